"""CPU check of the library's non-uniform-grid tables (mfc_grid_table, the
host code behind mfc_set_grid) against the oracle's, built independently from
the same definitions (oracle/nonuniform.py): candidate increments, ideal
weights, smoothness indicators and 1/dx of every cell, ghost cells included."""
import numpy as np
import pytest

import workloads
from oracle import nonuniform as nu


@pytest.fixture(scope="module")
def m():
    import paper_2305_09163_gb300 as mm
    mm.build()
    mm.load()
    return mm


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("kind", ["paper_stretching", "random"])
def test_library_tables_match_the_oracle(m, periodic, kind):
    if kind == "paper_stretching":
        faces = workloads.stretched_faces(24, -10.0, 10.0, 4.0, -1.2, 1.2)
    else:
        faces = np.concatenate([[0.0], np.cumsum(np.random.default_rng(5).uniform(0.3, 2.0, 19))])
    lib = m.mfc_grid_table(faces, periodic)
    T = lib[:, :, 0].astype(np.float64) + lib[:, :, 1].astype(np.float64)
    orc = nu.direction_tables(faces, periodic)
    assert T.shape[0] == orc.shape[0] == faces.size + 1
    rng = np.random.default_rng(1)
    for c in range(T.shape[0]):
        o = orc[c]
        cand = {0: o[0:15].reshape(3, 5), 1: o[15:30].reshape(3, 5)}
        ideal = {0: o[30:33], 1: o[33:36]}
        B = o[36:63].reshape(3, 3, 3)
        v = rng.standard_normal(5)
        D = np.diff(v)
        Da, Db = D[:3], D[1:]
        for side in (0, 1):
            for r in range(3):
                inc = T[c, 6 * side + 2 * r] * Da[r] + T[c, 6 * side + 2 * r + 1] * Db[r]
                assert inc == pytest.approx(cand[side][r] @ v - v[2], abs=1e-12)
            assert np.allclose(T[c, 12 + 3 * side:15 + 3 * side], ideal[side], rtol=1e-12, atol=1e-13)
        for r in range(3):
            beta = T[c, 18 + 3 * r] * Da[r] ** 2 + T[c, 19 + 3 * r] * Da[r] * Db[r] + T[c, 20 + 3 * r] * Db[r] ** 2
            assert beta == pytest.approx(v[r:r + 3] @ B[r] @ v[r:r + 3], rel=1e-11, abs=1e-12)
        assert T[c, 27] == pytest.approx(o[63], rel=1e-13)


def test_bad_faces_are_rejected(m):
    with pytest.raises(m.MFCError):
        m.mfc_grid_table(np.array([0.0, 1.0, 0.5, 2.0, 3.0]))
