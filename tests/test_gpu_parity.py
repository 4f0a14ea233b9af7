"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

The metric (``parity_util.rhs_error``) is a per-component relative L-infinity
error of one RHS call; the FP64 path must satisfy max_v err_v <= 1e-11.  Inputs
are seeded primitive fields from ``workloads``; each side converts them to
conserved variables with its own code.
"""
import numpy as np
import pytest

import oracle
import workloads
from parity_util import rhs_error, rhs_table, sampled_rhs_error, state_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-11


@pytest.fixture(scope="module")
def mfc():
    import paper_2305_09163_gb300 as m
    m.build()
    m.load()
    return m


def _problem(n, bc, gamma, pi_inf, fallback, eps=1e-6):
    return oracle.Problem(n, (0, 0, 0), (1, 1, 1), bc, gamma, pi_inf, eps=eps, fallback=fallback)


def _solver(mfc, pb, precision="fp64", **params):
    s = mfc.Solver(pb.n, pb.lo, pb.hi, pb.bc, pb.gamma, pb.pi_inf, precision=precision,
                   weno_eps=pb.eps, fallback=1 if pb.fallback else 0, **params)
    return s


CASES = [
    # (n, nf, bc, water_air, fallback)
    ((37,), 1, 1, False, False),
    ((37,), 2, 0, True, False),
    ((41,), 2, 2, True, True),
    ((29, 17), 2, 1, True, False),
    ((23, 19), 3, 0, True, True),
    ((37, 23, 19), 2, 1, True, False),
    ((37, 23, 19), 2, 0, True, True),
    ((21, 13, 11), 3, 2, True, False),
    ((16, 9, 7), 1, 1, False, False),
    ((19, 24, 13), 3, 1, True, True),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "n%s_nf%d_bc%d_fb%d" % ("x".join(map(str, c[0])), c[1], c[2], c[4]))
def test_rhs_parity_fp64_random_states(mfc, case):
    n, nf, bc, wa, fb = case
    gam, pin = workloads.fluids(nf, wa)
    pb = _problem(n, (bc,) * 6, gam, pin, fb)
    w = workloads.random_prims(n, nf, seed=hash(case) % 1000, water_air=wa)
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    s = _solver(mfc, pb)
    s.set_state_prim(torch.from_numpy(w).cuda())
    # conversion parity: the GPU's conserved state equals the oracle's
    qg = s.get_state().cpu().numpy()
    assert np.allclose(qg, q, rtol=1e-14, atol=0)
    R_gpu = s.rhs().cpu().numpy()
    err = rhs_error(pb, q, R_gpu, R_cpu, fmax)
    assert err.max() <= TOL_FP64, err


def test_rhs_parity_fp64_mixed_bcs(mfc):
    n = (17, 14, 12)
    gam, pin = workloads.fluids(2)
    bc = (2, 1, 0, 0, 1, 2)
    pb = _problem(n, bc, gam, pin, True)
    w = workloads.random_prims(n, 2, seed=5)
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    s = _solver(mfc, pb)
    s.set_state_prim(torch.from_numpy(w).cuda())
    R_gpu = s.rhs().cpu().numpy()
    assert rhs_error(pb, q, R_gpu, R_cpu, fmax).max() <= TOL_FP64


@pytest.mark.parametrize("seg,yz", [(8, 0), (16, 0), (64, 0), (8, 1), (64, 1)])
def test_rhs_parity_independent_of_segment_length(mfc, seg, yz):
    """Several pencil segments per direction with a ragged last segment, with
    either y/z kernel (pencil marching or the stream kernel)."""
    n = (70, 33, 21)
    gam, pin = workloads.fluids(2)
    pb = _problem(n, (1,) * 6, gam, pin, True)
    w = workloads.random_prims(n, 2, seed=7)
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    s = _solver(mfc, pb, segment=seg, yz_kernel=yz)
    s.set_state_prim(torch.from_numpy(w).cuda())
    R_gpu = s.rhs().cpu().numpy()
    assert rhs_error(pb, q, R_gpu, R_cpu, fmax).max() <= TOL_FP64


def test_rhs_parity_shock_bubble_small(mfc, capsys):
    """The shock-bubble geometry at 48^3: shocked water (1e9 Pa), tanh air bubble."""
    wl = workloads.shock_bubble(48)
    pb = oracle.Problem(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, fallback=True)
    w = wl.prims()
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    s = _solver(mfc, pb)
    s.set_state_prim(torch.from_numpy(w).cuda())
    R_gpu = s.rhs().cpu().numpy()
    with capsys.disabled():
        print("\nshock-bubble 48^3, FP64 RHS per component:\n" + rhs_table(pb, q, R_gpu, R_cpu, fmax))
    assert rhs_error(pb, q, R_gpu, R_cpu, fmax).max() <= TOL_FP64


@pytest.mark.parametrize("p_high,solid", [(1e12, True), (1e16, False)], ids=["stiff_solid_1e12", "jump_1e16"])
def test_rhs_parity_at_range_extremes(mfc, p_high, solid, capsys):
    """The FP64 path's WENO weights and HLLC run in float-float (float32 exponent
    range): three fluids with the stiff solid phase (gamma 3, pi_inf 1e10 Pa),
    either dominant (volume fraction ~0.98) beside a 1e5 -> 1e12 Pa pressure
    jump, or mixed with water and air across a 1e5 -> 1e16 Pa jump, near the top
    of the documented range.  Gate: the FP64 1e-11."""
    n = (29, 17, 13)
    gam, pin = workloads.fluids(3)
    assert pin[2] == 1e10
    pb = _problem(n, (1,) * 6, gam, pin, True)
    w = workloads.random_prims(n, 3, seed=404)
    nf, nd = 3, 3
    ip = nf + nd
    x = (np.arange(n[0]) + 0.5) / n[0]
    high = np.broadcast_to(x > 0.45, w[ip].shape)
    w[ip] = np.where(high, p_high, 1e5) * (1.0 + 0.05 * np.sin(7.0 * w[nf]))
    if solid:
        a = np.empty((nf,) + w[0].shape)
        a[0] = 0.01 * (1.0 + 0.5 * np.sin(3.0 * w[nf]))
        a[1] = 0.01 * (1.0 + 0.5 * np.cos(5.0 * w[nf + 1]))
        a[2] = 1.0 - a[0] - a[1]
        rho = (1000.0, 1.0, 2000.0)
        for k in range(nf):
            w[k] = a[k] * rho[k]
        for k in range(nf - 1):
            w[ip + 1 + k] = a[k]
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    s = _solver(mfc, pb)
    s.set_state_prim(torch.from_numpy(np.ascontiguousarray(w)).cuda())
    R_gpu = s.rhs().cpu().numpy()
    with capsys.disabled():
        print("\nrange extremes (p_high %.0e, solid-dominant %s), FP64 RHS per component:\n"
              % (p_high, solid) + rhs_table(pb, q, R_gpu, R_cpu, fmax))
    assert rhs_error(pb, q, R_gpu, R_cpu, fmax).max() <= TOL_FP64


def test_cfl_and_steps_match_oracle(mfc):
    """dt from the CFL reduction and five SSP-RK3 steps on the small shock-bubble."""
    wl = workloads.shock_bubble(24)
    pb = oracle.Problem(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, fallback=True)
    w = wl.prims()
    q = oracle.cons_from_prims(pb, w)
    s = _solver(mfc, pb)
    s.set_state_prim(torch.from_numpy(w).cuda())
    for _ in range(5):
        dt_cpu = oracle.cfl_dt(pb, q, 0.3)
        dt_gpu = s.cfl_dt(0.3)
        assert dt_gpu == pytest.approx(dt_cpu, rel=1e-13)
        q = oracle.rk3_step(pb, q, dt_cpu)
        s.step(dt_cpu)
    qg = s.get_state().cpu().numpy()
    err = state_error(pb, qg, q)
    assert err.max() <= 1e-10, err


def test_shock_tube_1d_matches_oracle_and_exact(mfc):
    """The 1000-cell water/air shock tube to t = 240 us on the GPU."""
    from oracle.exact_riemann import Side, sample
    wl = workloads.shock_tube(1000)
    pb = oracle.Problem(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, fallback=False)
    s = _solver(mfc, pb)
    s.set_state_prim(torch.from_numpy(wl.prims()).cuda())
    t, steps = 0.0, 0
    while t < wl.t_end:
        dt = s.cfl_dt(wl.cfl)
        dt = min(dt, wl.t_end - t)
        s.step(dt)
        t += dt
        steps += 1
    qg = s.get_state().cpu().numpy()
    wg = oracle.prims_from_cons(pb, qg)
    x = (np.arange(1000) + 0.5) / 1000
    rho_e, u_e, p_e, _ = sample(Side(1000.0, 0.0, 1e9, 4.4, 6e8), Side(1.0, 0.0, 1e5, 1.4, 0.0), (x - 0.7) / t)
    l1 = lambda a, b: np.abs(a - b).mean() / np.abs(b).mean()
    assert l1((wg[0] + wg[1]).ravel(), rho_e) < 5e-3
    assert l1(wg[2].ravel(), u_e) < 1.2e-2
    assert l1(wg[3].ravel(), p_e) < 5e-3
    # the oracle's own run: same number of steps, close states
    qo, to, so = oracle.run(pb, oracle.cons_from_prims(pb, wl.prims()), wl.t_end, wl.cfl)
    assert so == steps
    wo = oracle.prims_from_cons(pb, qo)
    assert np.abs(wg[3] - wo[3]).max() <= 1e-7 * np.abs(wo[3]).max()


def test_results_are_bitwise_reproducible_and_replicas_agree(mfc):
    n = (33, 20, 17)
    gam, pin = workloads.fluids(2)
    pb = _problem(n, (1,) * 6, gam, pin, True)
    w = torch.from_numpy(workloads.random_prims(n, 2, seed=3)).cuda()
    s1 = _solver(mfc, pb)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s2 = _solver(mfc, pb)
    s1.set_state_prim(w)
    s2.set_state_prim(w)
    torch.cuda.synchronize()
    for _ in range(3):
        s1.step(1e-7)
        s2.step(1e-7)
    torch.cuda.synchronize()
    a = s1.get_state()
    b = s2.get_state()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    r1 = s1.rhs()
    r2 = s1.rhs()
    assert torch.equal(r1, r2)


def test_checkpoint_restart_is_bitwise(mfc):
    wl = workloads.shock_bubble(20)
    pb = oracle.Problem(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, fallback=True)
    w = torch.from_numpy(wl.prims()).cuda()
    a = _solver(mfc, pb)
    a.set_state_prim(w)
    dt = 2e-8
    for _ in range(4):
        a.step(dt)
    ref = a.get_state()
    b = _solver(mfc, pb)
    b.set_state_prim(w)
    for _ in range(2):
        b.step(dt)
    host = b.get_state().cpu().numpy()
    c = _solver(mfc, pb)
    c.set_state(host)
    for _ in range(2):
        c.step(dt)
    assert torch.equal(c.get_state(), ref)


def test_nonphysical_state_is_reported(mfc):
    gam, pin = workloads.fluids(2)
    pb = _problem((12, 8, 8), (1,) * 6, gam, pin, True)
    w = workloads.random_prims(pb.n, 2, seed=4)
    q = oracle.cons_from_prims(pb, w)
    q[5, 3, 4, 5] = np.nan  # energy of one cell
    s = _solver(mfc, pb)
    s.set_state(q)
    with pytest.raises(mfc.MFCError) as ei:
        s.cfl_dt(0.3)
    assert ei.value.status == mfc.MFC_ERR_NONPHYSICAL
    # the context stays usable
    s.set_state_prim(torch.from_numpy(w).cuda())
    assert s.cfl_dt(0.3) > 0


def test_unset_state_and_bad_arguments(mfc):
    gam, pin = workloads.fluids(2)
    pb = _problem((8, 8, 8), (1,) * 6, gam, pin, True)
    s = _solver(mfc, pb)
    with pytest.raises(mfc.MFCError) as ei:
        s.rhs()
    assert ei.value.status == mfc.MFC_ERR_STATE_UNSET
    with pytest.raises(mfc.MFCError) as ei:
        s.set_param("weno_eps", -1.0)
    assert ei.value.status == mfc.MFC_ERR_ARG
    with pytest.raises(mfc.MFCError) as ei:
        s.set_param("no_such_thing", 1.0)
    assert ei.value.status == mfc.MFC_ERR_ARG
    s.set_state_prim(torch.from_numpy(workloads.random_prims(pb.n, 2, seed=1)).cuda())
    with pytest.raises(mfc.MFCError) as ei:
        s.step(float("nan"))
    assert ei.value.status == mfc.MFC_ERR_ARG


def test_rhs_to_host_buffer(mfc):
    gam, pin = workloads.fluids(2)
    pb = _problem((15, 11, 9), (0,) * 6, gam, pin, False)
    w = workloads.random_prims(pb.n, 2, seed=8)
    s = _solver(mfc, pb)
    s.set_state_prim(w)  # host numpy input
    host = np.empty(pb.shape())
    mfc.mfc_rhs(s.ctx, host)
    dev = s.rhs().cpu().numpy()
    assert np.array_equal(host, dev)


@pytest.mark.parametrize("wl_name", ["shock_bubble"])
def test_full_size_sampled_parity(mfc, wl_name, capsys):
    """The 256^3 shock-bubble workload in the bench's launch configuration:
    full GPU RHS, oracle at sampled cells (random, boundaries, interface, shock)."""
    wl = workloads.shock_bubble(256)
    pb = oracle.Problem(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, fallback=True)
    w = wl.prims()
    q = oracle.cons_from_prims(pb, w)
    s = _solver(mfc, pb)
    s.set_state_prim(torch.from_numpy(w).cuda())
    R = s.rhs().cpu().numpy().reshape(pb.sys_size, -1)
    rng = np.random.default_rng(11)
    n = 256
    pick = [rng.integers(0, pb.ncell, 1500)]
    # faces of the domain, the shock front and the bubble interface
    for (x, y, z) in [(0, 0, 0), (n - 1, n - 1, n - 1), (12, 100, 7), (13, 5, 255), (128, 128, 128 + 25),
                      (128 + 26, 128, 128), (128, 102, 128), (0, 255, 128)]:
        pick.append(np.array([(z * n + y) * n + x]))
    xs = rng.integers(8, 18, 300)
    ys = rng.integers(0, n, 300)
    zs = rng.integers(0, n, 300)
    pick.append((zs * n + ys) * n + xs)
    cells = np.unique(np.concatenate(pick))
    Rc, fmax = oracle.rhs_cells(pb, q, cells, return_fmax=True)
    err = sampled_rhs_error(pb, q, R, cells, Rc, fmax)
    with capsys.disabled():
        print("\nshock-bubble 256^3, FP64 RHS at %d sampled cells:\n" % cells.size
              + rhs_table(pb, q, R, Rc, fmax, cells=cells))
    assert err.max() <= TOL_FP64, err
