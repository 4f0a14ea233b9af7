"""The allocation-free right-hand side (mfc_rhs_noalloc).

Callers that cannot let a library allocate device memory (their own pool or
budget owns every byte, or they cannot take an allocation's synchronisation)
use this entry point; its scratch is a static device array of the library.
Checked through the C ABI against the context-based mfc_rhs on two calls in a
row with different states, so stale scratch contents would show.  Kept in a file
of its own that pytest collects last.
"""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11


def _rel_err(a, b):
    ns = b.shape[0]
    a = a.reshape(ns, -1)
    b = b.reshape(ns, -1)
    return max(float((a[v] - b[v]).abs().max() / max(float(b[v].abs().max()), 1e-300)) for v in range(ns))


def test_noalloc_rhs_matches_context_rhs_on_consecutive_calls():
    import paper_2305_09163_gb300 as m
    m.build()
    n = (37, 23, 19)
    gam, pin = workloads.fluids(2)
    bc = (1, 1, 2, 2, 0, 0)
    lo, hi = (0.0, 0.0, 0.0), (1.0, 0.8, 0.5)
    s = m.Solver(n, lo, hi, bc, gam, pin, precision="fp64", fallback=1)
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (31, 32):
        w = torch.from_numpy(workloads.random_prims(n, 2, seed=seed)).cuda()
        s.set_state_prim(w)
        q = s.get_state()
        ref = s.rhs()
        out = torch.full_like(ref, float("nan"))
        m.mfc_rhs_noalloc(q, out, n, lo, hi, bc, gam, pin, 1e-6, 1, stream)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel_err(out, ref) <= TOL
    s.close()


def test_noalloc_allocates_no_device_memory():
    """The property the entry point exists for: once the first call on the
    device has looked up the scratch array's address, a call (here with
    characteristic boundaries, whose context path keeps a side buffer) leaves
    the free device memory unchanged."""
    import paper_2305_09163_gb300 as m
    m.build()
    n = (24, 18, 16)
    gam, pin = workloads.fluids(2)
    bc = (3, 3, 1, 3, 3, 2)
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    s = m.Solver(n, lo, hi, bc, gam, pin, precision="fp64", fallback=1)
    s.set_state_prim(torch.from_numpy(workloads.random_prims(n, 2, seed=33)).cuda())
    q = s.get_state()
    ref = s.rhs()
    out = torch.empty_like(ref)
    stream = torch.cuda.current_stream().cuda_stream
    m.mfc_rhs_noalloc(q, out, n, lo, hi, bc, gam, pin, 1e-6, 1, stream)  # warm-up: address look-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    out.fill_(float("nan"))
    m.mfc_rhs_noalloc(q, out, n, lo, hi, bc, gam, pin, 1e-6, 1, stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert _rel_err(out, ref) <= TOL
    s.close()


def test_noalloc_rejects_grids_beyond_its_maximum():
    import paper_2305_09163_gb300 as m
    m.build()
    n = (65, 64, 64)  # one plane more than 64^3
    assert n[0] * n[1] * n[2] > m.NOALLOC_MAX_CELLS
    # buffers of the full size, so that no launch could ever overrun them
    q = torch.zeros((7, 64, 64, 65), dtype=torch.float64, device="cuda")
    rhs = torch.zeros_like(q)
    with pytest.raises(m.MFCError) as ei:
        m.mfc_rhs_noalloc(q, rhs, n, (0, 0, 0), (1, 1, 1), (1,) * 6, (4.4, 1.4), (6e8, 0.0))
    assert ei.value.status == m.MFC_ERR_ARG
    assert "MFC_NOALLOC_MAX_CELLS" in str(ei.value)
    assert not rhs.any()


def test_noalloc_binding_checks_buffer_sizes():
    """The C side trusts its pointers; the binding refuses buffers whose size
    does not match the grid before anything is launched."""
    import paper_2305_09163_gb300 as m
    m.build()
    n = (16, 8, 8)
    q = torch.zeros((7, 8, 8, 16), dtype=torch.float64, device="cuda")
    small = torch.zeros((7, 8, 8, 15), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        m.mfc_rhs_noalloc(q, small, n, (0, 0, 0), (1, 1, 1), (1,) * 6, (4.4, 1.4), (6e8, 0.0))
    with pytest.raises(ValueError):
        m.mfc_rhs_noalloc(small, q, n, (0, 0, 0), (1, 1, 1), (1,) * 6, (4.4, 1.4), (6e8, 0.0))
