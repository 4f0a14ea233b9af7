"""Learned-weight network kernels (BF16 tensor cores) against the FP64 oracle.

Tolerances are those of BF16 operands (8-bit mantissa) with FP32 accumulation:
weights omega within 2e-2 absolute, gradients within 5e-2 relative L2 norm
(and cosine similarity >= 0.995), the loss within 1e-2 relative."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import mlp as omlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import paper_2305_09163_gb300 as mm
    mm.build()
    mm.load()
    return mm


def _bf16(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _data(B, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(B, 5)).cumsum(axis=1) * rng.uniform(0.1, 10, size=(B, 1))
    v[: B // 4, 3:] += rng.normal(scale=20, size=(B // 4, 1))  # some jumps
    x, phat, s = omlp.stencil_features(v)
    t = (phat * rng.dirichlet([1, 1, 1], size=B)).sum(axis=1) + rng.normal(scale=0.05, size=B)
    mask = (rng.uniform(size=B) < 0.6).astype(np.float64)
    return x, phat, t, mask


def _theta(seed):
    return omlp.init_params(seed) + np.random.default_rng(seed + 100).normal(scale=0.1, size=omlp.N_PARAMS)


@pytest.mark.parametrize("impl", ["mma", "tc"])
@pytest.mark.parametrize("B", [16, 1000, 65536 + 5])
def test_forward_matches_oracle(m, B, impl):
    """mfc_mlp_forward (warp-level mma.sync) and mfc_mlp_forward_tc (tcgen05,
    128-sample tiles, accumulators in tensor memory)."""
    x, _, _, _ = _data(B, 1)
    theta = _theta(2)
    P = torch.tensor(theta, dtype=torch.float32, device="cuda")
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    om = torch.full((B, 3), float("nan"), dtype=torch.float32, device="cuda")
    (m.mfc_mlp_forward_tc if impl == "tc" else m.mfc_mlp_forward)(P, xd, om)
    torch.cuda.synchronize()
    if impl == "tc":
        assert m.mfc_mlp_tc_status() == 0
        om_mma = torch.empty_like(om)
        m.mfc_mlp_forward(P, xd, om_mma)
        # the same BF16 roundings; FP32 accumulation order and bias placement differ
        assert (om - om_mma).abs().max().item() <= 2e-3
    om_ref, _ = omlp.forward(theta, x)
    err = np.abs(om.cpu().numpy() - om_ref).max()
    assert err <= 2e-2, err
    # the same network with BF16-rounded weights and inputs: only activation rounding remains
    p = omlp.unpack(theta)
    for k in ("W1", "W2", "W3"):
        p[k] = _bf16(p[k])
    om_bf, _ = omlp.forward(omlp.pack(p), _bf16(x))
    assert np.abs(om.cpu().numpy() - om_bf).max() <= 1e-2
    assert np.allclose(om.cpu().numpy().sum(axis=1), 1.0, atol=1e-5)


@pytest.mark.parametrize("impl", ["tc", "mma"])
@pytest.mark.parametrize("B", [100, 40000, 200003])
def test_gradient_matches_oracle(m, B, impl):
    """mfc_mlp_grad (tcgen05; 40000 and 200003 samples give CTAs several
    128-sample tiles, so the weight gradients accumulate in tensor memory) and
    mfc_mlp_grad_mma against the FP64 oracle."""
    grad_fn = m.mfc_mlp_grad if impl == "tc" else m.mfc_mlp_grad_mma
    x, phat, t, mask = _data(B, 3)
    theta = _theta(4)
    lam = 0.3
    L_ref, g_ref = omlp.loss_and_grad(theta, x, phat, t, mask, lam)
    dev = lambda a: torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()
    P = dev(theta)
    grad = torch.empty(omlp.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    work = torch.empty(m.MLP_WORK_FLOATS, dtype=torch.float32, device="cuda")
    grad_fn(P, dev(x), dev(phat), dev(t), dev(mask), lam, grad, loss, work)
    torch.cuda.synchronize()
    if impl == "tc":
        assert m.mfc_mlp_tc_status() == 0
    g = grad.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    cos = g @ g_ref / (np.linalg.norm(g) * np.linalg.norm(g_ref))
    assert rel <= 5e-2 and cos >= 0.995, (rel, cos)
    assert loss.item() == pytest.approx(L_ref, rel=1e-2)
    # every parameter block gets its gradient (no unwritten workspace slot)
    gp, gr = omlp.unpack(g), omlp.unpack(g_ref)
    for k in gp:
        assert np.linalg.norm(gp[k] - gr[k]) <= 0.1 * np.linalg.norm(gr[k]) + 1e-6, k
    # deterministic
    grad2 = torch.empty_like(grad)
    grad_fn(P, dev(x), dev(phat), dev(t), dev(mask), lam, grad2, None, work)
    torch.cuda.synchronize()
    assert torch.equal(grad, grad2)


def test_adam_matches_oracle(m):
    rng = np.random.default_rng(5)
    theta = rng.normal(size=omlp.N_PARAMS)
    mom = np.zeros(omlp.N_PARAMS)
    vel = np.zeros(omlp.N_PARAMS)
    P = torch.tensor(theta, dtype=torch.float32, device="cuda")
    M = torch.zeros_like(P)
    V = torch.zeros_like(P)
    for step in range(1, 4):
        g = rng.normal(size=omlp.N_PARAMS)
        theta, mom, vel = omlp.adam_step(theta, g, mom, vel, step, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8)
        G = torch.tensor(g, dtype=torch.float32, device="cuda")
        m.mfc_mlp_adam(P, G, M, V, 1e-2, 0.9, 0.999, 1e-8, step)
    torch.cuda.synchronize()
    assert np.allclose(P.cpu().numpy(), theta, rtol=1e-5, atol=1e-6)


def test_primitives_match_oracle(m):
    gam, pin = workloads.fluids(3)
    pb = oracle.Problem((11, 7, 5), (0,) * 3, (1,) * 3, (1,) * 6, gam, pin)
    w = workloads.random_prims(pb.n, 3, seed=6)
    q = oracle.cons_from_prims(pb, w)
    s = m.Solver(pb.n, pb.lo, pb.hi, pb.bc, gam, pin)
    s.set_state(q)
    wg = s.get_prims().cpu().numpy()
    wo = oracle.prims_from_cons(pb, q)
    for v in range(pb.sys_size):
        scale = np.abs(wo[v]).max()
        assert np.abs(wg[v] - wo[v]).max() <= 1e-12 * scale + (1e-9 * 1e6 if v == 6 else 0), v


def _harvest(m, w, n, nf, N, seed, tau=1e3, eps=1e-6):
    outs = [torch.empty(s, dtype=torch.float32, device="cuda") for s in ((N, 5), (N, 3), (N,), (N,), (N,))]
    m.mfc_harvest(torch.from_numpy(w).cuda(), n, nf, eps, tau, N, seed, *outs)
    torch.cuda.synchronize()
    return [o.cpu().numpy().astype(np.float64) for o in outs]


def test_harvest_samples_are_consistent(m):
    """On a smooth 3D field: inputs are normalised, the WENO5-JS value matches the
    oracle on the restricted stencil, and the fine target is close to it."""
    n = 32
    g = np.meshgrid(*[(np.arange(n) + 0.5) / n] * 3, indexing="ij")
    prof = np.sin(2 * np.pi * g[2]) * np.cos(2 * np.pi * g[1]) + 0.5 * np.sin(2 * np.pi * g[0])
    w = np.stack([1000 + 50 * prof, 1 + 0.1 * prof, 10 * prof, 5 * prof, 2 * prof, 1e5 * (1 + 0.1 * prof),
                  0.5 + 0.2 * prof])
    x, phat, t, smooth, js = _harvest(m, w, (n, n, n), 2, 20000, 7)
    assert np.allclose(x[:, 2], 0) and np.allclose(np.abs(x).max(axis=1), 1.0, atol=1e-6)
    assert smooth.mean() > 0.7
    # the coarse WENO5-JS edge, re-evaluated by the oracle on the normalised stencil
    # (WENO5 is affine invariant up to the epsilon, which is negligible here)
    for k in range(0, 2000, 97):
        ref = oracle.weno5(x[k], 1e-6 / 1e12)
        assert js[k] == pytest.approx(ref, abs=2e-3)
    # smooth data: target and JS value agree closely; candidates bracket the target
    assert np.abs(t - js).mean() < 0.02


def test_harvest_sensor_trips_at_a_step(m):
    n = 32
    w = np.zeros((5, 1, 1, n))
    w[0] = 1.0
    w[1] = 0.0
    w[2] = np.where(np.arange(n) < n // 2, 1.0, 0.1)
    w[3] = 1.0
    w[4] = 0.5
    x, phat, t, smooth, js = _harvest(m, w.reshape(5, 1, 1, n), (n,), 2, 4000, 9)
    # stencils containing the step (|x| not a smooth ramp) trip the sensor
    has_step = np.abs(np.diff(x, axis=1)).max(axis=1) > 0.99
    assert (smooth[has_step] == 0).all()
