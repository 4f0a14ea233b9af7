"""Training the learned WENO weights on the GPU.

Orchestration only: every computation is a call into libmfc_gb300.so — the
fine solver run (mfc_step / mfc_cfl_dt), primitive output (mfc_get_prims),
sample harvest (mfc_harvest), forward/backward on BF16 tensor cores
(mfc_mlp_grad, on the tcgen05 tensor cores) and the Adam update (mfc_mlp_adam).  Harvested samples are
already in hash-random order, so consecutive batches need no shuffle.

The paper has no learned part: the network stands in for the WENO5-JS nonlinear
weights of Sec. 3.2 (5 normalised stencil differences -> 32 -> 32 ReLU -> 3
softmax weights), trained on stencils of the plain method's own runs with the
fine-grid (2x) face value as target.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import (MFC_ERR_TIMEOUT, MFCError, MLP_PARAMS, MLP_WORK_FLOATS, Solver, mfc_harvest, mfc_mlp_adam,
               mfc_mlp_grad, mfc_mlp_tc_status)

IDEAL = (0.1, 0.6, 0.3)
HIDDEN = 32


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal hidden layers, small output layer biased to the ideal weights."""
    rng = np.random.default_rng(seed)
    w1 = rng.normal(0.0, np.sqrt(2.0 / 5), (HIDDEN, 5))
    w2 = rng.normal(0.0, np.sqrt(2.0 / HIDDEN), (HIDDEN, HIDDEN))
    w3 = rng.normal(0.0, 0.1 / np.sqrt(HIDDEN), (3, HIDDEN))
    parts = [w1.ravel(), np.zeros(HIDDEN), w2.ravel(), np.zeros(HIDDEN), w3.ravel(), np.log(IDEAL)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == MLP_PARAMS
    return p


@dataclass
class Samples:
    x: object        # [N,5] normalised stencils
    phat: object     # [N,3] normalised candidate increments
    target: object   # [N] normalised fine-grid face value
    smooth: object   # [N] 1 where the discontinuity sensor does not trip
    js: object       # [N] normalised WENO5-JS value

    def __len__(self):
        return self.x.shape[0]

    def slice(self, a, b):
        return Samples(self.x[a:b], self.phat[a:b], self.target[a:b], self.smooth[a:b], self.js[a:b])

    @staticmethod
    def cat(parts):
        import torch
        return Samples(*[torch.cat([getattr(p, f) for p in parts]) for f in ("x", "phat", "target", "smooth", "js")])


def harvest(w_fine, n_fine, num_fluids, count, seed, weno_eps=1e-6, tau=100.0) -> Samples:
    """`count` samples from one fine primitive field (device float64 tensor)."""
    import torch
    dev = w_fine.device
    out = Samples(torch.empty((count, 5), dtype=torch.float32, device=dev),
                  torch.empty((count, 3), dtype=torch.float32, device=dev),
                  torch.empty(count, dtype=torch.float32, device=dev),
                  torch.empty(count, dtype=torch.float32, device=dev),
                  torch.empty(count, dtype=torch.float32, device=dev))
    mfc_harvest(w_fine, n_fine, num_fluids, weno_eps, tau, count, seed, out.x, out.phat, out.target, out.smooth,
                out.js)
    return out


def harvest_run(workload, steps, snapshots, per_snapshot, seed, precision="mixed", cfl=0.3):
    """Run the plain method on a (fine) workload and harvest samples at the given
    step counts (0 = initial state)."""
    s = Solver(workload.n, workload.lo, workload.hi, workload.bc, workload.gamma, workload.pi_inf,
               precision=precision, fallback=1)
    s.set_state_prim(workload.prims())
    parts = []
    for k in range(steps + 1):
        if k in snapshots:
            parts.append(harvest(s.get_prims(), workload.n, workload.nf, per_snapshot, seed + 7919 * k))
        if k < steps:
            s.step(s.cfl_dt(cfl))
    s.close()
    return Samples.cat(parts)


def smooth_part(samples: Samples) -> Samples:
    """The samples where the discontinuity sensor does not trip: the only places
    the learned weights are used."""
    keep = samples.smooth > 0.5
    return Samples(samples.x[keep], samples.phat[keep], samples.target[keep], samples.smooth[keep],
                   samples.js[keep])


def train(samples: Samples, epochs=15, batch=65536, lr=2e-3, lam=1.0, seed=0, params=None, log=None,
          smooth_only=True):
    """Adam on the harvested samples (by default only those where the sensor does
    not trip); returns (params as a device float32 tensor, per-epoch mean losses)."""
    import torch
    if smooth_only:
        samples = smooth_part(samples)
    dev = samples.x.device
    P = torch.tensor(init_params(seed) if params is None else params, dtype=torch.float32, device=dev)
    M = torch.zeros_like(P)
    V = torch.zeros_like(P)
    G = torch.empty_like(P)
    L = torch.empty(1, dtype=torch.float32, device=dev)
    work = torch.empty(MLP_WORK_FLOATS, dtype=torch.float32, device=dev)
    n = len(samples)
    step = 0
    history = []
    for ep in range(epochs):
        tot, nb = 0.0, 0
        for a in range(0, n - batch + 1 if n >= batch else 1, batch):
            b = min(a + batch, n)
            sb = samples.slice(a, b)
            mfc_mlp_grad(P, sb.x, sb.phat, sb.target, sb.smooth, lam, G, L, work)
            step += 1
            mfc_mlp_adam(P, G, M, V, lr, 0.9, 0.999, 1e-8, step)
            tot += L.item()
            nb += 1
        history.append(tot / max(nb, 1))
        if log:
            log("epoch %d loss %.6g" % (ep, history[-1]))
    if mfc_mlp_tc_status():
        raise MFCError(MFC_ERR_TIMEOUT, "a tensor-core wait of mfc_mlp_grad gave up")
    return P, history
