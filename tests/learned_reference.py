"""FP64 CPU reference of the learned form's right-hand side, composed from the
oracle's pieces (primitive recovery, HLLC, the network of ``oracle.mlp``), for
the parity tests of the fused tensor-core inference in the sweeps.

Test infrastructure only.  Periodic boundaries; every edge takes the network's
weights (the library is run with the sensor and the range safeguard off).  With
``bf16=True`` the network inputs, the weights W1..W3 and the two hidden
activations are rounded to BF16 (round to nearest even) at the points where the
tensor-core kernels round them; biases, logits, softmax and the edge value stay
FP64.  The finite-volume assembly follows the semi-discrete form of Sec. 2-3:
R_v = sum_d (F_{v,i-1/2} - F_{v,i+1/2}) / dx_d, and for the volume fractions
the source alpha_i (u~_{i+1/2} - u~_{i-1/2}) / dx_d with u~ the HLLC face velocity.
"""
import numpy as np

import oracle
from oracle import mlp


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def network_weights(theta, V, rounded=True):
    """Softmax weights [B,3] of the network for stencils V[B,5] (edge at i+1/2)."""
    p = mlp.unpack(theta)
    x, _, _ = mlp.stencil_features(V)
    r = bf16 if rounded else (lambda a: np.asarray(a, dtype=np.float64))
    h1 = r(np.maximum(r(x) @ r(p["W1"]).T + p["b1"], 0.0))
    h2 = r(np.maximum(h1 @ r(p["W2"]).T + p["b2"], 0.0))
    z = h2 @ r(p["W3"]).T + p["b3"]
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def learned_edges(theta, V, rounded=True, shift=0):
    """Edge values at i+1/2 of stencils V[B,5].  shift != 0 plants a mistake for
    the tests: each stencil takes the weights of the stencil `shift` rows on."""
    _, phat, s = mlp.stencil_features(V)
    om = network_weights(theta, V, rounded)
    if shift:
        om = np.roll(om, -shift, axis=0)
    return V[:, 2] + s * (om * phat).sum(axis=1)


def learned_rhs(pb, q, theta, rounded=True, shift=0):
    """(R, fmax): the learned-form right-hand side [ns, nz, ny, nx] of the
    conserved state q on the periodic grid of pb, and max |F_v| over all faces."""
    assert all(b == 0 for b in pb.bc[:2 * pb.ndim]), "periodic boundaries only"
    w = oracle.prims_from_cons(pb, q)
    ns, nf, nd = pb.sys_size, pb.nf, pb.ndim
    ia = nf + nd + 1
    R = np.zeros_like(w)
    fmax = np.zeros(ns)
    for d in range(nd):
        ax = 3 - d                      # array axis of direction d in [v, z, y, x]
        n = w.shape[ax]
        st = np.stack([np.take(w, (np.arange(n) + k) % n, axis=ax) for k in (-2, -1, 0, 1, 2)], axis=-1)
        flat = st.reshape(-1, 5)
        eL = learned_edges(theta, flat, rounded, shift).reshape(w.shape)          # at i+1/2, from cell i
        eR = learned_edges(theta, flat[:, ::-1], rounded, shift).reshape(w.shape)  # at i-1/2, from cell i
        left = eL
        right = np.roll(eR, -1, axis=ax)   # face i+1/2: right state from cell i+1
        F = np.zeros_like(w)
        U = np.zeros(w.shape[1:])
        for idx in np.ndindex(*w.shape[1:]):
            f, u = oracle.hllc(pb, d, left[(slice(None),) + idx], right[(slice(None),) + idx])
            F[(slice(None),) + idx] = f
            U[idx] = u
        fmax = np.maximum(fmax, np.abs(F).reshape(ns, -1).max(axis=1))
        Fm = np.roll(F, 1, axis=ax)          # face i-1/2
        Um = np.roll(U, 1, axis=ax - 1)
        R += (Fm - F) / pb.dx[d]
        R[ia:] += w[ia:] * (U - Um)[None] / pb.dx[d]
    return R, fmax
