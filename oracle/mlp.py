"""FP64 reference of the learned WENO weights: network, loss and gradients.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper has no learned part; this is the reference for the library's learned
form, which replaces the WENO5-JS nonlinear weights of Sec. 3.2 by a small
network.  For one five-cell stencil v_{i-2..i+2} and the edge at i+1/2:

  * inputs  x_k = (v_{i+k} - v_i) / s,  k = -2..2,  s = max_k |v_{i+k} - v_i| + 1e-30
  * network h1 = relu(W1 x + b1) (32), h2 = relu(W2 h1 + b2) (32),
            z = W3 h2 + b3 (3),  omega = softmax(z)
  * value   v_i + s * sum_r omega_r phat_r, where phat_r are the WENO5 candidate
            increments (p_r - v_i)/s of the three three-cell stencils
            (r = 0: i-2..i, r = 1: i-1..i+1, r = 2: i..i+2).
The edge at i-1/2 uses the same network on the reversed stencil.

Training loss over a batch of B samples with targets t_b (normalised like the
candidates) and smooth-region mask m_b:
  L = (1/B) sum_b [ (sum_r omega_br phat_br - t_b)^2 + lam * m_b * sum_r (omega_br - d_r)^2 ],
with the ideal weights d = (0.1, 0.6, 0.3).

Parameter blob (float32 on the GPU): W1[32][5], b1[32], W2[32][32], b2[32],
W3[3][32], b3[3] -- 1347 values.
"""
from __future__ import annotations

import numpy as np

H = 32
NIN = 5
NOUT = 3
D_IDEAL = np.array([0.1, 0.6, 0.3])
SIZES = [("W1", (H, NIN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (NOUT, H)), ("b3", (NOUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == N_PARAMS
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SIZES])


def init_params(seed=0):
    """He-style initialisation; output layer biased toward the ideal weights."""
    rng = np.random.default_rng(seed)
    p = {
        "W1": rng.normal(0, np.sqrt(2.0 / NIN), (H, NIN)),
        "b1": np.zeros(H),
        "W2": rng.normal(0, np.sqrt(2.0 / H), (H, H)),
        "b2": np.zeros(H),
        "W3": rng.normal(0, 0.1 * np.sqrt(1.0 / H), (NOUT, H)),
        "b3": np.log(D_IDEAL),
    }
    return pack(p)


def stencil_features(v):
    """Normalised inputs x[B,5], candidate increments phat[B,3] and scale s[B]
    of stencils v[B,5] (cells i-2..i+2) for the edge at i+1/2."""
    v = np.asarray(v, dtype=np.float64)
    dv = v - v[:, 2:3]
    s = np.abs(dv).max(axis=1) + 1e-30
    x = dv / s[:, None]
    # candidate values minus v_i (Jiang-Shu candidates, Sec. 3.2)
    p0 = (2 * v[:, 0] - 7 * v[:, 1] + 11 * v[:, 2]) / 6 - v[:, 2]
    p1 = (-v[:, 1] + 5 * v[:, 2] + 2 * v[:, 3]) / 6 - v[:, 2]
    p2 = (2 * v[:, 2] + 5 * v[:, 3] - v[:, 4]) / 6 - v[:, 2]
    phat = np.stack([p0, p1, p2], axis=1) / s[:, None]
    return x, phat, s


def forward(theta, x):
    """Network outputs: (omega[B,3], cache) for inputs x[B,5]."""
    p = unpack(theta)
    a1 = x @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["W3"].T + p["b3"]
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    om = e / e.sum(axis=1, keepdims=True)
    return om, (x, a1, h1, a2, h2, om)


def edge_value(theta, v):
    """Learned reconstruction of the edge at i+1/2 for stencils v[B,5]."""
    x, phat, s = stencil_features(v)
    om, _ = forward(theta, x)
    return v[:, 2] + s * (om * phat).sum(axis=1)


def loss(theta, x, phat, t, mask, lam):
    om, _ = forward(theta, x)
    y = (om * phat).sum(axis=1)
    B = x.shape[0]
    return float(((y - t) ** 2).sum() / B + lam * (mask[:, None] * (om - D_IDEAL) ** 2).sum() / B)


def loss_and_grad(theta, x, phat, t, mask, lam):
    """Loss and its gradient with respect to every parameter (backpropagation)."""
    p = unpack(theta)
    om, (x, a1, h1, a2, h2, _) = forward(theta, x)
    B = x.shape[0]
    y = (om * phat).sum(axis=1)
    L = float(((y - t) ** 2).sum() / B + lam * (mask[:, None] * (om - D_IDEAL) ** 2).sum() / B)
    dom = (2.0 / B) * (y - t)[:, None] * phat + (2.0 * lam / B) * mask[:, None] * (om - D_IDEAL)
    dz = om * (dom - (om * dom).sum(axis=1, keepdims=True))
    g = {}
    g["W3"] = dz.T @ h2
    g["b3"] = dz.sum(axis=0)
    dh2 = dz @ p["W3"]
    da2 = dh2 * (a2 > 0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * (a1 > 0)
    g["W1"] = da1.T @ x
    g["b1"] = da1.sum(axis=0)
    return L, pack(g)


def adam_step(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (Kingma & Ba 2015) with bias correction; returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
