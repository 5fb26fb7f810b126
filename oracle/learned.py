"""CPU FP64 reference of the learned predictor residual (plain numpy).

TEST INFRASTRUCTURE ONLY (part of the oracle): nothing in the product imports it.

Reading R13 of the design notes (the paper has no learned component; the
workload asks for one):
  features  u_k = R^T F_k / (|a| sigma^k),  k = 0 .. 2p-1, then 1 + log10(sigma),
            F_k = h^k a^(k) / k!  (the scaled stack of Eq. 1, h = dt/2),
            R = [e1 e2 e3], e1 = a/|a|, e2 along the part of a-dot normal to a,
            e3 = e1 x e2, sigma = max_{1<=k<2p} (|F_k| / |F_0|)^(1/k), the
            shortest time scale the stack shows in units of h (omega h on a
            Kepler orbit), so every |u_k| <= 1;
  targets   y = (R^T dx / (|a| h^2 sigma^6), R^T dv / (|a| h sigma^6)),
            dx, dv = converged corrector result minus the Taylor prediction.
A body is left out (mask False) when |a| = 0, sigma = 0, or sigma > sigma_max.

MLP: n_in -> H -> H -> n_out, SiLU activations, mean-squared-error loss over
all outputs.  With bf16=True every GEMM input (features, weights, hidden
activations, back-propagated errors) is rounded to bfloat16 (round to nearest
even) at the same points as the GPU kernels, and all sums run in FP64.
"""
from __future__ import annotations

import numpy as np

SIGMA_MAX = 0.5


def bf16(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = rounded.astype(np.uint32).view(np.float32)
    out = np.where(np.isfinite(f), out, f)
    return out.astype(np.float64)


def frames(d: np.ndarray):
    """(R (N,3,3) with columns e1 e2 e3, |a|, valid) from a^(0), a^(1) (d: (N,K,3))."""
    a, j = d[:, 0], d[:, 1]
    na = np.linalg.norm(a, axis=1)
    ok = na > 0
    e1 = a / np.where(ok, na, 1.0)[:, None]
    u = j - (j * e1).sum(1)[:, None] * e1
    nu = np.linalg.norm(u, axis=1)
    # a-dot parallel to a: take any direction normal to e1
    alt = np.where(np.abs(e1[:, 0:1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    alt = alt - (alt * e1).sum(1)[:, None] * e1
    use_alt = nu <= 1e-300
    u = np.where(use_alt[:, None], alt, u)
    e2 = u / np.linalg.norm(u, axis=1)[:, None]
    e3 = np.cross(e1, e2)
    R = np.stack([e1, e2, e3], axis=2)
    return R, na, ok


def features(d: np.ndarray, dt: float):
    """(u (N, 3K+1), R, |a|, sigma, mask) of the derivative stacks d (N, K, 3)."""
    N, K, _ = d.shape
    h = 0.5 * dt
    fact = np.cumprod(np.concatenate([[1.0], np.arange(1, K)]))
    F = d * (h ** np.arange(K) / fact)[None, :, None]
    R, na, ok = frames(d)
    nF = np.linalg.norm(F, axis=2)                               # (N, K)
    nF0 = nF[:, 0]
    ratio = nF[:, 1:] / np.where(nF0 > 0, nF0, 1.0)[:, None]
    sigma = np.where(nF0 > 0, (ratio ** (1.0 / np.arange(1, K))[None, :]).max(axis=1), 0.0)
    mask = ok & (sigma > 0) & (sigma <= SIGMA_MAX)
    s = np.where(mask, sigma, 1.0)
    Fr = np.einsum("nji,nkj->nki", R, F)                       # R^T F_k
    u = Fr / (np.where(mask, na, 1.0)[:, None, None] * s[:, None, None] ** np.arange(K)[None, :, None])
    u = np.where(mask[:, None, None], u, 0.0).reshape(N, 3 * K)
    ls = np.where(mask, 1.0 + np.log10(np.where(mask, sigma, 1.0)), 0.0)
    return np.concatenate([u, ls[:, None]], axis=1), R, na, sigma, mask


def targets(dx: np.ndarray, dv: np.ndarray, R, na, sigma, mask, dt: float):
    h = 0.5 * dt
    s6 = np.where(mask, sigma, 1.0) ** 6
    den = np.where(mask, na, 1.0) * s6
    yx = np.einsum("nji,nj->ni", R, dx) / (den * h * h)[:, None]
    yv = np.einsum("nji,nj->ni", R, dv) / (den * h)[:, None]
    y = np.concatenate([yx, yv], axis=1)
    return np.where(mask[:, None], y, 0.0)


def residual(y: np.ndarray, R, na, sigma, mask, dt: float):
    """Inverse of targets(): (dx, dv) from network outputs y."""
    h = 0.5 * dt
    s6 = np.where(mask, sigma, 1.0) ** 6
    den = np.where(mask, na, 1.0) * s6
    dx = np.einsum("nij,nj->ni", R, y[:, :3]) * (den * h * h)[:, None]
    dv = np.einsum("nij,nj->ni", R, y[:, 3:]) * (den * h)[:, None]
    return np.where(mask[:, None], dx, 0.0), np.where(mask[:, None], dv, 0.0)


# --------------------------------------------------------------------------- #
# MLP
# --------------------------------------------------------------------------- #

def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


SHAPES = lambda n_in, H, n_out: [("W1", (H, n_in)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
                                 ("W3", (n_out, H)), ("b3", (n_out,))]


def unflatten(flat, n_in, H, n_out):
    out, o = {}, 0
    for name, shp in SHAPES(n_in, H, n_out):
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def flatten(p, n_in, H, n_out):
    return np.concatenate([p[name].ravel() for name, _ in SHAPES(n_in, H, n_out)])


def forward(p, X, bf=False):
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    W1, W2, W3 = r(p["W1"]), r(p["W2"]), r(p["W3"])
    X = r(X)
    Z1 = X @ W1.T + p["b1"]
    H1 = r(silu(Z1))
    Z2 = H1 @ W2.T + p["b2"]
    H2 = r(silu(Z2))
    Y = H2 @ W3.T + p["b3"]
    return Y, (X, Z1, H1, Z2, H2)


def loss_grad(p, X, T, bf=False):
    """MSE loss (mean over samples and outputs) and its gradient (dict)."""
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    Y, (Xr, Z1, H1, Z2, H2) = forward(p, X, bf)
    B, n_out = Y.shape
    diff = Y - T
    loss = float((diff ** 2).mean())
    dY = r(2.0 * diff / (B * n_out))
    W2, W3 = r(p["W2"]), r(p["W3"])
    g = {"W3": dY.T @ H2, "b3": dY.sum(0)}
    dZ2 = r((dY @ W3) * dsilu(Z2))
    g["W2"] = dZ2.T @ H1
    g["b2"] = dZ2.sum(0)
    dZ1 = r((dZ2 @ W2) * dsilu(Z1))
    g["W1"] = dZ1.T @ Xr
    g["b1"] = dZ1.sum(0)
    return loss, g


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of every parameter, in place."""
    for k in p:
        m[k] = b1 * m[k] + (1 - b1) * g[k]
        v[k] = b2 * v[k] + (1 - b2) * g[k] ** 2
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
