"""Shared helpers of the test suite (comparison norms and synthetic inputs)."""
from math import factorial

import numpy as np


def rel_rows(got, ref, floor_frac=1e-9):
    """max_i |got_i - ref_i| / max(|ref_i|, floor_frac * max_i |ref_i|) over the
    last axis (3-vectors)."""
    got, ref = np.asarray(got), np.asarray(ref)
    d = np.linalg.norm(got - ref, axis=-1)
    r = np.linalg.norm(ref, axis=-1)
    floor = floor_frac * max(r.max(), 1e-300)
    return float((d / np.maximum(r, floor)).max())


def scaled_stack_err(got, ref, dt):
    """Error of the derivative stacks (N, K, 3) in the scaled form of Eq. 1,
    F_k = h^k a^(k) / k! with h = dt/2, relative to max_k |F_k| per body."""
    got, ref = np.asarray(got), np.asarray(ref)
    K = ref.shape[1]
    h = abs(dt) / 2
    sc = np.array([h ** k / factorial(k) for k in range(K)])[None, :, None]
    Fg, Fr = got * sc, ref * sc
    per = np.linalg.norm(Fg - Fr, axis=-1).max(axis=1)
    scale = np.linalg.norm(Fr, axis=-1).max(axis=1)
    return float((per / np.maximum(scale, 1e-300)).max())


def kepler_traj(m, x, v, P, central=0):
    """Evaluation input built from the inputs alone (no integrator involved):
    rows x, v and, for P >= 2 / 3, the Kepler acceleration and jerk about the
    central body.  Returns a (N, P+1, 3) array."""
    N = len(m)
    out = np.zeros((N, P + 1, 3))
    out[:, 0] = x
    out[:, 1] = v
    r = x - x[central]
    u = v - v[central]
    d = np.linalg.norm(r, axis=1)
    d[central] = 1.0
    mu = m[central]
    a = -mu * r / d[:, None] ** 3
    rv = (r * u).sum(1)
    j = -mu * (u / d[:, None] ** 3 - 3 * rv[:, None] * r / d[:, None] ** 5)
    a[central] = 0.0
    j[central] = 0.0
    if P >= 2:
        out[:, 2] = a
    if P >= 3:
        out[:, 3] = j
    return out
