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


def dd_diff(a2, b2):
    """(a_hi + a_lo) - (b_hi + b_lo) for double-double arrays (..., 2), keeping
    the low words: the high words' difference is exact when they are within a
    factor of two of each other (Sterbenz), which holds wherever the values agree."""
    a2, b2 = np.asarray(a2), np.asarray(b2)
    return (a2[..., 0] - b2[..., 0]) + (a2[..., 1] - b2[..., 1])


def dd_scaled_stack_err(got2, ref2, dt):
    """scaled_stack_err for double-double stacks (N, K, 3, 2)."""
    ref = np.asarray(ref2)[..., 0] + np.asarray(ref2)[..., 1]
    d = dd_diff(got2, ref2)
    K = ref.shape[1]
    h = abs(dt) / 2
    sc = np.array([h ** k / factorial(k) for k in range(K)])[None, :, None]
    per = np.linalg.norm(d * sc, axis=-1).max(axis=1)
    scale = np.linalg.norm(ref * sc, axis=-1).max(axis=1)
    return float((per / np.maximum(scale, 1e-300)).max())
