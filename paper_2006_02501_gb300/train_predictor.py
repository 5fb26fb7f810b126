"""Training pipeline of the learned predictor residual (host orchestration).

All arithmetic runs in the library's kernels: the samples come from
mh_collect_samples (converged corrector outputs), training is mh_mlp_train
(BF16 tensor-core forward/backward, Adam).  This module only selects rows,
standardises the targets and folds the standardisation into the last layer.

    net = fit(collect(sim, dt, steps=24, n_iter=10), n_hidden=128)
    sim2.set_predictor(net)
"""
from __future__ import annotations

import numpy as np

from . import MLP, _capi  # noqa: F401


def collect(sim, dt: float, steps: int, n_iter: int = 10):
    """(features, targets) device tensors of `steps` converged steps of `sim`."""
    import torch
    n_in = 6 * sim.p + 1
    F = torch.zeros((steps * sim.N, n_in), dtype=torch.float32, device="cuda")
    T = torch.zeros((steps * sim.N, 6), dtype=torch.float32, device="cuda")
    for k in range(steps):
        sim.collect_samples(dt, n_iter, F[k * sim.N:(k + 1) * sim.N], T[k * sim.N:(k + 1) * sim.N])
    return F, T


def _shapes(n_in, H, n_out):
    return [("W1", (H, n_in)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (n_out, H)), ("b3", (n_out,))]


def fit(samples, n_hidden: int = 128, epochs: int = 80, batch: int = 512, lr: float = 1e-3, seed: int = 0,
        max_abs_target: float = 1e3, oversample: int = 3):
    """Train an MLP on (features, targets).

    Rows without a frame (all-zero features) and rows with a target beyond
    max_abs_target are dropped; rows are resampled with weight
    clip(10^(6 (log10 sigma - median)), 1, 30) (the sigma of a row is its last
    feature), which favours the short-time-scale bodies that set the pass
    count; targets are standardised per output and the standardisation is
    folded into the last layer, so the returned network predicts raw targets."""
    import torch
    F, T = samples
    Fn, Tn = F.cpu().numpy(), T.cpu().numpy()
    keep = (np.abs(Tn).max(1) < max_abs_target) & (np.abs(Fn).max(1) > 0)
    Fn, Tn = Fn[keep], Tn[keep]
    if len(Fn) == 0:
        raise ValueError("no usable training rows")
    ls = Fn[:, -1]
    w = np.clip(10.0 ** (6.0 * (ls - np.median(ls))), 1.0, 30.0)
    rng = np.random.default_rng(seed)
    sel = rng.choice(len(Fn), size=oversample * len(Fn), p=w / w.sum())
    Fn, Tn = Fn[sel], Tn[sel]
    mu = Tn.mean(0)
    sd = Tn.std(0) + 1e-30
    n_in = Fn.shape[1]
    net = MLP(n_in, n_hidden, Tn.shape[1], seed=seed + 1)
    net.train(torch.from_numpy(np.ascontiguousarray(Fn)).cuda(),
              torch.from_numpy(((Tn - mu) / sd).astype(np.float32)).cuda(),
              epochs=epochs, batch=batch, lr=lr, seed=seed + 2)
    flat = net.get_params().astype(np.float64)
    o, parts = 0, {}
    for name, shp in _shapes(n_in, n_hidden, Tn.shape[1]):
        n = int(np.prod(shp))
        parts[name] = flat[o:o + n].reshape(shp)
        o += n
    parts["W3"] = parts["W3"] * sd[:, None]
    parts["b3"] = parts["b3"] * sd + mu
    net.set_params(np.concatenate([parts[name].ravel() for name, _ in _shapes(n_in, n_hidden, Tn.shape[1])])
                   .astype(np.float32))
    return net
