"""GB300-native modified Hermite N-body integrators (Dittmann 2020), orders 4, 6, 8.

Thin Python binding over the C ABI of include/mh.h.  Every step of the
integration runs in the library's CUDA kernels; this module only marshals
arguments (numpy arrays for host data, torch tensors or raw pointers for
device data and streams).

    sim = Simulation(order=8, m=m, x=x, v=v, eps=1e-4)
    sim.step(dt, n_iter=3)
    t, x, v, derivs = sim.sync()
    E, ecc = sim.diagnostics(central=0)
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi
from ._capi import (MH_BETA_MODIFIED, MH_BETA_STANDARD, MH_PREC_FP32PAIR, MH_PREC_FP64,  # noqa: F401
                    MHError, check)

__all__ = ["Simulation", "Batch", "DDSimulation", "DDBatch", "MLP", "pair_eval", "MHError", "build_library", "MH_PREC_FP64", "MH_PREC_FP32PAIR",
           "MH_BETA_MODIFIED", "MH_BETA_STANDARD"]

_DP = ctypes.POINTER(ctypes.c_double)


def build_library(force: bool = False) -> str:
    """Compile lib/libmh.so (nvcc, sm_103a) if it is missing or stale."""
    from .build import build as _b
    return _b(force=force)


def _host(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        a = a.reshape(shape)
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)        # torch.cuda.Stream


def _config(order, precision, beta, G, split_j, heavy_frac, block, symmetric, fp32_variant, timesym_eta,
            compensated) -> "_capi.Config":
    cfg = _capi.Config()
    _capi.lib().mh_config_default(ctypes.byref(cfg))
    cfg.order, cfg.precision, cfg.beta_mode, cfg.G, cfg.split_j = order, precision, beta, G, split_j
    if heavy_frac is not None:
        cfg.heavy_frac = heavy_frac
    cfg.symmetric = int(symmetric)
    cfg.fp32_variant = int(fp32_variant)
    cfg.compensated = 1 if compensated else 0
    if timesym_eta is not None:
        cfg.step_mode = _capi.MH_STEP_TIMESYM
        cfg.eta = float(timesym_eta)
    if block is not None:
        cfg.step_mode = _capi.MH_STEP_BLOCK
        cfg.dt_max = float(block.get("dt_max", cfg.dt_max))
        cfg.k_max = int(block.get("k_max", cfg.k_max))
        cfg.eta = float(block.get("eta", cfg.eta))
    return cfg


class Simulation:
    """One N-body system advanced by the shared-step P(EC)^n scheme.

    order: 4, 6, 8, 10 or 12 (10 and 12: FP64 form, shared or time-symmetric
    steps); precision: MH_PREC_FP64 or MH_PREC_FP32PAIR; beta:
    MH_BETA_MODIFIED (Eq. 20) or MH_BETA_STANDARD (beta = 1); stream: a
    torch.cuda.Stream, a raw cudaStream_t integer, or None (library stream);
    heavy_frac: precision form, mass fraction above which a source body's
    pairs run in FP64 (None = library default 1e-3, 0 = all pairs FP32);
    block: None for shared steps, or {"dt_max", "k_max", "eta"} for block time
    steps (order 6 or 8; step() then needs a multiple of dt_max);
    symmetric: FP64 evaluation of each unordered pair once, both bodies
    updated: 1/True = from 2048 padded bodies up (default), 2 = always,
    0/False = never (every ordered pair);
    fp32_variant: precision form evaluation kernel, 0 = autotuned, 1/2/3 fixed
    (one i-body per thread, two, two in packed FP32x2 lanes);
    timesym_eta: not None for time-symmetric variable shared steps with this
    eta of Eq. 24 (FP64; advance with step_timesym());
    compensated: compensated summation of the x, v updates (shared steps).
    """

    def __init__(self, order: int, m, x, v, eps: float, precision: int = MH_PREC_FP64,
                 beta: int = MH_BETA_MODIFIED, G: float = 1.0, stream=None, split_j: int = 0,
                 heavy_frac: float | None = None, block: dict | None = None,
                 symmetric: int = 1, fp32_variant: int = 0, timesym_eta: float | None = None,
                 compensated: bool = False):
        L = _capi.lib()
        m = _host(m)
        N = m.shape[0]
        x, v = _host(x, (N, 3)), _host(v, (N, 3))
        cfg = _config(order, precision, beta, G, split_j, heavy_frac, block, symmetric, fp32_variant,
                      timesym_eta, compensated)
        h = ctypes.c_void_p()
        check(L.mh_create(ctypes.byref(h), N, order, _ptr(m), _ptr(x), _ptr(v), float(eps),
                          ctypes.byref(cfg), _stream_handle(stream)))
        self._adopt(h, N, order, eps, G, precision, block)

    def _adopt(self, h, N, order, eps, G, precision, block):
        self._h = h
        self.N, self.order, self.p = N, order, order // 2 - 1
        self.eps, self.G, self.precision = eps, G, precision
        self.block = block is not None

    @classmethod
    def restore(cls, order: int, m, state: dict, eps: float, precision: int = MH_PREC_FP64,
                beta: int = MH_BETA_MODIFIED, G: float = 1.0, stream=None, split_j: int = 0,
                heavy_frac: float | None = None, block: dict | None = None, symmetric: int = 1,
                fp32_variant: int = 0, timesym_eta: float | None = None, compensated: bool = False):
        """A simulation created from checkpoint() output (mh_restore): no
        initialisation passes; continuing it reproduces the uninterrupted run bit
        for bit for shared and block steps.  The other arguments as for __init__."""
        m = _host(m)
        N = m.shape[0]
        x, v = _host(state["x"], (N, 3)), _host(state["v"], (N, 3))
        d = _host(state["derivs"], (N, 2 * (order // 2 - 1), 3))
        lv = state.get("level")
        lp = None
        if lv is not None:
            lv = np.ascontiguousarray(lv, dtype=np.int32)
            lp = lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        st = _capi.StateC(float(state["t"]), _ptr(x), _ptr(v), _ptr(d), lp)
        cfg = _config(order, precision, beta, G, split_j, heavy_frac, block, symmetric, fp32_variant,
                      timesym_eta, compensated)
        h = ctypes.c_void_p()
        check(_capi.lib().mh_restore(ctypes.byref(h), N, order, _ptr(m), ctypes.byref(st), float(eps),
                                     ctypes.byref(cfg), _stream_handle(stream)))
        sim = cls.__new__(cls)
        sim._adopt(h, N, order, eps, G, precision, block)
        return sim

    def checkpoint(self) -> dict:
        """{t, x, v, derivs[, level]}: everything mh_restore needs."""
        t, x, v, d = self.sync()
        out = {"t": t, "x": x, "v": v, "derivs": d}
        if self.block:
            out["level"] = self.levels()
        return out

    def close(self) -> None:
        if getattr(self, "_h", None):
            _capi.lib().mh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def step(self, dt: float, n_iter: int, nsteps: int = 1) -> None:
        L = _capi.lib()
        for _ in range(nsteps):
            check(L.mh_step(self._h, float(dt), int(n_iter)))

    def step_timesym(self, nsteps: int, n_iter: int, backward: bool = False) -> None:
        """nsteps time-symmetric variable steps (Section 3.3), stream-ordered."""
        check(_capi.lib().mh_step_timesym(self._h, int(nsteps), int(n_iter), 1 if backward else 0))

    def sync(self):
        """(t, x (N,3), v (N,3), derivs (N,2p,3)) copied to the host."""
        x = np.zeros((self.N, 3))
        v = np.zeros((self.N, 3))
        d = np.zeros((self.N, 2 * self.p, 3))
        st = _capi.StateC(0.0, _ptr(x), _ptr(v), _ptr(d), None)
        check(_capi.lib().mh_sync(self._h, ctypes.byref(st)))
        return st.t, x, v, d

    def levels(self) -> np.ndarray:
        """Block steps: the level of every body (step dt_max 2^-level)."""
        lv = np.zeros(self.N, dtype=np.int32)
        st = _capi.StateC(0.0, None, None, None, lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        check(_capi.lib().mh_sync(self._h, ctypes.byref(st)))
        return lv

    def set_state(self, x, v, derivs=None, t: float = 0.0, level=None) -> None:
        x, v = _host(x, (self.N, 3)), _host(v, (self.N, 3))
        dp = lp = None
        if derivs is not None:
            derivs = _host(derivs, (self.N, 2 * self.p, 3))
            dp = _ptr(derivs)
        if level is not None:
            level = np.ascontiguousarray(level, dtype=np.int32)
            lp = level.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        st = _capi.StateC(float(t), _ptr(x), _ptr(v), dp, lp)
        check(_capi.lib().mh_set_state(self._h, ctypes.byref(st)))

    def diagnostics(self, central: int = 0, energy: bool = True, ecc: bool = True):
        e = ctypes.c_double(0.0)
        ev = np.zeros((self.N, 3)) if ecc else None
        check(_capi.lib().mh_diagnostics(self._h, ctypes.byref(e) if energy else None,
                                         _ptr(ev) if ecc else None, int(central)))
        return (e.value if energy else None), ev

    def energy(self) -> float:
        return self.diagnostics(energy=True, ecc=False)[0]

    def step_converge(self, dt: float, tol: float, max_iter: int) -> int:
        """One step with evaluate-correct passes until the largest position change
        is at most tol * max|x| (at most max_iter); returns the passes used."""
        n = ctypes.c_int(0)
        check(_capi.lib().mh_step_converge(self._h, float(dt), float(tol), int(max_iter), ctypes.byref(n)))
        return n.value

    def predict(self, dt: float):
        """(x, v) the predictor gives for t + dt (Taylor, plus the learned residual
        when a network is set); the state is not advanced."""
        x = np.zeros((self.N, 3))
        v = np.zeros((self.N, 3))
        check(_capi.lib().mh_predict(self._h, float(dt), _ptr(x), _ptr(v)))
        return x, v

    def set_predictor(self, net) -> None:
        """Use the learned residual of `net` (an MLP) on the Taylor predictor; None = plain."""
        check(_capi.lib().mh_set_predictor(self._h, None if net is None else net._h))
        self._net = net                     # keep the network alive while it is used

    def collect_samples(self, dt: float, n_iter: int, feats, targets) -> None:
        """One plain step with n_iter passes; writes N rows of features and targets
        into the device tensors feats (N x (6p+1) float32) and targets (N x 6 float32)."""
        check(_capi.lib().mh_collect_samples(self._h, float(dt), int(n_iter), _dev_ptr(feats), _dev_ptr(targets)))

    def set_timing(self, on: bool) -> None:
        """Bracket every O(N^2) evaluation launch with CUDA events (see counters())."""
        check(_capi.lib().mh_set_timing(self._h, 1 if on else 0))

    def counters(self) -> dict:
        n, o, c = ctypes.c_int64(), ctypes.c_int(), _capi.Counters()
        check(_capi.lib().mh_info(self._h, ctypes.byref(n), ctypes.byref(o), ctypes.byref(c)))
        out = {f: getattr(c, f) for f, _ in c._fields_}
        out["pair_tune_ms_x1000"] = list(out["pair_tune_ms_x1000"])
        return out


class MLP:
    """n_in -> hidden -> hidden -> n_out SiLU network on the GPU (BF16 operands,
    FP32 accumulation on the tensor cores); trained by the library's kernels."""

    def __init__(self, n_in: int, n_hidden: int = 128, n_out: int = 6, seed: int = 0):
        h = ctypes.c_void_p()
        check(_capi.lib().mh_mlp_create(ctypes.byref(h), int(n_in), int(n_hidden), int(n_out), int(seed)))
        self._h = h
        self.n_in, self.n_hidden, self.n_out = n_in, n_hidden, n_out
        c = ctypes.c_int64()
        check(_capi.lib().mh_mlp_num_params(self._h, ctypes.byref(c)))
        self.n_params = c.value

    def close(self) -> None:
        if getattr(self, "_h", None):
            _capi.lib().mh_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        check(_capi.lib().mh_mlp_get_params(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), out.size))
        return out

    def set_params(self, flat) -> None:
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        check(_capi.lib().mh_mlp_set_params(self._h, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), flat.size))

    def forward(self, x, y, stream=None) -> None:
        """y = net(x) on device tensors (rows x n_in, rows x n_out, float32)."""
        check(_capi.lib().mh_mlp_forward(self._h, _dev_ptr(x), _dev_ptr(y), int(x.shape[0]),
                                         _stream_handle(stream)))

    def loss_grad(self, x, t, stream=None):
        """(loss, gradient as n_params float32 on the host)."""
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = ctypes.c_double()
        check(_capi.lib().mh_mlp_loss_grad(self._h, _dev_ptr(x), _dev_ptr(t), int(x.shape[0]), ctypes.byref(loss),
                                           g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _stream_handle(stream)))
        return loss.value, g

    def train(self, x, t, epochs: int, batch: int, lr: float, seed: int = 0, stream=None) -> float:
        loss = ctypes.c_double()
        check(_capi.lib().mh_mlp_train(self._h, _dev_ptr(x), _dev_ptr(t), int(x.shape[0]), int(epochs), int(batch),
                                       float(lr), int(seed), ctypes.byref(loss), _stream_handle(stream)))
        return loss.value


class Batch:
    """Many independent small systems (1..64 bodies each) advanced together by
    one persistent kernel launch per call (FP64, shared steps per system).

    offsets: (S+1,) int64 body offsets; m, x, v: the concatenated bodies;
    dt: (S,) step of each system.
    """

    def __init__(self, order: int, offsets, m, x, v, dt, eps: float, beta: int = MH_BETA_MODIFIED,
                 G: float = 1.0, stream=None):
        L = _capi.lib()
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        S = offsets.shape[0] - 1
        m = _host(m)
        N = m.shape[0]
        x, v, dt = _host(x, (N, 3)), _host(v, (N, 3)), _host(dt, (S,))
        cfg = _capi.Config()
        L.mh_config_default(ctypes.byref(cfg))
        cfg.order, cfg.beta_mode, cfg.G = order, beta, G
        h = ctypes.c_void_p()
        check(L.mh_create_batch(ctypes.byref(h), S, offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                _ptr(m), _ptr(x), _ptr(v), _ptr(dt), float(eps), order, ctypes.byref(cfg),
                                _stream_handle(stream)))
        self._h = h
        self.S, self.N, self.order, self.p = S, N, order, order // 2 - 1
        self.offsets = offsets

    close = Simulation.close
    __del__ = Simulation.__del__
    __enter__ = Simulation.__enter__
    __exit__ = Simulation.__exit__
    sync = Simulation.sync
    counters = Simulation.counters

    def step(self, n_steps: int, n_iter: int) -> None:
        check(_capi.lib().mh_step_batch(self._h, int(n_steps), int(n_iter)))

    def tune(self, probe_steps: int = 8, n_iter: int = 2):
        w, o = ctypes.c_int(), ctypes.c_int()
        check(_capi.lib().mh_batch_tune(self._h, int(probe_steps), int(n_iter), ctypes.byref(w), ctypes.byref(o)))
        return w.value, o.value

    def energies(self) -> np.ndarray:
        e = np.zeros(self.S)
        check(_capi.lib().mh_batch_energy(self._h, _ptr(e)))
        return e


def _dd_host(a, N: int, K: int = 3) -> np.ndarray:
    """(N, K, 2) double-double pairs from pairs or from plain doubles (lo = 0)."""
    a = np.asarray(a, dtype=np.float64)
    if a.ndim >= 1 and a.shape[-1] == 2 and a.size == N * K * 2:
        return np.ascontiguousarray(a.reshape(N, K, 2))
    a = a.reshape(N, K)
    return np.ascontiguousarray(np.stack([a, np.zeros_like(a)], axis=-1))


class DDSimulation:
    """One system integrated in double-double arithmetic (mh_dd_*): the state,
    the prediction, every pair term and every sum carry ~106 bits, so that the
    high-order schemes can be run below the round-off of FP64 (Section 3.1;
    Discussion).  Shared constant steps, orders 4 to 12.

    x, v: (N, 3) doubles or (N, 3, 2) (hi, lo) pairs.  Results come back as
    (..., 2) pairs; value = hi + lo.  symmetric: each unordered pair evaluated
    once for both bodies (k_dd_pair_sym), 1 = from 2048 bodies up (default),
    2 = always, 0 = never.
    """

    def __init__(self, order: int, m, x, v, eps: float, beta: int = MH_BETA_MODIFIED, G: float = 1.0,
                 stream=None, symmetric: int = 1):
        L = _capi.lib()
        m = _host(m)
        N = m.shape[0]
        x2, v2 = _dd_host(x, N), _dd_host(v, N)
        cfg = _capi.Config()
        L.mh_config_default(ctypes.byref(cfg))
        cfg.order, cfg.beta_mode, cfg.G, cfg.symmetric = order, beta, G, int(symmetric)
        h = ctypes.c_void_p()
        check(L.mh_dd_create(ctypes.byref(h), N, order, _ptr(m), _ptr(x2), _ptr(v2), float(eps),
                             ctypes.byref(cfg), _stream_handle(stream)))
        self._h = h
        self.N, self.order, self.p = N, order, order // 2 - 1

    def close(self) -> None:
        if getattr(self, "_h", None):
            _capi.lib().mh_dd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def step(self, dt: float, n_iter: int, nsteps: int = 1) -> None:
        check(_capi.lib().mh_dd_step(self._h, float(dt), int(n_iter), int(nsteps)))

    def sync(self):
        """(t2, x2, v2, d2): time (2,), positions and velocities (N, 3, 2), a^(0..2p-1) (N, 2p, 3, 2)."""
        t2 = np.zeros(2)
        x2, v2 = np.zeros((self.N, 3, 2)), np.zeros((self.N, 3, 2))
        d2 = np.zeros((self.N, 2 * self.p, 3, 2))
        check(_capi.lib().mh_dd_sync(self._h, _ptr(t2), _ptr(x2), _ptr(v2), _ptr(d2)))
        return t2, x2, v2, d2

    def set_state(self, x, v, derivs=None, t2=None) -> None:
        x2, v2 = _dd_host(x, self.N), _dd_host(v, self.N)
        d2 = None if derivs is None else _dd_host(derivs, self.N, 2 * self.p * 3)
        t2 = None if t2 is None else np.ascontiguousarray(t2, dtype=np.float64).reshape(2)
        check(_capi.lib().mh_dd_set_state(self._h, None if t2 is None else _ptr(t2), _ptr(x2), _ptr(v2),
                                          None if d2 is None else _ptr(d2)))

    def diagnostics(self, central: int = 0):
        """(E2, ecc2): the energy as a (2,) pair and the eccentricity vectors (N, 3, 2)."""
        E2 = np.zeros(2)
        e2 = np.zeros((self.N, 3, 2))
        check(_capi.lib().mh_dd_diagnostics(self._h, _ptr(E2), _ptr(e2), int(central)))
        return E2, e2

    def counters(self) -> dict:
        c = _capi.Counters()
        check(_capi.lib().mh_dd_info(self._h, None, None, ctypes.byref(c)))
        return {f: getattr(c, f) for f, _ in c._fields_ if f != "pair_tune_ms_x1000"}


class DDBatch(DDSimulation):
    """Many independent systems (1..64 bodies each) in double-double, advanced
    together with shared steps of each system's own dt (mh_dd_create_batch).

    offsets: (S+1,) int64 body offsets; m, x, v: the concatenated bodies (x, v as
    doubles or (hi, lo) pairs); dt: (S,) steps.
    """

    def __init__(self, order: int, offsets, m, x, v, dt, eps: float, beta: int = MH_BETA_MODIFIED,
                 G: float = 1.0, stream=None):
        L = _capi.lib()
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        S = offsets.shape[0] - 1
        m = _host(m)
        N = m.shape[0]
        x2, v2 = _dd_host(x, N), _dd_host(v, N)
        dt = _host(dt, (S,))
        cfg = _capi.Config()
        L.mh_config_default(ctypes.byref(cfg))
        cfg.order, cfg.beta_mode, cfg.G = order, beta, G
        h = ctypes.c_void_p()
        check(L.mh_dd_create_batch(ctypes.byref(h), S, offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                   _ptr(m), _ptr(x2), _ptr(v2), _ptr(dt), float(eps), order,
                                   ctypes.byref(cfg), _stream_handle(stream)))
        self._h = h
        self.S, self.N, self.order, self.p = S, N, order, order // 2 - 1
        self.offsets = offsets

    def step(self, nsteps: int, n_iter: int) -> None:          # noqa: D401 (batched signature)
        check(_capi.lib().mh_dd_step_batch(self._h, int(nsteps), int(n_iter)))

    def energies(self) -> np.ndarray:
        """(S, 2) energies of the systems as (hi, lo) pairs."""
        e = np.zeros((self.S, 2))
        check(_capi.lib().mh_dd_batch_energy(self._h, _ptr(e)))
        return e


def _dev_ptr(t) -> int:
    if isinstance(t, int):
        return t
    return int(t.data_ptr())


def pair_eval(P: int, precision: int, m, traj, eps: float, out, G: float = 1.0, i0: int = 0,
              i1: int | None = None, stream=None) -> None:
    """Direct-summation a^(0..P) of bodies i0..i1-1 on DEVICE memory.

    m: (N,) float64 device tensor; traj: ((P+1)*3, N) float64 device tensor (row
    3k+c = component c of x, v, a, a-dot, ...); out: ((P+1)*3, i1-i0) float64
    device tensor.  Stream-ordered on `stream` (default: torch's current stream).
    """
    N = int(m.shape[0]) if hasattr(m, "shape") else None
    if N is None:
        raise ValueError("m must be a device tensor")
    i1 = N if i1 is None else i1
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    check(_capi.lib().mh_pair_eval(int(P), int(precision), N, _dev_ptr(m), _dev_ptr(traj), float(eps),
                                   float(G), int(i0), int(i1), _dev_ptr(out), _stream_handle(stream)))


def measure_peaks() -> dict:
    """Measured FP64 / FP32 / packed FP32x2 multiply-add TFLOP/s and MUFU
    reciprocal square roots (10^12/s) of the current device (mh_measure_peaks)."""
    out = (ctypes.c_double * 4)()
    check(_capi.lib().mh_measure_peaks(out))
    return {"fp64_tflops": out[0], "fp32_tflops": out[1], "fp32x2_tflops": out[2], "rsqrt_tera_per_s": out[3]}


def dd_pair_eval(P: int, m, tr2, eps: float, G: float = 1.0, i0: int = 0, i1: int | None = None,
                 symmetric: int = 1) -> np.ndarray:
    """a^(0..P) of bodies i0 .. i1-1 in double-double (mh_dd_pair_eval): tr2 is
    (N, P+1, 3, 2) (hi, lo) trajectory records x, v, a, ...; returns
    (i1-i0, P+1, 3, 2).  symmetric as in DDSimulation."""
    m = _host(m)
    N = m.shape[0]
    tr2 = np.ascontiguousarray(tr2, dtype=np.float64)
    if tr2.shape != (N, P + 1, 3, 2):
        raise ValueError(f"tr2 must be ({N}, {P + 1}, 3, 2)")
    i1 = N if i1 is None else int(i1)
    out = np.zeros((max(i1 - int(i0), 0), P + 1, 3, 2))
    check(_capi.lib().mh_dd_pair_eval(int(P), N, _ptr(m), _ptr(tr2), float(eps), float(G), int(i0), i1,
                                      int(symmetric), _ptr(out)))
    return out


def dd_sym_check(N: int) -> dict:
    """Host-side check of the symmetric double-double kernel's work map for N
    bodies (mh_dd_sym_check; no device needed).  Raises MHError when a block
    pair or a (slot, block) entry is not covered exactly once."""
    info = (ctypes.c_int * 5)()
    check(_capi.lib().mh_dd_sym_check(int(N), info))
    return {"blocks": info[0], "items": info[1], "bad_pairs": info[2], "bad_slots": info[3],
            "bad_body_pairs": info[4]}


def sym_schedule_check(N: int, slots: int, precision: int = MH_PREC_FP64) -> dict:
    """Host-side check of the pair-symmetric evaluation's ordered accumulation
    for N bodies, `slots` resident CTAs and a form (MH_PREC_FP64 or
    MH_PREC_FP32PAIR) (mh_sym_schedule_check; no device needed).  Raises
    MHError when a property fails; returns the plan."""
    info = (ctypes.c_int * 7)()
    check(_capi.lib().mh_sym_schedule_check(int(N), int(slots), int(precision), info))
    return {"blocks": info[0], "chunks": info[1], "distances_per_chunk": info[2], "cyclic": bool(info[3]),
            "grid": info[4], "chains": info[5], "rows_per_item": info[6]}
