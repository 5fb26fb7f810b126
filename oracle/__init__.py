"""CPU FP64 oracle for the modified Hermite integrators (Dittmann 2020).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_2006_02501_gb300``) never imports, links or runs it, and the two share
no code: the oracle is plain C (``mh_oracle.c``, compiled with gcc and
``-ffp-contract=off``) plus the exact-rational algebra in ``coeffs.py``.

Array conventions (all float64, C-contiguous):
  m        (N,)
  x2, ...  (..., 2)      double-double values (hi, lo), value = hi + lo, for the
                         binary128 oracle of the double-double form (dd_*)
  x, v     (N, 3)
  derivs   (N, 2p, 3)    a^(0) .. a^(2p-1) of each particle
  traj     (N, P+1, 3)   x, v, a, a-dot, ... fed to a direct-summation evaluation
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mh_oracle.c")
_LIB = os.path.join(_HERE, "libmh_oracle.so")
_lock = threading.Lock()
_lib = None


_SRC_Q = os.path.join(_HERE, "mh_oracle_q.c")
_LIB_Q = os.path.join(_HERE, "libmh_oracle_q.so")
_lib_q = None


def _compile(src: str, lib: str, force: bool) -> None:
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", src, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)


def build(force: bool = False) -> str:
    """Compile the C oracles with gcc (plain -O2, no FMA contraction, OpenMP over
    i): the FP64 oracle and its binary128 twin for the double-double form."""
    _compile(_SRC, _LIB, force)
    _compile(_SRC_Q, _LIB_Q, force)
    return _LIB


_D = ctypes.POINTER(ctypes.c_double)


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i, d = ctypes.c_int, ctypes.c_double
            lib.orc_beta.argtypes = [i]
            lib.orc_beta.restype = d
            lib.orc_corrector_weights.argtypes = [i, i, _D, _D]
            lib.orc_hermite_interp.argtypes = [i, d, _D, _D, i, _D]
            lib.orc_pair_derivs.argtypes = [i, _D, d, d, _D]
            lib.orc_evaluate.argtypes = [i, i, _D, _D, d, d, i, i, _D]
            lib.orc_initialise.argtypes = [i, i, _D, _D, _D, d, d, _D]
            lib.orc_predict.argtypes = [i, i, d, _D, _D, _D, _D, _D, _D]
            lib.orc_correct.argtypes = [i, i, i, d, _D, _D, _D, _D, _D, _D]
            lib.orc_step.argtypes = [i, i, i, i, d, _D, d, d, _D, _D, _D]
            lib.orc_run.argtypes = [i, i, i, i, d, i, _D, d, d, _D, _D, _D]
            lib.orc_run_comp.argtypes = [i, i, i, i, d, i, _D, d, d, _D, _D, _D, _D]
            lib.orc_energy.argtypes = [i, _D, _D, _D, d, d]
            lib.orc_energy.restype = d
            lib.orc_ecc.argtypes = [i, _D, _D, _D, d, i, _D]
            lib.orc_timestep_H.argtypes = [i, _D, _D, d, d, d]
            lib.orc_run_timesym.argtypes = [i, i, i, i, i, d, i, _D, d, d, _D, _D, _D, _D, _D]
            lib.orc_run_timesym.restype = d
            lib.orc_timestep_H.restype = d
            LL = ctypes.POINTER(ctypes.c_longlong)
            IP = ctypes.POINTER(ctypes.c_int)
            lib.orc_aarseth_dt.argtypes = [_D, d]
            lib.orc_aarseth_dt.restype = d
            lib.orc_block_level.argtypes = [d, d, i, i, ctypes.c_longlong]
            lib.orc_block_init_levels.argtypes = [i, i, _D, d, d, i, IP]
            lib.orc_block_step.argtypes = [i, i, i, i, d, i, d, _D, d, d, _D, _D, _D, LL, IP, LL]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def order_to_p(order: int) -> int:
    """Order 2(p+1) -> p (Section 2: p derivatives of a give order 2(p+1)); the
    paper's schemes are of arbitrary order, the oracle takes 4 .. 12."""
    if order not in (4, 6, 8, 10, 12):
        raise ValueError("order must be 4, 6, 8, 10 or 12")
    return order // 2 - 1


# --------------------------------------------------------------------------- #
# Hermite algebra (Section 2)
# --------------------------------------------------------------------------- #

def beta(p: int) -> float:
    return _lib_handle().orc_beta(p)


def corrector_weights(p: int, modified: bool = True):
    """(cv, cx) on the F+- vectors, from solving the Eq. 8 system in double."""
    cv = np.zeros(8)
    cx = np.zeros(8)
    _lib_handle().orc_corrector_weights(p, 0 if modified else 1, _p(cv), _p(cx))
    return cv[:p + 1].copy(), cx[:p + 2].copy()


def hermite_interp(p: int, dt: float, f0, f1, nout: int) -> np.ndarray:
    """f^(0..nout-1) at the end of the step from f^(0..p) at both ends."""
    f0, f1 = _f64(f0).reshape(p + 1, 3), _f64(f1).reshape(p + 1, 3)
    out = np.zeros((nout, 3))
    _lib_handle().orc_hermite_interp(p, dt, _p(f0), _p(f1), nout, _p(out))
    return out


# --------------------------------------------------------------------------- #
# pair derivatives and direct summation (Section 3)
# --------------------------------------------------------------------------- #

def pair_derivs(P: int, r, eps: float, Gm: float) -> np.ndarray:
    """Time derivatives 0..P of G m r (r.r+eps^2)^(-3/2); r: (P+1, 3) relative
    trajectory derivatives."""
    r = _f64(r).reshape(P + 1, 3)
    out = np.zeros((P + 1, 3))
    _lib_handle().orc_pair_derivs(P, _p(r), eps * eps, Gm, _p(out))
    return out


def evaluate(m, traj, eps: float, G: float = 1.0, i0: int = 0, i1: int | None = None) -> np.ndarray:
    """Direct-summation derivatives a^(0..P) for particles i0..i1-1."""
    m = _f64(m)
    traj = _f64(traj)
    N, K, _ = traj.shape
    i1 = N if i1 is None else i1
    out = np.zeros((i1 - i0, K, 3))
    _lib_handle().orc_evaluate(N, K - 1, _p(m), _p(traj), eps, G, i0, i1, _p(out))
    return out


def initialise(order: int, m, x, v, eps: float, G: float = 1.0) -> np.ndarray:
    """a^(0..2p-1) at t = 0 by explicit pair derivatives (Section 3 intro)."""
    p = order_to_p(order)
    m, x, v = _f64(m), _f64(x), _f64(v)
    N = m.shape[0]
    d = np.zeros((N, 2 * p, 3))
    _lib_handle().orc_initialise(N, p, _p(m), _p(x), _p(v), eps, G, _p(d))
    return d


def predict(order: int, dt: float, x, v, derivs):
    p = order_to_p(order)
    x, v, derivs = _f64(x), _f64(v), _f64(derivs)
    N = x.shape[0]
    xp, vp = np.zeros((N, 3)), np.zeros((N, 3))
    ap = np.zeros((N, max(p - 1, 1), 3))
    _lib_handle().orc_predict(N, p, dt, _p(x), _p(v), _p(derivs), _p(xp), _p(vp), _p(ap))
    return xp, vp, ap[:, :max(p - 1, 0)]


def correct(order: int, dt: float, x0, v0, d0, d1, modified: bool = True):
    """Corrector (Eqs. 5-7): d0, d1 are (N, p+1, 3) derivative stacks at t, t+dt."""
    p = order_to_p(order)
    x0, v0, d0, d1 = _f64(x0), _f64(v0), _f64(d0), _f64(d1)
    N = x0.shape[0]
    x1, v1 = np.zeros((N, 3)), np.zeros((N, 3))
    _lib_handle().orc_correct(N, p, 0 if modified else 1, dt, _p(x0), _p(v0), _p(d0), _p(d1),
                              _p(x1), _p(v1))
    return x1, v1


class State:
    """A simulation state held by the oracle: x, v, derivs (a^(0..2p-1)), m."""

    def __init__(self, order: int, m, x, v, eps: float, G: float = 1.0, derivs=None,
                 modified: bool = True):
        self.order = order
        self.p = order_to_p(order)
        self.m = _f64(m).copy()
        self.x = _f64(x).copy()
        self.v = _f64(v).copy()
        self.eps = float(eps)
        self.G = float(G)
        self.modified = modified
        self.t = 0.0
        self.derivs = initialise(order, self.m, self.x, self.v, eps, G) if derivs is None \
            else _f64(derivs).copy()

    @property
    def N(self) -> int:
        return self.m.shape[0]

    def step(self, dt: float, n_iter: int, nsteps: int = 1, compensated: bool = False) -> None:
        """nsteps shared P(EC)^n steps of constant dt (negative dt runs backward).
        compensated: Kahan-compensated summation of the x, v updates (Section
        3.2); the compensation is carried in self.comp between calls."""
        if compensated:
            if getattr(self, "comp", None) is None:
                self.comp = np.zeros((self.N, 6))
            _lib_handle().orc_run_comp(self.N, self.p, 0 if self.modified else 1, n_iter, dt, nsteps,
                                       _p(self.m), self.eps, self.G, _p(self.x), _p(self.v),
                                       _p(self.derivs), _p(self.comp))
        else:
            _lib_handle().orc_run(self.N, self.p, 0 if self.modified else 1, n_iter, dt, nsteps,
                                  _p(self.m), self.eps, self.G, _p(self.x), _p(self.v),
                                  _p(self.derivs))
        self.t += dt * nsteps

    def step_timesym(self, eta: float, n_iter: int, nsteps: int = 1, backward: bool = False) -> np.ndarray:
        """nsteps time-symmetric variable steps (Section 3.3): dt = (H- + H+)/2 with
        H of Eq. 24, H+ re-evaluated in every pass of P(EC)^n.  H- of the first
        step is Eq. 24 at the current positions unless a previous call left the
        next step's H- (self.H).  Returns the step sizes taken."""
        if getattr(self, "H", None) is None or getattr(self, "H_eta", None) != eta:
            self.H = timestep_H(self.m, self.x, self.eps, eta, self.G)
            self.H_eta = eta
        Hc = ctypes.c_double(self.H)
        dts = np.zeros(nsteps)
        adv = _lib_handle().orc_run_timesym(self.N, self.p, 0 if self.modified else 1, n_iter,
                                            -1 if backward else 1, eta, nsteps, _p(self.m), self.eps,
                                            self.G, _p(self.x), _p(self.v), _p(self.derivs),
                                            ctypes.byref(Hc), _p(dts))
        self.H = Hc.value
        self.t += adv
        return dts

    def energy(self) -> float:
        return energy(self.m, self.x, self.v, self.eps, self.G)

    def ecc(self, central: int = 0) -> np.ndarray:
        return ecc(self.m, self.x, self.v, self.G, central)

    def copy(self) -> "State":
        s = State.__new__(State)
        s.__dict__.update({k: (v.copy() if isinstance(v, np.ndarray) else v)
                           for k, v in self.__dict__.items()})
        return s


def energy(m, x, v, eps: float, G: float = 1.0) -> float:
    m, x, v = _f64(m), _f64(x), _f64(v)
    return _lib_handle().orc_energy(m.shape[0], _p(m), _p(x), _p(v), eps, G)


def ecc(m, x, v, G: float = 1.0, central: int = 0) -> np.ndarray:
    m, x, v = _f64(m), _f64(x), _f64(v)
    e = np.zeros_like(x)
    _lib_handle().orc_ecc(m.shape[0], _p(m), _p(x), _p(v), G, central, _p(e))
    return e


def timestep_H(m, x, eps: float, eta: float, G: float = 1.0) -> float:
    """Eq. 24: eta times the shortest two-body time scale sqrt(s^1.5 / (G (m_i + m_j)))."""
    m, x = _f64(m), _f64(x)
    return _lib_handle().orc_timestep_H(m.shape[0], _p(m), _p(x), eps, eta, G)


# --------------------------------------------------------------------------- #
# block time steps (Section 4 option; scheme of reading R12)
# --------------------------------------------------------------------------- #

def aarseth_dt(d, eta: float) -> float:
    d = _f64(d).reshape(-1, 3)
    return _lib_handle().orc_aarseth_dt(_p(d), eta)


def block_level(dt_c: float, dt_max: float, k_max: int, k_old: int = -1, T: int = 0) -> int:
    return _lib_handle().orc_block_level(dt_c, dt_max, k_max, k_old, T)


class BlockState(State):
    """Oracle state advanced by block time steps: every body has its own tick
    T (units of dt_max 2^-k_max) and level (step dt_max 2^-level)."""

    def __init__(self, order: int, m, x, v, eps: float, dt_max: float, k_max: int, eta: float,
                 G: float = 1.0, modified: bool = True, derivs=None, level=None):
        super().__init__(order, m, x, v, eps, G=G, derivs=derivs, modified=modified)
        if self.p < 2:
            raise ValueError("block steps need order 6 or 8")
        self.dt_max, self.k_max, self.eta = float(dt_max), int(k_max), float(eta)
        self.T = np.zeros(self.N, dtype=np.int64)
        if level is None:
            self.level = np.zeros(self.N, dtype=np.int32)
            _lib_handle().orc_block_init_levels(self.N, self.p, _p(self.derivs), self.eta, self.dt_max,
                                                self.k_max, self.level.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        else:
            self.level = np.ascontiguousarray(level, dtype=np.int32).copy()
        self.block_steps = 0
        self.active_total = 0

    @property
    def tick(self) -> float:
        return self.dt_max * 2.0 ** -self.k_max

    def block_step(self, n_iter: int) -> int:
        Tn = ctypes.c_longlong(0)
        n_act = _lib_handle().orc_block_step(
            self.N, self.p, 0 if self.modified else 1, n_iter, self.dt_max, self.k_max, self.eta,
            _p(self.m), self.eps, self.G, _p(self.x), _p(self.v), _p(self.derivs),
            self.T.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
            self.level.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.byref(Tn))
        self.block_steps += 1
        self.active_total += n_act
        self.t = Tn.value * self.tick
        return n_act

    def advance(self, dt: float, n_iter: int) -> None:
        """Block steps until every body reaches the current time + dt (a multiple of dt_max)."""
        target = int(round((self.T.max() * self.tick + dt) / self.tick))
        while self.T.min() < target:
            self.block_step(n_iter)


# --------------------------------------------------------------------------- #
# binary128 oracle of the double-double form (mh_oracle_q.c)
# --------------------------------------------------------------------------- #

def _lib_q_handle():
    global _lib_q
    with _lock:
        if _lib_q is None:
            build()
            lib = ctypes.CDLL(_LIB_Q)
            i, d = ctypes.c_int, ctypes.c_double
            lib.orq_corrector_weights.argtypes = [i, i, _D, _D]
            lib.orq_hermite_interp.argtypes = [i, d, _D, _D, i, _D]
            lib.orq_run.argtypes = [i, i, i, i, d, i, _D, d, d, i, _D, _D, _D]
            lib.orq_energy.argtypes = [i, _D, _D, _D, d, d, _D]
            lib.orq_evaluate.argtypes = [i, i, _D, _D, d, d, i, i, _D]
            lib.orq_ecc.argtypes = [i, _D, _D, _D, d, i, _D]
            _lib_q = lib
    return _lib_q


def as_dd(a) -> np.ndarray:
    """Doubles as a double-double array (..., 2) with lo = 0."""
    a = np.asarray(a, dtype=np.float64)
    return np.ascontiguousarray(np.stack([a, np.zeros_like(a)], axis=-1))


def dd_value(a2) -> np.ndarray:
    """hi + lo rounded to double (for display and FP64 comparisons)."""
    a2 = np.asarray(a2)
    return a2[..., 0] + a2[..., 1]


def dd_corrector_weights(p: int, modified: bool = True):
    """(cv, cx) on the F+- vectors from the Eq. 8 system solved in binary128,
    as double-double pairs: (p+1, 2) and (p+2, 2)."""
    cv, cx = np.zeros((8, 2)), np.zeros((8, 2))
    _lib_q_handle().orq_corrector_weights(p, 0 if modified else 1, _p(cv), _p(cx))
    return cv[:p + 1].copy(), cx[:p + 2].copy()


def dd_hermite_interp(p: int, dt: float, f0_2, f1_2, nout: int) -> np.ndarray:
    """f^(0..nout-1) at the end of the step (binary128), from (p+1, 3, 2) pairs."""
    f0_2 = _f64(f0_2).reshape(p + 1, 3, 2)
    f1_2 = _f64(f1_2).reshape(p + 1, 3, 2)
    out = np.zeros((nout, 3, 2))
    _lib_q_handle().orq_hermite_interp(p, dt, _p(f0_2), _p(f1_2), nout, _p(out))
    return out


def dd_run(order: int, m, x2, v2, eps: float, dt: float, n_iter: int, nsteps: int,
           G: float = 1.0, modified: bool = True, d2=None):
    """Initialise (d2 None) and take nsteps constant P(EC)^n steps, all in
    binary128.  x2, v2: (N, 3, 2) pairs (or (N, 3) doubles); d2: (N, 2p, 3, 2).
    Returns (x2, v2, d2) rounded to double-double pairs."""
    p = order_to_p(order)
    m = _f64(m)
    N = m.shape[0]
    x2 = _f64(x2).copy() if np.asarray(x2).ndim == 3 else as_dd(x2)
    v2 = _f64(v2).copy() if np.asarray(v2).ndim == 3 else as_dd(v2)
    init = d2 is None
    d2 = np.zeros((N, 2 * p, 3, 2)) if init else _f64(d2).copy()
    _lib_q_handle().orq_run(N, p, 0 if modified else 1, n_iter, dt, nsteps, _p(m), eps, G,
                            1 if init else 0, _p(x2), _p(v2), _p(d2))
    return x2, v2, d2


def dd_evaluate(m, traj2, eps: float, G: float = 1.0, i0: int = 0, i1: int | None = None) -> np.ndarray:
    """Direct-summation a^(0..P) in binary128 for bodies i0..i1-1 (pairs out):
    traj2 (N, P+1, 3, 2) trajectory pairs x, v, a, ...; returns (i1-i0, P+1, 3, 2)."""
    m, traj2 = _f64(m), _f64(traj2)
    N, K = traj2.shape[0], traj2.shape[1]
    i1 = N if i1 is None else i1
    out = np.zeros((i1 - i0, K, 3, 2))
    _lib_q_handle().orq_evaluate(N, K - 1, _p(m), _p(traj2), eps, G, i0, i1, _p(out))
    return out


def dd_energy(m, x2, v2, eps: float, G: float = 1.0) -> np.ndarray:
    """Energy (R4) in binary128 as a (hi, lo) pair."""
    m, x2, v2 = _f64(m), _f64(x2), _f64(v2)
    E2 = np.zeros(2)
    _lib_q_handle().orq_energy(m.shape[0], _p(m), _p(x2), _p(v2), eps, G, _p(E2))
    return E2


def dd_ecc(m, x2, v2, G: float = 1.0, central: int = 0) -> np.ndarray:
    """Eccentricity vectors (Eq. A1) in binary128 as (N, 3, 2) pairs."""
    m, x2, v2 = _f64(m), _f64(x2), _f64(v2)
    e2 = np.zeros_like(x2)
    _lib_q_handle().orq_ecc(m.shape[0], _p(m), _p(x2), _p(v2), G, central, _p(e2))
    return e2
