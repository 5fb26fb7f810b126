"""C-ABI checks that need no GPU: the library builds and loads, exports every
entry point that include/*.h declares, and rejects bad arguments before
touching the device."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2006_02501_gb300.build import build
    build()
    from paper_2006_02501_gb300 import _capi
    return _capi.lib()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names.update(re.findall(r"\b(mh_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert "mh_create" in names and "mh_step" in names and "mh_sync" in names and "mh_diagnostics" in names
    for n in names:
        assert hasattr(L, n), n
    from paper_2006_02501_gb300 import _capi
    assert sorted(_capi.EXPORTS) == names


def test_config_default(L):
    from paper_2006_02501_gb300 import _capi
    c = _capi.Config()
    L.mh_config_default(ctypes.byref(c))
    assert c.order == 8 and c.G == 1.0 and c.precision == 0 and c.beta_mode == 0 and c.k_max == 12


def _create(L, N, order, m, x, v, eps):
    h = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    ptr = lambda a: None if a is None else a.ctypes.data_as(dp)
    rc = L.mh_create(ctypes.byref(h), N, order, ptr(m), ptr(x), ptr(v), eps, None, None)
    return rc, h


def test_invalid_arguments_rejected_before_device_use(L):
    m = np.ones(4)
    x = np.zeros((4, 3))
    v = np.zeros((4, 3))
    rc, h = _create(L, 4, 5, m, x, v, 0.1)        # order must be 4, 6, 8
    assert rc == -1 and not h.value
    assert b"order" in L.mh_last_error()
    rc, h = _create(L, 0, 8, m, x, v, 0.1)        # N >= 1
    assert rc == -1
    rc, h = _create(L, 4, 8, m, x, v, -1.0)       # eps >= 0
    assert rc == -1
    rc, h = _create(L, 4, 8, None, x, v, 0.1)     # NULL masses
    assert rc == -1
    bad = x.copy()
    bad[2, 1] = np.nan
    rc, h = _create(L, 4, 8, m, bad, v, 0.1)      # non-finite input
    assert rc == -4
    mneg = m.copy()
    mneg[0] = -1
    rc, h = _create(L, 4, 8, mneg, x, v, 0.1)
    assert rc == -1
    assert L.mh_step(None, 0.1, 3) == -1          # NULL handle
    assert L.mh_sync(None, None) == -1
    assert L.mh_diagnostics(None, None, None, 0) == -1
    L.mh_destroy(None)                            # no-op


def test_pair_eval_argument_checks(L):
    # unsupported P / precision combinations fail before any device call
    assert L.mh_pair_eval(6, 0, 10, 1, 1, 0.0, 1.0, 0, 10, 1, None) == -1
    assert L.mh_pair_eval(4, 1, 10, 1, 1, 0.0, 1.0, 0, 10, 1, None) == -1
    assert L.mh_pair_eval(3, 0, 10, 1, 1, 0.0, 1.0, 5, 5, 1, None) == -1   # empty range
    assert L.mh_pair_eval(3, 0, 10, 1, 1, 0.0, 1.0, 0, 11, 1, None) == -1  # i1 > N
    assert L.mh_pair_eval(3, 0, 10, 0, 1, 0.0, 1.0, 0, 10, 1, None) == -1  # NULL m


def test_python_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2006_02501_gb300 import _capi
    monkeypatch.setattr(_capi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_capi, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _capi.lib()


def test_create_batch_argument_checks(L):
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    m = np.ones(70)
    x = np.zeros((70, 3))
    dt = np.full(2, 0.01)
    ptr = lambda a: a.ctypes.data_as(dp)
    h = ctypes.c_void_p()
    off = np.array([0, 5, 70], dtype=np.int64)                 # second system has 65 bodies
    rc = L.mh_create_batch(ctypes.byref(h), 2, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                           ptr(m), ptr(x), ptr(x), ptr(dt), 1e-3, 6, None, None)
    assert rc == -1 and b"64" in L.mh_last_error()
    off = np.array([1, 5, 9], dtype=np.int64)                  # offsets[0] != 0
    rc = L.mh_create_batch(ctypes.byref(h), 2, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                           ptr(m), ptr(x), ptr(x), ptr(dt), 1e-3, 6, None, None)
    assert rc == -1
    assert L.mh_step_batch(None, 10, 2) == -1


def test_double_double_and_restore_arguments_rejected_before_device_use(L):
    from paper_2006_02501_gb300 import _capi
    dp = ctypes.POINTER(ctypes.c_double)
    ptr = lambda a: None if a is None else a.ctypes.data_as(dp)
    m = np.ones(3)
    x2 = np.zeros((3, 3, 2))
    x2[:, 0, 0] = [0.0, 1.0, 2.0]
    v2 = np.zeros((3, 3, 2))
    h = ctypes.c_void_p()
    assert L.mh_dd_create(ctypes.byref(h), 3, 7, ptr(m), ptr(x2), ptr(v2), 0.0, None, None) == _capi.MH_EINVAL
    assert L.mh_dd_create(ctypes.byref(h), 3, 8, ptr(m), None, ptr(v2), 0.0, None, None) == _capi.MH_EINVAL
    assert L.mh_dd_create(ctypes.byref(h), 3, 8, ptr(m), ptr(x2), ptr(v2), -1.0, None, None) == _capi.MH_EINVAL
    bad = x2.copy()
    bad[1, 2, 1] = np.inf                       # a non-finite low word
    assert L.mh_dd_create(ctypes.byref(h), 3, 8, ptr(m), ptr(bad), ptr(v2), 0.0, None, None) == _capi.MH_ENONFINITE
    assert not h.value
    i64 = ctypes.POINTER(ctypes.c_int64)
    off = np.array([0, 65], dtype=np.int64)      # one system of 65 bodies
    mm, xx, vv = np.ones(65), np.zeros((65, 3, 2)), np.zeros((65, 3, 2))
    dt = np.array([0.01])
    assert L.mh_dd_create_batch(ctypes.byref(h), 1, off.ctypes.data_as(i64), ptr(mm), ptr(xx), ptr(vv), ptr(dt),
                                0.0, 8, None, None) == _capi.MH_EINVAL
    off = np.array([0, 2, 3], dtype=np.int64)
    dt = np.array([0.01, 0.0])                   # a zero step
    assert L.mh_dd_create_batch(ctypes.byref(h), 2, off.ctypes.data_as(i64), ptr(m), ptr(x2), ptr(v2), ptr(dt),
                                0.0, 8, None, None) == _capi.MH_EINVAL
    cfg = _capi.Config()
    L.mh_config_default(ctypes.byref(cfg))
    cfg.symmetric = 3
    assert L.mh_dd_create(ctypes.byref(h), 3, 8, ptr(m), ptr(x2), ptr(v2), 0.0, ctypes.byref(cfg),
                          None) == _capi.MH_EINVAL
    # the direct double-double evaluation checks its arguments first
    tr2 = np.zeros((3, 4, 3, 2))
    out = np.zeros((3, 4, 3, 2))
    assert L.mh_dd_pair_eval(6, 3, ptr(m), ptr(tr2), 0.0, 1.0, 0, 3, 1, ptr(out)) == _capi.MH_EINVAL
    assert L.mh_dd_pair_eval(3, 3, ptr(m), ptr(tr2), 0.0, 1.0, 0, 4, 1, ptr(out)) == _capi.MH_EINVAL
    assert L.mh_dd_pair_eval(3, 3, ptr(m), ptr(tr2), 0.0, 1.0, 2, 1, 1, ptr(out)) == _capi.MH_EINVAL
    assert L.mh_dd_pair_eval(3, 3, ptr(m), ptr(tr2), 0.0, 1.0, 0, 3, 3, ptr(out)) == _capi.MH_EINVAL
    assert L.mh_dd_pair_eval(3, 3, None, ptr(tr2), 0.0, 1.0, 0, 3, 1, ptr(out)) == _capi.MH_EINVAL
    assert L.mh_dd_pair_eval(3, 3, ptr(m), ptr(tr2), -1.0, 1.0, 0, 3, 1, ptr(out)) == _capi.MH_EINVAL
    assert L.mh_dd_pair_eval(3, 3, ptr(m), ptr(tr2), 0.0, 1.0, 1, 1, 1, None) == _capi.MH_OK   # empty range
    assert L.mh_dd_sym_check(0, None) == _capi.MH_EINVAL
    assert L.mh_dd_step(None, 0.01, 3, 1) == _capi.MH_EINVAL
    assert L.mh_dd_step_batch(None, 1, 3) == _capi.MH_EINVAL
    assert L.mh_dd_batch_energy(None, None) == _capi.MH_EINVAL
    L.mh_dd_destroy(None)
    # mh_restore needs x, v and derivs before anything is created
    st = _capi.StateC(0.0, ptr(np.zeros((3, 3))), ptr(np.zeros((3, 3))), None, None)
    assert L.mh_restore(ctypes.byref(h), 3, 8, ptr(m), ctypes.byref(st), 0.0, None, None) == _capi.MH_EINVAL
    assert not h.value


def test_double_double_marshalling():
    from paper_2006_02501_gb300 import _dd_host
    x = np.arange(12.0).reshape(4, 3)
    x2 = _dd_host(x, 4)
    assert x2.shape == (4, 3, 2) and np.array_equal(x2[..., 0], x) and not x2[..., 1].any()
    assert x2.flags.c_contiguous
    pairs = np.random.default_rng(0).normal(size=(4, 3, 2))
    assert np.array_equal(_dd_host(pairs, 4), pairs)
    d = np.arange(4 * 6 * 3, dtype=float).reshape(4, 6, 3)
    d2 = _dd_host(d, 4, 18)
    assert d2.shape == (4, 18, 2) and np.array_equal(d2[..., 0].reshape(4, 6, 3), d)
