"""GPU: checkpoint and resume (mh_sync -> mh_restore).

Every reduction of the library has a fixed order, so a run of 2k steps and a
run of k steps, checkpointed, restored into a new handle and continued for k
more, must agree bit for bit: shared steps of both FP64 kernels and of the
precision form (fixed kernel variant), and block steps (levels and derivative
stacks restored, all bodies synchronised at a multiple of dt_max).  The
time-symmetric step restarts its H- from Eq. 24 at the restored positions and
compensated summation restarts its compensation at zero: those continue within
rounding."""
import numpy as np
import pytest

from paper_2006_02501_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_02501_gb300 as pkg
    pkg.build_library()
    return pkg


def _resume(mh, order, m, x, v, eps, advance, k, **kw):
    """(uninterrupted 2k, checkpointed k + restored k) final checkpoints."""
    with mh.Simulation(order, m, x, v, eps, **kw) as a:
        for _ in range(2 * k):
            advance(a)
        full = a.checkpoint()
    with mh.Simulation(order, m, x, v, eps, **kw) as b:
        for _ in range(k):
            advance(b)
        ck = b.checkpoint()
    with mh.Simulation.restore(order, m, ck, eps, **kw) as c:
        for _ in range(k):
            advance(c)
        again = c.checkpoint()
        counters = c.counters()
    return full, again, counters


@pytest.mark.parametrize("symmetric", [0, 2])
@pytest.mark.parametrize("order", [6, 8, 12])
def test_resume_bitwise_fp64(mh, order, symmetric):
    m, x, v = I.smbh_disc(seed=41, N=300)
    dt = 2 * np.pi * 1e-3
    full, again, c = _resume(mh, order, m, x, v, 1e-4, lambda s: s.step(dt, 3), 3, symmetric=symmetric)
    for key in ("x", "v", "derivs"):
        assert np.array_equal(full[key], again[key]), key
    assert full["t"] == again["t"]
    assert c["steps"] == 3 and c["evaluations"] == 9    # no initialisation pass counted or run


def test_resume_bitwise_fp32_pair(mh):
    m, x, v = I.smbh_disc(seed=42, N=500)
    dt = 2 * np.pi * 1e-3
    full, again, _ = _resume(mh, 8, m, x, v, 1e-4, lambda s: s.step(dt, 3), 2,
                             precision=mh.MH_PREC_FP32PAIR, fp32_variant=1)
    for key in ("x", "v", "derivs"):
        assert np.array_equal(full[key], again[key]), key


@pytest.mark.parametrize("order", [6, 8])
def test_resume_bitwise_block_steps(mh, order):
    m, x, v = I.smbh_disc(seed=43, N=400)
    blk = dict(dt_max=2.0 ** -5, k_max=10, eta=0.05)
    full, again, _ = _resume(mh, order, m, x, v, 1e-4, lambda s: s.step(blk["dt_max"], 3), 2, block=blk)
    assert len(np.unique(full["level"])) > 1             # several levels in play
    for key in ("x", "v", "derivs", "level"):
        assert np.array_equal(full[key], again[key]), key


def test_resume_timesym_and_compensated_within_rounding(mh):
    m, x, v = I.kepler_pair(a=1.0, e=0.5, M=1.0, m=1e-3)
    full, again, _ = _resume(mh, 8, m, x, v, 0.0, lambda s: s.step_timesym(10, 3), 3, timesym_eta=0.05)
    scale = np.abs(full["x"]).max()
    assert np.abs(full["x"] - again["x"]).max() < 1e-12 * scale
    assert abs(full["t"] - again["t"]) < 1e-12 * abs(full["t"])
    full, again, _ = _resume(mh, 8, m, x, v, 0.0, lambda s: s.step(0.01, 3), 50, compensated=True)
    assert np.abs(full["x"] - again["x"]).max() < 1e-13 * np.abs(full["x"]).max()


def test_restore_needs_derivatives(mh):
    from paper_2006_02501_gb300 import _capi
    m, x, v = I.smbh_disc(seed=44, N=50)
    with mh.Simulation(8, m, x, v, 1e-4) as s:
        ck = s.checkpoint()
    ck_bad = dict(ck)
    ck_bad["derivs"] = None
    with pytest.raises((mh.MHError, TypeError, ValueError)):
        mh.Simulation.restore(8, m, ck_bad, 1e-4)
    st = _capi.StateC(0.0, None, None, None, None)
    import ctypes
    h = ctypes.c_void_p()
    mm = np.ascontiguousarray(m)
    rc = _capi.lib().mh_restore(ctypes.byref(h), len(m), 8, mm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                ctypes.byref(st), 1e-4, None, None)
    assert rc == _capi.MH_EINVAL and not h.value
