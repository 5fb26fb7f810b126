"""GPU: failure detection by host-side fault injection (MH_FAULT).

No fault is made on the device.  The library reports, on request, an
allocation failure (creation must return MH_ENOMEM, free what it allocated and
leave *out NULL), a failed launch or an expired bounded wait (the step must
return MH_ECUDA / MH_ETIMEOUT before queuing work, so that after the fault is
cleared the run continues exactly as one that never saw it), and a non-finite
state at sync."""
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


def _case():
    m, x, v = I.smbh_disc(seed=51, N=200)
    return m, x, v, 2 * np.pi * 1e-3


def test_injected_allocation_failure(mh, monkeypatch):
    from paper_2006_02501_gb300 import _capi
    m, x, v, dt = _case()
    monkeypatch.setenv("MH_FAULT", "alloc")
    for make in (lambda: mh.Simulation(8, m, x, v, 1e-4),
                 lambda: mh.DDSimulation(8, m[:5], x[:5], v[:5], 0.0),
                 lambda: mh.Batch(6, np.array([0, 5, 12]), m[:12], x[:12], v[:12], np.array([dt, dt]), 1e-8)):
        with pytest.raises(mh.MHError) as e:
            make()
        assert e.value.code == _capi.MH_ENOMEM
        assert "MH_FAULT=alloc" in str(e.value)
    monkeypatch.delenv("MH_FAULT")
    with mh.Simulation(8, m, x, v, 1e-4) as sim:          # nothing left behind
        sim.step(dt, 3)
        sim.sync()


@pytest.mark.parametrize("fault,code", [("launch", -3), ("timeout", -5)])
def test_injected_step_fault_leaves_state_unchanged(mh, monkeypatch, fault, code):
    m, x, v, dt = _case()
    with mh.Simulation(8, m, x, v, 1e-4) as a, mh.Simulation(8, m, x, v, 1e-4) as b:
        a.step(dt, 3)
        b.step(dt, 3)
        monkeypatch.setenv("MH_FAULT", fault)
        with pytest.raises(mh.MHError) as e:
            a.step(dt, 3)
        assert e.value.code == code
        monkeypatch.delenv("MH_FAULT")
        assert a.counters()["steps"] == 1
        a.step(dt, 3)
        b.step(dt, 3)
        for qa, qb in zip(a.sync(), b.sync()):
            assert np.array_equal(qa, qb)


@pytest.mark.parametrize("fault,code", [("launch", -3), ("timeout", -5)])
def test_injected_step_fault_double_double(mh, monkeypatch, fault, code):
    m, x, v, dt = _case()
    with mh.DDSimulation(8, m[:7], x[:7], v[:7], 0.0) as a, mh.DDSimulation(8, m[:7], x[:7], v[:7], 0.0) as b:
        monkeypatch.setenv("MH_FAULT", "x," + fault)
        with pytest.raises(mh.MHError) as e:
            a.step(dt, 3, nsteps=2)
        assert e.value.code == code
        monkeypatch.delenv("MH_FAULT")
        a.step(dt, 3, nsteps=2)
        b.step(dt, 3, nsteps=2)
        for qa, qb in zip(a.sync(), b.sync()):
            assert np.array_equal(qa, qb)


def test_injected_nonfinite_at_sync(mh, monkeypatch):
    m, x, v, dt = _case()
    with mh.Simulation(8, m, x, v, 1e-4) as sim, mh.DDSimulation(8, m[:4], x[:4], v[:4], 0.0) as dsim:
        sim.step(dt, 3)
        monkeypatch.setenv("MH_FAULT", "nonfinite")
        for s in (sim, dsim):
            with pytest.raises(mh.MHError) as e:
                s.sync()
            assert e.value.code == -4
        monkeypatch.delenv("MH_FAULT")
        t, xs, _, _ = sim.sync()
        assert np.isfinite(xs).all() and t == pytest.approx(dt)


def test_unrelated_fault_names_are_ignored(mh, monkeypatch):
    m, x, v, dt = _case()
    monkeypatch.setenv("MH_FAULT", "allocx,launc,,")
    with mh.Simulation(8, m, x, v, 1e-4) as sim:
        sim.step(dt, 3)
        sim.sync()


@pytest.mark.parametrize("N,precision", [(8000, 0), (8000, 1), (40000, 0)])
def test_ordered_accumulation_wait_runs_out(mh, monkeypatch, N, precision):
    """The pair-symmetric evaluation's turns are bounded waits.  MH_FAULT=symwait
    makes every turn unreachable (an awaited count nothing sets) and shortens
    the limit to 20 ms: the launch must still end, the sync must report
    MH_ETIMEOUT, and the device must stay usable, a new simulation stepping to
    the same bits as one that never saw the fault.  8000 bodies: every item
    resident at once (distance order); 40000 bodies: items handed out in row
    order over several waves."""
    from paper_2006_02501_gb300 import _capi
    m, x, v = I.smbh_disc(seed=52, N=N - 1)
    dt = 2 * np.pi * 1e-3
    with mh.Simulation(8, m, x, v, 1e-4, precision=precision) as sim:
        monkeypatch.setenv("MH_FAULT", "symwait")
        sim.step(dt, 3)
        monkeypatch.delenv("MH_FAULT")
        with pytest.raises(mh.MHError) as e:
            sim.sync()
        assert e.value.code == _capi.MH_ETIMEOUT
    with mh.Simulation(8, m, x, v, 1e-4, precision=precision) as a, \
            mh.Simulation(8, m, x, v, 1e-4, precision=precision) as b:
        a.step(dt, 3)
        b.step(dt, 3)
        np.testing.assert_array_equal(a.sync()[1], b.sync()[1])
