"""GPU: the batched double-double form (mh_dd_create_batch / mh_dd_step_batch)
against the binary128 oracle run on each system alone.

Systems of 1, 2 and 64 bodies (the edge sizes) sit beside a random ensemble of
planetary systems, each with its own dt.  The tolerance is that of the
single-system form (1e-27 relative; see test_gpu_dd.py)."""
import numpy as np
import pytest

from helpers import dd_diff
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


def _ensemble():
    """(offsets, m, x, v, dt) of 10 random systems plus a single body, a Kepler
    pair and a 64-body system."""
    parts = []
    off, m, x, v, pmin = I.planetary_systems(seed=31, S=10, nmin=3, nmax=40)
    for s in range(10):
        a, b = off[s], off[s + 1]
        parts.append((m[a:b], x[a:b], v[a:b], pmin[s] / 64))
    parts.append((np.array([1.0]), np.array([[0.3, -0.2, 0.1]]), np.array([[0.01, 0.02, -0.03]]), 0.01))
    km, kx, kv = I.kepler_pair(a=1.0, e=0.5, M=1.0, m=1e-3)
    parts.append((km, kx, kv, 2.0 ** -6))
    o64, m64, x64, v64, p64 = I.planetary_systems(seed=32, S=1, nmin=64, nmax=64)
    parts.append((m64, x64, v64, p64[0] / 64))
    offsets = np.cumsum([0] + [len(p[0]) for p in parts]).astype(np.int64)
    return (offsets, np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]),
            np.concatenate([p[2] for p in parts]), np.array([p[3] for p in parts]))


def _rel(got2, ref2):
    ref = np.asarray(ref2)[..., 0] + np.asarray(ref2)[..., 1]
    return float(np.abs(dd_diff(got2, ref2)).max() / max(np.abs(ref).max(), 1e-300))


@pytest.mark.parametrize("order", [6, 8, 12])
def test_dd_batch_matches_oracle_per_system(mh, orc, order):
    off, m, x, v, dt = _ensemble()
    with mh.DDBatch(order, off, m, x, v, dt, 0.0) as b:
        b.step(5, 3)
        t2, x2, v2, d2 = b.sync()
    assert t2[0] == 5
    for s in range(len(dt)):
        a, e = off[s], off[s + 1]
        xr, vr, dr = orc.dd_run(order, m[a:e], x[a:e], v[a:e], 0.0, dt[s], 3, 5)
        assert _rel(x2[a:e], xr) < 1e-27, (s, _rel(x2[a:e], xr))
        assert _rel(v2[a:e], vr) < 1e-27, (s, _rel(v2[a:e], vr))


def test_dd_batch_matches_single_system_form(mh):
    off, m, x, v, dt = _ensemble()
    with mh.DDBatch(8, off, m, x, v, dt, 1e-4) as b:
        b.step(4, 2)
        _, x2, v2, _ = b.sync()
    for s in (0, 10, 11, 12):
        a, e = off[s], off[s + 1]
        with mh.DDSimulation(8, m[a:e], x[a:e], v[a:e], 1e-4) as one:
            one.step(dt[s], 2, nsteps=4)
            _, xs, vs, _ = one.sync()
        # the two forms sum the j terms in different orders: rounding level only
        assert _rel(x2[a:e], xs) < 1e-29 and _rel(v2[a:e], vs) < 1e-29, s


def test_dd_batch_energies(mh, orc):
    off, m, x, v, dt = _ensemble()
    with mh.DDBatch(8, off, m, x, v, dt, 1e-3) as b:
        b.step(3, 3)
        _, x2, v2, _ = b.sync()
        E2 = b.energies()
    for s in range(len(dt)):
        a, e = off[s], off[s + 1]
        Er = orc.dd_energy(m[a:e], x2[a:e], v2[a:e], 1e-3)
        assert abs(dd_diff(E2[s], Er)) <= 1e-29 * max(abs(Er[0]), 1e-300), s


def test_dd_batch_graph_replay_and_counters(mh):
    off, m, x, v, dt = _ensemble()
    with mh.DDBatch(8, off, m, x, v, dt, 0.0) as a, mh.DDBatch(8, off, m, x, v, dt, 0.0) as b:
        a.step(6, 3)
        for _ in range(6):
            b.step(1, 3)
        ra, rb = a.sync(), b.sync()
        c = a.counters()
    for qa, qb in zip(ra, rb):
        assert np.array_equal(qa, qb)
    n = np.diff(off)
    assert c["steps"] == 6 and c["evaluations"] == 18
    assert c["pair_interactions"] == 18 * float((n * (n - 1)).sum())
    assert c["particle_steps"] == 6 * off[-1]


def test_dd_batch_argument_errors(mh):
    from paper_2006_02501_gb300 import _capi
    off, m, x, v, dt = _ensemble()
    big = np.array([0, 65], dtype=np.int64)
    mb, xb, vb = I.planetesimal_ring(seed=3, n=64)
    with pytest.raises(mh.MHError):
        mh.DDBatch(8, big, mb, xb, vb, np.array([0.01]), 0.0)          # 65 bodies in one system
    bad_dt = dt.copy()
    bad_dt[3] = 0.0
    with pytest.raises(mh.MHError):
        mh.DDBatch(8, off, m, x, v, bad_dt, 0.0)
    with mh.DDBatch(8, off, m, x, v, dt, 0.0) as b:
        L = _capi.lib()
        assert L.mh_dd_step(b._h, 0.01, 3, 1) == _capi.MH_EINVAL
        assert L.mh_dd_diagnostics(b._h, None, None, 0) == _capi.MH_EINVAL
        with pytest.raises(mh.MHError):
            b.step(1, 0)
    with mh.DDSimulation(8, m[:5], x[:5], v[:5], 0.0) as one:
        assert _capi.lib().mh_dd_step_batch(one._h, 1, 3) == _capi.MH_EINVAL
        assert _capi.lib().mh_dd_batch_energy(one._h, None) == _capi.MH_EINVAL
