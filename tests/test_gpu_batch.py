"""Batched form: many independent systems in one persistent launch.  Each
system must match the oracle run alone, and the single-system GPU path, to
1e-12 (same precision, FP64)."""
import numpy as np
import pytest

from helpers import rel_rows, scaled_stack_err
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


def _systems(S, seed, sizes=None):
    off, m, x, v, pmin = I.planetary_systems(seed=seed, S=S)
    if sizes is not None:                       # force edge sizes into the first systems
        parts = []
        for k in range(S):
            n = off[k + 1] - off[k]
            n2 = min(n, sizes[k]) if k < len(sizes) else n
            parts.append((m[off[k]:off[k] + n2], x[off[k]:off[k] + n2], v[off[k]:off[k] + n2]))
        off = np.concatenate([[0], np.cumsum([len(p[0]) for p in parts])]).astype(np.int64)
        m = np.concatenate([p[0] for p in parts])
        x = np.concatenate([p[1] for p in parts])
        v = np.concatenate([p[2] for p in parts])
    return off, m, x, v, pmin / 128.0


@pytest.mark.parametrize("order,n_iter", [(6, 2), (4, 3), (8, 2)])
def test_batch_matches_oracle_per_system(mh, orc, order, n_iter):
    off, m, x, v, dt = _systems(40, seed=41, sizes=[1, 2, 3, 64])
    eps, nst = 1e-8, 25
    with mh.Batch(order, off, m, x, v, dt, eps) as b:
        b.step(nst, n_iter)
        _, xg, vg, dg = b.sync()
        E = b.energies()
    for k in range(len(off) - 1):
        sl = slice(off[k], off[k + 1])
        ref = orc.State(order, m[sl], x[sl], v[sl], eps)
        ref.step(dt[k], n_iter, nst)
        assert rel_rows(xg[sl], ref.x) < 1e-12, k
        assert rel_rows(vg[sl], ref.v, 1e-6) < 1e-12, k
        if off[k + 1] - off[k] > 1:
            assert scaled_stack_err(dg[sl], ref.derivs, dt[k]) < 1e-10, k
            assert abs(E[k] / ref.energy() - 1) < 1e-13, k


def test_batch_matches_single_system_gpu_path(mh):
    off, m, x, v, dt = _systems(12, seed=42)
    eps = 1e-8
    with mh.Batch(6, off, m, x, v, dt, eps) as b:
        b.step(40, 2)
        _, xg, vg, _ = b.sync()
    for k in range(len(off) - 1):
        sl = slice(off[k], off[k + 1])
        with mh.Simulation(6, m[sl], x[sl], v[sl], eps) as s:
            s.step(dt[k], 2, nsteps=40)
            _, xs, vs, _ = s.sync()
        assert rel_rows(xg[sl], xs) < 1e-12
        assert rel_rows(vg[sl], vs, 1e-6) < 1e-12


def test_batch_autotune_graph_replay_and_continuation(mh):
    off, m, x, v, dt = _systems(600, seed=43)
    eps = 1e-8
    with mh.Batch(6, off, m, x, v, dt, eps) as b:
        w, o = b.tune(probe_steps=4, n_iter=2)
        assert w in (2, 4, 6, 8) and o in (0, 1)
        b.step(10, 2)
        b.step(10, 2)                          # replays the captured graph
        _, x2, v2, _ = b.sync()
        c = b.counters()
    with mh.Batch(6, off, m, x, v, dt, eps) as b1:
        b1.step(20, 2)
        _, x1, v1, _ = b1.sync()
    np.testing.assert_array_equal(x1, x2)      # deterministic, independent of the split of calls
    np.testing.assert_array_equal(v1, v2)
    assert c["steps"] == 20


def test_batch_rejects_oversize_system(mh):
    m = np.full(65, 1e-3)
    x = np.random.default_rng(0).normal(size=(65, 3))
    v = np.zeros((65, 3))
    with pytest.raises(mh.MHError):
        mh.Batch(6, np.array([0, 65]), m, x, v, np.array([0.01]), 1e-3)
