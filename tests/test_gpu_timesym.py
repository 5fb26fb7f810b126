"""GPU parity of the time-symmetric variable shared step (Section 3.3) against
the oracle.

The GPU keeps dt on the device: every evaluation also finds the maximum over
pairs of G (m_i + m_j) s^(-3/2), H = eta w_max^(-1/2) (Eq. 24), and the
predictor and corrector compute dt = (H- + H+)/2 from those words.  Both sides
take H from the same formula; they differ only in rounding (the GPU forms w,
the oracle its inverse square root), so the step sizes agree to ~1e-15 and the
states to the FP64 form's 1e-12.
"""
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


def test_timesym_kepler_e09_parity(mh, orc):
    m, x, v = I.kepler_pair(a=1.0, e=0.9, M=1.0, m=1e-3)
    eta, n, K = 0.02, 5, 150
    with mh.Simulation(8, m, x, v, 0.0, timesym_eta=eta) as sim:
        sim.step_timesym(K, n)
        t, xg, vg, dg = sim.sync()
    ref = orc.State(8, m, x, v, 0.0)
    ref.step_timesym(eta, n, K)
    assert abs(t - ref.t) / ref.t < 1e-13
    assert rel_rows(xg, ref.x) < 1e-12 and rel_rows(vg, ref.v) < 1e-12
    assert scaled_stack_err(dg, ref.derivs, ref.H) < 1e-10


@pytest.mark.parametrize("n_bodies,seed", [(100, 5), (300, 6)])    # one block of 128 / several
def test_timesym_disc_parity(mh, orc, n_bodies, seed):
    """Section 3.3 disc (bodies of 1e-5 around a unit mass, log-spaced a in
    [0.1, 10], eps = 1e-6), eta = 0.02, n = 4; 300 bodies spread the pairs over
    the off-diagonal blocks of the pair-symmetric kernel as well."""
    m, x, v = I.disc_100(seed=seed, n=n_bodies)
    eta, n, K, eps = 0.02, 4, 30, 1e-6
    with mh.Simulation(8, m, x, v, eps, timesym_eta=eta) as sim:
        sim.step_timesym(K, n)
        t, xg, vg, dg = sim.sync()
    ref = orc.State(8, m, x, v, eps)
    dts = ref.step_timesym(eta, n, K)
    assert np.ptp(dts) > 0                         # the step really varies
    assert abs(t - ref.t) / ref.t < 1e-12
    assert rel_rows(xg, ref.x) < 1e-12 and rel_rows(vg, ref.v, 1e-3) < 1e-11


def test_timesym_reversible_on_gpu(mh):
    m, x, v = I.kepler_pair(a=1.0, e=0.9, M=1.0, m=1e-3)
    with mh.Simulation(8, m, x, v, 0.0, timesym_eta=0.02) as sim:
        sim.step_timesym(300, 10)
        t1, *_ = sim.sync()
        sim.step_timesym(300, 10, backward=True)
        t, xg, vg, _ = sim.sync()
    assert t1 > 1.0
    assert abs(t) < 1e-12
    assert np.abs(xg - x).max() < 1e-12 and np.abs(vg - v).max() < 1e-12


def test_timesym_circular_constant_step(mh, orc):
    m, x, v = I.kepler_pair(a=1.0, e=0.0, M=1.0, m=1e-3)
    eta = 0.05
    H0 = orc.timestep_H(m, x, 0.0, eta)
    with mh.Simulation(8, m, x, v, 0.0, timesym_eta=eta) as sim:
        sim.step_timesym(64, 3)
        t, xg, vg, _ = sim.sync()
    assert t == pytest.approx(64 * H0, rel=1e-13)


def test_timesym_rejects_bad_use(mh):
    m, x, v = I.kepler_pair(a=1.0, e=0.5)
    with mh.Simulation(8, m, x, v, 0.0, timesym_eta=0.02) as sim:
        with pytest.raises(mh.MHError):
            sim.step(0.01, 3)                        # variable steps only
    with pytest.raises(mh.MHError):
        mh.Simulation(8, m, x, v, 0.0, timesym_eta=0.02, precision=mh.MH_PREC_FP32PAIR)
    with pytest.raises(mh.MHError):
        mh.Simulation(8, m[:1], x[:1], v[:1], 0.0, timesym_eta=0.02)


def test_timesym_graph_replay_matches_plain_launches(mh):
    """Pairs of steps replay a captured CUDA graph unless per-launch timing is
    on; both paths run the same kernels on the same data, so the states agree
    bit for bit."""
    m, x, v = I.disc_100(seed=7, n=60)
    out = []
    for timing in (False, True):
        with mh.Simulation(8, m, x, v, 1e-6, timesym_eta=0.04) as sim:
            sim.set_timing(timing)
            sim.step_timesym(41, 4)
            t, xg, vg, dg = sim.sync()
            c = sim.counters()
        out.append((t, xg, vg, dg))
        assert c["steps"] == 41 and c["evaluations"] == 41 * 4
    assert out[0][0] == out[1][0]
    for a, b in zip(out[0][1:], out[1][1:]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("n_bodies", [60, 300])
def test_timesym_pair_symmetric_kernel(mh, orc, n_bodies):
    """The Eq. 24 maximum inside the pair-symmetric kernel (forced with
    symmetric = 2; by default small systems take the ordered kernel): its
    diagonal blocks (ordered pairs, guarded self pair) and its off-diagonal
    blocks (each pair once) both feed w_max."""
    m, x, v = I.disc_100(seed=8, n=n_bodies)
    eta, n, K, eps = 0.02, 4, 20, 1e-6
    with mh.Simulation(8, m, x, v, eps, timesym_eta=eta, symmetric=2) as sim:
        sim.step_timesym(K, n)
        t, xg, vg, _ = sim.sync()
    ref = orc.State(8, m, x, v, eps)
    ref.step_timesym(eta, n, K)
    assert abs(t - ref.t) / ref.t < 1e-12
    assert rel_rows(xg, ref.x) < 1e-12 and rel_rows(vg, ref.v, 1e-3) < 1e-11
