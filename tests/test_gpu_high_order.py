"""GPU parity of the 10th- and 12th-order schemes (p = 4, 5; Section 2 gives
the correctors for any order, the paper prints them up to 8th order) against
the oracle: the explicit initialisation to a^(2p-1), one P(EC)^n step with a
coarse dt, time symmetry, and the variable time-symmetric step.  Tolerances as
for the FP64 form (1e-12 on states, the scaled stacks within rounding)."""
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


@pytest.mark.parametrize("order", [10, 12])
@pytest.mark.parametrize("symmetric", [1, 2])          # 2: the pair-symmetric kernel (P <= 5) forced
def test_high_order_initialisation(mh, orc, order, symmetric):
    m, x, v = I.smbh_disc(seed=41, N=400)
    with mh.Simulation(order, m, x, v, 1e-4, symmetric=symmetric) as sim:
        _, _, _, dg = sim.sync()
    ref = orc.initialise(order, m, x, v, 1e-4)
    assert dg.shape == ref.shape == (401, order - 2, 3)
    assert scaled_stack_err(dg, ref, 0.05) < 1e-11


@pytest.mark.parametrize("order", [10, 12])
@pytest.mark.parametrize("beta,symmetric", [(0, 1), (1, 1), (0, 2)])
def test_high_order_one_step(mh, orc, order, beta, symmetric):
    m, x, v = I.planetesimal_ring(seed=42, n=200, m=1e-6, a_lo=0.5, a_hi=1.5, sigma_e=0.1, sigma_i=0.05)
    dt, eps = 0.08, 1e-3
    with mh.Simulation(order, m, x, v, eps, beta=beta, symmetric=symmetric) as sim:
        sim.step(dt, 3)
        _, xg, vg, dg = sim.sync()
    ref = orc.State(order, m, x, v, eps, modified=(beta == 0))
    ref.step(dt, 3)
    assert rel_rows(xg - x, ref.x - x) < 1e-11
    assert rel_rows(vg - v, ref.v - v) < 1e-11
    assert rel_rows(xg, ref.x) < 1e-12 and rel_rows(vg, ref.v) < 1e-12
    assert scaled_stack_err(dg, ref.derivs, dt) < 1e-9


@pytest.mark.parametrize("order", [10, 12])
def test_high_order_kepler_and_symmetry(mh, orc, order):
    m, x, v = I.kepler_pair(a=1.0, e=0.5)
    dt, K = 2 * np.pi / 64, 64
    with mh.Simulation(order, m, x, v, 0.0) as sim:
        sim.step(dt, 6, nsteps=K)
        _, xf, vf, _ = sim.sync()
        sim.step(-dt, 6, nsteps=K)
        _, xb, vb, _ = sim.sync()
    ref = orc.State(order, m, x, v, 0.0)
    ref.step(dt, 6, K)
    assert rel_rows(xf, ref.x) < 1e-12 and rel_rows(vf, ref.v) < 1e-12
    assert np.abs(xb - x).max() < 1e-11 and np.abs(vb - v).max() < 1e-11


def test_tenth_order_time_symmetric_variable_step(mh, orc):
    m, x, v = I.kepler_pair(a=1.0, e=0.9, M=1.0, m=1e-3)
    with mh.Simulation(10, m, x, v, 0.0, timesym_eta=0.03) as sim:
        sim.step_timesym(80, 4)
        t, xg, vg, _ = sim.sync()
    ref = orc.State(10, m, x, v, 0.0)
    ref.step_timesym(0.03, 4, 80)
    assert abs(t - ref.t) / ref.t < 1e-13
    assert rel_rows(xg, ref.x) < 1e-12 and rel_rows(vg, ref.v) < 1e-12


def test_high_order_rejects_unsupported_forms(mh):
    m, x, v = I.kepler_pair(a=1.0, e=0.5)
    with pytest.raises(mh.MHError):
        mh.Simulation(10, m, x, v, 0.0, precision=mh.MH_PREC_FP32PAIR)
    with pytest.raises(mh.MHError):
        mh.Simulation(12, m, x, v, 0.0, block=dict(dt_max=2.0 ** -5, k_max=8, eta=0.05))
    with pytest.raises(mh.MHError):
        mh.Simulation(14, m, x, v, 0.0)


def test_tenth_order_variable_step_pair_symmetric(mh, orc):
    m, x, v = I.disc_100(seed=9, n=150)
    with mh.Simulation(10, m, x, v, 1e-6, timesym_eta=0.03, symmetric=2) as sim:
        sim.step_timesym(20, 4)
        t, xg, vg, _ = sim.sync()
    ref = orc.State(10, m, x, v, 1e-6)
    ref.step_timesym(0.03, 4, 20)
    assert abs(t - ref.t) / ref.t < 1e-12
    assert rel_rows(xg, ref.x) < 1e-12 and rel_rows(vg, ref.v, 1e-3) < 1e-11
