"""GPU: compensated summation of the x, v updates (Section 3.2, after Kahan).

The GPU forms each increment minus the carried compensation with one fused
multiply-add (the product v dt is exact inside it), so its exact reference for a
free body is x0 + K v dt in rational arithmetic; the oracle's is the sum of the
rounded products.  Parity with the oracle on a long Kepler run at 1e-12."""
from fractions import Fraction

import numpy as np
import pytest

from helpers import rel_rows
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


def test_gpu_free_body_sum(mh):
    m = np.array([1.0])
    x = np.array([[0.1, -0.7, 3.3]])
    v = np.array([[1.0 / 3.0, 2.0 / 7.0, -1.0 / 9.0]])
    dt, K = 0.01, 100000
    out = {}
    for comp in (False, True):
        with mh.Simulation(8, m, x, v, 0.0, compensated=comp) as sim:
            sim.step(dt, 2, nsteps=K)
            out[comp] = sim.sync()[1][0]
    for c in range(3):
        exact = Fraction(float(x[0, c])) + K * Fraction(float(v[0, c])) * Fraction(dt)
        ulp = abs(float(np.spacing(float(exact))))
        assert abs(Fraction(float(out[True][c])) - exact) <= 2 * ulp
        assert abs(Fraction(float(out[False][c])) - exact) > 50 * ulp


def test_gpu_compensated_kepler_parity(mh, orc):
    """20 orbits: the GPU (fused multiply-adds) and the oracle (none) round
    differently, and their orbital phases drift apart by ~1e-14 per orbit
    (3e-12 after 200 orbits), so the 1e-12 parity is checked over 20."""
    m, x, v = I.kepler_pair(a=1.0, e=0.1, M=1.0, m=1e-3)
    dt, K = 2 * np.pi / 128, 128 * 20
    with mh.Simulation(8, m, x, v, 0.0, compensated=True) as sim:
        sim.step(dt, 3, nsteps=K)
        _, xg, vg, _ = sim.sync()
    ref = orc.State(8, m, x, v, 0.0)
    ref.step(dt, 3, K, compensated=True)
    assert rel_rows(xg, ref.x) < 1e-12 and rel_rows(vg, ref.v) < 1e-12


def test_gpu_compensation_lowers_rounding_error(mh):
    m, x, v = I.kepler_pair(a=1.0, e=0.1, M=1.0, m=1e-3)
    dt, K = 2 * np.pi / 128, 128 * 200
    worst = {}
    for comp in (False, True):
        with mh.Simulation(8, m, x, v, 0.0, compensated=comp) as sim:
            E0 = sim.energy()
            w = 0.0
            for _ in range(20):
                sim.step(dt, 3, nsteps=K // 20)
                w = max(w, abs(sim.energy() / E0 - 1))
        worst[comp] = w
    assert worst[True] < worst[False] / 2, worst


def test_compensated_rejected_outside_shared_steps(mh):
    m, x, v = I.kepler_pair(a=1.0, e=0.5)
    with pytest.raises(mh.MHError):
        mh.Simulation(8, m, x, v, 0.0, compensated=True, timesym_eta=0.02)
