"""GPU parity of the pair-symmetric FP64 evaluation (each unordered pair once,
its odd terms added to both bodies).

The symmetric kernel runs in FP64 simulations of 2048 or more padded bodies by
default (symmetric = 2 forces it at any size); here it is checked against the CPU oracle at sizes that cover every branch of its
block schedule (one block, odd and even block counts, ragged padding, eps = 0
with its guarded diagonal) and against the ordered-pair kernel at the full
SMBH-disc size.  Tolerance: 1e-12 relative, as for the plain FP64 form.
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


# padded to a multiple of 256: 2, 2, 2, 2, 2, 4, 6 and 10 blocks of 128 bodies
# (one row of blocks with its half-distance pair, ragged padding, several chunks)
@pytest.mark.parametrize("N", [1, 2, 3, 129, 256, 257, 700, 1100])
@pytest.mark.parametrize("order", [4, 6, 8])
def test_symmetric_initialisation_parity(mh, orc, N, order):
    m, x, v = I.smbh_disc(seed=20 + N, N=max(N - 1, 1))
    m, x, v = m[:N], x[:N], v[:N]
    with mh.Simulation(order, m, x, v, 1e-4, symmetric=2) as sim:
        _, _, _, dg = sim.sync()
    ref = orc.initialise(order, m, x, v, 1e-4)
    if N == 1:
        assert np.all(dg == 0.0)
    else:
        assert scaled_stack_err(dg, ref, 0.05) < 1e-12


def test_symmetric_unsoftened(mh, orc):
    """eps = 0: the diagonal block skips i = j instead of evaluating r = 0."""
    m, x, v = I.planetesimal_ring(seed=1)
    with mh.Simulation(8, m, x, v, 0.0, symmetric=2) as sim:
        _, _, _, dg = sim.sync()
    assert np.all(np.isfinite(dg))
    assert scaled_stack_err(dg, orc.initialise(8, m, x, v, 0.0), 0.05) < 1e-12


@pytest.mark.parametrize("N", [383, 640])          # 384 and 641 bodies: 4 and 6 blocks
@pytest.mark.parametrize("order", [6, 8])
def test_symmetric_step_parity(mh, orc, N, order):
    m, x, v = I.planetesimal_ring(seed=N, n=N, m=1e-6, a_lo=0.5, a_hi=1.5, sigma_e=0.1, sigma_i=0.05)
    dt, eps = 0.08, 1e-3
    with mh.Simulation(order, m, x, v, eps, symmetric=2) as sim:
        sim.step(dt, 3)
        _, xg, vg, dg = sim.sync()
    ref = orc.State(order, m, x, v, eps)
    ref.step(dt, 3)
    assert rel_rows(xg - x, ref.x - x) < 1e-12
    assert rel_rows(vg - v, ref.v - v) < 1e-12
    p = order // 2 - 1
    assert scaled_stack_err(dg[:, :p + 1], ref.derivs[:, :p + 1], dt) < 1e-12
    assert scaled_stack_err(dg, ref.derivs, dt) < 1e-12


def test_symmetric_matches_ordered_full_size(mh):
    """SMBH disc, 65536 stars + SMBH, 8th order, P(EC)^3, one step: the symmetric
    and ordered kernels differ only in summation order.  The initial stacks
    agree to 1e-13; after a step, close star passages and the interpolated
    a^(4), a^(5) amplify the rounding differences (measured 3.7e-13 in the
    scaled stack), which the FP64 form's 1e-12 tolerance bounds."""
    m, x, v = I.smbh_disc(seed=2, N=65536)
    dt, eps = 2 * np.pi * 1e-3, 1e-4
    out = {}
    for sym in (True, False):
        with mh.Simulation(8, m, x, v, eps, symmetric=sym) as sim:
            _, _, _, d_init = sim.sync()
            sim.step(dt, 3)
            _, xg, vg, dg = sim.sync()
        out[sym] = (d_init, xg, vg, dg)
    a, b = out[True], out[False]
    assert scaled_stack_err(a[0], b[0], dt) < 1e-13
    assert rel_rows(a[1], b[1]) < 1e-14 and rel_rows(a[2], b[2]) < 1e-13
    assert scaled_stack_err(a[3], b[3], dt) < 1e-12


def test_symmetric_full_size_sampled_against_oracle(mh, orc):
    """The headline kernel at the size it is timed at: SMBH disc, 65536 stars +
    SMBH (514 blocks of 128, rows cut into chunks, items handed out in row
    order).  The three initialisation passes of an 8th-order simulation run
    the pair-symmetric kernel with P = 1, 3, 5; each pass is compared with the
    oracle's direct summation on the same inputs (x, v and the derivatives the
    earlier passes left on the device) for three ranges of 40 bodies, the SMBH
    among them, element by element at 1e-12 relative (a^(4), a^(5) in the
    scaled form of Eq. 1 with the workload's dt, as the step tests hold them)."""
    m, x, v = I.smbh_disc(seed=2, N=65536)
    eps, dt = 1e-4, 2 * np.pi * 1e-3
    with mh.Simulation(8, m, x, v, eps) as sim:
        _, _, _, d = sim.sync()
    N = len(m)
    xv = np.stack([x, v], 1)
    for i0 in (0, 31337, N - 40):
        i1 = min(i0 + 40, N)
        g = d[i0:i1]
        r1 = orc.evaluate(m, xv, eps, i0=i0, i1=i1)
        r3 = orc.evaluate(m, np.concatenate([xv, d[:, 0:2]], 1), eps, i0=i0, i1=i1)
        r5 = orc.evaluate(m, np.concatenate([xv, d[:, 0:4]], 1), eps, i0=i0, i1=i1)
        for k in (0, 1):
            assert rel_rows(g[:, k], r1[:, k]) < 1e-12, (i0, k)
        for k in (2, 3):
            assert rel_rows(g[:, k], r3[:, k]) < 1e-12, (i0, k)
        ref = np.concatenate([r1[:, 0:2], r3[:, 2:4], r5[:, 4:6]], 1)
        assert scaled_stack_err(g, ref, dt) < 1e-12, i0


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("N", [8000, 65536])
def test_symmetric_bitwise_reproducible(mh, N, precision):
    """Several rows add into each j-side slot, one after another in a fixed
    order: two runs give the same bits (8000 bodies: all items resident at
    once; 65537: items handed out over several waves)."""
    m, x, v = I.smbh_disc(seed=2, N=N)
    dt, eps = 2 * np.pi * 1e-3, 1e-4
    runs = []
    for _ in range(2):
        with mh.Simulation(8, m, x, v, eps, precision=precision) as sim:
            sim.step(dt, 3)
            runs.append(sim.sync()[1:])
            assert sim.counters()["pair_variant"] == (4 if precision else 0)
    for a, b in zip(*runs):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("N", [2, 3, 129, 300, 1100])
def test_symmetric_fp32_small_sizes(mh, orc, N):
    """The precision form's pair-symmetric kernel forced at small sizes (one
    block of 128 with its ring guard, ragged padding, several blocks): the
    accelerations after one step within 2e-6 of the oracle's."""
    m, x, v = I.smbh_disc(seed=50 + N, N=max(N - 1, 1), m_total=N * 1e-9)
    m, x, v = m[:N], x[:N], v[:N]
    dt, eps = 2 * np.pi * 1e-3, 1e-4
    with mh.Simulation(8, m, x, v, eps, precision=mh.MH_PREC_FP32PAIR, symmetric=2) as sim:
        sim.step(dt, 3)
        _, _, _, dg = sim.sync()
        assert sim.counters()["pair_variant"] == 4
    ref = orc.State(8, m, x, v, eps)
    ref.step(dt, 3)
    assert rel_rows(dg[:, 0], ref.derivs[:, 0]) < 2e-6
