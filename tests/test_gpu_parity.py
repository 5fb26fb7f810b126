"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances
  FP64 form: 1e-12 relative on derivatives (in the scaled form of Eq. 1 for
  derivative stacks) and on states, as the plain form requires.
  FP32-pair form: acceleration within 2e-6 relative per body; the higher
  derivatives within the bounds written in each test.
Step-parity cases use coarse time steps so that every term of the predictor
and corrector lies well above rounding and a wrong coefficient shows.
"""
import numpy as np
import pytest

from helpers import kepler_traj, rel_rows, scaled_stack_err
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _pair_eval(mh, P, prec, m, traj, eps, i0=0, i1=None):
    N = len(m)
    i1 = N if i1 is None else i1
    rows = np.ascontiguousarray(traj[:, :P + 1].transpose(1, 2, 0).reshape((P + 1) * 3, N))
    out = torch.zeros(((P + 1) * 3, i1 - i0), dtype=torch.float64, device="cuda")
    mh.pair_eval(P, prec, _dev(m), _dev(rows), eps, out, i0=i0, i1=i1)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(P + 1, 3, i1 - i0).transpose(2, 0, 1)


# --------------------------------------------------------------------------- #
# evaluation (the O(N^2) kernel alone)
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("P", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("N", [1, 2, 3, 257, 777])
def test_pair_eval_fp64_random(mh, orc, P, N):
    rng = np.random.default_rng(P * 1000 + N)
    m = rng.uniform(0.1, 1.0, N)
    traj = rng.normal(size=(N, P + 1, 3))
    got = _pair_eval(mh, P, mh.MH_PREC_FP64, m, traj, 0.05)
    ref = orc.evaluate(m, traj, 0.05)
    for k in range(P + 1):
        if N == 1:
            assert np.all(got == 0.0)
        else:
            assert rel_rows(got[:, k], ref[:, k], 1e-6) < 1e-12, k


def test_pair_eval_fp64_unsoftened_self_term(mh, orc):
    # eps = 0: the i = j term must be skipped, not evaluated at r = 0
    m, x, v = I.kepler_pair(e=0.3)
    traj = kepler_traj(m, x, v, 3)
    got = _pair_eval(mh, 3, mh.MH_PREC_FP64, m, traj, 0.0)
    ref = orc.evaluate(m, traj, 0.0)
    assert np.all(np.isfinite(got))
    assert rel_rows(got.reshape(-1, 3), ref.reshape(-1, 3), 1e-6) < 1e-12


@pytest.mark.parametrize("P", [1, 2, 3])
def test_pair_eval_fp32_disc(mh, orc, P):
    m, x, v = I.smbh_disc(seed=11, N=1500)
    traj = kepler_traj(m, x, v, P)
    got = _pair_eval(mh, P, mh.MH_PREC_FP32PAIR, m, traj, 1e-4)
    ref = orc.evaluate(m, traj, 1e-4)
    assert rel_rows(got[:, 0], ref[:, 0]) < 2e-6
    for k in range(1, P + 1):
        assert rel_rows(got[:, k], ref[:, k], 1e-3) < 5e-5, k


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-6)])
def test_pair_eval_full_size_sampled(mh, orc, prec, tol):
    """N = 65537 disc (SMBH + 65536 stars), 8th-order evaluation (P = 3) in the
    launch configuration of the integrator, on three sampled ranges of bodies."""
    m, x, v = I.smbh_disc(seed=2, N=65536)
    traj = kepler_traj(m, x, v, 3)
    N = len(m)
    for i0 in (0, 31337, N - 40):
        i1 = min(i0 + 40, N)
        got = _pair_eval(mh, 3, prec, m, traj, 1e-4, i0, i1)
        ref = orc.evaluate(m, traj, 1e-4, i0=i0, i1=i1)
        assert rel_rows(got[:, 0], ref[:, 0]) < tol
        if prec == 0:
            for k in range(1, 4):
                assert rel_rows(got[:, k], ref[:, k], 1e-6) < tol


# --------------------------------------------------------------------------- #
# the integrator through mh_create / mh_step / mh_sync
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("order", [4, 6, 8])
def test_initialisation_parity(mh, orc, order):
    m, x, v = I.smbh_disc(seed=3, N=999)
    with mh.Simulation(order, m, x, v, 1e-4) as sim:
        _, xg, vg, dg = sim.sync()
    ref = orc.initialise(order, m, x, v, 1e-4)
    np.testing.assert_array_equal(xg, x)
    np.testing.assert_array_equal(vg, v)
    assert scaled_stack_err(dg, ref, 0.05) < 1e-12


@pytest.mark.parametrize("order", [4, 6, 8])
@pytest.mark.parametrize("n_iter", [1, 2, 3])
@pytest.mark.parametrize("beta", [0, 1])
def test_one_step_parity_coarse_dt(mh, orc, order, n_iter, beta):
    """One P(EC)^n step from an identical state with a coarse dt, so that every
    corrector and predictor term is far above rounding."""
    m, x, v = I.planetesimal_ring(seed=4, n=300, m=1e-6, a_lo=0.5, a_hi=1.5, sigma_e=0.1, sigma_i=0.05)
    dt = 0.08
    eps = 1e-3
    with mh.Simulation(order, m, x, v, eps, beta=beta) as sim:
        sim.step(dt, n_iter)
        _, xg, vg, dg = sim.sync()
    ref = orc.State(order, m, x, v, eps, modified=(beta == 0))
    ref.step(dt, n_iter)
    # increments relative to their own size: catches any wrong coefficient
    assert rel_rows(xg - x, ref.x - x) < 1e-12
    assert rel_rows(vg - v, ref.v - v) < 1e-12
    assert rel_rows(xg, ref.x) < 1e-12 and rel_rows(vg, ref.v) < 1e-12
    p = order // 2 - 1
    # a^(0..p): evaluated at the end of the step; a^(p+1..2p-1): interpolated (Eqs. 2-5)
    assert scaled_stack_err(dg[:, :p + 1], ref.derivs[:, :p + 1], dt) < 1e-12
    assert scaled_stack_err(dg, ref.derivs, dt) < 1e-12


def test_trajectory_parity_planetesimal_ring(mh, orc):
    """Central mass + 64 planetesimals (m = 1e-9), 6th order, P(EC)^2,
    dt = 2 pi / 256, eps = 0, 1000 steps."""
    m, x, v = I.planetesimal_ring(seed=1)
    dt = 2 * np.pi / 256
    with mh.Simulation(6, m, x, v, 0.0) as sim:
        sim.step(dt, 2, nsteps=1000)
        t, xg, vg, dg = sim.sync()
        E = sim.energy()
    ref = orc.State(6, m, x, v, 0.0)
    ref.step(dt, 2, 1000)
    assert abs(t - 1000 * dt) < 1e-9
    assert rel_rows(xg, ref.x) < 1e-12
    assert rel_rows(vg, ref.v) < 1e-12
    assert abs(E - ref.energy()) / abs(ref.energy()) < 1e-13


def test_trajectory_parity_disc_8th(mh, orc):
    """SMBH disc (N = 1025), 8th order, P(EC)^3, dt = 2 pi 1e-3, eps = 1e-4, 40 steps."""
    m, x, v = I.smbh_disc(seed=2, N=1024)
    dt, eps = 2 * np.pi * 1e-3, 1e-4
    with mh.Simulation(8, m, x, v, eps) as sim:
        sim.step(dt, 3, nsteps=40)
        _, xg, vg, dg = sim.sync()
        E, ecc = sim.diagnostics(central=0)
    ref = orc.State(8, m, x, v, eps)
    ref.step(dt, 3, 40)
    # single steps agree to 1e-12 (test_one_step_parity_coarse_dt); over 40
    # steps of this collisional disc the rounding differences of each step
    # (FMA contraction, summation order) accumulate and are amplified by
    # close star-star passages, so the trajectory is held to 1e-11
    assert rel_rows(xg, ref.x) < 1e-12
    assert rel_rows(vg, ref.v) < 1e-11
    assert scaled_stack_err(dg[:, :4], ref.derivs[:, :4], dt) < 1e-11
    assert abs(E - ref.energy()) / abs(ref.energy()) < 1e-13
    assert rel_rows(ecc[1:], ref.ecc()[1:]) < 1e-10


def test_trajectory_parity_disc_4097_200_steps(mh, orc):
    """The survey's trajectory case: the SMBH disc of the 8th-order workload cut
    to 4096 stars + SMBH (total star mass 0.01, so m = 2.4e-6 per star),
    P(EC)^3, dt = 2 pi 1e-3, eps = 1e-4, 200 steps, through the pair-symmetric
    kernel.  At this size the disc is collisional: star pairs pass within a few
    eps, and two runs that start one rounding apart separate exponentially,
    reaching O(1) differences in the passing stars by step 200 (the oracle's own
    relative energy error there is ~7e-3).  So the GPU run is held to the
    oracle at the size that rounding alone produces: at steps 20, 50, 100 and
    200, the GPU-oracle differences of x and v (their maximum, 90th percentile
    and median over bodies, relative to the system's position and velocity
    scales) lie within 10x of the differences between the oracle and the
    oracle started with every coordinate moved by one ulp (plus 1e-15 of the
    scale).  A wrong term would separate the runs from the first step on.  At
    step 20 the energies also agree to 1e-13.  The SMBH row, 7e-5 from the
    barycentre, is measured against the system's scale like every other row."""
    m, x, v = I.smbh_disc(seed=2, N=4096)
    dt, eps = 2 * np.pi * 1e-3, 1e-4
    marks = (20, 50, 100, 200)
    gpu = {}
    with mh.Simulation(8, m, x, v, eps) as sim:
        done = 0
        for k in marks:
            sim.step(dt, 3, nsteps=k - done)
            done = k
            _, xg, vg, _ = sim.sync()
            gpu[k] = (xg, vg, sim.energy())
    rng = np.random.default_rng(5)
    xp = x * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], size=x.shape))
    ref, pert = orc.State(8, m, x, v, eps), orc.State(8, m, xp, v, eps)
    done = 0
    for k in marks:
        ref.step(dt, 3, k - done)
        pert.step(dt, 3, k - done)
        done = k
        xg, vg, Eg = gpu[k]
        for got, base, other in ((xg, ref.x, pert.x), (vg, ref.v, pert.v)):
            scale = np.abs(base).max()
            dg = np.linalg.norm(got - base, axis=1) / scale
            dp = np.linalg.norm(other - base, axis=1) / scale
            for q in (100, 90, 50):
                a, b = np.percentile(dg, q), np.percentile(dp, q)
                assert a <= 10 * b + 1e-15, (k, q, a, b)
        if k == 20:
            assert abs(Eg - ref.energy()) / abs(ref.energy()) < 1e-13


def test_diagnostics_parity(mh, orc):
    m, x, v = I.smbh_disc(seed=8, N=700)
    with mh.Simulation(6, m, x, v, 1e-4) as sim:
        E, ecc = sim.diagnostics(central=0)
    assert abs(E - orc.energy(m, x, v, 1e-4)) / abs(E) < 1e-13
    np.testing.assert_allclose(ecc, orc.ecc(m, x, v), rtol=1e-12, atol=1e-14)
    assert np.all(ecc[0] == 0)


@pytest.mark.parametrize("order", [4, 6, 8])
def test_time_symmetry_on_gpu(mh, order):
    m, x, v = I.kepler_pair(e=0.5)
    dt, K = 2 * np.pi / 128, 64
    with mh.Simulation(order, m, x, v, 0.0) as sim:
        sim.step(dt, 12, nsteps=K)
        sim.step(-dt, 12, nsteps=K)
        _, xg, vg, _ = sim.sync()
    assert np.abs(xg - x).max() < 1e-11 and np.abs(vg - v).max() < 1e-11


def test_single_body_moves_freely(mh):
    m = np.array([1.0])
    x = np.array([[0.1, 0.2, 0.3]])
    v = np.array([[1.0, -2.0, 0.5]])
    with mh.Simulation(8, m, x, v, 0.0) as sim:
        sim.step(0.25, 3, nsteps=4)
        t, xg, vg, dg = sim.sync()
    np.testing.assert_allclose(xg, x + v * 1.0, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(vg, v)
    assert np.all(dg == 0)


def test_set_state_and_counters(mh, orc):
    m, x, v = I.smbh_disc(seed=9, N=300)
    with mh.Simulation(8, m, x, v, 1e-4) as sim:
        sim.step(0.01, 3, nsteps=2)
        c = sim.counters()
        assert c["steps"] == 2 and c["evaluations"] == 6
        n = len(m)
        assert c["pair_interactions"] == 6 * n * (n - 1)
        sim.set_state(x, v, t=0.0)          # derivatives recomputed by initialisation
        _, xg, vg, dg = sim.sync()
    np.testing.assert_array_equal(xg, x)
    assert scaled_stack_err(dg, orc.initialise(8, m, x, v, 1e-4), 0.05) < 1e-12


def test_nonfinite_state_reported(mh):
    m = np.array([1.0, 1.0])
    x = np.array([[0.0, 0.0, 0.0], [1e-200, 0.0, 0.0]])   # r^2 underflows with eps = 0
    v = np.zeros((2, 3))
    with pytest.raises(mh.MHError) as ei:
        with mh.Simulation(4, m, x, v, 0.0) as sim:
            sim.step(0.1, 1)
            sim.sync()
    assert ei.value.code == -4


@pytest.fixture(scope="module")
def fp32_disc_case(orc):
    m, x, v = I.smbh_disc(seed=12, N=1023, m_total=1023e-9)
    dt, eps, nst = 2 * np.pi * 1e-3, 1e-4, 50
    ref = orc.State(8, m, x, v, eps)
    ref.step(dt, 3, nst)
    return m, x, v, dt, eps, nst, ref


@pytest.mark.parametrize("variant,symmetric", [(1, 1), (2, 1), (3, 1), (0, 2)])
def test_fp32_pair_form_accuracy(mh, orc, fp32_disc_case, variant, symmetric):
    """Precision form: the relative energy error after the run within 1e-9 of
    the oracle's, and accelerations within 2e-6 of the oracle's, for each
    evaluation kernel.  Stars of 1e-9 each keep star-star encounters
    negligible, so the energy error is the deterministic truncation error of
    the inner orbits (about 31 steps per orbit at r = 0.1) rather than a
    chaotic quantity."""
    m, x, v, dt, eps, nst, ref = fp32_disc_case
    with mh.Simulation(8, m, x, v, eps, precision=mh.MH_PREC_FP32PAIR, fp32_variant=variant,
                       symmetric=symmetric) as s32:
        E0 = s32.energy()
        s32.step(dt, 3, nsteps=nst)
        assert s32.counters()["pair_variant"] == (4 if symmetric == 2 else variant)
        _, x32, v32, d32 = s32.sync()
        E32 = s32.energy()
    dE_ref = ref.energy() / orc.energy(m, x, v, eps) - 1
    dE_32 = E32 / E0 - 1
    assert abs(dE_ref) > 1e-8                     # the quantity compared is well resolved
    assert abs(dE_32 - dE_ref) < 1e-9
    assert rel_rows(d32[:, 0], ref.derivs[:, 0]) < 2e-6


def test_fp32_variants_full_size(mh):
    """SMBH disc, 65536 stars + SMBH, one 8th-order P(EC)^3 step in the precision
    form with each evaluation kernel (three ordered-pair variants and the
    pair-symmetric default): one and two i-bodies per thread agree bit for bit;
    every kernel's accelerations lie within 2e-6 of the FP64 form's (itself
    held to the oracle at 1e-12)."""
    m, x, v = I.smbh_disc(seed=2, N=65536)
    dt, eps = 2 * np.pi * 1e-3, 1e-4
    with mh.Simulation(8, m, x, v, eps) as s64:
        s64.step(dt, 3)
        _, _, _, d64 = s64.sync()
    got = {}
    for variant in (1, 2, 3, 0):                  # 0: the default, each unordered pair once
        with mh.Simulation(8, m, x, v, eps, precision=mh.MH_PREC_FP32PAIR, fp32_variant=variant) as s32:
            s32.step(dt, 3)
            _, _, _, d32 = s32.sync()
            assert s32.counters()["pair_variant"] == (variant or 4)
        got[variant] = d32
        assert rel_rows(d32[:, 0], d64[:, 0]) < 2e-6, variant
    np.testing.assert_array_equal(got[1][:, :4], got[2][:, :4])
