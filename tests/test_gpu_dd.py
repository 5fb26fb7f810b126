"""GPU: the double-double form (mh_dd_*) against the binary128 oracle.

Tolerances.  Each double-double operation errs by a small multiple of u^2
(u = 2^-53, u^2 ~ 1.2e-32); a pair evaluation chains ~10^2 of them and a step a
few evaluations and a corrector, so positions and velocities after ten steps
carry ~1e-30 of relative rounding.  The tests allow 1e-27 (1e-25 after a
thousand steps), ten decades below what the FP64 form can reach; the binary128
oracle's own rounding (~1e-34) does not enter.  Derivative stacks are compared
in the scaled form of Eq. 1 (F_k = h^k a^(k) / k!)."""
import ctypes

import numpy as np
import pytest

from helpers import dd_diff, dd_scaled_stack_err
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


def _planets(N=7, seed=21):
    offs, m, x, v, pmin = I.planetary_systems(seed=seed, S=1, nmin=N, nmax=N)
    return m, x, v, float(pmin[0])


def _rel(got2, ref2):
    ref = np.asarray(ref2)[..., 0] + np.asarray(ref2)[..., 1]
    return float(np.abs(dd_diff(got2, ref2)).max() / np.abs(ref).max())


@pytest.mark.parametrize("order", [4, 6, 8, 10, 12])
def test_dd_initialisation_parity(mh, orc, order):
    m, x, v, pmin = _planets()
    dt = pmin / 64
    _, _, d_ref = orc.dd_run(order, m, x, v, 0.0, dt, 3, 0)
    with mh.DDSimulation(order, m, x, v, 0.0) as sim:
        _, x2, v2, d2 = sim.sync()
    assert np.array_equal(x2[..., 0], x) and not x2[..., 1].any()
    err = dd_scaled_stack_err(d2, d_ref, dt)
    assert err < 1e-27, err


@pytest.mark.parametrize("order", [4, 6, 8, 10, 12])
@pytest.mark.parametrize("modified", [True, False])
def test_dd_steps_parity(mh, orc, order, modified):
    m, x, v, pmin = _planets()
    dt = pmin / 64
    xr, vr, dr = orc.dd_run(order, m, x, v, 0.0, dt, 3, 10, modified=modified)
    beta = mh.MH_BETA_MODIFIED if modified else mh.MH_BETA_STANDARD
    with mh.DDSimulation(order, m, x, v, 0.0, beta=beta) as sim:
        sim.step(dt, 3, nsteps=10)
        t2, x2, v2, d2 = sim.sync()
    assert _rel(x2, xr) < 1e-27, _rel(x2, xr)
    assert _rel(v2, vr) < 1e-27, _rel(v2, vr)
    err = dd_scaled_stack_err(d2, dr, dt)
    assert err < 1e-25, err
    assert t2[0] + t2[1] == pytest.approx(10 * dt, rel=1e-15)


def test_dd_ragged_multi_chunk(mh, orc):
    """133 bodies: two 128-thread i-blocks (the second ragged) and 34 j-chunks of
    4 with a one-body tail; softened, 8th order, two steps of n = 3."""
    m, x, v = I.planetesimal_ring(seed=9, n=132, m=1e-7)
    dt = 2 * np.pi / 256
    xr, vr, dr = orc.dd_run(8, m, x, v, 1e-3, dt, 3, 2)
    with mh.DDSimulation(8, m, x, v, 1e-3) as sim:
        sim.step(dt, 3, nsteps=2)
        _, x2, v2, d2 = sim.sync()
    assert _rel(x2, xr) < 1e-27, _rel(x2, xr)
    assert _rel(v2, vr) < 1e-27, _rel(v2, vr)
    assert dd_scaled_stack_err(d2, dr, dt) < 1e-25


def test_dd_single_body(mh, orc):
    """One body: no pairs, a free flight x0 + v0 t in double-double."""
    m = np.array([1.0])
    x = np.array([[0.1, -0.7, 3.3]])
    v = np.array([[1.0 / 3.0, 2.0 / 7.0, -1.0 / 9.0]])
    with mh.DDSimulation(8, m, x, v, 0.0) as sim:
        sim.step(0.01, 2, nsteps=100)
        _, x2, v2, d2 = sim.sync()
    assert not d2.any()
    xr, _, _ = orc.dd_run(8, m, x, v, 0.0, 0.01, 2, 100)
    assert _rel(x2, xr) < 1e-30


@pytest.mark.parametrize("order", [10, 12])
def test_dd_kepler_pair(mh, orc, order):
    """Two bodies: the Kepler pair of Section 3.1 at 10th and 12th order."""
    m, x, v = I.kepler_pair(a=1.0, e=0.1, M=1.0, m=1e-3)
    xr, vr, _ = orc.dd_run(order, m, x, v, 0.0, 2.0 ** -4, 3, 20)
    with mh.DDSimulation(order, m, x, v, 0.0) as sim:
        sim.step(2.0 ** -4, 3, nsteps=20)
        _, x2, v2, _ = sim.sync()
    assert _rel(x2, xr) < 1e-27 and _rel(v2, vr) < 1e-27


def test_dd_diagnostics_parity(mh, orc):
    m, x, v, pmin = _planets()
    with mh.DDSimulation(8, m, x, v, 1e-4) as sim:
        sim.step(pmin / 64, 3, nsteps=5)
        _, x2, v2, _ = sim.sync()
        E2, e2 = sim.diagnostics(central=0)
    Er = orc.dd_energy(m, x2, v2, 1e-4)
    assert abs(dd_diff(E2, Er)) < 1e-29 * abs(Er[0])
    er = orc.dd_ecc(m, x2, v2, 1.0, 0)
    assert np.abs(dd_diff(e2, er)).max() < 1e-28
    assert not e2[0].any()


def test_dd_graph_replay_matches_single_steps(mh):
    m, x, v, pmin = _planets()
    dt = pmin / 64
    with mh.DDSimulation(8, m, x, v, 0.0) as a, mh.DDSimulation(8, m, x, v, 0.0) as b:
        a.step(dt, 3, nsteps=6)
        for _ in range(6):
            b.step(dt, 3)
        ra, rb = a.sync(), b.sync()
        ca = a.counters()
    for qa, qb in zip(ra, rb):
        assert np.array_equal(qa, qb)
    assert ca["steps"] == 6 and ca["evaluations"] == 18
    assert ca["pair_interactions"] == 18 * 7 * 6


def test_dd_set_state_round_trip(mh):
    m, x, v, pmin = _planets()
    dt = pmin / 64
    with mh.DDSimulation(10, m, x, v, 0.0) as a, mh.DDSimulation(10, m, x, v, 0.0) as b:
        a.step(dt, 2, nsteps=3)
        t2, x2, v2, d2 = a.sync()
        b.set_state(x2, v2, d2, t2)
        a.step(dt, 2, nsteps=3)
        b.step(dt, 2, nsteps=3)
        for qa, qb in zip(a.sync(), b.sync()):
            assert np.array_equal(qa, qb)


@pytest.mark.parametrize("order,bound", [(10, 1e-17), (12, 1e-21)])
def test_dd_section31_energy_below_fp64(mh, orc, order, bound):
    """a = 1, e = 0.1, dt = 2^-4, n = 3, ten orbits: the 10th- and 12th-order
    double-double runs keep the energy error below 1e-17 and 1e-21 (the binary128
    oracle gives 9e-19 and 2.5e-22), the FP64 form's stays at round-off."""
    m, x, v = I.kepler_pair(a=1.0, e=0.1, M=1.0, m=1e-3)
    dt = 2.0 ** -4
    from fractions import Fraction
    val = lambda E2: Fraction(float(E2[0])) + Fraction(float(E2[1]))
    worst, worst64 = 0.0, 0.0
    with mh.DDSimulation(order, m, x, v, 0.0) as sim, mh.Simulation(order, m, x, v, 0.0) as ref:
        E0 = val(sim.diagnostics()[0])
        E0f = ref.diagnostics(central=0)[0]
        for _ in range(20):
            sim.step(dt, 3, nsteps=50)
            ref.step(dt, 3, nsteps=50)
            worst = max(worst, float(abs((val(sim.diagnostics()[0]) - E0) / E0)))
            worst64 = max(worst64, abs(ref.diagnostics(central=0)[0] / E0f - 1))
        _, x2, v2, _ = sim.sync()
    assert worst < bound, worst
    assert worst64 > 3e-16 and worst < worst64 / 1e3, (worst, worst64)
    xr, vr, _ = orc.dd_run(order, m, x, v, 0.0, dt, 3, 1000)
    assert _rel(x2, xr) < 1e-25 and _rel(v2, vr) < 1e-25


def test_dd_argument_errors(mh):
    from paper_2006_02501_gb300 import _capi
    m, x, v, pmin = _planets()
    for order in (2, 7, 14):
        with pytest.raises(mh.MHError) as e:
            mh.DDSimulation(order, m, x, v, 0.0)
        assert e.value.code == _capi.MH_EINVAL
    with pytest.raises(mh.MHError):
        mh.DDSimulation(8, m, x, v, -1.0)
    bad = x.copy()
    bad[2, 1] = np.nan
    with pytest.raises(mh.MHError) as e:
        mh.DDSimulation(8, m, bad, v, 0.0)
    assert e.value.code == _capi.MH_ENONFINITE
    with mh.DDSimulation(8, m, x, v, 0.0) as sim:
        for args in ((0.0, 3), (float("inf"), 3), (0.01, 0), (0.01, 65)):
            with pytest.raises(mh.MHError):
                sim.step(*args)
        sim.step(0.01, 3, nsteps=0)
        with pytest.raises(mh.MHError):
            sim.diagnostics(central=7)
        L = _capi.lib()
        assert L.mh_dd_step(None, 0.01, 3, 1) == _capi.MH_EINVAL
        assert L.mh_dd_sync(None, None, None, None, None) == _capi.MH_EINVAL
        n = ctypes.c_int64()
        assert L.mh_dd_info(sim._h, ctypes.byref(n), None, None) == 0 and n.value == 7


def test_dd_bench_size_sampled_start(mh, orc):
    """The double-double form at the size bench.py times (the SMBH disc cut to
    4096 bodies, 8th order, eps = 1e-4; 32 i-blocks x 38 j-chunks): a and a-dot
    of the start (the first initialisation pass, from x and v alone) for sampled
    bodies, including the SMBH and the last i-block's tail, against binary128 sums
    over all 4096 bodies.  Tolerance 1e-26 of each row: the SMBH's acceleration
    is a ~30-fold cancelling sum of 4095 star terms."""
    m, x, v = I.smbh_disc(seed=2, N=4095)
    with mh.DDSimulation(8, m, x, v, 1e-4) as sim:
        _, _, _, d2 = sim.sync()
    tr = np.stack([orc.as_dd(x), orc.as_dd(v)], axis=1)
    for i0, i1 in ((0, 3), (1000, 1001), (2047, 2049), (4093, 4096)):
        ref = orc.dd_evaluate(m, tr, 1e-4, 1.0, i0, i1)
        for k in range(2):
            diff = np.linalg.norm(dd_diff(d2[i0:i1, k], ref[:, k]), axis=-1)
            scale = np.linalg.norm(ref[:, k, :, 0], axis=-1)
            assert (diff <= 1e-26 * scale).all(), (i0, k, diff / scale)


# ---- pair-symmetric double-double evaluation (k_dd_pair_sym) ----

def _dd_traj(seed, N, P):
    """Seeded evaluation input of N bodies: an SMBH disc's x, v with the Kepler
    a, a-dot (helpers.kepler_traj), normal rows above a-dot, and low words of
    up to 2^-54 of each value (so every double-word is normalised and the low
    words take part)."""
    from helpers import kepler_traj
    m, x, v = I.smbh_disc(seed=seed, N=N - 1)
    traj = kepler_traj(m, x, v, min(P, 3))
    rng = np.random.default_rng(seed)
    if P > 3:
        traj = np.concatenate([traj, rng.normal(size=(N, P - 3, 3))], axis=1)
    lo = traj * 2.0 ** -54 * rng.uniform(-1.0, 1.0, size=traj.shape)
    return m, np.ascontiguousarray(np.stack([traj, lo], axis=-1))


def _rows_ok(got2, ref2, tol):
    diff = np.linalg.norm(dd_diff(got2, ref2), axis=-1)
    scale = np.linalg.norm(np.asarray(ref2)[..., 0], axis=-1)
    return float((diff / scale).max()) <= tol, float((diff / scale).max())


@pytest.mark.parametrize("N", [2100, 2500])      # 33 blocks of 64 (odd) and 40 (even), both ragged
@pytest.mark.parametrize("P", [1, 3, 5])
def test_dd_symmetric_eval_sampled_against_oracle(mh, orc, N, P):
    """Each unordered pair once, both bodies from one evaluation: sampled bodies
    (the SMBH, a block boundary, the middle, the ragged tail) against binary128
    direct sums over all N bodies, at 1e-26 of each row as the bench-size test;
    the ordered kernel on the same input gives the same rows."""
    m, tr2 = _dd_traj(40 + P, N, P)
    for i0, i1 in ((0, 3), (127, 130), (1234, 1236), (N - 5, N)):
        ref = orc.dd_evaluate(m, tr2, 1e-4, 1.0, i0, i1)
        got = mh.dd_pair_eval(P, m, tr2, 1e-4, 1.0, i0, i1, symmetric=2)
        ordered = mh.dd_pair_eval(P, m, tr2, 1e-4, 1.0, i0, i1, symmetric=0)
        for k in range(P + 1):
            ok, e = _rows_ok(got[:, k], ref[:, k], 1e-26)
            assert ok, (i0, k, e)
            ok, e = _rows_ok(ordered[:, k], ref[:, k], 1e-26)
            assert ok, (i0, k, e, "ordered")


def test_dd_symmetric_matches_ordered_all_bodies(mh):
    """All 4096 bodies of the bench-size disc at P = 3: the symmetric and the
    ordered kernels agree to 1e-27 of each row (both sit ~1e-31 from the exact
    sums), and two symmetric runs are bit-identical (the slots are added in a
    fixed order)."""
    m, tr2 = _dd_traj(44, 4096, 3)
    sym = mh.dd_pair_eval(3, m, tr2, 1e-4, 1.0, symmetric=2)
    ordered = mh.dd_pair_eval(3, m, tr2, 1e-4, 1.0, symmetric=0)
    for k in range(4):
        ok, e = _rows_ok(sym[:, k], ordered[:, k], 1e-27)
        assert ok, (k, e)
    again = mh.dd_pair_eval(3, m, tr2, 1e-4, 1.0, symmetric=2)
    assert np.array_equal(sym, again)


@pytest.mark.parametrize("order", [4, 12])
def test_dd_symmetric_steps_parity_planets(mh, orc, order):
    """Ten steps of a 7-body planetary system with the symmetric kernel forced
    (one diagonal item: the ring distances 1 .. 16 of one subtile, 57 empty
    lanes) against the binary128 oracle, at the tolerances of the ordered tests."""
    m, x, v, pmin = _planets()
    dt = pmin / 64
    xr, vr, dr = orc.dd_run(order, m, x, v, 0.0, dt, 3, 10)
    with mh.DDSimulation(order, m, x, v, 0.0, symmetric=2) as sim:
        sim.step(dt, 3, nsteps=10)
        _, x2, v2, d2 = sim.sync()
    assert _rel(x2, xr) < 1e-27, _rel(x2, xr)
    assert _rel(v2, vr) < 1e-27, _rel(v2, vr)
    assert dd_scaled_stack_err(d2, dr, dt) < 1e-25


def test_dd_symmetric_steps_parity_ragged(mh, orc):
    """The 133-body softened ring of test_dd_ragged_multi_chunk with the
    symmetric kernel forced: three blocks of 64 bodies (three diagonal items and
    three at distance 1, the third block ragged with 5 bodies), two steps of n = 3."""
    m, x, v = I.planetesimal_ring(seed=9, n=132, m=1e-7)
    dt = 2 * np.pi / 256
    xr, vr, dr = orc.dd_run(8, m, x, v, 1e-3, dt, 3, 2)
    with mh.DDSimulation(8, m, x, v, 1e-3, symmetric=2) as sim:
        sim.step(dt, 3, nsteps=2)
        _, x2, v2, d2 = sim.sync()
    assert _rel(x2, xr) < 1e-27, _rel(x2, xr)
    assert _rel(v2, vr) < 1e-27, _rel(v2, vr)
    assert dd_scaled_stack_err(d2, dr, dt) < 1e-25
