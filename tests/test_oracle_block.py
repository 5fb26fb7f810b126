"""Pins for the oracle's block time steps (the Section 4 option, scheme of
reading R12: ticks of dt_max 2^-k_max, levels from an Aarseth-type estimate,
halving freely, doubling only when commensurate)."""
import numpy as np
import pytest

from paper_2006_02501_gb300 import inputs as I


def test_aarseth_estimate_circular_orbit_closed_form(orc):
    # circular motion at rate w: |a^(k)| = w^(k+2) R, so the estimate is eta / w
    w, R, eta = 1.7, 0.8, 0.05
    d = np.array([[np.cos(k * np.pi / 2), np.sin(k * np.pi / 2), 0.0] for k in range(4)])
    d = d * np.array([w ** (k + 2) * R for k in range(4)])[:, None]
    assert orc.aarseth_dt(d, eta) == pytest.approx(eta / w, rel=1e-14)


def test_level_rules(orc):
    dt_max, k_max = 1.0, 6
    assert orc.block_level(2.0, dt_max, k_max) == 0          # estimate above dt_max
    assert orc.block_level(0.3, dt_max, k_max) == 2          # 0.25 <= 0.3
    assert orc.block_level(1e-9, dt_max, k_max) == k_max     # clamped
    # shrinking is free
    assert orc.block_level(0.1, dt_max, k_max, k_old=1, T=3) == 4
    # growing: one level at most, and only at a commensurate tick (span of level 2 = 16 ticks)
    assert orc.block_level(0.9, dt_max, k_max, k_old=3, T=16) == 2
    assert orc.block_level(0.9, dt_max, k_max, k_old=3, T=8) == 3


@pytest.mark.parametrize("order", [6, 8])
def test_block_equals_shared_steps_when_levels_stay_fixed(orc, order):
    """Circular two-body orbit: the estimate is constant, every body keeps one
    level, and the block scheme reduces to shared steps of dt_max 2^-k exactly."""
    m, x, v = I.kepler_pair(a=1.0, e=0.0, M=1.0, m=1e-3)
    dt_max, k_max, eta = 2.0 ** -2, 10, 0.05
    B = orc.BlockState(order, m, x, v, 0.0, dt_max, k_max, eta)
    k = int(B.level[0])
    assert np.all(B.level == k) and k > 0
    B.advance(4 * dt_max, 3)
    assert np.all(B.level == k)
    S = orc.State(order, m, x, v, 0.0)
    S.step(dt_max * 2.0 ** -k, 3, 4 * 2 ** k)
    np.testing.assert_array_equal(B.x, S.x)
    np.testing.assert_array_equal(B.v, S.v)
    assert B.block_steps == 4 * 2 ** k


def test_block_hierarchical_system_against_dop853(orc):
    """A tight inner pair and a wide outer body get different levels; the block
    integration agrees with an independent DOP853 integration."""
    from scipy.integrate import solve_ivp
    m = np.array([1.0, 1e-3, 1e-4])
    x = np.array([[0.0, 0, 0], [0.3, 0, 0], [-2.0, 0.2, 0.0]])
    v = np.array([[0.0, -0.0577, 0], [0.0, np.sqrt(1.001 / 0.3), 0.0], [0.1, -0.7, 0.05]])
    mt = m.sum()
    x -= (m[:, None] * x).sum(0) / mt
    v -= (m[:, None] * v).sum(0) / mt
    eps = 1e-6
    B = orc.BlockState(8, m, x, v, eps, dt_max=2.0 ** -3, k_max=10, eta=0.02)
    assert len(set(B.level.tolist())) >= 2
    E0 = B.energy()
    B.advance(2.0, 3)
    assert np.all(B.T == B.T[0])

    def rhs(t, y):
        X = y[:9].reshape(3, 3)
        A = np.zeros_like(X)
        for i in range(3):
            for j in range(3):
                if i != j:
                    d = X[j] - X[i]
                    A[i] += m[j] * d / (d @ d + eps * eps) ** 1.5
        return np.concatenate([y[9:], A.ravel()])
    sol = solve_ivp(rhs, (0, 2.0), np.concatenate([x.ravel(), v.ravel()]), method="DOP853",
                    rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(B.x.ravel(), sol.y[:9, -1], atol=1e-9)
    assert abs(B.energy() / E0 - 1) < 1e-10


def test_block_disc_synchronises_and_conserves_energy(orc):
    m, x, v = I.smbh_disc(seed=3, N=300)
    B = orc.BlockState(6, m, x, v, 1e-4, dt_max=2.0 ** -5, k_max=12, eta=0.05)
    E0 = B.energy()
    B.advance(2 * 2.0 ** -5, 3)
    assert np.all(B.T == 2 * 2 ** 12)
    assert B.active_total < B.block_steps * B.N          # fewer updates than shared steps
    assert abs(B.energy() / E0 - 1) < 1e-9
