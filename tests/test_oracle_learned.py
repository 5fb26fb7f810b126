"""Pins for the CPU reference of the learned predictor (oracle/learned.py):
bfloat16 rounding on exact values, MLP gradients against central finite
differences, rotation invariance of the features, and targets/residual being
inverse maps."""
import numpy as np
import pytest

from oracle import learned as Lr


def test_bf16_rounding_exact_values():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 1 + 2 ** -7, 3.0e38], dtype=np.float32)
    got = Lr.bf16(x)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: to even (1.0); 1 + 3*2^-8 rounds up to 1 + 2^-6
    assert got[0] == 1.0 and got[1] == 1.0 and got[2] == 1 + 2 ** -6
    assert got[3] == -2.5 and got[4] == 1 + 2 ** -7
    assert np.isfinite(got[5])


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    n_in, H, n_out, B = 18, 16, 6, 7
    p = {k: rng.normal(scale=0.4, size=s) for k, s in Lr.SHAPES(n_in, H, n_out)}
    X = rng.normal(size=(B, n_in))
    T = rng.normal(size=(B, n_out))
    loss, g = Lr.loss_grad(p, X, T)
    flat = Lr.flatten(p, n_in, H, n_out)
    gflat = Lr.flatten(g, n_in, H, n_out)
    for idx in rng.choice(flat.size, 40, replace=False):
        e = np.zeros_like(flat)
        e[idx] = 1e-6
        lp, _ = Lr.loss_grad(Lr.unflatten(flat + e, n_in, H, n_out), X, T)
        lm, _ = Lr.loss_grad(Lr.unflatten(flat - e, n_in, H, n_out), X, T)
        fd = (lp - lm) / 2e-6
        assert fd == pytest.approx(gflat[idx], rel=1e-6, abs=1e-9)


def _random_rotation(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


def test_features_rotation_invariant_and_targets_invertible():
    rng = np.random.default_rng(1)
    N, K, dt = 50, 6, 0.01
    d = rng.normal(size=(N, K, 3)) * (2.0 ** -np.arange(K))[None, :, None]
    u, R, na, sig, mask = Lr.features(d, dt)
    Q = _random_rotation(rng)
    u2, R2, na2, sig2, mask2 = Lr.features(d @ Q.T, dt)
    assert np.array_equal(mask, mask2) and mask.any()
    np.testing.assert_allclose(u2[mask], u[mask], rtol=0, atol=1e-12)
    # F_0 in its own frame is (1, 0, 0); F_1 has no e3 component
    np.testing.assert_allclose(u[mask][:, :3], np.tile([1.0, 0, 0], (mask.sum(), 1)), atol=1e-14)
    np.testing.assert_allclose(u[mask][:, 5], 0.0, atol=1e-14)
    dx = rng.normal(size=(N, 3)) * 1e-9
    dv = rng.normal(size=(N, 3)) * 1e-8
    y = Lr.targets(dx, dv, R, na, sig, mask, dt)
    bx, bv = Lr.residual(y, R, na, sig, mask, dt)
    np.testing.assert_allclose(bx[mask], dx[mask], rtol=1e-12, atol=0)
    np.testing.assert_allclose(bv[mask], dv[mask], rtol=1e-12, atol=0)
