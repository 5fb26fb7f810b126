"""Learned predictor residual: the GPU network against the FP64 CPU reference
(with bfloat16 rounding at the same points), sample collection against the
oracle, convergence-controlled stepping, and what a trained network gains."""
import numpy as np
import pytest

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


@pytest.fixture(scope="module")
def Lr():
    from oracle import learned
    return learned


def _net(mh, Lr, n_in=18, H=128, n_out=6, seed=0):
    net = mh.MLP(n_in, H, n_out, seed=1)
    rng = np.random.default_rng(seed)
    p = {k: rng.normal(scale=0.5 / np.sqrt(s[-1]), size=s) for k, s in Lr.SHAPES(n_in, H, n_out)}
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(scale=0.1, size=p[k].shape)
    flat = Lr.flatten(p, n_in, H, n_out).astype(np.float32)
    net.set_params(flat)
    return net, Lr.unflatten(flat.astype(np.float64), n_in, H, n_out)


@pytest.mark.parametrize("B", [1, 100, 1000])
def test_mlp_forward_matches_reference(mh, Lr, B):
    net, p = _net(mh, Lr)
    X = np.random.default_rng(2).normal(size=(B, 18)).astype(np.float32)
    y = torch.zeros((B, 6), dtype=torch.float32, device="cuda")
    net.forward(torch.from_numpy(X).cuda(), y)
    torch.cuda.synchronize()
    ref, _ = Lr.forward(p, X.astype(np.float64), bf=True)
    err = np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 5e-3


def test_mlp_gradient_matches_reference(mh, Lr):
    net, p = _net(mh, Lr, seed=3)
    rng = np.random.default_rng(4)
    B = 777
    X = rng.normal(size=(B, 18)).astype(np.float32)
    T = rng.normal(size=(B, 6)).astype(np.float32)
    loss, g = net.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    loss_ref, g_ref = Lr.loss_grad(p, X.astype(np.float64), T.astype(np.float64), bf=True)
    assert loss == pytest.approx(loss_ref, rel=1e-3)
    gd = Lr.unflatten(g.astype(np.float64), 18, 128, 6)
    for k in g_ref:
        rel = np.linalg.norm(gd[k] - g_ref[k]) / np.linalg.norm(g_ref[k])
        assert rel < 2e-2, (k, rel)


def test_mlp_training_reduces_loss(mh):
    rng = np.random.default_rng(5)
    n = 16384
    X = rng.normal(size=(n, 18)).astype(np.float32)
    T = np.stack([np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2], np.tanh(X[:, 3]), X[:, 4] ** 2 - 1,
                  np.cos(X[:, 5]), 0.3 * X[:, 6], X[:, 7] * X[:, 8]], axis=1).astype(np.float32)
    net = mh.MLP(18, 128, 6, seed=7)
    xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    l0, _ = net.loss_grad(xd, td)
    l1 = net.train(xd, td, epochs=20, batch=512, lr=2e-3, seed=1)
    assert l1 < 0.1 * l0


def test_collect_samples_match_reference(mh, orc, Lr):
    """One converged step (P(EC)^8) of a ring with dt = 0.1: features and targets
    of every body against the oracle's step and predictor (FP64)."""
    m, x, v = I.planetesimal_ring(seed=6, n=400, m=1e-9, a_lo=0.8, a_hi=1.3, sigma_e=0.05, sigma_i=0.02)
    dt, eps = 0.1, 1e-6
    N = len(m)
    f = torch.zeros((N, 19), dtype=torch.float32, device="cuda")
    t = torch.zeros((N, 6), dtype=torch.float32, device="cuda")
    ref = orc.State(8, m, x, v, eps)
    d0 = ref.derivs.copy()
    with mh.Simulation(8, m, x, v, eps) as sim:
        sim.collect_samples(dt, 8, f, t)
    xp, vp, _ = orc.predict(8, dt, x, v, d0)
    ref.step(dt, 8)
    u, R, na, sig, mask = Lr.features(d0, dt)
    y = Lr.targets(ref.x - xp, ref.v - vp, R, na, sig, mask, dt)
    fg, tg = f.cpu().numpy(), t.cpu().numpy()
    assert mask[1:].all()
    np.testing.assert_allclose(fg[mask], u[mask], rtol=0, atol=1e-5 * np.abs(u[mask]).max())
    scale = np.abs(y[mask]).max()
    assert scale > 0.1
    assert np.abs(tg[mask] - y[mask]).max() < 1e-3 * scale


def test_step_converge_matches_fixed_passes(mh):
    m, x, v = I.smbh_disc(seed=7, N=2000)
    dt, eps = 2 * np.pi * 1e-3, 1e-4
    with mh.Simulation(8, m, x, v, eps) as a, mh.Simulation(8, m, x, v, eps) as b:
        n = a.step_converge(dt, 1e-13, 12)
        assert 2 <= n <= 12
        b.step(dt, n)
        _, xa, va, _ = a.sync()
        _, xb, vb, _ = b.sync()
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)


def test_learned_predictor_gain(mh):
    """Train on converged corrector outputs of one collisionless ring (24 steps),
    then on a fresh ring compare with the plain Taylor predictor: the worst
    body's predicted x and v errors (against a converged step), the error after
    one evaluate-correct pass, and the passes to a 1e-13 convergence tolerance.

    The gain claimed is the prediction's: x and v errors at least 2x lower
    (measured 2.7x and 3.5x), and a lower error after the first pass (1.14x).
    No pass is saved: the P(EC)^n iteration contracts by about 1e3 per pass
    here, so a predictor a few times better does not remove one at 1e-13
    (measured 4.05 passes per step with either predictor).  The pass count is
    held to no loss beyond one pass in the 20 steps."""
    from paper_2006_02501_gb300 import train_predictor as tp
    eps, dt, tol = 1e-6, 0.15, 1e-13
    ring = lambda seed: I.planetesimal_ring(seed=seed, n=4000, m=1e-12, a_lo=0.7, a_hi=1.2, sigma_e=0.05,
                                            sigma_i=0.02)
    m, x, v = ring(100)
    with mh.Simulation(8, m, x, v, eps) as sim:
        net = tp.fit(tp.collect(sim, dt, steps=24, n_iter=10), epochs=80, seed=0)
    m2, x2, v2 = ring(1000)
    with mh.Simulation(8, m2, x2, v2, eps) as c:
        c.step(dt, 12)
        _, xc, vc, _ = c.sync()
    with mh.Simulation(8, m2, x2, v2, eps) as a, mh.Simulation(8, m2, x2, v2, eps) as b:
        b.set_predictor(net)
        xa, va = a.predict(dt)
        xb, vb = b.predict(dt)
        a.step(dt, 1)
        b.step(dt, 1)
        _, x1a, _, _ = a.sync()
        _, x1b, _, _ = b.sync()
    ex_plain, ex_learn = np.abs(xc - xa).max(), np.abs(xc - xb).max()
    ev_plain, ev_learn = np.abs(vc - va).max(), np.abs(vc - vb).max()
    e1_plain, e1_learn = np.abs(xc - x1a).max(), np.abs(xc - x1b).max()
    print(f"worst x prediction error plain {ex_plain:.3e} learned {ex_learn:.3e}; "
          f"v {ev_plain:.3e} {ev_learn:.3e}; after one pass {e1_plain:.3e} {e1_learn:.3e}")
    assert ex_learn < 0.5 * ex_plain
    assert ev_learn < 0.5 * ev_plain
    assert e1_learn < e1_plain
    plain, learned = [], []
    with mh.Simulation(8, m2, x2, v2, eps) as a, mh.Simulation(8, m2, x2, v2, eps) as b:
        b.set_predictor(net)
        for _ in range(20):
            plain.append(a.step_converge(dt, tol, 20))
            learned.append(b.step_converge(dt, tol, 20))
        _, xa, _, _ = a.sync()
        _, xb, _, _ = b.sync()
    print("passes to 1e-13: plain", np.mean(plain), "learned", np.mean(learned))
    assert np.mean(learned) <= np.mean(plain) + 0.05
    assert np.abs(xa - xb).max() < 1e-11                     # both converge to the same solution
