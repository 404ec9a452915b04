"""Pins of the reaction-path landscape, the Gaussian policy head and returns."""
import numpy as np
import pytest

from paper_2408_00930_gb300 import inputs


def test_energy_single_gaussian_matches_scipy_mvn(orc):
    stats = pytest.importorskip("scipy.stats")
    g = inputs.rng(0)
    for D in (1, 3, 24):
        c = g.uniform(-3, 3, (1, D)); w = np.array([0.7]); a = np.array([-1.3])
        for _ in range(5):
            x = c[0] + g.normal(0, 0.8, D)
            ref = a[0] * (2 * np.pi * w[0] ** 2) ** (D / 2) * stats.multivariate_normal(
                mean=c[0], cov=w[0] ** 2 * np.eye(D)).pdf(x)
            assert orc.landscape_energy(c, w, a, x) == pytest.approx(ref, rel=1e-10, abs=1e-300)
    # at a centre the single Gaussian gives exactly its amplitude
    assert orc.landscape_energy(c, w, a, c[0]) == a[0]


def test_energy_direct_vs_expanded_form(orc):
    g = inputs.rng(1)
    c, w, a = inputs.landscape_params(g, 64, 24)
    for _ in range(10):
        x = g.uniform(-3, 3, 24)
        d2 = (x * x).sum() + (c * c).sum(1) - 2 * c @ x
        ref = (a * np.exp(-d2 / (2 * w * w))).sum()
        scale = (np.abs(a) * np.exp(-d2 / (2 * w * w))).sum()
        E = orc.landscape_energy(c, w, a, x)
        assert abs(E - ref) <= 1e-9 * max(scale, 1e-300)
        assert orc.landscape_energy_scale(c, w, a, x) == pytest.approx(scale, rel=1e-9)


def test_gradient_vs_central_differences(orc):
    g = inputs.rng(2)
    for D, M in [(1, 1), (2, 3), (3, 4)]:
        c = g.uniform(-1, 1, (M, D)); w = np.exp(0.3 * g.standard_normal(M))
        a = g.standard_normal(M)
        for _ in range(5):
            x = g.uniform(-1.5, 1.5, D)
            gr = orc.landscape_grad(c, w, a, x)
            h = 1e-6
            fd = np.array([(orc.landscape_energy(c, w, a, x + h * e) -
                            orc.landscape_energy(c, w, a, x - h * e)) / (2 * h)
                           for e in np.eye(D)])
            np.testing.assert_allclose(gr, fd, rtol=1e-7, atol=1e-9)


def test_landscape_init_distributions(orc):
    stats = pytest.importorskip("scipy.stats")
    c, w, a = orc.landscape_init(21, 24, 4096)
    assert c.shape == (4096, 24)
    assert np.all(np.abs(c) <= 3.0)
    assert stats.kstest(c.ravel(), "uniform", args=(-3, 6)).pvalue > 1e-4
    assert stats.kstest(np.log(w) / 0.3, "norm").pvalue > 1e-4
    assert stats.kstest(a, "norm").pvalue > 1e-4
    # coordinates are exact FP32 uniform draws
    wd = orc.draw(21, 5, 0, 0, orc.TAG_LANDSCAPE_INIT, 1)
    assert c[5, 4] == orc.uniform_f32(int(wd[0]), -3, 3)


def test_gaussian_head_logp_and_clip(orc):
    stats = pytest.importorskip("scipy.stats")
    g = inputs.rng(3)
    D = 24
    for _ in range(20):
        out = np.concatenate([g.normal(0, 0.05, D), g.normal(-2.5, 3, D)])
        z = g.standard_normal(D)
        dx, lp = orc.gaussian_action(out, z, 0.1)
        ls = np.clip(out[D:], -5, 2)
        sample = out[:D] + np.exp(ls) * z
        ref = stats.norm(loc=out[:D], scale=np.exp(ls)).logpdf(sample).sum()
        assert lp == pytest.approx(ref, rel=1e-10)
        assert np.all(np.abs(dx) <= 0.1)
        inside = np.abs(sample) < 0.1
        np.testing.assert_allclose(dx[inside], sample[inside], rtol=1e-15)
        assert np.all(dx[~inside] == np.sign(sample[~inside]) * 0.1)


def test_landscape_rollout_semantics(orc):
    g = inputs.rng(4)
    D, M = 6, 32
    c, w, a = orc.landscape_init(3, D, M)
    widths = [D, 16, 16, 2 * D]
    p = inputs.policy_params(g, widths)
    r = orc.landscape_rollout(c, w, a, p, 16, 16, seed=8, env_ids=[0, 5], n_steps=12,
                              episode_limit=10, noise_sigma=0.05, step_clip=0.1)
    for e, env in enumerate([0, 5]):
        np.testing.assert_array_equal(r["obs"][0, e], orc.landscape_reset_draw(8, orc.STEP_INIT, env, D))
        for t in range(11):
            if t == 9:
                assert r["done"][t, e] == 1
                np.testing.assert_array_equal(r["obs"][t + 1, e], orc.landscape_reset_draw(8, 9, env, D))
            else:
                assert r["done"][t, e] == 0
                np.testing.assert_allclose(r["obs"][t + 1, e], r["obs"][t, e] + r["act"][t, e],
                                           rtol=0, atol=0)
            # energy record is E of the post-step state
            E = orc.landscape_energy(c, w, a, r["obs"][t, e] + r["act"][t, e])
            assert r["energy"][t, e] == E
        # reward telescopes: r_t = Eobs_t - Eobs_{t+1} with Eobs = E + sigma * noise
        eobs_prev = (orc.landscape_energy(c, w, a, r["obs"][0, e]) +
                     0.05 * orc.landscape_noise(8, orc.STEP_INIT, env, 1))
        for t in range(9):
            eobs = r["energy"][t, e] + 0.05 * orc.landscape_noise(8, t, env, 0)
            assert r["reward"][t, e] == pytest.approx(eobs_prev - eobs, abs=1e-15)
            eobs_prev = eobs


def test_returns_closed_form_and_library(orc):
    signal = pytest.importorskip("scipy.signal")
    T, gam = 1000, 0.99
    r = np.ones((T, 3)); d = np.zeros((T, 3), np.uint8)
    G = orc.returns(r, d, gam)
    t = np.arange(T)
    np.testing.assert_allclose(G[:, 0], (1 - gam ** (T - t)) / (1 - gam), rtol=1e-13)
    g = inputs.rng(5)
    r, _ = inputs.rewards_dones(g, 300, 4)
    d = np.zeros_like(r, dtype=np.uint8)
    G = orc.returns(r, d, gam)
    for s in range(4):
        ref = signal.lfilter([1.0], [1.0, -gam], r[::-1, s])[::-1]
        np.testing.assert_allclose(G[:, s], ref, rtol=1e-12)


def test_returns_done_cuts_bootstrap(orc):
    r = np.array([[1.0], [2.0], [4.0], [8.0]])
    d = np.array([[0], [1], [0], [0]], np.uint8)
    G = orc.returns(r, d, 0.5)
    # t=3: 8; t=2: 4 + 0.5*8 = 8; t=1 (done): 2; t=0: 1 + 0.5*2 = 2
    np.testing.assert_allclose(G[:, 0], [2.0, 2.0, 8.0, 8.0])


def test_landscape_energy_target_terminal(orc):
    """Energy-target terminal condition (App. C: an episode runs until the
    reaction's terminal state): done when the pure energy of the post-step
    state falls below the target, checked against the closed form of a single
    Gaussian well E(x) = -exp(-|x|^2 / 2) on the recorded positions."""
    g = inputs.rng(5)
    D = 2
    c, w, a = np.zeros((1, D)), np.ones(1), -np.ones(1)
    widths = [D, 8, 8, 2 * D]
    p = inputs.policy_params(g, widths)
    n, T = 40, 30
    x0 = g.uniform(-1.5, 1.5, (n, D))
    eobs0 = np.zeros(n)
    t0 = np.zeros(n, np.int32)
    kw = dict(seed=3, env_ids=np.arange(n), n_steps=T, episode_limit=25, noise_sigma=0.0,
              step_clip=0.1, x0=x0, eobs0=eobs0, t0=t0)
    target = -0.6
    r = orc.landscape_rollout(c, w, a, p, 8, 8, energy_target=target, **kw)
    n_target = 0
    for e in range(n):
        t = 0
        for s in range(T):
            y = r["obs"][s, e] + r["act"][s, e]
            E = -np.exp(-(y * y).sum() / 2)
            assert r["energy"][s, e] == pytest.approx(E, rel=1e-14)
            t += 1
            want = E < target or t >= 25
            assert r["done"][s, e] == want, (e, s)
            n_target += int(E < target)
            if want:
                t = 0
                if s + 1 < T:
                    np.testing.assert_array_equal(r["obs"][s + 1, e],
                                                  orc.landscape_reset_draw(3, s, e, D))
    assert 0 < n_target < n * T
    # +inf ends every episode after one step; -inf is the plain step limit
    r_all = orc.landscape_rollout(c, w, a, p, 8, 8, energy_target=np.inf, **kw)
    assert r_all["done"].all()
    r_off = orc.landscape_rollout(c, w, a, p, 8, 8, energy_target=-np.inf, **kw)
    r_none = orc.landscape_rollout(c, w, a, p, 8, 8, **kw)
    for f in ("obs", "act", "done", "energy", "reward"):
        np.testing.assert_array_equal(r_off[f], r_none[f])
    assert r_none["done"].sum() == n
