"""Pins of the control environment, the policy MLP and the categorical sampler."""
import os

import numpy as np
import pytest

from paper_2408_00930_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _hand_steps():
    rows = []
    for ln in open(os.path.join(GOLDEN, "control_hand_steps.txt")):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        lhs, rhs = ln.split("|")
        a = [float(v) for v in lhs.split()]
        rows.append((np.array(a[:4]), int(a[4]), np.array([float(v) for v in rhs.split()])))
    return rows


def test_control_hand_steps(orc):
    for s, a, ref in _hand_steps():
        got = orc.control_dynamics(s, a)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9)


def test_control_done_thresholds(orc):
    assert orc.control_done([2.41, 0, 0, 0], 1, 200)[0]
    assert orc.control_done([-2.41, 0, 0, 0], 1, 200)[0]
    assert not orc.control_done([2.4, 0, 0, 0], 1, 200)[0]      # strict
    assert orc.control_done([0, 0, 0.2101, 0], 1, 200)[0]
    assert not orc.control_done([0, 0, -0.21, 0], 1, 200)[0]
    assert orc.control_done([0, 0, 0, 0], 200, 200)[0]
    assert not orc.control_done([0, 0, 0, 0], 199, 200)[0]


def test_control_reset_draw_in_range_and_keyed(orc):
    s = orc.control_reset_draw(7, 12, 3)
    assert np.all(np.abs(s) <= 0.05)
    w = orc.draw(7, 12, 3, 0, orc.TAG_RESET, 0)
    for d in range(4):
        assert s[d] == orc.uniform_f32(int(w[d]), -0.05, 0.05)
    assert not np.array_equal(s, orc.control_reset_draw(7, 13, 3))
    assert not np.array_equal(s, orc.control_reset_draw(8, 12, 3))


def test_mlp_matches_torch_functional(orc):
    torch = pytest.importorskip("torch")
    g = inputs.rng(0)
    for widths in ([4, 64, 64, 2], [16, 128, 128, 20], [24, 32, 16, 48], [3, 5, 1]):
        p = inputs.policy_params(g, widths)
        x = g.standard_normal((5, widths[0]))
        got = orc.mlp_forward(widths, p, x)
        a = torch.from_numpy(x)
        off = 0
        pt = torch.from_numpy(p.astype(np.float64))
        for l, (ni, no) in enumerate(zip(widths[:-1], widths[1:])):
            W = pt[off:off + ni * no].reshape(ni, no)
            b = pt[off + ni * no: off + ni * no + no]
            off += ni * no + no
            a = torch.nn.functional.linear(a, W.T, b)
            if l < len(widths) - 2:
                a = torch.tanh(a)
        np.testing.assert_allclose(got, a.numpy(), rtol=1e-13, atol=1e-13)


def test_mlp_bf16_layers_match_torch_bf16_rounding(orc):
    torch = pytest.importorskip("torch")
    g = inputs.rng(1)
    widths = [4, 32, 32, 2]
    p = inputs.policy_params(g, widths)
    x = g.standard_normal((3, 4))
    got = orc.mlp_forward(widths, p, x, bf16_layers=0b010)
    pt = torch.from_numpy(p)
    W1 = pt[:128].reshape(4, 32).double(); b1 = pt[128:160].double()
    W2 = pt[160:160 + 1024].reshape(32, 32); b2 = pt[1184:1216].double()
    W3 = pt[1216:1280].reshape(32, 2).double(); b3 = pt[1280:1282].double()
    h1 = torch.tanh(torch.from_numpy(x) @ W1 + b1)
    h1b = h1.float().to(torch.bfloat16).double()
    h2 = torch.tanh(h1b @ W2.to(torch.bfloat16).double() + b2)
    ref = h2 @ W3 + b3
    np.testing.assert_allclose(got, ref.numpy(), rtol=1e-12, atol=1e-12)


def test_policy_init_bounds_and_distribution(orc):
    widths = [4, 256, 256, 2]
    p = orc.policy_init(42, 0, widths)
    assert p.dtype == np.float32 and p.size == orc.policy_param_count(widths)
    off = 0
    stats = pytest.importorskip("scipy.stats")
    for ni, no in zip(widths[:-1], widths[1:]):
        n = ni * no + no
        b = np.float32(1.0) / np.sqrt(np.float32(ni))
        seg = p[off:off + n]
        assert np.all(np.abs(seg) <= b)
        if n > 1000:
            assert stats.kstest(seg, "uniform", args=(-b, 2 * b)).pvalue > 1e-4
        off += n
    q = orc.policy_init(42, 1, widths)
    assert not np.array_equal(p, q)   # policy id keys the stream


def test_sampler_two_class_closed_form(orc):
    """Two classes: action 1 iff u >= 1 - sigmoid(l1 - l0); logp = log-sigmoid."""
    g = np.random.default_rng(2)
    for _ in range(500):
        l = g.normal(0, 2, 2)
        u = g.random()
        a, lp, mg = orc.sample_categorical(l, u)
        p0 = 1.0 / (1.0 + np.exp(l[1] - l[0]))
        assert a == (0 if u < p0 else 1)
        assert lp == pytest.approx(np.log(p0 if a == 0 else 1 - p0), rel=1e-12, abs=1e-12)
        assert mg == pytest.approx(abs(u - p0), abs=1e-15)


def test_sampler_frequencies_chi2(orc):
    special = pytest.importorskip("scipy.special")
    stats = pytest.importorskip("scipy.stats")
    g = np.random.default_rng(3)
    logits = g.normal(0, 1, 20)
    p = special.softmax(logits)
    n = 100_000
    us = g.random(n)
    counts = np.bincount([orc.sample_categorical(logits, u)[0] for u in us], minlength=20)
    assert stats.chisquare(counts, p * n).pvalue > 1e-4
    lsm = special.log_softmax(logits)
    for i, u in enumerate(us[:200]):
        a, lp, _ = orc.sample_categorical(logits, u)
        assert lp == pytest.approx(lsm[a], rel=1e-12, abs=1e-12)


def test_sampler_edges(orc):
    assert orc.sample_categorical([0.0, 0.0], 0.0)[0] == 0
    assert orc.sample_categorical([0.0, 0.0], 0.5)[0] == 1        # u < CDF is strict
    assert orc.sample_categorical([0.0, 0.0], 0.4999999)[0] == 0
    assert orc.sample_categorical([-1e4, 0.0, -1e4], 0.999999)[0] == 1
    assert orc.sample_categorical([50.0, -50.0], 0.9999999)[0] == 0


def test_control_rollout_semantics(orc):
    widths = [4, 64, 64, 2]
    p = orc.policy_init(1, 0, widths)
    T, ids = 200, np.arange(40)
    r = orc.control_rollout(p, 64, 64, seed=5, env_ids=ids, n_steps=T, episode_limit=200)
    assert np.all(r["reward"] == 1.0)
    assert r["done"].sum() > 40          # episodes end well before the limit
    for e in range(len(ids)):
        # initial observation is the full-reset draw
        np.testing.assert_array_equal(r["obs"][0, e], orc.control_reset_draw(5, orc.STEP_INIT, e))
        for t in range(T - 1):
            if r["done"][t, e]:
                np.testing.assert_array_equal(r["obs"][t + 1, e], orc.control_reset_draw(5, t, e))
            else:
                nxt = orc.control_dynamics(r["obs"][t, e], r["action"][t, e])
                np.testing.assert_array_equal(r["obs"][t + 1, e], nxt)
                assert not orc.control_done(nxt, 1, 10**9)[0]
    # chunking: 120 + 80 steps from the saved state equals 200 steps
    a = orc.control_rollout(p, 64, 64, seed=5, env_ids=ids, n_steps=120, episode_limit=200)
    b = orc.control_rollout(p, 64, 64, seed=5, env_ids=ids, n_steps=80, episode_limit=200,
                            k0=120, state0=a["state"], t0=a["t"])
    np.testing.assert_array_equal(b["action"], r["action"][120:])
    np.testing.assert_array_equal(b["obs"], r["obs"][120:])


def test_control_episode_limit_forces_done(orc):
    widths = [4, 8, 8, 2]
    p = np.zeros(orc.policy_param_count(widths), np.float32)
    # zero policy -> 50/50 pushes; start at rest with t = limit - 1
    r = orc.control_rollout(p, 8, 8, seed=1, env_ids=[0, 1], n_steps=1, episode_limit=10,
                            state0=np.zeros((2, 4)), t0=[9, 3])
    assert list(r["done"][0]) == [1, 0]
    assert r["t"][0] == 0 and r["t"][1] == 4
