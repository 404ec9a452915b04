"""Pins of the oracle's PPO clipped-surrogate loss and gradients: central
finite differences of the loss with rows in all three regimes of the clip
(below, inside and above [1 - eps, 1 + eps]), PyTorch autograd (float64) on the
loss written with torch.minimum / torch.clamp, the reduction to the actor-critic
gradient when the behaviour policy is the current one and eps is unbounded,
and the fully clipped case, where the surrogate passes no gradient; for the
categorical head and for the diagonal Gaussian head (behaviour samples scored
under the current mean and sigma, the clamp of log sigma binding on some
outputs; on policy it reduces to the Gaussian actor-critic gradient)."""
import numpy as np
import pytest

from paper_2408_00930_gb300 import inputs


def setup(seed=0, R=48, od=4, h=8, na=3, spread=0.6):
    g = inputs.rng(seed)
    actor = inputs.policy_params(g, [od, h, h, na], scale=2.0)
    critic = inputs.policy_params(g, [od, h, h, 1], scale=2.0)
    obs = g.normal(size=(R, od))
    act = g.integers(0, na, R).astype(np.int32)
    ret = g.normal(size=R) * 3
    adv = g.normal(size=R) * 2
    lp = log_pi(actor, obs, act, od, h, na)
    logp_old = lp + g.uniform(-spread, spread, R)
    return actor, critic, obs, act, ret, adv, logp_old, h, na


def log_pi(actor, obs, act, od, h, na):
    """log pi(a | s) of each row from the actor's logits (numpy log-softmax)."""
    from oracle import mlp_forward
    out = []
    for o, a in zip(obs, act):
        lg = np.asarray(mlp_forward([od, h, h, na], actor, o), np.float64)
        m = lg.max()
        out.append(lg[a] - m - np.log(np.exp(lg - m).sum()))
    return np.array(out)


def total(st, c_v, c_e):
    return st[0] + c_v * st[1] - c_e * st[2]


def test_ppo_gradient_matches_finite_differences(orc):
    eps, c_v, c_e = 0.2, 0.5, 0.01
    actor, critic, obs, act, ret, adv, logp_old, h, na = setup()
    od = obs.shape[1]
    rho = np.exp(log_pi(actor, obs, act, od, h, na) - logp_old)
    # rows in every regime, none within the reach of the difference step of a kink
    assert (rho < 1 - eps).sum() >= 5 and (rho > 1 + eps).sum() >= 5
    assert (np.abs(rho - 1) < eps).sum() >= 5
    assert np.abs(np.abs(rho - 1) - eps).min() > 1e-3
    st, ga, gc = orc.ppo(actor, critic, obs, act, ret, adv, logp_old, h, h, na, eps, c_v, c_e)
    assert st[3] == pytest.approx(np.mean(np.abs(rho - 1) > eps), abs=0)
    g = np.random.default_rng(2)
    for idx in g.choice(len(actor), 30, replace=False):
        up, dn = actor.copy(), actor.copy()
        up[idx] += np.float32(2.0 ** -16)
        dn[idx] -= np.float32(2.0 ** -16)
        lu = total(orc.ppo(up, critic, obs, act, ret, adv, logp_old, h, h, na, eps, c_v, c_e,
                           grads=False)[0], 0.0, c_e)
        ld = total(orc.ppo(dn, critic, obs, act, ret, adv, logp_old, h, h, na, eps, c_v, c_e,
                           grads=False)[0], 0.0, c_e)
        fd = (lu - ld) / (float(up[idx]) - float(dn[idx]))
        assert fd == pytest.approx(ga[idx], rel=2e-6, abs=1e-10), idx
    for idx in g.choice(len(critic), 20, replace=False):
        up, dn = critic.copy(), critic.copy()
        up[idx] += np.float32(2.0 ** -16)
        dn[idx] -= np.float32(2.0 ** -16)
        lu = orc.ppo(actor, up, obs, act, ret, adv, logp_old, h, h, na, eps, c_v, c_e,
                     grads=False)[0][1] * c_v
        ld = orc.ppo(actor, dn, obs, act, ret, adv, logp_old, h, h, na, eps, c_v, c_e,
                     grads=False)[0][1] * c_v
        fd = (lu - ld) / (float(up[idx]) - float(dn[idx]))
        assert fd == pytest.approx(gc[idx], rel=2e-6, abs=1e-10), idx


def test_ppo_matches_torch_autograd(orc):
    torch = pytest.importorskip("torch")
    eps, c_v, c_e = 0.15, 0.3, 0.05
    actor, critic, obs, act, ret, adv, logp_old, h, na = setup(seed=4, R=64, na=4)
    od = obs.shape[1]
    st, ga, gc = orc.ppo(actor, critic, obs, act, ret, adv, logp_old, h, h, na, eps, c_v, c_e)

    def layers(p, w):
        out, off = [], 0
        for a, b in zip(w[:-1], w[1:]):
            out.append(torch.tensor(p[off:off + a * b].reshape(a, b), dtype=torch.float64,
                                    requires_grad=True))
            out.append(torch.tensor(p[off + a * b:off + a * b + b], dtype=torch.float64,
                                    requires_grad=True))
            off += a * b + b
        return out

    def mlp(ps, x):
        for i in range(3):
            x = x @ ps[2 * i] + ps[2 * i + 1]
            if i < 2:
                x = torch.tanh(x)
        return x

    pa, pc = layers(actor, [od, h, h, na]), layers(critic, [od, h, h, 1])
    x = torch.tensor(obs)
    logp = torch.log_softmax(mlp(pa, x), 1)
    v = mlp(pc, x)[:, 0]
    A, G, lpo = torch.tensor(adv), torch.tensor(ret), torch.tensor(logp_old)
    lp_a = logp.gather(1, torch.tensor(act, dtype=torch.int64)[:, None])[:, 0]
    rho = torch.exp(lp_a - lpo)
    surr = torch.minimum(rho * A, torch.clamp(rho, 1 - eps, 1 + eps) * A)
    ent = -(logp.exp() * logp).sum(1)
    loss = -surr.mean() + c_v * ((G - v) ** 2).mean() - c_e * ent.mean()
    loss.backward()
    ref_a = np.concatenate([t.grad.numpy().ravel() for t in pa])
    ref_c = np.concatenate([t.grad.numpy().ravel() for t in pc])
    np.testing.assert_allclose(ga, ref_a, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(gc, ref_c, rtol=1e-9, atol=1e-12)
    assert st[0] == pytest.approx(float(-surr.mean().detach()), rel=1e-12)
    assert st[1] == pytest.approx(float(((G - v) ** 2).mean().detach()), rel=1e-12)
    assert st[2] == pytest.approx(float(ent.mean().detach()), rel=1e-12)
    frac = float((torch.abs(rho - 1) > eps).double().mean())
    assert 0 < frac < 1 and st[3] == frac


def test_ppo_reduces_to_actor_critic_on_policy(orc):
    """Behaviour policy = the current one (rho = 1) and eps unbounded: the
    surrogate's gradient is the policy gradient -A grad log pi of or_a2c."""
    actor, critic, obs, act, ret, adv, _, h, na = setup(seed=7)
    od = obs.shape[1]
    lp = log_pi(actor, obs, act, od, h, na)
    st, ga, gc = orc.ppo(actor, critic, obs, act, ret, adv, lp, h, h, na, 1e9, 0.5, 0.02)
    st2, ga2, gc2 = orc.a2c(actor, critic, obs, act, ret, h, h, na, c_v=0.5, c_e=0.02, adv=adv)
    np.testing.assert_allclose(ga, ga2, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(gc, gc2, rtol=1e-12, atol=1e-15)
    assert st[0] == pytest.approx(-adv.mean(), rel=1e-12)     # -rho A with rho = 1
    assert st[1:3] == pytest.approx(st2[1:3], rel=1e-12) and st[3] == 0


def test_ppo_fully_clipped_passes_no_policy_gradient(orc):
    """Every row on the held side of the clip (rho > 1 + eps where A > 0, rho <
    1 - eps where A < 0): without the entropy term the actor gets no gradient;
    the surrogate is (1 +- eps) A per row."""
    eps = 0.1
    actor, critic, obs, act, ret, adv, _, h, na = setup(seed=9)
    od = obs.shape[1]
    lp = log_pi(actor, obs, act, od, h, na)
    logp_old = lp - np.sign(adv) * 0.5           # rho = e^{+-0.5}: outside on the held side
    st, ga, gc = orc.ppo(actor, critic, obs, act, ret, adv, logp_old, h, h, na, eps, 0.5, 0.0)
    assert np.all(ga == 0) and st[3] == 1.0
    assert st[0] == pytest.approx(-np.mean((1 + np.sign(adv) * eps) * adv), rel=1e-12)
    # the other side (rho pulled towards the inside of the range by the sign of A) keeps it
    st, ga, _ = orc.ppo(actor, critic, obs, act, ret, adv, lp + np.sign(adv) * 0.5, h, h, na, eps,
                        0.5, 0.0)
    assert np.abs(ga).max() > 1e-3 and st[3] == 1.0


def gauss_setup(seed=0, R=48, D=3, h=8, spread=0.6):
    """Gaussian head: samples u = mean + sigma z of the actor itself, the
    behaviour log-densities moved by up to +-spread (rows in all clip regimes);
    the actor's scale makes the clamp of log sigma bind on some outputs."""
    from oracle import mlp_forward
    g = inputs.rng(seed)
    actor = inputs.policy_params(g, [D, h, h, 2 * D], scale=3.0)
    critic = inputs.policy_params(g, [D, h, h, 1], scale=2.0)
    obs, z = g.normal(size=(R, D)), g.normal(size=(R, D))
    out = np.asarray(mlp_forward([D, h, h, 2 * D], actor, obs))
    ls = np.clip(out[:, D:], -5.0, 2.0)
    u = out[:, :D] + np.exp(ls) * z
    lp = (-0.5 * z * z - ls - 0.5 * np.log(2 * np.pi)).sum(1)
    ret, adv = g.normal(size=R) * 3, g.normal(size=R) * 2
    return actor, critic, obs, z, u, lp, lp + g.uniform(-spread, spread, R), ret, adv, h, out


def test_ppo_gauss_gradient_matches_finite_differences(orc):
    eps, c_v, c_e = 0.2, 0.5, 0.01
    actor, critic, obs, _, u, lp, lpo, ret, adv, h, out = gauss_setup()
    D = obs.shape[1]
    rho = np.exp(lp - lpo)
    assert (rho < 1 - eps).sum() >= 5 and (rho > 1 + eps).sum() >= 5
    assert (np.abs(rho - 1) < eps).sum() >= 5
    assert np.abs(np.abs(rho - 1) - eps).min() > 1e-3
    raw = out[:, D:]
    assert (raw < -5).any() or (raw > 2).any()          # the clamp binds somewhere
    st, ga, gc = orc.ppo_gauss(actor, critic, obs, u, ret, adv, lpo, h, h, eps, c_v, c_e)
    assert st[3] == pytest.approx(np.mean(np.abs(rho - 1) > eps), abs=0)
    g = np.random.default_rng(3)
    for idx in g.choice(len(actor), 30, replace=False):
        up, dn = actor.copy(), actor.copy()
        up[idx] += np.float32(2.0 ** -16)
        dn[idx] -= np.float32(2.0 ** -16)
        lu = total(orc.ppo_gauss(up, critic, obs, u, ret, adv, lpo, h, h, eps, c_v, c_e,
                                 grads=False)[0], 0.0, c_e)
        ld = total(orc.ppo_gauss(dn, critic, obs, u, ret, adv, lpo, h, h, eps, c_v, c_e,
                                 grads=False)[0], 0.0, c_e)
        fd = (lu - ld) / (float(up[idx]) - float(dn[idx]))
        assert fd == pytest.approx(ga[idx], rel=2e-6, abs=1e-10), idx


def test_ppo_gauss_matches_torch_autograd(orc):
    torch = pytest.importorskip("torch")
    eps, c_v, c_e = 0.15, 0.3, 0.02
    actor, critic, obs, _, u, _, lpo, ret, adv, h, _ = gauss_setup(seed=5, R=64, D=4)
    D = obs.shape[1]
    st, ga, gc = orc.ppo_gauss(actor, critic, obs, u, ret, adv, lpo, h, h, eps, c_v, c_e)

    def layers(p, w):
        out, off = [], 0
        for a, b in zip(w[:-1], w[1:]):
            out.append(torch.tensor(p[off:off + a * b].reshape(a, b), dtype=torch.float64,
                                    requires_grad=True))
            out.append(torch.tensor(p[off + a * b:off + a * b + b], dtype=torch.float64,
                                    requires_grad=True))
            off += a * b + b
        return out

    def mlp(ps, x):
        for i in range(3):
            x = x @ ps[2 * i] + ps[2 * i + 1]
            if i < 2:
                x = torch.tanh(x)
        return x

    pa, pc = layers(actor, [D, h, h, 2 * D]), layers(critic, [D, h, h, 1])
    x = torch.tensor(obs)
    out, v = mlp(pa, x), mlp(pc, x)[:, 0]
    mean, ls = out[:, :D], torch.clamp(out[:, D:], -5.0, 2.0)
    dist = torch.distributions.Normal(mean, torch.exp(ls))
    logp = dist.log_prob(torch.tensor(u)).sum(1)
    A, G = torch.tensor(adv), torch.tensor(ret)
    rho = torch.exp(logp - torch.tensor(lpo))
    surr = torch.minimum(rho * A, torch.clamp(rho, 1 - eps, 1 + eps) * A)
    ent = dist.entropy().sum(1)
    loss = -surr.mean() + c_v * ((G - v) ** 2).mean() - c_e * ent.mean()
    loss.backward()
    ref_a = np.concatenate([t.grad.numpy().ravel() for t in pa])
    ref_c = np.concatenate([t.grad.numpy().ravel() for t in pc])
    np.testing.assert_allclose(ga, ref_a, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(gc, ref_c, rtol=1e-9, atol=1e-12)
    assert st[0] == pytest.approx(float(-surr.mean().detach()), rel=1e-12)
    assert st[2] == pytest.approx(float(ent.mean().detach()), rel=1e-12)
    assert 0 < st[3] < 1


def test_ppo_gauss_reduces_to_actor_critic_on_policy(orc):
    """u = mean + sigma z of the current actor, logp_old its own density and
    eps unbounded: the gradient of or_a2c_gauss with the same normals z."""
    actor, critic, obs, z, u, lp, _, ret, adv, h, _ = gauss_setup(seed=8)
    st, ga, gc = orc.ppo_gauss(actor, critic, obs, u, ret, adv, lp, h, h, 1e9, 0.5, 0.02)
    st2, ga2, gc2 = orc.a2c_gauss(actor, critic, obs, z, ret, h, h, c_v=0.5, c_e=0.02, adv=adv)
    np.testing.assert_allclose(ga, ga2, rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(gc, gc2, rtol=1e-12, atol=1e-15)
    assert st[1:3] == pytest.approx(st2[1:3], rel=1e-12) and st[3] == 0
