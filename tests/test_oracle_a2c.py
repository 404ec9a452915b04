"""Pins of the oracle's actor-critic loss and gradients (A2C with Monte-Carlo
returns over recorded transitions): central finite differences of the loss,
PyTorch autograd (float64) on the same loss written with library ops, and the
special cases that must give zero gradient."""
import numpy as np
import pytest

from paper_2408_00930_gb300 import inputs


def setup(seed=0, R=40, od=4, h=8, na=3):
    g = inputs.rng(seed)
    actor = inputs.policy_params(g, [od, h, h, na], scale=2.0)
    critic = inputs.policy_params(g, [od, h, h, 1], scale=2.0)
    obs = g.normal(size=(R, od))
    act = g.integers(0, na, R).astype(np.int32)
    ret = g.normal(size=R) * 3
    return actor, critic, obs, act, ret, h, na


def total(st, c_v, c_e):
    return st[0] + c_v * st[1] - c_e * st[2]


@pytest.mark.parametrize("na", [2, 3])
def test_a2c_gradient_matches_finite_differences(orc, na):
    actor, critic, obs, act, ret, h, _ = setup(na=na)
    c_v, c_e = 0.5, 0.01
    st, ga, gc = orc.a2c(actor, critic, obs, act, ret, h, h, na, c_v=c_v, c_e=c_e)
    # the actor's advantage is a constant of its loss: hold it while perturbing
    V = np.array([orc.mlp_forward([obs.shape[1], h, h, 1], critic, o)[0] for o in obs])
    adv = ret - V
    g = np.random.default_rng(1)
    for idx in g.choice(len(actor), 25, replace=False):
        up, dn = actor.copy(), actor.copy()
        up[idx] += np.float32(2.0 ** -16)
        dn[idx] -= np.float32(2.0 ** -16)
        lu = total(orc.a2c(up, critic, obs, act, ret, h, h, na, c_v, c_e, adv=adv, grads=False)[0],
                   0.0, c_e)
        ld = total(orc.a2c(dn, critic, obs, act, ret, h, h, na, c_v, c_e, adv=adv, grads=False)[0],
                   0.0, c_e)
        fd = (lu - ld) / (float(up[idx]) - float(dn[idx]))
        assert fd == pytest.approx(ga[idx], rel=2e-6, abs=1e-10), idx
    for idx in g.choice(len(critic), 25, replace=False):
        up, dn = critic.copy(), critic.copy()
        up[idx] += np.float32(2.0 ** -16)
        dn[idx] -= np.float32(2.0 ** -16)
        lu = orc.a2c(actor, up, obs, act, ret, h, h, na, c_v, c_e, grads=False)[0][1] * c_v
        ld = orc.a2c(actor, dn, obs, act, ret, h, h, na, c_v, c_e, grads=False)[0][1] * c_v
        fd = (lu - ld) / (float(up[idx]) - float(dn[idx]))
        assert fd == pytest.approx(gc[idx], rel=2e-6, abs=1e-10), idx


def test_a2c_matches_torch_autograd(orc):
    torch = pytest.importorskip("torch")
    actor, critic, obs, act, ret, h, na = setup(seed=3, R=64, na=3)
    c_v, c_e = 0.25, 0.05
    st, ga, gc = orc.a2c(actor, critic, obs, act, ret, h, h, na, c_v=c_v, c_e=c_e)
    od = obs.shape[1]

    def layers(p, w):
        out, off = [], 0
        for a, b in zip(w[:-1], w[1:]):
            W = torch.tensor(p[off:off + a * b].reshape(a, b), dtype=torch.float64,
                             requires_grad=True)
            bb = torch.tensor(p[off + a * b:off + a * b + b], dtype=torch.float64,
                              requires_grad=True)
            out += [W, bb]
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
    logits, v = mlp(pa, x), mlp(pc, x)[:, 0]
    G = torch.tensor(ret)
    logp = torch.log_softmax(logits, 1)
    ent = -(logp.exp() * logp).sum(1)
    A = (G - v).detach()
    lp_a = logp.gather(1, torch.tensor(act, dtype=torch.int64)[:, None])[:, 0]
    loss = (-A * lp_a).mean() + c_v * ((G - v) ** 2).mean() - c_e * ent.mean()
    loss.backward()
    ref_a = np.concatenate([t.grad.numpy().ravel() for t in pa])
    ref_c = np.concatenate([t.grad.numpy().ravel() for t in pc])
    np.testing.assert_allclose(ga, ref_a, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(gc, ref_c, rtol=1e-9, atol=1e-12)
    assert st[0] == pytest.approx(float((-A * lp_a).mean().detach()), rel=1e-12)
    assert st[1] == pytest.approx(float(((G - v) ** 2).mean().detach()), rel=1e-12)
    assert st[2] == pytest.approx(float(ent.mean().detach()), rel=1e-12)


def test_a2c_zero_gradient_cases(orc):
    actor, critic, obs, act, ret, h, na = setup(seed=5)
    V = np.array([orc.mlp_forward([obs.shape[1], h, h, 1], critic, o)[0] for o in obs])
    # returns equal to the critic's values: no advantage and no value error
    st, ga, gc = orc.a2c(actor, critic, obs, act, V, h, h, na, c_v=0.5, c_e=0.0)
    assert np.abs(ga).max() < 1e-15 and np.abs(gc).max() < 1e-15 and st[1] < 1e-30
    # c_v = 0: the critic gets no gradient whatever the returns
    _, _, gc = orc.a2c(actor, critic, obs, act, ret, h, h, na, c_v=0.0)
    assert np.all(gc == 0)


def test_a2c_gauss_matches_torch_autograd(orc):
    """Gaussian head: the loss written with torch.distributions at the sample
    x = mean + sigma z (the clamp of log sigma included), autograd float64."""
    torch = pytest.importorskip("torch")
    g = inputs.rng(7)
    D, h, R = 3, 8, 50
    actor = inputs.policy_params(g, [D, h, h, 2 * D], scale=3.0)
    critic = inputs.policy_params(g, [D, h, h, 1], scale=2.0)
    obs, z, ret = g.normal(size=(R, D)), g.normal(size=(R, D)), g.normal(size=R)
    c_v, c_e = 0.3, 0.02
    st, ga, gc = orc.a2c_gauss(actor, critic, obs, z, ret, h, h, c_v=c_v, c_e=c_e)

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
    mu, ls = out[:, :D], torch.clamp(out[:, D:], -5.0, 2.0)
    sample = (mu + ls.exp() * torch.tensor(z)).detach()     # the recorded sample
    dist = torch.distributions.Normal(mu, ls.exp())
    logp = dist.log_prob(sample).sum(1)
    ent = dist.entropy().sum(1)
    G = torch.tensor(ret)
    A = (G - v).detach()
    loss = (-A * logp).mean() + c_v * ((G - v) ** 2).mean() - c_e * ent.mean()
    loss.backward()
    ref_a = np.concatenate([t.grad.numpy().ravel() for t in pa])
    ref_c = np.concatenate([t.grad.numpy().ravel() for t in pc])
    np.testing.assert_allclose(ga, ref_a, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(gc, ref_c, rtol=1e-9, atol=1e-12)
    assert st[0] == pytest.approx(float((-A * logp).mean().detach()), rel=1e-12)
    assert st[2] == pytest.approx(float(ent.mean().detach()), rel=1e-12)
    # the clamp really binds somewhere in this draw
    raw = out[:, D:].detach().numpy()
    assert ((raw < -5) | (raw > 2)).any()
