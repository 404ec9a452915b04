"""Pins of the acrobot oracle (App. C classic control, the Sutton & Barto
two-link acrobot): the equations of motion against a symbolic Euler-Lagrange
derivation from the links' kinetic and potential energy; the integrator's
fifth-order one-step error against a tight reference integration; the
equilibrium, wrap, clip, terminal height and reset draw; roll-out semantics."""
import numpy as np
import pytest

from paper_2408_00930_gb300 import inputs


def lagrangian_accels():
    """(th1'', th2'') as functions of (th1, th2, w1, w2, tau), derived here
    from L = T - V of two rigid links (masses m, lengths l, centres of mass at
    lc, inertias I about the centre of mass; angles from hanging down; the
    torque acts on the second joint)."""
    sp = pytest.importorskip("sympy")
    t = sp.symbols("t")
    tau = sp.symbols("tau")
    m1 = m2 = l1 = I1 = I2 = 1
    lc1 = lc2 = sp.Rational(1, 2)
    g = sp.Rational(98, 10)
    th1, th2 = sp.Function("th1")(t), sp.Function("th2")(t)
    x1, y1 = lc1 * sp.sin(th1), -lc1 * sp.cos(th1)
    x2 = l1 * sp.sin(th1) + lc2 * sp.sin(th1 + th2)
    y2 = -l1 * sp.cos(th1) - lc2 * sp.cos(th1 + th2)
    v2 = lambda x, y: sp.diff(x, t) ** 2 + sp.diff(y, t) ** 2
    T = (m1 * v2(x1, y1) / 2 + I1 * sp.diff(th1, t) ** 2 / 2 + m2 * v2(x2, y2) / 2 +
         I2 * sp.diff(th1 + th2, t) ** 2 / 2)
    V = m1 * g * y1 + m2 * g * y2
    L = T - V
    eqs = [sp.diff(sp.diff(L, sp.diff(q, t)), t) - sp.diff(L, q) - Q
           for q, Q in ((th1, 0), (th2, tau))]
    a1, a2 = sp.diff(th1, t, 2), sp.diff(th2, t, 2)
    sol = sp.solve(eqs, [a1, a2], dict=True)[0]
    q1, q2, w1, w2 = sp.symbols("q1 q2 w1 w2")
    rep = {sp.diff(th1, t): w1, sp.diff(th2, t): w2}
    exprs = []
    for a in (a1, a2):
        e = sol[a].subs(rep).subs({th1: q1, th2: q2})
        exprs.append(sp.lambdify((q1, q2, w1, w2, tau), e, "math"))
    return exprs


def test_dynamics_match_euler_lagrange(orc):
    f1, f2 = lagrangian_accels()
    g = inputs.rng(40)
    for _ in range(200):
        s = np.concatenate([g.uniform(-np.pi, np.pi, 2), g.uniform(-8, 8, 2)])
        for tau in (-1.0, 0.0, 1.0):
            ds = orc.acrobot_deriv(s, tau)
            assert ds[0] == s[2] and ds[1] == s[3]
            ref = np.array([f1(*s, tau), f2(*s, tau)])
            np.testing.assert_allclose(ds[2:], ref, rtol=1e-11, atol=1e-11)


def test_rk4_one_step_error_is_fifth_order(orc):
    """The local error of one step against a tight integration of the same
    equations shrinks ~32x per halving of dt: a fourth-order method."""
    integrate = pytest.importorskip("scipy.integrate")
    g = inputs.rng(41)
    for _ in range(5):
        s0 = np.concatenate([g.uniform(-1, 1, 2), g.uniform(-1, 1, 2)])
        a = int(g.integers(0, 3))

        def rhs(_t, y):
            return orc.acrobot_deriv(y, a - 1.0)

        errs = []
        for dt in (0.2, 0.1, 0.05):
            ref = integrate.solve_ivp(rhs, (0, dt), s0, method="DOP853", rtol=1e-13,
                                      atol=1e-13).y[:, -1]
            _, raw = orc.acrobot_step(s0, a, dt)
            errs.append(np.abs(raw - ref).max())
        r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
        assert 20 < r1 < 45 and 24 < r2 < 40, (errs, r1, r2)
        assert errs[0] < 5e-3


def test_equilibrium_wrap_clip_terminal_and_reset(orc):
    # hanging at rest without torque stays exactly at rest
    s, raw = orc.acrobot_step(np.zeros(4), 1, 0.2)
    assert np.all(s == 0) and np.all(raw == 0)
    # with torque the second joint turns, the first reacts the other way
    s, _ = orc.acrobot_step(np.zeros(4), 2, 0.2)
    assert s[3] > 0 and s[2] < 0
    # wrap into [-pi, pi] and velocity clip at 4 pi / 9 pi
    s, raw = orc.acrobot_step(np.array([3.1, -3.1, 12.0, -27.0]), 1, 0.2)
    for i in (0, 1):
        assert -np.pi <= s[i] <= np.pi
        k = (raw[i] - s[i]) / (2 * np.pi)
        assert abs(k - round(k)) < 1e-12
    assert abs(s[2]) <= 4 * np.pi + 1e-12 and abs(s[3]) <= 9 * np.pi + 1e-12
    s, raw = orc.acrobot_step(np.array([0.0, 0.0, 20.0, -40.0]), 1, 0.2)
    assert s[2] == pytest.approx(np.clip(raw[2], -4 * np.pi, 4 * np.pi), abs=0)
    assert s[3] == pytest.approx(np.clip(raw[3], -9 * np.pi, 9 * np.pi), abs=0)
    # tip height -cos th1 - cos(th1 + th2) > 1 (strict)
    assert orc.acrobot_terminal([np.pi, 0, 0, 0])[0]                      # straight up: 2
    assert not orc.acrobot_terminal([np.pi / 2, 0, 0, 0])[0]              # horizontal: 0
    assert not orc.acrobot_terminal([0, 0, 0, 0])[0]                      # hanging: -2
    t, mg = orc.acrobot_terminal([2 * np.pi / 3, 0, 0, 0])                # exactly 1
    assert mg < 1e-12
    assert orc.acrobot_terminal([2 * np.pi / 3 + 0.01, 0, 0, 0])[0]       # just above 1
    assert not orc.acrobot_terminal([np.pi / 2, np.pi / 2 - 0.01, 0, 0])[0]  # cos(0.01) < 1
    # observation
    o = orc.acrobot_obs([0.3, -1.2, 2.0, -3.0])
    np.testing.assert_array_equal(o, [np.cos(0.3), np.sin(0.3), np.cos(-1.2), np.sin(-1.2), 2.0,
                                      -3.0])
    # reset draw: four exact FP32 uniforms in [-0.1, 0.1) from RESET(k, env)
    w = orc.draw(9, 17, 3, 0, orc.TAG_RESET, 0)
    r = orc.acrobot_reset_draw(9, 17, 3)
    assert list(r) == [orc.uniform_f32(int(x), -0.1, 0.1) for x in w]


def test_acrobot_rollout_semantics(orc):
    g = inputs.rng(42)
    widths = [6, 16, 16, 3]
    p = inputs.policy_params(g, widths, scale=3.0)
    n, T, limit = 12, 80, 50
    r = orc.acrobot_rollout(p, 16, 16, seed=5, env_ids=np.arange(n), n_steps=T,
                            episode_limit=limit)
    for e in range(n):
        np.testing.assert_array_equal(r["state"][0, e], orc.acrobot_reset_draw(5, orc.STEP_INIT, e))
        t = 0
        for s in range(T):
            st = r["state"][s, e]
            np.testing.assert_array_equal(r["obs"][s, e], orc.acrobot_obs(st))
            out = orc.mlp_forward(widths, p, r["obs"][s, e])
            np.testing.assert_allclose(r["logits"][s, e], out, rtol=1e-15)
            nxt, _ = orc.acrobot_step(st, r["action"][s, e])
            term = orc.acrobot_terminal(nxt)[0]
            t += 1
            assert r["reward"][s, e] == (0.0 if term else -1.0)
            assert r["done"][s, e] == (term or t >= limit)
            if s + 1 < T:
                if r["done"][s, e]:
                    np.testing.assert_array_equal(r["state"][s + 1, e],
                                                  orc.acrobot_reset_draw(5, s, e))
                    t = 0
                else:
                    np.testing.assert_array_equal(r["state"][s + 1, e], nxt)
    assert set(np.unique(r["action"])) == {0, 1, 2}
    assert r["done"].sum() >= n
