"""Pins of the oracle's differentiation (no counterpart in the paper): the
vector-Jacobian product of the force and the gradient of a fixed shared-step
Hermite trajectory.

The force VJP is checked against central differences of the oracle force
(itself pinned to derivatives of the potential) and against translation
invariance; the trajectory gradient against central differences of the
trajectory and against the closed-form response to a translation of all
positions and a boost of all velocities.
"""
import numpy as np
import pytest

from synth import plummer


def _system(n, seed):
    r = np.random.default_rng(seed)
    m = r.uniform(0.2, 1.0, n)
    m /= m.sum()
    x = r.normal(0, 0.5, (n, 3))
    v = r.normal(0, 0.5, (n, 3))
    return m, x, v


@pytest.mark.parametrize("n,eps", [(2, 0.1), (5, 0.05), (8, 0.0)])
def test_force_vjp_matches_central_differences(orc, n, eps):
    m, x, v = _system(n, 10 + n)
    r = np.random.default_rng(1)
    abar, kbar = r.normal(size=(n, 3)), r.normal(size=(n, 3))
    xb, vb, mb = orc.force_vjp(m, x, v, eps, abar, kbar)

    def f(mm, xx, vv):
        a, k, _ = orc.force(mm, xx, vv, eps)
        return np.sum(abar * a) + np.sum(kbar * k)

    h = 1e-6
    for trial in range(4):
        dx, dv, dm = r.normal(size=(n, 3)), r.normal(size=(n, 3)), r.normal(size=n)
        fd = (f(m + h * dm, x + h * dx, v + h * dv) - f(m - h * dm, x - h * dx, v - h * dv)) / (2 * h)
        an = np.sum(xb * dx) + np.sum(vb * dv) + np.sum(mb * dm)
        assert an == pytest.approx(fd, rel=1e-7, abs=1e-7 * (abs(fd) + 1.0))
    # single coordinates
    for (i, c) in [(0, 0), (n - 1, 2)]:
        e = np.zeros((n, 3))
        e[i, c] = 1.0
        fd = (f(m, x + h * e, v) - f(m, x - h * e, v)) / (2 * h)
        assert xb[i, c] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_force_vjp_translation_invariance(orc):
    # Forces depend on differences only, so the VJP sums to zero over particles.
    m, x, v = plummer(200, 3)
    r = np.random.default_rng(2)
    xb, vb, mb = orc.force_vjp(m, x, v, 1 / 256, r.normal(size=(200, 3)), r.normal(size=(200, 3)))
    assert np.abs(xb.sum(0)).max() < 1e-10 * np.abs(xb).sum()
    assert np.abs(vb.sum(0)).max() < 1e-10 * np.abs(vb).sum()


@pytest.mark.parametrize("n,steps,dt,eps", [(3, 6, 1 / 32, 0.1), (6, 10, 1 / 64, 0.05)])
def test_trajectory_gradient_matches_central_differences(orc, n, steps, dt, eps):
    m, x, v = _system(n, 20 + n)
    tgt = np.random.default_rng(3).normal(0, 0.5, (n, 3))

    def loss(mm, xx, vv):
        xt, _ = orc.traj_final(mm, xx, vv, eps, dt, steps)
        return np.sum((xt - tgt) ** 2)

    xt, vt = orc.traj_final(m, x, v, eps, dt, steps)
    _, _, xb, vb, mb = orc.traj_vjp(m, x, v, eps, dt, steps, 2 * (xt - tgt), np.zeros((n, 3)))
    r = np.random.default_rng(4)
    h = 1e-6
    for trial in range(4):
        dx, dv, dm = r.normal(size=(n, 3)), r.normal(size=(n, 3)), r.normal(size=n) * 0.01
        fd = (loss(m + h * dm, x + h * dx, v + h * dv) - loss(m - h * dm, x - h * dx, v - h * dv)) / (2 * h)
        an = np.sum(xb * dx) + np.sum(vb * dv) + np.sum(mb * dm)
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_trajectory_gradient_translation_and_boost(orc):
    # Shifting every x0 by c shifts x_T by c (v_T unchanged); boosting every v0
    # by u adds u T to x_T and u to v_T.  Hence, for any cotangents,
    # sum_k xbar_0 = sum_k xbar_T and sum_k vbar_0 = T sum_k xbar_T + sum_k vbar_T.
    n, steps, dt = 40, 12, 1 / 128
    m, x, v = plummer(n, 5)
    r = np.random.default_rng(6)
    xbT, vbT = r.normal(size=(n, 3)), r.normal(size=(n, 3))
    _, _, xb, vb, _ = orc.traj_vjp(m, x, v, 1 / 64, dt, steps, xbT, vbT)
    T = steps * dt
    assert np.allclose(xb.sum(0), xbT.sum(0), rtol=1e-9, atol=1e-9)
    assert np.allclose(vb.sum(0), T * xbT.sum(0) + vbT.sum(0), rtol=1e-9, atol=1e-9)


def test_trajectory_forward_equals_shared_step_integrator(orc):
    # The trajectory's forward pass is the integrator with every particle on
    # the shared step 2^-k.
    m, x, v = plummer(50, 7)
    xt, vt = orc.traj_final(m, x, v, 1 / 256, 2.0 ** -10, 16)
    it = orc.Integrator(m, x, v, 1 / 256, kfix=10)
    for _ in range(16):
        it.step()
    assert np.array_equal(xt, it.x) and np.array_equal(vt, it.v)


@pytest.mark.parametrize("dt,steps", [(1 / 8, 4), (1 / 16, 6)])
def test_trajectory_vjp_large_steps_general_cotangents(orc, dt, steps):
    # Large steps make every dt^2 and dt^3 term of the corrector and predictor
    # transposes visible; random cotangents on both x_T and v_T exercise all of
    # them.  f = <xbar_T, x_T> + <vbar_T, v_T>; its directional derivatives by
    # central differences must match the VJP to 1e-7.
    n, eps = 5, 0.2
    m, x, v = _system(n, 40)
    r = np.random.default_rng(41)
    xbT, vbT = r.normal(size=(n, 3)), r.normal(size=(n, 3))

    def f(mm, xx, vv):
        xt, vt = orc.traj_final(mm, xx, vv, eps, dt, steps)
        return np.sum(xbT * xt) + np.sum(vbT * vt)

    _, _, xb, vb, mb = orc.traj_vjp(m, x, v, eps, dt, steps, xbT, vbT)
    h = 1e-5
    for trial in range(6):
        dx, dv, dm = r.normal(size=(n, 3)), r.normal(size=(n, 3)), r.normal(size=n) * 0.01
        fd = (f(m + h * dm, x + h * dx, v + h * dv) - f(m - h * dm, x - h * dx, v - h * dv)) / (2 * h)
        an = np.sum(xb * dx) + np.sum(vb * dv) + np.sum(mb * dm)
        assert an == pytest.approx(fd, rel=1e-7, abs=1e-9)
