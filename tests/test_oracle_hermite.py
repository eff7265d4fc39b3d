"""Pins of the oracle's Hermite integrator and block time steps (Section 2).

Polynomial trajectories fix the predictor (exact for cubic motion) and the
corrector (exact for quintic motion, since it interpolates a cubic
acceleration); a circular orbit fixes the time-step criterion in closed form;
the Kepler problem fixes the integrated orbit; the paper's own fits and energy
figures bound the Plummer runs.
"""
import json
import math
import os

import numpy as np
import pytest

from synth import plummer

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _quintic(seed):
    r = np.random.default_rng(seed)
    return r.uniform(-1, 1, (6, 3))  # c[n] multiplies t^n


def _derivs(c, t):
    x = sum(c[n] * t ** n for n in range(6))
    v = sum(n * c[n] * t ** (n - 1) for n in range(1, 6))
    a = sum(n * (n - 1) * c[n] * t ** (n - 2) for n in range(2, 6))
    k = sum(n * (n - 1) * (n - 2) * c[n] * t ** (n - 3) for n in range(3, 6))
    return x, v, a, k


@pytest.mark.parametrize("dt", [2.0 ** -3, 2.0 ** -7, 0.3])
def test_predictor_exact_for_cubic_motion(orc, dt):
    c = _quintic(1)
    c[4:] = 0.0
    x0, v0, a0, k0 = _derivs(c, 0.0)
    x1, v1, _, _ = _derivs(c, dt)
    xp, vp = orc.predict_one(x0, v0, a0, k0, dt)
    assert np.allclose(xp, x1, rtol=1e-15, atol=1e-15)
    assert np.allclose(vp, v1, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("dt", [2.0 ** -3, 2.0 ** -6, 0.2])
def test_corrector_exact_for_quintic_motion(orc, dt):
    c = _quintic(2)
    x0, v0, a0, k0 = _derivs(c, 0.0)
    x1, v1, a1, k1 = _derivs(c, dt)
    xp, vp = orc.predict_one(x0, v0, a0, k0, dt)
    xc, vc, a2, a3 = orc.correct_one(xp, vp, a0, k0, a1, k1, dt)
    assert np.allclose(xc, x1, rtol=1e-14, atol=1e-14)
    assert np.allclose(vc, v1, rtol=1e-14, atol=1e-14)
    # a2 = (dk/dt) dt^2 / 2 and a3 = (d2k/dt2) dt^3 / 6 at the start of the step (Section 2)
    assert np.allclose(a2, 24 * c[4] * dt * dt / 2, rtol=1e-12, atol=1e-14)
    assert np.allclose(a3, 120 * c[5] * dt ** 3 / 6, rtol=1e-12, atol=1e-14)


def test_corrector_not_exact_beyond_quintic(orc):
    # A sextic term is outside what a two-point cubic interpolation of a(t) can carry.
    dt = 0.25
    x0, v0, a0, k0 = np.zeros(3), np.zeros(3), np.zeros(3), np.zeros(3)
    c6 = np.array([1.0, 0.0, 0.0])
    a1 = 30 * c6 * dt ** 4
    k1 = 120 * c6 * dt ** 3
    xp, vp = orc.predict_one(x0, v0, a0, k0, dt)
    xc, _, _, _ = orc.correct_one(xp, vp, a0, k0, a1, k1, dt)
    assert abs(xc[0] - dt ** 6) > 1e-6 * dt ** 6


@pytest.mark.parametrize("omega,R,eta", [(1.0, 1.0, 0.01), (3.0, 0.2, 0.02), (0.5, 7.0, 0.001)])
def test_aarseth_circular_orbit_closed_form(orc, omega, R, eta):
    # On a circular orbit |a| = w^2 R, |k| = w^3 R, |snap| = w^4 R, |crackle| = w^5 R,
    # so the Aarseth criterion reduces to sqrt(eta) / w.
    th = 0.7
    dt = 2.0 ** -5
    r = R * np.array([math.cos(th), math.sin(th), 0.0])
    u = R * omega * np.array([-math.sin(th), math.cos(th), 0.0])
    a1 = -omega ** 2 * r
    k1 = -omega ** 2 * u
    snap = omega ** 4 * r
    crackle = omega ** 4 * u
    a3 = crackle * dt ** 3 / 6
    a2 = (snap - crackle * dt) * dt * dt / 2
    got = orc.aarseth_dt(a1, k1, a2, a3, dt, eta)
    assert got == pytest.approx(math.sqrt(eta) / omega, rel=1e-13)


def test_initial_dt(orc):
    a = np.array([3.0, 4.0, 0.0])
    k = np.array([0.0, 0.0, 2.0])
    assert orc.initial_dt(a, k, 0.01) == pytest.approx(0.025)
    assert math.isinf(orc.initial_dt(a, np.zeros(3), 0.01))


@pytest.mark.parametrize("dt_raw,kmin,rc,level", [
    (0.125, 3, 0, 3), (0.12, 3, 0, 4), (1.0, 3, 0, 3), (0.0625, 3, 0, 4),
    (0.0625 * (1 + 1e-15), 3, 0, 4), (0.0625 * (1 - 1e-16), 3, 0, 5), (2.0 ** -40, 3, 0, 40),
    (2.0 ** -40 * 0.999, 3, -4, 0), (float("nan"), 3, -4, 0), (float("inf"), 3, 0, 3),
    (0.5, 4, 0, 4), (3e-5, 3, 0, 16)])
def test_level_of(orc, dt_raw, kmin, rc, level):
    got_rc, got_level = orc.level_of(dt_raw, kmin)
    assert got_rc == rc
    if rc == 0:
        assert got_level == level


def test_next_level_rules(orc):
    T = 1 << 40
    # halving (any depth) is immediate
    assert orc.next_level(5, 8, T // 32, 3) == 8
    # doubling needs the new time to be a multiple of the doubled step
    assert orc.next_level(5, 3, T // 16, 3) == 4
    assert orc.next_level(5, 3, T // 32, 3) == 5
    # at most one doubling per step, never above dt_max
    assert orc.next_level(3, 3, T, 3) == 3
    assert orc.next_level(4, 3, T // 8, 4) == 4
    assert orc.next_level(6, 6, T // 64 * 3, 3) == 6


def _kepler_position(t, a, e, gm):
    n = math.sqrt(gm / a ** 3)
    M = n * t
    E = M if e < 0.8 else math.pi
    for _ in range(60):
        E -= (E - e * math.sin(E) - M) / (1 - e * math.cos(E))
    return np.array([a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E), 0.0])


def _kepler_run(orc, e, eta):
    a_, gm = 1.0, 1.0
    rp = a_ * (1 - e)
    vp = math.sqrt(gm * (1 + e) / rp)
    m = np.array([0.5, 0.5])
    x = np.array([[-rp / 2, 0, 0], [rp / 2, 0, 0]])
    v = np.array([[0, -vp / 2, 0], [0, vp / 2, 0]])
    it = orc.Integrator(m, x, v, 0.0, eta=eta, eta_init=eta)
    E0 = it.energy()
    L0 = np.cross(it.x[1] - it.x[0], it.v[1] - it.v[0])
    it.run(8.0)
    assert it.synchronised() and it.t[0] == 8 * orc.TICKS_PER_UNIT
    err = np.linalg.norm(it.x[1] - it.x[0] - _kepler_position(8.0, a_, e, gm))
    dE = abs(it.energy() - E0) / abs(E0)
    dL = np.linalg.norm(np.cross(it.x[1] - it.x[0], it.v[1] - it.v[0]) - L0)
    assert np.abs((m[:, None] * it.v).sum(0)).max() < 1e-14
    return err, dE, dL


@pytest.mark.parametrize("e", [0.0, 0.5])
def test_kepler_two_body_fourth_order(orc, e):
    # Equal masses 1/2, unsoftened, relative orbit with a = 1 and G M = 1 (period
    # 2 pi), started at pericentre and integrated to t = 8; compared with the
    # closed-form Kepler solution.  Each 4x cut in eta halves every step, so a
    # fourth-order Hermite scheme must cut the position error about 16x.
    errs = []
    for eta in (0.01, 0.0025, 0.000625):
        err, dE, dL = _kepler_run(orc, e, eta)
        errs.append(err)
        assert dE < 1e-5 and dL < 1e-5
    assert errs[-1] < 1e-7
    for coarse, fine in zip(errs, errs[1:]):
        assert 11.0 < coarse / fine < 22.0


def test_block_step_invariants(orc):
    m, x, v = plummer(96, 7)
    it = orc.Integrator(m, x, v, 1.0 / 256)
    t_prev = 0
    T = orc.TICKS_PER_UNIT
    for _ in range(300):
        ends = it.t + (np.int64(1) << (40 - it.lev.astype(np.int64)))
        want_t = ends.min()
        want_act = np.nonzero(ends == want_t)[0]
        tn, act = it.step()
        assert tn == want_t and np.array_equal(act, want_act)
        assert act.size > 0 and tn >= t_prev
        t_prev = tn
        assert np.all(it.lev >= 3) and np.all(it.lev <= 40)
        dt_ticks = np.int64(1) << (40 - it.lev.astype(np.int64))
        assert np.all(it.t % dt_ticks == 0)
        assert np.all(it.t[act] == tn)
    assert t_prev <= T


def test_energy_and_paper_fits_n1024(orc):
    # Plummer N = 1024, eps = 1/256, eta = 0.01, t = 0 -> 1.  The paper reports
    # |dE/E| ~ 2e-7 for the host and GRAPE and < 1e-6 for its GPUs (Section 6,
    # abstract); the FP64 oracle must meet the 1e-6 bound.  Block size and step
    # count are checked against the paper's fits within a factor of 3 (Section 5).
    m, x, v = plummer(1024, 1)
    it = orc.Integrator(m, x, v, 1.0 / 256, nthreads=4)
    E0 = it.energy()
    steps, inter, hist = it.run(1.0)
    assert it.synchronised()
    dE = abs(it.energy() - E0) / abs(E0)
    assert dE <= GOLDEN["energy_bound_gpu"]["value"]
    nb = GOLDEN["n_block_fit"]
    ns = GOLDEN["n_steps_fit"]
    fit_block = nb["coef"] * 1024 ** nb["exp"]
    fit_steps = ns["coef"] * 1024 ** ns["exp"]
    assert fit_block / 3 < hist.mean() < fit_block * 3
    assert fit_steps / 3 < steps < fit_steps * 3
    assert inter == int(hist.astype(np.int64).sum()) * 1023


def test_shared_level_mode(orc):
    # kfix > 0: every particle advances with the same step 2^-kfix (fixed shared step).
    m, x, v = plummer(64, 8)
    it = orc.Integrator(m, x, v, 1.0 / 256, kfix=10)
    for s in range(5):
        tn, act = it.step()
        assert act.size == 64 and tn == (s + 1) * (orc.TICKS_PER_UNIT >> 10)
