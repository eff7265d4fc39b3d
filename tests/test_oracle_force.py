"""Pins of the oracle's direct-summation force (Eq. 1 and the Appendix A kernel).

The pins tie acc, jerk and pot to things other than their own formulas:
acc is the gradient of the softened potential, jerk is the time derivative of
acc along the motion (both by high-precision numerical differentiation of the
potential alone), Newton's third law gives momentum conservation, and the
shell theorem fixes the potential and force at the centre of a symmetric shell.
"""
import numpy as np
import pytest

from synth import plummer

mpmath = pytest.importorskip("mpmath")


def _rand_system(n, seed, spread=1.0):
    r = np.random.default_rng(seed)
    m = r.uniform(0.1, 1.0, n)
    x = r.normal(0, spread, (n, 3))
    v = r.normal(0, 1.0, (n, 3))
    return m, x, v


def _potential_field(m, x, v, i, eps):
    """F(y0, y1, y2, t) = sum_{j != i} m_j / sqrt(|d_j(t) - y|^2 + eps^2), d_j(t) the
    position of j relative to i when both move on straight lines.  The softened
    potential of i is -F, so acc_i = grad_y F and jerk_i = d/dt grad_y F at 0."""
    mp = mpmath.mp
    d = [[mp.mpf(x[j, c]) - mp.mpf(x[i, c]) for c in range(3)] for j in range(len(m))]
    w = [[mp.mpf(v[j, c]) - mp.mpf(v[i, c]) for c in range(3)] for j in range(len(m))]
    e2 = mp.mpf(eps) ** 2

    def F(y0, y1, y2, t):
        s = mp.mpf(0)
        y = (y0, y1, y2)
        for j in range(len(m)):
            if j == i:
                continue
            q = sum((d[j][c] + w[j][c] * t - y[c]) ** 2 for c in range(3))
            s += mp.mpf(m[j]) / mp.sqrt(q + e2)
        return s
    return F


@pytest.mark.parametrize("n,eps,seed", [(2, 0.0, 1), (3, 0.1, 2), (5, 1.0 / 256, 3), (8, 0.05, 4)])
def test_acc_is_gradient_and_jerk_is_time_derivative(orc, n, eps, seed):
    mpmath.mp.dps = 40
    m, x, v = _rand_system(n, seed)
    acc, jerk, pot = orc.force(m, x, v, eps)
    for i in range(n):
        F = _potential_field(m, x, v, i, eps)
        z = (0, 0, 0, 0)
        for c in range(3):
            order = [0, 0, 0, 0]
            order[c] = 1
            g = float(mpmath.diff(F, z, tuple(order)))
            order[3] = 1
            h = float(mpmath.diff(F, z, tuple(order)))
            assert acc[i, c] == pytest.approx(g, rel=1e-12, abs=1e-13 * np.abs(acc[i]).max())
            assert jerk[i, c] == pytest.approx(h, rel=1e-11, abs=1e-12 * np.abs(jerk[i]).max())
        assert pot[i] == pytest.approx(-float(F(0, 0, 0, 0)), rel=1e-14)


def test_two_body_closed_form(orc):
    # Two bodies: the force on each is m_other d / (|d|^2 + eps^2)^(3/2), attractive.
    m = np.array([0.3, 0.7])
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    v = np.zeros((2, 3))
    eps = 0.5
    acc, jerk, pot = orc.force(m, x, v, eps)
    s = (1.0 + eps * eps) ** 1.5
    assert acc[0] == pytest.approx([0.7 / s, 0, 0])
    assert acc[1] == pytest.approx([-0.3 / s, 0, 0])
    assert np.all(jerk == 0)
    assert pot == pytest.approx([-0.7 / 1.25 ** 0.5, -0.3 / 1.25 ** 0.5])


def test_momentum_conservation_plummer(orc):
    # Pairwise antisymmetry (Newton's third law) makes sum m_i a_i and sum m_i k_i vanish.
    m, x, v = plummer(512, 2)
    acc, jerk, _ = orc.force(m, x, v, 1.0 / 256)
    scale_a = np.abs(m[:, None] * acc).sum()
    scale_k = np.abs(m[:, None] * jerk).sum()
    assert np.abs((m[:, None] * acc).sum(0)).max() < 1e-14 * scale_a
    assert np.abs((m[:, None] * jerk).sum(0)).max() < 1e-14 * scale_k


def test_shell_theorem_center(orc):
    # Six equal masses on the vertices of an octahedron of radius R around a probe:
    # by symmetry acc = jerk = 0 at the centre, and pot = -M / sqrt(R^2 + eps^2).
    R, eps, M = 2.0, 0.25, 1.5
    pts = [[R, 0, 0], [-R, 0, 0], [0, R, 0], [0, -R, 0], [0, 0, R], [0, 0, -R]]
    x = np.array([[0.0, 0.0, 0.0]] + pts)
    m = np.array([1e-3] + [M / 6] * 6)
    v = np.zeros_like(x)
    acc, jerk, pot = orc.force(m, x, v, eps, idx=np.array([0], dtype=np.int32))
    assert np.abs(acc).max() < 1e-16
    assert np.abs(jerk).max() == 0.0
    assert pot[0] == pytest.approx(-M / np.sqrt(R * R + eps * eps), rel=1e-15)


def test_self_term_excluded_and_idx_subset(orc):
    m, x, v = plummer(64, 3)
    eps = 1.0 / 256
    acc, jerk, pot = orc.force(m, x, v, eps)
    sub = np.array([3, 17, 40], dtype=np.int32)
    a2, k2, p2 = orc.force(m, x, v, eps, idx=sub)
    assert np.array_equal(a2, acc[sub]) and np.array_equal(k2, jerk[sub]) and np.array_equal(p2, pot[sub])
    # a lone particle feels nothing: the self term is not in the sum
    a1, k1, p1 = orc.force(m[:1], x[:1], v[:1], eps)
    assert np.all(a1 == 0) and np.all(k1 == 0) and np.all(p1 == 0)


def test_energy_definition_consistency(orc):
    # W from the pair sum equals 1/2 sum m_i pot_i from the force routine; T = 1/2 sum m v^2.
    m, x, v = plummer(300, 4)
    eps = 1.0 / 256
    ek, ep = orc.energy(m, x, v, eps)
    _, _, pot = orc.force(m, x, v, eps)
    assert ep == pytest.approx(0.5 * np.sum(m * pot), rel=1e-13)
    assert ek == pytest.approx(0.5 * np.sum(m * (v * v).sum(1)), rel=1e-14)
    # Plummer realisation with T = 1/4, W(unsoftened) = -1/2: softening raises W a little
    assert -0.5 < ep < -0.49


def test_threads_do_not_change_results(orc):
    m, x, v = plummer(700, 5)
    r1 = orc.force(m, x, v, 1 / 256, nthreads=1)
    r4 = orc.force(m, x, v, 1 / 256, nthreads=4)
    for p, q in zip(r1, r4):
        assert np.array_equal(p, q)
