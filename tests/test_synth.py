"""Pins of the seeded input generator (Plummer sphere, Section 4 of the paper)."""
import math

import numpy as np
import pytest

from synth import plummer, rng, sample_active, salpeter_masses, ensemble, ensemble_member
from synth.plummer import LENGTH_UNIT, kinetic_energy, unsoftened_potential_energy


def test_splitmix64_published_vector():
    # SplitMix64 started from state 1234567: the first five outputs of the
    # reference implementation (the standard test vector for this generator).
    s = np.uint64(1234567)
    with np.errstate(over="ignore"):
        got = [int(rng.mix64(s + np.uint64(k) * rng.GAMMA)) for k in range(1, 6)]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]


def test_uniform_range_and_moments():
    u = rng.uniform(7, 1, np.arange(200000))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3
    assert abs(u.var() - 1.0 / 12.0) < 2e-3


def test_deterministic_and_seed_dependent():
    a = plummer(256, 5)
    b = plummer(256, 5)
    c = plummer(256, 6)
    for p, q in zip(a, b):
        assert np.array_equal(p, q)
    assert not np.array_equal(a[1], c[1])


def test_nbody_units_exact_virial():
    m, x, v = plummer(1024, 1)
    assert m.sum() == pytest.approx(1.0, abs=1e-15)
    assert kinetic_energy(m, v) == pytest.approx(0.25, rel=1e-12)
    assert unsoftened_potential_energy(m, x) == pytest.approx(-0.5, rel=1e-12)
    assert np.abs((m[:, None] * x).sum(0)).max() < 1e-15
    assert np.abs((m[:, None] * v).sum(0)).max() < 1e-15


def test_plummer_mass_profile_ks():
    # Cumulative mass of a Plummer sphere (scale radius 1): M(<r) = r^3 / (1 + r^2)^(3/2),
    # truncated at the cut.  Analytic unit conversion only (no rescale) keeps radii in
    # known units.
    n = 1 << 16
    m, x, v = plummer(n, 11, exact_virial_max=0)
    r = np.sort(np.linalg.norm(x, axis=1)) / LENGTH_UNIT
    rc = 22.8 / LENGTH_UNIT
    cdf = lambda s: s ** 3 / (1 + s * s) ** 1.5
    f = cdf(r) / cdf(rc)
    emp = np.arange(1, n + 1) / n
    d = np.max(np.abs(emp - f))
    assert d < 1.63 / math.sqrt(n)  # KS at the 1% level
    assert r.max() <= rc


def test_plummer_speed_distribution_mean_square():
    # In N-body units a Plummer sphere has <v^2> = 2 T / M = 1/2 (virial equilibrium).
    m, x, v = plummer(1 << 16, 12, exact_virial_max=0)
    v2 = np.einsum("ij,ij->i", v, v).mean()
    assert v2 == pytest.approx(0.5, rel=0.02)
    # isotropy: each component carries a third of it
    for c in range(3):
        assert (v[:, c] ** 2).mean() == pytest.approx(v2 / 3, rel=0.03)


def test_sample_active():
    idx = sample_active(1000, 100, 3)
    assert idx.dtype == np.int32
    assert len(np.unique(idx)) == 100
    assert np.all(np.diff(idx) > 0)
    assert idx.min() >= 0 and idx.max() < 1000
    assert np.array_equal(sample_active(1000, 1000, 3), np.arange(1000))
    assert sample_active(10, 0, 3).size == 0


def test_salpeter_and_ensemble():
    mm = salpeter_masses(100000, 4)
    assert mm.sum() == pytest.approx(1.0)
    ratio = mm.max() / mm.min()
    assert ratio <= 1000.0 * (1 + 1e-12)
    # slope of the mass function: the median of m^-1.35-distributed masses on [0.1, 100]
    raw = mm / mm.min() * 0.1
    a = -1.35
    med_theory = (0.5 * (0.1 ** a + 100 ** a)) ** (1 / a)
    assert np.median(raw) == pytest.approx(med_theory, rel=0.05)
    clusters = ensemble(6, 9)
    for (m, x, v) in clusters:
        assert 32 <= m.shape[0] <= 4096
        q = kinetic_energy(m, v) / -unsoftened_potential_energy(m, x)
        assert 0.3 - 1e-9 <= q <= 0.7 + 1e-9


def test_ensemble_workers_give_the_same_clusters():
    # clusters come from their own counter-based streams: a process pool
    # (spawned) must reproduce the sequential generator bit for bit
    seq = ensemble(12, 4, n_lo=32, n_hi=1500)
    par = ensemble(12, 4, n_lo=32, n_hi=1500, workers=2)
    assert len(seq) == len(par)
    for a, b in zip(seq, par):
        for p, q in zip(a, b):
            assert np.array_equal(p, q)


def test_ensemble_member_is_the_same_cluster():
    full = ensemble(9, 6, n_lo=32, n_hi=700)
    for ci in (0, 4, 8):
        one = ensemble_member(9, 6, ci, n_lo=32, n_hi=700)
        for p, q in zip(full[ci], one):
            assert np.array_equal(p, q)
