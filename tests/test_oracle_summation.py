"""Pins of the oracle's summation variants (Section 6 on accuracy: GRAPE-6's
64-bit fixed-point accumulation, and the suggestion to sum the smallest
forces first on the GPU).

The single-precision pair terms are pinned against the FP64 definition
(itself pinned in test_oracle_force.py); the summations are redone here from
the exposed terms with Python integers and numpy's sequential float32
accumulation; the fixed-point scales are derived from their definition with
math.frexp; exact momentum conservation and order independence are
properties the fixed-point sum must have.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

import oracle
from synth import plummer, salpeter_masses

EPS = 1.0 / 256


@pytest.fixture(scope="module")
def system():
    return plummer(512, 11)


def _exp_above(x32):
    """Smallest e with x < 2^e from the exponent field (-126 for 0, subnormals)."""
    x = float(x32)
    if x == 0.0:
        return -126
    return max(math.frexp(x)[1], -126)


def _scales_by_definition(m, v, eps):
    eps2 = float(np.float32(eps * eps))
    F = math.frexp(eps2)[1] - 1
    m32 = m.astype(np.float32)
    v32 = np.abs(v.astype(np.float32))
    v1 = (v32[:, 0] + v32[:, 1]) + v32[:, 2]     # float32 arithmetic
    Em = max(_exp_above(m32.max()), -64)
    Ev = max(_exp_above(v1.max()), -64)
    e = [Em - F, 3 + Em + Ev - (3 * F) // 2, Em - F // 2]
    return tuple(min(56 - q, 126) for q in e)


def _to_double(Y):
    """The oracle's integer-to-double rule: |Y| = H 2^64 + L, fl(fl(H) 2^64 + fl(L))."""
    H, L = divmod(abs(Y), 1 << 64)
    d = float(H) * 2.0 ** 64 + float(L)
    return -d if Y < 0 else d


# ---------------------------------------------------------------------------
# the single-precision pair terms


@pytest.mark.parametrize("masses", ["equal", "salpeter"])
def test_terms_sum_to_the_fp64_force(masses):
    n = 384
    mm = None if masses == "equal" else salpeter_masses(n, 4)
    m, x, v = plummer(n, 21, masses=mm)
    a64, k64, p64 = oracle.force(m, x, v, EPS)
    for i in (0, 7, 100, 383):
        t, _, ok = oracle.pair_terms32(m, x, v, EPS, i)
        assert not ok[i] and ok.sum() == n - 1
        t64 = t.astype(np.float64)
        got = t64.sum(axis=0)
        S = np.abs(t64).sum(axis=0)          # sum of term magnitudes per component
        ref = np.concatenate([a64[i], k64[i], [p64[i]]])
        # each FP32 term carries a few ulps of relative error
        assert np.all(np.abs(got - ref) <= 4e-7 * S + 1e-300), (i, got, ref)


def test_terms_keep_double_single_positions(system):
    # far from the origin the separations only survive in hi + lo: the force
    # of the shifted system must still be the (translation-invariant) FP64 one
    m, x, v = system
    xs = x + np.array([100.0, -50.0, 25.0])
    a64, k64, p64 = oracle.force(m, x, v, EPS)
    for i in (0, 200):
        t, _, ok = oracle.pair_terms32(m, xs, v, EPS, i)
        t64 = t.astype(np.float64)
        ref = np.concatenate([a64[i], k64[i], [p64[i]]])
        assert np.all(np.abs(t64.sum(axis=0) - ref) <= 4e-7 * np.abs(t64).sum(axis=0)), i


def test_term_keys_are_pair_force_magnitudes(system):
    m, x, v = system
    t, key, ok = oracle.pair_terms32(m, x, v, EPS, 3)
    fmag = np.linalg.norm(t[:, :3].astype(np.float64), axis=1)
    assert np.all(np.abs(key[ok] - fmag[ok]) <= 4e-7 * fmag[ok])
    assert key[3] == 0.0


def test_equal_mass_fixed_force_conserves_momentum_exactly(system):
    # For equal masses the single-precision pair terms of (i, j) and (j, i)
    # are exact negatives, and so are their rounded fixed-point values: the
    # fixed-point sums conserve momentum exactly.
    m, x, v = system
    acc, jerk, _ = oracle.force_summed(m, x, v, EPS, mode=oracle.SUM_FIXED)
    for comp in (acc, jerk):
        for c in range(3):
            assert sum(Fraction(float(q)) for q in comp[:, c]) == 0
    # FP32 running sums do not have this property
    acc32, _, _ = oracle.force_summed(m, x, v, EPS, mode=oracle.SUM_FP32)
    assert any(sum(Fraction(float(q)) for q in acc32[:, c]) != 0 for c in range(3))


# ---------------------------------------------------------------------------
# fixed-point scales and sums


@pytest.mark.parametrize("eps", [1.0 / 256, 1.0 / 1024, 2.0 ** -5.5, 3.0, 1e-3])
@pytest.mark.parametrize("vscale", [1.0, 1e-3, 1e3, 0.0])
def test_fixed_scales_follow_their_definition(system, eps, vscale):
    m, _, v = system
    v = v * vscale
    assert oracle.fixed_scales(m, v, eps) == _scales_by_definition(m, v, eps)


def test_fixed_scales_reject_unusable_softening(system):
    m, x, v = system
    for eps in (0.0, 1e-30):
        with pytest.raises(ValueError):
            oracle.fixed_scales(m, v, eps)
        with pytest.raises(ValueError):
            oracle.force_summed(m, x, v, eps, mode=oracle.SUM_FIXED)


@pytest.mark.parametrize("masses", ["equal", "salpeter"])
def test_fixed_sum_is_the_exact_sum_of_rounded_terms(masses):
    n = 300
    mm = None if masses == "equal" else salpeter_masses(n, 9)
    m, x, v = plummer(n, 31, masses=mm)
    s = oracle.fixed_scales(m, v, EPS)
    idx = np.array([0, 1, 150, 299], dtype=np.int32)
    acc, jerk, pot = oracle.force_summed(m, x, v, EPS, idx, mode=oracle.SUM_FIXED)
    out = np.concatenate([acc, jerk, pot[:, None]], axis=1)
    for r, i in enumerate(idx):
        t, _, ok = oracle.pair_terms32(m, x, v, EPS, i, scaled=True)
        for q in range(7):
            Y = sum(round(float(tt)) for tt in t[ok, q])   # round half to even
            want = _to_double(Y) * 2.0 ** -s[0 if q < 3 else (1 if q < 6 else 2)]
            assert out[r, q] == want, (i, q)


def test_fixed_terms_stay_below_the_bound():
    # a close pair at the distance that maximises m |dx| / r^3, with a large
    # relative velocity, inside a Plummer sphere
    m, x, v = plummer(256, 41)
    x[1] = x[0] + np.array([EPS / math.sqrt(2.0), 0.0, 0.0])
    v[1] = v[0] + np.array([3.0, 0.5, 0.0])
    worst = 0.0
    for i in (0, 1, 2):
        t, _, ok = oracle.pair_terms32(m, x, v, EPS, i, scaled=True)
        worst = max(worst, float(np.abs(t[ok]).max()))
    assert worst < 2.0 ** 56 * (1 + 2.0 ** -10)
    assert worst > 2.0 ** 50     # the bound is within a factor 64 of this pair


def test_fixed_sum_is_independent_of_particle_order(system):
    m, x, v = system
    perm = np.random.default_rng(5).permutation(m.shape[0])
    a0, k0, p0 = oracle.force_summed(m, x, v, EPS, mode=oracle.SUM_FIXED)
    a1, k1, p1 = oracle.force_summed(m[perm], x[perm], v[perm], EPS, mode=oracle.SUM_FIXED)
    assert np.array_equal(a1, a0[perm]) and np.array_equal(k1, k0[perm])
    assert np.array_equal(p1, p0[perm])
    # the test can see order dependence: the index-order FP32 sums change
    b0, _, _ = oracle.force_summed(m, x, v, EPS, mode=oracle.SUM_FP32)
    b1, _, _ = oracle.force_summed(m[perm], x[perm], v[perm], EPS, mode=oracle.SUM_FP32)
    assert not np.array_equal(b1, b0[perm])


# ---------------------------------------------------------------------------
# FP32 running sums


@pytest.mark.parametrize("mode", [oracle.SUM_FP32, oracle.SUM_FP32_SORTED])
def test_fp32_sums_are_sequential_in_their_order(system, mode):
    m, x, v = system
    idx = np.array([0, 5, 211, 511], dtype=np.int32)
    acc, jerk, pot = oracle.force_summed(m, x, v, EPS, idx, mode=mode)
    out = np.concatenate([acc, jerk, pot[:, None]], axis=1)
    for r, i in enumerate(idx):
        t, key, ok = oracle.pair_terms32(m, x, v, EPS, i)
        j = np.nonzero(ok)[0]
        if mode == oracle.SUM_FP32_SORTED:
            j = j[np.lexsort((j, key[j].view(np.uint32)))]
        for q in range(7):
            run = np.add.accumulate(t[j, q], dtype=np.float32)   # strictly sequential
            assert out[r, q] == float(run[-1]), (i, q)


def test_sorted_order_is_smallest_force_first(system):
    m, x, v = system
    _, key, ok = oracle.pair_terms32(m, x, v, EPS, 9)
    j = np.nonzero(ok)[0]
    order = j[np.lexsort((j, key[j].view(np.uint32)))]
    assert np.all(np.diff(key[order]) >= 0)


def test_sorted_ties_go_in_index_order():
    # particle 0 at the centre of a cubic lattice: its pair forces come in
    # groups of exactly equal magnitude, summed in increasing j
    g = np.arange(-2, 3, dtype=np.float64) * 0.25
    pts = np.array([(a, b, c) for a in g for b in g for c in g])
    pts = np.concatenate([[[0.0, 0.0, 0.0]], pts[np.any(pts != 0.0, axis=1)]])
    n = pts.shape[0]
    m = np.full(n, 1.0 / n)
    v = np.zeros((n, 3))
    t, key, ok = oracle.pair_terms32(m, pts, v, EPS, 0)
    j = np.nonzero(ok)[0]
    assert len(np.unique(key[j])) < len(j) // 4       # many exact ties
    order = j[np.lexsort((j, key[j].view(np.uint32)))]
    acc, _, pot = oracle.force_summed(m, pts, v, EPS, np.array([0], np.int32),
                                      mode=oracle.SUM_FP32_SORTED)
    for q in range(3):
        assert acc[0, q] == float(np.add.accumulate(t[order, q], dtype=np.float32)[-1])
    # the reversed tie order gives a different sum for some component
    rev = j[np.lexsort((-j, key[j].view(np.uint32)))]
    sums_rev = [float(np.add.accumulate(t[rev, q], dtype=np.float32)[-1]) for q in range(3)]
    assert any(acc[0, q] != sums_rev[q] for q in range(3))


def test_sorting_and_fixed_point_improve_accuracy():
    # Section 6: FP32 sums lose accuracy; smallest-first sums should do
    # better, and exact (fixed-point) sums leave only the terms' own error.
    n = 4096
    m, x, v = plummer(n, 13)
    idx = np.random.default_rng(2).choice(n, 256, replace=False).astype(np.int32)
    a64, k64, p64 = oracle.force(m, x, v, EPS, idx, nthreads=oracle.max_threads())
    err = {}
    for mode in (oracle.SUM_FIXED, oracle.SUM_FP32, oracle.SUM_FP32_SORTED):
        a, k, p = oracle.force_summed(m, x, v, EPS, idx, mode=mode, nthreads=oracle.max_threads())
        err[mode] = (np.median(np.linalg.norm(a - a64, axis=1) / np.linalg.norm(a64, axis=1)),
                     np.median(np.abs(p - p64) / np.abs(p64)))
    for q in range(2):
        assert err[oracle.SUM_FP32_SORTED][q] < err[oracle.SUM_FP32][q]
        assert err[oracle.SUM_FIXED][q] < 0.5 * err[oracle.SUM_FP32_SORTED][q]


# ---------------------------------------------------------------------------
# the integrator with a summation variant


@pytest.mark.parametrize("mode", [oracle.SUM_FIXED, oracle.SUM_FP32_SORTED])
def test_integrator_with_summation_variant_tracks_fp64(mode):
    m, x, v = plummer(256, 1)
    ref = oracle.Integrator(m, x, v, EPS)
    var = oracle.Integrator(m, x, v, EPS, summation=mode)
    a0, k0, _ = oracle.force_summed(m, x, v, EPS, mode=mode)
    assert np.array_equal(var.a, a0) and np.array_equal(var.k, k0)
    e0 = ref.energy()
    ref.run(0.125)
    var.run(0.125)
    assert var.synchronised() and np.all(var.t == ref.t)
    assert abs(var.energy() - e0) / abs(e0) < 1e-5
    assert np.max(np.abs(var.x - ref.x)) < 1e-4
