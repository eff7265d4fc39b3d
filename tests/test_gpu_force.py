"""Parity of the CUDA force sweep (nb_force) with the FP64 oracle.

Sizes span several tiles and ragged tails, block sizes cover the edges of
the i-blocks and of the automatic regimes (one or four i per pass of the
j-parallel kernel at 2/3, j-parallel up to 96, the one-i-per-thread kernel
for 97..192, 257..384 and 513..576, four i per thread otherwise), both
kernels are forced as well as chosen automatically, and both precisions are
checked.
"""
import numpy as np
import pytest

import oracle
from synth import plummer, sample_active
from nbtest import TOL_DS, TOL_F64, assert_force_close, force_errors, nb, pair_magnitudes  # noqa: F401

pytestmark = pytest.mark.gpu

EPS = 1.0 / 256


def _check(nb, m, x, v, eps, idx, precision, mode=0, split=0, label=""):
    o = nb.nb_default_opts(precision=precision, force_mode=mode, split_j=split)
    ctx = nb.nb_init(m, x, v, eps, o)
    try:
        got = nb.nb_force(ctx, idx)
    finally:
        nb.nb_free(ctx)
    ref = oracle.force(m, x, v, eps, idx, nthreads=8)
    mags = pair_magnitudes(m, x, v, eps, idx)
    tol = TOL_F64 if precision == nb.NB_FP64 else TOL_DS
    return assert_force_close(got, ref, mags, tol, label), got


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n", [2, 3, 8, 130, 1024, 4099])
def test_full_sweep(nb, n, precision):
    m, x, v = plummer(n, 100 + n)
    _check(nb, m, x, v, EPS, np.arange(n, dtype=np.int32), precision, label="n=%d" % n)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("na", [1, 2, 3, 7, 16, 17, 31, 32, 33, 64, 65, 96, 97, 191, 192, 193, 255, 256,
                                257, 384, 385, 576, 577, 1000])
def test_block_sizes_and_kernels(nb, na, mode, precision):
    n = 3001
    m, x, v = plummer(n, 7)
    idx = sample_active(n, na, 11 + na)
    _check(nb, m, x, v, EPS, idx, precision, mode, label="na=%d mode=%d" % (na, mode))


@pytest.mark.parametrize("split", [1, 2, 5, 23])
def test_forced_split_counts(nb, split):
    n = 2048 + 77
    m, x, v = plummer(n, 8)
    idx = sample_active(n, 300, 3)
    _check(nb, m, x, v, EPS, idx, 0, 1, split, label="split=%d" % split)


def test_unsorted_active_order(nb):
    n = 1500
    m, x, v = plummer(n, 9)
    idx = sample_active(n, 200, 4)[::-1].copy()
    _check(nb, m, x, v, EPS, idx, 0)


@pytest.mark.parametrize("precision", [0, 1])
def test_unsoftened_two_body_and_small(nb, precision):
    # eps = 0 runs the guarded kernel; no coincident particles here.
    rng = np.random.default_rng(5)
    for n in (2, 3, 9, 200):
        m = rng.uniform(0.1, 1.0, n)
        x = rng.normal(size=(n, 3))
        v = rng.normal(size=(n, 3))
        _check(nb, m, x, v, 0.0, np.arange(n, dtype=np.int32), precision, label="eps0 n=%d" % n)


def test_single_particle_feels_nothing(nb):
    for precision in (0, 1):
        ctx = nb.nb_init([1.0], [[0.3, 0.1, -2.0]], [[1.0, 0, 0]], EPS,
                         nb.nb_default_opts(precision=precision))
        acc, jerk, pot = nb.nb_force(ctx, [0])
        nb.nb_free(ctx)
        assert np.all(acc == 0) and np.all(jerk == 0)
        assert abs(pot[0]) < 1e-6 if precision == 0 else pot[0] == 0.0


def test_coincident_particles_softened(nb):
    # Two particles at the same place: only softening keeps the pair finite.
    m, x, v = plummer(300, 12)
    x[5] = x[17]
    v[5] = v[17] + 0.1
    _check(nb, m, x, v, EPS, np.arange(300, dtype=np.int32), 0)
    _check(nb, m, x, v, EPS, np.arange(300, dtype=np.int32), 1)


def test_mass_spread_1e6(nb):
    m, x, v = plummer(2000, 13)
    m = m * np.exp(np.random.default_rng(1).uniform(0, np.log(1e6), 2000))
    m /= m.sum()
    _check(nb, m, x, v, EPS, sample_active(2000, 500, 2), 0)


def test_offset_cluster_needs_double_single(nb):
    # A cluster far from the origin: plain FP32 positions would lose the close
    # separations, the double-single difference keeps them.
    m, x, v = plummer(1024, 14)
    x = x + np.array([1000.0, -3000.0, 500.0])
    _check(nb, m, x, v, EPS, sample_active(1024, 200, 5), 0, label="offset")


def test_deterministic_bitwise(nb):
    m, x, v = plummer(5000, 15)
    idx = sample_active(5000, 700, 6)
    outs = []
    for _ in range(2):
        ctx = nb.nb_init(m, x, v, EPS)
        outs.append(nb.nb_force(ctx, idx))
        nb.nb_free(ctx)
    for p, q in zip(*outs):
        assert np.array_equal(p, q)


def test_dev_pointer_variant_matches_host(nb):
    torch = pytest.importorskip("torch")
    m, x, v = plummer(3000, 16)
    idx = sample_active(3000, 123, 7)
    stream = torch.cuda.current_stream()
    ctx = nb.nb_init(m, x, v, EPS, nb.nb_default_opts(stream=stream.cuda_stream))
    try:
        host = nb.nb_force(ctx, idx)
        d_idx = torch.from_numpy(idx).cuda()
        d_acc = torch.empty((len(idx), 3), dtype=torch.float64, device="cuda")
        d_jerk = torch.empty_like(d_acc)
        d_pot = torch.empty(len(idx), dtype=torch.float64, device="cuda")
        nb.nb_force_dev(ctx, d_idx, len(idx), d_acc, d_jerk, d_pot)
        torch.cuda.synchronize()
        assert np.array_equal(d_acc.cpu().numpy(), host[0])
        assert np.array_equal(d_jerk.cpu().numpy(), host[1])
        assert np.array_equal(d_pot.cpu().numpy(), host[2])
        bad = torch.tensor([0, 5, 5], dtype=torch.int32, device="cuda")
        with pytest.raises(nb.NbError) as ei:
            nb.nb_force_dev(ctx, bad, 3, d_acc, d_jerk, d_pot)
        assert ei.value.code == nb.NB_EINVAL
        oob = torch.tensor([0, 3000], dtype=torch.int32, device="cuda")
        with pytest.raises(nb.NbError):
            nb.nb_force_dev(ctx, oob, 2, d_acc, d_jerk, d_pot)
    finally:
        nb.nb_free(ctx)


def test_host_argument_errors(nb):
    m, x, v = plummer(64, 17)
    ctx = nb.nb_init(m, x, v, EPS)
    try:
        for idx in ([0, 64], [-1], [3, 3]):
            with pytest.raises(nb.NbError) as ei:
                nb.nb_force(ctx, idx)
            assert ei.value.code == nb.NB_EINVAL
        with pytest.raises(nb.NbError) as ei:
            nb.nb_predict(ctx, 0.1)   # not on the 2^-40 grid
        assert ei.value.code == nb.NB_EINVAL
        with pytest.raises(nb.NbError) as ei:
            nb.nb_correct(ctx, [1, 2], 0.125)  # no matching nb_force
        assert ei.value.code == nb.NB_ESTATE
        acc, jerk, pot = nb.nb_force(ctx, np.zeros(0, dtype=np.int32))
        assert acc.shape == (0, 3)
    finally:
        nb.nb_free(ctx)


@pytest.mark.parametrize("na", [1, 2, 3, 32, 96, 97, 256, 300, 577, 4096])
def test_full_size_sampled(nb, na):
    # N = 2^20, eps = 1/1024: the benchmark's sweep configuration; 64 of the
    # active particles are checked one by one against the oracle.
    n, eps = 1 << 20, 1.0 / 1024
    m, x, v = plummer(n, 3)
    idx = sample_active(n, na, 3 + na)
    ctx = nb.nb_init(m, x, v, eps)
    try:
        got = nb.nb_force(ctx, idx)
    finally:
        nb.nb_free(ctx)
    pick = np.random.default_rng(na).choice(na, size=min(64, na), replace=False)
    ref = oracle.force(m, x, v, eps, idx[pick], nthreads=8)
    mags = pair_magnitudes(m, x, v, eps, idx[pick], chunk=4)
    assert_force_close(tuple(g[pick] for g in got), ref, mags, TOL_DS, "N=2^20 na=%d" % na)


@pytest.mark.parametrize("precision", [0, 1])
def test_whole_and_sliced_blocks(nb, precision):
    # More i-blocks than one wave of resident CTAs (all 300001 particles
    # active): the i-blocks of the full waves (on a GB300, the first
    # 608 x 256 = 155648 particles for DS, 2432 x 64 for FP64) take all j
    # in one item, the remaining ones run in j slices whose partials are
    # summed in slice order; the last i-block and the last slice are ragged.
    # Sampled particles on both sides of the boundary against the oracle,
    # and bitwise the same result on a second call.
    n, eps = 300001, 1.0 / 1024
    m, x, v = plummer(n, 31)
    idx = np.arange(n, dtype=np.int32)
    ctx = nb.nb_init(m, x, v, eps, nb.nb_default_opts(precision=precision, flags=nb.NB_INIT_NO_FORCE))
    try:
        got = nb.nb_force(ctx, idx)
        again = nb.nb_force(ctx, idx)
    finally:
        nb.nb_free(ctx)
    for g, h in zip(got, again):
        assert np.array_equal(g, h)
    edges = [0, 1, 155647, 155648, 155649, 155903, 155904, 299775, 299776, n - 1]
    pick = np.unique(np.concatenate([np.random.default_rng(5).choice(n, 190, replace=False),
                                     edges])).astype(np.int32)
    ref = oracle.force(m, x, v, eps, pick, nthreads=8)
    mags = pair_magnitudes(m, x, v, eps, pick, chunk=8)
    assert_force_close(tuple(g[pick] for g in got), ref, mags, TOL_F64 if precision else TOL_DS,
                       "whole and sliced i-blocks, precision %d" % precision)


def test_jpar_slice_counters_reset_between_calls(nb):
    # The DS j-parallel kernel sums its slices in the CTA that finishes a
    # chunk last, found by per-chunk arrival counters that this CTA resets.
    # Alternating block sizes (one i per pass, four i per pass, different
    # chunk and slice counts) must give bitwise the same result every time.
    n = 300000
    m, x, v = plummer(n, 21)
    ctx = nb.nb_init(m, x, v, EPS, nb.nb_default_opts(flags=nb.NB_INIT_NO_FORCE))
    try:
        blocks = [sample_active(n, na, 40 + na) for na in (5, 1, 2, 31, 3)]
        first = [nb.nb_force(ctx, idx) for idx in blocks]
        again = [nb.nb_force(ctx, idx) for idx in reversed(blocks)][::-1]
    finally:
        nb.nb_free(ctx)
    for f, g in zip(first, again):
        for p, q in zip(f, g):
            assert np.array_equal(p, q)
    ref = oracle.force(m, x, v, EPS, blocks[0], nthreads=8)
    mags = pair_magnitudes(m, x, v, EPS, blocks[0])
    assert_force_close(first[0], ref, mags, TOL_DS, "na=5 N=300000")
