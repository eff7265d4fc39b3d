"""Parity of the summation variants (Section 6: GRAPE-style 64-bit fixed-point
sums; FP32 sums in index order and smallest force first) with the oracle.

Every variant evaluates its single-precision pair terms with IEEE
round-to-nearest operations in a fixed order, so the GPU must reproduce the
oracle bit for bit: forces on every block size, kernel split and ragged tail,
and (fixed point) whole block-step trajectories.
"""
import numpy as np
import pytest

import oracle
from synth import plummer, salpeter_masses, sample_active
from nbtest import nb  # noqa: F401

pytestmark = pytest.mark.gpu

EPS = 1.0 / 256
MODES = {"fixed": (1, oracle.SUM_FIXED), "fp32": (2, oracle.SUM_FP32),
         "sorted": (3, oracle.SUM_FP32_SORTED)}


def _gpu_force(nb, m, x, v, eps, idx, summation, split=0, no_force=False):
    o = nb.nb_default_opts(summation=summation, split_j=split,
                           flags=nb.NB_INIT_NO_FORCE if no_force else 0)
    ctx = nb.nb_init(m, x, v, eps, o)
    try:
        return nb.nb_force(ctx, idx)
    finally:
        nb.nb_free(ctx)


def _assert_same(got, ref, label):
    for name, g, r in zip(("acc", "jerk", "pot"), got, ref):
        bad = np.nonzero(~((g == r) | (np.isnan(g) & np.isnan(r))).reshape(len(g), -1).all(axis=1))[0]
        assert bad.size == 0, "%s %s differs at %d particles, first %d: %r vs %r" % (
            label, name, bad.size, bad[0], g[bad[0]], r[bad[0]])


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("n", [2, 3, 130, 1031, 4099])
def test_full_sweep_bit_exact(nb, mode, n):
    m, x, v = plummer(n, 200 + n)
    idx = np.arange(n, dtype=np.int32)
    if mode == "sorted" and n > 1100:
        idx = sample_active(n, 300, 5)
    got = _gpu_force(nb, m, x, v, EPS, idx, MODES[mode][0])
    ref = oracle.force_summed(m, x, v, EPS, idx, mode=MODES[mode][1], nthreads=8)
    _assert_same(got, ref, "%s n=%d" % (mode, n))


@pytest.mark.parametrize("split", [0, 1, 3, 17])
@pytest.mark.parametrize("na", [1, 7, 33, 128, 129, 255, 256, 257, 1000, 3001])
def test_fixed_block_sizes_and_splits_bit_exact(nb, na, split):
    n = 3001
    m, x, v = plummer(n, 7)
    idx = sample_active(n, na, 11 + na)
    got = _gpu_force(nb, m, x, v, EPS, idx, nb.NB_SUM_FIXED, split=split)
    ref = oracle.force_summed(m, x, v, EPS, idx, mode=oracle.SUM_FIXED, nthreads=8)
    _assert_same(got, ref, "na=%d split=%d" % (na, split))


@pytest.mark.parametrize("mode", ["fp32", "sorted"])
@pytest.mark.parametrize("na", [1, 5, 129, 700])
def test_fp32_block_sizes_bit_exact(nb, mode, na):
    n = 2053
    m, x, v = plummer(n, 17)
    idx = sample_active(n, na, 3 + na)
    got = _gpu_force(nb, m, x, v, EPS, idx, MODES[mode][0])
    ref = oracle.force_summed(m, x, v, EPS, idx, mode=MODES[mode][1], nthreads=8)
    _assert_same(got, ref, "%s na=%d" % (mode, na))


@pytest.mark.parametrize("mode", sorted(MODES))
def test_unequal_masses_far_from_origin_bit_exact(nb, mode):
    n = 1500
    m, x, v = plummer(n, 23, masses=salpeter_masses(n, 23))
    x = x + np.array([100.0, -50.0, 25.0])
    idx = sample_active(n, 200, 9)
    got = _gpu_force(nb, m, x, v, EPS, idx, MODES[mode][0])
    ref = oracle.force_summed(m, x, v, EPS, idx, mode=MODES[mode][1], nthreads=8)
    _assert_same(got, ref, mode)


def test_fixed_is_independent_of_particle_order(nb):
    n = 2500
    m, x, v = plummer(n, 31)
    perm = np.random.default_rng(4).permutation(n)
    idx = np.arange(n, dtype=np.int32)
    a0, k0, p0 = _gpu_force(nb, m, x, v, EPS, idx, nb.NB_SUM_FIXED)
    a1, k1, p1 = _gpu_force(nb, m[perm], x[perm], v[perm], EPS, idx, nb.NB_SUM_FIXED, split=5)
    assert np.array_equal(a1, a0[perm]) and np.array_equal(k1, k0[perm])
    assert np.array_equal(p1, p0[perm])


@pytest.mark.parametrize("mode", ["fp32", "sorted"])
def test_fp32_unsoftened_coincident_pair_is_skipped(nb, mode):
    m, x, v = plummer(300, 3)
    x[7] = x[3]                     # distinct particles at one point, eps = 0
    idx = np.array([3, 7, 100], dtype=np.int32)
    got = _gpu_force(nb, m, x, v, 0.0, idx, MODES[mode][0])
    ref = oracle.force_summed(m, x, v, 0.0, idx, mode=MODES[mode][1])
    assert np.all(np.isfinite(got[0]))
    _assert_same(got, ref, mode)


def test_fixed_rejects_unrepresentable_units(nb):
    # masses of 1e30 with eps = 1e-10 put the jerk unit below 2^-126: the
    # kernel reports it and the start-up sweep fails cleanly
    m, x, v = plummer(64, 2)
    with pytest.raises(nb.NbError) as ei:
        nb.nb_init(m * 1e30, x, v * 1e10, 1e-10, nb.nb_default_opts(summation=nb.NB_SUM_FIXED))
    assert ei.value.code == nb.NB_EINVAL


def test_fixed_force_dev_matches_host_call(nb):
    import torch
    n = 1200
    m, x, v = plummer(n, 5)
    idx = sample_active(n, 150, 2)
    ctx = nb.Context(m, x, v, EPS, summation=nb.NB_SUM_FIXED)
    try:
        host = ctx.nb_force(idx)
        d_idx = torch.tensor(idx, device="cuda")
        acc = torch.empty((len(idx), 3), dtype=torch.float64, device="cuda")
        jerk = torch.empty_like(acc)
        pot = torch.empty(len(idx), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        ctx.nb_force_dev(d_idx.data_ptr(), len(idx), acc.data_ptr(), jerk.data_ptr(), pot.data_ptr())
        nb.nb_get_state(ctx.ctx)    # synchronises the context's stream
        assert np.array_equal(acc.cpu().numpy(), host[0])
        assert np.array_equal(jerk.cpu().numpy(), host[1])
        assert np.array_equal(pot.cpu().numpy(), host[2])
    finally:
        ctx.nb_free()


# ---------------------------------------------------------------------------
# trajectories: with fixed-point sums the whole block-step integration is
# reproducible, so the device-driven steps must equal the oracle bit for bit


def _assert_state_equal(st, orc, label):
    for key, ref in (("x", orc.x), ("v", orc.v), ("a", orc.a), ("k", orc.k), ("t", orc.t),
                     ("level", orc.lev)):
        assert np.array_equal(st[key], ref), "%s: %s differs at %d particles" % (
            label, key, int(np.sum(np.any((st[key] != ref).reshape(len(ref), -1), axis=1))))


def test_fixed_block_steps_bit_exact(nb):
    n = 1024
    m, x, v = plummer(n, 1)
    orc = oracle.Integrator(m, x, v, EPS, summation=oracle.SUM_FIXED, nthreads=8)
    ctx = nb.Context(m, x, v, EPS, summation=nb.NB_SUM_FIXED)
    try:
        _assert_state_equal(ctx.nb_get_state(), orc, "start")
        for s in range(64):
            t, na = ctx.nb_step()
            tn, act = orc.step()
            assert t == tn / oracle.TICKS_PER_UNIT and na == len(act), s
            _assert_state_equal(ctx.nb_get_state(), orc, "step %d" % s)
    finally:
        ctx.nb_free()


def test_fixed_graph_run_bit_exact(nb):
    n = 1500
    m, x, v = plummer(n, 4, masses=salpeter_masses(n, 4))
    orc = oracle.Integrator(m, x, v, EPS, summation=oracle.SUM_FIXED, nthreads=8)
    ctx = nb.Context(m, x, v, EPS, summation=nb.NB_SUM_FIXED)
    try:
        steps, _ = ctx.nb_run(1.0 / 32)
        osteps, _, _ = orc.run(1.0 / 32)
        assert steps == osteps
        _assert_state_equal(ctx.nb_get_state(), orc, "t=1/32")
    finally:
        ctx.nb_free()


# ---------------------------------------------------------------------------
# the full-size system: sampled particles computed one by one by the oracle


@pytest.mark.parametrize("mode", sorted(MODES))
def test_million_body_sampled_bit_exact(nb, mode):
    n = 1 << 20
    m, x, v = plummer(n, 3, exact_virial_max=0)
    eps = 1.0 / 1024
    na = 16 if mode == "sorted" else 64
    idx = sample_active(n, na, 3 + na)
    got = _gpu_force(nb, m, x, v, eps, idx, MODES[mode][0], no_force=True)
    ref = oracle.force_summed(m, x, v, eps, idx, mode=MODES[mode][1], nthreads=oracle.max_threads())
    _assert_same(got, ref, "%s n=2^20" % mode)
