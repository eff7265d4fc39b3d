"""The persistent nb_run (the whole block-step loop in one launch for n <=
16384) against the oracle and against the per-stage graph.

With the fixed-point summation the sums are exact, so the persistent run, the
per-stage graph and the oracle's integrator must agree bit for bit over whole
runs; with the compensated sums the persistent run adds its partials in
another order, so it is checked against the graph run and the oracle by
closeness and energy.
"""
import numpy as np
import pytest

import oracle
from synth import plummer, salpeter_masses
from nbtest import nb  # noqa: F401

pytestmark = pytest.mark.gpu

EPS = 1.0 / 256
T = oracle.TICKS_PER_UNIT
KEYS = (("x", "x"), ("v", "v"), ("a", "a"), ("k", "k"), ("t", "t"), ("level", "lev"))


def _state_equal_oracle(st, orc, label):
    for key, okey in KEYS:
        ref = getattr(orc, okey)
        assert np.array_equal(st[key], ref), "%s: %s differs at %d particles" % (
            label, key, int(np.sum(np.any((st[key] != ref).reshape(len(ref), -1), axis=1))))


@pytest.mark.parametrize("n,seed,t_end,salpeter", [(1024, 1, 1.0 / 16, False), (3000, 4, 1.0 / 32, True),
                                                   (33, 2, 1.0 / 8, False)])
def test_fixed_point_run_matches_oracle_bitwise(nb, n, seed, t_end, salpeter):
    m, x, v = plummer(n, seed, masses=salpeter_masses(n, seed) if salpeter else None)
    orc = oracle.Integrator(m, x, v, EPS, summation=oracle.SUM_FIXED, nthreads=8)
    ctx = nb.Context(m, x, v, EPS, summation=nb.NB_SUM_FIXED)
    try:
        steps, inter = ctx.nb_run(t_end)
        osteps, ointer, _ = orc.run(t_end)
        assert steps == osteps and inter == ointer
        _state_equal_oracle(ctx.nb_get_state(), orc, "n=%d" % n)
        assert ctx.nb_get_stats()["kernel_launches"] >= 1
    finally:
        ctx.nb_free()


def test_fixed_point_persistent_equals_graph_bitwise(nb):
    n = 2000
    m, x, v = plummer(n, 9)
    a = nb.Context(m, x, v, EPS, summation=nb.NB_SUM_FIXED)
    b = nb.Context(m, x, v, EPS, summation=nb.NB_SUM_FIXED, flags=nb.NB_RUN_GRAPH)
    try:
        sa, ia = a.nb_run(1.0 / 16)
        sb, ib = b.nb_run(1.0 / 16)
        assert (sa, ia) == (sb, ib)
        ra, rb = a.nb_get_state(), b.nb_get_state()
        for key in ra:
            assert np.array_equal(ra[key], rb[key]), key
        ea, eb = a.nb_energy(), b.nb_energy()
        assert ea == eb
    finally:
        a.nb_free()
        b.nb_free()


def test_stop_at_max_steps_and_resume_bitwise(nb):
    n = 1500
    m, x, v = plummer(n, 12)
    a = nb.Context(m, x, v, EPS, summation=nb.NB_SUM_FIXED)
    b = nb.Context(m, x, v, EPS, summation=nb.NB_SUM_FIXED)
    try:
        s1, _ = a.nb_run(1.0 / 8, max_steps=7)
        assert s1 == 7
        s2, _ = a.nb_run(1.0 / 8, max_steps=0)
        assert s2 == 0
        s3, _ = a.nb_run(1.0 / 8)
        sb, _ = b.nb_run(1.0 / 8)
        assert s1 + s3 == sb
        ra, rb = a.nb_get_state(), b.nb_get_state()
        for key in ra:
            assert np.array_equal(ra[key], rb[key]), key
    finally:
        a.nb_free()
        b.nb_free()


@pytest.mark.parametrize("n", [2, 257, 4096])
def test_compensated_run_close_to_graph_run(nb, n):
    m, x, v = plummer(n, 20 + n)
    # dt_max = 1/32, so that every particle meets at t = 1/32
    a = nb.Context(m, x, v, EPS, level_min=5)
    b = nb.Context(m, x, v, EPS, level_min=5, flags=nb.NB_RUN_GRAPH)
    try:
        e0 = sum(a.nb_energy())
        sa, _ = a.nb_run(1.0 / 32)
        sb, _ = b.nb_run(1.0 / 32)
        ra, rb = a.nb_get_state(), b.nb_get_state()
        assert np.all(ra["t"] == T // 32) and np.all(rb["t"] == T // 32)
        assert abs(sa - sb) <= max(2, 0.01 * sb)
        # the partials are added in another order: forces differ in the last
        # bits, and a particle whose step lies near a power of two may take the
        # other level, which changes its truncation error
        assert np.max(np.abs(ra["x"] - rb["x"])) < 1e-6
        assert np.max(np.abs(ra["v"] - rb["v"])) < 1e-5
        e1 = sum(a.nb_energy())
        assert abs(e1 - e0) / abs(e0) < 1e-6
    finally:
        a.nb_free()
        b.nb_free()


def test_compensated_run_against_oracle(nb):
    n = 1024
    m, x, v = plummer(n, 1)
    ctx = nb.Context(m, x, v, EPS)
    orc = oracle.Integrator(m, x, v, EPS, nthreads=8)
    try:
        steps, _ = ctx.nb_run(1.0 / 16)
        osteps, _, _ = orc.run(1.0 / 16)
        st = ctx.nb_get_state()
        assert abs(steps - osteps) <= 0.02 * osteps
        assert np.all(st["t"] == orc.t)
        assert np.max(np.abs(st["x"] - orc.x)) < 1e-6
    finally:
        ctx.nb_free()


def test_persistent_run_reports_nb_estep(nb):
    m = np.array([0.5, 0.5])
    x = np.array([[0.0, 0.0, 0.0], [1e-9, 0.0, 0.0]])
    v = np.zeros((2, 3))
    ctx = nb.nb_init(m, x, v, 0.0, nb.nb_default_opts(level_min=40))
    try:
        with pytest.raises(nb.NbError) as ei:
            nb.nb_run(ctx, 2.0 ** -37)
        assert ei.value.code == nb.NB_ESTEP
    finally:
        nb.nb_free(ctx)


@pytest.mark.parametrize("n", [1, 4097, 8193, 16384, 16385])
def test_sizes_at_the_edges(nb, n):
    # one particle; the first sizes past 64 CTAs of 64 and of 64 CTAs of 128
    # particles (new layouts); the largest persistent size; the first graph size
    m, x, v = plummer(n, 30, exact_virial_max=0)
    a = nb.Context(m, x, v, EPS, summation=nb.NB_SUM_FIXED)
    b = nb.Context(m, x, v, EPS, summation=nb.NB_SUM_FIXED, flags=nb.NB_RUN_GRAPH)
    try:
        t_end = 1.0 / 8 if n < 100 else 1.0 / 512
        sa = a.nb_run(t_end)
        sb = b.nb_run(t_end)
        assert sa == sb
        ra, rb = a.nb_get_state(), b.nb_get_state()
        for key in ra:
            assert np.array_equal(ra[key], rb[key]), key
    finally:
        a.nb_free()
        b.nb_free()


def test_bounded_wait_times_out_and_the_context_stays_usable(nb):
    # failure detection without a fault: the persistent run's wait loop on a
    # counter that nothing increments must give up after its limit, report
    # NB_ETIMEOUT, and leave the context working
    import time
    m, x, v = plummer(600, 41)
    a = nb.Context(m, x, v, EPS, summation=nb.NB_SUM_FIXED)
    b = nb.Context(m, x, v, EPS, summation=nb.NB_SUM_FIXED)
    try:
        t0 = time.perf_counter()
        with pytest.raises(nb.NbError) as ei:
            a.nb_check_wait(100)
        el = time.perf_counter() - t0
        assert ei.value.code == nb.NB_ETIMEOUT
        assert 0.05 < el < 3.0
        with pytest.raises(nb.NbError) as ei:
            a.nb_check_wait(0)
        assert ei.value.code == nb.NB_EINVAL
        a.nb_run(1.0 / 16)
        b.nb_run(1.0 / 16)
        ra, rb = a.nb_get_state(), b.nb_get_state()
        for key in ra:
            assert np.array_equal(ra[key], rb[key]), key
    finally:
        a.nb_free()
        b.nb_free()
