"""Parity of the ensemble path (many clusters, one launch per ensemble step)
with the FP64 oracle and with the single-system path.

Clusters: Salpeter masses, virial ratio 0.3-0.7, N from 1 to a few thousand.
Start-up forces are checked per cluster with the force error metric; the first
ensemble step must pick each cluster's block exactly and correct it bit for
bit (given the GPU's own forces, as in the single-system test); energies over
a run are checked against the oracle's own runs of the same clusters.
"""
import math

import numpy as np
import pytest

import oracle
from synth import ensemble, ensemble_member, plummer
from nbtest import TOL_DS, assert_force_close, nb, pair_magnitudes  # noqa: F401

pytestmark = pytest.mark.gpu

EPS = 1.0 / 256
T = oracle.TICKS_PER_UNIT


def _flatten(clusters):
    off = np.zeros(len(clusters) + 1, dtype=np.int64)
    for c, (m, _, _) in enumerate(clusters):
        off[c + 1] = off[c] + m.shape[0]
    m = np.concatenate([c[0] for c in clusters])
    x = np.concatenate([c[1] for c in clusters])
    v = np.concatenate([c[2] for c in clusters])
    return off, m, x, v


def _clusters():
    cl = ensemble(10, 3, n_lo=32, n_hi=1500)
    cl.append(plummer(1, 4))           # a lone particle
    cl.append(plummer(2, 5))
    cl.append(plummer(4096, 6, exact_virial_max=0))  # the largest allowed
    return cl


@pytest.mark.parametrize("threads,gmax", [(512, 8), (256, 1), (128, 32)])
def test_startup_force_and_levels(nb, threads, gmax):
    cl = _clusters()
    off, m, x, v = _flatten(cl)
    e = nb.Ensemble(off, m, x, v, EPS)
    try:
        e.nb_ens_configure(threads, gmax)
        acc, jerk, pot = e.nb_ens_force()
        st = e.nb_ens_get_state()
    finally:
        e.nb_ens_free()
    for c, (mc, xc, vc) in enumerate(cl):
        s, t = off[c], off[c + 1]
        if t - s < 2:
            assert np.all(acc[s:t] == 0) and np.all(jerk[s:t] == 0)
            continue
        ref = oracle.force(mc, xc, vc, EPS, nthreads=8)
        idx = np.arange(t - s)
        mags = pair_magnitudes(mc, xc, vc, EPS, idx)
        assert_force_close((acc[s:t], jerk[s:t], pot[s:t]), ref, mags, TOL_DS, "cluster %d" % c)
    # start-up levels follow from the start-up forces exactly
    for i in range(0, off[-1], 7):
        rc, lv = oracle.level_of(oracle.initial_dt(st["a"][i], st["k"][i], 0.01), 3)
        assert rc == 0 and st["level"][i] == lv


def test_first_step_blocks_and_corrector_bit_exact(nb):
    cl = _clusters()
    off, m, x, v = _flatten(cl)
    e = nb.Ensemble(off, m, x, v, EPS)
    try:
        before = e.nb_ens_get_state()
        e.nb_ens_step()
        after = e.nb_ens_get_state()
    finally:
        e.nb_ens_free()
    for c in range(len(cl)):
        s, t = off[c], off[c + 1]
        ends = before["t"][s:t] + (np.int64(1) << (40 - before["level"][s:t].astype(np.int64)))
        tn = ends.min()
        act = np.nonzero(ends == tn)[0] + s
        rest = np.setdiff1d(np.arange(s, t), act)
        assert np.all(after["t"][act] == tn) and np.array_equal(after["t"][rest], before["t"][rest])
        assert after["steps"][c] == 1 and after["interactions"][c] == len(act) * (t - s - 1)
        for i in act[:50]:
            dt = (tn - before["t"][i]) / T
            xp, vp = oracle.predict_one(before["x"][i], before["v"][i], before["a"][i], before["k"][i], dt)
            xc, vc, a2, a3 = oracle.correct_one(xp, vp, before["a"][i], before["k"][i],
                                                after["a"][i], after["k"][i], dt)
            assert np.array_equal(after["x"][i], xc) and np.array_equal(after["v"][i], vc)
            rc, kq = oracle.level_of(oracle.aarseth_dt(after["a"][i], after["k"][i], a2, a3, dt, 0.01), 3)
            assert after["level"][i] == oracle.next_level(int(before["level"][i]), kq, int(tn), 3)
        for i in rest[:20]:
            assert np.array_equal(after["x"][i], before["x"][i])


def test_deterministic_under_dynamic_scheduling(nb):
    cl = ensemble(40, 7, n_lo=16, n_hi=600)
    off, m, x, v = _flatten(cl)
    runs = []
    for _ in range(2):
        e = nb.Ensemble(off, m, x, v, EPS)
        try:
            e.nb_ens_run(1.0, max_launches=60)
            runs.append(e.nb_ens_get_state())
        finally:
            e.nb_ens_free()
    for key in runs[0]:
        assert np.array_equal(runs[0][key], runs[1][key]), key


def test_energy_over_one_time_unit_vs_oracle_runs(nb):
    cl = ensemble(8, 11, n_lo=32, n_hi=200)
    off, m, x, v = _flatten(cl)
    e = nb.Ensemble(off, m, x, v, EPS)
    try:
        k0, p0 = e.nb_ens_energy()
        launches, inter = e.nb_ens_run(1.0)
        k1, p1 = e.nb_ens_energy()
        st = e.nb_ens_get_state()
    finally:
        e.nb_ens_free()
    assert np.all(st["t"] == T)
    for c, (mc, xc, vc) in enumerate(cl):
        ek, ep = oracle.energy(mc, xc, vc, EPS)
        assert abs(k0[c] + p0[c] - (ek + ep)) <= 1e-12 * abs(ek + ep)
        it = oracle.Integrator(mc, xc, vc, EPS)
        E0 = it.energy()
        steps, _, _ = it.run(1.0)
        d_orc = abs(it.energy() - E0) / abs(E0)
        d_gpu = abs(k1[c] + p1[c] - (k0[c] + p0[c])) / abs(k0[c] + p0[c])
        assert d_gpu <= max(1e-6, 3 * d_orc), (c, d_gpu, d_orc)
        assert abs(st["steps"][c] - steps) <= 0.05 * steps + 5
    # launches go out in batches of 32 between completion checks
    assert st["steps"].max() + 1 <= launches < st["steps"].max() + 1 + 32


def test_energy_outliers_match_the_oracle(nb):
    # The clusters of the 4096-cluster benchmark ensemble (seed 5) whose energy
    # the GPU conserves worst (358 and 114 bodies; close pairs of massive
    # stars, the encounters Section 2 leaves out), next to two ordinary ones.
    # The oracle's FP64 integrator must show the same error on the same
    # cluster: the outliers are the method's, not the GPU's.
    picks = (2923, 1231, 7, 100)
    cl = [ensemble_member(4096, 5, ci) for ci in picks]
    off, m, x, v = _flatten(cl)
    e = nb.Ensemble(off, m, x, v, EPS)
    try:
        k0, p0 = e.nb_ens_energy()
        e.nb_ens_run(1.0)
        k1, p1 = e.nb_ens_energy()
    finally:
        e.nb_ens_free()
    for c, (mc, xc, vc) in enumerate(cl):
        it = oracle.Integrator(mc, xc, vc, EPS, nthreads=8)
        E0 = it.energy()
        it.run(1.0)
        d_orc = abs(it.energy() - E0) / abs(E0)
        d_gpu = abs(k1[c] + p1[c] - (k0[c] + p0[c])) / abs(k0[c] + p0[c])
        assert d_gpu <= max(1e-6, 3 * d_orc), (picks[c], d_gpu, d_orc)
        if c < 2:
            # a real outlier of the integrator, reproduced within a factor 3
            assert d_orc > 1e-5 and d_gpu >= d_orc / 3, (picks[c], d_gpu, d_orc)


def test_matches_single_system_path(nb):
    mc, xc, vc = ensemble(1, 13, n_lo=700, n_hi=700)[0]
    off = np.array([0, mc.shape[0]])
    e = nb.Ensemble(off, mc, xc, vc, EPS)
    ctx = nb.Context(mc, xc, vc, EPS)
    try:
        e.nb_ens_run(0.125)
        ctx.nb_run(0.125)
        a, b = e.nb_ens_get_state(), ctx.nb_get_state()
        assert np.array_equal(a["t"], b["t"])
        assert np.abs(a["x"] - b["x"]).max() < 1e-6
        ea = sum(x_[0] for x_ in e.nb_ens_energy())
        eb = sum(ctx.nb_energy())
        assert abs(ea - eb) < 1e-7 * abs(eb)
    finally:
        e.nb_ens_free()
        ctx.nb_free()


def test_tune_keeps_state_and_picks_a_candidate(nb):
    cl = ensemble(24, 17, n_lo=32, n_hi=1000)
    off, m, x, v = _flatten(cl)
    e = nb.Ensemble(off, m, x, v, EPS)
    try:
        before = e.nb_ens_get_state()
        th, g, ms = e.nb_ens_tune(3)
        after = e.nb_ens_get_state()
        assert th in (128, 256, 512) and g in (1, 2, 4, 8, 16, 32) and ms > 0
        for key in before:
            assert np.array_equal(before[key], after[key]), key
    finally:
        e.nb_ens_free()


def test_bad_arguments(nb):
    m, x, v = plummer(10, 1)
    for off in ([1, 10], [0, 5, 4], [0, 10, 5000]):
        with pytest.raises((nb.NbError, ValueError)):
            mm = np.resize(m, max(off[-1], 1))
            nb.Ensemble(np.array(off), mm, np.resize(x, (max(off[-1], 1), 3)),
                        np.resize(v, (max(off[-1], 1), 3)), EPS)
    big = plummer(4097, 2, exact_virial_max=0)
    with pytest.raises(nb.NbError) as ei:
        nb.Ensemble(np.array([0, 4097]), *big, EPS)
    assert ei.value.code == nb.NB_EINVAL
