"""nb_force_few_noalloc: the force on a few particles for callers that may not
allocate device memory (a host that pre-partitions the GPU and forbids later
cudaMalloc calls, a real-time loop, a plug-in whose host owns the allocator).

It is checked through the C ABI against the library's regular entry point,
nb_force, on two calls in a row, within the force tolerance the other GPU
tests use, and against the FP64 oracle directly: with many j slices and a
short last slice (2^18 + 37 bodies, one and 64 active), with long per-thread
runs (64 active on 2^20 bodies), and without softening.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import os

import numpy as np
import pytest

import oracle
from synth import plummer, sample_active
from nbtest import TOL_DS, assert_force_close, nb, pair_magnitudes  # noqa: F401

pytestmark = pytest.mark.gpu

EPS = 1.0 / 256


def _noalloc(nb, torch, n, d_m, d_x, d_v, eps, idx, calls=1):
    """Runs the entry point `calls` times in a row on the same inputs (outputs
    poisoned with NaN before each call) and returns the last result; every
    call must give the same bits."""
    na = len(idx)
    d_idx = torch.from_numpy(idx).cuda()
    prev = None
    for _ in range(calls):
        d_acc = torch.full((na, 3), float("nan"), dtype=torch.float64, device="cuda")
        d_jerk = torch.full_like(d_acc, float("nan"))
        d_pot = torch.full((na,), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        nb.nb_force_few_noalloc(n, d_m, d_x, d_v, eps, d_idx, na, d_acc, d_jerk, d_pot, stream)
        torch.cuda.synchronize()
        got = (d_acc.cpu().numpy(), d_jerk.cpu().numpy(), d_pot.cpu().numpy())
        if prev is not None:
            assert all(np.array_equal(a, b) for a, b in zip(got, prev))
        prev = got
    return prev


def test_noalloc_force_matches_nb_force_on_consecutive_calls(nb):
    torch = pytest.importorskip("torch")
    n = 5003
    m, x, v = plummer(n, 21)
    ctx = nb.Context(m, x, v, EPS)
    try:
        d_m = torch.from_numpy(m).cuda()
        d_x = torch.from_numpy(x).cuda()
        d_v = torch.from_numpy(v).cuda()
        for call, na in enumerate((nb.NB_NOALLOC_MAX_ACTIVE, 7, 1, nb.NB_NOALLOC_MAX_ACTIVE)):
            idx = sample_active(n, na, 31 + call)
            ref = ctx.nb_force(idx)
            got = _noalloc(nb, torch, n, d_m, d_x, d_v, EPS, idx)
            assert np.all(np.isfinite(got[0])) and np.all(np.isfinite(got[2]))
            mags = pair_magnitudes(m, x, v, EPS, idx)
            assert_force_close(got, ref, mags, TOL_DS, "no-alloc call %d (n_active=%d)" % (call, na))
    finally:
        ctx.nb_free()


@pytest.mark.parametrize("n,na,eps", [((1 << 18) + 37, 1, EPS), ((1 << 18) + 37, 64, EPS),
                                      (1 << 20, 64, 1.0 / 1024), (5003, 64, 0.0)])
def test_noalloc_force_matches_the_oracle(nb, n, na, eps):
    # Many slices (2^18 + 37 bodies: 304 slices for one active particle, the
    # last one short), long per-thread runs (64 active on 2^20 bodies: about
    # 216 j per thread per slice) and no softening, each compared with the
    # FP64 oracle on the same particles and with nb_force, two calls in a row.
    torch = pytest.importorskip("torch")
    m, x, v = plummer(n, 23)
    idx = sample_active(n, na, 41 + na)
    d_m, d_x, d_v = (torch.from_numpy(a).cuda() for a in (m, x, v))
    got = _noalloc(nb, torch, n, d_m, d_x, d_v, eps, idx, calls=2)
    ref = oracle.force(m, x, v, eps, idx, nthreads=os.cpu_count() or 1)
    mags = pair_magnitudes(m, x, v, eps, idx, chunk=8)
    assert_force_close(got, ref, mags, TOL_DS, "no-alloc n=%d n_active=%d eps=%g" % (n, na, eps))
    ctx = nb.Context(m, x, v, eps, flags=nb.NB_INIT_NO_FORCE)
    try:
        lib_ref = ctx.nb_force(idx)
    finally:
        ctx.nb_free()
    assert_force_close(got, lib_ref, mags, TOL_DS, "no-alloc vs nb_force n=%d n_active=%d" % (n, na))


def test_noalloc_rejects_sizes_beyond_the_maximum(nb):
    torch = pytest.importorskip("torch")
    n = 100
    m, x, v = plummer(n, 22)
    d_m, d_x, d_v = (torch.from_numpy(a).cuda() for a in (m, x, v))
    too_many = nb.NB_NOALLOC_MAX_ACTIVE + 1
    d_idx = torch.arange(too_many, dtype=torch.int32, device="cuda")
    out = torch.empty((too_many, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(nb.NbError) as ei:
        nb.nb_force_few_noalloc(n, d_m, d_x, d_v, EPS, d_idx, too_many, out, None, None)
    assert ei.value.code == nb.NB_EINVAL
    with pytest.raises(nb.NbError):
        nb.nb_force_few_noalloc(n, d_m, d_x, d_v, -1.0, d_idx, 3, out, None, None)
    # tensors of the wrong type or too short are refused before the C call
    with pytest.raises(ValueError):
        nb.nb_force_few_noalloc(n, d_m, d_x.float(), d_v, EPS, d_idx, 3, out, None, None)
    with pytest.raises(ValueError):
        nb.nb_force_few_noalloc(n, d_m, d_x, d_v, EPS, d_idx.long(), 3, out, None, None)
    with pytest.raises(ValueError):
        nb.nb_force_few_noalloc(n, d_m, d_x[:50], d_v, EPS, d_idx, 3, out, None, None)
