"""Shared helpers of the GPU parity tests.

Error metric for the force (FP32 pair arithmetic cannot give a small relative
error on an acceleration that nearly cancels, e.g. at the cluster centre):
  err_a,i = |a_gpu,i - a_ref,i| / max(|a_ref,i|, S_a,i / 10)
with S_a,i = sum_j |m_j dx / r^3| the sum of the pair magnitudes, and the same
for the jerk with S_k,i = sum_j |k_ij|.  The potential is a sum of terms of
one sign, so its plain relative error is used.  Tolerances (per particle):
DS 2e-6 (acc, pot) and 1e-5 (jerk); FP64 1e-12.
"""
import numpy as np
import pytest

TOL_DS = {"acc": 2e-6, "jerk": 1e-5, "pot": 2e-6}
TOL_F64 = {"acc": 1e-12, "jerk": 1e-12, "pot": 1e-12}


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def nb():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_cs_0702135_gb300 import build
    build.build()
    import paper_cs_0702135_gb300 as nbmod
    nbmod.lib()
    return nbmod


def pair_magnitudes(m, x, v, eps, idx, chunk=32):
    """S_a, S_k per listed i (sums of |pair acc| and |pair jerk|), j != i."""
    sa = np.empty(len(idx))
    sk = np.empty(len(idx))
    for s in range(0, len(idx), chunk):
        ii = np.asarray(idx[s:s + chunk])
        d = x[None, :, :] - x[ii, None, :]
        w = v[None, :, :] - v[ii, None, :]
        r2 = np.einsum("ijk,ijk->ij", d, d) + eps * eps
        rv = np.einsum("ijk,ijk->ij", d, w)
        with np.errstate(divide="ignore", invalid="ignore"):
            rinv = 1.0 / np.sqrt(r2)
            r3 = rinv ** 3
            fa = m[None, :] * np.sqrt(r2 - eps * eps) * r3
            kk = m[None, :, None] * (w * r3[..., None] - 3 * rv[..., None] * d * (r3 * rinv * rinv)[..., None])
            fk = np.linalg.norm(kk, axis=2)
        rows = np.arange(len(ii))
        fa[rows, ii] = 0.0
        fk[rows, ii] = 0.0
        sa[s:s + len(ii)] = np.nansum(fa, axis=1)
        sk[s:s + len(ii)] = np.nansum(fk, axis=1)
    return sa, sk


def force_errors(got, ref, mags):
    """Per-particle errors (err_a, err_k, err_p) of got=(acc, jerk, pot) vs ref."""
    sa, sk = mags
    ea = np.linalg.norm(got[0] - ref[0], axis=1) / np.maximum(np.linalg.norm(ref[0], axis=1), sa / 10)
    ek = np.linalg.norm(got[1] - ref[1], axis=1) / np.maximum(np.linalg.norm(ref[1], axis=1), sk / 10)
    ep = np.abs(got[2] - ref[2]) / np.abs(ref[2])
    return ea, ek, ep


def assert_force_close(got, ref, mags, tol, label=""):
    ea, ek, ep = force_errors(got, ref, mags)
    msg = "%s max err acc %.3g jerk %.3g pot %.3g" % (label, ea.max(), ek.max(), ep.max())
    assert ea.max() <= tol["acc"], msg
    assert ek.max() <= tol["jerk"], msg
    assert ep.max() <= tol["pot"], msg
    return ea.max(), ek.max(), ep.max()
