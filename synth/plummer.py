"""Seeded synthetic initial conditions: Plummer spheres in N-body units.

The paper's workload (Section 4, "Results") is an equal-mass Plummer (1911)
sphere drawn with the method of Aarseth, Henon & Wielen (1974) and scaled to
virial equilibrium, run in standard N-body units (G = M = 1, E = -1/4;
Heggie & Mathieu 1986).  This module builds that input and nothing else: it
contains none of the force, predictor, corrector or time-step arithmetic.

Sampling, in Plummer units (scale radius 1, G = M = 1):

* radius from the enclosed-mass fraction X1 ~ U(0,1):
  r = (X1^(-2/3) - 1)^(-1/2); a draw whose N-body radius exceeds ``r_cut``
  (22.8) is redrawn;
* isotropic direction: z = (1 - 2 X2) r, azimuth 2 pi X3;
* speed q * v_esc with v_esc = sqrt(2) (1 + r^2)^(-1/4) and q drawn by von
  Neumann rejection against g(q) = q^2 (1 - q^2)^(7/2) < 0.1;
* isotropic velocity direction from X6, X7.

Then lengths are multiplied by 3 pi / 16 and speeds by sqrt(16 / (3 pi)) (the
Plummer model's energy is -3 pi / 64 in Plummer units), the centre of mass is
moved to rest at the origin, and, for N <= ``exact_virial_max``, positions and
velocities are rescaled so that the realisation has exactly T = 1/4 and
W = -1/2 (unsoftened).  Above that size the O(N^2) rescale is skipped and the
analytic unit conversion alone sets the scale (E = -1/4 in expectation).
"""
from __future__ import annotations

import math

import numpy as np

from . import rng

# Independent streams, one per kind of draw.
_S_RADIUS, _S_POSDIR, _S_SPEED, _S_VELDIR, _S_ACTIVE = 1, 2, 3, 4, 5
_S_ENS_N, _S_ENS_IMF, _S_ENS_Q, _S_PAIRS = 11, 12, 13, 14

_ATTEMPTS = 1 << 16          # counter space reserved per particle for redraws
LENGTH_UNIT = 3.0 * math.pi / 16.0
SPEED_UNIT = math.sqrt(16.0 / (3.0 * math.pi))


def _draw_radius(n: int, seed: int, r_cut: float) -> np.ndarray:
    r = np.empty(n)
    pending = np.arange(n, dtype=np.int64)
    attempt = 0
    while pending.size:
        x1 = rng.uniform(seed, _S_RADIUS, pending * _ATTEMPTS + attempt)
        with np.errstate(divide="ignore"):
            rr = 1.0 / np.sqrt(x1 ** (-2.0 / 3.0) - 1.0)
        ok = rr * LENGTH_UNIT <= r_cut
        r[pending[ok]] = rr[ok]
        pending = pending[~ok]
        attempt += 1
        if attempt >= _ATTEMPTS:
            raise RuntimeError("radius rejection did not terminate")
    return r


def _draw_q(n: int, seed: int) -> np.ndarray:
    q = np.empty(n)
    pending = np.arange(n, dtype=np.int64)
    attempt = 0
    while pending.size:
        base = (pending * _ATTEMPTS + attempt) * 2
        x4 = rng.uniform(seed, _S_SPEED, base)
        x5 = rng.uniform(seed, _S_SPEED, base + 1)
        ok = 0.1 * x5 < x4 * x4 * (1.0 - x4 * x4) ** 3.5
        q[pending[ok]] = x4[ok]
        pending = pending[~ok]
        attempt += 1
        if attempt >= _ATTEMPTS:
            raise RuntimeError("speed rejection did not terminate")
    return q


def _isotropic(length: np.ndarray, seed: int, stream: int) -> np.ndarray:
    n = length.shape[0]
    c = np.arange(n, dtype=np.int64) * 2
    u = rng.uniform(seed, stream, c)
    w = rng.uniform(seed, stream, c + 1)
    z = (1.0 - 2.0 * u) * length
    rho = np.sqrt(np.maximum(length * length - z * z, 0.0))
    phi = 2.0 * math.pi * w
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def kinetic_energy(m: np.ndarray, v: np.ndarray) -> float:
    return 0.5 * float(np.sum(m * np.einsum("ij,ij->i", v, v)))


def unsoftened_potential_energy(m: np.ndarray, x: np.ndarray, chunk: int = 1024) -> float:
    """W = -sum_{i<j} m_i m_j / |x_i - x_j|, used only to scale the realisation."""
    n = m.shape[0]
    w = 0.0
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        d = x[s:e, None, :] - x[None, :, :]
        r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
        rows = np.arange(s, e)
        r[rows - s, rows] = np.inf
        w -= float(np.sum(m[s:e, None] * m[None, :] / r))
    return 0.5 * w


def sampled_potential_energy(m: np.ndarray, x: np.ndarray, seed: int, pairs: int) -> float:
    """W estimated from `pairs` uniformly drawn pairs i != j (seeded):
    W ~ -(n (n - 1) / 2) * mean(m_i m_j / |x_i - x_j|); relative error ~ pairs^-1/2."""
    n = m.shape[0]
    c = np.arange(pairs, dtype=np.int64)
    i = (rng.u64(seed, _S_PAIRS, 2 * c) % np.uint64(n)).astype(np.int64)
    j = (rng.u64(seed, _S_PAIRS, 2 * c + 1) % np.uint64(n - 1)).astype(np.int64)
    j = j + (j >= i)
    r = np.linalg.norm(x[i] - x[j], axis=1)
    return -0.5 * n * (n - 1) * float(np.mean(m[i] * m[j] / r))


def plummer(n: int, seed: int, r_cut: float = 22.8, masses: np.ndarray | None = None,
            virial_ratio: float = 0.5, exact_virial_max: int = 16384, sample_pairs: int = 0):
    """Plummer sphere of ``n`` bodies; returns (m[n], x[n,3], v[n,3]) in float64.

    ``masses`` (normalised to total 1) replaces the equal masses 1/n.  With
    unequal masses or ``virial_ratio`` Q != 1/2 the realisation is always
    rescaled exactly, to W = -1/2 and T = Q / 2 (Q = T / |W|).
    """
    if n < 1:
        raise ValueError("n must be positive")
    r = _draw_radius(n, seed, r_cut)
    x = _isotropic(r, seed, _S_POSDIR)
    q = _draw_q(n, seed)
    speed = q * math.sqrt(2.0) * (1.0 + r * r) ** -0.25
    v = _isotropic(speed, seed, _S_VELDIR)
    x *= LENGTH_UNIT
    v *= SPEED_UNIT
    if masses is None:
        m = np.full(n, 1.0 / n)
    else:
        m = np.asarray(masses, dtype=np.float64).copy()
        m /= m.sum()
    x -= (m[:, None] * x).sum(axis=0) / m.sum()
    v -= (m[:, None] * v).sum(axis=0) / m.sum()
    if n >= 2 and (n <= exact_virial_max or masses is not None or virial_ratio != 0.5):
        if n > exact_virial_max and sample_pairs > 0:
            w = sampled_potential_energy(m, x, seed, sample_pairs)
        else:
            w = unsoftened_potential_energy(m, x)
        t = kinetic_energy(m, v)
        x *= w / -0.5
        v *= math.sqrt(0.5 * virial_ratio / t)
    return np.ascontiguousarray(m), np.ascontiguousarray(x), np.ascontiguousarray(v)


def sample_active(n: int, n_active: int, seed: int) -> np.ndarray:
    """``n_active`` distinct indices of [0, n) drawn uniformly, ascending int32."""
    if not 0 <= n_active <= n:
        raise ValueError("n_active out of range")
    keys = rng.u64(seed, _S_ACTIVE, np.arange(n, dtype=np.int64))
    pick = np.argsort(keys, kind="stable")[:n_active]
    return np.sort(pick).astype(np.int32)


def salpeter_masses(n: int, seed: int, stream_offset: int = 0, slope: float = -2.35,
                    m_lo: float = 0.1, m_hi: float = 100.0) -> np.ndarray:
    """Masses from dN/dm ~ m^slope on [m_lo, m_hi] by inverse CDF, sum = 1."""
    u = rng.uniform(seed, _S_ENS_IMF + 16 * stream_offset, np.arange(n, dtype=np.int64))
    a = slope + 1.0
    lo, hi = m_lo ** a, m_hi ** a
    m = (lo + u * (hi - lo)) ** (1.0 / a)
    return m / m.sum()


def _ensemble_cluster(job):
    nc, sub, q = job
    m = salpeter_masses(nc, sub)
    return plummer(nc, sub, masses=m, virial_ratio=q, exact_virial_max=1024, sample_pairs=200000)


def _ensemble_jobs(n_clusters, seed, n_lo, n_hi, q_lo, q_hi):
    c = np.arange(n_clusters, dtype=np.int64)
    un = rng.uniform(seed, _S_ENS_N, c)
    sizes = np.floor(np.exp(math.log(n_lo) + un * (math.log(n_hi + 1) - math.log(n_lo)))).astype(np.int64)
    sizes = np.clip(sizes, n_lo, n_hi)
    uq = rng.uniform(seed, _S_ENS_Q, c)
    return [(int(sizes[ci]), (seed * 1000003 + ci) & 0x7FFFFFFFFFFFFFFF,
             float(q_lo + uq[ci] * (q_hi - q_lo))) for ci in range(n_clusters)]


def ensemble_member(n_clusters: int, seed: int, index: int, n_lo: int = 32, n_hi: int = 4096,
                    q_lo: float = 0.3, q_hi: float = 0.7):
    """Cluster ``index`` of ``ensemble(n_clusters, seed, ...)`` alone, bit for bit."""
    return _ensemble_cluster(_ensemble_jobs(n_clusters, seed, n_lo, n_hi, q_lo, q_hi)[index])


def ensemble(n_clusters: int, seed: int, n_lo: int = 32, n_hi: int = 4096,
             q_lo: float = 0.3, q_hi: float = 0.7, workers: int = 1):
    """Independent clusters: N log-uniform in [n_lo, n_hi], Salpeter masses,
    virial ratio uniform in [q_lo, q_hi].  Returns a list of (m, x, v).  Clusters
    above 1024 bodies are scaled with W estimated from 2e5 sampled pairs.
    Every cluster draws from its own counter-based streams, so ``workers`` > 1
    (processes started by spawn) gives the same clusters."""
    jobs = _ensemble_jobs(n_clusters, seed, n_lo, n_hi, q_lo, q_hi)
    if workers > 1 and n_clusters > 1:
        import multiprocessing
        with multiprocessing.get_context("spawn").Pool(workers) as pool:
            return pool.map(_ensemble_cluster, jobs, chunksize=max(1, n_clusters // (8 * workers)))
    return [_ensemble_cluster(j) for j in jobs]
