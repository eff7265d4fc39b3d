"""Python access to the FP64 CPU oracle (``nbody_oracle.c``).

TEST INFRASTRUCTURE, NOT THE PRODUCT.  The oracle is the plain definition of
the direct N-body Hermite block-step method (Section 2 and Appendix A of the
paper) in FP64 C.  Only the tests, the smoke check and the benchmark's CPU
baseline may import this package; the CUDA library shares no code with it.

Pins (tests that tie the oracle to something other than itself) live in
``tests/test_oracle_*.py``.  Every routine here is pinned; none is "parity
unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

TICK_BITS = 40
# Summation of the force (same numbers as the library's NB_SUM_* options):
SUM_FP64 = 0           # the FP64 definition (orc_force)
SUM_FIXED = 1          # single-precision pair terms, 64-bit fixed-point sums (GRAPE-style)
SUM_FP32 = 2           # single-precision pair terms, FP32 running sum in index order
SUM_FP32_SORTED = 3    # the same, smallest pair force first
TICKS_PER_UNIT = 1 << TICK_BITS
ESTEP = -4

_lib = None

_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double


def lib():
    """Loads (building first if needed) the oracle's shared library."""
    global _lib
    if _lib is None:
        # NBODY_ORACLE_LIB lets the mutation test load a deliberately broken copy.
        path = os.environ.get("NBODY_ORACLE_LIB") or _build.build()
        L = ctypes.CDLL(path)
        L.orc_force.argtypes = [_i64, _f64p, _f64p, _f64p, _dbl, _i64, _i32p, _f64p, _f64p, _f64p, _int]
        L.orc_force.restype = None
        L.orc_energy.argtypes = [_i64, _f64p, _f64p, _f64p, _dbl, ctypes.POINTER(_dbl),
                                 ctypes.POINTER(_dbl), _int]
        L.orc_energy.restype = None
        L.orc_predict_one.argtypes = [_f64p, _f64p, _f64p, _f64p, _dbl, _f64p, _f64p]
        L.orc_predict_one.restype = None
        L.orc_correct_one.argtypes = [_f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _dbl,
                                      _f64p, _f64p, _f64p, _f64p]
        L.orc_correct_one.restype = None
        L.orc_aarseth_dt.argtypes = [_f64p, _f64p, _f64p, _f64p, _dbl, _dbl]
        L.orc_aarseth_dt.restype = _dbl
        L.orc_initial_dt.argtypes = [_f64p, _f64p, _dbl]
        L.orc_initial_dt.restype = _dbl
        L.orc_level_of.argtypes = [_dbl, _int, ctypes.POINTER(_int)]
        L.orc_level_of.restype = _int
        L.orc_next_level.argtypes = [_int, _int, _i64, _int]
        L.orc_next_level.restype = _int
        L.orc_init.argtypes = [_i64, _f64p, _f64p, _f64p, _dbl, _dbl, _int, _int, _f64p, _f64p,
                               _f64p, _i64p, _i32p, _int, _int]
        L.orc_init.restype = _int
        L.orc_next_time.argtypes = [_i64, _i64p, _i32p]
        L.orc_next_time.restype = _i64
        L.orc_step.argtypes = [_i64, _f64p, _dbl, _dbl, _int, _int, _i64, _f64p, _f64p, _f64p,
                               _f64p, _i64p, _i32p, _i32p, ctypes.POINTER(_i64), ctypes.c_void_p,
                               _int, _int]
        L.orc_step.restype = _i64
        L.orc_run.argtypes = [_i64, _f64p, _dbl, _dbl, _int, _int, _i64, _i64, _f64p, _f64p,
                              _f64p, _f64p, _i64p, _i32p, ctypes.c_void_p, ctypes.POINTER(_i64),
                              _int, _int]
        L.orc_run.restype = _i64
        L.orc_force_vjp.argtypes = [_i64, _f64p, _f64p, _f64p, _dbl, _f64p, _f64p, _f64p, _f64p,
                                    _f64p]
        L.orc_force_vjp.restype = None
        L.orc_traj_vjp.argtypes = [_i64, _f64p, _f64p, _f64p, _dbl, _dbl, _i64, _f64p, _f64p, _f64p,
                                   _f64p, _f64p]
        L.orc_traj_vjp.restype = _int
        L.orc_force_summed.argtypes = [_int, _i64, _f64p, _f64p, _f64p, _dbl, _i64, _i32p, _f64p,
                                       _f64p, _f64p, _int]
        L.orc_force_summed.restype = _int
        L.orc_fixed_scales.argtypes = [_i64, _f64p, _f64p, _dbl, _i32p]
        L.orc_fixed_scales.restype = _int
        L.orc_pair_terms32.argtypes = [_i64, _f64p, _f64p, _f64p, _dbl, _i64, _int, _f32p, _f32p,
                                       _i32p]
        L.orc_pair_terms32.restype = _int
        L.orc_max_threads.argtypes = []
        L.orc_max_threads.restype = _int
        _lib = L
    return _lib


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def max_threads() -> int:
    return int(lib().orc_max_threads())


def force(m, x, v, eps, idx=None, nthreads=1):
    """acc[n_act,3], jerk[n_act,3], pot[n_act] on the listed i (all if None)."""
    m, x, v = _c(m), _c(x), _c(v)
    n = m.shape[0]
    idx = np.arange(n, dtype=np.int32) if idx is None else _c(idx, np.int32)
    na = idx.shape[0]
    acc = np.zeros((na, 3))
    jerk = np.zeros((na, 3))
    pot = np.zeros(na)
    lib().orc_force(n, m, x, v, float(eps), na, idx, acc, jerk, pot, int(nthreads))
    return acc, jerk, pot


def force_summed(m, x, v, eps, idx=None, mode=SUM_FIXED, nthreads=1):
    """acc, jerk, pot on the listed i with a summation variant (SUM_FIXED,
    SUM_FP32 or SUM_FP32_SORTED) of the single-precision pair terms."""
    m, x, v = _c(m), _c(x), _c(v)
    n = m.shape[0]
    idx = np.arange(n, dtype=np.int32) if idx is None else _c(idx, np.int32)
    na = idx.shape[0]
    acc = np.zeros((na, 3))
    jerk = np.zeros((na, 3))
    pot = np.zeros(na)
    rc = lib().orc_force_summed(int(mode), n, m, x, v, float(eps), na, idx, acc, jerk, pot,
                                int(nthreads))
    if rc != 0:
        raise ValueError("summation variant %d rejected the input (%d)" % (mode, rc))
    return acc, jerk, pot


def fixed_scales(m, v, eps):
    """(s_acc, s_jerk, s_pot): fixed-point units 2^-s of the GRAPE-style sums."""
    s = np.zeros(3, dtype=np.int32)
    rc = lib().orc_fixed_scales(_c(m).shape[0], _c(m), _c(v), float(eps), s)
    if rc != 0:
        raise ValueError("no fixed-point scales for this input (%d)" % rc)
    return tuple(int(q) for q in s)


def pair_terms32(m, x, v, eps, i, scaled=False):
    """Single-precision pair terms of every j on particle i: (t[n][7] float32,
    key[n] float32, ok[n] bool); scaled=True applies the fixed-point scales."""
    m, x, v = _c(m), _c(x), _c(v)
    n = m.shape[0]
    t = np.zeros((n, 7), dtype=np.float32)
    key = np.zeros(n, dtype=np.float32)
    ok = np.zeros(n, dtype=np.int32)
    rc = lib().orc_pair_terms32(n, m, x, v, float(eps), int(i), int(bool(scaled)), t, key, ok)
    if rc != 0:
        raise ValueError("no fixed-point scales for this input (%d)" % rc)
    return t, key, ok.astype(bool)


def energy(m, x, v, eps, nthreads=1):
    """(T, W) with the softened potential energy."""
    ek, ep = _dbl(), _dbl()
    m, x, v = _c(m), _c(x), _c(v)
    lib().orc_energy(m.shape[0], m, x, v, float(eps), ctypes.byref(ek), ctypes.byref(ep),
                     int(nthreads))
    return ek.value, ep.value


def force_vjp(m, x, v, eps, abar, kbar):
    """(xbar, vbar, mbar): VJP of every particle's acc and jerk w.r.t. x, v, m."""
    m, x, v = _c(m), _c(x), _c(v)
    n = m.shape[0]
    xb, vb, mb = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
    lib().orc_force_vjp(n, m, x, v, float(eps), _c(abar), _c(kbar), xb, vb, mb)
    return xb, vb, mb


def traj_vjp(m, x0, v0, eps, dt, steps, xbar_T, vbar_T):
    """Fixed shared-step Hermite trajectory from (x0, v0): returns
    (x_T, v_T, xbar_0, vbar_0, mbar) for cotangents (xbar_T, vbar_T)."""
    m = _c(m)
    n = m.shape[0]
    x, v = _c(x0).copy(), _c(v0).copy()
    xb, vb, mb = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
    rc = lib().orc_traj_vjp(n, m, x, v, float(eps), float(dt), int(steps), _c(xbar_T), _c(vbar_T),
                            xb, vb, mb)
    if rc != 0:
        raise RuntimeError("oracle trajectory failed: %d" % rc)
    return x, v, xb, vb, mb


def traj_final(m, x0, v0, eps, dt, steps):
    """Final (x, v) of the fixed shared-step trajectory (no gradient)."""
    n = _c(m).shape[0]
    z = np.zeros((n, 3))
    x, v, _, _, _ = traj_vjp(m, x0, v0, eps, dt, steps, z, z)
    return x, v


def predict_one(x, v, a, k, dt):
    xp, vp = np.zeros(3), np.zeros(3)
    lib().orc_predict_one(_c(x), _c(v), _c(a), _c(k), float(dt), xp, vp)
    return xp, vp


def correct_one(xp, vp, a, k, ap, kp, dt):
    x, v, a2, a3 = np.zeros(3), np.zeros(3), np.zeros(3), np.zeros(3)
    lib().orc_correct_one(_c(xp), _c(vp), _c(a), _c(k), _c(ap), _c(kp), float(dt), x, v, a2, a3)
    return x, v, a2, a3


def aarseth_dt(a1, k1, a2, a3, dt, eta):
    return float(lib().orc_aarseth_dt(_c(a1), _c(k1), _c(a2), _c(a3), float(dt), float(eta)))


def initial_dt(a, k, eta_init):
    return float(lib().orc_initial_dt(_c(a), _c(k), float(eta_init)))


def level_of(dt_raw, kmin=3):
    """(status, level) of the largest power-of-two step <= dt_raw."""
    lv = _int()
    rc = lib().orc_level_of(float(dt_raw), int(kmin), ctypes.byref(lv))
    return int(rc), int(lv.value)


def next_level(k_old, k_q, t_new, kmin=3):
    return int(lib().orc_next_level(int(k_old), int(k_q), int(t_new), int(kmin)))


def time_to_ticks(t: float) -> int:
    ticks = t * TICKS_PER_UNIT
    if ticks != math.floor(ticks):
        raise ValueError("time is not on the 2^-40 tick grid")
    return int(ticks)


class Integrator:
    """FP64 Hermite block-step integrator state (the oracle's step loop)."""

    def __init__(self, m, x, v, eps, eta=0.01, eta_init=0.01, kmin=3, kfix=0, nthreads=1,
                 summation=SUM_FP64):
        self.m = _c(m).copy()
        self.x = _c(x).copy()
        self.v = _c(v).copy()
        self.n = self.m.shape[0]
        self.eps, self.eta, self.eta_init = float(eps), float(eta), float(eta_init)
        self.kmin, self.kfix, self.nthreads = int(kmin), int(kfix), int(nthreads)
        self.summation = int(summation)
        self.a = np.zeros((self.n, 3))
        self.k = np.zeros((self.n, 3))
        self.pot = np.zeros(self.n)
        self.t = np.zeros(self.n, dtype=np.int64)
        self.lev = np.zeros(self.n, dtype=np.int32)
        rc = lib().orc_init(self.n, self.m, self.x, self.v, self.eps, self.eta_init, self.kmin,
                            self.kfix, self.a, self.k, self.pot, self.t, self.lev, self.nthreads,
                            self.summation)
        if rc != 0:
            raise RuntimeError("oracle init failed: %d" % rc)
        self._act = np.zeros(self.n, dtype=np.int32)

    def step(self, t_end_ticks=None):
        """One block step: returns (block time in ticks, ascending active indices)."""
        t_end = (1 << 62) if t_end_ticks is None else int(t_end_ticks)
        tn = _i64()
        pot = np.zeros(self.n)
        na = lib().orc_step(self.n, self.m, self.eps, self.eta, self.kmin, self.kfix, t_end,
                            self.x, self.v, self.a, self.k, self.t, self.lev, self._act,
                            ctypes.byref(tn), pot.ctypes.data_as(ctypes.c_void_p), self.nthreads,
                            self.summation)
        if na < 0:
            raise RuntimeError("oracle step failed: %d" % na)
        act = self._act[:na].copy()
        self.pot[act] = pot[act]
        return int(tn.value), act

    def run(self, t_end, max_steps=1 << 40):
        """Steps until all particles reach t_end; returns (steps, interactions, hist)."""
        t_end_ticks = time_to_ticks(t_end)
        cap = int(min(max_steps, 1 << 21))
        hist = np.zeros(cap, dtype=np.int32)
        inter = _i64()
        steps = lib().orc_run(self.n, self.m, self.eps, self.eta, self.kmin, self.kfix,
                              t_end_ticks, cap, self.x, self.v, self.a, self.k, self.t, self.lev,
                              hist.ctypes.data_as(ctypes.c_void_p), ctypes.byref(inter),
                              self.nthreads, self.summation)
        if steps < 0:
            raise RuntimeError("oracle run failed: %d" % steps)
        return int(steps), int(inter.value), hist[:steps].copy()

    def energy(self):
        ek, ep = energy(self.m, self.x, self.v, self.eps, self.nthreads)
        return ek + ep

    def synchronised(self):
        return bool(np.all(self.t == self.t[0]))
