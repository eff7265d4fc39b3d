"""Python binding of the C ABI in ``include/nb.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does
nothing but convert arguments: all work runs in ``libnb_gb300.so``.  The
library must have been built (``__graft_entry__.build()`` or
``python -m paper_cs_0702135_gb300.build``); loading fails loudly otherwise,
and there is no fallback implementation.

Device-pointer variants accept torch CUDA tensors; pass the tensor's stream as
``stream`` in the options (``torch.cuda.current_stream().cuda_stream``) when
mixing the library with torch work on the same data.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libnb_gb300.so")

NB_OK, NB_EINVAL, NB_ENOMEM, NB_ECUDA, NB_ESTEP, NB_ETIMEOUT, NB_ESTATE = 0, -1, -2, -3, -4, -5, -6
NB_DS, NB_FP64 = 0, 1
NB_FORCE_AUTO, NB_FORCE_IPAR, NB_FORCE_JPAR = 0, 1, 2
NB_SUM_COMPENSATED, NB_SUM_FIXED, NB_SUM_FP32, NB_SUM_FP32_SORTED = 0, 1, 2, 3
NB_TICK_BITS = 40
NB_INIT_NO_FORCE = 1
NB_RUN_GRAPH = 2
NB_NOALLOC_MAX_ACTIVE = 64
TICKS_PER_UNIT = 1 << NB_TICK_BITS

_ERRNAMES = {NB_EINVAL: "NB_EINVAL", NB_ENOMEM: "NB_ENOMEM", NB_ECUDA: "NB_ECUDA",
             NB_ESTEP: "NB_ESTEP", NB_ETIMEOUT: "NB_ETIMEOUT", NB_ESTATE: "NB_ESTATE"}


class NbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_ERRNAMES.get(code, "error"), code, msg))
        self.code = code


class nb_opts(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("eta_init", ctypes.c_double),
                ("level_min", ctypes.c_int), ("level_fixed", ctypes.c_int),
                ("precision", ctypes.c_int), ("force_mode", ctypes.c_int),
                ("split_j", ctypes.c_int), ("flags", ctypes.c_int),
                ("summation", ctypes.c_int), ("stream", ctypes.c_void_p)]


class nb_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("interactions", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("force_launches", ctypes.c_int64),
                ("force_ms", ctypes.c_double)]


_c_dp = ctypes.POINTER(ctypes.c_double)
_c_ip = ctypes.POINTER(ctypes.c_int32)
_c_lp = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p
_lib = None

# (name, restype, argtypes) of every entry point of include/nb.h
SIGNATURES = [
    ("nb_default_opts", None, [ctypes.POINTER(nb_opts)]),
    ("nb_init", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int64, _vp, _vp, _vp, ctypes.c_double,
                               ctypes.POINTER(nb_opts)]),
    ("nb_init_dev", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int64, _vp, _vp, _vp,
                                   ctypes.c_double, ctypes.POINTER(nb_opts)]),
    ("nb_get_state_dev", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("nb_traj_backward_dev", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    ("nb_predict", ctypes.c_int, [_vp, ctypes.c_double]),
    ("nb_force", ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp, _vp, _vp]),
    ("nb_force_dev", ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp, _vp, _vp]),
    ("nb_correct", ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.c_double, _vp, _vp]),
    ("nb_step", ctypes.c_int, [_vp, _c_dp, _c_ip]),
    ("nb_check_wait", ctypes.c_int, [_vp, ctypes.c_int32]),
    ("nb_run", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int64, _c_lp, _c_lp]),
    ("nb_energy", ctypes.c_int, [_vp, _c_dp, _c_dp]),
    ("nb_get_state", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("nb_set_state", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("nb_get_active", ctypes.c_int, [_vp, _vp, ctypes.c_int32, _c_ip, _c_lp]),
    ("nb_force_vjp", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    ("nb_traj_forward", ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int64]),
    ("nb_traj_backward", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    ("nb_ens_init", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int32, _vp, _vp, _vp, _vp,
                                    ctypes.c_double, ctypes.POINTER(nb_opts)]),
    ("nb_ens_configure", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    ("nb_ens_tune", ctypes.c_int, [_vp, ctypes.c_int, _c_ip, _c_ip, _c_dp]),
    ("nb_ens_run", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int64, _c_lp, _c_lp]),
    ("nb_ens_step", ctypes.c_int, [_vp]),
    ("nb_ens_force", ctypes.c_int, [_vp, _vp, _vp, _vp]),
    ("nb_ens_energy", ctypes.c_int, [_vp, _vp, _vp]),
    ("nb_ens_get_state", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("nb_ens_set_state", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("nb_ens_last_error", ctypes.c_char_p, [_vp]),
    ("nb_ens_free", None, [_vp]),
    ("nb_set_profiling", ctypes.c_int, [_vp, ctypes.c_int]),
    ("nb_get_stats", ctypes.c_int, [_vp, ctypes.POINTER(nb_stats), ctypes.c_int]),
    ("nb_force_few_noalloc", ctypes.c_int, [ctypes.c_int64, _vp, _vp, _vp, ctypes.c_double, _vp,
                                            ctypes.c_int32, _vp, _vp, _vp, _vp]),
    ("nb_num_particles", ctypes.c_int64, [_vp]),
    ("nb_last_error", ctypes.c_char_p, [_vp]),
    ("nb_free", None, [_vp]),
]


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("%s is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _dptr(t):
    """Device pointer of a torch tensor (or an int address, or None)."""
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(t.data_ptr())


def _dev(t, dtype, count, name, required=True):
    """Device address of a torch CUDA tensor after checking that it is a
    contiguous CUDA tensor of `dtype` ("float64" or "int32") holding at least
    `count` elements, so the C side never reads or writes past its end.  An int
    is taken as a raw device address that the caller vouches for; None is a
    null pointer (a ValueError when the argument is required)."""
    if t is None:
        if required:
            raise ValueError("%s is required" % name)
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    dt = str(getattr(t, "dtype", type(t).__name__)).replace("torch.", "")
    if dt != dtype:
        raise ValueError("%s must be a %s tensor, got %s" % (name, dtype, dt))
    if not getattr(t, "is_cuda", False):
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.numel() < count:
        raise ValueError("%s holds %d elements, %d needed" % (name, t.numel(), count))
    return ctypes.c_void_p(t.data_ptr())


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        raise ValueError("expected shape %s, got %s" % (shape, a.shape))
    return a


def _check(ctx, rc):
    if rc != NB_OK:
        raise NbError(rc, lib().nb_last_error(ctx).decode())


def nb_default_opts(**overrides) -> nb_opts:
    o = nb_opts()
    lib().nb_default_opts(ctypes.byref(o))
    names = {f[0] for f in nb_opts._fields_}
    for k, v in overrides.items():
        if k not in names:
            raise TypeError("nb_opts has no field %r" % k)
        setattr(o, k, v)
    return o


def nb_init(m, x, v, eps, opts=None):
    """Returns a context handle (c_void_p)."""
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    v = _f64(v, (n, 3))
    ctx = ctypes.c_void_p()
    rc = lib().nb_init(ctypes.byref(ctx), n, _ptr(m), _ptr(x), _ptr(v), float(eps),
                       None if opts is None else ctypes.byref(opts))
    if rc != NB_OK:
        raise NbError(rc, lib().nb_last_error(None).decode())
    return ctx


def nb_init_dev(n, d_m, d_x, d_v, eps, opts=None):
    """nb_init from device arrays (torch CUDA float64 tensors m[n], x[n,3],
    v[n,3], or raw device addresses); returns a context handle."""
    n = int(n)
    nn = max(n, 0)
    args = (_dev(d_m, "float64", nn, "d_m"), _dev(d_x, "float64", 3 * nn, "d_x"),
            _dev(d_v, "float64", 3 * nn, "d_v"))
    ctx = ctypes.c_void_p()
    rc = lib().nb_init_dev(ctypes.byref(ctx), n, *args, float(eps),
                           None if opts is None else ctypes.byref(opts))
    if rc != NB_OK:
        raise NbError(rc, lib().nb_last_error(None).decode())
    return ctx


def nb_predict(ctx, t):
    _check(ctx, lib().nb_predict(ctx, float(t)))


def nb_force(ctx, active_idx):
    """(acc[n,3], jerk[n,3], pot[n]) on host for the listed particles."""
    idx = np.ascontiguousarray(active_idx, dtype=np.int32)
    na = idx.shape[0]
    acc = np.empty((na, 3))
    jerk = np.empty((na, 3))
    pot = np.empty(na)
    _check(ctx, lib().nb_force(ctx, _ptr(idx), na, _ptr(acc), _ptr(jerk), _ptr(pot)))
    return acc, jerk, pot


def nb_force_into(ctx, active_idx, acc, jerk, pot):
    """nb_force writing into caller-provided host arrays (any may be None)."""
    idx = np.ascontiguousarray(active_idx, dtype=np.int32)
    _check(ctx, lib().nb_force(ctx, _ptr(idx), idx.shape[0], _ptr(acc), _ptr(jerk), _ptr(pot)))


def nb_force_dev(ctx, d_active_idx, n_active, d_acc=None, d_jerk=None, d_pot=None):
    """Device-pointer variant: torch CUDA tensors (int32 indices, float64 outputs)."""
    na = max(int(n_active), 0)
    _check(ctx, lib().nb_force_dev(ctx, _dev(d_active_idx, "int32", na, "d_active_idx", na > 0),
                                   int(n_active), _dev(d_acc, "float64", 3 * na, "d_acc", False),
                                   _dev(d_jerk, "float64", 3 * na, "d_jerk", False),
                                   _dev(d_pot, "float64", na, "d_pot", False)))


def nb_correct(ctx, active_idx, t, acc=None, jerk=None):
    idx = np.ascontiguousarray(active_idx, dtype=np.int32)
    na = idx.shape[0]
    a = None if acc is None else _f64(acc, (na, 3))
    k = None if jerk is None else _f64(jerk, (na, 3))
    _check(ctx, lib().nb_correct(ctx, _ptr(idx), na, float(t), _ptr(a), _ptr(k)))


def nb_step(ctx, wait=True):
    """One device-driven block step; returns (t, n_active) when wait, else None."""
    if not wait:
        _check(ctx, lib().nb_step(ctx, None, None))
        return None
    t = ctypes.c_double()
    na = ctypes.c_int32()
    _check(ctx, lib().nb_step(ctx, ctypes.byref(t), ctypes.byref(na)))
    return t.value, na.value


def nb_run(ctx, t_end, max_steps=1 << 62):
    """Block steps to t_end; returns (steps, interactions)."""
    s = ctypes.c_int64()
    it = ctypes.c_int64()
    _check(ctx, lib().nb_run(ctx, float(t_end), int(max_steps), ctypes.byref(s), ctypes.byref(it)))
    return s.value, it.value


def nb_check_wait(ctx, ms):
    """Runs the bounded device wait on a counter nothing sets; raises NbError
    with NB_ETIMEOUT when the wait ran out, as it must."""
    _check(ctx, lib().nb_check_wait(ctx, int(ms)))


def nb_energy(ctx):
    """(kinetic, potential) energy."""
    ek = ctypes.c_double()
    ep = ctypes.c_double()
    _check(ctx, lib().nb_energy(ctx, ctypes.byref(ek), ctypes.byref(ep)))
    return ek.value, ep.value


def nb_get_state(ctx):
    """dict with x, v, a, k [n,3], t (int64 ticks) and level (int32)."""
    n = int(lib().nb_num_particles(ctx))
    st = {"x": np.empty((n, 3)), "v": np.empty((n, 3)), "a": np.empty((n, 3)),
          "k": np.empty((n, 3)), "t": np.empty(n, dtype=np.int64), "level": np.empty(n, dtype=np.int32)}
    _check(ctx, lib().nb_get_state(ctx, _ptr(st["x"]), _ptr(st["v"]), _ptr(st["a"]), _ptr(st["k"]),
                                   _ptr(st["t"]), _ptr(st["level"])))
    return st


def nb_get_state_dev(ctx, d_x=None, d_v=None, d_a=None, d_k=None, d_t=None, d_level=None):
    """nb_get_state into device tensors (float64 [n,3]; int64 / int32 [n]),
    enqueued on the context's stream."""
    n = int(lib().nb_num_particles(ctx))
    _check(ctx, lib().nb_get_state_dev(ctx, _dev(d_x, "float64", 3 * n, "d_x", False),
                                       _dev(d_v, "float64", 3 * n, "d_v", False),
                                       _dev(d_a, "float64", 3 * n, "d_a", False),
                                       _dev(d_k, "float64", 3 * n, "d_k", False),
                                       _dev(d_t, "int64", n, "d_t", False),
                                       _dev(d_level, "int32", n, "d_level", False)))


def nb_set_state(ctx, x, v, a, k, t, level):
    n = int(lib().nb_num_particles(ctx))
    arrs = [_f64(x, (n, 3)), _f64(v, (n, 3)), _f64(a, (n, 3)), _f64(k, (n, 3)),
            np.ascontiguousarray(t, dtype=np.int64), np.ascontiguousarray(level, dtype=np.int32)]
    _check(ctx, lib().nb_set_state(ctx, *[_ptr(q) for q in arrs]))


def nb_get_active(ctx):
    """(ascending indices of the last block, block time in ticks)."""
    n = int(lib().nb_num_particles(ctx))
    na = ctypes.c_int32()
    tt = ctypes.c_int64()
    _check(ctx, lib().nb_get_active(ctx, None, 0, ctypes.byref(na), ctypes.byref(tt)))
    idx = np.empty(max(na.value, 1), dtype=np.int32)
    _check(ctx, lib().nb_get_active(ctx, _ptr(idx), na.value, ctypes.byref(na), ctypes.byref(tt)))
    return idx[:na.value].copy(), tt.value


def nb_force_vjp(ctx, abar, kbar):
    """(xbar[n,3], vbar[n,3], mbar[n]) for cotangents of every acc and jerk."""
    n = int(lib().nb_num_particles(ctx))
    a, k = _f64(abar, (n, 3)), _f64(kbar, (n, 3))
    xb, vb, mb = np.empty((n, 3)), np.empty((n, 3)), np.empty(n)
    _check(ctx, lib().nb_force_vjp(ctx, _ptr(a), _ptr(k), _ptr(xb), _ptr(vb), _ptr(mb)))
    return xb, vb, mb


def nb_traj_forward(ctx, steps, checkpoint_every):
    _check(ctx, lib().nb_traj_forward(ctx, int(steps), int(checkpoint_every)))


def nb_traj_backward(ctx, xbar_T, vbar_T=None):
    """(xbar0[n,3], vbar0[n,3], mbar[n]) for cotangents of the final x, v."""
    n = int(lib().nb_num_particles(ctx))
    xt = _f64(xbar_T, (n, 3))
    vt = None if vbar_T is None else _f64(vbar_T, (n, 3))
    xb, vb, mb = np.empty((n, 3)), np.empty((n, 3)), np.empty(n)
    _check(ctx, lib().nb_traj_backward(ctx, _ptr(xt), _ptr(vt), _ptr(xb), _ptr(vb), _ptr(mb)))
    return xb, vb, mb


def nb_traj_backward_dev(ctx, d_xbar_T, d_vbar_T=None, d_xbar0=None, d_vbar0=None, d_mbar=None):
    """nb_traj_backward with device tensors (float64): cotangents of the final
    x, v in, gradients with respect to the initial x, v and the masses out."""
    n = int(lib().nb_num_particles(ctx))
    _check(ctx, lib().nb_traj_backward_dev(ctx, _dev(d_xbar_T, "float64", 3 * n, "d_xbar_T"),
                                           _dev(d_vbar_T, "float64", 3 * n, "d_vbar_T", False),
                                           _dev(d_xbar0, "float64", 3 * n, "d_xbar0", False),
                                           _dev(d_vbar0, "float64", 3 * n, "d_vbar0", False),
                                           _dev(d_mbar, "float64", n, "d_mbar", False)))


def nb_set_profiling(ctx, enable=True):
    _check(ctx, lib().nb_set_profiling(ctx, 1 if enable else 0))


def nb_get_stats(ctx, reset=False):
    """dict of the context counters (see nb_stats in include/nb.h)."""
    st = nb_stats()
    _check(ctx, lib().nb_get_stats(ctx, ctypes.byref(st), 1 if reset else 0))
    return {name: getattr(st, name) for name, _ in nb_stats._fields_}


def nb_force_few_noalloc(n, d_m, d_x, d_v, eps, d_active_idx, n_active, d_acc=None, d_jerk=None,
                         d_pot=None, stream=None):
    """Context-free force on at most NB_NOALLOC_MAX_ACTIVE particles from device
    arrays (torch CUDA tensors or addresses), for callers that may not allocate
    device memory; enqueued on `stream` (an int cudaStream_t, None = default)."""
    n, na = int(n), int(n_active)
    nn, nk = max(n, 0), max(na, 0)
    args = (_dev(d_m, "float64", nn, "d_m"), _dev(d_x, "float64", 3 * nn, "d_x"),
            _dev(d_v, "float64", 3 * nn, "d_v"), float(eps),
            _dev(d_active_idx, "int32", nk, "d_active_idx"), na,
            _dev(d_acc, "float64", 3 * nk, "d_acc", False),
            _dev(d_jerk, "float64", 3 * nk, "d_jerk", False),
            _dev(d_pot, "float64", nk, "d_pot", False))
    rc = lib().nb_force_few_noalloc(n, *args, None if not stream else ctypes.c_void_p(stream))
    if rc != NB_OK:
        raise NbError(rc, "nb_force_few_noalloc rejected n=%d n_active=%d eps=%r (limit %d)"
                      % (n, n_active, eps, NB_NOALLOC_MAX_ACTIVE))


def _echeck(ens, rc):
    if rc != NB_OK:
        raise NbError(rc, lib().nb_ens_last_error(ens).decode())


def nb_ens_init(offsets, m, x, v, eps, opts=None):
    """Ensemble of clusters offsets[c] .. offsets[c+1]-1; returns a handle."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    C = off.shape[0] - 1
    P = int(off[-1])
    m = _f64(m)
    x = _f64(x, (P, 3))
    v = _f64(v, (P, 3))
    e = ctypes.c_void_p()
    rc = lib().nb_ens_init(ctypes.byref(e), C, _ptr(off), _ptr(m), _ptr(x), _ptr(v), float(eps),
                           None if opts is None else ctypes.byref(opts))
    if rc != NB_OK:
        raise NbError(rc, lib().nb_ens_last_error(None).decode())
    return e


def nb_ens_configure(ens, threads, gmax):
    _echeck(ens, lib().nb_ens_configure(ens, int(threads), int(gmax)))


def nb_ens_tune(ens, launches_per_candidate=10):
    th, g, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _echeck(ens, lib().nb_ens_tune(ens, int(launches_per_candidate), ctypes.byref(th),
                                   ctypes.byref(g), ctypes.byref(ms)))
    return th.value, g.value, ms.value


def nb_ens_run(ens, t_end, max_launches=1 << 62):
    n, it = ctypes.c_int64(), ctypes.c_int64()
    _echeck(ens, lib().nb_ens_run(ens, float(t_end), int(max_launches), ctypes.byref(n), ctypes.byref(it)))
    return n.value, it.value


def nb_ens_step(ens):
    _echeck(ens, lib().nb_ens_step(ens))


def nb_ens_force(ens, P):
    acc, jerk, pot = np.empty((P, 3)), np.empty((P, 3)), np.empty(P)
    _echeck(ens, lib().nb_ens_force(ens, _ptr(acc), _ptr(jerk), _ptr(pot)))
    return acc, jerk, pot


def nb_ens_energy(ens, C):
    ek, ep = np.empty(C), np.empty(C)
    _echeck(ens, lib().nb_ens_energy(ens, _ptr(ek), _ptr(ep)))
    return ek, ep


def nb_ens_get_state(ens, C, P):
    st = {"x": np.empty((P, 3)), "v": np.empty((P, 3)), "a": np.empty((P, 3)), "k": np.empty((P, 3)),
          "t": np.empty(P, dtype=np.int64), "level": np.empty(P, dtype=np.int32),
          "steps": np.empty(C, dtype=np.int64), "interactions": np.empty(C, dtype=np.int64)}
    _echeck(ens, lib().nb_ens_get_state(ens, *[_ptr(st[k]) for k in
                                              ("x", "v", "a", "k", "t", "level", "steps", "interactions")]))
    return st


def nb_ens_set_state(ens, x, v, a, k, t, level):
    arrs = [_f64(x), _f64(v), _f64(a), _f64(k), np.ascontiguousarray(t, dtype=np.int64),
            np.ascontiguousarray(level, dtype=np.int32)]
    _echeck(ens, lib().nb_ens_set_state(ens, *[_ptr(q) for q in arrs]))


def nb_ens_last_error(ens) -> str:
    return lib().nb_ens_last_error(ens).decode()


def nb_ens_free(ens):
    if ens is not None and ens.value:
        lib().nb_ens_free(ens)
        ens.value = None


class Ensemble:
    """Owns one nb_ens; each method calls the entry point of the same name."""

    def __init__(self, offsets, m, x, v, eps, **opts):
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.C = self.offsets.shape[0] - 1
        self.P = int(self.offsets[-1])
        self.ens = nb_ens_init(self.offsets, m, x, v, eps, nb_default_opts(**opts) if opts else None)

    def nb_ens_configure(self, threads, gmax):
        return nb_ens_configure(self.ens, threads, gmax)

    def nb_ens_tune(self, launches_per_candidate=10):
        return nb_ens_tune(self.ens, launches_per_candidate)

    def nb_ens_run(self, t_end, max_launches=1 << 62):
        return nb_ens_run(self.ens, t_end, max_launches)

    def nb_ens_step(self):
        return nb_ens_step(self.ens)

    def nb_ens_force(self):
        return nb_ens_force(self.ens, self.P)

    def nb_ens_energy(self):
        return nb_ens_energy(self.ens, self.C)

    def nb_ens_get_state(self):
        return nb_ens_get_state(self.ens, self.C, self.P)

    def nb_ens_set_state(self, x, v, a, k, t, level):
        return nb_ens_set_state(self.ens, x, v, a, k, t, level)

    def nb_ens_free(self):
        nb_ens_free(self.ens)

    def __del__(self):
        try:
            self.nb_ens_free()
        except Exception:
            pass


def nb_num_particles(ctx) -> int:
    return int(lib().nb_num_particles(ctx))


def nb_last_error(ctx) -> str:
    return lib().nb_last_error(ctx).decode()


def nb_free(ctx):
    if ctx is not None and ctx.value:
        lib().nb_free(ctx)
        ctx.value = None


class Context:
    """Owns one nb_ctx; each method calls the entry point of the same name."""

    def __init__(self, m, x, v, eps, **opts):
        o = nb_default_opts(**opts) if opts else None
        self.ctx = nb_init(m, x, v, eps, o)
        self.n = nb_num_particles(self.ctx)

    @classmethod
    def from_device(cls, d_m, d_x, d_v, eps, n=None, **opts):
        """A context made by nb_init_dev from device tensors (float64 m[n],
        x[n,3], v[n,3]); n is needed only for raw addresses."""
        self = cls.__new__(cls)
        n = d_m.numel() if n is None else int(n)
        o = nb_default_opts(**opts) if opts else None
        self.ctx = nb_init_dev(n, d_m, d_x, d_v, eps, o)
        self.n = nb_num_particles(self.ctx)
        return self

    def nb_get_state_dev(self, d_x=None, d_v=None, d_a=None, d_k=None, d_t=None, d_level=None):
        return nb_get_state_dev(self.ctx, d_x, d_v, d_a, d_k, d_t, d_level)

    def nb_traj_backward_dev(self, d_xbar_T, d_vbar_T=None, d_xbar0=None, d_vbar0=None, d_mbar=None):
        return nb_traj_backward_dev(self.ctx, d_xbar_T, d_vbar_T, d_xbar0, d_vbar0, d_mbar)

    def nb_predict(self, t):
        return nb_predict(self.ctx, t)

    def nb_force(self, active_idx):
        return nb_force(self.ctx, active_idx)

    def nb_force_dev(self, d_active_idx, n_active, d_acc=None, d_jerk=None, d_pot=None):
        return nb_force_dev(self.ctx, d_active_idx, n_active, d_acc, d_jerk, d_pot)

    def nb_correct(self, active_idx, t, acc=None, jerk=None):
        return nb_correct(self.ctx, active_idx, t, acc, jerk)

    def nb_step(self, wait=True):
        return nb_step(self.ctx, wait)

    def nb_run(self, t_end, max_steps=1 << 62):
        return nb_run(self.ctx, t_end, max_steps)

    def nb_energy(self):
        return nb_energy(self.ctx)

    def nb_check_wait(self, ms):
        return nb_check_wait(self.ctx, ms)

    def nb_get_state(self):
        return nb_get_state(self.ctx)

    def nb_set_state(self, x, v, a, k, t, level):
        return nb_set_state(self.ctx, x, v, a, k, t, level)

    def nb_get_active(self):
        return nb_get_active(self.ctx)

    def nb_force_vjp(self, abar, kbar):
        return nb_force_vjp(self.ctx, abar, kbar)

    def nb_traj_forward(self, steps, checkpoint_every):
        return nb_traj_forward(self.ctx, steps, checkpoint_every)

    def nb_traj_backward(self, xbar_T, vbar_T=None):
        return nb_traj_backward(self.ctx, xbar_T, vbar_T)

    def nb_set_profiling(self, enable=True):
        return nb_set_profiling(self.ctx, enable)

    def nb_get_stats(self, reset=False):
        return nb_get_stats(self.ctx, reset)

    def nb_free(self):
        nb_free(self.ctx)

    def __del__(self):
        try:
            self.nb_free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.nb_free()

    def __del__(self):
        try:
            self.nb_free()
        except Exception:
            pass
