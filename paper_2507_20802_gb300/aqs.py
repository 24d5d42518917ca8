"""Thin Python binding of the C ABI in include/aqs.h (argument marshalling only).

Every compute step runs in the CUDA library ``_build/libaqs.so``; this module
converts numpy arrays / torch tensors to pointers and checks status codes.
Importing it loads the library and raises if it is missing: there is no CPU
fallback.  The functions keep the C names (``aqs_create_system`` ...); the
``System`` class is a small convenience wrapper over them.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MAX_TYPES = 4
AQS_OK, AQS_ERR_INVALID_ARG, AQS_ERR_CUDA, AQS_ERR_OOM = 0, 1, 2, 3
AQS_ERR_NOT_CONVERGED, AQS_ERR_NONFINITE, AQS_ERR_NLIST_OVERFLOW = 4, 5, 6
AQS_ERR_BOX_TOO_SMALL, AQS_ERR_TIMEOUT, AQS_ERR_UNSUPPORTED = 7, 8, 9
AQS_FP64, AQS_MIXED = 0, 1

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class aqs_potential(C.Structure):
    _fields_ = [("n_types", C.c_int),
                ("sigma", C.c_double * (MAX_TYPES * MAX_TYPES)),
                ("eps", C.c_double * (MAX_TYPES * MAX_TYPES)),
                ("rc_factor", C.c_double)]


class aqs_system_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_replicas", C.c_int),
                ("n_atoms", C.POINTER(C.c_int64)), ("box", C.POINTER(C.c_double)),
                ("pos", C.c_void_p), ("types", C.c_void_p),
                ("pot", aqs_potential), ("precision", C.c_int), ("skin", C.c_double),
                ("nlist_capacity", C.c_int), ("cluster_size", C.c_int),
                ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", C.c_void_p)]


class aqs_fire_params(C.Structure):
    _fields_ = [("dt0", C.c_double), ("alpha0", C.c_double), ("f_inc", C.c_double),
                ("f_dec", C.c_double), ("f_alpha", C.c_double), ("dt_max", C.c_double),
                ("dt_min", C.c_double), ("max_step", C.c_double), ("tol", C.c_double),
                ("n_min", C.c_int), ("max_iter", C.c_int64),
                ("ref_ratio", C.c_double), ("ref_dmax", C.c_double)]


class aqs_min_result(C.Structure):
    _fields_ = [("iters", C.c_int64), ("evals64", C.c_int64), ("rebuilds", C.c_int64),
                ("energy", C.c_double), ("fmax", C.c_double), ("tau", C.c_double),
                ("nonaffine", C.c_double), ("status", C.c_int)]


class aqs_parallel_params(C.Structure):
    _fields_ = [("dgamma", C.c_double), ("K", C.c_int), ("P", C.c_int),
                ("n_steps", C.c_int64), ("eq_tol", C.c_double),
                ("event_threshold", C.c_double), ("max_iterations", C.c_int64),
                ("warm_start", C.c_int), ("run_discarded", C.c_int), ("K_max", C.c_int),
                ("F_steps", C.POINTER(C.c_double))]


class aqs_parallel_result(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("accepted_steps", C.c_int64),
                ("rejections", C.c_int64), ("fire_iters_total", C.c_int64),
                ("evals64_total", C.c_int64), ("chains_stopped", C.c_int64),
                ("K_pass", C.POINTER(C.c_int32)), ("K_next", C.c_int32),
                ("energy", C.POINTER(C.c_double)), ("tau", C.POINTER(C.c_double)),
                ("fire_iters", C.POINTER(C.c_int64)), ("nonaffine", C.POINTER(C.c_double)),
                ("event", C.POINTER(C.c_uint8)),
                ("log_cap", C.c_int64), ("n_log", C.c_int64),
                ("log_iter", C.POINTER(C.c_int64)), ("log_i", C.POINTER(C.c_int32)),
                ("log_eq", C.POINTER(C.c_uint8)), ("log_m", C.POINTER(C.c_double))]


class aqs_kernel_stats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("kernel_ms", C.c_double), ("evals32", C.c_int64),
                ("evals64", C.c_int64), ("pairs32", C.c_int64), ("pairs64", C.c_int64),
                ("atom_iters", C.c_int64), ("rebuilds", C.c_int64)]


# exported symbols and their signatures (kept in the order of include/aqs.h)
_SIGS = {
    "aqs_fire_params_default": (None, [C.POINTER(aqs_fire_params)]),
    "aqs_create_system": (C.c_int, [C.POINTER(aqs_system_desc), C.POINTER(C.c_void_p)]),
    "aqs_destroy_system": (None, [C.c_void_p]),
    "aqs_affine_shear": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "aqs_minimize": (C.c_int, [C.c_void_p, C.POINTER(aqs_fire_params), C.POINTER(C.c_uint8),
                               C.POINTER(aqs_min_result)]),
    "aqs_run_sequential": (C.c_int, [C.c_void_p, C.POINTER(aqs_fire_params), C.c_double,
                                     C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "aqs_parallel_step": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(aqs_fire_params),
                                    C.POINTER(aqs_parallel_params),
                                    C.POINTER(aqs_parallel_result)]),
    "aqs_deform": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "aqs_run_history": (C.c_int, [C.c_void_p, C.POINTER(aqs_fire_params), C.POINTER(C.c_double),
                                  C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "aqs_get_frame": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "aqs_compare_configs": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_double,
                                      C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "aqs_num_replicas": (C.c_int, [C.c_void_p]),
    "aqs_num_atoms": (C.c_int64, [C.c_void_p, C.c_int]),
    "aqs_get_positions": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "aqs_set_positions": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "aqs_get_box": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "aqs_set_box": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "aqs_energy_forces": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_void_p,
                                    C.POINTER(C.c_double)]),
    "aqs_warm_num_params": (C.c_int, []),
    "aqs_warm_create": (C.c_int, [C.c_int, C.c_int, C.c_uint64, C.c_void_p, C.POINTER(C.c_void_p)]),
    "aqs_warm_destroy": (None, [C.c_void_p]),
    "aqs_warm_get_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "aqs_warm_set_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "aqs_warm_features": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "aqs_warm_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "aqs_warm_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                     C.POINTER(C.c_float), C.POINTER(C.c_double)]),
    "aqs_warm_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_double,
                                      C.c_double, C.POINTER(C.c_double)]),
    "aqs_warm_collect": (C.c_int, [C.c_void_p, C.POINTER(aqs_fire_params), C.c_double, C.c_int64,
                                   C.c_void_p, C.c_void_p]),
    "aqs_run_sequential_warm": (C.c_int, [C.c_void_p, C.POINTER(aqs_fire_params), C.c_void_p,
                                          C.c_double, C.c_int64, C.c_double,
                                          C.POINTER(C.c_double), C.POINTER(C.c_double),
                                          C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                          C.POINTER(C.c_uint8)]),
    "aqs_energy_forces_noalloc": (C.c_int, [C.c_int, C.c_int64, C.c_void_p, C.c_void_p,
                                            C.POINTER(C.c_double), C.POINTER(aqs_potential),
                                            C.c_void_p, C.c_void_p, C.c_void_p]),
    "aqs_autotune_clusters": (C.c_int, [C.c_void_p, C.POINTER(aqs_fire_params), C.c_int64,
                                        C.POINTER(C.c_uint8), C.POINTER(C.c_int),
                                        C.POINTER(C.c_int), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double)]),
    "aqs_set_autotune": (C.c_int, [C.c_void_p, C.c_int64]),
    "aqs_set_launch_budget": (C.c_int, [C.c_void_p, C.c_int64]),
    "aqs_set_threads_per_atom": (C.c_int, [C.c_void_p, C.c_int]),
    "aqs_threads_per_atom": (C.c_int, [C.c_void_p]),
    "aqs_max_active_clusters": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]),
    "aqs_set_grid_barrier": (C.c_int, [C.c_void_p, C.c_int]),
    "aqs_grid_barrier": (C.c_int, [C.c_void_p, C.c_int]),
    "aqs_set_staging": (C.c_int, [C.c_void_p, C.c_int]),
    "aqs_staging": (C.c_int, [C.c_void_p, C.c_int]),
    "aqs_set_kernel_timing": (None, [C.c_int]),
    "aqs_get_kernel_stats": (None, [C.POINTER(aqs_kernel_stats)]),
    "aqs_reset_kernel_stats": (None, []),
    "aqs_last_error": (C.c_char_p, []),
    "aqs_launch_count": (C.c_int64, []),
    "aqs_mean_neighbours": (C.c_double, [C.c_void_p, C.c_int]),
    "aqs_cluster_size": (C.c_int, [C.c_void_p, C.c_int]),
}

_lib = None


def lib(build_if_missing: bool = True):
    """Load libaqs.so (building it when it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path}")
        lib_ = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib_, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib_
    return _lib


class AqsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"aqs status {status}: {msg}")
        self.status = status


def check(status):
    if status != AQS_OK:
        raise AqsError(status, lib().aqs_last_error().decode())
    return status


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _ptr(a):
    """Pointer of a numpy array or a torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def make_potential(sigma, eps, rc_factor=2.5) -> aqs_potential:
    sigma = np.asarray(sigma, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    nt = sigma.shape[0]
    p = aqs_potential()
    p.n_types, p.rc_factor = nt, rc_factor
    for a in range(nt):
        for b in range(nt):
            p.sigma[a * nt + b] = sigma[a, b]
            p.eps[a * nt + b] = eps[a, b]
    return p


def fire_params(**kw) -> aqs_fire_params:
    f = aqs_fire_params()
    lib().aqs_fire_params_default(C.byref(f))
    for k, v in kw.items():
        setattr(f, k, v)
    return f


# ------------------------------------------------------------ C-name wrappers
def aqs_create_system(desc: aqs_system_desc) -> C.c_void_p:
    h = C.c_void_p()
    check(lib().aqs_create_system(C.byref(desc), C.byref(h)))
    return h


def aqs_destroy_system(h):
    lib().aqs_destroy_system(h)


def aqs_affine_shear(h, dgamma):
    dg = np.ascontiguousarray(dgamma, dtype=np.float64)
    check(lib().aqs_affine_shear(h, _dp(dg)))


def aqs_minimize(h, fire, n_replicas, mask=None):
    res = (aqs_min_result * n_replicas)()
    m = None
    if mask is not None:
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        m = mask.ctypes.data_as(C.POINTER(C.c_uint8))
    st = lib().aqs_minimize(h, C.byref(fire), m, res)
    return st, res


def aqs_run_sequential(h, fire, dgamma, n_steps, n_replicas):
    E = np.zeros((n_steps, n_replicas))
    tau = np.zeros((n_steps, n_replicas))
    it = np.zeros((n_steps, n_replicas), dtype=np.int64)
    D = np.zeros((n_steps, n_replicas))
    check(lib().aqs_run_sequential(h, C.byref(fire), C.c_double(dgamma), C.c_int64(n_steps),
                                   _dp(E), _dp(tau), it.ctypes.data_as(C.POINTER(C.c_int64)),
                                   _dp(D)))
    return dict(E=E, tau=tau, iters=it, D=D)


def aqs_parallel_step(h, replica, fire, dgamma, K, P, n_steps, eq_tol=1e-6,
                      event_threshold=1e-2, max_iterations=0, warm_start=0, log_cap=100000,
                      run_discarded=0, K_max=0, F_steps=None):
    p = aqs_parallel_params(dgamma=dgamma, K=K, P=P, n_steps=n_steps, eq_tol=eq_tol,
                            event_threshold=event_threshold, max_iterations=max_iterations,
                            warm_start=warm_start, run_discarded=run_discarded, K_max=K_max)
    Fh = None
    if F_steps is not None:
        Fh = np.ascontiguousarray(F_steps, dtype=np.float64)
        p.F_steps = _dp(Fh)
    n = max(int(n_steps), 1)
    E, tau, D = np.zeros(n), np.zeros(n), np.zeros(n)
    it = np.zeros(n, dtype=np.int64)
    ev = np.zeros(n, dtype=np.uint8)
    li = np.zeros(log_cap, dtype=np.int64)
    lc = np.zeros(log_cap, dtype=np.int32)
    le = np.zeros(log_cap, dtype=np.uint8)
    lm = np.zeros(log_cap)
    r = aqs_parallel_result()
    r.energy, r.tau, r.nonaffine = _dp(E), _dp(tau), _dp(D)
    r.fire_iters = it.ctypes.data_as(C.POINTER(C.c_int64))
    r.event = ev.ctypes.data_as(C.POINTER(C.c_uint8))
    r.log_cap = log_cap
    r.log_iter = li.ctypes.data_as(C.POINTER(C.c_int64))
    r.log_i = lc.ctypes.data_as(C.POINTER(C.c_int32))
    r.log_eq = le.ctypes.data_as(C.POINTER(C.c_uint8))
    r.log_m = _dp(lm)
    kp = np.zeros(n, dtype=np.int32)
    r.K_pass = kp.ctypes.data_as(C.POINTER(C.c_int32))
    check(lib().aqs_parallel_step(h, replica, C.byref(fire), C.byref(p), C.byref(r)))
    k = r.accepted_steps
    nl = min(r.n_log, log_cap)
    return dict(E=E[:k], tau=tau[:k], iters=it[:k], D=D[:k], event=ev[:k],
                iterations=r.iterations, accepted=r.accepted_steps, rejections=r.rejections,
                fire_iters_total=r.fire_iters_total, evals64_total=r.evals64_total,
                chains_stopped=r.chains_stopped, K_pass=kp[:r.iterations], K_next=r.K_next,
                log_iter=li[:nl], log_i=lc[:nl], log_eq=le[:nl], log_m=lm[:nl])


def aqs_deform(h, F):
    F = np.ascontiguousarray(F, dtype=np.float64)
    check(lib().aqs_deform(h, _dp(F)))


def aqs_run_history(h, fire, F_steps, n_replicas):
    F = np.ascontiguousarray(F_steps, dtype=np.float64)
    n_steps = F.shape[0]
    E = np.zeros((n_steps, n_replicas))
    tau = np.zeros((n_steps, n_replicas))
    it = np.zeros((n_steps, n_replicas), dtype=np.int64)
    D = np.zeros((n_steps, n_replicas))
    check(lib().aqs_run_history(h, C.byref(fire), _dp(F), C.c_int64(n_steps), _dp(E), _dp(tau),
                                it.ctypes.data_as(C.POINTER(C.c_int64)), _dp(D)))
    return dict(E=E, tau=tau, iters=it, D=D)


def aqs_get_frame(h, replica, dim):
    Q = np.zeros((dim, dim))
    check(lib().aqs_get_frame(h, replica, _dp(Q)))
    return Q


def aqs_compare_configs(ha, ra, hb, rb, tol):
    m, eq = C.c_double(), C.c_int()
    check(lib().aqs_compare_configs(ha, ra, hb, rb, C.c_double(tol), C.byref(m), C.byref(eq)))
    return m.value, bool(eq.value)


def aqs_get_positions(h, replica, out):
    check(lib().aqs_get_positions(h, replica, _ptr(out)))
    return out


def aqs_set_positions(h, replica, pos):
    check(lib().aqs_set_positions(h, replica, _ptr(pos)))


def aqs_get_box(h, replica, dim):
    H = np.zeros((dim, dim))
    check(lib().aqs_get_box(h, replica, _dp(H)))
    return H


def aqs_set_box(h, replica, H):
    H = np.ascontiguousarray(H, dtype=np.float64)
    check(lib().aqs_set_box(h, replica, _dp(H)))


def aqs_energy_forces(h, replica, forces=None):
    e, tau = C.c_double(), C.c_double()
    check(lib().aqs_energy_forces(h, replica, C.byref(e), _ptr(forces), C.byref(tau)))
    return e.value, tau.value


def aqs_launch_count() -> int:
    return int(lib().aqs_launch_count())


def aqs_set_kernel_timing(on: bool):
    lib().aqs_set_kernel_timing(1 if on else 0)


def aqs_get_kernel_stats() -> dict:
    s = aqs_kernel_stats()
    lib().aqs_get_kernel_stats(C.byref(s))
    return {k: getattr(s, k) for k, _ in aqs_kernel_stats._fields_}


def aqs_reset_kernel_stats():
    lib().aqs_reset_kernel_stats()


# ------------------------------------------------------------ warm start
WARM_IN = 80


class Warm:
    """The learned warm-start network (device weights); thin wrapper over the
    aqs_warm_* calls.  Device buffers are torch tensors (memory only)."""

    def __init__(self, dim=2, n_types=2, seed=0, stream=None):
        self.dim, self.n_types = dim, n_types
        h = C.c_void_p()
        check(lib().aqs_warm_create(dim, n_types, seed, C.c_void_p(stream) if stream else None,
                                    C.byref(h)))
        self.h = h
        self.n_params = lib().aqs_warm_num_params()

    def close(self):
        if getattr(self, "h", None):
            lib().aqs_warm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        p = np.zeros(self.n_params, np.float32)
        check(lib().aqs_warm_get_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float))))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        check(lib().aqs_warm_set_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float))))

    def predict(self, feat, out):
        check(lib().aqs_warm_predict(self.h, _ptr(feat), feat.shape[0], _ptr(out)))
        return out

    def loss_grad(self, feat, target):
        g = np.zeros(self.n_params, np.float32)
        loss = C.c_double()
        check(lib().aqs_warm_loss_grad(self.h, _ptr(feat), _ptr(target), feat.shape[0],
                                       g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)))
        return loss.value, g

    def train_step(self, feat, target, lr, weight_decay=0.0):
        loss = C.c_double()
        check(lib().aqs_warm_train_step(self.h, _ptr(feat), _ptr(target), feat.shape[0],
                                        C.c_double(lr), C.c_double(weight_decay), C.byref(loss)))
        return loss.value


def unpack_params(p, dim=2, n_in=WARM_IN, hid=128, out_pad=16):
    """Split the flat parameter vector into (weights, biases) lists."""
    shapes = [(hid, n_in), (hid, hid), (hid, hid), (out_pad, hid)]
    Ws, k = [], 0
    for s in shapes:
        Ws.append(p[k:k + s[0] * s[1]].reshape(s))
        k += s[0] * s[1]
    bs = []
    for n in [hid, hid, hid, out_pad]:
        bs.append(p[k:k + n])
        k += n
    return Ws, bs


# ------------------------------------------------------------ convenience
class System:
    """Owns one aqs_system.  ``pos`` (N_tot x d) and ``types`` may be numpy
    arrays (host) or CUDA tensors (device); ``boxes`` is R x d x d."""

    def __init__(self, pos, types, boxes, n_atoms, sigma, eps, rc_factor=2.5,
                 precision=AQS_MIXED, skin=0.3, nlist_capacity=0, cluster_size=0,
                 stream=None):
        self.n_atoms = np.ascontiguousarray(n_atoms, dtype=np.int64)
        self.R = len(self.n_atoms)
        self.boxes = np.ascontiguousarray(boxes, dtype=np.float64).reshape(self.R, -1)
        self.dim = int(round(np.sqrt(self.boxes.shape[1])))
        self._pos = pos if hasattr(pos, "data_ptr") else np.ascontiguousarray(pos, np.float64)
        self._types = types if hasattr(types, "data_ptr") else np.ascontiguousarray(types, np.int32)
        d = aqs_system_desc()
        d.dim, d.n_replicas = self.dim, self.R
        d.n_atoms = self.n_atoms.ctypes.data_as(C.POINTER(C.c_int64))
        d.box = self.boxes.ctypes.data_as(C.POINTER(C.c_double))
        d.pos = _ptr(self._pos)
        d.types = _ptr(self._types)
        d.pot = make_potential(sigma, eps, rc_factor)
        d.precision = precision
        d.skin = skin
        d.nlist_capacity = nlist_capacity
        d.cluster_size = cluster_size
        d.stream = C.c_void_p(stream) if stream else None
        self.h = aqs_create_system(d)

    def close(self):
        if getattr(self, "h", None):
            aqs_destroy_system(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def positions(self, replica=0):
        out = np.zeros((int(self.n_atoms[replica]), self.dim))
        return aqs_get_positions(self.h, replica, out)

    def set_positions(self, pos, replica=0):
        pos = pos if hasattr(pos, "data_ptr") else np.ascontiguousarray(pos, np.float64)
        aqs_set_positions(self.h, replica, pos)

    def box(self, replica=0):
        return aqs_get_box(self.h, replica, self.dim)

    def shear(self, dgamma):
        dg = np.broadcast_to(np.asarray(dgamma, np.float64), (self.R,))
        aqs_affine_shear(self.h, dg)

    def minimize(self, fire=None, mask=None, check_status=True):
        fire = fire or fire_params()
        st, res = aqs_minimize(self.h, fire, self.R, mask)
        if check_status:
            check(st)
        return [dict(iters=r.iters, evals64=r.evals64, rebuilds=r.rebuilds, E=r.energy,
                     fmax=r.fmax, tau=r.tau, D=r.nonaffine, status=r.status) for r in res]

    def energy_forces(self, replica=0):
        F = np.zeros((int(self.n_atoms[replica]), self.dim))
        e, tau = aqs_energy_forces(self.h, replica, F)
        return e, F, tau

    def run_sequential(self, dgamma, n_steps, fire=None):
        return aqs_run_sequential(self.h, fire or fire_params(), dgamma, n_steps, self.R)

    def run_history(self, F_steps, fire=None):
        return aqs_run_history(self.h, fire or fire_params(), F_steps, self.R)

    def deform(self, F):
        F = np.broadcast_to(np.asarray(F, np.float64), (self.R, self.dim, self.dim))
        aqs_deform(self.h, F)

    def frame(self, replica=0):
        return aqs_get_frame(self.h, replica, self.dim)

    def parallel_step(self, dgamma, K, P, n_steps, fire=None, replica=0, **kw):
        return aqs_parallel_step(self.h, replica, fire or fire_params(), dgamma, K, P, n_steps,
                                 **kw)

    def warm_features(self, feat_bf16, feat_f64=None, replica=-1):
        check(lib().aqs_warm_features(self.h, replica, _ptr(feat_bf16), _ptr(feat_f64)))

    def warm_collect(self, dgamma, n_steps, feat_out, target_out, fire=None):
        check(lib().aqs_warm_collect(self.h, C.byref(fire or fire_params()), C.c_double(dgamma),
                                     C.c_int64(n_steps), _ptr(feat_out), _ptr(target_out)))

    def run_sequential_warm(self, warm, dgamma, n_steps, gate=0.0, fire=None):
        R = self.R
        E, tau, D = (np.zeros((n_steps, R)) for _ in range(3))
        it = np.zeros((n_steps, R), dtype=np.int64)
        used = np.zeros((n_steps, R), dtype=np.uint8)
        check(lib().aqs_run_sequential_warm(self.h, C.byref(fire or fire_params()), warm.h,
                                            C.c_double(dgamma), C.c_int64(n_steps),
                                            C.c_double(gate), _dp(E), _dp(tau),
                                            it.ctypes.data_as(C.POINTER(C.c_int64)), _dp(D),
                                            used.ctypes.data_as(C.POINTER(C.c_uint8))))
        return dict(E=E, tau=tau, iters=it, D=D, used=used)

    def mean_neighbours(self, replica=0):
        return lib().aqs_mean_neighbours(self.h, replica)

    def cluster_size(self, replica=0):
        return lib().aqs_cluster_size(self.h, replica)

    def autotune(self, iters=200, fire=None, mask=None):
        """Times every feasible cluster size, then every staging mode at the
        fastest size, on `iters` FIRE iterations and keeps the fastest.
        Returns (C, staging, {C: ms per iteration}, {mode: ms per iteration})."""
        best, mode = C.c_int(0), C.c_int(-1)
        ms = np.zeros(17)
        mm = np.zeros(4)
        m = None
        if mask is not None:
            mk = np.ascontiguousarray(mask, dtype=np.uint8)
            m = mk.ctypes.data_as(C.POINTER(C.c_uint8))
        check(lib().aqs_autotune_clusters(self.h, C.byref(fire or fire_params()), C.c_int64(iters),
                                          m, C.byref(best), C.byref(mode), _dp(ms), _dp(mm)))
        return (best.value, mode.value, {c: float(ms[c]) for c in range(1, 17) if ms[c] >= 0},
                {k: float(mm[k]) for k in range(4) if mm[k] >= 0})

    def set_launch_budget(self, iters):
        check(lib().aqs_set_launch_budget(self.h, C.c_int64(iters)))

    def set_threads_per_atom(self, tpa):
        check(lib().aqs_set_threads_per_atom(self.h, int(tpa)))

    def threads_per_atom(self):
        return lib().aqs_threads_per_atom(self.h)

    def set_grid_barrier(self, on):
        """True / False fixes the barrier mode; None lets the autotuner choose."""
        check(lib().aqs_set_grid_barrier(self.h, -1 if on is None else (1 if on else 0)))

    def grid_barrier(self, chains=False):
        """1 grid barriers, 0 clusters, -1 chains not run yet."""
        return lib().aqs_grid_barrier(self.h, 1 if chains else 0)

    def max_active_clusters(self, C, staging=-1, tpa=1, replica=0):
        return lib().aqs_max_active_clusters(self.h, replica, C, staging, tpa)

    def set_staging(self, mode):
        check(lib().aqs_set_staging(self.h, int(mode)))

    def staging(self, replica=0):
        return lib().aqs_staging(self.h, replica)

    def set_autotune(self, iters):
        check(lib().aqs_set_autotune(self.h, C.c_int64(iters)))
