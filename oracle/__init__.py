"""FP64 CPU oracle for AQS parallel stepping -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously correct definition that the CUDA
library is checked against.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import it; the product path never does.
It shares no code with the CUDA library (its own C sources under this folder,
built with gcc into ``oracle/_build/liboracle.so``).

Every function here is a thin ctypes wrapper over the C functions declared in
``oracle.h``; the arithmetic lives in the C files, each citing the passage of
the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["geometry.c", "potential.c", "minimize.c", "aqs.c", "mlp.c"]

ORC_OK, ORC_ERR_INVALID_ARG, ORC_ERR_NOT_CONVERGED, ORC_ERR_NONFINITE, ORC_ERR_BOX_TOO_SMALL = 0, 1, 4, 5, 7
MAX_TYPES = 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags, no FMA contraction)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    hdr = os.path.join(_HERE, "oracle.h")
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(p) <= so_t for p in srcs + [hdr, __file__]):
            return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", "-shared",
           "-pthread", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Potential(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_types", C.c_int),
                ("sigma", C.c_double * (MAX_TYPES * MAX_TYPES)),
                ("eps", C.c_double * (MAX_TYPES * MAX_TYPES)),
                ("rc_factor", C.c_double)]


class FireParams(C.Structure):
    _fields_ = [("dt0", C.c_double), ("alpha0", C.c_double), ("f_inc", C.c_double),
                ("f_dec", C.c_double), ("f_alpha", C.c_double), ("dt_max", C.c_double),
                ("dt_min", C.c_double), ("max_step", C.c_double), ("tol", C.c_double),
                ("n_min", C.c_int), ("max_iter", C.c_int64)]


class ParallelStats(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("fire_iters_total", C.c_int64), ("n_log", C.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_half_min_width.restype = C.c_double
        _lib.orc_volume.restype = C.c_double
        _lib.orc_max_rel_disp.restype = C.c_double
        _lib.orc_fmax.restype = C.c_double
        _lib.orc_alg1_decide.restype = C.c_int64
        _lib.orc_mlp_loss_grad.restype = C.c_double
    return _lib


def _p(a, ctype=C.c_double):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


def make_potential(dim, sigma, eps, rc_factor=2.5) -> Potential:
    sigma = np.asarray(sigma, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    nt = sigma.shape[0]
    p = Potential()
    p.dim, p.n_types, p.rc_factor = dim, nt, rc_factor
    for a in range(nt):
        for b in range(nt):
            p.sigma[a * nt + b] = sigma[a, b]
            p.eps[a * nt + b] = eps[a, b]
    return p


def make_fire(**kw) -> FireParams:
    f = FireParams()
    for k, v in kw.items():
        setattr(f, k, v)
    return f


def _pos(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _types(t):
    return np.ascontiguousarray(t, dtype=np.int32)


def volume(H):
    H = _pos(H)
    return lib().orc_volume(H.shape[0], _p(H))


def half_min_width(H):
    H = _pos(H)
    return lib().orc_half_min_width(H.shape[0], _p(H))


def min_image(H, d):
    H = _pos(H)
    d = _pos(d).copy()
    flat = d.reshape(-1, H.shape[0])
    for row in flat:
        r = np.ascontiguousarray(row)
        lib().orc_min_image(H.shape[0], _p(H), _p(r))
        row[:] = r
    return flat.reshape(d.shape)


def affine_shear(x, H, dgamma):
    x, H = _pos(x).copy(), _pos(H).copy()
    lib().orc_affine_shear(H.shape[0], x.shape[0], _p(x), _p(H), C.c_double(dgamma))
    return x, H


def affine_map(x, H, F):
    x, H, F = _pos(x).copy(), _pos(H).copy(), _pos(F)
    lib().orc_affine_map(H.shape[0], x.shape[0], _p(x), _p(H), _p(F))
    return x, H


def pair_sflj(s, sigma, eps, rc):
    u, du = C.c_double(), C.c_double()
    lib().orc_pair_sflj(C.c_double(s), C.c_double(sigma), C.c_double(eps), C.c_double(rc),
                        C.byref(u), C.byref(du))
    return u.value, du.value


def energy_forces(pot, x, types, H):
    x, t, H = _pos(x), _types(types), _pos(H)
    F = np.zeros_like(x)
    E, tau = C.c_double(), C.c_double()
    st = lib().orc_energy_forces(C.byref(pot), x.shape[0], _p(x), _p(t, C.c_int32), _p(H),
                                 C.byref(E), _p(F), C.byref(tau))
    if st != ORC_OK:
        raise RuntimeError(f"orc_energy_forces status {st}")
    return E.value, F, tau.value


def fire(pot, fp, x, types, H, trace_cap=0):
    x, t, H = _pos(x).copy(), _types(types), _pos(H)
    it, E, fm = C.c_int64(), C.c_double(), C.c_double()
    et = np.zeros(trace_cap) if trace_cap else None
    rt = np.zeros(trace_cap, dtype=np.uint8) if trace_cap else None
    st = lib().orc_fire(C.byref(pot), C.byref(fp), x.shape[0], _p(x), _p(t, C.c_int32), _p(H),
                        C.byref(it), C.byref(E), C.byref(fm), _p(et), _p(rt, C.c_uint8),
                        C.c_int64(trace_cap))
    out = dict(x=x, status=st, iters=it.value, E=E.value, fmax=fm.value)
    if trace_cap:
        n = min(trace_cap, it.value + 1)
        out["e_trace"], out["reset_trace"] = et[:n], rt[:n]
    return out


def cg(pot, x, types, H, tol, max_iter, trace_cap=0):
    x, t, H = _pos(x).copy(), _types(types), _pos(H)
    it, E, fm = C.c_int64(), C.c_double(), C.c_double()
    et = np.zeros(trace_cap) if trace_cap else None
    st = lib().orc_cg(C.byref(pot), x.shape[0], _p(x), _p(t, C.c_int32), _p(H), C.c_double(tol),
                      C.c_int64(max_iter), C.byref(it), C.byref(E), C.byref(fm), _p(et),
                      C.c_int64(trace_cap))
    out = dict(x=x, status=st, iters=it.value, E=E.value, fmax=fm.value)
    if trace_cap:
        out["e_trace"] = et[:min(trace_cap, it.value + 1)]
    return out


def max_rel_disp(a, b, H):
    a, b, H = _pos(a), _pos(b), _pos(H)
    return lib().orc_max_rel_disp(H.shape[0], a.shape[0], _p(a), _p(b), _p(H))


def aqs(pot, fp, x, types, H, dgamma, n_steps):
    x, t, H = _pos(x).copy(), _types(types), _pos(H).copy()
    E = np.zeros(n_steps)
    tau = np.zeros(n_steps)
    D = np.zeros(n_steps)
    it = np.zeros(n_steps, dtype=np.int64)
    st = lib().orc_aqs(C.byref(pot), C.byref(fp), x.shape[0], _p(x), _p(t, C.c_int32), _p(H),
                       C.c_double(dgamma), n_steps, _p(E), _p(tau), _p(it, C.c_int64), _p(D))
    return dict(x=x, H=H, status=st, E=E, tau=tau, iters=it, D=D)


def wrap(x, H):
    x, H = _pos(x).copy(), _pos(H)
    lib().orc_wrap(H.shape[0], x.shape[0], _p(x), _p(H))
    return x


def triangularise(x, H):
    x, H = _pos(x).copy(), _pos(H).copy()
    lib().orc_triangularise(H.shape[0], x.shape[0], _p(x), _p(H))
    return x, H


def deform(x, H, F, Hlab=None):
    """One increment of a deformation history; returns (x, H, Hlab)."""
    x, H, F = _pos(x).copy(), _pos(H).copy(), _pos(F)
    Hl = H.copy() if Hlab is None else _pos(Hlab).copy()
    lib().orc_deform(H.shape[0], x.shape[0], _p(x), _p(H), _p(Hl), _p(F))
    return x, H, Hl


def aqs_history(pot, fp, x, types, H, F_steps, Hlab=None):
    x, t, H = _pos(x).copy(), _types(types), _pos(H).copy()
    Hl = H.copy() if Hlab is None else _pos(Hlab).copy()
    F = _pos(F_steps)
    n_steps = F.shape[0]
    E, tau, D = np.zeros(n_steps), np.zeros(n_steps), np.zeros(n_steps)
    it = np.zeros(n_steps, dtype=np.int64)
    st = lib().orc_aqs_history(C.byref(pot), C.byref(fp), x.shape[0], _p(x), _p(t, C.c_int32),
                               _p(H), _p(Hl), C.c_double(0.0), _p(F), n_steps, _p(E), _p(tau),
                               _p(it, C.c_int64), _p(D))
    return dict(x=x, H=H, Hlab=Hl, status=st, E=E, tau=tau, iters=it, D=D)


def parallel(pot, fp, x, types, H, dgamma, K, P, n_steps, eq_tol, n_threads=1, log_cap=100000,
             K_max=0, wrap_ends=False, F_steps=None, Hlab=None):
    x, t, H = _pos(x).copy(), _types(types), _pos(H).copy()
    Hl = H.copy() if Hlab is None else _pos(Hlab).copy()
    Fs = None if F_steps is None else _pos(F_steps)
    E, tau, D = np.zeros(n_steps), np.zeros(n_steps), np.zeros(n_steps)
    it = np.zeros(n_steps, dtype=np.int64)
    li = np.zeros(log_cap, dtype=np.int64)
    lc = np.zeros(log_cap, dtype=np.int32)
    le = np.zeros(log_cap, dtype=np.uint8)
    lm = np.zeros(log_cap)
    stats = ParallelStats()
    Kp = np.zeros(max(1, n_steps), dtype=np.int32)
    st = lib().orc_parallel(C.byref(pot), C.byref(fp), x.shape[0], _p(x), _p(t, C.c_int32), _p(H),
                            C.c_double(dgamma), K, P, n_steps, C.c_double(eq_tol), n_threads,
                            _p(E), _p(tau), _p(it, C.c_int64), _p(D), _p(li, C.c_int64),
                            _p(lc, C.c_int32), _p(le, C.c_uint8), _p(lm), C.c_int64(log_cap),
                            C.byref(stats), int(K_max), _p(Kp, C.c_int32), int(bool(wrap_ends)),
                            _p(Fs), _p(Hl) if Fs is not None else None)
    n = min(stats.n_log, log_cap)
    return dict(x=x, H=H, Hlab=Hl, status=st, E=E, tau=tau, iters=it, D=D,
                log_iter=li[:n], log_i=lc[:n], log_eq=le[:n], log_m=lm[:n],
                iterations=stats.iterations, fire_iters_total=stats.fire_iters_total,
                K_pass=Kp[:stats.iterations])


def alg1_decide(K_i, eq):
    K_i = np.ascontiguousarray(K_i, dtype=np.int32)
    eq = np.ascontiguousarray(eq, dtype=np.uint8)
    ff = C.c_int32()
    q = lib().orc_alg1_decide(len(K_i), _p(K_i, C.c_int32), _p(eq, C.c_uint8), C.byref(ff))
    return q, ff.value


def knn_features(x, types, H, n_types, n_nb):
    x, t, H = _pos(x), _types(types), _pos(H)
    dim = H.shape[0]
    feat = np.zeros((x.shape[0], n_nb * dim + n_types))
    st = lib().orc_knn_features(dim, x.shape[0], _p(x), _p(t, C.c_int32), _p(H), n_types, n_nb,
                                _p(feat))
    if st != ORC_OK:
        raise RuntimeError(f"orc_knn_features status {st}")
    return feat


def _mlp_args(Ws, bs):
    Ws = [np.ascontiguousarray(w, dtype=np.float64) for w in Ws]
    bs = [np.ascontiguousarray(b, dtype=np.float64) for b in bs]
    width = np.array([Ws[0].shape[1]] + [w.shape[0] for w in Ws], dtype=np.int32)
    L = len(Ws)
    Wp = (C.POINTER(C.c_double) * L)(*[_p(w) for w in Ws])
    bp = (C.POINTER(C.c_double) * L)(*[_p(b) for b in bs])
    return Ws, bs, width, L, Wp, bp


def mlp_forward(Ws, bs, X):
    Ws, bs, width, L, Wp, bp = _mlp_args(Ws, bs)
    X = _pos(X)
    Y = np.zeros((X.shape[0], width[-1]))
    lib().orc_mlp_forward(L, _p(width, C.c_int32), Wp, bp, C.c_int64(X.shape[0]), _p(X), _p(Y))
    return Y


def mlp_loss_grad(Ws, bs, X, T):
    Ws, bs, width, L, Wp, bp = _mlp_args(Ws, bs)
    X, T = _pos(X), _pos(T)
    dW = [np.zeros_like(w) for w in Ws]
    db = [np.zeros_like(b) for b in bs]
    dWp = (C.POINTER(C.c_double) * L)(*[_p(w) for w in dW])
    dbp = (C.POINTER(C.c_double) * L)(*[_p(b) for b in db])
    loss = lib().orc_mlp_loss_grad(L, _p(width, C.c_int32), Wp, bp, C.c_int64(X.shape[0]), _p(X),
                                   _p(T), dWp, dbp)
    return loss, dW, db
