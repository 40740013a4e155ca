"""FP64 CPU oracle for the multiscale symmetric debiased Sinkhorn solver
(Feydy et al., "Fast and Scalable Optimal Transport for Brain Tractograms").

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library and its Python binding never import, link or call it, and it imports
nothing from them.

The arithmetic lives in ``oracle.c`` (plain C, double precision, OpenMP over
independent rows); this module compiles it with gcc and exposes thin ctypes
wrappers that take numpy arrays.  ``mlp.py`` holds the FP64 oracle of the
warm-start network.  Every function states the passage of the paper it follows
in ``oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no FP contraction so that
    the float cell decisions of the grid clustering are plain IEEE single)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               "-std=c11", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        ci, cd = C.c_int, C.c_double
        lib.oracle_threads.argtypes = []; lib.oracle_threads.restype = ci
        lib.oracle_set_threads.argtypes = [ci]; lib.oracle_set_threads.restype = None
        lib.oracle_flip_fibers.argtypes = [f32p, ci, ci, f32p]; lib.oracle_flip_fibers.restype = None
        lib.oracle_select_flips.argtypes = [f64p, i32p, ci, i32p, i32p, f64p]; lib.oracle_select_flips.restype = None
        lib.oracle_grad_x.argtypes = [f32p, f32p, ci, f32p, f32p, ci, ci, ci, cd, f64p, f64p, f64p, f64p]
        lib.oracle_grad_x.restype = None
        lib.oracle_cost.argtypes = [f32p, f32p, ci, ci]; lib.oracle_cost.restype = cd
        lib.oracle_rho.argtypes = [cd, ci]; lib.oracle_rho.restype = cd
        lib.oracle_lambda.argtypes = [cd, cd, ci]; lib.oracle_lambda.restype = cd
        lib.oracle_softmin.argtypes = [ci, f32p, ci, f32p, f32p, f64p, ci, ci, cd, cd, f64p]
        lib.oracle_softmin.restype = None
        lib.oracle_diameter.argtypes = [f32p, ci, f32p, ci, ci]; lib.oracle_diameter.restype = cd
        lib.oracle_schedule.argtypes = [cd, cd, cd, C.c_void_p, ci]; lib.oracle_schedule.restype = ci
        lib.oracle_sinkhorn_step.argtypes = [f32p, f32p, ci, f32p, f32p, ci, ci, ci, cd, cd, f64p, f64p, f64p, f64p]
        lib.oracle_sinkhorn_step.restype = cd
        lib.oracle_divergence.argtypes = [f32p, ci, f32p, ci, cd, cd, f64p, f64p, f64p, f64p]
        lib.oracle_divergence.restype = cd
        lib.oracle_sinkhorn.argtypes = [f32p, f32p, ci, f32p, f32p, ci, ci, ci, cd, cd, cd, cd, cd, ci,
                                        f64p, f64p, f64p, f64p, C.POINTER(cd), f64p]
        lib.oracle_sinkhorn.restype = ci
        lib.oracle_ot_dual.argtypes = [f32p, f32p, ci, f32p, f32p, ci, ci, ci, cd, cd, f64p, f64p]
        lib.oracle_ot_dual.restype = cd
        lib.oracle_ot_primal.argtypes = [f32p, f32p, ci, f32p, f32p, ci, ci, ci, cd, cd, f64p, f64p, C.POINTER(cd)]
        lib.oracle_ot_primal.restype = cd
        lib.oracle_transport_apply.argtypes = [f32p, ci, f32p, f32p, ci, ci, ci, cd, f64p, f64p, i32p, ci,
                                               f64p, i32p, f64p]
        lib.oracle_transport_apply.restype = None
        lib.oracle_cluster_grid.argtypes = [f32p, ci, ci, C.c_float, i32p, i32p, i32p, u32p]
        lib.oracle_cluster_grid.restype = ci
        lib.oracle_kmeans.argtypes = [f32p, C.c_void_p, ci, ci, ci, ci, f32p, i32p, f64p]
        lib.oracle_kmeans.restype = None
        _lib = lib
    return _lib


def threads() -> int:
    """Threads of the oracle's OpenMP row loops (the host cores its timings use)."""
    return int(_load().oracle_threads())


def set_threads(n: int) -> None:
    """Threads of the row loops from now on (timings on one core use 1)."""
    _load().oracle_set_threads(int(n))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _pts(a):
    a = _f32(a)
    return a.reshape(a.shape[0], -1) if a.ndim == 2 else a.reshape(-1, 1)


def rho(reach, p=2):
    return _load().oracle_rho(float(reach), int(p))


def lam(sigma, reach, p=2):
    return _load().oracle_lambda(float(sigma), float(reach), int(p))


def cost(u, v, p=2):
    u, v = _f32(u).ravel(), _f32(v).ravel()
    return _load().oracle_cost(u, v, u.size, int(p))


def softmin(q, pts, w, pot, eps, lam=1.0, p=2):
    """out_i = -lam*eps*log sum_k w_k exp((pot_k - C(pts_k, q_i))/eps)."""
    q, pts = _pts(q), _pts(pts)
    out = np.empty(q.shape[0], np.float64)
    _load().oracle_softmin(q.shape[0], q, pts.shape[0], pts, _f32(w), _f64(pot), q.shape[1], int(p),
                           float(eps), float(lam), out)
    return out


def diameter(x, y):
    x, y = _pts(x), _pts(y)
    return _load().oracle_diameter(x, x.shape[0], y, y.shape[0], x.shape[1])


def schedule(d, blur, q):
    n = _load().oracle_schedule(float(d), float(blur), float(q), None, 0)
    out = np.empty(n, np.float64)
    _load().oracle_schedule(float(d), float(blur), float(q), out.ctypes.data_as(C.c_void_p), n)
    return out


def sinkhorn_step(x, alpha, y, beta, eps, lam, a, b, f, g, p=2):
    """One averaged step in place on (a, b, f, g) (float64 arrays); returns max|delta|/eps."""
    x, y = _pts(x), _pts(y)
    return _load().oracle_sinkhorn_step(x, _f32(alpha), x.shape[0], y, _f32(beta), y.shape[0], x.shape[1],
                                        int(p), float(eps), float(lam), a, b, f, g)


def divergence(alpha, beta, eps, rho_, a, b, f, g):
    return _load().oracle_divergence(_f32(alpha), len(alpha), _f32(beta), len(beta), float(eps), float(rho_),
                                     _f64(a), _f64(b), _f64(f), _f64(g))


def sinkhorn(x, alpha, y, beta, blur, reach=0.0, scaling=0.5, p=2, diameter=0.0, tol=1e-13, max_iters=100000):
    """Converged FP64 solve.  Returns dict(S, a, b, f, g, iters, sched_len, delta, converged)."""
    x, y = _pts(x), _pts(y)
    N, M, D = x.shape[0], y.shape[0], x.shape[1]
    a, f = np.zeros(N), np.zeros(N)
    b, g = np.zeros(M), np.zeros(M)
    S = C.c_double()
    info = np.zeros(3)
    rc = _load().oracle_sinkhorn(x, _f32(alpha), N, y, _f32(beta), M, D, int(p), float(blur), float(reach),
                                 float(scaling), float(diameter), float(tol), int(max_iters), a, b, f, g,
                                 C.byref(S), info)
    return dict(S=S.value, a=a, b=b, f=f, g=g, iters=int(info[0]), sched_len=int(info[1]), delta=info[2],
                converged=(rc == 0))


def grad_x(x, alpha, y, beta, eps, a, f, g, p=2):
    """dS/dx (N x D) at the converged duals: a = a^{alpha<->alpha}, f = b^{beta->alpha},
    g = a^{alpha->beta}.  For dS/dy pass (y, beta, x, alpha, eps, b, g, f)."""
    x, y = _pts(x), _pts(y)
    out = np.empty(x.shape, np.float64)
    _load().oracle_grad_x(x, _f32(alpha), x.shape[0], y, _f32(beta), y.shape[0], x.shape[1], int(p), float(eps),
                          _f64(a), _f64(f), _f64(g), out)
    return out


def ot_dual(x, alpha, y, beta, eps, rho_, f, g, p=2):
    x, y = _pts(x), _pts(y)
    return _load().oracle_ot_dual(x, _f32(alpha), x.shape[0], y, _f32(beta), y.shape[0], x.shape[1], int(p),
                                  float(eps), float(rho_), _f64(f), _f64(g))


def ot_primal(x, alpha, y, beta, eps, rho_, f, g, p=2):
    """Returns (primal value at the plan of Eq. (4), max marginal error)."""
    x, y = _pts(x), _pts(y)
    err = C.c_double()
    v = _load().oracle_ot_primal(x, _f32(alpha), x.shape[0], y, _f32(beta), y.shape[0], x.shape[1], int(p),
                                 float(eps), float(rho_), _f64(f), _f64(g), C.byref(err))
    return v, err.value


def transport_apply(x, y, beta, eps, f, g, labels, L, p=2):
    """Returns (scores N x L, argmax int32[N], row_mass[N])."""
    x, y = _pts(x), _pts(y)
    N = x.shape[0]
    sc = np.empty((N, L), np.float64)
    am = np.empty(N, np.int32)
    rm = np.empty(N, np.float64)
    _load().oracle_transport_apply(x, N, y, _f32(beta), y.shape[0], x.shape[1], int(p), float(eps), _f64(f),
                                   _f64(g), np.ascontiguousarray(labels, np.int32), int(L), sc, am, rm)
    return sc, am, rm


def flip_fibers(x, P=20):
    """2N x 3P: the N fibers, then their mirror flips (points in reverse order)."""
    x = _f32(x)
    N = x.shape[0]
    out = np.empty((2 * N, x.shape[1]), np.float32)
    _load().oracle_flip_fibers(x, N, int(P), out)
    return out


def select_flips(row_mass, argmax, N):
    """Per fiber: (label, version 0/1, row mass) of the version with the larger
    row mass among rows i and N + i of flip-augmented data."""
    label = np.empty(N, np.int32)
    version = np.empty(N, np.int32)
    mass = np.empty(N, np.float64)
    _load().oracle_select_flips(_f64(row_mass), np.ascontiguousarray(argmax, np.int32), int(N), label, version, mass)
    return label, version, mass


def cluster_grid(x, cell):
    """Returns (labels, perm, offsets, keys) of the Morton-ordered grid clustering."""
    x = _pts(x)
    N, D = x.shape
    labels = np.empty(N, np.int32)
    perm = np.empty(N, np.int32)
    offsets = np.empty(N + 1, np.int32)
    keys = np.empty(max(N, 1), np.uint32)
    n = _load().oracle_cluster_grid(x, N, D, float(cell), labels, perm, offsets, keys)
    if n < 0:
        raise ValueError("grid too fine: more than 1024 cells along an axis")
    return labels, perm, offsets[: n + 1].copy(), keys[:N]


def kmeans(x, w, K, iters, init):
    """Weighted Lloyd iterations from `init` (K x D). Returns (labels, centroids float64)."""
    x = _pts(x)
    N, D = x.shape
    labels = np.empty(N, np.int32)
    cent = np.empty((K, D), np.float64)
    wp = None if w is None else _f32(w)
    _load().oracle_kmeans(x, None if wp is None else wp.ctypes.data_as(C.c_void_p), N, D, int(K), int(iters),
                          _f32(init), labels, cent)
    return labels, cent
