"""Thin ctypes binding of libotgb.so (include/otgb.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Tensors are torch CUDA tensors (device memory and streams come from
PyTorch); the functions keep the C names.  The library must be built
(``paper_2107_02010_gb300.build.build()``); there is no CPU fallback and a
missing library raises immediately.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

_lib = None


class Params(C.Structure):
    _fields_ = [
        ("p", C.c_int),
        ("blur", C.c_double),
        ("reach", C.c_double),
        ("scaling", C.c_double),
        ("diameter", C.c_double),
        ("multiscale", C.c_int),
        ("cluster", C.c_int),
        ("cell", C.c_double),
        ("k_clusters", C.c_int),
        ("kmeans_iters", C.c_int),
        ("seed", C.c_ulonglong),
        ("sigma_switch", C.c_double),
        ("trunc_tau", C.c_double),
        ("tol", C.c_double),
        ("min_iters", C.c_int),
        ("max_iters", C.c_int),
        ("check_every", C.c_int),
        ("fixed_iters", C.c_int),
        ("precision", C.c_int),
        ("f_init", C.c_void_p),
        ("g_init", C.c_void_p),
        ("a_init", C.c_void_p),
        ("b_init", C.c_void_p),
        ("sigma_start", C.c_double),
        ("translation", C.c_int),
        ("anderson", C.c_int),
        ("rows_per_thread", C.c_int),
        ("init_g_from_f", C.c_int),
        ("warm_max_iters", C.c_int),
        ("debug_wait_probe", C.c_int),
        ("polish", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("iters_total", C.c_int),
        ("iters_coarse", C.c_int),
        ("iters_fine", C.c_int),
        ("n_clusters_x", C.c_int),
        ("n_clusters_y", C.c_int),
        ("schedule_len", C.c_int),
        ("diameter", C.c_double),
        ("sigma_switch", C.c_double),
        ("pairs_evaluated", C.c_double),
        ("pairs_dense", C.c_double),
        ("kept_fraction", C.c_double),
        ("softmin_ms", C.c_double),
        ("total_ms", C.c_double),
        ("last_delta", C.c_double),
        ("last_rel_change", C.c_double),
        ("fallback_rows", C.c_longlong),
        ("warm_start", C.c_int),
        ("warm_iters", C.c_int),
        ("warm_ms", C.c_double),
        ("prep_ms", C.c_double),
        ("coarse_ms", C.c_double),
        ("fine_ms", C.c_double),
        ("final_ms", C.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


STATUS = {0: "OK", -1: "EINVAL", -2: "ECUDA", -3: "ENOMEM", -4: "ENOCONV", -5: "ENONFINITE", -6: "ETIMEOUT",
          -7: "EINTERNAL"}

EXPORTS = ["otgb_default_params", "otgb_create", "otgb_destroy", "otgb_last_error", "sinkhorn_divergence",
           "transport_apply", "otgb_plan_free", "cluster_grid", "cluster_kmeans", "otgb_softmin",
           "otgb_kernel_launches", "otgb_softmin_noalloc", "otgb_mlp_create", "otgb_mlp_destroy",
           "otgb_mlp_n_params", "otgb_mlp_fit_normalization", "otgb_mlp_set_normalization",
           "otgb_mlp_get_normalization", "otgb_mlp_set_params", "otgb_mlp_get_params", "otgb_mlp_grad",
           "otgb_mlp_adam_step", "otgb_mlp_train_step", "otgb_mlp_train_epoch", "otgb_mlp_infer", "otgb_mlp_save",
           "otgb_mlp_load", "sinkhorn_divergence_warm", "sinkhorn_grad_x", "sinkhorn_barycenter", "otgb_flip_fibers",
           "otgb_select_flips", "otgb_unit_rates"]


def kernel_launches() -> int:
    return int(load().otgb_kernel_launches())


class OtgbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libotgb.so (building it first if asked).  Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libotgb.so is not built; run paper_2107_02010_gb300.build.build()")
    lib = C.CDLL(_build.LIB)
    vp, ci, cd = C.c_void_p, C.c_int, C.c_double
    lib.otgb_default_params.argtypes = [C.POINTER(Params)]
    lib.otgb_default_params.restype = None
    lib.otgb_create.argtypes = [C.POINTER(vp), ci, vp]
    lib.otgb_destroy.argtypes = [vp]
    lib.otgb_last_error.argtypes = [vp]
    lib.otgb_last_error.restype = C.c_char_p
    lib.sinkhorn_divergence.argtypes = [vp, vp, vp, ci, vp, vp, ci, ci, C.POINTER(Params), C.POINTER(cd), vp, vp,
                                        vp, vp, C.POINTER(vp), C.POINTER(Stats)]
    lib.transport_apply.argtypes = [vp, vp, vp, vp, vp, ci, vp, vp, vp]
    lib.otgb_plan_free.argtypes = [vp]
    lib.otgb_plan_free.restype = None
    lib.cluster_grid.argtypes = [vp, vp, vp, ci, ci, C.c_float, vp, vp, vp, C.POINTER(ci), vp]
    lib.cluster_kmeans.argtypes = [vp, vp, vp, ci, ci, ci, ci, C.c_ulonglong, vp, vp, vp, vp, vp]
    lib.otgb_softmin.argtypes = [vp, vp, ci, vp, vp, vp, ci, ci, cd, cd, vp, cd, vp]
    lib.otgb_softmin_noalloc.argtypes = [vp, ci, vp, vp, vp, ci, ci, cd, cd, vp, cd, vp, vp]
    lib.otgb_softmin_noalloc.restype = ci
    lib.otgb_kernel_launches.argtypes = []
    lib.otgb_kernel_launches.restype = C.c_ulonglong
    fp = C.POINTER(C.c_float)
    lib.otgb_mlp_create.argtypes = [vp, ci, ci, C.c_ulonglong, C.POINTER(vp)]
    lib.otgb_mlp_destroy.argtypes = [vp]
    lib.otgb_mlp_n_params.argtypes = [vp]
    lib.otgb_mlp_fit_normalization.argtypes = [vp, vp, vp, ci]
    lib.otgb_mlp_set_normalization.argtypes = [vp, fp, fp, cd, cd]
    lib.otgb_mlp_get_normalization.argtypes = [vp, fp, fp, C.POINTER(cd), C.POINTER(cd)]
    lib.otgb_mlp_set_params.argtypes = [vp, fp, ci]
    lib.otgb_mlp_get_params.argtypes = [vp, fp, ci]
    lib.otgb_mlp_grad.argtypes = [vp, vp, vp, ci, C.POINTER(cd), vp]
    lib.otgb_mlp_adam_step.argtypes = [vp, vp, C.c_float]
    lib.otgb_mlp_train_step.argtypes = [vp, vp, vp, ci, C.c_float, C.POINTER(cd)]
    lib.otgb_mlp_train_epoch.argtypes = [vp, vp, vp, ci, ci, C.c_float, C.c_ulonglong, C.POINTER(cd)]
    lib.otgb_mlp_infer.argtypes = [vp, vp, ci, vp]
    lib.otgb_mlp_save.argtypes = [vp, C.c_char_p]
    lib.otgb_mlp_load.argtypes = [vp, C.c_char_p]
    lib.sinkhorn_divergence_warm.argtypes = [vp, vp, vp, vp, ci, vp, vp, ci, ci, C.POINTER(Params), vp,
                                             C.POINTER(cd), vp, vp, vp, vp, C.POINTER(vp), C.POINTER(Stats)]
    lib.sinkhorn_grad_x.argtypes = [vp, vp, vp, ci, vp, vp, ci, ci, ci, cd, vp, vp, vp, vp]
    lib.sinkhorn_barycenter.argtypes = [vp, vp, vp, ci, ci, C.POINTER(vp), C.POINTER(vp), C.POINTER(ci), ci,
                                        C.POINTER(Params), ci, cd, C.POINTER(cd)]
    lib.otgb_flip_fibers.argtypes = [vp, vp, ci, ci, vp]
    lib.otgb_unit_rates.argtypes = [vp, C.POINTER(cd), C.POINTER(cd), C.POINTER(cd)]
    lib.otgb_unit_rates.restype = ci
    lib.otgb_select_flips.argtypes = [vp, vp, vp, ci, vp, vp, vp]
    for name in ("otgb_flip_fibers", "otgb_select_flips", "sinkhorn_grad_x", "sinkhorn_barycenter", "otgb_create", "otgb_destroy", "sinkhorn_divergence",
                 "transport_apply", "cluster_grid",
                 "cluster_kmeans", "otgb_softmin", "otgb_mlp_create", "otgb_mlp_destroy", "otgb_mlp_n_params",
                 "otgb_mlp_fit_normalization", "otgb_mlp_set_normalization", "otgb_mlp_get_normalization",
                 "otgb_mlp_set_params", "otgb_mlp_get_params", "otgb_mlp_grad", "otgb_mlp_adam_step",
                 "otgb_mlp_train_step", "otgb_mlp_train_epoch", "otgb_mlp_infer", "otgb_mlp_save", "otgb_mlp_load",
                 "sinkhorn_divergence_warm"):
        getattr(lib, name).restype = ci
    _lib = lib
    return lib


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _f32(t):
    if t.dtype != torch.float32:
        raise TypeError("expected float32, got %s" % t.dtype)
    return _ptr(t)


def default_params(**kw) -> Params:
    p = Params()
    load().otgb_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Context:
    """An otgb context bound to the current CUDA device and stream."""

    def __init__(self, device=None, stream=None):
        lib = load()
        dev = torch.cuda.current_device() if device is None else int(device)
        st = torch.cuda.current_stream(dev) if stream is None else stream
        self.stream = st
        h = C.c_void_p()
        rc = lib.otgb_create(C.byref(h), dev, C.c_void_p(st.cuda_stream))
        if rc != 0:
            raise OtgbError(rc, lib.otgb_last_error(None).decode())
        self.h = h

    def check(self, rc):
        if rc != 0:
            raise OtgbError(rc, load().otgb_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            load().otgb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    def __init__(self, handle, keep):
        self.h = handle
        self._keep = keep  # the non-owning views must outlive the plan

    def __del__(self):
        if getattr(self, "h", None):
            load().otgb_plan_free(self.h)
            self.h = None


def sinkhorn_divergence(ctx: Context, x, a, y, b, params: Params | None = None, want_self=False,
                        want_plan=False, want_stats=True, raise_on_noconv=True):
    """Returns dict(S, f, g, [a_self, b_self], [plan], [stats], status)."""
    N, D = x.shape
    M = y.shape[0]
    f = torch.empty(N, device=x.device, dtype=torch.float32)
    g = torch.empty(M, device=x.device, dtype=torch.float32)
    aa = torch.empty(N, device=x.device, dtype=torch.float32) if want_self else None
    bb = torch.empty(M, device=x.device, dtype=torch.float32) if want_self else None
    cost = C.c_double()
    plan = C.c_void_p() if want_plan else None
    st = Stats() if want_stats else None
    p = params if params is not None else default_params()
    rc = load().sinkhorn_divergence(ctx.h, _f32(x), _f32(a), N, _f32(y), _f32(b), M, D, C.byref(p), C.byref(cost),
                                    _ptr(f), _ptr(g), _ptr(aa), _ptr(bb),
                                    C.byref(plan) if plan is not None else None,
                                    C.byref(st) if st is not None else None)
    if rc != 0 and not (rc == -4 and not raise_on_noconv):
        ctx.check(rc)
    out = dict(S=cost.value, f=f, g=g, status=rc)
    if want_self:
        out["a_self"], out["b_self"] = aa, bb
    if want_plan:
        out["plan"] = Plan(plan, (x, y, b))
    if want_stats:
        out["stats"] = st.as_dict()
    return out


def transport_apply(ctx: Context, plan: Plan, f, g, labels, L, want_scores=True):
    N = f.shape[0]
    sc = torch.empty((N, L), device=f.device, dtype=torch.float32) if want_scores else None
    am = torch.empty(N, device=f.device, dtype=torch.int32)
    rm = torch.empty(N, device=f.device, dtype=torch.float32)
    if labels.dtype != torch.int32:
        raise TypeError("labels must be int32")
    ctx.check(load().transport_apply(ctx.h, plan.h, _f32(f), _f32(g), _ptr(labels), int(L), _ptr(sc), _ptr(am),
                                     _ptr(rm)))
    return sc, am, rm


def sinkhorn_grad_x(ctx: Context, x, alpha, y, beta, eps, f, g, a_self, p=2):
    """dS(alpha, beta)/dx (N x D) from the duals of a solve (sinkhorn_grad_x).
    For dS/dy call sinkhorn_grad_x(ctx, y, beta, x, alpha, eps, g, f, b_self)."""
    N, D = x.shape
    M = y.shape[0]
    if y.shape[1] != D or alpha.numel() != N or beta.numel() != M:
        raise ValueError("sinkhorn_grad_x: shapes of x, alpha, y, beta do not match")
    if f.numel() != N or a_self.numel() != N or g.numel() != M:
        raise ValueError("sinkhorn_grad_x: f and a_self need N entries, g needs M")
    grad = torch.empty((N, D), device=x.device, dtype=torch.float32)
    ctx.check(load().sinkhorn_grad_x(ctx.h, _f32(x), _f32(alpha), N, _f32(y), _f32(beta), M, D, int(p), float(eps),
                                     _f32(f), _f32(g), _f32(a_self), _ptr(grad)))
    return grad


def sinkhorn_barycenter(ctx: Context, x, alpha, ys, betas, params: Params | None = None, iters=5, lr=1.0):
    """Free-support barycenter (sinkhorn_barycenter): moves x (N x D, float32,
    in place) and returns the objective history (iters + 1 values)."""
    N, D = x.shape
    K = len(ys)
    if len(betas) != K or K < 1:
        raise ValueError("sinkhorn_barycenter: one weight vector per measure")
    for y, b in zip(ys, betas):
        if y.dim() != 2 or y.shape[1] != D or b.numel() != y.shape[0]:
            raise ValueError("sinkhorn_barycenter: each measure needs M x D points and M weights")
    yp = (C.c_void_p * K)(*[_f32(y).value for y in ys])
    bp = (C.c_void_p * K)(*[_f32(b).value for b in betas])
    ms = (C.c_int * K)(*[int(y.shape[0]) for y in ys])
    hist = (C.c_double * (iters + 1))()
    p = params if params is not None else default_params()
    ctx.check(load().sinkhorn_barycenter(ctx.h, _f32(x), _f32(alpha), N, K, yp, bp, ms, D, C.byref(p), int(iters),
                                         float(lr), hist))
    return list(hist)


def unit_rates(ctx: Context):
    """otgb_unit_rates: measured lane operations per clock per SM of MUFU ex2,
    scalar FP32 FMA and packed FP32x2 FMA."""
    e, f, f2 = C.c_double(), C.c_double(), C.c_double()
    ctx.check(load().otgb_unit_rates(ctx.h, C.byref(e), C.byref(f), C.byref(f2)))
    return {"ex2": e.value, "fma": f.value, "fma2": f2.value}


def flip_fibers(ctx: Context, x, P=20):
    """otgb_flip_fibers: 2N x 3P, the fibers then their mirror flips."""
    N, D = x.shape
    if D != 3 * P:
        raise ValueError("flip_fibers: rows must hold 3P = %d coordinates" % (3 * P))
    out = torch.empty((2 * N, D), device=x.device, dtype=torch.float32)
    ctx.check(load().otgb_flip_fibers(ctx.h, _f32(x), N, int(P), _ptr(out)))
    return out


def select_flips(ctx: Context, row_mass, argmax):
    """otgb_select_flips on 2N augmented rows: (label, version, mass) per fiber."""
    if row_mass.numel() % 2 or argmax.numel() != row_mass.numel() or argmax.dtype != torch.int32:
        raise ValueError("select_flips: row_mass (float32) and argmax (int32) of 2N rows")
    N = row_mass.numel() // 2
    lab = torch.empty(N, device=row_mass.device, dtype=torch.int32)
    ver = torch.empty(N, device=row_mass.device, dtype=torch.int32)
    mass = torch.empty(N, device=row_mass.device, dtype=torch.float32)
    ctx.check(load().otgb_select_flips(ctx.h, _f32(row_mass), _ptr(argmax), N, _ptr(lab), _ptr(ver), _ptr(mass)))
    return lab, ver, mass


def cluster_grid(ctx: Context, x, cell, w=None, want_centroids=True):
    N, D = x.shape
    labels = torch.empty(N, device=x.device, dtype=torch.int32)
    perm = torch.empty(N, device=x.device, dtype=torch.int32)
    offsets = torch.empty(N + 1, device=x.device, dtype=torch.int32)
    cent = torch.empty((N, D), device=x.device, dtype=torch.float32) if want_centroids else None
    n = C.c_int()
    ctx.check(load().cluster_grid(ctx.h, _f32(x), _f32(w) if w is not None else None, N, D, float(cell),
                                  _ptr(labels), _ptr(perm), _ptr(offsets), C.byref(n), _ptr(cent)))
    k = n.value
    return labels, perm, offsets[: k + 1], (cent[:k] if cent is not None else None)


def cluster_kmeans(ctx: Context, x, K, iters=10, seed=0, w=None, init=None):
    N, D = x.shape
    labels = torch.empty(N, device=x.device, dtype=torch.int32)
    cent = torch.empty((K, D), device=x.device, dtype=torch.float32)
    perm = torch.empty(N, device=x.device, dtype=torch.int32)
    offsets = torch.empty(K + 1, device=x.device, dtype=torch.int32)
    ctx.check(load().cluster_kmeans(ctx.h, _f32(x), _f32(w) if w is not None else None, N, D, int(K), int(iters),
                                    int(seed), _f32(init) if init is not None else None, _ptr(labels), _ptr(cent),
                                    _ptr(perm), _ptr(offsets)))
    return labels, cent, perm, offsets


def _check_softmin_args(q, p, w, pot, old, out):
    """Shapes, dtypes and devices of a softmin call, checked before any pointer
    reaches the library (the kernels trust the sizes they are given)."""
    if q.dim() != 2 or p.dim() != 2:
        raise ValueError("q and p must be 2-D (rows x D, columns x D)")
    n_out, D = q.shape
    n_in = p.shape[0]
    if p.shape[1] != D:
        raise ValueError("p has %d coordinates, q has %d" % (p.shape[1], D))
    if w.numel() != n_in or pot.numel() != n_in:
        raise ValueError("w and pot must have one entry per column of p (%d)" % n_in)
    if old is not None and old.numel() != n_out:
        raise ValueError("old must have one entry per row of q (%d)" % n_out)
    if out is not None and out.numel() != n_out:
        raise ValueError("out must have one entry per row of q (%d)" % n_out)
    for name, t in (("q", q), ("p", p), ("w", w), ("pot", pot), ("old", old), ("out", out)):
        if t is None:
            continue
        if t.dtype != torch.float32:
            raise ValueError("%s must be float32, got %s" % (name, t.dtype))
        if t.device != q.device:
            raise ValueError("%s is on %s, q on %s: all tensors must be on one device" % (name, t.device, q.device))
    if not q.is_cuda:
        raise ValueError("expected CUDA tensors")
    return n_out, n_in, D


def softmin(ctx: Context, q, p, w, pot, eps, lam=1.0, old=None, omega=0.5):
    n_out, n_in, D = _check_softmin_args(q, p, w, pot, old, None)
    out = torch.empty(n_out, device=q.device, dtype=torch.float32)
    ctx.check(load().otgb_softmin(ctx.h, _f32(q), n_out, _f32(p), _f32(w), _f32(pot), n_in, D, float(eps),
                                  float(lam), _f32(old) if old is not None else None, float(omega), _ptr(out)))
    return out


def softmin_noalloc(q, p, w, pot, eps, lam=1.0, old=None, omega=0.5, out=None, stream=None):
    """otgb_softmin_noalloc: no context, no device allocation inside the call.
    `out` may be passed preallocated (float32, n_out) so that nothing at all
    is allocated on the device during the call.  The call runs with q's
    device current (the library looks up its fixed scratch array on the
    current device)."""
    n_out, n_in, D = _check_softmin_args(q, p, w, pot, old, out)
    lib = load()
    with torch.cuda.device(q.device):
        if out is None:
            out = torch.empty(n_out, device=q.device, dtype=torch.float32)
        st = torch.cuda.current_stream(q.device) if stream is None else stream
        rc = lib.otgb_softmin_noalloc(_f32(q), n_out, _f32(p), _f32(w), _f32(pot), n_in, D, float(eps),
                                      float(lam), _f32(old) if old is not None else None, float(omega), _ptr(out),
                                      C.c_void_p(st.cuda_stream))
    if rc != 0:
        raise OtgbError(rc, lib.otgb_last_error(None).decode())
    return out


class Mlp:
    """The warm-start network of a context (otgb_mlp_*): D -> H -> H -> H -> 1."""

    def __init__(self, ctx: Context, D: int, hidden: int = 256, seed: int = 0):
        h = C.c_void_p()
        ctx.check(load().otgb_mlp_create(ctx.h, int(D), int(hidden), int(seed), C.byref(h)))
        self.ctx, self.h, self.D, self.H = ctx, h, int(D), int(hidden)
        self.n_params = int(load().otgb_mlp_n_params(h))

    def close(self):
        if getattr(self, "h", None):
            load().otgb_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def fit_normalization(self, x, f=None):
        self.ctx.check(load().otgb_mlp_fit_normalization(self.h, _f32(x), _f32(f) if f is not None else None,
                                                         x.shape[0]))

    def set_normalization(self, in_mean, in_scale, out_mean, out_scale):
        import numpy as np
        m = np.ascontiguousarray(in_mean, dtype=np.float32)
        s = np.ascontiguousarray(in_scale, dtype=np.float32)
        fp = C.POINTER(C.c_float)
        self.ctx.check(load().otgb_mlp_set_normalization(self.h, m.ctypes.data_as(fp), s.ctypes.data_as(fp),
                                                         float(out_mean), float(out_scale)))

    def get_normalization(self):
        import numpy as np
        m = np.zeros(self.D, np.float32)
        s = np.zeros(self.D, np.float32)
        om, os_ = C.c_double(), C.c_double()
        fp = C.POINTER(C.c_float)
        self.ctx.check(load().otgb_mlp_get_normalization(self.h, m.ctypes.data_as(fp), s.ctypes.data_as(fp),
                                                         C.byref(om), C.byref(os_)))
        return m, s, om.value, os_.value

    def set_params(self, theta):
        import numpy as np
        t = np.ascontiguousarray(theta, dtype=np.float32)
        self.ctx.check(load().otgb_mlp_set_params(self.h, t.ctypes.data_as(C.POINTER(C.c_float)), t.size))

    def get_params(self):
        import numpy as np
        t = np.zeros(self.n_params, np.float32)
        self.ctx.check(load().otgb_mlp_get_params(self.h, t.ctypes.data_as(C.POINTER(C.c_float)), t.size))
        return t

    def grad(self, x, f):
        g = torch.empty(self.n_params, device=x.device, dtype=torch.float32)
        loss = C.c_double()
        self.ctx.check(load().otgb_mlp_grad(self.h, _f32(x), _f32(f), x.shape[0], C.byref(loss), _ptr(g)))
        return loss.value, g

    def adam_step(self, grad, lr):
        self.ctx.check(load().otgb_mlp_adam_step(self.h, _f32(grad), float(lr)))

    def train_step(self, x, f, lr):
        loss = C.c_double()
        self.ctx.check(load().otgb_mlp_train_step(self.h, _f32(x), _f32(f), x.shape[0], float(lr), C.byref(loss)))
        return loss.value

    def train_epoch(self, x, f, batch, lr, seed):
        loss = C.c_double()
        self.ctx.check(load().otgb_mlp_train_epoch(self.h, _f32(x), _f32(f), x.shape[0], int(batch), float(lr),
                                                   int(seed), C.byref(loss)))
        return loss.value

    def infer(self, x):
        out = torch.empty(x.shape[0], device=x.device, dtype=torch.float32)
        self.ctx.check(load().otgb_mlp_infer(self.h, _f32(x), x.shape[0], _ptr(out)))
        return out

    def save(self, path):
        self.ctx.check(load().otgb_mlp_save(self.h, str(path).encode()))

    def load_file(self, path):
        self.ctx.check(load().otgb_mlp_load(self.h, str(path).encode()))


def sinkhorn_divergence_warm(ctx: Context, mlp: Mlp, x, a, y, b, params: Params | None = None, b_atlas=None,
                             want_self=False, want_plan=False, raise_on_noconv=True):
    """Warm-started solve (sinkhorn_divergence_warm); returns the dict of
    sinkhorn_divergence with stats (stats["warm_start"]: 1 warm, 2 fell back)."""
    N, D = x.shape
    M = y.shape[0]
    f = torch.empty(N, device=x.device, dtype=torch.float32)
    g = torch.empty(M, device=x.device, dtype=torch.float32)
    aa = torch.empty(N, device=x.device, dtype=torch.float32) if want_self else None
    bb = torch.empty(M, device=x.device, dtype=torch.float32) if want_self else None
    cost = C.c_double()
    plan = C.c_void_p() if want_plan else None
    st = Stats()
    p = params if params is not None else default_params()
    rc = load().sinkhorn_divergence_warm(ctx.h, mlp.h, _f32(x), _f32(a), N, _f32(y), _f32(b), M, D, C.byref(p),
                                         _f32(b_atlas) if b_atlas is not None else None, C.byref(cost), _ptr(f),
                                         _ptr(g), _ptr(aa), _ptr(bb), C.byref(plan) if plan is not None else None,
                                         C.byref(st))
    if rc != 0 and not (rc == -4 and not raise_on_noconv):
        ctx.check(rc)
    out = dict(S=cost.value, f=f, g=g, status=rc, stats=st.as_dict())
    if want_self:
        out["a_self"], out["b_self"] = aa, bb
    if want_plan:
        out["plan"] = Plan(plan, (x, y, b))
    return out
