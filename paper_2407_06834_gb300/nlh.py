"""Python binding of libnlh (include/nlh.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this
module converts torch CUDA tensors to device pointers and the current torch
stream to a cudaStream_t.  It raises if the native library cannot be loaded:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libnlh.so")
_lock = threading.Lock()
_lib = None

NLH_OK, NLH_ERR_NOT_CONVERGED = 0, 1
NLH_FP64, NLH_FP32, NLH_DF32 = 0, 1, 2
PREC_PA, PREC_PB = 0, 1      # Jacobi P_a, and P_b' of Sec. 4.3.3
CG, PCG_JACOBI, PCG_DEFLATED, CG_DEFLATED = 0, 1, 2, 3
SOLVE_FP64, SOLVE_MIXED, SOLVE_DF32 = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "NOT_CONVERGED", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_OOM",
                -4: "ERR_BREAKDOWN", -5: "ERR_TIMEOUT"}


# nlh_reduce_fn: (buf, n, stream, ctx) -> None, called on the host at enqueue time.
REDUCE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p)


class PlanDesc(C.Structure):
    _fields_ = [("N", C.c_int64), ("D", C.c_int), ("L", C.c_int),
                ("windows", C.POINTER(C.c_int32)), ("sigma", C.c_double), ("M", C.c_int),
                ("n_os", C.c_int), ("m", C.c_int), ("precision", C.c_int),
                ("torus_fill", C.c_double), ("max_items_pts", C.c_int),
                ("nfft_eps", C.c_double), ("unit_points", C.c_int), ("team", C.c_int * 3),
                ("window_first", C.c_int), ("window_count", C.c_int), ("reduce", REDUCE_FN),
                ("reduce_ctx", C.c_void_p), ("image", C.c_void_p), ("image_n1", C.c_int),
                ("image_n2", C.c_int), ("patch_radius", C.c_int), ("patch_pad", C.c_int)]


class PlanInfo(C.Structure):
    _fields_ = [("N", C.c_int64), ("L", C.c_int), ("M", C.c_int), ("n_os", C.c_int),
                ("m", C.c_int), ("precision", C.c_int), ("sigma", C.c_double),
                ("torus_fill", C.c_double), ("scale", C.c_double), ("sigma_torus", C.c_double),
                ("max_range", C.c_double), ("n_items", C.c_int64),
                ("occupied_cells", C.c_int64), ("est_trunc_err", C.c_double),
                ("est_alias_err", C.c_double), ("device_bytes", C.c_int64),
                ("n_units", C.c_int64), ("max_items_pts", C.c_int), ("unit_points", C.c_int),
                ("team", C.c_int * 3), ("window_first", C.c_int), ("window_count", C.c_int),
                ("coords_from_image", C.c_int)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("method", C.c_int),
                ("arith", C.c_int), ("inner_tol", C.c_double), ("max_outer", C.c_int),
                ("x0", C.c_void_p), ("diag_scale", C.c_void_p), ("hist", C.c_void_p),
                ("hist_len", C.c_int), ("check_every", C.c_int), ("x0_check", C.c_int),
                ("precond", C.c_int)]


class NetBatch(C.Structure):
    _fields_ = [("B", C.c_int), ("H", C.c_int), ("W", C.c_int), ("f", C.c_void_p),
                ("sigma", C.POINTER(C.c_double)), ("alpha", C.POINTER(C.c_double)),
                ("ustar", C.c_void_p), ("e0", C.c_void_p), ("r0", C.c_void_p),
                ("deg", C.c_void_p), ("beta", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("outer", C.c_int), ("matvecs_fp64", C.c_int),
                ("matvecs_fp32", C.c_int), ("rel_res", C.c_double),
                ("rel_res_true", C.c_double), ("seconds", C.c_double),
                ("used_fallback", C.c_int), ("status", C.c_int), ("x0_rejected", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# Every entry point of include/nlh.h with its ctypes signature.
SIGNATURES = {
    "nlh_patch_features": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.c_void_p, C.c_void_p]),
    "nlh_plan_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(PlanDesc), C.c_void_p,
                                  C.c_void_p]),
    "nlh_plan_set_sigma": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p]),
    "nlh_plan_get_info": (C.c_int, [C.c_void_p, C.POINTER(PlanInfo)]),
    "nlh_matvec": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_void_p,
                             C.c_void_p, C.c_void_p]),
    "nlh_solve": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                            C.POINTER(SolveOpts), C.POINTER(SolveInfo), C.c_void_p]),
    "nlh_solve_batched": (C.c_int, [C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_double),
                                    C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                    C.POINTER(SolveOpts), C.POINTER(SolveInfo), C.c_void_p]),
    "nlh_plan_retile": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "nlh_plan_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int),
                                    C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double),
                                    C.c_void_p]),
    "nlh_plan_set_team": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "nlh_plan_destroy": (C.c_int, [C.c_void_p]),
    "nlh_last_error": (C.c_char_p, []),
    "nlh_version": (C.c_char_p, []),
    "nlh_residual_norms_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                             C.c_void_p, C.c_void_p]),
    "nlh_plan_get_degrees": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "nlh_net_create": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "nlh_net_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
    "nlh_net_layer": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                C.POINTER(C.c_int)]),
    "nlh_net_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "nlh_net_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "nlh_net_get_grads": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "nlh_net_forward": (C.c_int, [C.c_void_p, C.POINTER(NetBatch), C.c_void_p, C.c_void_p,
                                  C.c_void_p]),
    "nlh_net_residual_error": (C.c_int, [C.c_void_p, C.POINTER(NetBatch), C.c_void_p,
                                         C.c_void_p]),
    "nlh_net_loss_grad": (C.c_int, [C.c_void_p, C.POINTER(NetBatch), C.POINTER(C.c_double),
                                    C.c_void_p]),
    "nlh_net_adam": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double,
                               C.c_void_p]),
    "nlh_net_set_engine": (C.c_int, [C.c_void_p, C.c_int]),
    "nlh_net_get_engine": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "nlh_net_check": (C.c_int, [C.c_void_p, C.c_void_p]),
    "nlh_net_destroy": (C.c_int, [C.c_void_p]),
    "nlh_bilevel_misfit": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.POINTER(C.c_double), C.c_void_p]),
    "nlh_bilevel_gradient_term": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.POINTER(C.c_double), C.c_void_p]),
    "nlh_mis_windows": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "nlh_selftest_plan_timeout": (C.c_int, [C.c_void_p, C.c_void_p]),
    "nlh_selftest_net_timeout": (C.c_int, [C.c_void_p, C.c_void_p]),
    "nlh_selftest_inner_tolerance": (C.c_double, [C.c_double, C.c_double, C.c_double]),
    "nlh_selftest_convergence": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_int]),
    "nlh_kernel_launches": (C.c_int64, []),
    "nlh_profile_enable": (C.c_int, [C.c_int]),
    "nlh_profile_reset": (C.c_int, []),
    "nlh_profile_read": (C.c_int, [C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
}


def lib_path() -> str:
    return _LIB_PATH


def load(build_if_missing: bool = True):
    """Load libnlh.so (building it in-tree first if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH) and build_if_missing:
            from . import build_native
            build_native.build()
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError("libnlh.so not found at %s; run __graft_entry__.build()" % _LIB_PATH)
        lib = C.CDLL(_LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class NLHError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(status, "?"), status, msg))
        self.status = status


def _check(status: int, allow_not_converged: bool = False) -> int:
    if status == NLH_OK or (allow_not_converged and status == NLH_ERR_NOT_CONVERGED):
        return status
    raise NLHError(status, load().nlh_last_error().decode())


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None) -> int:
    torch = _torch()
    st = stream if stream is not None else torch.cuda.current_stream()
    return int(st.cuda_stream)


def _iptr(t) -> int:
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int32
            and t.is_contiguous()):
        raise TypeError("expected a contiguous int32 CUDA tensor")
    return int(t.data_ptr())


def _dptr(t, n: Optional[int] = None) -> int:
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError("expected %d elements, got %d" % (n, t.numel()))
    return int(t.data_ptr())


def patch_features(image, radius: int, pad: str = "reflect", stream=None):
    """(n1 n2, (2 radius + 1)^2) patch features of a CUDA float64 image."""
    torch = _torch()
    n1, n2 = image.shape
    D = (2 * radius + 1) ** 2
    out = torch.empty((n1 * n2, D), dtype=torch.float64, device=image.device)
    _check(load().nlh_patch_features(_dptr(image), n1, n2, radius, 1 if pad == "reflect" else 0,
                                     _dptr(out), _stream_ptr(stream)))
    return out


def mis_windows(image, radius: int, pad: str = "reflect", bins: int = 64, want_counts=False,
                stream=None):
    """Feature windows ranked by mutual information (include/nlh_mis.h).

    Returns (mis, windows, counts): mis a CUDA float64 tensor of the D
    scores, windows an int32 (L, 3) host array for Plan, counts the CUDA
    int32 (D, bins, bins) joint histograms or None."""
    torch = _torch()
    n1, n2 = image.shape
    D = (2 * radius + 1) ** 2
    L = -(-D // 3)
    mis = torch.empty(D, dtype=torch.float64, device=image.device)
    win = torch.empty((L, 3), dtype=torch.int32, device=image.device)
    cnt = (torch.empty((D, bins, bins), dtype=torch.int32, device=image.device)
           if want_counts else None)
    _check(load().nlh_mis_windows(_dptr(image), n1, n2, int(radius),
                                  1 if pad == "reflect" else 0, int(bins), _dptr(mis),
                                  _iptr(win), None if cnt is None else _iptr(cnt),
                                  _stream_ptr(stream)))
    return mis, win.cpu().numpy(), cnt


@dataclass
class SolveResult:
    u: object
    info: dict
    hist: np.ndarray


def _device_view(ptr: int, n: int):
    """A torch view of n device FP64 values at ptr (no copy), through the CUDA
    array interface."""
    torch = _torch()

    class _View:
        __cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8",
                                    "data": (int(ptr), False), "version": 3, "strides": None}
    return torch.as_tensor(_View(), device="cuda")


class Plan:
    """An NFFT plan for one feature matrix (see nlh_plan_create).

    window_range=(first, count) builds the plan of that range of the windows
    only; reduce, a callable (buf, stream) -> None that sums the FP64 CUDA
    tensor buf in place over all ranks on that torch stream, makes such a
    plan act as the operator of all windows (nlh_reduce_fn)."""

    def __init__(self, features, windows, sigma: float, M: int = 32, n_os: int = 64, m: int = 4,
                 precision: int = 3, torus_fill: float = 0.0, max_items_pts: int = 0,
                 nfft_eps: float = 0.0, unit_points: int = 0, autotune: bool = False,
                 team=None, window_range=None, reduce=None, image=None, stream=None):
        """image: None, or (image, radius, pad) when the features are that
        image's patches; the plan then recomputes coordinates from it."""
        lib = load()
        N, D = features.shape
        win = np.ascontiguousarray(np.asarray(windows, dtype=np.int32).reshape(-1, 3))
        self._win = win
        tuned = None
        if autotune and nfft_eps == 0.0 and not max_items_pts and not unit_points:
            from . import autotune as _at
            tuned = _at.lookup(n_os, m, win.shape[0], N)
            if tuned:
                max_items_pts, unit_points = tuned["max_items_pts"], tuned["unit_points"]
                team = tuned.get("team", team)
        wf, wc = window_range if window_range is not None else (0, 0)
        self._reduce = None
        if reduce is not None:
            torch = _torch()

            def _cb(buf, n, stream_ptr, ctx, _fn=reduce):
                st = torch.cuda.ExternalStream(int(stream_ptr or 0)) if stream_ptr else \
                    torch.cuda.default_stream()
                _fn(_device_view(buf, n), st)
            self._reduce = REDUCE_FN(_cb)
        desc = PlanDesc(N=N, D=D, L=win.shape[0],
                        windows=win.ctypes.data_as(C.POINTER(C.c_int32)), sigma=float(sigma),
                        M=M, n_os=n_os, m=m, precision=precision,
                        torus_fill=float(torus_fill), max_items_pts=max_items_pts,
                        nfft_eps=float(nfft_eps), unit_points=unit_points,
                        team=(C.c_int * 3)(*(team or (0, 0, 0))), window_first=int(wf),
                        window_count=int(wc),
                        reduce=self._reduce if self._reduce is not None else REDUCE_FN(),
                        reduce_ctx=None)
        if image is not None:
            img, radius, pad = image
            n1, n2 = img.shape
            desc.image = _dptr(img, n1 * n2)
            desc.image_n1, desc.image_n2 = int(n1), int(n2)
            desc.patch_radius = int(radius)
            desc.patch_pad = 1 if pad == "reflect" else 0
        h = C.c_void_p()
        _check(lib.nlh_plan_create(C.byref(h), C.byref(desc), _dptr(features),
                                   _stream_ptr(stream)))
        self._h = h
        self.N = N
        self.L = win.shape[0]
        if autotune and not tuned and window_range is None:
            from . import autotune as _at
            hit = None
            if nfft_eps > 0.0:
                # the class (n_os, m) is known only now: apply a cached result
                inf = self.info()
                hit = _at.lookup(inf["n_os"], inf["m"], self.L, N)
            if hit:
                self.retile(hit["max_items_pts"], hit["unit_points"], stream=stream)
                for arith, shape in enumerate(hit.get("team", (0, 0, 0))):
                    self.set_team(arith, shape)
            else:
                _at.tune_and_record(self, stream=stream)

    @classmethod
    def from_image(cls, image, radius: int, windows, sigma: float, pad: str = "reflect",
                   coords_from_image: bool = False, **kw):
        """Plan of the image's patch features.  coords_from_image: the NFFT
        kernels recompute the points' coordinates from the image instead of
        reading stored offsets (less memory and DRAM traffic, slower)."""
        feats = patch_features(image, radius, pad, kw.get("stream"))
        img = image.contiguous() if coords_from_image else None
        return cls(feats, windows, sigma, image=(img, radius, pad) if coords_from_image else None,
                   **kw)

    @property
    def handle(self) -> int:
        return self._h.value

    def info(self) -> dict:
        inf = PlanInfo()
        _check(load().nlh_plan_get_info(self._h, C.byref(inf)))
        d = {k: getattr(inf, k) for k, _ in inf._fields_}
        d["team"] = list(inf.team)
        return d

    def retile(self, max_items_pts: int, unit_points: int, stream=None):
        _check(load().nlh_plan_retile(self._h, int(max_items_pts), int(unit_points),
                                      _stream_ptr(stream)))

    def autotune(self, precisions: int = 0, reps: int = 3, stream=None):
        k, u, ms = C.c_int(0), C.c_int(0), C.c_double(0)
        t = (C.c_int * 3)()
        _check(load().nlh_plan_autotune(self._h, precisions, reps, C.byref(k), C.byref(u), t,
                                        C.byref(ms), _stream_ptr(stream)))
        return {"max_items_pts": k.value, "unit_points": u.value, "team": list(t),
                "ms": ms.value}

    def set_team(self, arith: int, shape: int):
        _check(load().nlh_plan_set_team(self._h, int(arith), int(shape)))

    def degrees(self, out=None, stream=None):
        """d = Gamma_full 1 in pixel order (nlh_plan_get_degrees)."""
        torch = _torch()
        d = out if out is not None else torch.empty(self.N, dtype=torch.float64, device="cuda")
        _check(load().nlh_plan_get_degrees(self._h, _dptr(d, self.N), _stream_ptr(stream)))
        return d

    def set_sigma(self, sigma: float, stream=None):
        _check(load().nlh_plan_set_sigma(self._h, float(sigma), _stream_ptr(stream)))

    def matvec(self, x, op: int = 0, precision: int = NLH_FP64, alpha: float = 0.0, out=None,
               stream=None):
        torch = _torch()
        y = out if out is not None else torch.empty_like(x)
        _check(load().nlh_matvec(self._h, op, precision, float(alpha), _dptr(x, self.N),
                                 _dptr(y, self.N), _stream_ptr(stream)))
        return y

    def solve(self, alpha: float, b, tol: float = 1e-6, maxit: int = 200,
              method: int = PCG_DEFLATED, arith: int = SOLVE_FP64, inner_tol: float = 0.0,
              max_outer: int = 0, x0=None, diag_scale=None, u=None, check_every: int = 0,
              x0_check: bool = False, precond: int = 0,
              hist_len: int = 256, stream=None) -> SolveResult:
        torch = _torch()
        u = u if u is not None else torch.empty_like(b)
        hist = np.zeros(hist_len)
        opts = SolveOpts(tol=tol, maxit=maxit, method=method, arith=arith, inner_tol=inner_tol,
                         max_outer=max_outer,
                         x0=None if x0 is None else _dptr(x0, self.N),
                         diag_scale=None if diag_scale is None else _dptr(diag_scale, self.N),
                         hist=hist.ctypes.data, hist_len=hist_len, check_every=check_every,
                         x0_check=1 if x0_check else 0, precond=int(precond))
        info = SolveInfo()
        st = load().nlh_solve(self._h, float(alpha), _dptr(b, self.N), _dptr(u, self.N),
                              C.byref(opts), C.byref(info), _stream_ptr(stream))
        _check(st, allow_not_converged=True)
        d = info.as_dict()
        n = (d["iters"] + 1) if arith != SOLVE_MIXED else d["outer"]
        return SolveResult(u, d, hist[:max(0, min(n, hist_len))].copy())

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().nlh_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batched(plans, alphas, bs, us=None, tol: float = 1e-6, maxit: int = 200,
                  method: int = PCG_DEFLATED, arith: int = SOLVE_MIXED, inner_tol: float = 0.0,
                  max_outer: int = 0, precond: int = 0, stream=None):
    """Solve (alpha_i I + L_i) u_i = b_i for many plans at once (nlh_solve_batched)."""
    torch = _torch()
    n = len(plans)
    us = us if us is not None else [torch.empty_like(b) for b in bs]
    hp = (C.c_void_p * n)(*[p.handle for p in plans])
    ha = (C.c_double * n)(*[float(a) for a in alphas])
    hb = (C.c_void_p * n)(*[_dptr(b, p.N) for b, p in zip(bs, plans)])
    hu = (C.c_void_p * n)(*[_dptr(u, p.N) for u, p in zip(us, plans)])
    opts = SolveOpts(tol=tol, maxit=maxit, method=method, arith=arith, inner_tol=inner_tol,
                     max_outer=max_outer, x0=None, diag_scale=None, hist=None, hist_len=0,
                     check_every=0, x0_check=0, precond=int(precond))
    infos = (SolveInfo * n)()
    st = load().nlh_solve_batched(n, hp, ha, hb, hu, C.byref(opts), infos, _stream_ptr(stream))
    _check(st, allow_not_converged=True)
    return us, [infos[i].as_dict() for i in range(n)]


def bilevel_misfit(u, uc, r=None, stream=None) -> float:
    """||u - uc||^2, and r = u - uc when given (nlh_bilevel_misfit)."""
    n = u.numel()
    sq = C.c_double(0)
    _check(load().nlh_bilevel_misfit(n, _dptr(u, n), _dptr(uc, n),
                                     None if r is None else _dptr(r, n), C.byref(sq),
                                     _stream_ptr(stream)))
    return sq.value


def bilevel_gradient_term(p, f, u, stream=None) -> float:
    """<p, f - u> (nlh_bilevel_gradient_term)."""
    n = u.numel()
    dot = C.c_double(0)
    _check(load().nlh_bilevel_gradient_term(n, _dptr(p, n), _dptr(f, n), _dptr(u, n),
                                            C.byref(dot), _stream_ptr(stream)))
    return dot.value


class Net:
    """The learned warm start and diagonal correction (include/nlh_net.h).

    Images are CUDA float64 tensors of shape (B, H, W) (or (H, W)); sigma and
    alpha are sequences of B floats."""

    def __init__(self, base: int = 32, levels: int = 4):
        h = C.c_void_p()
        _check(load().nlh_net_create(int(base), int(levels), C.byref(h)))
        self._h = h
        self.base, self.levels = base, levels
        nl, npar = C.c_int(), C.c_int64()
        _check(load().nlh_net_info(h, C.byref(nl), C.byref(npar)))
        self.n_params = npar.value
        self.layers = []
        for i in range(nl.value):
            a, b, k = C.c_int(), C.c_int(), C.c_int()
            _check(load().nlh_net_layer(h, i, C.byref(a), C.byref(b), C.byref(k)))
            self.layers.append((a.value, b.value, k.value))

    ENGINE_MMA_SYNC, ENGINE_TCGEN05 = 0, 1

    @property
    def engine(self) -> int:
        """Engine of the 3x3 convolutions: 1 = tcgen05 (default), 0 = mma.sync."""
        e = C.c_int()
        _check(load().nlh_net_get_engine(self._h, C.byref(e)))
        return e.value

    @engine.setter
    def engine(self, value: int) -> None:
        _check(load().nlh_net_set_engine(self._h, int(value)))

    def check(self, stream=None) -> None:
        """Synchronise and raise if a bounded tensor-core wait gave up."""
        _check(load().nlh_net_check(self._h, _stream_ptr(stream)))

    def shapes(self):
        """(cout, k, cin) per layer, the order of the parameter vector."""
        return [(cout, k, cin) for cin, cout, k in self.layers]

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        _check(load().nlh_net_set_params(self._h, th.ctypes.data, th.size))

    def params(self) -> np.ndarray:
        th = np.empty(self.n_params, dtype=np.float32)
        _check(load().nlh_net_get_params(self._h, th.ctypes.data, th.size))
        return th

    def grads(self) -> np.ndarray:
        g = np.empty(self.n_params, dtype=np.float32)
        _check(load().nlh_net_get_grads(self._h, g.ctypes.data, g.size))
        return g

    @staticmethod
    def _batch(f, sigma, alpha, ustar=None, e0=None, r0=None, deg=None, beta=0.0):
        if f.dim() == 2:
            f = f.unsqueeze(0)
        B, H, W = f.shape
        n = B * H * W
        sig = (C.c_double * B)(*[float(x) for x in np.broadcast_to(np.asarray(sigma, float), (B,))])
        alp = (C.c_double * B)(*[float(x) for x in np.broadcast_to(np.asarray(alpha, float), (B,))])
        opt = lambda t: None if t is None else _dptr(t, n)
        nb = NetBatch(B=B, H=H, W=W, f=_dptr(f, n), sigma=sig, alpha=alp, ustar=opt(ustar),
                      e0=opt(e0), r0=opt(r0), deg=opt(deg), beta=float(beta))
        nb._keep = (sig, alp)
        return nb, f.shape

    def forward(self, f, sigma, alpha, u0=None, scale=None, want=("u0", "scale"), stream=None):
        """Return (u0, scale) as CUDA float64 tensors shaped like f."""
        torch = _torch()
        nb, shape = self._batch(f, sigma, alpha)
        if "u0" in want and u0 is None:
            u0 = torch.empty(shape, dtype=torch.float64, device=f.device)
        if "scale" in want and scale is None:
            scale = torch.empty(shape, dtype=torch.float64, device=f.device)
        n = nb.B * nb.H * nb.W
        _check(load().nlh_net_forward(self._h, C.byref(nb),
                                      None if u0 is None else _dptr(u0, n),
                                      None if scale is None else _dptr(scale, n),
                                      _stream_ptr(stream)))
        return u0, scale

    def residual_error(self, f, sigma, alpha, ustar, e0=None, stream=None):
        """e0 = ustar - u0 for the current parameters."""
        torch = _torch()
        nb, shape = self._batch(f, sigma, alpha, ustar=ustar)
        e0 = e0 if e0 is not None else torch.empty(shape, dtype=torch.float64, device=f.device)
        _check(load().nlh_net_residual_error(self._h, C.byref(nb), _dptr(e0, e0.numel()),
                                             _stream_ptr(stream)))
        return e0

    def loss_grad(self, f, sigma, alpha, ustar, e0=None, r0=None, deg=None, beta=0.0,
                  want_loss=True, stream=None):
        nb, _ = self._batch(f, sigma, alpha, ustar, e0, r0, deg, beta)
        loss = C.c_double(float("nan"))
        _check(load().nlh_net_loss_grad(self._h, C.byref(nb), C.byref(loss) if want_loss else None,
                                        _stream_ptr(stream)))
        return loss.value if want_loss else None

    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
             stream=None):
        _check(load().nlh_net_adam(self._h, float(lr), float(beta1), float(beta2), float(eps),
                                   _stream_ptr(stream)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().nlh_net_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
