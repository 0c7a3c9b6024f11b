"""CPU FP64 oracle: Python binding of oracle.c plus plain NumPy helpers.

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference legs may import this module.  It shares no code with
the CUDA library (it does not import the package that holds it), and nothing
on the product path calls it.

What it computes (arXiv 2407.06834):
  * patch features and window coordinates (Sec. 5);
  * direct O(N^2) ANOVA kernel sums, Eq. discrete_ANOVA, with the zero
    diagonal of Sec. 2.3 (Gamma) or with it kept (Gamma_full);
  * eta = Gamma 1, L = diag(eta) - Gamma, A = lambda I + mu L
    (Eq. discretized-state);
  * the Helmert change of basis U of Eq. ULap and its transpose;
  * the deflated CG of Sec. 4.1 / 4.3.2 in U coordinates (P_{U,a}, I_U) and
    CG / Jacobi-PCG in the original basis (Sec. 5.3-5.4);
  * the truncated Fourier series of the Gaussian that the fast summation of
    Sec. 3 evaluates, summed directly.

All pins of these functions live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        L = C.c_long
        sig = {
            "orc_num_threads": (C.c_int, []),
            "orc_patch_features": (None, [_dp, C.c_int, C.c_int, C.c_int, C.c_int, _dp]),
            "orc_window_coords": (None, [_dp, L, C.c_int, C.c_int, _ip, _dp]),
            "orc_gamma_full_rows": (None, [_dp, L, C.c_int, C.c_double, _dp, C.c_void_p, L, _dp]),
            "orc_gamma_full_matvec": (None, [_dp, L, C.c_int, C.c_double, _dp, _dp]),
            "orc_gamma_matvec": (None, [_dp, L, C.c_int, C.c_double, _dp, _dp]),
            "orc_gamma_dense": (None, [_dp, L, C.c_int, C.c_double, _dp]),
            "orc_degrees": (None, [_dp, L, C.c_int, C.c_double, _dp]),
            "orc_pb_diag": (None, [_dp, L, C.c_int, C.c_double, C.c_double, C.c_double, _dp]),
            "orc_A_apply": (None, [_dp, L, C.c_int, C.c_double, C.c_double, C.c_double, _dp, _dp, _dp]),
            "orc_gauss_fourier_coeff": (C.c_double, [C.c_double, C.c_double]),
            "orc_trig_kernel_1d": (C.c_double, [C.c_double, C.c_double, C.c_int]),
            "orc_torus_map": (C.c_double, [_dp, L, C.c_int, C.c_double, _dp]),
            "orc_trig_full_matvec": (None, [_dp, L, C.c_int, C.c_double, C.c_int, _dp, _dp]),
            "orc_U_apply": (None, [_dp, L, _dp]),
            "orc_Ut_apply": (None, [_dp, L, _dp]),
            "orc_pcg_deflated": (C.c_int, [_dp, L, C.c_int, C.c_double, C.c_double, C.c_double,
                                           _dp, C.c_double, C.c_int, C.c_int, _dp, _dp,
                                           C.POINTER(C.c_int)]),
            "orc_cg": (C.c_int, [_dp, L, C.c_int, C.c_double, C.c_double, C.c_double, _dp,
                                 C.c_void_p, C.c_double, C.c_int, C.c_int, _dp, _dp,
                                 C.POINTER(C.c_int)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().orc_num_threads())


# ---------------------------------------------------------------- features
def patch_features(img: np.ndarray, radius: int, pad: str = "reflect") -> np.ndarray:
    """n x (2 rho + 1)^2 patch features of Sec. 5 (row-major pixels)."""
    img = _f64(img)
    n1, n2 = img.shape
    D = (2 * radius + 1) ** 2
    out = np.empty((n1 * n2, D), dtype=np.float64)
    _load().orc_patch_features(img, n1, n2, radius, 1 if pad == "reflect" else 0, out)
    return out


def window_coords(feat: np.ndarray, windows: np.ndarray) -> np.ndarray:
    """(L, N, 3) window coordinates W_l[f]; -1 entries give zero dims."""
    feat = _f64(feat)
    N, D = feat.shape
    win = np.ascontiguousarray(windows, dtype=np.int32)
    L = win.shape[0]
    out = np.empty((L, N, 3), dtype=np.float64)
    _load().orc_window_coords(feat, N, D, L, win, out)
    return out


def image_coords(img: np.ndarray, radius: int, windows: np.ndarray,
                 pad: str = "reflect") -> np.ndarray:
    return window_coords(patch_features(img, radius, pad), windows)


# ---------------------------------------------------------------- kernel sums
def gamma_full_matvec(coords: np.ndarray, sigma: float, v: np.ndarray) -> np.ndarray:
    coords = _f64(coords)
    L, N, _ = coords.shape
    y = np.empty(N)
    _load().orc_gamma_full_matvec(coords, N, L, sigma, _f64(v), y)
    return y


def gamma_full_rows(coords: np.ndarray, sigma: float, v: np.ndarray,
                    rows: np.ndarray) -> np.ndarray:
    coords = _f64(coords)
    L, N, _ = coords.shape
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    y = np.empty(rows.shape[0])
    _load().orc_gamma_full_rows(coords, N, L, sigma, _f64(v),
                                rows.ctypes.data_as(C.c_void_p), rows.shape[0], y)
    return y


def gamma_matvec(coords: np.ndarray, sigma: float, v: np.ndarray) -> np.ndarray:
    coords = _f64(coords)
    L, N, _ = coords.shape
    y = np.empty(N)
    _load().orc_gamma_matvec(coords, N, L, sigma, _f64(v), y)
    return y


def gamma_dense(coords: np.ndarray, sigma: float) -> np.ndarray:
    coords = _f64(coords)
    L, N, _ = coords.shape
    G = np.empty((N, N))
    _load().orc_gamma_dense(coords, N, L, sigma, G)
    return G


def degrees(coords: np.ndarray, sigma: float) -> np.ndarray:
    coords = _f64(coords)
    L, N, _ = coords.shape
    eta = np.empty(N)
    _load().orc_degrees(coords, N, L, sigma, eta)
    return eta


def A_apply(coords: np.ndarray, sigma: float, lam: float, mu: float,
            v: np.ndarray, eta: np.ndarray | None = None) -> np.ndarray:
    coords = _f64(coords)
    L, N, _ = coords.shape
    if eta is None:
        eta = degrees(coords, sigma)
    y = np.empty(N)
    _load().orc_A_apply(coords, N, L, sigma, lam, mu, _f64(eta), _f64(v), y)
    return y


def laplacian_apply(coords, sigma, v, eta=None):
    """L v = diag(eta) v - Gamma v (lambda = 0, mu = 1)."""
    return A_apply(coords, sigma, 0.0, 1.0, v, eta)


# ---------------------------------------------------------------- Fourier side
def gauss_fourier_coeff(s: float, k) -> np.ndarray:
    lib = _load()
    k = np.atleast_1d(np.asarray(k, dtype=np.float64))
    return np.array([lib.orc_gauss_fourier_coeff(s, float(x)) for x in k])


def trig_kernel_1d(t, s: float, M: int) -> np.ndarray:
    lib = _load()
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    return np.array([lib.orc_trig_kernel_1d(float(x), s, M) for x in t])


def torus_map(coords: np.ndarray, fill: float):
    """Return (tcoords, s): x~ = s (x - midrange), s = fill / max range."""
    coords = _f64(coords)
    L, N, _ = coords.shape
    out = np.empty_like(coords)
    s = _load().orc_torus_map(coords, N, L, fill, out)
    return out, float(s)


def trig_full_matvec(tcoords: np.ndarray, sigma_s: float, M: int,
                     v: np.ndarray) -> np.ndarray:
    tcoords = _f64(tcoords)
    L, N, _ = tcoords.shape
    y = np.empty(N)
    _load().orc_trig_full_matvec(tcoords, N, L, sigma_s, M, _f64(v), y)
    return y


# ---------------------------------------------------------------- change of basis
def U_apply(x: np.ndarray) -> np.ndarray:
    x = _f64(x)
    u = np.empty_like(x)
    _load().orc_U_apply(x, x.shape[0], u)
    return u


def Ut_apply(x: np.ndarray) -> np.ndarray:
    x = _f64(x)
    g = np.empty_like(x)
    _load().orc_Ut_apply(x, x.shape[0], g)
    return g


# ---------------------------------------------------------------- solvers
class SolveResult:
    def __init__(self, u, hist, iters, status):
        self.u, self.hist, self.iters, self.status = u, hist, iters, status

    def __repr__(self):
        return "SolveResult(iters=%d, status=%d, res=%.3e)" % (
            self.iters, self.status, self.hist[self.iters])


def pcg_deflated(coords, sigma, lam, mu, b, tol=1e-6, maxit=200, precond=True):
    """The paper's decoupled CG in U coordinates: precond True / 1 = P_{U,a},
    2 = with P_b' (Sec. 4.3.3), False / 0 = I_U."""
    coords = _f64(coords)
    L, N, _ = coords.shape
    u = np.empty(N)
    hist = np.zeros(maxit + 1)
    it = C.c_int(0)
    st = _load().orc_pcg_deflated(coords, N, L, sigma, lam, mu, _f64(b), tol, maxit,
                                  int(precond), u, hist, C.byref(it))
    return SolveResult(u, hist, it.value, st)


def pb_diag(coords, sigma, lam, mu):
    """The diagonal of P_b' (Sec. 4.3.3, Eq. ANOVA_Norm_2_Prec)."""
    coords = _f64(coords)
    L, N, _ = coords.shape
    P = np.empty(N)
    _load().orc_pb_diag(coords, N, L, sigma, lam, mu, P)
    return P


def cg(coords, sigma, lam, mu, b, x0=None, tol=1e-6, maxit=200, precond=False):
    """CG (precond False / 0), Jacobi-PCG with P_a (True / 1) or with P_b'
    (2, Sec. 4.3.3), original basis."""
    coords = _f64(coords)
    L, N, _ = coords.shape
    u = np.empty(N)
    hist = np.zeros(maxit + 1)
    it = C.c_int(0)
    x0a = None if x0 is None else _f64(x0)
    st = _load().orc_cg(coords, N, L, sigma, lam, mu, _f64(b),
                        None if x0a is None else x0a.ctypes.data_as(C.c_void_p),
                        tol, maxit, int(precond), u, hist, C.byref(it))
    return SolveResult(u, hist, it.value, st)
