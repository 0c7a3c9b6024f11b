"""CPU FP64 oracle of the bilevel parameter learning (Sec. 2 and Sec. 5.5).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference legs may import this module.  It shares no code with
the CUDA library and nothing on the product path calls it.

For training pairs (u_c,t clean, f_t noisy), t = 1..T, and mu = 1, alpha =
lambda (Eq. BilevelProblem):
    j(alpha) = (1/T) sum_t ||u_c,t - u_t(alpha)||^2,
    (alpha I + L_t) u_t = alpha f_t          (the lower-level problem).
Differentiating the constraint gives u_t + A_t u_t' = f_t, so with the
adjoint states A_t p_t = u_t - u_c,t (second line of the optimality system,
Eq. Optimality_System_Regularization):
    dj/dalpha = (2/T) sum_t <p_t, f_t - u_t>.
The system matrices are dense (oracle.gamma_dense), the solves LAPACK.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

from . import oracle as orc


def laplacians(coords_list: Sequence[np.ndarray], sigma: float) -> List[np.ndarray]:
    """Dense L_t = diag(Gamma 1) - Gamma (zero-diagonal Gamma) per image."""
    out = []
    for coords in coords_list:
        G = orc.gamma_dense(coords, sigma)
        out.append(np.diag(G.sum(axis=1)) - G)
    return out


def lower_level(L: np.ndarray, f: np.ndarray, alpha: float) -> np.ndarray:
    n = f.size
    return np.linalg.solve(alpha * np.eye(n) + L, alpha * f)


def objective_and_gradient(Ls: Sequence[np.ndarray], fs: Sequence[np.ndarray],
                           ucs: Sequence[np.ndarray], alpha: float) -> Tuple[float, float]:
    """(j(alpha), dj/dalpha) by the adjoint formula."""
    T = len(Ls)
    j = 0.0
    g = 0.0
    for L, f, uc in zip(Ls, fs, ucs):
        n = f.size
        A = alpha * np.eye(n) + L
        u = np.linalg.solve(A, alpha * f)
        p = np.linalg.solve(A, u - uc)
        j += np.sum((uc - u) ** 2)
        g += 2.0 * np.dot(p, f - u)
    return j / T, g / T


def learn_alpha(Ls, fs, ucs, bounds=(1e-3, 10.0), xatol=1e-6):
    """Brent's bounded minimisation of j over log alpha (scipy's
    implementation of Brent's method)."""
    from scipy.optimize import minimize_scalar
    fun = lambda la: objective_and_gradient(Ls, fs, ucs, float(np.exp(la)))[0]
    res = minimize_scalar(fun, bounds=(np.log(bounds[0]), np.log(bounds[1])), method="bounded",
                          options={"xatol": xatol})
    return float(np.exp(res.x)), float(res.fun), int(res.nfev)
