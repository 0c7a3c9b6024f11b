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
The joint learning of (alpha, theta = sigma^-2) of Sec. 5.5 minimises
j(alpha, sigma) by L-BFGS-B with a central difference in log theta.
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


def objective_sigma(coords_list, fs, ucs, alpha: float, sigma: float) -> float:
    """j(alpha, sigma) with the Laplacians rebuilt for sigma."""
    return objective_and_gradient(laplacians(coords_list, sigma), fs, ucs, alpha)[0]


def learn_alpha_theta(coords_list, fs, ucs, alpha0, sigma0, bounds_alpha=(1e-3, 1e3),
                      bounds_sigma=(0.05, 1.0), rel_step=1e-4):
    """Joint (alpha, theta = sigma^-2) learning (Sec. 5.5) by L-BFGS-B over
    (log alpha, log theta); dj/dalpha by the adjoint formula, dj/dtheta by a
    central difference in log theta."""
    from scipy.optimize import minimize

    def fg(z):
        a, th = float(np.exp(z[0])), float(np.exp(z[1]))
        j, ga = objective_and_gradient(laplacians(coords_list, th ** -0.5), fs, ucs, a)
        jp = objective_sigma(coords_list, fs, ucs, a, float(np.exp(z[1] + rel_step)) ** -0.5)
        jm = objective_sigma(coords_list, fs, ucs, a, float(np.exp(z[1] - rel_step)) ** -0.5)
        return j, np.array([ga * a, (jp - jm) / (2 * rel_step)])

    lt_b = (np.log(bounds_sigma[1] ** -2), np.log(bounds_sigma[0] ** -2))
    res = minimize(fg, np.array([np.log(alpha0), np.log(sigma0 ** -2)]), jac=True,
                   method="L-BFGS-B",
                   bounds=[(np.log(bounds_alpha[0]), np.log(bounds_alpha[1])), lt_b],
                   options={"maxiter": 50, "ftol": 1e-12, "gtol": 1e-8})
    th = float(np.exp(res.x[1]))
    return float(np.exp(res.x[0])), th ** -0.5, float(res.fun)
