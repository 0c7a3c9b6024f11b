"""Bilevel learning of the fidelity weight alpha = lambda / mu (Sec. 2 and
Sec. 5.5, Eq. BilevelProblem), on top of the library's batched solves.

For training pairs (u_c,t clean, f_t noisy):
    j(alpha) = (1/T) sum_t ||u_c,t - u_t(alpha)||^2,  (alpha I + L_t) u_t = alpha f_t.
Every evaluation of j is one batched call of lower-level solves (one plan per
image, built once); its derivative takes one more batched call of adjoint
solves (alpha I + L_t) p_t = u_t - u_c,t (the optimality system of Sec. 2):
    dj/dalpha = (2/T) sum_t <p_t, f_t - u_t>.
The outer minimisation over log alpha in [Lambda_min, Lambda_max] is Brent's
method, as in Sec. 5.5 (scipy's bounded implementation).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import nlh
from .inputs import raster_windows


def _torch():
    import torch
    return torch


@dataclass
class LearnResult:
    alpha: float
    j: float
    evaluations: int
    seconds: float
    solves: int
    cg_iters_mean: float
    history: List[tuple] = field(default_factory=list)   # (alpha, j) per evaluation


class Bilevel:
    """The bilevel problem for a set of (clean, noisy) image pairs."""

    def __init__(self, pairs, sigma: float, radius: int = 1, pad: str = "reflect",
                 tol: float = 1e-8, arith: int = nlh.SOLVE_MIXED, precision: int = 6,
                 nfft_eps: float = 1e-7, plan_kw=None):
        torch = _torch()
        self.tol, self.arith = tol, arith
        self.f, self.uc, self.plans = [], [], []
        kw = dict(precision=precision, nfft_eps=nfft_eps, m=0)
        if plan_kw:
            kw = dict(plan_kw)
        for clean, noisy in pairs:
            f = torch.as_tensor(np.ascontiguousarray(noisy, dtype=np.float64), device="cuda")
            self.f.append(f.reshape(-1))
            self.uc.append(torch.as_tensor(np.ascontiguousarray(clean, dtype=np.float64).ravel(),
                                           device="cuda"))
            self.plans.append(nlh.Plan.from_image(f, radius, raster_windows(radius), sigma,
                                                  pad=pad, **kw))
        self.u = [torch.empty_like(f) for f in self.f]
        self.p = [torch.empty_like(f) for f in self.f]
        self.r = [torch.empty_like(f) for f in self.f]
        self.solves = 0
        self.cg_iters = 0
        self.sigma = sigma

    @property
    def T(self) -> int:
        return len(self.plans)

    def _solve(self, alpha, bs, us):
        _, infos = nlh.solve_batched(self.plans, [alpha] * self.T, bs, us, tol=self.tol,
                                     arith=self.arith, inner_tol=1e-3)
        self.solves += len(infos)
        self.cg_iters += sum(i["iters"] for i in infos)
        bad = [i for i in infos if i["status"] != 0]
        if bad:
            raise nlh.NLHError(bad[0]["status"], "a lower-level or adjoint solve failed")
        return infos

    def objective(self, alpha: float) -> float:
        """j(alpha); keeps the lower-level solutions in self.u."""
        bs = [f * alpha for f in self.f]
        self._solve(alpha, bs, self.u)
        return sum(nlh.bilevel_misfit(u, uc) for u, uc in zip(self.u, self.uc)) / self.T

    def objective_and_gradient(self, alpha: float):
        """(j(alpha), dj/dalpha) with the adjoint solves."""
        bs = [f * alpha for f in self.f]
        self._solve(alpha, bs, self.u)
        j = sum(nlh.bilevel_misfit(u, uc, r) for u, uc, r in zip(self.u, self.uc, self.r))
        self._solve(alpha, self.r, self.p)
        g = sum(2.0 * nlh.bilevel_gradient_term(p, f, u) for p, f, u in zip(self.p, self.f, self.u))
        return j / self.T, g / self.T

    def learn(self, bounds=(1e-3, 1e3), xatol: float = 1e-4) -> LearnResult:
        """Brent's bounded minimisation of j over log alpha."""
        from scipy.optimize import minimize_scalar
        torch = _torch()
        hist = []
        s0, c0 = self.solves, self.cg_iters

        def fun(la):
            a = float(math.exp(la))
            j = self.objective(a)
            hist.append((a, j))
            return j

        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = minimize_scalar(fun, bounds=(math.log(bounds[0]), math.log(bounds[1])),
                              method="bounded", options={"xatol": xatol})
        torch.cuda.synchronize()
        n_s = self.solves - s0
        return LearnResult(float(math.exp(res.x)), float(res.fun), int(res.nfev),
                           time.perf_counter() - t0, n_s,
                           (self.cg_iters - c0) / max(1, n_s), hist)

    def set_sigma(self, sigma: float):
        """Kernel width of every lower-level system (multiplier tables and
        degrees; the torus map and the window weights are kept)."""
        for P in self.plans:
            P.set_sigma(sigma)
        self.sigma = sigma

    def learn_alpha_theta(self, alpha0: float, sigma0: float, bounds_alpha=(1e-3, 1e3),
                          bounds_sigma=(0.05, 1.0), rel_step: float = 1e-4,
                          maxiter: int = 50) -> dict:
        """Joint learning of (alpha, theta = sigma^-2) (Sec. 5.5) with
        L-BFGS-B over (log alpha, log theta): dj/dalpha by the adjoint
        solves, dj/dtheta by a central difference in log theta (the paper
        used two-point differences for both)."""
        from scipy.optimize import minimize
        torch = _torch()
        evals = []
        s0, c0 = self.solves, self.cg_iters

        def fg(z):
            la, lt = float(z[0]), float(z[1])
            a, th = math.exp(la), math.exp(lt)
            self.set_sigma(th ** -0.5)
            j, ga = self.objective_and_gradient(a)
            h = rel_step
            self.set_sigma(math.exp(lt + h) ** -0.5)
            jp = self.objective(a)
            self.set_sigma(math.exp(lt - h) ** -0.5)
            jm = self.objective(a)
            self.set_sigma(th ** -0.5)
            evals.append((a, th ** -0.5, j))
            return j, np.array([ga * a, (jp - jm) / (2 * h)])

        lt_b = (math.log(bounds_sigma[1] ** -2), math.log(bounds_sigma[0] ** -2))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = minimize(fg, np.array([math.log(alpha0), math.log(sigma0 ** -2)]), jac=True,
                       method="L-BFGS-B",
                       bounds=[(math.log(bounds_alpha[0]), math.log(bounds_alpha[1])), lt_b],
                       options={"maxiter": maxiter, "ftol": 1e-12, "gtol": 1e-8})
        torch.cuda.synchronize()
        a, th = math.exp(res.x[0]), math.exp(res.x[1])
        self.set_sigma(th ** -0.5)
        return {"alpha": a, "sigma": th ** -0.5, "theta": th, "j": float(res.fun),
                "iterations": int(res.nit), "evaluations": len(evals),
                "seconds": time.perf_counter() - t0, "solves": self.solves - s0,
                "cg_iters_mean": (self.cg_iters - c0) / max(1, self.solves - s0),
                "history": evals}

    def close(self):
        for P in self.plans:
            P.close()
        self.plans = []
