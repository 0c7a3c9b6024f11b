"""Learned warm start and diagonal correction (include/nlh_net.h).

* `make_triples`: (noisy image, sigma, alpha) -> converged solution u*,
  produced by the method itself (batched mixed-precision deflated
  Jacobi-PCG solves to 1e-6), together with the degrees d = Gamma_full 1 and
  the snapshot e0 = u* - u0, r0 = A e0 (= b - A u0) of the preconditioner
  term of the loss.
* `train`: Adam on the network with the library's forward / backward / Adam
  kernels.
* `learned_solve`: u0 and the preconditioner factor from the network, then
  the deflated PCG with x0 = u0 and P_c = P_a * scale; the solver drops the
  factor and restarts plain from its last iterate if the learned run fails,
  and the final residual is always the FP64-accurate ||b - A u|| / ||b||.

The paper has no learned component.  Only library calls and device-memory
plumbing happen here; images come from the seeded synthetic generator.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import nlh
from .inputs import learned_draws, net_init, raster_windows, synthetic_image


def _torch():
    import torch
    return torch


def _gen_image(args):
    H, W, seed = args
    return synthetic_image(H, W, seed)[1]


def host_images(seeds, H, W, workers: int = 0):
    """Noisy synthetic images for the given seeds, generated on the host
    cores (a spawn-started process pool when workers > 1)."""
    if workers <= 1 or len(seeds) < 32:
        return [_gen_image((H, W, s)) for s in seeds]
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_gen_image, [(H, W, s) for s in seeds], chunksize=16))


@dataclass
class TripleSet:
    H: int
    W: int
    f: object            # (S, H, W) float64 CUDA
    ustar: object
    deg: object
    e0: object
    r0: object
    sigma: np.ndarray
    alpha: np.ndarray
    seeds: np.ndarray
    iters: np.ndarray
    seconds: float = 0.0
    worst_rel_res: float = 0.0

    @property
    def count(self) -> int:
        return int(self.sigma.size)


def _plan(f2d, sigma, precision=6):
    return nlh.Plan.from_image(f2d, 1, raster_windows(1), sigma, precision=precision,
                               nfft_eps=1e-7, m=0)


def make_triples(count: int, H: int = 256, W: int = 256, seed: int = 0, per_image: int = 4,
                 net: nlh.Net = None, chunk: int = 16, tol: float = 1e-6,
                 workers: int = 0) -> TripleSet:
    """Generate `count` training triples with the method itself.

    Draws (sigma, alpha) log-uniform over the bilevel search ranges; every
    `per_image` consecutive draws share one synthetic image; the draws are
    then shuffled so that a batch mixes images.  Each draw gets its own plan
    (NFFT parameters for a 1e-7 per-dim error); chunks of plans are solved
    in one batched call.  e0 and r0 are the snapshot for the current
    parameters of `net`."""
    torch = _torch()
    t0 = time.perf_counter()
    draws = learned_draws(count, seed)
    n_img = (count + per_image - 1) // per_image
    img_seeds = [draws[k * per_image][0] for k in range(n_img)]
    imgs = host_images(img_seeds, H, W, workers)
    IMG = torch.as_tensor(np.stack(imgs), device="cuda")
    order = np.random.Generator(np.random.PCG64(seed + 7)).permutation(count)
    S = count
    f = torch.empty((S, H, W), dtype=torch.float64, device="cuda")
    ustar = torch.empty_like(f)
    deg = torch.empty_like(f)
    e0 = torch.empty_like(f)
    r0 = torch.empty_like(f)
    sig = np.empty(S)
    alp = np.empty(S)
    seeds = np.empty(S, dtype=np.int64)
    iters = np.empty(S, dtype=np.int64)
    worst = 0.0
    for c0 in range(0, S, chunk):
        ks = list(range(c0, min(S, c0 + chunk)))
        plans, bs, us, alphas = [], [], [], []
        for k in ks:
            j = int(order[k])
            seeds[k], sig[k], alp[k] = draws[j]
            f[k].copy_(IMG[j // per_image])
            P = _plan(f[k], sig[k])
            plans.append(P)
            bs.append(f[k].reshape(-1) * alp[k])
            us.append(ustar[k].view(-1))
            alphas.append(alp[k])
            P.degrees(out=deg[k].view(-1))
        _, infos = nlh.solve_batched(plans, alphas, bs, us, tol=tol, arith=nlh.SOLVE_MIXED,
                                     inner_tol=1e-3)
        for k, inf in zip(ks, infos):
            iters[k] = inf["iters"]
            worst = max(worst, inf["rel_res_true"])
        _snapshot(net, plans, f, ustar, e0, r0, sig, alp, ks)
        for P in plans:
            P.close()
    del IMG
    torch.cuda.synchronize()
    return TripleSet(H, W, f, ustar, deg, e0, r0, sig, alp, seeds, iters,
                     time.perf_counter() - t0, worst)


def _snapshot(net, plans, f, ustar, e0, r0, sig, alp, ks):
    """e0 = u* - u0 (u0 from the network) and r0 = A e0 per draw."""
    for P, k in zip(plans, ks):
        net.residual_error(f[k], [sig[k]], [alp[k]], ustar[k], e0=e0[k])
        P.matvec(e0[k].view(-1), op=2, alpha=float(alp[k]), precision=nlh.NLH_FP32,
                 out=r0[k].view(-1))


def refresh_snapshot(net: nlh.Net, data: TripleSet, chunk: int = 16) -> float:
    """Recompute e0, r0 for the network's current parameters (one plan per
    draw again).  Returns the seconds it took."""
    torch = _torch()
    t0 = time.perf_counter()
    for c0 in range(0, data.count, chunk):
        ks = list(range(c0, min(data.count, c0 + chunk)))
        plans = [_plan(data.f[k], data.sigma[k]) for k in ks]
        _snapshot(net, plans, data.f, data.ustar, data.e0, data.r0, data.sigma, data.alpha, ks)
        for P in plans:
            P.close()
    torch.cuda.synchronize()
    return time.perf_counter() - t0


@dataclass
class TrainLog:
    steps: int = 0
    seconds: float = 0.0
    losses: List[float] = field(default_factory=list)   # (step, loss) pairs flattened
    refresh_seconds: float = 0.0


def new_net(seed: int = 0, base: int = 32, levels: int = 4) -> nlh.Net:
    net = nlh.Net(base, levels)
    net.set_params(net_init(net.shapes(), seed))
    return net


def train(net: nlh.Net, data: TripleSet, epochs: float = 1.0, batch: int = 16,
          lr: float = 1e-3, lr_final: float = 1e-5, beta: float = 0.25,
          beta_from: float = 0.5, seed: int = 0, log_every: int = 50,
          refresh: bool = True) -> TrainLog:
    """Adam with a cosine learning-rate decay.  The preconditioner term
    (weight beta) is switched on after the fraction `beta_from` of the
    steps, with the e0 / r0 snapshot refreshed for the network at that
    point when `refresh`."""
    torch = _torch()
    nb = data.count // batch
    total = max(1, int(round(epochs * nb)))
    rng = np.random.Generator(np.random.PCG64(seed + 11))
    order = np.concatenate([rng.permutation(nb) for _ in range(int(math.ceil(total / nb)))])
    log = TrainLog()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b_on = int(beta_from * total)
    for step in range(total):
        if step == b_on and beta > 0 and refresh:
            log.refresh_seconds += refresh_snapshot(net, data)
        i0 = int(order[step]) * batch
        sl = slice(i0, i0 + batch)
        bt = beta if step >= b_on else 0.0
        want = (step % log_every == 0) or step == total - 1
        loss = net.loss_grad(data.f[sl], data.sigma[sl], data.alpha[sl], data.ustar[sl],
                             e0=data.e0[sl], r0=data.r0[sl], deg=data.deg[sl], beta=bt,
                             want_loss=want)
        if want:
            log.losses.append((step, bt, loss))
        lr_t = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * step / total))
        net.adam(lr_t)
    torch.cuda.synchronize()
    log.steps = total
    log.seconds = time.perf_counter() - t0 - log.refresh_seconds
    return log


def learned_solve(net: nlh.Net, plan: nlh.Plan, f, sigma: float, alpha: float,
                  tol: float = 1e-6, arith: int = nlh.SOLVE_MIXED, use_x0: bool = True,
                  use_scale: bool = True, maxit: int = 200):
    """The network's u0 and preconditioner factor, then the deflated PCG.
    Returns (SolveResult, seconds of the network forward)."""
    torch = _torch()
    H, W = f.shape
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    u0, scale = net.forward(f, [sigma], [alpha])
    ev[1].record()
    b = f.reshape(-1) * alpha
    res = plan.solve(alpha, b, tol=tol, maxit=maxit, arith=arith, inner_tol=1e-3,
                     x0=u0.view(-1) if use_x0 else None,
                     diag_scale=scale.view(-1) if use_scale else None, x0_check=True)
    torch.cuda.synchronize()
    return res, ev[0].elapsed_time(ev[1]) * 1e-3
