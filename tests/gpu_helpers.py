"""Shared helpers of the GPU parity tests (inputs only; no method arithmetic)."""
import numpy as np

from paper_2407_06834_gb300.inputs import raster_windows, synthetic_image


def cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def image(n1, n2=None, seed=0):
    return synthetic_image(n1, n2 or n1, seed)[1]


def make_plan(img, radius=1, sigma=0.2, M=32, n_os=64, m=4, fill=0.0, precision=3, pad="reflect",
              kmax=0):
    from paper_2407_06834_gb300 import nlh
    return nlh.Plan.from_image(cuda(img), radius, raster_windows(radius), sigma, pad=pad, M=M,
                               n_os=n_os, m=m, precision=precision, torus_fill=fill,
                               max_items_pts=kmax)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
