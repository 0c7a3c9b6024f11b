"""CPU FP64 oracle of the feature-window selection by mutual information (Sec. 5).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference legs may import this module.  It shares no code with
the CUDA library and nothing on the product path calls it.

Sec. 5 ranks the (2 rho + 1)^2 patch dimensions by their mutual information
score (MIS) against the noisy pixel values f, which stand in for the clean
image, and groups the ranked dimensions into L = ceil(D / 3) windows.  The
paper does not fix the estimator.  The reading taken here is the plug-in
(maximum-likelihood) mutual information, in nats, of the equal-width B x B
joint histogram of (feature d, f):
    lo, hi = min and max of the variable over the N pixels,
    bin(x) = min(B - 1, floor((x - lo) * (B / (hi - lo))))   (0 when hi = lo),
    MIS_d  = sum over cells with c_ab > 0 of (c_ab / N) log(c_ab N / (c_a c_b)),
c_ab the joint counts and c_a, c_b the marginal counts.  The bin index is
computed in FP64 exactly as written (one subtraction, one product with the
precomputed B / (hi - lo)), so it is an integer decision both sides take in
the same precision.  Ranking: MIS descending, ties to the lower dimension.
Windows: the ranked dimensions in consecutive triples, the last one
completed with -1 (a zero-valued dimension), as in the raster-order default.
"""
from __future__ import annotations

import numpy as np

from . import oracle as orc


def bin_index(x: np.ndarray, bins: int) -> np.ndarray:
    """Equal-width bin of every value of x over [min x, max x]."""
    x = np.asarray(x, dtype=np.float64)
    lo, hi = float(x.min()), float(x.max())
    if hi == lo:
        return np.zeros(x.shape, dtype=np.int64)
    inv = bins / (hi - lo)
    k = np.floor((x - lo) * inv).astype(np.int64)
    return np.minimum(k, bins - 1)


def joint_counts(x: np.ndarray, y: np.ndarray, bins: int) -> np.ndarray:
    """B x B integer histogram c[a, b] = #{i : bin(x_i) = a, bin(y_i) = b}."""
    a, b = bin_index(x, bins), bin_index(y, bins)
    c = np.zeros((bins, bins), dtype=np.int64)
    np.add.at(c, (a, b), 1)
    return c


def mi_from_counts(c: np.ndarray) -> float:
    """Plug-in mutual information (nats) of a joint count table."""
    c = np.asarray(c, dtype=np.float64)
    n = c.sum()
    ca, cb = c.sum(axis=1), c.sum(axis=0)
    s = 0.0
    for a in range(c.shape[0]):
        for b in range(c.shape[1]):
            if c[a, b] > 0:
                s += (c[a, b] / n) * np.log(c[a, b] * n / (ca[a] * cb[b]))
    return float(s)


def mis_scores(img: np.ndarray, radius: int, pad: str = "reflect", bins: int = 64):
    """(MIS per patch dimension, joint counts per dimension)."""
    feat = orc.patch_features(img, radius, pad)
    y = np.asarray(img, dtype=np.float64).reshape(-1)
    counts = [joint_counts(feat[:, d], y, bins) for d in range(feat.shape[1])]
    return np.array([mi_from_counts(c) for c in counts]), counts


def rank_windows(mis: np.ndarray) -> np.ndarray:
    """Dimensions by MIS descending (ties: lower index first) in triples."""
    D = mis.size
    order = sorted(range(D), key=lambda d: (-mis[d], d))
    L = -(-D // 3)
    w = np.full((L, 3), -1, dtype=np.int32)
    for r, d in enumerate(order):
        w[r // 3, r % 3] = d
    return w


def mis_windows(img: np.ndarray, radius: int, pad: str = "reflect", bins: int = 64):
    """(MIS per dimension, (L, 3) windows) for an image."""
    mis, _ = mis_scores(img, radius, pad, bins)
    return mis, rank_windows(mis)
