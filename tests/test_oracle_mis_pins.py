"""Pins of the mutual-information window selection oracle (Sec. 5) against
closed forms, special cases and brute force; none re-derives the oracle's
own formula."""
import math

import numpy as np
import pytest

from oracle import mis
from paper_2407_06834_gb300.inputs import synthetic_image


def test_two_by_two_table_closed_form():
    # values at two levels with joint counts [[3, 1], [1, 3]] (x 25): p = 3/8
    # on the diagonal, 1/8 off it, uniform marginals 1/2
    x = np.array([0.0] * 75 + [0.0] * 25 + [1.0] * 25 + [1.0] * 75)
    y = np.array([0.0] * 75 + [1.0] * 25 + [0.0] * 25 + [1.0] * 75)
    c = mis.joint_counts(x, y, 2)
    assert c.tolist() == [[75, 25], [25, 75]]
    ref = 0.75 * math.log(1.5) + 0.25 * math.log(0.5)
    assert mis.mi_from_counts(c) == pytest.approx(ref, rel=1e-14)


def test_constant_variable_carries_no_information():
    r = np.random.default_rng(0)
    y = r.standard_normal(1000)
    assert mis.mi_from_counts(mis.joint_counts(np.full(1000, 0.3), y, 16)) == 0.0


def test_identical_variables_give_the_entropy():
    # MI(Y; Y) = H(binned Y), here from scipy's entropy of the bin frequencies
    from scipy.stats import entropy
    r = np.random.default_rng(1)
    y = r.standard_normal(5000)
    counts = np.bincount(mis.bin_index(y, 32), minlength=32)
    h = entropy(counts[counts > 0] / counts.sum())
    assert mis.mi_from_counts(mis.joint_counts(y, y, 32)) == pytest.approx(h, rel=1e-12)


def test_symmetry_and_exact_scaling_invariance():
    r = np.random.default_rng(2)
    x = r.standard_normal(4000)
    y = 0.6 * x + r.standard_normal(4000)
    a = mis.mi_from_counts(mis.joint_counts(x, y, 24))
    b = mis.mi_from_counts(mis.joint_counts(y, x, 24))
    # x -> 4 x - 1 keeps every bin (powers of two scale exactly)
    c = mis.mi_from_counts(mis.joint_counts(4.0 * x, y, 24))
    assert a == pytest.approx(b, rel=1e-13)
    assert a == pytest.approx(c, rel=1e-13)


def test_gaussian_pair_approaches_the_closed_form():
    # bivariate normal with correlation rho: I = -1/2 log(1 - rho^2); the
    # plug-in histogram estimate is within discretisation + bias of it
    r = np.random.default_rng(3)
    n, rho = 400_000, 0.8
    x = r.standard_normal(n)
    y = rho * x + math.sqrt(1 - rho * rho) * r.standard_normal(n)
    est = mis.mi_from_counts(mis.joint_counts(x, y, 48))
    assert est == pytest.approx(-0.5 * math.log(1 - rho * rho), abs=0.04)


def test_bins_match_brute_force_on_a_tiny_input():
    r = np.random.default_rng(4)
    x, y = r.uniform(-1, 2, 37), r.uniform(0, 1, 37)
    c = mis.joint_counts(x, y, 5)
    lo, hi = x.min(), x.max()
    ly, hy = y.min(), y.max()
    ref = np.zeros((5, 5), dtype=np.int64)
    for xi, yi in zip(x, y):
        a = 0
        while a < 4 and xi >= lo + (a + 1) * (hi - lo) / 5 + 1e-12:
            a += 1
        b = 0
        while b < 4 and yi >= ly + (b + 1) * (hy - ly) / 5 + 1e-12:
            b += 1
        ref[a, b] += 1
    assert (c == ref).all()


def test_windows_rank_the_center_pixel_first():
    # the center patch dimension is f itself: the largest score
    _, img = synthetic_image(48, 40, 7)
    for radius, pad in ((1, "reflect"), (2, "zero")):
        D = (2 * radius + 1) ** 2
        s, w = mis.mis_windows(img, radius, pad, bins=32)
        assert w[0, 0] == D // 2
        assert np.argmax(s) == D // 2
        flat = [d for d in w.reshape(-1) if d >= 0]
        assert sorted(flat) == list(range(D))
        assert all(s[flat[i]] >= s[flat[i + 1]] for i in range(D - 1))
        assert (w.reshape(-1)[D:] == -1).all()


def test_ties_go_to_the_lower_dimension():
    w = mis.rank_windows(np.array([0.5, 0.7, 0.5, 0.7, 0.1]))
    assert w.tolist() == [[1, 3, 0], [2, 4, -1]]
