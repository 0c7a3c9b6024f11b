"""Pins of the bilevel oracle (oracle/bilevel.py): the adjoint gradient
against central differences of the objective, the closed-form limits of the
lower-level solution (alpha -> infinity: u -> f; alpha -> 0: u -> the mean
of f, the kernel of L), and first-order optimality of Brent's minimiser."""
import numpy as np
import pytest

from oracle import bilevel, oracle as orc
from paper_2407_06834_gb300.inputs import raster_windows, synthetic_image


@pytest.fixture(scope="module")
def pairs():
    ucs, fs, coords = [], [], []
    for seed in (3, 4):
        clean, noisy = synthetic_image(12, 12, seed)
        ucs.append(clean.ravel())
        fs.append(noisy.ravel())
        coords.append(orc.image_coords(noisy, 1, raster_windows(1)))
    Ls = bilevel.laplacians(coords, 0.1)
    return Ls, fs, ucs


def test_laplacian_is_the_oracles(pairs):
    Ls, fs, _ = pairs
    v = np.random.Generator(np.random.PCG64(1)).standard_normal(fs[0].size)
    L = Ls[0]
    assert np.max(np.abs(L @ np.ones(v.size))) < 1e-12 * np.max(np.abs(L))
    np.testing.assert_allclose(L, L.T, atol=1e-15)


@pytest.mark.parametrize("alpha", [0.01, 0.3, 4.0])
def test_adjoint_gradient_equals_finite_differences(pairs, alpha):
    Ls, fs, ucs = pairs
    j, g = bilevel.objective_and_gradient(Ls, fs, ucs, alpha)
    h = 1e-4 * alpha   # O(h^2) truncation; larger than the solves' rounding / h
    jp = bilevel.objective_and_gradient(Ls, fs, ucs, alpha + h)[0]
    jm = bilevel.objective_and_gradient(Ls, fs, ucs, alpha - h)[0]
    assert g == pytest.approx((jp - jm) / (2 * h), rel=1e-6, abs=1e-12)


def test_limits_of_the_lower_level(pairs):
    Ls, fs, ucs = pairs
    j_inf = np.mean([np.sum((uc - f) ** 2) for uc, f in zip(ucs, fs)])
    j_zero = np.mean([np.sum((uc - f.mean()) ** 2) for uc, f in zip(ucs, fs)])
    assert bilevel.objective_and_gradient(Ls, fs, ucs, 1e9)[0] == pytest.approx(j_inf, rel=1e-6)
    assert bilevel.objective_and_gradient(Ls, fs, ucs, 1e-9)[0] == pytest.approx(j_zero, rel=1e-5)
    u = bilevel.lower_level(Ls[0], fs[0], 1e-9)
    np.testing.assert_allclose(u, np.full(u.size, fs[0].mean()), atol=1e-6)


def test_brent_minimiser_is_stationary(pairs):
    Ls, fs, ucs = pairs
    lo, hi = 1e-3, 1e3
    a, j, nfev = bilevel.learn_alpha(Ls, fs, ucs, bounds=(lo, hi), xatol=1e-8)
    assert nfev > 3 and lo * 1.1 < a < hi / 1.1       # an interior minimum here
    # there the derivative vanishes (scale: the change of j over 10% of alpha)
    _, g = bilevel.objective_and_gradient(Ls, fs, ucs, a)
    jl = bilevel.objective_and_gradient(Ls, fs, ucs, a * 0.9)[0]
    assert abs(g) * a < 1e-3 * abs(jl - j)
    for b in (lo, hi, a * 0.9, a * 1.1):
        assert j <= bilevel.objective_and_gradient(Ls, fs, ucs, b)[0]


def test_joint_learning_improves_on_alpha_alone():
    """The joint (alpha, theta) minimum is no worse than the alpha-only one
    at the initial sigma, and stationary in alpha."""
    ucs, fs, coords = [], [], []
    for seed in (3, 4):
        clean, noisy = synthetic_image(10, 10, seed)
        ucs.append(clean.ravel())
        fs.append(noisy.ravel())
        coords.append(orc.image_coords(noisy, 1, raster_windows(1)))
    Ls = bilevel.laplacians(coords, 0.1)
    a1, j1, _ = bilevel.learn_alpha(Ls, fs, ucs, bounds=(1e-3, 1e3), xatol=1e-8)
    a2, s2, j2 = bilevel.learn_alpha_theta(coords, fs, ucs, a1, 0.1, bounds_sigma=(0.05, 0.5))
    assert j2 <= j1 * (1 + 1e-9)
    assert 0.05 <= s2 <= 0.5
    _, g = bilevel.objective_and_gradient(bilevel.laplacians(coords, s2), fs, ucs, a2)
    if 1.1e-3 < a2 < 1e3 / 1.1:
        assert abs(g * a2) < 1e-3 * j2
