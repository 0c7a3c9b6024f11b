"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every test here runs on the CPU (no GPU marker).  None compares the oracle
with a retyped copy of itself: each check is a closed form, a library routine
that a special case reduces to (np.pad, scipy.linalg.helmert, LAPACK solves,
numpy FFT), an invariant, or one of the paper's spectral lemmas checked on a
dense eigendecomposition.  A plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand) breaks at least one of them.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
from math import erfc

from oracle import oracle as orc
from paper_2407_06834_gb300.inputs import raster_windows, synthetic_image, random_vector

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _img(n, seed=0):
    return synthetic_image(n, n, seed)[1]


def _coords(n, radius=1, seed=0, pad="reflect"):
    return orc.image_coords(_img(n, seed), radius, raster_windows(radius), pad)


def _golden_limits():
    rows = {}
    for line in open(os.path.join(GOLD, "limit_spectra.txt")):
        if line.startswith("#") or not line.strip():
            continue
        case, n, lam, mu, v1, v2 = line.split()
        rows.setdefault(case, []).append((int(n), float(lam), float(mu), float(v1), float(v2)))
    return rows


# ------------------------------------------------------------------ features
@pytest.mark.parametrize("radius", [1, 2])
@pytest.mark.parametrize("pad,npmode", [("reflect", "reflect"), ("zero", "constant")])
def test_patch_features_match_numpy_pad(radius, pad, npmode):
    """Sec. 5 patches == sliding windows of np.pad (library routine)."""
    img = _img(7)[:7, :5]
    feat = orc.patch_features(img, radius, pad)
    P = 2 * radius + 1
    padded = np.pad(img, radius, mode=npmode)
    win = np.lib.stride_tricks.sliding_window_view(padded, (P, P))
    expect = win.reshape(img.shape[0] * img.shape[1], P * P)
    np.testing.assert_array_equal(feat, expect)


def test_window_coords_zero_pad_dims():
    """The 9th window of a 5x5 patch holds dim 24 and two zero dims."""
    img = _img(8)
    w = raster_windows(2)
    assert w.shape == (9, 3) and list(w[-1]) == [24, -1, -1]
    feat = orc.patch_features(img, 2)
    c = orc.window_coords(feat, w)
    np.testing.assert_array_equal(c[8, :, 0], feat[:, 24])
    assert np.all(c[8, :, 1:] == 0.0)
    np.testing.assert_array_equal(c[2, :, :], feat[:, 6:9])


# ------------------------------------------------------------------ kernel sums
def test_constant_image_gives_complete_graph():
    """Identical features => Gamma = 11^T - I for every sigma (Sec. 4.3.3,
    limit A_inf; Sec. 4.2 K_n example)."""
    c = orc.image_coords(np.full((6, 6), 0.37), 1, raster_windows(1))
    v = random_vector(36, 1)
    for sigma in (0.01, 0.2, 5.0):
        np.testing.assert_allclose(orc.gamma_matvec(c, sigma, v), v.sum() - v, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(orc.gamma_full_matvec(c, sigma, v),
                                   np.full(36, v.sum()), rtol=1e-13)


def test_two_point_kernel_closed_form():
    """Eq. discrete_ANOVA on two points: windows at squared distance sigma^2
    and 0 give gamma_12 = (e^-1 + 1)/2, and 4 sigma^2 gives e^-4."""
    sigma = 0.3
    c = np.zeros((2, 2, 3))
    c[0, 1, :] = [sigma, 0.0, 0.0]             # window 1: r^2 = sigma^2
    G = orc.gamma_dense(c, sigma)
    assert G[0, 0] == 0.0 and G[1, 1] == 0.0
    assert G[0, 1] == pytest.approx(0.5 * (np.exp(-1.0) + 1.0), rel=1e-15)
    c2 = np.zeros((1, 2, 3))
    c2[0, 1, :] = [0.0, sigma, sigma * np.sqrt(3.0)]   # r^2 = 4 sigma^2
    assert orc.gamma_dense(c2, sigma)[1, 0] == pytest.approx(np.exp(-4.0), rel=1e-14)


def test_diagonal_convention_and_symmetry():
    """Gamma_full = Gamma + I (gamma_ii = 1, Sec. 2.3) and Gamma symmetric."""
    c = _coords(12)
    N = c.shape[1]
    v, w = random_vector(N, 2), random_vector(N, 3)
    np.testing.assert_allclose(orc.gamma_full_matvec(c, 0.2, v) - orc.gamma_matvec(c, 0.2, v), v,
                               rtol=1e-12, atol=1e-12)
    a = w @ orc.gamma_matvec(c, 0.2, v)
    b = v @ orc.gamma_matvec(c, 0.2, w)
    assert a == pytest.approx(b, rel=1e-13)


def test_gamma_rows_subset_matches_full():
    c = _coords(10)
    N = c.shape[1]
    v = random_vector(N, 4)
    rows = np.array([0, 5, N - 1, 37])
    np.testing.assert_allclose(orc.gamma_full_rows(c, 0.2, v, rows),
                               orc.gamma_full_matvec(c, 0.2, v)[rows], rtol=1e-14)


def test_sigma_to_zero_limits():
    """Sec. 4.3.3: with all window features distinct, sigma -> 0 gives
    A_{1,sigma->0} = lambda I.  With coinciding windows (reflect padding makes
    row -1 of pixel (0, c) equal row +1 of pixel (2, c)) the limit is
    A_{2,sigma->0} with Gamma -> E, E_ij = (1/L) #{l : W_l x_i = W_l x_j}."""
    rng = np.random.Generator(np.random.PCG64(11))
    c = rng.uniform(0.0, 1.0, size=(3, 50, 3))
    v = random_vector(50, 5)
    np.testing.assert_allclose(orc.A_apply(c, 1e-4, 0.7, 1.0, v), 0.7 * v, rtol=1e-12)
    c = _coords(8)
    L, N, _ = c.shape
    E = np.zeros((N, N))
    for l in range(L):
        same = np.all(c[l][:, None, :] == c[l][None, :, :], axis=2)
        E += same / L
    np.fill_diagonal(E, 0.0)
    assert E.max() > 0
    np.testing.assert_allclose(orc.gamma_dense(c, 1e-4), E, atol=1e-300)


def test_laplacian_invariants():
    """L 1 = 0, A 1 = lambda 1, Gamma 1 = eta (Sec. 4.2)."""
    c = _coords(12)
    N = c.shape[1]
    eta = orc.degrees(c, 0.2)
    one = np.ones(N)
    np.testing.assert_allclose(orc.gamma_matvec(c, 0.2, one), eta, rtol=1e-14)
    Lone = orc.laplacian_apply(c, 0.2, one, eta)
    assert np.max(np.abs(Lone)) <= 1e-13 * np.max(eta)
    np.testing.assert_allclose(orc.A_apply(c, 0.2, 0.3, 2.0, one, eta), 0.3 * one,
                               rtol=1e-12, atol=1e-12 * np.max(eta))


# ------------------------------------------------------------------ spectra
@pytest.fixture(scope="module")
def dense16():
    c = _coords(16)
    G = orc.gamma_dense(c, 0.2)
    eta = G.sum(axis=1)
    Lm = np.diag(eta) - G
    return c, G, eta, Lm


def test_dense_matches_matvec(dense16):
    c, G, eta, Lm = dense16
    v = random_vector(G.shape[0], 6)
    np.testing.assert_allclose(G @ v, orc.gamma_matvec(c, 0.2, v), rtol=1e-12)
    np.testing.assert_allclose(eta, orc.degrees(c, 0.2), rtol=1e-13)
    np.testing.assert_allclose(Lm @ v, orc.laplacian_apply(c, 0.2, v), rtol=1e-10, atol=1e-11)


def test_spectral_bounds_of_L(dense16):
    """Lemma general_spectral_bounds: max eta <= rho(L) < 2 max eta;
    Lemma UpperConnectivity: a(L) <= n/(n-1) min eta;
    Lemma lower_bound_algebraic_connectivity: Sigma(E) >= min Gamma_{2:n,1}
    and a(A) >= mu min Gamma_{2:n,1} + lambda (read with rows 2:n)."""
    c, G, eta, Lm = dense16
    n = G.shape[0]
    ev = np.linalg.eigvalsh(Lm)
    assert abs(ev[0]) < 1e-10 * ev[-1]
    rho, a = ev[-1], ev[1]
    assert eta.max() <= rho * (1 + 1e-12) and rho < 2 * eta.max()
    assert a <= n / (n - 1) * eta.min() * (1 + 1e-12)
    E = Lm[1:, 1:] + np.outer(G[1:, 0], np.ones(n - 1))
    evE = np.linalg.eigvals(E).real
    assert evE.min() >= G[1:, 0].min() * (1 - 1e-9)
    lam, mu = 1e-3, 1.0
    evA = np.linalg.eigvalsh(lam * np.eye(n) + mu * Lm)
    assert evA[1] >= mu * G[1:, 0].min() + lam - 1e-12


def test_jacobi_and_projected_spectral_bounds(dense16):
    """Lemma Rayleigh_Diag_Jac, Lemma Equivalence_Diag_Precs, Lemma
    Spectral_Control_Pa_on_D (with X = U of Eq. ULap)."""
    c, G, eta, Lm = dense16
    n = G.shape[0]
    lam, mu = 1e-2, 1.0
    A = lam * np.eye(n) + mu * Lm
    Pa = lam + mu * eta
    evL = np.linalg.eigvalsh(Lm)
    rhoL, aL = evL[-1], evL[1]
    s = 1.0 / np.sqrt(Pa)
    ev = np.linalg.eigvalsh(s[:, None] * A * s[None, :])        # Sigma(P_a^-1 A)
    assert ev[0] >= lam / (lam + mu * eta.max()) * (1 - 1e-10)
    assert ev[-1] <= min(2.0, n / (n - 1) * rhoL / aL) * (1 + 1e-10)
    Pb = np.sqrt(mu ** 2 * (G ** 2).sum(axis=1) + Pa ** 2)        # Eq. Prec_rel_a_b
    assert np.all(Pa <= Pb * (1 + 1e-15)) and np.all(Pb <= np.sqrt(2) * Pa * (1 + 1e-15))
    U = np.column_stack([orc.U_apply(e) for e in np.eye(n)])
    D_inv = U.T @ np.diag(1.0 / Pa) @ U                           # (U^-1 P_a U)^-1
    Atil = U.T @ A @ U
    proj = D_inv[1:, 1:] @ Atil[1:, 1:]
    evp = np.sort(np.linalg.eigvals(proj).real)
    assert evp[0] > 0
    assert evp[0] >= ev[0] - lam / (lam + mu * eta.min()) - 1e-10
    assert evp[-1] <= ev[-1] * (1 + 1e-10)


def test_change_of_basis_block_form(dense16):
    """Eq. ChangeOfBasisOfA with Q of Eq. QLap:
    Q^-1 A Q = [[lambda, 0], [0, mu (L_22 + Gamma_{2:n,1} 1^T) + lambda I]]."""
    c, G, eta, Lm = dense16
    n = G.shape[0]
    lam, mu = 0.3, 1.7
    A = lam * np.eye(n) + mu * Lm
    Q = np.zeros((n, n))
    Q[:, 0] = 1.0
    Q[0, 1:] = 1.0
    Q[1:, 1:] = -np.eye(n - 1)
    Qinv = np.ones((n, n)) / n - np.diag(np.r_[0.0, np.ones(n - 1)])   # Eq. QLap
    np.testing.assert_allclose(Qinv @ Q, np.eye(n), atol=1e-13)
    B = Qinv @ A @ Q
    assert B[0, 0] == pytest.approx(lam, rel=1e-10)
    assert np.max(np.abs(B[0, 1:])) < 1e-10 and np.max(np.abs(B[1:, 0])) < 1e-10
    expect = mu * (Lm[1:, 1:] + np.outer(G[1:, 0], np.ones(n - 1))) + lam * np.eye(n - 1)
    np.testing.assert_allclose(B[1:, 1:], expect, atol=1e-10)


def test_golden_limit_spectra():
    """Closed-form spectra printed in the paper (tests/golden/limit_spectra.txt)."""
    g = _golden_limits()
    for n, lam, mu, v1, v2 in g["K_n"]:
        side = int(np.sqrt(n))
        c = orc.image_coords(np.full((side, side), 0.5), 1, raster_windows(1))
        Lm = np.diag(orc.degrees(c, 0.2)) - orc.gamma_dense(c, 0.2)
        ev = np.linalg.eigvalsh(Lm)
        assert ev[0] == pytest.approx(v1, abs=1e-12)
        np.testing.assert_allclose(ev[1:], v2, rtol=1e-12)
    for case in ("A_inf", "PaA_inf"):
        for n, lam, mu, v1, v2 in g[case]:
            side = int(np.sqrt(n))
            c = orc.image_coords(np.full((side, side), 0.5), 1, raster_windows(1))
            G = orc.gamma_dense(c, 0.2)
            eta = G.sum(axis=1)
            A = lam * np.eye(n) + mu * (np.diag(eta) - G)
            if case == "PaA_inf":
                s = 1.0 / np.sqrt(lam + mu * eta)
                A = s[:, None] * A * s[None, :]
            ev = np.linalg.eigvalsh(A)
            assert ev[0] == pytest.approx(v1, rel=1e-10)
            np.testing.assert_allclose(ev[1:], v2, rtol=1e-12)


# ------------------------------------------------------------------ change of basis U
@pytest.mark.parametrize("n", [1, 2, 3, 7, 64])
def test_helmert_matches_scipy(n):
    """Eq. ULap: U equals the (transposed) Helmert matrix of scipy."""
    U = np.column_stack([orc.U_apply(e) for e in np.eye(n)])
    np.testing.assert_allclose(U, sla.helmert(n, full=True).T, atol=1e-15)
    Ut = np.column_stack([orc.Ut_apply(e) for e in np.eye(n)])
    np.testing.assert_allclose(Ut, U.T, atol=1e-15)


def test_helmert_orthogonal_large():
    n = 5000
    x = random_vector(n, 7)
    np.testing.assert_allclose(orc.Ut_apply(orc.U_apply(x)), x, atol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(orc.U_apply(x)), np.linalg.norm(x), rtol=1e-13)
    g = orc.Ut_apply(np.ones(n))
    assert g[0] == pytest.approx(np.sqrt(n), rel=1e-14) and np.max(np.abs(g[1:])) < 1e-11


# ------------------------------------------------------------------ solvers
@pytest.fixture(scope="module")
def sys24():
    img = _img(24)
    c = orc.image_coords(img, 1, raster_windows(1))
    G = orc.gamma_dense(c, 0.2)
    return img.ravel(), c, G


@pytest.mark.parametrize("lam", [0.5, 1e-3])
def test_solvers_match_lapack(sys24, lam):
    """All oracle solvers reach the LAPACK solution of the dense system."""
    f, c, G = sys24
    n = f.size
    A = lam * np.eye(n) + np.diag(G.sum(axis=1)) - G
    b = lam * f
    u_ref = np.linalg.solve(A, b)
    for res in (orc.pcg_deflated(c, 0.2, lam, 1.0, b, tol=1e-10, maxit=500),
                orc.pcg_deflated(c, 0.2, lam, 1.0, b, tol=1e-10, maxit=500, precond=False),
                orc.cg(c, 0.2, lam, 1.0, b, tol=1e-10, maxit=2000, precond=True),
                orc.cg(c, 0.2, lam, 1.0, b, x0=f, tol=1e-10, maxit=2000)):
        assert res.status == 0, res
        np.testing.assert_allclose(res.u, u_ref, rtol=0, atol=1e-7 * np.abs(u_ref).max())
        r = b - A @ res.u
        assert np.linalg.norm(r) <= 2e-10 * np.linalg.norm(b)


def test_deflated_history_is_true_residual(sys24):
    """||r_k|| of the second block equals ||b - A u_k||: check at the end."""
    f, c, G = sys24
    lam = 0.05
    A = lam * np.eye(f.size) + np.diag(G.sum(axis=1)) - G
    res = orc.pcg_deflated(c, 0.2, lam, 1.0, lam * f, tol=1e-6)
    true = np.linalg.norm(lam * f - A @ res.u) / np.linalg.norm(lam * f)
    assert true == pytest.approx(res.hist[res.iters], rel=1e-6)


def test_deflated_pcg_constant_image_one_iteration():
    """Constant image: on 1^perp, P_a^-1 A_inf is a multiple of the identity,
    so the deflated Jacobi-PCG converges in one iteration (Sec. 4.3.3)."""
    c = orc.image_coords(np.full((8, 8), 0.25), 1, raster_windows(1))
    b = random_vector(64, 8)
    res = orc.pcg_deflated(c, 0.2, 1e-3, 1.0, b, tol=1e-12)
    assert res.status == 0 and res.iters == 1


def test_maximum_principle(sys24):
    """Thm Uniqueness_LLP: min f <= u <= max f for A u = lambda f."""
    f, c, G = sys24
    for lam in (1.0, 1e-2):
        u = orc.pcg_deflated(c, 0.2, lam, 1.0, lam * f, tol=1e-12, maxit=500).u
        assert u.min() >= f.min() - 1e-9 and u.max() <= f.max() + 1e-9


def test_deflated_iteration_trend_matches_table3(sys24):
    """Table 3: the P_{U,a} count does not move as lambda drops from 1e-3 to
    1e-9, while Jacobi-PCG in the original basis grows or fails."""
    table = np.loadtxt(os.path.join(GOLD, "table3_deflated_iters.txt"))
    assert np.all(table[:, 2] == table[:, 3]) and np.all(table[:, 3] == table[:, 4])
    f, c, _ = sys24
    its_defl, its_jac = [], []
    for lam in (1e-3, 1e-6, 1e-9):
        its_defl.append(orc.pcg_deflated(c, 0.2, lam, 1e-2, lam * f, tol=1e-8, maxit=60).iters)
        r = orc.cg(c, 0.2, lam, 1e-2, lam * f, tol=1e-8, maxit=60, precond=True)
        its_jac.append(r.iters if r.status == 0 else 10 ** 6)
    assert max(its_defl) - min(its_defl) <= 1
    assert its_jac[-1] > its_defl[-1]


def test_pi_form_equals_u_form(sys24):
    """CG on 1^perp with Pi P_a^-1 Pi is iterate-for-iterate the paper's CG on
    pi_2(U^T A U) with pi_2(U^T P_a^-1 U): compare residual histories."""
    f, c, G = sys24
    lam = 1e-3
    n = f.size
    A = lam * np.eye(n) + np.diag(G.sum(axis=1)) - G
    Pa = lam + G.sum(axis=1)
    b = lam * f
    res = orc.pcg_deflated(c, 0.2, lam, 1.0, b, tol=1e-10, maxit=50)
    # plain dense Pi-form
    Pi = lambda x: x - x.mean()
    r = Pi(b)
    z = Pi(r / Pa)
    p = z.copy()
    rz = r @ z
    hist = [np.linalg.norm(r) / np.linalg.norm(b)]
    for _ in range(res.iters):
        q = A @ p
        a = rz / (p @ q)
        r = r - a * q
        hist.append(np.linalg.norm(r) / np.linalg.norm(b))
        z = Pi(r / Pa)
        rz, rz_old = r @ z, rz
        p = z + rz / rz_old * p
    np.testing.assert_allclose(hist, res.hist[:res.iters + 1], rtol=1e-7, atol=1e-13)


def test_breakdown_reported_on_nan_rhs(sys24):
    f, c, _ = sys24
    b = 0.5 * f.copy()
    b[3] = np.nan
    res = orc.pcg_deflated(c, 0.2, 0.5, 1.0, b, tol=1e-6)
    assert res.status != 0


# ------------------------------------------------------------------ Fourier side
def test_gauss_fourier_coeff_vs_fft():
    """Closed-form Gaussian coefficients == DFT of the sampled, periodised
    Gaussian (numpy FFT)."""
    for s in (0.05, 0.1, 0.3):
        nf = 4096
        t = np.arange(nf) / nf
        gper = sum(np.exp(-((t + r) ** 2) / s ** 2) for r in range(-6, 7))
        coef = np.fft.fft(gper).real / nf
        k = np.arange(0, 40)
        np.testing.assert_allclose(orc.gauss_fourier_coeff(s, k), coef[:40],
                                   rtol=1e-10, atol=1e-15)


def test_trig_kernel_truncation_bound():
    """|K_M(t) - g_per(t)| <= erfc(pi s (M/2 - 1)) (tail of the Gaussian
    coefficients), and the error falls as M grows."""
    s = 0.07
    t = np.linspace(-0.5, 0.5, 41)
    gper = sum(np.exp(-((t + r) ** 2) / s ** 2) for r in range(-4, 5))
    prev = np.inf
    for M in (8, 16, 24, 32, 48):
        err = np.max(np.abs(orc.trig_kernel_1d(t, s, M) - gper))
        assert err <= erfc(np.pi * s * (M / 2 - 1)) + 1e-15
        assert err < prev or err < 1e-15
        prev = err


def test_torus_map_range():
    c = _coords(16)
    tc, s = orc.torus_map(c, 0.6)
    rng = tc.max(axis=1) - tc.min(axis=1)
    assert rng.max() == pytest.approx(0.6, rel=1e-14)
    assert np.all(np.abs(tc) <= 0.3 + 1e-15)
    np.testing.assert_allclose(tc[1] - tc[1].mean(axis=0), s * (c[1] - c[1].mean(axis=0)), atol=1e-15)


def test_trig_sum_approaches_gaussian_sum():
    """The truncated-Fourier kernel sum tends to the direct Gaussian sum as M
    grows (alias error exp(-((1 - fill)/sigma_s)^2) is negligible here)."""
    c = _coords(8)
    N = c.shape[1]
    v = np.abs(random_vector(N, 9))
    sigma = 0.2
    ref = orc.gamma_full_matvec(c, sigma, v)
    scale = v.sum() / np.max(np.abs(ref))
    # small fill: aliasing negligible, the truncation error falls with M
    tc, s = orc.torus_map(c, 0.4)
    errs = []
    for M in (16, 24, 32, 48):
        y = orc.trig_full_matvec(tc, s * sigma, M, v)
        errs.append(np.max(np.abs(y - ref)) / np.max(np.abs(ref)))
        assert errs[-1] <= 3 * erfc(np.pi * s * sigma * (M / 2 - 1)) * scale
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-9
    # large fill: the error stalls at the alias level 2 exp(-((1-fill)/sigma_s)^2)
    fill = 0.6
    tc, s = orc.torus_map(c, fill)
    y = orc.trig_full_matvec(tc, s * sigma, 64, v)
    err = np.max(np.abs(y - ref)) / np.max(np.abs(ref))
    alias = 2 * np.exp(-((1 - fill) / (s * sigma)) ** 2)
    assert 1e-3 * alias * scale < err <= 3 * alias * scale
