"""Pins of the P_b' preconditioner in the oracle (Sec. 4.3.3): for a single
window it equals P_b of Eq. Prec_rel_a_b computed from the dense kernel
matrix; its squared kernel is the kernel at sigma / sqrt(2); the chain
P_a <= P_b' <= P_b <= sqrt(2) P_a (remark after Eq. ANOVA_Norm_2_Prec) and
the spectral bounds of lem. Prec_Norm_2_Diag hold; the solvers with P_b'
reach the LAPACK solution."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2407_06834_gb300.inputs import raster_windows, synthetic_image

LAM, MU, SIG = 0.5, 1.0, 0.2


def _coords(n, radius=1, seed=1):
    img = synthetic_image(n, n, seed)[1]
    return img, orc.image_coords(img, radius, raster_windows(radius))


def _pa_pb(coords):
    G = orc.gamma_dense(coords, SIG)
    eta = G.sum(axis=1)
    pa = LAM + MU * eta
    pb = np.sqrt(MU ** 2 * (G ** 2).sum(axis=1) + pa ** 2)
    return pa, pb


def test_single_window_equals_pb():
    _, c = _coords(10)
    c1 = c[:1]
    pa, pb = _pa_pb(c1)
    np.testing.assert_allclose(orc.pb_diag(c1, SIG, LAM, MU), pb, rtol=1e-13)
    # the squared kernel is the kernel at sigma / sqrt(2): P_b'^2 - P_a^2 = eta(sigma/sqrt 2)
    eta2 = orc.degrees(c1, SIG / np.sqrt(2.0))
    np.testing.assert_allclose(orc.pb_diag(c1, SIG, LAM, MU) ** 2 - pa ** 2, MU ** 2 * eta2,
                               rtol=1e-11)


def test_chain_and_spectral_bounds():
    _, c = _coords(8)
    pa, pb = _pa_pb(c)
    pbp = orc.pb_diag(c, SIG, LAM, MU)
    assert np.all(pa <= pbp * (1 + 1e-15)) and np.all(pbp <= pb * (1 + 1e-15))
    assert np.all(pb <= np.sqrt(2.0) * pa)
    G = orc.gamma_dense(c, SIG)
    A = LAM * np.eye(len(pa)) + MU * (np.diag(G.sum(axis=1)) - G)
    lam_a = np.linalg.eigvals(A / pa[:, None]).real
    lam_b = np.linalg.eigvals(A / pbp[:, None]).real
    assert lam_b.min() >= 2 ** -0.5 * lam_a.min() * (1 - 1e-10)
    assert lam_b.max() <= lam_a.max() * (1 + 1e-10)


def test_solvers_with_pb_reach_lapack():
    img, c = _coords(12, seed=2)
    b = LAM * img.ravel()
    G = orc.gamma_dense(c, SIG)
    A = LAM * np.eye(b.size) + MU * (np.diag(G.sum(axis=1)) - G)
    ref = np.linalg.solve(A, b)
    r = orc.pcg_deflated(c, SIG, LAM, MU, b, tol=1e-12, maxit=500, precond=2)
    assert r.status == 0 and np.linalg.norm(r.u - ref) <= 1e-9 * np.linalg.norm(ref)
    r2 = orc.cg(c, SIG, LAM, MU, b, tol=1e-12, maxit=500, precond=2)
    assert r2.status == 0 and np.linalg.norm(r2.u - ref) <= 1e-9 * np.linalg.norm(ref)
    # iteration counts comparable to P_a (Table 3)
    ra = orc.pcg_deflated(c, SIG, LAM, MU, b, tol=1e-6, precond=True)
    rb = orc.pcg_deflated(c, SIG, LAM, MU, b, tol=1e-6, precond=2)
    assert abs(ra.iters - rb.iters) <= max(2, ra.iters // 2)
