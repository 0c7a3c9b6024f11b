"""GPU parity of the Krylov solves against the CPU oracle (through the C ABI).

The solve target is the relative residual 1e-6.  Parity criteria:
  * the GPU's own FP64 residual ||b - A~ u|| / ||b|| <= 1e-6 (A~: the NFFT
    operator), recomputed from u by an extra FP64 matvec;
  * at tight NFFT parameters the oracle's direct operator also certifies
    u: ||b - A u|| / ||b|| <= 2e-6;
  * the deflated CG iterates equal the oracle's CG in the paper's Helmert
    coordinates: residual histories agree to 1e-7 relative per iteration;
  * u agrees with the oracle's solution to the conditioning-scaled error.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2407_06834_gb300.inputs import random_vector, raster_windows
from gpu_helpers import cuda, host, image, make_plan, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2407_06834_gb300 import nlh  # noqa: E402

SIGMA, ALPHA = 0.2, 0.5


@pytest.fixture(scope="module")
def tight64():
    img = image(64)
    coords = orc.image_coords(img, 1, raster_windows(1))
    P = make_plan(img, M=64, n_os=128, m=8, fill=0.5, precision=3)
    return img, coords, P


def test_deflated_fp64_solve_matches_oracle(tight64):
    img, coords, P = tight64
    f = img.ravel()
    b = ALPHA * f
    res = P.solve(ALPHA, cuda(b), tol=1e-6, method=nlh.PCG_DEFLATED, arith=nlh.SOLVE_FP64)
    assert res.info["status"] == 0
    assert res.info["rel_res_true"] <= 1.5e-6
    u = host(res.u)
    # the direct operator certifies the GPU solution
    r = b - orc.A_apply(coords, SIGMA, ALPHA, 1.0, u)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 2e-6
    ref = orc.pcg_deflated(coords, SIGMA, ALPHA, 1.0, b, tol=1e-12, maxit=500)
    assert rel(u, ref.u) < 1e-5
    # iterate-for-iterate equality with the paper's U-coordinates CG
    o = orc.pcg_deflated(coords, SIGMA, ALPHA, 1.0, b, tol=1e-6, maxit=200)
    assert res.info["iters"] == o.iters
    np.testing.assert_allclose(res.hist, o.hist[:o.iters + 1], rtol=1e-7)


@pytest.mark.parametrize("method,oracle_kw", [
    (nlh.CG, dict(precond=False)), (nlh.PCG_JACOBI, dict(precond=True))])
def test_original_basis_methods_match_oracle(tight64, method, oracle_kw):
    img, coords, P = tight64
    f = img.ravel()
    b = ALPHA * f
    res = P.solve(ALPHA, cuda(b), tol=1e-6, maxit=400, method=method, x0=cuda(f))
    o = orc.cg(coords, SIGMA, ALPHA, 1.0, b, x0=f, tol=1e-6, maxit=400, **oracle_kw)
    assert res.info["status"] == 0 and o.status == 0
    assert abs(res.info["iters"] - o.iters) <= 1
    n = min(res.info["iters"], o.iters) + 1
    np.testing.assert_allclose(res.hist[:n], o.hist[:n], rtol=1e-6)
    assert res.info["rel_res_true"] <= 1.5e-6


def test_unpreconditioned_deflated_matches_oracle(tight64):
    img, coords, P = tight64
    b = ALPHA * img.ravel()
    res = P.solve(ALPHA, cuda(b), tol=1e-6, method=nlh.CG_DEFLATED)
    o = orc.pcg_deflated(coords, SIGMA, ALPHA, 1.0, b, tol=1e-6, precond=False)
    assert res.info["iters"] == o.iters
    np.testing.assert_allclose(res.hist, o.hist[:o.iters + 1], rtol=1e-7)


def test_mixed_precision_reaches_fp64_residual():
    img = image(64)
    P = make_plan(img, precision=3)
    b = ALPHA * img.ravel()
    r64 = P.solve(ALPHA, cuda(b), tol=1e-6, arith=nlh.SOLVE_FP64)
    rmx = P.solve(ALPHA, cuda(b), tol=1e-6, arith=nlh.SOLVE_MIXED, inner_tol=1e-3)
    assert rmx.info["status"] == 0
    assert rmx.info["rel_res_true"] <= 1e-6
    assert rmx.info["matvecs_fp32"] > 0 and rmx.info["outer"] >= 1
    assert rel(host(rmx.u), host(r64.u)) < 1e-5


def test_df32_solve_matches_oracle_iterates(tight64):
    """The double-float solve follows the oracle's U-coordinate CG and its
    solution is certified by the direct operator."""
    img, coords, _ = tight64
    P = make_plan(img, M=64, n_os=128, m=8, fill=0.5, precision=6)
    b = ALPHA * img.ravel()
    res = P.solve(ALPHA, cuda(b), tol=1e-6, arith=nlh.SOLVE_DF32)
    o = orc.pcg_deflated(coords, SIGMA, ALPHA, 1.0, b, tol=1e-6, maxit=200)
    assert res.info["iters"] == o.iters
    np.testing.assert_allclose(res.hist, o.hist[:o.iters + 1], rtol=1e-7)
    r = b - orc.A_apply(coords, SIGMA, ALPHA, 1.0, host(res.u))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 2e-6
    # mixed form with double-float refinement residuals
    rmx = P.solve(ALPHA, cuda(b), tol=1e-6, arith=nlh.SOLVE_MIXED, inner_tol=1e-3)
    assert rmx.info["status"] == 0 and rmx.info["rel_res_true"] <= 1e-6
    r = b - orc.A_apply(coords, SIGMA, ALPHA, 1.0, host(rmx.u))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 2e-6


@pytest.mark.parametrize("arith", [nlh.SOLVE_FP64, nlh.SOLVE_MIXED])
def test_graph_solve_equals_host_loop(tight64, arith):
    """The solve as one CUDA graph (device-side WHILE loop) and the
    host-driven loop run the same kernels: same iterations, and histories and
    solutions equal up to the run-to-run rounding of the atomic grid sums."""
    img, coords, P = tight64
    b = cuda(ALPHA * img.ravel())
    # FP32 atomic sums round differently from run to run (~1e-7 relative);
    # in the mixed form that reaches the refinement residuals
    hist_tol, u_tol = (1e-8, 1e-10) if arith == nlh.SOLVE_FP64 else (1e-2, 1e-6)
    g = P.solve(ALPHA, b, tol=1e-7, arith=arith, inner_tol=1e-3)
    h = P.solve(ALPHA, b, tol=1e-7, arith=arith, inner_tol=1e-3, check_every=3)
    assert abs(g.info["iters"] - h.info["iters"]) <= (0 if arith == nlh.SOLVE_FP64 else 1)
    assert g.info["outer"] == h.info["outer"]
    np.testing.assert_allclose(g.hist, h.hist, rtol=hist_tol)
    assert rel(host(g.u), host(h.u)) < u_tol
    # a second graph launch (cached graph) reproduces the first
    g2 = P.solve(ALPHA, b, tol=1e-7, arith=arith, inner_tol=1e-3)
    assert g2.info["rel_res_true"] <= 1e-7 * (1.5 if arith == nlh.SOLVE_FP64 else 1.0)
    assert rel(host(g2.u), host(g.u)) < u_tol


def test_warm_start_and_diag_scale(tight64):
    img, coords, P = tight64
    b = ALPHA * img.ravel()
    ref = P.solve(ALPHA, cuda(b), tol=1e-8)
    # exact warm start: converged at iteration 0
    res = P.solve(ALPHA, cuda(b), tol=1e-6, x0=ref.u.clone())
    assert res.info["iters"] == 0 and res.info["rel_res_true"] <= 1e-6
    # a constant positive diagonal scale is a no-op for CG (z scales, p too)
    res2 = P.solve(ALPHA, cuda(b), tol=1e-6, diag_scale=cuda(np.full(img.size, 3.0)))
    res1 = P.solve(ALPHA, cuda(b), tol=1e-6)
    assert res2.info["iters"] == res1.info["iters"]
    # a harmful scale still ends at the tolerance (fallback if needed)
    bad = np.exp(np.random.Generator(np.random.PCG64(3)).uniform(-4, 4, img.size))
    res3 = P.solve(ALPHA, cuda(b), tol=1e-6, maxit=60, diag_scale=cuda(bad))
    assert res3.info["rel_res_true"] <= 1.5e-6


def test_constant_image_one_iteration():
    img = np.full((16, 16), 0.3)
    P = make_plan(img, precision=3)
    b = random_vector(256, 4)
    res = P.solve(1e-3, cuda(b), tol=1e-8, method=nlh.PCG_DEFLATED)
    assert res.info["iters"] <= 1


def test_maximum_principle(tight64):
    img, coords, P = tight64
    f = img.ravel()
    u = host(P.solve(0.05, cuda(0.05 * f), tol=1e-8).u)
    assert u.min() >= f.min() - 1e-6 and u.max() <= f.max() + 1e-6


def test_breakdown_and_argument_errors(tight64):
    img, coords, P = tight64
    b = ALPHA * img.ravel()
    bad = b.copy()
    bad[17] = np.nan
    with pytest.raises(nlh.NLHError) as e:
        P.solve(ALPHA, cuda(bad), tol=1e-6)
    assert e.value.status == -4
    with pytest.raises(nlh.NLHError):
        P.solve(0.0, cuda(b))
    res = P.solve(ALPHA, cuda(b), tol=1e-14, maxit=2)
    assert res.info["status"] == 1 and res.info["iters"] == 2


def test_solve_512_fp64_and_mixed():
    """The timed workload: every form reaches the 1e-6 FP64-accurate residual
    and they agree."""
    img = image(512)
    P = make_plan(img, precision=7)
    b = ALPHA * img.ravel()
    r64 = P.solve(ALPHA, cuda(b), tol=1e-6, arith=nlh.SOLVE_FP64)
    rmx = P.solve(ALPHA, cuda(b), tol=1e-6, arith=nlh.SOLVE_MIXED, inner_tol=1e-3)
    rdf = P.solve(ALPHA, cuda(b), tol=1e-6, arith=nlh.SOLVE_DF32)
    assert r64.info["rel_res_true"] <= 1.5e-6 and rmx.info["rel_res_true"] <= 1e-6
    assert rdf.info["rel_res_true"] <= 1.5e-6
    assert rel(host(rmx.u), host(r64.u)) < 1e-5
    assert rel(host(rdf.u), host(r64.u)) < 1e-9
    # the mixed form's double-float residual agrees with an FP64 matvec
    q = host(P.matvec(rmx.u, op=2, alpha=ALPHA, precision=nlh.NLH_FP64))
    assert np.linalg.norm(b - q) / np.linalg.norm(b) <= 1.01e-6
    # maximum principle on the large image
    u = host(r64.u)
    assert u.min() >= img.min() - 1e-4 and u.max() <= img.max() + 1e-4


def test_warm_start_screening(tight64):
    """With x0_check a warm start whose residual is not below that of the
    method's own start is dropped (the solve equals the plain one); a good
    one is kept."""
    img, coords, P = tight64
    b = ALPHA * img.ravel()
    plain = P.solve(ALPHA, cuda(b), tol=1e-6)
    bad = cuda(img.ravel() + random_vector(img.size, 31))
    r = P.solve(ALPHA, cuda(b), tol=1e-6, x0=bad, x0_check=True)
    assert r.info["x0_rejected"] == 1 and r.info["iters"] == plain.info["iters"]
    np.testing.assert_allclose(r.hist, plain.hist, rtol=1e-9)   # FP64 atomic-order rounding
    good = P.solve(ALPHA, cuda(b), tol=1e-3).u
    r = P.solve(ALPHA, cuda(b), tol=1e-6, x0=good, x0_check=True)
    assert r.info["x0_rejected"] == 0 and r.info["iters"] < plain.info["iters"]
    for arith in (nlh.SOLVE_MIXED,):
        m0 = P.solve(ALPHA, cuda(b), tol=1e-6, arith=arith, inner_tol=1e-3)
        m1 = P.solve(ALPHA, cuda(b), tol=1e-6, arith=arith, inner_tol=1e-3, x0=bad, x0_check=True)
        assert m1.info["x0_rejected"] == 1 and m1.info["rel_res_true"] <= 1e-6
        assert abs(m1.info["iters"] - m0.info["iters"]) <= 1
        m2 = P.solve(ALPHA, cuda(b), tol=1e-6, arith=arith, inner_tol=1e-3, x0=good, x0_check=True)
        assert m2.info["x0_rejected"] == 0 and m2.info["rel_res_true"] <= 1e-6
    # without the check the paper's CG start (x0 = f) is used as given
    r = P.solve(ALPHA, cuda(b), tol=1e-6, method=nlh.CG, x0=cuda(img.ravel()))
    assert r.info["x0_rejected"] == 0


def test_pb_preconditioner_matches_oracle(tight64):
    """P_b' (Sec. 4.3.3): the deflated CG with P_b' follows the oracle's
    U-coordinate CG with P_b' residual by residual; Jacobi-PCG with P_b' from
    x0 = f follows the oracle's; the mixed form reaches the tolerance."""
    img, coords, P = tight64
    f = img.ravel()
    b = ALPHA * f
    res = P.solve(ALPHA, cuda(b), tol=1e-6, method=nlh.PCG_DEFLATED, precond=nlh.PREC_PB)
    o = orc.pcg_deflated(coords, SIGMA, ALPHA, 1.0, b, tol=1e-6, maxit=200, precond=2)
    assert res.info["status"] == 0 and res.info["iters"] == o.iters
    np.testing.assert_allclose(res.hist, o.hist[:o.iters + 1], rtol=1e-7)
    r2 = P.solve(ALPHA, cuda(b), tol=1e-6, maxit=400, method=nlh.PCG_JACOBI, x0=cuda(f),
                 precond=nlh.PREC_PB)
    o2 = orc.cg(coords, SIGMA, ALPHA, 1.0, b, x0=f, tol=1e-6, maxit=400, precond=2)
    assert abs(r2.info["iters"] - o2.iters) <= 1
    n = min(r2.info["iters"], o2.iters) + 1
    np.testing.assert_allclose(r2.hist[:n], o2.hist[:n], rtol=1e-6)
    # P_b' and P_a need comparable iteration counts (Table 3)
    ra = P.solve(ALPHA, cuda(b), tol=1e-6, method=nlh.PCG_DEFLATED)
    assert abs(ra.info["iters"] - res.info["iters"]) <= max(2, ra.info["iters"] // 2)
    # after a change of sigma the P_b' term is recomputed
    P.set_sigma(0.3)
    r3 = P.solve(ALPHA, cuda(b), tol=1e-6, method=nlh.PCG_DEFLATED, precond=nlh.PREC_PB)
    o3 = orc.pcg_deflated(coords, 0.3, ALPHA, 1.0, b, tol=1e-6, maxit=200, precond=2)
    P.set_sigma(SIGMA)
    assert r3.info["iters"] == o3.iters
    np.testing.assert_allclose(r3.hist, o3.hist[:o3.iters + 1], rtol=1e-7)
    Pm = make_plan(img, precision=6)
    rm = Pm.solve(ALPHA, cuda(b), tol=1e-6, arith=nlh.SOLVE_MIXED, inner_tol=1e-3,
                  precond=nlh.PREC_PB)
    assert rm.info["rel_res_true"] <= 1e-6
    with pytest.raises(nlh.NLHError):
        P.solve(ALPHA, cuda(b), precond=2)
