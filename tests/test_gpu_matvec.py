"""GPU parity of the NFFT matvec against the CPU oracle (through the C ABI).

Tolerances (relative, max-norm over the output vector):
  * FP64 path at tight NFFT parameters (M = 64, n_os = 128, m = 8, fill 0.5)
    vs the oracle's direct Gaussian sum: 1e-10.  At these parameters the
    truncation term erfc(pi sigma_s (M/2 - 1)) ~ 1e-17, the alias term
    exp(-((1 - fill)/sigma_s)^2) ~ 1e-28 and the Kaiser-Bessel window error
    ~ 1e-15, so 1e-10 leaves room for the O(N) rounding of the sums.
  * FP64 path at the configured parameters (M = 32, n_os = 64, m = 4) vs the
    oracle's truncated-Fourier kernel sum at the same torus map: 1e-6
    (only the window error of the NFFT remains), and vs the direct Gaussian
    sum: within 10 x the a-priori estimate.
  * FP32 path vs the oracle's direct sum at tight parameters, vs its
    truncated-Fourier sum at the configured parameters, and vs the FP64
    path: 1e-5 (element-wise, relative to the largest output).
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2407_06834_gb300.inputs import random_vector, raster_windows
from gpu_helpers import cuda, host, image, make_plan, relmax, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2407_06834_gb300 import nlh  # noqa: E402

SIGMA = 0.2


@pytest.mark.parametrize("shape,radius,pad", [((17, 23), 1, "reflect"), ((8, 5), 2, "zero"),
                                              ((64, 64), 1, "reflect"), ((1, 1), 1, "reflect")])
def test_patch_features_bit_exact(shape, radius, pad):
    img = image(*shape)
    got = host(nlh.patch_features(cuda(img), radius, pad))
    np.testing.assert_array_equal(got, orc.patch_features(img, radius, pad))


@pytest.fixture(scope="module")
def img64():
    img = image(64)
    coords = orc.image_coords(img, 1, raster_windows(1))
    return img, coords


def test_fp64_tight_parameters_match_direct_sum(img64):
    img, coords = img64
    P = make_plan(img, M=64, n_os=128, m=8, fill=0.5, precision=1)
    for seed in (1, 2):
        v = random_vector(img.size, seed)
        y = host(P.matvec(cuda(v), op=0, precision=nlh.NLH_FP64))
        ref = orc.gamma_full_matvec(coords, SIGMA, v)
        assert relmax(y, ref) < 1e-10, relmax(y, ref)


def test_df32_tight_parameters_match_direct_sum(img64):
    """The double-float path (pairs of floats) is FP64-accurate: same 1e-10
    bar against the direct sum as the FP64 path."""
    img, coords = img64
    P = make_plan(img, M=64, n_os=128, m=8, fill=0.5, precision=5)
    v = random_vector(img.size, 21)
    ref = orc.gamma_full_matvec(coords, SIGMA, v)
    y = host(P.matvec(cuda(v), op=0, precision=nlh.NLH_DF32))
    assert relmax(y, ref) < 1e-10, relmax(y, ref)
    y64 = host(P.matvec(cuda(v), op=0, precision=nlh.NLH_FP64))
    assert relmax(y, y64) < 1e-12


def test_df32_configured_parameters_and_laplacian(img64):
    img, coords = img64
    P = make_plan(img, precision=7)
    N = img.size
    v = random_vector(N, 22)
    y64 = host(P.matvec(cuda(v), op=2, alpha=0.5, precision=nlh.NLH_FP64))
    ydf = host(P.matvec(cuda(v), op=2, alpha=0.5, precision=nlh.NLH_DF32))
    assert relmax(ydf, y64) < 1e-11, relmax(ydf, y64)
    one = cuda(np.ones(N))
    d = host(P.matvec(one, op=0, precision=nlh.NLH_DF32))
    L1 = host(P.matvec(one, op=1, precision=nlh.NLH_DF32))
    assert np.max(np.abs(L1)) < 1e-12 * np.max(d)


@pytest.mark.parametrize("m,shape,kmax", [(8, (64, 64), 0), (6, (64, 64), 0), (8, (37, 53), 7)])
def test_fp32_tight_parameters_match_direct_sum(m, shape, kmax):
    """The FP32 path (FP32 window weights, grid sums, convolution and
    interpolation) against the oracle's direct Gaussian sum at tight NFFT
    parameters (M = 64, n_os = 128, fill 0.5, where the NFFT's own error is
    far below FP32 rounding): element-wise within 1e-5 of max |Gamma_full v|,
    the FP32 accuracy bar of the matvec (Sec. 5.3).  The ragged image with
    7-point items spans many tiles and partial items."""
    img = image(*shape, seed=m)
    coords = orc.image_coords(img, 1, raster_windows(1))
    P = make_plan(img, M=64, n_os=128, m=m, fill=0.5, precision=6, kmax=kmax)
    for seed in (31, 32):
        v = random_vector(img.size, seed)
        ref = orc.gamma_full_matvec(coords, SIGMA, v)
        y32 = host(P.matvec(cuda(v), op=0, precision=nlh.NLH_FP32))
        assert relmax(y32, ref) < 1e-5, relmax(y32, ref)
    ones = np.ones(img.size)
    d32 = host(P.matvec(cuda(ones), op=0, precision=nlh.NLH_FP32))
    assert relmax(d32, orc.gamma_full_matvec(coords, SIGMA, ones)) < 1e-5


def test_fp32_configured_5x5_windows_match_truncated_fourier_sum():
    """5x5 patches (L = 9 windows, the last zero-padded) at the NFFT
    parameters of the 2048 x 2048 workload (M = 64, n_os = 128, m = 6) on a
    small image: FP32 and double-float against the oracle's truncated-Fourier
    kernel sum at the plan's torus map (the NFFT's window error only), and
    against the direct Gaussian sum within the a-priori estimate."""
    img = image(30, 26, seed=8)
    win = raster_windows(2)
    coords = orc.image_coords(img, 2, win)
    P = nlh.Plan.from_image(cuda(img), 2, win, SIGMA, M=64, n_os=128, m=6, precision=6)
    info = P.info()
    tc, s = orc.torus_map(coords, info["torus_fill"])
    assert info["scale"] == pytest.approx(s, rel=1e-14) and info["L"] == 9
    v = random_vector(img.size, 33)
    trig = orc.trig_full_matvec(tc, s * SIGMA, 64, v)
    y32 = host(P.matvec(cuda(v), op=0, precision=nlh.NLH_FP32))
    ydf = host(P.matvec(cuda(v), op=0, precision=nlh.NLH_DF32))
    assert relmax(ydf, trig) < 1e-8, relmax(ydf, trig)
    assert relmax(y32, trig) < 1e-5, relmax(y32, trig)
    ref = orc.gamma_full_matvec(coords, SIGMA, v)
    est = max(info["est_trunc_err"], info["est_alias_err"])
    scale = np.abs(v).sum() / np.max(np.abs(ref))
    assert relmax(y32, ref) < 10 * est * scale + 1e-5


@pytest.mark.parametrize("radius,pad,shape", [(1, "reflect", (33, 29)), (2, "zero", (20, 24)),
                                              (2, "reflect", (1, 40))])
def test_image_coordinates_match_stored_offsets(radius, pad, shape):
    """A plan that recomputes the points' coordinates from the image
    against one that stores each point's cell offsets (the default): the same operator in every arithmetic (FP64 and double-float
    coordinates agree to ~1e-14, the FP32 path's to FP32 rounding), with
    less device memory; reflect and zero padding, a one-row image."""
    img = image(*shape, seed=radius)
    win = raster_windows(radius)
    f = cuda(img)
    kw = dict(pad=pad, M=32, n_os=64, m=4, precision=7)
    a = nlh.Plan.from_image(f, radius, win, SIGMA, coords_from_image=True, **kw)
    b = nlh.Plan.from_image(f, radius, win, SIGMA, **kw)
    ia, ib = a.info(), b.info()
    assert ia["coords_from_image"] == 1 and ib["coords_from_image"] == 0
    assert ia["device_bytes"] < ib["device_bytes"]
    assert ia["n_items"] == ib["n_items"] and ia["scale"] == ib["scale"]
    v = cuda(random_vector(img.size, 9))
    for prec, tol in ((nlh.NLH_FP64, 1e-12), (nlh.NLH_DF32, 1e-12), (nlh.NLH_FP32, 1e-5)):
        for op in (0, 2):
            ya = host(a.matvec(v, op=op, alpha=0.5, precision=prec))
            yb = host(b.matvec(v, op=op, alpha=0.5, precision=prec))
            assert relmax(ya, yb) < tol, (prec, op, relmax(ya, yb))
    assert relmax(host(a.degrees()), host(b.degrees())) < 1e-12
    coords = orc.image_coords(img, radius, win, pad)
    ref = orc.gamma_full_matvec(coords, SIGMA, host(v))
    y32 = host(a.matvec(v, op=0, precision=nlh.NLH_FP32))
    y64 = host(a.matvec(v, op=0, precision=nlh.NLH_FP64))
    assert relmax(y32, y64) < 1e-5
    est = max(ia["est_trunc_err"], ia["est_alias_err"])
    assert relmax(y64, ref) < 10 * est * np.abs(host(v)).sum() / np.max(np.abs(ref)) + 1e-6


@pytest.mark.parametrize("M,n_os,m,tol", [(16, 32, 3, 1e-4), (64, 128, 5, 1e-6),
                                          (100, 256, 4, 1e-6)])
def test_grid_sizes_match_truncated_fourier_sum(M, n_os, m, tol):
    """Every grid size of the convolution: n_os = 32 and 128 (x and y in one
    plane kernel, then z) and 256 (three axis passes), against the oracle's
    truncated-Fourier kernel sum at the plan's torus map (the window error
    of the NFFT only, bounded by tol for the cutoff and oversampling), the
    double-float path against FP64 and FP32 within 1e-5."""
    img = image(20, 24, seed=M)
    coords = orc.image_coords(img, 1, raster_windows(1))
    P = make_plan(img, M=M, n_os=n_os, m=m, precision=7)
    info = P.info()
    assert (info["n_os"], info["M"], info["m"]) == (n_os, M, m)
    tc, s = orc.torus_map(coords, info["torus_fill"])
    v = random_vector(img.size, 40)
    trig = orc.trig_full_matvec(tc, s * SIGMA, M, v)
    y64 = host(P.matvec(cuda(v), op=0, precision=nlh.NLH_FP64))
    ydf = host(P.matvec(cuda(v), op=0, precision=nlh.NLH_DF32))
    y32 = host(P.matvec(cuda(v), op=0, precision=nlh.NLH_FP32))
    assert relmax(y64, trig) < tol, relmax(y64, trig)
    assert relmax(ydf, y64) < 1e-12, relmax(ydf, y64)
    assert relmax(y32, y64) < 1e-5, relmax(y32, y64)
    ones = cuda(np.ones(img.size))
    for prec, t in ((nlh.NLH_FP64, 1e-12), (nlh.NLH_DF32, 1e-11), (nlh.NLH_FP32, 1e-5)):
        l1 = host(P.matvec(ones, op=1, precision=prec))
        assert np.abs(l1).max() < t * host(P.degrees()).max(), (prec, np.abs(l1).max())


def test_two_pixel_image():
    """The smallest plan (N = 2, one row of two pixels, reflect padding):
    every arithmetic against the direct sum at tight parameters, and a
    solve certified by the direct operator.  The two points are close
    against sigma, so the torus fill is chosen by the plan (a fixed fill of
    0.5 would make sigma on the torus ~1 and the periodic copies overlap;
    the plan's alias estimate reports that)."""
    img = image(1, 2, seed=9)
    coords = orc.image_coords(img, 1, raster_windows(1))
    P = make_plan(img, M=64, n_os=128, m=8, precision=7)
    info = P.info()
    assert max(info["est_trunc_err"], info["est_alias_err"]) < 1e-12, info
    v = random_vector(2, 41)
    ref = orc.gamma_full_matvec(coords, SIGMA, v)
    for prec, tol in ((nlh.NLH_FP64, 1e-10), (nlh.NLH_DF32, 1e-10), (nlh.NLH_FP32, 1e-5)):
        y = host(P.matvec(cuda(v), op=0, precision=prec))
        assert relmax(y, ref) < tol, (prec, relmax(y, ref))
    b = 0.5 * img.ravel()
    res = P.solve(0.5, cuda(b), tol=1e-6, arith=nlh.SOLVE_MIXED, inner_tol=1e-3)
    r = b - orc.A_apply(coords, SIGMA, 0.5, 1.0, host(res.u))
    assert res.info["status"] == 0 and np.linalg.norm(r) / np.linalg.norm(b) <= 2e-6


def test_fp64_ragged_image_tight(img64):
    img = image(37, 53, seed=3)
    coords = orc.image_coords(img, 1, raster_windows(1))
    P = make_plan(img, M=64, n_os=128, m=8, fill=0.5, precision=1, kmax=7)
    v = random_vector(img.size, 4)
    y = host(P.matvec(cuda(v), op=0, precision=nlh.NLH_FP64))
    assert relmax(y, orc.gamma_full_matvec(coords, SIGMA, v)) < 1e-10


def test_configured_parameters_window_error_only(img64):
    img, coords = img64
    P = make_plan(img, precision=3)
    info = P.info()
    fill, s = info["torus_fill"], info["scale"]
    tc, s_orc = orc.torus_map(coords, fill)
    assert s == pytest.approx(s_orc, rel=1e-14)
    v = random_vector(img.size, 5)
    y64 = host(P.matvec(cuda(v), op=0, precision=nlh.NLH_FP64))
    trig = orc.trig_full_matvec(tc, s * SIGMA, 32, v)
    assert relmax(y64, trig) < 1e-6, relmax(y64, trig)
    ref = orc.gamma_full_matvec(coords, SIGMA, v)
    est = max(info["est_trunc_err"], info["est_alias_err"])
    scale = np.abs(v).sum() / np.max(np.abs(ref))
    assert relmax(y64, ref) < 10 * est * scale + 1e-6
    y32 = host(P.matvec(cuda(v), op=0, precision=nlh.NLH_FP32))
    assert relmax(y32, y64) < 1e-5, relmax(y32, y64)
    assert relmax(y32, trig) < 1e-5, relmax(y32, trig)


def test_error_falls_with_cutoff_m(img64):
    img, coords = img64
    fill = 0.55
    tc, s = orc.torus_map(coords, fill)
    v = np.abs(random_vector(img.size, 6))
    trig = orc.trig_full_matvec(tc, s * SIGMA, 32, v)
    errs = []
    for m in (2, 3, 4, 5, 6):
        P = make_plan(img, m=m, fill=fill, precision=1)
        errs.append(relmax(host(P.matvec(cuda(v), precision=nlh.NLH_FP64)), trig))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-9


def test_error_falls_with_bandwidth_M(img64):
    img, coords = img64
    v = np.abs(random_vector(img.size, 7))
    ref = orc.gamma_full_matvec(coords, SIGMA, v)
    errs = []
    for M, n in ((8, 32), (16, 32), (24, 64), (32, 64), (48, 128)):
        P = make_plan(img, M=M, n_os=n, m=8 if n > 32 else 6, fill=0.5, precision=1)
        errs.append(relmax(host(P.matvec(cuda(v), precision=nlh.NLH_FP64)), ref))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs


def test_laplacian_ops_invariants(img64):
    img, coords = img64
    P = make_plan(img, precision=3)
    N = img.size
    one = cuda(np.ones(N))
    for prec, tol in ((nlh.NLH_FP64, 1e-12), (nlh.NLH_FP32, 1e-5)):
        d = host(P.matvec(one, op=0, precision=prec))
        L1 = host(P.matvec(one, op=1, precision=prec))
        assert np.max(np.abs(L1)) < tol * np.max(d)
        A1 = host(P.matvec(one, op=2, precision=prec, alpha=0.5))
        assert np.max(np.abs(A1 - 0.5)) < tol * np.max(d)
    v, w = random_vector(N, 8), random_vector(N, 9)
    Lv = host(P.matvec(cuda(v), op=1))
    Lw = host(P.matvec(cuda(w), op=1))
    assert w @ Lv == pytest.approx(v @ Lw, rel=1e-12)
    # degrees against the oracle's eta = Gamma 1 (diagonal removed)
    eta = orc.degrees(coords, SIGMA)
    d = host(P.matvec(one, op=0))
    assert relmax(d - 1.0, eta) < 1e-5


def test_constant_image_complete_graph():
    """Identical features: Gamma_full = 1 1^T up to the NFFT error."""
    img = np.full((16, 16), 0.4)
    P = make_plan(img, precision=3)
    v = random_vector(256, 10)
    y = host(P.matvec(cuda(v), precision=nlh.NLH_FP64))
    assert relmax(y, np.full(256, v.sum())) < 1e-6
    Lv = host(P.matvec(cuda(v), op=1, precision=nlh.NLH_FP64))
    np.testing.assert_allclose(Lv, 256 * v - v.sum() * np.ones(256), atol=1e-5 * 256 * np.abs(v).max())


def test_full_size_512_sampled_rows():
    """The timed workload (512 x 512, 3 windows, M = 32, n_os = 64, m = 4):
    sampled rows against direct sums, and FP32 against FP64 everywhere."""
    img = image(512)
    coords = orc.image_coords(img, 1, raster_windows(1))
    P = make_plan(img, precision=3)
    info = P.info()
    v = random_vector(img.size, 11)
    y64 = host(P.matvec(cuda(v), precision=nlh.NLH_FP64))
    y32 = host(P.matvec(cuda(v), precision=nlh.NLH_FP32))
    assert relmax(y32, y64) < 1e-5, relmax(y32, y64)
    rng = np.random.Generator(np.random.PCG64(12))
    rows = np.sort(rng.choice(img.size, 48, replace=False))
    ref = orc.gamma_full_rows(coords, SIGMA, v, rows)
    est = max(info["est_trunc_err"], info["est_alias_err"])
    bound = 10 * est * np.abs(v).sum() / np.max(np.abs(ref))
    err = np.max(np.abs(y64[rows] - ref)) / np.max(np.abs(ref))
    assert err < bound + 1e-6, err
    err32 = np.max(np.abs(y32[rows] - ref)) / np.max(np.abs(ref))
    assert err32 < bound + 1e-5, err32


def test_set_sigma_matches_fresh_plan(img64):
    img, coords = img64
    P = make_plan(img, M=64, n_os=128, m=8, fill=0.5, precision=1)
    P.set_sigma(0.3)
    v = random_vector(img.size, 13)
    y = host(P.matvec(cuda(v), precision=nlh.NLH_FP64))
    assert relmax(y, orc.gamma_full_matvec(coords, 0.3, v)) < 1e-10


def test_argument_errors():
    img = image(8)
    P = make_plan(img, precision=1)
    x = cuda(np.ones(64))
    with pytest.raises(nlh.NLHError):
        P.matvec(x, precision=nlh.NLH_FP32)        # FP32 path not built
    with pytest.raises(nlh.NLHError):
        P.matvec(x, op=7)
    with pytest.raises(nlh.NLHError):
        make_plan(img, n_os=48)                    # not a power of two
    with pytest.raises(nlh.NLHError):
        make_plan(img, M=5)


def test_double_float_weights_without_fp64_path(img64):
    """Plans without the FP64 path evaluate the window polynomials in
    double-float arithmetic; their double-float operator agrees with the one
    built from FP64-evaluated weights (a plan with both paths) to the
    double-float rounding, and the FP32 operator to FP32 rounding."""
    img, coords = img64
    P5 = make_plan(img, precision=5)   # FP64 + double-float: FP64 Horner
    P6 = make_plan(img, precision=6)   # FP32 + double-float: double-float Horner
    v = random_vector(img.size, 23)
    y5 = host(P5.matvec(cuda(v), op=2, alpha=0.5, precision=nlh.NLH_DF32))
    y6 = host(P6.matvec(cuda(v), op=2, alpha=0.5, precision=nlh.NLH_DF32))
    assert relmax(y6, y5) < 1e-11, relmax(y6, y5)
    y32 = host(P6.matvec(cuda(v), op=2, alpha=0.5, precision=nlh.NLH_FP32))
    assert relmax(y32, y5) < 1e-5
    one = cuda(np.ones(img.size))
    d = host(P6.matvec(one, op=0, precision=nlh.NLH_DF32))
    L1 = host(P6.matvec(one, op=1, precision=nlh.NLH_FP32))
    assert np.max(np.abs(L1)) < 1e-5 * np.max(d)
    assert relmax(host(P6.degrees()), host(P5.degrees())) < 1e-12


@pytest.mark.parametrize("m,shape,kmax", [(4, (64, 64), 0), (6, (37, 53), 0), (3, (16, 24), 7),
                                          (4, (16, 16), 0)])
def test_launch_shapes_and_tilings_agree(m, shape, kmax):
    """Every launch shape of the spreading kernel and small work items: the
    same sums in another order, for every arithmetic, on ragged images; the
    16 x 16 constant image puts every point into one cell (items of many
    chunks).  L 1 = 0 to rounding with the degrees of the shape in use."""
    img = image(*shape, seed=m) if shape != (16, 16) else np.full((16, 16), 0.3)
    P = make_plan(img, M=32, n_os=64, m=m, precision=7, kmax=kmax)
    v = cuda(random_vector(img.size, 5 + m))
    ref = {prec: host(P.matvec(v, op=0, precision=prec))
           for prec in (nlh.NLH_FP64, nlh.NLH_FP32, nlh.NLH_DF32)}
    assert relmax(ref[nlh.NLH_DF32], ref[nlh.NLH_FP64]) < 1e-12
    assert relmax(ref[nlh.NLH_FP32], ref[nlh.NLH_FP64]) < 1e-5
    for prec, tol in ((nlh.NLH_FP64, 1e-13), (nlh.NLH_DF32, 1e-12), (nlh.NLH_FP32, 1e-5)):
        for sh in (1, 2, 0):
            P.set_team(prec, sh)
            assert relmax(host(P.matvec(v, op=0, precision=prec)), ref[prec]) < tol, (prec, sh)
    ones = cuda(np.ones(img.size))
    d = host(P.degrees())
    for prec, tol in ((nlh.NLH_DF32, 1e-9), (nlh.NLH_FP32, 1e-5)):
        l1 = host(P.matvec(ones, op=1, precision=prec))
        assert np.abs(l1).max() < tol * d.max(), (prec, np.abs(l1).max() / d.max())
    P.close()
