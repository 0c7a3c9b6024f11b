"""The bilevel learning of alpha on the GPU (batched lower-level and adjoint
solves through the C ABI) against the dense FP64 oracle (oracle/bilevel.py).

At tight NFFT parameters (M = 64, n_os = 128, m = 8, fill 0.5; a-priori
error < 1e-14) and FP64 solves to 1e-11, j and dj/dalpha agree with the
dense solution to 1e-7 relative; Brent's minimiser on the GPU objective
agrees with the oracle's to 1e-4 in alpha (both with xatol 1e-7 in log
alpha); the mixed-precision form changes j by less than 1e-6."""
import numpy as np
import pytest

from oracle import bilevel as obl, oracle as orc
from paper_2407_06834_gb300.inputs import raster_windows, synthetic_image

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2407_06834_gb300 import bilevel, nlh  # noqa: E402

SIGMA = 0.2
TIGHT = dict(M=64, n_os=128, m=8, torus_fill=0.5, precision=5)


@pytest.fixture(scope="module")
def problem():
    pairs = [synthetic_image(16, 16, s) for s in (3, 4)]
    coords = [orc.image_coords(noisy, 1, raster_windows(1)) for _, noisy in pairs]
    Ls = obl.laplacians(coords, SIGMA)
    fs = [noisy.ravel() for _, noisy in pairs]
    ucs = [clean.ravel() for clean, _ in pairs]
    B = bilevel.Bilevel(pairs, SIGMA, tol=1e-11, arith=nlh.SOLVE_FP64, plan_kw=TIGHT)
    yield B, (Ls, fs, ucs), pairs
    B.close()


@pytest.mark.parametrize("alpha", [0.1, 5.0, 40.0])
def test_objective_and_gradient_match_oracle(problem, alpha):
    B, (Ls, fs, ucs), _ = problem
    j, g = B.objective_and_gradient(alpha)
    jo, go = obl.objective_and_gradient(Ls, fs, ucs, alpha)
    assert j == pytest.approx(jo, rel=1e-7)
    assert g == pytest.approx(go, rel=1e-6, abs=1e-9 * abs(jo))
    assert B.objective(alpha) == pytest.approx(j, rel=1e-12)


def test_learned_alpha_matches_oracle(problem):
    B, (Ls, fs, ucs), _ = problem
    res = B.learn(bounds=(1e-3, 1e3), xatol=1e-7)
    ao, jo, _ = obl.learn_alpha(Ls, fs, ucs, bounds=(1e-3, 1e3), xatol=1e-7)
    assert res.alpha == pytest.approx(ao, rel=1e-4)
    assert res.j == pytest.approx(jo, rel=1e-8)
    assert 1e-3 * 1.1 < res.alpha < 1e3 / 1.1
    assert res.solves == 2 * res.evaluations and res.cg_iters_mean > 0
    # the adjoint gradient vanishes at the learned alpha
    _, g = B.objective_and_gradient(res.alpha)
    jl = B.objective(res.alpha * 0.9)
    assert abs(g) * res.alpha < 1e-3 * abs(jl - res.j)


def test_mixed_precision_objective(problem):
    _, _, pairs = problem
    Bm = bilevel.Bilevel(pairs, SIGMA, tol=1e-8, plan_kw=dict(TIGHT, precision=6))
    Bf = bilevel.Bilevel(pairs, SIGMA, tol=1e-11, arith=nlh.SOLVE_FP64, plan_kw=TIGHT)
    try:
        for alpha in (0.5, 20.0):
            assert Bm.objective(alpha) == pytest.approx(Bf.objective(alpha), rel=1e-6)
    finally:
        Bm.close()
        Bf.close()


def test_reduction_argument_errors():
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert nlh.load().nlh_bilevel_misfit(0, x.data_ptr(), x.data_ptr(), None, None, None) == -1
    assert nlh.bilevel_gradient_term(x + 1, x + 3, x + 1) == pytest.approx(8.0)
    r = torch.empty_like(x)
    assert nlh.bilevel_misfit(x + 2, x, r) == pytest.approx(16.0)
    assert torch.all(r == 2)


def test_joint_alpha_theta_matches_oracle(problem):
    """Joint (alpha, theta = sigma^-2) learning (Sec. 5.5): L-BFGS-B with the
    adjoint alpha-derivative and a central difference in log theta, on the
    GPU and in the oracle, from the same start; sigma is kept in [0.15, 0.5],
    where the tight NFFT parameters stay below 1e-9."""
    B, (Ls, fs, ucs), pairs = problem
    coords = [orc.image_coords(noisy, 1, raster_windows(1)) for _, noisy in pairs]
    try:
        res = B.learn_alpha_theta(30.0, SIGMA, bounds_sigma=(0.15, 0.5))
        ao, so, jo = obl.learn_alpha_theta(coords, fs, ucs, 30.0, SIGMA, bounds_sigma=(0.15, 0.5))
        assert res["j"] == pytest.approx(jo, rel=1e-6)
        assert res["alpha"] == pytest.approx(ao, rel=1e-3)
        assert res["sigma"] == pytest.approx(so, rel=1e-3)
        j_alpha_only = obl.objective_and_gradient(Ls, fs, ucs, 30.0)[0]
        assert res["j"] <= j_alpha_only * (1 + 1e-9)
    finally:
        B.set_sigma(SIGMA)
