"""GPU test of nlh_residual_norms_noalloc, the entry point that allocates
nothing (its partial sums live in a fixed array inside the library), for
callers that cannot allocate device memory when they need a residual.

It is checked through the C ABI against the residual that the existing
nlh_solve entry point reports (rel_res_true), on two calls in a row with
different data, so that a stale or unreset scratch array would show.  This
file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2407_06834_gb300 import nlh  # noqa: E402
from gpu_helpers import cuda, host, image, make_plan  # noqa: E402


def _norms(b, q, res=None):
    lib = nlh.load()
    norms = torch.empty(2, dtype=torch.float64, device=b.device)
    st = lib.nlh_residual_norms_noalloc(b.data_ptr(), q.data_ptr(), b.numel(),
                                        None if res is None else res.data_ptr(),
                                        norms.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.nlh_last_error().decode()
    torch.cuda.synchronize()
    return host(norms)


def test_noalloc_residual_matches_solver_on_two_calls():
    img = image(64)
    P = make_plan(img, precision=3)
    seen = []
    for alpha, tol in ((0.5, 1e-6), (0.05, 1e-8)):
        b = cuda(alpha * img.ravel())
        res_solve = P.solve(alpha, b, tol=tol)
        q = P.matvec(res_solve.u, op=2, precision=nlh.NLH_FP64, alpha=alpha)
        r = torch.empty_like(b)
        nr, nb = _norms(b, q, r)
        # the existing entry point's FP64 residual of the same solution
        assert nr / nb == pytest.approx(res_solve.info["rel_res_true"], rel=1e-6)
        np.testing.assert_array_equal(host(r), host(b) - host(q))
        assert nb == pytest.approx(float(torch.linalg.norm(b)), rel=1e-13)
        seen.append(nr / nb)
    assert seen[0] != seen[1]


def test_noalloc_many_blocks_matches_solver_on_two_calls():
    """512 x 512 pixels: 64 blocks of 4096 elements, so the finishing
    reduction sums partials of many slots of the library's array."""
    img = image(512)
    P = make_plan(img, precision=3)
    prev = None
    for alpha in (0.5, 2.0):
        b = cuda(alpha * img.ravel())
        res_solve = P.solve(alpha, b, tol=1e-6)
        q = P.matvec(res_solve.u, op=2, precision=nlh.NLH_FP64, alpha=alpha)
        nr, nb = _norms(b, q)
        assert nr / nb == pytest.approx(res_solve.info["rel_res_true"], rel=1e-6)
        hb, hq = host(b), host(q)
        assert nr == pytest.approx(float(np.linalg.norm(hb - hq)), rel=1e-12)
        assert nb == pytest.approx(float(np.linalg.norm(hb)), rel=1e-13)
        assert prev is None or nb != prev
        prev = nb
    P.close()


def test_noalloc_rejects_sizes_beyond_the_array():
    lib = nlh.load()
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = lib.nlh_residual_norms_noalloc(x.data_ptr(), x.data_ptr(), (1 << 25) + 1, None,
                                        x.data_ptr(), None)
    assert st == -1
    assert "exceeds the maximum" in lib.nlh_last_error().decode()
