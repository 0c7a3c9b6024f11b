"""GPU parity of the mutual-information window selection (include/nlh_mis.h)
against the FP64 oracle (oracle/mis.py).

Bars: joint counts and windows bit-exact (integer work; both sides bin in
FP64 with the same two rounded operations); scores within 1e-12 relative
(the same terms summed in a different order, and CUDA's log against the
host's, each within an ulp or two).  Where two scores tie up to that
tolerance their order may differ; then only the set of dimensions in the
tied ranks is compared."""
import numpy as np
import pytest

from oracle import mis as omis
from paper_2407_06834_gb300.inputs import synthetic_image
from gpu_helpers import cuda, host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2407_06834_gb300 import nlh  # noqa: E402


def _check_windows(w_gpu, w_ref, s_ref):
    a, b = w_gpu.reshape(-1), w_ref.reshape(-1)
    D = s_ref.size
    assert (a[D:] == -1).all() and sorted(a[:D].tolist()) == list(range(D))
    i = 0
    while i < D:
        j = i + 1
        while j < D and abs(s_ref[b[j]] - s_ref[b[i]]) <= 1e-12 * abs(s_ref[b[i]]):
            j += 1
        assert sorted(a[i:j].tolist()) == sorted(b[i:j].tolist()), (i, j)
        i = j


@pytest.mark.parametrize("n1,n2,radius,pad,bins", [
    (64, 64, 1, "reflect", 64), (37, 53, 1, "zero", 16), (96, 80, 2, "reflect", 32),
    (40, 40, 2, "zero", 128), (1, 7, 1, "reflect", 8), (33, 5, 3, "zero", 2)])
def test_matches_oracle(n1, n2, radius, pad, bins):
    _, img = synthetic_image(n1, n2, 11)
    s, w, c = nlh.mis_windows(cuda(img), radius, pad, bins, want_counts=True)
    torch.cuda.synchronize()
    s_ref, c_ref = omis.mis_scores(img, radius, pad, bins)
    assert (host(c).astype(np.int64) == np.stack(c_ref)).all()
    np.testing.assert_allclose(host(s), s_ref, rtol=1e-12, atol=1e-300)
    _check_windows(w, omis.rank_windows(s_ref), s_ref)


def test_constant_image_and_degenerate_sizes():
    img = np.full((9, 11), 0.25)
    s, w, c = nlh.mis_windows(cuda(img), 1, "reflect", 8, want_counts=True)
    assert (host(s) == 0.0).all()
    assert w.reshape(-1).tolist() == list(range(9))
    assert (host(c)[:, 0, 0] == 99).all() and host(c).sum() == 9 * 99
    s, w, _ = nlh.mis_windows(cuda(np.arange(5.0).reshape(1, 5)), 0, "zero", 4)
    assert w.tolist() == [[0, -1, -1]] and host(s)[0] > 0


def test_full_size_sampled():
    """2048 x 2048 with 5 x 5 patches: the counts of sampled dimensions are
    integer sums over all pixels, so they are checked against the oracle's
    histogram of those dimensions (the scores follow from the counts)."""
    n, radius, bins = 2048, 2, 64
    _, img = synthetic_image(n, n, 0)
    s, w, c = nlh.mis_windows(cuda(img), radius, "reflect", bins, want_counts=True)
    torch.cuda.synchronize()
    ch = host(c).astype(np.int64)
    from oracle import oracle as orc
    y = img.reshape(-1)
    P = 2 * radius + 1
    for d in (0, 7, 12, 24):
        dr, dc = d // P - radius, d % P - radius
        rows = np.abs(np.arange(n) + dr)
        rows = np.where(rows >= n, 2 * (n - 1) - rows, rows)
        cols = np.abs(np.arange(n) + dc)
        cols = np.where(cols >= n, 2 * (n - 1) - cols, cols)
        x = img[np.ix_(rows, cols)].reshape(-1)
        ref = omis.joint_counts(x, y, bins)
        assert (ch[d] == ref).all(), d
        assert host(s)[d] == pytest.approx(omis.mi_from_counts(ref), rel=1e-12)
    assert w[0, 0] == 12  # the center pixel is the target itself
    assert ch.sum() == 25 * n * n
    del orc


def test_argument_errors():
    img = cuda(np.zeros((8, 8)))
    with pytest.raises(nlh.NLHError):
        nlh.mis_windows(img, 7)
    with pytest.raises(nlh.NLHError):
        nlh.mis_windows(img, 1, bins=1)
    with pytest.raises(nlh.NLHError):
        nlh.mis_windows(img, 1, bins=129)


def test_windows_feed_a_plan():
    """Ranked windows build a plan whose operator matches the oracle's
    direct sum on those windows (tight NFFT parameters, FP64 path)."""
    from oracle import oracle as orc
    _, img = synthetic_image(32, 32, 5)
    _, w, _ = nlh.mis_windows(cuda(img), 1, "reflect", 32)
    assert sorted(w.reshape(-1).tolist()) == list(range(9))
    P = nlh.Plan.from_image(cuda(img), 1, w, 0.2, pad="reflect", M=64, n_os=128, m=8,
                            precision=1, torus_fill=0.5)
    v = np.random.default_rng(0).standard_normal(32 * 32)
    y = host(P.matvec(cuda(v), op=0, precision=nlh.NLH_FP64))
    ref = orc.gamma_full_matvec(orc.image_coords(img, 1, w), 0.2, v)
    assert np.max(np.abs(y - ref)) < 1e-10 * np.max(np.abs(ref))
    P.close()
