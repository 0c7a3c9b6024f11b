"""Window-range plans on one GPU (the matvec of Sec. 3 split over windows):
two plans of complementary ranges add up to the plan of all windows, in
every NFFT arithmetic, and a range plan whose reduce callback supplies the
other range's share acts as the operator of all windows (degrees, L x and
(alpha I + L) x).  The callback here adds precomputed shares in the order
the library calls it; across GPUs it is an all-reduce (shard.allreduce_sum),
whose reduction the gloo test covers on CPU ranks."""
import numpy as np
import pytest

from paper_2407_06834_gb300.inputs import random_vector, raster_windows
from gpu_helpers import cuda, host, image, relmax

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2407_06834_gb300 import nlh  # noqa: E402

WIN = raster_windows(2)          # 5x5 patches: L = 9 windows


def _plan(f, precision, **kw):
    return nlh.Plan.from_image(f, 2, WIN, 0.2, M=32, n_os=64, m=4, precision=precision, **kw)


@pytest.mark.parametrize("shape", [(40, 36), (17, 29)])
def test_complementary_ranges_sum_to_the_full_plan(shape):
    img = image(*shape, seed=3)
    f = cuda(img)
    full = _plan(f, 7)
    a = _plan(f, 7, window_range=(0, 5))
    b = _plan(f, 7, window_range=(5, 4))
    assert a.info()["window_count"] == 5 and b.info()["window_first"] == 5
    # the torus map is the full list's in every range plan
    assert a.info()["scale"] == full.info()["scale"] == b.info()["scale"]
    v = cuda(random_vector(img.size, 4))
    for prec, tol in ((nlh.NLH_FP64, 1e-13), (nlh.NLH_DF32, 1e-12), (nlh.NLH_FP32, 1e-5)):
        y = host(full.matvec(v, op=0, precision=prec))
        ya = host(a.matvec(v, op=0, precision=prec))
        yb = host(b.matvec(v, op=0, precision=prec))
        assert relmax(ya + yb, y) < tol, (prec, relmax(ya + yb, y))
    # without a reduce callback only the share (op 0) is defined
    with pytest.raises(nlh.NLHError):
        a.matvec(v, op=2, alpha=0.5)
    with pytest.raises(nlh.NLHError):
        _plan(f, 3, window_range=(5, 5))          # beyond the 9 windows


def test_reduce_callback_makes_a_range_plan_the_full_operator():
    img = image(48, 40, seed=5)
    f = cuda(img)
    full = _plan(f, 3)
    b = _plan(f, 3, window_range=(4, 5))
    ones = cuda(np.ones(img.size))
    x = cuda(random_vector(img.size, 6))
    # the other range's shares, in the order plan creation and the matvecs
    # call the callback: degrees (FP64, then FP32), then each matvec
    queue = [b.matvec(ones, op=0, precision=nlh.NLH_FP64),
             b.matvec(ones, op=0, precision=nlh.NLH_FP32),
             b.matvec(x, op=0, precision=nlh.NLH_FP64),
             b.matvec(x, op=0, precision=nlh.NLH_FP64),
             b.matvec(x, op=0, precision=nlh.NLH_FP32)]
    torch.cuda.synchronize()
    calls = []

    def reduce(buf, stream):
        with torch.cuda.stream(stream):
            buf.add_(queue[len(calls)])
        calls.append(buf.numel())

    a = _plan(f, 3, window_range=(0, 4), reduce=reduce)
    assert len(calls) == 2
    assert relmax(host(a.degrees()), host(full.degrees())) < 1e-13
    y2 = host(a.matvec(x, op=2, alpha=0.5, precision=nlh.NLH_FP64))
    assert relmax(y2, host(full.matvec(x, op=2, alpha=0.5, precision=nlh.NLH_FP64))) < 1e-12
    y1 = host(a.matvec(x, op=1, precision=nlh.NLH_FP64))
    assert relmax(y1, host(full.matvec(x, op=1, precision=nlh.NLH_FP64))) < 1e-11
    y32 = host(a.matvec(x, op=2, alpha=0.5, precision=nlh.NLH_FP32))
    assert relmax(y32, y2) < 1e-5
    assert calls == [img.size] * 5
