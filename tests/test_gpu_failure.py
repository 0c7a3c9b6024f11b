"""Failure detection of the bounded device waits, made without a GPU fault
(include/nlh_selftest.h): a wait on an mbarrier that nothing completes runs
out, records NLH_ERR_TIMEOUT in the plan's or the network's error word, and
the next synchronising call reports it; the context and the object stay
usable afterwards."""
import time

import numpy as np
import pytest

from paper_2407_06834_gb300.inputs import synthetic_image
from gpu_helpers import cuda, host, make_plan

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2407_06834_gb300 import nlh  # noqa: E402

TIMEOUT = -5


def _timed(fn):
    t0 = time.perf_counter()
    fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t0


def test_plan_wait_timeout_is_reported_once_and_the_plan_recovers():
    _, img = synthetic_image(40, 40, 2)
    P = make_plan(img, precision=3)
    b = cuda(img.reshape(-1) * 0.5)
    ref = P.solve(0.5, b, tol=1e-6)
    dt = _timed(lambda: nlh._check(nlh.load().nlh_selftest_plan_timeout(P._h, None)))
    assert dt < 30.0, dt
    with pytest.raises(nlh.NLHError) as e:
        P.solve(0.5, b, tol=1e-6)
    assert e.value.status == TIMEOUT
    again = P.solve(0.5, b, tol=1e-6)
    assert again.info["status"] == 0 and again.info["iters"] == ref.info["iters"]
    np.testing.assert_allclose(host(again.u), host(ref.u), rtol=0, atol=1e-12)
    P.close()


def test_net_wait_timeout_is_reported_once_and_the_net_recovers():
    net = nlh.Net(32, 2)
    f = cuda(synthetic_image(16, 16, 3)[1][None])
    u_ref, _ = net.forward(f, [0.2], [0.5])
    net.check()
    dt = _timed(lambda: nlh._check(nlh.load().nlh_selftest_net_timeout(net._h, None)))
    assert dt < 30.0, dt
    with pytest.raises(nlh.NLHError) as e:
        net.check()
    assert e.value.status == TIMEOUT
    net.check()  # reported once, then cleared
    u, _ = net.forward(f, [0.2], [0.5])
    net.check()
    assert torch.equal(u, u_ref)
    net.close()


def test_hooks_reject_null_objects():
    assert nlh.load().nlh_selftest_plan_timeout(None, None) == -1
    assert nlh.load().nlh_selftest_net_timeout(None, None) == -1
