// selftest.cu -- test hooks for the failure path of the bounded device waits
// (include/nlh_selftest.h).  The network's hook sits in net.cu, next to the
// network's definition.
#include "common.cuh"
#include "async_copy.cuh"
#include "../../include/nlh_selftest.h"

namespace nlh {

__global__ void k_selftest_wait_nothing(int *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const uint32_t addr = smem_addr(&bar);
    for (int i = 0; i < kMbarSpinLimit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(addr)
            : "memory");
        if (ok) return;  // cannot happen: nothing arrives on the barrier
    }
    if (err) atomicExch(err, (int)NLH_ERR_TIMEOUT);
}

}  // namespace nlh

using namespace nlh;

extern "C" nlh_status nlh_selftest_plan_timeout(nlh_plan plan, void *stream) {
    clear_error();
    try {
        NLH_REQUIRE(plan, "nlh_selftest_plan_timeout: NULL plan");
        k_selftest_wait_nothing<<<1, 32, 0, (cudaStream_t)stream>>>(plan->err);
        NLH_CHECK_LAUNCH();
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}
