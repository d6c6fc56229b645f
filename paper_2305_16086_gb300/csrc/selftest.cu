// Self-test of the bounded device waits (no fault, no hang): a wait on an
// mbarrier phase that never completes and a spin on a device flag that is
// never set, each limited in time, must give up and report through a status
// word, leaving the CUDA context usable. The mbarrier wait is the helper the
// TMA hop kernel uses for its staged row gathers.
#include "hop_tma.cuh"

namespace sc {

__global__ void k_selftest_waits(const volatile int32_t *flag, uint64_t limit_ns, int32_t *status) {
    __shared__ alignas(8) uint64_t bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    // phase 0 never completes: nothing arrives on the barrier
    status[0] = mbar_wait_bounded(smem_u32(&bar), 0u, limit_ns) ? 0 : 1;
    // a flag that nothing sets
    const uint64_t t0 = global_ns();
    int32_t expired = 0;
    while (*flag == 0) {
        if (global_ns() - t0 > limit_ns) {
            expired = 1;
            break;
        }
    }
    status[1] = expired;
}

}  // namespace sc

extern "C" sc_status sc_selftest_bounded_waits(uint32_t limit_us) {
    int32_t h_status[2] = {0, 0};
    const sc_status st = sc::guarded([&] {
        if (limit_us < 1 || limit_us > 1000000u) SC_FAIL(SC_ERR_INVALID_ARG, "limit_us %u not in [1, 1e6]", limit_us);
        sc::DevBuf<int32_t> buf;
        buf.reserve(4);
        SC_CUDA(cudaMemset(buf.get(), 0, 4 * sizeof(int32_t)));  // flag = 0, status = 0
        sc::k_selftest_waits<<<1, 32>>>(buf.get(), static_cast<uint64_t>(limit_us) * 1000ull, buf.get() + 1);
        SC_LAUNCH_CHECK();
        SC_CUDA(cudaMemcpy(h_status, buf.get() + 1, sizeof(h_status), cudaMemcpyDeviceToHost));
    });
    if (st != SC_OK) return st;
    if (h_status[0] == 1 && h_status[1] == 1) {
        sc::set_detail("both bounded waits gave up after %u us, as designed", limit_us);
        return SC_ERR_TIMEOUT;
    }
    sc::set_detail("a bounded wait did not report its expiry (mbarrier %d, flag %d)", h_status[0], h_status[1]);
    return SC_ERR_CUDA;
}
