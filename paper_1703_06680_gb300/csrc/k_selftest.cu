// Self-test of the bounded device-side waits (fault handling).
//
// Every wait of the library's kernels -- the decoupled look-back polls of the
// scans and the mbarrier waits of the TMA bulk copies -- gives up after a
// bounded number of polls, raises DDM_ERR_DEVICE_TIMEOUT in the status word
// and returns, so that a lost hand-off can never hang the GPU.  This kernel
// runs those same wait helpers against a hand-off that never comes, with a
// short limit, so that a test can watch the timeout path work: the kernel
// returns, the host reads DDM_ERR_DEVICE_TIMEOUT, and the context stays usable.
//   which = 0: warp_lookback_u64 for tile 1 over a zeroed status word (tile 0
//              never publishes its aggregate);
//   which = 1: mbar_wait_bounded on an mbarrier whose expected transaction
//              bytes never arrive (no copy is issued, so nothing is in flight
//              when the block leaves).
// The paper has no counterpart: its multicore algorithm has no device waits.
#include "common.cuh"

namespace ddm {

__global__ void k_wait_selftest(int which, uint32_t limit, unsigned long long* status,
                                DevStatus* st) {
    pdl_begin();
    if (which == 0) {
        if (threadIdx.x < 32) (void)warp_lookback_u64(status, 1, st, 90, limit);
        return;
    }
    __shared__ alignas(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, 16);  // one arrival with 16 bytes pending that never land
    }
    __syncthreads();
    (void)mbar_wait_bounded(&bar, 0, st, 91, limit);
}

// status: one zeroed u64 word (device).  Returns the number of launches.
int launch_wait_selftest(int which, uint32_t limit, unsigned long long* status, DevStatus* st,
                         cudaStream_t s) {
    launch_k(k_wait_selftest, 1, 64, 0, s, which, limit, status, st);
    return 1;
}

}  // namespace ddm
