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

// ---------------------------------------------------------------------------
// Write-pattern reference (a measurement aid, not part of the method): the
// stores of the window emission without its filter.  Segment s holds pairs
// [off[s], off[s+1]) of the output; one warp writes a segment in steps of 32
// consecutive 8-byte pairs (streaming stores), and warps take segments either
// in id order (concurrent segments adjacent in memory) or in a scattered order
// s = g * step mod nseg (step coprime to nseg), which is how the emission meets
// them: its windows hold subscriptions of unrelated ids.  The bandwidth this
// reaches is the ceiling of the emission's write pattern on the device.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t wp_hash(uint32_t x) {  // integer mix (xorshift-multiply)
    x ^= x >> 16; x *= 0x7feb352du; x ^= x >> 15; x *= 0x846ca68bu; x ^= x >> 16;
    return x;
}

// Segment lengths: mean_len/2 + hash(s) mod (mean_len + 1), mean about mean_len.
__global__ void k_wp_lengths(uint32_t* len, uint32_t nseg, uint32_t mean_len, uint32_t seed) {
    pdl_begin();
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg;
         s += gridDim.x * blockDim.x)
        len[s] = mean_len / 2 + wp_hash(s ^ seed) % (mean_len + 1);
}

__global__ void __launch_bounds__(256) k_wp_write(int2* out, const unsigned long long* off,
                                                  uint32_t nseg, uint32_t step) {
    pdl_begin();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t g = gw; g < nseg; g += nw) {
        const uint32_t s = step ? (uint32_t)(((uint64_t)g * step) % nseg) : g;
        const unsigned long long a = off[s], b = off[s + 1];
        for (unsigned long long k = a + lane; k < b; k += 32)
            __stcs(&out[k], make_int2((int)s, (int)(k - a)));
    }
}

int launch_wp_lengths(uint32_t* len, uint32_t nseg, uint32_t mean_len, uint32_t seed,
                      cudaStream_t s) {
    launch_k(k_wp_lengths, 152 * 4, 256, 0, s, len, nseg, mean_len, seed);
    return 1;
}

int launch_wp_write(int2* out, const unsigned long long* off, uint32_t nseg, uint32_t step,
                    cudaStream_t s) {
    launch_k(k_wp_write, 152 * 16, 256, 0, s, out, off, nseg, step);
    return 1;
}

}  // namespace ddm
