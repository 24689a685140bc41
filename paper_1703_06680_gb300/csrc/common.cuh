// Shared device-side helpers of the SBM library (sm_103a).
#pragma once

#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

#include "ddm.h"

namespace ddm {

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  The kernels of one call run back to back on
// one stream.  Launched with the programmatic-serialization attribute, a
// kernel's blocks may be scheduled while its predecessor is still finishing,
// which hides the launch and ramp-up of every grid behind the tail of the
// previous one.  Memory ordering is unchanged: every kernel begins with
// griddepcontrol.wait, which returns once the predecessor grid has completed
// and its writes are visible (and, transitively, those of all earlier
// kernels), before the kernel touches global memory.  It then lets its own
// dependent be scheduled; that grid is launched only once every block of this
// one has started, so waiting dependents occupy free slots only.  Without the
// attribute both instructions are no-ops.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Host switch for the attribute, set per call by the entry points (PdlScope).
extern thread_local bool g_pdl;

struct PdlScope {
    bool prev;
    explicit PdlScope(bool on) : prev(g_pdl) { g_pdl = on; }
    ~PdlScope() { g_pdl = prev; }
};

// Launches kernel k on stream s, with the programmatic-serialization
// attribute when the calling entry point enabled it.
template <typename... P, typename... A>
inline cudaError_t launch_k(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = g_pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

// ---------------------------------------------------------------------------
// Endpoint payload: (kind << 30) | id, kind 0 = S lower, 1 = U lower,
// 2 = S upper, 3 = U upper.  The key build lays endpoints out in exactly this
// kind order ([S lowers | U lowers | S uppers | U uppers]), so a stable sort
// by coordinate key puts every lower endpoint before every upper endpoint at
// equal coordinates: touching closed intervals are then reported, as
// Algorithm 1 requires.
// ---------------------------------------------------------------------------
constexpr uint32_t KIND_SLO = 0, KIND_ULO = 1, KIND_SHI = 2, KIND_UHI = 3;
constexpr uint32_t ID_MASK = (1u << 30) - 1;

__host__ __device__ __forceinline__ uint32_t payload(uint32_t kind, uint32_t id) {
    return (kind << 30) | id;
}

// Order-preserving map float32 -> uint32: a < b (IEEE) iff key(a) < key(b).
// -0 is first mapped to +0, so the two compare equal as IEEE says.  Negative
// floats have their bits inverted, non-negative ones get the sign bit set.
__device__ __forceinline__ uint32_t float_key(float x) {
    uint32_t u = __float_as_uint(x);
    if (u == 0x80000000u) u = 0u;
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Inverse of float_key (-0 comes back as +0).
__device__ __forceinline__ float key_float(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__device__ __forceinline__ bool is_nan_bits(float x) {
    return (__float_as_uint(x) & 0x7fffffffu) > 0x7f800000u;
}

// ---------------------------------------------------------------------------
// Device status block, one per context.  The first error wins.
// ---------------------------------------------------------------------------
struct DevStatus {
    int error;                 // DDM_OK or a DDM_ERR_* code
    int detail;                // where a timeout or check fired (diagnostics)
    unsigned long long K;      // number of pairs (after the offsets scan)
    unsigned long long aux[6]; // per-call diagnostics / plans
    unsigned long long flagged; // host copy only: subscriptions sent to the range path
};

__device__ __forceinline__ void raise_error(DevStatus* st, int code, int detail) {
    if (atomicCAS(&st->error, 0, code) == 0) st->detail = detail;
}

__device__ __forceinline__ int read_error(const DevStatus* st) {
    return *(volatile const int*)&st->error;
}

// ---------------------------------------------------------------------------
// Acquire / release accesses for single-pass scans with decoupled look-back.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Every device-side wait is bounded: after SPIN_LIMIT polls (with a growing
// nanosleep back-off, well over a second in total) the waiter raises
// DDM_ERR_DEVICE_TIMEOUT and proceeds with a neutral value, so a kernel can
// never hang the GPU; the host then reports the error.  The wait helpers take
// the limit as an argument (SPIN_LIMIT unless given) so that the self-test of
// ddm_debug_wait_timeout can run the same code out in milliseconds.
constexpr uint32_t SPIN_LIMIT = 1u << 21;

__device__ __forceinline__ void backoff(uint32_t iter) {
    __nanosleep(iter < 64 ? 32 : (iter < 4096 ? 256 : 1024));
}

// 64-bit look-back words: [flag:2 | value:62], flag 1 = tile aggregate,
// 2 = inclusive prefix.  A zero word means "not yet published".
constexpr unsigned long long LB64_AGG = 1ull << 62, LB64_INC = 2ull << 62;
constexpr unsigned long long LB64_VAL = (1ull << 62) - 1;

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Warp-cooperative look-back: exclusive prefix of tile `tile` over the values
// published by tiles 0..tile-1 in `status`.  Called by all 32 lanes of one warp.
// Each step examines the 128 nearest unexamined predecessors (four words per
// lane, loaded together) and sums back to the nearest inclusive prefix.  Each
// word carries its own flag and value, so relaxed loads suffice and can be
// pipelined; the publisher's release store makes the word visible whole.
__device__ __forceinline__ unsigned long long warp_lookback_u64(unsigned long long* status,
                                                                long long tile, DevStatus* st,
                                                                int where,
                                                                uint32_t limit = SPIN_LIMIT) {
    const int lane = threadIdx.x & 31;
    unsigned long long sum = 0;
    long long p = tile - 1;
    while (p >= 0) {
        unsigned long long v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long q = p - (j * 32 + lane);
            v[j] = q >= 0 ? ld_relaxed_u64(status + q) : LB64_INC;  // before tile 0: prefix 0
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long q = p - (j * 32 + lane);
            uint32_t it = 0;
            while (v[j] == 0ull) {  // not yet published: wait (bounded)
                if (++it > limit) {
                    raise_error(st, DDM_ERR_DEVICE_TIMEOUT, where);
                    v[j] = LB64_INC;
                    break;
                }
                backoff(it);
                v[j] = ld_relaxed_u64(status + q);
            }
        }
        int first = 128;  // distance index (j * 32 + lane) of the nearest inclusive prefix
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            const unsigned inc = __ballot_sync(0xffffffffu, (v[j] >> 62) == 2ull);
            if (inc) first = j * 32 + __ffs(inc) - 1;
        }
        unsigned long long mine = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j * 32 + lane <= first) mine += v[j] & LB64_VAL;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
        sum += mine;
        if (first < 128) break;
        p -= 128;
    }
    return sum;
}

// ---------------------------------------------------------------------------
// TMA bulk copies (global -> shared) completing on an mbarrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D bulk copy; dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of an mbarrier.  On timeout the error is
// raised and the wait continues (bounded again) so that no copy is still in
// flight into shared memory when the block leaves; returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, DevStatus* st,
                                                  int where, uint32_t limit = SPIN_LIMIT) {
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 16) __nanosleep(64);
    }
    raise_error(st, DDM_ERR_DEVICE_TIMEOUT, where);
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) break;
        __nanosleep(1024);
    }
    return false;
}

// Instance of a global id in a batch: base[b] <= id < base[b + 1], base[0] = 0.
__device__ __forceinline__ int inst_of(const int64_t* base, int num, int64_t id) {
    int lo = 0, hi = num;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (base[mid] <= id) lo = mid; else hi = mid;
    }
    return lo;
}

__host__ __device__ __forceinline__ uint64_t ceil_div(uint64_t a, uint64_t b) {
    return (a + b - 1) / b;
}

}  // namespace ddm
