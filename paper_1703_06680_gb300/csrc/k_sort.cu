// a1: endpoint key build with fused digit histograms.
// a2: onesweep LSD radix sort (one kernel per 8-bit digit place, single pass
//     over the data per digit, decoupled look-back on per-digit tile counts,
//     warp-level ranking with __match_any_sync).
//
// Paper: Algorithm 4 ("Insert x.lower and x.upper in T"; "Sort T in
// non-decreasing order"), parallel sort phase of Section 4 (Asymptotic
// Analysis, phase 1).  The paper uses a comparison-based parallel sort; on the
// GPU an LSD radix sort on order-preserving integer keys is the natural
// replacement.  Stability of the LSD passes keeps the [lowers | uppers]
// layout order among equal coordinates.
#include "sort.cuh"

namespace ddm {

// ---------------------------------------------------------------------------
// a1: key build
// ---------------------------------------------------------------------------
constexpr int KB_BLOCK = 256;

__global__ void __launch_bounds__(KB_BLOCK)
k_keybuild_d0(const float* __restrict__ sub_lo, const float* __restrict__ sub_hi,
              const float* __restrict__ upd_lo, const float* __restrict__ upd_hi, int64_t n,
              int64_t m, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
              uint32_t* __restrict__ hist, DevStatus* st) {
    __shared__ uint32_t sh[4][RADIX];
    for (int t = threadIdx.x; t < 4 * RADIX; t += blockDim.x) (&sh[0][0])[t] = 0;
    __syncthreads();
    const int64_t R = n + m;
    bool bad = false;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R;
         r += (int64_t)gridDim.x * blockDim.x) {
        const bool upd = r >= n;
        const int64_t id = upd ? r - n : r;
        const float lo = upd ? upd_lo[id] : sub_lo[id];
        const float hi = upd ? upd_hi[id] : sub_hi[id];
        bad |= is_nan_bits(lo) || is_nan_bits(hi) || !(lo <= hi);
        const uint32_t klo = float_key(lo), khi = float_key(hi);
        keys[r] = klo;
        keys[R + r] = khi;
        vals[r] = payload(upd ? KIND_ULO : KIND_SLO, (uint32_t)id);
        vals[R + r] = payload(upd ? KIND_UHI : KIND_SHI, (uint32_t)id);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            atomicAdd(&sh[p][(klo >> (8 * p)) & 0xFF], 1u);
            atomicAdd(&sh[p][(khi >> (8 * p)) & 0xFF], 1u);
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) raise_error(st, DDM_ERR_INVALID, 1);
    for (int t = threadIdx.x; t < 4 * RADIX; t += blockDim.x) {
        uint32_t c = (&sh[0][0])[t];
        if (c) atomicAdd(&hist[t], c);
    }
}

int launch_keybuild_d0(const float* sub_lo, const float* sub_hi, const float* upd_lo,
                        const float* upd_hi, int64_t n, int64_t m, uint32_t* keys,
                        uint32_t* vals, uint32_t* hist, DevStatus* st, cudaStream_t s) {
    const int64_t R = n + m;
    if (R == 0) return 0;
    int grid = (int)ceil_div((uint64_t)R, (uint64_t)KB_BLOCK * 8);
    grid = grid < 1 ? 1 : (grid > 152 * 16 ? 152 * 16 : grid);
    k_keybuild_d0<<<grid, KB_BLOCK, 0, s>>>(sub_lo, sub_hi, upd_lo, upd_hi, n, m, keys, vals,
                                             hist, st);
    return 1;
}

// ---------------------------------------------------------------------------
// a2: onesweep pass
// ---------------------------------------------------------------------------

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ uint32_t block_excl_scan_256(uint32_t v, uint32_t* warp_tmp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < 8 ? warp_tmp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < 8) warp_tmp[8 + lane] = t;  // inclusive warp totals
    }
    __syncthreads();
    uint32_t before = warp == 0 ? 0u : warp_tmp[8 + warp - 1];
    return before + x - v;
}

template <typename KeyT>
__device__ __forceinline__ uint32_t digit_of(KeyT k, int shift) {
    return (uint32_t)(k >> shift) & (RADIX - 1);
}

template <typename KeyT, int ITEMS>
struct SortSmem {
    static constexpr int TILE = SORT_BLOCK * ITEMS;
    union {
        KeyT keys[TILE];
        uint32_t vals[TILE];
    } x;
    uint32_t whist[SORT_BLOCK / 32][RADIX];  // per-warp digit counters
    uint32_t tile_start[RADIX];              // exclusive scan of tile counts over digits
    uint32_t gbase[RADIX];                   // global output base of each digit
    uint32_t warp_tmp[16];
    uint32_t tile_id;
};

template <typename KeyT, int ITEMS>
__global__ void __launch_bounds__(SORT_BLOCK)
k_onesweep(const KeyT* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
           KeyT* __restrict__ keys_out, uint32_t* __restrict__ vals_out, uint32_t E, int shift,
           const uint32_t* __restrict__ hist_pass, uint32_t* __restrict__ lookback,
           uint32_t* __restrict__ tile_counter, int write_keys, DevStatus* st) {
    using Smem = SortSmem<KeyT, ITEMS>;
    constexpr int TILE = Smem::TILE;
    constexpr int WARPS = SORT_BLOCK / 32;
    __shared__ Smem sm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (tid == 0) sm.tile_id = atomicAdd(tile_counter, 1u);
    for (int t = tid; t < WARPS * RADIX; t += SORT_BLOCK) (&sm.whist[0][0])[t] = 0;
    __syncthreads();
    const uint32_t tile = sm.tile_id;
    const uint64_t tile_base = (uint64_t)tile * TILE;

    // Warp-striped load: warp w owns TILE/WARPS consecutive keys of the tile.
    KeyT key[ITEMS];
    uint32_t dig[ITEMS], rank[ITEMS];
    const uint64_t wbase = tile_base + (uint64_t)warp * (32 * ITEMS);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint64_t e = wbase + (uint64_t)i * 32 + lane;
        key[i] = e < E ? keys_in[e] : ~(KeyT)0;  // tail: all-ones key, digit 255, last in order
        dig[i] = digit_of(key[i], shift);
    }

    // Stable ranking inside the warp: items in (i, lane) order.
    const unsigned lt = (1u << lane) - 1u;
    uint32_t* wh = sm.whist[warp];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const unsigned peers = __match_any_sync(0xffffffffu, dig[i]);
        const int leader = __ffs(peers) - 1;
        const uint32_t c = wh[dig[i]];
        __syncwarp();
        if (lane == leader) wh[dig[i]] = c + __popc(peers);
        __syncwarp();
        rank[i] = c + __popc(peers & lt);
    }
    __syncthreads();

    // Per digit (thread = digit): tile count and exclusive prefix over warps.
    const int b = tid;
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
        uint32_t c = sm.whist[w][b];
        sm.whist[w][b] = cnt;
        cnt += c;
    }
    // Publish the tile count, then look back for the prefix of earlier tiles.
    uint32_t* my_lb = lookback + (uint64_t)tile * RADIX + b;
    if (tile == 0) {
        st_release_u32(my_lb, LB32_INC | cnt);
    } else {
        st_release_u32(my_lb, LB32_AGG | cnt);
    }
    uint32_t prefix = 0;
    for (int64_t p = (int64_t)tile - 1; p >= 0; --p) {
        const uint32_t* q = lookback + (uint64_t)p * RADIX + b;
        uint32_t v;
        uint32_t it = 0;
        while (((v = ld_acquire_u32(q)) >> 30) == 0u) {
            if (++it > SPIN_LIMIT) {
                raise_error(st, DDM_ERR_DEVICE_TIMEOUT, 2);
                v = LB32_INC;
                break;
            }
            backoff(it);
        }
        prefix += v & LB32_VAL;
        if ((v >> 30) == 2u) break;
    }
    if (tile != 0) st_release_u32(my_lb, LB32_INC | (prefix + cnt));

    // Global base per digit: exclusive scan of the global histogram + prefix.
    const uint32_t gexcl = block_excl_scan_256(hist_pass[b], sm.warp_tmp);
    sm.gbase[b] = gexcl + prefix;
    const uint32_t tstart = block_excl_scan_256(cnt, sm.warp_tmp + 0);
    sm.tile_start[b] = tstart;
    __syncthreads();

    // Exchange through shared memory into digit-major order, then write out
    // runs of equal digits to consecutive global positions (coalesced).
    uint32_t slot[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        slot[i] = sm.tile_start[dig[i]] + sm.whist[warp][dig[i]] + rank[i];
        sm.x.keys[slot[i]] = key[i];
    }
    __syncthreads();
    uint32_t opos[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int s = tid + i * SORT_BLOCK;
        const KeyT k = sm.x.keys[s];
        const uint32_t d = digit_of(k, shift);
        opos[i] = sm.gbase[d] + (uint32_t)(s - sm.tile_start[d]);
        if (write_keys && opos[i] < E) keys_out[opos[i]] = k;
    }
    __syncthreads();
    // Values follow the same permutation.
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        uint64_t e = wbase + (uint64_t)i * 32 + lane;
        sm.x.vals[slot[i]] = e < E ? vals_in[e] : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int s = tid + i * SORT_BLOCK;
        if (opos[i] < E) vals_out[opos[i]] = sm.x.vals[s];
    }
}

template <typename KeyT>
int launch_radix_sort(KeyT* keys0, uint32_t* vals0, KeyT* keys1, uint32_t* vals1, uint64_t E,
                       int passes, const uint32_t* hist, uint32_t* lookback, bool skip_last_keys,
                       DevStatus* st, cudaStream_t s) {
    if (E == 0) return 0;
    constexpr int ITEMS = sort_items<KeyT>();
    constexpr int TILE = sort_tile<KeyT>();
    const uint64_t tiles = ceil_div(E, TILE);
    KeyT* kb[2] = {keys0, keys1};
    uint32_t* vb[2] = {vals0, vals1};
    for (int p = 0; p < passes; ++p) {
        uint32_t* lb = lookback + (size_t)p * (tiles * RADIX + 32);
        uint32_t* counter = lb + tiles * RADIX;
        const int write_keys = !(skip_last_keys && p == passes - 1);
        k_onesweep<KeyT, ITEMS><<<(unsigned)tiles, SORT_BLOCK, 0, s>>>(
            kb[p & 1], vb[p & 1], kb[(p + 1) & 1], vb[(p + 1) & 1], (uint32_t)E, 8 * p,
            hist + (size_t)p * RADIX, lb, counter, write_keys, st);
    }
    return passes;
}

template int launch_radix_sort<uint32_t>(uint32_t*, uint32_t*, uint32_t*, uint32_t*, uint64_t,
                                          int, const uint32_t*, uint32_t*, bool, DevStatus*,
                                          cudaStream_t);
template int launch_radix_sort<unsigned long long>(unsigned long long*, uint32_t*,
                                                    unsigned long long*, uint32_t*, uint64_t, int,
                                                    const uint32_t*, uint32_t*, bool,
                                                    DevStatus*, cudaStream_t);

}  // namespace ddm
