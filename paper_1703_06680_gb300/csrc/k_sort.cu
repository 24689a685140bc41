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


// Warp-parallel look-back over the per-digit tile counts.  Warp w resolves
// digits 32w .. 32w+31 together: in one step lane l reads the 32 words of
// predecessor tile p - l (eight 16-byte loads), and for every digit the warp
// sums the published values back to the nearest inclusive prefix.  A step
// thus covers 32 predecessor tiles, so even when every tile of the sort runs
// in the same wave the chain of L2 round trips stays short.  Returns the
// exclusive prefix of digit 32w + lane.  Each word carries its own flag, so
// plain volatile loads suffice.  Waits are bounded (SPIN_LIMIT).
__device__ __forceinline__ uint32_t warp_lookback_digits(const uint32_t* lookback, uint32_t tile,
                                                         int warp, int lane, DevStatus* st) {
    uint32_t my_prefix = 0;
    if (tile == 0) return 0;
    uint32_t done = 0;  // bit dd: digit 32w+dd found its inclusive prefix
    int64_t p = (int64_t)tile - 1;
    uint32_t it = 0;
    while (done != 0xffffffffu) {
        const int64_t q = p - lane;
        uint32_t v[32];
        if (q >= 0) {
            const uint4* src = reinterpret_cast<const uint4*>(lookback + (uint64_t)q * RADIX + 32 * warp);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint4 x = __ldcv(src + k);
                v[4 * k] = x.x; v[4 * k + 1] = x.y; v[4 * k + 2] = x.z; v[4 * k + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 32; ++k) v[k] = LB32_INC;  // before tile 0: prefix 0
        }
        // A window is usable for a digit when every word up to its nearest
        // inclusive prefix is published.
        bool ready = true;
#pragma unroll
        for (int dd = 0; dd < 32; ++dd) {
            if (done & (1u << dd)) continue;
            const unsigned inc = __ballot_sync(0xffffffffu, (v[dd] >> 30) == 2u);
            const unsigned zero = __ballot_sync(0xffffffffu, (v[dd] >> 30) == 0u);
            const unsigned need = inc ? (0xffffffffu >> (31 - (__ffs(inc) - 1))) : 0xffffffffu;
            if (zero & need) ready = false;
        }
        if (!ready) {
            if (++it > SPIN_LIMIT) {
                raise_error(st, DDM_ERR_DEVICE_TIMEOUT, 2);
                return my_prefix;
            }
            backoff(it);
            continue;
        }
#pragma unroll
        for (int dd = 0; dd < 32; ++dd) {
            if (done & (1u << dd)) continue;
            const unsigned inc = __ballot_sync(0xffffffffu, (v[dd] >> 30) == 2u);
            const int stop = inc ? __ffs(inc) - 1 : 31;
            uint32_t x = lane <= stop ? (v[dd] & LB32_VAL) : 0u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == dd) my_prefix += x;
            if (inc) done |= 1u << dd;
        }
        p -= 32;
    }
    return my_prefix;
}

template <typename KeyT, int ITEMS>
struct SortSmem {
    static constexpr int TILE = SORT_BLOCK * ITEMS;
    KeyT keys[TILE];                          // keys staged in digit-major tile order
    uint32_t vals[TILE];                      // values, same order
    uint32_t whist[SORT_BLOCK / 32][RADIX];   // per-warp digit counters
    uint32_t tile_start[RADIX];               // exclusive scan of tile counts over digits
    uint32_t gbase[RADIX];                    // global output base of each digit
    uint32_t warp_tmp[16];
    uint32_t tile_id;
};

// Stable rank of each lane's digit among the lanes of its warp holding the same
// digit: the peer mask is built from one ballot per digit bit (warp multisplit).
__device__ __forceinline__ unsigned digit_peers(uint32_t d) {
    unsigned peers = 0xffffffffu;
#pragma unroll
    for (int bit = 0; bit < RADIX_BITS; ++bit) {
        const unsigned b = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
        peers &= ((d >> bit) & 1u) ? b : ~b;
    }
    return peers;
}

template <typename KeyT, int ITEMS>
__global__ void __launch_bounds__(SORT_BLOCK, 3)
k_onesweep(const KeyT* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
           KeyT* __restrict__ keys_out, uint32_t* __restrict__ vals_out, uint32_t E, int shift,
           const uint32_t* __restrict__ hist_pass, uint32_t* __restrict__ lookback,
           uint32_t* __restrict__ tile_counter, int write_keys, DevStatus* st) {
    using Smem = SortSmem<KeyT, ITEMS>;
    constexpr int WARPS = SORT_BLOCK / 32;
    __shared__ Smem sm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (tid == 0) sm.tile_id = atomicAdd(tile_counter, 1u);
    for (int t = tid; t < WARPS * RADIX; t += SORT_BLOCK) (&sm.whist[0][0])[t] = 0;
    __syncthreads();
    const uint32_t tile = sm.tile_id;
    const uint64_t tile_base = (uint64_t)tile * Smem::TILE;

    // Warp-striped load: warp w owns 32*ITEMS consecutive keys of the tile.
    KeyT key[ITEMS];
    uint32_t dig[ITEMS], rank[ITEMS];
    const uint64_t wbase = tile_base + (uint64_t)warp * (32 * ITEMS);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint64_t e = wbase + (uint64_t)i * 32 + lane;
        key[i] = e < E ? keys_in[e] : ~(KeyT)0;  // tail: all-ones key, digit 255, last in order
        dig[i] = digit_of(key[i], shift);
    }
    // Stable ranking inside the warp: items in (i, lane) order.
    const unsigned lt = (1u << lane) - 1u;
    uint32_t* wh = sm.whist[warp];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const unsigned peers = digit_peers(dig[i]);
        const int leader = __ffs(peers) - 1;
        uint32_t c = 0;
        if (lane == leader) {
            c = wh[dig[i]];
            wh[dig[i]] = c + __popc(peers);
        }
        c = __shfl_sync(0xffffffffu, c, leader);
        rank[i] = c + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();

    // Per digit (thread = digit): tile count, exclusive prefix over warps,
    // digit starts inside the tile and in the global output.
    const int b = tid;
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
        const uint32_t c = sm.whist[w][b];
        sm.whist[w][b] = cnt;
        cnt += c;
    }
    uint32_t* my_lb = lookback + (uint64_t)tile * RADIX + b;
    st_release_u32(my_lb, (tile == 0 ? LB32_INC : LB32_AGG) | cnt);
    const uint32_t gexcl = block_excl_scan_256(hist_pass[b], sm.warp_tmp);
    sm.tile_start[b] = block_excl_scan_256(cnt, sm.warp_tmp);
    __syncthreads();

    // Stage keys and values in digit-major order before the look-back, so the
    // look-back runs with few live registers.
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t slot = sm.tile_start[dig[i]] + sm.whist[warp][dig[i]] + rank[i];
        sm.keys[slot] = key[i];
        const uint64_t e = wbase + (uint64_t)i * 32 + lane;
        sm.vals[slot] = e < E ? vals_in[e] : 0u;
    }
    const uint32_t prefix = warp_lookback_digits(lookback, tile, warp, lane, st);
    if (tile != 0) st_release_u32(my_lb, LB32_INC | (prefix + cnt));
    sm.gbase[b] = gexcl + prefix;
    __syncthreads();

    // Runs of equal digits go to consecutive global positions (coalesced).
#pragma unroll 4
    for (int i = 0; i < ITEMS; ++i) {
        const int s = tid + i * SORT_BLOCK;
        const KeyT k = sm.keys[s];
        const uint32_t d = digit_of(k, shift);
        const uint32_t pos = sm.gbase[d] + (uint32_t)(s - sm.tile_start[d]);
        if (pos < E) {
            if (write_keys) keys_out[pos] = k;
            vals_out[pos] = sm.vals[s];
        }
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
