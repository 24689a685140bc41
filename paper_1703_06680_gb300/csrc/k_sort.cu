// a1: endpoint key build.
// a2: LSD radix sort, 8-bit digits, per pass: tile digit histograms (upsweep),
//     the (digit, tile) output bases -- for up to 1024 tiles computed inside
//     the downsweep from group sums, else by one flat exclusive scan of the
//     digit-major table with decoupled look-back (k_offsets) -- and a
//     downsweep that ranks keys stably with warp ballots and scatters runs of
//     equal digits coalesced.
//
// Paper: Algorithm 4 ("Insert x.lower and x.upper in T"; "Sort T in
// non-decreasing order"), parallel sort phase of Section 4 (Asymptotic
// Analysis, phase 1).  The paper uses a comparison-based parallel sort; on the
// GPU an LSD radix sort on order-preserving integer keys is the natural
// replacement.  Stability of the LSD passes keeps the [lowers | uppers]
// layout order among equal coordinates.
#include <atomic>

#include "sort.cuh"
#include "sweep.cuh"

namespace ddm {

// ---------------------------------------------------------------------------
// a1: key build
// ---------------------------------------------------------------------------
constexpr int KB_BLOCK = 256;

// Four consecutive regions of one set per thread: 16-byte loads and stores
// where the quad is whole and the arrays line up, scalar accesses otherwise
// (the ragged end of each set, caller arrays or output offsets that are not
// 16-byte aligned).
__device__ __forceinline__ void st_u32x4(uint32_t* p, const uint32_t (&v)[4]) {
    *reinterpret_cast<uint4*>(p) = make_uint4(v[0], v[1], v[2], v[3]);
}

__global__ void __launch_bounds__(KB_BLOCK)
k_keybuild_d0(const float* __restrict__ sub_lo, const float* __restrict__ sub_hi,
              const float* __restrict__ upd_lo, const float* __restrict__ upd_hi, int64_t n,
              int64_t m, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, DevStatus* st) {
    pdl_begin();
    const int64_t R = n + m;
    const int64_t qs = (n + 3) >> 2, qall = qs + ((m + 3) >> 2);  // quads of subs, then of updates
    bool bad = false;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < qall;
         q += (int64_t)gridDim.x * blockDim.x) {
        const bool upd = q >= qs;
        const int64_t id0 = (upd ? q - qs : q) << 2;
        const int64_t left = (upd ? m : n) - id0;
        const int c = left < 4 ? (int)left : 4;
        const float* plo = (upd ? upd_lo : sub_lo) + id0;
        const float* phi = (upd ? upd_hi : sub_hi) + id0;
        float lo[4], hi[4];
        const uintptr_t in_bits = reinterpret_cast<uintptr_t>(plo) | reinterpret_cast<uintptr_t>(phi);
        if (c == 4 && (in_bits & 15u) == 0) {
            const float4 a = *reinterpret_cast<const float4*>(plo);
            const float4 b = *reinterpret_cast<const float4*>(phi);
            lo[0] = a.x; lo[1] = a.y; lo[2] = a.z; lo[3] = a.w;
            hi[0] = b.x; hi[1] = b.y; hi[2] = b.z; hi[3] = b.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                lo[k] = k < c ? plo[k] : 0.f;
                hi[k] = k < c ? phi[k] : 0.f;
            }
        }
        uint32_t kl[4], kh[4], vl[4], vh[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (k < c) bad |= is_nan_bits(lo[k]) || is_nan_bits(hi[k]) || !(lo[k] <= hi[k]);
            kl[k] = float_key(lo[k]);
            kh[k] = float_key(hi[k]);
            vl[k] = payload(upd ? KIND_ULO : KIND_SLO, (uint32_t)(id0 + k));
            vh[k] = payload(upd ? KIND_UHI : KIND_SHI, (uint32_t)(id0 + k));
        }
        const int64_t r = (upd ? n : 0) + id0;  // layout [S lo | U lo | S hi | U hi]
        if (c == 4 && ((r | R) & 3) == 0) {     // keys and vals start 256-byte aligned
            st_u32x4(keys + r, kl);
            st_u32x4(keys + R + r, kh);
            st_u32x4(vals + r, vl);
            st_u32x4(vals + R + r, vh);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (k < c) {
                    keys[r + k] = kl[k];
                    keys[R + r + k] = kh[k];
                    vals[r + k] = vl[k];
                    vals[R + r + k] = vh[k];
                }
            }
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) raise_error(st, DDM_ERR_INVALID, 1);
}

int launch_keybuild_d0(const float* sub_lo, const float* sub_hi, const float* upd_lo,
                       const float* upd_hi, int64_t n, int64_t m, uint32_t* keys, uint32_t* vals,
                       DevStatus* st, cudaStream_t s) {
    const int64_t R = n + m;
    if (R == 0) return 0;
    const uint64_t quads = (uint64_t)((n + 3) >> 2) + (uint64_t)((m + 3) >> 2);
    int grid = (int)ceil_div(quads, (uint64_t)KB_BLOCK);
    grid = grid < 1 ? 1 : (grid > 152 * 16 ? 152 * 16 : grid);
    launch_k(k_keybuild_d0, grid, KB_BLOCK, 0, s, sub_lo, sub_hi, upd_lo, upd_hi, n, m, keys, vals, st);
    return 1;
}

// ---------------------------------------------------------------------------
// a2: one pass per digit (upsweep histogram, downsweep ranking and scatter)
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

// Upsweep: digit histogram of one tile.  Flat-scan mode (grp == NULL): stored
// digit-major (tile_hist[d * tiles + tile]) so that one flat exclusive scan
// yields every (digit, tile) output base: all smaller digits first, then
// earlier tiles.  Fused mode: stored tile-major (tile_hist[tile * 256 + d])
// and added into the sums of the tile's group (grp[group * 256 + d]).
// A full tile arrives in shared memory by one TMA bulk copy.
template <typename KeyT, int ITEMS>
__global__ void __launch_bounds__(SORT_BLOCK)
k_upsweep(const KeyT* __restrict__ keys, uint32_t E, int shift, uint32_t* __restrict__ tile_hist,
          uint32_t tiles, uint32_t* __restrict__ grp, DevStatus* st) {
    pdl_begin();
    constexpr int TILE = SORT_BLOCK * ITEMS;
    __shared__ alignas(128) KeyT sk[TILE];
    __shared__ uint32_t h[RADIX];
    __shared__ alignas(8) uint64_t bar;
    const int tid = threadIdx.x;
    const uint32_t tile = blockIdx.x;
    const uint64_t base = (uint64_t)tile * TILE;
    const bool full = base + TILE <= E;
    h[tid] = 0;
    if (tid == 0 && full) mbar_init(&bar, 1);
    __syncthreads();
    if (full) {
        if (tid == 0) {
            mbar_expect_tx(&bar, TILE * sizeof(KeyT));
            tma_load_1d(sk, keys + base, TILE * sizeof(KeyT), &bar);
        }
        mbar_wait_bounded(&bar, 0, st, 13);
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) atomicAdd(&h[digit_of(sk[i * SORT_BLOCK + tid], shift)], 1u);
    } else {
        for (int i = 0; i < ITEMS; ++i) {
            const uint64_t e = base + i * SORT_BLOCK + tid;
            if (e < E) atomicAdd(&h[digit_of(keys[e], shift)], 1u);
        }
    }
    __syncthreads();
    if (grp) {
        tile_hist[(uint64_t)tile * RADIX + tid] = h[tid];
        if (h[tid]) atomicAdd(&grp[(tile >> SORT_GROUP_SHIFT) * RADIX + tid], h[tid]);
    } else {
        tile_hist[(uint64_t)tid * tiles + tile] = h[tid];
    }
}

// Shared memory of one downsweep tile (dynamic, > 48 KB).
template <typename KeyT, int ITEMS>
struct DownSmem {
    static constexpr int TILE = SORT_BLOCK * ITEMS;
    KeyT keys[TILE];                          // raw tile, then keys in digit-major order
    uint32_t vals_raw[TILE];                  // raw tile values
    struct {
        uint32_t vals[TILE];                  // values in digit-major order (after ranking)
    } u;
    uint32_t whist[SORT_BLOCK / 32][RADIX];   // per-warp digit counters
    uint32_t tile_start[RADIX];               // exclusive scan of tile counts over digits
    uint32_t gbase[RADIX];                    // global output base of each digit
    uint32_t warp_tmp[16];
    uint64_t bar;
};

// Adds one endpoint of the sorted output to the kind counters of its scan tile
// (see launch_radix_sort): lanes with the same (tile, kind) are counted by one
// atomic of their lowest lane.  Called by all lanes of the warp.
__device__ __forceinline__ void count_kind(uint32_t* kinds, uint32_t pos, uint32_t E, uint32_t v,
                                           int lane) {
    static_assert((SCAN_TILE & (SCAN_TILE - 1)) == 0, "scan tiles are a power of two");
    const uint32_t kind = v >> 30;
    const bool use = pos < E && kind != KIND_UHI;
    const uint32_t key = use ? ((pos / SCAN_TILE) << 2 | kind) : 0xffffffffu;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (use && lane == __ffs(peers) - 1) atomicAdd(&kinds[key], (uint32_t)__popc(peers));
}

// Downsweep: the tile arrives by TMA bulk copies (keys and values); stable
// rank of every key inside the tile (per-warp peer masks, warp-ordered
// prefix); exchange through shared memory into digit-major order; runs of
// equal digits are written to consecutive output positions starting at the
// scanned (digit, tile) base.
template <typename KeyT, int ITEMS>
__global__ void __launch_bounds__(SORT_BLOCK, 3)
k_downsweep(const KeyT* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
            KeyT* __restrict__ keys_out, uint32_t* __restrict__ vals_out, uint32_t E, int shift,
            const unsigned long long* __restrict__ base, const uint32_t* __restrict__ tile_hist,
            const uint32_t* __restrict__ grp, uint32_t tiles, int write_keys,
            uint4* __restrict__ clr, uint64_t clr_words, uint32_t* __restrict__ kinds,
            DevStatus* st) {
    pdl_begin();
    using Smem = DownSmem<KeyT, ITEMS>;
    constexpr int TILE = Smem::TILE;
    constexpr int WARPS = SORT_BLOCK / 32;
    extern __shared__ __align__(128) unsigned char dsm[];
    Smem& sm = *reinterpret_cast<Smem*>(dsm);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t tile = blockIdx.x;
    const uint64_t tbase = (uint64_t)tile * TILE;
    const bool full = tbase + TILE <= E;
    if (tid == 0 && full) {  // the tile is in flight while the digit offsets are formed
        mbar_init(&sm.bar, 1);
        mbar_expect_tx(&sm.bar, TILE * (sizeof(KeyT) + (vals_in ? sizeof(uint32_t) : 0)));
        tma_load_1d(sm.keys, keys_in + tbase, TILE * sizeof(KeyT), &sm.bar);
        if (vals_in) tma_load_1d(sm.vals_raw, vals_in + tbase, TILE * sizeof(uint32_t), &sm.bar);
    }
    for (int t = tid; t < WARPS * RADIX; t += SORT_BLOCK) (&sm.whist[0][0])[t] = 0;
    if (grp) {  // fused offsets (thread = digit)
        const uint32_t g = tile >> SORT_GROUP_SHIFT;
        const uint32_t ngroups = (tiles + (1u << SORT_GROUP_SHIFT) - 1) >> SORT_GROUP_SHIFT;
        // Every load is issued before the first sum (predicated, fixed counts),
        // so the bases cost about two L2 round trips rather than one per batch.
        constexpr int MAXG = (int)(SORT_FUSED_MAX_TILES >> SORT_GROUP_SHIFT);
        constexpr int GT = 1 << SORT_GROUP_SHIFT;
        uint32_t gv[MAXG], tv[GT - 1];
#pragma unroll
        for (int q = 0; q < MAXG; ++q) gv[q] = (uint32_t)q < ngroups ? grp[q * RADIX + tid] : 0u;
        const uint32_t t0 = g << SORT_GROUP_SHIFT;
#pragma unroll
        for (int k = 0; k < GT - 1; ++k)
            tv[k] = t0 + k < tile ? tile_hist[(uint64_t)(t0 + k) * RADIX + tid] : 0u;
        uint32_t total = 0, before = 0;
#pragma unroll
        for (int q = 0; q < MAXG; ++q) {
            total += gv[q];
            before += (uint32_t)q < g ? gv[q] : 0u;
        }
#pragma unroll
        for (int k = 0; k < GT - 1; ++k) before += tv[k];
        sm.gbase[tid] = block_excl_scan_256(total, sm.warp_tmp) + before;
    } else {
        sm.gbase[tid] = (uint32_t)base[(uint64_t)tid * tiles + tile];
    }
    __syncthreads();
    if (clr) {  // this block's share of a zero fill, while the tile is in flight
        const uint64_t share = (clr_words + gridDim.x - 1) / gridDim.x;
        const uint64_t c0 = (uint64_t)blockIdx.x * share;
        const uint64_t c1 = c0 + share < clr_words ? c0 + share : clr_words;
        for (uint64_t i = c0 + tid; i < c1; i += SORT_BLOCK) clr[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (full) {
        mbar_wait_bounded(&sm.bar, 0, st, 14);
    } else {
        for (int i = tid; i < TILE; i += SORT_BLOCK) {
            const uint64_t e = tbase + i;
            sm.keys[i] = e < E ? keys_in[e] : ~(KeyT)0;  // tail: all-ones key, digit 255, last
            sm.vals_raw[i] = e < E && vals_in ? vals_in[e] : 0u;
        }
        __syncthreads();
    }

    // Warp-striped view: warp w owns 32*ITEMS consecutive keys of the tile.
    KeyT key[ITEMS];
    uint32_t dig[ITEMS], rank[ITEMS];
    const int wofs = warp * (32 * ITEMS);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        key[i] = sm.keys[wofs + i * 32 + lane];
        dig[i] = digit_of(key[i], shift);
    }
    // Stable ranking inside the warp, items in (i, lane) order: the lanes
    // holding the same digit find each other with one ballot per digit bit
    // (no shared-memory round trip); the lowest such lane advances the warp's
    // counter for that digit.
    const unsigned lt = (1u << lane) - 1u;
    uint32_t* wh = sm.whist[warp];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        unsigned peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < RADIX_BITS; ++b) {
            const bool bit = (dig[i] >> b) & 1u;
            const unsigned m = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? m : ~m;
        }
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
    {   // per digit (thread = digit): exclusive prefix over warps; digit start in the tile
        const int b = tid;
        uint32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) {
            const uint32_t c = sm.whist[w][b];
            sm.whist[w][b] = cnt;
            cnt += c;
        }
        sm.tile_start[b] = block_excl_scan_256(cnt, sm.warp_tmp);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t slot = sm.tile_start[dig[i]] + sm.whist[warp][dig[i]] + rank[i];
        sm.keys[slot] = key[i];
        if (vals_in) sm.u.vals[slot] = sm.vals_raw[wofs + i * 32 + lane];
    }
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
            if (vals_out) vals_out[pos] = sm.u.vals[s];
        }
        if (kinds) count_kind(kinds, pos, E, sm.u.vals[s], lane);
    }
}

template <typename KeyT, int ITEMS>
static int radix_sort_items(KeyT* keys0, uint32_t* vals0, KeyT* keys1, uint32_t* vals1,
                            uint64_t E, int passes, const SortScratch& sc, bool skip_last_keys,
                            DevStatus* st, cudaStream_t s, void* clear_ptr,
                            uint64_t clear_words, uint32_t* kinds) {
    const uint64_t tiles = ceil_div(E, (uint64_t)SORT_BLOCK * ITEMS);
    KeyT* kb[2] = {keys0, keys1};
    uint32_t* vb[2] = {vals0, vals1};
    const uint64_t cells = tiles * RADIX;
    const int smem = (int)sizeof(DownSmem<KeyT, ITEMS>);
    // The dynamic shared-memory opt-in is per device; set it once for each.
    static std::atomic<unsigned long long> attr_set{0};  // server threads launch concurrently
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !(attr_set.load() & (1ull << dev))) {
        cudaFuncSetAttribute(k_downsweep<KeyT, ITEMS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
        if (dev >= 0 && dev < 64) attr_set.fetch_or(1ull << dev);
    }
    const bool fused = sc.grp && tiles <= SORT_FUSED_MAX_TILES;
    int launches = 0;
    for (int p = 0; p < passes; ++p) {
        const int write_keys = !(skip_last_keys && p == passes - 1);
        uint32_t* grp = fused ? sc.grp + (size_t)p * sort_groups(tiles) * RADIX : nullptr;
        launch_k(k_upsweep<KeyT, ITEMS>, (unsigned)tiles, SORT_BLOCK, 0, s, kb[p & 1], (uint32_t)E,
                 8 * p, sc.tile_hist, (uint32_t)tiles, grp, st);
        ++launches;
        if (!fused)
            launches += launch_offsets(sc.tile_hist, (int64_t)cells, sc.offs, ~0ull, sc.total,
                                       sc.status + (size_t)p * sort_status_stride(E), st, s);
        const bool last = p == passes - 1;
        launch_k(k_downsweep<KeyT, ITEMS>, (unsigned)tiles, SORT_BLOCK, smem, s, kb[p & 1],
                 vb[p & 1], kb[(p + 1) & 1], vb[(p + 1) & 1], (uint32_t)E, 8 * p, sc.offs,
                 sc.tile_hist, grp, (uint32_t)tiles, write_keys,
                 last ? static_cast<uint4*>(clear_ptr) : static_cast<uint4*>(nullptr),
                 last ? clear_words : 0ull, last && vals0 ? kinds : nullptr, st);
        ++launches;
    }
    return launches;
}

template <typename KeyT>
int launch_radix_sort(KeyT* keys0, uint32_t* vals0, KeyT* keys1, uint32_t* vals1, uint64_t E,
                      int passes, const SortScratch& sc, bool skip_last_keys, DevStatus* st,
                      cudaStream_t s, void* clear_ptr, uint64_t clear_words, int items,
                      uint32_t* kinds) {
    if (E == 0) return 0;
    if (sizeof(KeyT) == 8 || items == 0) items = sort_items<KeyT>();
    switch (items) {  // the tile sizes a context may choose (DDM_PARAM_SORT_ITEMS)
        case 12:
            return radix_sort_items<KeyT, 12>(keys0, vals0, keys1, vals1, E, passes, sc,
                                              skip_last_keys, st, s, clear_ptr, clear_words, kinds);
        case 16:
            return radix_sort_items<KeyT, 16>(keys0, vals0, keys1, vals1, E, passes, sc,
                                              skip_last_keys, st, s, clear_ptr, clear_words, kinds);
        default:
            return radix_sort_items<KeyT, SORT_ITEMS_32>(keys0, vals0, keys1, vals1, E, passes,
                                                         sc, skip_last_keys, st, s, clear_ptr,
                                                         clear_words, kinds);
    }
}

template int launch_radix_sort<uint32_t>(uint32_t*, uint32_t*, uint32_t*, uint32_t*, uint64_t,
                                         int, const SortScratch&, bool, DevStatus*, cudaStream_t,
                                         void*, uint64_t, int, uint32_t*);
template int launch_radix_sort<unsigned long long>(unsigned long long*, uint32_t*,
                                                   unsigned long long*, uint32_t*, uint64_t, int,
                                                   const SortScratch&, bool, DevStatus*,
                                                   cudaStream_t, void*, uint64_t, int, uint32_t*);

}  // namespace ddm
