// a3: sweep scan over the sorted endpoint stream.
// a4: exact per-extent match counts by rank arithmetic.
// a5: exclusive scan of the counts into output offsets.
//
// Paper: Algorithm 4 sweeps the sorted endpoints keeping the active sets
// SubSet and UpdSet (an extent is active between its lower and upper
// endpoint, Section 3 "Sort-Based Matching"); Section 4 computes the state at
// segment boundaries with a prefix computation (inclusive / exclusive scans,
// "Prefix computations") and Algorithm 6.  Here the sweep keeps only the
// SIZES of the active sets, as four running counts (S lowers, U lowers,
// S uppers, U uppers seen so far), computed for every position at once by a
// single-pass scan with decoupled look-back -- the GPU form of the paper's
// master combine of per-segment Sadd/Sdel/Uadd/Udel.
//
// Counting (a4).  With lowers before uppers at equal coordinates, S_i and U_j
// intersect iff pos(U_j.lo) < pos(S_i.hi) and pos(S_i.lo) < pos(U_j.hi).
// The updates with pos(lo) < pos(S_i.hi) number B_i = cUlo(pos S_i.hi); those
// among them that fail the second condition are exactly the updates whose
// upper endpoint precedes S_i's lower one, C_i = cUhi(pos S_i.lo) (an update
// whose upper precedes S_i.lo also has its lower before S_i.hi).  Hence
// |{j : S_i and U_j intersect}| = B_i - C_i, and symmetrically for updates.
#include "offsets.cuh"
#include "sweep.cuh"

namespace ddm {

// Packed per-thread counts: S lower [0,21), U lower [21,42), S upper [42,63).
__device__ __forceinline__ unsigned long long kind_inc(uint32_t kind) {
    return kind == KIND_SLO ? 1ull : kind == KIND_ULO ? (1ull << 21)
                                   : kind == KIND_SHI ? (1ull << 42) : 0ull;
}

// One thread's walk over its SCAN_ITEMS endpoints with exact exclusive counts:
// the rank records, the order arrays, the per-id-tile count sums and (DBG) the
// diagnostics.  FULL: every item lies before E, so there is no end test.
// Adds x (< 2^32) to the 64-bit sum held as {low, high} 32-bit words in shared
// memory: a native 32-bit atomic, and one more for the rare carry.
__device__ __forceinline__ void add_u64_pair(uint32_t* w, uint32_t x) {
    const uint32_t old = atomicAdd(&w[0], x);
    if (old + x < old) atomicAdd(&w[1], 1u);
}

template <bool FULL, bool DBG>
__device__ __forceinline__ void sweep_walk(const uint32_t (&v)[SCAN_ITEMS], uint64_t base,
                                           uint32_t E, uint32_t n, uint32_t m,
                                           const Records& rec, uint32_t* s_agg,
                                           bool agg, uint32_t& cSlo, uint32_t& cUlo,
                                           uint32_t& cShi, DevStatus* st) {
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const uint64_t p64 = base + k;
        if (!FULL && p64 >= E) break;
        const uint32_t p = (uint32_t)p64;
        const uint32_t kind = v[k] >> 30, id = v[k] & ID_MASK;
        const uint32_t cUhi = p - cSlo - cUlo - cShi;
        // Guard: a payload or rank out of range means an upstream fault; skip it.
        if (id >= ((kind & 1u) ? m : n) || cSlo > n || cUlo > m) {
            raise_error(st, DDM_ERR_INTERNAL, 3);
            continue;
        }
        // One record store per endpoint, address and value selected by kind.
        const bool is_upd = kind & 1u, is_upper = kind >> 1;
        uint4* const tab =
            is_upper ? (is_upd ? rec.u_hi : rec.s_hi) : (is_upd ? rec.u_lo : rec.s_lo);
        const uint32_t y = is_upd ? cSlo : cUlo;  // lower endpoints seen of the other set
        // Lowers: uppers of the other set seen; uppers: own rank among this set's uppers.
        const uint32_t z = is_upper ? (is_upd ? cUhi : cShi) : (is_upd ? cShi : cUhi);
        const uint32_t w = is_upper ? 0u : (is_upd ? cUlo : cSlo);
        tab[id] = make_uint4(p, y, z, w);
        // B_i at S_i's upper endpoint, C_i at its lower one, summed apart: id tile t
        // holds {B low, B high, C low, C high} at s_agg[4t].
        if (agg && !is_upd)
            add_u64_pair(&s_agg[4 * (id / OFF_TILE) + (is_upper ? 0 : 2)], is_upper ? y : z);
        if (!is_upper && rec.sub_order && w < (is_upd ? m : n))
            (is_upd ? rec.upd_order : rec.sub_order)[w] = id;
        cSlo += kind == KIND_SLO;
        cUlo += kind == KIND_ULO;
        cShi += kind == KIND_SHI;
        if (DBG) {
            const uint32_t cUhi_after = p + 1 - cSlo - cUlo - cShi;
            rec.dbg_who[p] = v[k];
            rec.dbg_subset[p] = cSlo - cShi;
            rec.dbg_updset[p] = cUlo - cUhi_after;
        }
    }
}

// Two ways to the counts before a tile.  With `kinds` (the tile aggregates that
// the sort's last pass formed), the block sums the aggregates of all earlier
// tiles itself; no tile waits for another.  Without, each tile publishes its
// aggregate and looks back (decoupled look-back, tiles numbered in start order).
// At most 64 registers: four blocks per SM keep every tile of 2e6 endpoints resident.
// DBG: also the per-position diagnostics.
template <bool DBG>
__global__ void __launch_bounds__(SCAN_BLOCK, 4)
k_sweep_scan(const uint32_t* __restrict__ vals, uint32_t E, uint32_t n, uint32_t m,
             Records rec, unsigned long long* __restrict__ status,
             uint32_t* __restrict__ tile_counter, const uint4* __restrict__ kinds,
             unsigned long long* __restrict__ cnt_agg, uint32_t cnt_tiles, DevStatus* st) {
    pdl_begin();
    __shared__ unsigned long long warp_sum[SCAN_BLOCK / 32];
    __shared__ uint32_t kind_sum[SCAN_BLOCK / 32][3];
    __shared__ unsigned long long tile_prefix[3];
    __shared__ uint32_t tile_id_s;
    extern __shared__ uint32_t s_agg[];  // 4 words per id tile when cnt_agg is set
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) tile_id_s = kinds ? blockIdx.x : atomicAdd(tile_counter, 1u);
    if (cnt_agg)
        for (uint32_t t = tid; t < 4 * cnt_tiles; t += SCAN_BLOCK) s_agg[t] = 0u;
    __syncthreads();
    const uint32_t tile = tile_id_s;
    const uint64_t base = (uint64_t)tile * SCAN_TILE + (uint64_t)tid * SCAN_ITEMS;

    uint32_t v[SCAN_ITEMS];
    if (base + SCAN_ITEMS <= E) {
        const uint4* p4 = reinterpret_cast<const uint4*>(vals + base);
#pragma unroll
        for (int q = 0; q < SCAN_ITEMS / 4; ++q) {
            const uint4 a = p4[q];
            v[4 * q] = a.x; v[4 * q + 1] = a.y; v[4 * q + 2] = a.z; v[4 * q + 3] = a.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) v[k] = base + k < E ? vals[base + k] : 0xFFFFFFFFu;
    }
    uint32_t ka = 0, kb = 0, kc = 0;  // S lowers, U lowers, S uppers in earlier tiles
    if (kinds) {
#pragma unroll 4
        for (uint32_t t = tid; t < tile; t += SCAN_BLOCK) {
            const uint4 q = kinds[t];
            ka += q.x; kb += q.y; kc += q.z;
        }
    }
    unsigned long long mine = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < E) mine += kind_inc(v[k] >> 30);

    // Block-wide exclusive scan of the packed counts.
    unsigned long long x = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    if (kinds) {
        ka = __reduce_add_sync(0xffffffffu, ka);
        kb = __reduce_add_sync(0xffffffffu, kb);
        kc = __reduce_add_sync(0xffffffffu, kc);
        if (lane == 0) {
            kind_sum[warp][0] = ka; kind_sum[warp][1] = kb; kind_sum[warp][2] = kc;
        }
    }
    __syncthreads();
    unsigned long long wexcl = 0, total = 0;
#pragma unroll
    for (int w = 0; w < SCAN_BLOCK / 32; ++w) {
        unsigned long long t = warp_sum[w];
        if (w < warp) wexcl += t;
        total += t;
    }
    unsigned long long excl = wexcl + x - mine;

    if (kinds) {
        if (tid < 3) {
            unsigned long long pre = 0;
#pragma unroll
            for (int w = 0; w < SCAN_BLOCK / 32; ++w) pre += kind_sum[w][tid];
            tile_prefix[tid] = pre;
        }
    } else if (warp < 3) {
        // Publish the tile aggregate, one look-back word per counter, then look back.
        const unsigned long long agg = (total >> (21 * warp)) & ((1ull << 21) - 1);
        const uint64_t stride = gridDim.x + 1ull;
        unsigned long long* word = status + (uint64_t)warp * stride + tile;
        if (lane == 0) st_release_u64(word, (tile == 0 ? LB64_INC : LB64_AGG) | agg);
        unsigned long long pre = tile == 0 ? 0ull
                                           : warp_lookback_u64(status + (uint64_t)warp * stride,
                                                               tile, st, 3);
        if (lane == 0) {
            if (tile != 0) st_release_u64(word, LB64_INC | (pre + agg));
            tile_prefix[warp] = pre;
        }
    }
    __syncthreads();

    // Walk this thread's items with exact exclusive counts.
    uint32_t cSlo = (uint32_t)(tile_prefix[0] + (excl & ((1ull << 21) - 1)));
    uint32_t cUlo = (uint32_t)(tile_prefix[1] + ((excl >> 21) & ((1ull << 21) - 1)));
    uint32_t cShi = (uint32_t)(tile_prefix[2] + ((excl >> 42) & ((1ull << 21) - 1)));
    // A window boundary (a multiple of 2^win_shift >= SCAN_ITEMS) can only be
    // a thread's first position; the counts there are this thread's start.
    if (rec.windows && base < E && (base & ((1ull << rec.win_shift) - 1)) == 0)
        rec.windows[base >> rec.win_shift] =
            make_uint4(cSlo, cUlo, (uint32_t)base - cSlo - cUlo - cShi, (uint32_t)base);
    const bool agg = cnt_agg != nullptr;
    if (base + SCAN_ITEMS <= E)
        sweep_walk<true, DBG>(v, base, E, n, m, rec, s_agg, agg, cSlo, cUlo, cShi, st);
    else
        sweep_walk<false, DBG>(v, base, E, n, m, rec, s_agg, agg, cSlo, cUlo, cShi, st);
    // The thread holding position E - 1 writes the closing entry at E.
    if (rec.windows && base < E && base + SCAN_ITEMS >= E)
        rec.windows[(E + (1u << rec.win_shift) - 1) >> rec.win_shift] =
            make_uint4(cSlo, cUlo, E - cSlo - cUlo - cShi, E);
    if (cnt_agg) {
        __syncthreads();
        for (uint32_t t = tid; t < cnt_tiles; t += SCAN_BLOCK) {
            const uint32_t* w = s_agg + 4 * t;
            const unsigned long long b = ((unsigned long long)w[1] << 32) | w[0];
            const unsigned long long c = ((unsigned long long)w[3] << 32) | w[2];
            if (b != c) atomicAdd(&cnt_agg[t], b - c);  // mod 2^64: all blocks' terms add up
        }
    }
}

int launch_sweep_scan(const uint32_t* vals, uint64_t E, int64_t n, int64_t m, const Records& rec,
                       unsigned long long* status, DevStatus* st, cudaStream_t s,
                       const uint32_t* kinds, unsigned long long* cnt_agg) {
    if (E == 0) return 0;
    const uint64_t tiles = ceil_div(E, SCAN_TILE);
    // layout: 3 counters x (tiles + 1) words; the last word of counter 0's row
    // region doubles as the tile counter.
    uint32_t* counter = reinterpret_cast<uint32_t*>(status + 3 * (tiles + 1));
    if (tiles > SCAN_KINDS_MAX_TILES) kinds = nullptr;
    const uint64_t ctiles = ceil_div((uint64_t)n, (uint64_t)OFF_TILE);
    if (ctiles > CNT_AGG_MAX_TILES) cnt_agg = nullptr;
    const uint32_t ct = cnt_agg ? (uint32_t)ctiles : 0u;
    // Window boundaries fall on a thread's first position (see k_sweep_scan).
    if (rec.windows && (1ull << rec.win_shift) % SCAN_ITEMS != 0) return -1;
    launch_k(rec.dbg_who ? k_sweep_scan<true> : k_sweep_scan<false>, (unsigned)tiles, SCAN_BLOCK,
             4 * ct * sizeof(uint32_t), s, vals, (uint32_t)E, (uint32_t)n, (uint32_t)m, rec,
             status, counter, reinterpret_cast<const uint4*>(kinds), cnt_agg, ct, st);
    return 1;
}

// ---------------------------------------------------------------------------
// a4
// ---------------------------------------------------------------------------
__global__ void k_rank_count(const uint4* __restrict__ lo, const uint4* __restrict__ hi,
                             int64_t count, uint32_t* __restrict__ cnt, DevStatus* st) {
    pdl_begin();
    if (read_error(st)) return;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = hi[i].y, c = lo[i].z;
        bad |= b < c;
        cnt[i] = b - c;
    }
    if (bad) raise_error(st, DDM_ERR_INTERNAL, 4);
}

int launch_rank_count(const Records& rec, int64_t n, int64_t m, uint32_t* cnt,
                       uint32_t* upd_cnt, DevStatus* st, cudaStream_t s) {
    auto grid = [](int64_t c) {
        int64_t g = ceil_div((uint64_t)c, 256ull * 4);
        return (unsigned)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
    };
    int launches = 0;
    if (n > 0)
        launch_k(k_rank_count, grid(n), 256, 0, s, rec.s_lo, rec.s_hi, n, cnt, st), ++launches;
    if (upd_cnt && m > 0)
        launch_k(k_rank_count, grid(m), 256, 0, s, rec.u_lo, rec.u_hi, m, upd_cnt, st), ++launches;
    return launches;
}

// ---------------------------------------------------------------------------
// a5
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(OFF_BLOCK)
k_offsets(OffsetSource src, uint32_t n, unsigned long long* __restrict__ off,
          unsigned long long cap, unsigned long long* total_out,
          unsigned long long* __restrict__ status, uint32_t* __restrict__ tile_counter,
          DevStatus* st) {
    pdl_begin();
    offsets_tile(src, n, off, cap, total_out, status, tile_counter, st, blockIdx.x);
}

int launch_offsets(const uint32_t* cnt, int64_t n, unsigned long long* off, uint64_t cap,
                   unsigned long long* total, unsigned long long* status, DevStatus* st,
                   cudaStream_t s) {
    if (n == 0) return 0;
    const uint64_t tiles = ceil_div((uint64_t)n, OFF_TILE);
    uint32_t* counter = reinterpret_cast<uint32_t*>(status + tiles);
    OffsetSource src{};
    src.kind = 0;
    src.cnt = cnt;
    launch_k(k_offsets, (unsigned)tiles, OFF_BLOCK, 0, s, src, (uint32_t)n, off, cap, total, status,
             counter, st);
    return 1;
}

int launch_rank_offsets(const Records& rec, int64_t n, uint32_t* cnt, unsigned long long* off,
                        uint64_t cap, unsigned long long* total, unsigned long long* status,
                        DevStatus* st, cudaStream_t s, const unsigned long long* cnt_agg,
                        SubRank* srank) {
    if (n == 0) return 0;
    const uint64_t tiles = ceil_div((uint64_t)n, OFF_TILE);
    uint32_t* counter = reinterpret_cast<uint32_t*>(status + tiles);
    const OffsetSource src = rank_offset_source(rec, n, cnt, cnt_agg, srank);
    launch_k(k_offsets, (unsigned)tiles, OFF_BLOCK, 0, s, src, (uint32_t)n, off, cap, total, status,
             counter, st);
    return 1;
}

int launch_window_offsets(const uint4* windows, uint32_t num_win, uint32_t lcap,
                          unsigned long long* off, unsigned long long* total,
                          unsigned long long* status, DevStatus* st, cudaStream_t s) {
    if (num_win == 0) return 0;
    const uint64_t tiles = ceil_div((uint64_t)num_win, OFF_TILE);
    uint32_t* counter = reinterpret_cast<uint32_t*>(status + tiles);
    OffsetSource src{};
    src.kind = 2;
    src.windows = windows;
    src.lcap = lcap;
    launch_k(k_offsets, (unsigned)tiles, OFF_BLOCK, 0, s, src, num_win, off, ~0ull, total, status,
             counter, st);
    return 1;
}

}  // namespace ddm
