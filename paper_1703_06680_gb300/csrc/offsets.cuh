// a5: the offsets scan (exclusive scan of per-subscription counts into output
// offsets, decoupled look-back or precomputed tile sums) as a per-block device
// function, so that a kernel can run it beside other independent work
// (k_offsets alone; k_rank_tables with the update rank tables of the window
// emission).
#pragma once

#include "sweep.cuh"

namespace ddm {

// Padded shared-memory index (one extra word every 32) against bank conflicts
// when a thread walks its own run of OFF_ITEMS consecutive elements.
__device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }

// Where the scanned values come from (so that the producing step needs no
// kernel of its own).
struct OffsetSource {
    int kind;                 // 0: cnt[i]
                              // 1: rank-arithmetic count B_i - C_i = hi[i].y - lo[i].z
                              //    of a4, also stored to cnt_out[i]
                              // 2: boundary-list size of window i,
                              //    s = windows[i].y - windows[i].z, or 0 when s > lcap
    const uint32_t* cnt;
    const uint4* lo;
    const uint4* hi;
    uint32_t* cnt_out;
    const uint4* windows;
    uint32_t lcap;
    const unsigned long long* agg;  // kind 1: per-tile sums of the counts, or NULL
    // kind 1, window emission (or NULL): the subscriptions' rank table, entry
    // r = the rank of S_i's lower endpoint (its record's w field), scattered
    // from id order.
    SubRank* srank;
};

// Kinds 0 and 2 (kind 1 is read inside k_offsets).
__device__ __forceinline__ uint32_t offset_value(const OffsetSource& src, uint64_t i) {
    if (src.kind == 2) {
        const uint4 t = src.windows[i];
        const uint32_t sz = t.y - t.z;
        return sz <= src.lcap ? sz : 0u;
    }
    return src.cnt[i];
}

// One tile (OFF_TILE values, one block of OFF_BLOCK threads) of the offsets
// scan; `block` numbers the scan's blocks (the tile when src.agg is set, else
// tiles are numbered in start order by the ticket counter).  Called once per
// block, after the kernel's programmatic-launch wait.
__device__ __forceinline__ void offsets_tile(const OffsetSource& src, uint32_t n,
                                             unsigned long long* __restrict__ off,
                                             unsigned long long cap,
                                             unsigned long long* total_out,
                                             unsigned long long* __restrict__ status,
                                             uint32_t* __restrict__ tile_counter, DevStatus* st,
                                             uint32_t block) {
    __shared__ uint32_t s_in[OFF_TILE + OFF_TILE / 32];
    __shared__ unsigned long long s_out[OFF_TILE + OFF_TILE / 32];
    __shared__ unsigned long long warp_sum[OFF_BLOCK / 32];
    __shared__ unsigned long long agg_sum[OFF_BLOCK / 32];
    __shared__ unsigned long long tile_prefix;
    __shared__ uint32_t tile_id_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) tile_id_s = src.agg ? block : atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = tile_id_s;
    const uint64_t tbase = (uint64_t)tile * OFF_TILE;
    // Coalesced load (striped), then each thread takes OFF_ITEMS consecutive values.
    // Counts from rank records: every load is issued before the first store of
    // a count, which the compiler could not otherwise move loads across.
    unsigned long long pre_part = 0;
    uint32_t pl[OFF_ITEMS], ph[OFF_ITEMS], rk[OFF_ITEMS];  // kind 1: positions and rank
    {
        bool bad = false;
        if (src.kind == 1) {
            uint32_t b[OFF_ITEMS], c[OFF_ITEMS];
#pragma unroll
            for (int k = 0; k < OFF_ITEMS; ++k) {
                const uint64_t i = tbase + k * OFF_BLOCK + tid;
                const uint4 lo = i < n ? src.lo[i] : make_uint4(0u, 0u, 0u, 0u);
                const uint4 hi = i < n ? src.hi[i] : make_uint4(0u, 0u, 0u, 0u);
                b[k] = hi.y;
                c[k] = lo.z;
                pl[k] = lo.x;
                rk[k] = lo.w;
                ph[k] = hi.x;
            }
            if (src.agg)  // this thread's share of the earlier tiles' sums
                for (uint32_t t = tid; t < tile; t += OFF_BLOCK) pre_part += src.agg[t];
#pragma unroll
            for (int k = 0; k < OFF_ITEMS; ++k) {
                const int i = k * OFF_BLOCK + tid;
                bad |= b[k] < c[k];
                s_in[pad32(i)] = b[k] - c[k];
                if (tbase + i < n) src.cnt_out[tbase + i] = b[k] - c[k];
            }
        } else {
#pragma unroll
            for (int k = 0; k < OFF_ITEMS; ++k) {
                const int i = k * OFF_BLOCK + tid;
                s_in[pad32(i)] = tbase + i < n ? offset_value(src, tbase + i) : 0u;
            }
        }
        if (bad) raise_error(st, DDM_ERR_INTERNAL, 4);
    }
    __syncthreads();
    uint32_t c[OFF_ITEMS];
    unsigned long long mine = 0;
#pragma unroll
    for (int k = 0; k < OFF_ITEMS; ++k) {
        c[k] = s_in[pad32(tid * OFF_ITEMS + k)];
        mine += c[k];
    }
    unsigned long long x = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pre_part += __shfl_xor_sync(0xffffffffu, pre_part, o);
    if (lane == 0) agg_sum[warp] = pre_part;
    __syncthreads();
    unsigned long long wexcl = 0, total = 0;
#pragma unroll
    for (int w = 0; w < OFF_BLOCK / 32; ++w) {
        unsigned long long t = warp_sum[w];
        if (w < warp) wexcl += t;
        total += t;
    }
    if (src.agg) {
        if (tid == 0) {
            unsigned long long pre = 0;
#pragma unroll
            for (int w = 0; w < OFF_BLOCK / 32; ++w) pre += agg_sum[w];
            tile_prefix = pre;
            if (src.agg[tile] != total) raise_error(st, DDM_ERR_INTERNAL, 4);
        }
    } else if (warp == 0) {
        unsigned long long* word = status + tile;
        if (lane == 0) st_release_u64(word, (tile == 0 ? LB64_INC : LB64_AGG) | total);
        unsigned long long pre = tile == 0 ? 0ull : warp_lookback_u64(status, tile, st, 5);
        if (lane == 0) {
            if (tile != 0) st_release_u64(word, LB64_INC | (pre + total));
            tile_prefix = pre;
        }
    }
    __syncthreads();
    unsigned long long run = tile_prefix + wexcl + x - mine;
#pragma unroll
    for (int k = 0; k < OFF_ITEMS; ++k) {
        s_out[pad32(tid * OFF_ITEMS + k)] = run;
        run += c[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < OFF_ITEMS; ++k) {
        const int i = k * OFF_BLOCK + tid;
        if (tbase + i < n) {
            const unsigned long long o = s_out[pad32(i)];
            off[tbase + i] = o;
            if (src.srank) {
                if (rk[k] < n) {
                    SubRank e;
                    e.e = make_uint4((uint32_t)(tbase + i), pl[k], ph[k], s_in[pad32(i)]);
                    e.off = o;
                    e.pad = 0ull;
                    src.srank[rk[k]] = e;
                } else {
                    raise_error(st, DDM_ERR_INTERNAL, 4);
                }
            }
        }
    }
    // The thread holding the last element also writes off[n] and the total.
    const uint64_t mybase = tbase + (uint64_t)tid * OFF_ITEMS;
    if (mybase < n && mybase + OFF_ITEMS >= n) {
        off[n] = run;
        *total_out = run;
        if (run > cap) raise_error(st, DDM_ERR_CAPACITY, 5);
    }
}

// The source of the rank-count scan (a4 + a5): cnt[i] = B_i - C_i from the
// subscriptions' records; see launch_rank_offsets.
inline OffsetSource rank_offset_source(const Records& rec, int64_t n, uint32_t* cnt,
                                       const unsigned long long* cnt_agg, SubRank* srank) {
    OffsetSource src{};
    src.kind = 1;
    src.lo = rec.s_lo;
    src.hi = rec.s_hi;
    src.cnt_out = cnt;
    src.agg = ceil_div((uint64_t)n, (uint64_t)OFF_TILE) <= CNT_AGG_MAX_TILES ? cnt_agg : nullptr;
    src.srank = srank;
    return src;
}

}  // namespace ddm
