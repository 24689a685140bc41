// a6 pair emission and a7 filter on dimensions 1..d-1: interfaces.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "sweep.cuh"

namespace ddm {

// Coordinates of all dimensions (device pointers), passed by value to kernels.
struct DimPtrs {
    const float* sub_lo[DDM_MAX_DIMS];
    const float* sub_hi[DDM_MAX_DIMS];
    const float* upd_lo[DDM_MAX_DIMS];
    const float* upd_hi[DDM_MAX_DIMS];
};

struct EmitArgs {
    int d;
    int64_t n, m;
    DimPtrs dims;
    Records rec;
    uint32_t* cnt;                  // per-subscription match counts
    const unsigned long long* off;  // n + 1 segment offsets
    uint32_t* cnt_a;                // d > 1: class (a) survivors per subscription
    uint32_t* cursor_b;             // per-subscription class (b) write cursor (zeroed)
    uint2* subK;                    // (d-1) x n keys of dims 1.., in sub_order layout
    uint2* updK;                    // (d-1) x m keys of dims 1.., in upd_order layout
    int32_t* pairs;                 // 2 * cap ints
    unsigned long long cap;
    int id_bits;                    // bits of the largest update id (radix passes)
    // Batched mode: ids are written local to their instance (see batch code).
    const int64_t* inst_sub_base;   // NULL in plain mode
    const int64_t* inst_upd_base;
    int num_inst;
    // Window path (d = 1): subscriptions it could not serve are flagged and
    // left to the range path; flag == NULL means "every subscription".
    uint8_t* flag;
    uint32_t* num_flagged;          // device counter; range path skipped when 0
    // Window lists: active updates at each window boundary.
    const uint4* windows;           // (cSlo, cUlo, cUhi, p) at p = w << win_shift, numWin + 1
    int win_shift;
    uint32_t num_win;
    unsigned long long* lw_off;     // list offsets (exclusive scan of the capped list sizes,
                                    // 0 for a list over lcap), numWin + 1; NULL: list w
                                    // has the fixed slot [w * lcap, (w + 1) * lcap)
    uint32_t* lw_fill;              // per-window fill cursor (zeroed)
    uint4* lw;                      // list storage {id, pos(U.hi), rank, 0}, lw_cap entries
    uint32_t lcap;                  // longest boundary list a window may use
    uint4* urank;                   // {id, pos(lo), pos(hi), 0} by lower-endpoint rank, m
    SubRank* srank;                 // window path: subscriptions by rank, n (or NULL)
    uint4* wmeta;                   // window path: {r0, ns, |W|, first wcand entry} per window
                                    // (ns = 0: skip), numWin
    uint2* wcand;                   // window path: id-sorted packed candidates, cand_cap entries
    unsigned long long* cand_fill;  // window path: entries of wcand reserved so far (zeroed)
    unsigned long long cand_cap;
    unsigned long long lw_cap;
    // d > 1, tiled join: the count pass also records every survivor as the key
    // (i << id_bits) | j into surv; window w, whose subscriptions have the
    // lower-endpoint ranks r0 .. r0 + ns, uses entries [r0 surv_cap,
    // (r0 + ns) surv_cap) (fill counter surv_fill[w]); NULL: not recorded.
    unsigned long long* surv;
    unsigned long long surv_cap;
    unsigned long long* surv_fill;
    const uint32_t* vals;           // sorted endpoint stream (payloads)
    bool sort_all;                  // segment sort every subscription, not only flagged ones
};

// First entry of window w's boundary list.
__device__ __forceinline__ unsigned long long list_base(const EmitArgs& a, uint32_t w) {
    return a.lw_off ? a.lw_off[w] : (unsigned long long)w * a.lcap;
}

// d > 1: tiled join of windows of subscriptions with chunks of candidates.
int launch_join(const EmitArgs& a, bool write, DevStatus* st, cudaStream_t s);
// Window w's used survivor entries (fill[w], padded holes included) into
// dst[pos[w] .. pos[w] + fill[w]).
int launch_surv_compact(const unsigned long long* surv, const unsigned long long* fill,
                        const uint4* windows, uint32_t num_win, unsigned long long per_sub,
                        const unsigned long long* pos, unsigned long long* dst, cudaStream_t s);

// Window path for d = 1.
int launch_tile_active(const EmitArgs& a, DevStatus* st, cudaStream_t s);
// Window path (fixed-slot lists), in one launch: the counts and offsets of
// launch_rank_offsets with the subscription rank table a.srank, and from the
// updates' records in id order the update rank table a.urank and the boundary
// lists.  Returns -1 when not on the window path (n == 0, no windows, or no
// srank).
int launch_rank_tables(const Records& rec, int64_t n, uint32_t* cnt, unsigned long long* off,
                       uint64_t cap, unsigned long long* total, unsigned long long* status,
                       const unsigned long long* cnt_agg, const EmitArgs& a, DevStatus* st,
                       cudaStream_t s);
int launch_win_setup(const EmitArgs& a, DevStatus* st, cudaStream_t s);
int launch_emit_window(const EmitArgs& a, DevStatus* st, cudaStream_t s);

// d > 1: permute keys of dims 1..d-1 into sub_order / upd_order layout and
// validate those dimensions (no NaN, lo <= hi).
int launch_permute_keys(const EmitArgs& a, DevStatus* st, cudaStream_t s);

// d > 1 count pass: cnt[i] = survivors of the filter among S_i's dim-0 matches.
int launch_filter_count(const EmitArgs& a, DevStatus* st, cudaStream_t s);

// Write pass: every match of S_i lands in out[off_i .. off_i + cnt_i), in any
// order, followed by the per-segment sort by update id.
int launch_emit_ranges(const EmitArgs& a, DevStatus* st, cudaStream_t s);
int launch_segment_sort(const EmitArgs& a, DevStatus* st, cudaStream_t s);

}  // namespace ddm
