// a3 sweep scan, a4 rank-arithmetic counts, a5 offsets: interfaces.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace ddm {

constexpr int SCAN_BLOCK = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;
constexpr int OFF_BLOCK = 256;
constexpr int OFF_ITEMS = 8;
constexpr int OFF_TILE = OFF_BLOCK * OFF_ITEMS;

// Per-region rank records written by the sweep scan.  Position p is an
// index into the sorted endpoint stream; cSlo(p), cUlo(p), cShi(p), cUhi(p)
// count the S lowers, U lowers, S uppers and U uppers strictly before p.
// Each endpoint event writes ONE packed record (a single scattered store):
//   s_lo[i] = {pos(S_i.lo), A = cUlo(pos lo), C = cUhi(pos lo), cSlo(pos lo)}
//   s_hi[i] = {pos(S_i.hi), B = cUlo(pos hi), 0, 0}
//   u_lo[j] = {pos(U_j.lo), A = cSlo(pos lo), C = cShi(pos lo), cUlo(pos lo)}
//   u_hi[j] = {pos(U_j.hi), B = cSlo(pos hi), 0, 0}
// All four are 16-byte records so that the scan writes every endpoint's record
// with one store through a computed address (no divergent branch per kind).
// sub_order[r] (upd_order[r]) is the id of the subscription (update) whose
// lower endpoint is the r-th S (U) lower endpoint of the stream.
struct Records {
    uint4* s_lo;
    uint4* s_hi;
    uint4* u_lo;
    uint4* u_hi;
    uint32_t *sub_order, *upd_order;  // ids by lower-endpoint rank (NULL: not written)
    uint4* windows;       // (cSlo, cUlo, cUhi, p) at p = w << win_shift, or NULL
    int win_shift;
    uint32_t *dbg_who, *dbg_subset, *dbg_updset;  // optional diagnostics (may be NULL)
};

// Status words: 3 * (ceil(E / SCAN_TILE) + 1) u64, zeroed.  kinds (may be NULL):
// the tile aggregates that launch_radix_sort's last pass formed (4 u32 per
// SCAN_TILE positions); with them, and at most SCAN_KINDS_MAX_TILES tiles, the
// tiles take their prefixes from the aggregates and the status words go unused.
// cnt_agg (may be NULL; ceil(n / OFF_TILE) u64, zeroed): the scan also adds up,
// per OFF_TILE subscription ids, the counts B_i - C_i of launch_rank_offsets
// (each block in shared memory, then one atomic per id tile), so that the
// offsets scan needs no look-back.  Used only with at most CNT_AGG_MAX_TILES
// id tiles; the caller passes the same pointer to launch_rank_offsets.
constexpr uint64_t SCAN_KINDS_MAX_TILES = 4096;
constexpr uint64_t CNT_AGG_MAX_TILES = 2048;
int launch_sweep_scan(const uint32_t* vals, uint64_t E, int64_t n, int64_t m, const Records& rec,
                       unsigned long long* status, DevStatus* st, cudaStream_t s,
                       const uint32_t* kinds = nullptr, unsigned long long* cnt_agg = nullptr);

// cnt[i] = B_i - C_i; optional upd_cnt[j] = B_j - C_j.
int launch_rank_count(const Records& rec, int64_t n, int64_t m, uint32_t* cnt,
                       uint32_t* upd_cnt, DevStatus* st, cudaStream_t s);

// off[i] = sum_{i' < i} cnt[i'] (u64), off[n] = *total = the sum; raises
// DDM_ERR_CAPACITY when the sum exceeds cap.  Status words: ceil(n / OFF_TILE)
// + 2 u64, zeroed.  *total must be zero on entry (it is left 0 when n == 0).
int launch_offsets(const uint32_t* cnt, int64_t n, unsigned long long* off, uint64_t cap,
                   unsigned long long* total, unsigned long long* status, DevStatus* st,
                   cudaStream_t s);

// a4 + a5 in one kernel: cnt[i] = B_i - C_i of the subscriptions' records and
// off[] / *total as launch_offsets gives for those counts.  Same status words.
// One subscription of the window emission, by the rank r of its lower
// endpoint among the subscriptions' lower endpoints: e = {i, pos(S_i.lo),
// pos(S_i.hi), cnt[i]} and off = off[i].  32 bytes: one sector per store.
struct SubRank {
    uint4 e;
    unsigned long long off, pad;
};

// cnt_agg: the per-id-tile sums from launch_sweep_scan (or NULL): each tile
// then takes its prefix from them instead of looking back.  srank (or NULL):
// the window emission's subscription rank table (n entries), scattered from
// id order.
int launch_rank_offsets(const Records& rec, int64_t n, uint32_t* cnt, unsigned long long* off,
                        uint64_t cap, unsigned long long* total, unsigned long long* status,
                        DevStatus* st, cudaStream_t s,
                        const unsigned long long* cnt_agg = nullptr, SubRank* srank = nullptr);

// Offsets of the boundary lists: value of window w = windows[w].y - windows[w].z
// (updates active at the window boundary), or 0 when that exceeds lcap.
int launch_window_offsets(const uint4* windows, uint32_t num_win, uint32_t lcap,
                          unsigned long long* off, unsigned long long* total,
                          unsigned long long* status, DevStatus* st, cudaStream_t s);

}  // namespace ddm
