// a3 sweep scan, a4 rank-arithmetic counts, a5 offsets: interfaces.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace ddm {

constexpr int SCAN_BLOCK = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;
constexpr int OFF_BLOCK = 256;
constexpr int OFF_ITEMS = 16;
constexpr int OFF_TILE = OFF_BLOCK * OFF_ITEMS;

// Per-region rank records written by the sweep scan.  Position p is an
// index into the sorted endpoint stream; cSlo(p), cUlo(p), cShi(p), cUhi(p)
// count the S lowers, U lowers, S uppers and U uppers strictly before p.
//   S_i: pos_lo, pos_hi, A = cUlo(pos_lo), B = cUlo(pos_hi), C = cUhi(pos_lo)
//   U_j: pos_lo, pos_hi, A = cSlo(pos_lo), B = cSlo(pos_hi), C = cShi(pos_lo)
// sub_order[r] (upd_order[r]) is the id of the subscription (update) whose
// lower endpoint is the r-th S (U) lower endpoint of the stream.
struct Records {
    uint32_t *s_pos_lo, *s_pos_hi, *s_A, *s_B, *s_C;
    uint32_t *u_pos_lo, *u_pos_hi, *u_A, *u_B, *u_C;
    uint32_t *sub_order, *upd_order;
    uint4* windows;       // (cSlo, cUlo, cUhi, p) at p = w << win_shift, or NULL
    int win_shift;
    uint32_t *dbg_who, *dbg_subset, *dbg_updset;  // optional diagnostics (may be NULL)
};

// Status words: 3 * (ceil(E / SCAN_TILE) + 1) u64, zeroed.
int launch_sweep_scan(const uint32_t* vals, uint64_t E, int64_t n, int64_t m, const Records& rec,
                       unsigned long long* status, DevStatus* st, cudaStream_t s);

// cnt[i] = B_i - C_i; optional upd_cnt[j] = B_j - C_j.
int launch_rank_count(const Records& rec, int64_t n, int64_t m, uint32_t* cnt,
                       uint32_t* upd_cnt, DevStatus* st, cudaStream_t s);

// off[i] = sum_{i' < i} cnt[i'] (u64), off[n] = K, st->K = K; raises
// DDM_ERR_CAPACITY when K > cap.  Status words: ceil(n / OFF_TILE) + 1 u64, zeroed.
int launch_offsets(const uint32_t* cnt, int64_t n, unsigned long long* off, uint64_t cap,
                    unsigned long long* status, DevStatus* st, cudaStream_t s);

}  // namespace ddm
