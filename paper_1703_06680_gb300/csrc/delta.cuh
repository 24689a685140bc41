// Incremental matching for served sessions (the change report): interfaces.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "emit.cuh"

namespace ddm {

// One change report between the reference coordinates (those of the last
// delivered report) and the current ones.  A pair's status changes only if
// one of its elementary comparisons changes: c1(k) = [U.lo_k <= S.hi_k] or
// c2(k) = [S.lo_k <= U.hi_k] for some dimension k (on order-preserving keys,
// ties as in Algorithm 1).  If a comparison of two endpoints changed, the two
// are now at most 2 disp[k] apart, disp[k] being the largest displacement of
// any endpoint along k: candidates are the endpoint pairs that close.
struct DeltaArgs {
    int d;
    uint32_t n, m;
    DimPtrs now, ref;               // current and reference coordinates (device)
    // Dimension 0: the sorted endpoint stream of the current count phase.
    uint32_t E;
    const uint32_t* keys;           // sorted keys (E)
    const uint32_t* vals;           // sorted payloads (kind << 30) | id (E)
    // Dimensions 1..d-1: the updates' current bounds sorted by key, per dimension
    // (index k - 1): lower bounds (c1 candidates) and upper bounds (c2).
    const uint32_t* lo_key[DDM_MAX_DIMS - 1];
    const uint32_t* lo_id[DDM_MAX_DIMS - 1];
    const uint32_t* hi_key[DDM_MAX_DIMS - 1];
    const uint32_t* hi_id[DDM_MAX_DIMS - 1];
    const uint4* pk;                // dimension 0, per stream position: {current key,
                                    // reference key, payload, w} (E); w = for a
                                    // subscription bound the start of its walk in the
                                    // stream of the other kind (below), else 0
    // Dimension 0, the updates' bounds of one kind in stream order: entry r of
    // ulo for the r-th update lower endpoint, of uhi for the r-th upper, each 32
    // bytes at [2r, 2r + 1]: {current key, reference key, update id, 0} and the
    // update's other bound {current key, reference key, 0, 0} (2m uint4 each).
    // An S upper at stream position p walks ulo from cUlo(p), an S lower walks
    // uhi from cUhi(p).
    uint4* ulo;
    uint4* uhi;
    Records rec;                    // the count phase's rank records
    unsigned long long* disp;       // per dimension: bits of the largest |now - ref| (float,
                                    // rounded up, in the low 32 bits)
    unsigned long long* counters;   // [0] added, [1] removed, [2] write cursor
    unsigned long long* keys_out;   // (removed << (ibits + jbits)) | (i << jbits) | j per
                                    // changed pair, at most cap entries
    unsigned long long cap;
    int ibits, jbits;
};

// Outcome flags of a report, set on the device (flags[0]).
constexpr uint32_t DELTA_RERUN = 1u;     // more changed pairs than keys_out holds
constexpr uint32_t DELTA_CAPACITY = 2u;  // more than the caller's buffers hold

// disp[k] for every dimension (disp zeroed).
int launch_delta_disp(const DeltaArgs& a, DevStatus* st, cudaStream_t s);

// Keys and ids of the updates' bounds of dimensions 1..d-1, unsorted, into
// a.lo_key/lo_id/hi_key/hi_id (the caller then sorts each pair by key).
int launch_delta_keys(const DeltaArgs& a, cudaStream_t s);

// pk[p] = {keys[p], reference key (dimension 0) of the endpoint at stream
// position p, vals[p], walk start}, the per-kind update streams ulo / uhi, and
// disp[0].
int launch_delta_refk(const DeltaArgs& a, uint4* pk, cudaStream_t s);

// The changed pairs, each exactly once: counters[0], [1] count them, and their
// keys go to keys_out while there is room.
int launch_delta_cand(const DeltaArgs& a, DevStatus* st, cudaStream_t s);

// keys_out[q] = ~0 for q in [count, cap), so that a sort of all cap entries
// leaves the pairs first.
int launch_delta_pad(const DeltaArgs& a, cudaStream_t s);

// From the sorted keys: the added pairs into `added`, the removed ones into
// `removed` (flag bit stripped), unless they overflow keys_out (flags |=
// DELTA_RERUN) or the caller's capacities (flags |= DELTA_CAPACITY); then, if
// no flag is set, the current coordinates become the reference.
int launch_delta_finish(const DeltaArgs& a, const unsigned long long* sorted, int32_t* added,
                        uint64_t cap_added, int32_t* removed, uint64_t cap_removed,
                        uint32_t* flags, float* ref_coords, const float* coords,
                        uint64_t coord_count, cudaStream_t s);

// Sorted pair keys (i << jbits) | j into interleaved int32 pairs
// (pairs[2q] = key >> jbits, pairs[2q + 1] = key & ((1 << jbits) - 1)).
int launch_delta_unpack(const unsigned long long* keys, uint64_t count, int jbits, int32_t* pairs,
                        cudaStream_t s);

}  // namespace ddm
