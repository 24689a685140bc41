// Change report between two sorted pair lists of one session (incremental
// matching): interfaces.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace ddm {

// Two lists of (sub, upd) pairs, both sorted lexicographically and grouped by
// subscription through their offsets (off[i] .. off[i+1] is sub i's segment).
struct DeltaArgs {
    int64_t n;                                 // subscriptions
    const int32_t* prev;                       // previous list (2 ints per pair)
    const unsigned long long* prev_off;        // n + 1
    const int32_t* cur;                        // current list
    const unsigned long long* cur_off;         // n + 1
    uint32_t* add_cnt;                         // count pass: |cur_i \ prev_i|
    uint32_t* rem_cnt;                         // count pass: |prev_i \ cur_i|
    const unsigned long long* add_off;         // write pass: exclusive scans of the counts
    const unsigned long long* rem_off;
    int32_t* added;                            // write pass: pairs of cur not in prev
    int32_t* removed;                          // write pass: pairs of prev not in cur
};

// Count pass (write = false) or write pass (write = true), one warp per
// subscription.  The write pass checks its counts against the offsets and
// raises DDM_ERR_INTERNAL on a mismatch.
int launch_delta(const DeltaArgs& a, bool write, DevStatus* st, cudaStream_t s);

}  // namespace ddm
