// In-library comparison matchers: Brute-Force matching (Algorithm 2) and
// Interval-Tree matching (Algorithm 3), as GPU kernels.  They compute the same
// sorted pair list as the sort-based path, by the paper's other two methods,
// so that the library can time them against it and use brute force as a
// second, independent GPU-side check at moderate sizes.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "emit.cuh"
#include "sort.cuh"

namespace ddm {

// Brute force, count pass: cnt[i] = number of updates intersecting S_i in all
// d dimensions (every pair tested).  Raises DDM_ERR_INVALID for NaN or
// lo > hi in any dimension of either set.
int launch_bf_count(const DimPtrs& dims, int d, int64_t n, int64_t m, uint32_t* cnt,
                    DevStatus* st, cudaStream_t s);

// Brute force, write pass: S_i's partners into pairs[2 off[i] ..), in
// increasing update id (the loop order of Algorithm 2), so segments need no
// sort.  Skipped when an earlier stage raised an error.
int launch_bf_write(const DimPtrs& dims, int d, int64_t n, int64_t m,
                    const unsigned long long* off, int32_t* pairs, DevStatus* st,
                    cudaStream_t s);

// Interval tree over the updates (dimension 0), a static balanced tree:
// leaves are the updates sorted by lower key; node k of the heap layout
// (children 2k and 2k + 1, leaves at P + r, P a power of two >= m) covers a
// run of leaves; its maxupper is tree[k], its minlower is the lower key of its
// first leaf.
struct ItmTree {
    uint32_t P;                 // leaves (power of two, >= m, >= 1)
    uint32_t m;
    const uint32_t* lo_sorted;  // lower keys in sorted order (m)
    const uint32_t* id_sorted;  // update ids in sorted order (m)
    uint32_t* tree;             // 2P max-upper keys (tree[0] unused)
};

// Key build of the updates' dimension-0 lower bounds: keys[j] = key(lo_j),
// vals[j] = j; validates every dimension of the updates.
int launch_itm_keys(const DimPtrs& dims, int d, int64_t m, uint32_t* keys, uint32_t* vals,
                    DevStatus* st, cudaStream_t s);

// tree[P + r] = key(upd_hi[id_sorted[r]]) (0 for padding), then the max of
// each node's children, bottom-up.
int launch_itm_build(const ItmTree& t, const float* upd_hi, DevStatus* st, cudaStream_t s);

// Interval-Query of every subscription against the tree (Algorithm 3, with
// the subscriptions as queries), filtered on dimensions 1..d-1.  Count pass
// (pairs == NULL): cnt[i]; write pass: the partners of S_i in tree (lower-key)
// order into pairs[2 off[i] ..); the caller then sorts each segment by id.
int launch_itm_query(const ItmTree& t, const DimPtrs& dims, int d, int64_t n, int64_t m,
                     uint32_t* cnt, const unsigned long long* off, int32_t* pairs,
                     DevStatus* st, cudaStream_t s);

}  // namespace ddm
