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

namespace ddm {

// Grid-Based matching (Section 2): a regular mesh over the first dg = min(d, 3)
// dimensions of the routing space.
constexpr int GRID_MAX_DIMS = 3;
constexpr uint32_t GRID_MAX_CELLS = 1u << 24;

struct GridPlan {
    int dg;                         // gridded dimensions
    uint32_t g[GRID_MAX_DIMS];      // cells along each
    uint32_t stride[GRID_MAX_DIMS]; // cell index = sum c_k * stride[k]
    float lo[GRID_MAX_DIMS];        // the mesh starts at the smallest lower bound
    float inv_w[GRID_MAX_DIMS];     // cells per unit length
    uint32_t G;                     // cells in all
};

// Device scratch of the grid matcher's first pass (zeroed before the call).
struct GridScratch {
    uint32_t kmax_hi[GRID_MAX_DIMS];      // max key of the upper bounds
    uint32_t kmin_lo_inv[GRID_MAX_DIMS];  // ~(min key of the lower bounds)
    double side_sum[GRID_MAX_DIMS];
};

// Bounding box and summed sides of the gridded dimensions (validating every
// dimension of both sets) into *gs.
int launch_grid_bounds(const DimPtrs& dims, int d, int64_t n, int64_t m, GridScratch* gs,
                       DevStatus* st, cudaStream_t s);

// The mesh, on the host, from the measured bounds: cells_per_dim > 0 fixes the
// cells along each gridded dimension; else cells about as wide as the mean
// extent side, with at least about one extent per cell (G <= GRID_MAX_CELLS).
GridPlan grid_plan(const GridScratch& h, int d, uint64_t total, uint32_t cells_per_dim);

// Per-cell membership counts of both sets (cnt_* zeroed, G entries each).
int launch_grid_count(const DimPtrs& dims, int64_t n, int64_t m, const GridPlan& p,
                      uint32_t* cnt_s, uint32_t* cnt_u, DevStatus* st, cudaStream_t s);

// Memberships sorted by cell (cell_off_* from the scans of the counts, cursors
// zeroed), then brute force inside each cell, reporting a pair only in the cell
// that holds max(S.lo, U.lo) along the gridded dimensions.  Count pass
// (pairs == NULL): cnt[i] (zeroed) accumulates; write pass: the pairs into
// pairs[2 off[i] ..) through cursor[i] (zeroed), in any order.
int launch_grid_fill(const DimPtrs& dims, int64_t n, int64_t m, const GridPlan& p,
                     const unsigned long long* cell_off_s, const unsigned long long* cell_off_u,
                     uint32_t* cur_s, uint32_t* cur_u, uint32_t* ent_s, uint32_t* ent_u,
                     DevStatus* st, cudaStream_t s);
int launch_grid_match(const DimPtrs& dims, int d, const GridPlan& p,
                      const unsigned long long* cell_off_s, const unsigned long long* cell_off_u,
                      const uint32_t* ent_s, const uint32_t* ent_u, uint32_t* cnt,
                      const unsigned long long* off, uint32_t* cursor, int32_t* pairs,
                      DevStatus* st, cudaStream_t s);

}  // namespace ddm
