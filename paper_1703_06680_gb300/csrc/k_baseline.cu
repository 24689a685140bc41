// Comparison matchers of the paper, on the GPU.
//
// Brute-Force matching (Algorithm 2): every (S_i, U_j) pair is tested with
// Algorithm 1 in every dimension (Section 3's logical "and").  One warp walks
// the updates in id order for one subscription at a time, 32 updates per step,
// and compacts the hits by ballot, so each subscription's segment is written
// in increasing update id -- the loop order of Algorithm 2.  The updates pass
// through shared memory in tiles, as order-preserving integer keys (so -0 and
// +0 compare equal and nothing is flushed, as on the sort-based path).
//
// Interval-Tree matching (Algorithm 3): an interval tree -- nodes ordered by
// lower bound, each subtree carrying its minimum lower and maximum upper
// bound -- answers Interval-Query for each query interval, leaving out every
// subtree whose maxupper is below the query's lower bound or whose minlower is
// above its upper bound.  The paper builds an AVL tree on S and queries it with
// every U_j; it notes that other balanced trees serve as well.  Here the tree
// is static and balanced: the leaves are the updates sorted by lower key (one
// radix sort), internal node k of a heap layout covers a run of leaves, its
// maxupper is stored and its minlower is the lower key of its first leaf.  The
// roles of the two sets are exchanged (the tree holds the updates, every
// subscription queries it), which Algorithm 1's symmetry allows and which
// yields each subscription's partners directly; a per-segment sort then puts
// them in update-id order.
#include "baseline.cuh"

namespace ddm {

constexpr int BF_BLOCK = 256;
constexpr int BF_TILE = 1024;  // updates per shared-memory tile
constexpr uint32_t NO_LO = 0xffffffffu;  // padding: above every valid key (NaN excluded)

__device__ __forceinline__ bool bad_extent(float lo, float hi) {
    return is_nan_bits(lo) || is_nan_bits(hi) || !(lo <= hi);
}

// One block: subscriptions [256 b, 256 b + 256), lane l of warp w holding
// subscription 256 b + 32 w + l; all warps walk the same update tiles.
template <bool WRITE>
__global__ void __launch_bounds__(BF_BLOCK)
k_bf(DimPtrs dims, int d, uint32_t n, uint32_t m, uint32_t* __restrict__ cnt,
     const unsigned long long* __restrict__ off, int2* __restrict__ pairs, DevStatus* st) {
    pdl_begin();
    extern __shared__ uint32_t bsm[];  // [d][2][BF_TILE]: lower keys, then upper keys
    if (WRITE && read_error(st)) return;
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t i = blockIdx.x * BF_BLOCK + tid;
    const bool have = i < n;
    uint32_t sl[DDM_MAX_DIMS], sh[DDM_MAX_DIMS];
    bool bad = false;
#pragma unroll
    for (int k = 0; k < DDM_MAX_DIMS; ++k) {
        sl[k] = 0u;
        sh[k] = 0u;
        if (k < d && have) {
            const float lo = dims.sub_lo[k][i], hi = dims.sub_hi[k][i];
            bad |= bad_extent(lo, hi);
            sl[k] = float_key(lo);
            sh[k] = float_key(hi);
        }
    }
    uint32_t my_cnt = 0;
    int2* my_out = WRITE && have ? pairs + off[i] : nullptr;
    const uint32_t base_w = blockIdx.x * BF_BLOCK + (tid & ~31);  // the warp's first subscription
    const uint32_t nsub = base_w < n ? min(32u, n - base_w) : 0u;
    for (uint32_t t0 = 0; t0 < m; t0 += BF_TILE) {
        const uint32_t tn = min((uint32_t)BF_TILE, m - t0);
        __syncthreads();  // the previous tile is consumed
        for (uint32_t x = tid; x < (uint32_t)d * BF_TILE; x += BF_BLOCK) {
            const uint32_t k = x / BF_TILE, r = x % BF_TILE;
            uint32_t klo = NO_LO, khi = 0u;
            if (r < tn) {
                const float lo = dims.upd_lo[k][t0 + r], hi = dims.upd_hi[k][t0 + r];
                if (!WRITE) bad |= bad_extent(lo, hi);
                klo = float_key(lo);
                khi = float_key(hi);
            }
            bsm[(2 * k) * BF_TILE + r] = klo;
            bsm[(2 * k + 1) * BF_TILE + r] = khi;
        }
        __syncthreads();
        for (uint32_t s = 0; s < nsub; ++s) {
            uint32_t bl[DDM_MAX_DIMS], bh[DDM_MAX_DIMS];
#pragma unroll
            for (int k = 0; k < DDM_MAX_DIMS; ++k) {
                if (k < d) {
                    bl[k] = __shfl_sync(0xffffffffu, sl[k], s);
                    bh[k] = __shfl_sync(0xffffffffu, sh[k], s);
                }
            }
            uint32_t c = __shfl_sync(0xffffffffu, my_cnt, s);
            int2* out = WRITE ? reinterpret_cast<int2*>(__shfl_sync(
                                    0xffffffffu, reinterpret_cast<uintptr_t>(my_out), s))
                              : nullptr;
            for (uint32_t r0 = 0; r0 < tn; r0 += 32) {
                const uint32_t r = r0 + lane;
                bool hit = r < tn;
#pragma unroll
                for (int k = 0; k < DDM_MAX_DIMS; ++k) {
                    if (k < d && hit) {
                        const uint32_t ul = bsm[(2 * k) * BF_TILE + r];
                        const uint32_t uh = bsm[(2 * k + 1) * BF_TILE + r];
                        hit = ul <= bh[k] && bl[k] <= uh;  // Algorithm 1, closed intervals
                    }
                }
                const unsigned bm = __ballot_sync(0xffffffffu, hit);
                if (WRITE && hit)
                    out[__popc(bm & lt)] = make_int2((int32_t)(base_w + s), (int32_t)(t0 + r));
                if (WRITE) out += __popc(bm);
                c += __popc(bm);
            }
            if (lane == (int)s) {
                my_cnt = c;
                if (WRITE) my_out = out;
            }
        }
    }
    if (!WRITE) {
        if (have) cnt[i] = my_cnt;
        if (__syncthreads_or(bad) && tid == 0) raise_error(st, DDM_ERR_INVALID, 40);
    }
}

static size_t bf_smem(int d) { return (size_t)2 * d * BF_TILE * sizeof(uint32_t); }

template <bool WRITE>
static void bf_launch(const DimPtrs& dims, int d, int64_t n, int64_t m, uint32_t* cnt,
                      const unsigned long long* off, int32_t* pairs, DevStatus* st,
                      cudaStream_t s) {
    // Opt-in above 48 KB of shared memory (d > 6); cheap, so set on every launch
    // (it is per device).
    cudaFuncSetAttribute(k_bf<WRITE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bf_smem(DDM_MAX_DIMS));
    // At least one block: with n = 0 it still validates the updates.
    uint64_t grid = ceil_div((uint64_t)n, BF_BLOCK);
    if (grid < 1) grid = 1;
    launch_k(k_bf<WRITE>, (unsigned)grid, BF_BLOCK, bf_smem(d), s, dims, d, (uint32_t)n,
             (uint32_t)m, cnt, off, reinterpret_cast<int2*>(pairs), st);
}

int launch_bf_count(const DimPtrs& dims, int d, int64_t n, int64_t m, uint32_t* cnt,
                    DevStatus* st, cudaStream_t s) {
    if (n == 0 && m == 0) return 0;
    bf_launch<false>(dims, d, n, m, cnt, nullptr, nullptr, st, s);
    return 1;
}

int launch_bf_write(const DimPtrs& dims, int d, int64_t n, int64_t m,
                    const unsigned long long* off, int32_t* pairs, DevStatus* st,
                    cudaStream_t s) {
    if (n == 0 || m == 0) return 0;
    bf_launch<true>(dims, d, n, m, nullptr, off, pairs, st, s);
    return 1;
}

// ---------------------------------------------------------------------------
// Interval tree over the updates (dimension 0)
// ---------------------------------------------------------------------------
constexpr int ITM_BUILD_BLOCK = 1024;  // leaves per block of the bottom levels
constexpr int ITM_STACK = 32;          // > tree height (P <= 2^30)

// Update keys for the sort by lower bound; validates every dimension of the
// updates (the query kernel validates the subscriptions).
__global__ void k_itm_keys(DimPtrs dims, int d, uint32_t m, uint32_t* __restrict__ keys,
                           uint32_t* __restrict__ vals, DevStatus* st) {
    pdl_begin();
    bool bad = false;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        for (int k = 0; k < d; ++k) bad |= bad_extent(dims.upd_lo[k][j], dims.upd_hi[k][j]);
        keys[j] = float_key(dims.upd_lo[0][j]);
        vals[j] = j;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) raise_error(st, DDM_ERR_INVALID, 41);
}

int launch_itm_keys(const DimPtrs& dims, int d, int64_t m, uint32_t* keys, uint32_t* vals,
                    DevStatus* st, cudaStream_t s) {
    if (m == 0) return 0;
    uint64_t g = ceil_div((uint64_t)m, 256);
    g = g > 152 * 16 ? 152 * 16 : g;
    launch_k(k_itm_keys, (unsigned)g, 256, 0, s, dims, d, (uint32_t)m, keys, vals, st);
    return 1;
}

// Leaves and the bottom levels: block b owns leaves [1024 b, 1024 b + 1024)
// (all P leaves when P < 1024) and writes the maxupper of every node of its
// subtree, level by level in shared memory.
__global__ void __launch_bounds__(ITM_BUILD_BLOCK)
k_itm_build_low(ItmTree t, const float* __restrict__ upd_hi, DevStatus* st) {
    pdl_begin();
    __shared__ uint32_t v[ITM_BUILD_BLOCK];
    if (read_error(st)) return;
    const uint32_t width = t.P < ITM_BUILD_BLOCK ? t.P : ITM_BUILD_BLOCK;
    const uint32_t x0 = blockIdx.x * width, tid = threadIdx.x;
    if (tid < width) {
        const uint32_t r = x0 + tid;
        v[tid] = r < t.m ? float_key(upd_hi[t.id_sorted[r]]) : 0u;
        t.tree[t.P + r] = v[tid];
    }
    __syncthreads();
    for (uint32_t sz = width >> 1, h = 1; sz >= 1; sz >>= 1, ++h) {
        uint32_t val = 0;
        if (tid < sz) val = max(v[2 * tid], v[2 * tid + 1]);
        __syncthreads();
        if (tid < sz) {
            v[tid] = val;
            t.tree[(t.P >> h) + (x0 >> h) + tid] = val;
        }
        __syncthreads();
    }
}

// The levels above the blocks' subtrees (P > 1024): one block, level by level.
__global__ void __launch_bounds__(ITM_BUILD_BLOCK) k_itm_build_top(ItmTree t, DevStatus* st) {
    pdl_begin();
    if (read_error(st)) return;
    for (uint32_t nodes = t.P / (2 * ITM_BUILD_BLOCK); nodes >= 1; nodes >>= 1) {
        for (uint32_t q = threadIdx.x; q < nodes; q += ITM_BUILD_BLOCK) {
            const uint32_t k = nodes + q;
            t.tree[k] = max(t.tree[2 * k], t.tree[2 * k + 1]);
        }
        __syncthreads();
    }
}

int launch_itm_build(const ItmTree& t, const float* upd_hi, DevStatus* st, cudaStream_t s) {
    if (t.m == 0) return 0;
    const uint32_t blocks = t.P < ITM_BUILD_BLOCK ? 1u : t.P / ITM_BUILD_BLOCK;
    launch_k(k_itm_build_low, blocks, ITM_BUILD_BLOCK, 0, s, t, upd_hi, st);
    if (t.P <= ITM_BUILD_BLOCK) return 1;
    launch_k(k_itm_build_top, 1, ITM_BUILD_BLOCK, 0, s, t, st);
    return 2;
}

// Interval-Query (Algorithm 3) of subscription i, one thread each, with an
// explicit stack: a subtree is left out when its maxupper is below the query's
// lower key or its minlower (its first leaf's lower key) is above the query's
// upper key; a leaf that survives both tests intersects the query along
// dimension 0, and is kept if dimensions 1..d-1 intersect too.  Leaves are
// reached in lower-key order.
template <bool WRITE>
__global__ void k_itm_query(ItmTree t, DimPtrs dims, int d, uint32_t n,
                            uint32_t* __restrict__ cnt, const unsigned long long* __restrict__ off,
                            int2* __restrict__ pairs, DevStatus* st) {
    pdl_begin();
    if (read_error(st)) return;
    bool bad = false;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t ql[DDM_MAX_DIMS], qh[DDM_MAX_DIMS];
#pragma unroll
        for (int k = 0; k < DDM_MAX_DIMS; ++k) {
            ql[k] = qh[k] = 0u;
            if (k < d) {
                const float lo = dims.sub_lo[k][i], hi = dims.sub_hi[k][i];
                if (!WRITE) bad |= bad_extent(lo, hi);
                ql[k] = float_key(lo);
                qh[k] = float_key(hi);
            }
        }
        uint32_t c = 0;
        int2* out = WRITE ? pairs + off[i] : nullptr;
        uint32_t stack[ITM_STACK];
        int sp = 0;
        uint32_t node = t.m ? 1u : 0u;  // 0: nothing left to visit
        int level = 0;                  // depth of `node`
        uint32_t levels[ITM_STACK];
        while (node) {
            const uint32_t span = t.P >> level;
            const uint32_t first = (node - (1u << level)) * span;  // first leaf of the subtree
            bool go = first < t.m && t.tree[node] >= ql[0] && t.lo_sorted[first] <= qh[0];
            if (go && node >= t.P) {  // a leaf: U intersects S along dimension 0
                const uint32_t j = t.id_sorted[first];
                bool keep = true;
                for (int k = 1; k < d && keep; ++k)
                    keep = float_key(dims.upd_lo[k][j]) <= qh[k] &&
                           ql[k] <= float_key(dims.upd_hi[k][j]);
                if (keep) {
                    if (WRITE) out[c] = make_int2((int32_t)i, (int32_t)j);
                    ++c;
                }
                go = false;
            }
            if (go) {  // visit the left subtree now, the right one later
                if (sp < ITM_STACK) {
                    stack[sp] = 2 * node + 1;
                    levels[sp] = level + 1;
                    ++sp;
                } else {
                    raise_error(st, DDM_ERR_INTERNAL, 42);
                }
                node = 2 * node;
                ++level;
            } else if (sp > 0) {
                --sp;
                node = stack[sp];
                level = (int)levels[sp];
            } else {
                node = 0;
            }
        }
        if (!WRITE) cnt[i] = c;
    }
    if (!WRITE && __syncthreads_or(bad) && threadIdx.x == 0) raise_error(st, DDM_ERR_INVALID, 43);
}

int launch_itm_query(const ItmTree& t, const DimPtrs& dims, int d, int64_t n, int64_t m,
                     uint32_t* cnt, const unsigned long long* off, int32_t* pairs,
                     DevStatus* st, cudaStream_t s) {
    (void)m;
    if (n == 0) return 0;
    uint64_t g = ceil_div((uint64_t)n, 128);
    g = g > 152 * 32 ? 152 * 32 : g;
    if (pairs)
        launch_k(k_itm_query<true>, (unsigned)g, 128, 0, s, t, dims, d, (uint32_t)n, cnt, off,
                 reinterpret_cast<int2*>(pairs), st);
    else
        launch_k(k_itm_query<false>, (unsigned)g, 128, 0, s, t, dims, d, (uint32_t)n, cnt, off,
                 static_cast<int2*>(nullptr), st);
    return 1;
}

}  // namespace ddm
