// a6: pair emission by symmetric range expansion, then a per-segment sort.
// a7: filter of dimensions 1..d-1 (count mode and write mode).
//
// Paper: Algorithm 4 reports, at each upper endpoint, the extent against the
// opposite active set; Section 3 extends d = 1 matching to d dimensions by
// testing the other projections (Algorithm 1 per dimension, logical "and").
//
// Decomposition used here.  With lowers before uppers at equal coordinates,
// S_i and U_j intersect along dimension 0 iff exactly one of
//   (a) pos(S_i.lo) < pos(U_j.lo) < pos(S_i.hi)   -- U_j starts inside S_i
//   (b) pos(U_j.lo) < pos(S_i.lo) < pos(U_j.hi)   -- S_i starts inside U_j
// holds.  The class-(a) partners of S_i are the updates of lower-endpoint
// rank A_i .. B_i-1 (a contiguous run of upd_order), and the class-(b)
// partners of U_j are the subscriptions of lower-endpoint rank A_j .. B_j-1
// (a contiguous run of sub_order).  Both sides therefore expand contiguous
// ranges, and the total work is the output size (plus the filtered-out
// candidates when d > 1).  Class (a) pairs go to the front of S_i's output
// segment in range order, class (b) pairs behind them through an atomic
// cursor; a per-segment sort by update id then fixes the order, so the result
// is deterministic.
#include "emit.cuh"

namespace ddm {

constexpr int EMIT_BLOCK = 256;
constexpr int WARP_SORT_MAX = 512;
constexpr int BIG_BLOCK = 256;
constexpr int BIG_ITEMS = 4;

// Id of the update / subscription whose lower endpoint has rank r in its set:
// from the window path's rank tables when they exist (the sweep then writes
// no order arrays), else from the order arrays.
__device__ __forceinline__ uint32_t upd_at_rank(const EmitArgs& a, uint64_t r) {
    return a.srank ? a.urank[r].x : a.rec.upd_order[r];
}
__device__ __forceinline__ uint32_t sub_at_rank(const EmitArgs& a, uint64_t r) {
    return a.srank ? a.srank[r].e.x : a.rec.sub_order[r];
}

// ---------------------------------------------------------------------------
// a7 set-up: keys of dims 1..d-1 in rank order, with validation.
// ---------------------------------------------------------------------------
__global__ void k_permute_keys(EmitArgs a, DevStatus* st) {
    pdl_begin();
    bool bad = false;
    const int64_t total = a.n + a.m;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total;
         r += (int64_t)gridDim.x * blockDim.x) {
        const bool upd = r >= a.n;
        const int64_t rank = upd ? r - a.n : r;
        const uint32_t id = upd ? a.rec.upd_order[rank] : a.rec.sub_order[rank];
        for (int k = 1; k < a.d; ++k) {
            const float lo = upd ? a.dims.upd_lo[k][id] : a.dims.sub_lo[k][id];
            const float hi = upd ? a.dims.upd_hi[k][id] : a.dims.sub_hi[k][id];
            bad |= is_nan_bits(lo) || is_nan_bits(hi) || !(lo <= hi);
            const uint2 kk = make_uint2(float_key(lo), float_key(hi));
            if (upd) a.updK[(int64_t)(k - 1) * a.m + rank] = kk;
            else a.subK[(int64_t)(k - 1) * a.n + rank] = kk;
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) raise_error(st, DDM_ERR_INVALID, 7);
}

// Keys of one extent in dims 1..d-1, held in registers.
struct OwnKeys {
    uint32_t lo[DDM_MAX_DIMS - 1], hi[DDM_MAX_DIMS - 1];
};

__device__ __forceinline__ OwnKeys own_keys(const EmitArgs& a, bool upd, int64_t id) {
    OwnKeys o;
#pragma unroll
    for (int k = 1; k < DDM_MAX_DIMS; ++k) {
        if (k < a.d) {
            o.lo[k - 1] = float_key(upd ? a.dims.upd_lo[k][id] : a.dims.sub_lo[k][id]);
            o.hi[k - 1] = float_key(upd ? a.dims.upd_hi[k][id] : a.dims.sub_hi[k][id]);
        }
    }
    return o;
}

// Algorithm 1 on integer keys for dims 1..d-1; `other` is in rank layout.
__device__ __forceinline__ bool pass_filter(const EmitArgs& a, const OwnKeys& o,
                                            const uint2* other, int64_t stride, int64_t rank) {
    bool ok = true;
#pragma unroll
    for (int k = 1; k < DDM_MAX_DIMS; ++k) {
        if (k < a.d) {
            const uint2 u = other[(int64_t)(k - 1) * stride + rank];
            ok &= (o.lo[k - 1] <= u.y) && (u.x <= o.hi[k - 1]);
        }
    }
    return ok;
}

__device__ __forceinline__ void put_pair(const EmitArgs& a, unsigned long long pos, int32_t i,
                                         int32_t j, DevStatus* st) {
    if (pos >= a.cap) {
        raise_error(st, DDM_ERR_INTERNAL, 6);
        return;
    }
    reinterpret_cast<int2*>(a.pairs)[pos] = make_int2(i, j);
}

// ---------------------------------------------------------------------------
// Class (a): one warp per subscription, UloOrder[A_i .. B_i).
// WRITE = false: count survivors (d > 1 only).
// ---------------------------------------------------------------------------
template <bool WRITE, bool FILTER>
__device__ __forceinline__ void class_a_body(const EmitArgs& a, DevStatus* st, uint32_t bid,
                                             uint32_t nblocks) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t warps = (int64_t)nblocks * (EMIT_BLOCK / 32);
    // Subscriptions in id order: neighbouring warps fill neighbouring output
    // segments.  (Visiting them in lower-endpoint order would let neighbouring
    // warps share candidate keys in L1; measured, that only pays for the long
    // ranges of d >= 3, which the tiled join serves by default.)
    for (int64_t i = ((int64_t)bid * EMIT_BLOCK + threadIdx.x) >> 5; i < a.n; i += warps) {
        if (a.flag && !a.flag[i]) continue;
        const uint32_t A = a.rec.s_lo[i].y, B = a.rec.s_hi[i].y;
        if (A > B || B > (uint64_t)a.m) {  // guard against an upstream fault
            if (lane == 0) raise_error(st, DDM_ERR_INTERNAL, 8);
            continue;
        }
        OwnKeys o;
        if (FILTER) o = own_keys(a, false, i);
        unsigned long long base = WRITE ? a.off[i] : 0ull;
        int32_t out_i = (int32_t)i, sub_off_j = 0;
        if (WRITE && a.inst_sub_base) {
            const int b = inst_of(a.inst_sub_base, a.num_inst, i);
            out_i = (int32_t)(i - a.inst_sub_base[b]);
            sub_off_j = (int32_t)a.inst_upd_base[b];
        }
        uint32_t running = 0;
        for (uint32_t k0 = A; k0 < B; k0 += 32) {
            const uint32_t k = k0 + lane;
            bool pass = k < B;
            if (FILTER && pass) pass = pass_filter(a, o, a.updK, a.m, k);
            const unsigned bal = __ballot_sync(0xffffffffu, pass);
            if (WRITE && pass) {
                const int32_t j = (int32_t)upd_at_rank(a, k) - sub_off_j;
                put_pair(a, base + running + __popc(bal & lt), out_i, j, st);
            }
            running += __popc(bal);
        }
        if (!WRITE && lane == 0) {
            a.cnt_a[i] = running;
            a.cnt[i] = running;
        }
    }
}

// ---------------------------------------------------------------------------
// Class (b): one warp per update, SloOrder[A_j .. B_j).
// ---------------------------------------------------------------------------
template <bool WRITE, bool FILTER>
__device__ __forceinline__ void class_b_body(const EmitArgs& a, DevStatus* st, uint32_t bid,
                                             uint32_t nblocks) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)nblocks * (EMIT_BLOCK / 32);
    // Updates in id order: neighbouring updates in stream order would target the
    // same subscriptions' counters at once (atomic contention).
    for (int64_t j = ((int64_t)bid * EMIT_BLOCK + threadIdx.x) >> 5; j < a.m; j += warps) {
        const uint32_t A = a.rec.u_lo[j].y, B = a.rec.u_hi[j].y;
        if (A > B || B > (uint64_t)a.n) {  // guard against an upstream fault
            if (lane == 0) raise_error(st, DDM_ERR_INTERNAL, 9);
            continue;
        }
        OwnKeys o;
        if (FILTER) o = own_keys(a, true, j);
        int32_t out_j = (int32_t)j;
        int64_t sub_base = 0;
        if (WRITE && a.inst_upd_base) {
            const int b = inst_of(a.inst_upd_base, a.num_inst, j);
            out_j = (int32_t)(j - a.inst_upd_base[b]);
            sub_base = a.inst_sub_base[b];
        }
        for (uint32_t r = A + lane; r < B; r += 32) {
            if (FILTER && !pass_filter(a, o, a.subK, a.n, r)) continue;
            const uint32_t i = sub_at_rank(a, r);
            if (a.flag && !a.flag[i]) continue;
            if (!WRITE) {
                atomicAdd(&a.cnt[i], 1u);
            } else {
                const uint32_t ca = FILTER ? a.cnt_a[i] : a.rec.s_hi[i].y - a.rec.s_lo[i].y;
                const uint32_t p = atomicAdd(&a.cursor_b[i], 1u);
                put_pair(a, a.off[i] + ca + p, (int32_t)(i - sub_base), out_j, st);
            }
        }
    }
}

// Count pass: class (a) stores each subscription's count, class (b) then adds
// to it, so the two run as consecutive kernels.
template <bool FILTER>
__global__ void __launch_bounds__(EMIT_BLOCK) k_class_a_count(EmitArgs a, DevStatus* st) {
    pdl_begin();
    if (read_error(st)) return;
    if (a.flag && *(volatile uint32_t*)a.num_flagged == 0u) return;
    class_a_body<false, FILTER>(a, st, blockIdx.x, gridDim.x);
}
template <bool FILTER>
__global__ void __launch_bounds__(EMIT_BLOCK) k_class_b_count(EmitArgs a, DevStatus* st) {
    pdl_begin();
    if (read_error(st)) return;
    if (a.flag && *(volatile uint32_t*)a.num_flagged == 0u) return;
    class_b_body<false, FILTER>(a, st, blockIdx.x, gridDim.x);
}

// Write pass: both classes in one launch, blocks [0, ga) for class (a) and
// [ga, ga + gb) for class (b).  Class (a) fills the front of a segment from
// off[i], class (b) the back from off[i] + cnt_a[i] through its cursors: the
// roles share no data written in this launch.
template <bool FILTER>
__global__ void __launch_bounds__(EMIT_BLOCK) k_class_ab_write(EmitArgs a, DevStatus* st,
                                                               uint32_t ga, uint32_t gb) {
    pdl_begin();
    if (read_error(st)) return;
    if (a.flag && *(volatile uint32_t*)a.num_flagged == 0u) return;
    if (blockIdx.x < ga) class_a_body<true, FILTER>(a, st, blockIdx.x, ga);
    else class_b_body<true, FILTER>(a, st, blockIdx.x - ga, gb);
}

// One warp per item, grid-stride; at most 8 blocks of 256 threads per SM.
static unsigned warp_grid(int64_t items) {
    int64_t g = ceil_div((uint64_t)items, EMIT_BLOCK / 32);
    return (unsigned)(g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g));
}

int launch_permute_keys(const EmitArgs& a, DevStatus* st, cudaStream_t s) {
    const int64_t total = a.n + a.m;
    if (a.d <= 1 || total == 0) return 0;
    int64_t g = ceil_div((uint64_t)total, 256 * 4);
    launch_k(k_permute_keys, (unsigned)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g)), 256, 0, s, a, st);
    return 1;
}

int launch_filter_count(const EmitArgs& a, DevStatus* st, cudaStream_t s) {
    int launches = 0;
    const unsigned ga = a.flag ? 152u : warp_grid(a.n), gb = a.flag ? 152u : warp_grid(a.m);
    if (a.n > 0) launch_k(k_class_a_count<true>, ga, EMIT_BLOCK, 0, s, a, st), ++launches;
    if (a.m > 0) launch_k(k_class_b_count<true>, gb, EMIT_BLOCK, 0, s, a, st), ++launches;
    return launches;
}

// When the window path ran (flags in use), the range path only serves the few
// flagged subscriptions and usually finds none: a small grid keeps that cheap.
static unsigned fallback_grid(const EmitArgs& a, int64_t items) {
    return a.flag && !a.sort_all ? 152u : warp_grid(items);
}

int launch_emit_ranges(const EmitArgs& a, DevStatus* st, cudaStream_t s) {
    if (a.n == 0 && a.m == 0) return 0;
    if (a.d > 1) {
        const unsigned ga = a.n > 0 ? (a.flag ? 152u : warp_grid(a.n)) : 0u;
        const unsigned gb = a.m > 0 ? (a.flag ? 152u : warp_grid(a.m)) : 0u;
        launch_k(k_class_ab_write<true>, ga + gb, EMIT_BLOCK, 0, s, a, st, ga, gb);
    } else {
        const unsigned ga = a.n > 0 ? fallback_grid(a, a.n) : 0u;
        const unsigned gb = a.m > 0 ? fallback_grid(a, a.m) : 0u;
        launch_k(k_class_ab_write<false>, ga + gb, EMIT_BLOCK, 0, s, a, st, ga, gb);
    }
    return 1;
}

// ---------------------------------------------------------------------------
// Per-segment sort by update id, in one launch.  Blocks [0, gw) sort the
// segments of up to WARP_SORT_MAX pairs, one warp each (bitonic network in
// shared memory).  Blocks [gw, gw + gbig) find the longer segments themselves
// (256 subscriptions per scan step) and sort each with the whole block.  A
// segment is sorted when flags are off (every segment), when every segment is
// requested (sort_all), or when its subscription is flagged.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool segment_wanted(const EmitArgs& a, int64_t i) {
    return !a.flag || a.sort_all || a.flag[i];
}

__device__ __forceinline__ void segsort_warp_body(const EmitArgs& a, uint32_t* buf, uint32_t bid,
                                                  uint32_t nblocks) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)nblocks * (EMIT_BLOCK / 32);
    for (int64_t i = ((int64_t)bid * EMIT_BLOCK + threadIdx.x) >> 5; i < a.n; i += warps) {
        if (!segment_wanted(a, i)) continue;
        const uint32_t c = a.cnt[i];
        if (c < 2 || c > WARP_SORT_MAX) continue;  // longer ones: the block role
        int32_t* seg = a.pairs + 2 * a.off[i];
        uint32_t P = 2;
        while (P < c) P <<= 1;
        for (uint32_t k = lane; k < P; k += 32) buf[k] = k < c ? (uint32_t)seg[2 * k + 1] : 0xFFFFFFFFu;
        __syncwarp();
        for (uint32_t size = 2; size <= P; size <<= 1) {
            for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
                for (uint32_t t = lane; t < P / 2; t += 32) {
                    // 2 * stride * (t / stride) + t % stride, stride a power of two
                    const uint32_t lo = ((t & ~(stride - 1)) << 1) | (t & (stride - 1));
                    const uint32_t hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    const uint32_t x = buf[lo], y = buf[hi];
                    if ((x > y) == up) { buf[lo] = y; buf[hi] = x; }
                }
                __syncwarp();
            }
        }
        for (uint32_t k = lane; k < c; k += 32) seg[2 * k + 1] = (int32_t)buf[k];
        __syncwarp();
    }
}

struct BigSortSmem {
    uint32_t hist[256];
    uint32_t bucket[256];
    uint32_t whist[BIG_BLOCK / 32][256];
    uint32_t list[BIG_BLOCK];  // long segments found in one scan step
    uint32_t nlist;
};

// One long segment, sorted by the whole block: LSD radix sort of the update-id
// column, 8 bits per pass, using the segment's own subscription-id column as
// the ping-pong buffer; the subscription ids are rewritten at the end.
// Stable ranking: peers of equal digits found with match_any within a warp,
// warp-ordered chunks.
__device__ void segsort_big_one(const EmitArgs& a, BigSortSmem& sm, uint32_t i) {
    constexpr int WARPS = BIG_BLOCK / 32;
    constexpr int CHUNK = BIG_BLOCK * BIG_ITEMS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int passes = (a.id_bits + 7) / 8;
    const uint32_t c = a.cnt[i];
    int32_t* seg = a.pairs + 2 * a.off[i];
    for (int p = 0; p < passes; ++p) {
        const int src = (p & 1) ? 0 : 1, dst = 1 - src;  // column offsets
        const int shift = 8 * p;
        sm.hist[tid] = 0;
        __syncthreads();
        for (uint32_t k = tid; k < c; k += BIG_BLOCK)
            atomicAdd(&sm.hist[((uint32_t)seg[2 * k + src] >> shift) & 0xFF], 1u);
        __syncthreads();
        if (warp == 0) {
            uint32_t run = 0;
            for (int b0 = 0; b0 < 256; b0 += 32) {
                uint32_t v = sm.hist[b0 + lane], x = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                sm.bucket[b0 + lane] = run + x - v;
                run += __shfl_sync(0xffffffffu, x, 31);
            }
        }
        __syncthreads();
        for (uint32_t c0 = 0; c0 < c; c0 += CHUNK) {
            for (int t = tid; t < WARPS * 256; t += BIG_BLOCK) (&sm.whist[0][0])[t] = 0;
            __syncthreads();
            uint32_t val[BIG_ITEMS], dg[BIG_ITEMS], rk[BIG_ITEMS];
            const uint32_t wb = c0 + warp * 32 * BIG_ITEMS;
#pragma unroll
            for (int it = 0; it < BIG_ITEMS; ++it) {
                const uint32_t k = wb + it * 32 + lane;
                val[it] = k < c ? (uint32_t)seg[2 * k + src] : 0xFFFFFFFFu;
                dg[it] = (val[it] >> shift) & 0xFF;
                const unsigned peers = __match_any_sync(0xffffffffu, dg[it]);
                const uint32_t cc = sm.whist[warp][dg[it]];
                __syncwarp();
                if (lane == __ffs(peers) - 1) sm.whist[warp][dg[it]] = cc + __popc(peers);
                __syncwarp();
                rk[it] = cc + __popc(peers & lt);
            }
            __syncthreads();
            {   // per digit: exclusive prefix over warps, chunk total
                uint32_t run = 0;
#pragma unroll
                for (int w = 0; w < WARPS; ++w) {
                    uint32_t x = sm.whist[w][tid];
                    sm.whist[w][tid] = run;
                    run += x;
                }
                sm.hist[tid] = run;  // chunk count of digit tid (tail items sit in digit 255 last)
            }
            __syncthreads();
#pragma unroll
            for (int it = 0; it < BIG_ITEMS; ++it) {
                const uint32_t k = wb + it * 32 + lane;
                if (k < c) {
                    const uint32_t pos = sm.bucket[dg[it]] + sm.whist[warp][dg[it]] + rk[it];
                    seg[2 * pos + dst] = (int32_t)val[it];
                }
            }
            __syncthreads();
            sm.bucket[tid] += sm.hist[tid];
            __syncthreads();
        }
        __syncthreads();
    }
    // Result is in column (passes odd ? 0 : 1); move it to column 1 and
    // restore the subscription ids in column 0.
    int32_t out_i = (int32_t)i;
    if (a.inst_sub_base) out_i = (int32_t)(i - a.inst_sub_base[inst_of(a.inst_sub_base, a.num_inst, i)]);
    for (uint32_t k = tid; k < c; k += BIG_BLOCK) {
        if (passes & 1) seg[2 * k + 1] = seg[2 * k];
        seg[2 * k] = out_i;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(EMIT_BLOCK) k_segsort(EmitArgs a, DevStatus* st, uint32_t gw,
                                                        uint32_t gbig) {
    static_assert(EMIT_BLOCK == BIG_BLOCK, "one block size for both roles");
    pdl_begin();
    __shared__ __align__(16) unsigned char smem[sizeof(BigSortSmem) > 4 * WARP_SORT_MAX *
                                                                         (EMIT_BLOCK / 32)
                                                    ? sizeof(BigSortSmem)
                                                    : 4 * WARP_SORT_MAX * (EMIT_BLOCK / 32)];
    if (read_error(st)) return;
    if (a.flag && !a.sort_all && *(volatile uint32_t*)a.num_flagged == 0u) return;
    if (blockIdx.x < gw) {
        uint32_t* buf = reinterpret_cast<uint32_t*>(smem) + (threadIdx.x >> 5) * WARP_SORT_MAX;
        segsort_warp_body(a, buf, blockIdx.x, gw);
        return;
    }
    BigSortSmem& sm = *reinterpret_cast<BigSortSmem*>(smem);
    const uint32_t bid = blockIdx.x - gw;
    for (int64_t base = (int64_t)bid * BIG_BLOCK; base < a.n; base += (int64_t)gbig * BIG_BLOCK) {
        if (threadIdx.x == 0) sm.nlist = 0;
        __syncthreads();
        const int64_t i = base + threadIdx.x;
        if (i < a.n && segment_wanted(a, i) && a.cnt[i] > WARP_SORT_MAX)
            sm.list[atomicAdd(&sm.nlist, 1u)] = (uint32_t)i;
        __syncthreads();
        const uint32_t nl = sm.nlist;
        for (uint32_t q = 0; q < nl; ++q) segsort_big_one(a, sm, sm.list[q]);
        __syncthreads();
    }
}

int launch_segment_sort(const EmitArgs& a, DevStatus* st, cudaStream_t s) {
    if (a.n == 0) return 0;
    const unsigned gw = fallback_grid(a, a.n), gbig = 152;
    launch_k(k_segsort, gw + gbig, EMIT_BLOCK, 0, s, a, st, gw, gbig);
    return 1;
}

}  // namespace ddm
