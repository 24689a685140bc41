// Incremental matching for served sessions: the pairs that appeared and the
// pairs that disappeared between two timesteps.
//
// Paper: Section 6 names dynamic DDM (regions that move between timesteps) as
// future work; SBM itself recomputes the full match.  Here the full match of
// the new timestep is computed as usual and compared with the previous one.
// Both lists are sorted by (sub, upd) and grouped by subscription, so the
// comparison splits into one comparison per subscription of two short sorted
// runs of update ids: an id of the new run that is absent from the old run is
// an added pair, an id of the old run absent from the new one a removed pair.
// One warp per subscription stages both runs in shared memory and merges them
// (merge path split over the lanes); a run longer than DELTA_STAGE is instead
// searched in global memory, id by id, with ballots keeping the order.
#include "delta.cuh"

namespace ddm {

constexpr int DELTA_BLOCK = 256;
constexpr int DELTA_WARPS = DELTA_BLOCK / 32;
constexpr uint32_t DELTA_STAGE = 256;  // ids per run staged in shared memory

// Whether id v occurs in the ascending run ids[0..len).  Staged runs
// (len <= DELTA_STAGE, shared memory): a branch-free search of fixed length
// whose position never passes DELTA_STAGE - 1, so the final probe covers the
// last element.  Longer runs (global memory, ids at stride 2): a plain one.
__device__ __forceinline__ bool staged_has(const int32_t* ids, uint32_t len, int32_t v) {
    static_assert((DELTA_STAGE & (DELTA_STAGE - 1)) == 0, "power of two");
    uint32_t pos = 0;
#pragma unroll
    for (uint32_t step = DELTA_STAGE / 2; step > 0; step >>= 1)
        if (pos + step <= len && ids[pos + step - 1] < v) pos += step;
    return pos < len && ids[pos] == v;
}

__device__ __forceinline__ bool global_has(const int32_t* pair_ids, uint32_t len, int32_t v) {
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pair_ids[2 * mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo < len && pair_ids[2 * lo] == v;
}

// Pairs of the run `src` (len_src pairs; its ids staged in src_stage when it
// fits) whose update id is absent from the run `other`; returns how many, and
// in the write pass stores them in order from out.
template <bool WRITE>
__device__ __forceinline__ uint32_t run_minus(const int32_t* src, uint32_t len_src,
                                              const int32_t* src_stage, const int32_t* other,
                                              uint32_t len_other, const int32_t* other_stage,
                                              int32_t sub, int32_t* out, int lane) {
    const unsigned lt = (1u << lane) - 1u;
    uint32_t cnt = 0;
    for (uint32_t k0 = 0; k0 < len_src; k0 += 32) {
        const uint32_t k = k0 + lane;
        bool keep = false;
        int32_t v = 0;
        if (k < len_src) {
            v = src_stage ? src_stage[k] : src[2 * k + 1];
            keep = other_stage ? !staged_has(other_stage, len_other, v)
                               : !global_has(other + 1, len_other, v);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (WRITE && keep) {
            int32_t* p = out + 2 * (uint64_t)(cnt + __popc(bal & lt));
            p[0] = sub;
            p[1] = v;
        }
        cnt += __popc(bal);
    }
    return cnt;
}

// Both runs staged (shared memory, ascending ids): one merge of the two runs,
// split over the warp by merge path (ties take the old run first).  Lane l
// walks positions [l * seg, (l + 1) * seg) of the merged sequence.  A new id
// is old iff the old element just before it (in merge order) is equal; an old
// id survives iff the next new element is equal -- both looked up in the
// staged runs, so an equal pair split between two lanes is still seen.  The
// walk is done once to count and, in the write pass, again to store at the
// lane's offsets (warp exclusive scans), which keeps both outputs in order.
template <bool WRITE>
__device__ __forceinline__ void merge_minus(const int32_t* A, uint32_t la, const int32_t* B,
                                            uint32_t lb, int32_t sub, int32_t* out_add,
                                            int32_t* out_rem, int lane, uint32_t& n_add,
                                            uint32_t& n_rem) {
    const uint32_t L = la + lb;
    const uint32_t seg = (L + 31) / 32;
    const uint32_t d0 = min((uint32_t)lane * seg, L), d1 = min(d0 + seg, L);
    uint32_t lo = d0 > lb ? d0 - lb : 0u, hi = min(d0, la);
    while (lo < hi) {  // merge-path split point on diagonal d0
        const uint32_t mid = (lo + hi) >> 1;
        if (A[mid] <= B[d0 - mid - 1]) lo = mid + 1;
        else hi = mid;
    }
    const uint32_t i0 = lo, j0 = d0 - lo;
    uint32_t add = 0, rem = 0;
    {
        uint32_t i = i0, j = j0;
        for (uint32_t p = d0; p < d1; ++p) {
            if (i < la && (j >= lb || A[i] <= B[j])) {
                rem += (j < lb && B[j] == A[i]) ? 0u : 1u;
                ++i;
            } else {
                add += (i > 0 && A[i - 1] == B[j]) ? 0u : 1u;
                ++j;
            }
        }
    }
    uint32_t xa = add, xr = rem;  // inclusive warp scans
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t ya = __shfl_up_sync(0xffffffffu, xa, o);
        const uint32_t yr = __shfl_up_sync(0xffffffffu, xr, o);
        if (lane >= o) { xa += ya; xr += yr; }
    }
    n_add = __shfl_sync(0xffffffffu, xa, 31);
    n_rem = __shfl_sync(0xffffffffu, xr, 31);
    if (WRITE) {
        uint32_t oa = xa - add, orr = xr - rem;
        uint32_t i = i0, j = j0;
        for (uint32_t p = d0; p < d1; ++p) {
            if (i < la && (j >= lb || A[i] <= B[j])) {
                if (!(j < lb && B[j] == A[i])) {
                    out_rem[2 * (uint64_t)orr] = sub;
                    out_rem[2 * (uint64_t)orr + 1] = A[i];
                    ++orr;
                }
                ++i;
            } else {
                if (!(i > 0 && A[i - 1] == B[j])) {
                    out_add[2 * (uint64_t)oa] = sub;
                    out_add[2 * (uint64_t)oa + 1] = B[j];
                    ++oa;
                }
                ++j;
            }
        }
    }
}

template <bool WRITE>
__global__ void __launch_bounds__(DELTA_BLOCK) k_delta(DeltaArgs a, DevStatus* st) {
    pdl_begin();
    __shared__ int32_t s_a[DELTA_WARPS][DELTA_STAGE];
    __shared__ int32_t s_b[DELTA_WARPS][DELTA_STAGE];
    if (read_error(st)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t warps = (int64_t)gridDim.x * DELTA_WARPS;
    for (int64_t i = (int64_t)blockIdx.x * DELTA_WARPS + warp; i < a.n; i += warps) {
        if (WRITE && a.add_off[i + 1] == a.add_off[i] && a.rem_off[i + 1] == a.rem_off[i])
            continue;  // the count pass found nothing to report for this subscription
        const uint64_t pa0 = a.prev_off[i], pa1 = a.prev_off[i + 1];
        const uint64_t cb0 = a.cur_off[i], cb1 = a.cur_off[i + 1];
        if (pa1 < pa0 || cb1 < cb0) {
            if (lane == 0) raise_error(st, DDM_ERR_INTERNAL, 20);
            continue;
        }
        const uint32_t la = (uint32_t)(pa1 - pa0), lb = (uint32_t)(cb1 - cb0);
        const int32_t* A = a.prev + 2 * pa0;
        const int32_t* B = a.cur + 2 * cb0;
        const int32_t* sa = nullptr;
        const int32_t* sb = nullptr;
        __syncwarp();
        if (la <= DELTA_STAGE) {
            for (uint32_t k = lane; k < la; k += 32) s_a[warp][k] = A[2 * k + 1];
            sa = s_a[warp];
        }
        if (lb <= DELTA_STAGE) {
            for (uint32_t k = lane; k < lb; k += 32) s_b[warp][k] = B[2 * k + 1];
            sb = s_b[warp];
        }
        __syncwarp();
        int32_t* out_add = WRITE ? a.added + 2 * a.add_off[i] : nullptr;
        int32_t* out_rem = WRITE ? a.removed + 2 * a.rem_off[i] : nullptr;
        uint32_t na, nr;
        if (sa && sb) {
            merge_minus<WRITE>(sa, la, sb, lb, (int32_t)i, out_add, out_rem, lane, na, nr);
        } else {
            na = run_minus<WRITE>(B, lb, sb, A, la, sa, (int32_t)i, out_add, lane);
            nr = run_minus<WRITE>(A, la, sa, B, lb, sb, (int32_t)i, out_rem, lane);
        }
        if (lane == 0) {
            if (!WRITE) {
                a.add_cnt[i] = na;
                a.rem_cnt[i] = nr;
            } else if (a.add_off[i + 1] - a.add_off[i] != na ||
                       a.rem_off[i + 1] - a.rem_off[i] != nr) {
                raise_error(st, DDM_ERR_INTERNAL, 21);
            }
        }
    }
}

int launch_delta(const DeltaArgs& a, bool write, DevStatus* st, cudaStream_t s) {
    if (a.n <= 0) return 0;
    int64_t g = ceil_div((uint64_t)a.n, (uint64_t)DELTA_WARPS);
    const unsigned grid = (unsigned)(g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g));  // 8 blocks / SM
    if (write) launch_k(k_delta<true>, grid, DELTA_BLOCK, 0, s, a, st);
    else launch_k(k_delta<false>, grid, DELTA_BLOCK, 0, s, a, st);
    return 1;
}

}  // namespace ddm
