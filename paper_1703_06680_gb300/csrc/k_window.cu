// a6 (d = 1): fused window emission -- candidate set per window of the sorted
// stream, sorted once by update id, filtered per subscription in id order, so
// every output segment is written already sorted.
//
// Paper: Algorithm 5 splits the sorted endpoint list T into segments and gives
// each processor the active sets at its segment's start (SubSet[p] and
// UpdSet[p], computed by Algorithm 6 and the prefix recurrence of Section 4).
// Here a segment is a window of 2^win_shift stream positions, one thread block
// each.  The block starts from UpdSet at the window boundary -- the list L_w
// of updates with pos(lo) < w*T <= pos(hi), built by k_tile_active from the
// scan's counts, exactly the paper's UpdSet[p] -- and adds the updates whose
// lower endpoint lies between the boundary and the farthest upper endpoint of
// the window's subscriptions.  That union W contains every partner of every
// subscription starting in the window: a partner U of S either starts before
// the boundary (then it is still active there, because it ends after S
// starts) or starts before S ends.  W is sorted by update id in shared memory;
// each subscription then keeps the members with pos(U.lo) < pos(S.hi) and
// pos(S.lo) < pos(U.hi) (the closed-interval test of Algorithm 1 in stream
// positions) and writes them in that order.
//
// A warp takes 32 consecutive subscriptions (by lower endpoint) and first
// copies the members of W that can meet any of them into a list of its own
// (8-byte entries, positions relative to the window); it then filters that
// list for two subscriptions at a time, testing 32 entries per step and
// compacting the kept ones by ballot into each output segment.
//
// Subscriptions spanning more than LONG_SPAN positions, and every subscription
// of a window whose boundary list or candidate set exceeds WCAP entries (or
// the list storage), are flagged and served by the range path (k_emit.cu)
// followed by the per-segment sort.
#include <atomic>

#include "emit.cuh"
#include "offsets.cuh"

namespace ddm {

constexpr int WIN_BLOCK = 256;        // eight warps per window
constexpr int WIN_WARPS = WIN_BLOCK / 32;
// The longest boundary list a window may use is a.lcap = 2^win_shift on this
// path: list w has the fixed slot [w * lcap, (w + 1) * lcap) of the storage.
constexpr uint32_t WCAP = 1024;       // candidates per window
constexpr uint32_t LONG_SPAN = 512;   // positions; longer subscriptions use the range path
constexpr int MAX_WIN_SHIFT = 10;     // windows of at most 1024 positions
constexpr int SETUP_BITS = 8;         // log2 of the set-up block (threads per window)
constexpr int SETUP_BLOCK = 1 << SETUP_BITS;
constexpr int SETUP_WARPS = SETUP_BLOCK / 32;
constexpr int NBUCKET = SETUP_BLOCK;  // buckets of the per-window id sort: one per thread

constexpr uint32_t LCAP_W = 512;      // entries of a warp's candidate list (longer: in pieces)

// Candidates in the filter are 8 bytes: {update id, (hi << 16) | lo}, with lo
// and hi the stream positions relative to the window start wT.  lo is 0 for
// updates starting before the window and below T + LONG_SPAN otherwise; hi is
// clamped to 0xffff, which is above every subscription's lower position.
constexpr uint32_t REL_MAX = 0xffffu;
static_assert((1u << MAX_WIN_SHIFT) + LONG_SPAN < REL_MAX, "relative positions fit 16 bits");

// Dynamic shared memory of k_emit_window (at most): the per-warp candidate
// lists, then the window's candidates.
constexpr size_t WSM_TOTAL = (size_t)WIN_WARPS * (LCAP_W + 32) * 8 + (size_t)WCAP * 8;

__device__ __forceinline__ bool list_fits(const EmitArgs& a, uint32_t w, uint32_t s) {
    return s <= a.lcap && list_base(a, w) + s <= a.lw_cap;
}

// Tiled join (d > 1): one pass over the updates in lower-endpoint order (rank
// r, id = upd_order[r]):
//  - the rank table urank[r] = {id, pos(lo), pos(hi)}, so that windows read
//    their candidates contiguously;
//  - the boundary lists: U contributes {id, pos(U.hi), rank} to every boundary w*T
//    with pos(U.lo) < w*T <= pos(U.hi) (the paper's UpdSet at that boundary).
// The lanes of a warp hold consecutive ranks, whose lower endpoints are close
// in the stream, so they mostly cross the same boundaries: the warp walks the
// union of its lanes' boundary ranges and reserves the slots of all lanes
// crossing boundary w with one atomic (order inside a list is irrelevant: the
// join sorts its candidates by id).  The window path of d = 1 builds the same
// tables from id order instead (k_rank_tables).
__global__ void k_tile_active(EmitArgs a, DevStatus* st) {
    pdl_begin();
    if (read_error(st)) return;
    const int S = a.win_shift;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); r0 < a.m;
         r0 += stride) {
        const int64_t r = r0 + lane;
        const bool valid = r < a.m;
        uint32_t j = 0, ph = 0, wlo = 1, whi = 0;  // empty boundary range
        if (valid) {
            j = a.rec.upd_order[r];
            const uint32_t pl = a.rec.u_lo[j].x;
            ph = a.rec.u_hi[j].x;
            a.urank[r] = make_uint4(j, pl, ph, 0u);
            wlo = (pl >> S) + 1;
            whi = min(ph >> S, a.num_win - 1);
        }
        const bool any = valid && wlo <= whi;
        const uint32_t wmin = __reduce_min_sync(0xffffffffu, any ? wlo : 0xffffffffu);
        const uint32_t wmax = __reduce_max_sync(0xffffffffu, any ? whi : 0u);
        for (uint32_t w = wmin; w <= wmax; ++w) {  // no iteration when no lane crosses one
            const bool mine = any && wlo <= w && w <= whi;
            const unsigned mask = __ballot_sync(0xffffffffu, mine);
            if (!mask) continue;
            const uint4 t = a.windows[w];
            const uint32_t s = t.y - t.z;
            if (!list_fits(a, w, s)) continue;
            const int leader = __ffs(mask) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(&a.lw_fill[w], (uint32_t)__popc(mask));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (mine) {
                const uint32_t slot = base + __popc(mask & lt);
                if (slot < s) a.lw[list_base(a, w) + slot] = make_uint4(j, ph, (uint32_t)r, 0u);
                else raise_error(st, DDM_ERR_INTERNAL, 10);
            }
        }
    }
}

// Window path, the same for the updates in id order (no gather by rank): U_j's
// records give its positions and the rank r of its lower endpoint (w field),
// so urank[r] = {j, pos(lo), pos(hi), 0} is scattered, and U_j is added to the
// boundary list of every window boundary it spans, one atomic per list entry
// (about a fifth of the updates span one at the usual densities).  The
// subscriptions' rank tables come from the offsets scan (launch_rank_offsets).
__device__ __forceinline__ void upd_ranks_blocks(const EmitArgs& a, DevStatus* st,
                                                 uint32_t block, uint32_t nblocks) {
    if (read_error(st)) return;
    const int S = a.win_shift;
    const int64_t stride = (int64_t)nblocks * blockDim.x;
    for (int64_t j = (int64_t)block * blockDim.x + threadIdx.x; j < a.m; j += stride) {
        const uint4 lo = a.rec.u_lo[j];
        const uint32_t ph = a.rec.u_hi[j].x, pl = lo.x, r = lo.w;
        if (r >= a.m) {
            raise_error(st, DDM_ERR_INTERNAL, 10);
            continue;
        }
        a.urank[r] = make_uint4((uint32_t)j, pl, ph, 0u);
        const uint32_t whi = min(ph >> S, a.num_win - 1);
        for (uint32_t w = (pl >> S) + 1; w <= whi; ++w) {
            const uint4 t = a.windows[w];
            const uint32_t sz = t.y - t.z;
            if (!list_fits(a, w, sz)) continue;
            const uint32_t slot = atomicAdd(&a.lw_fill[w], 1u);
            if (slot < sz)
                a.lw[list_base(a, w) + slot] = make_uint4((uint32_t)j, ph, r, 0u);
            else
                raise_error(st, DDM_ERR_INTERNAL, 10);
        }
    }
}

// The window path's rank tables in one launch: blocks [0, off_blocks) run the
// offsets scan over the subscriptions' counts, which also scatters their rank
// table (offsets_tile); the others build the update table and the boundary
// lists.  Both read only the sweep's records, so their latencies overlap.
// Three blocks per SM (up to 85 registers) keep the scan part free of spills.
__global__ void __launch_bounds__(OFF_BLOCK, 3)
k_rank_tables(OffsetSource src, uint32_t n, unsigned long long* off, unsigned long long cap,
              unsigned long long* total_out, unsigned long long* status, uint32_t* tile_counter,
              uint32_t off_blocks, EmitArgs a, DevStatus* st) {
    pdl_begin();
    if (blockIdx.x < off_blocks)
        offsets_tile(src, n, off, cap, total_out, status, tile_counter, st, blockIdx.x);
    else
        upd_ranks_blocks(a, st, blockIdx.x - off_blocks, gridDim.x - off_blocks);
}

// One subscription of the filter: its relative bounds, output id, id base
// and next free slot of its segment.
struct FilterSub {
    uint32_t pl, ph;
    int32_t i;
    uint32_t jb;
    int2* out;
};

// Keeps the list entries (pos(lo) < ph and pl < pos(hi), relative positions)
// of two subscriptions, 32 entries per step.  The caller guarantees room for
// a whole list after each segment's next free slot.
__device__ __forceinline__ void filter_pair(const uint2* list, uint32_t n32, FilterSub& A,
                                            FilterSub& B, int lane) {
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll 2
    for (uint32_t kk = lane; kk < n32; kk += 32) {
        const uint2 c = list[kk];
        const uint32_t lo = c.y & 0xffffu, hi = c.y >> 16;
        const bool a = lo < A.ph && hi > A.pl;
        const bool b = lo < B.ph && hi > B.pl;
        const unsigned ma = __ballot_sync(0xffffffffu, a);
        const unsigned mb = __ballot_sync(0xffffffffu, b);
        if (a) __stcs(&A.out[__popc(ma & lt)], make_int2(A.i, (int32_t)(c.x - A.jb)));
        if (b) __stcs(&B.out[__popc(mb & lt)], make_int2(B.i, (int32_t)(c.x - B.jb)));
        A.out += __popc(ma);
        B.out += __popc(mb);
    }
}

// The same for one subscription, never writing past `end`: advances x.out
// and returns false if the segment would overflow (x.out then stops there).
__device__ __forceinline__ bool filter_checked(const uint2* list, uint32_t n32, FilterSub& x,
                                               int2* const end, int lane) {
    const unsigned lt = (1u << lane) - 1u;
    for (uint32_t kk = lane; kk < n32; kk += 32) {
        const uint2 c = list[kk];
        const bool pass = (c.y & 0xffffu) < x.ph && (c.y >> 16) > x.pl;
        const unsigned bm = __ballot_sync(0xffffffffu, pass);
        if (x.out + __popc(bm) > end) {
            x.out = end;
            return false;
        }
        if (pass) __stcs(&x.out[__popc(bm & lt)], make_int2(x.i, (int32_t)(c.x - x.jb)));
        x.out += __popc(bm);
    }
    return true;
}

// Lane l's segment pointer, to every lane.
__device__ __forceinline__ int2* shfl_ptr(int2* p, int l) {
    return reinterpret_cast<int2*>(__shfl_sync(0xffffffffu, reinterpret_cast<uintptr_t>(p), l));
}

// Emission set-up of window w (one block per window): the candidate set W of
// the window's subscriptions, sorted by update id, packed as 8-byte entries
// {update id, (hi << 16) | lo} (positions relative to the window start) into
// a reserved run of wcand, and the window's descriptor
// wmeta[w] = {r0, ns, |W|, first entry in wcand}; ns = 0 tells the filter
// kernel to skip the window (no subscription starts in it, or all of them go
// to the range path).  Also writes every subscription's flag (1 = range path)
// and counts the flagged ones.  Kept apart from the filter so that the
// latency of these dependent loads and the id sort does not hold the filter's
// block slots: the filter kernel starts writing pairs after one load round.
__global__ void __launch_bounds__(SETUP_BLOCK) k_win_setup(EmitArgs a, DevStatus* st) {
    pdl_begin();
    __shared__ uint4 raw[WCAP];                    // {id, lo, hi, arrival rank in bucket}
    __shared__ uint32_t byb[WCAP];                 // ids by bucket
    __shared__ uint32_t bcnt[NBUCKET], bstart[NBUCKET], warp_tmp[SETUP_WARPS];
    __shared__ uint32_t s_pmax, s_nlow, s_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t w = blockIdx.x;
    const int S = a.win_shift;
    const uint32_t wT = w << S;  // the window's first stream position
    // An earlier stage's error leaves the counters meaningless: no read below
    // (the filter kernel checks the error too).
    if (read_error(st)) return;
    // Every global read is issued in two dependent rounds.  Round 1: the
    // window's counters, and the counters at the farthest boundary a regular
    // subscription of this window can reach (it starts before (w+1)T and spans
    // at most LONG_SPAN positions).
    const uint32_t reach = (LONG_SPAN + (1u << S) - 1u) >> S;
    const uint32_t wl = min(w + 1 + reach, a.num_win);
    const uint4 t0 = a.windows[w], t1 = a.windows[w + 1];
    const uint32_t u_lim = a.windows[wl].y;
    const unsigned long long lwo = list_base(a, w);
    const uint32_t ns = t1.x - t0.x;  // subscriptions starting here
    if (ns == 0) {
        if (tid == 0) a.wmeta[w] = make_uint4(0u, 0u, 0u, 0u);
        return;
    }
    const uint32_t r0 = t0.x, u0 = t0.y, lw_n = t0.y - t0.z;
    const bool lfit = lw_n <= a.lcap && lwo + lw_n <= a.lw_cap;
    // Candidate k of W is list entry k for k < lw_n, else rank entry
    // u0 + k - lw_n; the rank entries that may start before pmax are
    // [u0, u_lim), and at most WCAP candidates are loaded.
    const uint32_t nspec = u_lim - u0;
    const uint64_t nall = (uint64_t)lw_n + nspec;
    const uint32_t nload = lfit ? (uint32_t)(nall < WCAP ? nall : WCAP) : 0u;
    if (tid == 0) { s_pmax = 0; s_nlow = 0; }
    for (int b = tid; b < NBUCKET; b += SETUP_BLOCK) bcnt[b] = 0;
    __syncthreads();
    // Round 2: the window's subscriptions (rank-ordered table; a first flag
    // for each: 1 = longer than LONG_SPAN), the boundary list and the rank
    // entries after the boundary.
    {
        uint32_t pm = 0, nlong = 0;
        for (uint32_t k = tid; k < ns; k += SETUP_BLOCK) {
            const uint4 e = a.srank[r0 + k].e;
            const bool lng = e.z - e.y > LONG_SPAN;
            a.flag[e.x] = lng ? 1 : 0;
            nlong += lng;
            if (!lng) pm = max(pm, e.z);
        }
        pm = __reduce_max_sync(0xffffffffu, pm);
        nlong = __reduce_add_sync(0xffffffffu, nlong);
        if (lane == 0) {
            if (pm) atomicMax(&s_pmax, pm);
            if (nlong) atomicAdd(a.num_flagged, nlong);
        }
    }
    for (uint32_t k0 = 0; k0 < nload; k0 += 4 * SETUP_BLOCK) {
        uint4 e[4];
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            const uint32_t k = k0 + tid + it * SETUP_BLOCK;
            e[it] = make_uint4(0u, 0u, 0u, 0u);
            if (k < nload) {
                if (k < lw_n) {  // starts before the window: pos(lo) < any pos(S.hi)
                    const uint4 v = a.lw[lwo + k];
                    e[it] = make_uint4(v.x, 0u, v.y, 0u);
                } else {
                    const uint4 v = a.urank[u0 + k - lw_n];
                    e[it] = make_uint4(v.x, v.y, v.z, 0u);
                }
            }
        }
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            const uint32_t k = k0 + tid + it * SETUP_BLOCK;
            if (k < nload) raw[k] = e[it];
        }
    }
    __syncthreads();
    // Updates starting in [wT, pmax): the rank table is sorted by pos(lo), so
    // the loaded entries below pmax are a prefix of it; their count is nlow.
    const uint32_t pmax = s_pmax;
    {
        uint32_t c = 0;
        for (uint32_t k = lw_n + tid; k < nload; k += SETUP_BLOCK)
            c += raw[k].y < pmax ? 1u : 0u;
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0 && c) atomicAdd(&s_nlow, c);
    }
    __syncthreads();
    const uint32_t nlow = s_nlow;
    const uint32_t W = lw_n + nlow;
    // Only the first WCAP candidates were loaded: if all loaded rank entries
    // qualify and more exist, W may exceed WCAP (treated as an overflow).
    const uint32_t room = WCAP - min(lw_n, WCAP);
    const bool clipped = nspec > room && nlow == room;
    bool overflow = !lfit || W > WCAP || clipped;
    if (!overflow) {  // a run of wcand for the packed candidates
        if (tid == 0) {
            const unsigned long long b = atomicAdd(a.cand_fill, (unsigned long long)W);
            s_base = b + W <= a.cand_cap ? (uint32_t)b : 0xffffffffu;
        }
        __syncthreads();
        overflow = s_base == 0xffffffffu;
    }
    if (overflow) {
        // The whole window goes to the range path.
        uint32_t nreg = 0;
        for (uint32_t k = tid; k < ns; k += SETUP_BLOCK) {
            const uint4 e = a.srank[r0 + k].e;
            if (e.z - e.y <= LONG_SPAN) { a.flag[e.x] = 1; ++nreg; }
        }
        nreg = __reduce_add_sync(0xffffffffu, nreg);
        if (lane == 0 && nreg) atomicAdd(a.num_flagged, nreg);
        if (tid == 0) a.wmeta[w] = make_uint4(r0, 0u, 0u, 0u);
        return;
    }
    const uint32_t base = s_base;

    // W sorted by id: bucket sort on the high id bits (bucket starts by a
    // block scan, arrival rank in the bucket by a shared atomic), then the
    // exact place inside a bucket by counting smaller ids among its members.
    const int bshift = a.id_bits > SETUP_BITS ? a.id_bits - SETUP_BITS : 0;
    for (uint32_t k = tid; k < W; k += SETUP_BLOCK)
        raw[k].w = atomicAdd(&bcnt[raw[k].x >> bshift], 1u);
    __syncthreads();
    {
        static_assert(NBUCKET == SETUP_BLOCK && SETUP_BLOCK <= 1024, "one bucket per thread");
        const uint32_t c = bcnt[tid];
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tmp[warp] = x;
        __syncthreads();
        uint32_t before = 0;
#pragma unroll
        for (int q = 0; q < SETUP_WARPS; ++q) before += q < warp ? warp_tmp[q] : 0u;
        bstart[tid] = before + x - c;
    }
    __syncthreads();
    for (uint32_t k = tid; k < W; k += SETUP_BLOCK) {
        const uint4 e = raw[k];
        byb[bstart[e.x >> bshift] + e.w] = e.x;
    }
    __syncthreads();
    uint2* const cand = a.wcand + base;
    for (uint32_t k = tid; k < W; k += SETUP_BLOCK) {
        const uint4 e = raw[k];
        const uint32_t b = e.x >> bshift, s0 = bstart[b], c = bcnt[b];
        uint32_t f = s0;
        for (uint32_t q = s0; q < s0 + c; ++q) f += byb[q] < e.x ? 1u : 0u;
        // Relative positions (list entries have lo = 0: before the window).
        const uint32_t lo = e.y ? e.y - wT : 0u;
        const uint32_t hi = min(e.z - wT, REL_MAX);
        cand[f] = make_uint2(e.x, (hi << 16) | lo);
    }
    if (tid == 0) a.wmeta[w] = make_uint4(r0, ns, W, base);
}

// Pair emission of window w: warp g takes subscriptions 32g .. 32g+31 (by
// lower endpoint) and filters the window's candidates, prepared by
// k_win_setup, for them.
template <bool BATCHED>
__global__ void __launch_bounds__(WIN_BLOCK, 4) k_emit_window(EmitArgs a, DevStatus* st) {
    pdl_begin();
    extern __shared__ __align__(16) unsigned char wsm[];
    uint2* const lists = reinterpret_cast<uint2*>(wsm);             // per-warp candidate lists
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nwarps = blockDim.x >> 5;  // one warp per 128 window positions
    uint2* const cand = reinterpret_cast<uint2*>(wsm + (size_t)nwarps * (LCAP_W + 32) * 8);
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t w = blockIdx.x;
    const uint32_t wT = w << a.win_shift;  // the window's first stream position
    if (read_error(st)) return;
    const uint4 md = a.wmeta[w];
    const uint32_t r0 = md.x, ns = md.y, W = md.z;
    if (ns == 0) return;
    // One load round: the candidates into shared memory, and the entries of
    // this thread's subscription in its warp's first group (k = tid).
    const uint2* const gcand = a.wcand + md.w;
    uint4 e_first = make_uint4(0u, 0u, 0u, 0u);
    unsigned long long off_first = 0;
    if ((uint32_t)tid < ns) {
        const SubRank q = a.srank[r0 + tid];
        e_first = q.e;
        off_first = q.off;
    }
    for (uint32_t k = tid; k < W; k += blockDim.x) cand[k] = __ldg(gcand + k);
    __syncthreads();

    // Filter: warp g takes subscriptions 32g .. 32g+31 (by lower endpoint).
    uint2* const my_list = lists + warp * (LCAP_W + 32);
    const uint32_t Wr = (W + 31) & ~31u;
    int2* const pairs = reinterpret_cast<int2*>(a.pairs);
    bool bad = false;
    for (uint32_t g = warp; g * 32 < ns; g += nwarps) {
        const uint32_t k = g * 32 + lane;
        uint4 e = make_uint4(0u, 0u, 0u, 0u);
        unsigned long long off = 0;
        if (g == (uint32_t)warp) { e = e_first; off = off_first; }  // zero when k >= ns
        else if (k < ns) {
            const SubRank q = a.srank[r0 + k];
            e = q.e;
            off = q.off;
        }
        const bool reg = k < ns && e.z - e.y <= LONG_SPAN;
        // Relative bounds; an idle lane tests [0xffff, 0]: lo < 0 never holds.
        const uint32_t pl = reg ? e.y - wT : REL_MAX, ph = reg ? e.z - wT : 0u;
        const uint32_t plmin = __reduce_min_sync(0xffffffffu, pl);
        const uint32_t phmax = __reduce_max_sync(0xffffffffu, ph);
        if (phmax == 0) continue;  // no regular subscription in this group
        int32_t i_out = (int32_t)e.x;
        uint32_t jb = 0;
        if (BATCHED && reg) {  // ids are written local to their instance
            const int b = inst_of(a.inst_sub_base, a.num_inst, i_out);
            i_out -= (int32_t)a.inst_sub_base[b];
            jb = (uint32_t)a.inst_upd_base[b];
        }
        int2* my_out = pairs + off;  // next free slot of this lane's segment
        int2* const my_end = my_out + (reg ? e.w : 0u);
        // Without a bound check per step: a subscription keeps at most W
        // candidates, and off + W <= cap for every segment of the group.
        const bool all_fit = __all_sync(0xffffffffu, off + W <= a.cap);
        // The members of W that can meet some subscription of the group, in
        // id order, copied into the warp's list; more than LCAP_W of them are
        // filtered in pieces (each piece in id order after the previous one).
        for (uint32_t kk0 = 0; kk0 < Wr;) {
            uint32_t nq = 0;
            for (; kk0 < Wr && nq + 32 <= LCAP_W; kk0 += 32) {
                const uint32_t kk = kk0 + lane;
                uint2 c = make_uint2(0u, 0u);
                bool pass = false;
                if (kk < W) {
                    c = cand[kk];
                    pass = (c.y & 0xffffu) < phmax && (c.y >> 16) > plmin;
                }
                const unsigned bm = __ballot_sync(0xffffffffu, pass);
                if (pass) my_list[nq + __popc(bm & lt)] = c;
                nq += __popc(bm);
            }
            const uint32_t nq32 = (nq + 31) & ~31u;
            // Padding that no subscription keeps (lo = 0xffff).
            if (lane < nq32 - nq) my_list[nq + lane] = make_uint2(0u, REL_MAX);
            __syncwarp();
            // Two subscriptions per pass over the list: each step loads one
            // entry per lane and tests it against both; the kept ones are
            // compacted by ballot into each segment, in id order.
            for (int l = 0; l < 32; l += 2) {
                FilterSub A, B;
                A.ph = __shfl_sync(0xffffffffu, ph, l);
                B.ph = __shfl_sync(0xffffffffu, ph, l + 1);
                if ((A.ph | B.ph) == 0) continue;  // both idle or long
                A.pl = __shfl_sync(0xffffffffu, pl, l);
                B.pl = __shfl_sync(0xffffffffu, pl, l + 1);
                A.i = __shfl_sync(0xffffffffu, i_out, l);
                B.i = __shfl_sync(0xffffffffu, i_out, l + 1);
                A.jb = BATCHED ? __shfl_sync(0xffffffffu, jb, l) : 0u;
                B.jb = BATCHED ? __shfl_sync(0xffffffffu, jb, l + 1) : 0u;
                A.out = shfl_ptr(my_out, l);
                B.out = shfl_ptr(my_out, l + 1);
                if (all_fit) {
                    filter_pair(my_list, nq32, A, B, lane);
                } else {
                    int2* const endA = shfl_ptr(my_end, l);
                    int2* const endB = shfl_ptr(my_end, l + 1);
                    if (!filter_checked(my_list, nq32, A, endA, lane)) bad = true;
                    if (!filter_checked(my_list, nq32, B, endB, lane)) bad = true;
                }
                if (lane == l) my_out = A.out;
                if (lane == l + 1) my_out = B.out;
            }
            __syncwarp();  // every lane is done with the list before it is rebuilt
        }
        if (my_out != my_end) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) raise_error(st, DDM_ERR_INTERNAL, 12);
}

static unsigned grid_for(uint64_t items, unsigned per_block, unsigned cap) {
    uint64_t g = ceil_div(items, per_block);
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

int launch_tile_active(const EmitArgs& a, DevStatus* st, cudaStream_t s) {
    if (a.num_win == 0) return 0;
    if (a.m == 0) return 0;
    launch_k(k_tile_active, grid_for((uint64_t)a.m, 256, 152 * 16), 256, 0, s, a, st);
    return 1;
}

int launch_rank_tables(const Records& rec, int64_t n, uint32_t* cnt, unsigned long long* off,
                       uint64_t cap, unsigned long long* total, unsigned long long* status,
                       const unsigned long long* cnt_agg, const EmitArgs& a, DevStatus* st,
                       cudaStream_t s) {
    if (n == 0 || a.num_win == 0 || !a.srank) return -1;
    const uint64_t tiles = ceil_div((uint64_t)n, (uint64_t)OFF_TILE);
    uint32_t* counter = reinterpret_cast<uint32_t*>(status + tiles);
    const OffsetSource src = rank_offset_source(rec, n, cnt, cnt_agg, a.srank);
    const unsigned ub = a.m ? grid_for((uint64_t)a.m, OFF_BLOCK * 4, 152 * 2) : 0u;
    launch_k(k_rank_tables, (unsigned)tiles + ub, OFF_BLOCK, 0, s, src, (uint32_t)n, off,
             (unsigned long long)cap, total, status, counter, (uint32_t)tiles, a, st);
    return 1;
}

int launch_win_setup(const EmitArgs& a, DevStatus* st, cudaStream_t s) {
    if (a.num_win == 0 || a.n == 0) return 0;
    launch_k(k_win_setup, a.num_win, SETUP_BLOCK, 0, s, a, st);
    return 1;
}

template <bool BATCHED>
static void launch_emit_window_t(const EmitArgs& a, DevStatus* st, cudaStream_t s) {
    static std::atomic<unsigned long long> attr_set{0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !(attr_set.load() & (1ull << dev))) {
        cudaFuncSetAttribute(k_emit_window<BATCHED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)WSM_TOTAL);
        if (dev >= 0 && dev < 64) attr_set.fetch_or(1ull << dev);
    }
    // One warp per 128 window positions (about 32 subscriptions), 1 to 8 warps.
    const int shift_w = a.win_shift > 7 ? a.win_shift - 7 : 0;
    const unsigned nwarps = 1u << (shift_w < 3 ? shift_w : 3);
    const size_t smem = (size_t)nwarps * (LCAP_W + 32) * 8 + (size_t)WCAP * 8;
    launch_k(k_emit_window<BATCHED>, a.num_win, 32 * nwarps, smem, s, a, st);
}

int launch_emit_window(const EmitArgs& a, DevStatus* st, cudaStream_t s) {
    if (a.num_win == 0 || a.n == 0) return 0;
    if (a.win_shift > MAX_WIN_SHIFT) return -1;
    if (a.inst_sub_base) launch_emit_window_t<true>(a, st, s);
    else launch_emit_window_t<false>(a, st, s);
    return 1;
}

}  // namespace ddm
