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
// Subscriptions spanning more than LONG_SPAN positions, and windows whose
// boundary list exceeds LCAP entries (or the list storage), are flagged and
// served by the range path (k_emit.cu) followed by the per-segment sort.
#include "emit.cuh"

namespace ddm {

constexpr int WIN_BLOCK = 256;
// The longest boundary list a window may use is a.lcap (1024 on this path).
constexpr uint32_t WCAP = 1024;       // candidates per window
constexpr uint32_t LONG_SPAN = 512;   // positions; longer subscriptions use the range path
constexpr int MAX_WIN_SHIFT = 9;      // windows of at most 512 positions
constexpr int NBUCKET = 256;          // buckets of the per-window id sort
constexpr int WITEMS = WCAP / WIN_BLOCK;

__device__ __forceinline__ bool list_fits(const EmitArgs& a, uint32_t w, uint32_t s) {
    return s <= a.lcap && a.lw_off[w] + s <= a.lw_cap;
}

// One pass over the updates in lower-endpoint order (rank r, id = upd_order[r]):
//  - the rank table urank[r] = {id, pos(lo), pos(hi)}, so that windows read
//    their candidates contiguously;
//  - the boundary lists: U contributes {id, pos(U.hi), rank} to every boundary w*T
//    with pos(U.lo) < w*T <= pos(U.hi) (the paper's UpdSet at that boundary).
// The lanes of a warp hold consecutive ranks, whose lower endpoints are close
// in the stream, so they mostly cross the same boundaries: the warp walks the
// union of its lanes' boundary ranges and reserves the slots of all lanes
// crossing boundary w with one atomic (order inside a list is irrelevant: the
// window kernel sorts its candidates by id).
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
                if (slot < s) a.lw[a.lw_off[w] + slot] = make_uint4(j, ph, (uint32_t)r, 0u);
                else raise_error(st, DDM_ERR_INTERNAL, 10);
            }
        }
    }
}

__global__ void __launch_bounds__(WIN_BLOCK) k_emit_window(EmitArgs a, DevStatus* st) {
    pdl_begin();
    constexpr uint32_t MAXSUB = 1u << MAX_WIN_SHIFT;
    __shared__ unsigned long long skey[WCAP];  // (update id << 32) | pos(U.lo)
    __shared__ uint32_t spay[WCAP];            // pos(U.hi)
    __shared__ uint32_t s_id[MAXSUB], s_lo[MAXSUB], s_hi[MAXSUB], s_cnt[MAXSUB];
    __shared__ unsigned long long s_off[MAXSUB];
    __shared__ uint32_t bcnt[NBUCKET], bstart[NBUCKET], warp_tmp[16];
    __shared__ uint32_t s_pmax, s_nreg;
    if (read_error(st)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t w = blockIdx.x;
    const int S = a.win_shift;
    const uint4 t0 = a.windows[w], t1 = a.windows[w + 1];
    const uint32_t r0 = t0.x, ns = t1.x - t0.x;  // subscriptions starting in this window
    if (ns == 0) return;
    if (ns > MAXSUB) {
        if (tid == 0) raise_error(st, DDM_ERR_INTERNAL, 11);
        return;
    }
    if (tid == 0) { s_pmax = 0; s_nreg = 0; }
    bcnt[tid] = 0;
    __syncthreads();
    for (uint32_t k = tid; k < ns; k += WIN_BLOCK) {
        const uint32_t i = a.rec.sub_order[r0 + k];
        const uint32_t pl = a.rec.s_lo[i].x, ph = a.rec.s_hi[i].x;
        s_id[k] = i; s_lo[k] = pl; s_hi[k] = ph;
        s_off[k] = a.off[i];
        s_cnt[k] = a.cnt[i];
        if (ph - pl <= LONG_SPAN) atomicMax(&s_pmax, ph);
    }
    __syncthreads();
    const uint32_t lw_n = t0.y - t0.z;
    const uint32_t wend = min(max((s_pmax >> S) + 1, w + 1), a.num_win);
    const uint32_t u0 = t0.y;
    // Updates starting in [wT, pmax): the rank table is sorted by pos(lo), so
    // the count of entries of [u0, cUlo(wend * T)) below pmax is the exact
    // length of the range (one parallel pass, no search).
    const uint32_t u1 = a.windows[wend].y;
    uint32_t nlow = 0;
    for (uint32_t r = u0; r < u1; r += WIN_BLOCK)
        nlow += __syncthreads_count(r + tid < u1 && a.urank[r + tid].y < s_pmax);
    const uint32_t W = lw_n + nlow;
    const bool overflow = !list_fits(a, w, lw_n) || W > WCAP;
    // Flags: 1 = served by the range path.
    for (uint32_t k = tid; k < ns; k += WIN_BLOCK) {
        const bool lng = overflow || (s_hi[k] - s_lo[k] > LONG_SPAN);
        a.flag[s_id[k]] = lng ? 1 : 0;
        if (lng) atomicAdd(a.num_flagged, 1u);
        else atomicAdd(&s_nreg, 1u);
    }
    if (overflow) return;

    // Candidate set W (boundary list, then updates starting in [wT, wend*T)),
    // held in registers: WITEMS per thread.
    const int bshift = a.id_bits > 8 ? a.id_bits - 8 : 0;
    unsigned long long key[WITEMS];
    uint32_t pay[WITEMS], bk[WITEMS], rk[WITEMS];
#pragma unroll
    for (int it = 0; it < WITEMS; ++it) {
        const uint32_t k = tid + it * WIN_BLOCK;
        if (k < W) {
            uint32_t id, pl;
            if (k < lw_n) {
                const uint4 e = a.lw[a.lw_off[w] + k];
                id = e.x; pl = 0u; pay[it] = e.y;  // starts before the window: pos(lo) < any pos(S.hi)
            } else {
                const uint4 e = a.urank[u0 + k - lw_n];
                id = e.x; pl = e.y; pay[it] = e.z;
            }
            key[it] = ((unsigned long long)id << 32) | pl;
            bk[it] = id >> bshift;
            rk[it] = atomicAdd(&bcnt[bk[it]], 1u);
        }
    }
    __syncthreads();
    // Bucket sort by the high id bits: bucket starts by a block scan, then the
    // exact position inside a bucket by counting smaller keys among its members.
    {
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
        for (int q = 0; q < WIN_BLOCK / 32; ++q) before += q < warp ? warp_tmp[q] : 0u;
        bstart[tid] = before + x - c;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < WITEMS; ++it) {
        const uint32_t k = tid + it * WIN_BLOCK;
        if (k < W) skey[bstart[bk[it]] + rk[it]] = key[it];
    }
    __syncthreads();
    uint32_t fin[WITEMS];
#pragma unroll
    for (int it = 0; it < WITEMS; ++it) {
        const uint32_t k = tid + it * WIN_BLOCK;
        if (k < W) {
            const uint32_t s0 = bstart[bk[it]], c = bcnt[bk[it]];
            uint32_t f = s0;
            for (uint32_t q = s0; q < s0 + c; ++q) f += skey[q] < key[it];
            fin[it] = f;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < WITEMS; ++it) {
        const uint32_t k = tid + it * WIN_BLOCK;
        if (k < W) {
            skey[fin[it]] = key[it];
            spay[fin[it]] = pay[it];
        }
    }
    // Pad W to whole warps with entries that no subscription keeps
    // (pos(lo) = 0xffffffff is never below a pos(S.hi)).
    const uint32_t Wpad = (W + 31) & ~31u;
    for (uint32_t k = W + tid; k < Wpad; k += WIN_BLOCK) {
        skey[k] = ~0ull;
        spay[k] = 0u;
    }
    __syncthreads();
    if (s_nreg == 0) return;

    // One warp per subscription: keep the members of W it intersects.
    const unsigned lt = (1u << lane) - 1u;
    for (uint32_t k = warp; k < ns; k += WIN_BLOCK / 32) {
        const uint32_t pl = s_lo[k], ph = s_hi[k];
        if (ph - pl > LONG_SPAN) continue;
        int32_t i = (int32_t)s_id[k];
        uint32_t j_base = 0;  // batched: ids are written local to the instance
        if (a.inst_sub_base) {
            const int b = inst_of(a.inst_sub_base, a.num_inst, i);
            i -= (int32_t)a.inst_sub_base[b];
            j_base = (uint32_t)a.inst_upd_base[b];
        }
        int2* out = reinterpret_cast<int2*>(a.pairs) + s_off[k];  // next free slot of the segment
        int2* const end = out + s_cnt[k];
        // Two 32-wide chunks per iteration for independent shared-memory loads.
        // Wpad is a multiple of 32, so every loop condition and the capacity
        // check are uniform across the warp.
        uint32_t kk = lane;
        for (; kk + 32 < Wpad; kk += 64) {
            const unsigned long long kv0 = skey[kk], kv1 = skey[kk + 32];
            const uint32_t p0 = spay[kk], p1 = spay[kk + 32];
            const bool pass0 = ((uint32_t)kv0 < ph) & (p0 > pl);
            const bool pass1 = ((uint32_t)kv1 < ph) & (p1 > pl);
            const unsigned b0 = __ballot_sync(0xffffffffu, pass0);
            const unsigned b1 = __ballot_sync(0xffffffffu, pass1);
            const int n0 = __popc(b0), n1 = __popc(b1);
            if (out + n0 + n1 > end) break;  // uniform: never write past the segment
            // Streaming stores: the pairs are written once and not read back here.
            if (pass0) __stcs(&out[__popc(b0 & lt)], make_int2(i, (int32_t)((uint32_t)(kv0 >> 32) - j_base)));
            if (pass1) __stcs(&out[n0 + __popc(b1 & lt)], make_int2(i, (int32_t)((uint32_t)(kv1 >> 32) - j_base)));
            out += n0 + n1;
        }
        for (; kk < Wpad; kk += 32) {
            const unsigned long long kv = skey[kk];
            const bool pass = ((uint32_t)kv < ph) & (spay[kk] > pl);
            const unsigned b = __ballot_sync(0xffffffffu, pass);
            if (out + __popc(b) > end) break;
            if (pass) __stcs(&out[__popc(b & lt)], make_int2(i, (int32_t)((uint32_t)(kv >> 32) - j_base)));
            out += __popc(b);
        }
        if (lane == 0 && (out != end || kk < Wpad)) raise_error(st, DDM_ERR_INTERNAL, 12);
    }
}

static unsigned grid_for(uint64_t items, unsigned per_block, unsigned cap) {
    uint64_t g = ceil_div(items, per_block);
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

int launch_tile_active(const EmitArgs& a, DevStatus* st, cudaStream_t s) {
    if (a.m == 0 || a.num_win == 0) return 0;
    launch_k(k_tile_active, grid_for(a.m, 256, 152 * 16), 256, 0, s, a, st);
    return 1;
}

int launch_emit_window(const EmitArgs& a, DevStatus* st, cudaStream_t s) {
    if (a.num_win == 0 || a.n == 0) return 0;
    if (a.win_shift > MAX_WIN_SHIFT) return -1;
    launch_k(k_emit_window, a.num_win, WIN_BLOCK, 0, s, a, st);
    return 1;
}

}  // namespace ddm
