// a7 for d > 1: the dimension-0 sweep joined with the filter of dims 1..d-1,
// tiled so that candidate keys are read once per window, not once per
// subscription.
//
// Paper: Section 3 reduces d dimensions to d = 1 -- two rectangles intersect
// iff every projection does -- and Algorithm 4 provides the dimension-0
// candidates.  As in the d = 1 window path (k_window.cu), a window of the
// sorted stream is one thread block; its dimension-0 candidates are the
// updates active at the window boundary (the paper's UpdSet[p], the list L_w)
// and the updates starting between the boundary and the farthest upper
// endpoint of the window's subscriptions.  Here the candidates are streamed
// through shared memory in chunks (positions plus keys of dims 1..d-1) and
// every subscription of the window tests each chunk: Algorithm 1 on stream
// positions for dimension 0 and on integer keys for the others.  The range
// part of the candidates is in lower-endpoint order, so a subscription stops
// at the first chunk that starts past its own upper endpoint.
//
// Pruning on dimension 1: each chunk is sorted in shared memory by its
// candidates' dimension-1 lower key.  With maxlen the largest dimension-1
// length hi - lo in the chunk (float, rounded up), a candidate can intersect
// S in dimension 1 only if its lower bound is at least S.lo1 - maxlen (rounded
// down): one below that ends before S starts.  The bound is taken back to key
// space (keys are order-preserving), so the candidates to test are those whose
// lower key lies in [key(S.lo1 - maxlen), key(S.hi1)]; each subscription finds
// that range by two warp-wide searches and tests only its members.  Lengths
// are measured on coordinates, not keys: a key difference grows with the
// exponent and would make the bound useless near 0.
//
// Pass 1 (count) stores each subscription's survivor count; after the offsets
// scan, pass 2 (write) appends the survivors to the subscription's segment.
// Segments are then sorted by update id (k_emit.cu).  Windows whose boundary
// list does not fit flag their subscriptions for the range path.
#include <atomic>

#include <algorithm>

#include "emit.cuh"

namespace ddm {

constexpr int JOIN_BLOCK = 512;
constexpr int JOIN_WARPS = JOIN_BLOCK / 32;
constexpr uint32_t JOIN_CHUNK = 512;
constexpr int JOIN_SHIFT = 11;  // windows of at most 2048 stream positions (DDM_PARAM_JOIN_SHIFT)
constexpr uint32_t JOIN_MAXSUB = 1u << JOIN_SHIFT;
constexpr uint32_t JOIN_LONG_RANGE = 16;  // candidate ranges walked by the whole warp
static_assert(JOIN_LONG_RANGE <= 32, "a short range's survivors fit a 32-bit mask");

// Dynamic shared memory of one join block for d dimensions.
__host__ __device__ inline size_t join_smem_bytes(int d) {
    return (size_t)JOIN_MAXSUB * sizeof(unsigned long long)   // sub output offsets
           + (size_t)JOIN_MAXSUB * 5 * sizeof(uint32_t)         // sub lo, hi, id, count, expected
           + (size_t)(d - 1) * JOIN_MAXSUB * sizeof(uint2)      // sub keys, dims 1..d-1
           + (size_t)JOIN_CHUNK * (sizeof(uint2) + sizeof(uint32_t))  // candidate pos, id
           + (size_t)(d - 1) * JOIN_CHUNK * sizeof(uint2)       // candidate keys, dims 1..d-1
           + 64;
}

// Number of sorted chunk keys sk[0..JOIN_CHUNK) below v / at most v (branch-free
// binary search, one thread).
__device__ __forceinline__ uint32_t chunk_count_below(const uint32_t* sk, uint32_t v) {
    uint32_t pos = 0;
#pragma unroll
    for (uint32_t step = JOIN_CHUNK / 2; step > 0; step >>= 1)
        pos += sk[pos + step - 1] < v ? step : 0u;
    return pos + (sk[pos] < v ? 1u : 0u);  // pos <= JOIN_CHUNK - 1 here
}
__device__ __forceinline__ uint32_t chunk_count_at_most(const uint32_t* sk, uint32_t v) {
    uint32_t pos = 0;
#pragma unroll
    for (uint32_t step = JOIN_CHUNK / 2; step > 0; step >>= 1)
        pos += sk[pos + step - 1] <= v ? step : 0u;
    return pos + (sk[pos] <= v ? 1u : 0u);
}

// DD > 0: compiled for DD = d - 1 extra dimensions; DD = 0: any d (arrays of
// DDM_MAX_DIMS - 1, runtime bound).
// Survivor slots of one warp: reserved from the window's fill counter in
// granules (one atomic per granule, not per warp step) of about 1/128 of the
// window's slice, between 32 and 512; slots a warp reserved but did not use
// are set to ~0 (sorted last).  All members are warp-uniform.
struct SurvSlots {
    unsigned long long next = 0, left = 0;
    uint32_t gran = 32;

    // Slots for cnt keys (cnt warp-uniform); returns the first.  Called by all
    // 32 lanes together.
    __device__ __forceinline__ unsigned long long take(uint32_t cnt, unsigned long long* sv,
                                                       unsigned long long* fill,
                                                       unsigned long long cap, int lane) {
        if (cnt > left) {
            pad(sv, cap, lane);
            const unsigned long long want = cnt > gran ? cnt : gran;
            unsigned long long b = 0;
            if (lane == 0) b = atomicAdd(fill, want);
            next = __shfl_sync(0xffffffffu, b, 0);
            left = want;
        }
        const unsigned long long r = next;
        next += cnt;
        left -= cnt;
        return r;
    }

    // The unused reserved slots become ~0.
    __device__ __forceinline__ void pad(unsigned long long* sv, unsigned long long cap, int lane) {
        for (unsigned long long q = lane; q < left; q += 32)
            if (next + q < cap) sv[next + q] = ~0ull;
        next += left;
        left = 0;
    }
};

template <bool WRITE, int DD>
__global__ void __launch_bounds__(JOIN_BLOCK) k_join(EmitArgs a, DevStatus* st) {
    constexpr int NK = DD > 0 ? DD : DDM_MAX_DIMS - 1;
    pdl_begin();
    extern __shared__ __align__(16) unsigned char jsm[];
    unsigned long long* s_off = reinterpret_cast<unsigned long long*>(jsm);
    uint32_t* s_lo = reinterpret_cast<uint32_t*>(s_off + JOIN_MAXSUB);
    uint32_t* s_hi = s_lo + JOIN_MAXSUB;
    uint32_t* s_id = s_hi + JOIN_MAXSUB;
    uint32_t* s_cnt = s_id + JOIN_MAXSUB;
    uint32_t* s_exp = s_cnt + JOIN_MAXSUB;  // write pass: the count from pass 1
    uint2* s_key = reinterpret_cast<uint2*>(s_exp + JOIN_MAXSUB);  // [(d-1)][JOIN_MAXSUB]
    uint2* c_pos = s_key + (size_t)(a.d - 1) * JOIN_MAXSUB;
    uint32_t* c_id = reinterpret_cast<uint32_t*>(c_pos + JOIN_CHUNK);
    uint2* c_key = reinterpret_cast<uint2*>(c_id + JOIN_CHUNK);  // [(d-1)][JOIN_CHUNK]
    __shared__ unsigned long long c_srt[JOIN_CHUNK];  // (dim-1 lo key << 32) | chunk index
    __shared__ uint32_t c_sk[JOIN_CHUNK];             // sorted dim-1 lo keys
    __shared__ uint32_t s_wmax[JOIN_WARPS];
    __shared__ uint32_t s_pmax, s_first;
    const bool rec_surv = !WRITE && a.surv != nullptr;

    if (read_error(st)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t w = blockIdx.x;
    const int S = a.win_shift;
    const int dd = DD > 0 ? DD : a.d - 1;
    const uint4 t0 = a.windows[w], t1 = a.windows[w + 1];
    const uint32_t r0 = t0.x, ns = t1.x - t0.x;
    if (ns == 0) return;
    if (ns > JOIN_MAXSUB) {
        if (tid == 0) raise_error(st, DDM_ERR_INTERNAL, 16);
        return;
    }
    // Count pass with survivor recording: this window's slice of the list,
    // surv_cap entries per subscription starting here (ranks r0 .. r0 + ns).
    unsigned long long* const sv_fill = rec_surv ? a.surv_fill + w : nullptr;
    unsigned long long* const sv = rec_surv ? a.surv + (uint64_t)r0 * a.surv_cap : nullptr;
    const unsigned long long sv_cap = (unsigned long long)ns * a.surv_cap;
    SurvSlots slots;
    slots.gran = (uint32_t)min(max(sv_cap / 128, 32ull), 512ull);
    const uint32_t lw_n = t0.y - t0.z;
    const bool overflow = !(lw_n <= a.lcap && a.lw_off[w] + lw_n <= a.lw_cap);
    if (tid == 0) s_pmax = 0;
    __syncthreads();
    for (uint32_t k = tid; k < ns; k += JOIN_BLOCK) {
        const uint32_t i = a.rec.sub_order[r0 + k];
        const uint32_t pl = a.rec.s_lo[i].x, ph = a.rec.s_hi[i].x;
        s_id[k] = i; s_lo[k] = pl; s_hi[k] = ph; s_cnt[k] = 0;
        if (WRITE) {
            s_off[k] = a.off[i];
            s_exp[k] = a.cnt[i];
        }
        for (int q = 0; q < a.d - 1; ++q)  // keys of dims 1..d-1 (sub_order rank layout)
            s_key[q * JOIN_MAXSUB + k] = a.subK[(int64_t)q * a.n + r0 + k];
        if (!WRITE) {  // the count pass decides the flags; the write pass reads them
            a.flag[i] = overflow ? 1 : 0;
            if (overflow) atomicAdd(a.num_flagged, 1u);
        }
        atomicMax(&s_pmax, ph);
    }
    __syncthreads();
    if (overflow) return;
    const uint32_t wend = min(max((s_pmax >> S) + 1, w + 1), a.num_win);
    const uint32_t u0 = t0.y, u1 = a.windows[wend].y;
    uint32_t nlow = 0;  // range part: updates starting in [wT, pmax), in rank order
    for (uint32_t r = u0; r < u1; r += JOIN_BLOCK)
        nlow += __syncthreads_count(r + tid < u1 && a.urank[r + tid].y < s_pmax);
    const uint32_t W = lw_n + nlow;

    static_assert(JOIN_BLOCK == JOIN_CHUNK, "one candidate per thread and chunk");
    for (uint32_t c0 = 0; c0 < W; c0 += JOIN_CHUNK) {
        const uint32_t clen = min(JOIN_CHUNK, W - c0);
        {   // one candidate per thread; entries past clen are never kept
            const uint32_t t = tid, k = c0 + t;
            uint32_t key1 = 0xffffffffu, len1 = 0;
            if (t < clen) {
                uint32_t id, pl, ph, rank;
                if (k < lw_n) {
                    const uint4 e = a.lw[a.lw_off[w] + k];
                    id = e.x; ph = e.y; rank = e.z; pl = 0u;  // starts before the window
                } else {
                    rank = u0 + (k - lw_n);
                    const uint4 e = a.urank[rank];
                    id = e.x; pl = e.y; ph = e.z;
                }
                c_pos[t] = make_uint2(pl, ph);
                c_id[t] = id;
                for (int q = 0; q < dd; ++q) c_key[q * JOIN_CHUNK + t] = a.updK[(int64_t)q * a.m + rank];
                const uint2 k1 = c_key[t];  // dimension 1 (q = 0)
                key1 = k1.x;
                const float lo1 = key_float(k1.x), hi1 = key_float(k1.y);
                // rounded up; a zero-length infinite extent (inf - inf) counts as 0
                const float len = hi1 == lo1 ? 0.0f : __fsub_ru(hi1, lo1);
                len1 = __float_as_uint(len);  // non-negative: bits order as values

            } else {
                c_pos[t] = make_uint2(0xffffffffu, 0u);  // fails the dimension-0 test
                c_id[t] = 0;
                for (int q = 0; q < dd; ++q) c_key[q * JOIN_CHUNK + t] = make_uint2(1u, 0u);
            }
            c_srt[t] = ((unsigned long long)key1 << 32) | t;
            uint32_t m1 = len1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m1 = max(m1, __shfl_xor_sync(0xffffffffu, m1, o));
            if (lane == 0) s_wmax[warp] = m1;
        }
        if (tid == 0) s_first = c0 >= lw_n ? c_pos[0].x : 0u;  // first pos(lo) of a range chunk
        __syncthreads();
        // Bitonic sort of the chunk's (dimension-1 lo key, index) words, ascending.
        for (uint32_t kk = 2; kk <= JOIN_CHUNK; kk <<= 1) {
            for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
                const uint32_t t = tid, u = t ^ j;
                if (u > t) {
                    const unsigned long long x = c_srt[t], y = c_srt[u];
                    const bool up = (t & kk) == 0;
                    if ((x > y) == up) { c_srt[t] = y; c_srt[u] = x; }
                }
                __syncthreads();
            }
        }
        {   // permute the chunk into sorted order (through registers, in place)
            const unsigned long long e = c_srt[tid];
            const uint32_t x = (uint32_t)e;
            const uint2 p = c_pos[x];
            const uint32_t id = c_id[x];
            uint2 kq[DDM_MAX_DIMS - 1];
#pragma unroll
            for (int q = 0; q < NK; ++q)
                if (q < dd) kq[q] = c_key[q * JOIN_CHUNK + x];
            __syncthreads();
            c_pos[tid] = p;
            c_id[tid] = id;
#pragma unroll
            for (int q = 0; q < NK; ++q)
                if (q < dd) c_key[q * JOIN_CHUNK + tid] = kq[q];
            const uint32_t key = (uint32_t)(e >> 32);
            c_sk[tid] = key;
        }
        __syncthreads();
        uint32_t maxbits = 0;
#pragma unroll
        for (int q = 0; q < JOIN_WARPS; ++q) maxbits = max(maxbits, s_wmax[q]);
        const float maxlen = __uint_as_float(maxbits);
        const uint32_t first = s_first;
        // One lane per subscription: two binary searches give its candidate
        // range; a short range is walked by the lane alone, a long one by the
        // whole warp (32 candidates per step, writes compacted by ballot).
        const uint32_t ns_pad = (ns + 31) & ~31u;
        for (uint32_t k = (uint32_t)tid; k < ns_pad; k += JOIN_BLOCK) {  // uniform per warp
            bool act = k < ns;
            uint32_t pl = 0, ph = 0;
            if (act) {
                pl = s_lo[k];
                ph = s_hi[k];
                act = !(c0 >= lw_n && first >= ph);  // every later candidate starts after S ends
            }
            uint2 own[NK];
            uint32_t b0 = 0, b1 = 0, cur = 0;
            if (act) {
#pragma unroll
                for (int q = 0; q < NK; ++q)
                    if (q < dd) own[q] = s_key[q * JOIN_MAXSUB + k];
                // candidates whose dimension-1 lower bound lies in [own.lo - maxlen, own.hi]
                const float bound = __fsub_rd(key_float(own[0].x), maxlen);
                const uint32_t lo_b = bound == bound ? float_key(bound) : 0u;  // NaN: inf - inf
                b0 = chunk_count_below(c_sk, lo_b);
                b1 = chunk_count_at_most(c_sk, own[0].y);
                cur = s_cnt[k];
            } else {
#pragma unroll
                for (int q = 0; q < NK; ++q) own[q] = make_uint2(0u, 0u);
            }
            unsigned long long obase = 0;  // write pass: segment start
            uint32_t c = 0;                // write pass: expected count
            int32_t i_out = 0;
            uint32_t j_base = 0;
            if (WRITE && act && b0 < b1) {
                const uint32_t i = s_id[k];
                obase = s_off[k];
                c = s_exp[k];
                i_out = (int32_t)i;
                if (a.inst_sub_base) {
                    const int b = inst_of(a.inst_sub_base, a.num_inst, i);
                    i_out -= (int32_t)a.inst_sub_base[b];
                    j_base = (uint32_t)a.inst_upd_base[b];
                }
            }
            const bool longr = b1 - b0 >= JOIN_LONG_RANGE;
            const uint32_t cur0 = cur;
            uint32_t passmask = 0;  // short range: bit x - b0 = candidate x survives
            if (b0 < b1 && !longr) {
                int2* seg = reinterpret_cast<int2*>(a.pairs) + obase;
                for (uint32_t x = b0; x < b1; ++x) {
                    const uint2 p = c_pos[x];
                    bool pass = (p.x < ph) & (p.y > pl);
#pragma unroll
                    for (int q = 0; q < NK; ++q) {
                        if (q < dd) {
                            const uint2 u = c_key[q * JOIN_CHUNK + x];
                            pass &= (own[q].x <= u.y) & (u.x <= own[q].y);
                        }
                    }
                    if (pass) {
                        if (WRITE && cur < c) seg[cur] = make_int2(i_out, (int32_t)(c_id[x] - j_base));
                        passmask |= 1u << (x - b0);
                        ++cur;
                    }
                }
            }
            if (rec_surv) {  // the short ranges' survivors: one shared reservation per warp
                const uint32_t mine = (b0 < b1 && !longr) ? cur - cur0 : 0u;
                uint32_t incl = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const uint32_t wtot = __shfl_sync(0xffffffffu, incl, 31);
                unsigned long long pos = 0;
                if (wtot) pos = slots.take(wtot, sv, sv_fill, sv_cap, lane) + incl - mine;
                if (mine) {  // the survivors of the short range, from its mask
                    const unsigned long long ihi = (unsigned long long)s_id[k] << a.id_bits;
                    for (uint32_t mm = passmask; mm; mm &= mm - 1u) {
                        const uint32_t x = b0 + (uint32_t)(__ffs(mm) - 1);
                        if (pos < sv_cap) sv[pos] = ihi | c_id[x];
                        ++pos;
                    }
                }
            }
            unsigned todo = __ballot_sync(0xffffffffu, longr);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const uint32_t spl = __shfl_sync(0xffffffffu, pl, src);
                const uint32_t sph = __shfl_sync(0xffffffffu, ph, src);
                const uint32_t sb0 = __shfl_sync(0xffffffffu, b0, src);
                const uint32_t sb1 = __shfl_sync(0xffffffffu, b1, src);
                const uint32_t sid_src = __shfl_sync(0xffffffffu, k < ns ? s_id[k] : 0u, src);
                uint32_t scur = __shfl_sync(0xffffffffu, cur, src);
                uint2 sown[NK];
#pragma unroll
                for (int q = 0; q < NK; ++q) {
                    if (q < dd) {
                        sown[q].x = __shfl_sync(0xffffffffu, own[q].x, src);
                        sown[q].y = __shfl_sync(0xffffffffu, own[q].y, src);
                    }
                }
                int2* sseg = nullptr;
                uint32_t sc = 0, sj = 0;
                int32_t si = 0;
                if (WRITE) {
                    sseg = reinterpret_cast<int2*>(a.pairs) + __shfl_sync(0xffffffffu, obase, src);
                    sc = __shfl_sync(0xffffffffu, c, src);
                    si = __shfl_sync(0xffffffffu, i_out, src);
                    sj = __shfl_sync(0xffffffffu, j_base, src);
                }
                for (uint32_t base = sb0; base < sb1; base += 32) {
                    const uint32_t x = base + lane;
                    const bool inr = x < sb1;
                    const uint32_t xx = inr ? x : sb0;
                    const uint2 p = c_pos[xx];
                    bool pass = inr & (p.x < sph) & (p.y > spl);
#pragma unroll
                    for (int q = 0; q < NK; ++q) {
                        if (q < dd) {
                            const uint2 u = c_key[q * JOIN_CHUNK + xx];
                            pass &= (sown[q].x <= u.y) & (u.x <= sown[q].y);
                        }
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, pass);
                    if (rec_surv && bal) {
                        const unsigned long long b =
                            slots.take((uint32_t)__popc(bal), sv, sv_fill, sv_cap, lane) +
                            __popc(bal & ((1u << lane) - 1u));
                        if (pass && b < sv_cap)
                            sv[b] = ((unsigned long long)sid_src << a.id_bits) | c_id[xx];
                    }
                    if (WRITE) {
                        const uint32_t r = scur + __popc(bal & ((1u << lane) - 1u));
                        if (pass && r < sc) sseg[r] = make_int2(si, (int32_t)(c_id[xx] - sj));
                    }
                    scur += __popc(bal);
                }
                if (lane == src) cur = scur;
            }
            if (act) s_cnt[k] = cur;
        }
        __syncthreads();
    }
    if (rec_surv) slots.pad(sv, sv_cap, lane);
    for (uint32_t k = tid; k < ns; k += JOIN_BLOCK) {
        const uint32_t i = s_id[k];
        if (!WRITE) a.cnt[i] = s_cnt[k];
        else if (s_cnt[k] != a.cnt[i]) raise_error(st, DDM_ERR_INTERNAL, 17);
    }
}

// One instantiation: sets its dynamic shared-memory limit once per device.
template <bool WRITE, int DD>
static void launch_join_t(const EmitArgs& a, size_t smem, DevStatus* st, cudaStream_t s) {
    static std::atomic<unsigned long long> attr_set{0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !(attr_set.load() & (1ull << dev))) {
        cudaFuncSetAttribute(k_join<WRITE, DD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)join_smem_bytes(DDM_MAX_DIMS));
        if (dev >= 0 && dev < 64) attr_set.fetch_or(1ull << dev);
    }
    launch_k(k_join<WRITE, DD>, a.num_win, JOIN_BLOCK, smem, s, a, st);
}

template <bool WRITE>
static void launch_join_w(const EmitArgs& a, size_t smem, DevStatus* st, cudaStream_t s) {
    switch (a.d - 1) {
        case 1: launch_join_t<WRITE, 1>(a, smem, st, s); break;
        case 2: launch_join_t<WRITE, 2>(a, smem, st, s); break;
        case 3: launch_join_t<WRITE, 3>(a, smem, st, s); break;
        default: launch_join_t<WRITE, 0>(a, smem, st, s); break;
    }
}

// Window w's used entries (its fill, holes included) moved to dst[pos[w] ..).
__global__ void k_surv_compact(const unsigned long long* __restrict__ surv,
                               const unsigned long long* __restrict__ fill,
                               const uint4* __restrict__ windows, unsigned long long per_sub,
                               const unsigned long long* __restrict__ pos,
                               unsigned long long* __restrict__ dst) {
    pdl_begin();
    const uint32_t w = blockIdx.x;
    const unsigned long long* src = surv + (uint64_t)windows[w].x * per_sub;
    unsigned long long* out = dst + pos[w];
    const unsigned long long f = fill[w];
    for (uint64_t q = threadIdx.x; q < f; q += blockDim.x) out[q] = src[q];
}

int launch_surv_compact(const unsigned long long* surv, const unsigned long long* fill,
                        const uint4* windows, uint32_t num_win, unsigned long long per_sub,
                        const unsigned long long* pos, unsigned long long* dst, cudaStream_t s) {
    if (num_win == 0) return 0;
    launch_k(k_surv_compact, num_win, 256, 0, s, surv, fill, windows, per_sub, pos, dst);
    return 1;
}

int launch_join(const EmitArgs& a, bool write, DevStatus* st, cudaStream_t s) {
    if (a.num_win == 0 || a.n == 0) return 0;
    if (a.win_shift > JOIN_SHIFT) return -1;  // shared memory holds at most 2^JOIN_SHIFT subs
    const size_t smem = join_smem_bytes(a.d);
    if (write) launch_join_w<true>(a, smem, st, s);
    else launch_join_w<false>(a, smem, st, s);
    return 1;
}

}  // namespace ddm
