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
#include "emit.cuh"

namespace ddm {

constexpr int JOIN_BLOCK = 512;
constexpr int JOIN_WARPS = JOIN_BLOCK / 32;
constexpr uint32_t JOIN_CHUNK = 512;
constexpr int JOIN_SHIFT = 11;  // windows of 2048 stream positions
constexpr uint32_t JOIN_MAXSUB = 1u << JOIN_SHIFT;

// Dynamic shared memory of one join block for d dimensions.
__host__ __device__ inline size_t join_smem_bytes(int d) {
    return (size_t)JOIN_MAXSUB * sizeof(unsigned long long)   // sub output offsets
           + (size_t)JOIN_MAXSUB * 5 * sizeof(uint32_t)         // sub lo, hi, id, count, expected
           + (size_t)(d - 1) * JOIN_MAXSUB * sizeof(uint2)      // sub keys, dims 1..d-1
           + (size_t)JOIN_CHUNK * (sizeof(uint2) + sizeof(uint32_t))  // candidate pos, id
           + (size_t)(d - 1) * JOIN_CHUNK * sizeof(uint2)       // candidate keys, dims 1..d-1
           + 64;
}

// Range [b0, b1) of the sorted chunk keys sk[0..JOIN_CHUNK) with lo <= key <= hi,
// found by one warp: a coarse ballot over the last key of each 16-entry
// segment (coarse[g] = sk[16 g + 15]) for both bounds at once, then a fine
// ballot inside the two segments (lanes 0-15 for the lower bound, 16-31 for
// the upper).
__device__ __forceinline__ void chunk_range(const uint32_t* sk, const uint32_t* coarse, uint32_t lo,
                                            uint32_t hi, int lane, uint32_t& b0, uint32_t& b1) {
    static_assert(JOIN_CHUNK == 32 * 16, "two-level search assumes 32 segments of 16");
    const uint32_t kc = coarse[lane];
    const uint32_t g0 = __popc(__ballot_sync(0xffffffffu, kc < lo));   // segments all < lo
    const uint32_t g1 = __popc(__ballot_sync(0xffffffffu, kc <= hi));  // segments all <= hi
    const int l = lane & 15;
    const uint32_t g = lane < 16 ? g0 : g1;
    const uint32_t kf = g < 32 ? sk[g * 16 + l] : 0xffffffffu;
    const unsigned f0 = __ballot_sync(0xffffffffu, lane < 16 && g0 < 32 && kf < lo);
    const unsigned f1 = __ballot_sync(0xffffffffu, lane >= 16 && g1 < 32 && kf <= hi);
    b0 = g0 < 32 ? g0 * 16 + __popc(f0) : JOIN_CHUNK;
    b1 = g1 < 32 ? g1 * 16 + __popc(f1) : JOIN_CHUNK;
}

template <bool WRITE>
__global__ void __launch_bounds__(JOIN_BLOCK) k_join(EmitArgs a, DevStatus* st) {
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
    __shared__ uint32_t c_coarse[32];                 // c_sk[16 g + 15]
    __shared__ uint32_t s_wmax[JOIN_WARPS];
    __shared__ uint32_t s_pmax, s_first;

    if (read_error(st)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t w = blockIdx.x;
    const int S = a.win_shift;
    const int dd = a.d - 1;
    const uint4 t0 = a.windows[w], t1 = a.windows[w + 1];
    const uint32_t r0 = t0.x, ns = t1.x - t0.x;
    if (ns == 0) return;
    if (ns > JOIN_MAXSUB) {
        if (tid == 0) raise_error(st, DDM_ERR_INTERNAL, 16);
        return;
    }
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
            for (int q = 0; q < DDM_MAX_DIMS - 1; ++q)
                if (q < dd) kq[q] = c_key[q * JOIN_CHUNK + x];
            __syncthreads();
            c_pos[tid] = p;
            c_id[tid] = id;
#pragma unroll
            for (int q = 0; q < DDM_MAX_DIMS - 1; ++q)
                if (q < dd) c_key[q * JOIN_CHUNK + tid] = kq[q];
            const uint32_t key = (uint32_t)(e >> 32);
            c_sk[tid] = key;
            if ((tid & 15) == 15) c_coarse[tid >> 4] = key;
        }
        __syncthreads();
        uint32_t maxbits = 0;
#pragma unroll
        for (int q = 0; q < JOIN_WARPS; ++q) maxbits = max(maxbits, s_wmax[q]);
        const float maxlen = __uint_as_float(maxbits);
        const uint32_t first = s_first;
        for (uint32_t k = warp; k < ns; k += JOIN_WARPS) {
            const uint32_t pl = s_lo[k], ph = s_hi[k];
            if (c0 >= lw_n && first >= ph) continue;  // every later candidate starts after S ends
            uint2 own[DDM_MAX_DIMS - 1];
#pragma unroll
            for (int q = 0; q < DDM_MAX_DIMS - 1; ++q)
                if (q < dd) own[q] = s_key[q * JOIN_MAXSUB + k];
            // candidates whose dimension-1 lower bound lies in [own.lo - maxlen, own.hi]
            const float bound = __fsub_rd(key_float(own[0].x), maxlen);
            const uint32_t lo_b = bound == bound ? float_key(bound) : 0u;  // NaN: inf - inf
            uint32_t b0, b1;
            chunk_range(c_sk, c_coarse, lo_b, own[0].y, lane, b0, b1);
            if (b0 >= b1) continue;
            const uint32_t i = s_id[k];
            uint32_t cur = s_cnt[k];
            int2* seg = nullptr;
            uint32_t c = 0;
            int32_t i_out = (int32_t)i;
            uint32_t j_base = 0;
            if (WRITE) {
                seg = reinterpret_cast<int2*>(a.pairs) + s_off[k];
                c = s_exp[k];
                if (a.inst_sub_base) {
                    const int b = inst_of(a.inst_sub_base, a.num_inst, i);
                    i_out -= (int32_t)a.inst_sub_base[b];
                    j_base = (uint32_t)a.inst_upd_base[b];
                }
            }
            for (uint32_t base = b0; base < b1; base += 32) {
                const uint32_t kk = base + lane;
                const bool inr = kk < b1;
                const uint32_t x = inr ? kk : 0u;
                const uint2 p = c_pos[x];
                bool pass = inr & (p.x < ph) & (p.y > pl);
#pragma unroll
                for (int q = 0; q < DDM_MAX_DIMS - 1; ++q) {
                    if (q < dd) {
                        const uint2 u = c_key[q * JOIN_CHUNK + x];
                        pass &= (own[q].x <= u.y) & (u.x <= own[q].y);
                    }
                }
                const unsigned bal = __ballot_sync(0xffffffffu, pass);
                if (WRITE) {
                    const uint32_t r = cur + __popc(bal & lt);
                    if (pass && r < c) seg[r] = make_int2(i_out, (int32_t)(c_id[x] - j_base));
                }
                cur += __popc(bal);
            }
            if (lane == 0) s_cnt[k] = cur;
        }
        __syncthreads();
    }
    for (uint32_t k = tid; k < ns; k += JOIN_BLOCK) {
        const uint32_t i = s_id[k];
        if (!WRITE) a.cnt[i] = s_cnt[k];
        else if (s_cnt[k] != a.cnt[i]) raise_error(st, DDM_ERR_INTERNAL, 17);
    }
}

int launch_join(const EmitArgs& a, bool write, DevStatus* st, cudaStream_t s) {
    if (a.num_win == 0 || a.n == 0) return 0;
    if (a.win_shift != JOIN_SHIFT) return -1;
    const size_t smem = join_smem_bytes(a.d);
    static unsigned long long attr_set[2] = {0, 0};  // per device, per pass
    int dev = 0;
    cudaGetDevice(&dev);
    const int w = write ? 1 : 0;
    if (dev < 0 || dev >= 64 || !(attr_set[w] & (1ull << dev))) {
        const size_t max_smem = join_smem_bytes(DDM_MAX_DIMS);
        if (write)
            cudaFuncSetAttribute(k_join<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
        else
            cudaFuncSetAttribute(k_join<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
        if (dev >= 0 && dev < 64) attr_set[w] |= 1ull << dev;
    }
    if (write) launch_k(k_join<true>, a.num_win, JOIN_BLOCK, smem, s, a, st);
    else launch_k(k_join<false>, a.num_win, JOIN_BLOCK, smem, s, a, st);
    return 1;
}

}  // namespace ddm
