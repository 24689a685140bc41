// Incremental matching for served sessions: the pairs that appeared and the
// pairs that disappeared since the last delivered report.
//
// Paper: Section 6 names dynamic DDM (regions that move between timesteps) as
// future work; SBM itself recomputes the full match.  Here nothing is
// recomputed in full.  By Algorithm 1 and Section 3 a pair intersects iff the
// 2d comparisons c1(k) = [U.lo_k <= S.hi_k] and c2(k) = [S.lo_k <= U.hi_k] all
// hold, so its status can change only if one of them changes.  If a
// comparison between endpoints a and b changed, then, with every endpoint of
// dimension k displaced by at most D_k, the two are now at most 2 D_k apart
// (a <= b before and a > b now give 0 < a' - b' <= (a' - a) - (b' - b)).  So
// the candidates of comparison (k, t) of S_i are the update bounds within
// 2 D_k of S_i's bound: for dimension 0 a walk among the update bounds of
// the one kind the comparison involves (c1: lowers, c2: uppers), kept in
// stream order from the sorted endpoint stream that the count phase has just
// produced and entered where the count phase's rank records place S_i's bound
// (subscription bounds taken in stream order, so neighbouring threads walk
// neighbouring ranges); for the other dimensions a binary search in the
// updates' bounds sorted per dimension.  A candidate is
// kept if its predicate differs between the reference and the current
// coordinates and (k, t) is the first of its comparisons, in the order
// c1(0), c2(0), c1(1), ..., that changed: each changed pair is found exactly
// once.
#include <algorithm>

#include "delta.cuh"

namespace ddm {

constexpr int DELTA_BLOCK = 256;
constexpr int DELTA_WALK = 4;  // entries read together per step of a neighbourhood walk

// |now - ref| along one bound; 0 when the value did not change (which also
// covers an infinite bound that stays infinite).
// Rounded up, so an upper bound of the exact distance (single precision with
// directed rounding: the radii below stay supersets of the exact ones).
__device__ __forceinline__ float moved(float now, float ref) {
    return now == ref ? 0.f : __fsub_ru(fmaxf(now, ref), fminf(now, ref));
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// Non-negative floats order like their bit patterns, so the maximum is kept
// as an integer maximum of the bits (in the low 32 bits of disp[k]).
__global__ void k_delta_disp(DeltaArgs a, DevStatus* st) {
    pdl_begin();
    if (read_error(st)) return;
    const uint64_t per_dim = 2ull * (a.n + a.m);
    for (int k = 1; k < a.d; ++k) {  // dimension 0: k_delta_refk
        float mx = 0.f;
        for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < per_dim;
             e += (uint64_t)gridDim.x * blockDim.x) {
            const bool upd = e >= 2ull * a.n;
            const uint64_t q = upd ? e - 2ull * a.n : e;
            const uint32_t cnt = upd ? a.m : a.n;
            const bool hi = q >= cnt;
            const uint32_t id = (uint32_t)(hi ? q - cnt : q);
            const float* pn = upd ? (hi ? a.now.upd_hi[k] : a.now.upd_lo[k])
                                  : (hi ? a.now.sub_hi[k] : a.now.sub_lo[k]);
            const float* pr = upd ? (hi ? a.ref.upd_hi[k] : a.ref.upd_lo[k])
                                  : (hi ? a.ref.sub_hi[k] : a.ref.sub_lo[k]);
            mx = fmaxf(mx, moved(pn[id], pr[id]));  // fmaxf drops a NaN (never produced)
        }
        const unsigned long long b = warp_max_u64((unsigned long long)__float_as_uint(mx));
        if ((threadIdx.x & 31) == 0 && b) atomicMax(&a.disp[k], b);
    }
}

int launch_delta_disp(const DeltaArgs& a, DevStatus* st, cudaStream_t s) {
    if (a.d < 2) return 0;
    uint64_t g = ceil_div(2ull * (a.n + a.m), DELTA_BLOCK);
    g = g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g);
    launch_k(k_delta_disp, (unsigned)g, DELTA_BLOCK, 0, s, a, st);
    return 1;
}

__global__ void k_delta_keys(DeltaArgs a) {
    pdl_begin();
    const uint64_t total = (uint64_t)(a.d - 1) * a.m;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const int k = 1 + (int)(e / a.m);
        const uint32_t j = (uint32_t)(e % a.m);
        const_cast<uint32_t*>(a.lo_key[k - 1])[j] = float_key(a.now.upd_lo[k][j]);
        const_cast<uint32_t*>(a.lo_id[k - 1])[j] = j;
        const_cast<uint32_t*>(a.hi_key[k - 1])[j] = float_key(a.now.upd_hi[k][j]);
        const_cast<uint32_t*>(a.hi_id[k - 1])[j] = j;
    }
}

int launch_delta_keys(const DeltaArgs& a, cudaStream_t s) {
    if (a.d < 2 || a.m == 0) return 0;
    uint64_t g = ceil_div((uint64_t)(a.d - 1) * a.m, DELTA_BLOCK);
    g = g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g);
    launch_k(k_delta_keys, (unsigned)g, DELTA_BLOCK, 0, s, a);
    return 1;
}

// Per dimension-0 stream position: the current key, the reference key of the
// same endpoint (one gather per endpoint) and the payload, packed; and the
// largest displacement along dimension 0 (disp[0]).  An update bound also goes
// to the stream of its kind at its rank among that kind (its rank record: w of
// a lower, z of an upper), with its update's other bound, so that a walk needs
// no gather by id; a subscription bound records where its walk starts in the
// stream of the other kind: the update lowers before it (an upper's y) or the
// update uppers before it (a lower's z).
__global__ void k_delta_refk(DeltaArgs a, uint4* __restrict__ pk) {
    pdl_begin();
    float mx = 0.f;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < a.E; p += gridDim.x * blockDim.x) {
        const uint32_t v = a.vals[p], kind = v >> 30, id = v & ID_MASK, key = a.keys[p];
        const float* src = kind == KIND_SLO ? a.ref.sub_lo[0] : kind == KIND_ULO ? a.ref.upd_lo[0]
                         : kind == KIND_SHI ? a.ref.sub_hi[0] : a.ref.upd_hi[0];
        const uint4* rec = kind == KIND_SLO ? a.rec.s_lo : kind == KIND_ULO ? a.rec.u_lo
                         : kind == KIND_SHI ? a.rec.s_hi : a.rec.u_hi;
        const float r = src[id];
        const uint4 rr = rec[id];
        const uint32_t rk = float_key(r);
        uint32_t start = 0;
        if (kind == KIND_SLO) start = rr.z;       // update uppers before S.lo
        else if (kind == KIND_SHI) start = rr.y;  // update lowers before S.hi
        else if ((kind == KIND_ULO && rr.w < a.m) || (kind == KIND_UHI && rr.z < a.m)) {
            const bool lo = kind == KIND_ULO;
            const uint32_t on = float_key(lo ? a.now.upd_hi[0][id] : a.now.upd_lo[0][id]);
            const uint32_t orf = float_key(lo ? a.ref.upd_hi[0][id] : a.ref.upd_lo[0][id]);
            uint4* const dst = lo ? a.ulo + 2ull * rr.w : a.uhi + 2ull * rr.z;
            dst[0] = make_uint4(key, rk, id, 0u);
            dst[1] = make_uint4(on, orf, 0u, 0u);
        }
        pk[p] = make_uint4(key, rk, v, start);
        mx = fmaxf(mx, moved(key_float(key), r));
    }
    const unsigned long long b = warp_max_u64((unsigned long long)__float_as_uint(mx));
    if ((threadIdx.x & 31) == 0 && b) atomicMax(&a.disp[0], b);
}

int launch_delta_refk(const DeltaArgs& a, uint4* pk, cudaStream_t s) {
    if (a.E == 0) return 0;
    uint64_t g = ceil_div((uint64_t)a.E, DELTA_BLOCK);
    g = g > 152 * 16 ? 152 * 16 : g;
    launch_k(k_delta_refk, (unsigned)g, DELTA_BLOCK, 0, s, a, pk);
    return 1;
}

// Comparison q = 2k + t of the pair (i, j) in the coordinates c: t = 0 is
// c1(k) = [U.lo_k <= S.hi_k], t = 1 is c2(k) = [S.lo_k <= U.hi_k].
__device__ __forceinline__ bool cmp_q(const DimPtrs& c, int q, uint32_t i, uint32_t j) {
    const int k = q >> 1;
    return (q & 1) ? float_key(c.sub_lo[k][i]) <= float_key(c.upd_hi[k][j])
                   : float_key(c.upd_lo[k][j]) <= float_key(c.sub_hi[k][i]);
}

// (i, j), whose comparison q changed, is kept if no earlier comparison changed
// and its predicate (all 2d comparisons) differs between reference and now;
// returns 0 (not kept), 1 (appeared) or 2 (disappeared).
__device__ __forceinline__ int first_change(const DeltaArgs& a, int q, uint32_t i, uint32_t j) {
    for (int q2 = 0; q2 < q; ++q2)
        if (cmp_q(a.ref, q2, i, j) != cmp_q(a.now, q2, i, j)) return 0;  // found through q2
    bool pr = true, pn = true;
    for (int q2 = 0; q2 < 2 * a.d && (pr || pn); ++q2) {
        pr = pr && cmp_q(a.ref, q2, i, j);
        pn = pn && cmp_q(a.now, q2, i, j);
    }
    return pr == pn ? 0 : (pn ? 1 : 2);
}

// A lane's changed pairs: the first DELTA_LANE_KEYS are held in registers and
// written after a warp-wide slot reservation; further ones take a slot each.
constexpr int DELTA_LANE_KEYS = 4;

struct LaneKeys {
    unsigned long long k[DELTA_LANE_KEYS];
    int nb = 0;
    unsigned long long n_add = 0, n_rem = 0;

    __device__ __forceinline__ void put(const DeltaArgs& a, int kind, uint32_t i, uint32_t j) {
        const unsigned long long which = kind == 1 ? 0ull : 1ull;
        (kind == 1 ? n_add : n_rem) += 1;
        const unsigned long long key =
            (which << (a.ibits + a.jbits)) | ((unsigned long long)i << a.jbits) | j;
        if (nb < DELTA_LANE_KEYS) {
#pragma unroll
            for (int q = 0; q < DELTA_LANE_KEYS; ++q)
                if (q == nb) k[q] = key;  // register-resident (no dynamic index)
            ++nb;
            return;
        }
        const unsigned long long slot = atomicAdd(&a.counters[2], 1ull);
        if (slot < a.cap) a.keys_out[slot] = key;
    }

    // Called by all 32 lanes of the warp together: the warp's keys into the
    // block's shared buffer (one shared atomic per warp); what does not fit
    // takes global slots directly.
    __device__ __forceinline__ void stage(const DeltaArgs& a, int lane, unsigned long long* sbuf,
                                          uint32_t* scnt, uint32_t scap) {
        uint32_t incl = (uint32_t)nb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        if (total == 0) return;
        uint32_t base = 0;
        if (lane == 31) base = atomicAdd(scnt, total);
        base = __shfl_sync(0xffffffffu, base, 31) + (incl - (uint32_t)nb);
#pragma unroll
        for (int q = 0; q < DELTA_LANE_KEYS; ++q) {
            if (q >= nb) break;
            if (base + q < scap) {
                sbuf[base + q] = k[q];
            } else {
                const unsigned long long slot = atomicAdd(&a.counters[2], 1ull);
                if (slot < a.cap) a.keys_out[slot] = k[q];
            }
        }
        nb = 0;
    }

    // Called by all 32 lanes of the warp together.
    __device__ __forceinline__ void flush(const DeltaArgs& a, int lane) {
        uint32_t incl = (uint32_t)nb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        if (total == 0) return;
        unsigned long long base = 0;
        if (lane == 31) base = atomicAdd(&a.counters[2], (unsigned long long)total);
        base = __shfl_sync(0xffffffffu, base, 31) + (incl - (uint32_t)nb);
#pragma unroll
        for (int q = 0; q < DELTA_LANE_KEYS; ++q)
            if (q < nb && base + q < a.cap) a.keys_out[base + q] = k[q];
        nb = 0;
    }
};

// Keys of the values within r of x (a superset: bounds rounded outwards;
// everything when r is not finite).
__device__ __forceinline__ void key_window(float x, float r, uint32_t& klo, uint32_t& khi) {
    if (!(r < INFINITY)) {
        klo = 0u;
        khi = 0xffffffffu;
        return;
    }
    const float lo = __fsub_rd(x, r), hi = __fadd_ru(x, r);
    klo = lo != lo ? 0u : float_key(lo);            // x infinite: a NaN cannot arise,
    khi = hi != hi ? 0xffffffffu : float_key(hi);   // kept for safety
}

__device__ __forceinline__ float disp_of(const DeltaArgs& a, int k) {
    return __uint_as_float((uint32_t)a.disp[k]);
}

// Dimension k >= 1: two endpoints whose comparison changed are now at most
// 2 D_k apart.
__device__ __forceinline__ float radius(const DeltaArgs& a, int k) {
    return __fmul_ru(2.f, disp_of(a, k));
}

// Dimension 0: the stream positions, 64 per warp step; the subscription
// bounds among them are handed out to the lanes (ballots), and each walks its
// neighbourhood in the stream of the update bounds it is compared with (c1 of
// an S upper: update lowers; c2 of an S lower: update uppers), testing them
// with the keys alone (current and reference keys, packed).  Dimensions
// k >= 1: items (k, t, i), 32 per warp step, by binary search.  The lanes of a
// warp reserve their output slots together.
__global__ void __launch_bounds__(DELTA_BLOCK) k_delta_cand(DeltaArgs a, DevStatus* st) {
    pdl_begin();
    if (read_error(st)) return;
    constexpr uint32_t SBUF = 2048;  // keys staged per block iteration
    __shared__ unsigned long long sbuf[SBUF];
    __shared__ uint32_t scnt;
    __shared__ unsigned long long sbase;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t warp_id = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    LaneKeys out;
    const float D0 = disp_of(a, 0);
    if (threadIdx.x == 0) scnt = 0;
    __syncthreads();
    // A block takes 8 x 64 stream positions per iteration (the same number of
    // iterations for all its warps), stages their keys in shared memory and
    // reserves global slots for all of them with one atomic.
    constexpr uint32_t CHUNK = (DELTA_BLOCK / 32) * 64;
    for (uint64_t cbase = (uint64_t)blockIdx.x * CHUNK; cbase < a.E;
         cbase += (uint64_t)gridDim.x * CHUNK) {
      const uint64_t base = cbase + (uint64_t)warp * 64;
      if (base < a.E) {
        const uint64_t p0 = base + lane, p1 = base + 32 + lane;
        const uint32_t k0 = p0 < a.E ? a.pk[p0].z >> 30 : KIND_ULO;
        const uint32_t k1 = p1 < a.E ? a.pk[p1].z >> 30 : KIND_ULO;
        const unsigned m0 = __ballot_sync(0xffffffffu, k0 == KIND_SHI || k0 == KIND_SLO);
        const unsigned m1 = __ballot_sync(0xffffffffu, k1 == KIND_SHI || k1 == KIND_SLO);
        const int c0 = __popc(m0), tot = c0 + __popc(m1);
        for (int r0 = 0; r0 < tot; r0 += 32) {  // up to 64 items: one or two rounds
          const int it = r0 + lane;
          if (it < tot) {
            // Lane l takes item r0 + l: the (r0 + l)-th subscription bound of the
            // 64 positions.
            unsigned mm = it < c0 ? m0 : m1;
            for (int t = it < c0 ? it : it - c0; t > 0; --t) mm &= mm - 1u;
            const uint64_t pos = base + (it < c0 ? 0 : 32) + (uint32_t)(__ffs(mm) - 1);
            const uint32_t p = (uint32_t)pos;
            const uint4 ep = a.pk[p < a.E ? p : 0];  // mm != 0 and p < E by construction
            const uint32_t kind = ep.z >> 30;
            const bool t0 = kind == KIND_SHI;           // c1: U lowers near S.hi
            const uint4* const ws = t0 ? a.ulo : a.uhi;  // c2: U uppers near S.lo
            const uint32_t i = ep.z & ID_MASK, kp = ep.x, rp = ep.y;
            const uint32_t start = ep.w < a.m ? ep.w : a.m;
            // The walk covers every update bound within |d_p| + D of this bound:
            // a changed comparison needs |now_q - now_p| <= |d_q - d_p| <= D + |d_p|.
            const float xp = key_float(kp);
            const float dp = moved(xp, key_float(rp));
            const float rad = D0 == 0.f ? 0.f : __fadd_ru(D0, dp);
            uint32_t klo, khi;
            key_window(xp, rad, klo, khi);
            // This subscription's other bound along dimension 0, loaded together
            // with the walk's first entries (most lanes meet a changed comparison).
            const uint32_t ko_now = float_key(t0 ? a.now.sub_lo[0][i] : a.now.sub_hi[0][i]);
            const uint32_t ko_ref = float_key(t0 ? a.ref.sub_lo[0][i] : a.ref.sub_hi[0][i]);
            auto test = [&](const uint4 eq, const uint4 eo) {
                const bool now = t0 ? eq.x <= kp : kp <= eq.x;
                const bool ref = t0 ? eq.y <= rp : rp <= eq.y;
                if (now == ref) return;
                const uint32_t j = eq.z;
                // The update's other bound, now and then (carried by the entry).
                const uint32_t uo_now = eo.x, uo_ref = eo.y;
                // c1 = [U.lo <= S.hi], c2 = [S.lo <= U.hi] along dimension 0.
                const bool c1n = t0 ? now : uo_now <= ko_now;
                const bool c1r = t0 ? ref : uo_ref <= ko_ref;
                const bool c2n = t0 ? ko_now <= uo_now : now;
                const bool c2r = t0 ? ko_ref <= uo_ref : ref;
                if (!t0 && c1n != c1r) return;  // found through c1(0)
                bool pn = c1n && c2n, pr = c1r && c2r;
                for (int q2 = 2; q2 < 2 * a.d && (pr || pn); ++q2) {
                    pr = pr && cmp_q(a.ref, q2, i, j);
                    pn = pn && cmp_q(a.now, q2, i, j);
                }
                if (pr != pn) out.put(a, pn ? 1 : 2, i, j);
            };
            // The update bounds of the wanted kind in stream order: those before
            // this bound end at `start`.  Each side is read DELTA_WALK entries at a
            // time (one round trip for the usual few entries within the radius).
            for (uint32_t q = start; q > 0;) {
                const uint32_t nq = q < DELTA_WALK ? q : DELTA_WALK;
                uint4 e4[DELTA_WALK], o4[DELTA_WALK];
#pragma unroll
                for (int u = 0; u < DELTA_WALK; ++u) {
                    const uint64_t at = 2ull * (q - 1 - u);
                    e4[u] = (uint32_t)u < nq ? ws[at] : make_uint4(0u, 0u, 0u, 0u);
                    o4[u] = (uint32_t)u < nq ? ws[at + 1] : make_uint4(0u, 0u, 0u, 0u);
                }
                bool stop = false;
#pragma unroll
                for (int u = 0; u < DELTA_WALK; ++u) {
                    if (stop || (uint32_t)u >= nq) continue;
                    if (e4[u].x < klo) stop = true;
                    else test(e4[u], o4[u]);
                }
                if (stop) break;
                q -= nq;
            }
            for (uint32_t q = start; q < a.m;) {
                const uint32_t nq = a.m - q < DELTA_WALK ? a.m - q : DELTA_WALK;
                uint4 e4[DELTA_WALK], o4[DELTA_WALK];
#pragma unroll
                for (int u = 0; u < DELTA_WALK; ++u) {
                    const uint64_t at = 2ull * (q + u);
                    e4[u] = (uint32_t)u < nq ? ws[at] : make_uint4(0u, 0u, 0u, 0u);
                    o4[u] = (uint32_t)u < nq ? ws[at + 1] : make_uint4(0u, 0u, 0u, 0u);
                }
                bool stop = false;
#pragma unroll
                for (int u = 0; u < DELTA_WALK; ++u) {
                    if (stop || (uint32_t)u >= nq) continue;
                    if (e4[u].x > khi) stop = true;
                    else test(e4[u], o4[u]);
                }
                if (stop) break;
                q += nq;
            }
          }
          out.stage(a, lane, sbuf, &scnt, SBUF);
        }
      }
      __syncthreads();
      const uint32_t ns = scnt < SBUF ? scnt : SBUF;
      if (threadIdx.x == 0) sbase = ns ? atomicAdd(&a.counters[2], (unsigned long long)ns) : 0ull;
      __syncthreads();
      for (uint32_t q = threadIdx.x; q < ns; q += DELTA_BLOCK)
          if (sbase + q < a.cap) a.keys_out[sbase + q] = sbuf[q];
      __syncthreads();
      if (threadIdx.x == 0) scnt = 0;
      __syncthreads();
    }
    (void)warp_id;
    (void)warps;
    const uint64_t other = 2ull * (a.d - 1) * a.n;
    for (uint64_t base = warp_id * 32; base < other; base += warps * 32) {
        const uint64_t r = base + lane;
        if (r < other) {
            const int k = 1 + (int)(r / (2ull * a.n));
            const int t = (int)((r / a.n) & 1);
            const uint32_t i = (uint32_t)(r % a.n);
            const uint32_t* key = t == 0 ? a.lo_key[k - 1] : a.hi_key[k - 1];
            const uint32_t* id = t == 0 ? a.lo_id[k - 1] : a.hi_id[k - 1];
            uint32_t klo, khi;
            key_window(t == 0 ? a.now.sub_hi[k][i] : a.now.sub_lo[k][i], radius(a, k), klo, khi);
            uint32_t lo = 0, hi = a.m;  // first key >= klo
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (key[mid] < klo) lo = mid + 1;
                else hi = mid;
            }
            for (uint32_t q = lo; q < a.m && key[q] <= khi; ++q) {
                const uint32_t j = id[q];
                if (cmp_q(a.ref, 2 * k + t, i, j) == cmp_q(a.now, 2 * k + t, i, j)) continue;
                const int c = first_change(a, 2 * k + t, i, j);
                if (c) out.put(a, c, i, j);
            }
        }
        out.flush(a, lane);
    }
    // The counts, one atomic per warp and kind.
    unsigned long long na = out.n_add, nr = out.n_rem;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        na += __shfl_xor_sync(0xffffffffu, na, o);
        nr += __shfl_xor_sync(0xffffffffu, nr, o);
    }
    if (lane == 0) {
        if (na) atomicAdd(&a.counters[0], na);
        if (nr) atomicAdd(&a.counters[1], nr);
    }
}

int launch_delta_cand(const DeltaArgs& a, DevStatus* st, cudaStream_t s) {
    const uint64_t warps_needed =
        std::max<uint64_t>(ceil_div(a.E, 64), ceil_div(2ull * (a.d - 1) * a.n, 32));
    if (warps_needed == 0) return 0;
    uint64_t g = ceil_div(warps_needed, DELTA_BLOCK / 32);
    g = g > 152 * 16 ? 152 * 16 : g;
    launch_k(k_delta_cand, (unsigned)g, DELTA_BLOCK, 0, s, a, st);
    return 1;
}

// Sorted pair keys (i << jbits) | j into interleaved int32 pairs.
__global__ void k_keys_unpack(const unsigned long long* __restrict__ keys, uint64_t count,
                              int jbits, int2* __restrict__ pairs) {
    pdl_begin();
    const unsigned long long mask = (1ull << jbits) - 1ull;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[q];
        pairs[q] = make_int2((int32_t)(k >> jbits), (int32_t)(k & mask));
    }
}

int launch_delta_unpack(const unsigned long long* keys, uint64_t count, int jbits, int32_t* pairs,
                        cudaStream_t s) {
    if (count == 0) return 0;
    uint64_t g = ceil_div(count, DELTA_BLOCK);
    g = g > 152 * 16 ? 152 * 16 : g;
    launch_k(k_keys_unpack, (unsigned)g, DELTA_BLOCK, 0, s, keys, count, jbits,
             reinterpret_cast<int2*>(pairs));
    return 1;
}

__global__ void k_delta_pad(DeltaArgs a) {
    pdl_begin();
    const unsigned long long used = a.counters[2];
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < a.cap;
         q += (uint64_t)gridDim.x * blockDim.x)
        if (q >= used) a.keys_out[q] = ~0ull;
}

int launch_delta_pad(const DeltaArgs& a, cudaStream_t s) {
    if (a.cap == 0) return 0;
    uint64_t g = ceil_div(a.cap, DELTA_BLOCK);
    g = g > 152 * 8 ? 152 * 8 : g;
    launch_k(k_delta_pad, (unsigned)g, DELTA_BLOCK, 0, s, a);
    return 1;
}

__global__ void k_delta_finish(DeltaArgs a, const unsigned long long* __restrict__ sorted,
                               int2* __restrict__ added, uint64_t cap_added,
                               int2* __restrict__ removed, uint64_t cap_removed,
                               uint32_t* flags, float* __restrict__ ref_coords,
                               const float* __restrict__ coords, uint64_t coord_count) {
    pdl_begin();
    const unsigned long long na = a.counters[0], nr = a.counters[1];
    uint32_t f = 0;
    if (na + nr > a.cap) f |= DELTA_RERUN;
    else if (na > cap_added || nr > cap_removed) f |= DELTA_CAPACITY;
    if (blockIdx.x == 0 && threadIdx.x == 0) flags[0] = f;
    if (f) return;
    const unsigned long long imask = (1ull << a.ibits) - 1ull, jmask = (1ull << a.jbits) - 1ull;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < na + nr; q += stride) {
        const unsigned long long k = sorted[q];
        const int2 pr = make_int2((int32_t)((k >> a.jbits) & imask), (int32_t)(k & jmask));
        if (q < na) added[q] = pr;
        else removed[q - na] = pr;
    }
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < coord_count; q += stride)
        ref_coords[q] = coords[q];  // the delivered report's coordinates: the next reference
}

int launch_delta_finish(const DeltaArgs& a, const unsigned long long* sorted, int32_t* added,
                        uint64_t cap_added, int32_t* removed, uint64_t cap_removed,
                        uint32_t* flags, float* ref_coords, const float* coords,
                        uint64_t coord_count, cudaStream_t s) {
    const uint64_t work = std::max<uint64_t>(a.cap, coord_count);
    uint64_t g = ceil_div(work > 0 ? work : 1, DELTA_BLOCK);
    g = g > 152 * 8 ? 152 * 8 : g;
    launch_k(k_delta_finish, (unsigned)g, DELTA_BLOCK, 0, s, a, sorted,
             reinterpret_cast<int2*>(added), cap_added, reinterpret_cast<int2*>(removed),
             cap_removed, flags, ref_coords, coords, coord_count);
    return 1;
}

}  // namespace ddm
