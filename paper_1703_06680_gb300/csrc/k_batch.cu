// a8: batched matching of many independent instances in one pipeline pass.
//
// The instances are concatenated on the device (subscriptions of all
// instances first, then all updates, each instance's extents contiguous, ids
// made global by the instance base).  The dimension-0 sort key of an endpoint
// is (instance << 32) | key(coordinate): one LSD sort then groups the stream
// by instance and orders each instance's endpoints exactly as a plain call
// would, lowers before uppers at equal coordinates.  Stream positions of
// different instances never interleave, so the sweep scan, the rank counts
// and the emission need no segment flags: every count at a position of
// instance b already includes all of instances 0..b-1, and ranges such as
// upd_order[A_i .. B_i) stay inside the instance.  The emission writes ids
// local to the instance.
#include "batch.cuh"

namespace ddm {

// One pass per region: the instance's coordinates of every dimension into the
// concatenated arrays, and the instance-tagged dimension-0 keys in
// [S lo | U lo | S hi | U hi] layout (one instance search per region).
__global__ void k_keybuild_batch(BatchArgs b, unsigned long long* __restrict__ keys,
                                 uint32_t* __restrict__ vals, DevStatus* st) {
    pdl_begin();
    const int64_t R = b.n + b.m;
    bool bad = false;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R;
         r += (int64_t)gridDim.x * blockDim.x) {
        const bool upd = r >= b.n;
        const int64_t g = upd ? r - b.n : r;
        const int inst = inst_of(upd ? b.m_base : b.n_base, b.num, g);
        const int64_t local = g - (upd ? b.m_base[inst] : b.n_base[inst]);
        const InstPtrs& ip = b.table[inst];
        float lo = 0.f, hi = 0.f;
        for (int k = 0; k < b.d; ++k) {
            const float l = upd ? ip.upd_lo[k][local] : ip.sub_lo[k][local];
            const float h = upd ? ip.upd_hi[k][local] : ip.sub_hi[k][local];
            (upd ? b.upd_lo[k] : b.sub_lo[k])[g] = l;
            (upd ? b.upd_hi[k] : b.sub_hi[k])[g] = h;
            if (k == 0) {
                lo = l;
                hi = h;
            }
        }
        bad |= is_nan_bits(lo) || is_nan_bits(hi) || !(lo <= hi);
        const unsigned long long tag = (unsigned long long)inst << 32;
        keys[r] = tag | float_key(lo);
        keys[R + r] = tag | float_key(hi);
        vals[r] = payload(upd ? KIND_ULO : KIND_SLO, (uint32_t)g);
        vals[R + r] = payload(upd ? KIND_UHI : KIND_SHI, (uint32_t)g);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) raise_error(st, DDM_ERR_INVALID, 15);
}

// inst_off[b] = first output pair of instance b = off[n_base[b]].
__global__ void k_inst_offsets(BatchArgs b, const unsigned long long* __restrict__ off,
                               unsigned long long* __restrict__ inst_off) {
    pdl_begin();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= b.num; i += gridDim.x * blockDim.x)
        inst_off[i] = b.n == 0 ? 0ull : off[b.n_base[i]];  // off[] exists only when n > 0
}

static unsigned grid_for(uint64_t items) {
    const uint64_t g = ceil_div(items, 256ull * 4);
    return (unsigned)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}


int launch_keybuild_batch(const BatchArgs& b, unsigned long long* keys, uint32_t* vals,
                          DevStatus* st, cudaStream_t s) {
    if (b.n + b.m == 0) return 0;
    launch_k(k_keybuild_batch, grid_for(b.n + b.m), 256, 0, s, b, keys, vals, st);
    return 1;
}

// Sorted survivor keys (i << jbits) | j of a batched d > 1 match, with global
// ids, to pairs of ids local to their instance (the instance of subscription i
// holds update j too: the join only pairs extents of one instance).
__global__ void k_batch_unpack(const unsigned long long* __restrict__ keys, uint64_t K, int jbits,
                               const int64_t* __restrict__ n_base,
                               const int64_t* __restrict__ m_base, int num,
                               int2* __restrict__ pairs) {
    pdl_begin();
    const unsigned long long jmask = (1ull << jbits) - 1ull;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K;
         k += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[k];
        const int64_t i = (int64_t)(key >> jbits), j = (int64_t)(key & jmask);
        const int b = inst_of(n_base, num, i);
        pairs[k] = make_int2((int32_t)(i - n_base[b]), (int32_t)(j - m_base[b]));
    }
}

int launch_batch_unpack(const unsigned long long* keys, uint64_t K, int jbits,
                        const int64_t* n_base, const int64_t* m_base, int num, int32_t* pairs,
                        cudaStream_t s) {
    if (K == 0) return 0;
    launch_k(k_batch_unpack, grid_for(K), 256, 0, s, keys, K, jbits, n_base, m_base, num,
             reinterpret_cast<int2*>(pairs));
    return 1;
}

int launch_inst_offsets(const BatchArgs& b, const unsigned long long* off,
                        unsigned long long* inst_off, cudaStream_t s) {
    launch_k(k_inst_offsets, grid_for(b.num + 1), 256, 0, s, b, off, inst_off);
    return 1;
}

}  // namespace ddm
