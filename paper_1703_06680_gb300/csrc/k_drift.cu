// a9 (served): drift of a simulation's resident extents between timesteps.
//
// Every extent moves by the same delta in lower and upper bound, per
// dimension: lo' = fl32(lo + delta), hi' = fl32(hi + delta); rounding is
// monotone, so lo' <= hi' still holds.  delta = f32(z * sigma) with z an
// approximately standard-normal draw computed exactly in integers: the
// Irwin-Hall sum of twelve uniforms, S = sum of twelve (x >> 11) values of
// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used as a counter-based
// generator, z = (S - 6 * 2^53) * 2^-53.  Element e of step t (e = k*n + i for
// S_i, d*n + k*m + j for U_j, along dimension k) uses stream draws
// (t * d(n+m) + e) * 12 .. +11.  All conversions round to nearest, so the
// result is reproducible bit for bit by any IEEE implementation of the same
// definition (the workload generator implements it independently).
#include "drift.cuh"

namespace ddm {

__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                            unsigned long long c) {
    unsigned long long z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_drift(DriftArgs a) {
    pdl_begin();
    const int64_t count = (int64_t)a.d * (a.n + a.m);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long c0 =
            ((unsigned long long)a.step * (unsigned long long)count + (unsigned long long)e) * 12ull;
        unsigned long long S = 0;
#pragma unroll
        for (int r = 0; r < 12; ++r) S += splitmix64_at(a.seed, c0 + r) >> 11;
        const double z = __ll2double_rn((long long)S - (long long)(6ull << 53)) * 0x1p-53;
        const float delta = __double2float_rn(__dmul_rn(z, a.sigma));
        const bool upd = e >= (int64_t)a.d * a.n;
        const int64_t rel = upd ? e - (int64_t)a.d * a.n : e;
        const int64_t cnt = upd ? a.m : a.n;
        const int k = (int)(rel / cnt);
        const int64_t id = rel - (int64_t)k * cnt;
        float* lo = upd ? a.upd_lo[k] : a.sub_lo[k];
        float* hi = upd ? a.upd_hi[k] : a.sub_hi[k];
        lo[id] = __fadd_rn(lo[id], delta);
        hi[id] = __fadd_rn(hi[id], delta);
    }
}

int launch_drift(const DriftArgs& a, cudaStream_t s) {
    const int64_t count = (int64_t)a.d * (a.n + a.m);
    if (count == 0) return 0;
    uint64_t g = ceil_div((uint64_t)count, 256ull * 4);
    launch_k(k_drift, (unsigned)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g)), 256, 0, s, a);
    return 1;
}

}  // namespace ddm
