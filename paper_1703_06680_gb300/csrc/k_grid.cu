// Grid-Based matching (Section 2, GB), the paper's third comparison method, on
// the GPU.  The routing space is cut into a regular mesh of cells (here over
// the first dg = min(d, 3) dimensions; the others are filtered per pair); every
// extent is registered in each cell it overlaps, and brute force runs inside
// each cell.  Two extents that intersect share a cell, because the cell map of
// a coordinate is monotone.  A pair that shares several cells is reported only
// in the cell holding the point max(S.lo, U.lo) (per gridded dimension), which
// lies in both extents when they intersect: each pair appears once.  The paper
// leaves the grid size G open (it depends on the workload and needs a
// heuristic); the caller may fix the cells per dimension, otherwise cells are
// made about as wide as the mean extent side, with at least about one extent
// per cell.
#include <cmath>
#include <cstring>

#include "baseline.cuh"

namespace ddm {

__device__ __forceinline__ bool grid_bad_extent(float lo, float hi) {
    return is_nan_bits(lo) || is_nan_bits(hi) || !(lo <= hi);
}

// Cell along gridded dimension k of coordinate x: monotone in x (a rounded
// subtraction, a product with a non-negative factor, a clamp and a
// truncation are all monotone).  NaN (only from -inf - -inf) clamps to 0.
__device__ __forceinline__ uint32_t cell_of(const GridPlan& p, int k, float x) {
    float t = (x - p.lo[k]) * p.inv_w[k];
    t = fminf(fmaxf(t, 0.f), (float)(p.g[k] - 1));
    return (uint32_t)t;
}

// Bounding box and summed sides of the gridded dimensions; validation of all.
__global__ void k_grid_bounds(DimPtrs dims, int d, int dg, uint32_t n, uint32_t m,
                              GridScratch* gs, DevStatus* st) {
    pdl_begin();
    __shared__ double ssum[GRID_MAX_DIMS][8];
    const uint32_t total = n + m;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t kmax[GRID_MAX_DIMS] = {}, kmin_inv[GRID_MAX_DIMS] = {};
    double side[GRID_MAX_DIMS] = {};
    bool bad = false;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += gridDim.x * blockDim.x) {
        const bool upd = e >= n;
        const uint32_t id = upd ? e - n : e;
        for (int k = 0; k < d; ++k) {
            const float lo = upd ? dims.upd_lo[k][id] : dims.sub_lo[k][id];
            const float hi = upd ? dims.upd_hi[k][id] : dims.sub_hi[k][id];
            bad |= grid_bad_extent(lo, hi);
            if (k < dg) {
                kmax[k] = max(kmax[k], float_key(hi));
                kmin_inv[k] = max(kmin_inv[k], ~float_key(lo));
                side[k] += (double)hi - (double)lo;
            }
        }
    }
    for (int k = 0; k < GRID_MAX_DIMS; ++k) {
        if (k >= dg) break;
        const uint32_t a = __reduce_max_sync(0xffffffffu, kmax[k]);
        const uint32_t b = __reduce_max_sync(0xffffffffu, kmin_inv[k]);
        double sk = side[k];
        for (int o = 16; o > 0; o >>= 1) sk += __shfl_xor_sync(0xffffffffu, sk, o);
        if (lane == 0) {
            if (a) atomicMax(&gs->kmax_hi[k], a);
            if (b) atomicMax(&gs->kmin_lo_inv[k], b);
            ssum[k][warp] = sk;
        }
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)dg) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ssum[threadIdx.x][w];
        if (t != 0) atomicAdd(&gs->side_sum[threadIdx.x], t);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) raise_error(st, DDM_ERR_INVALID, 50);
}

// Cells of an extent: the box [a_k, b_k] along the gridded dimensions.
struct CellBox {
    uint32_t a[GRID_MAX_DIMS], b[GRID_MAX_DIMS];
};

__device__ __forceinline__ CellBox box_of(const GridPlan& p, const DimPtrs& dims, bool upd,
                                          uint32_t id) {
    CellBox c{};
    for (int k = 0; k < p.dg; ++k) {
        c.a[k] = cell_of(p, k, upd ? dims.upd_lo[k][id] : dims.sub_lo[k][id]);
        c.b[k] = cell_of(p, k, upd ? dims.upd_hi[k][id] : dims.sub_hi[k][id]);
    }
    return c;
}

// Calls f(cell index) for every cell of the box.
template <typename F>
__device__ __forceinline__ void for_cells(const GridPlan& p, const CellBox& c, F&& f) {
    const uint32_t n0 = c.b[0] - c.a[0] + 1;
    const uint32_t n1 = p.dg > 1 ? c.b[1] - c.a[1] + 1 : 1u;
    const uint32_t n2 = p.dg > 2 ? c.b[2] - c.a[2] + 1 : 1u;
    for (uint32_t z = 0; z < n2; ++z)
        for (uint32_t y = 0; y < n1; ++y)
            for (uint32_t x = 0; x < n0; ++x) {
                uint32_t cell = (c.a[0] + x) * p.stride[0];
                if (p.dg > 1) cell += (c.a[1] + y) * p.stride[1];
                if (p.dg > 2) cell += (c.a[2] + z) * p.stride[2];
                f(cell);
            }
}

// Per-cell membership counts of both sets.
__global__ void k_grid_count(DimPtrs dims, uint32_t n, uint32_t m, GridPlan p,
                             uint32_t* cnt_s, uint32_t* cnt_u, DevStatus* st) {
    pdl_begin();
    if (read_error(st)) return;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n + m;
         e += gridDim.x * blockDim.x) {
        const bool upd = e >= n;
        uint32_t* cnt = upd ? cnt_u : cnt_s;
        for_cells(p, box_of(p, dims, upd, upd ? e - n : e),
                  [&](uint32_t cell) { atomicAdd(&cnt[cell], 1u); });
    }
}

static unsigned grid_blocks(uint64_t items) {
    uint64_t g = ceil_div(items, 256);
    return (unsigned)(g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g));
}

int launch_grid_bounds(const DimPtrs& dims, int d, int64_t n, int64_t m, GridScratch* gs,
                       DevStatus* st, cudaStream_t s) {
    const int dg = d < GRID_MAX_DIMS ? d : GRID_MAX_DIMS;
    launch_k(k_grid_bounds, grid_blocks((uint64_t)(n + m)), 256, 0, s, dims, d, dg, (uint32_t)n,
             (uint32_t)m, gs, st);
    return 1;
}

GridPlan grid_plan(const GridScratch& h, int d, uint64_t total, uint32_t cells_per_dim) {
    GridPlan p{};
    const int dg = d < GRID_MAX_DIMS ? d : GRID_MAX_DIMS;
    p.dg = dg;
    const uint32_t cap = 1u << (24 / dg);  // G <= 2^24 in all
    const double per_dim = std::ceil(std::pow((double)(total > 0 ? total : 1), 1.0 / dg));
    uint32_t G = 1;
    for (int k = 0; k < dg; ++k) {
        // Inverse of the order-preserving key map (the keys were reduced on the device).
        auto key_to_float = [](uint32_t key) {
            const uint32_t u = (key & 0x80000000u) ? (key & 0x7fffffffu) : ~key;
            float f;
            std::memcpy(&f, &u, sizeof f);
            return f;
        };
        const float lo = key_to_float(~h.kmin_lo_inv[k]), hi = key_to_float(h.kmax_hi[k]);
        const double span = (double)hi - (double)lo;
        uint32_t g = 1;
        if (std::isfinite(span) && span > 0 && total > 0) {
            double gg;
            if (cells_per_dim) {
                gg = cells_per_dim;
            } else {
                const double mean = h.side_sum[k] / (double)total;
                const double w = std::fmax(mean, span / per_dim);
                gg = std::floor(span / w);
            }
            g = gg < 1 ? 1u : (gg > cap ? cap : (uint32_t)gg);
        }
        p.g[k] = g;
        p.lo[k] = std::isfinite(lo) ? lo : 0.f;
        p.inv_w[k] = g > 1 ? (float)(g / span) : 0.f;
        p.stride[k] = G;
        G *= g;
    }
    p.G = G;
    return p;
}

int launch_grid_count(const DimPtrs& dims, int64_t n, int64_t m, const GridPlan& p,
                      uint32_t* cnt_s, uint32_t* cnt_u, DevStatus* st, cudaStream_t s) {
    launch_k(k_grid_count, grid_blocks((uint64_t)(n + m)), 256, 0, s, dims, (uint32_t)n,
             (uint32_t)m, p, cnt_s, cnt_u, st);
    return 1;
}

// Memberships sorted by cell: each extent writes its id into every cell of its
// box (order inside a cell is irrelevant: the segments are sorted at the end).
__global__ void k_grid_fill(DimPtrs dims, uint32_t n, uint32_t m, GridPlan p,
                            const unsigned long long* __restrict__ off_s,
                            const unsigned long long* __restrict__ off_u, uint32_t* cur_s,
                            uint32_t* cur_u, uint32_t* __restrict__ ent_s,
                            uint32_t* __restrict__ ent_u, DevStatus* st) {
    pdl_begin();
    if (read_error(st)) return;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n + m;
         e += gridDim.x * blockDim.x) {
        const bool upd = e >= n;
        const uint32_t id = upd ? e - n : e;
        const unsigned long long* off = upd ? off_u : off_s;
        uint32_t* cur = upd ? cur_u : cur_s;
        uint32_t* ent = upd ? ent_u : ent_s;
        for_cells(p, box_of(p, dims, upd, id), [&](uint32_t cell) {
            const unsigned long long pos = off[cell] + atomicAdd(&cur[cell], 1u);
            if (pos < off[cell + 1]) ent[pos] = id;
            else raise_error(st, DDM_ERR_INTERNAL, 51);
        });
    }
}

// Brute force inside each cell (one block per cell, grid-stride): thread t
// takes subscriptions t, t + blockDim, ... of the cell and tests every update
// of the cell (the same update for all threads at a time: broadcast loads).
// A pair is counted only in the cell of its reference point max(S.lo, U.lo).
template <bool WRITE>
__global__ void __launch_bounds__(128)
k_grid_match(DimPtrs dims, int d, GridPlan p, const unsigned long long* __restrict__ off_s,
             const unsigned long long* __restrict__ off_u, const uint32_t* __restrict__ ent_s,
             const uint32_t* __restrict__ ent_u, uint32_t* cnt,
             const unsigned long long* __restrict__ off, uint32_t* cursor, int2* pairs,
             DevStatus* st) {
    pdl_begin();
    if (read_error(st)) return;
    for (uint32_t c = blockIdx.x; c < p.G; c += gridDim.x) {
        uint32_t ck[GRID_MAX_DIMS];
        for (int k = 0; k < GRID_MAX_DIMS; ++k) ck[k] = k < p.dg ? (c / p.stride[k]) % p.g[k] : 0u;
        const unsigned long long s0 = off_s[c], s1 = off_s[c + 1];
        const unsigned long long u0 = off_u[c], u1 = off_u[c + 1];
        if (s0 == s1 || u0 == u1) continue;
        for (unsigned long long q = s0 + threadIdx.x; q < s1; q += blockDim.x) {
            const uint32_t i = ent_s[q];
            float slo_f[GRID_MAX_DIMS];
            uint32_t sl[DDM_MAX_DIMS], sh[DDM_MAX_DIMS];
#pragma unroll
            for (int k = 0; k < DDM_MAX_DIMS; ++k) {
                sl[k] = sh[k] = 0u;
                if (k < d) {
                    const float lo = dims.sub_lo[k][i];
                    if (k < GRID_MAX_DIMS) slo_f[k] = lo;
                    sl[k] = float_key(lo);
                    sh[k] = float_key(dims.sub_hi[k][i]);
                }
            }
            // Two passes in the write mode: count, reserve, then write.
            uint32_t found = 0;
            int2* out = nullptr;
            for (int pass = 0; pass < (WRITE ? 2 : 1); ++pass) {
                if (WRITE && pass == 1) {
                    if (found == 0) break;
                    out = pairs + off[i] + atomicAdd(&cursor[i], found);
                    found = 0;
                }
                for (unsigned long long r = u0; r < u1; ++r) {
                    const uint32_t j = ent_u[r];
                    bool hit = true;
#pragma unroll
                    for (int k = 0; k < DDM_MAX_DIMS; ++k) {
                        if (k < d && hit) {
                            const float ulo = dims.upd_lo[k][j];
                            const uint32_t kl = float_key(ulo), kh = float_key(dims.upd_hi[k][j]);
                            hit = kl <= sh[k] && sl[k] <= kh;  // Algorithm 1
                            if (hit && k < p.dg) {  // the reference point's cell
                                const float ref = kl > sl[k] ? ulo : slo_f[k < GRID_MAX_DIMS ? k : 0];
                                hit = cell_of(p, k, ref) == ck[k];
                            }
                        }
                    }
                    if (hit) {
                        if (WRITE && pass == 1) out[found] = make_int2((int32_t)i, (int32_t)j);
                        ++found;
                    }
                }
            }
            if (!WRITE && found) atomicAdd(&cnt[i], found);
        }
    }
}

int launch_grid_fill(const DimPtrs& dims, int64_t n, int64_t m, const GridPlan& p,
                     const unsigned long long* cell_off_s, const unsigned long long* cell_off_u,
                     uint32_t* cur_s, uint32_t* cur_u, uint32_t* ent_s, uint32_t* ent_u,
                     DevStatus* st, cudaStream_t s) {
    launch_k(k_grid_fill, grid_blocks((uint64_t)(n + m)), 256, 0, s, dims, (uint32_t)n,
             (uint32_t)m, p, cell_off_s, cell_off_u, cur_s, cur_u, ent_s, ent_u, st);
    return 1;
}

int launch_grid_match(const DimPtrs& dims, int d, const GridPlan& p,
                      const unsigned long long* cell_off_s, const unsigned long long* cell_off_u,
                      const uint32_t* ent_s, const uint32_t* ent_u, uint32_t* cnt,
                      const unsigned long long* off, uint32_t* cursor, int32_t* pairs,
                      DevStatus* st, cudaStream_t s) {
    const unsigned grid = p.G < 152u * 16 ? p.G : 152u * 16;
    if (pairs)
        launch_k(k_grid_match<true>, grid, 128, 0, s, dims, d, p, cell_off_s, cell_off_u, ent_s,
                 ent_u, cnt, off, cursor, reinterpret_cast<int2*>(pairs), st);
    else
        launch_k(k_grid_match<false>, grid, 128, 0, s, dims, d, p, cell_off_s, cell_off_u, ent_s,
                 ent_u, cnt, off, cursor, static_cast<int2*>(nullptr), st);
    return 1;
}

}  // namespace ddm
