// ddm_count_noalloc: the count of ddm_count for callers that cannot allocate
// device memory -- code running where cudaMalloc is unavailable or forbidden,
// such as under a custom allocator that owns all device memory, or in a
// real-time simulation loop that must not allocate after start-up.  Every
// scratch buffer of the count pipeline (sort keys and values, scan status
// words, rank records, counts, offsets, status word) is carved from one
// file-scope __device__ array of fixed size, so the call itself allocates
// nothing: no cudaMalloc, no cudaFree, no pinned host buffer.
//
// The array is held by every GPU that loads this library, until the process
// exits.  All calls share it and it keeps the last call's contents, so every
// call first clears the parts that must start at zero, and calls that overlap
// on the GPU (on two streams, or from two threads) race and give wrong
// results; serialise them.  The call synchronizes its stream before it
// returns, so it cannot run inside a host function enqueued on a stream.
#include "emit.cuh"
#include "sort.cuh"
#include "sweep.cuh"

using namespace ddm;

namespace {

constexpr int64_t NOALLOC_MAX_REGIONS = int64_t(1) << 17;  // n + m of one instance
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(24) << 20;  // 24 MiB per GPU
static_assert(NOALLOC_MAX_REGIONS == DDM_NOALLOC_MAX_REGIONS, "header and library agree");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// In host code g_noalloc_scratch names a host-side stand-in, not device
// memory.  The device address is looked up on every call, with the caller's
// device current: the lookup allocates nothing, and no address is cached that
// a cudaDeviceReset or another context on the same device would make stale.
int noalloc_scratch(char** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return DDM_ERR_CUDA;
    }
    *out = static_cast<char*>(p);
    return DDM_OK;
}

// Bump allocation inside the static array; every region 256-byte aligned.
struct Slab {
    char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
};

// Buffers of one count-only call.  Zeroed part first.
struct NoallocLayout {
    DevStatus* st;
    SortScratch sort;
    unsigned long long* scan_status;
    unsigned long long* off_status;
    size_t zero_bytes;
    uint32_t *keys0, *keys1, *vals0, *vals1;
    Records rec;
    uint32_t *cnt, *cnt_a;
    unsigned long long* off;
    uint2 *subK, *updK;
    size_t total;

    void carve(char* base, int d, int64_t n, int64_t m) {
        const uint64_t E = 2 * (uint64_t)(n + m);
        Slab s{base};
        st = s.take<DevStatus>(1);
        sort.status = s.take<unsigned long long>(4 * sort_status_stride(E));
        sort.total = s.take<unsigned long long>(1);
        {
            const size_t gw = sort_group_words(sort_tiles<uint32_t>(E), 4);
            sort.grp = s.take<uint32_t>(gw);
            if (gw == 0) sort.grp = nullptr;
        }
        scan_status = s.take<unsigned long long>(3 * (ceil_div(E, SCAN_TILE) + 1) + 1);
        off_status = s.take<unsigned long long>(ceil_div((uint64_t)n, OFF_TILE) + 2);
        zero_bytes = (s.off + 255) & ~(size_t)255;
        sort.tile_hist = s.take<uint32_t>(sort_tiles<uint32_t>(E) * RADIX);
        sort.offs = s.take<unsigned long long>(sort_tiles<uint32_t>(E) * RADIX + 1);
        keys0 = s.take<uint32_t>(E);
        keys1 = s.take<uint32_t>(E);
        vals0 = s.take<uint32_t>(E);
        vals1 = s.take<uint32_t>(E);
        rec = Records{};
        rec.s_lo = s.take<uint4>(n);
        rec.s_hi = s.take<uint4>(n);
        rec.u_lo = s.take<uint4>(m);
        rec.u_hi = s.take<uint4>(m);
        rec.sub_order = s.take<uint32_t>(n);
        rec.upd_order = s.take<uint32_t>(m);
        cnt = s.take<uint32_t>(n);
        cnt_a = s.take<uint32_t>(d > 1 ? n : 0);
        off = s.take<unsigned long long>(n + 1);
        subK = s.take<uint2>(d > 1 ? (size_t)(d - 1) * n : 0);
        updK = s.take<uint2>(d > 1 ? (size_t)(d - 1) * m : 0);
        total = s.off;
    }
};

}  // namespace

extern "C" int ddm_count_noalloc(const ddm_regions* r, void* cuda_stream, uint64_t* K_out) {
    if (!r || !K_out) return DDM_ERR_INVALID;
    if (r->d < 1 || r->d > DDM_MAX_DIMS || r->n < 0 || r->m < 0) return DDM_ERR_INVALID;
    if (r->n + r->m > NOALLOC_MAX_REGIONS) return DDM_ERR_INVALID;  // beyond the fixed scratch
    if (!r->sub_lo || !r->sub_hi || !r->upd_lo || !r->upd_hi) return DDM_ERR_INVALID;
    for (int k = 0; k < r->d; ++k) {
        if (r->n > 0 && (!r->sub_lo[k] || !r->sub_hi[k])) return DDM_ERR_INVALID;
        if (r->m > 0 && (!r->upd_lo[k] || !r->upd_hi[k])) return DDM_ERR_INVALID;
    }
    NoallocLayout L;
    L.carve(nullptr, r->d, r->n, r->m);
    if (L.total > NOALLOC_SCRATCH_BYTES) return DDM_ERR_INVALID;
    char* base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc) return rc;
    L.carve(base, r->d, r->n, r->m);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    PdlScope pdl_scope(true);
    const int64_t n = r->n, m = r->m;
    const uint64_t E = 2 * (uint64_t)(n + m);
    if (cudaMemsetAsync(base, 0, L.zero_bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return DDM_ERR_CUDA;
    }
    if (E > 0) {
        launch_keybuild_d0(r->sub_lo[0], r->sub_hi[0], r->upd_lo[0], r->upd_hi[0], n, m, L.keys0,
                           L.vals0, L.st, s);
        launch_radix_sort<uint32_t>(L.keys0, L.vals0, L.keys1, L.vals1, E, 4, L.sort, true, L.st, s);
        launch_sweep_scan(L.vals0, E, n, m, L.rec, L.scan_status, L.st, s);
        if (r->d == 1) {
            launch_rank_offsets(L.rec, n, L.cnt, L.off, ~0ull, &L.st->K, L.off_status, L.st, s);
        } else {
            EmitArgs a{};
            a.d = r->d; a.n = n; a.m = m;
            for (int k = 0; k < r->d; ++k) {
                a.dims.sub_lo[k] = r->sub_lo[k]; a.dims.sub_hi[k] = r->sub_hi[k];
                a.dims.upd_lo[k] = r->upd_lo[k]; a.dims.upd_hi[k] = r->upd_hi[k];
            }
            a.rec = L.rec;
            a.cnt = L.cnt; a.cnt_a = L.cnt_a; a.subK = L.subK; a.updK = L.updK;
            launch_permute_keys(a, L.st, s);
            launch_filter_count(a, L.st, s);
            launch_offsets(L.cnt, n, L.off, ~0ull, &L.st->K, L.off_status, L.st, s);
        }
    }
    if (cudaGetLastError() != cudaSuccess) return DDM_ERR_CUDA;
    DevStatus h{};
    if (cudaMemcpyAsync(&h, L.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return DDM_ERR_CUDA;
    }
    if (h.error == DDM_OK) *K_out = h.K;
    return h.error;
}
