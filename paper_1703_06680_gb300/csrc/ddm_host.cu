// C ABI of the SBM library: contexts, workspace, and the pipeline
// a1 key build -> a2 radix sort -> a3 sweep scan -> a4 counts (d = 1) or a7
// filter count (d > 1) -> a5 offsets -> a6 emission (+ a7 write filter) ->
// per-segment sort.  Everything is enqueued on the context's stream; device
// kernels gate on the device status word (an input error or a capacity
// overflow stops the later stages), and the host reads {status, K} once.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "baseline.cuh"
#include "batch.cuh"
#include "delta.cuh"
#include "drift.cuh"
#include "emit.cuh"
#include "sort.cuh"
#include "sweep.cuh"

using namespace ddm;

namespace ddm {
thread_local bool g_pdl = false;
int launch_wait_selftest(int which, uint32_t limit, unsigned long long* status, DevStatus* st,
                         cudaStream_t s);
// k_selftest.cu: the write-pattern reference of the window emission.
int launch_wp_lengths(uint32_t* len, uint32_t nseg, uint32_t mean_len, uint32_t seed,
                      cudaStream_t s);
int launch_wp_write(int2* out, const unsigned long long* off, uint32_t nseg, uint32_t step,
                    cudaStream_t s);
// k_status.cu: a call's zero fill (status and zeroed workspace) and the status
// copy into the mapped host mirror.
int launch_prologue(DevStatus* st, void* zero, uint64_t zero_bytes, cudaStream_t s);
int launch_publish(const DevStatus* st, DevStatus* host_mapped, const uint32_t* flagged,
                   cudaStream_t s);
}

struct ddm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0;
    size_t held = 0;  // device bytes held by ensure() buffers and session coordinates
    std::string err;
    char* ws = nullptr;
    size_t ws_size = 0;
    DevStatus* dstat = nullptr;  // device
    DevStatus* hstat = nullptr;  // pinned host mirror
    DevStatus* hstat_dev = nullptr;  // its device address when mapped (else NULL: copy)
    // ddm_match on the window path: the range path (flagged subscriptions) is
    // left out of the enqueued pipeline and launched after the one
    // synchronisation only if the status reports flagged subscriptions.
    bool defer_fallback = false;      // set by ddm_match around its enqueue
    bool fallback_pending = false;    // the last enqueue left the range path out
    EmitArgs fallback_args{};         // its arguments
    const uint32_t* flag_count = nullptr;  // the flagged counter, for the next finish only
    // host-buffer entry point staging (inputs, outputs)
    char* io = nullptr;
    size_t io_size = 0;
    char* out = nullptr;
    size_t out_size = 0;
    // counters and per-stage timing
    ddm_stats stats{};
    int prof = 0;  // 0 off, 1 every stage boundary, 2 + k only around stage k
    unsigned long long* last_inst_off = nullptr;  // device, batched calls
    int win_shift = 10;                           // DDM_PARAM_WIN_SHIFT
    int nd_path = 0;                              // DDM_PARAM_ND_PATH
    bool pdl = true;                              // DDM_PARAM_PDL
    bool keep_keys = false;  // sessions: the sort's last pass also writes the sorted keys
    int sort_items = 18;                          // DDM_PARAM_SORT_ITEMS
    // d > 1 matching: the join's count pass records its survivors here, so
    // that the pairs come from one sort of those keys instead of a second
    // filter pass and a per-segment sort (when all of them fit).
    char* sv = nullptr;
    size_t sv_size = 0;
    uint64_t surv_hint = 0;                       // K of the last d > 1 match
    uint64_t surv_fail_K = ~0ull;                 // K whose survivors did not fit
    unsigned long long* surv_keys = nullptr;      // non-NULL: record in this call
    uint64_t surv_cap = 0;
    int join_shift = 11;                          // DDM_PARAM_JOIN_SHIFT
    int nd_write = 0;                             // DDM_PARAM_ND_WRITE
    int sweep_dim = 0;                            // DDM_PARAM_SWEEP_DIM
    cudaEvent_t ev[DDM_STAGES + 1] = {};
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int fail(ddm_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(ddm_ctx* c, cudaError_t e, const char* what) {
    return fail(c, DDM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);     \
    } while (0)

// Bump allocator over one workspace allocation; every region 256-byte aligned.
struct Carve {
    size_t off = 0;
    char* base = nullptr;
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
};

// Grows one of the context's device buffers (*buf, *size) to hold `need`
// bytes.  c->held counts every byte the context (and its session, if any)
// holds on the device, so the budget covers all of them together.
int ensure(ddm_ctx* c, char** buf, size_t* size, size_t need) {
    if (need <= *size) return DDM_OK;
    const size_t other = c->held - *size;  // held includes this buffer's current size
    if (c->budget && (other > c->budget || need > c->budget - other))
        return fail(c, DDM_ERR_NOMEM, "device memory need of " + std::to_string(need) +
                                          " bytes exceeds the context budget (" +
                                          std::to_string(other) + " bytes held elsewhere)");
    if (*buf) {
        cudaFree(*buf);
        c->held -= *size;
        *buf = nullptr;
        *size = 0;
    }
    size_t grow = need + need / 8;
    if (c->budget && grow > c->budget - other) grow = c->budget - other;  // >= need (checked)
    cudaError_t e = cudaMalloc(buf, grow);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(buf, need);
        grow = need;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return fail(c, DDM_ERR_NOMEM, "cudaMalloc of " + std::to_string(need) + " bytes failed");
    }
    *size = grow;
    c->held += grow;
    return DDM_OK;
}

// Sort scratch of one radix sort of up to E KeyT keys in `passes` passes,
// carved with its zeroed part (status words, total, group sums) first;
// [zb, ze) is that part's byte range, to be cleared before every sort.
template <typename KeyT>
void carve_sort(Carve& cv, uint64_t E, int passes, SortScratch& sc, size_t& zb,
                       size_t& ze) {
    const uint64_t tiles = sort_tiles<KeyT>(E);
    zb = (cv.off + 255) & ~(size_t)255;
    sc.status = cv.take<unsigned long long>((size_t)passes * sort_status_stride(E));
    sc.total = cv.take<unsigned long long>(1);
    const size_t gw = sort_group_words(tiles, passes);
    sc.grp = gw ? cv.take<uint32_t>(gw) : nullptr;
    ze = cv.off;
    sc.tile_hist = cv.take<uint32_t>(tiles * RADIX);
    sc.offs = cv.take<unsigned long long>(tiles * RADIX + 1);
}

int check_regions(ddm_ctx* c, const ddm_regions* r) {
    if (!r) return fail(c, DDM_ERR_INVALID, "regions is NULL");
    if (r->d < 1 || r->d > DDM_MAX_DIMS) return fail(c, DDM_ERR_INVALID, "d out of range");
    if (r->n < 0 || r->m < 0 || r->n + r->m > DDM_MAX_REGIONS)
        return fail(c, DDM_ERR_INVALID, "n or m out of range");
    if (!r->sub_lo || !r->sub_hi || !r->upd_lo || !r->upd_hi)
        return fail(c, DDM_ERR_INVALID, "coordinate pointer arrays must not be NULL");
    for (int k = 0; k < r->d; ++k) {
        if (r->n > 0 && (!r->sub_lo[k] || !r->sub_hi[k]))
            return fail(c, DDM_ERR_INVALID, "NULL subscription coordinates");
        if (r->m > 0 && (!r->upd_lo[k] || !r->upd_hi[k]))
            return fail(c, DDM_ERR_INVALID, "NULL update coordinates");
    }
    return DDM_OK;
}

enum class Mode { Count, Match, Debug };

// Stage boundary k (0..DDM_STAGES): records an event when profiling.
void mark(ddm_ctx* c, int k) {
    if (c->prof == 1 || (c->prof >= 2 && (k == c->prof - 2 || k == c->prof - 1)))
        cudaEventRecord(c->ev[k], c->stream);
}

struct DebugOut {
    uint32_t *who, *subset, *updset, *sub_cnt, *upd_cnt;
};

// One call's work: a plain instance (device coordinate pointers) or a batch
// of instances (host array of descriptors, concatenated on the device).
struct Job {
    int d = 1;
    int64_t n = 0, m = 0;
    const ddm_regions* r = nullptr;     // plain: the instance
    int num_inst = 0;                   // batch: number of instances (0 = plain)
    const ddm_regions* inst = nullptr;  // batch: host descriptors
};

int ceil_log2(int64_t x) {
    int b = 0;
    while (((int64_t)1 << b) < x) ++b;
    return b;
}

// Lays out every buffer of one call.  With base == nullptr only sizes.
struct Plan {
    int64_t n, m, E;
    int d, num_inst, passes;
    // zeroed region
    SortScratch sort;
    unsigned long long* scan_status;
    unsigned long long* off_status;
    uint32_t* cursor_b;
    // window path (d = 1, match) and tiled join (d > 1)
    bool window, join;
    int win_shift;
    uint32_t lcap;
    uint32_t num_win;
    uint32_t* lw_fill;
    uint32_t* num_flagged;
    unsigned long long* cand_fill;
    unsigned long long* surv_fill;
    uint4* wmeta;
    uint2* wcand;
    unsigned long long cand_cap;
    unsigned long long* lw_total;
    unsigned long long* win_status;
    size_t zero_bytes;
    uint4* windows;
    unsigned long long* lw_off;
    uint4* lw;
    uint4* urank;
    SubRank* srank;
    unsigned long long lw_cap;
    uint8_t* flag;
    // the rest
    void *keys0, *keys1;
    uint32_t *vals0, *vals1;
    Records rec;
    uint32_t *cnt, *cnt_a, *upd_cnt;
    unsigned long long* off;
    uint2 *subK, *updK;
    // batch
    InstPtrs* table;
    int64_t *n_base, *m_base;
    float* cat[4][DDM_MAX_DIMS];
    unsigned long long* inst_off;
    size_t total;

    int sort_items;

    void layout(char* base, int d_, int64_t n_, int64_t m_, Mode mode, int num_inst_,
                int win_shift_ = 10, int nd_path = 0, int sort_items_ = 18, int join_shift = 11) {
        sort_items = sort_items_;
        d = d_; n = n_; m = m_; E = 2 * (n + m); num_inst = num_inst_;
        const bool batch = num_inst > 0;
        passes = batch ? (int)ceil_div(32 + ceil_log2(num_inst), RADIX_BITS) : 4;
        const uint64_t stiles = batch ? sort_tiles<unsigned long long>(E)
                                      : sort_tiles<uint32_t>(E, sort_items);
        Carve cv;
        cv.base = base;
        sort.status = cv.take<unsigned long long>((size_t)passes * sort_status_stride(E));
        sort.total = cv.take<unsigned long long>(1);
        {
            const size_t gw = sort_group_words(stiles, passes);
            sort.grp = cv.take<uint32_t>(gw);
            if (gw == 0) sort.grp = nullptr;
        }
        scan_status = cv.take<unsigned long long>(3 * (ceil_div(E, SCAN_TILE) + 1) + 1);
        off_status = cv.take<unsigned long long>(ceil_div(n, OFF_TILE) + 2);
        cursor_b = cv.take<uint32_t>(mode == Mode::Match ? n : 0);
        window = mode == Mode::Match && d == 1;
        join = d > 1 && mode != Mode::Debug && nd_path != 2;
        const bool lists = window || join;
        win_shift = join ? join_shift : win_shift_;
        // Window path: list w lives in a fixed slot of 2^win_shift entries at
        // w << win_shift (no offsets scan); longer lists overflow to the range
        // path.  Tiled join: lists of any length, placed by an offsets scan.
        lcap = join ? 0xffffffffu : (1u << win_shift);
        num_win = lists ? (uint32_t)ceil_div(E, 1ull << win_shift) : 0;
        lw_fill = cv.take<uint32_t>(num_win);
        num_flagged = cv.take<uint32_t>(1);
        cand_fill = cv.take<unsigned long long>(1);
        surv_fill = cv.take<unsigned long long>(join ? num_win : 0);
        lw_total = cv.take<unsigned long long>(1);
        win_status = cv.take<unsigned long long>(lists ? ceil_div(num_win, OFF_TILE) + 2 : 0);
        zero_bytes = (cv.off + 255) & ~(size_t)255;
        windows = cv.take<uint4>(lists ? num_win + 1 : 0);
        lw_off = cv.take<unsigned long long>(join ? num_win + 1 : 0);
        if (window) lw_cap = (unsigned long long)num_win << win_shift;
        else if (join) lw_cap = std::min<unsigned long long>(
            std::max<unsigned long long>(16ull * E, 16ull << 20), 64ull << 20);
        else lw_cap = 0;
        lw = cv.take<uint4>(lw_cap);
        // Window path: the id-sorted candidates of every window (about 360 per
        // window of 1024 positions at alpha = 100; windows that find no room
        // go to the range path).
        cand_cap = window ? 2 * (unsigned long long)E + 4096 : 0;
        wcand = cv.take<uint2>(cand_cap);
        wmeta = cv.take<uint4>(window ? num_win : 0);
        urank = cv.take<uint4>(lists ? m : 0);
        srank = cv.take<SubRank>(window ? n : 0);
        flag = cv.take<uint8_t>(lists ? n : 0);
        sort.tile_hist = cv.take<uint32_t>(stiles * RADIX);
        sort.offs = cv.take<unsigned long long>(stiles * RADIX + 1);
        const size_t ksz = batch ? 8 : 4;
        keys0 = cv.take<char>(E * ksz);
        keys1 = cv.take<char>(E * ksz);
        vals0 = cv.take<uint32_t>(E);
        vals1 = cv.take<uint32_t>(E);
        rec.s_lo = cv.take<uint4>(n);
        rec.s_hi = cv.take<uint4>(n);
        rec.u_lo = cv.take<uint4>(m);
        rec.u_hi = cv.take<uint4>(m);
        rec.sub_order = cv.take<uint32_t>(n);
        rec.upd_order = cv.take<uint32_t>(m);
        rec.windows = nullptr;
        rec.win_shift = 0;
        rec.dbg_who = rec.dbg_subset = rec.dbg_updset = nullptr;
        cnt = cv.take<uint32_t>(n);
        cnt_a = cv.take<uint32_t>(d > 1 ? n : 0);
        upd_cnt = nullptr;
        off = cv.take<unsigned long long>(n + 1);
        subK = cv.take<uint2>(d > 1 ? (size_t)(d - 1) * n : 0);
        updK = cv.take<uint2>(d > 1 ? (size_t)(d - 1) * m : 0);
        table = cv.take<InstPtrs>(num_inst);
        n_base = cv.take<int64_t>(batch ? num_inst + 1 : 0);
        m_base = cv.take<int64_t>(batch ? num_inst + 1 : 0);
        for (int a = 0; a < 4; ++a)
            for (int k = 0; k < DDM_MAX_DIMS; ++k)
                cat[a][k] = cv.take<float>(batch && k < d ? (a < 2 ? n : m) : 0);
        inst_off = cv.take<unsigned long long>(batch ? num_inst + 1 : 0);
        total = cv.off + 256;
    }
};

int id_bits(int64_t m) {
    int b = 1;
    while (b < 31 && ((int64_t)1 << b) < m) ++b;
    return b;
}

// Which part of the pipeline to enqueue: everything, only the stages up to
// and including the offsets scan (the exact K is then known), or only the
// emission stages that follow, on the state the prefix left in the workspace.
enum class Phase { All, Prefix, Suffix };

// Enqueues the pipeline (or a phase of it) for one job.  Does not synchronize.
int enqueue(ddm_ctx* c, const Job& job, Mode mode, int32_t* pairs, uint64_t cap,
            const DebugOut* dbg, Phase phase = Phase::All) {
    Plan pl;
    pl.layout(nullptr, job.d, job.n, job.m, mode, job.num_inst, c->win_shift, c->nd_path,
              c->sort_items, c->join_shift);
    if (phase == Phase::Suffix && pl.total > c->ws_size)
        return fail(c, DDM_ERR_INTERNAL, "emission phase without its prefix");
    int rc = ensure(c, &c->ws, &c->ws_size, pl.total);
    if (rc) return rc;
    pl.layout(c->ws, job.d, job.n, job.m, mode, job.num_inst, c->win_shift, c->nd_path,
              c->sort_items, c->join_shift);
    // Pairs are stored as 8-byte (i, j) units.
    if (pairs && (reinterpret_cast<uintptr_t>(pairs) & 7u))
        return fail(c, DDM_ERR_INVALID, "pairs must be 8-byte aligned");
    cudaStream_t s = c->stream;
    PdlScope pdl_scope(c->pdl);
    const bool batch = job.num_inst > 0;
    const bool do_prefix = phase != Phase::Suffix, do_suffix = phase != Phase::Prefix;
    uint64_t& L = c->stats.launches;
    if (do_prefix) {
        L += launch_prologue(c->dstat, c->ws, pl.zero_bytes, s);
        c->stats.calls++;
    }

    // Coordinates of every dimension as device arrays over the job's ids.
    DimPtrs dims{};
    BatchArgs ba{};
    if (batch) {
        const int num = job.num_inst;
        std::vector<InstPtrs> table(num);
        std::vector<int64_t> nb(num + 1, 0), mb(num + 1, 0);
        for (int b = 0; b < num; ++b) {
            const ddm_regions& r = job.inst[b];
            for (int k = 0; k < job.d; ++k) {
                table[b].sub_lo[k] = r.sub_lo[k]; table[b].sub_hi[k] = r.sub_hi[k];
                table[b].upd_lo[k] = r.upd_lo[k]; table[b].upd_hi[k] = r.upd_hi[k];
            }
            nb[b + 1] = nb[b] + r.n;
            mb[b + 1] = mb[b] + r.m;
        }
        if (do_prefix) {
            CK(cudaMemcpyAsync(pl.table, table.data(), num * sizeof(InstPtrs),
                               cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(pl.n_base, nb.data(), (num + 1) * sizeof(int64_t),
                               cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(pl.m_base, mb.data(), (num + 1) * sizeof(int64_t),
                               cudaMemcpyHostToDevice, s));
        }
        ba.d = job.d; ba.num = num; ba.n = pl.n; ba.m = pl.m;
        ba.table = pl.table; ba.n_base = pl.n_base; ba.m_base = pl.m_base;
        for (int k = 0; k < job.d; ++k) {
            ba.sub_lo[k] = pl.cat[0][k]; ba.sub_hi[k] = pl.cat[1][k];
            ba.upd_lo[k] = pl.cat[2][k]; ba.upd_hi[k] = pl.cat[3][k];
            dims.sub_lo[k] = pl.cat[0][k]; dims.sub_hi[k] = pl.cat[1][k];
            dims.upd_lo[k] = pl.cat[2][k]; dims.upd_hi[k] = pl.cat[3][k];
        }
    } else {
        for (int k = 0; k < job.d; ++k) {
            dims.sub_lo[k] = job.r->sub_lo[k]; dims.sub_hi[k] = job.r->sub_hi[k];
            dims.upd_lo[k] = job.r->upd_lo[k]; dims.upd_hi[k] = job.r->upd_hi[k];
        }
    }
    if (pl.E == 0) {
        if (do_prefix) {
            for (int k = 0; k <= DDM_STAGES; ++k) mark(c, k);  // zero-length stages
            if (batch) L += launch_inst_offsets(ba, pl.off, pl.inst_off, s);
        }
        c->last_inst_off = batch ? pl.inst_off : nullptr;
        return DDM_OK;
    }
    uint32_t* vals_sorted = (pl.passes & 1) ? pl.vals1 : pl.vals0;
    Records rec = pl.rec;
    // Window path: the emission's rank tables replace the order arrays (the
    // range path reads ids by rank from them), so the sweep does not write them.
    if (pl.window) rec.sub_order = rec.upd_order = nullptr;
    if (pl.window || pl.join) {
        rec.windows = pl.windows;
        rec.win_shift = pl.win_shift;
    }
    if (dbg) {
        rec.dbg_who = dbg->who;
        rec.dbg_subset = dbg->subset;
        rec.dbg_updset = dbg->updset;
        if (!rec.dbg_who || !rec.dbg_subset || !rec.dbg_updset)
            rec.dbg_who = rec.dbg_subset = rec.dbg_updset = nullptr;
    }
    EmitArgs a{};
    a.d = job.d; a.n = pl.n; a.m = pl.m;
    a.dims = dims;
    a.rec = rec;
    a.cnt = pl.cnt; a.off = pl.off; a.cnt_a = pl.cnt_a; a.cursor_b = pl.cursor_b;
    a.subK = pl.subK; a.updK = pl.updK;
    a.pairs = pairs; a.cap = cap;
    a.id_bits = id_bits(pl.m);
    a.inst_sub_base = batch ? pl.n_base : nullptr;
    a.inst_upd_base = batch ? pl.m_base : nullptr;
    a.num_inst = job.num_inst;
    a.flag = nullptr;
    a.num_flagged = pl.num_flagged;
    a.sort_all = pl.join;
    a.lcap = pl.lcap;
    if (pl.window || pl.join) {
        a.flag = pl.flag;
        a.windows = pl.windows;
        a.win_shift = pl.win_shift;
        a.num_win = pl.num_win;
        a.lw_off = pl.join ? pl.lw_off : nullptr;  // NULL: fixed slots
        a.lw_fill = pl.lw_fill;
        a.lw = pl.lw;
        a.urank = pl.urank;
        a.srank = pl.window ? pl.srank : nullptr;
        a.wmeta = pl.window ? pl.wmeta : nullptr;
        a.wcand = pl.window ? pl.wcand : nullptr;
        a.cand_fill = pl.cand_fill;
        a.cand_cap = pl.cand_cap;
        a.lw_cap = pl.lw_cap;
    }
    a.vals = vals_sorted;
    a.surv = nullptr;
    if (pl.join && mode == Mode::Match && c->surv_keys) {
        a.surv = c->surv_keys;
        a.surv_cap = c->surv_cap;
        a.surv_fill = pl.surv_fill;
    }
  if (do_prefix) {
    mark(c, 0);
    if (batch) {
        L += launch_keybuild_batch(ba, (unsigned long long*)pl.keys0, pl.vals0, c->dstat, s);
    } else {
        L += launch_keybuild_d0(dims.sub_lo[0], dims.sub_hi[0], dims.upd_lo[0], dims.upd_hi[0],
                                pl.n, pl.m, (uint32_t*)pl.keys0, pl.vals0, c->dstat, s);
    }
    mark(c, 1);
    // The sweep scan writes one 16-byte rank record per endpoint at a random
    // id.  Into sectors absent from L2 such partial writes cost a DRAM read
    // each; clearing the record tables first (full-sector writes) leaves them
    // resident in L2 (scan 57 -> 44 us, clear included, for E = 2e6).  The
    // blocks of the sort's last pass do the clear while their tiles load.
    // (Overlapping it with the sort on a second stream was no faster.)  The
    // tables start 256-byte aligned and the next buffer starts 256-byte
    // aligned too, so rounding up to 16-byte words stays inside them.
    const size_t rec_words =
        ((size_t)((char*)(pl.rec.upd_order + pl.m) - (char*)pl.rec.s_lo) + 15) / 16;
    // The sweep's tile aggregates (S lowers, U lowers, S uppers per SCAN_TILE
    // positions) are counted by the sort's last pass, which knows every output
    // position, into the scan status words (zeroed above, 24 bytes per tile
    // against the 16 used); the sweep's tiles then need no look-back.
    uint32_t* kinds = !batch && ceil_div(pl.E, (uint64_t)SCAN_TILE) <= SCAN_KINDS_MAX_TILES
                          ? reinterpret_cast<uint32_t*>(pl.scan_status)
                          : nullptr;
    if (batch) {
        L += launch_radix_sort<unsigned long long>(
            (unsigned long long*)pl.keys0, pl.vals0, (unsigned long long*)pl.keys1, pl.vals1, pl.E,
            pl.passes, pl.sort, true, c->dstat, s, rec.s_lo, rec_words);
    } else {
        L += launch_radix_sort<uint32_t>((uint32_t*)pl.keys0, pl.vals0, (uint32_t*)pl.keys1,
                                         pl.vals1, pl.E, pl.passes, pl.sort, !c->keep_keys,
                                         c->dstat, s, rec.s_lo, rec_words, pl.sort_items, kinds);
    }
    // d = 1: the counts are formed inside the offsets scan (one kernel for a4
    // and a5), except for diagnostics, which also want the update counts.  The
    // sweep adds up the counts per id tile into the offsets scan's status words
    // (zeroed above; one word per tile), so that scan needs no look-back.
    const bool fused_counts = job.d == 1 && !dbg;
    unsigned long long* cnt_agg = fused_counts ? pl.off_status : nullptr;
    mark(c, 2);
    const int lsw = launch_sweep_scan(vals_sorted, pl.E, pl.n, pl.m, rec, pl.scan_status,
                                      c->dstat, s, kinds, cnt_agg);
    if (lsw < 0) return fail(c, DDM_ERR_INTERNAL, "sweep launch configuration");
    L += lsw;
    mark(c, 3);
    if (job.d == 1) {
        if (!fused_counts)
            L += launch_rank_count(rec, pl.n, pl.m, pl.cnt, dbg ? dbg->upd_cnt : nullptr, c->dstat, s);
    } else {
        L += launch_permute_keys(a, c->dstat, s);
        if (pl.join) {
            L += launch_window_offsets(pl.windows, pl.num_win, pl.lcap, pl.lw_off, pl.lw_total,
                                       pl.win_status, c->dstat, s);
            L += launch_tile_active(a, c->dstat, s);
            const int lj = launch_join(a, false, c->dstat, s);
            if (lj < 0) return fail(c, DDM_ERR_INTERNAL, "join launch configuration");
            L += lj;
        }
        L += launch_filter_count(a, c->dstat, s);  // with the join: flagged subscriptions only
    }
    mark(c, 4);
    if (dbg && dbg->sub_cnt && pl.n > 0)
        CK(cudaMemcpyAsync(dbg->sub_cnt, pl.cnt, pl.n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    const uint64_t off_cap = mode == Mode::Match && phase == Phase::All ? cap : ~0ull;
    if (pl.window && !fused_counts)
        return fail(c, DDM_ERR_INTERNAL, "window path without fused counts");
    // Window path: the rank tables of the emission are scattered from id order
    // here, in one launch (subscriptions by the offsets scan, updates beside it).
    if (fused_counts && pl.window && pl.n > 0) {
        const int lr = launch_rank_tables(rec, pl.n, pl.cnt, pl.off, off_cap, &c->dstat->K,
                                          pl.off_status, cnt_agg, a, c->dstat, s);
        if (lr < 0) return fail(c, DDM_ERR_INTERNAL, "rank tables launch configuration");
        L += lr;
    } else if (fused_counts) {
        L += launch_rank_offsets(rec, pl.n, pl.cnt, pl.off, off_cap, &c->dstat->K, pl.off_status,
                                 c->dstat, s, cnt_agg);
    } else
        L += launch_offsets(pl.cnt, pl.n, pl.off, off_cap, &c->dstat->K, pl.off_status, c->dstat, s);
    if (batch) L += launch_inst_offsets(ba, pl.off, pl.inst_off, s);
  }
  if (do_suffix) {
    mark(c, 5);
    if (pl.window) L += launch_win_setup(a, c->dstat, s);
    mark(c, 6);
    if (pl.window) L += launch_emit_window(a, c->dstat, s);
    else if (pl.join && mode == Mode::Match) {
        const int lj = launch_join(a, true, c->dstat, s);
        if (lj < 0) return fail(c, DDM_ERR_INTERNAL, "join launch configuration");
        L += lj;
    }
    else if (mode == Mode::Match) L += launch_emit_ranges(a, c->dstat, s);
    mark(c, 7);
    if (c->defer_fallback && pl.window && mode == Mode::Match && phase == Phase::All) {
        c->fallback_args = a;  // range path of the flagged subscriptions, if any (ddm_match)
        c->fallback_pending = true;
        c->flag_count = pl.num_flagged;  // read by the next finish() only
    } else {
        if ((pl.window || pl.join) && mode == Mode::Match)
            L += launch_emit_ranges(a, c->dstat, s);  // flagged subscriptions only
        if (mode == Mode::Match) L += launch_segment_sort(a, c->dstat, s);
    }
    mark(c, 8);
  }
    CK(cudaGetLastError());
    c->last_inst_off = batch ? pl.inst_off : nullptr;
    return DDM_OK;
}

int enqueue_plain(ddm_ctx* c, const ddm_regions* r, Mode mode, int32_t* pairs, uint64_t cap,
                  const DebugOut* dbg) {
    Job job;
    job.d = r->d; job.n = r->n; job.m = r->m; job.r = r;
    return enqueue(c, job, mode, pairs, cap, dbg);
}

// Reads the device status and maps it to a return code.
int finish(ddm_ctx* c, uint64_t* K_out) {
    if (c->hstat_dev) {
        PdlScope pdl_scope(c->pdl);
        c->stats.launches += launch_publish(c->dstat, c->hstat_dev, c->flag_count, c->stream);
        c->flag_count = nullptr;  // one use: the workspace may move before the next call
        CK(cudaGetLastError());
    } else {
        CK(cudaMemcpyAsync(c->hstat, c->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                           c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    if (c->prof) {
        for (int k = 0; k < DDM_STAGES; ++k) {
            float ms = 0.f;
            if (c->prof >= 2 && k != c->prof - 2) {
                c->stats.stage_ms[k] = 0.0;
                continue;
            }
            if (cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]) != cudaSuccess) {
                cudaGetLastError();
                ms = 0.f;
            }
            c->stats.stage_ms[k] = ms;
        }
    }
    const DevStatus& h = *c->hstat;
    if (K_out) *K_out = h.K;
    switch (h.error) {
        case DDM_OK: c->err.clear(); return DDM_OK;
        case DDM_ERR_INVALID:
            return fail(c, DDM_ERR_INVALID, "input has NaN coordinates or lo > hi");
        case DDM_ERR_CAPACITY:
            return fail(c, DDM_ERR_CAPACITY, "output capacity too small for " +
                                                 std::to_string(h.K) + " pairs");
        case DDM_ERR_DEVICE_TIMEOUT:
            return fail(c, DDM_ERR_DEVICE_TIMEOUT,
                        "a device-side wait timed out (stage " + std::to_string(h.detail) + ")");
        default:
            return fail(c, DDM_ERR_INTERNAL,
                        "device consistency check failed (stage " + std::to_string(h.detail) + ")");
    }
}

}  // namespace

extern "C" {

int ddm_create(ddm_ctx** out, int device, void* cuda_stream, size_t mem_budget_bytes) {
    if (!out) return DDM_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return DDM_ERR_CUDA;
    }
    ddm_ctx* c = new ddm_ctx();
    c->device = device;
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    c->budget = mem_budget_bytes;
    DeviceGuard g(device);
    // The host mirror of the status is mapped pinned memory, which a kernel
    // writes directly (else plain pinned memory and a copy).
    if (cudaMalloc(&c->dstat, sizeof(DevStatus)) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return DDM_ERR_NOMEM;
    }
    if (cudaHostAlloc(&c->hstat, sizeof(DevStatus), cudaHostAllocMapped) == cudaSuccess) {
        if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->hstat_dev), c->hstat, 0) !=
            cudaSuccess) {
            cudaGetLastError();
            c->hstat_dev = nullptr;
        }
    } else {
        cudaGetLastError();
        c->hstat = nullptr;
        if (cudaMallocHost(&c->hstat, sizeof(DevStatus)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(c->dstat);
            delete c;
            return DDM_ERR_NOMEM;
        }
    }
    memset(c->hstat, 0, sizeof(DevStatus));
    *out = c;
    return DDM_OK;
}

int ddm_destroy(ddm_ctx* c) {
    if (!c) return DDM_OK;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->ws) cudaFree(c->ws);
    if (c->io) cudaFree(c->io);
    if (c->out) cudaFree(c->out);
    if (c->sv) cudaFree(c->sv);
    if (c->dstat) cudaFree(c->dstat);
    if (c->hstat) cudaFreeHost(c->hstat);
    delete c;
    return DDM_OK;
}

const char* ddm_last_error(const ddm_ctx* c) { return c ? c->err.c_str() : "null context"; }

int ddm_set_profiling(ddm_ctx* c, int enable) {
    if (!c) return DDM_ERR_INVALID;
    if (enable < 0 || enable >= 2 + DDM_STAGES)
        return fail(c, DDM_ERR_INVALID, "profiling mode must be 0, 1 or 2 + stage");
    DeviceGuard g(c->device);
    if (enable && !c->ev[0]) {
        for (auto& e : c->ev) CK(cudaEventCreate(&e));
    }
    c->prof = enable;
    return DDM_OK;
}

int ddm_set_param(ddm_ctx* c, int param, int64_t value) {
    if (!c) return DDM_ERR_INVALID;
    if (param == DDM_PARAM_WIN_SHIFT) {
        if (value < 6 || value > 10) return fail(c, DDM_ERR_INVALID, "window shift must be 6..10");
        c->win_shift = (int)value;
        return DDM_OK;
    }
    if (param == DDM_PARAM_ND_PATH) {
        if (value < 0 || value > 2) return fail(c, DDM_ERR_INVALID, "nd path must be 0..2");
        c->nd_path = (int)value;
        return DDM_OK;
    }
    if (param == DDM_PARAM_SWEEP_DIM) {
        if (value < 0 || value > 1) return fail(c, DDM_ERR_INVALID, "sweep dim must be 0 or 1");
        c->sweep_dim = (int)value;
        return DDM_OK;
    }
    if (param == DDM_PARAM_SORT_ITEMS) {
        if (value != 12 && value != 16 && value != 18)
            return fail(c, DDM_ERR_INVALID, "sort items must be 12, 16 or 18");
        c->sort_items = (int)value;
        return DDM_OK;
    }
    if (param == DDM_PARAM_JOIN_SHIFT) {
        if (value < 9 || value > 11) return fail(c, DDM_ERR_INVALID, "join shift must be 9..11");
        c->join_shift = (int)value;
        return DDM_OK;
    }
    if (param == DDM_PARAM_ND_WRITE) {
        if (value < 0 || value > 2) return fail(c, DDM_ERR_INVALID, "nd write must be 0..2");
        c->nd_write = (int)value;
        return DDM_OK;
    }
    if (param == DDM_PARAM_PDL) {
        if (value < 0 || value > 1) return fail(c, DDM_ERR_INVALID, "pdl must be 0 or 1");
        c->pdl = value != 0;
        return DDM_OK;
    }
    return fail(c, DDM_ERR_INVALID, "unknown parameter");
}

int ddm_get_stats(const ddm_ctx* c, ddm_stats* out) {
    if (!c || !out) return DDM_ERR_INVALID;
    *out = c->stats;
    return DDM_OK;
}

// Dimension order of a plain call (DDM_PARAM_SWEEP_DIM).  Section 3 of the
// paper reduces d dimensions to the logical "and" of d one-dimensional tests,
// so any order gives the same pairs; the cost, though, grows with the pairs
// that intersect in the swept dimension (every one is a candidate of the
// filter) and, for the tiled join, in the pruning dimension.  With the
// automatic choice each dimension's one-dimensional pair count is computed
// exactly (a d = 1 count pass) and the dimensions are taken in increasing
// order of it.  `out` receives the reordered descriptor; `hold` owns its
// pointer arrays.
int order_dims(ddm_ctx* c, const ddm_regions* r, ddm_regions* out,
               std::vector<const float*>& hold) {
    *out = *r;
    for (int k = 0; k < DDM_MAX_DIMS; ++k) c->stats.dim_order[k] = (uint32_t)k;
    const int d = r->d;
    if (c->sweep_dim != 1 || d < 2 || r->n == 0 || r->m == 0) return DDM_OK;
    std::vector<std::pair<uint64_t, int>> cnt(d);
    for (int k = 0; k < d; ++k) {
        ddm_regions r1{};
        r1.d = 1; r1.n = r->n; r1.m = r->m;
        r1.sub_lo = &r->sub_lo[k]; r1.sub_hi = &r->sub_hi[k];
        r1.upd_lo = &r->upd_lo[k]; r1.upd_hi = &r->upd_hi[k];
        uint64_t K = 0;
        int rc = enqueue_plain(c, &r1, Mode::Count, nullptr, 0, nullptr);
        if (rc) return rc;
        rc = finish(c, &K);
        if (rc) return rc;
        cnt[k] = {K, k};
    }
    std::stable_sort(cnt.begin(), cnt.end());
    hold.assign(4 * (size_t)d, nullptr);
    for (int k = 0; k < d; ++k) {
        const int src = cnt[k].second;
        hold[k] = r->sub_lo[src];
        hold[d + k] = r->sub_hi[src];
        hold[2 * d + k] = r->upd_lo[src];
        hold[3 * d + k] = r->upd_hi[src];
        c->stats.dim_order[k] = (uint32_t)src;
    }
    out->sub_lo = &hold[0];
    out->sub_hi = &hold[d];
    out->upd_lo = &hold[2 * d];
    out->upd_hi = &hold[3 * d];
    return DDM_OK;
}

int ddm_count(ddm_ctx* c, const ddm_regions* r, uint64_t* K_out) {
    if (!c) return DDM_ERR_INVALID;
    int rc = check_regions(c, r);
    if (rc) return rc;
    DeviceGuard g(c->device);
    ddm_regions ro;
    std::vector<const float*> hold;
    rc = order_dims(c, r, &ro, hold);
    if (rc) return rc;
    rc = enqueue_plain(c, &ro, Mode::Count, nullptr, 0, nullptr);
    if (rc) return rc;
    uint64_t K = 0;
    rc = finish(c, &K);
    if (K_out) *K_out = K;
    if (rc == DDM_OK && ro.d > 1) c->surv_hint = K;  // sizes the next d > 1 match
    return rc;
}

}  // extern "C"

namespace {

constexpr int MATCH_RETRY = 1;  // not an error code: take the general path

// d > 1 pairs from the count pass's survivors (one sort of K keys) or from a
// second filter pass and per-segment sorts.  Measured on GB300: the survivors
// win at d >= 3 (the filter dominates), and for a batched call at d = 2 when
// the output is sparse (K of the last d > 1 call at most 4 (n + m): the
// per-segment sorts of tens of millions of short segments dominate); a plain
// d = 2 call keeps the write pass (a tie at N = 1e6, alpha = 1; the survivors'
// extra host round trip loses at smaller sizes; the sort of K keys loses with
// dense output).  DDM_PARAM_ND_WRITE overrides.
bool use_survivors(const ddm_ctx* c, int d, int64_t n, int64_t m, bool batch) {
    if (d < 2 || c->nd_write == 1) return false;
    if (c->nd_write == 2 || d >= 3) return true;
    return batch && c->surv_hint > 0 && c->surv_hint <= 4 * (uint64_t)(n + m);
}

// d > 1 with the tiled join: the count pass records every survivor as the key
// (i << id_bits(m)) | j, and the sorted pair list is one radix sort of those
// keys, unpacked into `pairs` -- no second filter pass and no per-segment
// sort.  The keys' room follows the previous d > 1 call's K.  Returns
// MATCH_RETRY (nothing written, the error text cleared) when the room cannot be
// had, when not every survivor fitted, or when subscriptions of overflowing
// windows went to the range path; the caller then runs the general pipeline.
// A batched job (job.num_inst > 0) works the same way on global ids; its pairs
// are unpacked to ids local to their instance and inst_offsets (num + 1, host)
// receives the instances' first pairs.
int match_from_survivors(ddm_ctx* c, const Job& job, int32_t* pairs, uint64_t cap,
                         uint64_t* K_out, uint64_t* inst_offsets = nullptr) {
    const int64_t n = job.n, m = job.m;
    const int num = job.num_inst;
    // Room for the keys: one slice per join window, sized by the window's
    // subscriptions.
    Plan pl0;
    pl0.layout(nullptr, job.d, n, m, Mode::Match, num, c->win_shift, c->nd_path, c->sort_items,
               c->join_shift);
    const uint32_t slices = pl0.num_win;
    const uint64_t hint = c->surv_hint;  // 0: this attempt is not sized from a known K
    if (slices == 0 || (hint && hint == c->surv_fail_K)) return MATCH_RETRY;
    // Per subscription of a window: twice the last K's share, plus 8.
    const uint64_t per_sub = ceil_div(2 * hint, (uint64_t)n) + 8;
    const uint64_t room = per_sub * (uint64_t)n;
    const int passes = (int)ceil_div((uint64_t)(id_bits(n) + id_bits(m)), RADIX_BITS);
    SortScratch sc{};
    size_t zb = 0, ze = 0;
    unsigned long long* kb[2] = {};
    unsigned long long* dpos = nullptr;
    auto carve = [&](Carve& cv) {
        kb[0] = cv.take<unsigned long long>(room);  // the windows' slices, then sort buffer
        kb[1] = cv.take<unsigned long long>(room);  // the compacted keys
        dpos = cv.take<unsigned long long>(slices + 1);
        carve_sort<unsigned long long>(cv, room, passes, sc, zb, ze);
    };
    Carve sz;
    carve(sz);
    if (ensure(c, &c->sv, &c->sv_size, sz.off + 256) != DDM_OK) {
        c->err.clear();
        return MATCH_RETRY;  // no room for the keys: the general path needs none
    }
    Carve cv;
    cv.base = c->sv;
    carve(cv);
    c->surv_keys = kb[0];
    c->surv_cap = per_sub;
    int rc = enqueue(c, job, Mode::Match, nullptr, 0, nullptr, Phase::Prefix);
    c->surv_keys = nullptr;
    if (rc) return rc;
    uint64_t K = 0;
    rc = finish(c, &K);
    if (rc) return rc;
    c->surv_hint = K;
    Plan pl;
    pl.layout(c->ws, job.d, n, m, Mode::Match, num, c->win_shift, c->nd_path, c->sort_items,
              c->join_shift);
    if (num > 0)
        CK(cudaMemcpy(inst_offsets, pl.inst_off, (num + 1) * sizeof(uint64_t),
                      cudaMemcpyDeviceToHost));
    std::vector<unsigned long long> fill(slices);
    uint32_t flagged = 0;
    CK(cudaMemcpy(fill.data(), pl.surv_fill, slices * sizeof(unsigned long long),
                  cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&flagged, pl.num_flagged, sizeof flagged, cudaMemcpyDeviceToHost));
    if (K_out) *K_out = K;
    if (K > cap)
        return fail(c, DDM_ERR_CAPACITY, "output capacity too small for " + std::to_string(K) +
                                             " pairs");
    // Window w holds ns_w subscriptions: its slice has ns_w * per_sub entries.
    // Its fill counts reserved slots, unused ones (set to ~0) included.
    std::vector<uint4> win(slices + 1);
    CK(cudaMemcpy(win.data(), pl.windows, (slices + 1) * sizeof(uint4), cudaMemcpyDeviceToHost));
    std::vector<unsigned long long> pos(slices + 1, 0);
    bool fits = flagged == 0;
    for (uint32_t w = 0; w < slices; ++w) {
        pos[w + 1] = pos[w] + fill[w];
        fits = fits && fill[w] <= (uint64_t)(win[w + 1].x - win[w].x) * per_sub;
    }
    const uint64_t T = pos[slices];
    if (!fits || T < K) {
        // Skewed windows (or overflowing ones): the general path for this
        // output size from now on, so the count pass is not paid twice again.
        if (hint == K) c->surv_fail_K = K;
        return MATCH_RETRY;
    }
    // Stages 5 (no set-up here), 6 (the sort and unpack of the survivors) and
    // 7 (no per-segment sort).
    mark(c, 5);
    mark(c, 6);
    if (K > 0) {
        cudaStream_t s = c->stream;
        PdlScope pdl_scope(c->pdl);
        CK(cudaMemcpyAsync(dpos, pos.data(), (slices + 1) * sizeof(unsigned long long),
                           cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(c->sv + zb, 0, ze - zb, s));
        c->stats.launches += launch_surv_compact(kb[0], pl.surv_fill, pl.windows, slices,
                                                 per_sub, dpos, kb[1], s);
        // Keys only; the T - K unused slots (~0) sort last.
        c->stats.launches += launch_radix_sort<unsigned long long>(
            kb[1], nullptr, kb[0], nullptr, T, passes, sc, false, c->dstat, s);
        const unsigned long long* sorted = kb[(passes & 1) ? 0 : 1];
        if (num > 0)
            c->stats.launches += launch_batch_unpack(sorted, K, id_bits(m), pl.n_base, pl.m_base,
                                                     num, pairs, s);
        else
            c->stats.launches += launch_delta_unpack(sorted, K, id_bits(m), pairs, s);
    }
    mark(c, 7);
    mark(c, 8);
    c->stats.survivor_calls++;
    return finish(c, K_out);
}

}  // namespace

extern "C" {

int ddm_match(ddm_ctx* c, const ddm_regions* r, int32_t* pairs, uint64_t cap, uint64_t* K_out) {
    if (!c) return DDM_ERR_INVALID;
    int rc = check_regions(c, r);
    if (rc) return rc;
    if (!pairs && cap > 0) return fail(c, DDM_ERR_INVALID, "pairs is NULL but cap > 0");
    DeviceGuard g(c->device);
    ddm_regions ro;
    std::vector<const float*> hold;
    rc = order_dims(c, r, &ro, hold);
    if (rc) return rc;
    if (use_survivors(c, ro.d, ro.n, ro.m, false) && c->nd_path != 2 && ro.n > 0 && ro.m > 0 &&
        pairs) {
        Job job;
        job.d = ro.d; job.n = ro.n; job.m = ro.m; job.r = &ro;
        rc = match_from_survivors(c, job, pairs, cap, K_out);
        if (rc != MATCH_RETRY) return rc;
    }
    c->defer_fallback = c->hstat_dev != nullptr;  // the flagged count reaches the host
    c->fallback_pending = false;
    rc = enqueue_plain(c, &ro, Mode::Match, pairs, cap, nullptr);
    c->defer_fallback = false;
    if (rc) {
        c->fallback_pending = false;
        c->flag_count = nullptr;
        return rc;
    }
    uint64_t K = 0;
    rc = finish(c, &K);
    c->flag_count = nullptr;
    if (c->fallback_pending) {  // window path: the range path only when it has work
        c->fallback_pending = false;
        if (rc == DDM_OK && c->hstat->flagged > 0) {
            PdlScope pdl_scope(c->pdl);
            c->stats.launches += launch_emit_ranges(c->fallback_args, c->dstat, c->stream);
            c->stats.launches += launch_segment_sort(c->fallback_args, c->dstat, c->stream);
            CK(cudaGetLastError());
            rc = finish(c, &K);
        }
    }
    if (K_out) *K_out = K;
    if (ro.d > 1 && (rc == DDM_OK || rc == DDM_ERR_CAPACITY)) c->surv_hint = K;
    return rc;
}

int ddm_match_host(ddm_ctx* c, const ddm_regions* r, int32_t* pairs, uint64_t cap,
                   uint64_t* K_out) {
    if (!c) return DDM_ERR_INVALID;
    int rc = check_regions(c, r);
    if (rc) return rc;
    if (!pairs && cap > 0) return fail(c, DDM_ERR_INVALID, "pairs is NULL but cap > 0");
    DeviceGuard g(c->device);
    const int d = r->d;
    const int64_t n = r->n, m = r->m;
    const float* const* src[4] = {r->sub_lo, r->sub_hi, r->upd_lo, r->upd_hi};
    // Stage the coordinates into the io buffer.
    Carve sizing;
    for (int a = 0; a < 4; ++a)
        for (int k = 0; k < d; ++k) sizing.take<float>(a < 2 ? n : m);
    rc = ensure(c, &c->io, &c->io_size, sizing.off + 256);
    if (rc) return rc;
    Carve cv;
    cv.base = c->io;
    std::vector<const float*> dp(4 * d);
    for (int a = 0; a < 4; ++a) {
        const int64_t cnt = a < 2 ? n : m;
        for (int k = 0; k < d; ++k) {
            float* dst = cv.take<float>(cnt);
            if (cnt > 0)
                CK(cudaMemcpyAsync(dst, src[a][k], cnt * sizeof(float), cudaMemcpyHostToDevice,
                                   c->stream));
            dp[a * d + k] = dst;
        }
    }
    ddm_regions dr0 = *r;
    dr0.sub_lo = &dp[0];
    dr0.sub_hi = &dp[d];
    dr0.upd_lo = &dp[2 * d];
    dr0.upd_hi = &dp[3 * d];
    ddm_regions dr;
    std::vector<const float*> hold;
    rc = order_dims(c, &dr0, &dr, hold);
    if (rc) return rc;
    // Run the pipeline up to the exact K, size the device output, then emit.
    Job job;
    job.d = dr.d; job.n = dr.n; job.m = dr.m; job.r = &dr;
    uint64_t K = 0;
    rc = enqueue(c, job, Mode::Match, nullptr, 0, nullptr, Phase::Prefix);
    if (rc) return rc;
    rc = finish(c, &K);
    if (rc) return rc;
    if (K_out) *K_out = K;
    if (K > cap) return fail(c, DDM_ERR_CAPACITY, "output capacity too small for " +
                                                      std::to_string(K) + " pairs");
    if (K == 0) return DDM_OK;
    rc = ensure(c, &c->out, &c->out_size, 2 * K * sizeof(int32_t));
    if (rc) return rc;
    int32_t* dpairs = reinterpret_cast<int32_t*>(c->out);
    rc = enqueue(c, job, Mode::Match, dpairs, K, nullptr, Phase::Suffix);
    if (rc) return rc;
    CK(cudaMemcpyAsync(pairs, dpairs, 2 * K * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    return finish(c, K_out);
}

int ddm_match_batch(ddm_ctx* c, int num, const ddm_regions* inst, int32_t* pairs, uint64_t cap,
                    uint64_t* inst_offsets, uint64_t* K_out) {
    if (!c) return DDM_ERR_INVALID;
    if (num < 0 || num > DDM_MAX_BATCH) return fail(c, DDM_ERR_INVALID, "num out of range");
    if (!inst_offsets) return fail(c, DDM_ERR_INVALID, "inst_offsets is NULL");
    if (num > 0 && !inst) return fail(c, DDM_ERR_INVALID, "inst is NULL");
    Job job;
    job.num_inst = num;
    job.inst = inst;
    job.d = num > 0 ? inst[0].d : 1;
    for (int b = 0; b < num; ++b) {
        int rc = check_regions(c, &inst[b]);
        if (rc) return rc;
        if (inst[b].d != job.d) return fail(c, DDM_ERR_INVALID, "instances differ in d");
        job.n += inst[b].n;
        job.m += inst[b].m;
        if (job.n + job.m > DDM_MAX_REGIONS)
            return fail(c, DDM_ERR_INVALID, "the instances together exceed DDM_MAX_REGIONS");
    }
    inst_offsets[0] = 0;
    if (num == 0) {
        if (K_out) *K_out = 0;
        return DDM_OK;
    }
    DeviceGuard g(c->device);
    if (pairs && use_survivors(c, job.d, job.n, job.m, true) && c->nd_path != 2 && job.n > 0 &&
        job.m > 0) {
        int rc = match_from_survivors(c, job, pairs, cap, K_out, inst_offsets);
        if (rc != MATCH_RETRY) return rc;
    }
    const Mode mode = pairs ? Mode::Match : Mode::Count;
    int rc = enqueue(c, job, mode, pairs, pairs ? cap : 0, nullptr);
    if (rc) return rc;
    CK(cudaMemcpyAsync(inst_offsets, c->last_inst_off, (num + 1) * sizeof(uint64_t),
                       cudaMemcpyDeviceToHost, c->stream));
    uint64_t K = 0;
    rc = finish(c, &K);
    if (K_out) *K_out = K;
    if (job.d > 1 && (rc == DDM_OK || rc == DDM_ERR_CAPACITY)) c->surv_hint = K;
    return rc;
}

}  // extern "C"

struct ddm_session {
    ddm_ctx* ctx = nullptr;
    float* coords = nullptr;  // device: sub_lo, sub_hi (d x n each), upd_lo, upd_hi (d x m)
    const float* ptrs[4][DDM_MAX_DIMS] = {};
    ddm_regions regions{};
    bool counted = false;     // a pipeline prefix is held in the workspace
    uint64_t K = 0;
    // Incremental matching (ddm_session_emit_delta): the coordinates of the
    // last delivered report (same layout as coords), and a work area for the
    // report (displacements, counters, per-dimension sorted update bounds,
    // the change keys and their sort).
    float* ref_coords = nullptr;
    size_t ref_size = 0;
    bool have_ref = false;    // a report was delivered (else: everything is new)
    char* dwork = nullptr;
    size_t dwork_size = 0;
    uint64_t delta_cap = 0;   // room for the keys of one report's changed pairs
    // The count phase as a CUDA graph: a session's shapes, coordinates and
    // workspace do not change, so after one direct run the kernels of
    // ddm_session_count are captured once and then replayed with a single
    // launch (host launch overhead dominates small requests).
    cudaGraphExec_t prefix_exec = nullptr;
    const char* prefix_ws = nullptr;  // workspace the graph was captured against
    uint64_t prefix_launches = 0;     // kernels in the graph
    int prefix_runs = 0;              // direct runs so far
    bool no_graph = false;            // capture failed once: stay direct
};

namespace {

Job session_job(const ddm_session* s) {
    Job job;
    job.d = s->regions.d; job.n = s->regions.n; job.m = s->regions.m;
    job.r = &s->regions;
    return job;
}

}  // namespace

extern "C" {

int ddm_session_create(ddm_session** out, int device, const ddm_regions* initial,
                       size_t mem_budget_bytes) {
    if (!out) return DDM_ERR_INVALID;
    *out = nullptr;
    ddm_ctx* c = nullptr;
    int rc = ddm_create(&c, device, nullptr, mem_budget_bytes);
    if (rc) return rc;
    rc = check_regions(c, initial);
    if (rc) { ddm_destroy(c); return rc; }
    DeviceGuard g(device);
    ddm_session* s = new ddm_session();
    s->ctx = c;
    c->keep_keys = true;  // the change report walks the sorted endpoint stream
    const int d = initial->d;
    const int64_t n = initial->n, m = initial->m;
    const size_t floats = (size_t)2 * d * (n + m);
    if (c->budget && floats * sizeof(float) > c->budget) {
        ddm_destroy(c);
        delete s;
        return DDM_ERR_NOMEM;
    }
    if (floats > 0 && cudaMalloc(&s->coords, floats * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        ddm_destroy(c);
        delete s;
        return DDM_ERR_NOMEM;
    }
    c->held += floats * sizeof(float);  // the resident coordinates count against the budget
    const float* const* src[4] = {initial->sub_lo, initial->sub_hi, initial->upd_lo, initial->upd_hi};
    float* p = s->coords;
    for (int a = 0; a < 4; ++a) {
        const int64_t cnt = a < 2 ? n : m;
        for (int k = 0; k < d; ++k) {
            if (cnt > 0 && cudaMemcpy(p, src[a][k], cnt * sizeof(float),
                                      cudaMemcpyDeviceToDevice) != cudaSuccess) {
                cudaGetLastError();
                ddm_session_destroy(s);
                return DDM_ERR_CUDA;
            }
            s->ptrs[a][k] = p;
            p += cnt;
        }
    }
    s->regions.d = d;
    s->regions.n = n;
    s->regions.m = m;
    s->regions.sub_lo = s->ptrs[0];
    s->regions.sub_hi = s->ptrs[1];
    s->regions.upd_lo = s->ptrs[2];
    s->regions.upd_hi = s->ptrs[3];
    *out = s;
    return DDM_OK;
}

int ddm_session_destroy(ddm_session* s) {
    if (!s) return DDM_OK;
    if (s->ctx) {
        DeviceGuard g(s->ctx->device);
        if (s->coords) cudaFree(s->coords);  // every session call is synchronous
        if (s->ref_coords) cudaFree(s->ref_coords);
        if (s->dwork) cudaFree(s->dwork);
        if (s->prefix_exec) cudaGraphExecDestroy(s->prefix_exec);
        ddm_destroy(s->ctx);
    }
    delete s;
    return DDM_OK;
}

const ddm_regions* ddm_session_regions(const ddm_session* s) { return s ? &s->regions : nullptr; }

const char* ddm_session_last_error(const ddm_session* s) {
    return s && s->ctx ? s->ctx->err.c_str() : "null session";
}

int ddm_session_drift(ddm_session* s, void* stream, uint64_t seed, uint64_t step, double sigma) {
    if (!s) return DDM_ERR_INVALID;
    ddm_ctx* c = s->ctx;
    DeviceGuard g(c->device);
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    DriftArgs a{};
    a.d = s->regions.d; a.n = s->regions.n; a.m = s->regions.m;
    for (int k = 0; k < a.d; ++k) {
        a.sub_lo[k] = const_cast<float*>(s->ptrs[0][k]);
        a.sub_hi[k] = const_cast<float*>(s->ptrs[1][k]);
        a.upd_lo[k] = const_cast<float*>(s->ptrs[2][k]);
        a.upd_hi[k] = const_cast<float*>(s->ptrs[3][k]);
    }
    a.seed = seed; a.step = step; a.sigma = sigma;
    PdlScope pdl_scope(c->pdl);
    c->stats.launches += launch_drift(a, c->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    s->counted = false;
    return DDM_OK;
}

// The count phase of a session on c->stream: replayed from its graph when one
// exists, captured after the first direct run, direct otherwise (legacy default
// stream, profiling, or a capture that failed).
static int session_prefix(ddm_session* s) {
    ddm_ctx* c = s->ctx;
    const Job job = session_job(s);
    const bool graphable = c->stream != nullptr && !c->prof && !s->no_graph;
    if (s->prefix_exec && (!graphable || s->prefix_ws != c->ws)) {
        cudaGraphExecDestroy(s->prefix_exec);
        s->prefix_exec = nullptr;
    }
    if (graphable && !s->prefix_exec && s->prefix_runs >= 1) {
        cudaGraph_t graph = nullptr;
        const uint64_t l0 = c->stats.launches, calls0 = c->stats.calls;
        bool ok = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        int rc = ok ? enqueue(c, job, Mode::Match, nullptr, 0, nullptr, Phase::Prefix) : DDM_OK;
        ok = ok && cudaStreamEndCapture(c->stream, &graph) == cudaSuccess && rc == DDM_OK && graph;
        if (ok) ok = cudaGraphInstantiate(&s->prefix_exec, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (ok) {
            s->prefix_ws = c->ws;
            s->prefix_launches = c->stats.launches - l0;
        } else {
            s->prefix_exec = nullptr;
            s->no_graph = true;
        }
        c->stats.launches = l0;  // counted when the graph runs
        c->stats.calls = calls0;
    }
    if (s->prefix_exec) {
        CK(cudaGraphLaunch(s->prefix_exec, c->stream));
        c->stats.launches += s->prefix_launches;
        c->stats.calls++;
        return DDM_OK;
    }
    s->prefix_runs++;
    return enqueue(c, job, Mode::Match, nullptr, 0, nullptr, Phase::Prefix);
}

int ddm_session_count(ddm_session* s, void* stream, uint64_t* K_out) {
    if (!s) return DDM_ERR_INVALID;
    ddm_ctx* c = s->ctx;
    DeviceGuard g(c->device);
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    s->counted = false;
    int rc = session_prefix(s);
    if (rc) return rc;
    uint64_t K = 0;
    rc = finish(c, &K);
    if (rc) return rc;
    s->K = K;
    s->counted = true;
    if (K_out) *K_out = K;
    return DDM_OK;
}

int ddm_session_K(ddm_session* s, uint64_t* K_out) {
    if (!s || !K_out) return DDM_ERR_INVALID;
    *K_out = s->K;
    return DDM_OK;
}

int ddm_session_emit(ddm_session* s, void* stream, int32_t* pairs, uint64_t cap, uint64_t* K_out) {
    if (!s) return DDM_ERR_INVALID;
    ddm_ctx* c = s->ctx;
    if (!s->counted) return fail(c, DDM_ERR_INVALID, "ddm_session_emit needs ddm_session_count first");
    if (K_out) *K_out = s->K;
    if (s->K > cap) return fail(c, DDM_ERR_CAPACITY, "output capacity too small");
    if (!pairs && s->K > 0) return fail(c, DDM_ERR_INVALID, "pairs is NULL");
    DeviceGuard g(c->device);
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    s->counted = false;  // the emission consumes the kept state
    int rc = enqueue(c, session_job(s), Mode::Match, pairs, cap, nullptr, Phase::Suffix);
    if (rc) return rc;
    return finish(c, K_out);
}

int ddm_session_emit_delta(ddm_session* s, void* stream, int32_t* added, uint64_t cap_added,
                           int32_t* removed, uint64_t cap_removed, uint64_t* n_added,
                           uint64_t* n_removed) {
    if (!s) return DDM_ERR_INVALID;
    ddm_ctx* c = s->ctx;
    DeviceGuard g(c->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    c->stream = st;
    if (!s->counted && !s->have_ref)
        return fail(c, DDM_ERR_INVALID,
                    "the first ddm_session_emit_delta needs ddm_session_count first");
    if ((!added && cap_added) || (!removed && cap_removed))
        return fail(c, DDM_ERR_INVALID, "output is NULL but its capacity is not 0");
    if ((reinterpret_cast<uintptr_t>(added) | reinterpret_cast<uintptr_t>(removed)) & 7u)
        return fail(c, DDM_ERR_INVALID, "added and removed must be 8-byte aligned");
    const Job job = session_job(s);
    const int d = job.d;
    const int64_t n = job.n, m = job.m;
    const size_t coord_bytes = (size_t)2 * d * (n + m) * sizeof(float);
    int rc;
    // Room for the reference coordinates before anything is consumed.
    {
        char* p = reinterpret_cast<char*>(s->ref_coords);
        rc = ensure(c, &p, &s->ref_size, std::max<size_t>(coord_bytes, 16));
        s->ref_coords = reinterpret_cast<float*>(p);
        if (rc) return rc;
    }
    if (!s->have_ref) {  // the first report: every pair of this timestep is new
        if (n_added) *n_added = s->K;
        if (n_removed) *n_removed = 0;
        if (s->K > cap_added)
            return fail(c, DDM_ERR_CAPACITY, "change report does not fit: " +
                                                 std::to_string(s->K) + " added, 0 removed");
        if (s->K && !added) return fail(c, DDM_ERR_INVALID, "output is NULL");
        s->counted = false;  // the emission consumes the kept state
        rc = enqueue(c, job, Mode::Match, added, cap_added, nullptr, Phase::Suffix);
        if (rc) return rc;
        if (coord_bytes)
            CK(cudaMemcpyAsync(s->ref_coords, s->coords, coord_bytes, cudaMemcpyDeviceToDevice, st));
        rc = finish(c, nullptr);
        if (rc) return rc;
        s->have_ref = true;
        return DDM_OK;
    }
    // Later reports: candidates from the coordinates that moved.  A timestep
    // not counted yet is counted here, on the same stream without a host round
    // trip (the report needs the sorted stream and rank records, not K); its
    // prologue has cleared the status block.
    bool fresh = false;
    if (!s->counted) {
        rc = session_prefix(s);
        if (rc) return rc;
        s->counted = true;
        fresh = true;
    }
    Plan pl;  // the layout of the count phase that produced the sorted stream
    pl.layout(c->ws, d, n, m, Mode::Match, 0, c->win_shift, c->nd_path, c->sort_items,
              c->join_shift);
    DeltaArgs a{};
    a.d = d; a.n = (uint32_t)n; a.m = (uint32_t)m;
    a.E = (uint32_t)pl.E;
    a.keys = reinterpret_cast<const uint32_t*>((pl.passes & 1) ? pl.keys1 : pl.keys0);
    a.vals = (pl.passes & 1) ? pl.vals1 : pl.vals0;
    for (int q = 0; q < 4; ++q)
        for (int k = 0; k < d; ++k) {
            const float* nowp = s->ptrs[q][k];
            const float* refp = s->ref_coords + (nowp - s->coords);  // same layout
            switch (q) {
                case 0: a.now.sub_lo[k] = nowp; a.ref.sub_lo[k] = refp; break;
                case 1: a.now.sub_hi[k] = nowp; a.ref.sub_hi[k] = refp; break;
                case 2: a.now.upd_lo[k] = nowp; a.ref.upd_lo[k] = refp; break;
                default: a.now.upd_hi[k] = nowp; a.ref.upd_hi[k] = refp; break;
            }
        }
    a.rec = pl.rec;
    a.ibits = id_bits(n);
    a.jbits = id_bits(m);
    a.counters = &c->dstat->aux[2];  // [2] added, [3] removed, [4] write cursor
    uint32_t* flags = reinterpret_cast<uint32_t*>(&c->dstat->aux[5]);
    const int passes = (int)ceil_div((uint64_t)(1 + a.ibits + a.jbits), RADIX_BITS);
    // The change keys' room: grows when a report overflows it (then rerun).
    if (s->delta_cap == 0) s->delta_cap = std::max<uint64_t>(4096, s->K / 64);
    for (int attempt = 0; attempt < 3; ++attempt) {
        const uint64_t cap = s->delta_cap;
        SortScratch sc32{}, sc64{};
        size_t zb32 = 0, ze32 = 0, zb64 = 0, ze64 = 0;
        uint32_t *tmp[2] = {}, *vb[2] = {};
        uint4* pk = nullptr;
        unsigned long long* kb[2] = {};
        auto carve = [&](Carve& cv) {
            a.disp = cv.take<unsigned long long>(DDM_MAX_DIMS);
            for (int k = 1; k < d; ++k) {
                a.lo_key[k - 1] = cv.take<uint32_t>(m);
                a.lo_id[k - 1] = cv.take<uint32_t>(m);
                a.hi_key[k - 1] = cv.take<uint32_t>(m);
                a.hi_id[k - 1] = cv.take<uint32_t>(m);
            }
            tmp[0] = cv.take<uint32_t>(d > 1 ? m : 0);
            tmp[1] = cv.take<uint32_t>(d > 1 ? m : 0);
            if (d > 1) carve_sort<uint32_t>(cv, (uint64_t)m, 4, sc32, zb32, ze32);
            pk = cv.take<uint4>(pl.E);
            a.ulo = cv.take<uint4>(2 * m);
            a.uhi = cv.take<uint4>(2 * m);
            kb[0] = cv.take<unsigned long long>(cap);
            kb[1] = cv.take<unsigned long long>(cap);
            vb[0] = cv.take<uint32_t>(cap);
            vb[1] = cv.take<uint32_t>(cap);
            carve_sort<unsigned long long>(cv, cap, passes, sc64, zb64, ze64);
        };
        Carve sz;
        carve(sz);
        rc = ensure(c, &s->dwork, &s->dwork_size, sz.off + 256);
        if (rc) return rc;
        Carve cv;
        cv.base = s->dwork;
        carve(cv);
        a.pk = pk;
        a.keys_out = kb[0];
        a.cap = cap;
        PdlScope pdl_scope(c->pdl);
        uint64_t& L = c->stats.launches;
        if (!(fresh && attempt == 0)) CK(cudaMemsetAsync(c->dstat, 0, sizeof(DevStatus), st));
        CK(cudaMemsetAsync(a.disp, 0, DDM_MAX_DIMS * sizeof(unsigned long long), st));
        L += launch_delta_disp(a, c->dstat, st);
        L += launch_delta_refk(a, pk, st);
        if (d > 1 && m > 0) {
            L += launch_delta_keys(a, st);
            for (int k = 1; k < d; ++k)
                for (int b = 0; b < 2; ++b) {
                    CK(cudaMemsetAsync(s->dwork + zb32, 0, ze32 - zb32, st));
                    uint32_t* key = const_cast<uint32_t*>(b ? a.hi_key[k - 1] : a.lo_key[k - 1]);
                    uint32_t* id = const_cast<uint32_t*>(b ? a.hi_id[k - 1] : a.lo_id[k - 1]);
                    L += launch_radix_sort<uint32_t>(key, id, tmp[0], tmp[1], (uint64_t)m, 4,
                                                     sc32, false, c->dstat, st);
                }
        }
        L += launch_delta_cand(a, c->dstat, st);
        L += launch_delta_pad(a, st);
        CK(cudaMemsetAsync(s->dwork + zb64, 0, ze64 - zb64, st));
        L += launch_radix_sort<unsigned long long>(kb[0], vb[0], kb[1], vb[1], cap, passes, sc64,
                                                   false, c->dstat, st);
        L += launch_delta_finish(a, kb[passes & 1], added, cap_added, removed, cap_removed, flags,
                                 s->ref_coords, s->coords, coord_bytes / sizeof(float), st);
        rc = finish(c, nullptr);
        if (rc) return rc;
        if (fresh && attempt == 0) s->K = c->hstat->K;  // the count phase's K
        const uint64_t na = c->hstat->aux[2], nr = c->hstat->aux[3];
        const uint32_t f = static_cast<uint32_t>(c->hstat->aux[5]);
        if (n_added) *n_added = na;
        if (n_removed) *n_removed = nr;
        if (f & DELTA_RERUN) {  // nothing was written or committed: again, with room
            s->delta_cap = (na + nr) + (na + nr) / 4 + 4096;
            continue;
        }
        if (f & DELTA_CAPACITY)
            return fail(c, DDM_ERR_CAPACITY, "change report does not fit: " + std::to_string(na) +
                                                 " added, " + std::to_string(nr) + " removed");
        // The next report's room follows this one's size (the sort's cost is
        // proportional to the room).
        s->delta_cap = (na + nr) + (na + nr) / 4 + 4096;
        s->counted = false;  // one report per timestep: the next one needs a new count
        return DDM_OK;
    }
    return fail(c, DDM_ERR_INTERNAL, "change report: key room kept overflowing");
}

}  // extern "C"

extern "C" {

// The paper's comparison matchers (Algorithms 2 and 3) on the GPU, with the
// result contract of ddm_match.  `pairs` NULL (and cap 0): count only.
static int baseline_match(ddm_ctx* c, const ddm_regions* r, int32_t* pairs, uint64_t cap,
                          uint64_t* K_out, bool itm) {
    if (!c) return DDM_ERR_INVALID;
    int rc = check_regions(c, r);
    if (rc) return rc;
    if (!pairs && cap > 0) return fail(c, DDM_ERR_INVALID, "pairs is NULL but cap > 0");
    if (pairs && (reinterpret_cast<uintptr_t>(pairs) & 7u))
        return fail(c, DDM_ERR_INVALID, "pairs must be 8-byte aligned");
    DeviceGuard g(c->device);
    const int d = r->d;
    const int64_t n = r->n, m = r->m;
    // Workspace: zeroed part (offsets scan status, sort status and group
    // sums), then counts, offsets, and for the tree the sort buffers and nodes.
    uint32_t P = 1;
    while (P < (uint64_t)m) P <<= 1;
    const uint64_t stiles = sort_tiles<uint32_t>((uint64_t)m);
    const int passes = 4;
    auto carve = [&](Carve& cv, SortScratch& sc, unsigned long long*& ost, size_t& zero,
                     uint32_t*& cnt, unsigned long long*& off, uint32_t* kv[4], uint32_t*& tree) {
        ost = cv.take<unsigned long long>(ceil_div((uint64_t)n, OFF_TILE) + 2);
        sc.status = cv.take<unsigned long long>(itm ? (size_t)passes * sort_status_stride(m) : 0);
        sc.total = cv.take<unsigned long long>(1);
        const size_t gw = itm ? sort_group_words(stiles, passes) : 0;
        sc.grp = gw ? cv.take<uint32_t>(gw) : nullptr;
        zero = (cv.off + 255) & ~(size_t)255;
        cnt = cv.take<uint32_t>(n);
        off = cv.take<unsigned long long>(n + 1);
        sc.tile_hist = cv.take<uint32_t>(itm ? stiles * RADIX : 0);
        sc.offs = cv.take<unsigned long long>(itm ? stiles * RADIX + 1 : 0);
        for (int q = 0; q < 4; ++q) kv[q] = cv.take<uint32_t>(itm ? m : 0);
        tree = cv.take<uint32_t>(itm ? 2 * (size_t)P : 0);
    };
    Carve sizing;
    SortScratch sc{};
    unsigned long long *ost = nullptr, *off = nullptr;
    size_t zero = 0;
    uint32_t *cnt = nullptr, *tree = nullptr, *kv[4] = {};
    carve(sizing, sc, ost, zero, cnt, off, kv, tree);
    rc = ensure(c, &c->ws, &c->ws_size, sizing.off + 256);
    if (rc) return rc;
    Carve cv;
    cv.base = c->ws;
    carve(cv, sc, ost, zero, cnt, off, kv, tree);
    cudaStream_t s = c->stream;
    PdlScope pdl_scope(c->pdl);
    CK(cudaMemsetAsync(c->dstat, 0, sizeof(DevStatus), s));
    CK(cudaMemsetAsync(c->ws, 0, zero, s));
    c->stats.calls++;
    uint64_t& L = c->stats.launches;
    DimPtrs dims{};
    for (int k = 0; k < d; ++k) {
        dims.sub_lo[k] = r->sub_lo[k]; dims.sub_hi[k] = r->sub_hi[k];
        dims.upd_lo[k] = r->upd_lo[k]; dims.upd_hi[k] = r->upd_hi[k];
    }
    const uint64_t off_cap = pairs ? cap : ~0ull;
    if (!itm) {
        L += launch_bf_count(dims, d, n, m, cnt, c->dstat, s);
        L += launch_offsets(cnt, n, off, off_cap, &c->dstat->K, ost, c->dstat, s);
        if (pairs) L += launch_bf_write(dims, d, n, m, off, pairs, c->dstat, s);
    } else {
        L += launch_itm_keys(dims, d, m, kv[0], kv[1], c->dstat, s);
        if (m > 0)
            L += launch_radix_sort<uint32_t>(kv[0], kv[1], kv[2], kv[3], (uint64_t)m, passes, sc,
                                             false, c->dstat, s);
        ItmTree t{};
        t.P = P; t.m = (uint32_t)m;
        t.lo_sorted = kv[(passes & 1) * 2];
        t.id_sorted = kv[(passes & 1) * 2 + 1];
        t.tree = tree;
        L += launch_itm_build(t, dims.upd_hi[0], c->dstat, s);
        L += launch_itm_query(t, dims, d, n, m, cnt, nullptr, nullptr, c->dstat, s);
        L += launch_offsets(cnt, n, off, off_cap, &c->dstat->K, ost, c->dstat, s);
        if (pairs && n > 0 && m > 0) {
            L += launch_itm_query(t, dims, d, n, m, cnt, off, pairs, c->dstat, s);
            EmitArgs a{};  // per-segment sort by update id (every segment)
            a.d = d; a.n = n; a.m = m;
            a.cnt = cnt; a.off = off; a.pairs = pairs; a.cap = cap;
            a.id_bits = id_bits(m);
            L += launch_segment_sort(a, c->dstat, s);
        }
    }
    CK(cudaGetLastError());
    return finish(c, K_out);
}

int ddm_match_bruteforce(ddm_ctx* c, const ddm_regions* r, int32_t* pairs, uint64_t cap,
                         uint64_t* K_out) {
    return baseline_match(c, r, pairs, cap, K_out, false);
}

int ddm_match_itm(ddm_ctx* c, const ddm_regions* r, int32_t* pairs, uint64_t cap,
                  uint64_t* K_out) {
    return baseline_match(c, r, pairs, cap, K_out, true);
}

int ddm_match_grid(ddm_ctx* c, const ddm_regions* r, uint32_t cells_per_dim, int32_t* pairs,
                   uint64_t cap, uint64_t* K_out, uint32_t* grid_out) {
    if (!c) return DDM_ERR_INVALID;
    int rc = check_regions(c, r);
    if (rc) return rc;
    if (!pairs && cap > 0) return fail(c, DDM_ERR_INVALID, "pairs is NULL but cap > 0");
    if (pairs && (reinterpret_cast<uintptr_t>(pairs) & 7u))
        return fail(c, DDM_ERR_INVALID, "pairs must be 8-byte aligned");
    if (cells_per_dim > GRID_MAX_CELLS)
        return fail(c, DDM_ERR_INVALID, "cells_per_dim out of range");
    DeviceGuard g(c->device);
    const int d = r->d;
    const int64_t n = r->n, m = r->m;
    cudaStream_t s = c->stream;
    PdlScope pdl_scope(c->pdl);
    uint64_t& L = c->stats.launches;
    c->stats.calls++;
    DimPtrs dims{};
    for (int k = 0; k < d; ++k) {
        dims.sub_lo[k] = r->sub_lo[k]; dims.sub_hi[k] = r->sub_hi[k];
        dims.upd_lo[k] = r->upd_lo[k]; dims.upd_hi[k] = r->upd_hi[k];
    }
    if (grid_out)
        for (int k = 0; k < GRID_MAX_DIMS; ++k) grid_out[k] = 1;
    if (n + m == 0) {
        if (K_out) *K_out = 0;
        c->err.clear();
        return DDM_OK;
    }
    // 1. Bounding box of the gridded dimensions (and validation); the mesh.
    rc = ensure(c, &c->ws, &c->ws_size, 256 + sizeof(GridScratch));
    if (rc) return rc;
    GridScratch* gs = reinterpret_cast<GridScratch*>(c->ws);
    CK(cudaMemsetAsync(c->dstat, 0, sizeof(DevStatus), s));
    CK(cudaMemsetAsync(gs, 0, sizeof(GridScratch), s));
    L += launch_grid_bounds(dims, d, n, m, gs, c->dstat, s);
    GridScratch hg{};
    CK(cudaMemcpyAsync(&hg, gs, sizeof hg, cudaMemcpyDeviceToHost, s));
    rc = finish(c, nullptr);
    if (rc) return rc;
    const GridPlan plan = grid_plan(hg, d, (uint64_t)(n + m), cells_per_dim);
    if (grid_out)
        for (int k = 0; k < plan.dg; ++k) grid_out[k] = plan.g[k];
    // 2. Memberships per cell, and their offsets.
    const uint64_t G = plan.G;
    Carve sizing;
    auto layout = [&](Carve& cv, uint32_t** cz, unsigned long long** st2,
                      unsigned long long** offs, uint32_t*& cnt, uint32_t*& cursor,
                      unsigned long long*& ost, unsigned long long*& off, size_t& zero) {
        for (int q = 0; q < 4; ++q) cz[q] = cv.take<uint32_t>(G);  // counts s/u, cursors s/u
        for (int q = 0; q < 2; ++q) st2[q] = cv.take<unsigned long long>(ceil_div(G, OFF_TILE) + 2);
        cnt = cv.take<uint32_t>(n);
        cursor = cv.take<uint32_t>(n);
        ost = cv.take<unsigned long long>(ceil_div((uint64_t)n, OFF_TILE) + 2);
        zero = (cv.off + 255) & ~(size_t)255;
        for (int q = 0; q < 2; ++q) offs[q] = cv.take<unsigned long long>(G + 1);
        off = cv.take<unsigned long long>(n + 1);
    };
    uint32_t* cz[4];
    unsigned long long *st2[2], *offs[2], *ost, *off;
    uint32_t *cnt, *cursor;
    size_t zero = 0;
    layout(sizing, cz, st2, offs, cnt, cursor, ost, off, zero);
    rc = ensure(c, &c->ws, &c->ws_size, sizing.off + 256);
    if (rc) return rc;
    Carve cv;
    cv.base = c->ws;
    layout(cv, cz, st2, offs, cnt, cursor, ost, off, zero);
    CK(cudaMemsetAsync(c->ws, 0, zero, s));
    L += launch_grid_count(dims, n, m, plan, cz[0], cz[1], c->dstat, s);
    L += launch_offsets(cz[0], (int64_t)G, offs[0], ~0ull, &c->dstat->aux[0], st2[0], c->dstat, s);
    L += launch_offsets(cz[1], (int64_t)G, offs[1], ~0ull, &c->dstat->aux[1], st2[1], c->dstat, s);
    rc = finish(c, nullptr);
    if (rc) return rc;
    const uint64_t Ts = c->hstat->aux[0], Tu = c->hstat->aux[1];
    // 3. Memberships by cell, brute force per cell (count), offsets, write, sort.
    rc = ensure(c, &c->out, &c->out_size, 4 * (Ts + Tu) + 512);
    if (rc) return rc;
    uint32_t* ent_s = reinterpret_cast<uint32_t*>(c->out);
    uint32_t* ent_u = ent_s + ((Ts + 63) & ~63ull);
    L += launch_grid_fill(dims, n, m, plan, offs[0], offs[1], cz[2], cz[3], ent_s, ent_u,
                          c->dstat, s);
    L += launch_grid_match(dims, d, plan, offs[0], offs[1], ent_s, ent_u, cnt, nullptr, nullptr,
                           nullptr, c->dstat, s);
    L += launch_offsets(cnt, n, off, pairs ? cap : ~0ull, &c->dstat->K, ost, c->dstat, s);
    if (pairs && n > 0 && m > 0) {
        L += launch_grid_match(dims, d, plan, offs[0], offs[1], ent_s, ent_u, cnt, off, cursor,
                               pairs, c->dstat, s);
        EmitArgs a{};  // per-segment sort by update id (every segment)
        a.d = d; a.n = n; a.m = m;
        a.cnt = cnt; a.off = off; a.pairs = pairs; a.cap = cap;
        a.id_bits = id_bits(m);
        L += launch_segment_sort(a, c->dstat, s);
    }
    CK(cudaGetLastError());
    return finish(c, K_out);
}

int ddm_debug_wait_timeout(ddm_ctx* c, int which, uint32_t spin_limit) {
    if (!c) return DDM_ERR_INVALID;
    if (which < 0 || which > 1) return fail(c, DDM_ERR_INVALID, "which must be 0 or 1");
    if (spin_limit < 1 || spin_limit > (1u << 16))
        return fail(c, DDM_ERR_INVALID, "spin_limit must be 1 .. 65536");
    DeviceGuard g(c->device);
    // The status block is cleared first; its aux[0] word (zero) is the
    // look-back word that never gets published.
    CK(cudaMemsetAsync(c->dstat, 0, sizeof(DevStatus), c->stream));
    PdlScope pdl_scope(c->pdl);
    c->stats.launches += launch_wait_selftest(which, spin_limit, &c->dstat->aux[0], c->dstat,
                                              c->stream);
    CK(cudaGetLastError());
    return finish(c, nullptr);
}

int ddm_debug_write_pattern(ddm_ctx* c, uint32_t nseg, uint32_t mean_len, int scattered,
                            int reps, double* ms_out, uint64_t* bytes_out) {
    if (!c) return DDM_ERR_INVALID;
    if (!ms_out || nseg < 1 || nseg > (1u << 26) || mean_len < 1 || mean_len > 4096 ||
        reps < 1 || reps > 100)
        return fail(c, DDM_ERR_INVALID,
                    "write pattern: nseg 1..2^26, mean_len 1..4096, reps 1..100");
    DeviceGuard g(c->device);
    cudaStream_t s = c->stream;
    const uint64_t ntile = ceil_div((uint64_t)nseg, (uint64_t)OFF_TILE);
    uint32_t* len = nullptr;
    unsigned long long *off = nullptr, *st = nullptr;
    int2* out = nullptr;
    void* flush = nullptr;
    const size_t flush_bytes = 256u << 20;  // larger than L2: written between timed runs
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = DDM_OK;
    auto release = [&]() {
        cudaFree(len); cudaFree(off); cudaFree(st); cudaFree(out); cudaFree(flush);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMalloc(&len, nseg * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&off, (nseg + 1ull) * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&st, (ntile + 3) * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
        cudaGetLastError();
        release();
        return fail(c, DDM_ERR_NOMEM, "write pattern buffers");
    }
    // Lengths, then offsets by the library's scan (status words and total zeroed).
    unsigned long long K = 0;
    if (cudaMemsetAsync(c->dstat, 0, sizeof(DevStatus), s) != cudaSuccess ||
        cudaMemsetAsync(st, 0, (ntile + 3) * sizeof(unsigned long long), s) != cudaSuccess) {
        cudaGetLastError();
        release();
        return fail(c, DDM_ERR_CUDA, "write pattern set-up");
    }
    c->stats.launches += launch_wp_lengths(len, nseg, mean_len, 0x9e3779b9u, s);
    c->stats.launches += launch_offsets(len, nseg, off, ~0ull, st + ntile + 2, st, c->dstat, s);
    if (cudaMemcpyAsync(&K, st + ntile + 2, sizeof(K), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        release();
        return fail(c, DDM_ERR_CUDA, "write pattern offsets");
    }
    if (cudaMalloc(&out, K * sizeof(int2)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        release();
        return fail(c, DDM_ERR_NOMEM, "write pattern output");
    }
    // Scattered order: a step near 0.618 nseg, coprime to nseg.
    uint32_t step = 0;
    if (scattered && nseg > 2) {
        step = (uint32_t)(0.6180339887 * nseg) | 1u;
        auto gcd = [](uint32_t a, uint32_t b) {
            while (b) {
                const uint32_t t = a % b;
                a = b;
                b = t;
            }
            return a;
        };
        while (gcd(step, nseg) != 1) step += 2;
    }
    double best = 1e30;
    for (int r = 0; r < reps + 1 && rc == DDM_OK; ++r) {
        if (cudaMemsetAsync(flush, r & 0xff, flush_bytes, s) != cudaSuccess ||
            cudaEventRecord(e0, s) != cudaSuccess) { rc = DDM_ERR_CUDA; break; }
        c->stats.launches += launch_wp_write(out, off, nseg, step, s);
        float ms = 0.f;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { rc = DDM_ERR_CUDA; break; }
        if (r > 0 && ms < best) best = ms;  // the first run warms up
    }
    if (rc != DDM_OK) {
        cudaGetLastError();
        release();
        return fail(c, rc, "write pattern timing");
    }
    release();
    rc = finish(c, nullptr);
    if (rc) return rc;
    *ms_out = best;
    if (bytes_out) *bytes_out = K * sizeof(int2);
    return DDM_OK;
}

int ddm_debug_sweep(ddm_ctx* c, const ddm_regions* r, uint32_t* sorted_who,
                    uint32_t* subset_size, uint32_t* updset_size, uint32_t* sub_count,
                    uint32_t* upd_count) {
    if (!c) return DDM_ERR_INVALID;
    int rc = check_regions(c, r);
    if (rc) return rc;
    DeviceGuard g(c->device);
    ddm_regions r1 = *r;
    r1.d = 1;
    DebugOut dbg{sorted_who, subset_size, updset_size, sub_count, upd_count};
    rc = enqueue_plain(c, &r1, Mode::Debug, nullptr, 0, &dbg);
    if (rc) return rc;
    return finish(c, nullptr);
}

}  // extern "C"
