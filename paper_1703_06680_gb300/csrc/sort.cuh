// Endpoint key build (a1) and onesweep LSD radix sort (a2): interfaces.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "sweep.cuh"

namespace ddm {

constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int SORT_BLOCK = 256;        // threads per tile
constexpr int SORT_ITEMS_32 = 18;      // keys per thread, 32-bit keys
constexpr int SORT_ITEMS_64 = 12;      // keys per thread, 64-bit keys

template <typename KeyT>
constexpr int sort_items() { return sizeof(KeyT) == 4 ? SORT_ITEMS_32 : SORT_ITEMS_64; }

template <typename KeyT>
inline uint64_t sort_tiles(uint64_t E) {
    return ceil_div(E, (uint64_t)SORT_BLOCK * sort_items<KeyT>());
}

// Scratch of the sort besides the two ping-pong key/value buffers:
// tile_hist[256 * tiles] (u32), offs[256 * tiles + 1] (u64), per-pass scan
// status words (zeroed, sort_status_stride() u64 per pass) and one u64 total.
struct SortScratch {
    uint32_t* tile_hist;
    unsigned long long* offs;
    unsigned long long* status;
    unsigned long long* total;
};

// Status words of one pass's flat scan (sized for the 64-bit-key tiling, the
// larger of the two).
inline size_t sort_status_stride(uint64_t E) {
    return (size_t)ceil_div(sort_tiles<unsigned long long>(E) * RADIX, OFF_TILE) + 2;
}

// Dimension-0 key build for one instance: validates every extent of dim 0
// (no NaN, lo <= hi) and writes keys/payloads in [S lo | U lo | S hi | U hi]
// layout.
int launch_keybuild_d0(const float* sub_lo, const float* sub_hi, const float* upd_lo,
                       const float* upd_hi, int64_t n, int64_t m, uint32_t* keys, uint32_t* vals,
                       DevStatus* st, cudaStream_t s);

// Stable LSD radix sort of E (key, val) pairs by the low `passes` * 8 key bits.
// The result ends in (keys[r], vals[r]) with r = passes % 2 (buffer 0 = the
// input).  When `skip_last_keys` is set the last pass writes only values.
template <typename KeyT>
int launch_radix_sort(KeyT* keys0, uint32_t* vals0, KeyT* keys1, uint32_t* vals1, uint64_t E,
                      int passes, const SortScratch& sc, bool skip_last_keys, DevStatus* st,
                      cudaStream_t s);

}  // namespace ddm
