// Endpoint key build (a1) and LSD radix sort (a2): interfaces.
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

// Tiles of a sort of E keys; items = keys per thread (0: the default of KeyT;
// 32-bit keys may also use 12 or 16, see launch_radix_sort).
template <typename KeyT>
inline uint64_t sort_tiles(uint64_t E, int items = 0) {
    if (sizeof(KeyT) == 8 || items == 0) items = sort_items<KeyT>();
    return ceil_div(E, (uint64_t)SORT_BLOCK * items);
}

// Fused offsets: with at most SORT_FUSED_MAX_TILES tiles, the downsweep
// computes each (digit, tile) output base itself, and the flat scan between
// upsweep and downsweep is not launched.  The upsweep then stores its
// histogram tile-major and adds it into per-group sums (groups of 32 tiles);
// the downsweep's base for digit d is
//   sum over all groups and digits d' < d of the group sums   (digit start)
// + sum over earlier groups of the group sums of d
// + sum over earlier tiles of its own group of their counts of d,
// at most 32 + 31 independent loads per thread (thread = digit).
constexpr int SORT_GROUP_SHIFT = 5;
constexpr uint64_t SORT_FUSED_MAX_TILES = 1024;

// Scratch of the sort besides the two ping-pong key/value buffers:
// tile_hist[256 * tiles] (u32), offs[256 * tiles + 1] (u64), per-pass scan
// status words (zeroed, sort_status_stride() u64 per pass), one u64 total,
// and the per-pass group sums of the fused-offsets mode (zeroed,
// sort_group_words() u32 in all; NULL selects the flat scan).
struct SortScratch {
    uint32_t* tile_hist;
    unsigned long long* offs;
    unsigned long long* status;
    unsigned long long* total;
    uint32_t* grp;
};

inline uint64_t sort_groups(uint64_t tiles) { return ceil_div(tiles, 1ull << SORT_GROUP_SHIFT); }

// Group-sum words for `passes` passes (0 when the tiles exceed the fused limit).
inline size_t sort_group_words(uint64_t tiles, int passes) {
    return tiles <= SORT_FUSED_MAX_TILES ? (size_t)passes * sort_groups(tiles) * RADIX : 0;
}

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
// clear_ptr/clear_words (16-byte words, may be NULL/0): a buffer that the last
// pass's blocks zero while their tiles load (the rank-record tables of the
// sweep scan that follows).
// vals0 and vals1 may both be NULL: the keys alone are sorted.
// items: keys per thread of a 32-bit sort, 12, 16 or 18 (0: the default, 18);
// 64-bit keys always use 12.  The scratch must be sized for the same choice
// (sort_tiles<KeyT>(E, items)).
// kinds (may be NULL; needs values in endpoint-payload form): per SCAN_TILE
// positions of the sorted output, four u32 counters, zeroed by the caller, to
// which the last pass adds how many S lowers, U lowers and S uppers it writes
// into that range (the fourth stays 0).  These are the tile aggregates of the
// sweep scan (launch_sweep_scan), formed where the output positions are known.
template <typename KeyT>
int launch_radix_sort(KeyT* keys0, uint32_t* vals0, KeyT* keys1, uint32_t* vals1, uint64_t E,
                      int passes, const SortScratch& sc, bool skip_last_keys, DevStatus* st,
                      cudaStream_t s, void* clear_ptr = nullptr, uint64_t clear_words = 0,
                      int items = 0, uint32_t* kinds = nullptr);

}  // namespace ddm
