// Endpoint key build (a1) and onesweep LSD radix sort (a2): interfaces.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace ddm {

constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int SORT_BLOCK = 256;        // threads per onesweep tile (one per digit)
constexpr int SORT_ITEMS_32 = 16;      // keys per thread, 32-bit keys
constexpr int SORT_ITEMS_64 = 12;      // keys per thread, 64-bit keys
constexpr uint32_t LB32_AGG = 1u << 30, LB32_INC = 2u << 30, LB32_VAL = (1u << 30) - 1;

template <typename KeyT>
constexpr int sort_items() { return sizeof(KeyT) == 4 ? SORT_ITEMS_32 : SORT_ITEMS_64; }

template <typename KeyT>
constexpr int sort_tile() { return SORT_BLOCK * sort_items<KeyT>(); }

// Scratch the sort needs besides the two ping-pong key/value buffers:
// hist[passes][256] global digit counts, tile counters and the look-back words.
template <typename KeyT>
inline size_t sort_lookback_words(uint64_t E, int passes) {
    return (size_t)passes * (ceil_div(E, sort_tile<KeyT>()) * RADIX + 32);
}

// Dimension-0 key build for one instance: validates every extent of dim 0
// (no NaN, lo <= hi), writes keys/payloads in [S lo | U lo | S hi | U hi]
// layout and accumulates the digit histograms of all `passes` digit places
// into hist (which must be zeroed).
int launch_keybuild_d0(const float* sub_lo, const float* sub_hi, const float* upd_lo,
                        const float* upd_hi, int64_t n, int64_t m, uint32_t* keys,
                        uint32_t* vals, uint32_t* hist, DevStatus* st, cudaStream_t s);

// Stable LSD radix sort of E (key, val) pairs by the low `passes` * 8 key bits.
// hist must hold the digit histograms of all passes (from the key build);
// lookback must hold sort_lookback_words() zeroed words.  The result ends in
// (keys[r], vals[r]) with r = passes % 2 (buffer 0 = the input).  When
// `skip_last_keys` is set the last pass writes only values.
template <typename KeyT>
int launch_radix_sort(KeyT* keys0, uint32_t* vals0, KeyT* keys1, uint32_t* vals1, uint64_t E,
                       int passes, const uint32_t* hist, uint32_t* lookback,
                       bool skip_last_keys, DevStatus* st, cudaStream_t s);

}  // namespace ddm
