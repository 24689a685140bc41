// a8 batched mode: interfaces.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace ddm {

// Device copy of one instance's coordinate pointers (all dimensions).
struct InstPtrs {
    const float* sub_lo[DDM_MAX_DIMS];
    const float* sub_hi[DDM_MAX_DIMS];
    const float* upd_lo[DDM_MAX_DIMS];
    const float* upd_hi[DDM_MAX_DIMS];
};

struct BatchArgs {
    int d;
    int num;                  // instances
    int64_t n, m;             // totals
    const InstPtrs* table;    // num entries (device)
    const int64_t* n_base;    // num + 1 prefix sums of n_b (device)
    const int64_t* m_base;    // num + 1 prefix sums of m_b (device)
    float* sub_lo[DDM_MAX_DIMS];  // concatenated coordinates (device)
    float* sub_hi[DDM_MAX_DIMS];
    float* upd_lo[DDM_MAX_DIMS];
    float* upd_hi[DDM_MAX_DIMS];
};

int launch_keybuild_batch(const BatchArgs& b, unsigned long long* keys, uint32_t* vals,
                          DevStatus* st, cudaStream_t s);
int launch_inst_offsets(const BatchArgs& b, const unsigned long long* off,
                        unsigned long long* inst_off, cudaStream_t s);

// K sorted survivor keys (i << jbits) | j with global ids to int32 pairs local
// to the instance (n_base / m_base: the instances' first global ids, num + 1
// entries each, on the device).
int launch_batch_unpack(const unsigned long long* keys, uint64_t K, int jbits,
                        const int64_t* n_base, const int64_t* m_base, int num, int32_t* pairs,
                        cudaStream_t s);

}  // namespace ddm
