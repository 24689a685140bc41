// a9 served mode: drift kernel interface.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace ddm {

struct DriftArgs {
    int d;
    int64_t n, m;
    float* sub_lo[DDM_MAX_DIMS];
    float* sub_hi[DDM_MAX_DIMS];
    float* upd_lo[DDM_MAX_DIMS];
    float* upd_hi[DDM_MAX_DIMS];
    unsigned long long seed, step;
    double sigma;
};

int launch_drift(const DriftArgs& a, cudaStream_t s);

}  // namespace ddm
