// Start and end of every call as kernels: the zero fill that a call begins
// with (device status and the zeroed part of the workspace) and the copy of
// the device status to the host mirror that the host reads after its one
// synchronisation (with, on the window path, the number of subscriptions sent
// to the range path, so that the host launches that path only when needed).
// As kernels, both stay inside the chain of programmatic dependent launches
// that the call's other kernels form, where a memset or a copy-engine transfer
// would end it.
#include "common.cuh"

namespace ddm {

__global__ void __launch_bounds__(256) k_prologue(DevStatus* st, uint4* zero, uint64_t words) {
    pdl_begin();
    const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (i0 == 0) {
        st->error = 0;
        st->detail = 0;
        st->K = 0;
        for (int k = 0; k < 6; ++k) st->aux[k] = 0;
        st->flagged = 0;
    }
    for (uint64_t i = i0; i < words; i += stride) zero[i] = make_uint4(0u, 0u, 0u, 0u);
}

__global__ void k_publish(const DevStatus* st, DevStatus* host, const uint32_t* flagged) {
    pdl_begin();
    if (threadIdx.x == 0) {
        const volatile DevStatus* s = st;
        host->error = s->error;
        host->detail = s->detail;
        host->K = s->K;
        for (int k = 0; k < 6; ++k) host->aux[k] = s->aux[k];
        host->flagged = flagged ? *(const volatile uint32_t*)flagged : 0ull;
    }
}

int launch_prologue(DevStatus* st, void* zero, uint64_t zero_bytes, cudaStream_t s) {
    const uint64_t words = zero_bytes / 16;
    uint64_t g = ceil_div(words, (uint64_t)256 * 4);
    g = g < 1 ? 1 : (g > 152 * 4 ? 152 * 4 : g);
    launch_k(k_prologue, (unsigned)g, 256, 0, s, st, static_cast<uint4*>(zero), words);
    return 1;
}

int launch_publish(const DevStatus* st, DevStatus* host_mapped, const uint32_t* flagged,
                   cudaStream_t s) {
    launch_k(k_publish, 1, 32, 0, s, st, host_mapped, flagged);
    return 1;
}

}  // namespace ddm
