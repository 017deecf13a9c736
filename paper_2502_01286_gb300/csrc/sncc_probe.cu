// sncc_probe.cu - shared-memory read-bandwidth probe.  The segment-sum kernel
// reads one 32-bit shared-memory word per (offset, corner) with lane-
// consecutive addresses; this kernel performs the same access pattern with
// nothing else in the loop, so its rate is the on-chip ceiling the segment-sum
// kernel is compared against.
#include <cuda_runtime.h>

#include <cstdint>

#include "sncc.h"

namespace sncc {
namespace {

constexpr int kProbeWords = 8192;  // 32 KB

__global__ void __launch_bounds__(256) probe_smem_read(int32_t* __restrict__ sink, int iters) {
    __shared__ int32_t buf[kProbeWords];
    for (int i = threadIdx.x; i < kProbeWords; i += blockDim.x) buf[i] = i * 2654435761u;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    int base = warp * 1024 + lane;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 32; k += 4) {
            a0 += buf[(base + (k + 0) * 32) & (kProbeWords - 1)];
            a1 += buf[(base + (k + 1) * 32) & (kProbeWords - 1)];
            a2 += buf[(base + (k + 2) * 32) & (kProbeWords - 1)];
            a3 += buf[(base + (k + 3) * 32) & (kProbeWords - 1)];
        }
        base += 97 * 32;
    }
    sink[blockIdx.x * blockDim.x + threadIdx.x] = a0 ^ a1 ^ a2 ^ a3;
}

}  // namespace
}  // namespace sncc

extern "C" int sncc_probe_smem_read(int32_t* d_sink, int ctas, int iters, sncc_stream_t stream) {
    if (!d_sink || ctas <= 0 || iters <= 0) return SNCC_ERR_ARG;
    sncc::probe_smem_read<<<ctas, 256, 0, (cudaStream_t)stream>>>(d_sink, iters);
    return cudaGetLastError() == cudaSuccess ? SNCC_OK : SNCC_ERR_CUDA;
}
