// sncc_probe.cu - on-chip ceilings the kernels are compared against.
//
// Shared-memory read bandwidth: the segment-sum kernel reads one 32-bit
// shared-memory word per (offset, corner) with lane-consecutive addresses;
// probe_smem_read performs the same access pattern with nothing else in the
// loop.  Instruction rates: the segment-sum kernel adds one 32 x 32 -> 64-bit
// integer multiply-add per (offset, corner), and the exact comparator one
// four-way byte dot product (dp4a) per four template pixels; probe_alu issues
// only that instruction, in eight independent chains per thread.  HBM write
// bandwidth: the sum tables are almost all 16-byte stores (12 or 16 bytes
// written per pixel against 1 read); probe_hbm_write writes a buffer larger
// than L2 with 16-byte stores and nothing else.
#include <cuda_runtime.h>

#include <cstdint>

#include "sncc.h"
#include "sncc_internal.h"
#include "sncc_ptx.cuh"

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

constexpr int kChains = 8;

// kind 0: dp4a, 64 per thread and iteration
__global__ void __launch_bounds__(256) probe_dp4a(int32_t* __restrict__ sink, int iters, unsigned b) {
    unsigned a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = threadIdx.x * 7u + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = __dp4a(a[i], b + q, a[i]);
    }
    unsigned x = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) x ^= a[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = (int32_t)x;
}

__device__ __forceinline__ long long mad_wide(int a, int b, long long c) {
    long long d;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// kind 1: signed 32 x 32 -> 64-bit multiply-add into a 64-bit accumulator,
// 64 per thread and iteration; the multiplicands are the accumulators' low
// and high words at the start of the iteration, so nothing can be hoisted
__global__ void __launch_bounds__(256) probe_imad_wide(int32_t* __restrict__ sink, int iters) {
    long long acc[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i)
        acc[i] = (long long)((threadIdx.x * 7 + i + 1) * 0x10001u) << 16 | (threadIdx.x * 13 + i);
    for (int it = 0; it < iters; ++it) {
        int x[kChains], y[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            x[i] = (int)acc[i];
            y[i] = (int)(acc[i] >> 32);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int i = 0; i < kChains; ++i)
                acc[i] = mad_wide(x[(i + q) & (kChains - 1)], y[(i + 2 * q + 1) & (kChains - 1)], acc[i]);
    }
    long long x = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) x ^= acc[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = (int32_t)(x ^ (x >> 32));
}

// The bounded wait of the segment-sum kernel on an mbarrier that nothing
// completes: thread 0 gives up after the library's wait limit and records
// SNCC_STATUS_WAIT_TIMEOUT, the CTA returns, and the context stays usable.
__global__ void __launch_bounds__(32) probe_wait_timeout(int32_t* __restrict__ status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // one arrival expected; none comes
        fence_mbar_init();
    }
    __syncwarp();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0u)) atomicOr(status, SNCC_STATUS_WAIT_TIMEOUT);
}

// Grid-stride 16-byte stores of a pattern that depends on the address.
__global__ void __launch_bounds__(256) probe_hbm_write(int4* __restrict__ buf, size_t n16) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
        const uint32_t lo = (uint32_t)i, hi = (uint32_t)(i >> 32);
        buf[i] = make_int4((int)lo, (int)(hi ^ 0x5a5a5a5au), (int)(lo * 3u), (int)(lo ^ 0xffffu));
    }
}

}  // namespace
}  // namespace sncc

extern "C" int sncc_probe_hbm_write(void* d_buf, size_t bytes, sncc_stream_t stream) {
    if (!d_buf || bytes < 16 || (bytes & 15) || (reinterpret_cast<uintptr_t>(d_buf) & 15)) return SNCC_ERR_ARG;
    const int sms = sncc::sm_count() > 0 ? sncc::sm_count() : 1;
    sncc::probe_hbm_write<<<sms * 8, 256, 0, (cudaStream_t)stream>>>(static_cast<int4*>(d_buf), bytes / 16);
    return cudaGetLastError() == cudaSuccess ? SNCC_OK : SNCC_ERR_CUDA;
}

extern "C" int sncc_probe_smem_read(int32_t* d_sink, int ctas, int iters, sncc_stream_t stream) {
    if (!d_sink || ctas <= 0 || iters <= 0 || sncc::misaligned(d_sink, 4)) return SNCC_ERR_ARG;
    sncc::probe_smem_read<<<ctas, 256, 0, (cudaStream_t)stream>>>(d_sink, iters);
    return cudaGetLastError() == cudaSuccess ? SNCC_OK : SNCC_ERR_CUDA;
}

extern "C" int sncc_probe_alu(int kind, int32_t* d_sink, int ctas, int iters, sncc_stream_t stream) {
    if (!d_sink || ctas <= 0 || iters <= 0 || (kind != SNCC_PROBE_DP4A && kind != SNCC_PROBE_IMAD_WIDE) ||
        sncc::misaligned(d_sink, 4))
        return SNCC_ERR_ARG;
    if (kind == SNCC_PROBE_DP4A)
        sncc::probe_dp4a<<<ctas, 256, 0, (cudaStream_t)stream>>>(d_sink, iters, 0x01020304u);
    else
        sncc::probe_imad_wide<<<ctas, 256, 0, (cudaStream_t)stream>>>(d_sink, iters);
    return cudaGetLastError() == cudaSuccess ? SNCC_OK : SNCC_ERR_CUDA;
}

extern "C" int sncc_probe_wait_timeout(int32_t* d_status, sncc_stream_t stream) {
    if (!d_status || sncc::misaligned(d_status, 4)) return SNCC_ERR_ARG;
    sncc::probe_wait_timeout<<<1, 32, 0, (cudaStream_t)stream>>>(d_status);
    return cudaGetLastError() == cudaSuccess ? SNCC_OK : SNCC_ERR_CUDA;
}
