// sncc_refine.cu - the fine pass: exact NCC (Eq. 1) at every candidate the
// coarse pass kept (main algorithm, steps 7g-7j, with the second stage
// computed exactly), then the match list sorted by offset.
//
// One CTA per candidate (grid-stride over the device-side count, so no host
// synchronisation is needed): the CTA sums f*t, f and f^2 over the window in
// exact 64-bit integers, then thread 0 forms
//   rho = (n Sft - T Sf) / sqrt((n Sff - Sf^2)(n T2 - T^2))
// in double and appends (u, v, rho) when rho >= tau.  A sorted compaction
// (one bit per offset, a prefix count, a scatter: sncc_sort.cuh) then writes
// the matches in ascending v*U+u order, so the output is deterministic
// although candidates arrive in atomic order.
#include <cuda_runtime.h>

#include <cstdint>

#include "sncc.h"
#include "sncc_internal.h"
#include "sncc_sort.cuh"

namespace sncc {
namespace {

constexpr int kRefineThreads = 256;

__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kRefineThreads)
    refine_kernel(const uint8_t* __restrict__ f, int f_stride, const uint8_t* __restrict__ t, int W, int H,
                  int t_stride, long long T, long long T2, const int32_t* __restrict__ cand,
                  const int32_t* __restrict__ d_count, int cand_cap, float tau, int U, int V,
                  sncc_match_t* __restrict__ scratch, int scratch_cap, int32_t* __restrict__ d_nout,
                  int32_t* __restrict__ status) {
    __shared__ long long red[3][kRefineThreads / 32];
    const int count = min(*d_count, cand_cap);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long n = (long long)W * H;
    for (int i = blockIdx.x; i < count; i += gridDim.x) {
        const int idx = cand[i];
        if (idx < 0 || idx >= U * V) continue;  // not an offset: skip (uniform per CTA)
        const int u = idx % U, v = idx / U;
        long long sft = 0, sf = 0, sff = 0;
        for (int y = warp; y < H; y += kRefineThreads / 32) {
            const uint8_t* frow = f + (size_t)(v + y) * f_stride + u;
            const uint8_t* trow = t + (size_t)y * t_stride;
            for (int x = lane; x < W; x += 32) {
                const int fv = frow[x], tv = trow[x];
                sft += fv * tv;
                sf += fv;
                sff += fv * fv;
            }
        }
        sft = warp_sum(sft);
        sf = warp_sum(sf);
        sff = warp_sum(sff);
        if (lane == 0) {
            red[0][warp] = sft;
            red[1][warp] = sf;
            red[2][warp] = sff;
        }
        __syncthreads();
        if (tid == 0) {
            long long a = 0, b = 0, c = 0;
            for (int w = 0; w < kRefineThreads / 32; ++w) {
                a += red[0][w];
                b += red[1][w];
                c += red[2][w];
            }
            const long long num = n * a - T * b;
            const long long vf = n * c - b * b;
            const long long vt = n * T2 - T * T;
            const float rho = (vf > 0 && vt > 0) ? (float)((double)num / sqrt((double)vf * (double)vt)) : 0.0f;
            if (rho >= tau) {
                const int pos = atomicAdd(d_nout, 1);
                if (pos < scratch_cap) {
                    sncc_match_t m;
                    m.u = u;
                    m.v = v;
                    m.rho = rho;
                    scratch[pos] = m;
                } else {
                    atomicOr(status, SNCC_STATUS_MATCH_OVERFLOW);
                }
            }
        }
        __syncthreads();
    }
}

// The sort key of a match: its linear offset v*U + u.
struct MatchKey {
    int U;
    __device__ __forceinline__ long long operator()(const sncc_match_t& m) const { return (long long)m.v * U + m.u; }
};

}  // namespace

size_t match_sort_bytes(int U, int V) { return sort_layout((long long)U * V).total; }

cudaError_t launch_match_sort(const sncc_match_t* in, const int32_t* d_n, int cap, int U, int V, void* sort_ws,
                              sncc_match_t* out, cudaStream_t st) {
    const int ctas = 8 * (sm_count() > 0 ? sm_count() : 1);
    return launch_sorted_compaction(in, d_n, cap, MatchKey{U}, (long long)U * V, sort_ws, out, ctas, st);
}

size_t refine_workspace_bytes(int M, int N, int W, int H, int out_cap, size_t* sort_offset) {
    const size_t recs = ((size_t)(out_cap > 0 ? out_cap : 1) * sizeof(sncc_match_t) + 255) / 256 * 256;
    if (sort_offset) *sort_offset = recs;
    return recs + match_sort_bytes(M - W + 1, N - H + 1);
}

}  // namespace sncc

extern "C" size_t sncc_refine_workspace_bytes(int M, int N, int W, int H, int out_cap) {
    if (M <= 0 || N <= 0 || W <= 0 || H <= 0 || W > M || H > N || out_cap < 0) return 0;
    return sncc::refine_workspace_bytes(M, N, W, H, out_cap, nullptr);
}

extern "C" int sncc_refine(const uint8_t* d_f, int M, int N, int f_stride, const uint8_t* d_t, int W, int H,
                           int t_stride, int64_t T, int64_t T2, const int32_t* d_cand, const int32_t* d_count,
                           int cand_cap, float tau, sncc_match_t* d_out, int out_cap, int32_t* d_nout, void* d_ws,
                           size_t ws_bytes, int32_t* d_status, sncc_stream_t stream) {
    sncc::NvtxRange nvtx_range("sncc_refine");
    using namespace sncc;
    if (!d_f || !d_t || !d_count || !d_nout || !d_status || W <= 0 || H <= 0) return SNCC_ERR_ARG;
    if (f_stride < M || t_stride < W || M < W || N < H || cand_cap < 0 || out_cap < 0) return SNCC_ERR_ARG;
    if ((cand_cap > 0 && !d_cand) || (out_cap > 0 && !d_out)) return SNCC_ERR_ARG;
    if (misaligned(d_cand, 4) || misaligned(d_count, 4) || misaligned(d_out, 4) || misaligned(d_nout, 4) ||
        misaligned(d_status, 4))
        return SNCC_ERR_ARG;
    if ((int64_t)W * H > ((int64_t)1 << 23)) return SNCC_ERR_UNSUPPORTED;
    if (out_cap > 0 && (!d_ws || ws_bytes < sncc_refine_workspace_bytes(M, N, W, H, out_cap) ||
                        (reinterpret_cast<uintptr_t>(d_ws) & 15)))
        return SNCC_ERR_WORKSPACE;
    const int U = M - W + 1, V = N - H + 1;
    if ((int64_t)U * V >= ((int64_t)1 << 31)) return SNCC_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(d_nout, 0, sizeof(int32_t), st) != cudaSuccess) return SNCC_ERR_CUDA;
    if (cand_cap == 0) return SNCC_OK;
    sncc_match_t* scratch = static_cast<sncc_match_t*>(d_ws);
    const int cap_ctas = 8 * (sm_count() > 0 ? sm_count() : 1);
    const int grid = cand_cap < cap_ctas ? cand_cap : cap_ctas;
    refine_kernel<<<grid, kRefineThreads, 0, st>>>(d_f, f_stride, d_t, W, H, t_stride, (long long)T, (long long)T2,
                                                   d_cand, d_count, cand_cap, tau, U, V, scratch, out_cap, d_nout,
                                                   d_status);
    if (cudaGetLastError() != cudaSuccess) return SNCC_ERR_CUDA;
    if (out_cap > 0) {
        size_t sort_off = 0;
        refine_workspace_bytes(M, N, W, H, out_cap, &sort_off);
        if (launch_match_sort(scratch, d_nout, out_cap, U, V, static_cast<char*>(d_ws) + sort_off, d_out, st) !=
            cudaSuccess)
            return SNCC_ERR_CUDA;
    }
    return SNCC_OK;
}
