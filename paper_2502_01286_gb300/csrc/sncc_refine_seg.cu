// sncc_refine_seg.cu - the paper's own fine stage (Section 5, main algorithm
// steps 7g-7j): at every coarse candidate, segmented NCC (Eq. 12 - Eq. 18)
// with a second, finer approximation, thresholded into the match list.
//
// One warp per candidate.  The lanes stride over the fine plan's corner
// records (the same fixed-point corner form the coarse kernel uses) and read
// the global sum table directly: A = sum_p G_p s(u + bx + X_p, v + by + Y_p).
// Products and the sum are taken modulo 2^64, which is exact because the
// identity holds in integers and |A| < 2^63.  A warp-shuffle reduction gives
// A to lane 0, which normalises exactly as the coarse pass does.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "sncc.h"
#include "sncc_internal.h"

namespace sncc {
namespace {

constexpr int kWarpsPerCta = 8;

template <bool S64>
__device__ __forceinline__ long long table_at(const void* s, int pitch, int X, int Y) {
    if constexpr (S64)
        return static_cast<const long long*>(s)[(size_t)Y * pitch + X];
    else
        return static_cast<const int*>(s)[(size_t)Y * pitch + X];
}

struct RefineSegArgs {
    const int4* blocks;
    const int2* corners;
    int nblk, WP;
    const void* s;
    const int64_t* s2;
    int pitch, U, V, W, H;
    long long n;
    double rn;  // 1 / n in FP64
    float inv_n, Ek, scale;
    long long Q0;
    const int32_t* cand;
    const int32_t* count;
    int cand_cap;
    float tau;
    sncc_match_t* scratch;
    int scratch_cap;
    int32_t* nout;
    int32_t* status;
};

template <bool S64>
__global__ void __launch_bounds__(kWarpsPerCta * 32) refine_seg_kernel(const RefineSegArgs a) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
    const int nw = gridDim.x * kWarpsPerCta;
    const int count = min(*a.count, a.cand_cap);
    for (int i = gw; i < count; i += nw) {
        const int idx = a.cand[i];
        if (idx < 0 || idx >= a.U * a.V) continue;  // not an offset (warp-uniform)
        const int u = idx % a.U, v = idx / a.U;
        unsigned long long acc = 0ull;
        for (int b = 0; b < a.nblk; ++b) {
            const int4 blk = a.blocks[b];
            const int xb = u + blk.x, yb = v + blk.y;
            for (int p = lane; p < blk.w; p += 32) {
                const int2 c = __ldg(a.corners + blk.z + p);
                const int Y = c.x / a.WP, X = c.x - Y * a.WP;
                const long long sv = table_at<S64>(a.s, a.pitch, xb + X, yb + Y);
                acc += (unsigned long long)(long long)c.y * (unsigned long long)sv;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const long long sf = table_at<S64>(a.s, a.pitch, u + a.W, v + a.H) - table_at<S64>(a.s, a.pitch, u, v + a.H) -
                                 table_at<S64>(a.s, a.pitch, u + a.W, v) + table_at<S64>(a.s, a.pitch, u, v);
            const long long sf2 = a.s2[(size_t)(v + a.H) * a.pitch + u + a.W] - a.s2[(size_t)(v + a.H) * a.pitch + u] -
                                  a.s2[(size_t)v * a.pitch + u + a.W] + a.s2[(size_t)v * a.pitch + u];
            const long long var = a.n * sf2 - sf * sf;
            float rho = 0.0f;
            if (var > 0) {
                const double ef = (double)var * a.rn;
                const float den = sqrtf((float)ef * a.Ek);
                const float num = ((float)(long long)acc - (float)(a.Q0 * sf) * a.inv_n) * a.scale;
                rho = num / den;
            }
            if (rho >= a.tau) {
                const int pos = atomicAdd(a.nout, 1);
                if (pos < a.scratch_cap) {
                    sncc_match_t m;
                    m.u = u;
                    m.v = v;
                    m.rho = rho;
                    a.scratch[pos] = m;
                } else {
                    atomicOr(a.status, SNCC_STATUS_MATCH_OVERFLOW);
                }
            }
        }
    }
}

}  // namespace
}  // namespace sncc

extern "C" int sncc_refine_segmented(const sncc_segments* seg, const void* d_plan, const void* d_s, int s_bits,
                                     const int64_t* d_s2, int sat_pitch, int M, int N, const int32_t* d_cand,
                                     const int32_t* d_count, int cand_cap, float tau, sncc_match_t* d_out,
                                     int out_cap, int32_t* d_nout, void* d_ws, size_t ws_bytes, int32_t* d_status,
                                     sncc_stream_t stream) {
    sncc::NvtxRange nvtx_range("sncc_refine_segmented");
    using namespace sncc;
    const Plan* p = plan_of(seg);
    if (!seg || !p || !d_plan || !d_s || !d_s2 || !d_count || !d_nout || !d_status) return SNCC_ERR_ARG;
    if (cand_cap < 0 || out_cap < 0 || (cand_cap > 0 && !d_cand) || (out_cap > 0 && !d_out)) return SNCC_ERR_ARG;
    if (s_bits != 32 && s_bits != 64) return SNCC_ERR_ARG;
    if (!(seg->Ek > 0.0) || p->image.empty()) return SNCC_ERR_UNIFORM;
    const int W = seg->W, H = seg->H;
    const int U = M - W + 1, V = N - H + 1;
    if (U <= 0 || V <= 0 || sat_pitch < M + 1) return SNCC_ERR_ARG;
    if (misaligned(d_s, s_bits / 8) || misaligned(d_s2, 8) || misaligned(d_cand, 4) || misaligned(d_count, 4) ||
        misaligned(d_out, 4) || misaligned(d_nout, 4) || misaligned(d_status, 4))
        return SNCC_ERR_ARG;
    // the per-candidate walk reads table entries themselves: a 32-bit table
    // must hold them exactly
    if (s_bits == 32 && (int64_t)255 * M * N >= ((int64_t)1 << 31)) return SNCC_ERR_DTYPE;
    if ((int64_t)U * V >= ((int64_t)1 << 31)) return SNCC_ERR_UNSUPPORTED;
    if (reinterpret_cast<uintptr_t>(d_plan) & 15) return SNCC_ERR_ARG;
    if (out_cap > 0 && (!d_ws || ws_bytes < sncc_refine_workspace_bytes(M, N, W, H, out_cap) ||
                        (reinterpret_cast<uintptr_t>(d_ws) & 15)))
        return SNCC_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(d_nout, 0, sizeof(int32_t), st) != cudaSuccess) return SNCC_ERR_CUDA;
    if (cand_cap == 0) return SNCC_OK;

    RefineSegArgs a;
    const Layout& L = p->lay[0];
    a.blocks = reinterpret_cast<const int4*>(static_cast<const char*>(d_plan) + L.blocks_offset);
    a.corners = reinterpret_cast<const int2*>(static_cast<const char*>(d_plan) + L.corners_offset);
    a.nblk = L.nblk;
    a.WP = L.WP;
    a.s = d_s;
    a.s2 = d_s2;
    a.pitch = sat_pitch;
    a.U = U;
    a.V = V;
    a.W = W;
    a.H = H;
    a.n = (long long)W * H;
    a.rn = 1.0 / ((double)W * H);
    a.inv_n = (float)a.rn;
    a.Ek = (float)seg->Ek;
    a.scale = (float)std::ldexp(1.0, -p->F);
    a.Q0 = p->Q0;
    a.cand = d_cand;
    a.count = d_count;
    a.cand_cap = cand_cap;
    a.tau = tau;
    a.scratch = static_cast<sncc_match_t*>(d_ws);
    a.scratch_cap = out_cap;
    a.nout = d_nout;
    a.status = d_status;
    const int want = (cand_cap + kWarpsPerCta - 1) / kWarpsPerCta;
    const int cap_ctas = 16 * (sm_count() > 0 ? sm_count() : 1);
    const int grid = want < cap_ctas ? want : cap_ctas;
    if (s_bits == 64)
        refine_seg_kernel<true><<<grid, kWarpsPerCta * 32, 0, st>>>(a);
    else
        refine_seg_kernel<false><<<grid, kWarpsPerCta * 32, 0, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return SNCC_ERR_CUDA;
    if (out_cap > 0) {
        size_t sort_off = 0;
        refine_workspace_bytes(M, N, W, H, out_cap, &sort_off);
        if (launch_match_sort(a.scratch, d_nout, out_cap, U, V, static_cast<char*>(d_ws) + sort_off, d_out, st) !=
            cudaSuccess)
            return SNCC_ERR_CUDA;
    }
    return SNCC_OK;
}
