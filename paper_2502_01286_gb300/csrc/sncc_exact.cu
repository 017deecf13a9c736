// sncc_exact.cu - exact NCC (Eq. 1) at every offset by direct correlation,
// the paper's "naive algorithm" (Section 2, Table 1), kept as the same-GPU
// reference for speed and for the approximation error of segmented NCC.
//
// A CTA of 8 warps computes a 32 x 8R tile of offsets.  The template is cut
// into 64 x 64 blocks; for each block the CTA stages the template block and
// the source region its offsets touch in shared memory.  The region is kept
// as four byte-shifted copies (copy k, word j = bytes 4j+k .. 4j+k+3 of a
// row), so that the four source bytes a lane multiplies with four template
// bytes are always one aligned 32-bit word: lane l reads copy (l & 3), word
// (l >> 2) + x/4, and __dp4a multiplies and adds the four byte pairs.  The
// copies are spaced 8 words (mod 32) apart, so the 32 lanes hit 32 banks.
// A block adds at most 4096 * 65025 < 2^32 per offset, so the per-block
// sums are exact in uint32 and are flushed into 64-bit totals.  The window
// sums come from the sum tables; from the exact integers, the numerator and
// n^2 E_f are scaled by 1/n in FP64 and the ratio is finished in FP32 (a
// square root and a division per offset in FP64 would occupy GB300's slow
// FP64 pipe).
#include <cuda_runtime.h>

#include <cstdint>

#include "sncc.h"
#include "sncc_internal.h"
#include "sncc_tile.cuh"

namespace sncc {
namespace {

constexpr int kTB = 64;            // template block edge
constexpr int kRB = TILE_U + kTB + 4;  // source region row, bytes (100)
constexpr int kRW = kRB / 4;           // source region row, words (25)
constexpr int kTR = kTB + 8;           // staged template rows (8 >= R zero rows)

// words of one byte-shifted copy of a region of FR rows, padded so that the
// four copies start 8 banks apart
__host__ __device__ constexpr int copy_words(int FR) { return ((FR * kRW + 24) / 32) * 32 + 8; }

template <int R>
constexpr size_t exact_smem_bytes() {
    return (size_t)4 * copy_words(WARPS * R + kTB) * 4 + (size_t)kTR * kTB;
}

template <int R, bool S64>
__global__ void __launch_bounds__(256)
    exact_kernel(const uint8_t* __restrict__ f, int M, int N, int f_stride, const uint8_t* __restrict__ t, int W,
                 int H, int t_stride, long long T, long long T2, const void* __restrict__ s,
                 const int64_t* __restrict__ s2, int pitch, double rn, float etn, float* __restrict__ rho,
                 int rho_pitch) {
    constexpr int FR = WARPS * R + kTB;  // region rows (one spare)
    constexpr int CW = copy_words(FR);
    extern __shared__ __align__(16) uint32_t smx[];
    uint32_t* cp = smx;                                            // 4 copies x CW words
    uint8_t* ts = reinterpret_cast<uint8_t*>(smx + 4 * CW);        // kTR x kTB template bytes
    uint8_t* fb = reinterpret_cast<uint8_t*>(cp);                  // copy 0 viewed as bytes
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int u0 = blockIdx.x * TILE_U, v0 = blockIdx.y * (WARPS * R);
    const int U = M - W + 1, V = N - H + 1;
    unsigned long long acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0ull;
    // lane l's words: copy (l & 3), word (l >> 2) + x/4 of its rows
    const uint32_t* lbase = cp + (lane & 3) * CW + (warp * R) * kRW + (lane >> 2);

    for (int by = 0; by < H; by += kTB) {
        const int bh = min(kTB, H - by);
        for (int bx = 0; bx < W; bx += kTB) {
            const int bw = min(kTB, W - bx);
            const int bq = (bw + 3) >> 2;
            __syncthreads();
            // template block, zero-padded to a multiple of 4 columns and with
            // zero rows below it, read by the register window's last rows
            for (int i = tid; i < kTR * kTB; i += 256) {
                const int y = i / kTB, x = i - y * kTB;
                ts[i] = (y < bh && x < bw) ? t[(size_t)(by + y) * t_stride + bx + x] : (uint8_t)0;
            }
            // copy 0: the source region as bytes (rows of kRB), zero outside the image
            for (int i = tid; i < FR * kRB; i += 256) {
                const int Y = i / kRB, X = i - Y * kRB;
                const int gy = v0 + by + Y, gx = u0 + bx + X;
                fb[i] = (gy < N && gx < M) ? f[(size_t)gy * f_stride + gx] : (uint8_t)0;
            }
            __syncthreads();
            // copies 1..3: word j of copy k = bytes 4j+k .. 4j+k+3 of the row
            for (int i = tid; i < FR * kRW; i += 256) {
                const int Y = i / kRW, j = i - Y * kRW;
                const uint32_t w0 = cp[Y * kRW + j];
                const uint32_t w1 = (j + 1 < kRW) ? cp[Y * kRW + j + 1] : 0u;
                cp[1 * CW + i] = __byte_perm(w0, w1, 0x4321);
                cp[2 * CW + i] = __byte_perm(w0, w1, 0x5432);
                cp[3 * CW + i] = __byte_perm(w0, w1, 0x6543);
            }
            __syncthreads();
            // Column q of words outer, source rows j inner: the word a lane
            // reads at source row j serves all R offset rows of the warp (with
            // template row j - r for offset row r), and the last R template
            // words of column q stay in registers, so each j costs two shared
            // loads (source word, broadcast template word) and R dp4a.
            unsigned part[R];
#pragma unroll
            for (int r = 0; r < R; ++r) part[r] = 0u;
            const uint32_t* tw = reinterpret_cast<const uint32_t*>(ts);
            for (int q = 0; q < bq; ++q) {
                uint32_t win[R];  // win[j % R] = template word (row j, column q)
#pragma unroll
                for (int r = 0; r < R; ++r) win[r] = 0u;
                const uint32_t* lcol = lbase + q;
                const uint32_t* tcol = tw + q;
                for (int jb = 0; jb < bh + R - 1; jb += R) {
#pragma unroll
                    for (int jj = 0; jj < R; ++jj) {
                        const uint32_t w = lcol[(jb + jj) * kRW];
                        win[jj] = tcol[(jb + jj) * (kTB / 4)];
#pragma unroll
                        for (int r = 0; r < R; ++r) part[r] = __dp4a(w, win[(jj - r + R) % R], part[r]);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] += part[r];
        }
    }

    const int u = u0 + lane;
    const long long n = (long long)W * H;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = v0 + warp * R + r;
        if (u >= U || v >= V) continue;
        const long long sf = window_sum<S64>(s, pitch, u, v, W, H);
        const long long sf2 = s2[(size_t)(v + H) * pitch + u + W] - s2[(size_t)(v + H) * pitch + u] -
                              s2[(size_t)v * pitch + u + W] + s2[(size_t)v * pitch + u];
        const long long vf = n * sf2 - sf * sf;
        const long long num = n * (long long)acc[r] - T * sf;
        // rho = (num / n) / sqrt((vf / n) (vt / n)); etn = vt / n > 0
        const float out = vf > 0 ? (float)((double)num * rn) / sqrtf((float)((double)vf * rn) * etn) : 0.0f;
        rho[(size_t)v * rho_pitch + u] = out;
    }
}

template <int R>
cudaError_t launch_exact(bool s64, dim3 grid, cudaStream_t st, const uint8_t* f, int M, int N, int f_stride,
                         const uint8_t* t, int W, int H, int t_stride, long long T, long long T2, const void* s,
                         const int64_t* s2, int pitch, double rn, float etn, float* rho, int rho_pitch) {
    constexpr size_t sm = exact_smem_bytes<R>();
    cudaError_t attr = cudaFuncSetAttribute(exact_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (attr == cudaSuccess)
        attr = cudaFuncSetAttribute(exact_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (attr != cudaSuccess) return attr;
    if (s64)
        exact_kernel<R, true><<<grid, 256, sm, st>>>(f, M, N, f_stride, t, W, H, t_stride, T, T2, s, s2, pitch, rn,
                                                      etn, rho, rho_pitch);
    else
        exact_kernel<R, false><<<grid, 256, sm, st>>>(f, M, N, f_stride, t, W, H, t_stride, T, T2, s, s2, pitch,
                                                       rn, etn, rho, rho_pitch);
    return cudaGetLastError();
}

}  // namespace
}  // namespace sncc

extern "C" int sncc_exact_map(const uint8_t* d_f, int M, int N, int f_stride, const uint8_t* d_t, int W, int H,
                              int t_stride, int64_t T, int64_t T2, const void* d_s, int s_bits, const int64_t* d_s2,
                              int sat_pitch, float* d_rho, int rho_pitch, sncc_stream_t stream) {
    sncc::NvtxRange nvtx_range("sncc_exact_map");
    using namespace sncc;
    if (!d_f || !d_t || !d_s || !d_s2 || !d_rho || W <= 0 || H <= 0 || M < W || N < H) return SNCC_ERR_ARG;
    if (f_stride < M || t_stride < W || (s_bits != 32 && s_bits != 64) || sat_pitch < M + 1) return SNCC_ERR_ARG;
    if (misaligned(d_s, s_bits / 8) || misaligned(d_s2, 8) || misaligned(d_rho, 4)) return SNCC_ERR_ARG;
    const int U = M - W + 1, V = N - H + 1;
    if (rho_pitch < U) return SNCC_ERR_ARG;
    if ((int64_t)W * H > ((int64_t)1 << 23)) return SNCC_ERR_UNSUPPORTED;
    const long long n = (long long)W * H;
    if (n * T2 - T * T <= 0) return SNCC_ERR_UNIFORM;
    const double rn = 1.0 / (double)n;
    const float etn = (float)((double)(n * T2 - T * T) * rn);  // E_t
    const int tu = (U + TILE_U - 1) / TILE_U;
    const int sms = sm_count() > 0 ? sm_count() : 1;
    int R = 2;
    for (int c : {8, 4}) {
        if ((long long)tu * ((V + WARPS * c - 1) / (WARPS * c)) >= 2 * sms) { R = c; break; }
    }
    dim3 grid(tu, (V + WARPS * R - 1) / (WARPS * R));
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    const bool s64 = (s_bits == 64);
    if (R == 8)
        e = launch_exact<8>(s64, grid, st, d_f, M, N, f_stride, d_t, W, H, t_stride, T, T2, d_s, d_s2, sat_pitch,
                            rn, etn, d_rho, rho_pitch);
    else if (R == 4)
        e = launch_exact<4>(s64, grid, st, d_f, M, N, f_stride, d_t, W, H, t_stride, T, T2, d_s, d_s2, sat_pitch,
                            rn, etn, d_rho, rho_pitch);
    else
        e = launch_exact<2>(s64, grid, st, d_f, M, N, f_stride, d_t, W, H, t_stride, T, T2, d_s, d_s2, sat_pitch,
                            rn, etn, d_rho, rho_pitch);
    return e == cudaSuccess ? SNCC_OK : SNCC_ERR_CUDA;
}
