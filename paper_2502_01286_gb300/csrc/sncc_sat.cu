// sncc_sat.cu - exact integer sum tables of f and f^2 (Eq. 10 and Eq. 14).
//
// Layout: padded tables of (N+1) rows x pitch elements, entry [Y*pitch + X]
// = sum of f over x < X, y < Y (row 0 and column 0 are zero).
//
// Three passes, all coalesced along rows:
//   1. band column sums: for every band of R rows and every column x, the sum
//      of f (and f^2) over the band's rows (reads f once);
//   2. band scan: exclusive prefix of those sums over the bands, giving for
//      each band the column sums of everything above it;
//   3. emit: one CTA per band walks its rows, keeps the running column sums in
//      registers, scans each row across the full width and writes s and s^2.
// Algorithmic traffic: 1 B/px read, 4 or 8 B/px (s) + 8 B/px (s^2) written;
// passes 1-2 add one more read of f and a small band x width array.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "sncc.h"
#include "sncc_internal.h"

namespace sncc {
namespace {

constexpr int kTargetBands = 304;  // two bands per SM on 152 SMs

struct SatGeometry {
    int R;      // rows per band
    int nb;     // number of bands
    int E;      // output columns per thread in the emit pass
    int T;      // threads per emit CTA
};

SatGeometry sat_geometry(int M, int N) {
    SatGeometry g;
    g.R = (N + kTargetBands - 1) / kTargetBands;
    if (g.R < 1) g.R = 1;
    g.nb = (N + g.R - 1) / g.R;
    g.E = (M + 1 <= 8192) ? 8 : 16;
    const int threads = (M + 1 + g.E - 1) / g.E;
    g.T = (threads + 31) / 32 * 32;
    if (g.T < 32) g.T = 32;
    return g;
}

// Pass 1: cs1[b][x] = sum_{y in band b} f(x,y); cs2 the same for f^2.
__global__ void sat_band_colsum(const uint8_t* __restrict__ f, int M, int N, int stride, int R,
                                int32_t* __restrict__ cs1, int32_t* __restrict__ cs2) {
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    const int b = blockIdx.y;
    if (x0 >= M) return;
    const int y0 = b * R;
    const int y1 = min(y0 + R, N);
    int a0 = 0, a1 = 0, a2 = 0, a3 = 0, q0 = 0, q1 = 0, q2 = 0, q3 = 0;
    const bool vec = (x0 + 3 < M) && ((stride & 3) == 0) && ((reinterpret_cast<uintptr_t>(f) & 3) == 0);
    for (int y = y0; y < y1; ++y) {
        const uint8_t* row = f + (size_t)y * stride;
        int p0, p1, p2, p3;
        if (vec) {
            const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(row + x0));
            p0 = w & 0xff; p1 = (w >> 8) & 0xff; p2 = (w >> 16) & 0xff; p3 = w >> 24;
        } else {
            p0 = row[x0];
            p1 = (x0 + 1 < M) ? row[x0 + 1] : 0;
            p2 = (x0 + 2 < M) ? row[x0 + 2] : 0;
            p3 = (x0 + 3 < M) ? row[x0 + 3] : 0;
        }
        a0 += p0; a1 += p1; a2 += p2; a3 += p3;
        q0 += p0 * p0; q1 += p1 * p1; q2 += p2 * p2; q3 += p3 * p3;
    }
    int32_t* o1 = cs1 + (size_t)b * M + x0;
    int32_t* o2 = cs2 + (size_t)b * M + x0;
    o1[0] = a0; o2[0] = q0;
    if (x0 + 1 < M) { o1[1] = a1; o2[1] = q1; }
    if (x0 + 2 < M) { o1[2] = a2; o2[2] = q2; }
    if (x0 + 3 < M) { o1[3] = a3; o2[3] = q3; }
}

// Pass 2: in place, cs[b][x] := sum_{b' < b} cs[b'][x] (exclusive over bands).
// One CTA per 32 columns: lane = column (coalesced rows), warp w owns a
// contiguous chunk of bands; chunk totals are exchanged through shared memory
// so every warp walks only nb/8 bands, twice.
__global__ void __launch_bounds__(256) sat_band_scan(int M, int nb, int32_t* __restrict__ cs1,
                                                     int32_t* __restrict__ cs2) {
    __shared__ int32_t tot1[8][32], tot2[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x = blockIdx.x * 32 + lane;
    const int per = (nb + 7) / 8;
    const int b0 = min(warp * per, nb), b1 = min(b0 + per, nb);
    int32_t s1 = 0, s2 = 0;
    if (x < M) {
        int b = b0;
        for (; b + 8 <= b1; b += 8) {
            int32_t v1[8], v2[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                v1[i] = cs1[(size_t)(b + i) * M + x];
                v2[i] = cs2[(size_t)(b + i) * M + x];
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) { s1 += v1[i]; s2 += v2[i]; }
        }
        for (; b < b1; ++b) { s1 += cs1[(size_t)b * M + x]; s2 += cs2[(size_t)b * M + x]; }
    }
    tot1[warp][lane] = s1;
    tot2[warp][lane] = s2;
    __syncthreads();
    int32_t r1 = 0, r2 = 0;
    for (int w = 0; w < warp; ++w) { r1 += tot1[w][lane]; r2 += tot2[w][lane]; }
    if (x >= M) return;
    int b = b0;
    for (; b + 8 <= b1; b += 8) {
        int32_t v1[8], v2[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            v1[i] = cs1[(size_t)(b + i) * M + x];
            v2[i] = cs2[(size_t)(b + i) * M + x];
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            cs1[(size_t)(b + i) * M + x] = r1;
            cs2[(size_t)(b + i) * M + x] = r2;
            r1 += v1[i];
            r2 += v2[i];
        }
    }
    for (; b < b1; ++b) {
        const int32_t v1 = cs1[(size_t)b * M + x], v2 = cs2[(size_t)b * M + x];
        cs1[(size_t)b * M + x] = r1;
        cs2[(size_t)b * M + x] = r2;
        r1 += v1;
        r2 += v2;
    }
}

// Inclusive CTA-wide scan of two 64-bit values.  All threads call it.
__device__ __forceinline__ void block_scan2(int64_t& a, int64_t& b, int64_t* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t ta = __shfl_up_sync(0xffffffffu, a, o);
        const int64_t tb = __shfl_up_sync(0xffffffffu, b, o);
        if (lane >= o) { a += ta; b += tb; }
    }
    if (lane == 31) { sm[warp] = a; sm[32 + warp] = b; }
    __syncthreads();
    if (warp == 0) {
        int64_t wa = (lane < nw) ? sm[lane] : 0, wb = (lane < nw) ? sm[32 + lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t ta = __shfl_up_sync(0xffffffffu, wa, o);
            const int64_t tb = __shfl_up_sync(0xffffffffu, wb, o);
            if (lane >= o) { wa += ta; wb += tb; }
        }
        if (lane < nw) { sm[64 + lane] = wa; sm[96 + lane] = wb; }
    }
    __syncthreads();
    if (warp > 0) { a += sm[64 + warp - 1]; b += sm[96 + warp - 1]; }
    // no trailing barrier: callers alternate between two scratch copies, and
    // the next use of this copy is two scans (and two barriers) later
}

// Pass 3.  Thread t owns output columns X in [tE, tE+E), i.e. inputs
// x = X - 1 in [tE-1, tE+E-1); it keeps their running column sums (the
// column prefix of f above the current row) in registers.
template <int E, typename ST>
__global__ void sat_emit(const uint8_t* __restrict__ f, int M, int N, int stride, int R, int pitch,
                         const int32_t* __restrict__ cs1, const int32_t* __restrict__ cs2, ST* __restrict__ s,
                         int64_t* __restrict__ s2) {
    __shared__ int64_t sm[2][128];
    const int b = blockIdx.x;
    const int t = threadIdx.x;
    const int X0 = t * E;
    const int y0 = b * R;
    const int y1 = min(y0 + R, N);
    int32_t col[E], col2[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int x = X0 + e - 1;
        const bool in = (x >= 0) && (x < M);
        col[e] = in ? cs1[(size_t)b * M + x] : 0;
        col2[e] = in ? cs2[(size_t)b * M + x] : 0;
    }
    const bool full = (X0 + E - 1 <= M);
    if (b == 0) {  // row Y = 0 is all zero
        for (int e = 0; e < E; ++e)
            if (X0 + e <= M) { s[X0 + e] = 0; s2[X0 + e] = 0; }
    }
    const bool vec = ((stride & 7) == 0) && ((reinterpret_cast<uintptr_t>(f) & 7) == 0) && (E == 8) &&
                     (X0 + E - 1 < M) && (X0 >= 1);
    // Loads the E input bytes x = X0-1 .. X0+E-2 of row y (zero outside the row).
    auto load_row = [&](int y, int (&v)[E]) {
        const uint8_t* row = f + (size_t)y * stride;
        if (vec) {
            // one aligned 8-byte load (X0 .. X0+7, inside the row) plus the byte before
            const uint2 w = __ldg(reinterpret_cast<const uint2*>(row + X0));
            v[0] = row[X0 - 1];
            v[1] = w.x & 0xff; v[2] = (w.x >> 8) & 0xff; v[3] = (w.x >> 16) & 0xff; v[4] = w.x >> 24;
            v[5] = w.y & 0xff; v[6] = (w.y >> 8) & 0xff; v[7] = (w.y >> 16) & 0xff;
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int x = X0 + e - 1;
                v[e] = (x >= 0 && x < M) ? row[x] : 0;
            }
        }
    };
    int nxt[E];
    if (y0 < y1) load_row(y0, nxt);
    for (int y = y0; y < y1; ++y) {
        int v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = nxt[e];
        if (y + 1 < y1) load_row(y + 1, nxt);  // in flight during this row's scan
        int64_t p[E], p2[E];
        int64_t run = 0, run2 = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            col[e] += v[e];
            col2[e] += v[e] * v[e];
            run += col[e];
            run2 += col2[e];
            p[e] = run;
            p2[e] = run2;
        }
        int64_t inc = run, inc2 = run2;
        block_scan2(inc, inc2, sm[(y - y0) & 1]);
        const int64_t base = inc - run, base2 = inc2 - run2;
        ST* srow = s + (size_t)(y + 1) * pitch + X0;
        int64_t* s2row = s2 + (size_t)(y + 1) * pitch + X0;
        if (full) {
            if constexpr (sizeof(ST) == 4) {
#pragma unroll
                for (int e = 0; e < E; e += 4) {
                    int4 o;
                    o.x = (int)(base + p[e]); o.y = (int)(base + p[e + 1]);
                    o.z = (int)(base + p[e + 2]); o.w = (int)(base + p[e + 3]);
                    *reinterpret_cast<int4*>(srow + e) = o;
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; e += 2) {
                    longlong2 o;
                    o.x = base + p[e]; o.y = base + p[e + 1];
                    *reinterpret_cast<longlong2*>(srow + e) = o;
                }
            }
#pragma unroll
            for (int e = 0; e < E; e += 2) {
                longlong2 o;
                o.x = base2 + p2[e]; o.y = base2 + p2[e + 1];
                *reinterpret_cast<longlong2*>(s2row + e) = o;
            }
        } else {
            for (int e = 0; e < E; ++e)
                if (X0 + e <= M) {
                    srow[e] = (ST)(base + p[e]);
                    s2row[e] = base2 + p2[e];
                }
        }
    }
}

template <int E>
cudaError_t launch_emit(const SatGeometry& g, const uint8_t* f, int M, int N, int stride, int pitch,
                        const int32_t* cs1, const int32_t* cs2, void* s, int s_bits, int64_t* s2,
                        cudaStream_t st) {
    if (s_bits == 32)
        sat_emit<E, int32_t><<<g.nb, g.T, 0, st>>>(f, M, N, stride, g.R, pitch, cs1, cs2, (int32_t*)s, s2);
    else
        sat_emit<E, int64_t><<<g.nb, g.T, 0, st>>>(f, M, N, stride, g.R, pitch, cs1, cs2, (int64_t*)s, s2);
    return cudaGetLastError();
}

}  // namespace
}  // namespace sncc

extern "C" size_t sncc_integral_workspace_bytes(int M, int N) {
    if (M <= 0 || N <= 0) return 0;
    const sncc::SatGeometry g = sncc::sat_geometry(M, N);
    return (size_t)2 * g.nb * (size_t)M * sizeof(int32_t) + 256;
}

extern "C" int sncc_integral(const uint8_t* d_f, int M, int N, int f_stride, void* d_s, int s_bits, int64_t* d_s2,
                             int sat_pitch, void* d_ws, size_t ws_bytes, sncc_stream_t stream) {
    using namespace sncc;
    if (!d_f || !d_s || !d_s2 || M <= 0 || N <= 0 || f_stride < M) return SNCC_ERR_ARG;
    if (s_bits != 32 && s_bits != 64) return SNCC_ERR_ARG;
    if (M > 16383 || N > 65535) return SNCC_ERR_UNSUPPORTED;
    if (sat_pitch < M + 1 || (sat_pitch & 3)) return SNCC_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(d_s) & 15) || (reinterpret_cast<uintptr_t>(d_s2) & 15)) return SNCC_ERR_ARG;
    // s fits in int32 only while its largest entry 255*M*N does; the column
    // sums of f^2 kept in int32 need N*65025 < 2^31.
    if (s_bits == 32 && (int64_t)255 * M * N >= ((int64_t)1 << 31)) return SNCC_ERR_DTYPE;
    if ((int64_t)N * 65025 >= ((int64_t)1 << 31)) return SNCC_ERR_UNSUPPORTED;
    if (!d_ws || ws_bytes < sncc_integral_workspace_bytes(M, N) || (reinterpret_cast<uintptr_t>(d_ws) & 15))
        return SNCC_ERR_WORKSPACE;
    const SatGeometry g = sat_geometry(M, N);
    int32_t* cs1 = static_cast<int32_t*>(d_ws);
    int32_t* cs2 = cs1 + (size_t)g.nb * M;
    cudaStream_t st = (cudaStream_t)stream;
    dim3 g1((M / 4 + 1 + 255) / 256, g.nb);
    sat_band_colsum<<<g1, 256, 0, st>>>(d_f, M, N, f_stride, g.R, cs1, cs2);
    sat_band_scan<<<(M + 31) / 32, 256, 0, st>>>(M, g.nb, cs1, cs2);
    cudaError_t e = (g.E == 8) ? launch_emit<8>(g, d_f, M, N, f_stride, sat_pitch, cs1, cs2, d_s, s_bits, d_s2, st)
                               : launch_emit<16>(g, d_f, M, N, f_stride, sat_pitch, cs1, cs2, d_s, s_bits, d_s2, st);
    return e == cudaSuccess ? SNCC_OK : SNCC_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Allocation-free entry point.  The band sums normally live in the caller's
// workspace; here they live in this fixed array instead, which the library
// owns for the life of the process on every device that loads it.
// ---------------------------------------------------------------------------
static __device__ __align__(256) int32_t sncc_noalloc_scratch[SNCC_NOALLOC_SCRATCH_BYTES / sizeof(int32_t)];

namespace {

constexpr int kNoallocMaxDevices = 128;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoallocMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the array's name as a device pointer).
int noalloc_scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return SNCC_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_addr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, sncc_noalloc_scratch) != cudaSuccess || p == nullptr) return SNCC_ERR_CUDA;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return SNCC_OK;
}

}  // namespace

extern "C" int sncc_integral_noalloc(const uint8_t* d_f, int M, int N, int f_stride, void* d_s, int s_bits,
                                     int64_t* d_s2, int sat_pitch, sncc_stream_t stream) {
    if (!d_f || !d_s || !d_s2 || M <= 0 || N <= 0 || f_stride < M) return SNCC_ERR_ARG;
    if (sncc_integral_workspace_bytes(M, N) > (size_t)SNCC_NOALLOC_SCRATCH_BYTES) return SNCC_ERR_CAPACITY;
    void* scratch = nullptr;
    const int rc = noalloc_scratch_address(&scratch);
    if (rc != SNCC_OK) return rc;
    return sncc_integral(d_f, M, N, f_stride, d_s, s_bits, d_s2, sat_pitch, scratch, SNCC_NOALLOC_SCRATCH_BYTES,
                         stream);
}
