// sncc_sat.cu - exact integer sum tables of f and f^2 (Eq. 10 and Eq. 14).
//
// Layout: padded tables of (N+1) rows x pitch elements, entry [Y*pitch + X]
// = sum of f over x < X, y < Y (row 0 and column 0 are zero).
//
// The table is produced in tiles of (band of R rows) x (chunk of 1024
// columns), so that every tile is independent once two kinds of carry are
// known:
//   1. band column sums: for every band and column, the sum of f (and f^2)
//      over the band's rows;
//   2. band scan: exclusive prefix of those over the bands, i.e. for every
//      band and column the sum of the column above the band;
//   3. row carries (one warp per row): for every row and chunk, the sum of the
//      row left of the chunk;
//   4. tile emit (one CTA of 256 threads per tile, four output columns per
//      thread, 16-byte stores): s(X, Y) = corner + sum of the row carries of
//      the band's rows so far + CTA-wide prefix over the tile of the running
//      column sums, where corner = the band's column carries left of the tile.
// Algorithmic traffic: 1 B/px read, 4 or 8 B/px (s) + 8 B/px (s^2) written;
// passes 1 and 3 read f once more each, and the carries are small arrays.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "sncc.h"
#include "sncc_internal.h"

namespace sncc {
namespace {

constexpr int kThreads = 256;             // threads per emit CTA
constexpr int kPer = 4;                   // source columns per emit thread
constexpr int kChunk = kThreads * kPer;   // columns per tile
constexpr int kTargetTiles = 8 * 152;     // about eight emit CTAs per SM

struct SatGeometry {
    int R;   // rows per band
    int nb;  // bands
    int nc;  // column chunks
};

SatGeometry sat_geometry(int M, int N) {
    SatGeometry g;
    g.nc = (M + 1 + kChunk - 1) / kChunk;  // chunks cover output columns 0 .. M
    long long r = ((long long)N * g.nc + kTargetTiles - 1) / kTargetTiles;
    if (r < 2) r = 2;
    if (r > 64) r = 64;
    if (r > N) r = N;
    g.R = (int)r;
    g.nb = (N + g.R - 1) / g.R;
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

// Pass 3: rc[c][y] = sum of f (f^2) over source columns x < 1024c of row y.
// One warp per row: lane l reads bytes 1024c + 32l .. 32l+31 of each chunk,
// the warp reduces the chunk sums, and lane 0 writes their exclusive prefix.
// Chunk sums fit int32 (M <= 16383).
__global__ void __launch_bounds__(256) sat_row_carry(const uint8_t* __restrict__ f, int M, int N, int stride,
                                                     int nc, int32_t* __restrict__ rc1, int32_t* __restrict__ rc2) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int y = blockIdx.x * 8 + warp;
    if (y >= N) return;  // warp-uniform; no CTA barrier below
    const uint8_t* row = f + (size_t)y * stride;
    const bool vec = ((stride & 15) == 0) && ((reinterpret_cast<uintptr_t>(f) & 15) == 0);
    int32_t run1 = 0, run2 = 0;
    for (int c = 0; c < nc; ++c) {
        const int xb = c * kChunk + lane * 32;
        int s1 = 0, s2 = 0;
        if (vec && xb + 31 < M) {
            const uint4* q = reinterpret_cast<const uint4*>(row + xb);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint4 w = __ldg(q + h);
                const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int a = (ws[i] >> (8 * k)) & 0xff;
                        s1 += a;
                        s2 += a * a;
                    }
            }
        } else {
            for (int k = 0; k < 32; ++k)
                if (xb + k < M) {
                    const int v = row[xb + k];
                    s1 += v;
                    s2 += v * v;
                }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            rc1[(size_t)c * N + y] = run1;
            rc2[(size_t)c * N + y] = run2;
        }
        run1 += s1;
        run2 += s2;
    }
}

// Inclusive CTA-wide scan of two 64-bit values.  All threads call it; sm is
// one of two scratch copies that callers alternate (see below).
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

// Pass 4: one CTA per tile (chunk c = blockIdx.x, band b = blockIdx.y).
// Thread t owns output columns X = 1024c + 4t .. 4t+3 (16-byte aligned
// stores), i.e. source columns x = X - 1; the tile's inputs therefore start
// at x = 1024c - 1, and the left carry is the table at X = 1024c - 1:
//   corner  = sum_{x < 1024c-1} (column sums above the band),
//   row y   : sum_{x < 1024c-1} f(x, y) = rc[c][y] - f(1024c - 1, y).
template <typename ST>
__global__ void __launch_bounds__(kThreads) sat_tile_emit(const uint8_t* __restrict__ f, int M, int N, int stride,
                                                          int R, int pitch, const int32_t* __restrict__ cs1,
                                                          const int32_t* __restrict__ cs2,
                                                          const int32_t* __restrict__ rc1,
                                                          const int32_t* __restrict__ rc2, ST* __restrict__ s,
                                                          int64_t* __restrict__ s2) {
    __shared__ int64_t sm[2][128];
    __shared__ int32_t rcs1[64], rcs2[64];
    const int c = blockIdx.x, b = blockIdx.y, t = threadIdx.x;
    const int lane = t & 31;
    const int X0 = c * kChunk;          // first output column of the tile
    const int Xt = X0 + kPer * t;       // this thread's first output column
    const int xe = X0 - 1;              // the source column just left of the tile's own
    const int y0 = b * R, y1 = min(y0 + R, N);
    // corner = column sums above the band over x < X0 - 1
    int64_t k1 = 0, k2 = 0;
    for (int i = t; i < xe; i += kThreads) {
        k1 += cs1[(size_t)b * M + i];
        k2 += cs2[(size_t)b * M + i];
    }
    if (t < y1 - y0) {  // the band's row carries, to shared memory
        rcs1[t] = rc1[(size_t)c * N + y0 + t];
        rcs2[t] = rc2[(size_t)c * N + y0 + t];
    }
    block_scan2(k1, k2, sm[0]);  // inclusive: the last thread holds the totals
    __syncthreads();
    if (t == kThreads - 1) { sm[1][0] = k1; sm[1][1] = k2; }
    __syncthreads();
    int64_t left1 = sm[1][0], left2 = sm[1][1];
    __syncthreads();
    int32_t col1[kPer], col2[kPer];
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        const int x = Xt + e - 1;
        const bool in = (x >= 0) && (x < M);
        col1[e] = in ? cs1[(size_t)b * M + x] : 0;
        col2[e] = in ? cs2[(size_t)b * M + x] : 0;
    }
    const bool full = (Xt + kPer - 1 <= M);  // all four outputs exist
    if (b == 0) {  // row Y = 0 is all zero
#pragma unroll
        for (int e = 0; e < kPer; ++e)
            if (Xt + e <= M) { s[Xt + e] = 0; s2[Xt + e] = 0; }
    }
    // Inputs x = Xt-1 .. Xt+2: an aligned 4-byte load of Xt .. Xt+3 gives the
    // last three; the first is the previous lane's fourth byte (lane 0 loads it).
    const bool vec = ((stride & 3) == 0) && ((reinterpret_cast<uintptr_t>(f) & 3) == 0) && (Xt + kPer - 1 < M);
    auto load = [&](int y, int (&v)[kPer], int& edge) {
        const uint8_t* row = f + (size_t)y * stride;
        uint32_t w = 0;
        if (vec) {
            w = __ldg(reinterpret_cast<const uint32_t*>(row + Xt));
        } else {
#pragma unroll
            for (int e = 0; e < kPer; ++e)
                if (Xt + e < M) w |= (uint32_t)row[Xt + e] << (8 * e);
        }
        const uint32_t prev = __shfl_up_sync(0xffffffffu, w, 1);
        const int x_first = Xt - 1;
        v[0] = (lane > 0) ? (int)(prev >> 24) : ((x_first >= 0 && x_first < M) ? row[x_first] : 0);
#pragma unroll
        for (int e = 1; e < kPer; ++e) v[e] = (w >> (8 * (e - 1))) & 0xff;
        edge = (xe >= 0) ? row[xe] : 0;  // uniform
    };
    int nxt[kPer], nedge = 0;
    if (y0 < y1) load(y0, nxt, nedge);
    for (int y = y0; y < y1; ++y) {
        int v[kPer];
#pragma unroll
        for (int e = 0; e < kPer; ++e) v[e] = nxt[e];
        const int edge = nedge;
        if (y + 1 < y1) load(y + 1, nxt, nedge);  // in flight during this row's scan
        int64_t p1[kPer], p2[kPer];
        int64_t r1 = 0, r2 = 0;
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
            col1[e] += v[e];
            col2[e] += v[e] * v[e];
            r1 += col1[e];
            r2 += col2[e];
            p1[e] = r1;
            p2[e] = r2;
        }
        int64_t i1 = r1, i2 = r2;
        block_scan2(i1, i2, sm[(y - y0) & 1]);
        if (xe >= 0) {
            left1 += rcs1[y - y0] - edge;
            left2 += rcs2[y - y0] - edge * edge;
        }
        const int64_t base1 = left1 + i1 - r1, base2 = left2 + i2 - r2;
        ST* srow = s + (size_t)(y + 1) * pitch + Xt;
        int64_t* s2row = s2 + (size_t)(y + 1) * pitch + Xt;
        if (full) {
            if constexpr (sizeof(ST) == 4) {
                int4 o;
                o.x = (int)(base1 + p1[0]); o.y = (int)(base1 + p1[1]);
                o.z = (int)(base1 + p1[2]); o.w = (int)(base1 + p1[3]);
                *reinterpret_cast<int4*>(srow) = o;
            } else {
                *reinterpret_cast<longlong2*>(srow) = make_longlong2(base1 + p1[0], base1 + p1[1]);
                *reinterpret_cast<longlong2*>(srow + 2) = make_longlong2(base1 + p1[2], base1 + p1[3]);
            }
            *reinterpret_cast<longlong2*>(s2row) = make_longlong2(base2 + p2[0], base2 + p2[1]);
            *reinterpret_cast<longlong2*>(s2row + 2) = make_longlong2(base2 + p2[2], base2 + p2[3]);
        } else {
#pragma unroll
            for (int e = 0; e < kPer; ++e)
                if (Xt + e <= M) {
                    srow[e] = (ST)(base1 + p1[e]);
                    s2row[e] = base2 + p2[e];
                }
        }
    }
}

}  // namespace
}  // namespace sncc

extern "C" size_t sncc_integral_workspace_bytes(int M, int N) {
    if (M <= 0 || N <= 0) return 0;
    const sncc::SatGeometry g = sncc::sat_geometry(M, N);
    return (size_t)2 * g.nb * (size_t)M * sizeof(int32_t) + (size_t)2 * g.nc * (size_t)N * sizeof(int32_t) + 256;
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
    int32_t* rc1 = cs2 + (size_t)g.nb * M;
    int32_t* rc2 = rc1 + (size_t)g.nc * N;
    cudaStream_t st = (cudaStream_t)stream;
    dim3 g1((M / 4 + 1 + 255) / 256, g.nb);
    sat_band_colsum<<<g1, 256, 0, st>>>(d_f, M, N, f_stride, g.R, cs1, cs2);
    sat_band_scan<<<(M + 31) / 32, 256, 0, st>>>(M, g.nb, cs1, cs2);
    sat_row_carry<<<(N + 7) / 8, 256, 0, st>>>(d_f, M, N, f_stride, g.nc, rc1, rc2);
    dim3 g4(g.nc, g.nb);
    if (s_bits == 32)
        sat_tile_emit<int32_t><<<g4, kThreads, 0, st>>>(d_f, M, N, f_stride, g.R, sat_pitch, cs1, cs2, rc1, rc2,
                                                      static_cast<int32_t*>(d_s), d_s2);
    else
        sat_tile_emit<int64_t><<<g4, kThreads, 0, st>>>(d_f, M, N, f_stride, g.R, sat_pitch, cs1, cs2, rc1, rc2,
                                                      static_cast<int64_t*>(d_s), d_s2);
    return cudaGetLastError() == cudaSuccess ? SNCC_OK : SNCC_ERR_CUDA;
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
