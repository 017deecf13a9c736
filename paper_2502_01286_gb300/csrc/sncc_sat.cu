// sncc_sat.cu - exact integer sum tables of f and f^2 (Eq. 10 and Eq. 14).
//
// Layout: padded tables of (N+1) rows x pitch elements, entry [Y*pitch + X]
// = sum of f over x < X, y < Y (row 0 and column 0 are zero).
//
// The table is produced band by band (R rows each).  A band is independent
// once its column carries are known:
//   1. band column sums: for every band and column, the sum of f (and f^2)
//      over the band's rows;
//   2. band scan: exclusive prefix of those over the bands, i.e. for every
//      band and column the sum of the column above the band;
//   3. band emit (one CTA of 8 warps per band): the band's columns are cut
//      into 256-column tiles, one lane per 8 output columns.  The CTA first
//      sums, per tile, the column carries and every row's own values, and
//      prefixes those sums over the tiles (the corner above-left of each tile
//      and each row's sum left of it); then each warp walks its tiles row by
//      row: running column sums in registers, a lane prefix and one warp scan
//      per row (no CTA barrier), values relative to the tile in int32 and the
//      carries added in int64, and 16-byte stores.
// Algorithmic traffic: 1 B/px read, 4 or 8 B/px (s) + 8 B/px (s^2) written;
// pass 1 and the emit's first phase read f once more each (from L2), and the
// carries are small arrays.
#include <cuda_runtime.h>

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "sncc.h"
#include "sncc_internal.h"

namespace sncc {
namespace {

constexpr int kEmitWarps = 8;                 // warps per band-emit CTA
constexpr int kLaneCols = 8;                  // output columns per lane
constexpr int kTileCols = 32 * kLaneCols;     // output columns per warp tile
constexpr int kMaxTiles = 16384 / kTileCols;  // tiles of the widest table (M + 1 <= 16384)
constexpr int kMaxR = 64;                     // rows per band at most
constexpr int kTargetTiles = 4864;           // warp tiles (band x 256 columns) in all: about 32 per SM
                                              // of a 152-SM part; fixed, so that the workspace size
                                              // depends on the source size alone

struct SatGeometry {
    int R;   // rows per band
    int nb;  // bands
    int nc;  // 256-column tiles per band
};

SatGeometry sat_geometry(int M, int N) {
    SatGeometry g;
    g.nc = (M + 1 + kTileCols - 1) / kTileCols;  // tiles cover output columns 0 .. M
    // bands of R rows with about kTargetTiles warp tiles in all; the column-sum
    // workspace is then 2 * (N / R) * M * 4 bytes <= about 12.6 MB for any
    // source up to 10^8 pixels
    long long r = ((long long)N * g.nc + kTargetTiles - 1) / kTargetTiles;
    // at least N/256 rows (2 to 8): short sources keep about 256 bands for
    // parallelism, taller ones fewer, shorter passes over the bands (on a
    // 1920 x 1080 source N/256 took 23.7 us against 25.7 us for N/128 and
    // 31.9 us for N/512)
    const long long rmin = std::min(8LL, std::max(2LL, (long long)N / 256));
    if (r < rmin) r = rmin;
    if (r > kMaxR) r = kMaxR;
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
    auto word = [&](int y) -> uint32_t {
        const uint8_t* row = f + (size_t)y * stride;
        if (vec) return __ldg(reinterpret_cast<const uint32_t*>(row + x0));
        uint32_t w = row[x0];
        if (x0 + 1 < M) w |= (uint32_t)row[x0 + 1] << 8;
        if (x0 + 2 < M) w |= (uint32_t)row[x0 + 2] << 16;
        if (x0 + 3 < M) w |= (uint32_t)row[x0 + 3] << 24;
        return w;
    };
    auto add = [&](uint32_t w) {
        const int p0 = w & 0xff, p1 = (w >> 8) & 0xff, p2 = (w >> 16) & 0xff, p3 = w >> 24;
        a0 += p0; a1 += p1; a2 += p2; a3 += p3;
        q0 += p0 * p0; q1 += p1 * p1; q2 += p2 * p2; q3 += p3 * p3;
    };
    int y = y0;
    for (; y + 4 <= y1; y += 4) {  // four rows of loads in flight
        const uint32_t w0 = word(y), w1 = word(y + 1), w2 = word(y + 2), w3 = word(y + 3);
        add(w0); add(w1); add(w2); add(w3);
    }
    for (; y < y1; ++y) add(word(y));
    int32_t* o1 = cs1 + (size_t)b * M + x0;
    int32_t* o2 = cs2 + (size_t)b * M + x0;
    o1[0] = a0; o2[0] = q0;
    if (x0 + 1 < M) { o1[1] = a1; o2[1] = q1; }
    if (x0 + 2 < M) { o1[2] = a2; o2[2] = q2; }
    if (x0 + 3 < M) { o1[3] = a3; o2[3] = q3; }
}

// Pass 2: in place, cs[b][x] := sum_{b' < b} cs[b'][x] (exclusive over bands).
// One CTA per 32 columns: lane = column (coalesced rows), warp w of 32 owns a
// contiguous run of bands; run totals are exchanged through shared memory,
// so every warp walks only nb/32 bands, twice.
constexpr int kScanWarps = 32;

__global__ void __launch_bounds__(kScanWarps * 32) sat_band_scan(int M, int nb, int32_t* __restrict__ cs1,
                                                                 int32_t* __restrict__ cs2) {
    __shared__ int32_t tot1[kScanWarps][32], tot2[kScanWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x = blockIdx.x * 32 + lane;
    const int per = (nb + kScanWarps - 1) / kScanWarps;
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

// Pass 3: one CTA per band b.  Output column X of the table holds sources
// x < X, so tile c (outputs X = 256c .. 256c+255) owns the sources
// x = 256c - 1 .. 256c + 254, and lane l of a tile the sources
// 256c + 8l - 1 .. 256c + 8l + 6.  For output (X, Y) of the band, Y = y + 1:
//   s = [x < 256c-1, y < y0]        corner[c]        (prefix of P over tiles)
//     + [x < 256c-1, y0 <= y' <= y] sum of left[c][y'] (prefix of T over tiles)
//     + [own x <= X-1, y < y0]      top carry of the lane's column
//     + [own x <= X-1, y0 <= y' <= y] running column sums, prefixed along the tile.
// The first two come from the CTA's first phase (P: a tile's column carries
// summed; T: a tile's own values of one row summed), the last two from a lane
// prefix plus a warp scan.  Relative sums of one band and tile stay below
// 256 * 64 * 65025 < 2^31.

// Raw source bytes xa .. xa+7 of a row (zero from column M on), one 8-byte
// load when aligned and inside the row.
__device__ __forceinline__ uint2 load_word(const uint8_t* row, int M, int xa, bool vec) {
    if (vec && xa + 7 < M) return __ldg(reinterpret_cast<const uint2*>(row + xa));
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const uint32_t b = (xa + e < M) ? row[xa + e] : 0u;
        if (e < 4) lo |= b << (8 * e); else hi |= b << (8 * (e - 4));
    }
    return make_uint2(lo, hi);
}

// Lane l of a tile starting at output column X0 owns the sources
// x = X0 + 8l - 1 .. X0 + 8l + 6: bytes 0..6 of its own word (xa = X0 + 8l)
// and byte 7 of the previous lane's word; lane 0 reads x = X0 - 1 itself.
struct LaneRow {
    uint2 w;
    int edge;  // lane 0: source X0 - 1 (0 outside the row); other lanes unused
};

__device__ __forceinline__ LaneRow load_lane_row(const uint8_t* row, int M, int X0, int lane, bool vec) {
    const int xa = X0 + kLaneCols * lane;
    LaneRow r;
    r.w = load_word(row, M, xa, vec);
    r.edge = (lane == 0 && xa >= 1 && xa - 1 < M) ? row[xa - 1] : 0;
    return r;
}

__device__ __forceinline__ void unpack_lane_row(const LaneRow& r, int lane, int (&v)[8]) {
    const uint32_t prev = __shfl_up_sync(0xffffffffu, r.w.y, 1);
    v[0] = (lane > 0) ? (int)(prev >> 24) : r.edge;
#pragma unroll
    for (int e = 1; e < 8; ++e)
        v[e] = (int)(((e - 1 < 4) ? (r.w.x >> (8 * (e - 1))) : (r.w.y >> (8 * (e - 5)))) & 0xff);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_exclusive_scan(T v, int lane) {
    T inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    return inc - v;
}

constexpr int kAhead = 4;  // source rows in flight per warp
constexpr int kLaneStride = 80;  // staging bytes per lane: up to 64 data + 16 pad (conflict-free quarter-warps)
constexpr int kStageBytes = 32 * kLaneStride;

// Writes the lane's eight outputs a + col[0], a + col[0] + col[1], ... (as T)
// into the warp's staging buffer, then the warp stores the 256 values of the
// tile row to dst with 16-byte lane-consecutive stores (512 bytes each).
template <typename T>
__device__ __forceinline__ void stage_row(unsigned char* stage, int lane, const int32_t (&col)[kLaneCols], int64_t a,
                                          T* dst) {
    T o[kLaneCols];
#pragma unroll
    for (int e = 0; e < kLaneCols; ++e) {
        a += col[e];
        o[e] = (T)a;
    }
    unsigned char* mine = stage + lane * kLaneStride;
#pragma unroll
    for (int k = 0; k < (int)(kLaneCols * sizeof(T)) / 16; ++k)
        *reinterpret_cast<int4*>(mine + 16 * k) = *reinterpret_cast<const int4*>(reinterpret_cast<const char*>(o) + 16 * k);
    __syncwarp();
    constexpr int rowbytes = kTileCols * (int)sizeof(T);
#pragma unroll
    for (int j = 0; j < rowbytes / 512; ++j) {
        const int byte = 16 * lane + 512 * j;  // logical offset in the tile row
        const int4 v = *reinterpret_cast<const int4*>(stage + (byte / (kLaneCols * (int)sizeof(T))) * kLaneStride +
                                                      byte % (kLaneCols * (int)sizeof(T)));
        *reinterpret_cast<int4*>(reinterpret_cast<char*>(dst) + byte) = v;
    }
    __syncwarp();
}

template <typename ST>
__global__ void __launch_bounds__(kEmitWarps * 32, 3) sat_band_emit(const uint8_t* __restrict__ f, int M, int N,
                                                                 int stride, int R, int nc, int pitch,
                                                                 const int32_t* __restrict__ ca1,
                                                                 const int32_t* __restrict__ ca2,
                                                                 ST* __restrict__ s, int64_t* __restrict__ s2) {
    extern __shared__ __align__(16) unsigned char emit_smem[];
    // per-warp output staging (lane stride 80 bytes: 64 data + 16 pad), then
    // the per-tile row sums T (nc x R int32 each)
    unsigned char* stage = emit_smem + (size_t)(threadIdx.x >> 5) * kStageBytes;
    int32_t* T1 = reinterpret_cast<int32_t*>(emit_smem + kEmitWarps * kStageBytes);
    int32_t* T2 = T1 + (size_t)nc * R;
    __shared__ int64_t P1[kMaxTiles], P2[kMaxTiles];
    const int b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int y0 = b * R, nr = min(R, N - y0);
    const int32_t* cab1 = ca1 + (size_t)b * M;  // column sums above this band
    const int32_t* cab2 = ca2 + (size_t)b * M;
    const bool vec = ((stride & 7) == 0) && ((reinterpret_cast<uintptr_t>(f) & 7) == 0);
    const uint8_t* fband = f + (size_t)y0 * stride;

    // Phase 1: per tile, the column sums above the band over its sources (P)
    // and every row's own values (T), each summed over the tile.
    for (int c = warp; c < nc; c += kEmitWarps) {
        const int X0 = c * kTileCols;
        int64_t p1 = 0, p2 = 0;
#pragma unroll
        for (int e = 0; e < kLaneCols; ++e) {
            const int x = X0 + kLaneCols * lane - 1 + e;
            if (x >= 0 && x < M) {
                p1 += cab1[x];
                p2 += cab2[x];
            }
        }
        p1 = warp_sum(p1);
        p2 = warp_sum(p2);
        if (lane == 0) {
            P1[c] = p1;
            P2[c] = p2;
        }
        for (int r0 = 0; r0 < nr; r0 += kAhead) {
            LaneRow q[kAhead];
#pragma unroll
            for (int i = 0; i < kAhead; ++i)
                if (r0 + i < nr) q[i] = load_lane_row(fband + (size_t)(r0 + i) * stride, M, X0, lane, vec);
#pragma unroll
            for (int i = 0; i < kAhead; ++i) {
                if (r0 + i >= nr) break;
                int v[8];
                unpack_lane_row(q[i], lane, v);
                int t1 = 0, t2 = 0;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    t1 += v[e];
                    t2 += v[e] * v[e];
                }
                t1 = warp_sum(t1);
                t2 = warp_sum(t2);
                if (lane == 0) {
                    T1[c * R + r0 + i] = t1;
                    T2[c * R + r0 + i] = t2;
                }
            }
        }
    }
    __syncthreads();
    // Exclusive prefixes over the tiles: thread r < nr for row r, thread nr for P.
    if ((int)threadIdx.x < nr) {
        const int r = threadIdx.x;
        int32_t a1 = 0, a2 = 0;
        for (int c = 0; c < nc; ++c) {
            const int32_t t1 = T1[c * R + r], t2 = T2[c * R + r];
            T1[c * R + r] = a1;
            T2[c * R + r] = a2;
            a1 += t1;
            a2 += t2;
        }
    } else if ((int)threadIdx.x == nr) {
        int64_t a1 = 0, a2 = 0;
        for (int c = 0; c < nc; ++c) {
            const int64_t p1 = P1[c], p2 = P2[c];
            P1[c] = a1;
            P2[c] = a2;
            a1 += p1;
            a2 += p2;
        }
    }
    __syncthreads();

    // Phase 2: the band's outputs, tile by tile.  col holds the lane's
    // absolute column sums (above the band plus the band's rows so far), which
    // fit int32; the prefix along the tile is formed in int64 as it is stored.
    if (b == 0) {  // row Y = 0 of the table is zero
        for (int X = threadIdx.x; X <= M; X += blockDim.x) {
            s[X] = 0;
            s2[X] = 0;
        }
    }
    for (int c = warp; c < nc; c += kEmitWarps) {
        const int X0 = c * kTileCols, Xl = X0 + kLaneCols * lane;
        int32_t col1[kLaneCols], col2[kLaneCols];
#pragma unroll
        for (int e = 0; e < kLaneCols; ++e) {
            const int x = Xl - 1 + e;
            const bool in = (x >= 0 && x < M);
            col1[e] = in ? cab1[x] : 0;
            col2[e] = in ? cab2[x] : 0;
        }
        int64_t left1 = P1[c], left2 = P2[c];  // corner, then plus the rows' left sums
        const bool full_tile = (X0 + kTileCols - 1 <= M);  // warp-uniform
        LaneRow q[kAhead];
#pragma unroll
        for (int i = 0; i < kAhead; ++i)
            if (i < nr) q[i] = load_lane_row(fband + (size_t)i * stride, M, X0, lane, vec);
        for (int r = 0; r < nr; ++r) {
            int v[8];
            unpack_lane_row(q[0], lane, v);
#pragma unroll
            for (int i = 0; i < kAhead - 1; ++i) q[i] = q[i + 1];
            if (r + kAhead < nr) q[kAhead - 1] = load_lane_row(fband + (size_t)(r + kAhead) * stride, M, X0, lane, vec);
            int64_t t1 = 0, t2 = 0;
#pragma unroll
            for (int e = 0; e < kLaneCols; ++e) {
                col1[e] += v[e];
                col2[e] += v[e] * v[e];
                t1 += col1[e];
                t2 += col2[e];
            }
            left1 += T1[c * R + r];
            left2 += T2[c * R + r];
            int64_t a1 = left1 + warp_exclusive_scan(t1, lane), a2 = left2 + warp_exclusive_scan(t2, lane);
            ST* srow = s + (size_t)(y0 + r + 1) * pitch;
            int64_t* s2row = s2 + (size_t)(y0 + r + 1) * pitch;
            if (full_tile) {
                // through the warp's staging buffer, so that every global store
                // instruction writes 512 contiguous bytes
                stage_row<ST>(stage, lane, col1, a1, srow + X0);
                stage_row<int64_t>(stage, lane, col2, a2, s2row + X0);
            } else {
#pragma unroll
                for (int e = 0; e < kLaneCols; ++e) {
                    a1 += col1[e];
                    a2 += col2[e];
                    if (Xl + e <= M) {
                        srow[Xl + e] = (ST)a1;
                        s2row[Xl + e] = a2;
                    }
                }
            }
        }
    }
}

// The emit kernel's dynamic shared memory can exceed the 48 KB default
// (staging 20 KB + row sums up to 32 KB).
cudaError_t set_emit_attributes() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        const int most = kEmitWarps * kStageBytes + 2 * kMaxTiles * kMaxR * (int)sizeof(int32_t);
        err = cudaFuncSetAttribute(sat_band_emit<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(sat_band_emit<int64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    });
    return err;
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
    sncc::NvtxRange nvtx_range("sncc_integral");
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
    sat_band_scan<<<(M + 31) / 32, kScanWarps * 32, 0, st>>>(M, g.nb, cs1, cs2);
    const size_t smem = (size_t)kEmitWarps * kStageBytes + (size_t)2 * g.nc * g.R * sizeof(int32_t);
    if (set_emit_attributes() != cudaSuccess) return SNCC_ERR_CUDA;
    if (s_bits == 32)
        sat_band_emit<int32_t><<<g.nb, kEmitWarps * 32, smem, st>>>(d_f, M, N, f_stride, g.R, g.nc, sat_pitch, cs1,
                                                                   cs2, static_cast<int32_t*>(d_s), d_s2);
    else
        sat_band_emit<int64_t><<<g.nb, kEmitWarps * 32, smem, st>>>(d_f, M, N, f_stride, g.R, g.nc, sat_pitch, cs1,
                                                                   cs2, static_cast<int64_t*>(d_s), d_s2);
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
struct NoallocEntry {
    unsigned long long ctx_id;  // context the address was taken in (0 = none yet)
    void* addr;
};
std::mutex g_noalloc_mu;
NoallocEntry g_noalloc[kNoallocMaxDevices] = {};

// Unique identity of the calling thread's current context, 0 if unknown.
// A device reset, or a primary context released and retained again, gives a
// new identity, and the module (with its arrays) may then sit elsewhere.
unsigned long long current_context_id() {
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || c == nullptr || get_id(c, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the scratch array on the current device (host code
// cannot use the array's name as a device pointer).  Looked up once per
// device and context: a call in a context other than the one the cached
// address was taken in looks it up again; if the context cannot be
// identified, it is looked up on every call.
int noalloc_scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return SNCC_ERR_CUDA;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocEntry& e = g_noalloc[dev];
    if (ctx == 0 || e.ctx_id != ctx || e.addr == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, sncc_noalloc_scratch) != cudaSuccess || p == nullptr) return SNCC_ERR_CUDA;
        e.ctx_id = ctx;
        e.addr = p;
    }
    *out = e.addr;
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
