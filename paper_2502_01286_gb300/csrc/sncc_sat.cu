// sncc_sat.cu - exact integer sum tables of f and f^2 (Eq. 10 and Eq. 14).
//
// Layout: padded tables of (N+1) rows x pitch elements, entry [Y*pitch + X]
// = sum of f over x < X, y < Y (row 0 and column 0 are zero); a 32-bit s
// keeps the sums modulo 2^32.
//
// The table is produced band by band (R rows each) and, inside a band, tile
// by tile (256 output columns).  A (band, tile) is independent once three
// kinds of sums outside it are known, which the first two passes provide:
//   1. band column sums: for every band and column the sum of f (and f^2)
//      over the band's rows; and the row sums of every 256-column chunk of
//      every row;
//   2. band scan: exclusive prefix of the column sums over the bands (the
//      column carries: for every band and column the sum of the column
//      above the band), and per band the sums of the carries over every
//      32-column chunk;
//   3. band emit, one warp per (band, tile): from those it forms the corner
//      above-left of the tile and, per row, the row sum left of the tile;
//      then it walks the band's rows with running band-relative column sums
//      in registers (one lane per 8 columns), a lane prefix and a 32-bit
//      warp scan per row, adds one 64-bit base per lane, and stores each
//      tile row through a warp staging buffer as 512-byte stores.
// The scan and the emit are launched as programmatic dependents of the
// pass before them and wait for it in the kernel.
// Algorithmic traffic: 1 B/px read, 4 or 8 B/px (s) + 8 B/px (s^2) written;
// pass 1 and the emit read f once each (the second time mostly from L2), and
// the carry and chunk arrays are small.
#include <cuda_runtime.h>

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <type_traits>
#include <cstdint>
#include <mutex>

#include "sncc.h"
#include "sncc_internal.h"

namespace sncc {
namespace {

constexpr int kEmitWarps = 8;                 // warps per band-emit CTA, one (band, tile) each
constexpr int kEmitMinCtas = 24 / kEmitWarps;  // resident emit CTAs per SM the registers must allow (80 each)
constexpr int kColThreads = 32;               // threads per column-sum CTA (8 columns each): one-warp CTAs
                                              // spread the (band, chunk) warps evenly over the SMs
constexpr int kLaneCols = 8;                  // output columns per lane
constexpr int kTileCols = 32 * kLaneCols;     // output columns per warp tile
constexpr int kMaxR = 64;                     // rows per band at most
constexpr int kTargetTiles = 4864;           // warp tiles (band x 256 columns) in all, at most: sizes
                                              // the workspace, and bounds the launch's whole waves
constexpr int kCarryChunk = 32;               // columns per carry chunk sum (one scan CTA)

struct SatGeometry {
    int R;   // rows per band
    int nb;  // bands
    int nc;  // 256-column tiles per band (output columns 0 .. M)
    int nk;  // whole 256-column source chunks per row (the left sums read no other)
    int nj;  // whole 32-column carry chunks (the corners read no other)
};

// The workspace geometry: bands sized for about kTargetTiles warp tiles,
// fixed, so that the workspace size depends on the source size alone.
SatGeometry sat_geometry(int M, int N) {
    SatGeometry g;
    g.nc = (M + 1 + kTileCols - 1) / kTileCols;  // tiles cover output columns 0 .. M
    // tile c reads the chunks left of X0 = 256c <= M: whole ones only
    g.nk = M / kTileCols;
    g.nj = M / kCarryChunk;
    // bands of R rows with about kTargetTiles warp tiles in all; the column
    // sums are then 8 (N / R) M bytes, at most M N / 8 (12.5 MB for 10^8
    // pixels), the row chunk sums M N / 32 and the carry chunk sums M N / 128
    // at most
    long long r = ((long long)N * g.nc + kTargetTiles - 1) / kTargetTiles;
    // at least N/256 rows (2 to 8): short sources keep about 256 bands for
    // parallelism, taller ones fewer, shorter passes over the bands
    const long long rmin = std::min(8LL, std::max(2LL, (long long)N / 256));
    if (r < rmin) r = rmin;
    if (r > kMaxR) r = kMaxR;
    if (r > N) r = N;
    g.R = (int)r;
    g.nb = (N + g.R - 1) / g.R;
    return g;
}

// The launch geometry on a device with `slots` resident emit warps: bands no
// shorter than the workspace geometry's (so no more of them, and the
// workspace holds their sums), as short as lets every (band, tile) warp run
// in a whole number of waves, the largest that kTargetTiles allows.  With
// slots = 0 (unknown) it is the workspace geometry.
SatGeometry sat_launch_geometry(int M, int N, long long slots) {
    SatGeometry g = sat_geometry(M, N);
    if (slots <= 0) return g;
    const long long target = std::max(1LL, kTargetTiles / slots) * slots;
    const long long rmax = std::min<long long>(kMaxR, N);
    long long r = std::max<long long>(g.R, ((long long)N * g.nc + target - 1) / target);
    while (r < rmax && ((N + r - 1) / r) * g.nc > target) ++r;
    g.R = (int)std::min(r, rmax);
    g.nb = (N + g.R - 1) / g.R;
    return g;
}

// Workspace: column sums cs1, cs2 (nb x cp int32, cp = M rounded up to a
// multiple of 4 so that rows take 16-byte stores; carries after pass 2), row
// chunk sums rs1, rs2 (N x nk int32, by source row), carry chunk sums ch1,
// ch2 (nb x nj int64); a section may be empty.  Laid out for the workspace
// geometry, which has at least as many bands as any launch geometry.
struct SatWorkspace {
    size_t cs1, cs2, rs1, rs2, ch1, ch2, total;
};

int col_pitch(int M) { return (M + 3) & ~3; }

SatWorkspace sat_workspace(int M, int N, const SatGeometry& g) {
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    SatWorkspace w;
    size_t o = 0;
    w.cs1 = o;
    o = al(o + (size_t)g.nb * col_pitch(M) * 4);
    w.cs2 = o;
    o = al(o + (size_t)g.nb * col_pitch(M) * 4);
    w.rs1 = o;
    o = al(o + (size_t)N * g.nk * 4);
    w.rs2 = o;
    o = al(o + (size_t)N * g.nk * 4);
    w.ch1 = o;
    o = al(o + (size_t)g.nb * g.nj * 8);
    w.ch2 = o;
    o = al(o + (size_t)g.nb * g.nj * 8);
    w.total = o;
    return w;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp sum of non-negative 32-bit values whose total fits 32 bits: one
// reduction instruction.
__device__ __forceinline__ int32_t warp_sum_u32(int32_t v) {
    return (int32_t)__reduce_add_sync(0xffffffffu, (uint32_t)v);
}

// Warp sum of non-negative 32-bit values as a 64-bit total: the low and
// high halves reduced separately (each total below 2^21).
__device__ __forceinline__ int64_t warp_sum_wide(int32_t v) {
    const uint32_t lo = __reduce_add_sync(0xffffffffu, (uint32_t)v & 0xffffu);
    const uint32_t hi = __reduce_add_sync(0xffffffffu, (uint32_t)v >> 16);
    return ((int64_t)hi << 16) + (int64_t)lo;
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

__device__ __forceinline__ int byte_of(uint2 w, int e) {
    return (int)(((e < 4) ? (w.x >> (8 * e)) : (w.y >> (8 * (e - 4)))) & 0xffu);
}

// Pass 1: cs1[b][x] = sum_{y in band b} f(x, y), cs2 the same for f^2
// (rows of cp columns, those past M zero); and rs1[y nk + k] = sum of f
// over columns 256k .. 256k+255 of row y (rs2 for f^2), for the whole
// chunks k < nk.  A lane owns 8 columns, a warp one 256-column chunk; the
// next four rows load while four are summed.
constexpr int kColRows = 4;

__global__ void __launch_bounds__(kColThreads) sat_band_colsum(const uint8_t* __restrict__ f, int M, int N, int stride,
                                                       int R, int nk, int cp, int32_t* __restrict__ cs1,
                                                       int32_t* __restrict__ cs2, int32_t* __restrict__ rs1,
                                                       int32_t* __restrict__ rs2) {
    const int lane = threadIdx.x & 31;
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * kLaneCols;
    const int k = x0 / kTileCols;  // the warp's chunk
    if (x0 - kLaneCols * lane >= cp) return;  // the whole warp is past the row
    const int b = blockIdx.y;
    const int y0 = b * R, y1 = min(y0 + R, N);
    const bool vec = ((stride & 7) == 0) && ((reinterpret_cast<uintptr_t>(f) & 7) == 0);
    // column sums of f two to a word, in 16-bit halves (a band's sum is at
    // most 255 x 64 < 2^16): columns (0, 2), (1, 3), (4, 6), (5, 7)
    uint32_t a02 = 0, a13 = 0, a46 = 0, a57 = 0;
    int q[kLaneCols];
#pragma unroll
    for (int e = 0; e < kLaneCols; ++e) q[e] = 0;
    auto load_rows = [&](uint2 (&w)[kColRows], int y) {
#pragma unroll
        for (int i = 0; i < kColRows; ++i)
            w[i] = (x0 < M && y + i < y1) ? load_word(f + (size_t)(y + i) * stride, M, x0, vec) : make_uint2(0u, 0u);
    };
    uint2 cur[kColRows], nxt[kColRows];
    load_rows(cur, y0);
    for (int y = y0; y < y1; y += kColRows) {  // warp-uniform
        if (y + kColRows < y1) load_rows(nxt, y + kColRows);
        int s1[kColRows], s2[kColRows];
#pragma unroll
        for (int i = 0; i < kColRows; ++i) {
            const uint32_t lo = cur[i].x, hi = cur[i].y;
            a02 += lo & 0x00ff00ffu;
            a13 += (lo >> 8) & 0x00ff00ffu;
            a46 += hi & 0x00ff00ffu;
            a57 += (hi >> 8) & 0x00ff00ffu;
#pragma unroll
            for (int e = 0; e < kLaneCols; ++e) {
                const int p = byte_of(cur[i], e);
                q[e] += p * p;
            }
            // the row's sums over the lane's eight bytes: four byte products each
            s1[i] = (int)__dp4a(hi, 0x01010101u, __dp4a(lo, 0x01010101u, 0u));
            s2[i] = (int)__dp4a(hi, hi, __dp4a(lo, lo, 0u));
        }
#pragma unroll
        for (int i = 0; i < kColRows; ++i) {
            s1[i] = warp_sum_u32(s1[i]);  // at most 255^2 x 256 < 2^31
            s2[i] = warp_sum_u32(s2[i]);
        }
        if (lane == 0 && k < nk) {
#pragma unroll
            for (int i = 0; i < kColRows; ++i)
                if (y + i < y1) {
                    rs1[(size_t)(y + i) * nk + k] = s1[i];
                    rs2[(size_t)(y + i) * nk + k] = s2[i];
                }
        }
#pragma unroll
        for (int i = 0; i < kColRows; ++i) cur[i] = nxt[i];
    }
    // columns x0 .. x0+7 as two 16-byte stores each (cp and x0 are multiples
    // of 4; columns from M to cp hold zeros)
    const int a[kLaneCols] = {(int)(a02 & 0xffffu), (int)(a13 & 0xffffu), (int)(a02 >> 16), (int)(a13 >> 16),
                              (int)(a46 & 0xffffu), (int)(a57 & 0xffffu), (int)(a46 >> 16), (int)(a57 >> 16)};
#pragma unroll
    for (int h = 0; h < 2; ++h)
        if (x0 + 4 * h < cp) {
            *reinterpret_cast<int4*>(cs1 + (size_t)b * cp + x0 + 4 * h) =
                make_int4(a[4 * h], a[4 * h + 1], a[4 * h + 2], a[4 * h + 3]);
            *reinterpret_cast<int4*>(cs2 + (size_t)b * cp + x0 + 4 * h) =
                make_int4(q[4 * h], q[4 * h + 1], q[4 * h + 2], q[4 * h + 3]);
        }
}

// Pass 2: in place, cs[b][x] := sum_{b' < b} cs[b'][x] (exclusive over
// bands), and ch[b][j] = sum of the new cs[b][x] over the 32 columns of
// chunk j = blockIdx.x when it is whole (j < nj).  One CTA per 32 columns:
// lane = column (coalesced rows), warp w of 32 owns a contiguous run of
// bands; run totals are exchanged through shared memory, so every warp
// walks only nb/32 bands: once, held in registers, where that is at most
// kScanHold bands (4096 rows in bands of 20, 1080 in bands of 4), else twice,
// kScanBatch bands' loads at a time.
constexpr int kScanWarps = 32;
constexpr int kScanBatch = 4;
constexpr int kScanHold = 10;

__global__ void __launch_bounds__(kScanWarps * 32) sat_band_scan(int M, int nb, int nj, int cp,
                                                                 int32_t* __restrict__ cs1,
                                                                 int32_t* __restrict__ cs2,
                                                                 int64_t* __restrict__ ch1,
                                                                 int64_t* __restrict__ ch2) {
    __shared__ int32_t tot1[kScanWarps][32], tot2[kScanWarps][32];
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the column sums are complete
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x = blockIdx.x * 32 + lane;
    const bool in = x < M;
    const int per = (nb + kScanWarps - 1) / kScanWarps;
    const int b0 = min(warp * per, nb), b1 = min(b0 + per, nb);
    if (per <= kScanHold) {  // block-uniform: the warp's bands stay in registers
        int32_t v1[kScanHold], v2[kScanHold];
#pragma unroll
        for (int i = 0; i < kScanHold; ++i) {
            const bool ok = in && b0 + i < b1;
            v1[i] = ok ? cs1[(size_t)(b0 + i) * cp + x] : 0;
            v2[i] = ok ? cs2[(size_t)(b0 + i) * cp + x] : 0;
        }
        int32_t t1 = 0, t2 = 0;
#pragma unroll
        for (int i = 0; i < kScanHold; ++i) {
            t1 += v1[i];
            t2 += v2[i];
        }
        tot1[warp][lane] = t1;
        tot2[warp][lane] = t2;
        __syncthreads();
        int32_t r1 = 0, r2 = 0;
        for (int w = 0; w < warp; ++w) {
            r1 += tot1[w][lane];
            r2 += tot2[w][lane];
        }
#pragma unroll
        for (int i = 0; i < kScanHold; ++i) {
            if (b0 + i >= b1) break;  // warp-uniform
            const int32_t c1 = in ? r1 : 0, c2 = in ? r2 : 0;
            if (in) {
                cs1[(size_t)(b0 + i) * cp + x] = r1;
                cs2[(size_t)(b0 + i) * cp + x] = r2;
            }
            r1 += v1[i];
            r2 += v2[i];
            if ((int)blockIdx.x < nj) {  // block-uniform
                const int64_t h1 = warp_sum_wide(c1), h2 = warp_sum_wide(c2);
                if (lane == 0) {
                    ch1[(size_t)(b0 + i) * nj + blockIdx.x] = h1;
                    ch2[(size_t)(b0 + i) * nj + blockIdx.x] = h2;
                }
            }
        }
        return;
    }
    int32_t s1 = 0, s2 = 0;
    for (int b = b0; b < b1; b += kScanBatch) {  // warp-uniform
        int32_t v1[kScanBatch], v2[kScanBatch];
#pragma unroll
        for (int i = 0; i < kScanBatch; ++i) {
            const bool ok = in && b + i < b1;
            v1[i] = ok ? cs1[(size_t)(b + i) * cp + x] : 0;
            v2[i] = ok ? cs2[(size_t)(b + i) * cp + x] : 0;
        }
#pragma unroll
        for (int i = 0; i < kScanBatch; ++i) {
            s1 += v1[i];
            s2 += v2[i];
        }
    }
    tot1[warp][lane] = s1;
    tot2[warp][lane] = s2;
    __syncthreads();
    int32_t r1 = 0, r2 = 0;
    for (int w = 0; w < warp; ++w) {
        r1 += tot1[w][lane];
        r2 += tot2[w][lane];
    }
    // every lane stays in the loop (the chunk sums reduce over the warp);
    // columns past M contribute zeros
    for (int b = b0; b < b1; b += kScanBatch) {
        int32_t v1[kScanBatch], v2[kScanBatch];
#pragma unroll
        for (int i = 0; i < kScanBatch; ++i) {
            const bool ok = in && b + i < b1;
            v1[i] = ok ? cs1[(size_t)(b + i) * cp + x] : 0;
            v2[i] = ok ? cs2[(size_t)(b + i) * cp + x] : 0;
        }
        // v becomes the exclusive carries (zero past M)
#pragma unroll
        for (int i = 0; i < kScanBatch; ++i) {
            const int32_t t1 = v1[i], t2 = v2[i];
            v1[i] = in ? r1 : 0;
            v2[i] = in ? r2 : 0;
            if (in && b + i < b1) {
                cs1[(size_t)(b + i) * cp + x] = r1;
                cs2[(size_t)(b + i) * cp + x] = r2;
            }
            r1 += t1;
            r2 += t2;
        }
        if ((int)blockIdx.x < nj) {  // block-uniform
#pragma unroll
            for (int i = 0; i < kScanBatch; ++i) {
                const int64_t c1 = warp_sum_wide(v1[i]), c2 = warp_sum_wide(v2[i]);
                if (lane == 0 && b + i < b1) {
                    ch1[(size_t)(b + i) * nj + blockIdx.x] = c1;
                    ch2[(size_t)(b + i) * nj + blockIdx.x] = c2;
                }
            }
        }
    }
}

// Pass 3: one warp per (band b, tile c).  Output column X of the table holds
// sources x < X, so tile c (outputs X = 256c .. 256c+255, X0 = 256c) owns
// the sources x = X0 - 1 .. X0 + 254, and lane l the sources
// X0 + 8l - 1 .. X0 + 8l + 6: bytes 0..6 of its own word (xa = X0 + 8l) and
// byte 7 of the previous lane's word; lane 0 reads x = X0 - 1 itself.  For
// output (X, Y) with Y = y0 + r + 1 (row r of the band), X = X0 + 8l + e + ... :
//   s = P                               sum over x < X0-1, y < y0 (corner)
//     + L[r]                            sum over x < X0-1, y0 <= y <= y0+r (left)
//     + sum_{x' = X0-1 .. x} carry[x']  (above the band, own columns)
//     + sum_{x' = X0-1 .. x} rel_r[x']  (band rows so far, own columns)
// P and the carries of the lanes before this one form one 64-bit base per
// lane.  L[r] covers x < X0 - 1 and the band rows 0 .. r: int32 for f (at
// most 255 x 16383 x 64 < 2^31), int64 for f^2.  The band rows of the lanes
// before this one take a 32-bit scan (at most 31 x 8 x 64 x 255^2 < 2^31).
// Each of the lane's own columns (carry plus band rows, at most 255^2 N <
// 2^31) is then added to a 64-bit running sum that starts at the base plus
// those two.
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

// The lane's eight sources x = X0 + 8l - 1 + e as the bytes e of one packed
// pair: the previous lane's last byte (lane 0: the edge) and its own first
// seven.
__device__ __forceinline__ uint2 unpack_lane_row(const LaneRow& r, int lane) {
    const uint32_t prev = __shfl_up_sync(0xffffffffu, r.w.y, 1);
    const uint32_t first = (lane > 0) ? (prev >> 24) : (uint32_t)r.edge;
    return make_uint2((r.w.x << 8) | first, __funnelshift_l(r.w.x, r.w.y, 8));
}

constexpr int kAhead = 2;  // source rows in flight per warp
constexpr int kLaneStride = 80;  // staging bytes per lane: up to 64 data + 16 pad (conflict-free quarter-warps)
constexpr int kStageBytes = 32 * kLaneStride;
constexpr int kWarpSmem = kStageBytes + kMaxR * (4 + 8);  // staging, then the left sums L1[R] (int32), L2[R] (int64)
static_assert(kStageBytes % 16 == 0 && kWarpSmem % 16 == 0, "per-warp shared memory keeps 16-byte alignment");

// The warp stores the 256 values (as T) its lanes wrote into the staging
// buffer (lane l's eight at lane l * kLaneStride) to dst with 16-byte
// lane-consecutive stores (512 bytes each).
template <typename T>
__device__ __forceinline__ void stage_flush(const unsigned char* stage, int lane, T* dst) {
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
__global__ void __launch_bounds__(kEmitWarps * 32, kEmitMinCtas) sat_band_emit(const uint8_t* __restrict__ f, int M, int N,
                                                                 int stride, int R, int nb, int nc, int nk, int nj,
                                                                 int cp, int pitch, const int32_t* __restrict__ ca1,
                                                                 const int32_t* __restrict__ ca2,
                                                                 const int32_t* __restrict__ rs1,
                                                                 const int32_t* __restrict__ rs2,
                                                                 const int64_t* __restrict__ ch1,
                                                                 const int64_t* __restrict__ ch2, ST* __restrict__ s,
                                                                 int64_t* __restrict__ s2) {
    extern __shared__ __align__(16) unsigned char emit_smem[];
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the carries are complete
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pair = blockIdx.x * kEmitWarps + warp;
    if (pair >= nb * nc) return;  // whole warp
    const int b = pair / nc, c = pair % nc;
    unsigned char* stage = emit_smem + (size_t)warp * kWarpSmem;
    int32_t* L1 = reinterpret_cast<int32_t*>(stage + kStageBytes);
    int64_t* L2 = reinterpret_cast<int64_t*>(stage + kStageBytes + kMaxR * 4);
    const int y0 = b * R, nr = min(R, N - y0);
    const int X0 = c * kTileCols, Xl = X0 + kLaneCols * lane;
    const int32_t* cab1 = ca1 + (size_t)b * cp;  // column sums above this band
    const int32_t* cab2 = ca2 + (size_t)b * cp;
    const bool vec = ((stride & 7) == 0) && ((reinterpret_cast<uintptr_t>(f) & 7) == 0);
    const uint8_t* fband = f + (size_t)y0 * stride;

    // ---- prologue: the corner P and the left sums L[r] ----
    int64_t p1 = 0, p2 = 0;
    for (int j = lane; j < c * (kTileCols / kCarryChunk); j += 32) {
        p1 += ch1[(size_t)b * nj + j];
        p2 += ch2[(size_t)b * nj + j];
    }
    p1 = warp_sum(p1);
    p2 = warp_sum(p2);
    if (c > 0) {  // the chunks cover x < X0; the corner stops at X0 - 1
        p1 -= cab1[X0 - 1];
        p2 -= cab2[X0 - 1];
    }
    // lane l owns band rows l and l + 32: its row's chunk sums left of X0
    // less the edge pixel x = X0 - 1, then an inclusive scan over the rows
    int32_t cum1 = 0;  // running totals of the rows before this half
    int64_t cum2 = 0;
    for (int h = 0; h * 32 < nr; ++h) {
        const int r = h * 32 + lane;
        int32_t l1 = 0, l2 = 0;
        if (r < nr) {
            const int32_t* q1 = rs1 + (size_t)(y0 + r) * nk;
            const int32_t* q2 = rs2 + (size_t)(y0 + r) * nk;
#pragma unroll 4
            for (int k = 0; k < c; ++k) {
                l1 += q1[k];
                l2 += q2[k];
            }
            if (c > 0) {
                const int e = fband[(size_t)r * stride + X0 - 1];
                l1 -= e;
                l2 -= e * e;
            }
        }
        const int32_t i1 = cum1 + l1 + warp_exclusive_scan(l1, lane);
        const int64_t i2 = cum2 + (int64_t)l2 + warp_exclusive_scan((int64_t)l2, lane);
        if (r < nr) {
            L1[r] = i1;
            L2[r] = i2;
        }
        cum1 = __shfl_sync(0xffffffffu, i1, 31);
        cum2 = __shfl_sync(0xffffffffu, i2, 31);
    }
    // the lane's columns: col[e] = carry above the band plus the band's rows
    // so far (fits 32 bits: at most 65025 N < 2^31); the 64-bit base is the
    // corner plus the carries of the lanes before this one
    int32_t col1[kLaneCols], col2[kLaneCols];
    int64_t tc1 = 0, tc2 = 0;  // the lane's carry totals (8 x 255^2 N may pass 2^32)
#pragma unroll
    for (int e = 0; e < kLaneCols; ++e) {
        const int x = Xl - 1 + e;
        const bool in = (x >= 0 && x < M);
        col1[e] = in ? cab1[x] : 0;
        col2[e] = in ? cab2[x] : 0;
        tc1 += col1[e];
        tc2 += col2[e];
    }
    const int64_t base1 = p1 + warp_exclusive_scan(tc1, lane);
    const int64_t base2 = p2 + warp_exclusive_scan(tc2, lane);
    __syncwarp();

    if (b == 0) {  // row Y = 0 of the table is zero
        for (int X = X0 + lane; X < min(X0 + kTileCols, M + 1); X += 32) {
            s[X] = 0;
            s2[X] = 0;
        }
    }

    // ---- the band's rows ----
    const bool full_tile = (X0 + kTileCols - 1 <= M);  // warp-uniform
    unsigned char* mine = stage + lane * kLaneStride;
    // one row's outputs: running sums from the base plus the row part before
    // the lane, one column at a time (64-bit, or for a 32-bit s its low 32
    // bits, which is all the table keeps)
    using RunT = typename std::conditional<sizeof(ST) == 8, int64_t, uint32_t>::type;
    auto emit_row = [&](int r, int32_t pre1, int64_t pre2) {
        ST* srow = s + (size_t)(y0 + r + 1) * pitch;
        int64_t* s2row = s2 + (size_t)(y0 + r + 1) * pitch;
        RunT run1 = (RunT)(base1 + pre1);
        int64_t run2 = base2 + pre2;
        if (full_tile) {
            // through the warp's staging buffer, so that every global store
            // instruction writes 512 contiguous bytes
            if constexpr (sizeof(ST) == 8) {
#pragma unroll
                for (int e = 0; e < kLaneCols; e += 2) {
                    const int64_t o0 = (run1 += (RunT)col1[e]);
                    const int64_t o1 = (run1 += (RunT)col1[e + 1]);
                    *reinterpret_cast<longlong2*>(mine + 8 * e) = make_longlong2(o0, o1);
                }
            } else {
#pragma unroll
                for (int e = 0; e < kLaneCols; e += 4) {
                    int4 o;
                    o.x = (int)(run1 += (RunT)col1[e]);
                    o.y = (int)(run1 += (RunT)col1[e + 1]);
                    o.z = (int)(run1 += (RunT)col1[e + 2]);
                    o.w = (int)(run1 += (RunT)col1[e + 3]);
                    *reinterpret_cast<int4*>(mine + 4 * e) = o;
                }
            }
            stage_flush<ST>(stage, lane, srow + X0);
#pragma unroll
            for (int e = 0; e < kLaneCols; e += 2) {
                const int64_t o0 = (run2 += col2[e]);
                const int64_t o1 = (run2 += col2[e + 1]);
                *reinterpret_cast<longlong2*>(mine + 8 * e) = make_longlong2(o0, o1);
            }
            stage_flush<int64_t>(stage, lane, s2row + X0);
        } else {
#pragma unroll
            for (int e = 0; e < kLaneCols; ++e) {
                run1 += (RunT)col1[e];
                run2 += col2[e];
                if (Xl + e <= M) {
                    srow[Xl + e] = (ST)run1;
                    s2row[Xl + e] = run2;
                }
            }
        }
    };
    LaneRow q[kAhead];
#pragma unroll
    for (int i = 0; i < kAhead; ++i)
        if (i < nr) q[i] = load_lane_row(fband + (size_t)i * stride, M, X0, lane, vec);
    // the band's rows so far summed over the lane's columns, for the scans
    // (at most 8 x 64 x 255^2 < 2^31)
    uint32_t d1 = 0, d2 = 0;
    for (int r = 0; r < nr; ++r) {
        const uint2 va = unpack_lane_row(q[0], lane);
#pragma unroll
        for (int i = 0; i < kAhead - 1; ++i) q[i] = q[i + 1];
        if (r + kAhead < nr) q[kAhead - 1] = load_lane_row(fband + (size_t)(r + kAhead) * stride, M, X0, lane, vec);
#pragma unroll
        for (int e = 0; e < kLaneCols; ++e) {
            const int pa = byte_of(va, e);
            col1[e] += pa;
            col2[e] += pa * pa;
        }
        d1 = __dp4a(va.y, 0x01010101u, __dp4a(va.x, 0x01010101u, d1));
        d2 = __dp4a(va.y, va.y, __dp4a(va.x, va.x, d2));
        emit_row(r, L1[r] + (int32_t)warp_exclusive_scan(d1, lane), L2[r] + (int64_t)warp_exclusive_scan(d2, lane));
    }
}

// Emit warps resident on the whole current device at once (0 if unknown),
// cached per device: both table widths' kernels, the smaller.
long long emit_slots() {
    static std::atomic<long long> cached[kDeviceSlots];  // 0 = not yet queried
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 0;
    if (dev < kDeviceSlots) {
        const long long c = cached[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    const size_t smem = (size_t)kEmitWarps * kWarpSmem;
    int n32 = 0, n64 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n32, sat_band_emit<int32_t>, kEmitWarps * 32, smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n64, sat_band_emit<int64_t>, kEmitWarps * 32, smem) !=
            cudaSuccess)
        return 0;
    const long long n = (long long)std::min(n32, n64) * kEmitWarps * sm_count();
    if (n <= 0) return 0;
    if (dev < kDeviceSlots) cached[dev].store(n, std::memory_order_relaxed);
    return n;
}

cudaError_t set_emit_attributes() {
    static std::atomic<int> done[kDeviceSlots];
    return once_per_device(done, [] {
        const int smem = kEmitWarps * kWarpSmem;
        cudaError_t err = cudaFuncSetAttribute(sat_band_emit<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(sat_band_emit<int64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        return err;
    });
}

}  // namespace
}  // namespace sncc

extern "C" size_t sncc_integral_workspace_bytes(int M, int N) {
    if (M <= 0 || N <= 0) return 0;
    const sncc::SatGeometry g = sncc::sat_geometry(M, N);
    return sncc::sat_workspace(M, N, g).total;
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
    // A 32-bit s holds the sums modulo 2^32 (exact while 255*M*N < 2^31); the
    // column sums of f^2 kept in int32 need N*65025 < 2^31.
    if ((int64_t)N * 65025 >= ((int64_t)1 << 31)) return SNCC_ERR_UNSUPPORTED;
    if (!d_ws || ws_bytes < sncc_integral_workspace_bytes(M, N) || (reinterpret_cast<uintptr_t>(d_ws) & 15))
        return SNCC_ERR_WORKSPACE;
    const SatWorkspace w = sat_workspace(M, N, sat_geometry(M, N));
    const SatGeometry g = sat_launch_geometry(M, N, emit_slots());
    char* ws = static_cast<char*>(d_ws);
    int32_t* cs1 = reinterpret_cast<int32_t*>(ws + w.cs1);
    int32_t* cs2 = reinterpret_cast<int32_t*>(ws + w.cs2);
    int32_t* rs1 = reinterpret_cast<int32_t*>(ws + w.rs1);
    int32_t* rs2 = reinterpret_cast<int32_t*>(ws + w.rs2);
    int64_t* ch1 = reinterpret_cast<int64_t*>(ws + w.ch1);
    int64_t* ch2 = reinterpret_cast<int64_t*>(ws + w.ch2);
    cudaStream_t st = (cudaStream_t)stream;
    const dim3 g1((M + kColThreads * kLaneCols - 1) / (kColThreads * kLaneCols), g.nb);
    const int cp = col_pitch(M);
    sat_band_colsum<<<g1, kColThreads, 0, st>>>(d_f, M, N, f_stride, g.R, g.nk, cp, cs1, cs2, rs1, rs2);
    // the scan and the emit launch while their predecessor drains and wait
    // for it in the kernel (programmatic dependent launch)
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t c2 = {};
    c2.gridDim = dim3((M + kCarryChunk - 1) / kCarryChunk);
    c2.blockDim = dim3(kScanWarps * 32);
    c2.stream = st;
    c2.attrs = pdl;
    c2.numAttrs = 1;
    if (cudaLaunchKernelEx(&c2, sat_band_scan, M, g.nb, g.nj, cp, cs1, cs2, ch1, ch2) != cudaSuccess)
        return SNCC_ERR_CUDA;
    if (set_emit_attributes() != cudaSuccess) return SNCC_ERR_CUDA;
    cudaLaunchConfig_t c3 = c2;
    c3.gridDim = dim3((g.nb * g.nc + kEmitWarps - 1) / kEmitWarps);
    c3.blockDim = dim3(kEmitWarps * 32);
    c3.dynamicSmemBytes = (size_t)kEmitWarps * kWarpSmem;
    const cudaError_t e3 =
        s_bits == 32
            ? cudaLaunchKernelEx(&c3, sat_band_emit<int32_t>, d_f, M, N, f_stride, g.R, g.nb, g.nc, g.nk, g.nj, cp,
                                 sat_pitch, (const int32_t*)cs1, (const int32_t*)cs2, (const int32_t*)rs1,
                                 (const int32_t*)rs2, (const int64_t*)ch1, (const int64_t*)ch2,
                                 static_cast<int32_t*>(d_s), d_s2)
            : cudaLaunchKernelEx(&c3, sat_band_emit<int64_t>, d_f, M, N, f_stride, g.R, g.nb, g.nc, g.nk, g.nj, cp,
                                 sat_pitch, (const int32_t*)cs1, (const int32_t*)cs2, (const int32_t*)rs1,
                                 (const int32_t*)rs2, (const int64_t*)ch1, (const int64_t*)ch2,
                                 static_cast<int64_t*>(d_s), d_s2);
    return e3 == cudaSuccess && cudaGetLastError() == cudaSuccess ? SNCC_OK : SNCC_ERR_CUDA;
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
