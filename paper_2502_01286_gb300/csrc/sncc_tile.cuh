// sncc_tile.cuh - device building blocks shared by the single-problem and
// the batched segment-sum kernels (and the exact comparator's window sums):
// register staging of a re-based sum-table region, the corner sum, and the
// normalisation of Eq. 13 - Eq. 18.
#pragma once

#include <cstdint>

#include "sncc_internal.h"

namespace sncc {

// Reads a sum-table entry (int32 or int64 table) as a 64-bit integer.
template <bool S64>
__device__ __forceinline__ long long table_entry(const void* s, int pitch, int X, int Y) {
    if constexpr (S64)
        return static_cast<const long long*>(s)[(size_t)Y * pitch + X];
    else
        return static_cast<const int*>(s)[(size_t)Y * pitch + X];
}

// Sum of f over the W x H window at (u, v) from four table entries.  A
// 32-bit table may hold its entries modulo 2^32; the window sum (at most
// 255 W H < 2^31 for W H <= 2^23) is then exact as a wrapped 32-bit
// difference.
template <bool S64>
__device__ __forceinline__ long long window_sum(const void* s, int pitch, int u, int v, int W, int H) {
    if constexpr (S64) {
        const long long* t = static_cast<const long long*>(s);
        return t[(size_t)(v + H) * pitch + u + W] - t[(size_t)(v + H) * pitch + u] - t[(size_t)v * pitch + u + W] +
               t[(size_t)v * pitch + u];
    } else {
        const uint32_t* t = static_cast<const uint32_t*>(s);
        return (long long)(int32_t)(t[(size_t)(v + H) * pitch + u + W] - t[(size_t)(v + H) * pitch + u] -
                                    t[(size_t)v * pitch + u + W] + t[(size_t)v * pitch + u]);
    }
}

// Low 32 bits of entry (X, Y) of an int32 or int64 table (little endian).
template <bool S64>
__device__ __forceinline__ uint32_t table_low(const void* s, int pitch, int X, int Y) {
    const uint32_t* w = static_cast<const uint32_t*>(s);
    return S64 ? __ldg(w + 2 * ((size_t)Y * pitch + X)) : __ldg(w + (size_t)Y * pitch + X);
}

// Stages the region of a (M+1) x (N+1) sum table with origin (x0, y0) into
// buf (RH rows x WP words), re-based to the origin in wrapped 32-bit
// arithmetic: buf[Y][X] = s(x0+X, y0+Y) - s(x0+X, y0) - s(x0, y0+Y) + s(x0, y0)
// (mod 2^32), which is the box sum over the region and exact below 2^31.
// At least the first `cols` (<= WP) columns are written; warp w owns rows w,
// w + WARPS, ...
//
// Regions inside the table take the fast path: lane l loads entries
// x0 + 2j and x0 + 2j + 1 (j = l, l + 32, ...) with one 16-byte (int64
// table) or 8-byte (int32 table) load and stores their low words with one
// 8-byte store; the origin column comes from lane 0 by shuffle.  This needs
// x0 even, an even table pitch and a 16-byte aligned table, which the callers
// guarantee (x0 is a multiple of 32 plus a multiple of the block width 64,
// the pitch a multiple of 32).  Regions that cross the table's edge take the
// checked path, where entries past the table, which only offsets outside the
// map read, load as 0.
template <bool S64, int WP>
__device__ __forceinline__ void stage_region_checked(const void* s, int pitch, int M, int N, int* buf, int x0,
                                                     int y0, int RH, int lane, int warp, int cols) {
    constexpr int KX = (WP + 31) / 32;
    auto at = [&](int gx, int gy) -> uint32_t {
        return (gx <= M && gy <= N) ? table_low<S64>(s, pitch, gx, gy) : 0u;
    };
    const uint32_t c00 = at(x0, y0);
    uint32_t r0[KX];
#pragma unroll
    for (int k = 0; k < KX; ++k) r0[k] = at(x0 + lane + 32 * k, y0) - c00;
    for (int Y = warp; Y < RH; Y += WARPS) {
        const int gy = y0 + Y;
        const uint32_t cy = at(x0, gy);
        uint32_t v[KX];
#pragma unroll
        for (int k = 0; k < KX; ++k) v[k] = (lane + 32 * k < cols) ? at(x0 + lane + 32 * k, gy) : 0u;
#pragma unroll
        for (int k = 0; k < KX; ++k)
            if (lane + 32 * k < cols) buf[Y * WP + lane + 32 * k] = (int)(v[k] - r0[k] - cy);
    }
}

// Low words of table entries x0 + 2j and x0 + 2j + 1 of the row at `rowp`.
template <bool S64>
__device__ __forceinline__ uint2 load_pair(const char* rowp, int j) {
    if constexpr (S64) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(rowp) + j);
        return make_uint2(q.x, q.z);
    } else {
        return __ldg(reinterpret_cast<const uint2*>(rowp) + j);
    }
}

template <bool S64, int WP>
__device__ __forceinline__ void stage_region_regs(const void* s, int pitch, int M, int N, int* buf, int x0, int y0,
                                                  int RH, int lane, int warp, int cols = WP) {
    constexpr int KP = (WP / 2 + 31) / 32;  // column pairs per lane
    const int npairs = (cols + 1) >> 1;
    if (x0 + 2 * npairs - 1 > M || y0 + RH - 1 > N) {
        stage_region_checked<S64, WP>(s, pitch, M, N, buf, x0, y0, RH, lane, warp, cols);
        return;
    }
    constexpr size_t esz = S64 ? 8 : 4;
    const char* base = static_cast<const char*>(s) + ((size_t)y0 * pitch + x0) * esz;
    const size_t rstride = (size_t)pitch * esz;
    uint2 r0[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        const int j = lane + 32 * k;
        r0[k] = (j < npairs) ? load_pair<S64>(base, j) : make_uint2(0u, 0u);
    }
    const uint32_t c00 = __shfl_sync(0xffffffffu, r0[0].x, 0);
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        r0[k].x -= c00;
        r0[k].y -= c00;
    }
    for (int Y = warp; Y < RH; Y += WARPS) {
        const char* rowp = base + (size_t)Y * rstride;
        uint2 v[KP];
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const int j = lane + 32 * k;
            v[k] = (j < npairs) ? load_pair<S64>(rowp, j) : make_uint2(0u, 0u);
        }
        const uint32_t cy = __shfl_sync(0xffffffffu, v[0].x, 0);
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const int j = lane + 32 * k;
            if (j < npairs) {
                const uint2 o = make_uint2(v[k].x - r0[k].x - cy, v[k].y - r0[k].y - cy);
                *reinterpret_cast<uint2*>(buf + Y * WP + 2 * j) = o;
            }
        }
    }
}

// off is the corner's byte offset in the region (a plain add to the lane's
// base address).
template <int R, int WP>
__device__ __forceinline__ void apply_corner(long long (&acc)[R], const int* wbase, int off, int g) {
    const int* w = reinterpret_cast<const int*>(reinterpret_cast<const char*>(wbase) + off);
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] += (long long)g * (long long)w[r * WP];
}

// acc[r] += sum over the block's corner records of G * region(row r + Y, col X).
// Records come two per 16-byte load, four per iteration; `count` is a
// multiple of 4 (zero-weight padding) and `cq` 16-byte aligned.  The loads
// are issued at the top of each iteration and the loop is unrolled twice,
// so that the next group's loads overlap this group's multiply-adds without
// register copies (other warps hide the rest of their latency).
template <int R, int WP>
__device__ __forceinline__ void corner_sum(long long (&acc)[R], const int* wbase, const int4* cq, int count) {
    const int groups = count >> 2;
#pragma unroll 2
    for (int g = 0; g < groups; ++g) {
        const int4 c0 = __ldg(cq + 2 * g), c1 = __ldg(cq + 2 * g + 1);
        apply_corner<R, WP>(acc, wbase, c0.x, c0.y);
        apply_corner<R, WP>(acc, wbase, c0.z, c0.w);
        apply_corner<R, WP>(acc, wbase, c1.x, c1.y);
        apply_corner<R, WP>(acc, wbase, c1.z, c1.w);
    }
}

// A vertical run of L corners at rows Y, Y+T, .., Y+(L-1)T of column X
// (stride T = 1 or 2, idx = 4 (Y*WP + X)) with weights g[0..L-1]: offset
// row r needs the region words of rows Y+r+lT, so the R rows of a lane share
// R + (L-1)T loads, and each load feeds up to L multiply-adds instead of one.
template <int R, int WP, int L, int T = 1>
__device__ __forceinline__ void apply_run(long long (&acc)[R], const int* wbase, int idx, const int (&g)[L]) {
    const int* w = reinterpret_cast<const int*>(reinterpret_cast<const char*>(wbase) + idx);  // idx in bytes
    int v[R + (L - 1) * T];
#pragma unroll
    for (int i = 0; i < R + (L - 1) * T; ++i) v[i] = w[i * WP];
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] += (long long)g[l] * (long long)v[r + l * T];
}

// Corners at rows Y, Y+2 and Y+3 of one column (weights g0, g1, g2): R + 3
// shared loads for the three.
template <int R, int WP>
__device__ __forceinline__ void apply_t21(long long (&acc)[R], const int* wbase, int idx, int g0, int g1, int g2) {
    const int* w = reinterpret_cast<const int*>(reinterpret_cast<const char*>(wbase) + idx);  // idx in bytes
    int v[R + 3];
#pragma unroll
    for (int i = 0; i < R + 3; ++i) v[i] = w[i * WP];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] += (long long)g0 * (long long)v[r];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] += (long long)g1 * (long long)v[r + 2];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] += (long long)g2 * (long long)v[r + 3];
}

// All records {idx, g0, g1, g2} of the rows-(0, 2, 3) pattern of one block.
template <int R, int WP>
__device__ __forceinline__ void t21_class(long long (&acc)[R], const int* wbase, const int4* rec, int n) {
#pragma unroll 2
    for (int i = 0; i < n; ++i) {
        const int4 q = __ldg(rec + i);
        apply_t21<R, WP>(acc, wbase, q.x, q.y, q.z, q.w);
    }
}

// All runs of length L (stride T) of one block: `n` records of S int4 units
// each ({idx, G0, ...}), loaded at the top of each iteration (unrolled twice).
template <int R, int WP, int L, int S, int T = 1>
__device__ __forceinline__ void run_class(long long (&acc)[R], const int* wbase, const int4* rec, int n) {
#pragma unroll 2
    for (int i = 0; i < n; ++i) {
        int wd[4 * S];
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const int4 q = __ldg(rec + (size_t)i * S + k);
            wd[4 * k + 0] = q.x;
            wd[4 * k + 1] = q.y;
            wd[4 * k + 2] = q.z;
            wd[4 * k + 3] = q.w;
        }
        int g[L];
#pragma unroll
        for (int l = 0; l < L; ++l) g[l] = wd[1 + l];
        apply_run<R, WP, L, T>(acc, wbase, wd[0], g);
    }
}

// Two corners of one column D rows apart, weights g0 (row Y) and g1 (row
// Y + D): the lane's R rows share R + D region loads.
template <int R, int WP, int D>
__device__ __forceinline__ void apply_pair(long long (&acc)[R], const int* wbase, int idx, int g0, int g1) {
    const int* w = reinterpret_cast<const int*>(reinterpret_cast<const char*>(wbase) + idx);  // idx in bytes
    int v[R + D];
#pragma unroll
    for (int i = 0; i < R + D; ++i) v[i] = (i < R || i >= D) ? w[i * WP] : 0;
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] += (long long)g0 * (long long)v[r];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] += (long long)g1 * (long long)v[r + D];
}

// All pairs of gap D of one block: `n` records {idx, g0, g1, 0}.
template <int R, int WP, int D>
__device__ __forceinline__ void pair_class(long long (&acc)[R], const int* wbase, const int4* rec, int n) {
#pragma unroll 2
    for (int i = 0; i < n; ++i) {
        const int4 q = __ldg(rec + i);
        apply_pair<R, WP, D>(acc, wbase, q.x, q.y, q.z);
    }
}

// acc[r] += the block's corner sum, from its records: desc[0] = {first8,
// n8, first4, n4}, desc[1] = {first2, n2, first1, n1}, desc[2..4] = {first,
// n} of the pairs of gap 2 .. 7, desc[5] = {first, n} of the stride-2 runs
// of 8 and 4, desc[6] = {first, n} of the stride-2 runs of 3 and of the
// rows-(0, 2, 3) pattern (first* in int4 units of `runs`, n1 single corners
// in groups of four).
template <int R, int WP>
__device__ __forceinline__ void run_sum(long long (&acc)[R], const int* wbase, const int4* runs, const int4* desc) {
    static_assert(PAIR_MIN_GAP == 2 && PAIR_MAX_GAP == 7 && RUNBLK_INT4 == 7, "descriptor layout");
    const int4 d0 = __ldg(desc), d1 = __ldg(desc + 1), d2 = __ldg(desc + 2), d3 = __ldg(desc + 3),
               d4 = __ldg(desc + 4), d5 = __ldg(desc + 5), d6 = __ldg(desc + 6);
    run_class<R, WP, 8, 3>(acc, wbase, runs + d0.x, d0.y);
    run_class<R, WP, 4, 2>(acc, wbase, runs + d0.z, d0.w);
    run_class<R, WP, 2, 1>(acc, wbase, runs + d1.x, d1.y);
    run_class<R, WP, 8, 3, 2>(acc, wbase, runs + d5.x, d5.y);
    run_class<R, WP, 4, 2, 2>(acc, wbase, runs + d5.z, d5.w);
    run_class<R, WP, 3, 1, 2>(acc, wbase, runs + d6.x, d6.y);
    t21_class<R, WP>(acc, wbase, runs + d6.z, d6.w);
    pair_class<R, WP, 2>(acc, wbase, runs + d2.x, d2.y);
    pair_class<R, WP, 3>(acc, wbase, runs + d2.z, d2.w);
    pair_class<R, WP, 4>(acc, wbase, runs + d3.x, d3.y);
    pair_class<R, WP, 5>(acc, wbase, runs + d3.z, d3.w);
    pair_class<R, WP, 6>(acc, wbase, runs + d4.x, d4.y);
    pair_class<R, WP, 7>(acc, wbase, runs + d4.z, d4.w);
    corner_sum<R, WP>(acc, wbase, runs + d1.z, d1.w);
}

// rho at offset (u, v) from the exact numerator acc = 2^F num + Q0 * sum f / n
// (Eq. 13, 15, 16 exact in integers; E_f = var / n in FP64 as var times the
// FP64 reciprocal of n, within one FP64 ulp of the quotient; Eq. 17-18 in
// FP32).
// A uniform window gives 0.
template <bool S64>
__device__ __forceinline__ float normalise(long long acc, const void* s, const int64_t* s2, int pitch, int u, int v,
                                           int W, int H, long long n, double rn, float inv_n, float Ek,
                                           float scale, long long Q0) {
    const long long sf = window_sum<S64>(s, pitch, u, v, W, H);
    const long long sf2 = s2[(size_t)(v + H) * pitch + u + W] - s2[(size_t)(v + H) * pitch + u] -
                          s2[(size_t)v * pitch + u + W] + s2[(size_t)v * pitch + u];
    const long long var = n * sf2 - sf * sf;
    if (var <= 0) return 0.0f;
    const double ef = (double)var * rn;  // rn = 1/n rounded once in FP64
    const float den = sqrtf((float)ef * Ek);
    const float num = ((float)acc - (float)(Q0 * sf) * inv_n) * scale;
    return num / den;
}

}  // namespace sncc
