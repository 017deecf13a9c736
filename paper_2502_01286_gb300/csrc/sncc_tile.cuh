// sncc_tile.cuh - device building blocks shared by the single-problem and
// the batched segment-sum kernels: register staging of a re-based sum-table
// region, the corner sum, and the normalisation of Eq. 13 - Eq. 18.
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
// Lane l owns columns l, l+32, ...; warp w owns rows w, w+WARPS, ...; only
// columns below `cols` (<= WP) are written.
// Entries past the table, which only offsets outside the map read, load as 0.
template <bool S64, int WP>
__device__ __forceinline__ void stage_region_regs(const void* s, int pitch, int M, int N, int* buf, int x0, int y0,
                                                  int RH, int lane, int warp, int cols = WP) {
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

template <int R, int WP>
__device__ __forceinline__ void apply_corner(long long (&acc)[R], const int* wbase, int off, int g) {
    const int* w = wbase + off;
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] += (long long)g * (long long)w[r * WP];
}

// acc[r] += sum over the block's corner records of G * region(row r + Y, col X).
// Records come two per 16-byte load, one group of four ahead of their use;
// `count` is a multiple of 4 (zero-weight padding) and `cq` 16-byte aligned.
template <int R, int WP>
__device__ __forceinline__ void corner_sum(long long (&acc)[R], const int* wbase, const int4* cq, int count) {
    const int groups = count >> 2;
    if (groups <= 0) return;
    int4 n0 = __ldg(cq), n1 = __ldg(cq + 1);
    for (int g = 0; g < groups; ++g) {
        const int4 c0 = n0, c1 = n1;
        if (g + 1 < groups) {
            n0 = __ldg(cq + 2 * g + 2);
            n1 = __ldg(cq + 2 * g + 3);
        }
        apply_corner<R, WP>(acc, wbase, c0.x, c0.y);
        apply_corner<R, WP>(acc, wbase, c0.z, c0.w);
        apply_corner<R, WP>(acc, wbase, c1.x, c1.y);
        apply_corner<R, WP>(acc, wbase, c1.z, c1.w);
    }
}

// rho at offset (u, v) from the exact numerator acc = 2^F num + Q0 * sum f / n
// (Eq. 13, 15, 16 exact in integers; E_f divided in FP64; Eq. 17-18 in FP32).
// A uniform window gives 0.
template <bool S64>
__device__ __forceinline__ float normalise(long long acc, const void* s, const int64_t* s2, int pitch, int u, int v,
                                           int W, int H, long long n, float inv_n, float Ek, float scale,
                                           long long Q0) {
    const long long sf = table_entry<S64>(s, pitch, u + W, v + H) - table_entry<S64>(s, pitch, u, v + H) -
                         table_entry<S64>(s, pitch, u + W, v) + table_entry<S64>(s, pitch, u, v);
    const long long sf2 = s2[(size_t)(v + H) * pitch + u + W] - s2[(size_t)(v + H) * pitch + u] -
                          s2[(size_t)v * pitch + u + W] + s2[(size_t)v * pitch + u];
    const long long var = n * sf2 - sf * sf;
    if (var <= 0) return 0.0f;
    const double ef = (double)var / (double)n;
    const float den = sqrtf((float)ef * Ek);
    const float num = ((float)acc - (float)(Q0 * sf) * inv_n) * scale;
    return num / den;
}

}  // namespace sncc
