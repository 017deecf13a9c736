// sncc_diff.cu - the segmented-NCC loss L = sum_o (rho_k(o) - rho_t(o))^2 on a
// float source with a fixed segmentation, and its hand-written gradients with
// respect to the segment values k_i and the source image f.
//
// rho_k is segmented NCC (Eq. 9, Eq. 17, Eq. 18 with the weighted energy) of
// the approximation with values k_i; rho_t is exact NCC (Eq. 1).  With
// c_i = k_i - kbar (kbar of Eq. 7), g = 2 (rho_k - rho_t),
// a = g / sqrt(E_f E_k), b = g / sqrt(E_f E_t), h = g (rho_k - rho_t) / E_f:
//   dL/dk_j  = sum_{x in S_j} Gt(x) - n_j sum_o a fbar - n_j c_j sum_o g rho_k / E_k,
//              Gt(x) = sum_o a(o) f(o + x);
//   dL/df(p) = sum_{o : p in window(o)} a(o) c(p-o) - b(o) t0(p-o) + h(o) (fbar(o) - f(p)).
// Templates up to 256 x 256, taken in blocks of at most 64 x 64 (a block's
// window region and the block of the template fit in shared memory).  Sums
// run in FP32 along a template row (the forward pass: down a template column)
// and in compensated FP32 across rows (columns) and blocks.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "sncc.h"
#include "sncc_internal.h"

namespace sncc {
namespace {

constexpr int kDiffMax = 256;     // largest template edge
constexpr int kDiffBlk = 64;      // template block edge the forward and dL/df kernels stage at a time
constexpr int kFwXB = 4;          // forward: offset rows per thread (register window)
constexpr int kFwG = 2;           // forward: template-column groups per CTA
constexpr int kFwGT = 256 / kFwG;  // forward: threads per group (4 warps)
constexpr int kFwTX = 32;         // forward: offset columns per CTA (lane = column)
constexpr int kFwTY = (kFwGT / 32) * kFwXB;  // forward: offset rows per CTA (16)
constexpr int kGtChunks = 192;    // offset-row chunks of the Gt correlation
constexpr int kGtReduceLanes = 8;  // lanes summing the chunk partials of one Gt entry
constexpr int kGtYB = 16;         // template rows per Gt CTA
constexpr int kGtXB = 8;          // template columns per Gt thread (register window)
constexpr int kGtVS = 4;          // offset rows staged at a time
constexpr int kGtUS = 256;        // offset columns staged at a time
constexpr int kGtFW = kGtUS + 64;  // staged source row pitch: kGtUS + 8 * kGtXB - 1 columns used

// Workspace layout (bytes), 256-aligned sections.
struct DiffLayout {
    size_t scal, c, t0, ef, fbar, a, b, h, hf, rh, rhf, gtp, gt, total;
};

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

DiffLayout diff_layout(int M, int N, int W, int H) {
    const size_t U = (size_t)(M - W + 1), V = (size_t)(N - H + 1), T = (size_t)W * H, UV = U * V;
    (void)N;
    DiffLayout L;
    size_t o = 0;
    L.scal = o; o = al256(o + 8 * sizeof(double));
    L.c = o; o = al256(o + T * 4);
    L.t0 = o; o = al256(o + T * 4);
    L.ef = o; o = al256(o + UV * 4);
    L.fbar = o; o = al256(o + UV * 4);
    L.a = o; o = al256(o + UV * 4);
    L.b = o; o = al256(o + UV * 4);
    L.h = o; o = al256(o + UV * 4);
    L.hf = o; o = al256(o + UV * 4);
    L.rh = o; o = al256(o + V * (size_t)M * 4);
    L.rhf = o; o = al256(o + V * (size_t)M * 4);
    L.gtp = o; o = al256(o + (size_t)kGtChunks * T * sizeof(double));
    L.gt = o; o = al256(o + T * sizeof(double));
    L.total = o;
    return L;
}

__device__ __forceinline__ double block_sum_double(double v, double* sm) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sm[w];
    __syncthreads();
    return r;  // valid in thread 0
}

// Compensated (Kahan) FP32 sum: value() = s - c carries about twice the
// FP32 precision, so column sums add up across columns without FP64 adds
// (GB300's FP64 pipe runs at a small fraction of its FP32 rate).
struct KahanF {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// scal[0] = kbar, scal[1] = E_k, scal[2] = E_t, scal[3] = sum a fbar, scal[4] = sum g rho_k.
// Renders c(x) = k_i - kbar and t0 = t - tbar.  One CTA.
__global__ void __launch_bounds__(256) diff_prep_kernel(const float* __restrict__ t, int W, int H,
                                                        const int4* __restrict__ rects, const float* __restrict__ k,
                                                        int K, double* scal, float* c, float* t0) {
    __shared__ double sm[8];
    __shared__ double sh_kbar, sh_tbar;
    const double n = (double)W * H;
    double sk = 0.0, st = 0.0;
    for (int i = threadIdx.x; i < K; i += blockDim.x) sk += (double)rects[i].z * rects[i].w * (double)k[i];
    for (int i = threadIdx.x; i < W * H; i += blockDim.x) st += (double)t[i];
    sk = block_sum_double(sk, sm);
    st = block_sum_double(st, sm);
    if (threadIdx.x == 0) {
        sh_kbar = sk / n;
        sh_tbar = st / n;
    }
    __syncthreads();
    const double kbar = sh_kbar, tbar = sh_tbar;
    double ek = 0.0, et = 0.0;
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        const int4 r = rects[i];
        const double ci = (double)k[i] - kbar;
        ek += (double)r.z * r.w * ci * ci;
        // rectangles are clamped to the template, so a bad record cannot write outside c
        for (int y = max(r.y, 0); y < min(r.y + r.w, H); ++y)
            for (int x = max(r.x, 0); x < min(r.x + r.z, W); ++x) c[y * W + x] = (float)ci;
    }
    for (int i = threadIdx.x; i < W * H; i += blockDim.x) {
        const double d = (double)t[i] - tbar;
        t0[i] = (float)d;
        et += d * d;
    }
    ek = block_sum_double(ek, sm);
    et = block_sum_double(et, sm);
    if (threadIdx.x == 0) {
        scal[0] = kbar;
        scal[1] = ek;
        scal[2] = et;
        scal[3] = 0.0;
        scal[4] = 0.0;
    }
}

// Forward pass over a 32 x 16 tile of offsets.  The CTA's 256 threads are
// kFwG groups of 4 warps; within each template block group g takes the
// block's columns [g Wb / kFwG, (g+1) Wb / kFwG), and thread (warp w of the
// group, lane l) the offsets u0 + l, rows v0 + 4w .. +3.  Along a template
// column the thread keeps the 4 source values of its 4 offsets in a register
// window, so each template row costs one new source load and two broadcast
// loads (c, t0) for 4 x 4 floating-point operations.  Sums run in FP32 down a
// template column and in compensated FP32 across columns and blocks (a plain
// FP64 add per column and offset made the kernel FP64-bound); the groups'
// partial sums meet in shared memory, in FP64 and a fixed order.
//   pass 1: window means (sliding column sums), over every block;
//   pass 2: with d = f - fbar: sum d^2, sum c d, sum t0 d (E_f, numerator,
//           exact numerator), over every block again (a template of one
//           block is staged once for both passes).
__host__ __device__ constexpr int fw_region_w(int W) { return kFwTX + W - 1; }
__host__ __device__ constexpr int blk_edge(int E) { return E < kDiffBlk ? E : kDiffBlk; }
__host__ __device__ constexpr size_t fw_main_bytes(int W, int H) {
    // max(staged source, c, t0 of the largest block | pass-2 partials of groups 1..), rounded to 16 bytes
    return (((size_t)fw_region_w(blk_edge(W)) * (kFwTY + blk_edge(H) - 1) + 2 * (size_t)blk_edge(W) * blk_edge(H)) *
                        4 >
                    (size_t)(kFwG - 1) * kFwGT * kFwXB * 3 * 8
                ? ((size_t)fw_region_w(blk_edge(W)) * (kFwTY + blk_edge(H) - 1) +
                   2 * (size_t)blk_edge(W) * blk_edge(H)) *
                      4
                : (size_t)(kFwG - 1) * kFwGT * kFwXB * 3 * 8) +
               15 &
           ~(size_t)15;
}
__host__ __device__ constexpr size_t fw_smem_bytes(int W, int H) {
    return fw_main_bytes(W, H) + (size_t)kFwG * kFwGT * kFwXB * 8;  // + pass-1 partials
}

__global__ void __launch_bounds__(256) diff_forward_kernel(const float* __restrict__ f, int M, int N, int stride,
                                                           int W, int H, const float* __restrict__ c,
                                                           const float* __restrict__ t0, const double* scal,
                                                           float* __restrict__ rho_k, float* __restrict__ rho_t,
                                                           float* __restrict__ ef_out, float* __restrict__ fbar_out,
                                                           double* loss) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int Wb = blk_edge(W), Hb = blk_edge(H);  // the largest block
    const int RW = fw_region_w(Wb);                // region pitch
    const size_t main_bytes = fw_main_bytes(W, H);
    float* fs = reinterpret_cast<float*>(smraw);        // source region of a block, pitch RW
    float* cs = fs + RW * (kFwTY + Hb - 1);             // c of a block, pitch bw
    float* ts = cs + Wb * Hb;                           // t0 of a block, pitch bw
    double* red2 = reinterpret_cast<double*>(smraw);    // after pass 2: [g-1][t][j][3]
    double* red1 = reinterpret_cast<double*>(smraw + main_bytes);  // [g][t][j]
    __shared__ double red[8];
    const int U = M - W + 1, V = N - H + 1;
    const int u0 = blockIdx.x * kFwTX, v0 = blockIdx.y * kFwTY;
    const bool one_block = (W <= kDiffBlk && H <= kDiffBlk);
    // the source region of block (bx, by) of size bw x bh, and its c and t0
    auto stage = [&](int bx, int by, int bw, int bh, bool tmpl) {
        const int rw = fw_region_w(bw), rh = kFwTY + bh - 1;
        for (int i = threadIdx.x; i < rw * rh; i += blockDim.x) {
            const int Y = i / rw, X = i - Y * rw;
            const int gx = u0 + bx + X, gy = v0 + by + Y;
            fs[Y * RW + X] = (gx < M && gy < N) ? f[(size_t)gy * stride + gx] : 0.0f;
        }
        if (tmpl)
            for (int i = threadIdx.x; i < bw * bh; i += blockDim.x) {
                const int y = i / bw, x = i - y * bw;
                cs[i] = c[(by + y) * W + bx + x];
                ts[i] = t0[(by + y) * W + bx + x];
            }
    };
    const int g = threadIdx.x / kFwGT, t = threadIdx.x - g * kFwGT;
    const int lane = t & 31, wy = t >> 5;
    const float* base = fs + (wy * kFwXB) * RW + lane;  // region row of offset row 0, column of the lane
    const double n = (double)W * H;

    // ---- pass 1: window sums, sum over rows y of f(row y + j) per template column ----
    KahanF sp[kFwXB];
    for (int by = 0; by < H; by += kDiffBlk) {
        for (int bx = 0; bx < W; bx += kDiffBlk) {
            const int bw = min(kDiffBlk, W - bx), bh = min(kDiffBlk, H - by);
            __syncthreads();  // the previous block's reads are done
            stage(bx, by, bw, bh, one_block);
            __syncthreads();
            const int x_lo = g * bw / kFwG, x_hi = (g + 1) * bw / kFwG;
            for (int x = x_lo; x < x_hi; ++x) {
                const float* col = base + x;
                float s0 = 0.0f;
                for (int y = 0; y < bh; ++y) s0 += col[y * RW];
                float sj = s0;
                sp[0].add(s0);
#pragma unroll
                for (int j = 1; j < kFwXB; ++j) {  // slide the window one row
                    sj += col[(bh - 1 + j) * RW] - col[(j - 1) * RW];
                    sp[j].add(sj);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kFwXB; ++j) red1[(g * kFwGT + t) * kFwXB + j] = sp[j].value();
    __syncthreads();
    float fb[kFwXB];
#pragma unroll
    for (int j = 0; j < kFwXB; ++j) {
        double sf = 0.0;
        for (int q = 0; q < kFwG; ++q) sf += red1[(q * kFwGT + t) * kFwXB + j];
        fb[j] = (float)(sf / n);
    }

    // ---- pass 2: energy, approximate and exact numerators ----
    KahanF ek[kFwXB], nkk[kFwXB], ntk[kFwXB];
    for (int by = 0; by < H; by += kDiffBlk) {
        for (int bx = 0; bx < W; bx += kDiffBlk) {
            const int bw = min(kDiffBlk, W - bx), bh = min(kDiffBlk, H - by);
            if (!one_block) {
                __syncthreads();
                stage(bx, by, bw, bh, true);
                __syncthreads();
            }
            const int x_lo = g * bw / kFwG, x_hi = (g + 1) * bw / kFwG;
            for (int x = x_lo; x < x_hi; ++x) {
                const float* col = base + x;
                float re[kFwXB], rk[kFwXB], rt[kFwXB], win[kFwXB];
#pragma unroll
                for (int j = 0; j < kFwXB; ++j) {
                    re[j] = rk[j] = rt[j] = 0.0f;
                    win[j] = j < kFwXB - 1 ? col[j * RW] : 0.0f;  // rows 0 .. 2 in slots 0 .. 2
                }
                for (int y0 = 0; y0 < bh; y0 += kFwXB) {
#pragma unroll
                    for (int k = 0; k < kFwXB; ++k) {
                        const int y = y0 + k;
                        if (y < bh) {
                            win[(k + kFwXB - 1) % kFwXB] = col[(y + kFwXB - 1) * RW];  // row y + 3
                            const float cx = cs[y * bw + x], tx = ts[y * bw + x];
#pragma unroll
                            for (int j = 0; j < kFwXB; ++j) {
                                const float d = win[(k + j) % kFwXB] - fb[j];  // f(row y + j)
                                re[j] += d * d;
                                rk[j] += cx * d;
                                rt[j] += tx * d;
                            }
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < kFwXB; ++j) {
                    ek[j].add(re[j]);
                    nkk[j].add(rk[j]);
                    ntk[j].add(rt[j]);
                }
            }
        }
    }
    double e[kFwXB], nk[kFwXB], nt[kFwXB];
#pragma unroll
    for (int j = 0; j < kFwXB; ++j) {
        e[j] = ek[j].value();
        nk[j] = nkk[j].value();
        nt[j] = ntk[j].value();
    }
    __syncthreads();  // the staged region is reused for the groups' partials
    if (g > 0) {
#pragma unroll
        for (int j = 0; j < kFwXB; ++j) {
            double* o = red2 + (((g - 1) * kFwGT + t) * kFwXB + j) * 3;
            o[0] = e[j];
            o[1] = nk[j];
            o[2] = nt[j];
        }
    }
    __syncthreads();
    double contrib = 0.0;
    if (g == 0) {
        const int u = u0 + lane;
#pragma unroll
        for (int j = 0; j < kFwXB; ++j) {
            for (int q = 1; q < kFwG; ++q) {
                const double* o = red2 + (((q - 1) * kFwGT + t) * kFwXB + j) * 3;
                e[j] += o[0];
                nk[j] += o[1];
                nt[j] += o[2];
            }
            const int v = v0 + wy * kFwXB + j;
            if (u < U && v < V) {
                const double rk_ = nk[j] / sqrt(e[j] * scal[1]);
                const double rt_ = nt[j] / sqrt(e[j] * scal[2]);
                const size_t oi = (size_t)v * U + u;
                rho_k[oi] = (float)rk_;
                rho_t[oi] = (float)rt_;
                ef_out[oi] = (float)e[j];
                fbar_out[oi] = fb[j];
                contrib += (rk_ - rt_) * (rk_ - rt_);
            }
        }
    }
    const double sum = block_sum_double(contrib, red);
    if (threadIdx.x == 0) atomicAdd(loss, sum);
}

// Per-offset coefficients of the backward pass, and the sums A1, A2.  The
// coefficients are FP32 (inputs and outputs are FP32); each warp sums its 32
// terms of A1 and A2 in FP32 and the warps' sums meet in FP64.
__device__ __forceinline__ float warp_sum_float(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(256) diff_coeff_kernel(int UV, const float* __restrict__ rho_k,
                                                         const float* __restrict__ rho_t,
                                                         const float* __restrict__ ef,
                                                         const float* __restrict__ fbar, const double* dloss,
                                                         double* scal, float* a, float* b, float* h, float* hf) {
    __shared__ double red[2][8];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float s1 = 0.0f, s2 = 0.0f;
    if (i < UV) {
        const float d = rho_k[i] - rho_t[i];
        const float g = (float)(2.0 * (*dloss)) * d;
        const float e = ef[i];
        const float ai = g / sqrtf(e * (float)scal[1]);
        const float hi = g * d / e;
        a[i] = ai;
        b[i] = g / sqrtf(e * (float)scal[2]);
        h[i] = hi;
        hf[i] = hi * fbar[i];
        s1 = ai * fbar[i];
        s2 = g * rho_k[i];
    }
    s1 = warp_sum_float(s1);
    s2 = warp_sum_float(s2);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = s1;
        red[1][warp] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r1 = 0.0, r2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            r1 += red[0][w];
            r2 += red[1][w];
        }
        atomicAdd(&scal[3], r1);
        atomicAdd(&scal[4], r2);
    }
}

// Row sums of h and h*fbar over the template width, for the two window-sum
// terms of dL/df: rh(v, px) = sum_{x < W, 0 <= px-x < U} h(v, px - x) in FP32
// (x ascending), the same for hf.  Grid (ceil(M / 256), V).
__global__ void __launch_bounds__(256) diff_rowbox_kernel(int M, int U, int W, const float* __restrict__ h,
                                                          const float* __restrict__ hf, float* __restrict__ rh,
                                                          float* __restrict__ rhf) {
    const int px = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y;
    if (px >= M) return;
    const float* hr = h + (size_t)v * U;
    const float* hfr = hf + (size_t)v * U;
    float s = 0.0f, sf = 0.0f;
    for (int x = max(0, px - U + 1); x < min(W, px + 1); ++x) {
        s += hr[px - x];
        sf += hfr[px - x];
    }
    rh[(size_t)v * M + px] = s;
    rhf[(size_t)v * M + px] = sf;
}

// dL/df(p) = sum_x [a(p-x) c(x) - b(p-x) t0(x)] + sum_x hf(p-x) - f(p) sum_x h(p-x)
// over template positions x with p - x a valid offset.  A CTA covers 64 x 16
// pixels with kGfYG groups of threads; thread (g, ry, gx) owns pixels
// px0 + 8gx .. +7 of row py0 + ry for the rows y = g, g + kGfYG, ... of each
// template block, and the groups' partial sums meet in shared memory at the
// end.  For each block of at most 64 x 64 the a and b regions the tile needs
// are staged in shared memory, with the block's columns reversed
// (x' = bw-1-x, zero-padded to a multiple of 8), so that along x' the
// thread's eight pixels read one sliding window of eight consecutive region
// columns: each step loads one new a and one new b value and does 16
// multiply-adds.  The h and h*fbar window sums come from the row sums of
// diff_rowbox_kernel, summed over template rows in FP64.
constexpr int kGfTX = 64, kGfTY = 16, kGfXB = 8, kGfYG = 4;
constexpr int kGfGroup = (kGfTX / kGfXB) * kGfTY;  // threads of one group
constexpr int kGfThreads = kGfGroup * kGfYG;

__host__ __device__ inline int gf_w8(int W) { return (W + 7) & ~7; }
__host__ __device__ inline int gf_rw(int W) { return kGfTX + gf_w8(W) - 1 + 1; }  // region pitch (one spare)
// dynamic shared memory: the staged a, b regions and reversed c, t0 of the
// largest block, or the partial sums of groups 1.. (whichever is larger)
__host__ __device__ inline size_t gf_smem(int W, int H) {
    const int bw = blk_edge(W), bh = blk_edge(H);
    const size_t stage = (2 * (size_t)gf_rw(bw) * (kGfTY + bh - 1) + 2 * (size_t)bh * gf_w8(bw)) * 4;
    const size_t part = (size_t)(kGfYG - 1) * kGfGroup * kGfXB * 8;
    return stage > part ? stage : part;
}

__global__ void __launch_bounds__(kGfThreads, 2) diff_grad_f_kernel(const float* __restrict__ f, int M, int N,
                                                                 int stride, int W, int H, const float* __restrict__ c,
                                                                 const float* __restrict__ t0,
                                                                 const float* __restrict__ a,
                                                                 const float* __restrict__ b,
                                                                 const float* __restrict__ rh,
                                                                 const float* __restrict__ rhf,
                                                                 float* __restrict__ grad, int gstride) {
    extern __shared__ __align__(16) float sm[];
    const int RW = gf_rw(blk_edge(W)), RHmax = kGfTY + blk_edge(H) - 1;  // region pitch and rows of the largest block
    const int U = M - W + 1, V = N - H + 1;
    float* as = sm;
    float* bs = as + RW * RHmax;
    float* cr = bs + RW * RHmax;  // bh x w8 of a block, reversed columns
    float* tr = cr + blk_edge(H) * gf_w8(blk_edge(W));
    const int px0 = blockIdx.x * kGfTX, py0 = blockIdx.y * kGfTY;
    const int grp = threadIdx.x / kGfGroup, t = threadIdx.x - grp * kGfGroup;
    const int gx = t % (kGfTX / kGfXB), ry = t / (kGfTX / kGfXB);
    const int py = py0 + ry, pxb = px0 + gx * kGfXB;
    KahanF acck[kGfXB];
    for (int by = 0; by < H; by += kDiffBlk) {
        for (int bx = 0; bx < W; bx += kDiffBlk) {
            const int bw = min(kDiffBlk, W - bx), bh = min(kDiffBlk, H - by);
            const int w8 = gf_w8(bw), rw = kGfTX + w8, rh = kGfTY + bh - 1;
            // offsets o = p - x for x in the block: columns from px0 - (bx + bw - 1), rows from py0 - (by + bh - 1)
            const int ox0 = px0 - (bx + bw - 1), oy0 = py0 - (by + bh - 1);
            __syncthreads();  // the previous block's reads are done
            for (int i = threadIdx.x; i < rw * rh; i += blockDim.x) {
                const int Y = i / rw, X = i - Y * rw;
                const int ou = ox0 + X, ov = oy0 + Y;
                const bool in = (ou >= 0 && ov >= 0 && ou < U && ov < V);
                const size_t o = in ? (size_t)ov * U + ou : 0;
                as[Y * RW + X] = in ? a[o] : 0.0f;
                bs[Y * RW + X] = in ? b[o] : 0.0f;
            }
            for (int i = threadIdx.x; i < bh * w8; i += blockDim.x) {
                const int y = i / w8, xr = i - y * w8;
                const bool in = xr < bw;
                cr[i] = in ? c[(by + y) * W + bx + (bw - 1 - xr)] : 0.0f;
                tr[i] = in ? t0[(by + y) * W + bx + (bw - 1 - xr)] : 0.0f;
            }
            __syncthreads();
            if (py < N && pxb < M) {
                for (int y = grp; y < bh; y += kGfYG) {
                    // offset row py - (by + y)  ->  region row ry + bh - 1 - y; pixel pxb + j, block
                    // column bw-1-x'  ->  offset column pxb + j - bx - (bw-1-x')  ->  region column gx*8 + j + x'
                    const float* arow = as + (ry + bh - 1 - y) * RW + gx * kGfXB;
                    const float* brow = bs + (ry + bh - 1 - y) * RW + gx * kGfXB;
                    const float* crow = cr + y * w8;
                    const float* trow = tr + y * w8;
                    float r[kGfXB], wa[kGfXB], wb[kGfXB];
#pragma unroll
                    for (int j = 0; j < kGfXB; ++j) r[j] = 0.0f;
#pragma unroll
                    for (int j = 0; j < kGfXB - 1; ++j) {
                        wa[j] = arow[j];
                        wb[j] = brow[j];
                    }
                    for (int xq = 0; xq < w8; xq += kGfXB) {
#pragma unroll
                        for (int k = 0; k < kGfXB; ++k) {
                            // wa[(k + j) % 8] holds region column xq + k + j
                            wa[(k + kGfXB - 1) % kGfXB] = arow[xq + k + kGfXB - 1];
                            wb[(k + kGfXB - 1) % kGfXB] = brow[xq + k + kGfXB - 1];
                            const float cv = crow[xq + k], tv = trow[xq + k];
#pragma unroll
                            for (int j = 0; j < kGfXB; ++j)
                                r[j] += wa[(k + j) % kGfXB] * cv - wb[(k + j) % kGfXB] * tv;
                        }
                    }
#pragma unroll
                    for (int j = 0; j < kGfXB; ++j) acck[j].add(r[j]);
                }
            }
        }
    }
    // groups 1.. hand their partial sums to group 0 (the staging area is free now)
    __syncthreads();
    double* part = reinterpret_cast<double*>(sm);
    if (grp > 0) {
#pragma unroll
        for (int j = 0; j < kGfXB; ++j) part[((size_t)(grp - 1) * kGfXB + j) * kGfGroup + t] = acck[j].value();
    }
    __syncthreads();
    if (grp > 0 || py >= N || pxb >= M) return;
#pragma unroll
    for (int j = 0; j < kGfXB; ++j) {
        const int px = pxb + j;
        if (px >= M) break;
        double acc = acck[j].value();
        for (int g = 1; g < kGfYG; ++g) acc += part[((size_t)(g - 1) * kGfXB + j) * kGfGroup + t];
        KahanF hs, hfs;
        for (int y = max(0, py - V + 1); y < min(H, py + 1); ++y) {
            hs.add(rh[(size_t)(py - y) * M + px]);
            hfs.add(rhf[(size_t)(py - y) * M + px]);
        }
        grad[(size_t)py * gstride + px] =
            (float)(acc + hfs.value() - (double)f[(size_t)py * stride + px] * hs.value());
    }
}

// Partial Gt(x, y) = sum_{o in chunk} a(o) f(o + (x, y)): grid
// (ceil(H / kGtYB), kGtChunks, ceil(W / 64)), kGtYB * ceil(min(W, 64) / kGtXB)
// threads; in template column block z (columns 64z .. 64z+63) thread
// (yy, xg) owns template row y0 + yy and block columns xg*kGtXB .. +kGtXB-1.  The
// CTA stages up to kGtVS offset rows x kGtUS offset columns of a, and the source
// rows and columns they meet, in shared memory; along u the thread keeps the
// last kGtXB source values in registers, so each step is one broadcast load
// of a, one load of f and kGtXB multiply-adds.  Per offset row and column
// block the products are summed in FP32 (at most kGtUS terms), then in FP64.
__global__ void __launch_bounds__(128) diff_gt_kernel(const float* __restrict__ f, int M, int N, int stride, int W,
                                                      int H, const float* __restrict__ a, double* __restrict__ gtp) {
    __shared__ float fs[(kGtVS + kGtYB - 1) * kGtFW];
    __shared__ float as[kGtVS * kGtUS];
    const int U = M - W + 1, V = N - H + 1;
    const int xb = blockIdx.z * kDiffBlk, bw = min(kDiffBlk, W - xb);
    const int XG = (bw + kGtXB - 1) / kGtXB;
    const int y0 = blockIdx.x * kGtYB, chunk = blockIdx.y;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int yy = tid / XG, xg = tid - yy * XG;
    const int y = y0 + yy, x0 = xg * kGtXB;
    const bool active = yy < kGtYB && y < H;
    const int vb = (int)((long long)V * chunk / kGtChunks), ve = (int)((long long)V * (chunk + 1) / kGtChunks);
    KahanF accd[kGtXB];
    for (int vs = vb; vs < ve; vs += kGtVS) {
        for (int us = 0; us < U; us += kGtUS) {
            __syncthreads();  // the previous block's reads are done
            for (int i = tid; i < kGtVS * kGtUS; i += nthr) {
                const int vv = i / kGtUS, uu = i - vv * kGtUS;
                const int v = vs + vv, u = us + uu;
                as[i] = (v < ve && u < U) ? a[(size_t)v * U + u] : 0.0f;
            }
            for (int i = tid; i < (kGtVS + kGtYB - 1) * kGtFW; i += nthr) {
                const int rr = i / kGtFW, cc = i - rr * kGtFW;
                const int row = vs + y0 + rr, col = us + xb + cc;
                fs[i] = (row < N && col < M) ? f[(size_t)row * stride + col] : 0.0f;
            }
            __syncthreads();
            if (active) {
                for (int vv = 0; vv < kGtVS; ++vv) {
                    const float* fr = fs + (vv + yy) * kGtFW + x0;
                    const float* ar = as + vv * kGtUS;
                    float acc[kGtXB], win[kGtXB];
#pragma unroll
                    for (int j = 0; j < kGtXB; ++j) acc[j] = 0.0f;
#pragma unroll
                    for (int j = 0; j < kGtXB - 1; ++j) win[j] = fr[j];
                    for (int u = 0; u < kGtUS; u += kGtXB) {
#pragma unroll
                        for (int k = 0; k < kGtXB; ++k) {
                            // win[(k + j) % kGtXB] holds fr[u + k + j]
                            win[(k + kGtXB - 1) % kGtXB] = fr[u + k + kGtXB - 1];
                            const float av = ar[u + k];
#pragma unroll
                            for (int j = 0; j < kGtXB; ++j) acc[j] += av * win[(k + j) % kGtXB];
                        }
                    }
#pragma unroll
                    for (int j = 0; j < kGtXB; ++j) accd[j].add(acc[j]);
                }
            }
        }
    }
    if (active) {
#pragma unroll
        for (int j = 0; j < kGtXB; ++j)
            if (x0 + j < bw) gtp[((size_t)chunk * H + y) * W + xb + x0 + j] = accd[j].value();
    }
}

// Gt = the sum of the chunk partials, in a fixed order.
__global__ void __launch_bounds__(256) diff_gt_reduce_kernel(int T, const double* __restrict__ gtp,
                                                             double* __restrict__ gt) {
    // kGtReduceLanes lanes per entry, each summing every kGtReduceLanes-th
    // chunk, then a fixed shuffle tree
    const int e = (blockIdx.x * blockDim.x + threadIdx.x) / kGtReduceLanes;
    const int l = threadIdx.x % kGtReduceLanes;
    double s = 0.0;
    if (e < T)
        for (int ch = l; ch < kGtChunks; ch += kGtReduceLanes) s += gtp[(size_t)ch * T + e];
#pragma unroll
    for (int o = kGtReduceLanes / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, kGtReduceLanes);
    if (e < T && l == 0) gt[e] = s;
}

// dL/dk_j for every segment: sum of Gt over the rectangle, minus the mean and
// energy terms (one thread per segment).
__global__ void __launch_bounds__(256) diff_grad_k_kernel(int W, int H, const int4* __restrict__ rects,
                                                          const float* __restrict__ k, int K,
                                                          const double* __restrict__ gt, const double* scal,
                                                          float* __restrict__ grad_k) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= K) return;
    const int4 r = rects[j];
    double s = 0.0;
    for (int y = max(r.y, 0); y < min(r.y + r.w, H); ++y)
        for (int x = max(r.x, 0); x < min(r.x + r.z, W); ++x) s += gt[(size_t)y * W + x];
    const double nj = (double)r.z * r.w;
    const double cj = (double)k[j] - scal[0];
    grad_k[j] = (float)(s - nj * scal[3] - nj * cj * scal[4] / scal[1]);
}

// Opt-in shared-memory limits of the two large-tile kernels (once per device).
cudaError_t set_diff_attributes() {
    static std::atomic<int> done[kDeviceSlots];
    return once_per_device(done, [] {
        cudaError_t err =
            cudaFuncSetAttribute(diff_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(diff_grad_f_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024);
        return err;
    });
}

bool diff_args_ok(int M, int N, int W, int H, int K, int f_stride) {
    return M > 0 && N > 0 && W > 0 && H > 0 && W <= kDiffMax && H <= kDiffMax && W <= M && H <= N && K > 0 &&
           K <= W * H && f_stride >= M;
}

// The offset maps are indexed in int (U V < 2^31) and the backward row-box
// pass takes one grid row per offset row (V <= 65535).
bool diff_size_ok(int M, int N, int W, int H) {
    const int64_t U = M - W + 1, V = N - H + 1;
    return U * V < ((int64_t)1 << 31) && V <= 65535;
}

}  // namespace
}  // namespace sncc

extern "C" size_t sncc_diff_workspace_bytes(int M, int N, int W, int H) {
    if (M <= 0 || N <= 0 || W <= 0 || H <= 0 || W > M || H > N) return 0;
    return sncc::diff_layout(M, N, W, H).total;
}

extern "C" int sncc_diff_forward(const float* d_f, int M, int N, int f_stride, const float* d_t, int W, int H,
                                 const int32_t* d_rects, const float* d_k, int K, float* d_rho_k, float* d_rho_t,
                                 double* d_loss, void* d_ws, size_t ws_bytes, sncc_stream_t stream) {
    sncc::NvtxRange nvtx_range("sncc_diff_forward");
    using namespace sncc;
    if (!d_f || !d_t || !d_rects || !d_k || !d_rho_k || !d_rho_t || !d_loss) return SNCC_ERR_ARG;
    if (!diff_args_ok(M, N, W, H, K, f_stride)) return SNCC_ERR_ARG;
    if (!diff_size_ok(M, N, W, H)) return SNCC_ERR_UNSUPPORTED;
    if (misaligned(d_f, 4) || misaligned(d_t, 4) || misaligned(d_rects, 16) || misaligned(d_k, 4) ||
        misaligned(d_rho_k, 4) || misaligned(d_rho_t, 4) || misaligned(d_loss, 8))
        return SNCC_ERR_ARG;
    const DiffLayout L = diff_layout(M, N, W, H);
    if (!d_ws || ws_bytes < L.total || (reinterpret_cast<uintptr_t>(d_ws) & 255)) return SNCC_ERR_WORKSPACE;
    char* ws = static_cast<char*>(d_ws);
    double* scal = reinterpret_cast<double*>(ws + L.scal);
    float* c = reinterpret_cast<float*>(ws + L.c);
    float* t0 = reinterpret_cast<float*>(ws + L.t0);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(d_loss, 0, sizeof(double), st) != cudaSuccess) return SNCC_ERR_CUDA;
    diff_prep_kernel<<<1, 256, 0, st>>>(d_t, W, H, reinterpret_cast<const int4*>(d_rects), d_k, K, scal, c, t0);
    const int U = M - W + 1, V = N - H + 1;
    const size_t sm = fw_smem_bytes(W, H);
    if (set_diff_attributes() != cudaSuccess) return SNCC_ERR_CUDA;
    dim3 grid((U + kFwTX - 1) / kFwTX, (V + kFwTY - 1) / kFwTY);
    diff_forward_kernel<<<grid, 256, sm, st>>>(d_f, M, N, f_stride, W, H, c, t0, scal, d_rho_k, d_rho_t,
                                               reinterpret_cast<float*>(ws + L.ef),
                                               reinterpret_cast<float*>(ws + L.fbar), d_loss);
    return cudaGetLastError() == cudaSuccess ? SNCC_OK : SNCC_ERR_CUDA;
}

extern "C" int sncc_diff_backward(const float* d_f, int M, int N, int f_stride, int W, int H,
                                  const int32_t* d_rects, const float* d_k, int K, const float* d_rho_k,
                                  const float* d_rho_t, const double* d_dloss, float* d_grad_f, int grad_f_stride,
                                  float* d_grad_k, void* d_ws, size_t ws_bytes, sncc_stream_t stream) {
    sncc::NvtxRange nvtx_range("sncc_diff_backward");
    using namespace sncc;
    if (!d_f || !d_rects || !d_k || !d_rho_k || !d_rho_t || !d_dloss || !d_grad_f || !d_grad_k) return SNCC_ERR_ARG;
    if (!diff_args_ok(M, N, W, H, K, f_stride) || grad_f_stride < M) return SNCC_ERR_ARG;
    if (!diff_size_ok(M, N, W, H)) return SNCC_ERR_UNSUPPORTED;
    if (misaligned(d_f, 4) || misaligned(d_rects, 16) || misaligned(d_k, 4) || misaligned(d_rho_k, 4) ||
        misaligned(d_rho_t, 4) || misaligned(d_dloss, 8) || misaligned(d_grad_f, 4) || misaligned(d_grad_k, 4))
        return SNCC_ERR_ARG;
    const DiffLayout L = diff_layout(M, N, W, H);
    if (!d_ws || ws_bytes < L.total || (reinterpret_cast<uintptr_t>(d_ws) & 255)) return SNCC_ERR_WORKSPACE;
    char* ws = static_cast<char*>(d_ws);
    double* scal = reinterpret_cast<double*>(ws + L.scal);
    const float* c = reinterpret_cast<const float*>(ws + L.c);
    const float* t0 = reinterpret_cast<const float*>(ws + L.t0);
    float* a = reinterpret_cast<float*>(ws + L.a);
    float* b = reinterpret_cast<float*>(ws + L.b);
    float* h = reinterpret_cast<float*>(ws + L.h);
    float* hf = reinterpret_cast<float*>(ws + L.hf);
    double* gtp = reinterpret_cast<double*>(ws + L.gtp);
    cudaStream_t st = (cudaStream_t)stream;
    const int U = M - W + 1, V = N - H + 1;
    const int UV = U * V;
    if (set_diff_attributes() != cudaSuccess) return SNCC_ERR_CUDA;
    // A1, A2 are accumulated from zero (scal[3], scal[4])
    if (cudaMemsetAsync(scal + 3, 0, 2 * sizeof(double), st) != cudaSuccess) return SNCC_ERR_CUDA;
    diff_coeff_kernel<<<(UV + 255) / 256, 256, 0, st>>>(UV, d_rho_k, d_rho_t, reinterpret_cast<const float*>(ws + L.ef),
                                                        reinterpret_cast<const float*>(ws + L.fbar), d_dloss, scal, a,
                                                        b, h, hf);
    float* rh = reinterpret_cast<float*>(ws + L.rh);
    float* rhf = reinterpret_cast<float*>(ws + L.rhf);
    diff_rowbox_kernel<<<dim3((M + 255) / 256, V), 256, 0, st>>>(M, U, W, h, hf, rh, rhf);
    const size_t smf = gf_smem(W, H);
    dim3 gridf((M + kGfTX - 1) / kGfTX, (N + kGfTY - 1) / kGfTY);
    diff_grad_f_kernel<<<gridf, kGfThreads, smf, st>>>(d_f, M, N, f_stride, W, H, c, t0, a, b, rh, rhf, d_grad_f,
                                                       grad_f_stride);
    const int gt_threads = kGtYB * ((blk_edge(W) + kGtXB - 1) / kGtXB);
    diff_gt_kernel<<<dim3((H + kGtYB - 1) / kGtYB, kGtChunks, (W + kDiffBlk - 1) / kDiffBlk), gt_threads, 0, st>>>(
        d_f, M, N, f_stride, W, H, a, gtp);
    double* gt = reinterpret_cast<double*>(ws + L.gt);
    diff_gt_reduce_kernel<<<(W * H * kGtReduceLanes + 255) / 256, 256, 0, st>>>(W * H, gtp, gt);
    diff_grad_k_kernel<<<(K + 255) / 256, 256, 0, st>>>(W, H, reinterpret_cast<const int4*>(d_rects), d_k, K, gt,
                                                        scal, d_grad_k);
    return cudaGetLastError() == cudaSuccess ? SNCC_OK : SNCC_ERR_CUDA;
}
