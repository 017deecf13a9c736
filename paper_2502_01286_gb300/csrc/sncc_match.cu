// sncc_match.cu - the coarse pass of segmented NCC: for every offset the
// approximate numerator sum_i (k_i - kbar) S_i(u, v) (Eq. 9, Eq. 11, Eq. 12),
// normalised by the local energy and the approximation energy (Eq. 13 -
// Eq. 18), thresholded and compacted into a candidate list (main algorithm,
// steps 7a-7f); and, with a second approximation on the tiles that hold
// candidates, the paper's fine stage (steps 7g-7j).
//
// Kernel design (one CTA = 8 warps = a 32 x 8R tile of offsets):
//  * The segment values enter as fixed-point weights q_i = round(c_i 2^F),
//    c_i = k_i - kbar, and the CTA computes the exact integer correlation
//    A(u, v) = sum_{x,y} q(x, y) f(u+x, v+y) through the corner form of
//    Eq. 11: every segment contributes +-q_i at its four corners and corners
//    shared by neighbouring segments are combined on the host, so each
//    offset needs one 32x32->64-bit multiply-add per distinct corner.
//  * Staged mode: the template is processed in blocks (one block up to
//    64 x 64; larger templates in 64 x 64 blocks).  For each block the
//    sum-table region the tile touches is staged in shared memory and
//    re-based to its own origin (exact in wrapped 32-bit arithmetic, since
//    every re-based entry is a box sum below 2^31):
//      - one block, 32-bit table: a 2-D TMA tile load completing on an
//        mbarrier, then an in-place re-base;
//      - several blocks, or a 64-bit table: the low words (box sums only
//        need the table modulo 2^32) are loaded through registers, two
//        entries per load, and stored already re-based.  On textured
//        templates of 96 to 256 pixels this ran 1.3 to 1.45x faster than
//        32 x 32 blocks with double-buffered TMA copies (fewer block edges,
//        fewer corners, half the staged entries per corner).
//    The region is read with conflict-free 32-bit loads: lane l reads
//    column l, warp w its own R rows.  The corners come regrouped into
//    vertical runs of 8, 4, 2 and 1 corners (consecutive rows of one
//    column): a lane's R rows share R + L - 1 region loads per run of L, so
//    on dense templates the shared-memory reads drop well below one per
//    (offset, corner) and the 64-bit multiply-add is the only limit.  Run
//    records are loaded one ahead of their use.
//  * Direct mode: a template with at most 64 corners in all is summed by
//    reading the table at its corners in place (no staging, no block edges).
//  * Fused launch: several approximations of one template size (the
//    thresholds of a multi-threshold search) in one grid, slice z = one
//    approximation, the one with most corners first.  A launch of 8R-row
//    tiles leaves the last wave partly empty; over the whole set the lighter
//    slices fill it.
//  * Epilogue: window sums from the global tables, exact integer variance
//    n sum f^2 - (sum f)^2 times 1/n in FP64, rho in FP32; the coarse pass
//    appends candidates (v*U+u) with warp-aggregated atomics, the fine mode
//    appends (u, v, rho) records of the offsets whose candidate bit is set.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "sncc.h"
#include "sncc_internal.h"
#include "sncc_ptx.cuh"
#include "sncc_tile.cuh"

namespace sncc {
namespace {

// One approximation of a fused multi-plan launch (sncc_match_multi): its
// corner runs, normalisation constants, threshold and outputs.
struct MultiPlan {
    const int4* runblk;
    const int4* runs;
    long long Q0;
    float Ek, scale, tau;
    int cand_cap;
    float* rho;
    int32_t* cand;
    int32_t* count;
    int32_t* status;
};
constexpr int kMaxMultiPlans = SNCC_MULTI_MAX;

struct MatchArgs {
    const int4* blocks;
    const int4* runblk;  // RUNBLK_INT4 per block
    const int4* runs;
    int nblk;
    int RH;  // region rows = 8R + BH + 1
    int M, N;
    int U, V, W, H;
    const void* s;
    const int64_t* s2;
    int pitch;
    long long n;
    double rn;  // 1 / n in FP64
    float inv_n;
    float Ek;
    float scale;  // 2^-F
    long long Q0;
    float tau;
    float* rho;
    int rho_pitch;
    int32_t* cand;
    int cand_cap;
    int32_t* count;
    int32_t* status;
    // fine mode (sncc_refine_segmented_tiles): the tiles to evaluate, the
    // candidate bit of every offset and the (u, v, rho) output records
    const int32_t* tile_list;
    const int32_t* tile_count;
    int tiles_u;
    const uint32_t* cand_bits;
    sncc_match_t* out;
    int out_cap;
    int32_t* nout;
    // direct mode: the whole template's corners {X, Y, G, 0}, read in place
    const int4* direct;
    int ndirect;
    // multi-plan mode: several approximations of one template size, one block
    int nplans;
    MultiPlan mp[kMaxMultiPlans];
};

__host__ __device__ constexpr int align_up(int x, int a) { return (x + a - 1) / a * a; }

// Shared-memory layout (32-bit words from a 128-byte aligned base):
//   work[align32(RH*WP)] | row0[128] | col0[160] | mbarrier (8 B) | flag
__host__ __device__ constexpr int work_words(int RH, int WP) { return align_up(RH * WP, 32); }
__host__ __device__ constexpr int smem_words(int RH, int WP) { return work_words(RH, WP) + 128 + 160 + 4; }

// 32-bit tables: starts the TMA tile copy of a block's region into `buf`
// (thread 0 issues; completion on `bar`).
template <int WP>
__device__ __forceinline__ void stage_region_tma(const CUtensorMap* map, int* buf, uint64_t* bar, int x0, int y0,
                                                 int RH, int tid) {
    if (tid == 0) {
        fence_proxy_async();  // earlier generic accesses to buf precede the async write
        mbar_arrive_expect_tx(bar, (uint32_t)(RH * WP * 4));
        tma_load_2d(buf, map, x0, y0, bar);
    }
}

// Epilogue: normalise, threshold, compact (coarse: candidate indices and
// the rho map; fine: (u, v, rho) records of the offsets whose candidate bit
// is set).
template <int R, bool S64, bool FINE>
__device__ __forceinline__ void match_epilogue(const MatchArgs& a, const long long (&acc)[R], int u0, int v0, int lane,
                                               int warp, float Ek, float scale, long long Q0, float tau, float* rho_map,
                                               int32_t* cand, int cand_cap, int32_t* count, int32_t* status) {
    const int u = u0 + lane;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = v0 + warp * R + r;
        bool valid = (u < a.U) && (v < a.V);
        if constexpr (FINE) {
            if (valid) {
                const int idx = v * a.U + u;
                valid = (a.cand_bits[idx >> 5] >> (idx & 31)) & 1u;
            }
        }
        const float rho = valid ? normalise<S64>(acc[r], a.s, a.s2, a.pitch, u, v, a.W, a.H, a.n, a.rn, a.inv_n, Ek,
                                                 scale, Q0)
                                : 0.0f;
        if (!FINE && rho_map != nullptr && valid) rho_map[(size_t)v * a.rho_pitch + u] = rho;
        const bool pred = valid && (rho >= tau);
        const unsigned m = __ballot_sync(0xffffffffu, pred);
        if (m) {
            const int leader = __ffs(m) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(FINE ? a.nout : count, __popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (pred) {
                const int pos = base + __popc(m & ((1u << lane) - 1u));
                if constexpr (FINE) {
                    if (pos < a.out_cap) {
                        sncc_match_t rec;
                        rec.u = u;
                        rec.v = v;
                        rec.rho = rho;
                        a.out[pos] = rec;
                    } else {
                        atomicOr(status, SNCC_STATUS_MATCH_OVERFLOW);
                    }
                } else {
                    if (pos < cand_cap)
                        cand[pos] = v * a.U + u;
                    else
                        atomicOr(status, SNCC_STATUS_CAND_OVERFLOW);
                }
            }
        }
    }
}

template <int R, bool S64, int WP, bool FINE, bool DIRECT, bool MULTI, bool REGS>
__global__ void __launch_bounds__(256) match_kernel(const __grid_constant__ CUtensorMap tmap, const MatchArgs a) {
    constexpr bool TMA = !S64 && !REGS;  // else the region is staged through registers
    extern __shared__ __align__(128) unsigned char smem_base[];
    // The TMA destination must start on a 128-byte boundary of the shared
    // window; the host allocates 128 spare bytes for this adjustment.
    int* work = reinterpret_cast<int*>(smem_base + ((128u - (smem_u32(smem_base) & 127u)) & 127u));
    const int RH = a.RH;
    int* row0 = work + work_words(RH, WP);
    int* col0 = row0 + 128;
    uint64_t* bar = reinterpret_cast<uint64_t*>(col0 + 160);
    volatile int* flag = reinterpret_cast<volatile int*>(bar + 1);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int u0 = blockIdx.x * TILE_U, v0 = blockIdx.y * (WARPS * R);
    if constexpr (FINE) {  // a 1-D grid over the listed tiles; the rest exit at once
        if ((int)blockIdx.x >= *a.tile_count) return;
        const int t = a.tile_list[blockIdx.x];
        u0 = (t % a.tiles_u) * TILE_U;
        v0 = (t / a.tiles_u) * (WARPS * R);
    }

    if (tid == 0) {
        if constexpr (TMA) {
            mbar_init(bar, 1);
            fence_mbar_init();
        }
        *flag = 0;
    }
    __syncthreads();

    // the corner runs: this launch's plan, or (fused launch) plan blockIdx.z
    const int4* runs = a.runs;
    const int4* runblk = a.runblk;
    if constexpr (MULTI) {
        runs = a.mp[blockIdx.z].runs;
        runblk = a.mp[blockIdx.z].runblk;
    }
    long long acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0;
    if constexpr (DIRECT) {
        // Sparse template: A = sum_p G_p s(u + X_p, v + Y_p) over its few
        // corners, table entries read in place (full 64-bit entries of 64-bit
        // tables) and summed modulo 2^64, which is exact since |A| < 2^63.
        // Lanes and rows outside the map read the last valid offset's entries.
        const int uu = min(u0 + lane, a.U - 1);
        unsigned long long accu[R];
#pragma unroll
        for (int r = 0; r < R; ++r) accu[r] = 0ull;
        for (int q = 0; q < a.ndirect; ++q) {
            const int4 cr = __ldg(a.direct + q);
            const int x = uu + cr.x;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int y = min(v0 + warp * R + r, a.V - 1) + cr.y;
                const long long sv = table_entry<S64>(a.s, a.pitch, x, y);
                accu[r] += (unsigned long long)(long long)cr.z * (unsigned long long)sv;
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = (long long)accu[r];
    } else {
        uint32_t parity = 0u;  // phase parity expected next on bar
        const int* wbase = work + warp * R * WP + lane;
        for (int b = 0; b < a.nblk; ++b) {
            const int4 blk = a.blocks[b];
            if constexpr (TMA) {
                // ---- tile copy of block b's region, then re-base it in place ----
                stage_region_tma<WP>(&tmap, work, bar, u0 + blk.x, v0 + blk.y, RH, tid);
                if (tid == 0 && !mbar_wait_bounded(bar, parity)) *flag = 1;
                __syncthreads();
                if (*flag) {
                    if (tid == 0) atomicOr(MULTI ? a.mp[blockIdx.z].status : a.status, SNCC_STATUS_WAIT_TIMEOUT);
                    return;
                }
                (void)mbar_try_wait(bar, parity);  // phase complete: acquire for this thread
                parity ^= 1u;
                for (int X = tid; X < WP; X += WARPS * 32) row0[X] = work[X];
                for (int Y = tid; Y < RH; Y += WARPS * 32) col0[Y] = work[Y * WP];
                __syncthreads();
                const uint32_t c00 = (uint32_t)row0[0];
                for (int Y = warp; Y < RH; Y += WARPS) {
                    const uint32_t cy = (uint32_t)col0[Y] - c00;
                    for (int X = lane; X < WP; X += 32)
                        work[Y * WP + X] = (int)((uint32_t)work[Y * WP + X] - (uint32_t)row0[X] - cy);
                }
            } else {
                stage_region_regs<S64, WP>(a.s, a.pitch, a.M, a.N, work, u0 + blk.x, v0 + blk.y, RH, lane, warp);
            }
            __syncthreads();
            // ---- corner sum over vertical runs: one multiply-add per (offset, corner) ----
            run_sum<R, WP>(acc, wbase, runs, runblk + RUNBLK_INT4 * b);
            __syncthreads();  // the region buffer is restaged for the next block
        }
    }

    if constexpr (MULTI) {
        const MultiPlan& mp = a.mp[blockIdx.z];
        match_epilogue<R, S64, false>(a, acc, u0, v0, lane, warp, mp.Ek, mp.scale, mp.Q0, mp.tau, mp.rho, mp.cand,
                                      mp.cand_cap, mp.count, mp.status);
    } else {
        match_epilogue<R, S64, FINE>(a, acc, u0, v0, lane, warp, a.Ek, a.scale, a.Q0, a.tau, a.rho, a.cand,
                                     a.cand_cap, a.count, a.status);
    }
}

// Fine mode, step 1: the candidate bit of every listed offset, and a flag on
// every tile (32 x rows offsets) that holds a candidate.
__global__ void __launch_bounds__(256) mark_candidate_tiles(const int32_t* __restrict__ cand,
                                                            const int32_t* __restrict__ count, int cand_cap, int U,
                                                            int V, int tiles_u, int rows, uint32_t* __restrict__ bits,
                                                            int32_t* __restrict__ tile_flag) {
    const int n = min(*count, cand_cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int idx = cand[i];
        if (idx < 0 || idx >= U * V) continue;  // not an offset
        const int u = idx % U, v = idx / U;
        atomicOr(&bits[idx >> 5], 1u << (idx & 31));
        tile_flag[(v / rows) * tiles_u + u / TILE_U] = 1;
    }
}

// Fine mode, step 2: the flagged tiles as a list (any order).
__global__ void __launch_bounds__(256) list_tiles(const int32_t* __restrict__ tile_flag, int ntiles,
                                                  int32_t* __restrict__ tile_list, int32_t* __restrict__ tile_count) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x)
        if (tile_flag[t]) tile_list[atomicAdd(tile_count, 1)] = t;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

template <int R, bool S64, int WP, bool FINE, bool DIRECT, bool MULTI, bool REGS>
cudaError_t launch_match(const CUtensorMap& map, const MatchArgs& a, int BH, cudaStream_t st) {
    const int RH = DIRECT ? 0 : WARPS * R + BH + 1;  // direct mode stages nothing
    MatchArgs args = a;
    args.RH = RH;
    const size_t sm = 128 + (size_t)smem_words(RH, WP) * 4;
    static std::atomic<int> done[kDeviceSlots];
    const cudaError_t attr_err = once_per_device(done, [] {
        return cudaFuncSetAttribute(match_kernel<R, S64, WP, FINE, DIRECT, MULTI, REGS>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    128 + smem_words(WARPS * R + 64 + 1, WP) * 4);
    });
    if (attr_err != cudaSuccess) return attr_err;
    const int tu = (a.U + TILE_U - 1) / TILE_U, tv = (a.V + WARPS * R - 1) / (WARPS * R);
    const dim3 grid = FINE ? dim3(tu * tv) : dim3(tu, tv, MULTI ? a.nplans : 1);
    match_kernel<R, S64, WP, FINE, DIRECT, MULTI, REGS><<<grid, WARPS * 32, sm, st>>>(map, args);
    return cudaGetLastError();
}

template <bool S64, int WP, bool FINE, bool DIRECT = false, bool MULTI = false, bool REGS = false>
cudaError_t dispatch_r(int R, const CUtensorMap& map, const MatchArgs& a, int BH, cudaStream_t st) {
    switch (R) {
        case 8: return launch_match<8, S64, WP, FINE, DIRECT, MULTI, REGS>(map, a, BH, st);
        case 4: return launch_match<4, S64, WP, FINE, DIRECT, MULTI, REGS>(map, a, BH, st);
        default: return launch_match<2, S64, WP, FINE, DIRECT, MULTI, REGS>(map, a, BH, st);
    }
}

// The segment-sum launch on a prepared MatchArgs: picks the kernel instance
// for the layout and table width.  One block (32-bit tables): TMA staging;
// 64 x 64 blocks of a larger template, or 64-bit tables: register staging.
template <bool FINE>
cudaError_t launch_layout(const Layout& L, bool s64, int R, const CUtensorMap& map, const MatchArgs& a,
                          cudaStream_t st) {
    if (a.ndirect > 0)  // sparse template: no staging
        return s64 ? dispatch_r<true, 100, FINE, true>(R, map, a, 0, st)
                   : dispatch_r<false, 100, FINE, true>(R, map, a, 0, st);
    if (s64)
        return L.WP == 68 ? dispatch_r<true, 68, FINE>(R, map, a, L.BH, st)
                          : dispatch_r<true, 100, FINE>(R, map, a, L.BH, st);
    if (L.nblk > 1) return dispatch_r<false, 100, FINE, false, false, true>(R, map, a, L.BH, st);
    return L.WP == 68 ? dispatch_r<false, 68, FINE>(R, map, a, L.BH, st)
                      : dispatch_r<false, 100, FINE>(R, map, a, L.BH, st);
}

// Offsets per thread: the largest R in {8, 4, 2} that still gives two CTAs
// per SM.
int choose_r(int U, int V) {
    const int tu = (U + TILE_U - 1) / TILE_U;
    const int sms = sm_count() > 0 ? sm_count() : 1;
    for (int R : {8, 4}) {
        const long long ctas = (long long)tu * ((V + WARPS * R - 1) / (WARPS * R));
        if (ctas >= 2 * sms) return R;
    }
    return 2;
}

// Shared by sncc_match and sncc_refine_segmented_tiles: checks the common
// arguments and fills the kernel arguments and (32-bit tables) the TMA map.
int prepare_match(const sncc_segments* seg, const void* d_plan, const void* d_s, int s_bits, const int64_t* d_s2,
                  int sat_pitch, int M, int N, float tau, MatchArgs& a, CUtensorMap& map, int& R, const Layout*& Lout) {
    const Plan* p = plan_of(seg);
    if (!seg || !p || !d_plan || !d_s || !d_s2) return SNCC_ERR_ARG;
    if (s_bits != 32 && s_bits != 64) return SNCC_ERR_ARG;
    if (!(seg->Ek > 0.0) || p->image.empty()) return SNCC_ERR_UNIFORM;
    const int W = seg->W, H = seg->H;
    const int U = M - W + 1, V = N - H + 1;
    if (W <= 0 || H <= 0 || U <= 0 || V <= 0) return SNCC_ERR_ARG;
    if (sat_pitch < M + 1 || (sat_pitch & 3)) return SNCC_ERR_ARG;
    if (misaligned(d_plan, 16) || misaligned(d_s, 16) || misaligned(d_s2, 8)) return SNCC_ERR_ARG;
    if ((int64_t)U * V >= ((int64_t)1 << 31)) return SNCC_ERR_UNSUPPORTED;

    const bool s64 = (s_bits == 64);
    const Layout& L = layout_for(*p);
    Lout = &L;
    R = choose_r(U, V);
    const int RH = WARPS * R + L.BH + 1;
    std::memset(&map, 0, sizeof(map));
    if (!s64) {  // 2-D TMA tile map over the 32-bit table, box WP x RH
        PFN_cuTensorMapEncodeTiled_v12000 encode = get_encode();
        if (!encode) return SNCC_ERR_CUDA;
        cuuint64_t gdim[2] = {(cuuint64_t)(M + 1), (cuuint64_t)(N + 1)};
        cuuint64_t gstride[1] = {(cuuint64_t)sat_pitch * 4};
        cuuint32_t box[2] = {(cuuint32_t)L.WP, (cuuint32_t)RH};
        cuuint32_t estride[2] = {1, 1};
        CUresult cr = encode(&map, CU_TENSOR_MAP_DATA_TYPE_INT32, 2, const_cast<void*>(d_s), gdim, gstride, box,
                             estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) return SNCC_ERR_CUDA;
    }
    std::memset(&a, 0, sizeof(a));
    a.blocks = reinterpret_cast<const int4*>(static_cast<const char*>(d_plan) + L.blocks_offset);
    a.runblk = reinterpret_cast<const int4*>(static_cast<const char*>(d_plan) + L.runblk_offset);
    a.runs = reinterpret_cast<const int4*>(static_cast<const char*>(d_plan) + L.runs_offset);
    a.nblk = L.nblk;
    a.RH = RH;
    a.M = M;
    a.N = N;
    a.U = U;
    a.V = V;
    a.W = W;
    a.H = H;
    a.s = d_s;
    a.s2 = d_s2;
    a.pitch = sat_pitch;
    a.n = (long long)W * H;
    a.rn = 1.0 / ((double)W * H);
    a.inv_n = (float)a.rn;
    a.Ek = (float)seg->Ek;
    a.scale = (float)std::ldexp(1.0, -p->F);
    a.Q0 = p->Q0;
    a.tau = tau;
    a.tiles_u = (U + TILE_U - 1) / TILE_U;
    // The whole-template corner list reads table entries themselves, which a
    // 32-bit table holds only modulo 2^32 once 255*M*N reaches 2^31; staged
    // regions and window sums are differences below 2^31 (W*H <= 2^23), exact
    // in wrapped 32-bit arithmetic.
    const bool wraps = !s64 && (int64_t)255 * M * N >= ((int64_t)1 << 31);
    a.ndirect = wraps ? 0 : p->direct_count;
    a.direct = reinterpret_cast<const int4*>(static_cast<const char*>(d_plan) + p->direct_offset);
    return SNCC_OK;
}

// Workspace of sncc_refine_segmented_tiles, in order: match records
// (out_cap, 16-byte aligned), candidate bits (one per offset), tile flags,
// tile list, tile count, the sort scratch.
struct TilesLayout {
    size_t recs, bits, flags, list, count, sort, total;
    int ntiles, rows;
};

TilesLayout tiles_layout(int M, int N, int W, int H, int out_cap) {
    const int U = M - W + 1, V = N - H + 1;
    const int R = choose_r(U, V);
    TilesLayout t;
    t.rows = WARPS * R;
    t.ntiles = ((U + TILE_U - 1) / TILE_U) * ((V + t.rows - 1) / t.rows);
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    size_t o = 0;
    t.recs = o;
    o = al(o + (size_t)(out_cap > 0 ? out_cap : 1) * sizeof(sncc_match_t));
    t.bits = o;
    o = al(o + (((size_t)U * V + 31) / 32) * 4);
    t.flags = o;
    o = al(o + (size_t)t.ntiles * 4);
    t.list = o;
    o = al(o + (size_t)t.ntiles * 4);
    t.count = o;
    o = al(o + 16);
    t.sort = o;
    o = al(o + match_sort_bytes(U, V));
    t.total = o;
    return t;
}

}  // namespace

int multi_fusable(const sncc_segments* const* segs, const void* const* d_plans, int n) {
    if (!segs || !d_plans || n < 1 || n > SNCC_MULTI_MAX) return SNCC_ERR_ARG;
    // every approximation: the same template size and a plan
    for (int q = 0; q < n; ++q) {
        if (!segs[q] || !plan_of(segs[q]) || !d_plans[q] || (reinterpret_cast<uintptr_t>(d_plans[q]) & 15))
            return SNCC_ERR_ARG;
        if (segs[q]->W != segs[0]->W || segs[q]->H != segs[0]->H) return SNCC_ERR_ARG;
        if (!(segs[q]->Ek > 0.0) || plan_of(segs[q])->image.empty()) return SNCC_ERR_UNIFORM;
    }
    // and one staged block of the same layout each (templates up to 64 x 64
    // that are not summed directly)
    const Layout& L0 = layout_for(*plan_of(segs[0]));
    for (int q = 0; q < n; ++q) {
        const Plan* p = plan_of(segs[q]);
        const Layout& Lq = layout_for(*p);
        if (Lq.nblk != 1 || Lq.nbx * Lq.nby != 1 || Lq.WP != L0.WP || Lq.BH != L0.BH || p->direct_count > 0)
            return SNCC_ERR_UNSUPPORTED;
    }
    return SNCC_OK;
}

}  // namespace sncc

extern "C" int sncc_match(const sncc_segments* seg, const void* d_plan, const void* d_s, int s_bits,
                          const int64_t* d_s2, int sat_pitch, int M, int N, float tau, float* d_rho, int rho_pitch,
                          int32_t* d_cand, int cand_cap, int32_t* d_count, int32_t* d_status, sncc_stream_t stream) {
    sncc::NvtxRange nvtx_range("sncc_match");
    using namespace sncc;
    if (!d_count || !d_status || cand_cap < 0 || (cand_cap > 0 && !d_cand)) return SNCC_ERR_ARG;
    if (misaligned(d_rho, 4) || misaligned(d_cand, 4) || misaligned(d_count, 4) || misaligned(d_status, 4))
        return SNCC_ERR_ARG;
    MatchArgs a;
    CUtensorMap map;
    int R = 0;
    const Layout* L = nullptr;
    const int rc = prepare_match(seg, d_plan, d_s, s_bits, d_s2, sat_pitch, M, N, tau, a, map, R, L);
    if (rc != SNCC_OK) return rc;
    if (d_rho && rho_pitch < a.U) return SNCC_ERR_ARG;
    a.rho = d_rho;
    a.rho_pitch = rho_pitch;
    a.cand = d_cand;
    a.cand_cap = cand_cap;
    a.count = d_count;
    a.status = d_status;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(d_count, 0, sizeof(int32_t), st) != cudaSuccess) return SNCC_ERR_CUDA;
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), st) != cudaSuccess) return SNCC_ERR_CUDA;
    return launch_layout<false>(*L, s_bits == 64, R, map, a, st) == cudaSuccess ? SNCC_OK : SNCC_ERR_CUDA;
}

extern "C" size_t sncc_refine_segmented_tiles_workspace_bytes(int M, int N, int W, int H, int out_cap) {
    if (M <= 0 || N <= 0 || W <= 0 || H <= 0 || W > M || H > N || out_cap < 0) return 0;
    return sncc::tiles_layout(M, N, W, H, out_cap).total;
}

extern "C" int sncc_refine_segmented_tiles(const sncc_segments* seg, const void* d_plan, const void* d_s, int s_bits,
                                           const int64_t* d_s2, int sat_pitch, int M, int N, const int32_t* d_cand,
                                           const int32_t* d_count, int cand_cap, float tau, sncc_match_t* d_out,
                                           int out_cap, int32_t* d_nout, void* d_ws, size_t ws_bytes,
                                           int32_t* d_status, sncc_stream_t stream) {
    sncc::NvtxRange nvtx_range("sncc_refine_segmented_tiles");
    using namespace sncc;
    if (!d_count || !d_nout || !d_status || cand_cap < 0 || out_cap < 0) return SNCC_ERR_ARG;
    if ((cand_cap > 0 && !d_cand) || (out_cap > 0 && !d_out)) return SNCC_ERR_ARG;
    if (misaligned(d_cand, 4) || misaligned(d_count, 4) || misaligned(d_out, 4) || misaligned(d_nout, 4) ||
        misaligned(d_status, 4))
        return SNCC_ERR_ARG;
    MatchArgs a;
    CUtensorMap map;
    int R = 0;
    const Layout* L = nullptr;
    const int rc = prepare_match(seg, d_plan, d_s, s_bits, d_s2, sat_pitch, M, N, tau, a, map, R, L);
    if (rc != SNCC_OK) return rc;
    const TilesLayout t = tiles_layout(M, N, seg->W, seg->H, out_cap);
    if (!d_ws || ws_bytes < t.total || (reinterpret_cast<uintptr_t>(d_ws) & 255)) return SNCC_ERR_WORKSPACE;
    char* ws = static_cast<char*>(d_ws);
    uint32_t* bits = reinterpret_cast<uint32_t*>(ws + t.bits);
    int32_t* flags = reinterpret_cast<int32_t*>(ws + t.flags);
    int32_t* list = reinterpret_cast<int32_t*>(ws + t.list);
    int32_t* tcount = reinterpret_cast<int32_t*>(ws + t.count);
    sncc_match_t* recs = reinterpret_cast<sncc_match_t*>(ws + t.recs);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(d_nout, 0, sizeof(int32_t), st) != cudaSuccess) return SNCC_ERR_CUDA;
    if (cudaMemsetAsync(ws + t.bits, 0, t.list - t.bits, st) != cudaSuccess) return SNCC_ERR_CUDA;  // bits, flags
    if (cudaMemsetAsync(tcount, 0, sizeof(int32_t), st) != cudaSuccess) return SNCC_ERR_CUDA;
    if (cand_cap == 0) return SNCC_OK;
    const int sms = sm_count() > 0 ? sm_count() : 1;
    mark_candidate_tiles<<<2 * sms, 256, 0, st>>>(d_cand, d_count, cand_cap, a.U, a.V, a.tiles_u, t.rows, bits, flags);
    list_tiles<<<(t.ntiles + 255) / 256, 256, 0, st>>>(flags, t.ntiles, list, tcount);
    if (cudaGetLastError() != cudaSuccess) return SNCC_ERR_CUDA;
    a.tile_list = list;
    a.tile_count = tcount;
    a.cand_bits = bits;
    a.out = recs;
    a.out_cap = out_cap;
    a.nout = d_nout;
    a.status = d_status;
    if (launch_layout<true>(*L, s_bits == 64, R, map, a, st) != cudaSuccess) return SNCC_ERR_CUDA;
    if (out_cap > 0 && launch_match_sort(recs, d_nout, out_cap, a.U, a.V, ws + t.sort, d_out, st) != cudaSuccess)
        return SNCC_ERR_CUDA;
    return SNCC_OK;
}

extern "C" int sncc_match_multi(const sncc_segments* const* segs, const void* const* d_plans, int n, const void* d_s,
                                int s_bits, const int64_t* d_s2, int sat_pitch, int M, int N, const float* taus,
                                float* const* d_rho, int rho_pitch, int32_t* const* d_cand, int cand_cap,
                                int32_t* const* d_count, int32_t* const* d_status, sncc_stream_t stream) {
    sncc::NvtxRange nvtx_range("sncc_match_multi");
    using namespace sncc;
    if (!segs || !d_plans || !taus || !d_cand || !d_count || !d_status || n < 1 || n > SNCC_MULTI_MAX || cand_cap < 0)
        return SNCC_ERR_ARG;
    for (int q = 0; q < n; ++q) {  // every approximation has its own outputs
        if ((cand_cap > 0 && !d_cand[q]) || !d_count[q] || !d_status[q]) return SNCC_ERR_ARG;
        if ((d_rho && misaligned(d_rho[q], 4)) || misaligned(d_cand[q], 4) || misaligned(d_count[q], 4) ||
            misaligned(d_status[q], 4))
            return SNCC_ERR_ARG;
    }
    const int fz = multi_fusable(segs, d_plans, n);  // decided on the host before any CUDA call
    if (fz != SNCC_OK) return fz;
    MatchArgs a;
    CUtensorMap map;
    int R = 0;
    const Layout* L = nullptr;
    const int rc = prepare_match(segs[0], d_plans[0], d_s, s_bits, d_s2, sat_pitch, M, N, taus[0], a, map, R, L);
    if (rc != SNCC_OK) return rc;
    if (d_rho && rho_pitch < a.U) return SNCC_ERR_ARG;
    const bool s64 = (s_bits == 64);
    // grid slice z = 0 is dispatched first: the approximations with the most
    // corners go first, so that the lighter ones fill the last wave
    int order[kMaxMultiPlans];
    for (int q = 0; q < n; ++q) order[q] = q;
    std::stable_sort(order, order + n, [&](int x, int y) {
        return plan_of(segs[x])->template_corners > plan_of(segs[y])->template_corners;
    });
    for (int z = 0; z < n; ++z) {
        const int q = order[z];
        const Plan* p = plan_of(segs[q]);
        const Layout& Lq = layout_for(*p);
        MultiPlan& mp = a.mp[z];
        mp.runblk = reinterpret_cast<const int4*>(static_cast<const char*>(d_plans[q]) + Lq.runblk_offset);
        mp.runs = reinterpret_cast<const int4*>(static_cast<const char*>(d_plans[q]) + Lq.runs_offset);
        mp.Q0 = p->Q0;
        mp.Ek = (float)segs[q]->Ek;
        mp.scale = (float)std::ldexp(1.0, -p->F);
        mp.tau = taus[q];
        mp.cand_cap = cand_cap;
        mp.rho = d_rho ? d_rho[q] : nullptr;
        mp.cand = d_cand[q];
        mp.count = d_count[q];
        mp.status = d_status[q];
    }
    a.nplans = n;
    a.ndirect = 0;
    a.rho_pitch = rho_pitch;
    a.status = a.mp[0].status;
    cudaStream_t st = (cudaStream_t)stream;
    for (int q = 0; q < n; ++q)
        if (cudaMemsetAsync(d_count[q], 0, sizeof(int32_t), st) != cudaSuccess ||
            cudaMemsetAsync(d_status[q], 0, sizeof(int32_t), st) != cudaSuccess)
            return SNCC_ERR_CUDA;
    cudaError_t e;
    if (L->WP == 68)
        e = s64 ? dispatch_r<true, 68, false, false, true>(R, map, a, L->BH, st)
                : dispatch_r<false, 68, false, false, true>(R, map, a, L->BH, st);
    else
        e = s64 ? dispatch_r<true, 100, false, false, true>(R, map, a, L->BH, st)
                : dispatch_r<false, 100, false, false, true>(R, map, a, L->BH, st);
    return e == cudaSuccess ? SNCC_OK : SNCC_ERR_CUDA;
}
