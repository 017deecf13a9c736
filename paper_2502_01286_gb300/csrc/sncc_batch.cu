// sncc_batch.cu - many templates against several sources in one persistent
// launch: the coarse pass of segmented NCC (Eq. 9 - Eq. 18, main algorithm
// steps 7a-7f) for every (source, template) pair, then the exact refine of
// all candidates (Eq. 1, steps 7g-7j with an exact second stage).
//
// Design:
//  * Host: every template's plan is rebuilt with 64 x 64 blocks and one
//    region pitch (100 words), so a single kernel instance serves templates
//    of any size.  A work list of tiles (pair, tile column, tile row) is
//    built for each tile height R in {8, 4, 2} and ordered by estimated cost,
//    largest first (corner count plus staging), so that the dynamic schedule
//    below ends with the cheap tiles.
//  * Device: a persistent grid (occupancy x SMs) of 8-warp CTAs pulls tiles
//    with one atomic per tile; each tile runs the same staging / corner-sum /
//    normalisation code as the single-problem kernel (sncc_tile.cuh), with
//    the sources staged through registers.  Candidates are appended as
//    (pair, v*U+u) with warp-aggregated atomics.
//  * The tile height is chosen by an autotuner that times the variants on the
//    caller's data (sncc_batch_autotune) or given explicitly.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "sncc.h"
#include "sncc_internal.h"
#include "sncc_sort.cuh"
#include "sncc_tile.cuh"

namespace sncc {
namespace {

constexpr int kBatchWP = 100;  // region pitch of 64 x 64 blocks
constexpr int kBatchBlock = 64;
constexpr int kVariants[3] = {8, 4, 2};

struct TmplDesc {  // 80 bytes, one per template
    int W, H, nblk, blk_first;
    long long n, Q0;
    long long T, T2;
    float inv_n, Ek, scale, tau;
    float tau_exact;
    int pix_offset;
    double rn;  // 1 / n in FP64
};
static_assert(sizeof(TmplDesc) == 80, "template descriptor layout");

struct BatchArgs {
    const int4* pairs;  // {source, template, U, V}
    const TmplDesc* tmpl;
    const int4* blocks;
    const int4* runblk;  // RUNBLK_INT4 per block
    const int4* runs;
    const int2* items;  // {pair, (tile row << 16) | tile column}
    int n_items;
    int* counter;
    const void* s[SNCC_BATCH_MAX_SOURCES];
    const int64_t* s2[SNCC_BATCH_MAX_SOURCES];
    int pitch, M, N;
    int2* cand;
    int cand_cap;
    int* count;
    int* status;
};

template <int R, bool S64>
__global__ void __launch_bounds__(WARPS * 32) batch_match_kernel(const __grid_constant__ BatchArgs a) {
    constexpr int WP = kBatchWP;
    extern __shared__ __align__(16) int work[];
    __shared__ int item_sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int* wbase = work + warp * R * WP + lane;
    for (;;) {
        if (tid == 0) item_sh = atomicAdd(a.counter, 1);
        __syncthreads();
        const int it = item_sh;
        __syncthreads();  // item_sh is rewritten only after every thread has read it
        if (it >= a.n_items) break;
        const int2 item = a.items[it];
        const int4 pd = a.pairs[item.x];
        const TmplDesc& td = a.tmpl[pd.y];
        const int u0 = (item.y & 0xffff) * TILE_U, v0 = (item.y >> 16) * (WARPS * R);
        const void* s = a.s[pd.x];
        const int64_t* s2 = a.s2[pd.x];
        long long acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = 0;
        const int nblk = td.nblk;
        for (int b = 0; b < nblk; ++b) {
            const int4 blk = a.blocks[td.blk_first + b];
            const int bw = min(kBatchBlock, td.W - blk.x), bh = min(kBatchBlock, td.H - blk.y);
            stage_region_regs<S64, WP>(s, a.pitch, a.M, a.N, work, u0 + blk.x, v0 + blk.y, WARPS * R + bh + 1, lane,
                                       warp, TILE_U + bw + 1);
            __syncthreads();
            const int gb = td.blk_first + b;
            run_sum<R, WP>(acc, wbase, a.runs, a.runblk + RUNBLK_INT4 * gb);
            __syncthreads();
        }
        const int u = u0 + lane;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int v = v0 + warp * R + r;
            const bool valid = (u < pd.z) && (v < pd.w);
            const float rho = valid ? normalise<S64>(acc[r], s, s2, a.pitch, u, v, td.W, td.H, td.n, td.rn, td.inv_n, td.Ek,
                                                     td.scale, td.Q0)
                                    : 0.0f;
            const bool pred = valid && (rho >= td.tau);
            const unsigned m = __ballot_sync(0xffffffffu, pred);
            if (m) {
                const int leader = __ffs(m) - 1;
                int base = 0;
                if (lane == leader) base = atomicAdd(a.count, __popc(m));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (pred) {
                    const int pos = base + __popc(m & ((1u << lane) - 1u));
                    if (pos < a.cand_cap)
                        a.cand[pos] = make_int2(item.x, v * pd.z + u);
                    else
                        atomicOr(a.status, SNCC_STATUS_CAND_OVERFLOW);
                }
            }
        }
    }
}

struct BatchRefineArgs {
    const int4* pairs;
    const TmplDesc* tmpl;
    const uint8_t* pix;
    const uint8_t* f[SNCC_BATCH_MAX_SOURCES];
    int f_stride;
    const int2* cand;
    const int* count;
    int cand_cap;
    sncc_batch_match_t* scratch;
    int scratch_cap;
    int* nout;
    int* status;
};

__device__ __forceinline__ long long warp_sum64(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Exact NCC (Eq. 1) in integers at every candidate, one CTA per candidate.
__global__ void __launch_bounds__(256) batch_refine_kernel(const __grid_constant__ BatchRefineArgs a) {
    __shared__ long long red[3][8];
    const int count = min(*a.count, a.cand_cap);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = blockIdx.x; i < count; i += gridDim.x) {
        const int2 c = a.cand[i];
        const int4 pd = a.pairs[c.x];
        const TmplDesc& td = a.tmpl[pd.y];
        if (c.y < 0 || c.y >= pd.z * pd.w) continue;  // not an offset (uniform per CTA)
        const int u = c.y % pd.z, v = c.y / pd.z;
        const uint8_t* f = a.f[pd.x];
        const uint8_t* t = a.pix + td.pix_offset;
        long long sft = 0, sf = 0, sff = 0;
        for (int y = warp; y < td.H; y += 8) {
            const uint8_t* frow = f + (size_t)(v + y) * a.f_stride + u;
            const uint8_t* trow = t + (size_t)y * td.W;
            for (int x = lane; x < td.W; x += 32) {
                const int fv = frow[x], tv = trow[x];
                sft += fv * tv;
                sf += fv;
                sff += fv * fv;
            }
        }
        sft = warp_sum64(sft);
        sf = warp_sum64(sf);
        sff = warp_sum64(sff);
        if (lane == 0) {
            red[0][warp] = sft;
            red[1][warp] = sf;
            red[2][warp] = sff;
        }
        __syncthreads();
        if (tid == 0) {
            long long A = 0, B = 0, Cc = 0;
            for (int w = 0; w < 8; ++w) {
                A += red[0][w];
                B += red[1][w];
                Cc += red[2][w];
            }
            const long long num = td.n * A - td.T * B;
            const long long vf = td.n * Cc - B * B;
            const long long vt = td.n * td.T2 - td.T * td.T;
            const float rho = (vf > 0 && vt > 0) ? (float)((double)num / sqrt((double)vf * (double)vt)) : 0.0f;
            if (rho >= td.tau_exact) {
                const int pos = atomicAdd(a.nout, 1);
                if (pos < a.scratch_cap) {
                    sncc_batch_match_t m;
                    m.pair = c.x;
                    m.u = u;
                    m.v = v;
                    m.rho = rho;
                    a.scratch[pos] = m;
                } else {
                    atomicOr(a.status, SNCC_STATUS_MATCH_OVERFLOW);
                }
            }
        }
        __syncthreads();
    }
}

// The sort key of a batch match: its offset in the concatenation of every
// pair's offset space, pair-major (base[pair] + v*U + u), so that the sorted
// list is ordered by (pair, v*U+u).
struct BatchKey {
    const int4* pairs;
    const long long* base;
    __device__ __forceinline__ long long operator()(const sncc_batch_match_t& m) const {
        return base[m.pair] + (long long)m.v * pairs[m.pair].z + m.u;
    }
};

size_t align16(size_t x) { return (x + 15) / 16 * 16; }

}  // namespace
}  // namespace sncc

struct sncc_batch_s {
    int nt = 0, ns = 0, M = 0, N = 0;
    std::vector<sncc::TmplDesc> tmpl;
    std::vector<int32_t> corner_counts;    // nonzero corners per template in the 64 x 64 layout (the work)
    std::vector<int32_t> template_corners;  // corners of each whole template (the algorithmic count)
    size_t off_pairs = 0, off_pbase = 0, off_tmpl = 0, off_blocks = 0, off_runblk = 0, off_runs = 0, off_pix = 0,
           off_items[3] = {0, 0, 0};
    int n_items[3] = {0, 0, 0};
    std::vector<unsigned char> image;
    int variant = 8;
    int grid[3] = {0, 0, 0};
    double corner_offsets = 0.0;  // sum over pairs of U*V*(corners of the whole template)
    double offsets = 0.0;         // sum over pairs of U*V
};

namespace sncc {
namespace {

int variant_index(int R) { return R == 8 ? 0 : (R == 4 ? 1 : (R == 2 ? 2 : -1)); }

template <int R>
size_t batch_smem(void) {
    return (size_t)(WARPS * R + kBatchBlock + 1) * kBatchWP * 4;
}

template <int R, bool S64>
cudaError_t batch_launch(sncc_batch* b, const BatchArgs& args, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    static int per_sm = 0, sms = 0;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(batch_match_kernel<R, S64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)batch_smem<R>());
        if (attr == cudaSuccess)
            attr = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_match_kernel<R, S64>, WARPS * 32,
                                                                 batch_smem<R>());
        int dev = 0;
        if (attr == cudaSuccess) attr = cudaGetDevice(&dev);
        if (attr == cudaSuccess) attr = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    });
    if (attr != cudaSuccess) return attr;
    const int grid = std::max(1, per_sm) * std::max(1, sms);
    b->grid[variant_index(R)] = grid;
    batch_match_kernel<R, S64><<<grid, WARPS * 32, batch_smem<R>(), st>>>(args);
    return cudaGetLastError();
}

}  // namespace
}  // namespace sncc

extern "C" int sncc_batch_create(const sncc_segments* const* segs, const uint8_t* const* templates,
                                 const int* t_strides, const float* tau_coarse, const float* tau_exact,
                                 int n_templates, int n_sources, int M, int N, sncc_batch** out) {
    using namespace sncc;
    if (!segs || !templates || !t_strides || !tau_coarse || !tau_exact || !out) return SNCC_ERR_ARG;
    if (n_templates <= 0 || n_sources <= 0 || n_sources > SNCC_BATCH_MAX_SOURCES || M <= 0 || N <= 0)
        return SNCC_ERR_ARG;
    if ((int64_t)n_templates * n_sources > (1 << 20)) return SNCC_ERR_UNSUPPORTED;
    if (M > 16383 || N > 8192) return SNCC_ERR_UNSUPPORTED;
    *out = nullptr;
    sncc_batch* b = new (std::nothrow) sncc_batch();
    if (!b) return SNCC_ERR_NOMEM;
    try {
        b->nt = n_templates;
        b->ns = n_sources;
        b->M = M;
        b->N = N;
        std::vector<int32_t> blocks, runblk, runs;
        std::vector<unsigned char> pix;
        for (int t = 0; t < n_templates; ++t) {
            const sncc_segments* sg = segs[t];
            if (!sg || !templates[t] || t_strides[t] < sg->W) {
                delete b;
                return SNCC_ERR_ARG;
            }
            if (!(sg->Ek > 0.0)) {
                delete b;
                return SNCC_ERR_UNIFORM;
            }
            if (sg->W > M || sg->H > N || (int64_t)sg->W * sg->H > ((int64_t)1 << 23)) {
                delete b;
                return SNCC_ERR_ARG;
            }
            Plan p;
            build_plan(sg, p);
            const Layout& L = p.lay[1];  // blocks of at most 64 x 64, pitch 100
            TmplDesc d;
            std::memset(&d, 0, sizeof(d));
            d.W = sg->W;
            d.H = sg->H;
            d.nblk = L.nblk;
            d.blk_first = (int)(blocks.size() / 4);
            d.n = (long long)sg->W * sg->H;
            d.Q0 = p.Q0;
            d.T = sg->T;
            d.T2 = sg->T2;
            d.rn = 1.0 / (double)d.n;
            d.inv_n = (float)d.rn;
            d.Ek = (float)sg->Ek;
            d.scale = (float)std::ldexp(1.0, -p.F);
            d.tau = tau_coarse[t];
            d.tau_exact = tau_exact[t];
            d.pix_offset = (int)pix.size();
            for (int y = 0; y < sg->H; ++y)
                pix.insert(pix.end(), templates[t] + (size_t)y * t_strides[t],
                           templates[t] + (size_t)y * t_strides[t] + sg->W);
            while (pix.size() % 16) pix.push_back(0);
            const int run_base = (int)(runs.size() / 4);  // int4 units
            const int32_t* img_blocks = p.image.data() + L.blocks_offset / 4;
            const int32_t* img_runblk = p.image.data() + L.runblk_offset / 4;
            const int32_t* img_runs = p.image.data() + L.runs_offset / 4;
            const size_t run_words = (L.end_offset - L.runs_offset) / 4;
            for (int k = 0; k < L.nblk; ++k) {
                for (int j = 0; j < 4; ++j) blocks.push_back(img_blocks[4 * k + j]);
                for (int j = 0; j < 4 * RUNBLK_INT4; ++j)  // firsts (even words) move by run_base
                    runblk.push_back(img_runblk[4 * RUNBLK_INT4 * k + j] + ((j % 2 == 0) ? run_base : 0));
            }
            runs.insert(runs.end(), img_runs, img_runs + run_words);
            b->tmpl.push_back(d);
            b->corner_counts.push_back(L.nonzero_corners);
            b->template_corners.push_back(p.template_corners);
        }
        // pairs: source-major
        std::vector<int32_t> pairs;
        std::vector<double> cost;
        for (int s = 0; s < n_sources; ++s)
            for (int t = 0; t < n_templates; ++t) {
                const TmplDesc& d = b->tmpl[t];
                const int U = M - d.W + 1, V = N - d.H + 1;
                pairs.push_back(s);
                pairs.push_back(t);
                pairs.push_back(U);
                pairs.push_back(V);
                // per-tile cost: corner sum plus region staging per block
                cost.push_back((double)b->corner_counts[t] * 8.0 + (double)d.nblk * 1600.0);
                b->corner_offsets += (double)U * V * b->template_corners[t];
                b->offsets += (double)U * V;
            }
        const int npairs = n_templates * n_sources;
        std::vector<long long> pbase(npairs);  // first sort key of each pair
        long long key_end = 0;
        for (int pi = 0; pi < npairs; ++pi) {
            pbase[pi] = key_end;
            key_end += (long long)pairs[4 * pi + 2] * pairs[4 * pi + 3];
        }
        std::vector<int> order(npairs);
        for (int i = 0; i < npairs; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
        std::vector<int32_t> items[3];
        for (int vi = 0; vi < 3; ++vi) {
            const int R = kVariants[vi];
            for (int pi : order) {
                const int U = pairs[4 * pi + 2], V = pairs[4 * pi + 3];
                const int tu = (U + TILE_U - 1) / TILE_U, tv = (V + WARPS * R - 1) / (WARPS * R);
                for (int ty = 0; ty < tv; ++ty)
                    for (int tx = 0; tx < tu; ++tx) {
                        items[vi].push_back(pi);
                        items[vi].push_back((ty << 16) | tx);
                    }
            }
            b->n_items[vi] = (int)(items[vi].size() / 2);
        }
        // device image
        size_t off = 0;
        b->off_pairs = off;
        off = align16(off + pairs.size() * 4);
        b->off_pbase = off;
        off = align16(off + pbase.size() * 8);
        b->off_tmpl = off;
        off = align16(off + b->tmpl.size() * sizeof(TmplDesc));
        b->off_blocks = off;
        off = align16(off + blocks.size() * 4);
        b->off_runblk = off;
        off = align16(off + runblk.size() * 4);
        b->off_runs = off;
        off = align16(off + runs.size() * 4);
        b->off_pix = off;
        off = align16(off + pix.size());
        for (int vi = 0; vi < 3; ++vi) {
            b->off_items[vi] = off;
            off = align16(off + items[vi].size() * 4);
        }
        b->image.assign(off, 0);
        std::memcpy(b->image.data() + b->off_pairs, pairs.data(), pairs.size() * 4);
        std::memcpy(b->image.data() + b->off_pbase, pbase.data(), pbase.size() * 8);
        std::memcpy(b->image.data() + b->off_tmpl, b->tmpl.data(), b->tmpl.size() * sizeof(TmplDesc));
        std::memcpy(b->image.data() + b->off_blocks, blocks.data(), blocks.size() * 4);
        if (!runblk.empty()) std::memcpy(b->image.data() + b->off_runblk, runblk.data(), runblk.size() * 4);
        if (!runs.empty()) std::memcpy(b->image.data() + b->off_runs, runs.data(), runs.size() * 4);
        std::memcpy(b->image.data() + b->off_pix, pix.data(), pix.size());
        for (int vi = 0; vi < 3; ++vi)
            std::memcpy(b->image.data() + b->off_items[vi], items[vi].data(), items[vi].size() * 4);
    } catch (const std::bad_alloc&) {
        delete b;
        return SNCC_ERR_NOMEM;
    }
    *out = b;
    return SNCC_OK;
}

extern "C" void sncc_batch_destroy(sncc_batch* b) { delete b; }

extern "C" size_t sncc_batch_device_bytes(const sncc_batch* b) { return b ? b->image.size() : 0; }

extern "C" int sncc_batch_upload(const sncc_batch* b, void* d_buf, size_t bytes, sncc_stream_t stream) {
    if (!b || !d_buf) return SNCC_ERR_ARG;
    if (bytes < b->image.size() || (reinterpret_cast<uintptr_t>(d_buf) & 15)) return SNCC_ERR_WORKSPACE;
    if (cudaMemcpyAsync(d_buf, b->image.data(), b->image.size(), cudaMemcpyHostToDevice, (cudaStream_t)stream) !=
        cudaSuccess)
        return SNCC_ERR_CUDA;
    return SNCC_OK;
}

extern "C" int sncc_batch_set_variant(sncc_batch* b, int tile_rows) {
    if (!b || sncc::variant_index(tile_rows) < 0) return SNCC_ERR_ARG;
    b->variant = tile_rows;
    return SNCC_OK;
}

extern "C" int sncc_batch_get_info(const sncc_batch* b, sncc_batch_info* out) {
    if (!b || !out) return SNCC_ERR_ARG;
    out->n_templates = b->nt;
    out->n_sources = b->ns;
    out->tile_rows = b->variant;
    out->tiles = b->n_items[sncc::variant_index(b->variant)];
    out->offsets = b->offsets;
    out->corner_offsets = b->corner_offsets;
    return SNCC_OK;
}

extern "C" int sncc_batch_match(const sncc_batch* b, const void* d_buf, const void* const* d_s,
                                const int64_t* const* d_s2, int s_bits, int sat_pitch, int32_t* d_cand, int cand_cap,
                                int32_t* d_count, int32_t* d_counter, int32_t* d_status, sncc_stream_t stream) {
    sncc::NvtxRange nvtx_range("sncc_batch_match");
    using namespace sncc;
    if (!b || !d_buf || !d_s || !d_s2 || !d_count || !d_counter || !d_status || cand_cap < 0) return SNCC_ERR_ARG;
    if (cand_cap > 0 && !d_cand) return SNCC_ERR_ARG;
    if ((s_bits != 32 && s_bits != 64) || sat_pitch < b->M + 1) return SNCC_ERR_ARG;
    if (s_bits == 32 && (int64_t)255 * b->M * b->N >= ((int64_t)1 << 31)) return SNCC_ERR_DTYPE;
    if (reinterpret_cast<uintptr_t>(d_buf) & 15) return SNCC_ERR_ARG;
    BatchArgs a;
    std::memset(&a, 0, sizeof(a));
    const char* base = static_cast<const char*>(d_buf);
    const int vi = variant_index(b->variant);
    a.pairs = reinterpret_cast<const int4*>(base + b->off_pairs);
    a.tmpl = reinterpret_cast<const TmplDesc*>(base + b->off_tmpl);
    a.blocks = reinterpret_cast<const int4*>(base + b->off_blocks);
    a.runblk = reinterpret_cast<const int4*>(base + b->off_runblk);
    a.runs = reinterpret_cast<const int4*>(base + b->off_runs);
    a.items = reinterpret_cast<const int2*>(base + b->off_items[vi]);
    a.n_items = b->n_items[vi];
    a.counter = d_counter;
    for (int s = 0; s < b->ns; ++s) {
        if (!d_s[s] || !d_s2[s] || (reinterpret_cast<uintptr_t>(d_s[s]) & 15)) return SNCC_ERR_ARG;
        a.s[s] = d_s[s];
        a.s2[s] = d_s2[s];
    }
    a.pitch = sat_pitch;
    a.M = b->M;
    a.N = b->N;
    a.cand = reinterpret_cast<int2*>(d_cand);
    a.cand_cap = cand_cap;
    a.count = d_count;
    a.status = d_status;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(d_count, 0, sizeof(int32_t), st) != cudaSuccess) return SNCC_ERR_CUDA;
    if (cudaMemsetAsync(d_counter, 0, sizeof(int32_t), st) != cudaSuccess) return SNCC_ERR_CUDA;
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), st) != cudaSuccess) return SNCC_ERR_CUDA;
    sncc_batch* mb = const_cast<sncc_batch*>(b);
    cudaError_t e;
    const bool s64 = (s_bits == 64);
    switch (b->variant) {
        case 8: e = s64 ? batch_launch<8, true>(mb, a, st) : batch_launch<8, false>(mb, a, st); break;
        case 4: e = s64 ? batch_launch<4, true>(mb, a, st) : batch_launch<4, false>(mb, a, st); break;
        default: e = s64 ? batch_launch<2, true>(mb, a, st) : batch_launch<2, false>(mb, a, st); break;
    }
    return e == cudaSuccess ? SNCC_OK : SNCC_ERR_CUDA;
}

extern "C" int sncc_batch_autotune(sncc_batch* b, const void* d_buf, const void* const* d_s,
                                   const int64_t* const* d_s2, int s_bits, int sat_pitch, int32_t* d_cand,
                                   int cand_cap, int32_t* d_count, int32_t* d_counter, int32_t* d_status, int reps,
                                   sncc_stream_t stream, float* ms_out) {
    using namespace sncc;
    if (!b || reps <= 0) return SNCC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SNCC_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SNCC_ERR_CUDA;
    }
    int best = 8;
    float best_ms = 3.0e38f;
    int rc = SNCC_OK;
    for (int vi = 0; vi < 3 && rc == SNCC_OK; ++vi) {
        b->variant = kVariants[vi];
        // one untimed run, then the fastest of `reps` timed runs
        rc = sncc_batch_match(b, d_buf, d_s, d_s2, s_bits, sat_pitch, d_cand, cand_cap, d_count, d_counter, d_status,
                              stream);
        float ms_v = 3.0e38f;
        for (int r = 0; r < reps && rc == SNCC_OK; ++r) {
            cudaEventRecord(e0, st);
            rc = sncc_batch_match(b, d_buf, d_s, d_s2, s_bits, sat_pitch, d_cand, cand_cap, d_count, d_counter,
                                  d_status, stream);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = SNCC_ERR_CUDA;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms_v = std::min(ms_v, ms);
        }
        if (ms_out) ms_out[vi] = ms_v;
        if (ms_v < best_ms) {
            best_ms = ms_v;
            best = kVariants[vi];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->variant = best;
    return rc;
}

namespace {
// Match records (out_cap, padded to 256 bytes), then the sort scratch over
// every pair's offsets.
size_t batch_refine_ws(const sncc_batch* b, int out_cap, size_t* sort_offset) {
    const size_t recs = ((size_t)(out_cap > 0 ? out_cap : 1) * sizeof(sncc_batch_match_t) + 255) / 256 * 256;
    if (sort_offset) *sort_offset = recs;
    return recs + sncc::sort_layout((long long)b->offsets).total;
}
}  // namespace

extern "C" size_t sncc_batch_refine_workspace_bytes(const sncc_batch* b, int out_cap) {
    if (!b || out_cap < 0) return 0;
    return batch_refine_ws(b, out_cap, nullptr);
}

extern "C" int sncc_batch_refine(const sncc_batch* b, const void* d_buf, const uint8_t* const* d_f, int f_stride,
                                 const int32_t* d_cand, const int32_t* d_count, int cand_cap,
                                 sncc_batch_match_t* d_out, int out_cap, int32_t* d_nout, void* d_ws,
                                 size_t ws_bytes, int32_t* d_status, sncc_stream_t stream) {
    sncc::NvtxRange nvtx_range("sncc_batch_refine");
    using namespace sncc;
    if (!b || !d_buf || !d_f || !d_count || !d_nout || !d_status || f_stride < b->M || cand_cap < 0 || out_cap < 0)
        return SNCC_ERR_ARG;
    if ((cand_cap > 0 && !d_cand) || (out_cap > 0 && !d_out)) return SNCC_ERR_ARG;
    if (out_cap > 0 && (!d_ws || ws_bytes < sncc_batch_refine_workspace_bytes(b, out_cap) ||
                        (reinterpret_cast<uintptr_t>(d_ws) & 15)))
        return SNCC_ERR_WORKSPACE;
    BatchRefineArgs a;
    std::memset(&a, 0, sizeof(a));
    const char* base = static_cast<const char*>(d_buf);
    a.pairs = reinterpret_cast<const int4*>(base + b->off_pairs);
    a.tmpl = reinterpret_cast<const TmplDesc*>(base + b->off_tmpl);
    a.pix = reinterpret_cast<const uint8_t*>(base + b->off_pix);
    for (int s = 0; s < b->ns; ++s) {
        if (!d_f[s]) return SNCC_ERR_ARG;
        a.f[s] = d_f[s];
    }
    a.f_stride = f_stride;
    a.cand = reinterpret_cast<const int2*>(d_cand);
    a.count = d_count;
    a.cand_cap = cand_cap;
    a.scratch = static_cast<sncc_batch_match_t*>(d_ws);
    a.scratch_cap = out_cap;
    a.nout = d_nout;
    a.status = d_status;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(d_nout, 0, sizeof(int32_t), st) != cudaSuccess) return SNCC_ERR_CUDA;
    if (cand_cap == 0) return SNCC_OK;
    const int cap_ctas = 8 * (sm_count() > 0 ? sm_count() : 1);
    const int grid = cand_cap < cap_ctas ? cand_cap : cap_ctas;
    batch_refine_kernel<<<grid, 256, 0, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return SNCC_ERR_CUDA;
    if (out_cap > 0) {
        size_t sort_off = 0;
        batch_refine_ws(b, out_cap, &sort_off);
        const BatchKey key{a.pairs, reinterpret_cast<const long long*>(base + b->off_pbase)};
        if (launch_sorted_compaction(a.scratch, d_nout, out_cap, key, (long long)b->offsets,
                                     static_cast<char*>(d_ws) + sort_off, d_out, cap_ctas, st) != cudaSuccess)
            return SNCC_ERR_CUDA;
    }
    return SNCC_OK;
}
