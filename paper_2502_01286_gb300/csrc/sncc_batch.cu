// sncc_batch.cu - many templates against several sources in one persistent
// launch: the coarse pass of segmented NCC (Eq. 9 - Eq. 18, main algorithm
// steps 7a-7f) for every (source, template) pair, then the exact refine of
// all candidates (Eq. 1, steps 7g-7j with an exact second stage).
//
// Design:
//  * Host: every template's plan is rebuilt with two block layouts: blocks
//    of at most 64 x 64 (region pitch 100) and of at most 32 x 32 (pitch 68),
//    so that one kernel serves templates of any size.  Templates fall into
//    buckets by size (one 64 x 64 block, up to 4, more) and corner density
//    (corners per template pixel below 0.1, below 0.5, above).  Every
//    bucket has a variant: the tile height R in {8, 4, 2} (offset rows per
//    lane) and the block edge, 64 or 32 (corners per staging pass).  A work
//    list of tiles (pair, tile column, tile row) is built for every bucket
//    and tile height, ordered by estimated cost, largest first.
//  * Device: per variant in use, a persistent grid (occupancy x SMs) of
//    8-warp CTAs pulls tiles with one atomic per tile from the lists of the
//    buckets in that variant, one after another (heaviest bucket first, so
//    that the dynamic schedule ends with cheap tiles); each tile runs the
//    staging / corner-sum / normalisation code of the single-problem kernel
//    (sncc_tile.cuh), with the sources staged through registers.  One
//    kernel instance per variant keeps each at its own register count.
//    Candidates are appended as (pair, v*U+u) with warp-aggregated atomics.
//  * The variants are chosen per bucket by an autotuner that times each
//    bucket alone in every variant on the caller's data
//    (sncc_batch_autotune), or given explicitly.
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
constexpr int kBatchWP32 = 68;  // region pitch of 32 x 32 blocks
constexpr int kBatchBlock = 64;
constexpr int kVariants[3] = {8, 4, 2};
constexpr int kBuckets = SNCC_BATCH_BUCKETS;
constexpr int kBatchVariants = SNCC_BATCH_VARIANTS;  // variant v: R = kVariants[v % 3], block edge 64 >> (v / 3)

struct TmplDesc {  // 96 bytes, one per template
    int W, H;
    int nblk[2], blk_first[2];  // the 64 x 64 and the 32 x 32 block layouts
    long long n, Q0;
    long long T, T2;
    float inv_n, Ek, scale, tau;
    float tau_exact;
    int pix_offset;
    double rn;  // 1 / n in FP64
    int bucket, pad;
};
static_assert(sizeof(TmplDesc) == 96, "template descriptor layout");

// One bucket's share of a launch: items [first, first + count) of the item
// array (its list for tile height R), evaluated with R and the block edge.
struct BucketRun {
    int first, count, R, blk;
};

struct BatchArgs {
    const int4* pairs;  // {source, template, U, V}
    const TmplDesc* tmpl;
    const int4* blocks;
    const int4* runblk;  // RUNBLK_INT4 per block
    const int4* runs;
    const int2* items;  // {pair, (tile row << 16) | tile column}
    BucketRun run[kBuckets];  // in launch order
    int nruns;
    int n_items;  // over all runs
    int* counter;
    const void* s[SNCC_BATCH_MAX_SOURCES];
    const int64_t* s2[SNCC_BATCH_MAX_SOURCES];
    int pitch, M, N;
    int2* cand;
    int cand_cap;
    int* count;
    int* status;
};

// One tile of a pair with tile height R and region pitch WP (block edge 64
// for pitch 100, 32 for pitch 68; lay indexes the template's layout).
template <int R, int WP, bool S64>
__device__ __forceinline__ void batch_tile(const BatchArgs& a, int* work, int2 item, int lane, int warp) {
    constexpr int lay = (WP == kBatchWP) ? 0 : 1;
    constexpr int BB = (WP == kBatchWP) ? kBatchBlock : kBatchBlock / 2;
    const int4 pd = a.pairs[item.x];
    const TmplDesc& td = a.tmpl[pd.y];
    const int u0 = (item.y & 0xffff) * TILE_U, v0 = (item.y >> 16) * (WARPS * R);
    const void* s = a.s[pd.x];
    const int64_t* s2 = a.s2[pd.x];
    const int* wbase = work + warp * R * WP + lane;
    long long acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0;
    const int nblk = td.nblk[lay], first = td.blk_first[lay];
    for (int b = 0; b < nblk; ++b) {
        const int4 blk = a.blocks[first + b];
        const int bw = min(BB, td.W - blk.x), bh = min(BB, td.H - blk.y);
        stage_region_regs<S64, WP>(s, a.pitch, a.M, a.N, work, u0 + blk.x, v0 + blk.y, WARPS * R + bh + 1, lane, warp,
                                   TILE_U + bw + 1);
        __syncthreads();
        run_sum<R, WP>(acc, wbase, a.runs, a.runblk + RUNBLK_INT4 * (first + b));
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

// The persistent coarse pass of one variant (tile height R, region pitch
// WP) over the buckets listed in a.run.
template <int R, int WP, bool S64>
__global__ void __launch_bounds__(WARPS * 32) batch_match_kernel(const __grid_constant__ BatchArgs a) {
    extern __shared__ __align__(16) int work[];
    __shared__ int item_sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (;;) {
        if (tid == 0) item_sh = atomicAdd(a.counter, 1);
        __syncthreads();
        const int it = item_sh;
        __syncthreads();  // item_sh is rewritten only after every thread has read it
        if (it >= a.n_items) break;
        // the bucket run the item falls in (uniform per CTA)
        int k = 0, base = 0;
        while (k + 1 < a.nruns && it >= base + a.run[k].count) {
            base += a.run[k].count;
            ++k;
        }
        batch_tile<R, WP, S64>(a, work, a.items[a.run[k].first + (it - base)], lane, warp);
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
           off_items = 0;
    // items of bucket k for tile height kVariants[vi]: int2 units from item_first[k][vi]
    int item_first[sncc::kBuckets][3] = {};
    int item_count[sncc::kBuckets][3] = {};
    int bucket_templates[sncc::kBuckets] = {}, bucket_pairs[sncc::kBuckets] = {};
    double bucket_corner_offsets[sncc::kBuckets] = {};
    int bucket_order[sncc::kBuckets] = {};  // launch order: heaviest tiles first
    int variant[sncc::kBuckets] = {};       // chosen variant of every bucket
    float tuned_ms[sncc::kBuckets][sncc::kBatchVariants] = {};
    std::vector<unsigned char> image;
    double corner_offsets = 0.0;  // sum over pairs of U*V*(corners of the whole template)
    double offsets = 0.0;         // sum over pairs of U*V
};

namespace sncc {
namespace {

int variant_index(int R) { return R == 8 ? 0 : (R == 4 ? 1 : (R == 2 ? 2 : -1)); }
int variant_of(int R, int blk) {
    const int vi = variant_index(R);
    if (vi < 0 || (blk != kBatchBlock && blk != kBatchBlock / 2)) return -1;
    return vi + (blk == kBatchBlock ? 0 : 3);
}

// Shared memory of a variant: the region of one block for 8R offset rows.
template <int R, int WP>
constexpr size_t batch_smem() {
    return (size_t)(WARPS * R + (WP == kBatchWP ? kBatchBlock : kBatchBlock / 2) + 1) * WP * 4;
}

// Bucket of a template: size class (one 64 x 64 block, up to 4, more) x
// corner density (corners per template pixel below 0.1, below 0.5, above:
// sparse approximations of smooth or textured templates, mixed, and
// approximations close to the pixels).
int bucket_of(int W, int H, int corners) {
    const int nb = ((W + kBatchBlock - 1) / kBatchBlock) * ((H + kBatchBlock - 1) / kBatchBlock);
    const int sc = nb == 1 ? 0 : (nb <= 4 ? 1 : 2);
    const double d = (double)corners / ((double)W * H);
    const int dc = d < 0.1 ? 0 : (d < 0.5 ? 1 : 2);
    return sc * 3 + dc;
}

template <int R, int WP, bool S64>
cudaError_t batch_launch(const BatchArgs& args, cudaStream_t st) {
    static std::atomic<int> done[kDeviceSlots];
    static std::atomic<int> per_sm_of[kDeviceSlots];  // resident CTAs per SM, per device
    constexpr size_t smem = batch_smem<R, WP>();
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
    const bool slot = dev >= 0 && dev < kDeviceSlots;
    int per_sm = slot ? per_sm_of[dev].load(std::memory_order_relaxed) : 0;
    const cudaError_t attr = once_per_device(done, [&] {
        cudaError_t e = cudaFuncSetAttribute(batch_match_kernel<R, WP, S64>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_match_kernel<R, WP, S64>, WARPS * 32,
                                                              smem);
        if (e == cudaSuccess && slot) per_sm_of[dev].store(per_sm, std::memory_order_relaxed);
        return e;
    });
    if (attr != cudaSuccess) return attr;
    const int grid = std::max(1, per_sm) * std::max(1, sm_count());
    batch_match_kernel<R, WP, S64><<<grid, WARPS * 32, smem, st>>>(args);
    return cudaGetLastError();
}

template <bool S64>
cudaError_t batch_launch_variant(int v, const BatchArgs& args, cudaStream_t st) {
    switch (v) {
        case 0: return batch_launch<8, kBatchWP, S64>(args, st);
        case 1: return batch_launch<4, kBatchWP, S64>(args, st);
        case 2: return batch_launch<2, kBatchWP, S64>(args, st);
        case 3: return batch_launch<8, kBatchWP32, S64>(args, st);
        case 4: return batch_launch<4, kBatchWP32, S64>(args, st);
        default: return batch_launch<2, kBatchWP32, S64>(args, st);
    }
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
            build_plan(sg, p, true);
            const Layout& L = p.lay[1];  // blocks of at most 64 x 64, pitch 100
            TmplDesc d;
            std::memset(&d, 0, sizeof(d));
            d.W = sg->W;
            d.H = sg->H;
            d.bucket = bucket_of(sg->W, sg->H, p.template_corners);
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
            for (int li = 0; li < 2; ++li) {  // the 64 x 64 and the 32 x 32 block layouts
                const Layout& Ll = p.lay[li == 0 ? 1 : 2];
                d.nblk[li] = Ll.nblk;
                d.blk_first[li] = (int)(blocks.size() / 4);
                const int run_base = (int)(runs.size() / 4);  // int4 units
                const int32_t* img_blocks = p.image.data() + Ll.blocks_offset / 4;
                const int32_t* img_runblk = p.image.data() + Ll.runblk_offset / 4;
                const int32_t* img_runs = p.image.data() + Ll.runs_offset / 4;
                const size_t run_words = (Ll.end_offset - Ll.runs_offset) / 4;
                for (int k = 0; k < Ll.nblk; ++k) {
                    for (int j = 0; j < 4; ++j) blocks.push_back(img_blocks[4 * k + j]);
                    for (int j = 0; j < 4 * RUNBLK_INT4; ++j)  // firsts (even words) move by run_base
                        runblk.push_back(img_runblk[4 * RUNBLK_INT4 * k + j] + ((j % 2 == 0) ? run_base : 0));
                }
                runs.insert(runs.end(), img_runs, img_runs + run_words);
            }
            b->bucket_templates[d.bucket] += 1;
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
                cost.push_back((double)b->corner_counts[t] * 8.0 + (double)d.nblk[0] * 1600.0);
                b->corner_offsets += (double)U * V * b->template_corners[t];
                b->offsets += (double)U * V;
                b->bucket_pairs[d.bucket] += 1;
                b->bucket_corner_offsets[d.bucket] += (double)U * V * b->template_corners[t];
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
        // per bucket and tile height, that bucket's tiles, costliest pairs first
        std::vector<int32_t> items;
        double bucket_cost[kBuckets] = {};
        for (int k = 0; k < kBuckets; ++k) {
            for (int vi = 0; vi < 3; ++vi) {
                const int R = kVariants[vi];
                b->item_first[k][vi] = (int)(items.size() / 2);
                for (int pi : order) {
                    if (b->tmpl[pairs[4 * pi + 1]].bucket != k) continue;
                    if (vi == 0) bucket_cost[k] = std::max(bucket_cost[k], cost[pi]);
                    const int U = pairs[4 * pi + 2], V = pairs[4 * pi + 3];
                    const int tu = (U + TILE_U - 1) / TILE_U, tv = (V + WARPS * R - 1) / (WARPS * R);
                    for (int ty = 0; ty < tv; ++ty)
                        for (int tx = 0; tx < tu; ++tx) {
                            items.push_back(pi);
                            items.push_back((ty << 16) | tx);
                        }
                }
                b->item_count[k][vi] = (int)(items.size() / 2) - b->item_first[k][vi];
            }
            b->variant[k] = 0;  // R = 8, 64 x 64 blocks until tuned or set
            b->bucket_order[k] = k;
        }
        std::stable_sort(b->bucket_order, b->bucket_order + kBuckets,
                         [&](int x, int y) { return bucket_cost[x] > bucket_cost[y]; });
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
        b->off_items = off;
        off = align16(off + items.size() * 4);
        b->image.assign(off, 0);
        std::memcpy(b->image.data() + b->off_pairs, pairs.data(), pairs.size() * 4);
        std::memcpy(b->image.data() + b->off_pbase, pbase.data(), pbase.size() * 8);
        std::memcpy(b->image.data() + b->off_tmpl, b->tmpl.data(), b->tmpl.size() * sizeof(TmplDesc));
        std::memcpy(b->image.data() + b->off_blocks, blocks.data(), blocks.size() * 4);
        if (!runblk.empty()) std::memcpy(b->image.data() + b->off_runblk, runblk.data(), runblk.size() * 4);
        if (!runs.empty()) std::memcpy(b->image.data() + b->off_runs, runs.data(), runs.size() * 4);
        std::memcpy(b->image.data() + b->off_pix, pix.data(), pix.size());
        if (!items.empty()) std::memcpy(b->image.data() + b->off_items, items.data(), items.size() * 4);
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
    for (int k = 0; k < sncc::kBuckets; ++k) b->variant[k] = sncc::variant_of(tile_rows, sncc::kBatchBlock);
    return SNCC_OK;
}

extern "C" int sncc_batch_set_bucket_variant(sncc_batch* b, int bucket, int tile_rows, int block) {
    if (!b || bucket < 0 || bucket >= sncc::kBuckets) return SNCC_ERR_ARG;
    const int v = sncc::variant_of(tile_rows, block);
    if (v < 0) return SNCC_ERR_ARG;
    b->variant[bucket] = v;
    return SNCC_OK;
}

extern "C" int sncc_batch_get_info(const sncc_batch* b, sncc_batch_info* out) {
    using namespace sncc;
    if (!b || !out) return SNCC_ERR_ARG;
    out->n_templates = b->nt;
    out->n_sources = b->ns;
    int R = -1, tiles = 0;
    for (int k = 0; k < kBuckets; ++k) {
        if (b->bucket_pairs[k] == 0) continue;
        const int vi = b->variant[k] % 3;
        tiles += b->item_count[k][vi];
        R = (R == -1 || R == kVariants[vi]) ? kVariants[vi] : 0;
    }
    out->tile_rows = R < 0 ? 0 : R;
    out->tiles = tiles;
    out->offsets = b->offsets;
    out->corner_offsets = b->corner_offsets;
    return SNCC_OK;
}

extern "C" int sncc_batch_get_bucket(const sncc_batch* b, int bucket, sncc_batch_bucket* out) {
    using namespace sncc;
    if (!b || !out || bucket < 0 || bucket >= kBuckets) return SNCC_ERR_ARG;
    out->templates = b->bucket_templates[bucket];
    out->pairs = b->bucket_pairs[bucket];
    out->size_class = bucket / 3;
    out->density_class = bucket % 3;
    out->tile_rows = kVariants[b->variant[bucket] % 3];
    out->block = b->variant[bucket] < 3 ? kBatchBlock : kBatchBlock / 2;
    out->corner_offsets = b->bucket_corner_offsets[bucket];
    for (int v = 0; v < kBatchVariants; ++v) out->ms[v] = b->tuned_ms[bucket][v];
    return SNCC_OK;
}

namespace {

// The coarse pass over the buckets in `which` (all when which < 0, else
// that bucket alone), each with its variant.
int batch_match_run(const sncc_batch* b, const void* d_buf, const void* const* d_s, const int64_t* const* d_s2,
                    int s_bits, int sat_pitch, int32_t* d_cand, int cand_cap, int32_t* d_count, int32_t* d_counter,
                    int32_t* d_status, int which, sncc_stream_t stream) {
    using namespace sncc;
    if (!b || !d_buf || !d_s || !d_s2 || !d_count || !d_counter || !d_status || cand_cap < 0) return SNCC_ERR_ARG;
    if (cand_cap > 0 && !d_cand) return SNCC_ERR_ARG;
    if ((s_bits != 32 && s_bits != 64) || sat_pitch < b->M + 1 || (sat_pitch & 3)) return SNCC_ERR_ARG;
    if (misaligned(d_buf, 16) || misaligned(d_cand, 8) || misaligned(d_count, 4) || misaligned(d_counter, 4) ||
        misaligned(d_status, 4))
        return SNCC_ERR_ARG;
    BatchArgs a;
    std::memset(&a, 0, sizeof(a));
    const char* base = static_cast<const char*>(d_buf);
    a.pairs = reinterpret_cast<const int4*>(base + b->off_pairs);
    a.tmpl = reinterpret_cast<const TmplDesc*>(base + b->off_tmpl);
    a.blocks = reinterpret_cast<const int4*>(base + b->off_blocks);
    a.runblk = reinterpret_cast<const int4*>(base + b->off_runblk);
    a.runs = reinterpret_cast<const int4*>(base + b->off_runs);
    a.items = reinterpret_cast<const int2*>(base + b->off_items);
    a.counter = d_counter;
    for (int s = 0; s < b->ns; ++s) {
        if (!d_s[s] || !d_s2[s] || misaligned(d_s[s], 16) || misaligned(d_s2[s], 8)) return SNCC_ERR_ARG;
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
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), st) != cudaSuccess) return SNCC_ERR_CUDA;
    // one persistent launch per variant in use, over its buckets (heaviest
    // bucket first), the variants in the order of their heaviest buckets
    bool launched[kBatchVariants] = {};
    for (int j = 0; j < kBuckets; ++j) {
        const int k0 = b->bucket_order[j];
        if (b->bucket_pairs[k0] == 0 || (which >= 0 && k0 != which)) continue;
        const int v = b->variant[k0];
        if (launched[v]) continue;
        launched[v] = true;
        a.nruns = 0;
        a.n_items = 0;
        for (int jj = j; jj < kBuckets; ++jj) {
            const int k = b->bucket_order[jj];
            if (b->bucket_pairs[k] == 0 || (which >= 0 && k != which) || b->variant[k] != v) continue;
            BucketRun& r = a.run[a.nruns++];
            r.first = b->item_first[k][v % 3];
            r.count = b->item_count[k][v % 3];
            r.R = kVariants[v % 3];
            r.blk = v < 3 ? kBatchBlock : kBatchBlock / 2;
            a.n_items += r.count;
        }
        if (a.n_items == 0) continue;
        if (cudaMemsetAsync(d_counter, 0, sizeof(int32_t), st) != cudaSuccess) return SNCC_ERR_CUDA;
        const cudaError_t e = (s_bits == 64) ? batch_launch_variant<true>(v, a, st) : batch_launch_variant<false>(v, a, st);
        if (e != cudaSuccess) return SNCC_ERR_CUDA;
    }
    return SNCC_OK;
}

}  // namespace

extern "C" int sncc_batch_match(const sncc_batch* b, const void* d_buf, const void* const* d_s,
                                const int64_t* const* d_s2, int s_bits, int sat_pitch, int32_t* d_cand, int cand_cap,
                                int32_t* d_count, int32_t* d_counter, int32_t* d_status, sncc_stream_t stream) {
    sncc::NvtxRange nvtx_range("sncc_batch_match");
    return batch_match_run(b, d_buf, d_s, d_s2, s_bits, sat_pitch, d_cand, cand_cap, d_count, d_counter, d_status,
                           -1, stream);
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
    int rc = SNCC_OK;
    for (int k = 0; k < kBuckets && rc == SNCC_OK; ++k) {
        for (int v = 0; v < kBatchVariants; ++v) b->tuned_ms[k][v] = 0.0f;
        if (b->bucket_pairs[k] == 0) continue;
        int best = b->variant[k];
        float best_ms = 3.0e38f;
        for (int v = 0; v < kBatchVariants && rc == SNCC_OK; ++v) {
            b->variant[k] = v;
            // the bucket alone in variant v: one untimed run, then the fastest of `reps`
            rc = batch_match_run(b, d_buf, d_s, d_s2, s_bits, sat_pitch, d_cand, cand_cap, d_count, d_counter,
                                 d_status, k, stream);
            float ms_v = 3.0e38f;
            for (int r = 0; r < reps && rc == SNCC_OK; ++r) {
                cudaEventRecord(e0, st);
                rc = batch_match_run(b, d_buf, d_s, d_s2, s_bits, sat_pitch, d_cand, cand_cap, d_count, d_counter,
                                     d_status, k, stream);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) rc = SNCC_ERR_CUDA;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms_v = std::min(ms_v, ms);
            }
            b->tuned_ms[k][v] = ms_v;
            if (ms_v < best_ms) {
                best_ms = ms_v;
                best = v;
            }
        }
        b->variant[k] = best;
    }
    if (ms_out)
        for (int k = 0; k < kBuckets; ++k)
            for (int v = 0; v < kBatchVariants; ++v) ms_out[k * kBatchVariants + v] = b->tuned_ms[k][v];
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
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
    if (misaligned(d_buf, 16) || misaligned(d_cand, 8) || misaligned(d_count, 4) || misaligned(d_out, 4) ||
        misaligned(d_nout, 4) || misaligned(d_status, 4))
        return SNCC_ERR_ARG;
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
