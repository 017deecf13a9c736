// sncc_internal.h - private declarations shared by the library's translation
// units (host plan layout, tile geometry, launch helpers).  Not installed.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "sncc.h"

namespace sncc {

// Devices whose one-time kernel set-up is remembered (ordinals beyond this
// repeat it on every call, which is still correct).
constexpr int kDeviceSlots = 128;

// Runs `set` (a callable returning cudaError_t) for the current device
// unless it already succeeded there.  Kernel attributes such as the opt-in
// shared-memory limit, and occupancy figures, belong to a device, so a
// process that uses several GPUs sets them on each.
template <typename F>
cudaError_t once_per_device(std::atomic<int> (&done)[kDeviceSlots], F&& set) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool slot = dev >= 0 && dev < kDeviceSlots;
    if (slot && done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    e = set();
    if (e == cudaSuccess && slot) done[dev].store(1, std::memory_order_release);
    return e;
}

// True when p is not a multiple of `bytes` (a power of two).  Entry points
// reject such device pointers before any launch: the kernels load and store
// them by their element type (4, 8 or 16 bytes), and a misaligned access is
// a device fault, not an error code.
inline bool misaligned(const void* p, size_t bytes) {
    return (reinterpret_cast<uintptr_t>(p) & (bytes - 1)) != 0;
}

// An NVTX range around one ABI call (visible to profilers; a no-op otherwise).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------------------
// Segment-sum tile geometry.
//
// A CTA of 8 warps computes a tile of TILE_U x (8 * R) offsets: lane l of warp
// w owns offsets (u0 + l, v0 + w*R + r), r < R.  The template is cut into
// blocks of at most BLOCK x BLOCK pixels; for each block the CTA stages the
// sum-table region its offsets touch, (TILE_U + bw + 1) x (8R + bh + 1)
// entries, re-based to the region's own origin so every entry fits in 32 bits.
// ---------------------------------------------------------------------------
constexpr int TILE_U = 32;
constexpr int WARPS = 8;
constexpr int BLOCK_SINGLE_MAX = 64;  // a template up to 64 x 64 is one block
constexpr int BLOCK_MULTI = 32;       // first layout of larger templates: 32 x 32 blocks
constexpr int PAIR_MIN_GAP = 2, PAIR_MAX_GAP = 7;  // gaps of the corner-pair records
constexpr int PAIR_GAPS = PAIR_MAX_GAP - PAIR_MIN_GAP + 1;

// Host-side matching plan (built by sncc_build_segments).
//
// The zero-mean segment values c_i = k_i - kbar are quantised to
// q_i = round(c_i * 2^F).  With q(x, y) the rendered image of q_i, the kernel
// computes the exact integer correlation A(u, v) = sum_{x,y} q(x,y) f(u+x, v+y)
// as a sparse sum over corner points of each block:
//   A = sum_blocks sum_p G_p * s(u + bx + X_p, v + by + Y_p),
//   G(X, Y) = q(X-1, Y-1) - q(X, Y-1) - q(X-1, Y) + q(X, Y)   (block-local,
// q = 0 outside the block), i.e. Eq. 11 applied to every segment and summed,
// with the shared corners of neighbouring segments combined.
// One way of cutting the template into blocks, with its corner lists.
// Device image section (offsets in bytes from the start of the plan image,
// each array 16-byte aligned):
//  * int4 blocks[nblk] = {bx, by, first, count};
//  * int2 corners[total] = {Y * WP + X, G}, the plain corner list; each
//    block's list starts on a multiple of 4 corners and is padded with zero
//    weights to a multiple of 4;
//  * int4 runblk[RUNBLK_INT4 * nblk] = {first8, n8, first4, n4}, {first2,
//    n2, first1, n1}, {firstp2, np2, firstp3, np3}, {firstp4, np4, firstp5,
//    np5}, {firstp6, np6, firstp7, np7}, {firsts8, ns8, firsts4, ns4},
//    {firsts3, ns3, firstt, nt}: the same corners of block b regrouped into
//    vertical runs (a run of L corners occupies rows Y .. Y+L-1 of one
//    column X, every weight nonzero), stride-2 runs of 8, 4 and 3 (rows Y,
//    Y+2, .., none between), the rows-(Y, Y+2, Y+3) pattern, pairs (two
//    corners of one column D = 2 .. 7 rows apart, with no corner between
//    them) and single corners; first* index int4 units of runs[];
//  * int4 runs[]: a run of 8 is {idx, G0, G1, G2} {G3, G4, G5, G6}
//    {G7, 0, 0, 0}, a run of 4 is {idx, G0, G1, G2} {G3, 0, 0, 0}, a run of
//    2 is {idx, G0, G1, 0}, a pair is {idx, G0, G1, 0} (G1 at row Y + D),
//    stride-2 runs are laid out as runs of the same length, the (0, 2, 3)
//    pattern is {idx, G0, G1, G2},
//    with idx = 4 (Y * WP + X), the byte offset of the record's first word
//    in the region; single corners are int2 {idx, G}, two per int4, padded
//    with zero weights to a multiple of 4 (n1 counts corners, not int4
//    units).  A lane computing R offset rows reads R + L - 1 words for a run
//    of L, R + D for a pair and R for a single corner.
struct Layout {
    int BW = 0, BH = 0;     // block size (the last block in a row/column may be smaller)
    int nbx = 0, nby = 0;   // blocks across / down
    int nblk = 0;           // blocks that hold at least one corner (the others are dropped)
    int WP = 0;             // pitch (elements) of the re-based work region: 68 (BW <= 32) or 100
    int max_corners = 0;    // largest corner count of one block
    int total_corners = 0;  // including the zero-weight padding
    int nonzero_corners = 0;
    int runs[4] = {0, 0, 0, 0};  // vertical runs of 8, 4, 2 and 1 corners, over all blocks
    int pairs[PAIR_GAPS] = {};   // pairs of corners D = 2 .. 7 rows apart, over all blocks
    int runs2[3] = {0, 0, 0};    // stride-2 runs of 8, 4 and 3 corners, over all blocks
    int t21 = 0;                 // rows-(0, 2, 3) patterns, over all blocks
    int records = 0;             // run, pair and single-corner records, over all blocks
    long long extra_rows = 0;    // sum over records of the rows spanned beyond the first
    size_t blocks_offset = 0;
    size_t corners_offset = 0;
    size_t runblk_offset = 0;
    size_t runs_offset = 0;
    size_t end_offset = 0;  // one past the section
};

struct Plan {
    int W = 0, H = 0;
    int F = 0;              // fixed-point fraction bits of q_i
    int64_t Q0 = 0;         // sum over the template of q(x, y)
    double Ek = 0.0;        // weighted energy of the approximation
    double n = 0.0;         // W * H
    int template_corners = 0;  // corners of the whole template taken as one block
    // lay[0]: a template up to 64 x 64 is one block (pitch 68 when it is at
    // most 32 wide, else 100), the segment-sum kernel's layout for it;
    // larger ones use 32 x 32 blocks (pitch 68), read by the per-candidate
    // fine pass.  lay[1]: blocks of at most 64 x 64 with pitch 100, the
    // segment-sum kernels' layout for templates larger than 64 x 64 (fewer,
    // larger blocks halve the staged entries per corner).  lay[2] (built on
    // request, for the batched kernel): blocks of at most 32 x 32 with pitch
    // 68 for every template size.
    Layout lay[3];
    // Templates with at most DIRECT_MAX corners in all also carry their
    // whole-template corner list, int4 {X, Y, G, 0}, at direct_offset: the
    // segment-sum kernel then reads the table at those corners directly
    // instead of staging block regions (direct_count = 0 otherwise).
    int direct_count = 0;
    size_t direct_offset = 0;
    std::vector<int32_t> image;  // both layouts, the direct list, then 4 zero words
};

constexpr int DIRECT_MAX = SNCC_DIRECT_MAX_CORNERS;

// Lengths of the vertical corner runs and the int4 units one run occupies.
constexpr int RUN_LEN[4] = {8, 4, 2, 1};
constexpr int RUN_INT4[3] = {3, 2, 1};
// int4 descriptors per block (runblk), and the pair gaps 2 .. 7.
constexpr int RUNBLK_INT4 = 7;
// Stride-2 runs (corners every second row, none between) of 8, 4 and 3.
constexpr int RUN2_LEN[3] = {8, 4, 3};

Plan* plan_of(const sncc_segments* s);

// Fills p from seg's segment table (defined in sncc_host.cpp); with
// small_blocks, also lay[2].
int build_plan(const sncc_segments* seg, Plan& p, bool small_blocks = false);

// The layout the single-problem segment-sum kernel uses: one block for a
// template up to 64 x 64, else 64 x 64 blocks.
inline const Layout& layout_for(const Plan& p) { return (p.lay[0].nbx * p.lay[0].nby > 1) ? p.lay[1] : p.lay[0]; }

// Writes the first min(*d_n, cap) records of `in` to `out` in ascending
// v*U+u order (keys are distinct), with match_sort_bytes(U, V) bytes of
// scratch at sort_ws (16-byte aligned).  Defined in sncc_refine.cu.
size_t match_sort_bytes(int U, int V);
cudaError_t launch_match_sort(const sncc_match_t* in, const int32_t* d_n, int cap, int U, int V, void* sort_ws,
                              sncc_match_t* out, cudaStream_t st);

// Workspace of sncc_refine and sncc_refine_segmented: out_cap match records
// (padded to 256 bytes), then the sort scratch at *sort_offset.
size_t refine_workspace_bytes(int M, int N, int W, int H, int out_cap, size_t* sort_offset);

// Status helpers.
const char* error_string(int code);

// Streaming multiprocessors of the current device, queried once per device
// (grid sizes and tile heights are chosen against it); 0 if the query fails.
int sm_count();

// Whether sncc_match_multi can fuse these n approximations into one launch,
// decided on the host alone: SNCC_OK, SNCC_ERR_UNSUPPORTED (not fusable),
// SNCC_ERR_UNIFORM (some Ek = 0) or SNCC_ERR_ARG.  Defined in sncc_match.cu.
int multi_fusable(const sncc_segments* const* segs, const void* const* d_plans, int n);

}  // namespace sncc
