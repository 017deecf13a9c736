// sncc_sort.cuh - match lists written in ascending offset order in
// O(keys / 32 + n) work: one bit per key of the offset space, a prefix count
// of the set bits, and a scatter of every record to its rank.  Short lists
// (at most kSortSmall records) are ranked by direct comparison instead,
// which costs less than a pass over the bit array.
//
// The records are the first min(*d_n, cap) entries of `in`, with distinct
// keys in [0, nkeys); the caller gives the key of a record by a functor.
// Device work, in stream order (four launches, no host synchronisation):
//   1. clear the bit array and the block counter (one memset);
//   2. sort_mark: short list - rank by comparison and write `out`; else set
//      the bit of every record's key;
//   3. sort_scan: per block of kScanWords words the exclusive prefix of the
//      set-bit counts of its words, then the last block to finish turns the
//      block totals into their exclusive prefix;
//   4. sort_scatter: out[block prefix + word prefix + bits below] = record.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace sncc {

constexpr int kSortSmall = 2048;      // at most this many records: rank by comparison
constexpr int kSortThreads = 256;
constexpr int kScanWords = 4 * kSortThreads;  // bit-array words per scan block

// Byte layout of the sort scratch for a key space of nkeys keys (offsets
// from the scratch start, each 256-byte aligned).  The memset covers
// [bits, bits_end): the bit array (padded to whole scan blocks) and the
// block counter.
struct SortLayout {
    long long nwords = 0;  // 32-bit words of the bit array (a multiple of kScanWords)
    int nblocks = 0;       // scan blocks
    size_t bits = 0, counter = 0, bits_end = 0, wpre = 0, bpre = 0, total = 0;
};

inline SortLayout sort_layout(long long nkeys) {
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    SortLayout L;
    const long long words = (nkeys + 31) / 32;
    L.nblocks = (int)((words + kScanWords - 1) / kScanWords);
    if (L.nblocks < 1) L.nblocks = 1;
    L.nwords = (long long)L.nblocks * kScanWords;
    size_t o = 0;
    L.bits = o;
    o += (size_t)L.nwords * 4;
    L.counter = o;
    o += 16;
    L.bits_end = o;
    o = al(o);
    L.wpre = o;
    o = al(o + (size_t)L.nwords * 4);
    L.bpre = o;
    o = al(o + (size_t)L.nblocks * 4);
    L.total = o;
    return L;
}

// The kernels have internal linkage: each translation unit that includes
// this header gets its own copies.
namespace {
namespace sortk {

// Short list: out[rank(i)] = in[i], rank = records with a smaller key (the
// grid's first n / kSortThreads CTAs; keys staged in shared memory by
// chunks).  Long list: the bit of every key.
template <class Rec, class KeyFn>
__global__ void __launch_bounds__(kSortThreads)
    sort_mark(const Rec* __restrict__ in, const int32_t* __restrict__ d_n, int cap, KeyFn key,
              uint32_t* __restrict__ bits, Rec* __restrict__ out) {
    constexpr int CH = 1024;
    __shared__ long long keys[CH];
    const int n = min(*d_n, cap);
    if (n <= kSortSmall) {
        const int i = blockIdx.x * blockDim.x + threadIdx.x;
        if (blockIdx.x * blockDim.x >= n) return;  // uniform per CTA
        const bool mine = i < n;
        Rec me;
        long long k = 0;
        if (mine) {
            me = in[i];
            k = key(me);
        }
        int rank = 0;
        for (int c0 = 0; c0 < n; c0 += CH) {
            const int len = min(CH, n - c0);
            __syncthreads();
            for (int j = threadIdx.x; j < len; j += blockDim.x) keys[j] = key(in[c0 + j]);
            __syncthreads();
            if (mine)
                for (int j = 0; j < len; ++j) rank += (keys[j] < k) ? 1 : 0;
        }
        if (mine) out[rank] = me;
        return;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const long long k = key(in[i]);
        atomicOr(bits + (k >> 5), 1u << (k & 31));
    }
}

// Exclusive scan of v over the CTA (kSortThreads threads); returns the
// CTA's total through *total.
__device__ __forceinline__ int cta_exclusive_scan(int v, int* warp_tot, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < kSortThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kSortThreads / 32) warp_tot[lane] = w;  // inclusive
    }
    __syncthreads();
    const int before = (warp > 0 ? warp_tot[warp - 1] : 0) + x - v;
    *total = warp_tot[kSortThreads / 32 - 1];
    __syncthreads();  // warp_tot is reused by the next call
    return before;
}

// Word prefixes within each block and the blocks' exclusive prefix.
__global__ void __launch_bounds__(kSortThreads)
    sort_scan(const uint32_t* __restrict__ bits, const int32_t* __restrict__ d_n, int cap,
              int32_t* __restrict__ wpre, int32_t* __restrict__ bpre, unsigned int* __restrict__ counter) {
    __shared__ int warp_tot[kSortThreads / 32];
    __shared__ bool last;
    if (min(*d_n, cap) <= kSortSmall) return;
    const long long w0 = (long long)blockIdx.x * kScanWords + 4 * threadIdx.x;
    const uint4 q = *reinterpret_cast<const uint4*>(bits + w0);
    const int c0 = __popc(q.x), c1 = __popc(q.y), c2 = __popc(q.z), c3 = __popc(q.w);
    int total = 0;
    const int before = cta_exclusive_scan(c0 + c1 + c2 + c3, warp_tot, &total);
    *reinterpret_cast<int4*>(wpre + w0) = make_int4(before, before + c0, before + c0 + c1, before + c0 + c1 + c2);
    if (threadIdx.x == 0) {
        bpre[blockIdx.x] = total;
        __threadfence();  // the total is visible before the counter says so
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    // the last block: exclusive prefix of the block totals, in place
    __threadfence();
    int carry = 0;
    for (int b0 = 0; b0 < (int)gridDim.x; b0 += kSortThreads) {
        const int b = b0 + threadIdx.x;
        const int v = b < (int)gridDim.x ? __ldcg(bpre + b) : 0;
        int tot = 0;
        const int ex = cta_exclusive_scan(v, warp_tot, &tot);
        if (b < (int)gridDim.x) bpre[b] = carry + ex;
        carry += tot;
    }
}

template <class Rec, class KeyFn>
__global__ void __launch_bounds__(kSortThreads)
    sort_scatter(const Rec* __restrict__ in, const int32_t* __restrict__ d_n, int cap, KeyFn key,
                 const uint32_t* __restrict__ bits, const int32_t* __restrict__ wpre,
                 const int32_t* __restrict__ bpre, Rec* __restrict__ out) {
    const int n = min(*d_n, cap);
    if (n <= kSortSmall) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Rec r = in[i];
        const long long k = key(r);
        const long long w = k >> 5;
        const int pos = bpre[w / kScanWords] + wpre[w] + __popc(bits[w] & ((1u << (k & 31)) - 1u));
        out[pos] = r;
    }
}

}  // namespace sortk
}  // namespace

// Queues the sorted compaction of the first min(*d_n, cap) records of `in`
// into `out` (cap records), keys from `key` in [0, nkeys), scratch `ws` laid
// out by sort_layout(nkeys) (256-byte aligned).  `ctas` bounds the grid of
// the grid-stride kernels.
template <class Rec, class KeyFn>
cudaError_t launch_sorted_compaction(const Rec* in, const int32_t* d_n, int cap, KeyFn key, long long nkeys,
                                     void* ws, Rec* out, int ctas, cudaStream_t st) {
    if (cap <= 0) return cudaSuccess;
    const SortLayout L = sort_layout(nkeys);
    char* base = static_cast<char*>(ws);
    uint32_t* bits = reinterpret_cast<uint32_t*>(base + L.bits);
    unsigned int* counter = reinterpret_cast<unsigned int*>(base + L.counter);
    int32_t* wpre = reinterpret_cast<int32_t*>(base + L.wpre);
    int32_t* bpre = reinterpret_cast<int32_t*>(base + L.bpre);
    cudaError_t e = cudaMemsetAsync(base + L.bits, 0, L.bits_end - L.bits, st);
    if (e != cudaSuccess) return e;
    const int small_ctas = (kSortSmall + kSortThreads - 1) / kSortThreads;
    const int need = (cap + kSortThreads - 1) / kSortThreads;
    int grid = need < ctas ? need : ctas;
    if (grid < small_ctas) grid = small_ctas;
    sortk::sort_mark<Rec, KeyFn><<<grid, kSortThreads, 0, st>>>(in, d_n, cap, key, bits, out);
    sortk::sort_scan<<<L.nblocks, kSortThreads, 0, st>>>(bits, d_n, cap, wpre, bpre, counter);
    sortk::sort_scatter<Rec, KeyFn><<<grid, kSortThreads, 0, st>>>(in, d_n, cap, key, bits, wpre, bpre, out);
    return cudaGetLastError();
}

}  // namespace sncc
