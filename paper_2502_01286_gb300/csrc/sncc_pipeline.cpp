// sncc_pipeline.cpp - a native frame pipeline: segmented-NCC matching of a
// stream of host frames with one template at up to SNCC_MULTI_MAX std
// thresholds (Section 5, main algorithm with an exact second stage, once per
// frame).
//
// Two slots of caller-owned device buffers alternate.  Each slot's whole
// path (sum tables, the coarse pass of every approximation - fused into one
// launch where sncc_match_multi accepts them - and the exact refines) is
// captured once into a CUDA graph.  Per frame, one call:
//   - copies the frame host -> device on a copy stream, after the frame that
//     last used the slot has finished with it, and returns only once that
//     copy is complete (the caller may then refill its host buffer);
//   - launches the slot's graph on the compute stream once the copy is done;
//   - waits on a read-back stream for the previous frame only and copies its
//     match counts, records and status words to the caller's host memory.
// So the copies and the host's work overlap the GPU's, and the host issues a
// handful of CUDA calls per frame.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <new>

#include "sncc.h"
#include "sncc_internal.h"

struct sncc_pipeline_st {
    int n = 0;
    const sncc_segments* segs[SNCC_MULTI_MAX] = {};
    const void* plans[SNCC_MULTI_MAX] = {};
    float taus[SNCC_MULTI_MAX] = {};
    float tau_exact = 0.0f;
    const uint8_t* d_t = nullptr;
    int t_stride = 0, M = 0, N = 0, W = 0, H = 0, s_bits = 32, sat_pitch = 0, cand_cap = 0, out_cap = 0,
        rho_pitch = 0;
    sncc_pipeline_slot slot[2];
    bool fused = false;
    cudaStream_t compute = nullptr, copy = nullptr, readback = nullptr;
    cudaEvent_t copied[2] = {}, done[2] = {};
    cudaGraphExec_t exec[2] = {};
    bool used[2] = {false, false};
    long long frames = 0;
    int32_t* h_counts = nullptr;  // pinned staging for the read-back counts
};

namespace {

// The whole path of one slot on stream st (outside or inside a capture).
int run_slot(sncc_pipeline_st* p, int k, cudaStream_t st) {
    const sncc_pipeline_slot& b = p->slot[k];
    const sncc_stream_t s = (sncc_stream_t)st;
    int rc = sncc_integral(b.d_frame, p->M, p->N, p->M, b.d_s, p->s_bits, b.d_s2, p->sat_pitch, b.d_ws, b.ws_bytes, s);
    if (rc != SNCC_OK) return rc;
    if (p->fused) {
        rc = sncc_match_multi(p->segs, p->plans, p->n, b.d_s, p->s_bits, b.d_s2, p->sat_pitch, p->M, p->N, p->taus,
                              b.d_rho[0] ? b.d_rho : nullptr, p->rho_pitch, b.d_cand, p->cand_cap, b.d_count,
                              b.d_status, s);
        if (rc != SNCC_OK) return rc;
    } else {
        for (int q = 0; q < p->n; ++q) {
            rc = sncc_match(p->segs[q], p->plans[q], b.d_s, p->s_bits, b.d_s2, p->sat_pitch, p->M, p->N, p->taus[q],
                            b.d_rho[q], p->rho_pitch, b.d_cand[q], p->cand_cap, b.d_count[q], b.d_status[q], s);
            if (rc != SNCC_OK) return rc;
        }
    }
    for (int q = 0; q < p->n; ++q) {
        rc = sncc_refine(b.d_frame, p->M, p->N, p->M, p->d_t, p->W, p->H, p->t_stride, p->segs[q]->T,
                         p->segs[q]->T2, b.d_cand[q], b.d_count[q], p->cand_cap, p->tau_exact, b.d_out[q], p->out_cap,
                         b.d_nout[q], b.d_rws[q], b.rws_bytes, b.d_status[q], s);
        if (rc != SNCC_OK) return rc;
    }
    return SNCC_OK;
}

void release(sncc_pipeline_st* p) {
    if (!p) return;
    for (int k = 0; k < 2; ++k) {
        if (p->exec[k]) cudaGraphExecDestroy(p->exec[k]);
        if (p->copied[k]) cudaEventDestroy(p->copied[k]);
        if (p->done[k]) cudaEventDestroy(p->done[k]);
    }
    if (p->compute) cudaStreamDestroy(p->compute);
    if (p->copy) cudaStreamDestroy(p->copy);
    if (p->readback) cudaStreamDestroy(p->readback);
    if (p->h_counts) cudaFreeHost(p->h_counts);
    delete p;
}

// Copies the match lists of the frame in `k` (already complete on the
// device once done[k] is reached) to the caller's host memory.
int collect(sncc_pipeline_st* p, int k, sncc_match_t* const* h_out, int32_t* h_count, int32_t* h_status) {
    const sncc_pipeline_slot& b = p->slot[k];
    if (cudaStreamWaitEvent(p->readback, p->done[k], 0) != cudaSuccess) return SNCC_ERR_CUDA;
    for (int q = 0; q < p->n; ++q) {
        if (cudaMemcpyAsync(p->h_counts + q, b.d_nout[q], sizeof(int32_t), cudaMemcpyDeviceToHost, p->readback) !=
                cudaSuccess ||
            cudaMemcpyAsync(p->h_counts + SNCC_MULTI_MAX + q, b.d_status[q], sizeof(int32_t), cudaMemcpyDeviceToHost,
                            p->readback) != cudaSuccess)
            return SNCC_ERR_CUDA;
    }
    if (cudaStreamSynchronize(p->readback) != cudaSuccess) return SNCC_ERR_CUDA;
    bool any = false;
    for (int q = 0; q < p->n; ++q) {
        const int32_t c = p->h_counts[q];
        h_count[q] = c;
        if (h_status) h_status[q] = p->h_counts[SNCC_MULTI_MAX + q];
        const int m = c < p->out_cap ? c : p->out_cap;
        if (m > 0 && h_out && h_out[q]) {
            if (cudaMemcpyAsync(h_out[q], b.d_out[q], (size_t)m * sizeof(sncc_match_t), cudaMemcpyDeviceToHost,
                                p->readback) != cudaSuccess)
                return SNCC_ERR_CUDA;
            any = true;
        }
    }
    if (any && cudaStreamSynchronize(p->readback) != cudaSuccess) return SNCC_ERR_CUDA;
    return 1;
}

}  // namespace

extern "C" int sncc_pipeline_create(const sncc_segments* const* segs, const void* const* d_plans, int n,
                                    const uint8_t* d_t, int t_stride, int M, int N, int s_bits, int sat_pitch,
                                    const float* taus, float tau_exact, int cand_cap, int out_cap, int rho_pitch,
                                    const sncc_pipeline_slot* slots, sncc_pipeline* out) {
    sncc::NvtxRange nvtx_range("sncc_pipeline_create");
    if (!out) return SNCC_ERR_ARG;
    *out = nullptr;
    if (!segs || !d_plans || !taus || !slots || !d_t || n < 1 || n > SNCC_MULTI_MAX || cand_cap < 1 || out_cap < 1)
        return SNCC_ERR_ARG;
    for (int q = 0; q < n; ++q)
        if (!segs[q] || !d_plans[q] || segs[q]->W != segs[0]->W || segs[q]->H != segs[0]->H) return SNCC_ERR_ARG;
    const int W = segs[0]->W, H = segs[0]->H;
    if (M < W || N < H || t_stride < W) return SNCC_ERR_ARG;
    for (int k = 0; k < 2; ++k) {
        const sncc_pipeline_slot& b = slots[k];
        if (!b.d_frame || !b.d_s || !b.d_s2 || !b.d_ws) return SNCC_ERR_ARG;
        for (int q = 0; q < n; ++q)
            if (!b.d_cand[q] || !b.d_count[q] || !b.d_status[q] || !b.d_out[q] || !b.d_nout[q] || !b.d_rws[q] ||
                (b.d_rho[q] != nullptr) != (b.d_rho[0] != nullptr))
                return SNCC_ERR_ARG;
    }
    sncc_pipeline_st* p = new (std::nothrow) sncc_pipeline_st;
    if (!p) return SNCC_ERR_NOMEM;
    p->n = n;
    for (int q = 0; q < n; ++q) {
        p->segs[q] = segs[q];
        p->plans[q] = d_plans[q];
        p->taus[q] = taus[q];
    }
    p->tau_exact = tau_exact;
    p->d_t = d_t;
    p->t_stride = t_stride;
    p->M = M;
    p->N = N;
    p->W = W;
    p->H = H;
    p->s_bits = s_bits;
    p->sat_pitch = sat_pitch;
    p->cand_cap = cand_cap;
    p->out_cap = out_cap;
    p->rho_pitch = rho_pitch;
    p->slot[0] = slots[0];
    p->slot[1] = slots[1];
    if (cudaStreamCreateWithFlags(&p->compute, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->readback, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(&p->h_counts, 2 * SNCC_MULTI_MAX * sizeof(int32_t)) != cudaSuccess) {
        release(p);
        return SNCC_ERR_CUDA;
    }
    for (int k = 0; k < 2; ++k)
        if (cudaEventCreateWithFlags(&p->copied[k], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->done[k], cudaEventDisableTiming) != cudaSuccess) {
            release(p);
            return SNCC_ERR_CUDA;
        }
    // fuse the coarse passes if the library accepts the approximations (a
    // host-only decision; nothing is launched)
    if (n > 1) {
        const int rc = sncc::multi_fusable(p->segs, p->plans, n);
        if (rc != SNCC_OK && rc != SNCC_ERR_UNSUPPORTED) {
            release(p);
            return rc;
        }
        p->fused = (rc == SNCC_OK);
    }
    // one eager run per slot (the library's one-time setup happens outside
    // any capture), then one captured graph per slot
    for (int k = 0; k < 2; ++k) {
        int rc = run_slot(p, k, p->compute);
        if (rc == SNCC_OK && cudaStreamSynchronize(p->compute) != cudaSuccess) rc = SNCC_ERR_CUDA;
        if (rc != SNCC_OK) {
            release(p);
            return rc;
        }
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(p->compute, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            release(p);
            return SNCC_ERR_CUDA;
        }
        rc = run_slot(p, k, p->compute);
        const cudaError_t ce = cudaStreamEndCapture(p->compute, &g);
        if (rc == SNCC_OK && (ce != cudaSuccess || cudaGraphInstantiate(&p->exec[k], g, 0) != cudaSuccess))
            rc = SNCC_ERR_CUDA;
        if (g) cudaGraphDestroy(g);
        if (rc != SNCC_OK) {
            release(p);
            return rc;
        }
    }
    *out = p;
    return SNCC_OK;
}

extern "C" int sncc_pipeline_submit(sncc_pipeline p, const uint8_t* h_frame, sncc_match_t* const* h_out,
                                    int32_t* h_count, int32_t* h_status) {
    sncc::NvtxRange nvtx_range("sncc_pipeline_submit");
    if (!p || !h_frame || !h_count) return SNCC_ERR_ARG;
    const int k = (int)(p->frames & 1);
    // the slot's frame buffer is free once the frame two back is done
    if (p->used[k] && cudaStreamWaitEvent(p->copy, p->done[k], 0) != cudaSuccess) return SNCC_ERR_CUDA;
    if (cudaMemcpyAsync(p->slot[k].d_frame, h_frame, (size_t)p->M * p->N, cudaMemcpyHostToDevice, p->copy) !=
            cudaSuccess ||
        cudaEventRecord(p->copied[k], p->copy) != cudaSuccess ||
        cudaStreamWaitEvent(p->compute, p->copied[k], 0) != cudaSuccess ||
        cudaGraphLaunch(p->exec[k], p->compute) != cudaSuccess || cudaEventRecord(p->done[k], p->compute) != cudaSuccess)
        return SNCC_ERR_CUDA;
    p->used[k] = true;
    // the caller may refill h_frame once this returns: wait for its copy
    // (it overlaps the previous frame's matching, which is waited for next)
    if (cudaEventSynchronize(p->copied[k]) != cudaSuccess) return SNCC_ERR_CUDA;
    const bool prev = p->frames > 0;
    ++p->frames;
    return prev ? collect(p, k ^ 1, h_out, h_count, h_status) : 0;
}

extern "C" int sncc_pipeline_flush(sncc_pipeline p, sncc_match_t* const* h_out, int32_t* h_count,
                                   int32_t* h_status) {
    if (!p || !h_count) return SNCC_ERR_ARG;
    if (p->frames == 0) return 0;
    return collect(p, (int)((p->frames - 1) & 1), h_out, h_count, h_status);
}

extern "C" int sncc_pipeline_fused(sncc_pipeline p) { return p ? (p->fused ? 1 : 0) : SNCC_ERR_ARG; }

extern "C" sncc_stream_t sncc_pipeline_compute_stream(sncc_pipeline p) {
    return p ? (sncc_stream_t)p->compute : nullptr;
}

extern "C" void sncc_pipeline_destroy(sncc_pipeline p) {
    if (!p) return;
    if (p->compute) cudaStreamSynchronize(p->compute);
    if (p->copy) cudaStreamSynchronize(p->copy);
    if (p->readback) cudaStreamSynchronize(p->readback);
    release(p);
}
