/*
 * sncc.h - C ABI of the GB300 segmented-NCC library (libsncc.so).
 *
 * Method: Marusic, Popovic, Kalafatic, "Template Matching in Images using
 * Segmented Normalized Cross-Correlation" (arXiv 2502.01286).
 *
 * Conventions (paper Section 2)
 *   Source f: M x N pixels (M columns, N rows), uint8, row-major with a row
 *   stride in bytes, pixel (x, y) at f[y * f_stride + x].
 *   Template t: W x H pixels, uint8, t[y * t_stride + x].
 *   Offsets (u, v) in {0..M-W} x {0..N-H} (main algorithm, step 7):
 *   U = M-W+1 columns and V = N-H+1 rows of offsets, linear index v*U + u.
 *
 * Memory and ownership
 *   Every pointer named d_* is device memory owned by the caller.  The
 *   library never allocates device memory and never frees caller memory.
 *   sncc_segments is host memory owned by the library (sncc_free_segments).
 *   Scratch space is passed in as a caller-owned workspace whose size the
 *   matching *_workspace_bytes call returns.
 *   Alignment: every device array must be aligned to its element (4 bytes
 *   for int32 and float, 8 for int64, double and the candidate pairs of the
 *   batch calls, 16 for plans, rectangle lists and batch buffers); sum
 *   tables read by the segment-sum and batch calls must start on 16 bytes
 *   with a pitch that is a multiple of 4, as sncc_integral writes them.
 *   Byte arrays (sources, templates) have no alignment rule.  A call given a
 *   misaligned pointer returns SNCC_ERR_ARG before launching anything.
 *
 * Streams and errors
 *   Device entry points are asynchronous on the given stream (NULL = the
 *   legacy default stream).  Each returns SNCC_OK or a negative SNCC_ERR_*
 *   code for errors found on the host (bad arguments, launch failures).
 *   Errors found on the device (capacity overflow, a bounded wait that ran
 *   out) are OR-ed as SNCC_STATUS_* bits into a caller-owned int32 status
 *   word, which the caller reads after synchronising the stream; the calls
 *   that take one clear it first, in stream order.
 *
 * SNCC_STATUS_WAIT_TIMEOUT means that a copy into a CTA's shared memory did
 * not complete within one second.  The CTA then stops without waiting any
 * longer, so that copy may still land later in shared memory that another
 * CTA of the same or a later launch is using.  Discard the outputs of that
 * call and of every call queued after it on the stream, and do not trust
 * further results from the context; the limit exists so that a stuck copy
 * ends in an error instead of a hung GPU.
 *
 * Thread safety: calls are reentrant; concurrent calls must not share
 * output buffers or workspaces.
 */
#ifndef SNCC_H
#define SNCC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (cudaStream_t / CUstream); NULL selects the default stream. */
typedef struct CUstream_st* sncc_stream_t;

/* Host-side return codes. */
#define SNCC_OK 0
#define SNCC_ERR_ARG (-1)       /* bad argument: null pointer, size, stride, bits */
#define SNCC_ERR_UNIFORM (-2)   /* uniform template or zero-energy approximation (Section 2) */
#define SNCC_ERR_DTYPE (-3)     /* a wrapped 32-bit table where whole entries are read */
#define SNCC_ERR_CAPACITY (-4)  /* a host-visible capacity is too small */
#define SNCC_ERR_CUDA (-5)      /* a CUDA runtime call or kernel launch failed */
#define SNCC_ERR_WORKSPACE (-6) /* workspace missing, misaligned or too small */
#define SNCC_ERR_NOMEM (-7)     /* host allocation failed */
#define SNCC_ERR_UNSUPPORTED (-8) /* size or shape outside what the library supports */

/* Device status bits (OR-ed into the caller's int32 status word). */
#define SNCC_STATUS_CAND_OVERFLOW 1  /* more candidates than cand_cap; count is still exact */
#define SNCC_STATUS_MATCH_OVERFLOW 2 /* more matches than out_cap; count is still exact */
#define SNCC_STATUS_WAIT_TIMEOUT 4   /* a bounded wait on an asynchronous copy ran out: treat as
                                        fatal for the stream (see below) */
#define SNCC_STATUS_SORT_OVERFLOW 8  /* more matches than the sort scratch holds */

/* Human-readable text of a return code (static storage). */
const char* sncc_error_string(int code);

/* ------------------------------------------------------------------ */
/* Template preparation (host)                                         */
/* ------------------------------------------------------------------ */

/* One rectangular segment S_i, the 5-tuple of Eq. 6 plus its exact sum. */
typedef struct {
    int32_t x, y;  /* top-left corner in template coordinates */
    int32_t w, h;  /* width W_i and height H_i */
    int64_t sum;   /* exact sum of t over the rectangle */
    double mean;   /* k_i = sum / (w*h), Eq. 4 (double, correctly rounded) */
} sncc_seg;

/* The segmented approximation k of a template (Section 3). */
typedef struct {
    sncc_seg* seg;      /* K segments, ascending (y, x); owned by the library */
    int32_t K;          /* number of segments after merging */
    int32_t K_split;    /* number of segments split_segment produced */
    int32_t W, H;       /* template size */
    double sigma_used;  /* sigma_max of the last split (after K_max raises) */
    double kbar;        /* Eq. 7: mean of k (equal to the template mean) */
    double Ek;          /* energy of k: sum_i W_i H_i (k_i - kbar)^2 */
    double rho_max;     /* NCC(t, k) by steps 5-7 of precompute_template_approximation */
    int64_t T, T2;      /* sum of t and of t^2 (exact) */
    double err_bound;   /* bound on |rho_gpu - rho| from weight quantisation */
    void* plan;         /* library-private matching plan (host memory) */
    double sigma_t;     /* population std of the whole template, sqrt(n T2 - T^2) / n
                           (the input of sigma_max,fast = 0.99 sigma_t and
                           sigma_max,slow = 0.1 sigma_t, Section 5) */
} sncc_segments;

/*
 * sncc_build_segments - split-and-merge template approximation.
 * Paper: Section 3 (Eq. 2 - Eq. 7) and Section 5, functions
 * precompute_template_approximation, split_segment, merge_redundant_segments.
 *
 *   t, W, H, t_stride  host template (uint8, row stride in bytes >= W)
 *   sigma_max          std threshold of Eq. 2 (segments need std < sigma_max,
 *                      evaluated as n*S2 - S^2 < n^2 sigma_max^2 with the
 *                      segment's exact sum S, sum of squares S2, size n)
 *   k_max              segment cap; > 0 repeats the split with sigma_max + 1
 *                      until K_split <= k_max (steps 1-2); 0 = no cap
 *   out                receives the approximation (overwritten; call
 *                      sncc_free_segments when done)
 * Also builds the matching plan: fixed-point segment weights and the
 * per-block corner lists sncc_match reads (see sncc_plan_bytes).
 * Returns SNCC_OK, SNCC_ERR_ARG, SNCC_ERR_UNSUPPORTED (W*H > 2^23) or
 * SNCC_ERR_NOMEM.  A uniform template is not an error here (K = 1, Ek = 0);
 * sncc_match reports it.
 */
int sncc_build_segments(const uint8_t* t, int W, int H, int t_stride, double sigma_max, int k_max,
                        sncc_segments* out);

/* Releases what sncc_build_segments allocated; safe on a zeroed struct. */
void sncc_free_segments(sncc_segments* s);

/*
 * sncc_template_sigma - sigma_t, the population std of a template: the std
 * of Eq. 2 taken over the whole template, which the main algorithm of
 * Section 5 scales into its two thresholds (sigma_max,fast = 0.99 sigma_t,
 * sigma_max,slow = 0.1 sigma_t).  Computed as sqrt(n T2 - T^2) / n from the
 * exact sums T and T2 (the radicand exact in 64-bit integers).
 *   t, W, H, t_stride  host template (uint8)
 *   sigma_t            receives the value (0 for a uniform template)
 * Returns SNCC_OK, SNCC_ERR_ARG or SNCC_ERR_UNSUPPORTED (W*H > 2^23).
 */
int sncc_template_sigma(const uint8_t* t, int W, int H, int t_stride, double* sigma_t);

/* ------------------------------------------------------------------ */
/* Sum tables (GPU)                                                    */
/* ------------------------------------------------------------------ */

/* Row pitch, in elements, of the padded sum tables for an M-wide source:
 * the smallest multiple of 32 that is >= M+1. */
int sncc_sat_pitch(int M);

/* Scratch bytes sncc_integral needs for an M x N source. */
size_t sncc_integral_workspace_bytes(int M, int N);

/*
 * sncc_integral - sum tables of f and f^2 (Eq. 10 and Eq. 14).
 *
 *   d_f, M, N, f_stride  device source (uint8), f_stride >= M bytes
 *   d_s                  output, (N+1) rows x sat_pitch elements of int32
 *                        (s_bits = 32) or int64 (s_bits = 64); entry
 *                        [Y * pitch + X] = sum of f over x < X, y < Y, so row
 *                        0 and column 0 are zero and [(y+1)*pitch + (x+1)]
 *                        is s(x, y) of Eq. 10.  Columns beyond M are not
 *                        written.
 *   d_s2                 output, the same layout in int64, for f^2 (Eq. 14)
 *   sat_pitch            row pitch in elements, >= sncc_sat_pitch(M) and a
 *                        multiple of 4
 *   d_ws, ws_bytes       workspace, >= sncc_integral_workspace_bytes(M, N),
 *                        16-byte aligned
 * With s_bits = 32 the entries of s are the sums modulo 2^32 (two's
 * complement): exact while 255*M*N < 2^31, wrapped beyond.  Every window sum
 * the library forms from a table (at most 255*W*H < 2^31, as W*H <= 2^23) is
 * a difference of entries and exact in wrapped 32-bit arithmetic, so the
 * segment-sum, batch and exact-map calls take wrapped tables; only
 * sncc_refine_segmented, which reads whole entries, rejects them
 * (SNCC_ERR_DTYPE).  A 32-bit table writes 12 bytes per pixel instead of 16.
 */
int sncc_integral(const uint8_t* d_f, int M, int N, int f_stride, void* d_s, int s_bits, int64_t* d_s2,
                  int sat_pitch, void* d_ws, size_t ws_bytes, sncc_stream_t stream);

/* Templates with at most this many corners in all (sncc_plan_info.template_corners)
 * are summed by sncc_match straight from the corners' table entries, without
 * staging; that needs whole entries, so with a 32-bit s that may wrap
 * (255*M*N >= 2^31) they take the staged path instead. */
#define SNCC_DIRECT_MAX_CORNERS 64

/* Size of the library's built-in scratch array used by sncc_integral_noalloc. */
#define SNCC_NOALLOC_SCRATCH_BYTES (16u << 20)

/*
 * sncc_integral_noalloc - sncc_integral without a caller-supplied workspace
 * and without allocating anything.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory where they call it, e.g. plug-ins whose host
 * application owns the whole device-memory budget and forbids allocations by
 * libraries, latency-critical loops that cannot afford the device-wide
 * synchronisation cudaMalloc implies, or plain C callers that have no
 * allocator to hand for a workspace buffer.
 *
 * Arguments, layout and results are those of sncc_integral (same kernels);
 * the band sums live instead in a fixed array of SNCC_NOALLOC_SCRATCH_BYTES
 * (16 MiB) of device memory that every GPU which loads the library holds
 * until the process exits.  That covers every source of up to 100 million
 * pixels (e.g. 10000 x 10000 or 16383 x 6100); a source whose
 * sncc_integral_workspace_bytes exceeds it returns SNCC_ERR_CAPACITY and
 * launches nothing.  No call allocates or frees memory.
 *
 * The first call on a device (with that device current) looks up the
 * array's device address; make that first call before any stream capture.
 * The address is kept per device together with the identity of the context
 * it was taken in; a call made in another context (after cudaDeviceReset, or
 * once the primary context was destroyed and created again) looks it up
 * anew, so make the first call after such a reset outside a capture too.
 * Every call shares the one array and leaves its contents behind; nothing
 * in it needs to start at zero, because each call writes every entry it
 * later reads.  Calls whose executions overlap on the GPU (other streams,
 * other host threads) race on the array: serialise them.
 */
int sncc_integral_noalloc(const uint8_t* d_f, int M, int N, int f_stride, void* d_s, int s_bits, int64_t* d_s2,
                          int sat_pitch, sncc_stream_t stream);

/* ------------------------------------------------------------------ */
/* Coarse pass: segmented NCC, threshold, candidates (GPU)             */
/* ------------------------------------------------------------------ */

/* Device bytes of the matching plan of seg (corner lists and block table). */
size_t sncc_plan_bytes(const sncc_segments* seg);

/* Copies the plan into caller-owned device memory d_plan (>= sncc_plan_bytes,
 * 16-byte aligned), asynchronously on stream.  The host plan must stay alive
 * until the copy completes (it lives as long as seg). */
int sncc_plan_upload(const sncc_segments* seg, void* d_plan, size_t plan_bytes, sncc_stream_t stream);

/*
 * sncc_match - approximate NCC at every offset and its candidates.
 * Paper: Section 4, Eq. 9 - Eq. 18; Section 5 main algorithm steps 7a-7f.
 *
 * For each offset (u, v): num = sum_i (k_i - kbar) * S_i(u, v), where S_i is
 * the four-corner box sum (Eq. 11) of the source over segment i; the local
 * energy E_f = sum f^2 - (sum f)^2 / n (Eq. 13, 15, 16), formed exactly in
 * integers and divided in double; rho = num / sqrt(E_f * Ek) (Eq. 17, 18,
 * with the weighted template energy).  A uniform window gives rho = 0.
 * Offsets with rho >= tau are candidates.
 *
 *   seg, d_plan          approximation and its uploaded plan
 *   d_s, s_bits, d_s2    sum tables from sncc_integral, pitch sat_pitch (a
 *                        wrapped 32-bit s is fine: only differences below
 *                        2^31 are used, and a template of at most 64 corners
 *                        then takes the staged path instead of reading its
 *                        corners' entries directly)
 *   M, N                 source size
 *   tau                  coarse threshold (e.g. precision * rho_max)
 *   d_rho, rho_pitch     optional FP32 map, V rows x rho_pitch (>= U)
 *                        floats; NULL skips it
 *   d_cand, cand_cap     candidate linear indices v*U+u (unordered)
 *   d_count              int32, receives the exact candidate count (may
 *                        exceed cand_cap; then only cand_cap are stored and
 *                        SNCC_STATUS_CAND_OVERFLOW is set)
 *   d_status             int32 status word (cleared first)
 * Returns SNCC_ERR_UNIFORM when Ek = 0 (nothing launched).
 */
int sncc_match(const sncc_segments* seg, const void* d_plan, const void* d_s, int s_bits, const int64_t* d_s2,
               int sat_pitch, int M, int N, float tau, float* d_rho, int rho_pitch, int32_t* d_cand,
               int cand_cap, int32_t* d_count, int32_t* d_status, sncc_stream_t stream);

/* Most approximations sncc_match_multi fuses into one launch. */
#define SNCC_MULTI_MAX 4

/*
 * sncc_match_multi - sncc_match for n approximations of one template size
 * in a single launch (Section 5 step 7 once per approximation, as in the
 * multi-threshold search of Section 6).  The grid covers every (tile,
 * approximation) pair, the approximation with most corners first, so the
 * lighter ones fill the last wave of the heavier ones.  Output q (rho map,
 * candidates, count) is bit-identical to sncc_match with segs[q],
 * d_plans[q] and taus[q].
 *
 *   segs, d_plans, taus  n approximations, plans and thresholds
 *   n                    1 .. SNCC_MULTI_MAX
 *   d_rho                NULL, or n pointers (each NULL or a V x rho_pitch map)
 *   d_cand, d_count,     n pointers each; cand_cap applies to every list;
 *   d_status             status word q is cleared first and receives the
 *                        bits of approximation q
 * The other arguments are those of sncc_match.  Returns
 * SNCC_ERR_UNSUPPORTED unless every approximation has the same template
 * size, at most 64 x 64 (one staged block of the same layout), and more
 * than 64 corners (not summed in place); callers then use sncc_match.
 * SNCC_ERR_UNIFORM when some Ek = 0 (nothing launched).
 */
int sncc_match_multi(const sncc_segments* const* segs, const void* const* d_plans, int n, const void* d_s,
                     int s_bits, const int64_t* d_s2, int sat_pitch, int M, int N, const float* taus,
                     float* const* d_rho, int rho_pitch, int32_t* const* d_cand, int cand_cap,
                     int32_t* const* d_count, int32_t* const* d_status, sncc_stream_t stream);

/* ------------------------------------------------------------------ */
/* Fine pass: exact NCC at the candidates (GPU)                        */
/* ------------------------------------------------------------------ */

/* One match (u, v, rho) of the output collection (Section 5, "matches"). */
typedef struct {
    int32_t u, v;
    float rho;
} sncc_match_t;

/* Scratch bytes sncc_refine and sncc_refine_segmented need for out_cap
 * matches on an M x N source with a W x H template: the unsorted match
 * records, plus one bit per offset and a prefix count per 32 offsets for the
 * sorted write-out (about U*V/4 bytes).  0 for invalid sizes. */
size_t sncc_refine_workspace_bytes(int M, int N, int W, int H, int out_cap);

/*
 * sncc_refine - exact NCC (Eq. 1) at each candidate and the match list.
 * Paper: Eq. 1; Section 5 main algorithm steps 7g-7j, with the second
 * stage computed exactly instead of with a finer approximation.
 *
 * For candidate (u, v): rho_t = (n*Sft - T*Sf) / sqrt((n*Sff - Sf^2)(n*T2 - T^2))
 * with the exact integer sums Sft = sum f*t, Sf, Sff over the window and
 * T, T2 over the template, divided in double.  Matches have rho_t >= tau.
 *
 *   d_f, M, N, f_stride  device source
 *   d_t, W, H, t_stride  device template (uint8)
 *   T, T2                sum of t and t^2 (from sncc_segments)
 *   d_cand, d_count      candidates and their count from sncc_match; only
 *                        the first min(*d_count, cand_cap) are read
 *   tau                  exact threshold
 *   d_out, out_cap       matches sorted by v*U+u
 *   d_nout               int32, receives the exact match count (may exceed
 *                        out_cap: SNCC_STATUS_MATCH_OVERFLOW; then the
 *                        out_cap matches that were stored are written, sorted)
 *   d_ws, ws_bytes       workspace, >= sncc_refine_workspace_bytes(M, N, W, H,
 *                        out_cap), 16-byte aligned
 *   d_status             int32 status word (not cleared: sncc_match clears it)
 * The sort is a sorted compaction: one bit per offset, a prefix count of the
 * set bits and a scatter, O(U*V/32 + matches) work; lists of at most 2048
 * matches are ranked by direct comparison instead.  The candidates must be
 * distinct offsets (as sncc_match writes them).
 */
int sncc_refine(const uint8_t* d_f, int M, int N, int f_stride, const uint8_t* d_t, int W, int H, int t_stride,
                int64_t T, int64_t T2, const int32_t* d_cand, const int32_t* d_count, int cand_cap, float tau,
                sncc_match_t* d_out, int out_cap, int32_t* d_nout, void* d_ws, size_t ws_bytes,
                int32_t* d_status, sncc_stream_t stream);

/*
 * sncc_refine_segmented - the paper's own fine stage: segmented NCC with a
 * second, finer approximation at each candidate.
 * Paper: Section 5 main algorithm steps 7g-7j (k_slow, threshold_slow =
 * precision * rho_slow), Eq. 12 - Eq. 18.
 *
 * For candidate (u, v) of the coarse pass, rho is computed exactly as
 * sncc_match computes it, but with `seg` (the fine approximation, e.g.
 * sigma_max = 0.1 sigma_t with K_max = 5000) and only at the candidates.
 * Matches have rho >= tau.
 *
 *   seg, d_plan             fine approximation and its uploaded plan
 *   d_s, s_bits, d_s2       sum tables from sncc_integral, pitch sat_pitch;
 *                           a 32-bit s must not wrap (255*M*N < 2^31, else
 *                           SNCC_ERR_DTYPE): this walk reads whole entries
 *   M, N                    source size
 *   d_cand, d_count         candidates and count from sncc_match; the first
 *                           min(*d_count, cand_cap) are read
 *   tau                     fine threshold
 *   d_out, out_cap, d_nout  matches sorted by v*U+u and their exact count
 *                           (SNCC_STATUS_MATCH_OVERFLOW beyond out_cap)
 *   d_ws, ws_bytes          workspace, >= sncc_refine_workspace_bytes(M, N,
 *                           seg->W, seg->H, out_cap), 16-byte aligned
 *   d_status                int32 status word (not cleared)
 */
int sncc_refine_segmented(const sncc_segments* seg, const void* d_plan, const void* d_s, int s_bits,
                          const int64_t* d_s2, int sat_pitch, int M, int N, const int32_t* d_cand,
                          const int32_t* d_count, int cand_cap, float tau, sncc_match_t* d_out, int out_cap,
                          int32_t* d_nout, void* d_ws, size_t ws_bytes, int32_t* d_status, sncc_stream_t stream);

/*
 * sncc_refine_segmented_tiles - the same fine stage as sncc_refine_segmented
 * (Section 5 main algorithm steps 7g-7j, Eq. 12 - Eq. 18), evaluated tile by
 * tile: every tile of 32 x 8R offsets (R as sncc_match picks it) that holds a
 * candidate is computed by the segment-sum kernel of sncc_match with the
 * fine plan, and its candidates with rho >= tau become matches.  The result
 * is the same set (rho identical); the cost follows the number of tiles that
 * hold candidates rather than the number of candidates, which pays when the
 * coarse stage passes many.
 *
 *   arguments as sncc_refine_segmented, except the workspace:
 *   d_ws, ws_bytes          256-byte aligned workspace of at least
 *                           sncc_refine_segmented_tiles_workspace_bytes(M, N, W, H, out_cap)
 *                           (match records, one candidate bit per offset,
 *                           a flag and a list entry per tile, the sort
 *                           scratch)
 * Errors as sncc_refine_segmented; SNCC_ERR_WORKSPACE for a missing, short or
 * misaligned workspace.
 */
size_t sncc_refine_segmented_tiles_workspace_bytes(int M, int N, int W, int H, int out_cap);
int sncc_refine_segmented_tiles(const sncc_segments* seg, const void* d_plan, const void* d_s, int s_bits,
                                const int64_t* d_s2, int sat_pitch, int M, int N, const int32_t* d_cand,
                                const int32_t* d_count, int cand_cap, float tau, sncc_match_t* d_out, int out_cap,
                                int32_t* d_nout, void* d_ws, size_t ws_bytes, int32_t* d_status,
                                sncc_stream_t stream);

/* ------------------------------------------------------------------ */
/* Frame pipeline: a stream of host frames (GPU)                       */
/* ------------------------------------------------------------------ */

/* Caller-owned device buffers of one pipeline slot (two slots alternate).
 * Entries q < n of the per-approximation arrays are used; either every
 * d_rho[q] is NULL (no maps) or none is. */
typedef struct {
    uint8_t* d_frame;                    /* N x M source, row stride M bytes */
    void* d_s;                           /* sum tables (sncc_integral), s_bits / sat_pitch */
    int64_t* d_s2;
    void* d_ws;                          /* sncc_integral workspace */
    size_t ws_bytes;
    float* d_rho[SNCC_MULTI_MAX];        /* V x rho_pitch maps, or NULL */
    int32_t* d_cand[SNCC_MULTI_MAX];     /* cand_cap candidates each */
    int32_t* d_count[SNCC_MULTI_MAX];
    int32_t* d_status[SNCC_MULTI_MAX];
    sncc_match_t* d_out[SNCC_MULTI_MAX]; /* out_cap matches each */
    int32_t* d_nout[SNCC_MULTI_MAX];
    void* d_rws[SNCC_MULTI_MAX];         /* sncc_refine workspaces of rws_bytes
                                            (sncc_refine_workspace_bytes(M, N, W, H, out_cap)) */
    size_t rws_bytes;
} sncc_pipeline_slot;

typedef struct sncc_pipeline_st* sncc_pipeline;

/*
 * sncc_pipeline_create - a pipeline matching a stream of frames with one
 * template at n (1 .. SNCC_MULTI_MAX) std thresholds: per frame the sum
 * tables, the coarse pass of every approximation (one fused launch when
 * sncc_match_multi accepts them) and the exact refine of each (Section 5,
 * main algorithm with an exact second stage).  Each slot's path is captured
 * into a CUDA graph here, after one eager run per slot.
 *
 *   segs, d_plans, taus  the n approximations (same template size), their
 *                        uploaded plans and coarse thresholds
 *   d_t, t_stride        device template (uint8) for the exact refine
 *   M, N, s_bits, sat_pitch, rho_pitch, cand_cap, out_cap
 *                        as for sncc_integral / sncc_match / sncc_refine
 *   tau_exact            exact-refine threshold
 *   slots                two slots of device buffers (caller-owned; they
 *                        must outlive the pipeline)
 *   out                  receives the pipeline (sncc_pipeline_destroy)
 * The library allocates no device memory; it creates three streams, four
 * events, two graphs and a small pinned host array.
 */
int sncc_pipeline_create(const sncc_segments* const* segs, const void* const* d_plans, int n, const uint8_t* d_t,
                         int t_stride, int M, int N, int s_bits, int sat_pitch, const float* taus, float tau_exact,
                         int cand_cap, int out_cap, int rho_pitch, const sncc_pipeline_slot* slots,
                         sncc_pipeline* out);

/*
 * sncc_pipeline_submit - queues one frame (host memory, N x M, row stride M;
 * pinned for an asynchronous copy) and returns the previous frame's results.
 * The frame is copied on the pipeline's copy stream once the frame that last
 * used the slot has finished with it, and matched on the compute stream.
 * The call returns only after that copy has completed, so h_frame may be
 * refilled as soon as it returns.
 * Then the call waits for the previous frame only, and writes its match
 * count into h_count[q] and its status word into h_status[q] (if h_status is
 * not NULL).  Its first min(count, out_cap) matches, sorted by v*U+u, go to
 * h_out[q] (host memory, out_cap records; pinned for speed).
 * Returns 1 when a previous frame was reported, 0 on the first call, or a
 * negative code.
 */
int sncc_pipeline_submit(sncc_pipeline p, const uint8_t* h_frame, sncc_match_t* const* h_out, int32_t* h_count,
                         int32_t* h_status);

/* The results of the last submitted frame, as above (0 if none was submitted). */
int sncc_pipeline_flush(sncc_pipeline p, sncc_match_t* const* h_out, int32_t* h_count, int32_t* h_status);

/* 1 if the coarse passes run as one fused launch, 0 if one launch each. */
int sncc_pipeline_fused(sncc_pipeline p);

/* The stream frames are matched on, e.g. to queue other work between frames. */
sncc_stream_t sncc_pipeline_compute_stream(sncc_pipeline p);

/* Waits for the pipeline's streams and releases it; safe on NULL. */
void sncc_pipeline_destroy(sncc_pipeline p);

/* ------------------------------------------------------------------ */
/* Batched matching: many templates x several sources, one launch      */
/* ------------------------------------------------------------------ */

#define SNCC_BATCH_MAX_SOURCES 16
/* Template buckets of a batch: size class (0: one 64 x 64 block, 1: up to
 * four, 2: more) x corner density class (0: corners per template pixel below
 * 0.1, 1: below 0.5, 2: above); bucket = 3 * size_class + density_class. */
#define SNCC_BATCH_BUCKETS 9
/* Variants of a bucket: v = 0, 1, 2 are tile heights R = 8, 4, 2 with
 * 64 x 64 template blocks, v = 3, 4, 5 the same with 32 x 32 blocks. */
#define SNCC_BATCH_VARIANTS 6

/* Opaque host object describing a batch (library-owned host memory). */
typedef struct sncc_batch_s sncc_batch;

/* One match of a batch: pair = source * n_templates + template. */
typedef struct {
    int32_t pair;
    int32_t u, v;
    float rho;
} sncc_batch_match_t;

typedef struct {
    int32_t n_templates, n_sources;
    int32_t tile_rows;      /* R of every bucket's tile shape (32 x 8R offsets per tile); 0 if the
                               buckets differ */
    int32_t tiles;          /* work items under the current variants */
    double offsets;         /* sum over pairs of U*V */
    double corner_offsets;  /* sum over pairs of U*V*(nonzero corners of the whole template) */
} sncc_batch_info;

/* One bucket of a batch (sncc_batch_get_bucket). */
typedef struct {
    int32_t templates, pairs;  /* templates in the bucket and their (source, template) pairs */
    int32_t size_class, density_class;
    int32_t tile_rows;         /* the bucket's variant: tile height R ... */
    int32_t block;             /* ... and template block edge (64 or 32: corners per staging pass) */
    double corner_offsets;     /* sum over its pairs of U*V*(corners of the whole template) */
    float ms[SNCC_BATCH_VARIANTS]; /* the autotuner's time of the bucket alone in each variant (0 untimed) */
} sncc_batch_bucket;

/*
 * sncc_batch_create - plan the coarse pass of every (source, template) pair
 * of a batch in one persistent launch.  Paper: Eq. 9 - Eq. 18 and Section 5
 * steps 7a-7f, applied to n_sources x n_templates independent problems.
 *
 *   segs[i], templates[i], t_strides[i]  approximation and host pixels of
 *                          template i (pixels are kept for the exact refine)
 *   tau_coarse[i], tau_exact[i]          thresholds of template i
 *   n_templates, n_sources (<= SNCC_BATCH_MAX_SOURCES), M, N  all sources
 *                          are M x N
 *   out                    receives the batch (free with sncc_batch_destroy)
 * Every template's plan is rebuilt with 64 x 64 and 32 x 32 blocks and the
 * template goes into its bucket; work lists of tiles are ordered by
 * estimated cost (largest first) for each bucket and tile height.  Every
 * bucket starts with R = 8 and 64 x 64 blocks.
 * Returns SNCC_ERR_UNIFORM if an approximation has zero energy.
 */
int sncc_batch_create(const sncc_segments* const* segs, const uint8_t* const* templates, const int* t_strides,
                      const float* tau_coarse, const float* tau_exact, int n_templates, int n_sources, int M, int N,
                      sncc_batch** out);
void sncc_batch_destroy(sncc_batch* b);

/* Device bytes of the batch image, and its asynchronous upload into
 * caller-owned memory (16-byte aligned). */
size_t sncc_batch_device_bytes(const sncc_batch* b);
int sncc_batch_upload(const sncc_batch* b, void* d_buf, size_t bytes, sncc_stream_t stream);

/* Sets every bucket to tile height R (8, 4 or 2) with 64 x 64 blocks;
 * batch statistics. */
int sncc_batch_set_variant(sncc_batch* b, int tile_rows);
int sncc_batch_get_info(const sncc_batch* b, sncc_batch_info* out);

/* One bucket's variant (tile height 8, 4 or 2; block edge 64 or 32), and a
 * bucket's description.  SNCC_ERR_ARG for other values. */
int sncc_batch_set_bucket_variant(sncc_batch* b, int bucket, int tile_rows, int block);
int sncc_batch_get_bucket(const sncc_batch* b, int bucket, sncc_batch_bucket* out);

/*
 * sncc_batch_match - the coarse pass for all pairs: one persistent launch
 * per variant in use (one CTA per SM slot, tiles pulled through an atomic
 * work counter, every bucket's tiles in its own variant).
 *
 *   d_buf                  uploaded batch image
 *   d_s[s], d_s2[s]        sum tables of source s (sncc_integral), all with
 *                          the same s_bits and sat_pitch (a multiple of 4)
 *   d_cand, cand_cap       candidates as int32 pairs {pair, v*U+u}
 *                          (2*cand_cap int32), unordered
 *   d_count                exact candidate count (may exceed cand_cap:
 *                          SNCC_STATUS_CAND_OVERFLOW)
 *   d_counter              one int32 of device scratch (the work counter)
 *   d_status               status word (cleared first)
 */
int sncc_batch_match(const sncc_batch* b, const void* d_buf, const void* const* d_s, const int64_t* const* d_s2,
                     int s_bits, int sat_pitch, int32_t* d_cand, int cand_cap, int32_t* d_count, int32_t* d_counter,
                     int32_t* d_status, sncc_stream_t stream);

/*
 * sncc_batch_autotune - for every bucket that holds pairs, times the coarse
 * pass of that bucket alone in each of the SNCC_BATCH_VARIANTS variants on
 * the given data (one untimed run, then the fastest of `reps`) and keeps the
 * fastest variant per bucket for later calls.  Synchronises the stream.
 * ms_out (nullable) receives SNCC_BATCH_BUCKETS x SNCC_BATCH_VARIANTS times
 * in ms, bucket-major (0 for empty buckets); sncc_batch_get_bucket reports
 * them too.
 */
int sncc_batch_autotune(sncc_batch* b, const void* d_buf, const void* const* d_s, const int64_t* const* d_s2,
                        int s_bits, int sat_pitch, int32_t* d_cand, int cand_cap, int32_t* d_count,
                        int32_t* d_counter, int32_t* d_status, int reps, sncc_stream_t stream, float* ms_out);

/* Scratch bytes sncc_batch_refine needs for out_cap matches of batch b: the
 * unsorted records plus one bit per offset of every pair for the sorted
 * write-out.  0 for a NULL batch or a negative out_cap. */
size_t sncc_batch_refine_workspace_bytes(const sncc_batch* b, int out_cap);

/*
 * sncc_batch_refine - exact NCC (Eq. 1) at every batch candidate; matches
 * with rho >= the template's tau_exact, sorted by (pair, v*U+u).
 *   d_f[s], f_stride       device sources (uint8, M x N)
 *   d_cand, d_count, cand_cap  from sncc_batch_match
 *   d_out, out_cap, d_nout matches and their exact count
 *   d_ws, ws_bytes         workspace, >= sncc_batch_refine_workspace_bytes(b,
 *                          out_cap), 16-byte aligned
 *   d_status               status word (not cleared)
 */
int sncc_batch_refine(const sncc_batch* b, const void* d_buf, const uint8_t* const* d_f, int f_stride,
                      const int32_t* d_cand, const int32_t* d_count, int cand_cap, sncc_batch_match_t* d_out,
                      int out_cap, int32_t* d_nout, void* d_ws, size_t ws_bytes, int32_t* d_status,
                      sncc_stream_t stream);

/* ------------------------------------------------------------------ */
/* Differentiation: the approximation-error loss and its gradients     */
/* ------------------------------------------------------------------ */

/* Workspace bytes of sncc_diff_forward / sncc_diff_backward (the same buffer
 * must be passed to both: the backward pass reads what the forward left). */
size_t sncc_diff_workspace_bytes(int M, int N, int W, int H);

/*
 * sncc_diff_forward - loss of a fixed segmentation on a float source.
 * Paper: Eq. 1 (rho_t), Eq. 7, Eq. 9, Eq. 17, Eq. 18 (rho_k with raw segment
 * values k_i, c_i = k_i - kbar, weighted energy).
 *
 * L = sum over offsets (u, v) of (rho_k(u, v) - rho_t(u, v))^2.
 *   d_f, M, N, f_stride  float32 source (row stride in elements)
 *   d_t, W, H            float32 template, contiguous (W, H <= 256; the
 *                        kernels take it in blocks of at most 64 x 64)
 *   d_rects, d_k, K      segmentation: K records {x, y, w, h} (int32) tiling
 *                        the template, and the segment values (float32)
 *   d_rho_k, d_rho_t     outputs, (N-H+1) x (M-W+1) float32 each
 *   d_loss               output, one double
 *   d_ws, ws_bytes       workspace (256-byte aligned)
 * Every window is assumed non-uniform.  Offsets: (M-W+1)(N-H+1) < 2^31 and
 * N-H+1 <= 65535, else SNCC_ERR_UNSUPPORTED (also for sncc_diff_backward).
 */
int sncc_diff_forward(const float* d_f, int M, int N, int f_stride, const float* d_t, int W, int H,
                      const int32_t* d_rects, const float* d_k, int K, float* d_rho_k, float* d_rho_t,
                      double* d_loss, void* d_ws, size_t ws_bytes, sncc_stream_t stream);

/*
 * sncc_diff_backward - gradients of dloss * L with respect to k and f, after
 * sncc_diff_forward on the same inputs and workspace.
 * With g = 2 dloss (rho_k - rho_t), a = g / sqrt(E_f E_k), b = g / sqrt(E_f E_t),
 * h = g (rho_k - rho_t) / E_f:
 *   dL/dk_j  = sum_{x in S_j} sum_o a(o) f(o+x) - n_j sum_o a fbar - n_j c_j sum_o g rho_k / E_k
 *   dL/df(p) = sum_{o: p in window(o)} a(o) c(p-o) - b(o) t0(p-o) + h(o) (fbar(o) - f(p))
 *   d_dloss              upstream gradient (one double, device)
 *   d_grad_f, grad_f_stride  output N x M float32
 *   d_grad_k             output K float32
 */
int sncc_diff_backward(const float* d_f, int M, int N, int f_stride, int W, int H, const int32_t* d_rects,
                       const float* d_k, int K, const float* d_rho_k, const float* d_rho_t, const double* d_dloss,
                       float* d_grad_f, int grad_f_stride, float* d_grad_k, void* d_ws, size_t ws_bytes,
                       sncc_stream_t stream);

/* ------------------------------------------------------------------ */
/* Same-GPU comparator: exact NCC at every offset                      */
/* ------------------------------------------------------------------ */

/*
 * sncc_exact_map - Eq. 1 at every offset by direct correlation with exact
 * integer sums (the paper's "naive algorithm", Section 2 and Table 1), as
 * the same-GPU reference for speed and approximation error.
 *
 *   d_f, M, N, f_stride  device source; d_t, W, H, t_stride device template
 *   T, T2                sum of t and t^2
 *   d_s, s_bits, d_s2    sum tables from sncc_integral (window sums)
 *   d_rho, rho_pitch     FP32 map, V rows x rho_pitch floats
 * Returns SNCC_ERR_UNIFORM for a uniform template.
 */
int sncc_exact_map(const uint8_t* d_f, int M, int N, int f_stride, const uint8_t* d_t, int W, int H,
                   int t_stride, int64_t T, int64_t T2, const void* d_s, int s_bits, const int64_t* d_s2,
                   int sat_pitch, float* d_rho, int rho_pitch, sncc_stream_t stream);

/* ------------------------------------------------------------------ */
/* Introspection and measurement helpers                               */
/* ------------------------------------------------------------------ */

/* Shape of the matching plan built by sncc_build_segments.  blocks ..
 * runs1 describe the first block layout: one block for a template up to
 * 64 x 64 (the layout the segment-sum kernel uses for such templates),
 * else blocks of 32 x 32 (the per-candidate fine pass). */
typedef struct {
    int32_t F;            /* fraction bits of the fixed-point weights q_i */
    int32_t blocks;       /* template blocks that hold at least one corner */
    int32_t block_w;      /* block width and height (edge blocks may be smaller) */
    int32_t block_h;
    int32_t corners;      /* distinct corner points with a nonzero weight, summed over blocks */
    int32_t max_corners;  /* largest corner count of one block */
    int64_t Q0;           /* sum of the weights over all pixels, sum_i W_i H_i q_i */
    int32_t runs8;        /* the corners regrouped into vertical runs (consecutive rows of */
    int32_t runs4;        /* one column, all weights nonzero) of 8, 4, 2 and 1 corners: */
    int32_t runs2;        /* 8 runs8 + 4 runs4 + 2 runs2 + runs1 = corners.  The segment-sum */
    int32_t runs1;        /* kernels read R + L - 1 table words per run of L for R rows; the
                             pairs below R + D words for two corners D rows apart. */
    int32_t template_corners; /* nonzero corners of the whole template taken as one block: the
                                 algorithmic multiply-adds per offset (block edges add corners);
                                 at most SNCC_DIRECT_MAX_CORNERS: sncc_match reads these corners'
                                 table entries directly unless a 32-bit s may wrap */
    int32_t wide_blocks;  /* blocks and nonzero corners of the 64 x 64 block layout, which the */
    int32_t wide_corners; /* segment-sum kernels use for templates larger than 64 x 64 */
    int32_t pairs;        /* first layout: pairs of corners of one column 2 .. 7 rows apart with no
                             corner between them */
    int32_t sum_records;  /* the layout the segment-sum kernel walks (one block, else 64 x 64
                             blocks): its run, pair and single-corner records ... */
    int64_t sum_extra_rows; /* ... and the rows they span beyond their first, summed: a lane computing
                               R offset rows reads sum_records * R + sum_extra_rows table words */
    int32_t strided8;     /* first layout: runs of 8, 4 and 3 corners on every second row of one */
    int32_t strided4;     /* column (none between), and patterns of corners at rows Y, Y+2, Y+3: */
    int32_t strided3;     /* 8 runs8 + 4 runs4 + 2 runs2 + 2 pairs + runs1 + 8 strided8 + */
    int32_t t023;         /* 4 strided4 + 3 strided3 + 3 t023 = corners */
} sncc_plan_info;

/* Fills *out for seg; SNCC_ERR_UNIFORM when seg has no plan (Ek = 0). */
int sncc_get_plan_info(const sncc_segments* seg, sncc_plan_info* out);

/* Shared-memory read-bandwidth probe: `ctas` CTAs of 256 threads each read
 * 32-bit words from shared memory with conflict-free accesses, `iters`
 * rounds of 32 loads per thread, and store one checksum word per thread into
 * d_sink (ctas * 256 int32, device).  Bytes read = ctas*256*iters*32*4.
 * Used by the benchmark to measure the on-chip roofline of the segment-sum
 * kernel; not part of the matching path. */
int sncc_probe_smem_read(int32_t* d_sink, int ctas, int iters, sncc_stream_t stream);

/* Instruction-rate probe: `ctas` CTAs of 256 threads each issue `iters`
 * rounds of 64 instructions of one kind, in eight independent chains, and
 * store one checksum word per thread into d_sink (ctas * 256 int32, device).
 * kind SNCC_PROBE_DP4A: four-way unsigned byte dot product with 32-bit
 * accumulate (the exact comparator's multiply-add, 4 pixel MACs each);
 * kind SNCC_PROBE_IMAD_WIDE: signed 32 x 32 -> 64-bit multiply-add (the
 * segment-sum kernel's per-corner operation).  Instructions issued =
 * ctas*256*iters*64.  SNCC_ERR_ARG for another kind or a non-positive
 * size.  Used by the benchmark to measure ALU ceilings; not part of the
 * matching path. */
/* Bounded-wait test hook (no counterpart in the paper): one CTA waits on a
 * shared-memory mbarrier that nothing completes, with the same bounded wait
 * the segment-sum kernel uses for its TMA copies; after the wait limit (1 s)
 * it ORs SNCC_STATUS_WAIT_TIMEOUT into *d_status (int32, device) and returns.
 * No fault: the context stays usable.  SNCC_ERR_ARG for a null status. */
int sncc_probe_wait_timeout(int32_t* d_status, sncc_stream_t stream);

#define SNCC_PROBE_DP4A 0
#define SNCC_PROBE_IMAD_WIDE 1
int sncc_probe_alu(int kind, int32_t* d_sink, int ctas, int iters, sncc_stream_t stream);

/* HBM write-bandwidth probe: writes all `bytes` of d_buf (device, 16-byte
 * aligned, a multiple of 16, best larger than L2) with 16-byte stores; entry
 * i (16 bytes) becomes {lo, hi ^ 0x5a5a5a5a, 3 lo, lo ^ 0xffff} for the low
 * and high 32 bits of i.  The sum tables are almost all such stores, so the
 * benchmark reports them against this rate as well as against the copy
 * bandwidth; not part of the matching path.  SNCC_ERR_ARG for a null,
 * unaligned or ragged buffer. */
int sncc_probe_hbm_write(void* d_buf, size_t bytes, sncc_stream_t stream);

/* Library version string. */
const char* sncc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SNCC_H */
