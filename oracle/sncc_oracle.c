/*
 * sncc_oracle.c - plain, slow, FP64 CPU oracle for segmented normalized
 * cross-correlation (Marusic, Popovic, Kalafatic, "Template Matching in Images
 * using Segmented Normalized Cross-Correlation", arXiv 2502.01286).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * library: it is written from the paper's equations and pseudocode alone.
 *
 * Conventions (paper Section 2): an image f of size M x N is stored row-major,
 * f[y*M + x], x in [0, M) the column and y in [0, N) the row.  A template t of
 * size W x H is stored the same way, t[y*W + x].  Offsets (u, v) range over
 * {0..M-W} x {0..N-H} (main algorithm, step 7).  All arithmetic is double
 * precision; pixel values are passed in as doubles (uint8 images are exact).
 *
 * Readings of the paper that this file takes (each one is also listed in the
 * design notes of the repository):
 *  - Eq. 17 and step 6 of precompute_template_approximation print the
 *    template-approximation energy without the W_i*H_i weight.  Taken
 *    literally, rho is not bounded by [-1, 1] and does not equal the exact NCC
 *    when k = t.  The default here is the weighted energy
 *    sum_i W_i H_i (k_i - kbar)^2 = sum_{x,y} (k(x,y) - kbar)^2, consistent with
 *    Eq. 5 and Eq. 7; the literal unweighted form is available behind a flag.
 *  - Eq. 1 is undefined when the window or the template is uniform (Section 2
 *    rules those cases out of scope).  Here rho := 0 whenever either energy is
 *    exactly zero.
 *  - Eq. 2 is evaluated as  n*S2 - S*S < n*n*sigma^2  (S, S2 the segment's sum
 *    and sum of squares, n = W_i*H_i), which is sigma_i < sigma_max squared and
 *    multiplied by n^2; for integer images every term is exact in double.
 *  - split_segment splits the width only when width > height, so a square
 *    splits its height; the first half receives ceil(size/2).
 *  - merge_redundant_segments compares segment means with plain double
 *    equality, as printed.
 *
 * Parity status: every function here is pinned by the CPU tests (brute force,
 * library Pearson correlation, invariants, hand-worked split/merge cases).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Row-parallel driver: splits offset rows over plain pthreads.        */
/* Each offset is computed independently, so results do not depend on */
/* the thread count.                                                   */
/* ------------------------------------------------------------------ */
typedef void (*orc_row_fn)(void* ctx, int row);

typedef struct {
    orc_row_fn fn;
    void* ctx;
    const int* rows;
    int nrows;
    int tid;
    int nthreads;
} orc_job;

static void* orc_worker(void* p)
{
    orc_job* j = (orc_job*)p;
    for (int r = j->tid; r < j->nrows; r += j->nthreads) j->fn(j->ctx, j->rows[r]);
    return NULL;
}

static void orc_run_rows(orc_row_fn fn, void* ctx, const int* rows, int nrows, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > nrows) nthreads = nrows > 0 ? nrows : 1;
    pthread_t th[256];
    orc_job jobs[256];
    for (int i = 0; i < nthreads; ++i) {
        jobs[i].fn = fn; jobs[i].ctx = ctx; jobs[i].rows = rows; jobs[i].nrows = nrows;
        jobs[i].tid = i; jobs[i].nthreads = nthreads;
    }
    if (nthreads == 1) { orc_worker(&jobs[0]); return; }
    for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, orc_worker, &jobs[i]);
    for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
}

/* ------------------------------------------------------------------ */
/* Sum tables, Eq. 10 and Eq. 14.                                      */
/* s and s2 are (N+1) x (M+1), row-major; entry [(y+1)*(M+1) + (x+1)]  */
/* holds s(x, y).  Row 0 and column 0 hold s(-1, .) = s(., -1) = 0.    */
/* ------------------------------------------------------------------ */
void orc_sum_tables(const double* f, int M, int N, double* s, double* s2)
{
    const int P = M + 1;
    for (int X = 0; X < P; ++X) { s[X] = 0.0; s2[X] = 0.0; }
    for (int y = 0; y < N; ++y) {
        s[(y + 1) * P] = 0.0;
        s2[(y + 1) * P] = 0.0;
        for (int x = 0; x < M; ++x) {
            const double v = f[(size_t)y * M + x];
            /* Eq. 10: s(u,v) = f(u,v) + s(u-1,v) + s(u,v-1) - s(u-1,v-1) */
            s[(size_t)(y + 1) * P + (x + 1)] = v + s[(size_t)(y + 1) * P + x]
                                             + s[(size_t)y * P + (x + 1)] - s[(size_t)y * P + x];
            /* Eq. 14: the same recurrence on f^2 */
            s2[(size_t)(y + 1) * P + (x + 1)] = v * v + s2[(size_t)(y + 1) * P + x]
                                              + s2[(size_t)y * P + (x + 1)] - s2[(size_t)y * P + x];
        }
    }
}

/* s(x, y) of Eq. 10 with the zero border for x = -1 or y = -1. */
static inline double orc_s(const double* s, int M, int x, int y)
{
    return s[(size_t)(y + 1) * (M + 1) + (x + 1)];
}

/* Eq. 11: sum of f over the rectangle with top-left (X, Y) and size w x h,
 * read from the sum table at four corners. */
double orc_box_sum(const double* s, int M, int X, int Y, int w, int h)
{
    return orc_s(s, M, X - 1, Y - 1) - orc_s(s, M, X - 1, Y + h - 1)
         - orc_s(s, M, X + w - 1, Y - 1) + orc_s(s, M, X + w - 1, Y + h - 1);
}

/* ------------------------------------------------------------------ */
/* Exact NCC, Eq. 1, evaluated directly (two passes: means, then the   */
/* centred sums).                                                      */
/* ------------------------------------------------------------------ */
static double orc_template_mean(const double* t, int W, int H)
{
    double st = 0.0;
    for (int i = 0; i < W * H; ++i) st += t[i];
    return st / ((double)W * (double)H);
}

static double orc_template_energy(const double* t, int W, int H, double tbar)
{
    double et = 0.0;
    for (int i = 0; i < W * H; ++i) { const double d = t[i] - tbar; et += d * d; }
    return et;
}

static double orc_ncc_exact_one(const double* f, int M, const double* t, int W, int H,
                                double tbar, double et, int u, int v)
{
    double sf = 0.0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) sf += f[(size_t)(v + y) * M + (u + x)];
    const double fbar = sf / ((double)W * (double)H);
    double num = 0.0, ef = 0.0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const double df = f[(size_t)(v + y) * M + (u + x)] - fbar;
            const double dt = t[y * W + x] - tbar;
            num += df * dt;
            ef += df * df;
        }
    if (ef == 0.0 || et == 0.0) return 0.0; /* uniform window or template */
    return num / sqrt(ef * et);
}

typedef struct {
    const double* f; int M, N;
    const double* t; int W, H;
    double tbar, et;
    double* out; int U;
} orc_exact_ctx;

static void orc_exact_row(void* p, int v)
{
    orc_exact_ctx* c = (orc_exact_ctx*)p;
    for (int u = 0; u < c->U; ++u)
        c->out[(size_t)v * c->U + u] = orc_ncc_exact_one(c->f, c->M, c->t, c->W, c->H, c->tbar, c->et, u, v);
}

/* Exact NCC map over the given offset rows v (out is V x U, rows not listed
 * are left untouched). */
void orc_ncc_exact_map(const double* f, int M, int N, const double* t, int W, int H,
                       const int* rows, int nrows, double* out, int nthreads)
{
    orc_exact_ctx c;
    c.f = f; c.M = M; c.N = N; c.t = t; c.W = W; c.H = H;
    c.tbar = orc_template_mean(t, W, H);
    c.et = orc_template_energy(t, W, H, c.tbar);
    c.out = out; c.U = M - W + 1;
    orc_run_rows(orc_exact_row, &c, rows, nrows, nthreads);
}

/* Exact NCC at a list of offsets (u[i], v[i]). */
void orc_ncc_exact_at(const double* f, int M, int N, const double* t, int W, int H,
                      const int* u, const int* v, int n, double* out)
{
    (void)N;
    const double tbar = orc_template_mean(t, W, H);
    const double et = orc_template_energy(t, W, H, tbar);
    for (int i = 0; i < n; ++i) out[i] = orc_ncc_exact_one(f, M, t, W, H, tbar, et, u[i], v[i]);
}

/* ------------------------------------------------------------------ */
/* Segmented template approximation, Section 3 and Section 5.          */
/* ------------------------------------------------------------------ */
typedef struct {
    int x, y, w, h; /* top-left corner and size in template coordinates */
    double mu;      /* segment value k_i, Eq. 4 */
} orc_seg;

typedef struct {
    orc_seg* v;
    int n, cap;
} orc_segvec;

static void orc_push(orc_segvec* k, int x, int y, int w, int h, double mu)
{
    if (k->n == k->cap) {
        k->cap = k->cap ? 2 * k->cap : 64;
        k->v = (orc_seg*)realloc(k->v, (size_t)k->cap * sizeof(orc_seg));
    }
    orc_seg s = {x, y, w, h, mu};
    k->v[k->n++] = s;
}

/* function split_segment (Section 5). */
static void orc_split_segment(const double* t, int W, double sigma_max,
                              int x, int y, int width, int height, orc_segvec* k)
{
    /* step 1: a single pixel is always a segment */
    if (width == 1 && height == 1) {
        orc_push(k, x, y, 1, 1, t[y * W + x]);
        return;
    }
    /* step 2: mean and standard deviation of the segment (Eq. 2) */
    double S = 0.0, S2 = 0.0;
    for (int yy = y; yy < y + height; ++yy)
        for (int xx = x; xx < x + width; ++xx) {
            const double p = t[yy * W + xx];
            S += p;
            S2 += p * p;
        }
    const double n = (double)width * (double)height;
    const double mu = S / n;
    /* step 3: std < sigma_max, squared and scaled by n^2 */
    if (n * S2 - S * S < n * n * sigma_max * sigma_max) {
        orc_push(k, x, y, width, height, mu);
        return;
    }
    /* steps 4-5: halve the larger dimension, first half gets the ceiling */
    if (width > height) {
        const int a = (width + 1) / 2, b = width / 2;
        orc_split_segment(t, W, sigma_max, x, y, a, height, k);
        orc_split_segment(t, W, sigma_max, x + a, y, b, height, k);
    } else {
        const int a = (height + 1) / 2, b = height / 2;
        orc_split_segment(t, W, sigma_max, x, y, width, a, k);
        orc_split_segment(t, W, sigma_max, x, y + a, width, b, k);
    }
}

static int orc_cmp_xy(const void* pa, const void* pb)
{
    const orc_seg* a = (const orc_seg*)pa;
    const orc_seg* b = (const orc_seg*)pb;
    if (a->x != b->x) return a->x < b->x ? -1 : 1;
    if (a->y != b->y) return a->y < b->y ? -1 : 1;
    return 0;
}

static int orc_cmp_yx(const void* pa, const void* pb)
{
    const orc_seg* a = (const orc_seg*)pa;
    const orc_seg* b = (const orc_seg*)pb;
    if (a->y != b->y) return a->y < b->y ? -1 : 1;
    if (a->x != b->x) return a->x < b->x ? -1 : 1;
    return 0;
}

/* function merge_redundant_segments (Section 5). */
static void orc_merge_redundant_segments(orc_segvec* k)
{
    for (;;) {
        /* step 1: sort on (x, y) */
        qsort(k->v, (size_t)k->n, sizeof(orc_seg), orc_cmp_xy);
        /* step 2: merge vertically */
        int i = 0;
        while (i < k->n - 1) {
            if (k->v[i].w == 0 || k->v[i].h == 0) { i += 1; continue; }
            int j = i + 1;
            while (j < k->n && k->v[i].x == k->v[j].x && k->v[i].w == k->v[j].w &&
                   k->v[i].y + k->v[i].h == k->v[j].y && k->v[i].mu == k->v[j].mu) {
                k->v[i].h += k->v[j].h;
                k->v[j].h = 0;
                j += 1;
            }
            i = j;
        }
        /* step 3: sort on (y, x) */
        qsort(k->v, (size_t)k->n, sizeof(orc_seg), orc_cmp_yx);
        /* step 4: merge horizontally */
        i = 0;
        while (i < k->n - 1) {
            if (k->v[i].w == 0 || k->v[i].h == 0) { i += 1; continue; }
            int j = i + 1;
            while (j < k->n && k->v[i].y == k->v[j].y && k->v[i].h == k->v[j].h &&
                   k->v[i].x + k->v[i].w == k->v[j].x && k->v[i].mu == k->v[j].mu) {
                k->v[i].w += k->v[j].w;
                k->v[j].w = 0;
                j += 1;
            }
            i = j;
        }
        /* step 5: drop degenerate segments */
        int m = 0;
        for (int a = 0; a < k->n; ++a)
            if (k->v[a].w != 0 && k->v[a].h != 0) k->v[m++] = k->v[a];
        const int changed = (m != k->n);
        k->n = m;
        /* step 6 */
        if (!changed) return;
    }
}

/* function precompute_template_approximation (Section 5), extended to report
 * the quantities the matching stage needs.
 *
 *  t, W, H       template
 *  sigma_max     starting threshold of Eq. 2
 *  k_max         maximum segment count (0: no cap, the loop runs once)
 *  weighted      1: energy sum_i W_i H_i (k_i - kbar)^2; 0: literal Eq. 17
 *  out_segs      receives a malloc'ed array of K segments (caller frees with
 *                orc_free), in the order merge_redundant_segments leaves them
 *  info[0..6]    K, K before merging, sigma used by the last split, kbar,
 *                template-approximation energy, tbar, rho_max
 */
int orc_precompute_template_approximation(const double* t, int W, int H, double sigma_max, int k_max,
                                          int weighted, orc_seg** out_segs, double* info)
{
    orc_segvec k = {NULL, 0, 0};
    double sigma = sigma_max, sigma_used = sigma_max;
    /* step 1-2: repeat the split, raising sigma_max by one, until K <= K_max */
    for (;;) {
        k.n = 0;
        orc_split_segment(t, W, sigma, 0, 0, W, H, &k);
        sigma_used = sigma;
        sigma = sigma + 1.0;
        if (k_max <= 0 || k.n <= k_max) break;
    }
    const int k_split = k.n;
    /* step 3 */
    orc_merge_redundant_segments(&k);
    /* step 4: kbar (Eq. 7) and tbar */
    double sk = 0.0;
    for (int i = 0; i < k.n; ++i) sk += (double)k.v[i].w * (double)k.v[i].h * k.v[i].mu;
    const double n = (double)W * (double)H;
    const double kbar = sk / n;
    const double tbar = orc_template_mean(t, W, H);
    /* step 5: numerator, sum over segments of (segment sum - tbar n_i)(k_i - kbar) */
    double num = 0.0, ek = 0.0;
    for (int i = 0; i < k.n; ++i) {
        const orc_seg* s = &k.v[i];
        double ssum = 0.0;
        for (int yy = s->y; yy < s->y + s->h; ++yy)
            for (int xx = s->x; xx < s->x + s->w; ++xx) ssum += t[yy * W + xx];
        const double ni = (double)s->w * (double)s->h;
        const double c = s->mu - kbar;
        num += (ssum - tbar * ni) * c;
        ek += (weighted ? ni : 1.0) * c * c;
    }
    /* step 6: denominator */
    const double et = orc_template_energy(t, W, H, tbar);
    const double den = sqrt(et * ek);
    info[0] = (double)k.n;
    info[1] = (double)k_split;
    info[2] = sigma_used;
    info[3] = kbar;
    info[4] = ek;
    info[5] = tbar;
    info[6] = den > 0.0 ? num / den : 0.0;
    *out_segs = k.v;
    return k.n;
}

void orc_free(void* p) { free(p); }

/* Split alone (no merge), for the tests of split_segment. */
int orc_split_only(const double* t, int W, int H, double sigma_max, orc_seg** out_segs)
{
    orc_segvec k = {NULL, 0, 0};
    orc_split_segment(t, W, sigma_max, 0, 0, W, H, &k);
    *out_segs = k.v;
    return k.n;
}

/* Merge alone, on a caller-supplied list (copied), for the merge tests. */
int orc_merge_only(const orc_seg* in, int n, orc_seg** out_segs)
{
    orc_segvec k = {NULL, 0, 0};
    for (int i = 0; i < n; ++i) orc_push(&k, in[i].x, in[i].y, in[i].w, in[i].h, in[i].mu);
    orc_merge_redundant_segments(&k);
    *out_segs = k.v;
    return k.n;
}

/* ------------------------------------------------------------------ */
/* Segmented NCC.                                                      */
/* ------------------------------------------------------------------ */
typedef struct {
    const double* f; int M, N;
    const orc_seg* seg; int K; int W, H;
    double kbar, ek;
    const double* s; const double* s2; /* sum tables for the SAT route */
    double* out; int U;
} orc_segncc_ctx;

/* Eq. 9 evaluated pixel by pixel over each segment, before any sum table:
 * num = sum_i sum_{(x,y) in S_i} (f(u+x, v+y) - fbar) (k_i - kbar);
 * denominator sqrt(sum (f - fbar)^2 * energy of k). */
static void orc_segncc_direct_row(void* p, int v)
{
    orc_segncc_ctx* c = (orc_segncc_ctx*)p;
    const double n = (double)c->W * (double)c->H;
    for (int u = 0; u < c->U; ++u) {
        double sf = 0.0;
        for (int y = 0; y < c->H; ++y)
            for (int x = 0; x < c->W; ++x) sf += c->f[(size_t)(v + y) * c->M + (u + x)];
        const double fbar = sf / n;
        double ef = 0.0;
        for (int y = 0; y < c->H; ++y)
            for (int x = 0; x < c->W; ++x) {
                const double d = c->f[(size_t)(v + y) * c->M + (u + x)] - fbar;
                ef += d * d;
            }
        double num = 0.0;
        for (int i = 0; i < c->K; ++i) {
            const orc_seg* s = &c->seg[i];
            double part = 0.0;
            for (int y = s->y; y < s->y + s->h; ++y)
                for (int x = s->x; x < s->x + s->w; ++x)
                    part += c->f[(size_t)(v + y) * c->M + (u + x)] - fbar;
            num += part * (s->mu - c->kbar);
        }
        c->out[(size_t)v * c->U + u] = (ef == 0.0 || c->ek == 0.0) ? 0.0 : num / sqrt(ef * c->ek);
    }
}

/* Eq. 12 - Eq. 18 through the sum tables: window sums by Eq. 13 and Eq. 15,
 * local energy by Eq. 16, numerator by Eq. 12 (including the fbar W_i H_i
 * term), denominator by Eq. 17, rho by Eq. 18. */
static void orc_segncc_sat_row(void* p, int v)
{
    orc_segncc_ctx* c = (orc_segncc_ctx*)p;
    const int M = c->M, W = c->W, H = c->H;
    for (int u = 0; u < c->U; ++u) {
        /* Eq. 13 */
        const double sf = orc_s(c->s, M, u + W - 1, v + H - 1) - orc_s(c->s, M, u - 1, v + H - 1)
                        - orc_s(c->s, M, u + W - 1, v - 1) + orc_s(c->s, M, u - 1, v - 1);
        /* Eq. 15 */
        const double sf2 = orc_s(c->s2, M, u + W - 1, v + H - 1) - orc_s(c->s2, M, u - 1, v + H - 1)
                         - orc_s(c->s2, M, u + W - 1, v - 1) + orc_s(c->s2, M, u - 1, v - 1);
        /* step 7b */
        const double fbar = sf / ((double)W * (double)H);
        /* Eq. 12 */
        double num = 0.0;
        for (int i = 0; i < c->K; ++i) {
            const orc_seg* s = &c->seg[i];
            const double box = orc_box_sum(c->s, M, u + s->x, v + s->y, s->w, s->h);
            num += (box - fbar * (double)s->w * (double)s->h) * (s->mu - c->kbar);
        }
        /* Eq. 16 */
        const double ef = sf2 - fbar * sf;
        /* Eq. 17 and Eq. 18 */
        c->out[(size_t)v * c->U + u] = (ef <= 0.0 || c->ek == 0.0) ? 0.0 : num / sqrt(ef * c->ek);
    }
}

/* Segmented NCC map over the given offset rows.
 *  method 0: Eq. 9 pixel by pixel; method 1: sum tables (Eq. 10 - Eq. 18).
 *  seg/K, kbar, ek describe the approximation (ek as returned by
 *  orc_precompute_template_approximation). */
void orc_segncc_map(const double* f, int M, int N, const orc_seg* seg, int K, int W, int H,
                    double kbar, double ek, int method, const int* rows, int nrows,
                    double* out, int nthreads)
{
    orc_segncc_ctx c;
    c.f = f; c.M = M; c.N = N; c.seg = seg; c.K = K; c.W = W; c.H = H;
    c.kbar = kbar; c.ek = ek; c.out = out; c.U = M - W + 1;
    c.s = NULL; c.s2 = NULL;
    double* s = NULL;
    double* s2 = NULL;
    if (method == 1) {
        s = (double*)malloc(sizeof(double) * (size_t)(M + 1) * (size_t)(N + 1));
        s2 = (double*)malloc(sizeof(double) * (size_t)(M + 1) * (size_t)(N + 1));
        orc_sum_tables(f, M, N, s, s2);
        c.s = s; c.s2 = s2;
        orc_run_rows(orc_segncc_sat_row, &c, rows, nrows, nthreads);
    } else {
        orc_run_rows(orc_segncc_direct_row, &c, rows, nrows, nthreads);
    }
    free(s);
    free(s2);
}
