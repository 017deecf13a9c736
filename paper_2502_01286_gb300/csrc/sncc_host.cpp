// sncc_host.cpp - host side of the library: split-and-merge template
// approximation (Section 3, Section 5) and the matching plan.
//
// The segmentation follows the paper's definitions step for step (the table
// it produces is part of the method's result and is compared bit for bit),
// but the statistics of each candidate rectangle come from exact integer sum
// tables of the template instead of per-pixel loops.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "sncc.h"
#include "sncc_internal.h"

namespace sncc {

namespace {

// Exact integer sum tables of a uint8 template, padded with a zero row and
// column: tab[Y * (W+1) + X] = sum over x < X, y < Y.
struct TemplateSums {
    int W = 0, H = 0;
    std::vector<int64_t> s, s2;
    void build(const uint8_t* t, int W_, int H_, int stride) {
        W = W_;
        H = H_;
        const int P = W + 1;
        s.assign((size_t)P * (H + 1), 0);
        s2.assign((size_t)P * (H + 1), 0);
        for (int y = 0; y < H; ++y) {
            int64_t row = 0, row2 = 0;
            for (int x = 0; x < W; ++x) {
                const int64_t v = t[(size_t)y * stride + x];
                row += v;
                row2 += v * v;
                s[(size_t)(y + 1) * P + x + 1] = s[(size_t)y * P + x + 1] + row;
                s2[(size_t)(y + 1) * P + x + 1] = s2[(size_t)y * P + x + 1] + row2;
            }
        }
    }
    int64_t box(const std::vector<int64_t>& tab, int x, int y, int w, int h) const {
        const int P = W + 1;
        return tab[(size_t)(y + h) * P + x + w] - tab[(size_t)y * P + x + w] - tab[(size_t)(y + h) * P + x] +
               tab[(size_t)y * P + x];
    }
};

struct Seg {
    int x, y, w, h;
    int64_t sum;
    double mean;
};

// split_segment (Section 5), depth first with the first half before the
// second, as the recursion orders it.  Eq. 2 is tested as
// n*S2 - S*S < n*n*sigma^2 in double with the same association everywhere.
void split(const TemplateSums& ts, const uint8_t* t, int stride, double sigma, std::vector<Seg>& out) {
    struct R { int x, y, w, h; };
    std::vector<R> stack;
    stack.push_back({0, 0, ts.W, ts.H});
    out.clear();
    while (!stack.empty()) {
        const R r = stack.back();
        stack.pop_back();
        if (r.w == 1 && r.h == 1) {
            const int64_t v = t[(size_t)r.y * stride + r.x];
            out.push_back({r.x, r.y, 1, 1, v, (double)v});
            continue;
        }
        const int64_t S = ts.box(ts.s, r.x, r.y, r.w, r.h);
        const int64_t S2 = ts.box(ts.s2, r.x, r.y, r.w, r.h);
        const double n = (double)r.w * (double)r.h;
        const double Sd = (double)S, S2d = (double)S2;
        const double lhs = n * S2d - Sd * Sd;
        const double rhs = n * n * sigma * sigma;
        if (lhs < rhs) {
            out.push_back({r.x, r.y, r.w, r.h, S, Sd / n});
            continue;
        }
        if (r.w > r.h) {
            const int a = (r.w + 1) / 2;
            stack.push_back({r.x + a, r.y, r.w - a, r.h});
            stack.push_back({r.x, r.y, a, r.h});
        } else {
            const int a = (r.h + 1) / 2;
            stack.push_back({r.x, r.y + a, r.w, r.h - a});
            stack.push_back({r.x, r.y, r.w, a});
        }
    }
}

// merge_redundant_segments (Section 5): alternate a vertical pass over the
// (x, y)-sorted list and a horizontal pass over the (y, x)-sorted list, each
// extending a segment by the chain of equal-mean neighbours that share its
// column (row) span, until a round removes nothing.
void merge(std::vector<Seg>& k) {
    auto by_xy = [](const Seg& a, const Seg& b) { return a.x != b.x ? a.x < b.x : a.y < b.y; };
    auto by_yx = [](const Seg& a, const Seg& b) { return a.y != b.y ? a.y < b.y : a.x < b.x; };
    for (;;) {
        std::sort(k.begin(), k.end(), by_xy);
        for (size_t i = 0; i + 1 < k.size();) {
            if (k[i].w == 0 || k[i].h == 0) { ++i; continue; }
            size_t j = i + 1;
            while (j < k.size() && k[j].x == k[i].x && k[j].w == k[i].w && k[j].y == k[i].y + k[i].h &&
                   k[j].mean == k[i].mean) {
                k[i].h += k[j].h;
                k[i].sum += k[j].sum;
                k[j].h = 0;
                ++j;
            }
            i = j;
        }
        std::sort(k.begin(), k.end(), by_yx);
        for (size_t i = 0; i + 1 < k.size();) {
            if (k[i].w == 0 || k[i].h == 0) { ++i; continue; }
            size_t j = i + 1;
            while (j < k.size() && k[j].y == k[i].y && k[j].h == k[i].h && k[j].x == k[i].x + k[i].w &&
                   k[j].mean == k[i].mean) {
                k[i].w += k[j].w;
                k[i].sum += k[j].sum;
                k[j].w = 0;
                ++j;
            }
            i = j;
        }
        const size_t before = k.size();
        k.erase(std::remove_if(k.begin(), k.end(), [](const Seg& s) { return s.w == 0 || s.h == 0; }), k.end());
        if (k.size() == before) return;
    }
}

// round(num / den) to nearest, ties away from zero, den > 0.
__int128 round_div(__int128 num, __int128 den) {
    if (num >= 0) return (2 * num + den) / (2 * den);
    return -((2 * (-num) + den) / (2 * den));
}

}  // namespace

// Cuts the rendered weights qimg (W x H) into blocks of BW x BH with region
// pitch WP and appends the layout's arrays (blocks, corner list, run
// descriptors, runs) to `image`, recording their byte offsets in L.
static void build_layout(const std::vector<int32_t>& qimg, int W, int H, int BW, int BH, int WP, Layout& L,
                  std::vector<int32_t>& image) {
    L.BW = BW;
    L.BH = BH;
    L.WP = WP;
    L.nbx = (W + BW - 1) / BW;
    L.nby = (H + BH - 1) / BH;
    std::vector<int32_t> blocks, corners, runblk, runs;
    L.max_corners = 0;
    L.nonzero_corners = 0;
    L.records = 0;
    L.extra_rows = 0;
    for (int k = 0; k < 4; ++k) L.runs[k] = 0;
    for (int k = 0; k < PAIR_GAPS; ++k) L.pairs[k] = 0;
    for (int k = 0; k < 3; ++k) L.runs2[k] = 0;
    L.t21 = 0;
    for (int by_i = 0; by_i < L.nby; ++by_i) {
        for (int bx_i = 0; bx_i < L.nbx; ++bx_i) {
            const int bx = bx_i * BW, by = by_i * BH;
            const int bw = std::min(BW, W - bx), bh = std::min(BH, H - by);
            auto q = [&](int X, int Y) -> int64_t {  // block-local, zero outside
                if (X < 0 || Y < 0 || X >= bw || Y >= bh) return 0;
                return qimg[(size_t)(by + Y) * W + (bx + X)];
            };
            std::vector<int32_t> G((size_t)(bw + 1) * (bh + 1));  // G[X * (bh + 1) + Y], column-major
            const int first = (int)(corners.size() / 2);
            for (int Y = 0; Y <= bh; ++Y)
                for (int X = 0; X <= bw; ++X) {
                    const int64_t g = q(X - 1, Y - 1) - q(X, Y - 1) - q(X - 1, Y) + q(X, Y);
                    G[(size_t)X * (bh + 1) + Y] = (int32_t)g;
                    if (g != 0) {
                        corners.push_back(Y * WP + X);
                        corners.push_back((int32_t)g);
                        ++L.nonzero_corners;
                    }
                }
            // pad to a multiple of 4 corners with zero weights (16-byte loads
            // of two corners, groups of four, no tail in the kernel)
            while (((corners.size() / 2) - first) % 4 != 0) {
                corners.push_back(0);
                corners.push_back(0);
            }
            const int cnt = (int)(corners.size() / 2) - first;
            if (cnt == 0) continue;  // a block inside one segment adds nothing
            blocks.push_back(bx);
            blocks.push_back(by);
            blocks.push_back(first);
            blocks.push_back(cnt);
            L.max_corners = std::max(L.max_corners, cnt);

            // Vertical runs: walking each column downwards, the first
            // uncovered corner starts the longest run of 8, 4 or 2 whose rows
            // all hold corners (and stay inside the block's corner grid);
            // otherwise the longest stride-2 run of 8, 4 or 3 (corners every
            // second row, none between), or corners at rows Y, Y+2, Y+3
            // (none at Y+1), or it pairs with the next corner of the column
            // if that one is 2 .. 7 rows below (the rows between them hold
            // none), else it is a single corner.  A lane then reads each
            // table word its record spans once for all of the record's
            // corners.
            std::vector<int32_t> cls[4], pcls[PAIR_GAPS], s2cls[3], tcls;
            for (int X = 0; X <= bw; ++X) {
                const int32_t* col = &G[(size_t)X * (bh + 1)];
                for (int Y = 0; Y <= bh;) {
                    if (col[Y] == 0) {
                        ++Y;
                        continue;
                    }
                    int k = 3;
                    for (int c = 0; c < 3; ++c) {
                        const int len = RUN_LEN[c];
                        if (Y + len - 1 > bh) continue;
                        bool full = true;
                        for (int i = 0; i < len && full; ++i) full = col[Y + i] != 0;
                        if (full) {
                            k = c;
                            break;
                        }
                    }
                    ++L.records;
                    if (k == 3) {  // no run: a stride-2 run?
                        int k2 = -1;
                        for (int c = 0; c < 3 && k2 < 0; ++c) {
                            const int len = RUN2_LEN[c];
                            if (Y + 2 * (len - 1) > bh) continue;
                            bool ok = true;
                            for (int i = 0; i < len && ok; ++i) ok = col[Y + 2 * i] != 0;
                            for (int i = 0; i + 1 < len && ok; ++i) ok = col[Y + 2 * i + 1] == 0;
                            if (ok) k2 = c;
                        }
                        if (k2 >= 0) {
                            const int len = RUN2_LEN[k2];
                            std::vector<int32_t>& sc = s2cls[k2];
                            sc.push_back(4 * (Y * WP + X));
                            for (int i = 0; i < len; ++i) sc.push_back(col[Y + 2 * i]);
                            while (sc.size() % 4 != 0) sc.push_back(0);
                            ++L.runs2[k2];
                            L.extra_rows += 2 * (len - 1);
                            Y += 2 * (len - 1) + 1;
                            continue;
                        }
                        if (Y + 3 <= bh && col[Y + 1] == 0 && col[Y + 2] != 0 && col[Y + 3] != 0) {
                            tcls.push_back(4 * (Y * WP + X));
                            tcls.push_back(col[Y]);
                            tcls.push_back(col[Y + 2]);
                            tcls.push_back(col[Y + 3]);
                            ++L.t21;
                            L.extra_rows += 3;
                            Y += 4;
                            continue;
                        }
                    }
                    if (k == 3) {  // a pair with the next corner of the column?
                        int d = 1;
                        while (d <= PAIR_MAX_GAP && Y + d <= bh && col[Y + d] == 0) ++d;
                        if (d >= PAIR_MIN_GAP && d <= PAIR_MAX_GAP && Y + d <= bh) {
                            std::vector<int32_t>& pc = pcls[d - PAIR_MIN_GAP];
                            pc.push_back(4 * (Y * WP + X));
                            pc.push_back(col[Y]);
                            pc.push_back(col[Y + d]);
                            pc.push_back(0);
                            ++L.pairs[d - PAIR_MIN_GAP];
                            L.extra_rows += d;
                            Y += d + 1;
                            continue;
                        }
                    }
                    const int len = RUN_LEN[k];
                    cls[k].push_back(4 * (Y * WP + X));  // byte offset in the region
                    for (int i = 0; i < len; ++i) cls[k].push_back(col[Y + i]);
                    if (k < 3)  // pad the record to its int4 units
                        while (cls[k].size() % (4 * RUN_INT4[k]) != 0) cls[k].push_back(0);
                    ++L.runs[k];
                    L.extra_rows += len - 1;
                    Y += len;
                }
            }
            while (cls[3].size() % 8 != 0) cls[3].push_back(0);  // whole groups of 4 single corners
            for (int k = 0; k < 4; ++k) {
                runblk.push_back((int32_t)(runs.size() / 4));
                runblk.push_back(k < 3 ? (int32_t)(cls[k].size() / (4 * RUN_INT4[k])) : (int32_t)(cls[3].size() / 2));
                runs.insert(runs.end(), cls[k].begin(), cls[k].end());
            }
            for (int k = 0; k < PAIR_GAPS; ++k) {
                runblk.push_back((int32_t)(runs.size() / 4));
                runblk.push_back((int32_t)(pcls[k].size() / 4));
                runs.insert(runs.end(), pcls[k].begin(), pcls[k].end());
            }
            for (int k = 0; k < 3; ++k) {  // stride-2 runs: records of RUN_INT4[k] int4 units
                runblk.push_back((int32_t)(runs.size() / 4));
                const int units = k == 0 ? 3 : (k == 1 ? 2 : 1);
                runblk.push_back((int32_t)(s2cls[k].size() / (4 * units)));
                while (s2cls[k].size() % (4 * units) != 0) s2cls[k].push_back(0);
                runs.insert(runs.end(), s2cls[k].begin(), s2cls[k].end());
            }
            runblk.push_back((int32_t)(runs.size() / 4));
            runblk.push_back((int32_t)(tcls.size() / 4));
            runs.insert(runs.end(), tcls.begin(), tcls.end());
            static_assert(8 + 2 * PAIR_GAPS + 8 == 4 * RUNBLK_INT4, "runblk holds every record class");
        }
    }
    L.nblk = (int)(blocks.size() / 4);
    L.total_corners = (int)(corners.size() / 2);
    L.blocks_offset = image.size() * 4;
    image.insert(image.end(), blocks.begin(), blocks.end());
    L.corners_offset = image.size() * 4;
    image.insert(image.end(), corners.begin(), corners.end());
    L.runblk_offset = image.size() * 4;
    image.insert(image.end(), runblk.begin(), runblk.end());
    L.runs_offset = image.size() * 4;
    image.insert(image.end(), runs.begin(), runs.end());
    L.end_offset = image.size() * 4;
}

// Builds the fixed-point weights and the block layouts of the plan.
int build_plan(const sncc_segments* s, Plan& p, bool small_blocks) {
    const int W = s->W, H = s->H;
    const int64_t n = (int64_t)W * H;
    p.W = W;
    p.H = H;
    p.n = (double)n;
    p.Ek = s->Ek;

    // Fixed-point scale: every |G| <= 4 max|q_i| must stay below 2^31.
    double maxc = 0.0;
    for (int i = 0; i < s->K; ++i) maxc = std::max(maxc, std::fabs(s->seg[i].mean - s->kbar));
    int F = 30;
    if (maxc > 0.0) {
        while (F > 0 && maxc * std::ldexp(1.0, F) + 1.0 >= std::ldexp(1.0, 29)) --F;
    }
    p.F = F;

    // q_i = round(2^F (sum_i * n - T * n_i) / (n_i * n)), exact in 128 bits.
    std::vector<int32_t> qimg((size_t)W * H, 0);
    int64_t Q0 = 0;
    for (int i = 0; i < s->K; ++i) {
        const sncc_seg& g = s->seg[i];
        const int64_t ni = (int64_t)g.w * g.h;
        const __int128 num = ((__int128)g.sum * n - (__int128)s->T * ni) * ((__int128)1 << F);
        const __int128 q = round_div(num, (__int128)ni * n);
        const int32_t qi = (int32_t)q;
        for (int y = g.y; y < g.y + g.h; ++y)
            for (int x = g.x; x < g.x + g.w; ++x) qimg[(size_t)y * W + x] = qi;
        Q0 += (int64_t)qi * ni;
    }
    p.Q0 = Q0;

    // Corners of the whole template as one block: the algorithmic count, and
    // for sparse templates the direct corner list.
    p.template_corners = 0;
    auto qa = [&](int X, int Y) -> int64_t {
        return (X < 0 || Y < 0 || X >= W || Y >= H) ? 0 : qimg[(size_t)Y * W + X];
    };
    std::vector<int32_t> direct;
    for (int Y = 0; Y <= H; ++Y)
        for (int X = 0; X <= W; ++X) {
            const int64_t g = qa(X - 1, Y - 1) - qa(X, Y - 1) - qa(X - 1, Y) + qa(X, Y);
            if (g == 0) continue;
            ++p.template_corners;
            if ((int)direct.size() / 4 < DIRECT_MAX + 1) {
                direct.push_back(X);
                direct.push_back(Y);
                direct.push_back((int32_t)g);
                direct.push_back(0);
            }
        }

    // Region pitches are compile-time widths of the kernels, multiples of 4
    // so that a region row is a whole number of 16-byte units.
    p.image.clear();
    const bool single = W <= BLOCK_SINGLE_MAX && H <= BLOCK_SINGLE_MAX;
    const int bw0 = single ? W : std::min(W, BLOCK_MULTI), bh0 = single ? H : std::min(H, BLOCK_MULTI);
    build_layout(qimg, W, H, bw0, bh0, bw0 <= 32 ? 68 : 100, p.lay[0], p.image);
    build_layout(qimg, W, H, std::min(W, BLOCK_SINGLE_MAX), std::min(H, BLOCK_SINGLE_MAX), 100, p.lay[1], p.image);
    if (small_blocks)
        build_layout(qimg, W, H, std::min(W, BLOCK_MULTI), std::min(H, BLOCK_MULTI), 68, p.lay[2], p.image);
    p.direct_count = p.template_corners <= DIRECT_MAX ? p.template_corners : 0;
    p.direct_offset = p.image.size() * 4;
    if (p.direct_count > 0) p.image.insert(p.image.end(), direct.begin(), direct.begin() + 4 * p.direct_count);
    p.image.insert(p.image.end(), 4, 0);
    return SNCC_OK;
}

Plan* plan_of(const sncc_segments* s) { return s ? static_cast<Plan*>(s->plan) : nullptr; }

int sm_count() {
    static std::atomic<int> cached[kDeviceSlots];  // 0 = not yet queried
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 0;
    if (dev < kDeviceSlots) {
        const int c = cached[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 0;
    if (dev < kDeviceSlots) cached[dev].store(n, std::memory_order_relaxed);
    return n;
}

const char* error_string(int code) {
    switch (code) {
        case SNCC_OK: return "ok";
        case SNCC_ERR_ARG: return "invalid argument";
        case SNCC_ERR_UNIFORM: return "uniform template or zero-energy approximation";
        case SNCC_ERR_DTYPE: return "32-bit sum table wraps where whole entries are read";
        case SNCC_ERR_CAPACITY: return "capacity too small";
        case SNCC_ERR_CUDA: return "CUDA error";
        case SNCC_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case SNCC_ERR_NOMEM: return "host allocation failed";
        case SNCC_ERR_UNSUPPORTED: return "size not supported";
        default: return "unknown error";
    }
}

// The population std of a template from its exact sums (the Eq. 2 std taken
// over the whole template): sqrt(n T2 - T^2) / n, the radicand exact in int64.
double template_sigma(int64_t n, int64_t T, int64_t T2) {
    const int64_t var_n2 = n * T2 - T * T;
    return var_n2 > 0 ? std::sqrt((double)var_n2) / (double)n : 0.0;
}

}  // namespace sncc

extern "C" {

const char* sncc_error_string(int code) { return sncc::error_string(code); }

const char* sncc_version(void) { return "sncc 0.1 (sm_103a)"; }

void sncc_free_segments(sncc_segments* s) {
    if (!s) return;
    std::free(s->seg);
    delete static_cast<sncc::Plan*>(s->plan);
    std::memset(s, 0, sizeof(*s));
}

int sncc_build_segments(const uint8_t* t, int W, int H, int t_stride, double sigma_max, int k_max,
                        sncc_segments* out) {
    sncc::NvtxRange nvtx_range("sncc_build_segments");
    using namespace sncc;
    if (!t || !out || W <= 0 || H <= 0 || t_stride < W || !(sigma_max == sigma_max)) return SNCC_ERR_ARG;
    if ((int64_t)W * H > ((int64_t)1 << 23)) return SNCC_ERR_UNSUPPORTED;
    std::memset(out, 0, sizeof(*out));
    try {
        TemplateSums ts;
        ts.build(t, W, H, t_stride);
        std::vector<Seg> k;
        double sigma = sigma_max, used = sigma_max;
        // precompute_template_approximation steps 1-2
        for (;;) {
            split(ts, t, t_stride, sigma, k);
            used = sigma;
            sigma = sigma + 1.0;
            if (k_max <= 0 || (int64_t)k.size() <= k_max) break;
        }
        const int k_split = (int)k.size();
        merge(k);  // step 3

        const int64_t n = (int64_t)W * H;
        const int64_t T = ts.box(ts.s, 0, 0, W, H);
        const int64_t T2 = ts.box(ts.s2, 0, 0, W, H);
        out->K = (int32_t)k.size();
        out->K_split = k_split;
        out->W = W;
        out->H = H;
        out->sigma_used = used;
        out->T = T;
        out->T2 = T2;
        out->sigma_t = template_sigma(n, T, T2);
        // Eq. 7: sum_i n_i k_i = sum_i (segment sum) = T, so kbar = T / n.
        out->kbar = (double)T / (double)n;
        out->seg = static_cast<sncc_seg*>(std::malloc(sizeof(sncc_seg) * (k.size() ? k.size() : 1)));
        if (!out->seg) return SNCC_ERR_NOMEM;
        double Ek = 0.0;
        for (size_t i = 0; i < k.size(); ++i) {
            sncc_seg& g = out->seg[i];
            g.x = k[i].x;
            g.y = k[i].y;
            g.w = k[i].w;
            g.h = k[i].h;
            g.sum = k[i].sum;
            g.mean = k[i].mean;
            const double c = g.mean - out->kbar;
            Ek += (double)g.w * (double)g.h * c * c;
        }
        out->Ek = Ek;
        // Steps 4-7: the numerator sum_i (sum_i - tbar n_i)(k_i - kbar) equals
        // Ek because k_i n_i = sum_i and tbar = kbar, so rho_max = sqrt(Ek / Et)
        // with Et = (n T2 - T^2) / n exactly.
        const double Et = (double)(n * T2 - T * T) / (double)n;
        out->rho_max = (Et > 0.0 && Ek > 0.0) ? std::sqrt(Ek / Et) : 0.0;

        Plan* p = new Plan();
        out->plan = p;
        if (Ek > 0.0) {
            build_plan(out, *p);
            // |rho_gpu - rho| from quantising c_i to q_i / 2^F is at most
            // 2^-(F+1) sqrt(n / Ek); float rounding adds a few 1e-7.
            out->err_bound = std::ldexp(1.0, -(p->F + 1)) * std::sqrt((double)n / Ek) + 1e-6;
        }
    } catch (const std::bad_alloc&) {
        sncc_free_segments(out);
        return SNCC_ERR_NOMEM;
    }
    return SNCC_OK;
}

int sncc_template_sigma(const uint8_t* t, int W, int H, int t_stride, double* sigma_t) {
    if (!t || !sigma_t || W <= 0 || H <= 0 || t_stride < W) return SNCC_ERR_ARG;
    if ((int64_t)W * H > ((int64_t)1 << 23)) return SNCC_ERR_UNSUPPORTED;
    int64_t T = 0, T2 = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const int64_t v = t[(size_t)y * t_stride + x];
            T += v;
            T2 += v * v;
        }
    *sigma_t = sncc::template_sigma((int64_t)W * H, T, T2);
    return SNCC_OK;
}

int sncc_get_plan_info(const sncc_segments* seg, sncc_plan_info* out) {
    const sncc::Plan* p = sncc::plan_of(seg);
    if (!out || !p) return SNCC_ERR_ARG;
    if (p->image.empty()) return SNCC_ERR_UNIFORM;
    out->F = p->F;
    const sncc::Layout& L = p->lay[0];
    out->blocks = L.nblk;
    out->block_w = L.BW;
    out->block_h = L.BH;
    out->corners = L.nonzero_corners;
    out->max_corners = L.max_corners;
    out->Q0 = p->Q0;
    out->runs8 = L.runs[0];
    out->runs4 = L.runs[1];
    out->runs2 = L.runs[2];
    out->runs1 = L.runs[3];
    out->template_corners = p->template_corners;
    out->wide_blocks = p->lay[1].nblk;
    out->wide_corners = p->lay[1].nonzero_corners;
    out->pairs = 0;
    for (int k = 0; k < sncc::PAIR_GAPS; ++k) out->pairs += L.pairs[k];
    const sncc::Layout& S = sncc::layout_for(*p);
    out->sum_records = S.records;
    out->sum_extra_rows = S.extra_rows;
    out->strided8 = L.runs2[0];
    out->strided4 = L.runs2[1];
    out->strided3 = L.runs2[2];
    out->t023 = L.t21;
    return SNCC_OK;
}

int sncc_sat_pitch(int M) {
    if (M < 0) return -1;
    return ((M + 1) + 31) / 32 * 32;
}

size_t sncc_plan_bytes(const sncc_segments* seg) {
    const sncc::Plan* p = sncc::plan_of(seg);
    if (!p) return 0;
    return p->image.size() * sizeof(int32_t);
}

int sncc_plan_upload(const sncc_segments* seg, void* d_plan, size_t plan_bytes, sncc_stream_t stream) {
    const sncc::Plan* p = sncc::plan_of(seg);
    if (!p || !d_plan) return SNCC_ERR_ARG;
    if (p->image.empty()) return SNCC_ERR_UNIFORM;
    const size_t need = p->image.size() * sizeof(int32_t);
    if (plan_bytes < need || (reinterpret_cast<uintptr_t>(d_plan) & 15)) return SNCC_ERR_WORKSPACE;
    if (cudaMemcpyAsync(d_plan, p->image.data(), need, cudaMemcpyHostToDevice, (cudaStream_t)stream) != cudaSuccess)
        return SNCC_ERR_CUDA;
    return SNCC_OK;
}

}  // extern "C"
