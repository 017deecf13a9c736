"""Pins for the FP64 CPU oracle: each test checks the oracle against something
other than itself -- brute force, numpy's Pearson correlation (the textbook
form of Eq. 1), closed forms, invariants, and hand-derived split/merge
fixtures (tests/golden).  None of these needs a GPU."""
import numpy as np
import pytest

import oracle as O
from paper_2502_01286_gb300 import synth
from conftest import GOLDEN, load_golden


def pearson_map(f, t):
    """Eq. 1 through numpy's corrcoef on each window (library routine)."""
    f = np.asarray(f, np.float64)
    t = np.asarray(t, np.float64)
    N, M = f.shape
    H, W = t.shape
    out = np.zeros((N - H + 1, M - W + 1))
    tv = t.ravel()
    for v in range(N - H + 1):
        for u in range(M - W + 1):
            w = f[v:v + H, u:u + W].ravel()
            if w.std() == 0 or tv.std() == 0:
                out[v, u] = 0.0
            else:
                out[v, u] = np.corrcoef(w, tv)[0, 1]
    return out


# ---------------------------------------------------------------- sum tables
@pytest.mark.parametrize("M,N", [(1, 1), (7, 5), (13, 4), (3, 11)])
def test_sum_tables_brute_force(M, N):
    """Eq. 10 / Eq. 14 against the double sum over the upper-left rectangle."""
    f = synth.random_image(11 + M * N, M, N).astype(np.float64)
    s, s2 = O.sum_tables(f)
    assert s.shape == (N + 1, M + 1)
    assert np.all(s[0] == 0) and np.all(s[:, 0] == 0)
    for y in range(N):
        for x in range(M):
            assert s[y + 1, x + 1] == f[:y + 1, :x + 1].sum()
            assert s2[y + 1, x + 1] == (f[:y + 1, :x + 1] ** 2).sum()


def test_sum_tables_large_exact():
    """A 4096-wide table stays integer-exact (values up to 255*M*N)."""
    f = np.full((64, 4096), 255.0)
    s, s2 = O.sum_tables(f)
    assert s[-1, -1] == 255.0 * 64 * 4096
    assert s2[-1, -1] == 255.0 * 255.0 * 64 * 4096


def test_box_sum_eq11_against_slices():
    f = synth.random_image(5, 17, 9).astype(np.float64)
    s, _ = O.sum_tables(f)
    rng = np.random.default_rng(0)
    for _ in range(200):
        w = int(rng.integers(1, 18)); h = int(rng.integers(1, 10))
        X = int(rng.integers(0, 17 - w + 1)); Y = int(rng.integers(0, 9 - h + 1))
        assert O.box_sum(s, X, Y, w, h) == f[Y:Y + h, X:X + w].sum()


# ---------------------------------------------------------------- exact NCC
@pytest.mark.parametrize("shape", [((13, 9), (4, 3)), ((6, 17), (5, 2)), ((8, 8), (8, 8)), ((5, 7), (1, 6))])
def test_exact_ncc_vs_corrcoef(shape):
    """Eq. 1 against numpy's Pearson correlation, on non-square shapes so a
    transposed index fails."""
    (N, M), (H, W) = shape
    f = synth.random_image(101, M, N)
    t = synth.random_image(202, W, H)
    ref = pearson_map(f, t)
    got = O.ncc_exact_map(f, t)
    np.testing.assert_allclose(got, ref, atol=1e-12, rtol=0)


def test_exact_ncc_at_matches_map():
    f = synth.random_image(3, 21, 15)
    t = synth.random_image(4, 6, 5)
    mp = O.ncc_exact_map(f, t)
    u = np.array([0, 3, 15, 7]); v = np.array([0, 10, 2, 6])
    np.testing.assert_array_equal(O.ncc_exact_at(f, t, u, v), mp[v, u])


def test_exact_ncc_unaltered_crop_is_one():
    """An unaltered crop of the source matches with rho = 1 (P5)."""
    c = synth.case_plain(M=96, N=80, W=20, H=12, noise=0.0)
    u0, v0 = c.origin
    rho = O.ncc_exact_at(c.f, c.t, [u0], [v0])[0]
    assert abs(rho - 1.0) < 1e-12


def test_exact_ncc_bounds_and_affine():
    """rho in [-1, 1]; affine change a*t + b keeps rho for a > 0 and flips its
    sign for a < 0 (P4, P6)."""
    f = synth.random_image(7, 40, 30)
    t = synth.random_image(8, 9, 7).astype(np.float64)
    r = O.ncc_exact_map(f, t)
    assert np.all(np.abs(r) <= 1 + 1e-12)
    np.testing.assert_allclose(O.ncc_exact_map(f, 3 * t + 7), r, atol=1e-12)
    np.testing.assert_allclose(O.ncc_exact_map(f, -2 * t + 600), -r, atol=1e-12)


def test_exact_ncc_uniform_cases():
    """Uniform template or window: Eq. 1 is 0/0; the oracle's reading is 0."""
    f = synth.random_image(9, 20, 20)
    f[5:12, 5:12] = 77
    t = synth.random_image(10, 4, 4)
    r = O.ncc_exact_map(f, t)
    assert r[5, 5] == 0.0 and r[8, 8] == 0.0
    assert np.all(O.ncc_exact_map(f, np.full((4, 4), 3.0)) == 0.0)


def test_exact_ncc_rows_subset():
    f = synth.random_image(12, 30, 25)
    t = synth.random_image(13, 5, 6)
    full = O.ncc_exact_map(f, t)
    part = O.ncc_exact_map(f, t, rows=[0, 7, 19])
    for v in range(full.shape[0]):
        if v in (0, 7, 19):
            np.testing.assert_array_equal(part[v], full[v])
        else:
            assert np.all(np.isnan(part[v]))


# ---------------------------------------------------------------- segmentation
@pytest.mark.parametrize("name", GOLDEN)
def test_segmentation_golden(name):
    """Hand-derived split/merge fixtures (Section 5)."""
    g = load_golden(name)
    t = np.array(g["t"], np.float64)
    if g["split"] is not None:
        segs, mu = O.split_segments(t, g["sigma"])
        got = [tuple(int(v) for v in s) + (float(m),) for s, m in zip(segs, mu)]
        assert got == g["split"]
    ap = O.precompute_template_approximation(t, g["sigma"], g["kmax"])
    got = [tuple(int(v) for v in s) + (float(m),) for s, m in zip(ap.segments, ap.mu)]
    assert got == g["segments"]
    if "sigma_used" in g:
        assert ap.sigma_used == g["sigma_used"]
    if "rho_max" in g:
        assert abs(ap.rho_max - g["rho_max"]) < 1e-12


def _check_partition(ap, t, sigma):
    H, W = t.shape
    cover = np.zeros((H, W), np.int32)
    for (x, y, w, h), m in zip(ap.segments, ap.mu):
        assert w > 0 and h > 0 and x >= 0 and y >= 0 and x + w <= W and y + h <= H
        cover[y:y + h, x:x + w] += 1
        block = t[y:y + h, x:x + w]
        assert m == block.sum() / block.size
    assert np.all(cover == 1)


def _mergeable_pairs(ap):
    """Pairs that merge_redundant_segments would still join: same column span
    and vertically adjacent, or same row span and horizontally adjacent, with
    equal means."""
    segs = [tuple(int(v) for v in s) for s in ap.segments]
    mu = list(ap.mu)
    pos = {(s[0], s[1]): i for i, s in enumerate(segs)}
    bad = []
    for i, (x, y, w, h) in enumerate(segs):
        j = pos.get((x, y + h))
        if j is not None and segs[j][2] == w and mu[j] == mu[i]:
            bad.append((i, j))
        j = pos.get((x + w, y))
        if j is not None and segs[j][3] == h and mu[j] == mu[i]:
            bad.append((i, j))
    return bad


@pytest.mark.parametrize("sigma", [0.0, 2.0, 5.0, 10.0, 20.0])
def test_segmentation_invariants(sigma):
    """Segments tile the template, each satisfies Eq. 2 or is one pixel, the
    merge reached its fixpoint, and the table is ascending (y, x) (P7)."""
    c = synth.case_plain(M=120, N=100, W=37, H=29)
    t = c.t.astype(np.float64)
    ap = O.precompute_template_approximation(t, sigma)
    _check_partition(ap, t, sigma)
    for (x, y, w, h), m in zip(ap.segments, ap.mu):
        if w * h > 1:
            # a merged segment joins parts of equal mean; each part had std < sigma,
            # so the union's std is below sigma as well
            assert t[y:y + h, x:x + w].std() < sigma + 1e-9
    assert _mergeable_pairs(ap) == []
    keys = [(int(s[1]), int(s[0])) for s in ap.segments]
    assert keys == sorted(keys)


def test_split_emission_is_depth_first():
    """split_segment recurses into the first half before the second: with
    sigma = 0 every pixel is a segment and the emission order is the
    recursive-halving order (checked against an independent recursion)."""
    W, H = 5, 3
    t = np.arange(W * H, dtype=np.float64).reshape(H, W)
    segs, _ = O.split_segments(t, 0.0)

    def order(x, y, w, h):
        if w == 1 and h == 1:
            return [(x, y)]
        if w > h:
            a = (w + 1) // 2
            return order(x, y, a, h) + order(x + a, y, w - a, h)
        a = (h + 1) // 2
        return order(x, y, w, a) + order(x, y + a, w, h - a)

    assert [(int(s[0]), int(s[1])) for s in segs] == order(0, 0, W, H)


def test_sigma_above_template_std_gives_one_segment():
    """sigma_max above the template's std leaves a single segment (Section 3);
    its approximation is uniform, so its energy is 0 (P3)."""
    c = synth.case_plain(M=64, N=64, W=16, H=16)
    t = c.t.astype(np.float64)
    ap = O.precompute_template_approximation(t, t.std() + 0.01)
    assert ap.K == 1 and ap.ek == 0.0 and ap.rho_max == 0.0
    assert O.precompute_template_approximation(t, t.std() * 0.5).K > 1


def test_kmax_loop_raises_sigma():
    """Steps 1-2: sigma_max rises by one until K_split <= K_max; the previous
    sigma gave more than K_max segments."""
    c = synth.case_plain(M=96, N=96, W=40, H=40)
    t = c.t.astype(np.float64)
    ap0 = O.precompute_template_approximation(t, 0.0)
    kmax = max(2, ap0.k_split // 7)
    ap = O.precompute_template_approximation(t, 0.0, kmax)
    assert ap.k_split <= kmax and ap.sigma_used >= 1.0
    prev, _ = O.split_segments(t, ap.sigma_used - 1.0)
    assert len(prev) > kmax
    now, _ = O.split_segments(t, ap.sigma_used)
    assert len(now) == ap.k_split


def test_merge_only_joins_equal_means():
    segs = [(0, 0, 2, 1), (2, 0, 2, 1), (0, 1, 4, 1)]
    mu = [5.0, 5.0, 5.0]
    s, m = O.merge_segments(segs, mu)
    assert [tuple(int(v) for v in r) for r in s] == [(0, 0, 4, 2)]
    s, m = O.merge_segments(segs, [5.0, 6.0, 5.0])
    assert len(s) == 3


def test_rho_max_equals_exact_ncc_of_rendered_k():
    """rho_max (step 5-7) is NCC(t, k) by Eq. 1 with the rendered k."""
    c = synth.case_plain(M=80, N=80, W=24, H=20)
    t = c.t.astype(np.float64)
    ap = O.precompute_template_approximation(t, 6.0)
    k = ap.render()
    ref = np.corrcoef(t.ravel(), k.ravel())[0, 1]
    assert abs(ap.rho_max - ref) < 1e-12
    assert abs(ap.kbar - k.mean()) < 1e-12 and abs(ap.kbar - ap.tbar) < 1e-12
    assert abs(ap.ek - ((k - k.mean()) ** 2).sum()) < 1e-6


def test_literal_unweighted_energy_differs():
    """The unweighted reading of Eq. 17 drops the W_i*H_i weight: it only
    agrees with the weighted one when every segment is a single pixel."""
    c = synth.case_plain(M=64, N=64, W=16, H=16)
    t = c.t.astype(np.float64)
    a = O.precompute_template_approximation(t, 5.0, weighted=True)
    b = O.precompute_template_approximation(t, 5.0, weighted=False)
    n = a.segments[:, 2] * a.segments[:, 3]
    assert abs(a.ek - np.sum(n * (a.mu - a.kbar) ** 2)) < 1e-6
    assert abs(b.ek - np.sum((b.mu - b.kbar) ** 2)) < 1e-6
    assert (n > 1).any() and a.ek != b.ek


# ---------------------------------------------------------------- segmented NCC
@pytest.mark.parametrize("sigma", [3.0, 8.0, 15.0])
@pytest.mark.parametrize("method", ["direct", "sat"])
def test_segmented_ncc_is_pearson_of_rendered_k(sigma, method):
    """Segmented NCC (Eq. 9 / Eq. 12-18) equals Eq. 1 between f and the
    rendered approximation k, computed by numpy's Pearson correlation (P1).
    Non-square shapes catch transposed indices."""
    c = synth.case_plain(M=41, N=33, W=11, H=7)
    ap = O.precompute_template_approximation(c.t, sigma)
    ref = pearson_map(c.f, ap.render())
    got = O.segmented_ncc_map(c.f, ap, method=method)
    np.testing.assert_allclose(got, ref, atol=1e-10, rtol=0)


def test_segmented_equals_exact_at_sigma_zero():
    """sigma_max = 0 gives k = t, so segmented NCC equals exact NCC (P2)."""
    c = synth.case_plain(M=50, N=40, W=12, H=9)
    ap = O.precompute_template_approximation(c.t, 0.0)
    np.testing.assert_array_equal(ap.render(), c.t.astype(np.float64))
    np.testing.assert_allclose(O.segmented_ncc_map(c.f, ap, "sat"), O.ncc_exact_map(c.f, c.t), atol=1e-10)


def test_segmented_bounds_and_affine():
    """rho in [-1, 1]; the affine template a*t + b with sigma scaled by |a|
    gives the same segmentation and rho (a > 0) or -rho (a < 0)."""
    c = synth.case_plain(M=60, N=50, W=14, H=10)
    t = c.t.astype(np.float64)
    ap = O.precompute_template_approximation(t, 6.0)
    r = O.segmented_ncc_map(c.f, ap)
    assert np.all(np.abs(r) <= 1 + 1e-12)
    ap3 = O.precompute_template_approximation(3 * t + 7, 18.0)
    np.testing.assert_array_equal(ap3.segments, ap.segments)
    np.testing.assert_allclose(O.segmented_ncc_map(c.f, ap3), r, atol=1e-10)
    apn = O.precompute_template_approximation(-2 * t + 600, 12.0)
    np.testing.assert_array_equal(apn.segments, ap.segments)
    np.testing.assert_allclose(O.segmented_ncc_map(c.f, apn), -r, atol=1e-10)


def test_segmented_uniform_window_is_zero():
    c = synth.case_plain(M=40, N=40, W=8, H=8)
    f = c.f.copy()
    f[10:30, 10:30] = 90
    ap = O.precompute_template_approximation(c.t, 4.0)
    r = O.segmented_ncc_map(f, ap)
    assert np.all(r[10:23, 10:23] == 0.0)


def test_segmented_rows_subset_and_methods_agree():
    c = synth.case_plain(M=70, N=60, W=13, H=11)
    ap = O.precompute_template_approximation(c.t, 5.0)
    full = O.segmented_ncc_map(c.f, ap, "sat")
    part = O.segmented_ncc_map(c.f, ap, "direct", rows=[3, 40])
    np.testing.assert_allclose(part[[3, 40]], full[[3, 40]], atol=1e-11)


def test_f_bar_term_of_eq9_vanishes():
    """Eq. 9's fbar*W_i*H_i*(k_i - kbar) terms sum to zero by Eq. 7, so the
    numerator equals sum_i (box sum_i)(k_i - kbar) (checked with raw numpy)."""
    c = synth.case_plain(M=30, N=30, W=9, H=8)
    ap = O.precompute_template_approximation(c.t, 4.0)
    n = ap.segments[:, 2] * ap.segments[:, 3]
    assert abs(np.sum(n * (ap.mu - ap.kbar))) < 1e-9 * np.sum(n * np.abs(ap.mu))


# ---------------------------------------------------------------- two-stage search
def test_candidates_and_refine_brute_force():
    """Step 7 with the exact second stage: matches are exactly the offsets
    where the segmented rho passes tau_c and the exact rho passes tau_e."""
    c = synth.case_plain(M=48, N=40, W=10, H=8, noise=1.0)
    ap = O.precompute_template_approximation(c.t, 6.0)
    seg = pearson_map(c.f, ap.render())
    ex = pearson_map(c.f, c.t)
    tau_c, tau_e = 0.5, 0.6
    cand = O.candidates(O.segmented_ncc_map(c.f, ap), tau_c)
    U = ex.shape[1]
    idx, rho = O.refine(c.f, c.t, cand, U, tau_e)
    want = np.flatnonzero(((seg >= tau_c) & (ex >= tau_e)).ravel())
    np.testing.assert_array_equal(idx, want)
    np.testing.assert_allclose(rho, ex.ravel()[want], atol=1e-12)
    u0, v0 = c.origin
    assert v0 * U + u0 in set(idx.tolist())


def test_main_algorithm_two_approximations_brute_force():
    """Section 5 main algorithm: matches are the offsets where Eq. 1 against
    the rendered k_fast passes precision * rho_fast and Eq. 1 against the
    rendered k_slow passes precision * rho_slow (numpy Pearson correlation),
    with sigma_fast = 0.99 sigma_t and sigma_slow = 0.1 sigma_t."""
    c = synth.case_plain(M=56, N=44, W=12, H=10, noise=1.0, seed=4321)
    p = 0.6
    r = O.main_algorithm(c.f, c.t, precision=p)
    st = c.t.astype(np.float64).std()
    ap_f = O.precompute_template_approximation(c.t, 0.99 * st, 5000)
    ap_s = O.precompute_template_approximation(c.t, 0.1 * st, 5000)
    np.testing.assert_array_equal(r["fast"].segments, ap_f.segments)
    np.testing.assert_array_equal(r["slow"].segments, ap_s.segments)
    pf = pearson_map(c.f, ap_f.render())
    ps = pearson_map(c.f, ap_s.render())
    want = np.flatnonzero(((pf >= p * ap_f.rho_max) & (ps >= p * ap_s.rho_max)).ravel())
    np.testing.assert_array_equal(r["idx"], want)
    np.testing.assert_allclose(r["rho"], ps.ravel()[want], atol=1e-10)
    assert len(want) > 0 and ap_s.K > ap_f.K


# ---------------------------------------------------------------- differentiable loss
def _diff_problem(seed=3, M=15, N=12, W=6, H=5, sigma=4.0):
    from oracle import diff as D  # noqa: F401
    g = np.random.default_rng(seed)
    f = g.uniform(0, 255, size=(N, M))
    t = f[3:3 + H, 4:4 + W] + g.normal(0, 3.0, size=(H, W))
    ap = O.precompute_template_approximation(t, sigma)
    kv = ap.mu + g.normal(0, 2.0, size=ap.K)  # move off the fitted means
    return f, t, ap.segments, kv


def test_diff_forward_matches_segmented_ncc():
    """The differentiable forward with k_i = the segment means is the
    segmented NCC of Eq. 18 (weighted energy) and Eq. 1."""
    from oracle import diff as D
    f, t, rects, _ = _diff_problem()
    ap = O.precompute_template_approximation(t, 4.0)
    fw = D.forward(f, t, rects, ap.mu)
    np.testing.assert_allclose(fw["rho_k"], O.segmented_ncc_map(f, ap, "direct"), atol=1e-12)
    np.testing.assert_allclose(fw["rho_t"], O.ncc_exact_map(f, t), atol=1e-12)


def test_diff_gradients_vs_central_differences():
    """Analytic dL/dk and dL/df against FP64 central differences of the loss
    (step 1e-5 in intensity units)."""
    from oracle import diff as D
    f, t, rects, kv = _diff_problem()
    gr = D.gradients(f, t, rects, kv)
    eps = 1e-5
    num_k = np.empty(len(kv))
    for j in range(len(kv)):
        kp = kv.copy(); kp[j] += eps
        km = kv.copy(); km[j] -= eps
        num_k[j] = (D.forward(f, t, rects, kp)["loss"] - D.forward(f, t, rects, km)["loss"]) / (2 * eps)
    np.testing.assert_allclose(gr["dk"], num_k, rtol=1e-6, atol=1e-9 * np.abs(num_k).max())
    rng = np.random.default_rng(0)
    for _ in range(25):
        y, x = int(rng.integers(0, f.shape[0])), int(rng.integers(0, f.shape[1]))
        fp = f.copy(); fp[y, x] += eps
        fm = f.copy(); fm[y, x] -= eps
        num = (D.forward(fp, t, rects, kv)["loss"] - D.forward(fm, t, rects, kv)["loss"]) / (2 * eps)
        assert abs(gr["df"][y, x] - num) <= 1e-6 * max(1e-3, np.abs(gr["df"]).max())
    assert np.abs(gr["df"]).max() > 0 and np.abs(gr["dk"]).max() > 0


def test_diff_loss_zero_when_k_is_t():
    """With every pixel its own segment and k = t, rho_k = rho_t and L = 0,
    so both gradients vanish."""
    from oracle import diff as D
    f, t, _, _ = _diff_problem()
    H, W = t.shape
    rects = np.array([(x, y, 1, 1) for y in range(H) for x in range(W)])
    gr = D.gradients(f, t, rects, t.ravel())
    assert gr["loss"] < 1e-20
    assert np.abs(gr["dk"]).max() < 1e-9 and np.abs(gr["df"]).max() < 1e-9
