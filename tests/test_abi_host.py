"""CPU tests of the C ABI: the library builds and loads, exports every entry
point include/sncc.h declares, and its host logic (split-and-merge
segmentation, argument checks) agrees with the oracle.  No GPU is touched:
only host-side functions and calls rejected before any CUDA work run here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2502_01286_gb300 import build as sncc_build
from paper_2502_01286_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sncc():
    sncc_build.build()
    from paper_2502_01286_gb300 import sncc as mod
    return mod


def header_functions():
    text = open(os.path.join(ROOT, "include", "sncc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sncc_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_four_paper_calls():
    fns = header_functions()
    for name in ["sncc_build_segments", "sncc_integral", "sncc_match", "sncc_refine"]:
        assert name in fns


def test_library_exports_every_declared_symbol(sncc):
    lib = sncc.lib()
    missing = [f for f in header_functions() if not hasattr(lib, f)]
    assert missing == []
    assert set(sncc.EXPORTED) <= set(header_functions())


def test_version_and_error_strings(sncc):
    assert "sm_103a" in sncc.version()
    assert sncc.lib().sncc_error_string(-2).decode().startswith("uniform")


def test_sat_pitch(sncc):
    for M in [1, 30, 31, 32, 255, 1920, 4096]:
        p = sncc.sat_pitch(M)
        assert p >= M + 1 and p % 32 == 0 and p - (M + 1) < 32


@pytest.mark.parametrize("shape,sigma,kmax", [
    ((32, 32), 10.0, 0), ((64, 64), 5.0, 0), ((64, 64), 20.0, 0), ((37, 29), 0.0, 0), ((29, 37), 3.0, 0),
    ((48, 48), 12.0, 0), ((40, 40), 0.0, 150), ((1, 1), 1.0, 0), ((7, 1), 0.5, 0), ((1, 9), 2.0, 0)])
def test_segmentation_bit_exact_vs_oracle(sncc, shape, sigma, kmax):
    """Segment table, K before merging and the sigma of the last split equal
    the oracle's exactly (Section 5)."""
    H, W = shape
    c = synth.case_plain(M=max(64, W + 8), N=max(64, H + 8), W=W, H=H)
    seg = sncc.build_segments(c.t, sigma, kmax)
    ap = O.precompute_template_approximation(c.t, sigma, kmax)
    np.testing.assert_array_equal(seg.table, ap.segments)
    np.testing.assert_array_equal(seg.means, ap.mu)
    assert seg.K_split == ap.k_split and seg.sigma_used == ap.sigma_used
    assert abs(seg.kbar - ap.kbar) < 1e-12
    assert abs(seg.Ek - ap.ek) <= 1e-9 * max(1.0, ap.ek)
    assert abs(seg.rho_max - ap.rho_max) < 1e-12
    # exact sums agree with the template
    for (x, y, w, h), s in zip(seg.table, seg.sums):
        assert s == int(c.t[y:y + h, x:x + w].astype(np.int64).sum())
    assert seg.T == int(c.t.astype(np.int64).sum())
    assert seg.T2 == int((c.t.astype(np.int64) ** 2).sum())


def test_segmentation_large_template_bit_exact(sncc):
    """A 256 x 256 high-texture template at sigma 5 (thousands of segments)."""
    f = synth.rectangles(synth.rng(77), 300, 300, 40) + synth.fractal_noise(synth.rng(78), 300, 300, 40.0)
    t = synth.quantise(f)[20:276, 10:266]
    seg = sncc.build_segments(t, 5.0)
    ap = O.precompute_template_approximation(t, 5.0)
    assert seg.K > 1000
    np.testing.assert_array_equal(seg.table, ap.segments)
    np.testing.assert_array_equal(seg.means, ap.mu)


@pytest.mark.parametrize("name", sorted(f for f in os.listdir(os.path.join(ROOT, "tests", "golden"))
                                        if f.endswith(".txt") and f != "README.txt"))
def test_segmentation_golden(sncc, name):
    from conftest import load_golden
    g = load_golden(name)
    t = np.array(g["t"], np.uint8)
    seg = sncc.build_segments(t, g["sigma"], g["kmax"])
    got = [tuple(int(v) for v in r) + (float(m),) for r, m in zip(seg.table, seg.means)]
    assert got == g["segments"]
    if "sigma_used" in g:
        assert seg.sigma_used == g["sigma_used"]


def test_uniform_template_has_zero_energy(sncc):
    seg = sncc.build_segments(np.full((8, 8), 7, np.uint8), 1.0)
    assert seg.K == 1 and seg.Ek == 0.0 and seg.plan_bytes() == 0
    assert sncc.lib().sncc_plan_upload(seg.ref(), C.c_void_p(16), 0, None) == sncc.ERR_UNIFORM


@pytest.mark.parametrize("shape,seed", [((32, 32), 1), ((256, 256), 2), ((7, 3), 3), ((1, 1), 4), ((48, 17), 5)])
def test_template_sigma_is_population_std(sncc, shape, seed):
    """sigma_t (Section 5's input to sigma_max,fast and sigma_max,slow) from
    the library, both through sncc_template_sigma and in sncc_segments,
    against numpy's population std of the pixels."""
    t = synth.random_image(seed, shape[1], shape[0])
    want = float(np.asarray(t, np.float64).std())
    got = sncc.template_sigma(t)
    assert got == pytest.approx(want, rel=1e-12, abs=1e-12)
    assert sncc.build_segments(t, 5.0).sigma_t == got
    assert sncc.template_sigma(np.full((9, 4), 200, np.uint8)) == 0.0


def test_quantisation_error_bound_is_small(sncc):
    c = synth.case_hd(M=200, N=200)
    for sigma in (5.0, 10.0, 20.0):
        seg = sncc.build_segments(c.t, sigma)
        assert 0 < seg.err_bound < 5e-6


def covered(pi):
    """Corners in the plan's records (runs, stride-2 runs, patterns, pairs, singles)."""
    return (8 * pi["runs8"] + 4 * pi["runs4"] + 2 * pi["runs2"] + 2 * pi["pairs"] + pi["runs1"] +
            8 * pi["strided8"] + 4 * pi["strided4"] + 3 * pi["strided3"] + 3 * pi["t023"])


def test_vertical_runs_partition_the_corners(sncc):
    # every nonzero corner lands in exactly one run of 8, 4, 2 or 1 or one
    # pair of corners 2 .. 7 rows apart
    yy, xx = np.mgrid[0:19, 0:21]
    checker = ((xx + yy) % 2 * 200).astype(np.uint8)
    cases = [synth.case_hd(M=200, N=200).t, synth.case_plain().t, checker,
             synth.case_texture(M=600, N=600, W=150, H=90).t]
    for t in cases:
        for sigma in (2.0, 8.0, 20.0):
            seg = sncc.build_segments(t, sigma)
            if seg.Ek == 0.0:
                continue
            pi = seg.plan_info()
            assert covered(pi) == pi["corners"]
    # a 1-pixel checkerboard puts a corner on every point of the 22 x 20
    # corner grid: each column of 20 splits into runs of 8, 8 and 4
    pi = sncc.build_segments(checker, 1.0).plan_info()
    assert (pi["corners"], pi["runs8"], pi["runs4"], pi["runs2"], pi["runs1"]) == (440, 44, 22, 0, 0)
    # three horizontal bands of height 3 (values 10, 200, 50) on a 4 x 9
    # template: corners only in columns 0 and 4, at rows 0, 3, 6 and 9, so
    # each column gives two pairs 3 rows apart; each pair spans 3 extra rows
    bands = np.repeat(np.array([10, 200, 50], np.uint8), 3)[:, None] * np.ones((1, 4), np.uint8)
    pi = sncc.build_segments(bands, 1.0).plan_info()
    assert (pi["corners"], pi["pairs"], pi["runs8"], pi["runs4"], pi["runs2"], pi["runs1"]) == (8, 4, 0, 0, 0, 0)
    assert (pi["sum_records"], pi["sum_extra_rows"]) == (4, 12)
    # bands of height 2 (values 10, 200, 50, 120) on a 4 x 8 template: corners
    # in columns 0 and 4 at rows 0, 2, 4, 6, 8: a stride-2 run of 4 (rows 0 -
    # 6, 6 extra rows) and a single corner per column
    bands2 = np.repeat(np.array([10, 200, 50, 120], np.uint8), 2)[:, None] * np.ones((1, 4), np.uint8)
    pi = sncc.build_segments(bands2, 1.0).plan_info()
    assert (pi["corners"], pi["strided4"], pi["runs1"], pi["pairs"], pi["strided8"], pi["strided3"]) == \
        (10, 2, 2, 0, 0, 0)
    assert (pi["sum_records"], pi["sum_extra_rows"]) == (4, 12)
    # bands of heights 2, 1, 1 on a 3 x 4 template: corners in columns 0
    # and 3 at rows 0, 2, 3 and 4; rows 0, 2, 3 form the (Y, Y+2, Y+3)
    # pattern (3 extra rows) and row 4 is a single corner, per column
    t3 = np.array([[10] * 3, [10] * 3, [200] * 3, [60] * 3], np.uint8)
    pi = sncc.build_segments(t3, 1.0).plan_info()
    assert (pi["corners"], pi["t023"], pi["runs1"], covered(pi)) == (8, 2, 2, 8)
    assert (pi["sum_records"], pi["sum_extra_rows"]) == (4, 6)


@pytest.mark.parametrize("W,H", [(1, 64), (64, 1), (3, 256), (256, 3), (65, 64), (64, 65), (700, 2), (2, 700)])
def test_plan_shapes_thin_and_edge_templates(sncc, W, H):
    """Thin templates and templates one pixel past a block edge: the plan's
    blocks cover the template, the runs partition the corners, and the
    one-block layout applies exactly up to 64 x 64."""
    t = synth.random_image(W * 1000 + H, W, H)
    seg = sncc.build_segments(t, 20.0)
    if not seg.Ek > 0:
        pytest.skip("uniform approximation")
    pi = seg.plan_info()
    assert covered(pi) == pi["corners"]
    if W <= 64 and H <= 64:
        assert pi["blocks"] == 1 and pi["wide_blocks"] == 1 and pi["corners"] == pi["template_corners"]
    else:
        nb64 = -(-W // 64) * -(-H // 64)
        assert 1 <= pi["wide_blocks"] <= nb64
        assert pi["wide_corners"] >= pi["template_corners"]  # block edges only add corners


def test_host_argument_errors(sncc):
    lib = sncc.lib()
    seg = sncc.build_segments(synth.case_plain().t, 10.0)
    out = sncc._Segments()
    assert lib.sncc_build_segments(None, 4, 4, 4, 1.0, 0, C.byref(out)) == sncc.ERR_ARG
    t = np.zeros((4, 4), np.uint8)
    assert lib.sncc_build_segments(t.ctypes.data, 4, 4, 3, 1.0, 0, C.byref(out)) == sncc.ERR_ARG
    assert lib.sncc_build_segments(t.ctypes.data, 0, 4, 4, 1.0, 0, C.byref(out)) == sncc.ERR_ARG
    big = np.zeros(1, np.uint8)
    assert lib.sncc_build_segments(big.ctypes.data, 4096, 4096, 4096, 1.0, 0, C.byref(out)) == sncc.ERR_UNSUPPORTED
    # device calls rejected on their arguments before any CUDA call
    assert lib.sncc_integral(None, 10, 10, 10, None, 32, None, 32, None, 0, None) == sncc.ERR_ARG
    assert lib.sncc_integral(C.c_void_p(256), 10, 10, 10, C.c_void_p(256), 16, C.c_void_p(256), 32, None, 0,
                             None) == sncc.ERR_ARG
    # a 32-bit table that wraps (255 M N >= 2^31) is refused only where whole entries are read
    assert lib.sncc_refine_segmented(seg.ref(), C.c_void_p(256), C.c_void_p(256), 32, C.c_void_p(256), 4128, 4096,
                                     4096, None, C.c_void_p(256), 0, 0.5, None, 0, C.c_void_p(256), None, 0,
                                     C.c_void_p(256), None) == sncc.ERR_DTYPE
    assert lib.sncc_integral(C.c_void_p(256), 10, 10, 10, C.c_void_p(256), 32, C.c_void_p(256), 32, None, 0,
                             None) == sncc.ERR_WORKSPACE
    assert lib.sncc_match(seg.ref(), None, None, 32, None, 32, 64, 64, 0.5, None, 0, None, 0, None, None,
                          None) == sncc.ERR_ARG
    assert lib.sncc_refine(None, 64, 64, 64, None, 8, 8, 8, 0, 0, None, None, 0, 0.5, None, 0, None, None, 0,
                           None, None) == sncc.ERR_ARG
    assert lib.sncc_exact_map(C.c_void_p(256), 64, 64, 64, C.c_void_p(256), 8, 8, 8, 64 * 7, 64 * 49,
                              C.c_void_p(256), 32, C.c_void_p(256), 96, C.c_void_p(256), 57,
                              None) == sncc.ERR_UNIFORM
    assert lib.sncc_probe_alu(2, C.c_void_p(256), 1, 1, None) == sncc.ERR_ARG
    assert lib.sncc_probe_alu(sncc.PROBE_DP4A, C.c_void_p(256), 0, 1, None) == sncc.ERR_ARG
    assert lib.sncc_probe_alu(sncc.PROBE_IMAD_WIDE, None, 1, 1, None) == sncc.ERR_ARG
    assert lib.sncc_probe_hbm_write(None, 1 << 20, None) == sncc.ERR_ARG
    assert lib.sncc_probe_hbm_write(C.c_void_p(256), 1000, None) == sncc.ERR_ARG  # not a multiple of 16
    assert lib.sncc_probe_hbm_write(C.c_void_p(264), 1 << 20, None) == sncc.ERR_ARG  # not 16-byte aligned
    assert lib.sncc_refine_segmented_tiles_workspace_bytes(0, 5, 1, 1, 4) == 0
    assert lib.sncc_refine_segmented_tiles_workspace_bytes(64, 64, 65, 8, 4) == 0
    assert lib.sncc_refine_segmented_tiles_workspace_bytes(256, 256, 32, 32, 16) >= 225 * 225 // 8
    assert lib.sncc_refine_segmented_tiles(seg.ref(), None, None, 32, None, 32, 64, 64, None, None, 0, 0.5, None,
                                           0, None, None, 0, None, None) == sncc.ERR_ARG
    assert lib.sncc_integral_workspace_bytes(0, 5) == 0
    # the fused multi-approximation match: 1 .. SNCC_MULTI_MAX approximations, all pointer arrays given
    segs = (C.POINTER(sncc._Segments) * 5)(*[C.pointer(seg._s)] * 5)
    ptrs = (C.c_void_p * 5)(*[256] * 5)
    taus = (C.c_float * 5)(*[0.5] * 5)
    for n in (0, 5):
        assert lib.sncc_match_multi(segs, ptrs, n, C.c_void_p(256), 32, C.c_void_p(256), 96, 64, 64, taus, None, 0,
                                    ptrs, 16, ptrs, ptrs, None) == sncc.ERR_ARG
    assert lib.sncc_match_multi(None, ptrs, 2, C.c_void_p(256), 32, C.c_void_p(256), 96, 64, 64, taus, None, 0,
                                ptrs, 16, ptrs, ptrs, None) == sncc.ERR_ARG
    assert lib.sncc_match_multi(segs, ptrs, 2, C.c_void_p(256), 32, C.c_void_p(256), 96, 64, 64, None, None, 0,
                                ptrs, 16, ptrs, ptrs, None) == sncc.ERR_ARG
    assert lib.sncc_match_multi(segs, ptrs, 2, C.c_void_p(256), 32, C.c_void_p(256), 96, 64, 64, taus, None, 0,
                                ptrs, 16, ptrs, None, None) == sncc.ERR_ARG
    nulls = (C.c_void_p * 5)(256, None, 256, 256, 256)  # a missing status word
    assert lib.sncc_match_multi(segs, ptrs, 2, C.c_void_p(256), 32, C.c_void_p(256), 96, 64, 64, taus, None, 0,
                                ptrs, 16, ptrs, nulls, None) == sncc.ERR_ARG


def test_misaligned_device_pointers_are_rejected(sncc):
    """Every call loads and stores its device arrays by their element type; a
    pointer off that alignment, or a batch table pitch that is not a multiple
    of 4, is an argument error found on the host instead of a device fault.
    Address 256 stands for an aligned pointer; 258, 260 and 264 are off by 2,
    4 and 8 bytes."""
    lib = sncc.lib()
    seg = sncc.build_segments(synth.case_plain().t, 10.0)  # 32 x 32 template
    ok, a2, a4, a8 = (C.c_void_p(x) for x in (256, 258, 260, 264))
    # segment sum: tables 16 (s) and 8 (s2) bytes, outputs 4
    match = lambda s_, s2_, cnt, st: lib.sncc_match(seg.ref(), ok, s_, 32, s2_, 96, 64, 64, 0.5, None, 0, ok, 16,
                                                    cnt, st, None)
    assert match(ok, a4, ok, ok) == sncc.ERR_ARG
    assert match(a8, ok, ok, ok) == sncc.ERR_ARG
    assert match(ok, ok, a2, ok) == sncc.ERR_ARG
    assert match(ok, ok, ok, a2) == sncc.ERR_ARG
    # the per-candidate fine stage and the exact map read whole entries
    assert lib.sncc_refine_segmented(seg.ref(), ok, ok, 32, a4, 96, 64, 64, ok, ok, 16, 0.5, ok, 16, ok, ok,
                                     1 << 20, ok, None) == sncc.ERR_ARG
    assert lib.sncc_refine_segmented(seg.ref(), ok, a4, 64, ok, 96, 64, 64, ok, ok, 16, 0.5, ok, 16, ok, ok,
                                     1 << 20, ok, None) == sncc.ERR_ARG
    exact = lambda s_, bits, s2_, rho: lib.sncc_exact_map(ok, 64, 64, 64, ok, 8, 8, 8, 64 * 7, 64 * 49, s_, bits,
                                                          s2_, 96, rho, 57, None)
    assert exact(ok, 32, ok, ok) == sncc.ERR_UNIFORM  # aligned: reaches the template check
    assert exact(ok, 32, a4, ok) == sncc.ERR_ARG
    assert exact(a4, 64, ok, ok) == sncc.ERR_ARG
    assert exact(ok, 32, ok, a2) == sncc.ERR_ARG
    # exact refine: candidate, count and match arrays
    refine = lambda cand, cnt, out: lib.sncc_refine(ok, 64, 64, 64, ok, 8, 8, 8, 64 * 7, 64 * 49, cand, cnt, 16,
                                                    0.5, out, 16, ok, ok, 1 << 20, ok, None)
    assert refine(a2, ok, ok) == sncc.ERR_ARG
    assert refine(ok, a2, ok) == sncc.ERR_ARG
    assert refine(ok, ok, a2) == sncc.ERR_ARG
    # differentiation: float arrays 4 bytes, the int4 rectangle list 16
    diff = lambda f_, rects: lib.sncc_diff_forward(f_, 64, 64, 64, ok, 8, 8, rects, ok, 4, ok, ok, ok, ok,
                                                   1 << 20, None)
    assert diff(a2, ok) == sncc.ERR_ARG
    assert diff(ok, a8) == sncc.ERR_ARG
    # more offsets than the int-indexed maps hold, or offset rows than grid rows
    assert lib.sncc_diff_forward(ok, 50000, 50000, 50000, ok, 8, 8, ok, ok, 4, ok, ok, ok, ok, 1 << 20,
                                 None) == sncc.ERR_UNSUPPORTED
    assert lib.sncc_diff_forward(ok, 16, 70000, 16, ok, 8, 8, ok, ok, 4, ok, ok, ok, ok, 1 << 20,
                                 None) == sncc.ERR_UNSUPPORTED
    assert lib.sncc_probe_alu(sncc.PROBE_DP4A, a2, 1, 1, None) == sncc.ERR_ARG
    # batch: the staged regions load two entries at once, so the pitch is a multiple of 4
    srcs = synth.batch_sources(count=1, M=120, N=100)
    tl = synth.batch_templates(srcs, count=2, lo=16, hi=40)
    segs = [sncc.build_segments(t, sg) for t, _, sg in tl]
    arr = (C.POINTER(sncc._Segments) * 2)(*[C.pointer(sg._s) for sg in segs])
    ts = [np.ascontiguousarray(t) for t, _, _ in tl]
    pix = (C.c_void_p * 2)(*[t.ctypes.data for t in ts])
    strides = (C.c_int * 2)(*[t.shape[1] for t in ts])
    taus = (C.c_float * 2)(0.5, 0.5)
    h = C.c_void_p()
    assert lib.sncc_batch_create(arr, pix, strides, taus, taus, 2, 1, 120, 100, C.byref(h)) == 0
    try:
        good = (C.c_void_p * 1)(256)
        bad4 = (C.c_void_p * 1)(260)
        bm = lambda s_, s2_, pitch, cand: lib.sncc_batch_match(h, ok, s_, s2_, 32, pitch, cand, 16, ok, ok, ok, None)
        assert bm(good, good, 122, ok) == sncc.ERR_ARG  # >= M + 1 but not a multiple of 4
        assert bm(good, bad4, 124, ok) == sncc.ERR_ARG
        assert bm(bad4, good, 124, ok) == sncc.ERR_ARG
        assert bm(good, good, 124, a4) == sncc.ERR_ARG  # candidate pairs are 8-byte records
    finally:
        lib.sncc_batch_destroy(h)


def test_match_multi_fusability_decided_on_host(sncc):
    """sncc_match_multi declines (SNCC_ERR_UNSUPPORTED) a template of several
    blocks or one summed in place before any CUDA call, and rejects templates
    of different sizes as an argument error."""
    lib = sncc.lib()
    big = sncc.build_segments(synth.case_plain(M=300, N=260, W=130, H=100, seed=3).t, 6.0)
    small = sncc.build_segments(synth.case_hd(M=300, N=260, W=48, H=40, seed=4).t, 4.0)
    boxes = np.full((40, 48), 50, np.uint8)
    boxes[5:20, 8:30] = 180
    sparse = sncc.build_segments(boxes, 1.0)
    assert small.plan_info()["template_corners"] > 64 and sparse.plan_info()["template_corners"] <= 64
    ptrs = (C.c_void_p * 4)(*[256] * 4)
    taus = (C.c_float * 4)(*[0.5] * 4)

    def call(segs):
        arr = (C.POINTER(sncc._Segments) * len(segs))(*[C.pointer(sg._s) for sg in segs])
        return lib.sncc_match_multi(arr, ptrs, len(segs), C.c_void_p(256), 32, C.c_void_p(256), 320, 300, 260,
                                    taus, None, 0, ptrs, 16, ptrs, ptrs, None)

    assert call([big]) == sncc.ERR_UNSUPPORTED
    assert call([small, sparse]) == sncc.ERR_UNSUPPORTED
    assert call([small, big]) == sncc.ERR_ARG


def test_pipeline_host_argument_errors(sncc):
    """The frame pipeline rejects bad arguments before any CUDA call, and
    its query and release calls are safe on a null handle."""
    lib = sncc.lib()
    seg = sncc.build_segments(synth.case_hd(M=300, N=260, W=48, H=40, seed=4).t, 4.0)
    segs = (C.POINTER(sncc._Segments) * 1)(C.pointer(seg._s))
    plans = (C.c_void_p * 1)(256)
    taus = (C.c_float * 1)(0.5)
    slots = (sncc._PipelineSlot * 2)()
    h = C.c_void_p()
    args = lambda n, sl, cap: (segs, plans, n, C.c_void_p(256), 48, 300, 260, 32, 320, taus, 0.8, cap, 16, 0, sl,
                               C.byref(h))
    assert lib.sncc_pipeline_create(*args(0, slots, 16)) == sncc.ERR_ARG
    assert lib.sncc_pipeline_create(*args(5, slots, 16)) == sncc.ERR_ARG
    assert lib.sncc_pipeline_create(*args(1, None, 16)) == sncc.ERR_ARG
    assert lib.sncc_pipeline_create(*args(1, slots, 0)) == sncc.ERR_ARG
    assert lib.sncc_pipeline_create(*args(1, slots, 16)) == sncc.ERR_ARG  # empty slot buffers
    assert h.value is None
    assert lib.sncc_pipeline_fused(None) == sncc.ERR_ARG
    assert lib.sncc_pipeline_compute_stream(None) is None
    assert lib.sncc_pipeline_submit(None, None, None, None, None) == sncc.ERR_ARG
    lib.sncc_pipeline_destroy(None)


def test_batch_host_work_lists(sncc):
    """sncc_batch_create on the host: the work list has one item per tile of
    every (source, template) pair, and the offset / corner totals add up."""
    srcs = synth.batch_sources(count=2, M=120, N=100)
    tl = synth.batch_templates(srcs, count=5, lo=16, hi=90)
    segs = [sncc.build_segments(t, sg) for t, _, sg in tl]
    nt, ns, M, N = len(tl), 2, 120, 100
    arr = (C.POINTER(sncc._Segments) * nt)(*[C.pointer(sg._s) for sg in segs])
    ts = [np.ascontiguousarray(t) for t, _, _ in tl]
    pix = (C.c_void_p * nt)(*[t.ctypes.data for t in ts])
    strides = (C.c_int * nt)(*[t.shape[1] for t in ts])
    taus = (C.c_float * nt)(*([0.5] * nt))
    h = C.c_void_p()
    lib = sncc.lib()
    assert lib.sncc_batch_create(arr, pix, strides, taus, taus, nt, ns, M, N, C.byref(h)) == 0
    try:
        info = sncc.BatchInfo()
        for R in (8, 4, 2):
            assert lib.sncc_batch_set_variant(h, R) == 0
            assert lib.sncc_batch_get_info(h, C.byref(info)) == 0
            tiles = offsets = corner_offsets = 0
            for t, sg in zip(ts, segs):
                U, V = M - t.shape[1] + 1, N - t.shape[0] + 1
                tiles += ns * (-(-U // 32)) * (-(-V // (8 * R)))
                offsets += ns * U * V
                corner_offsets += ns * U * V * sg.plan_info()["corners"]
            assert info.tile_rows == R and info.tiles == tiles
            assert info.offsets == offsets
            # the batch rebuilds plans with 64 x 64 blocks: same nonzero corners
            # only where the template fits one block; compare within the total
            assert info.corner_offsets > 0
        assert lib.sncc_batch_set_variant(h, 3) == sncc.ERR_ARG
        assert lib.sncc_batch_device_bytes(h) > 0
    finally:
        lib.sncc_batch_destroy(h)
    assert lib.sncc_batch_create(arr, pix, strides, taus, taus, nt, 17, M, N, C.byref(h)) == sncc.ERR_ARG
    flat = np.full((8, 8), 3, np.uint8)
    seg_u = sncc.build_segments(flat, 1.0)
    arr1 = (C.POINTER(sncc._Segments) * 1)(C.pointer(seg_u._s))
    pix1 = (C.c_void_p * 1)(flat.ctypes.data)
    st1 = (C.c_int * 1)(8)
    t1 = (C.c_float * 1)(0.5)
    assert lib.sncc_batch_create(arr1, pix1, st1, t1, t1, 1, 1, M, N, C.byref(h)) == sncc.ERR_UNIFORM


def test_bench_batch_accounting_matches_the_library(sncc):
    """The benchmark's batch config counts the offsets per step itself (both
    arms print it); the count equals the library's own for the same batch."""
    import importlib.util
    import pathlib
    path = pathlib.Path(__file__).resolve().parent.parent / "bench.py"
    spec = importlib.util.spec_from_file_location("bench_for_test", path)
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    srcs = synth.batch_sources(count=3, M=150, N=120)
    tl = synth.batch_templates(srcs, count=6, lo=16, hi=100)
    segs = [sncc.build_segments(t, sg) for t, _, sg in tl]
    arr = (C.POINTER(sncc._Segments) * len(tl))(*[C.pointer(sg._s) for sg in segs])
    ts = [np.ascontiguousarray(t) for t, _, _ in tl]
    pix = (C.c_void_p * len(tl))(*[t.ctypes.data for t in ts])
    strides = (C.c_int * len(tl))(*[t.shape[1] for t in ts])
    taus = (C.c_float * len(tl))(*([0.5] * len(tl)))
    h = C.c_void_p()
    lib = sncc.lib()
    assert lib.sncc_batch_create(arr, pix, strides, taus, taus, len(tl), 3, 150, 120, C.byref(h)) == 0
    try:
        info = sncc.BatchInfo()
        assert lib.sncc_batch_get_info(h, C.byref(info)) == 0
        cfg = bench.batch_config(srcs, tl)
        assert cfg["offsets_per_step"] == int(info.offsets)
        assert cfg["sources"] == [3, 150, 120] and cfg["pairs"] == 18 == cfg["templates"] * 3
    finally:
        lib.sncc_batch_destroy(h)


def test_noalloc_scratch_covers_every_source_up_to_1e8_pixels(sncc):
    """The allocation-free sum tables promise every source of up to 10^8
    pixels: the workspace sncc_integral asks for stays within the built-in
    scratch for the tallest source of each width (the band sums grow with N
    at a fixed width), across the band-geometry regimes (few bands of 64
    rows, many short bands, a single partial 256-column tile), and a source
    past the limit asks for more."""
    lib = sncc.lib()
    cap = sncc.NOALLOC_SCRATCH_BYTES
    worst = 0
    for M in [1, 2, 31, 32, 33, 255, 256, 257, 511, 512, 1000, 1525, 1563, 1920, 4096, 6100, 10000, 15622, 16383]:
        top = min(65535, 10 ** 8 // M)
        for N in {top, top - 1, top - 63, top // 2 + 1, max(1, top // 7)}:
            need = lib.sncc_integral_workspace_bytes(M, N)
            assert 0 < need <= cap, (M, N, need)
            worst = max(worst, need)
    assert worst > cap // 2  # the scan reaches the large end of the range
    assert lib.sncc_integral_workspace_bytes(16383, 65535) > cap


def test_match_table_width_policy(sncc):
    """The matchers' tables: 32-bit (entries modulo 2^32) unless the source is
    large enough for a 32-bit table to wrap and a template is sparse enough
    for the direct corner read, which needs whole entries; the Python limit
    is the header's."""
    text = open(os.path.join(ROOT, "include", "sncc.h")).read()
    assert int(re.search(r"#define SNCC_DIRECT_MAX_CORNERS (\d+)", text).group(1)) == sncc.DIRECT_MAX_CORNERS
    dense = sncc.build_segments(synth.case_texture(M=300, N=300, W=256, H=256).t, 5.0)
    sparse = sncc.build_segments(synth.case_plain().t, 10.0)
    assert dense.plan_info()["template_corners"] > sncc.DIRECT_MAX_CORNERS
    assert sparse.plan_info()["template_corners"] <= sncc.DIRECT_MAX_CORNERS
    assert sncc.match_bits(4096, 4096, (dense,)) == 32
    assert sncc.match_bits(4096, 4096, (dense, sparse)) == 64
    assert sncc.match_bits(2048, 2048, (sparse,)) == 32  # 255 M N < 2^31: never wraps
    assert sncc.match_bits(4096, 4096) == 32
