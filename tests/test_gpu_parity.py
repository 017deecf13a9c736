"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Bars: sum tables and segment tables bit-exact; NCC maps within 1e-5 absolute;
candidate and match sets exact outside a +-1e-5 band around each threshold
(inside the band the FP32 decision may legitimately go either way, and such
offsets are counted); match values within 1e-5."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from conftest import record_band_count
from paper_2502_01286_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5


@pytest.fixture(scope="module")
def sncc():
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA GPU")
    from paper_2502_01286_gb300 import build
    build.build()
    from paper_2502_01286_gb300 import sncc as mod
    return mod


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def run_match(sncc, f, t, sigma, tau, cand_cap=1 << 20, k_max=0, s_bits=None):
    N, M = f.shape
    seg = sncc.build_segments(t, sigma, k_max)
    fd = dev(f)
    tb = sncc.integral(fd, s_bits=s_bits)
    plan = sncc.upload_plan(seg)
    mb = sncc.alloc_match(M, N, seg.W, seg.H, cand_cap)
    sncc.match(seg, plan, tb, tau, mb)
    torch.cuda.synchronize()
    return seg, fd, tb, mb


def check_candidates(rho64, cand, count, tau, rows=None, what=""):
    """Every offset with rho64 >= tau + TOL is a candidate and every one with
    rho64 < tau - TOL is not; the number of offsets inside the band (where
    either decision is right) is recorded for the session summary and
    returned."""
    V, U = rho64.shape
    cand = np.asarray(cand, np.int64)
    assert len(np.unique(cand)) == len(cand) == count
    got = np.zeros(U * V, bool)
    got[cand] = True
    got = got.reshape(V, U)
    sel = slice(None) if rows is None else rows
    r = rho64[sel]
    g = got[sel]
    assert np.all(g[r >= tau + TOL])
    assert not np.any(g[r < tau - TOL])
    band = int(np.sum((r >= tau - TOL) & (r < tau + TOL)))
    record_band_count(what or "candidates at tau %.6f" % tau, band, r.size)
    return band


# ------------------------------------------------------------------ sum tables
@pytest.mark.parametrize("M,N", [(1, 1), (5, 3), (33, 17), (257, 129), (256, 256), (1920, 1080), (4095, 7),
                                 (300, 20000)])
@pytest.mark.parametrize("bits", [32, 64])
def test_integral_bit_exact(sncc, M, N, bits):
    """Every entry against the oracle's tables.  The 300 x 20000 source is
    bright (values 200 to 255): a lane's eight carries of f^2 then sum past
    2^32 in the lower bands."""
    f = synth.random_image(1000 + M + N, M, N, lo=200 if N > 8192 else 0)
    tb = sncc.integral(dev(f), s_bits=bits)
    torch.cuda.synchronize()
    s, s2 = O.sum_tables(f)
    got_s = tb.s[:, :M + 1].cpu().numpy().astype(np.int64)
    got_s2 = tb.s2[:, :M + 1].cpu().numpy()
    np.testing.assert_array_equal(got_s, s.astype(np.int64))
    np.testing.assert_array_equal(got_s2, s2.astype(np.int64))


def test_integral_strided_source(sncc):
    """A source that is a column window of a wider image (row stride > M)."""
    big = synth.random_image(5, 300, 90)
    fd = dev(big)[:, 17:17 + 211]
    tb = sncc.integral(fd, s_bits=32)
    torch.cuda.synchronize()
    s, s2 = O.sum_tables(big[:, 17:17 + 211])
    np.testing.assert_array_equal(tb.s[:, :212].cpu().numpy().astype(np.int64), s.astype(np.int64))
    np.testing.assert_array_equal(tb.s2[:, :212].cpu().numpy(), s2.astype(np.int64))


def test_integral_int64_full_size(sncc):
    """4096 x 4096 at full intensity: entries reach 255*4096^2 > 2^31."""
    f = synth.random_image(9, 4096, 4096, lo=200)
    tb = sncc.integral(dev(f))
    assert tb.s_bits == 64
    torch.cuda.synchronize()
    s, s2 = O.sum_tables(f)
    for rows in (slice(0, 3), slice(2000, 2003), slice(4094, 4097)):
        np.testing.assert_array_equal(tb.s[rows, :4097].cpu().numpy(), s[rows].astype(np.int64))
        np.testing.assert_array_equal(tb.s2[rows, :4097].cpu().numpy(), s2[rows].astype(np.int64))
    assert int(tb.s[-1, 4096]) == int(s[-1, -1])


@pytest.mark.parametrize("bits", [32, 64])
def test_table_pitch_any_multiple_of_4(sncc, bits):
    """Tables whose pitch is a multiple of 4 but not of 32 (304 for a
    300-column source): the sums, the segment-sum maps of a one-block
    template (TMA staging on a 32-bit table) and of a multi-block template
    (register staging), the exact map, and the batch's candidates and matches
    equal those of the default pitch bit for bit."""
    M, N, P = 300, 260, 304
    assert P % 4 == 0 and P % 32 != 0 and P >= M + 1 and sncc.sat_pitch(M) != P
    one = synth.case_hd(M=M, N=N, W=48, H=40, seed=4)
    multi = synth.case_plain(M=M, N=N, W=130, H=100, seed=3)
    fd = dev(one.f)
    ref = sncc.integral(fd, s_bits=bits)
    dt = torch.int32 if bits == 32 else torch.int64
    tb = sncc.Tables(torch.zeros((N + 1, P), dtype=dt, device="cuda"),
                     torch.zeros((N + 1, P), dtype=torch.int64, device="cuda"), bits, P, M, N)
    sncc.integral(fd, tb)
    torch.cuda.synchronize()
    assert torch.equal(tb.s[:, :M + 1], ref.s[:, :M + 1]) and torch.equal(tb.s2[:, :M + 1], ref.s2[:, :M + 1])
    for t, sigma in ((one.t, 4.0), (multi.t, 6.0)):
        seg = sncc.build_segments(t, sigma)
        plan = sncc.upload_plan(seg)
        out = []
        for tables in (ref, tb):
            mb = sncc.alloc_match(M, N, seg.W, seg.H, 1 << 16)
            sncc.match(seg, plan, tables, 0.0, mb)
            rho = sncc.exact_map(fd, dev(t), seg.T, seg.T2, tables)
            torch.cuda.synchronize()
            n = int(mb.count.item())
            assert int(mb.status.item()) == 0 and n > 0
            out.append((mb.rho.clone(), sorted(mb.cand[:n].tolist()), rho.clone()))
        assert torch.equal(out[0][0], out[1][0]) and out[0][1] == out[1][1] and torch.equal(out[0][2], out[1][2])
    # the batch's staged regions at the same pitch
    tl = [(one.t, 4.0), (multi.t, 6.0)]
    res = []
    for pitch in (None, P):
        b = sncc.Batch([t for t, _ in tl], [sg for _, sg in tl], M, N, 1, precision=0.7)
        if pitch is not None:
            b.tables = [sncc.Tables(torch.zeros((N + 1, P), dtype=b.tables[0].s.dtype, device="cuda"),
                                    torch.zeros((N + 1, P), dtype=torch.int64, device="cuda"), b.s_bits, P, M, N)]
            b._s = (C.c_void_p * 1)(b.tables[0].s.data_ptr())
            b._s2 = (C.c_void_p * 1)(b.tables[0].s2.data_ptr())
            b.pitch = P
        b.run([fd])
        torch.cuda.synchronize()
        assert int(b.status.item()) == 0
        pair, idx = b.candidates()
        res.append((sorted(zip(pair.tolist(), idx.tolist())), [a.tolist() for a in b.matches()]))
    assert res[0][1][0] and res[0] == res[1]


def wrap32(a):
    """Exact sums as the int32 entries of a 32-bit table: modulo 2^32, two's
    complement."""
    return (np.asarray(a).astype(np.int64) & 0xFFFFFFFF).astype(np.uint32).view(np.int32)


def _random_sat_shapes(n=24, seed=2026120301):
    """Seeded random sources for the sum tables: general, tall and narrow,
    wide and short, and medium shapes (every band height, tile count and
    ragged edge the launch geometry picks), each a column window of a wider
    image at a random (often odd) offset."""
    g = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = i % 4
        if kind == 0:
            M, N = int(g.integers(1, 5000)), int(g.integers(1, 3000))
        elif kind == 1:
            M, N = int(g.integers(1, 300)), int(g.integers(3000, 24000))
        elif kind == 2:
            M, N = int(g.integers(3000, 16384)), int(g.integers(1, 200))
        else:
            M, N = int(g.integers(200, 2500)), int(g.integers(200, 2500))
        pad = int(g.integers(0, 40))
        out.append((i, M, N, pad, int(g.integers(0, pad + 1)), (32, 64)[i % 2], int(g.integers(0, 1 << 30))))
    return out


@pytest.mark.parametrize("i,M,N,pad,x0,bits,seed", _random_sat_shapes())
def test_integral_random_shapes(sncc, i, M, N, pad, x0, bits, seed):
    """Both tables of a random source against the oracle's, bit for bit (the
    32-bit s modulo 2^32)."""
    big = synth.random_image_u8(seed, M + pad, N)
    tb = sncc.integral(dev(big)[:, x0:x0 + M], s_bits=bits)
    torch.cuda.synchronize()
    s, s2 = O.sum_tables(np.ascontiguousarray(big[:, x0:x0 + M]))
    want = s.astype(np.int64) if bits == 64 else wrap32(s).astype(np.int64)
    np.testing.assert_array_equal(tb.s[:, :M + 1].cpu().numpy().astype(np.int64), want)
    np.testing.assert_array_equal(tb.s2[:, :M + 1].cpu().numpy(), s2.astype(np.int64))


def test_integral_int32_wraps_modulo_2_32(sncc):
    """A 32-bit s on a source whose sums pass 2^32 (8192 x 3000, values 200
    to 255): sampled rows hold the exact sums modulo 2^32, and window sums
    formed from them in wrapped 32-bit arithmetic equal the exact ones."""
    M, N = 8192, 3000
    f = synth.random_image(19, M, N, lo=200)
    tb = sncc.integral(dev(f), s_bits=32)
    torch.cuda.synchronize()
    s, s2 = O.sum_tables(f)
    assert s[-1, -1] > 2 ** 32  # the entries wrap at least once
    for rows in (slice(0, 3), slice(1500, 1503), slice(N - 2, N + 1)):
        np.testing.assert_array_equal(tb.s[rows, :M + 1].cpu().numpy(), wrap32(s[rows]))
        np.testing.assert_array_equal(tb.s2[rows, :M + 1].cpu().numpy(), s2[rows].astype(np.int64))
    t32 = tb.s[:, :M + 1].cpu().numpy()
    g = np.random.default_rng(4)
    for _ in range(200):
        W, H = int(g.integers(1, 2897)), int(g.integers(1, 2897))  # 255 W H < 2^31
        u, v = int(g.integers(0, M - W + 1)), int(g.integers(0, N - H + 1))
        d = (int(t32[v + H, u + W]) - int(t32[v + H, u]) - int(t32[v, u + W]) + int(t32[v, u])) & 0xFFFFFFFF
        got = d - (1 << 32) if d >= 1 << 31 else d
        want = int(s[v + H, u + W] - s[v + H, u] - s[v, u + W] + s[v, u])  # exact in float64 (< 2^53)
        assert got == want, (u, v, W, H)


@pytest.fixture(scope="module")
def max_source():
    """The largest source sncc_integral takes, 16383 x 33025 (M <= 16383, and
    N 65025 < 2^31 for the int32 column sums of f^2), bright (values 200 to
    255), and its exact table rows Y = 0, 1, 2, 16512, N - 1, N by the
    definition: the column sums of the rows above Y, prefix-summed along the
    row (in chunks of rows, so no full-size int64 copy is made)."""
    M, N = 16383, 33025
    f = synth.random_image_u8(41, M, N, lo=200)
    rows = [0, 1, 2, 16512, N - 1, N]
    want, want2 = {}, {}
    acc = np.zeros(M, np.int64)
    acc2 = np.zeros(M, np.int64)
    prev = 0
    for Y in rows:
        for y in range(prev, Y, 1024):
            blk = f[y:min(Y, y + 1024)].astype(np.int64)
            acc += blk.sum(0)
            acc2 += (blk * blk).sum(0)
        prev = Y
        want[Y] = np.concatenate([[0], np.cumsum(acc)])
        want2[Y] = np.concatenate([[0], np.cumsum(acc2)])
    return f, rows, want, want2


@pytest.mark.parametrize("bits", [32, 64])
def test_integral_maximum_source(sncc, max_source, bits):
    """Sampled rows of the tables of the largest source: s2 exact, s exact
    (64-bit) or modulo 2^32 (32-bit, wrapping about ten times)."""
    f, rows, want, want2 = max_source
    N, M = f.shape
    tb = sncc.integral(dev(f), s_bits=bits)
    torch.cuda.synchronize()
    assert want[N][-1] > 8 * 2 ** 32
    for Y in rows:
        got = tb.s[Y, :M + 1].cpu().numpy()
        np.testing.assert_array_equal(got, want[Y] if bits == 64 else wrap32(want[Y]))
        np.testing.assert_array_equal(tb.s2[Y, :M + 1].cpu().numpy(), want2[Y])
    del tb
    torch.cuda.empty_cache()


def test_match_maximum_template_area(sncc):
    """The largest template area (W H = 2^23: 2048 x 4096), where a window sum
    of f can reach 255 W H, just under 2^31, on a 2100 x 4600 source of
    values 200 to 255 whose 32-bit table wraps (sum of f past 2^31).  The
    approximation (sigma 1: 4637 segments, 2048 blocks of 64 x 64) equals the
    oracle's; the rho maps on 32- and 64-bit tables are identical and within
    1e-5 of the oracle on sampled rows; the crop offset gives rho_max."""
    c = synth.case_plain(M=2100, N=4600, W=2048, H=4096, noise=0.0)
    f = (200 + (c.f.astype(np.int64) - 39) * 55 // 189).clip(0, 255).astype(np.uint8)
    u0, v0 = c.origin
    t = np.ascontiguousarray(f[v0:v0 + 4096, u0:u0 + 2048])
    N, M = f.shape
    U, V = M - 2048 + 1, N - 4096 + 1
    assert int(f.astype(np.int64).sum()) >= 2 ** 31
    ap = O.precompute_template_approximation(t, 1.0)
    seg = sncc.build_segments(t, 1.0)
    assert seg.K == ap.K
    plan = sncc.upload_plan(seg)
    fd = dev(f)
    maps = {}
    for bits in (32, 64):
        tb = sncc.integral(fd, s_bits=bits)
        mb = sncc.alloc_match(M, N, 2048, 4096, U * V)
        sncc.match(seg, plan, tb, 0.9 * seg.rho_max, mb)
        torch.cuda.synchronize()
        assert int(mb.status.item()) == 0
        maps[bits] = mb.rho.clone()
    assert torch.equal(maps[32], maps[64])
    rows = np.unique(np.r_[0, 1, v0, V - 1, np.random.default_rng(7).choice(V, 12, replace=False)])
    ref = O.segmented_ncc_map(f, ap, "sat", rows=rows)
    got = maps[32].cpu().numpy()
    assert np.abs(got[rows] - ref[rows]).max() <= TOL
    assert abs(got[v0, u0] - ap.rho_max) <= TOL


def test_wrapped_tables_equal_int64_texture(sncc):
    """The texture workload (4096 x 4096 source, the 256 x 256 template at
    sigma 5, precision 0.5) on the 32-bit tables the
    matchers use and on 64-bit tables: the staged region words, window sums
    and integer numerators are the same, so the rho maps, candidate sets,
    refined matches and the exact comparator's map are identical."""
    c = synth.case_texture()
    N, M = c.f.shape
    H, W = c.t.shape
    U, V = M - W + 1, N - H + 1
    seg = sncc.build_segments(c.t, 5.0)
    plan = sncc.upload_plan(seg)
    fd, td = dev(c.f), dev(c.t)
    out = {}
    for bits in (32, 64):
        tb = sncc.integral(fd, s_bits=bits)
        mb = sncc.alloc_match(M, N, W, H, U * V // 8)
        sncc.match(seg, plan, tb, 0.5 * seg.rho_max, mb)
        rb = sncc.alloc_refine(M, N, W, H, 1 << 20)
        sncc.refine(fd, td, seg, mb, 0.5, rb)
        ex = sncc.exact_map(fd, td, seg.T, seg.T2, tb)
        torch.cuda.synchronize()
        assert int(mb.status.item()) == 0
        cnt = int(mb.count.item())
        out[bits] = (mb.rho.clone(), np.sort(mb.cand[:cnt].cpu().numpy()), sncc.matches_to_numpy(rb), ex.clone())
    assert 255 * M * N >= 2 ** 31  # a size whose 32-bit table may wrap (the sparse-template test wraps one)
    a, b = out[32], out[64]
    assert torch.equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert a[1].size > 1000
    for x, y in zip(a[2], b[2]):
        np.testing.assert_array_equal(x, y)
    assert torch.equal(a[3], b[3])


def test_wrapped_tables_sparse_template(sncc):
    """A template of at most 64 corners reads its corners' table entries
    directly; on a wrapping 32-bit table it takes the staged path instead.
    Its rho map equals the direct read of 64-bit tables exactly (the same
    integer numerator either way), on a bright 4096 x 3000 source (values 150
    to 255, sums past 2^31) holding the template, three boxes on a flat
    background, at one offset.  The exact comparator's map and the paper's
    tile-by-tile fine stage are identical on both tables as well."""
    f = synth.random_image(23, 4096, 3000, lo=150)
    t = np.full((48, 48), 160, np.uint8)
    t[5:20, 8:30] = 230
    t[25:45, 3:15] = 185
    t[30:40, 28:44] = 205
    u0, v0 = 1234, 2001
    f[v0:v0 + 48, u0:u0 + 48] = t
    seg = sncc.build_segments(t, 10.0)
    assert seg.plan_info()["template_corners"] <= 64
    fine = sncc.build_segments(t, 2.0)
    N, M = f.shape
    plan, plan_fine = sncc.upload_plan(seg), sncc.upload_plan(fine)
    fd, td = dev(f), dev(t)
    maps, exact, lists = {}, {}, {}
    for bits in (32, 64):
        tb = sncc.integral(fd, s_bits=bits)
        mb = sncc.alloc_match(M, N, 48, 48, 1 << 16)
        sncc.match(seg, plan, tb, 0.9 * seg.rho_max, mb)
        exact[bits] = sncc.exact_map(fd, td, seg.T, seg.T2, tb)  # window sums from the table
        # the paper's fine stage on the tiles that hold the coarse candidates, from the same table
        rb = sncc.alloc_refine(M, N, 48, 48, 1 << 16)
        ws = sncc.tiles_workspace(M, N, 48, 48, 1 << 16)
        sncc.refine_segmented_tiles(fine, plan_fine, tb, mb, 0.9 * fine.rho_max, rb, ws)
        torch.cuda.synchronize()
        assert int(mb.status.item()) == 0
        maps[bits] = mb.rho.clone()
        lists[bits] = sncc.matches_to_numpy(rb)
    assert int(f.astype(np.int64).sum()) >= 2 ** 31
    assert torch.equal(maps[32], maps[64])
    assert abs(float(maps[32][v0, u0]) - seg.rho_max) <= TOL
    assert torch.equal(exact[32], exact[64])
    assert abs(float(exact[32][v0, u0]) - 1.0) <= TOL
    for x, y in zip(lists[32], lists[64]):
        np.testing.assert_array_equal(x, y)
    assert (v0 * (M - 47) + u0) in (lists[32][1].astype(np.int64) * (M - 47) + lists[32][0]).tolist()


# ------------------------------------------------------------------ coarse pass
SHAPES = [
    # (M, N, W, H, sigma)
    (256, 256, 32, 32, 3.0),    # 256^2 source, 32^2 template (std 5.5 with this seed: sigma 3)
    (70, 45, 13, 9, 3.0),       # ragged tail in both directions
    (100, 100, 64, 64, 5.0),    # largest single-block template
    (130, 90, 100, 70, 6.0),    # multi-block template (64 x 64 blocks, ragged)
    (40, 300, 40, 17, 4.0),     # U = 1
    (300, 40, 23, 40, 4.0),     # V = 1
    (120, 110, 37, 29, 0.0),    # sigma 0: every pixel its own segment before merging
    (97, 61, 2, 1, 0.5),        # two-pixel template
    (300, 60, 256, 3, 2.0),     # wide, three rows: 64 x 64 blocks along one axis
    (30, 900, 3, 700, 2.0),     # tall, three columns: 11 blocks down one column
]


@pytest.mark.parametrize("M,N,W,H,sigma", SHAPES)
def test_match_map_and_candidates(sncc, M, N, W, H, sigma):
    c = synth.case_plain(M=M, N=N, W=W, H=H, seed=4242 + M * 7 + W)
    seg = sncc.build_segments(c.t, sigma)
    if not seg.Ek > 0:
        pytest.skip("uniform approximation")
    ap = O.precompute_template_approximation(c.t, sigma)
    np.testing.assert_array_equal(seg.table, ap.segments)
    tau = 0.8 * seg.rho_max
    seg, fd, tb, mb = run_match(sncc, c.f, c.t, sigma, tau)
    ref = O.segmented_ncc_map(c.f, ap, "sat")
    got = mb.rho.cpu().numpy().astype(np.float64)
    assert got.shape == ref.shape
    err = np.abs(got - ref).max()
    assert err <= TOL, err
    assert int(mb.status.item()) == 0
    cnt = int(mb.count.item())
    check_candidates(ref, mb.cand[:cnt].cpu().numpy(), cnt, tau, what="%dx%d t%dx%d sigma %g" % (M, N, W, H, sigma))


def _random_cases(n=20, seed=20261203):
    """Seeded random problems: the three source generators, templates of 2 to
    159 pixels a side, sources up to 160 columns and 140 rows wider, std
    thresholds from 0 (every pixel its own segment) to 12, both table widths."""
    g = np.random.default_rng(seed)
    cases = []
    for i in range(n):
        W, H = int(g.integers(2, 160)), int(g.integers(2, 160))
        M, N = W + int(g.integers(0, 160)), H + int(g.integers(0, 140))
        sigma = float(g.choice([0.0, 1.0, 3.0, 6.0, 12.0]))
        p = float(g.choice([0.5, 0.7, 0.9]))
        cases.append((i, ("plain", "texture", "hd")[i % 3], M, N, W, H, sigma, (32, 64)[(i // 3) % 2], p,
                      int(g.integers(0, 1 << 30))))
    return cases


@pytest.mark.parametrize("i,kind,M,N,W,H,sigma,bits,p,seed", _random_cases())
def test_random_problems_whole_path(sncc, i, kind, M, N, W, H, sigma, bits, p, seed):
    """The whole path on a random problem against the oracle: the segment
    table bit for bit, the map within 1e-5, the candidate set by the band
    rule, and the exact refine's sorted matches (values within 1e-5, the set
    equal outside the two threshold bands)."""
    c = getattr(synth, "case_" + kind)(M=M, N=N, W=W, H=H, seed=seed)
    seg = sncc.build_segments(c.t, sigma)
    if not seg.Ek > 0:
        pytest.skip("uniform approximation")
    ap = O.precompute_template_approximation(c.t, sigma)
    np.testing.assert_array_equal(seg.table, ap.segments)
    tau_c = p * ap.rho_max
    U, V = M - W + 1, N - H + 1
    seg, fd, tb, mb = run_match(sncc, c.f, c.t, sigma, tau_c, cand_cap=U * V, s_bits=bits)
    ref = O.segmented_ncc_map(c.f, ap, "sat")
    assert np.abs(mb.rho.cpu().numpy() - ref).max() <= TOL
    assert int(mb.status.item()) == 0
    cnt = int(mb.count.item())
    check_candidates(ref, mb.cand[:cnt].cpu().numpy(), cnt, tau_c,
                     what="random %d: %s %dx%d t%dx%d sigma %g" % (i, kind, M, N, W, H, sigma))
    rb = sncc.alloc_refine(M, N, W, H, U * V)
    sncc.refine(fd, dev(c.t), seg, mb, p, rb)
    torch.cuda.synchronize()
    assert int(mb.status.item()) == 0
    u, v, rho = sncc.matches_to_numpy(rb)
    key = v.astype(np.int64) * U + u
    assert np.all(np.diff(key) > 0)
    assert np.abs(rho - O.ncc_exact_at(c.f, c.t, u, v)).max(initial=0) <= TOL
    idx_o, _ = O.refine(c.f, c.t, O.candidates(ref, tau_c), U, p)
    diff = np.setxor1d(key, idx_o)
    if diff.size:
        ex = O.ncc_exact_at(c.f, c.t, (diff % U).astype(np.int32), (diff // U).astype(np.int32))
        amb = (np.abs(ref.ravel()[diff] - tau_c) < TOL) | (np.abs(ex - p) < TOL)
        assert np.all(amb), diff[~amb][:10]


@pytest.mark.parametrize("M,N,W,H", [(200, 150, 48, 40), (300, 260, 130, 129), (420, 150, 97, 65)])
@pytest.mark.parametrize("bits", [32, 64])
def test_match_table_width_independent(sncc, bits, M, N, W, H):
    """The same source through 32- and 64-bit sum tables gives one map: one
    TMA-staged block, and templates of several 64 x 64 blocks staged through
    registers (ragged edge blocks; tiles inside the table and on its edge)."""
    c = synth.case_plain(M=M, N=N, W=W, H=H, seed=11 + W)
    ap = O.precompute_template_approximation(c.t, 7.0)
    seg, _, _, mb = run_match(sncc, c.f, c.t, 7.0, 0.5, s_bits=bits)
    if W > 64 or H > 64:
        pi = seg.plan_info()
        assert pi["blocks"] > 1 and pi["wide_blocks"] > 1 and pi["wide_blocks"] < pi["blocks"]
    ref = O.segmented_ncc_map(c.f, ap, "sat")
    assert np.abs(mb.rho.cpu().numpy() - ref).max() <= TOL


@pytest.mark.parametrize("bits", [32, 64])
def test_match_direct_sparse_multiblock_template(sncc, bits):
    """A 200 x 150 template approximated by a few segments (sigma near the
    template's own std, as the paper's k_fast) has few corners in all; the
    kernel reads the table at those corners directly instead of staging
    blocks.  Map against the oracle, with 32- and 64-bit tables."""
    c = synth.case_plain(M=420, N=330, W=200, H=150, seed=23)
    sigma = 0.99 * sncc.template_sigma(c.t)
    seg = sncc.build_segments(c.t, sigma)
    pi = seg.plan_info()
    assert pi["blocks"] > 1 and 0 < pi["template_corners"] <= 64
    ap = O.precompute_template_approximation(c.t, sigma)
    _, _, _, mb = run_match(sncc, c.f, c.t, sigma, 0.5 * seg.rho_max, s_bits=bits)
    ref = O.segmented_ncc_map(c.f, ap, "sat")
    assert np.abs(mb.rho.cpu().numpy() - ref).max() <= TOL
    cnt = int(mb.count.item())
    check_candidates(ref, mb.cand[:cnt].cpu().numpy(), cnt, 0.5 * seg.rho_max, what="direct %d-bit" % bits)


MULTI_CASES = [
    # (M, N, W, H, bits, sigmas)
    (256, 256, 32, 32, 32, (2.0, 4.0, 8.0)),
    (70, 45, 13, 9, 32, (0.5, 1.0, 2.0, 3.0)),        # ragged tails, four approximations
    (300, 200, 64, 48, 64, (3.0, 6.0)),               # 64-bit tables
    (1920, 1080, 64, 64, 32, (5.0, 10.0, 20.0)),      # the HD workload's three thresholds
    (130, 90, 40, 40, 32, (5.0,)),                    # a single approximation
]


@pytest.mark.parametrize("M,N,W,H,bits,sigmas", MULTI_CASES)
def test_match_multi_equals_separate_calls(sncc, M, N, W, H, bits, sigmas):
    """sncc_match_multi stages each tile once for all approximations; every
    output (map, candidate set, count) is bit-identical to its own
    sncc_match, and the maps agree with the oracle."""
    c = synth.case_hd(M=M, N=N, W=W, H=H, seed=77 + W + len(sigmas))
    segs = [sncc.build_segments(c.t, s) for s in sigmas]
    for sg in segs:
        assert sg.Ek > 0 and sg.plan_info()["template_corners"] > 64
    fd = dev(c.f)
    tb = sncc.integral(fd, s_bits=bits)
    plans = [sncc.upload_plan(sg) for sg in segs]
    taus = [0.6 * sg.rho_max for sg in segs]
    sep = [sncc.alloc_match(M, N, W, H, 1 << 20) for _ in segs]
    for sg, pl, tau, mb in zip(segs, plans, taus, sep):
        sncc.match(sg, pl, tb, tau, mb)
    fused = [sncc.alloc_match(M, N, W, H, 1 << 20) for _ in segs]
    sncc.match_multi(segs, plans, tb, taus, fused)
    torch.cuda.synchronize()
    assert all(int(b.status.item()) == 0 for b in fused)
    V, U = N - H + 1, M - W + 1
    rows = np.unique(np.r_[0, V - 1, np.random.default_rng(M).choice(V, min(V, 6), replace=False)])
    for q, (a, b) in enumerate(zip(sep, fused)):
        assert torch.equal(a.rho, b.rho), q
        n = int(a.count.item())
        assert int(b.count.item()) == n
        np.testing.assert_array_equal(np.sort(a.cand[:n].cpu().numpy()), np.sort(b.cand[:n].cpu().numpy()))
        ap = O.precompute_template_approximation(c.t, sigmas[q])
        ref = O.segmented_ncc_map(c.f, ap, "sat", rows=rows)
        assert np.abs(b.rho.cpu().numpy()[rows] - ref[rows]).max() <= TOL


def test_match_multi_overflow_per_approximation(sncc):
    """Each approximation's count stays exact and its own status word gets
    the overflow bit when its list is longer than cand_cap."""
    c = synth.case_hd(M=200, N=150, W=40, H=40, seed=31)
    segs = [sncc.build_segments(c.t, s) for s in (2.0, 6.0)]
    fd = dev(c.f)
    tb = sncc.integral(fd)
    plans = [sncc.upload_plan(sg) for sg in segs]
    bufs = [sncc.alloc_match(200, 150, 40, 40, 64) for _ in segs]
    sncc.match_multi(segs, plans, tb, [-1.0, 2.0], bufs)  # every offset / no offset
    torch.cuda.synchronize()
    assert int(bufs[0].count.item()) == 161 * 111
    assert int(bufs[0].status.item()) == sncc.STATUS_CAND_OVERFLOW
    assert int(bufs[1].count.item()) == 0 and int(bufs[1].status.item()) == 0


def test_multi_matcher_graph_and_separate_matchers(sncc):
    """MultiMatcher fuses three thresholds of one template; a captured run
    replayed on a new source equals the eager run, and each threshold's
    match list equals that of its own Matcher."""
    a = synth.case_hd(M=400, N=300, W=48, H=48, seed=41)
    b = synth.case_hd(M=400, N=300, W=48, H=48, seed=42)
    sig = (3.0, 6.0, 12.0)
    mm = sncc.MultiMatcher(b.t, sig, 400, 300, precision=0.6)
    fd = dev(a.f)
    g = mm.capture(fd)
    assert mm.fused is True
    fd.copy_(dev(b.f))
    g.replay()
    torch.cuda.synchronize()
    got = [[x.copy() for x in sncc.matches_to_numpy(rb)] for rb in mm.rbs]
    mm.run(fd)
    torch.cuda.synchronize()
    assert mm.status() == 0
    for q, s in enumerate(sig):
        want = sncc.matches_to_numpy(mm.rbs[q])
        assert len(want[0]) > 0
        for x, y in zip(got[q], want):
            np.testing.assert_array_equal(x, y)
        one = sncc.Matcher(b.t, s, 400, 300, precision=0.6)
        one.run(fd)
        torch.cuda.synchronize()
        assert torch.equal(one.mb.rho, mm.mbs[q].rho)
        for x, y in zip(sncc.matches_to_numpy(one.rb), want):
            np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("sigmas", [(3.0, 6.0, 12.0), (5.0,)])
def test_stream_matcher_equals_one_frame_at_a_time(sncc, sigmas):
    """Five different frames through the pipelined StreamMatcher (the
    library's native frame pipeline) give, frame by frame, the match lists
    of a MultiMatcher run on each frame alone, and the last frame's rho maps
    equal that run's."""
    frames = [synth.case_hd(M=400, N=300, W=48, H=48, seed=60 + i) for i in range(5)]
    t = frames[0].t
    sm = sncc.StreamMatcher(t, sigmas, 400, 300, precision=0.6, keep_rho=True)
    got = []
    for c in frames:
        r = sm.submit(torch.as_tensor(c.f).pin_memory())
        if r is not None:
            got.append(r)
    got.append(sm.flush())
    assert sm.status() == 0
    ref = sncc.MultiMatcher(t, sigmas, 400, 300, precision=0.6)
    assert sm.fused == (len(sigmas) > 1)
    nonempty = 0
    for c, lists in zip(frames, got):
        fd = dev(c.f)
        ref.run(fd)
        torch.cuda.synchronize()
        for q, rb in enumerate(ref.rbs):
            want = sncc.matches_to_numpy(rb)
            nonempty += len(want[0]) > 0
            for x, y in zip(lists[q], want):
                np.testing.assert_array_equal(x, y)
    assert nonempty > 0
    # the last frame's maps in its slot equal the one-frame run's
    last = sm._bufs[(len(frames) - 1) % 2][3]
    for q in range(len(sigmas)):
        assert torch.equal(last[q].rho, ref.mbs[q].rho)


def test_stream_matcher_reuses_one_pinned_frame(sncc):
    """A caller that refills one pinned host buffer for every frame, and
    overwrites it as soon as submit returns, gets each frame's own match
    lists: submit returns only once the frame's copy is done."""
    frames = [synth.case_hd(M=400, N=300, W=48, H=48, seed=80 + i) for i in range(4)]
    t = frames[0].t
    sm = sncc.StreamMatcher(t, (4.0,), 400, 300, precision=0.6)
    buf = torch.empty((300, 400), dtype=torch.uint8).pin_memory()
    got = []
    for c in frames:
        buf.copy_(torch.as_tensor(c.f))
        r = sm.submit(buf)
        buf.fill_(0)  # the next frame's data would land here now
        if r is not None:
            got.append(r)
    got.append(sm.flush())
    assert sm.status() == 0
    ref = sncc.Matcher(t, 4.0, 400, 300, precision=0.6)
    nonempty = 0
    for c, lists in zip(frames, got):
        ref.run(dev(c.f))
        torch.cuda.synchronize()
        want = sncc.matches_to_numpy(ref.rb)
        nonempty += len(want[0]) > 0
        for x, y in zip(lists[0], want):
            np.testing.assert_array_equal(x, y)
    assert nonempty > 0


def test_match_multi_rejects_what_it_cannot_fuse(sncc):
    """Templates of different sizes are an argument error; a multi-block
    template, or one summed in place (at most 64 corners), is not fused
    (SNCC_ERR_UNSUPPORTED) and needs sncc_match."""
    c = synth.case_plain(M=300, N=260, W=130, H=100, seed=3)
    fd = dev(c.f)
    tb = sncc.integral(fd)
    small = synth.case_hd(M=300, N=260, W=48, H=40, seed=4)
    boxes = np.full((40, 48), 50, np.uint8)   # three flat rectangles: a handful of corners
    boxes[5:20, 8:30] = 180
    boxes[25:35, 10:40] = 90
    sparse = sncc.build_segments(boxes, 1.0)
    assert 0 < sparse.plan_info()["template_corners"] <= 64
    cases = [
        ([sncc.build_segments(c.t, 6.0)], sncc.ERR_UNSUPPORTED),                      # 130 x 100
        ([sncc.build_segments(small.t, 4.0), sncc.build_segments(c.t, 4.0)], sncc.ERR_ARG),
        ([sncc.build_segments(small.t, 4.0), sparse], sncc.ERR_UNSUPPORTED),
    ]
    for segs, code in cases:
        plans = [sncc.upload_plan(sg) for sg in segs]
        bufs = [sncc.alloc_match(300, 260, segs[0].W, segs[0].H, 1024) for _ in segs]
        with pytest.raises(sncc.SnccError) as e:
            sncc.match_multi(segs, plans, tb, [0.5] * len(segs), bufs)
        assert e.value.code == code


def test_match_repeatable(sncc):
    c = synth.case_plain()
    _, _, _, a = run_match(sncc, c.f, c.t, 10.0, 0.5)
    _, _, _, b = run_match(sncc, c.f, c.t, 10.0, 0.5)
    assert torch.equal(a.rho, b.rho)
    ca = np.sort(a.cand[:int(a.count.item())].cpu().numpy())
    cb = np.sort(b.cand[:int(b.count.item())].cpu().numpy())
    np.testing.assert_array_equal(ca, cb)


def test_match_uniform_windows_are_zero(sncc):
    c = synth.case_plain(M=120, N=100, W=20, H=16)
    f = c.f.copy()
    f[30:70, 40:90] = 111
    _, _, _, mb = run_match(sncc, f, c.t, 6.0, 0.5)
    rho = mb.rho.cpu().numpy()
    assert np.all(rho[30:55, 40:71] == 0.0)


def test_match_candidate_overflow(sncc):
    c = synth.case_plain()
    _, _, _, full = run_match(sncc, c.f, c.t, 10.0, -1.0)
    n = int(full.count.item())
    assert n == (256 - 31) ** 2
    _, _, _, small = run_match(sncc, c.f, c.t, 10.0, -1.0, cand_cap=100)
    assert int(small.count.item()) == n
    assert int(small.status.item()) & sncc.STATUS_CAND_OVERFLOW
    stored = small.cand[:100].cpu().numpy()
    assert len(np.unique(stored)) == 100 and stored.min() >= 0 and stored.max() < n


def test_match_uniform_template_rejected(sncc):
    t = np.full((16, 16), 50, np.uint8)
    seg = sncc.build_segments(t, 3.0)
    tb = sncc.integral(dev(synth.random_image(1, 64, 64)))
    mb = sncc.alloc_match(64, 64, 16, 16, 10)
    plan = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(sncc.SnccError) as e:
        sncc.match(seg, plan, tb, 0.5, mb)
    assert e.value.code == sncc.ERR_UNIFORM


def test_match_kmax(sncc):
    c = synth.case_plain(M=150, N=150, W=40, H=40)
    seg = sncc.build_segments(c.t, 0.0, 200)
    ap = O.precompute_template_approximation(c.t, 0.0, 200)
    assert seg.K_split <= 200 and seg.sigma_used == ap.sigma_used
    _, _, _, mb = run_match(sncc, c.f, c.t, 0.0, 0.5, k_max=200)
    assert np.abs(mb.rho.cpu().numpy() - O.segmented_ncc_map(c.f, ap, "sat")).max() <= TOL


@pytest.mark.parametrize("sigma", [5.0, 10.0, 20.0])
def test_match_hd_full_size_sampled(sncc, sigma):
    """1920 x 1080 source, 64 x 64 template (the HD workload), full launch;
    the oracle checks a seeded sample of offset rows."""
    c = synth.case_hd(sigma_max=sigma)
    ap = O.precompute_template_approximation(c.t, sigma)
    tau = c.precision * ap.rho_max
    seg, fd, tb, mb = run_match(sncc, c.f, c.t, sigma, tau)
    V = c.f.shape[0] - 64 + 1
    rows = np.unique(np.r_[np.random.default_rng(int(sigma)).choice(V, 10, replace=False), 0, V - 1,
                            c.origin[1]])
    ref = O.segmented_ncc_map(c.f, ap, "sat", rows=rows)
    got = mb.rho.cpu().numpy()
    assert np.abs(got[rows] - ref[rows]).max() <= TOL
    cnt = int(mb.count.item())
    check_candidates(ref, mb.cand[:min(cnt, mb.cand.numel())].cpu().numpy(), cnt, tau, rows=rows,
                     what="hd sigma %g, %d rows" % (sigma, len(rows)))


def test_match_texture_full_size_sampled(sncc):
    """4096 x 4096 high-texture source with a 256 x 256 template at sigma 5
    (thousands of segments, 64-bit sum tables, the register-staged 64 x 64
    block instance of the segment-sum kernel), full launch in the bench's
    configuration, on sampled offset rows: the map, the candidate set (G13
    rule at tau_c = 0.85 rho_max) and the exact refine's matches (Eq. 1;
    main algorithm steps 7a-7j with the exact second stage) against the
    oracle.  A second run at precision 0.5 gives about 7.6e5 candidates in
    all, and thousands of candidates and matches on those rows."""
    c = synth.case_texture()
    N, M = c.f.shape
    H, W = c.t.shape
    U, V = M - W + 1, N - H + 1
    ap = O.precompute_template_approximation(c.t, 5.0)
    assert ap.K > 1000
    rows = np.unique(np.r_[0, 1, 1234, c.origin[1] - 1, c.origin[1], c.origin[1] + 1, V - 1,
                           np.random.default_rng(3).choice(V, 9, replace=False)])
    ref = O.segmented_ncc_map(c.f, ap, "sat", rows=rows)
    u0, v0 = c.origin
    td = dev(c.t)
    for p in (c.precision, 0.5):
        tau = p * ap.rho_max
        seg, fd, tb, mb = run_match(sncc, c.f, c.t, 5.0, tau, cand_cap=U * V)
        assert tb.s_bits == 64
        got = mb.rho.cpu().numpy()
        assert np.abs(got[rows] - ref[rows]).max() <= TOL
        assert abs(got[v0, u0] - ap.rho_max) <= TOL  # noise-free crop: rho = NCC(t, k)
        cnt = int(mb.count.item())
        assert int(mb.status.item()) == 0
        check_candidates(ref, mb.cand[:cnt].cpu().numpy(), cnt, tau, rows=rows,
                         what="texture p %g, %d rows" % (p, len(rows)))
        # exact refine of the full candidate list; its matches on the sampled
        # rows against the oracle's refine of the oracle's candidates there
        rb = sncc.alloc_refine(M, N, W, H, U * V // 4)
        sncc.refine(fd, td, seg, mb, p, rb)
        torch.cuda.synchronize()
        assert int(mb.status.item()) == 0
        u, v, rho = sncc.matches_to_numpy(rb)
        key = v.astype(np.int64) * U + u
        assert np.all(np.diff(key) > 0)
        sel = np.isin(v, rows)
        assert np.abs(rho[sel] - O.ncc_exact_at(c.f, c.t, u[sel], v[sel])).max(initial=0) <= TOL
        idx_o, rho_o = O.refine(c.f, c.t, O.candidates(ref, tau), U, p)
        diff = np.setxor1d(key[sel], idx_o)
        if diff.size:
            ex = O.ncc_exact_at(c.f, c.t, (diff % U).astype(np.int32), (diff // U).astype(np.int32))
            amb = (np.abs(ref.ravel()[diff] - tau) < TOL) | (np.abs(ex - p) < TOL)
            assert np.all(amb), diff[~amb][:10]
        assert v0 * U + u0 in set(key.tolist())
        if p < 0.6:
            assert sel.sum() > 500  # many candidates and matches on the sampled rows


# ------------------------------------------------------------------ fine pass
def oracle_matches(f, t, ap, tau_c, tau_e):
    rho_seg = O.segmented_ncc_map(f, ap, "sat")
    cand = O.candidates(rho_seg, tau_c)
    U = rho_seg.shape[1]
    idx, rho = O.refine(f, t, cand, U, tau_e)
    return rho_seg, idx, rho


@pytest.mark.parametrize("M,N,W,H,sigma,p", [(256, 256, 32, 32, 6.0, 0.9), (180, 140, 48, 30, 4.0, 0.7),
                                             (90, 70, 90, 20, 3.0, 0.5)])
def test_refine_matches_oracle(sncc, M, N, W, H, sigma, p):
    c = synth.case_plain(M=M, N=N, W=W, H=H, seed=99 + M)
    ap = O.precompute_template_approximation(c.t, sigma)
    tau_c, tau_e = p * ap.rho_max, p
    rho_seg, idx_o, rho_o = oracle_matches(c.f, c.t, ap, tau_c, tau_e)
    seg, fd, tb, mb = run_match(sncc, c.f, c.t, sigma, tau_c)
    td = dev(c.t)
    rb = sncc.alloc_refine(M, N, W, H, 1 << 14)
    sncc.refine(fd, td, seg, mb, tau_e, rb)
    torch.cuda.synchronize()
    assert int(mb.status.item()) == 0
    u, v, rho = sncc.matches_to_numpy(rb)
    U = M - W + 1
    key = v * U + u
    assert np.all(np.diff(key) > 0)  # sorted, distinct
    ex = O.ncc_exact_at(c.f, c.t, u, v)
    assert np.abs(rho - ex).max(initial=0) <= TOL
    # sets agree outside the threshold bands
    band_c = np.abs(rho_seg.ravel() - tau_c) < TOL
    exact_all = O.ncc_exact_map(c.f, c.t).ravel()
    band_e = np.abs(exact_all - tau_e) < TOL
    amb = band_c | band_e
    got = set(key.tolist())
    want = set(idx_o.tolist())
    diff = got ^ want
    assert all(amb[d] for d in diff), sorted(diff)[:10]
    if W == 32:
        assert c.origin[1] * U + c.origin[0] in got


def test_refine_many_matches_sorted(sncc):
    """Over 10^5 matches (a 1024 x 1024 source, every offset a candidate,
    exact threshold 0.1): the sorted write-out (one bit per offset, prefix
    counts, scatter) returns exactly the oracle's matches in ascending
    v*U+u order with their exact rho (Eq. 1); matches within the tolerance
    of the threshold may go either way."""
    c = synth.case_hd(M=1024, N=1024, W=32, H=32, seed=2024)
    N, M = c.f.shape
    H, W = c.t.shape
    U, V = M - W + 1, N - H + 1
    seg, fd, tb, mb = run_match(sncc, c.f, c.t, 6.0, -1.0, cand_cap=U * V)
    assert int(mb.count.item()) == U * V
    rb = sncc.alloc_refine(M, N, W, H, U * V)
    sncc.refine(fd, dev(c.t), seg, mb, 0.1, rb)
    torch.cuda.synchronize()
    assert int(mb.status.item()) == 0
    u, v, rho = sncc.matches_to_numpy(rb)
    assert len(u) == int(rb.nout.item()) > 100000
    key = v.astype(np.int64) * U + u
    assert np.all(np.diff(key) > 0)
    ex = O.ncc_exact_map(c.f, c.t)
    assert np.abs(rho - ex[v, u]).max() <= TOL
    want = np.flatnonzero(ex.ravel() >= 0.1)
    diff = np.setxor1d(key, want)
    assert np.all(np.abs(ex.ravel()[diff] - 0.1) < TOL), diff[:10]


def test_refine_output_overflow(sncc):
    c = synth.case_plain()
    seg, fd, tb, mb = run_match(sncc, c.f, c.t, 10.0, -1.0)
    rb = sncc.alloc_refine(256, 256, 32, 32, 10)
    sncc.refine(fd, dev(c.t), seg, mb, -1.0, rb)
    torch.cuda.synchronize()
    assert int(rb.nout.item()) == (256 - 31) ** 2
    assert int(mb.status.item()) & sncc.STATUS_MATCH_OVERFLOW
    u, v, rho = sncc.matches_to_numpy(rb)
    assert len(u) == 10 and np.all(np.diff(v * 225 + u) > 0)


# ------------------------------------------------------------------ exact comparator
@pytest.mark.parametrize("M,N,W,H", [(256, 256, 32, 32), (70, 45, 13, 9), (200, 150, 100, 70), (97, 61, 97, 3)])
def test_exact_map_vs_oracle(sncc, M, N, W, H):
    c = synth.case_plain(M=M, N=N, W=W, H=H, seed=7 + W)
    fd = dev(c.f)
    tb = sncc.integral(fd)
    seg = sncc.build_segments(c.t, 1.0)
    rho = sncc.exact_map(fd, dev(c.t), seg.T, seg.T2, tb)
    torch.cuda.synchronize()
    ref = O.ncc_exact_map(c.f, c.t)
    assert np.abs(rho.cpu().numpy() - ref).max() <= TOL


def test_exact_map_int64_tables_multi_block(sncc):
    # a 130 x 129 template spans 3 x 3 template blocks with ragged edges; 64-bit tables
    c = synth.case_plain(M=300, N=260, W=130, H=129, seed=31)
    fd = dev(c.f)
    tb = sncc.integral(fd, s_bits=64)
    seg = sncc.build_segments(c.t, 1.0)
    rho = sncc.exact_map(fd, dev(c.t), seg.T, seg.T2, tb)
    torch.cuda.synchronize()
    ref = O.ncc_exact_map(c.f, c.t)
    assert np.abs(rho.cpu().numpy() - ref).max() <= TOL


def test_exact_map_hd_sampled(sncc):
    c = synth.case_hd()
    fd = dev(c.f)
    tb = sncc.integral(fd)
    seg = sncc.build_segments(c.t, 10.0)
    rho = sncc.exact_map(fd, dev(c.t), seg.T, seg.T2, tb).cpu().numpy()
    rows = np.array([0, 500, c.origin[1], 1016])
    ref = O.ncc_exact_map(c.f, c.t, rows=rows)
    assert np.abs(rho[rows] - ref[rows]).max() <= TOL
    assert abs(rho[c.origin[1], c.origin[0]] - ref[c.origin[1], c.origin[0]]) <= TOL


# ------------------------------------------------------------------ whole path
def test_matcher_end_to_end(sncc):
    c = synth.case_plain()
    m = sncc.Matcher(c.t, c.sigma_max, 256, 256, precision=c.precision)
    fd = dev(c.f)
    m.run(fd)
    torch.cuda.synchronize()
    ap = O.precompute_template_approximation(c.t, c.sigma_max)
    rho_seg, idx_o, rho_o = oracle_matches(c.f, c.t, ap, c.precision * ap.rho_max, c.precision)
    u, v, rho = sncc.matches_to_numpy(m.rb)
    assert m.status() == 0
    np.testing.assert_array_equal(v * 225 + u, idx_o)
    assert np.abs(rho - rho_o).max(initial=0) <= TOL


def test_matcher_graph_replay_matches_eager(sncc):
    """A captured step replayed on a new source gives the eager results."""
    a = synth.case_plain(seed=synth.BASE_SEED + 3)
    b = synth.case_plain(seed=synth.BASE_SEED + 4)
    m = sncc.Matcher(a.t, 3.0, 256, 256, precision=0.5)
    fd = dev(a.f)
    g = m.capture(fd)
    fd.copy_(dev(b.f))
    g.replay()
    torch.cuda.synchronize()
    got = [x.copy() for x in sncc.matches_to_numpy(m.rb)]
    rho_g = m.mb.rho.clone()
    m.run(fd)
    torch.cuda.synchronize()
    want = sncc.matches_to_numpy(m.rb)
    assert torch.equal(rho_g, m.mb.rho)
    assert len(want[0]) > 0
    for x, y in zip(got, want):
        np.testing.assert_array_equal(x, y)


# ------------------------------------------------------------------ the paper's two-approximation search
@pytest.mark.parametrize("M,N,W,H,p,seed", [(256, 256, 32, 32, 0.9, 0), (300, 220, 64, 48, 0.8, 5),
                                            (200, 180, 100, 70, 0.7, 9)])
def test_paper_two_stage_matches_oracle(sncc, M, N, W, H, p, seed):
    """Coarse k_fast at every offset, k_slow at the candidates (Section 5),
    through sncc_match + sncc_refine_segmented_tiles, against the oracle's
    main algorithm; sets agree outside the +-TOL bands of both thresholds."""
    c = synth.case_plain(M=M, N=N, W=W, H=H, seed=synth.BASE_SEED + seed)
    r = O.main_algorithm(c.f, c.t, precision=p)
    m = sncc.PaperMatcher(c.t, M, N, precision=p)
    np.testing.assert_array_equal(m.fast.table, r["fast"].segments)
    np.testing.assert_array_equal(m.slow.table, r["slow"].segments)
    fd = dev(c.f)
    m.run(fd)
    torch.cuda.synchronize()
    assert m.status() == 0
    assert np.abs(m.mb.rho.cpu().numpy() - r["rho_fast"]).max() <= TOL
    u, v, rho = sncc.matches_to_numpy(m.rb)
    U = M - W + 1
    key = v * U + u
    assert np.all(np.diff(key) > 0)
    ap_s = r["slow"]
    rows = np.unique(v)
    ref_s = O.segmented_ncc_map(c.f, ap_s, "sat", rows=rows) if rows.size else None
    if rows.size:
        assert np.abs(rho - ref_s[v, u]).max() <= TOL
    # set agreement outside the bands
    full_s = O.segmented_ncc_map(c.f, ap_s, "sat").ravel()
    amb = (np.abs(r["rho_fast"].ravel() - r["thr_fast"]) < TOL) | (np.abs(full_s - r["thr_slow"]) < TOL)
    diff = set(key.tolist()) ^ set(r["idx"].tolist())
    assert all(amb[d] for d in diff), sorted(diff)[:10]
    assert len(r["idx"]) > 0


def _random_paper_problems(n=6, seed=2026120304):
    """Seeded random problems for the paper's own search: the three source
    generators, templates of 8 to 150 pixels a side, precision 0.3 to 0.9."""
    g = np.random.default_rng(seed)
    out = []
    for i in range(n):
        W, H = int(g.integers(8, 151)), int(g.integers(8, 151))
        M, N = W + int(g.integers(20, 200)), H + int(g.integers(20, 160))
        out.append((i, ("plain", "texture", "hd")[i % 3], M, N, W, H, float(g.choice([0.3, 0.5, 0.7, 0.9])),
                    int(g.integers(0, 1 << 30))))
    return out


@pytest.mark.parametrize("i,kind,M,N,W,H,p,seed", _random_paper_problems())
def test_paper_two_stage_random_problems(sncc, i, kind, M, N, W, H, p, seed):
    """The paper's two-approximation search on random problems against the
    oracle's main algorithm: both segment tables bit for bit, the k_fast map
    within 1e-5, the k_slow values of the matches within 1e-5, and the match
    set equal outside the two threshold bands."""
    c = getattr(synth, "case_" + kind)(M=M, N=N, W=W, H=H, seed=seed)
    r = O.main_algorithm(c.f, c.t, precision=p)
    m = sncc.PaperMatcher(c.t, M, N, precision=p)
    np.testing.assert_array_equal(m.fast.table, r["fast"].segments)
    np.testing.assert_array_equal(m.slow.table, r["slow"].segments)
    m.run(dev(c.f))
    torch.cuda.synchronize()
    assert m.status() == 0
    assert np.abs(m.mb.rho.cpu().numpy() - r["rho_fast"]).max() <= TOL
    u, v, rho = sncc.matches_to_numpy(m.rb)
    U = M - W + 1
    key = v.astype(np.int64) * U + u
    assert np.all(np.diff(key) > 0)
    full_s = O.segmented_ncc_map(c.f, r["slow"], "sat")
    if u.size:
        assert np.abs(rho - full_s[v, u]).max() <= TOL
    amb = (np.abs(r["rho_fast"].ravel() - r["thr_fast"]) < TOL) | (np.abs(full_s.ravel() - r["thr_slow"]) < TOL)
    diff = set(key.tolist()) ^ set(r["idx"].tolist())
    assert all(amb[d] for d in diff), sorted(diff)[:10]


@pytest.mark.parametrize("M,N,W,H,p,seed,bits", [(300, 220, 64, 48, 0.6, 5, 32), (260, 200, 100, 70, 0.5, 9, 64),
                                                 (256, 256, 32, 32, 0.3, 0, 32)])
def test_fine_stage_per_candidate_and_tiled_agree(sncc, M, N, W, H, p, seed, bits):
    """The two implementations of the paper's fine stage return the same
    match list (same offsets, identical rho) on the same coarse candidates,
    with many candidates (low precision) and both table widths."""
    c = synth.case_plain(M=M, N=N, W=W, H=H, seed=synth.BASE_SEED + seed)
    m = sncc.PaperMatcher(c.t, M, N, precision=p)
    fd = dev(c.f)
    tb = sncc.integral(fd, s_bits=bits)
    sncc.match(m.fast, m.plan_fast, tb, m.tau_fast, m.mb)
    rb1 = sncc.alloc_refine(M, N, W, H, 1 << 16)
    sncc.refine_segmented(m.slow, m.plan_slow, tb, m.mb, m.tau_slow, rb1)
    rb2 = sncc.alloc_refine(M, N, W, H, 1 << 16)
    ws = sncc.tiles_workspace(M, N, W, H, 1 << 16)
    sncc.refine_segmented_tiles(m.slow, m.plan_slow, tb, m.mb, m.tau_slow, rb2, ws)
    torch.cuda.synchronize()
    assert int(m.mb.count.item()) > 100
    a, b = sncc.matches_to_numpy(rb1), sncc.matches_to_numpy(rb2)
    assert int(rb1.nout.item()) == int(rb2.nout.item()) > 0
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_fine_stage_tiled_output_overflow(sncc):
    c = synth.case_plain(seed=synth.BASE_SEED)
    m = sncc.PaperMatcher(c.t, 256, 256, precision=0.2)
    fd = dev(c.f)
    tb = sncc.integral(fd)
    sncc.match(m.fast, m.plan_fast, tb, m.tau_fast, m.mb)
    rb = sncc.alloc_refine(256, 256, 32, 32, 7)
    ws = sncc.tiles_workspace(256, 256, 32, 32, 7)
    sncc.refine_segmented_tiles(m.slow, m.plan_slow, tb, m.mb, m.tau_slow, rb, ws)
    torch.cuda.synchronize()
    assert int(rb.nout.item()) > 7
    assert int(m.mb.status.item()) & sncc.STATUS_MATCH_OVERFLOW
    u, v, rho = sncc.matches_to_numpy(rb)
    assert len(u) == 7 and np.all(np.diff(v * 225 + u) > 0)


def test_paper_two_stage_texture_full_size_sampled(sncc):
    """The 4096 x 4096 / 256 x 256 workload through the two-stage search
    (k_fast summed directly at its few corners, k_slow on the tiles that hold
    the ~1.3 M candidates), against the oracle on sampled offset rows: the
    coarse map and the matches of those rows agree outside the bands."""
    c = synth.case_texture()
    N, M = c.f.shape
    H, W = c.t.shape
    U, V = M - W + 1, N - H + 1
    m = sncc.PaperMatcher(c.t, M, N, precision=c.precision, cand_cap=U * V)
    assert m.fast.plan_info()["template_corners"] <= 64
    fd = dev(c.f)
    m.run(fd)
    torch.cuda.synchronize()
    assert m.status() == 0
    rows = np.array([0, 777, c.origin[1], V - 1])
    ap_f, ap_s = O.precompute_template_approximation(c.t, 0.99 * sncc.template_sigma(c.t), 5000), \
        O.precompute_template_approximation(c.t, 0.1 * sncc.template_sigma(c.t), 5000)
    np.testing.assert_array_equal(m.fast.table, ap_f.segments)
    np.testing.assert_array_equal(m.slow.table, ap_s.segments)
    rf = O.segmented_ncc_map(c.f, ap_f, "sat", rows=rows)
    rs = O.segmented_ncc_map(c.f, ap_s, "sat", rows=rows)
    got_f = m.mb.rho.cpu().numpy()
    assert np.abs(got_f[rows] - rf[rows]).max() <= TOL
    thr_f, thr_s = c.precision * ap_f.rho_max, c.precision * ap_s.rho_max
    u, v, rho = sncc.matches_to_numpy(m.rb)
    sel = np.isin(v, rows)
    got = set((v[sel] * U + u[sel]).tolist())
    want, amb = set(), set()
    for r in rows:
        for x in range(U):
            a, b = rf[r, x], rs[r, x]
            if (a >= thr_f + TOL) and (b >= thr_s + TOL):
                want.add(r * U + x)
            elif abs(a - thr_f) < TOL or abs(b - thr_s) < TOL:
                amb.add(r * U + x)
    assert (got ^ want) <= amb
    assert c.origin[1] * U + c.origin[0] in got
    assert np.abs(rho[sel] - rs[v[sel], u[sel]]).max() <= TOL
