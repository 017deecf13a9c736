"""GPU parity of the batched path (many templates x several sources in one
persistent launch) against the FP64 oracle, pair by pair."""
import numpy as np
import pytest

import oracle as O
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


@pytest.fixture(scope="module")
def problem():
    M, N = 200, 150
    srcs = synth.batch_sources(count=3, M=M, N=N)
    tl = synth.batch_templates(srcs, count=7, lo=16, hi=100)
    p = 0.7
    ref = []
    for t, _, sg in tl:
        ap = O.precompute_template_approximation(t, sg)
        ref.append(ap)
    maps = {}
    for s, f in enumerate(srcs):
        for ti, ap in enumerate(ref):
            maps[(s, ti)] = O.segmented_ncc_map(f, ap, "sat")
    return M, N, srcs, tl, ref, maps, p


def _check_batch(sncc, b, problem):
    M, N, srcs, tl, ref, maps, p = problem
    nt = len(tl)
    pair, idx = b.candidates()
    assert int(b.status.item()) == 0
    got = set(zip(pair.tolist(), idx.tolist()))
    assert len(got) == len(pair)
    for s in range(len(srcs)):
        for ti, ap in enumerate(ref):
            rho = maps[(s, ti)].ravel()
            tau = p * ap.rho_max
            pid = s * nt + ti
            mine = {i for (q, i) in got if q == pid}
            must = set(np.flatnonzero(rho >= tau + TOL).tolist())
            never = set(np.flatnonzero(rho < tau - TOL).tolist())
            assert must <= mine, (pid, len(must - mine))
            assert not (mine & never), (pid, sorted(mine & never)[:5])
    return got


def test_batch_coarse_and_refine_vs_oracle(sncc, problem):
    M, N, srcs, tl, ref, maps, p = problem
    b = sncc.Batch([t for t, _, _ in tl], [sg for _, _, sg in tl], M, N, len(srcs), precision=p)
    fd = [torch.as_tensor(f).cuda() for f in srcs]
    b.run(fd)
    torch.cuda.synchronize()
    _check_batch(sncc, b, problem)
    pair, u, v, rho = b.matches()
    nt = len(tl)
    order_keys = [(int(q), int(vv) * (M - tl[int(q) % nt][0].shape[1] + 1) + int(uu)) for q, uu, vv in zip(pair, u, v)]
    assert order_keys == sorted(order_keys)
    for q, uu, vv, r in zip(pair, u, v, rho):
        s, ti = int(q) // nt, int(q) % nt
        ex = O.ncc_exact_at(srcs[s], tl[ti][0], [int(uu)], [int(vv)])[0]
        assert abs(ex - r) <= TOL and ex >= p - TOL
    # every exact match among the coarse candidates is reported (outside the bands)
    want = set()
    for s in range(len(srcs)):
        for ti, ap in enumerate(ref):
            U = M - tl[ti][0].shape[1] + 1
            cand = O.candidates(maps[(s, ti)], p * ap.rho_max + TOL)
            idx, r = O.refine(srcs[s], tl[ti][0], cand, U, p + TOL)
            want |= {(s * nt + ti, int(i)) for i in idx}
    got = {(int(q), int(vv) * (M - tl[int(q) % nt][0].shape[1] + 1) + int(uu)) for q, uu, vv in zip(pair, u, v)}
    assert want <= got


def test_batch_variants_agree_and_autotune_per_bucket(sncc, problem):
    """Every tile height and block edge gives the same candidate set; the
    autotuner times each bucket in each variant and keeps its fastest."""
    M, N, srcs, tl, ref, maps, p = problem
    b = sncc.Batch([t for t, _, _ in tl], [sg for _, _, sg in tl], M, N, len(srcs), precision=p)
    fd = [torch.as_tensor(f).cuda() for f in srcs]
    sets = []
    for R in (8, 4, 2):
        b.set_tile_rows(R)
        b.run(fd)
        torch.cuda.synchronize()
        sets.append(_check_batch(sncc, b, problem))
        assert b.info()["tile_rows"] == R
    # 32 x 32 template blocks in every bucket give the same candidates
    for k in range(sncc.BATCH_BUCKETS):
        b.set_bucket_variant(k, 4, 32)
    b.run(fd)
    torch.cuda.synchronize()
    sets.append(_check_batch(sncc, b, problem))
    assert sets[0] == sets[1] == sets[2] == sets[3]
    ms = b.autotune(fd, reps=2)
    buckets = b.buckets()
    assert set(ms) == {k for k, bb in enumerate(buckets) if bb["pairs"]} and len(ms) >= 2
    for k, times in ms.items():
        assert len(times) == 6 and all(v > 0 for v in times.values())
        assert (buckets[k]["tile_rows"], buckets[k]["block"]) == min(times, key=times.get)
    assert sum(bb["pairs"] for bb in buckets) == len(srcs) * len(tl)
    # the tuned (mixed) variants still give the same candidates
    b.run(fd)
    torch.cuda.synchronize()
    assert _check_batch(sncc, b, problem) == sets[0]


def test_batch_cuda_graph_replay(sncc, problem):
    M, N, srcs, tl, ref, maps, p = problem
    b = sncc.Batch([t for t, _, _ in tl], [sg for _, _, sg in tl], M, N, len(srcs), precision=p)
    fd = [torch.as_tensor(f).cuda() for f in srcs]
    g = b.capture(fd)
    b.count.zero_()
    b.nout.zero_()
    g.replay()
    torch.cuda.synchronize()
    first = _check_batch(sncc, b, problem)
    m1 = b.matches()
    # new pixels in the same buffers, replay again: results follow the data
    fd[0].copy_(torch.as_tensor(srcs[1]).cuda())
    g.replay()
    torch.cuda.synchronize()
    pair, idx = b.candidates()
    nt = len(tl)
    got0 = {(int(q), int(i)) for q, i in zip(pair, idx) if int(q) < nt}
    got1 = {(int(q) - nt, int(i)) for q, i in zip(pair, idx) if nt <= int(q) < 2 * nt}
    assert got0 == got1 and len(got0) > 0  # source 0 now holds source 1's pixels
    fd[0].copy_(torch.as_tensor(srcs[0]).cuda())
    g.replay()
    torch.cuda.synchronize()
    assert _check_batch(sncc, b, problem) == first
    m2 = b.matches()
    for a, c in zip(m1, m2):
        np.testing.assert_array_equal(a, c)


def test_batch_config4_full_size_sampled(sncc):
    """The batched workload at its real size: 8 sources of 1024 x 1024 and
    64 templates with sides 16 .. 256 and std thresholds 4 .. 25 (512 pairs,
    K from about 100 to 38000) in one persistent launch at precision 0.85.
    For every pair one random offset row, and for each template the row of
    its own crop in its own source, go through the oracle: candidates obey
    the band rule (Eq. 17 - 18, steps 7a-7f) and the exact matches on those
    rows (Eq. 1, steps 7g-7j) equal the oracle's outside the bands, with rho
    within the tolerance."""
    srcs = synth.batch_sources()
    tl = synth.batch_templates(srcs)
    M = N = 1024
    p = 0.85
    nt, ns = len(tl), len(srcs)
    b = sncc.Batch([t for t, _, _ in tl], [sg for _, _, sg in tl], M, N, ns, precision=p, cand_cap=1 << 22,
                   out_cap=1 << 18)
    fd = [torch.as_tensor(f).cuda() for f in srcs]
    b.run(fd)
    torch.cuda.synchronize()
    assert int(b.status.item()) == 0
    pair, idx = b.candidates()
    cand = {}
    for q, i in zip(pair.tolist(), idx.tolist()):
        cand.setdefault(q, set()).add(i)
    mp, mu, mv, mrho = b.matches()
    matches = {}
    for q, uu, vv, r in zip(mp.tolist(), mu.tolist(), mv.tolist(), mrho.tolist()):
        matches.setdefault(q, {})[(uu, vv)] = r
    rng = np.random.default_rng(2025)
    checked = positives = 0
    for ti, (t, org, sg) in enumerate(tl):
        ap = O.precompute_template_approximation(t, sg)
        H, W = t.shape
        U, V = M - W + 1, N - H + 1
        tau = p * ap.rho_max
        for s in range(ns):
            rows = [int(rng.integers(0, V))]
            if s == ti % ns:
                rows.append(int(org[1]))  # the template's own crop
            rows = np.unique(rows)
            rho = O.segmented_ncc_map(srcs[s], ap, "sat", rows=rows)
            q = s * nt + ti
            mine = cand.get(q, set())
            for r in rows:
                row_idx = {i - r * U for i in mine if i // U == r}
                must = set(np.flatnonzero(rho[r] >= tau + TOL).tolist())
                never = set(np.flatnonzero(rho[r] < tau - TOL).tolist())
                assert must <= row_idx, (q, r)
                assert not (row_idx & never), (q, r)
                checked += U
                # exact refine of the oracle's candidates on this row
                oc = np.flatnonzero(rho[r] >= tau)
                ex = O.ncc_exact_at(srcs[s], t, oc.astype(np.int32), np.full(oc.size, r, np.int32)) \
                    if oc.size else np.zeros(0)
                want = {int(u) for u, e in zip(oc, ex) if e >= p + TOL}
                got = {uu for (uu, vv) in matches.get(q, {}) if vv == r}
                amb = {int(u) for u, e in zip(oc, ex) if abs(e - p) < TOL} | \
                      {int(u) for u in np.flatnonzero(np.abs(rho[r] - tau) < TOL)}
                assert (got ^ want) <= amb, (q, r, sorted(got ^ want)[:5])
                for uu in got:
                    e = O.ncc_exact_at(srcs[s], t, [uu], [r])[0]
                    assert abs(matches[q][(uu, r)] - e) <= TOL
                positives += len(want)
    assert checked > 400000 and positives >= 32


def test_batch_on_wrapping_sources_equals_single_matches_on_int64_tables(sncc):
    """Two bright textured 4096 x 2800 sources (values 150 to 255: sums past
    2^31, so the batch's 32-bit tables wrap) and two templates cropped from
    the first (128 x 96 and 200 x 150, std threshold 5: 202 and 814
    segments): every pair's
    candidate set and exact match list equal those of the single-template
    path on 64-bit tables (the same integer numerators and window sums)."""
    M, N = 4096, 2800
    base = synth.case_texture(M=M, N=N, W=200, H=150)
    srcs = [(150 + base.f.astype(np.int64) * 105 // 255).astype(np.uint8)]
    srcs.append(np.ascontiguousarray(srcs[0][::-1, ::-1]))
    assert int(srcs[0].astype(np.int64).sum()) >= 2 ** 31
    u0, v0 = base.origin
    tl = [np.ascontiguousarray(srcs[0][v0:v0 + 96, u0:u0 + 128]), np.ascontiguousarray(srcs[0][v0:v0 + 150, u0:u0 + 200])]
    sig, p = 5.0, 0.95
    b = sncc.Batch(tl, [sig, sig], M, N, 2, precision=p, cand_cap=1 << 23, out_cap=1 << 20)
    fd = [torch.as_tensor(f).cuda() for f in srcs]
    b.run(fd)
    torch.cuda.synchronize()
    assert int(b.status.item()) == 0
    pair, idx = b.candidates()
    mp, mu, mv, mrho = b.matches()
    nt = len(tl)
    total = 0
    for s, f in enumerate(fd):
        tb = sncc.integral(f, s_bits=64)
        for ti, t in enumerate(tl):
            seg = sncc.build_segments(t, sig)
            plan = sncc.upload_plan(seg)
            H, W = t.shape
            mb = sncc.alloc_match(M, N, W, H, 1 << 23)
            sncc.match(seg, plan, tb, p * seg.rho_max, mb)
            rb = sncc.alloc_refine(M, N, W, H, 1 << 20)
            sncc.refine(f, torch.as_tensor(t).cuda(), seg, mb, p, rb)
            torch.cuda.synchronize()
            q = s * nt + ti
            want = np.sort(mb.cand[:int(mb.count.item())].cpu().numpy())
            got = np.sort(idx[pair == q])
            np.testing.assert_array_equal(got, want)
            u, v, rho = sncc.matches_to_numpy(rb)
            sel = mp == q
            np.testing.assert_array_equal(mu[sel], u)
            np.testing.assert_array_equal(mv[sel], v)
            np.testing.assert_array_equal(mrho[sel], rho)
            assert int(mb.status.item()) == 0
            total += len(want)
    assert total > 0 and len(mu) > 0


def _random_batches(n=3, seed=2026120302):
    """Seeded random batches: source size, source and template counts,
    template sides from 8 up to the source, precision, and one variant (tile
    height, template block edge) per bucket."""
    g = np.random.default_rng(seed)
    out = []
    for i in range(n):
        M, N = int(g.integers(150, 420)), int(g.integers(150, 420))
        out.append((i, M, N, int(g.integers(1, 4)), int(g.integers(4, 8)), min(M, N, 256) - 1,
                    float(g.choice([0.6, 0.75, 0.9])), int(g.integers(0, 1 << 30)),
                    [(int(g.choice([8, 4, 2])), int(g.choice([64, 32]))) for _ in range(16)]))
    return out


@pytest.mark.parametrize("i,M,N,ns,nt,hi,p,seed,variants", _random_batches())
def test_batch_random_problems_vs_oracle(sncc, i, M, N, ns, nt, hi, p, seed, variants):
    """A random batch in mixed per-bucket variants: every pair's candidates by
    the band rule against the oracle's map, and the exact matches (sorted,
    values within 1e-5, every oracle match outside the bands present)."""
    srcs = synth.batch_sources(count=ns, M=M, N=N, seed=seed)
    tl = synth.batch_templates(srcs, count=nt, seed=seed + 1, lo=8, hi=hi)
    ref = [O.precompute_template_approximation(t, sg) for t, _, sg in tl]
    b = sncc.Batch([t for t, _, _ in tl], [sg for _, _, sg in tl], M, N, ns, precision=p)
    for k in range(sncc.BATCH_BUCKETS):
        b.set_bucket_variant(k, *variants[k % len(variants)])
    b.run([torch.as_tensor(f).cuda() for f in srcs])
    torch.cuda.synchronize()
    assert int(b.status.item()) == 0
    pair, idx = b.candidates()
    got = set(zip(pair.tolist(), idx.tolist()))
    assert len(got) == len(pair)
    mp, mu, mv, mrho = b.matches()
    keys = [(int(q), int(vv) * (M - tl[int(q) % nt][0].shape[1] + 1) + int(uu)) for q, uu, vv in zip(mp, mu, mv)]
    assert keys == sorted(keys)
    for s in range(ns):
        for ti, ap in enumerate(ref):
            W = tl[ti][0].shape[1]
            U = M - W + 1
            rho = O.segmented_ncc_map(srcs[s], ap, "sat")
            flat = rho.ravel()
            tau = p * ap.rho_max
            pid = s * nt + ti
            mine = {j for (q, j) in got if q == pid}
            assert set(np.flatnonzero(flat >= tau + TOL).tolist()) <= mine, pid
            assert not (mine & set(np.flatnonzero(flat < tau - TOL).tolist())), pid
            sel = mp == pid
            u, v, r = mu[sel], mv[sel], mrho[sel]
            if u.size:
                ex = O.ncc_exact_at(srcs[s], tl[ti][0], u.astype(np.int32), v.astype(np.int32))
                assert np.abs(ex - r).max() <= TOL and ex.min() >= p - TOL
            idx_o, _ = O.refine(srcs[s], tl[ti][0], O.candidates(rho, tau + TOL), U, p + TOL)
            assert set(idx_o.tolist()) <= set((v.astype(np.int64) * U + u).tolist()), pid
