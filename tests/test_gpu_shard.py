"""The band split of one source (one rank per band) run on the GPU: every
band goes through the library's own path on its source rows (sum tables of
the band, coarse pass, exact refine), the band lists are mapped back to the
full source's offsets and merged, and the result equals one launch over the
whole source bit for bit - same offsets, identical rho - because every box
sum, window sum and exact sum is the same integer whichever table it comes
from (main algorithm step 7: every offset is independent)."""
import numpy as np
import pytest

from paper_2502_01286_gb300 import shard, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sncc():
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA GPU")
    from paper_2502_01286_gb300 import build
    build.build()
    from paper_2502_01286_gb300 import sncc as mod
    return mod


def run_full(sncc, c, sigma, p, cand_cap, out_cap):
    N, M = c.f.shape
    m = sncc.Matcher(c.t, sigma, M, N, precision=p, cand_cap=cand_cap, out_cap=out_cap)
    m.run(torch.as_tensor(c.f).cuda())
    torch.cuda.synchronize()
    assert m.status() == 0
    u, v, rho = sncc.matches_to_numpy(m.rb)
    return m, v.astype(np.int64) * (M - c.t.shape[1] + 1) + u, rho


def run_bands(sncc, c, sigma, p, world, cand_cap, out_cap):
    """Each band one after another on this GPU, as its rank would run it."""
    N, M = c.f.shape
    H, W = c.t.shape
    U = M - W + 1
    parts, maps = [], []
    for b in shard.bands(N, H, world):
        if b.empty:
            continue
        sub = np.ascontiguousarray(c.f[b.src_y0:b.src_y1])
        m = sncc.Matcher(c.t, sigma, M, sub.shape[0], precision=p, cand_cap=cand_cap, out_cap=out_cap)
        m.run(torch.as_tensor(sub).cuda())
        torch.cuda.synchronize()
        assert m.status() == 0
        u, v, rho = sncc.matches_to_numpy(m.rb)
        parts.append((shard.to_global(b, U, u, v), rho))
        maps.append((b, m.mb.rho.cpu()))
    idx, rho = shard.merge(parts)
    return idx, rho, maps


@pytest.mark.parametrize("world", [2, 3])
def test_bands_equal_one_launch_texture(sncc, world):
    """The 4096 x 4096 / 256 x 256 texture workload (sigma 5, 64-bit tables
    on the full source) split into 2 and 3 bands with an H - 1 row halo:
    the merged match list and every band's rho rows equal the full launch's
    exactly; precision 0.6 gives thousands of matches across the bands."""
    c = synth.case_texture()
    N, M = c.f.shape
    H, W = c.t.shape
    U, V = M - W + 1, N - H + 1
    full, idx_full, rho_full = run_full(sncc, c, 5.0, 0.6, U * V // 8, 1 << 20)
    idx, rho, maps = run_bands(sncc, c, 5.0, 0.6, world, U * V // 8, 1 << 20)
    assert idx_full.size > 1000
    np.testing.assert_array_equal(idx, idx_full)
    np.testing.assert_array_equal(rho, rho_full)
    full_rho = full.mb.rho.cpu()
    for b, r in maps:
        assert torch.equal(r, full_rho[b.v0:b.v1])
    # the matches are spread over the bands
    per_band = [int(np.sum((idx // U >= b.v0) & (idx // U < b.v1))) for b in shard.bands(N, H, world)]
    assert sum(1 for n in per_band if n > 0) > 1, per_band


def test_bands_equal_one_launch_hd_ragged(sncc):
    """HD source (1920 x 1080, 64 x 64 template) in 7 bands of 145 or 146
    offset rows: tile heights and table widths change per band, the list
    does not (precision 0.25)."""
    c = synth.case_hd()
    N, M = c.f.shape
    H, W = c.t.shape
    U, V = M - W + 1, N - H + 1
    _, idx_full, rho_full = run_full(sncc, c, 10.0, 0.25, U * V, 1 << 20)
    idx, rho, _ = run_bands(sncc, c, 10.0, 0.25, 7, U * V, 1 << 20)
    assert idx_full.size > 1000  # about 6000 at precision 0.25, spread over every band
    np.testing.assert_array_equal(idx, idx_full)
    np.testing.assert_array_equal(rho, rho_full)
