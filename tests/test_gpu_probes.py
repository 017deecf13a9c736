"""The ceiling probes compute what their header says: each thread's checksum
equals a host replay of its instruction chains (dp4a as the unsigned
four-byte dot product, the wide multiply-add as signed 32 x 32 -> 64-bit
arithmetic modulo 2^64)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sncc():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA GPU")
    from paper_2502_01286_gb300 import build
    build.build()
    from paper_2502_01286_gb300 import sncc as mod
    return mod


def _dp4a(x, y, c):
    return (sum(((x >> (8 * k)) & 255) * ((y >> (8 * k)) & 255) for k in range(4)) + c) & 0xFFFFFFFF


def _s32(x):
    x &= 0xFFFFFFFF
    return x - (1 << 32) if x >> 31 else x


def _s64(x):
    x &= (1 << 64) - 1
    return x - (1 << 64) if x >> 63 else x


def _replay_dp4a(tid, iters):
    a = [(tid * 7 + i) & 0xFFFFFFFF for i in range(8)]
    for _ in range(iters):
        for q in range(8):
            a = [_dp4a(a[i], 0x01020304 + q, a[i]) for i in range(8)]
    x = 0
    for v in a:
        x ^= v
    return _s32(x)


def _replay_imad_wide(tid, iters):
    acc = [((((tid * 7 + i + 1) * 0x10001) & 0xFFFFFFFF) << 16) | (tid * 13 + i) for i in range(8)]
    for _ in range(iters):
        x = [_s32(a) for a in acc]
        y = [_s32(a >> 32) for a in acc]
        for q in range(8):
            acc = [_s64(acc[i] + x[(i + q) & 7] * y[(i + 2 * q + 1) & 7]) for i in range(8)]
    r = 0
    for a in acc:
        r ^= a
    r = _s64(r)
    return _s32(r ^ (r >> 32))


def test_alu_probes_match_host_replay(sncc):
    import torch
    sink = torch.zeros(2 * 256, dtype=torch.int32, device="cuda")
    for kind, replay in [(sncc.PROBE_DP4A, _replay_dp4a), (sncc.PROBE_IMAD_WIDE, _replay_imad_wide)]:
        n = sncc.probe_alu(kind, sink, 2, 3)
        assert n == 2 * 256 * 3 * 64
        torch.cuda.synchronize()
        got = sink.cpu().numpy()
        want = np.array([replay(t % 256, 3) for t in range(512)], np.int64)
        assert np.array_equal(got.astype(np.int64), want)


def test_smem_probe_runs(sncc):
    import torch
    sink = torch.zeros(4 * 256, dtype=torch.int32, device="cuda")
    assert sncc.probe_smem_read(sink, 4, 2) == 4 * 256 * 2 * 32 * 4
    torch.cuda.synchronize()


def test_hbm_write_probe_writes_every_entry(sncc):
    """Every 16-byte entry i of a buffer larger than L2 holds the header's
    pattern {lo, hi ^ 0x5a5a5a5a, 3 lo, lo ^ 0xffff} after the probe."""
    import torch
    buf = torch.full((160 << 20,), 7, dtype=torch.uint8, device="cuda")
    assert sncc.probe_hbm_write(buf) == 160 << 20
    torch.cuda.synchronize()
    got = buf.view(torch.int32).view(-1, 4).cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    i = np.arange(got.shape[0], dtype=np.int64)
    lo, hi = i & 0xFFFFFFFF, i >> 32
    want = np.stack([lo, hi ^ 0x5A5A5A5A, (lo * 3) & 0xFFFFFFFF, lo ^ 0xFFFF], axis=1)
    assert np.array_equal(got, want)


def test_bounded_wait_gives_up_and_reports(sncc):
    """A wait that nothing completes ends after the wait limit with the
    timeout status bit, and the context keeps working afterwards."""
    import time
    import torch
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sncc.probe_wait_timeout(status)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    assert int(status.item()) & sncc.STATUS_WAIT_TIMEOUT
    assert 0.5 < secs < 30.0
    sink = torch.zeros(256, dtype=torch.int32, device="cuda")
    sncc.probe_alu(sncc.PROBE_DP4A, sink, 1, 1)
    torch.cuda.synchronize()
    assert int(sink[0].item()) == _replay_dp4a(0, 1)
