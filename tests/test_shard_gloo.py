"""The multi-rank path on CPU: world_size-2 gloo process groups split one
source into bands of offset rows, each rank computes its band (the FP64
oracle stands in for the GPU here, since these tests run without one) and
the gathered match list equals the single-rank result exactly."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2502_01286_gb300 import shard, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_bands_partition_offsets():
    for N, H, world in [(100, 10, 2), (100, 10, 3), (50, 50, 4), (64, 1, 7), (12, 5, 8)]:
        bs = shard.bands(N, H, world)
        V = N - H + 1
        rows = [v for b in bs for v in range(b.v0, b.v1)]
        assert rows == list(range(V))
        for b in bs:
            if not b.empty:
                assert b.src_y0 == b.v0 and b.src_y1 == b.v1 + H - 1 <= N
        sizes = [b.v1 - b.v0 for b in bs]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.bands(10, 11, 2)


def test_merge_rejects_overlap():
    with pytest.raises(ValueError):
        shard.merge([(np.array([3, 5]), np.array([0.1, 0.2])), (np.array([5]), np.array([0.3]))])
    idx, rho = shard.merge([(np.array([9, 2]), np.array([0.9, 0.2])), (np.array([4]), np.array([0.4]))])
    assert idx.tolist() == [2, 4, 9] and np.allclose(rho, [0.2, 0.4, 0.9])


def _band_matches(f, t, sigma, p, band):
    """One rank's work: the whole path on its band only (oracle stand-in)."""
    H, W = t.shape
    sub = f[band.src_y0:band.src_y1]
    ap = O.precompute_template_approximation(t, sigma)
    rho = O.segmented_ncc_map(sub, ap, "sat")
    cand = O.candidates(rho, p * ap.rho_max)
    U = f.shape[1] - W + 1
    idx_local, r = O.refine(sub, t, cand, U, p)
    return shard.to_global(band, U, idx_local % U, idx_local // U), r


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = synth.case_hd(M=150, N=111, W=24, H=18, seed=77)
        band = shard.bands(c.f.shape[0], c.t.shape[0], world)[rank]
        idx, rho = _band_matches(c.f, c.t, 10.0, 0.3, band) if not band.empty else (np.zeros(0, np.int64),
                                                                                   np.zeros(0, np.float32))
        got = shard.gather_matches(idx, rho)
        if rank == 0:
            out.put((got[0].tolist(), np.asarray(got[1], np.float64).tolist()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks_match_single_rank(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got_idx, got_rho = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    c = synth.case_hd(M=150, N=111, W=24, H=18, seed=77)
    full_band = shard.bands(c.f.shape[0], c.t.shape[0], 1)[0]
    want_idx, want_rho = _band_matches(c.f, c.t, 10.0, 0.3, full_band)
    assert got_idx == [int(i) for i in want_idx]
    np.testing.assert_allclose(got_rho, want_rho, atol=1e-12)
    # matches come from both bands (65 in the first, 105 in the second)
    b0 = shard.bands(c.f.shape[0], c.t.shape[0], world)[0]
    U = c.f.shape[1] - c.t.shape[1] + 1
    first = sum(1 for i in got_idx if i // U < b0.v1)
    assert 0 < first < len(got_idx)
