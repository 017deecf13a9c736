#!/usr/bin/env python3
"""Benchmark of the segmented-NCC hot path on GB300.

Workload (default "texture"): a 4096 x 4096 uint8 high-texture source (300
random rectangles plus 1/f noise) and a 256 x 256 template cropped from it,
std threshold 5 (a few thousand segments), coarse precision 0.85
(tau_c = 0.85 * rho_max), exact refine threshold 0.85, 64-bit sum tables,
exact direct NCC timed on the same GPU beside it.  One step = one pass of the
whole path over the source: the sum tables, the coarse pass (segmented NCC
map, threshold, candidates) and the exact refine of the candidates.  The
metric counts offsets evaluated: U * V per step and threshold.  Other
workloads (--workload): "hd" (1920 x 1080, 64 x 64, thresholds 5, 10, 20),
"plain", "batch", "diff".

Printed: one JSON line (rank 0).  Timing: CUDA events on the launching stream
around every step, an L2 flush (a 256 MiB write) between steps outside the
events, a barrier and synchronize on both sides of the timed region, the max
over ranks.  --impl reference times the FP64 CPU oracle on a bounded sample
of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "segmented-NCC Goffsets/s vs exact NCC on same GB300 at stated max |dNCC|"
UNIT = "Goffsets/s"
L2_FLUSH_BYTES = 256 << 20

# name -> (case factory name, std thresholds swept in one step, precision p).
# "texture" is the workload the metric is quoted on (the largest single
# problem, where the comparison with exact NCC on the same GPU is made); the
# others are measured on request (--workload) and are otherwise parity-test
# cases.
WORKLOADS = {
    "hd": ("case_hd", (5.0, 10.0, 20.0), 0.85),
    "plain": ("case_plain", (10.0,), 0.9),
    "texture": ("case_texture", (5.0,), 0.85),
    "batch": ("batch", None, 0.85),
    "diff": ("diff", None, None),
}
SIGMAS = WORKLOADS["hd"][1]
PRECISION = WORKLOADS["hd"][2]


def make_case(workload: str, seed_offset: int = 0):
    from paper_2502_01286_gb300 import synth
    factory, sigmas, precision = WORKLOADS[workload]
    fn = getattr(synth, factory)
    return fn(seed=case_seed_of(workload, seed_offset)), sigmas, precision


def case_seed_of(workload: str, seed_offset: int = 0) -> int:
    from paper_2502_01286_gb300 import synth
    factory = WORKLOADS[workload][0]
    return synth.BASE_SEED + {"case_plain": 0, "case_hd": 1, "case_texture": 2}[factory] + seed_offset


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["sncc", "reference"], default="sncc")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["crossover"], default="texture")
    ap.add_argument("--shard", choices=["replicas", "bands"], default="replicas",
                    help="N > 1: each rank its own problem (replicas, weak scaling) or one source split into bands "
                         "of offset rows with an H - 1 row halo (bands, strong scaling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle baseline")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; no collective on the data path)
# ---------------------------------------------------------------------------
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "sncc" else "gloo"
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        if backend == "nccl":
            import torch
            # bind this rank's GPU before the first collective, so that every
            # barrier and reduction runs on the rank's own device
            torch.cuda.set_device(local)
            dist.init_process_group(backend=backend, device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, value: float) -> float:
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, value: float) -> float:
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append((time.time(), ln.strip()))

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [ln for (ts, ln) in self.lines if self.t0 is not None and self.t0 <= ts <= (self.t1 or ts) + 0.1]
        if not rows:
            rows = [ln for (_, ln) in self.lines]
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in rows:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 10:
                continue
            try:
                sm.append(float(p[2]))
                smax.append(float(p[3]))
                power.append(float(p[4]))
            except ValueError:
                continue
            for nm, val in zip(names, p[6:10]):
                if val == "Active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(case, sigmas, rows_per_sigma, seed=0, precision=None):
    """Runs the oracle's version of one step on `rows_per_sigma` offset rows
    per threshold: sum tables + segmented NCC (Eq. 10 - 18) on those rows,
    candidates, exact refine.  Returns (offsets, seconds, threads, maps) with
    maps[sigma] = (rows, rho map (NaN outside the rows), matches (ascending
    v*U+u), their exact rho)."""
    import oracle as O
    f, t = case.f, case.t
    N, M = f.shape
    H, W = t.shape
    U, V = M - W + 1, N - H + 1
    rng = np.random.default_rng(seed)
    p = case.precision if precision is None else precision
    threads = O.default_threads()
    total, secs, maps = 0, 0.0, {}
    for s in sigmas:
        ap = O.precompute_template_approximation(t, s)
        rows = np.sort(rng.choice(V, size=min(rows_per_sigma, V), replace=False))
        t0 = time.perf_counter()
        rho = O.segmented_ncc_map(f, ap, "sat", rows=rows, nthreads=threads)
        cand = O.candidates(rho, p * ap.rho_max)
        idx, rho_e = O.refine(f, t, cand, U, p)
        secs += time.perf_counter() - t0
        total += len(rows) * U
        maps[s] = (rows, rho, idx, rho_e)
    return total, secs, threads, maps


TOL = 1e-5  # the parity bar: |rho_gpu - rho_oracle| and the G13 decision band


def sampled_set_check(f, t, rows, rho64, idx_o, rho_o, cand_gpu, match_gpu, U, tau_c, tau_e):
    """The GPU's candidate and match sets on the oracle's sampled offset rows.
    G13: every offset with rho64 >= tau_c + TOL must be a candidate and every
    one with rho64 < tau_c - TOL must not; offsets inside the band may go
    either way and are counted.  The match lists may differ only at offsets
    inside the coarse band or inside the exact band around tau_e."""
    import oracle as O
    V = rho64.shape[0]
    on_rows = np.zeros(V, bool)
    on_rows[rows] = True
    got_c = np.zeros(rho64.shape, bool)
    cg = np.asarray(cand_gpu, np.int64)
    got_c.ravel()[cg] = True
    r, g = rho64[rows], got_c[rows]
    band = (r >= tau_c - TOL) & (r < tau_c + TOL)
    violations = int(np.sum(g & (r < tau_c - TOL)) + np.sum(~g & (r >= tau_c + TOL)))
    mu, mv, mrho = match_gpu
    sel = on_rows[mv]
    key_g = mv[sel].astype(np.int64) * U + mu[sel]
    diff = np.setxor1d(key_g, idx_o)
    if diff.size:
        ex = O.ncc_exact_at(f, t, (diff % U).astype(np.int32), (diff // U).astype(np.int32))
        amb = (np.abs(rho64.ravel()[diff] - tau_c) < TOL) | (np.abs(ex - tau_e) < TOL)
        outside = int(np.sum(~amb))
    else:
        outside = 0
    common, ig, io = np.intersect1d(key_g, idx_o, return_indices=True)
    drho = float(np.abs(mrho[sel][ig].astype(np.float64) - rho_o[io]).max()) if common.size else 0.0
    return {"g13_band_offsets": int(band.sum()), "g13_violations": violations,
            "candidates_on_rows": int(g.sum()), "matches_oracle": int(idx_o.size), "matches_gpu": int(key_g.size),
            "match_diff_outside_bands": outside, "max_abs_drho_matches": drho}


def calibrate_rows(case, sigmas, budget_s: float) -> int:
    """Rows per threshold so that one oracle_sample takes about budget_s.
    The oracle spreads rows over all host threads, so the fit uses one and
    three rounds of rows per thread: time = fixed + per_row * rows."""
    import oracle as O
    T = O.default_threads()
    _, t_small, _, _ = oracle_sample(case, sigmas, T, seed=12345)
    _, t_large, _, _ = oracle_sample(case, sigmas, 3 * T, seed=12346)
    per_row = max((t_large - t_small) / (2.0 * T), 1e-7)
    fixed = max(t_small - T * per_row, 0.0)
    return max(1, int((budget_s - fixed) / per_row))


def run_reference(args, world, rank, pg):
    """The reference arm: the FP64 CPU oracle as it stands, timed on the host
    cores, each step a bounded sample of the same workload."""
    if rank != 0:
        return
    if args.workload == "crossover":
        print(json.dumps({"impl": "reference", "unavailable": "the crossover sweep compares two GPU kernels; "
                                                              "the oracle's timing is reported per workload"}))
        return
    if args.workload == "batch":
        return run_reference_batch(args)
    if args.workload == "diff":
        return run_reference_diff(args)
    case, sigmas, precision = make_case(args.workload)
    N, M = case.f.shape
    H, W = case.t.shape
    U, V = M - W + 1, N - H + 1
    budget_total = 150.0
    rows = calibrate_rows(case, sigmas, budget_total / max(1, args.steps + args.warmup))
    for i in range(args.warmup):
        oracle_sample(case, sigmas, rows, seed=i)
    offsets, secs, threads = 0, 0.0, 1
    for i in range(args.steps):
        o, s, threads, _ = oracle_sample(case, sigmas, rows, seed=1000 + i)
        offsets += o
        secs += s
    value = offsets / secs / 1e9
    sample = "%d random offset rows x %d offsets per threshold per step (of %d rows), thresholds %s" % (
        min(rows, V), U, V, list(sigmas))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(args.workload, case, sigmas, precision, U, V, case_seed_of(args.workload)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def diff_config(seg):
    """The differentiation workload as both arms describe it."""
    return {"workload": "diff-512x512f32-t48x48-sigma12", "segments": int(seg.K),
            "l2": "flushed between steps (256 MiB write)"}


def run_reference_diff(args):
    """The oracle's FP64 loss and analytic gradients (oracle/diff.py) on a
    128 x 128 crop of the differentiation source with the same template."""
    from oracle import diff as D
    from paper_2502_01286_gb300 import sncc, synth
    f, t, org, sigma = synth.case_diff()
    seg = sncc.build_segments(np.rint(np.clip(t, 0, 255)).astype(np.uint8), sigma)
    rects = seg.table
    k0 = np.array([t[y:y + h, x:x + w].mean() for x, y, w, h in rects])
    fc = f[:128, :128].astype(np.float64)
    U = V = 128 - 48 + 1
    for _ in range(args.warmup):
        D.gradients(fc, t.astype(np.float64), rects, k0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        D.gradients(fc, t.astype(np.float64), rects, k0)
    secs = time.perf_counter() - t0
    value = args.steps * U * V / secs / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": diff_config(seg),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "loss + analytic gradients on a 128 x 128 crop (81 x 81 offsets) per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_batch(args):
    srcs, tl = batch_problem(0)
    rng = np.random.default_rng(5)
    pairs = [(int(rng.integers(0, len(srcs))), int(rng.integers(0, len(tl)))) for _ in range(8)]
    import oracle as O
    T = O.default_threads()
    _, s1, _ = batch_oracle_sample(srcs, tl, T, pairs, seed=1)
    rows = max(1, int(T * 150.0 / max(1, args.steps + args.warmup) / max(s1, 1e-3)))
    for i in range(args.warmup):
        batch_oracle_sample(srcs, tl, rows, pairs, seed=10 + i)
    offs, secs, threads = 0, 0.0, 1
    for i in range(args.steps):
        o, s_, threads = batch_oracle_sample(srcs, tl, rows, pairs, seed=100 + i)
        offs += o
        secs += s_
    value = offs / secs / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": batch_config(srcs, tl),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "up to %d random offset rows of each of 8 random pairs per step" % rows},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(name, case, sigmas, precision, U, V, seed):
    """The workload as both arms describe it (the same dict in each)."""
    N, M = case.f.shape
    H, W = case.t.shape
    return {"workload": "%s-%dx%d-t%dx%d-sigma%s" % (name, M, N, W, H, "-".join("%g" % s for s in sigmas)),
            "source": [M, N], "template": [W, H], "sigma_max": list(sigmas), "precision": precision,
            "offsets_per_step": len(sigmas) * U * V, "l2": "flushed between steps (256 MiB write)",
            "sum_tables": "s int32 (modulo 2^32), s2 int64", "seed": seed}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def kernel_hash() -> str:
    h = hashlib.sha256()
    for fn in ("sncc_match.cu", "sncc_ptx.cuh", "sncc_internal.h", "sncc_tile.cuh"):
        with open(os.path.join(ROOT, "paper_2502_01286_gb300", "csrc", fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str):
    """DRAM bytes per launch of the segment-sum kernel on this workload from
    the committed ncu records, if one was taken on the current kernel
    source; else None."""
    p = os.path.join(ROOT, "profiles", "match_kernel_traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    for r in d.get("records", []):
        if r.get("workload") == workload and r.get("kernel_hash") == kernel_hash():
            return r.get("dram_bytes_per_launch")
    return None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def measure_ceilings(sncc, torch, stream, dev):
    """Ceilings measured live by the library's probes (best of 5):
    shared-memory read GB/s, dp4a and 32x32->64-bit multiply-add
    instructions per second (lane operations), and the HBM write rate of
    16-byte stores over 1 GiB."""
    set_sm_count(torch, dev)
    ctas = SM_COUNT * 8
    sink = torch.empty(ctas * 256, dtype=torch.int32, device=dev)

    def best(launch):
        launch(8)
        rates = []
        for _ in range(5):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            n = launch(2048)
            b.record(stream)
            torch.cuda.synchronize()
            rates.append(n / (a.elapsed_time(b) * 1e-3))
        return max(rates)

    wbuf = torch.empty(1 << 30, dtype=torch.uint8, device=dev)
    sncc.probe_hbm_write(wbuf)
    wrates = []
    for _ in range(5):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        n = sncc.probe_hbm_write(wbuf)
        b.record(stream)
        torch.cuda.synchronize()
        wrates.append(n / (a.elapsed_time(b) * 1e-3))
    del wbuf
    return {"smem_gbs": best(lambda it: sncc.probe_smem_read(sink, ctas, it)) / 1e9,
            "dp4a_per_s": best(lambda it: sncc.probe_alu(sncc.PROBE_DP4A, sink, ctas, it // 4)),
            "imad_wide_per_s": best(lambda it: sncc.probe_alu(sncc.PROBE_IMAD_WIDE, sink, ctas, it // 4)),
            "hbm_write_gbs": max(wrates) / 1e9}


IMAD_WIDE_PER_CLK_SM = 32  # 16-lane integer multiplier per SM sub-partition, two passes per 64-bit product
# GB300's figures, replaced by the device's own at the first measurement
SM_COUNT, SM_MAX_MHZ = 152, 2070


def device_max_sm_mhz(gpu_index: int):
    """The maximum SM clock nvidia-smi reports for this GPU (None if it
    cannot be read)."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        return int(float(out.stdout.strip().splitlines()[0]))
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        return None


def set_sm_count(torch, dev):
    """The SM count and maximum SM clock of the device the bench runs on
    (for the nominal peaks)."""
    global SM_COUNT, SM_MAX_MHZ
    SM_COUNT = int(torch.cuda.get_device_properties(dev).multi_processor_count)
    mhz = device_max_sm_mhz(dev.index if dev.index is not None else 0)
    if mhz:
        SM_MAX_MHZ = mhz


def match_tile_rows(U, V):
    """Tile height the library picks for one match launch (largest R in
    {8, 4} giving at least two CTAs per SM, else 2)."""
    tu = -(-U // 32)
    for R in (8, 4):
        if tu * -(-V // (8 * R)) >= 2 * SM_COUNT:
            return R
    return 2


def segsum_roofline(kernel, corner_ops, ms, ceil, traffic=None, smem_words=None, **extra):
    """The segment-sum kernel against its ALU ceiling: one 32x32->64-bit
    multiply-add per (offset, corner), peak from unit counts and the maximum
    SM clock; the live probe and the shared-memory reads are reported beside it."""
    achieved = corner_ops / (ms * 1e-3) / 1e12
    peak = SM_COUNT * IMAD_WIDE_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    out = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "Tops/s",
           "frac": achieved / peak, "traffic": traffic, "ops_per_launch": corner_ops, "ms_per_launch": ms,
           "peak_source": "%d SMs x 32 IMAD.WIDE lane-ops/clk/SM x %d MHz (nominal)" % (SM_COUNT, SM_MAX_MHZ),
           "imad_wide_probe": {"peak": ceil["imad_wide_per_s"] / 1e12, "unit": "Tops/s",
                               "frac": achieved * 1e12 / ceil["imad_wide_per_s"],
                               "source": "measured: IMAD.WIDE instruction probe (all SMs), this run"}}
    if smem_words is not None:
        gbs = smem_words * 4 / (ms * 1e-3) / 1e9
        out["smem"] = {"words_per_launch": smem_words, "achieved": gbs, "peak": ceil["smem_gbs"], "unit": "GB/s",
                       "frac": gbs / ceil["smem_gbs"],
                       "source": "measured: shared-memory read probe (all SMs), this run"}
    out.update(extra)
    return out


def exact_roofline(macs, ms, ceil):
    """The exact comparator against the dp4a ceiling (4 pixel MACs each)."""
    achieved = macs / (ms * 1e-3) / 1e12
    peak = 4 * ceil["dp4a_per_s"] / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TMAC/s", "frac": achieved / peak,
            "peak_source": "measured: dp4a instruction probe (all SMs) x 4 MACs, this run"}


def run_gpu(args, world, rank, local, pg):
    import torch
    from paper_2502_01286_gb300 import build as lib_build
    if rank == 0 or not os.path.exists(lib_build.LIB):
        lib_build.build()
    barrier(pg)
    from paper_2502_01286_gb300 import sncc, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    set_sm_count(torch, dev)
    stream = torch.cuda.current_stream()
    band = None
    if args.shard == "bands" and world > 1:
        # one source for every rank: rank r runs the unchanged path on its
        # band of offset rows (source rows [v0, v1 + H - 1)); the only
        # exchange is the gather of the match lists after the timed region
        import dataclasses
        from paper_2502_01286_gb300 import shard
        case, SIGMAS, PRECISION = make_case(args.workload, 0)
        case_seed = case_seed_of(args.workload, 0)
        full_N, full_M = case.f.shape
        band = shard.bands(full_N, case.t.shape[0], world)[rank]
        if band.empty:
            raise SystemExit("more ranks than offset rows")
        full_case = case
        case = dataclasses.replace(case, f=np.ascontiguousarray(case.f[band.src_y0:band.src_y1]))
    else:
        case, SIGMAS, PRECISION = make_case(args.workload, rank)  # independent problem per rank
        case_seed = case_seed_of(args.workload, rank)
    N, M = case.f.shape
    H, W = case.t.shape
    U, V = M - W + 1, N - H + 1
    offsets_per_step = len(SIGMAS) * U * V

    # --- preparation (host template approximation, plans, buffers) ---
    t_prep = time.perf_counter()
    segs = [sncc.build_segments(case.t, s) for s in SIGMAS]
    prep_s = time.perf_counter() - t_prep
    fd = torch.as_tensor(case.f).to(dev)
    td = torch.as_tensor(case.t).to(dev)
    plans = [sncc.upload_plan(s, dev) for s in segs]
    tables = sncc.alloc_tables(M, N, sncc.match_bits(M, N, segs), dev)
    ws = sncc.integral_workspace(M, N, dev)
    cand_cap, out_cap = U * V, 1 << 16
    mbs = [sncc.alloc_match(M, N, W, H, cand_cap, True, dev) for _ in SIGMAS]
    rbs = [sncc.alloc_refine(M, N, W, H, out_cap, dev) for _ in SIGMAS]
    taus = [PRECISION * s.rho_max for s in segs]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    match_ev = []
    refine_ev = []
    # the thresholds' segment sums as one launch over (tile, threshold)
    # pairs where the library can fuse them (same template, one block each)
    fused = len(segs) > 1
    if fused:
        sncc.integral(fd, tables, workspace=ws)
        try:
            sncc.match_multi(segs, plans, tables, taus, mbs)
        except sncc.SnccError as e:
            if e.code != sncc.ERR_UNSUPPORTED:
                raise
            fused = False

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    sides = [torch.cuda.Stream(dev) for _ in segs[1:]]

    def step(record_match=False):
        sncc.integral(fd, tables, workspace=ws)
        if fused:
            a = ev() if record_match else None
            sncc.match_multi(segs, plans, tables, taus, mbs)
            prev = ev() if record_match else None
            if record_match:  # refines one after another, each timed
                match_ev.append((-1, a, prev))
                for i, s in enumerate(segs):
                    sncc.refine(fd, td, s, mbs[i], PRECISION, rbs[i])
                    c = ev()
                    refine_ev.append((i, prev, c))
                    prev = c
                return
            # the refines are independent: parallel branches of the graph
            main = torch.cuda.current_stream()
            for i, s in enumerate(segs):
                st = main if i == 0 else sides[i - 1]
                if i:
                    st.wait_stream(main)
                sncc.refine(fd, td, s, mbs[i], PRECISION, rbs[i], stream=st)
            for st in sides:
                main.wait_stream(st)
            return
        for i, s in enumerate(segs):
            a = ev() if record_match else None
            sncc.match(s, plans[i], tables, taus[i], mbs[i])
            b = ev() if record_match else None
            sncc.refine(fd, td, s, mbs[i], PRECISION, rbs[i])
            if record_match:
                c = ev()
                match_ev.append((i, a, b))
                refine_ev.append((i, b, c))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # the step as one CUDA graph (sum tables, then per threshold the segment
    # sum, the exact refine and its sort), replayed on the resident source
    graph = sncc.capture_graph(step)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(pg)
    torch.cuda.synchronize()
    clocks.mark_start()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        starts[k].record(stream)
        graph.replay()
        ends[k].record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    wall = time.perf_counter() - wall0
    clocks.mark_end()
    clk = clocks.stop()
    ms_steps = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    ms_per_step = max_over_ranks(pg, sum(ms_steps) / args.steps)
    status = [int(m.status.item()) for m in mbs]
    counts = [int(m.count.item()) for m in mbs]
    nmatch = [int(r.nout.item()) for r in rbs]

    # per-kernel time of the segment-sum launches: the same step launched
    # eagerly with events around each segment-sum launch (same stream)
    for k in range(max(3, min(args.steps, 50))):
        flush.fill_(k & 0xff)
        step(record_match=True)
    torch.cuda.synchronize()
    per_sigma_ms = {i: [] for i in range(-1, len(SIGMAS))}
    for i, a, b in match_ev:
        per_sigma_ms[i].append(a.elapsed_time(b))
    if fused:  # each threshold's segment sum launched on its own, for the per-threshold figures
        for k in range(max(3, min(args.steps, 50))):
            for i, s in enumerate(segs):
                flush.fill_(k & 0xff)
                a = ev()
                sncc.match(s, plans[i], tables, taus[i], mbs[i])
                b = ev()
                per_sigma_ms[i].append((a, b))
        torch.cuda.synchronize()
        for i in range(len(SIGMAS)):
            per_sigma_ms[i] = [a.elapsed_time(b) for a, b in per_sigma_ms[i]]
        step()  # leave the step's own outputs in the buffers
        torch.cuda.synchronize()
    refine_ms = {i: [] for i in range(len(SIGMAS))}
    for i, a, b in refine_ev:
        refine_ms[i].append(a.elapsed_time(b))

    # --- end to end through the public API: a stream of frames from pinned
    # host memory (StreamMatcher: the next frame's copy and the previous
    # frame's read-back overlap the current frame's matching) ---
    f_host = torch.as_tensor(case.f).pin_memory()
    e2e_steps = max(3, min(args.steps, 200))
    h2d = f_host.numel()
    sm = sncc.StreamMatcher(case.t, SIGMAS, M, N, precision=PRECISION, cand_cap=cand_cap, out_cap=out_cap,
                            keep_rho=True, device=dev)

    def e2e_frames(count):
        for k in range(count):
            with torch.cuda.stream(sm.compute):  # L2 flush before every frame, inside the timed region
                flush.fill_(k & 0xff)
            sm.submit(f_host)
        return sm.flush()

    e2e_frames(args.warmup)
    torch.cuda.synchronize()
    d2h0 = sm.d2h_bytes
    barrier(pg)
    t0 = time.perf_counter()
    last = e2e_frames(e2e_steps)
    t1 = time.perf_counter()
    e2e_ms_step = max_over_ranks(pg, 1e3 * (t1 - t0) / e2e_steps)
    d2h_total = sm.d2h_bytes - d2h0
    # the streamed lists are the step's own
    for (u, v, rho), rb in zip(last, rbs):
        if len(u) != min(int(rb.nout.item()), rb.cap):
            raise RuntimeError("streamed match list differs from the step's")
    e2e_status = sm.status()
    del sm

    # --- the same-GPU comparator: exact NCC map ---
    exact_rho = torch.empty((V, U), dtype=torch.float32, device=dev)
    for _ in range(3):
        sncc.exact_map(fd, td, segs[0].T, segs[0].T2, tables, exact_rho)
    ex_ms = []
    for k in range(10):
        flush.fill_(k)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sncc.exact_map(fd, td, segs[0].T, segs[0].T2, tables, exact_rho)
        b.record(stream)
        torch.cuda.synchronize()
        ex_ms.append(a.elapsed_time(b))
    exact_ms = statistics.median(ex_ms)
    max_dncc = [float((m.rho - exact_rho).abs().max().item()) for m in mbs]

    # --- sum tables alone: HBM roofline of the three sum-table kernels,
    # replayed from a graph as in the step ---
    sat_graph = sncc.capture_graph(lambda: sncc.integral(fd, tables, workspace=ws))
    sat_ms = []
    for k in range(20):
        flush.fill_(k)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sat_graph.replay()
        b.record(stream)
        torch.cuda.synchronize()
        sat_ms.append(a.elapsed_time(b))
    sat_med = statistics.median(sat_ms)
    # the same after a read pass over the flush buffer: the write flush leaves
    # up to an L2 of dirty lines, whose write-back otherwise lands inside the
    # next timed call; the read pass writes them back before the events
    sat_rd_ms = []
    for k in range(20):
        flush.fill_(k)
        flush.view(torch.int64).max()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sat_graph.replay()
        b.record(stream)
        torch.cuda.synchronize()
        sat_rd_ms.append(a.elapsed_time(b))
    sat_rd_med = statistics.median(sat_rd_ms)
    sat_bytes = M * N * (1 + tables.s_bits // 8 + 8)  # read f, write s and s2
    # context for the fraction: a device copy moving the same bytes (half
    # read, half written) after the same write flush; the measured copy peak
    # comes from far larger buffers
    cp_src = torch.ones(sat_bytes // 2, dtype=torch.uint8, device=dev)
    cp_dst = torch.empty_like(cp_src)
    cp_ms = []
    for k in range(20):
        flush.fill_(k)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        cp_dst.copy_(cp_src)
        b.record(stream)
        torch.cuda.synchronize()
        cp_ms.append(a.elapsed_time(b))
    copy_gbs = 2 * cp_src.numel() / (statistics.median(cp_ms) * 1e-3) / 1e9
    del cp_src, cp_dst
    peaks_hbm = measured_peaks().get("hbm_gbs")

    # --- the paper's own two-approximation search on the same source ---
    two = None
    try:
        pm = sncc.PaperMatcher(case.t, M, N, precision=PRECISION, cand_cap=U * V, device=dev)
        for _ in range(3):
            pm.run(fd)
        tw_ms = []
        for k in range(20):
            flush.fill_(k)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pm.run(fd)
            b.record(stream)
            torch.cuda.synchronize()
            tw_ms.append(a.elapsed_time(b))
        two = {"value": U * V / (statistics.median(tw_ms) * 1e-3) / 1e9, "unit": UNIT,
               "ms": statistics.median(tw_ms), "K_fast": pm.fast.K, "K_slow": pm.slow.K,
               "corners_fast": pm.fast.plan_info()["template_corners"],
               "corners_slow": pm.slow.plan_info()["template_corners"],
               "candidates": int(pm.mb.count.item()), "matches": int(pm.rb.nout.item()), "status": pm.status(),
               "max_abs_dncc_fast_vs_exact": float((pm.mb.rho - exact_rho).abs().max().item()),
               "what": "sum tables + coarse k_fast (0.99 sigma_t) at every offset + k_slow (0.1 sigma_t, "
                       "K_max 5000) on the tiles that hold candidates (Section 5 main algorithm)"}
    except sncc.SnccError as e:
        two = {"unavailable": str(e)}

    # --- on-chip ceilings of the segment-sum kernel and the comparator ---
    ceil = measure_ceilings(sncc, torch, stream, dev)

    # dominant kernel: the fused segment-sum launch, else the one with the
    # most corners
    infos = [s.plan_info() for s in segs]
    dom_set = list(range(len(SIGMAS))) if fused else \
        [max(range(len(SIGMAS)), key=lambda i: infos[i]["template_corners"])]
    dom = dom_set[0] if not fused else -1
    dom_ms = statistics.mean(per_sigma_ms[dom])
    # one multiply-add per (offset, corner)
    dom_ops = U * V * sum(infos[i]["template_corners"] for i in dom_set)
    Rt = match_tile_rows(U, V)
    # table words a lane reads per R offset rows: R per record (run, pair or
    # single corner) plus the rows each record spans beyond its first
    dom_words = U * V * sum(infos[i]["sum_records"] * Rt + infos[i]["sum_extra_rows"] for i in dom_set) / Rt
    dom_runs = {L: sum(infos[i]["runs%d" % L] for i in dom_set) for L in (8, 4, 2, 1)}
    dom_runs["pairs"] = sum(infos[i]["pairs"] for i in dom_set)

    value = sum_over_ranks(pg, offsets_per_step) / (ms_per_step * 1e-3) / 1e9
    e2e_value = sum_over_ranks(pg, offsets_per_step) / (e2e_ms_step * 1e-3) / 1e9
    band_info = None
    if band is not None:
        # the one exchange of the band split: every rank's match list, in the
        # full source's offsets, gathered on rank 0 (after the timed region)
        from paper_2502_01286_gb300 import shard
        U_full = full_M - W + 1
        per_sigma = []
        for i, rb in enumerate(rbs):
            u_, v_, rho_ = sncc.matches_to_numpy(rb)
            got = shard.gather_matches(shard.to_global(band, U_full, u_, v_), rho_)
            if rank == 0:
                per_sigma.append({"sigma_max": SIGMAS[i], "matches": int(got[0].size)})
        band_info = {"ranks": world, "rows": [band.v0, band.v1], "source_rows": [band.src_y0, band.src_y1],
                     "source": [full_M, full_N], "gathered": per_sigma,
                     "how": "rank r owns offset rows [v0, v1) and reads source rows [v0, v1 + H - 1); its own sum "
                            "tables give the same box sums; one gather of the match lists to rank 0"}

    cpu = None
    oracle_check = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rows = calibrate_rows(case, SIGMAS, args.cpu_seconds)
        offs, secs, threads, maps = oracle_sample(case, SIGMAS, rows, seed=7)
        cpu = {"value": offs / secs / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "%d random offset rows x %d offsets per threshold (of %d rows), thresholds %s; "
                         "sum tables + segmented NCC + candidates + exact refine" % (min(rows, V), U, V,
                                                                                  list(SIGMAS)),
               "seconds": secs}
        errs, nrows, sets = [], 0, {}
        for i, s in enumerate(SIGMAS):
            rws, rho, idx_o, rho_o = maps[s]
            g = mbs[i].rho[torch.as_tensor(rws, device=dev)].cpu().numpy().astype(np.float64)
            errs.append(float(np.abs(g - rho[rws]).max()))
            nrows += len(rws)
            n_c = min(counts[i], mbs[i].cand.numel())
            sets[str(s)] = sampled_set_check(case.f, case.t, rws, rho, idx_o, rho_o,
                                             mbs[i].cand[:n_c].cpu().numpy(), sncc.matches_to_numpy(rbs[i]),
                                             U, taus[i], PRECISION)
        oracle_check = {"max_abs_drho_vs_oracle": max(errs), "offset_rows_checked": nrows,
                        "offsets_checked": nrows * U, "tolerance": TOL,
                        "candidate_and_match_sets": sets,
                        "g13_band_offsets": sum(v["g13_band_offsets"] for v in sets.values()),
                        "g13_violations": sum(v["g13_violations"] for v in sets.values())}

    peaks = measured_peaks()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "strong" if band is not None else "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": workload_config(args.workload, case, SIGMAS, PRECISION, U, V, case_seed) if band is None else
                  workload_config(args.workload, full_case, SIGMAS, PRECISION, full_M - W + 1, full_N - H + 1,
                                  case_seed),
        "launch": ("one CUDA graph per step: sum tables, one segment-sum launch over every (tile, threshold) "
                   "pair, then per threshold exact refine and sort (parallel branches)") if fused else
                  "one CUDA graph per step: sum tables, then per threshold segment sum, exact refine and sort",
        "exact_ncc": {"value": U * V / (exact_ms * 1e-3) / 1e9, "unit": UNIT, "ms": exact_ms,
                      "kernel": "direct integer correlation, dp4a (4 byte MACs per instruction)",
                      "roofline": exact_roofline(U * V * W * H, exact_ms, ceil)},
        "speedup_vs_exact": value / (U * V / (exact_ms * 1e-3) / 1e9),
        "max_abs_dncc_vs_exact": dict(zip([str(s) for s in SIGMAS], max_dncc)),
        "per_sigma": [{"sigma_max": s, "K": seg.K, "corners": infos[i]["template_corners"],
                       "block_corners": infos[i]["corners"] if infos[i]["blocks"] == 1
                       else infos[i]["wide_corners"], "rho_max": seg.rho_max,
                       "tau_c": taus[i], "match_ms": statistics.mean(per_sigma_ms[i]),
                       "refine_ms": statistics.mean(refine_ms[i]),
                       "candidates": counts[i], "matches": nmatch[i], "status": status[i],
                       "goffsets_s_coarse": U * V / (statistics.mean(per_sigma_ms[i]) * 1e-3) / 1e9}
                      for i, (s, seg) in enumerate(zip(SIGMAS, segs))],
        "prep_s": prep_s,
        "sum_tables": {"ms": sat_med, "algorithmic_bytes": sat_bytes,
                       "achieved_gbs": sat_bytes / (sat_med * 1e-3) / 1e9,
                       "frac_of_hbm": (sat_bytes / (sat_med * 1e-3) / 1e9) / peaks_hbm if peaks_hbm else None,
                       "peak": "MEASURED_PEAKS hbm_gbs",
                       # the tables are almost all 16-byte stores: also against the write rate of such stores
                       "write_probe_gbs": ceil["hbm_write_gbs"],
                       "frac_of_write_probe": (sat_bytes / (sat_med * 1e-3) / 1e9) / ceil["hbm_write_gbs"],
                       "write_probe_source": "measured: 16-byte store probe over 1 GiB (all SMs), this run",
                       "size_matched_copy": {"gbs": copy_gbs,
                                             "frac": (sat_bytes / (sat_med * 1e-3) / 1e9) / copy_gbs,
                                             "how": "device copy of the same bytes (half read, half written) "
                                                    "after the same write flush, this run"},
                       "clean_l2": {"ms": sat_rd_med,
                                    "frac_of_hbm": (sat_bytes / (sat_rd_med * 1e-3) / 1e9) / peaks_hbm
                                    if peaks_hbm else None,
                                    "how": "the same write flush, then a read pass over the 256 MiB flush buffer "
                                           "(its dirty lines written back before the timed call)"}},
        "paper_two_stage": two,
        "roofline": segsum_roofline("match_kernel" + (" (fused over %d thresholds)" % len(SIGMAS) if fused else ""),
                                    dom_ops, dom_ms, ceil, traffic=recorded_traffic(args.workload),
                                    smem_words=dom_words, sigma_max=[SIGMAS[i] for i in dom_set], tile_rows=Rt,
                                    runs=dom_runs, hbm_peak_gbs=peaks.get("hbm_gbs")),
        "coarse_fused": {"ms": dom_ms, "separate_ms": sum(statistics.mean(per_sigma_ms[i]) for i in dom_set),
                         "goffsets_s": len(SIGMAS) * U * V / (dom_ms * 1e-3) / 1e9} if fused else None,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h_total / e2e_steps, "ms_per_step": e2e_ms_step, "status": e2e_status,
                "how": "StreamMatcher over %d frames: per frame an L2 flush and the frame's graph on the compute "
                       "stream, the host-to-device copy on a copy stream, the previous frame's match lists read "
                       "back on a third stream; wall clock from the first submit to the last list" % e2e_steps},
        "gpu_launches": args.steps * (sncc.INTEGRAL_KERNELS + (1 if fused else len(SIGMAS)) +
                                      sncc.REFINE_KERNELS * len(SIGMAS)),
        "clocks": clk, "wall_s_timed": wall,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if oracle_check is not None:
        line["oracle_check"] = oracle_check
    if band_info is not None:
        line["shard"] = band_info
    if rank == 0:
        print(json.dumps(line), flush=True)


def batch_config(srcs, tl):
    """The batch workload as both arms describe it (the same dict in each)."""
    N, M = srcs[0].shape
    offsets = len(srcs) * sum((M - t.shape[1] + 1) * (N - t.shape[0] + 1) for t, _, _ in tl)
    return {"workload": "batch-8x1024x1024-64templates-16to256-sigma4to25", "sources": [len(srcs), M, N],
            "templates": len(tl), "pairs": len(srcs) * len(tl), "offsets_per_step": offsets,
            "precision": PRECISION, "l2": "flushed between steps (256 MiB write)"}


def batch_problem(rank: int = 0):
    """8 sources of 1024 x 1024 (blobs + 1/f noise) and 64 templates with
    sides U{16..256} and std thresholds U(4, 25): all 512 pairs."""
    from paper_2502_01286_gb300 import synth
    srcs = synth.batch_sources(seed=synth.BASE_SEED + 3 + 1000 * rank)
    tl = synth.batch_templates(srcs, seed=synth.BASE_SEED + 4 + 1000 * rank)
    return srcs, tl


def batch_oracle_sample(srcs, tl, rows_per_pair: int, pairs, seed=0):
    """The oracle on `rows_per_pair` random offset rows of each listed pair
    (sum tables + segmented NCC + candidates + exact refine)."""
    import oracle as O
    rng = np.random.default_rng(seed)
    total, secs = 0, 0.0
    for (si, ti) in pairs:
        f = srcs[si]
        t, _, sg = tl[ti]
        H, W = t.shape
        U, V = f.shape[1] - W + 1, f.shape[0] - H + 1
        ap = O.precompute_template_approximation(t, sg)
        rows = np.sort(rng.choice(V, size=min(rows_per_pair, V), replace=False))
        t0 = time.perf_counter()
        rho = O.segmented_ncc_map(f, ap, "sat", rows=rows)
        cand = O.candidates(rho, PRECISION * ap.rho_max)
        O.refine(f, t, cand, U, PRECISION)
        secs += time.perf_counter() - t0
        total += len(rows) * U
    return total, secs, O.default_threads()


def run_gpu_batch(args, world, rank, local, pg):
    import torch
    from paper_2502_01286_gb300 import build as lib_build
    if rank == 0 or not os.path.exists(lib_build.LIB):
        lib_build.build()
    barrier(pg)
    from paper_2502_01286_gb300 import sncc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    set_sm_count(torch, dev)
    stream = torch.cuda.current_stream()
    srcs, tl = batch_problem(rank)
    N, M = srcs[0].shape
    t_prep = time.perf_counter()
    b = sncc.Batch([t for t, _, _ in tl], [sg for _, _, sg in tl], M, N, len(srcs), precision=PRECISION,
                   cand_cap=1 << 22, out_cap=1 << 18, device=dev)
    prep_s = time.perf_counter() - t_prep
    info = b.info()
    fd = [torch.as_tensor(f).to(dev) for f in srcs]
    t_tune = time.perf_counter()
    tune = b.autotune(fd, reps=2)
    tune_s = time.perf_counter() - t_tune
    buckets = [{"bucket": bb["bucket"], "size_class": bb["size_class"], "density_class": bb["density_class"],
                "templates": bb["templates"], "pairs": bb["pairs"], "tile_rows": bb["tile_rows"],
                "block": bb["block"],
                "ms_per_variant": {"R%d-b%d" % key: ms for key, ms in tune.get(bb["bucket"], {}).items()}}
               for bb in b.buckets() if bb["pairs"]]
    g = b.capture(fd)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(pg)
    torch.cuda.synchronize()
    clocks.mark_start()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        starts[k].record(stream)
        g.replay()
        ends[k].record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    wall = time.perf_counter() - wall0
    clocks.mark_end()
    clk = clocks.stop()
    ms_per_step = max_over_ranks(pg, sum(a.elapsed_time(e) for a, e in zip(starts, ends)) / args.steps)
    status = int(b.status.item())
    ncand, nmatch = int(b.count.item()), int(b.nout.item())

    # the persistent coarse launch alone (dominant kernel)
    mk = []
    for k in range(5):
        flush.fill_(k)
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sncc._check(sncc._lib.sncc_batch_match(*b._match_args(), sncc._stream(None)), "sncc_batch_match")
        e.record(stream)
        torch.cuda.synchronize()
        mk.append(a.elapsed_time(e))
    match_ms = statistics.median(mk)
    ceil = measure_ceilings(sncc, torch, stream, dev)

    # end to end: sources from pinned host memory, graph replay, matches back
    host = [torch.as_tensor(f).pin_memory() for f in srcs]
    e2e_ms, d2h = [], 0
    e2e_steps = max(3, min(args.steps, 20))
    for k in range(args.warmup + e2e_steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d_, h_ in zip(fd, host):
            d_.copy_(h_, non_blocking=True)
        g.replay()
        n = min(int(b.nout.item()), b.out_cap)
        if n:
            b.out[:n].cpu()
        t1 = time.perf_counter()
        if k >= args.warmup:
            e2e_ms.append(1e3 * (t1 - t0))
            d2h += 4 + 16 * n
    e2e_ms_step = max_over_ranks(pg, statistics.mean(e2e_ms))

    # exact NCC of every pair on the same GPU (the comparator), timed once
    tb = b.tables
    rho_buf = torch.empty(M * N, dtype=torch.float32, device=dev)
    segs = b.segs
    t_devs = [torch.as_tensor(t).to(dev) for t, _, _ in tl]
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    exact_macs = 0
    for si in range(len(srcs)):
        for ti, (t, _, _) in enumerate(tl):
            H, W = t.shape
            exact_macs += (N - H + 1) * (M - W + 1) * H * W
            out = rho_buf[:(N - H + 1) * (M - W + 1)].view(N - H + 1, M - W + 1)
            sncc.exact_map(fd[si], t_devs[ti], segs[ti].T, segs[ti].T2, tb[si], out)
    e.record(stream)
    torch.cuda.synchronize()
    exact_ms = a.elapsed_time(e)

    offsets = sum_over_ranks(pg, info["offsets"])
    value = offsets / (ms_per_step * 1e-3) / 1e9
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rng = np.random.default_rng(5)
        pairs = [(int(rng.integers(0, len(srcs))), int(rng.integers(0, len(tl)))) for _ in range(8)]
        import oracle as O
        T = O.default_threads()
        _, s1, _ = batch_oracle_sample(srcs, tl, T, pairs, seed=1)  # one round of rows per host thread
        rows = max(1, int(T * args.cpu_seconds / max(s1, 1e-3)))
        o, secs, threads = batch_oracle_sample(srcs, tl, rows, pairs, seed=2)
        cpu = {"value": o / secs / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "up to %d random offset rows of each of 8 random (source, template) pairs" % rows,
               "seconds": secs}
    peaks = measured_peaks()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic",
        "config": batch_config(srcs, tl),
        "launch": {"graph": "sum tables x8, one persistent coarse launch per variant in use, refine, sort",
                   "buckets": buckets, "autotune_s": tune_s,
                   "autotune": "per template bucket (size class x corner density class), the fastest of tile "
                               "height R in {8, 4, 2} x template block edge {64, 32}, each bucket timed alone"},
        "exact_ncc": {"value": info["offsets"] / (exact_ms * 1e-3) / 1e9, "unit": UNIT, "ms": exact_ms,
                      "kernel": "direct integer correlation, dp4a (4 byte MACs per instruction), one launch "
                                "per pair", "roofline": exact_roofline(exact_macs, exact_ms, ceil)},
        "speedup_vs_exact": value / (info["offsets"] / (exact_ms * 1e-3) / 1e9),
        "candidates": ncand, "matches": nmatch, "status": status, "prep_s": prep_s,
        "roofline": segsum_roofline("batch_match_kernel", info["corner_offsets"], match_ms, ceil,
                                    hbm_peak_gbs=peaks.get("hbm_gbs")),
        "e2e": {"value": offsets / (e2e_ms_step * 1e-3) / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": sum(f.size for f in srcs), "d2h_bytes_per_step": d2h / e2e_steps,
                "ms_per_step": e2e_ms_step},
        "gpu_launches": args.steps * (sncc.INTEGRAL_KERNELS * len(srcs) + len({(x["tile_rows"], x["block"])
                                                                                for x in buckets}) +
                                      sncc.REFINE_KERNELS),
        "clocks": clk, "wall_s_timed": wall,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)


CROSSOVER_SIGMAS = (2.75, 3.0, 3.25, 3.5, 3.75, 4.0, 4.25, 4.5, 5.0, 6.0, 8.0, 12.0, 20.0, 40.0)


def run_gpu_crossover(args, world, rank, local, pg):
    """Where segmented NCC stops beating exact NCC on this GPU: the 4096^2 /
    256^2 texture workload at std thresholds from 2.75 to 40, so that the
    approximation's corners per template pixel, P / (W H), run from about 0.4
    down to 0.01.  At each threshold: the whole path (sum tables, coarse
    pass, exact refine, one graph per step) timed with CUDA events after an
    L2 flush, the same-GPU exact comparator, and max |rho_seg - rho_exact|
    over every offset (the accuracy the speedup is bought with)."""
    import torch
    from paper_2502_01286_gb300 import build as lib_build
    if rank == 0 or not os.path.exists(lib_build.LIB):
        lib_build.build()
    barrier(pg)
    from paper_2502_01286_gb300 import sncc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    set_sm_count(torch, dev)
    stream = torch.cuda.current_stream()
    case, _, precision = make_case("texture", rank)
    N, M = case.f.shape
    H, W = case.t.shape
    U, V = M - W + 1, N - H + 1
    fd = torch.as_tensor(case.f).to(dev)
    td = torch.as_tensor(case.t).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    tables = sncc.alloc_tables(M, N, sncc.match_bits(M, N), dev)
    ws = sncc.integral_workspace(M, N, dev)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        out = []
        for k in range(reps):
            flush.fill_(k & 0xff)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            out.append(a.elapsed_time(b))
        return statistics.median(out)

    sncc.integral(fd, tables, workspace=ws)
    exact_rho = torch.empty((V, U), dtype=torch.float32, device=dev)
    seg0 = sncc.build_segments(case.t, 5.0)
    exact_ms = timed(lambda: sncc.exact_map(fd, td, seg0.T, seg0.T2, tables, exact_rho), 10)
    exact_value = U * V / (exact_ms * 1e-3) / 1e9
    clocks = ClockSampler(local)
    clocks.mark_start()
    sweep = []
    for sigma in CROSSOVER_SIGMAS:
        t0 = time.perf_counter()
        seg = sncc.build_segments(case.t, sigma)
        prep_s = time.perf_counter() - t0
        if not seg.Ek > 0:
            continue
        pi = seg.plan_info()
        plan = sncc.upload_plan(seg, dev)
        mb = sncc.alloc_match(M, N, W, H, U * V, True, dev)
        rb = sncc.alloc_refine(M, N, W, H, 1 << 16, dev)
        tau = precision * seg.rho_max

        def step():
            sncc.integral(fd, tables, workspace=ws)
            sncc.match(seg, plan, tables, tau, mb)
            sncc.refine(fd, td, seg, mb, precision, rb)

        g = sncc.capture_graph(step)
        reps = 5
        step_ms = timed(g.replay, reps)
        match_ms = timed(lambda: sncc.match(seg, plan, tables, tau, mb), reps)
        g.replay()
        torch.cuda.synchronize()
        value = U * V / (step_ms * 1e-3) / 1e9
        sweep.append({"sigma_max": sigma, "K": seg.K, "corners": pi["template_corners"],
                      "corners_per_pixel": pi["template_corners"] / float(W * H), "prep_s": prep_s,
                      "step_ms": step_ms, "match_ms": match_ms, "value": value,
                      "speedup_vs_exact": value / exact_value,
                      "max_abs_dncc_vs_exact": float((mb.rho - exact_rho).abs().max().item()),
                      "candidates": int(mb.count.item()), "matches": int(rb.nout.item()),
                      "status": int(mb.status.item())})
        del g, mb, rb, plan
    clocks.mark_end()
    clk = clocks.stop()
    # the crossover: where the speedup falls through 1, interpolated in
    # log(corners per pixel) between the two bracketing thresholds
    cross = None
    pts = sorted(sweep, key=lambda e: e["corners_per_pixel"])
    for lo, hi in zip(pts, pts[1:]):
        if lo["speedup_vs_exact"] >= 1.0 > hi["speedup_vs_exact"]:
            import math
            t = (math.log(lo["speedup_vs_exact"])) / (math.log(lo["speedup_vs_exact"]) - math.log(hi["speedup_vs_exact"]))
            cpp = math.exp(math.log(lo["corners_per_pixel"]) +
                           t * (math.log(hi["corners_per_pixel"]) - math.log(lo["corners_per_pixel"])))
            cross = {"corners_per_pixel": cpp, "corners": cpp * W * H,
                     "between_sigma": [lo["sigma_max"], hi["sigma_max"]], "between_K": [lo["K"], hi["K"]],
                     "how": "speedup interpolated linearly in log(speedup) against log(P / (W H))"}
    ref = next((e for e in sweep if e["sigma_max"] == 5.0), sweep[0])
    line = {"metric": METRIC, "value": ref["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ref["step_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "crossover-texture-4096x4096-t256x256-sigma%g-%g" % (CROSSOVER_SIGMAS[0],
                                                                                         CROSSOVER_SIGMAS[-1]),
                       "precision": precision, "l2": "flushed before every timed call (256 MiB write)",
                       "value_is": "the sigma 5 point of the sweep"},
            "exact_ncc": {"value": exact_value, "unit": UNIT, "ms": exact_ms,
                          "kernel": "direct integer correlation, dp4a (4 byte MACs per instruction)"},
            "sweep": sweep, "crossover": cross, "clocks": clk,
            "gpu_launches": args.steps * (sncc.INTEGRAL_KERNELS + 1 + sncc.REFINE_KERNELS)}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_gpu_diff(args, world, rank, local, pg):
    """Differentiation workload: loss between segmented and exact NCC over a
    512 x 512 float source (48 x 48 template, segmentation at std 12), one
    step = forward + hand-written backward w.r.t. segment values and source."""
    import torch
    from paper_2502_01286_gb300 import build as lib_build
    if rank == 0 or not os.path.exists(lib_build.LIB):
        lib_build.build()
    barrier(pg)
    from paper_2502_01286_gb300 import sncc, synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    set_sm_count(torch, dev)
    stream = torch.cuda.current_stream()
    f, t, org, sigma = synth.case_diff(seed=synth.BASE_SEED + 5 + 1000 * rank)
    N, M = f.shape
    seg = sncc.build_segments(np.rint(np.clip(t, 0, 255)).astype(np.uint8), sigma)
    rects = seg.table
    k0 = np.array([t[y:y + h, x:x + w].mean() for x, y, w, h in rects], np.float32)
    pb = sncc.DiffProblem(t, rects, M, N, device=dev)
    fd = torch.as_tensor(f).to(dev).requires_grad_(True)
    kd = torch.as_tensor(k0).to(dev).requires_grad_(True)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        fd.grad = None
        kd.grad = None
        loss = pb.loss(fd, kd)
        loss.backward()
        return loss

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier(pg)
    torch.cuda.synchronize()
    clocks.mark_start()
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    clocks.mark_end()
    barrier(pg)
    clk = clocks.stop()
    ms = max_over_ranks(pg, sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / args.steps)
    U, V = pb.U, pb.V
    H, W = t.shape

    # end to end: the source from pinned host memory every step, loss and dL/dk read back
    host_f = torch.as_tensor(f).pin_memory()
    e2e_ms = []
    for k in range(max(3, min(args.steps, 20))):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fe = host_f.to(dev, non_blocking=True).requires_grad_(True)
        ke = kd.detach().clone().requires_grad_(True)
        loss = pb.loss(fe, ke)
        loss.backward()
        out_loss = loss.detach().to("cpu", non_blocking=True)
        out_dk = ke.grad.to("cpu", non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e_ms_step = max_over_ranks(pg, statistics.mean(e2e_ms))

    # the backward call alone (coefficients, dL/df, template-space correlation, dL/dk)
    fdet, kdet = fd.detach(), kd.detach().contiguous()
    rho_k, rho_t, _ = sncc._diff_forward(pb, fdet, kdet)
    dl = torch.ones(1, dtype=torch.float64, device=dev)
    gf = torch.empty((N, M), dtype=torch.float32, device=dev)
    gk = torch.empty(pb.K, dtype=torch.float32, device=dev)

    def backward_call():
        sncc._check(sncc._lib.sncc_diff_backward(fdet.data_ptr(), M, N, fdet.stride(0), W, H, pb.rects.data_ptr(),
                                                 kdet.data_ptr(), pb.K, rho_k.data_ptr(), rho_t.data_ptr(),
                                                 dl.data_ptr(), gf.data_ptr(), M, gk.data_ptr(), pb.ws_ptr,
                                                 pb.ws_bytes, sncc._stream(None)), "sncc_diff_backward")

    def forward_call():
        sncc._diff_forward(pb, fdet, kdet)

    def timed(fn, reps=20):
        fn()
        torch.cuda.synchronize()
        out = []
        for k in range(reps):
            flush.fill_(k & 0xff)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            out.append(a.elapsed_time(b))
        return statistics.median(out)

    bwd_ms = timed(backward_call)
    fwd_ms = timed(forward_call)
    pairs = U * V * W * H
    # algorithmic work of the backward call: per (offset, template pixel) two
    # FP32 multiply-adds of dL/df (a c and b t0) and one of Gt (a f)
    bwd_flops = 2 * 3 * pairs
    bwd_tflops = bwd_flops / (bwd_ms * 1e-3) / 1e12
    fp32_peak = SM_COUNT * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12  # 128 FP32 FMA lanes per SM

    _, losses = sncc.refit_segment_values(pb, fd.detach(), k0, steps=50, lr=0.5)
    value = sum_over_ranks(pg, U * V) / (ms * 1e-3) / 1e9

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import diff as OD
        rects_np = np.asarray(rects)

        def sample(rows):
            sub = f[:rows + H - 1]
            t0_ = time.perf_counter()
            OD.gradients(sub, t, rects_np, k0)
            return time.perf_counter() - t0_

        s1 = sample(4)
        rows = int(max(4, min(V, 4 * args.cpu_seconds / max(s1, 1e-3))))
        secs = sample(rows)
        cpu = {"value": rows * U / secs / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "loss and both gradients (FP64 numpy, one thread) over the first %d of %d offset rows"
                         % (rows, V), "seconds": secs}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": diff_config(seg),
            "step": "loss forward + backward w.r.t. segment values and source (kernel launches: forward 2: prep, "
                    "forward; backward 6: coefficients, row sums, dL/df, Gt, Gt reduce, dL/dk)",
            "forward_call_ms": fwd_ms, "backward_call_ms": bwd_ms,
            "roofline": {"bound": "alu", "kernel": "sncc_diff_backward (diff_coeff, diff_rowbox, diff_grad_f, diff_gt, "
                                                    "diff_gt_reduce, diff_grad_k)",
                         "achieved": bwd_tflops, "peak": fp32_peak, "unit": "TFLOP/s", "frac": bwd_tflops / fp32_peak,
                         "traffic": None, "flops_per_launch": bwd_flops, "ms_per_launch": bwd_ms,
                         "peak_source": "%d SMs x 128 FP32 FMA lanes x 2 x %d MHz (nominal)" % (SM_COUNT,
                                                                                                 SM_MAX_MHZ)},
            "e2e": {"value": sum_over_ranks(pg, U * V) / (e2e_ms_step * 1e-3) / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": M * N * 4, "d2h_bytes_per_step": 8 + 4 * pb.K, "ms_per_step": e2e_ms_step},
            "refit": {"steps": 50, "loss_first": losses[0], "loss_last": losses[-1]},
            "gpu_launches": args.steps * 8, "clocks": clk}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank, pg)
    elif args.workload == "diff":
        run_gpu_diff(args, world, rank, local, pg)
    elif args.workload == "crossover":
        run_gpu_crossover(args, world, rank, local, pg)
    elif args.workload == "batch":
        run_gpu_batch(args, world, rank, local, pg)
    else:
        run_gpu(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
