#!/usr/bin/env python3
"""Throughput of the lambda(omega)-mapped triangular kernels on one GB300.

Default workload: the high-dimensional EDM, N = 65536 points of d = 128 FP32
features drawn N(0,1) with 1% duplicated rows, every pair i >= j written to a
packed lower triangle (2,147,516,416 distances, 8.59 GB).  A step is one full
tri_edm call over that input (all kernels of the chosen precision path); the
metric is pairs per second.  Beside it the line carries the bounding-box map
on the same input and GPU (the paper's improvement factor I = t_BB / t_lambda),
the FP32 and tensor-core arms, the roofline of the dominant kernel, an
end-to-end figure through host buffers, and the CPU oracle timed on a bounded
sample on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--prec fp32|bf16x3|bf16x6] [--split] [--suite]

With N > 1 (torchrun), every rank runs its own full instance of the workload
(weak scaling, no collective on the data path); rank 0 prints the line.  With
--split the ranks share one triangle instead, each computing a band of rows
of equal pair count (strong scaling).  --suite prints one line per other
hot-path row (maps, FP32 EDM, Life, Axilrod-Teller, collisions, batched EDM).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_PTS, D_FEAT, DUP = 65536, 128, 0.01
WORKLOAD = "edm_n65536_d128_normal_dup1pct"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
NUM_SMS = 152
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) of one Gram-kernel launch, from the ncu capture
# summarised in profiles/gram_kernel_lambda_bf16x6_n65536_d128.md (taken at
# N = 16384 and scaled by the number of pairs).  Keyed by (prec, n, d); a
# kernel change makes the figure stale, and it is then removed.
NCU_TRAFFIC = {("bf16x6", 65536, 128): 7.912e9}


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except (OSError, ValueError):
        return dict(FALLBACK), "fallback"


def host_cores() -> int:
    return len(os.sched_getaffinity(0))


# ----------------------------------------------------------- clocks --------
class ClockSampler:
    """nvidia-smi samples (every 20 ms, with timestamps) around the timed
    region; the summary keeps the samples that fall inside it (mark_begin /
    mark_end), and says how many there were."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 20
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.begin = self.end = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.INTERVAL_MS)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def mark_begin(self):
        self.begin = _now()

    def mark_end(self):
        self.end = _now()

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        try:
            with open(self.path) as f:
                lines = f.readlines()
        except OSError:
            lines = []
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        return self.summarize(lines, self.begin, self.end)

    @classmethod
    def summarize(cls, lines, begin=None, end=None):
        """Median SM clock, maximum clock and active throttle reasons of the
        samples within [begin, end] (widened by one interval on each side),
        or of all samples when none fall inside."""
        import datetime
        rows = []
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                sm, smax = float(f[2]), float(f[3])
            except ValueError:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f")
            except ValueError:
                ts = None  # an unexpected timestamp format: the sample counts only in the overall summary
            rs = {nm for nm, v in zip(cls.REASONS, f[6:10]) if v.lower() in ("active", "1", "yes")}
            rows.append((ts, sm, smax, rs))
        inside = rows
        if begin is not None and end is not None:
            pad = datetime.timedelta(milliseconds=cls.INTERVAL_MS)
            inside = [r for r in rows if r[0] is not None and begin - pad <= r[0] <= end + pad]
        use = inside if inside else rows
        return {"sm_mhz": statistics.median(r[1] for r in use) if use else None,
                "sm_max_mhz": max(r[2] for r in use) if use else None,
                "reasons": sorted(set().union(*[r[3] for r in use])) if use else [],
                "samples": len(rows), "samples_in_timed_region": len(inside),
                "interval_ms": cls.INTERVAL_MS}


def _now():
    import datetime
    return datetime.datetime.now()


# ------------------------------------------------------ reference arm -------
def cpu_oracle_sample(x: np.ndarray, target_s: float = 12.0, with_time: bool = False):
    """Time the CPU oracle on a band of full rows at the end of the triangle.

    Returns (pairs/s, threads, sample description[, seconds of the timed band])."""
    import oracle
    n = x.shape[0]
    probe = 64
    t0 = time.perf_counter()
    oracle.edm_rows(x, n - probe, n)
    dt = time.perf_counter() - t0
    pairs_probe = (n * (n + 1) - (n - probe) * (n - probe + 1)) // 2
    rate = pairs_probe / max(dt, 1e-9)
    rows = int(max(probe, min(n, target_s * rate / n)))
    r0 = n - rows
    t0 = time.perf_counter()
    oracle.edm_rows(x, r0, n)
    dt = time.perf_counter() - t0
    pairs = (n * (n + 1) - r0 * (r0 + 1)) // 2
    desc = f"rows [{r0}, {n}) of the triangle: {pairs} pairs in {dt:.2f} s"
    if with_time:
        return pairs / dt, oracle.threads(), desc, dt
    return pairs / dt, oracle.threads(), desc


def headline_config(prec: str) -> dict:
    """The workload the headline line (and the reference arm beside it) runs."""
    P = N_PTS * (N_PTS + 1) // 2
    return {"workload": WORKLOAD, "n": N_PTS, "d": D_FEAT, "dup_frac": DUP, "map": "lambda",
            "tile": (("16x16 threads x 8x8 pairs" if D_FEAT >= 32 else "16x16 threads x 4x4 pairs")
                     if prec == "fp32"
                     else "2x2 blocks of 128x128 tiles per CTA pair (tcgen05.mma.cta_group::2, M=N=256)"),
            "prec": prec, "pairs_per_step": P,
            "l2": (f"each step writes the {4 * P / 1e9:.2f} GB triangle (> 129 MB L2), which flushes L2 "
                   "between steps" if 4 * P > 129e6 else
                   f"the {4 * P / 1e6:.1f} MB triangle fits in L2: no flush between steps")}


def max_over_ranks(values, world: int, device=None):
    """Each timing's maximum over the ranks: in a replica run the slowest rank
    bounds the job.  Collective over the default process group when world > 1."""
    values = [float(v) for v in values]
    if world <= 1:
        return values
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_rate(world: int, units_per_rank: float, ms_per_step: float) -> float:
    """Whole-job throughput: the units every rank processed in one step over
    the slowest rank's step time."""
    return world * units_per_rank / (ms_per_step * 1e-3)


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    from paper_1609_01490_gb300 import inputs
    x = inputs.edm_normal_points(N_PTS, D_FEAT, seed=1609, dup_frac=DUP)
    total_pairs = N_PTS * (N_PTS + 1) // 2
    vals, secs = [], []
    for s in range(args.warmup + args.steps):
        rate, thr, sample, dt = cpu_oracle_sample(x, target_s=4.0, with_time=True)
        if s >= args.warmup:
            vals.append(rate)
            secs.append(dt)
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": "pairs/s", "value": value, "unit": "pairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        # each step is one bounded band of rows, timed as run (not the whole triangle)
        "ms_per_step": 1e3 * statistics.median(secs),
        "ms_per_step_note": "wall time of one step's band of rows; the whole triangle would take "
                            f"{1e3 * total_pairs / value:.0f} ms at this rate",
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": headline_config("bf16x6"),
        "impl_note": "CPU oracle (FP64 direct differences), each step a bounded band of rows",
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": thr, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def graph_time_ms(fn, reps, stream):
    """Mean ms of fn, captured `reps` times into one CUDA graph, best of 3 replays
    timed with CUDA events on `stream`."""
    import torch
    fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s2 = torch.cuda.Stream()
    s2.wait_stream(stream)
    with torch.cuda.stream(s2):
        fn()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s2):
            for _ in range(reps):
                fn()
    stream.wait_stream(s2)
    g.replay()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.replay()
        b.record(stream)
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b) / reps)
    return best


def paper_comparison(tri, inputs, dev, stream):
    """The other workloads beside the headline, each timed on this GPU as the
    mean of launches captured in one CUDA graph: the paper's own comparison
    (Section 5) of lambda, the bounding box and the rectangular box on the
    paper-size EDM (N = 2048, d = 3, one pair per thread, rho = 16, as the
    paper launches it) and on one triangular Life step (n = 16384, rho = 32);
    the Life workload's 100 steps through tri_ca_run; the Axilrod-Teller energy under the tetrahedral maps; and the 1000-instance
    batched EDM against separate launches.  I = t_BB / t_map."""
    import torch
    out = {}
    x = torch.from_numpy(inputs.edm_uniform_points(2048, 3, seed=1609)).to(dev)
    o = torch.empty(2048 * 2049 // 2, dtype=torch.float32, device=dev)
    t = {nm: graph_time_ms(lambda: tri.tri_edm(x, o, map=m, rho=16, reg=1), 200, stream)
         for nm, m in (("lambda", tri.MAP_LAMBDA), ("bb", tri.MAP_BB), ("rb", tri.MAP_RB))}
    out["edm_n2048_d3_rho16_reg1"] = {"ms": t, "I_bb_over": {k: t["bb"] / v for k, v in t.items()}}
    n = 16384
    a = torch.from_numpy(inputs.ca_grid(n, seed=1609)).to(dev)
    b = torch.zeros_like(a)

    def life(m):
        def run():
            for k in range(10):
                src, dst = (a, b) if k % 2 == 0 else (b, a)
                tri.tri_ca_step(src, dst, n, map=m, rho=32)
        return run
    t = {nm: graph_time_ms(life(m), 1, stream) / 10
         for nm, m in (("lambda", tri.MAP_LAMBDA), ("bb", tri.MAP_BB), ("rb", tri.MAP_RB))}
    out["life_n16384_step_rho32"] = {"ms": t, "I_bb_over": {k: t["bb"] / v for k, v in t.items()}}
    # the Life workload as configured, 100 steps, through tri_ca_run (up to 16
    # steps per pass through memory)
    c = torch.zeros_like(a)
    t = {nm: graph_time_ms(lambda: tri.tri_ca_run(a, b, n, 100, scratch=c, map=m, rho=32), 1, stream)
         for nm, m in (("lambda", tri.MAP_LAMBDA), ("bb", tri.MAP_BB), ("rb", tri.MAP_RB))}
    out["life_n16384_100steps_run"] = {"ms": t, "I_bb_over": {k: t["bb"] / v for k, v in t.items()},
                                       "cell_updates_per_s": 100 * (n * (n + 1) // 2) / (t["lambda"] * 1e-3)}
    del x, o, a, b, c
    # the Axilrod-Teller energy over the tetrahedral domain (Section 6), N = 1536, rho = 32:
    # the cubic-root map, the table of layer starts (Section 7) and the m^3 box
    pts = torch.from_numpy(inputs.at_points(1536, seed=1610)).to(dev)
    e = torch.zeros(1, dtype=torch.float64, device=dev)
    ws = torch.empty(tri.tet_at_workspace_size(1536, 32, tri.MAP_BB) // 8 + 1, dtype=torch.float64, device=dev)
    t = {nm: graph_time_ms(lambda: tri.tet_at_energy(pts, e, 1.0, m, 32, ws), 20, stream)
         for nm, m in (("lambda", tri.MAP_LAMBDA), ("lambda_table", tri.MAP_TET_TABLE), ("bb", tri.MAP_BB))}
    out["at_energy_n1536_rho32"] = {"ms": t, "I_bb_over": {k: t["bb"] / v for k, v in t.items()}}
    del pts, e, ws
    # 1000 uneven EDM triangles (N log-uniform in [64, 8192], d = 64): one
    # persistent launch at the autotuner's tile against 1000 separate lambda
    # launches, each captured in a CUDA graph
    from paper_1609_01490_gb300 import autotune
    sizes = inputs.batched_sizes(1000, seed=1609)
    xc, pt_off = inputs.batched_points(sizes, 64, seed=1609)
    tl = sizes.astype(np.int64) * (sizes.astype(np.int64) + 1) // 2
    oo = np.zeros(len(sizes), dtype=np.uint64)
    oo[1:] = np.cumsum(tl)[:-1]
    xd = torch.from_numpy(xc).to(dev)
    oc = torch.empty(int(tl.sum()), dtype=torch.float32, device=dev)
    pto = torch.from_numpy(pt_off.view(np.int64)).to(dev)
    nk = torch.from_numpy(sizes.astype(np.int32)).to(dev)
    ood = torch.from_numpy(oo.view(np.int64)).to(dev)
    wsb = torch.empty(tri.tri_edm_batched_workspace_size(1000) // 8 + 1, dtype=torch.int64, device=dev)
    rho_b, reg_b, _ = autotune.best_batched(sizes, 64, reps=3)
    t_b = graph_time_ms(lambda: tri.tri_edm_batched(xd, pto, nk, oc, ood, rho=rho_b, reg=reg_b, workspace=wsb), 1,
                        stream)
    views = [(xd[int(pt_off[k]): int(pt_off[k]) + int(sizes[k])], oc[int(oo[k]): int(oo[k]) + int(tl[k])])
             for k in range(1000)]

    def separate():
        for xv, ov in views:
            tri.tri_edm(xv, ov, map=tri.MAP_LAMBDA, rho=16, reg=0)
    t_s = graph_time_ms(separate, 1, stream)
    out["edm_batched_1000_d64"] = {"ms": {"persistent": t_b, "separate_1000_launches": t_s},
                                   "tile": {"rho": rho_b, "reg": reg_b}, "pairs": int(tl.sum()),
                                   "speedup_over_separate": t_s / t_b}
    del xd, oc, views
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------ row suite -----
def run_suite(args):
    """One JSON line per remaining hot-path row, each timed with CUDA events
    (CUDA graphs for launches shorter than the launch overhead), lambda beside
    the bounding box and a roofline fraction."""
    import torch
    from paper_1609_01490_gb300 import inputs
    from paper_1609_01490_gb300 import tri

    dev = torch.device("cuda")
    peaks, peak_src = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    clk = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = NUM_SMS * FP32_LANES_PER_SM * 2 * clk * 1e6 / 1e12
    stream = torch.cuda.current_stream()

    def graph_ms(fn, reps):
        return graph_time_ms(fn, reps, stream)

    only = set(args.only.split(",")) if args.only else None

    def want(section):
        return only is None or section in only

    def measure_alu_peaks():
        """FP32 (scalar and f32x2) and FP64 FMA throughput of this GPU in TFLOP/s,
        from the library's FMA probe (full occupancy, 8 chains per thread)."""
        blocks = NUM_SMS * 8
        sink = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
        out = {}
        for name, kind, iters in (("fp32", 0, 4096), ("fp32x2", 1, 4096), ("fp64", 2, 128)):
            flop = tri.tri_peak_probe(kind, blocks, iters, sink)
            ms = graph_ms(lambda: tri.tri_peak_probe(kind, blocks, iters, sink), 10)
            out[name] = flop / (ms * 1e-3) / 1e12
        return out

    def emit(d):
        d.setdefault("data", "synthetic")
        d.setdefault("peaks", {"source": peak_src})
        print(json.dumps(d), flush=True)

    use_cpu = not args.no_cpu
    if use_cpu:
        import oracle
        oracle.lib()
        cores = oracle.threads()

    def cpu_leg(fn, units, unit, sample):
        """The oracle on a bounded sample of the row's workload, on the host cores."""
        if not use_cpu:
            return None
        t0 = time.perf_counter()
        fn()
        dt = time.perf_counter() - t0
        return {"value": units / dt, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample}

    peaks_alu = measure_alu_peaks()
    fp32_derived = fp32_peak
    fp32_peak = peaks_alu["fp32"]
    emit({"row": "alu_peaks", "metric": "TFLOP/s", "unit": "TFLOP/s", "value": peaks_alu,
          "config": {"workload": "FMA probe: 152 x 8 blocks of 256 threads, 8 chains per thread"},
          "derived_fp32": fp32_derived,
          "note": "ALU rooflines below use the measured scalar FP32 figure"})

    if want("maps"):
        # a1-a4: the maps alone (sentinel body), n = 65536, rho = 16
        n = 65536
        out = torch.zeros(4, dtype=torch.int32, device=dev)
        times = {}
        for name, m, sq in (("lambda_X", tri.MAP_LAMBDA, tri.SQRT_X), ("lambda_R", tri.MAP_LAMBDA, tri.SQRT_R),
                            ("lambda_N", tri.MAP_LAMBDA, tri.SQRT_N), ("lambda_pdelta_R", tri.MAP_LAMBDA_PDELTA, tri.SQRT_R),
                            ("bb", tri.MAP_BB, tri.SQRT_R), ("rb", tri.MAP_RB, tri.SQRT_R),
                            ("rec", tri.MAP_REC, tri.SQRT_R), ("utm", tri.MAP_UTM, tri.SQRT_R)):
            times[name] = graph_ms(lambda: tri.tri_map_launch(m, sq, n, 16, True, tri.BODY_SENTINEL, out), 20)
        elems = n * (n + 1) // 2
        emit({"row": "map_only", "metric": "mapped elements/s", "unit": "elements/s",
              "config": {"workload": "sentinel body (map cost only)", "n": n, "rho": 16},
              "ms": times, "value": {k: elems / (v * 1e-3) for k, v in times.items()},
              "I_bb_over": {k: times["bb"] / v for k, v in times.items()},
          "cpu_baseline": cpu_leg(lambda: oracle.lambda_enum(16384), 16384 * 16385 // 2, "elements/s",
                                  "enumeration matrix walk, m = 16384 rows")})

    if want("maps"):
        # the square-root strategies of Section 4.1 over n (the map-only sweep
        # of the paper's dummy-kernel test): time per launch of the sentinel
        # body under lambda_X, lambda_R, lambda_N and the bounding box
        sweep = {}
        for n in (1024, 2048, 4096, 8192, 16384, 32768, 65536):
            reps = max(3, min(200, (1 << 34) // (n * n)))
            sweep[n] = {name: graph_ms(lambda: tri.tri_map_launch(m, sq, n, 16, True, tri.BODY_SENTINEL, out), reps)
                        for name, m, sq in (("lambda_X", tri.MAP_LAMBDA, tri.SQRT_X),
                                            ("lambda_R", tri.MAP_LAMBDA, tri.SQRT_R),
                                            ("lambda_N", tri.MAP_LAMBDA, tri.SQRT_N),
                                            ("bb", tri.MAP_BB, tri.SQRT_R))}
        emit({"row": "map_sqrt_sweep", "metric": "ms per launch", "unit": "ms",
              "config": {"workload": "sentinel body, rho = 16, n = 1024 ... 65536"},
              "ms": sweep, "I_bb_over_lambda_R": {n: v["bb"] / v["lambda_R"] for n, v in sweep.items()},
              "lambda_N_over_lambda_X": {n: v["lambda_N"] / v["lambda_X"] for n, v in sweep.items()},
              "lambda_R_over_lambda_X": {n: v["lambda_R"] / v["lambda_X"] for n, v in sweep.items()}})

    if want("maps"):
        # Section 4.1 / 4.2 taken as printed, without the exact integer step:
        # the first omega (of all below 2^32) where each square-root estimate
        # (with the paper's eps = 1e-4 for lambda_N and lambda_R) floors to the
        # wrong row, and the first thread k where UTM's FP32 formula is wrong
        fb = torch.empty(1, dtype=torch.int64, device=dev)

        def first_error(map_id, sq, n_items, end):
            fb.fill_(-1)
            tri.tri_map_first_error(map_id, sq, n_items, 0, end, fb)
            torch.cuda.synchronize()
            v = int(fb.item()) & (2 ** 64 - 1)
            return None if v == 2 ** 64 - 1 else v

        lam = {}
        for name, sq in (("lambda_X", tri.SQRT_X), ("lambda_R", tri.SQRT_R), ("lambda_N", tri.SQRT_N)):
            w = first_error(tri.MAP_LAMBDA, sq, 0, 1 << 32)
            row = None if w is None else int((math.isqrt(8 * w + 1) - 1) // 2)
            lam[name] = {"first_bad_omega": w, "exact_rows_below": row}
        utm = {}
        for items in (1000, 2000, 3000, 4000, 6000, 8000, 16000, 32768):
            utm[items] = first_error(tri.MAP_UTM, tri.SQRT_X, items, items * (items - 1) // 2)
        emit({"row": "printed_formula_exactness", "metric": "first failing index", "unit": "index",
              "config": {"workload": "every omega < 2^32 (lambda); every thread of n items (UTM)"},
              "lambda": lam, "utm_first_bad_k": utm,
              "note": "exact_rows_below rows of blocks map correctly: n <= rows x rho elements"})

    if want("edm"):
        # a5: the paper-size EDM, N = 2048, d = 3, rho = 16 (8.4 MB output,
        # L2-resident across back-to-back launches, so HBM does not bound it).
        # Its bounds: the launch-and-map floor (the map alone, sentinel body,
        # on the same grid of blocks) and the L2-resident write bandwidth (a
        # fill of the same 8.4 MB buffer).  Times per launch, 200 launches in
        # one CUDA graph.
        xh = inputs.edm_uniform_points(2048, 3, seed=1609)
        x = torch.from_numpy(xh).to(dev)
        o = torch.empty(2048 * 2049 // 2, dtype=torch.float32, device=dev)
        P = 2048 * 2049 // 2
        maps5 = (("lambda", tri.MAP_LAMBDA), ("lambda_pdelta", tri.MAP_LAMBDA_PDELTA), ("bb", tri.MAP_BB),
                 ("rb", tri.MAP_RB), ("rec", tri.MAP_REC), ("utm", tri.MAP_UTM))
        t = {nm: graph_ms(lambda: tri.tri_edm(x, o, map=m, rho=16, reg=1), 200) for nm, m in maps5}
        t4 = {nm: graph_ms(lambda: tri.tri_edm(x, o, map=m, rho=16, reg=4), 200) for nm, m in maps5 if nm != "utm"}
        fill_ms = graph_ms(lambda: o.fill_(1.0), 200)
        l2_gbs = 4.0 * P / (fill_ms * 1e-3) / 1e9
        o4 = torch.zeros(4, dtype=torch.int32, device=dev)
        # the same grids with the map alone: 128 block rows of 16 x 16 threads
        # (one pair per thread), 32 block rows (4 x 4 pairs per thread: 512 "elements" at rho 16)
        floor1 = graph_ms(lambda: tri.tri_map_launch(tri.MAP_LAMBDA, tri.SQRT_R, 2048, 16, True, tri.BODY_SENTINEL,
                                                     o4), 200)
        floor4 = graph_ms(lambda: tri.tri_map_launch(tri.MAP_LAMBDA, tri.SQRT_R, 512, 16, True, tri.BODY_SENTINEL,
                                                     o4), 200)
        best4 = min(t4.values())
        ach = 4.0 * P / (t4["lambda"] * 1e-3) / 1e9
        emit({"row": "edm_fp32_paper_size", "metric": "pairs/s", "unit": "pairs/s",
              "value": P / (t4["lambda"] * 1e-3),
              "config": {"workload": "edm_n2048_d3_uniform", "rho": 16, "reg": 4, "launches_per_graph": 200},
              "ms_reg4": t4, "ms_reg1_paper_shape": t, "I_bb_over_lambda": t4["bb"] / t4["lambda"],
              "I_bb_over_lambda_reg1": t["bb"] / t["lambda"],
              "bounds": {"launch_and_map_floor_ms_reg1": floor1, "launch_and_map_floor_ms_reg4": floor4,
                         "l2_fill_ms": fill_ms, "l2_write_gbs": l2_gbs,
                         "note": "floors: the sentinel-body map kernel on the same grids (8256 and 528 blocks); "
                                 "L2 write bandwidth: a fill of the same 8.4 MB buffer"},
              "roofline": {"bound": "l2", "achieved": ach, "peak": l2_gbs, "unit": "GB/s", "frac": ach / l2_gbs,
                           "frac_of_time_bound": max(fill_ms, floor4) / t4["lambda"],
                           "note": "8.4 MB output stays in L2 across back-to-back launches; time bound = "
                                   "max(L2 fill time, launch-and-map floor)"},
              "fastest": min(t4, key=t4.get), "fastest_ms": best4,
              "cpu_baseline": cpu_leg(lambda: [oracle.edm_rows(xh) for _ in range(50)], 50 * P, "pairs/s",
                                      "the whole triangle 50 times, FP64")})

    if want("edm"):
        # a2/a5 at scale: N = 65536, d = 3 (store-bound, 8.6 GB of output) with the
        # paper's block shape (one pair per thread, rho = 16) and with 4 x 4 pairs per thread
        xh = inputs.edm_uniform_points(65536, 3, seed=1609)
        x = torch.from_numpy(xh).to(dev)
        o = torch.empty(65536 * 65537 // 2, dtype=torch.float32, device=dev)
        P = 65536 * 65537 // 2
        for reg in (1, 4):
            t = {nm: graph_ms(lambda: tri.tri_edm(x, o, map=m, rho=16, reg=reg), 3)
                 for nm, m in (("lambda", tri.MAP_LAMBDA), ("bb", tri.MAP_BB), ("rb", tri.MAP_RB),
                               ("rec", tri.MAP_REC))}
            gbs = 4.0 * P / (t["lambda"] * 1e-3) / 1e9
            emit({"row": f"edm_fp32_n65536_d3_reg{reg}", "metric": "pairs/s", "unit": "pairs/s",
                  "value": P / (t["lambda"] * 1e-3),
                  "config": {"workload": "edm_n65536_d3_uniform", "rho": 16, "reg": reg,
                             "pairs_per_thread": reg * reg}, "ms": t, "I_bb_over_lambda": t["bb"] / t["lambda"],
                  "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm},
                  "cpu_baseline": cpu_leg(lambda: oracle.edm_rows(xh, 63488, 65536),
                                          65536 * 65537 // 2 - 63488 * 63489 // 2, "pairs/s",
                                          "rows 63488 .. 65535 (the last 2048 rows), FP64")})
        del x, o
        torch.cuda.empty_cache()

    if want("life"):
        # a6: triangular Life, n = 16384, 100 steps, rho = 16
        n = 16384
        gh = inputs.ca_grid(n, seed=1609)
        a = torch.from_numpy(gh).to(dev)
        b = torch.zeros_like(a)

        def life(m, rho):
            def run():
                for s in range(100):
                    src, dst = (a, b) if s % 2 == 0 else (b, a)
                    tri.tri_ca_step(src, dst, n, map=m, rho=rho)
            return run
        # 128 x 128 cell tiles (rho = 32) are the fastest; rho = 16 beside them
        t = {nm: graph_ms(life(m, 32), 1) / 100 for nm, m in (("lambda", tri.MAP_LAMBDA), ("bb", tri.MAP_BB),
                                                              ("rb", tri.MAP_RB), ("rec", tri.MAP_REC))}
        t16 = {nm: graph_ms(life(m, 16), 1) / 100 for nm, m in (("lambda", tri.MAP_LAMBDA), ("bb", tri.MAP_BB))}
        cells = n * (n + 1) // 2
        gbs = 2.0 * cells / (t["lambda"] * 1e-3) / 1e9
        emit({"row": "life_step", "metric": "cell updates/s", "unit": "cells/s", "value": cells / (t["lambda"] * 1e-3),
              "config": {"workload": "life_n16384_bernoulli05_100steps", "rho": 32}, "ms_per_step": t,
              "ms_per_step_rho16": t16,
              "I_bb_over_lambda": t["bb"] / t["lambda"],
              "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                           "algorithmic_bytes_per_step": 2 * cells},
              "cpu_baseline": cpu_leg(lambda: oracle.ca_step(gh), cells, "cells/s", "one step of the n = 16384 grid")})
        # the same 100 steps through tri_ca_run: up to 16 steps per pass through
        # memory (one warp per tile: read once with a 16-cell halo, stepped as
        # bits in registers, written once), 7 passes
        c = torch.zeros_like(a)

        def run100(m):
            def go():
                tri.tri_ca_run(a, b, n, 100, scratch=c, map=m, rho=32)
            return go
        tr = {nm: graph_ms(run100(m), 1) for nm, m in (("lambda", tri.MAP_LAMBDA), ("bb", tri.MAP_BB),
                                                        ("rb", tri.MAP_RB), ("rec", tri.MAP_REC))}
        passes = -(-100 // 16)
        gbs_run = 2.0 * cells * passes / (tr["lambda"] * 1e-3) / 1e9
        emit({"row": "life_run", "metric": "cell updates/s", "unit": "cells/s",
              "value": 100 * cells / (tr["lambda"] * 1e-3),
              "config": {"workload": "life_n16384_bernoulli05_100steps", "rho": 32, "steps_per_pass": 16},
              "ms_per_100_steps": tr, "I_bb_over_lambda": tr["bb"] / tr["lambda"],
              "speedup_over_step_by_step": 100 * t["lambda"] / tr["lambda"],
              "roofline": {"bound": "hbm", "achieved": gbs_run, "peak": hbm, "unit": "GB/s", "frac": gbs_run / hbm,
                           "algorithmic_bytes_per_pass": 2 * cells, "passes": passes,
                           "note": "one read and one write of every cell per pass; the 16-cell halos are re-read; "
                                   "the kernel is bound by its ALU pipe (ncu), not by these bytes"},
              "cpu_baseline": cpu_leg(lambda: oracle.ca_run(gh, 4), 4 * cells, "cells/s",
                                      "four steps of the n = 16384 grid")})

    if want("at"):
        # a7: Axilrod-Teller energy over the tetrahedral domain, N = 1536, rho = 16
        n = 1536
        ph = inputs.at_points(n, seed=1610)
        p = torch.from_numpy(ph).to(dev)
        e = torch.zeros(1, dtype=torch.float64, device=dev)
        ws = torch.empty(max(tri.tet_at_workspace_size(n, r, tri.MAP_BB) for r in (16, 32)) // 8 + 1,
                         dtype=torch.float64, device=dev)
        # 32 x 32 threads with 32 values of k each are the fastest; rho = 16 beside them
        t = {nm: graph_ms(lambda: tri.tet_at_energy(p, e, 1.0, m, 32, ws), 20)
             for nm, m in (("lambda", tri.MAP_LAMBDA), ("lambda_table", tri.MAP_TET_TABLE), ("bb", tri.MAP_BB))}
        t16 = {nm: graph_ms(lambda: tri.tet_at_energy(p, e, 1.0, m, 16, ws), 20)
               for nm, m in (("lambda", tri.MAP_LAMBDA), ("lambda_table", tri.MAP_TET_TABLE), ("bb", tri.MAP_BB))}
        trip = n * (n - 1) * (n - 2) // 6
        tf = 40.0 * trip / (t["lambda"] * 1e-3) / 1e12
        emit({"row": "at_energy", "metric": "triplets/s", "unit": "triplets/s", "value": trip / (t["lambda"] * 1e-3),
              "value_layer_table": trip / (t["lambda_table"] * 1e-3),
              "config": {"workload": "at_n1536_uniform_unit_density", "rho": 32}, "ms": t, "ms_rho16": t16,
              "I_bb_over_lambda": t["bb"] / t["lambda"],
              "roofline": {"bound": "alu", "achieved": tf, "peak": fp32_peak, "unit": "TFLOP/s", "frac": tf / fp32_peak,
                           "note": "about 40 FP32 flop per triplet (plus one MUFU rsqrt)"},
              "cpu_baseline": cpu_leg(lambda: oracle.at_energy(ph[:1000]), 1000 * 999 * 998 // 6, "triplets/s",
                                      "the first 1000 points (1.66e8 triplets), FP64")})

    if want("at"):
        # Section 6 / Section 7: the tetrahedral map alone (sentinel body), the
        # closed-form cubic root against the table of layer starts and the m^3 box
        n = 16384
        o4 = torch.zeros(4, dtype=torch.int32, device=dev)
        t = {nm: graph_ms(lambda: tri.tet_map_ex(m, n, 16, tri.BODY_SENTINEL, o4), 3)
             for nm, m in (("lambda_cubic", tri.MAP_LAMBDA), ("lambda_table", tri.MAP_TET_TABLE),
                           ("bb", tri.MAP_BB))}
        mm = n // 16
        emit({"row": "tet_map_only", "metric": "blocks/s", "unit": "blocks/s",
              "value": mm * (mm + 1) * (mm + 2) // 6 / (t["lambda_table"] * 1e-3),
              "config": {"workload": "sentinel body, n = 16384, rho = 16 (179,481,600 tetrahedral blocks)"},
              "ms": t, "I_bb_over": {k: t["bb"] / v for k, v in t.items()},
              "table_over_cubic": t["lambda_table"] / t["lambda_cubic"],
              "cpu_baseline": cpu_leg(lambda: oracle.tet_enum(800), 800 * 801 * 802 // 6, "blocks/s",
                                      "tetrahedral enumeration, m = 800 layers")})

    if want("collide"):
        # Section 5, test 3: collision detection of 65,536 spheres (smaller
        # counts are for profiling) with about 4 contacts each, 1-D and 3-D,
        # under each map, with the paper's block shape (one pair per thread)
        # and with 4 x 4 and 8 x 8 pairs per thread
        n = args.collide_n
        npairs = torch.zeros(1, dtype=torch.int64, device=dev)
        cnt = torch.zeros(n, dtype=torch.int32, device=dev)
        plist = torch.zeros((4 * n, 2), dtype=torch.int32, device=dev)
        P = n * (n - 1) // 2
        alu_peak = fp32_peak / 2  # FP32 results per second (an FMA counts 2 flop)
        for dim in (1, 3):
            cs, rs = inputs.spheres(n, dim)
            cd, rd = torch.from_numpy(cs).to(dev), torch.from_numpy(rs).to(dev)
            ops = 4 if dim == 1 else 10  # FP32 sub, mul, add per pair (no fused multiply-add)
            r0 = max(0, n - 8192)
            cpu_base = cpu_leg(lambda: oracle.collide_pairs(cs, rs, r0, n), n * (n - 1) // 2 - r0 * (r0 - 1) // 2,
                               "pairs/s", f"rows {r0} .. {n - 1} (every pair j < i), FP32 test")
            for reg in (1, 4, 8):
                maps = [("lambda", tri.MAP_LAMBDA), ("bb", tri.MAP_BB), ("rb", tri.MAP_RB), ("rec", tri.MAP_REC)]
                if reg == 1:
                    maps.append(("utm", tri.MAP_UTM))
                t = {nm: graph_ms(lambda: tri.tri_collide(cd, rd, npairs, count=cnt, pairs=plist, map=m, rho=16,
                                                          reg=reg), 5) for nm, m in maps}
                top = ops * P / (t["lambda"] * 1e-3) / 1e12
                emit({"row": f"collide_{dim}d_n{n}_reg{reg}", "metric": "pairs/s", "unit": "pairs/s",
                      "value": P / (t["lambda"] * 1e-3),
                      "config": {"workload": f"spheres_{dim}d_n{n}_kappa4", "rho": 16, "reg": reg,
                                 "pairs_per_thread": reg * reg}, "ms": t, "contacts": int(npairs.item()),
                      "I_bb_over_lambda": t["bb"] / t["lambda"],
                      "roofline": {"bound": "alu", "achieved": top, "peak": alu_peak, "unit": "TOP/s",
                                   "frac": top / alu_peak,
                                   "note": f"{ops} FP32 operations per pair; peak: measured FFMA results/s"},
                      "cpu_baseline": cpu_base})
            del cd, rd
        del npairs, cnt, plist

    if want("batched"):
        # a9: 1000 uneven EDM triangles: one persistent launch vs 1000 tri_edm launches (both in CUDA graphs)
        sizes = inputs.batched_sizes(1000, seed=1609)
        xc, pt_off = inputs.batched_points(sizes, 64, seed=1609)
        tri_len = sizes.astype(np.int64) * (sizes.astype(np.int64) + 1) // 2
        out_off = np.zeros(len(sizes), dtype=np.uint64)
        out_off[1:] = np.cumsum(tri_len)[:-1]
        total = int(tri_len.sum())
        xd = torch.from_numpy(xc).to(dev)
        oc = torch.empty(total, dtype=torch.float32, device=dev)
        pto = torch.from_numpy(pt_off.view(np.int64)).to(dev)
        nk = torch.from_numpy(sizes.astype(np.int32)).to(dev)
        oo = torch.from_numpy(out_off.view(np.int64)).to(dev)
        wsb = torch.empty(tri.tri_edm_batched_workspace_size(1000) // 8 + 1, dtype=torch.int64, device=dev)
        # the tile (rho threads per side, reg x reg pairs per thread) picked by
        # the autotuner over every candidate, then the persistent launch timed
        # in a CUDA graph at the pick and at each rho with 4 x 4 pairs
        from paper_1609_01490_gb300 import autotune
        tuned = autotune.tune_batched(sizes, 64, use_cache=False)
        rho_b, reg_b = (int(v) for v in min(tuned, key=tuned.get).split("/"))
        tb = {}
        for rho in (8, 16, 32):
            tb[f"persistent_rho{rho}_reg4"] = graph_ms(lambda: tri.tri_edm_batched(xd, pto, nk, oc, oo, rho=rho, reg=4,
                                                                                    workspace=wsb), 1)
        tb[f"persistent_tuned_rho{rho_b}_reg{reg_b}"] = graph_ms(
            lambda: tri.tri_edm_batched(xd, pto, nk, oc, oo, rho=rho_b, reg=reg_b, workspace=wsb), 1)
        views = [(xd[int(pt_off[k]): int(pt_off[k]) + int(sizes[k])], oc[int(out_off[k]): int(out_off[k]) + int(tri_len[k])])
                 for k in range(1000)]

        def separate():
            for xv, ov in views:
                tri.tri_edm(xv, ov, map=tri.MAP_LAMBDA, rho=16, reg=0)
        tb["separate_1000_launches"] = graph_ms(separate, 1)
        best = min(v for k, v in tb.items() if k.startswith("persistent"))
        tf = 3.0 * 64 * total / (best * 1e-3) / 1e12
        emit({"row": "edm_batched", "metric": "pairs/s", "unit": "pairs/s", "value": total / (best * 1e-3),
              "config": {"workload": "1000 instances, N log-uniform [64, 8192], d = 64", "pairs": total,
                         "tuned_tile": {"rho": rho_b, "reg": reg_b}}, "ms": tb, "autotune_ms": tuned,
              "speedup_over_separate": tb["separate_1000_launches"] / best,
              "roofline": {"bound": "alu", "achieved": tf, "peak": fp32_peak, "unit": "TFLOP/s", "frac": tf / fp32_peak},
              "cpu_baseline": cpu_leg(lambda: [oracle.edm_rows(xc[int(pt_off[k]): int(pt_off[k]) + int(sizes[k])])
                                               for k in range(20)], int(tri_len[:20].sum()), "pairs/s",
                                      "the first 20 instances, FP64")})


def run_split(args, rank: int, world: int, local: int):
    """One triangle split across the ranks (--split): rank r computes the band
    of rows tri_edm_partition gives it (equal pair counts, disjoint packed
    ranges, no exchange while computing) with tri_edm_rows; the job's value is
    the triangle's pairs over the slowest rank's time (strong scaling).  The
    bands stay on their GPUs: gathering them is not part of the EDM."""
    import torch
    import torch.distributed as dist
    from paper_1609_01490_gb300 import inputs
    from paper_1609_01490_gb300 import tri

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    prec = {"bf16x3": tri.BF16X3, "bf16x6": tri.BF16X6}[args.prec]
    x_host = inputs.edm_normal_points(N_PTS, D_FEAT, seed=1609, dup_frac=DUP)  # the same points on every rank
    P = N_PTS * (N_PTS + 1) // 2
    rb, re_, pb, pe = tri.tri_edm_partition(N_PTS, world, rank)
    x = torch.from_numpy(x_host).to(dev)
    band = torch.empty(max(pe - pb, 4), dtype=torch.float32, device=dev)
    ws = torch.empty(tri.tri_edm_workspace_size(N_PTS, D_FEAT, prec), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        tri.tri_edm_rows(x, rb, re_, band, map=tri.MAP_LAMBDA, prec=prec, workspace=ws)

    def timed(fn, k, w, sampler=None):
        for _ in range(w):
            fn()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.mark_begin()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if sampler:
            sampler.mark_end()
        if world > 1:
            dist.barrier()
        return e0.elapsed_time(e1) / k

    sampler = ClockSampler(local)
    sampler.start()
    ms = max_over_ranks([timed(step, args.steps, args.warmup, sampler)], world, dev)[0]
    clocks = sampler.stop()
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(x_host).pin_memory()
        bh = torch.empty(band.numel(), dtype=torch.float32).pin_memory()

        def e2e_step():
            x.copy_(xh, non_blocking=True)
            step()
            bh.copy_(band, non_blocking=True)
        ms_e2e = max_over_ranks([timed(e2e_step, max(2, min(args.steps, 5)), args.warmup)], world, dev)[0]
        e2e = {"value": P / (ms_e2e * 1e-3), "ms_per_step": ms_e2e, "unit": "pairs/s",
               "h2d_bytes_per_step": xh.numel() * 4, "d2h_bytes_per_step": (pe - pb) * 4,
               "path": "copies around tri_edm_rows (each rank's band)"}
    cfg = headline_config(args.prec)
    cfg["parallelism"] = f"one triangle split in {world} row bands of equal pair count (tri_edm_partition)"
    line = {"metric": "pairs/s", "value": P / (ms * 1e-3), "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic", "config": cfg, "clocks": clocks,
            "gpu_launches": args.steps * 3, "band": {"rows": [rb, re_], "pairs": pe - pb}}
    if e2e:
        line["e2e"] = e2e
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_profile_case(args):
    """A few launches of one kernel on its small case, for ncu captures
    (select the launch with -k and -s / -c): the Life step (n = 16384,
    lambda, rho 32), 32 Life steps through tri_ca_run (two passes, twice), the AT energy (N = 1536, table map, rho 32), the FP32
    EDM (N = 16384, d = 64, lambda, rho 16 x 8 x 8 pairs), the batched EDM
    (100 of the seeded instances, d = 64, rho 16 x 8 x 8) and the collision
    test (16384 spheres in 3-D, rho 16 x 8 x 8).  Four launches each."""
    import torch
    from paper_1609_01490_gb300 import inputs
    from paper_1609_01490_gb300 import tri
    dev = torch.device("cuda")
    case = args.profile
    if case == "life":
        n = 16384
        a = torch.from_numpy(inputs.ca_grid(n, seed=1609)).to(dev)
        b = torch.zeros_like(a)
        for _ in range(4):
            tri.tri_ca_step(a, b, n, map=tri.MAP_LAMBDA, rho=32)
            a, b = b, a
    elif case == "life_run":
        n = 16384
        a = torch.from_numpy(inputs.ca_grid(n, seed=1609)).to(dev)
        b, c = torch.zeros_like(a), torch.zeros_like(a)
        for _ in range(2):
            tri.tri_ca_run(a, b, n, 32, scratch=c, map=tri.MAP_LAMBDA, rho=32)  # two passes each
    elif case == "at":
        p = torch.from_numpy(inputs.at_points(1536, seed=1610)).to(dev)
        e = torch.zeros(1, dtype=torch.float64, device=dev)
        ws = torch.empty(tri.tet_at_workspace_size(1536, 32, tri.MAP_TET_TABLE) // 8 + 1, dtype=torch.float64,
                         device=dev)
        for _ in range(4):
            tri.tet_at_energy(p, e, 1.0, tri.MAP_TET_TABLE, 32, ws)
    elif case == "edm":
        x = torch.from_numpy(inputs.edm_normal_points(16384, 64, seed=1609)).to(dev)
        o = torch.empty(16384 * 16385 // 2, device=dev)
        for _ in range(4):
            tri.tri_edm(x, o, map=tri.MAP_LAMBDA, rho=16, reg=8)
    elif case == "batched":
        sizes = inputs.batched_sizes(100, seed=1609)
        xc, pt_off = inputs.batched_points(sizes, 64, seed=1609)
        tl = sizes.astype(np.int64) * (sizes.astype(np.int64) + 1) // 2
        oo = np.zeros(len(sizes), dtype=np.uint64)
        oo[1:] = np.cumsum(tl)[:-1]
        oc = torch.empty(int(tl.sum()), device=dev)
        ws = torch.empty(tri.tri_edm_batched_workspace_size(100) // 8 + 1, dtype=torch.int64, device=dev)
        args_b = (torch.from_numpy(xc).to(dev), torch.from_numpy(pt_off.view(np.int64)).to(dev),
                  torch.from_numpy(sizes.astype(np.int32)).to(dev), oc, torch.from_numpy(oo.view(np.int64)).to(dev))
        for _ in range(4):
            tri.tri_edm_batched(*args_b, rho=16, reg=8, workspace=ws)
    elif case == "collide":
        c, r = inputs.spheres(16384, 3)
        cd, rd = torch.from_numpy(c).to(dev), torch.from_numpy(r).to(dev)
        npairs = torch.zeros(1, dtype=torch.int64, device=dev)
        cnt = torch.zeros(16384, dtype=torch.int32, device=dev)
        for _ in range(4):
            tri.tri_collide(cd, rd, npairs, count=cnt, map=tri.MAP_LAMBDA, rho=16, reg=8)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": case, "ok": True}))


    # -------------------------------------------------------------- our arm -----


def main():
    global N_PTS, D_FEAT, WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x6", choices=["fp32", "bf16x3", "bf16x6"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end pass")
    ap.add_argument("--no-arms", action="store_true", help="skip the BB and FP32 comparison arms")
    ap.add_argument("--split", action="store_true",
                    help="split one triangle across the ranks in row bands (strong scaling) instead of "
                         "one triangle per rank (weak scaling, the default)")
    ap.add_argument("--n", type=int, default=N_PTS, help="points (smaller cases are for profiling only)")
    ap.add_argument("--d", type=int, default=D_FEAT, help="features (smaller cases are for profiling only)")
    ap.add_argument("--suite", action="store_true", help="one JSON line per other hot-path row instead")
    ap.add_argument("--only", default="", help="suite sections to run (maps,edm,life,at,collide,batched)")
    ap.add_argument("--collide-n", type=int, default=65536, help="spheres in the collision rows")
    ap.add_argument("--profile", default="", choices=["", "life", "life_run", "at", "edm", "batched", "collide"],
                    help="run a few launches of one kernel's small case (for ncu captures) and exit")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if (args.n, args.d) != (N_PTS, D_FEAT):  # a smaller case, for profiling and tests
        N_PTS, D_FEAT = args.n, args.d
        WORKLOAD = f"edm_n{N_PTS}_d{D_FEAT}_normal_dup1pct"

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.profile:
        run_profile_case(args)
        return
    if args.suite:
        run_suite(args)
        return
    if args.split:
        if args.prec == "fp32":
            ap.error("--split runs the tensor-core path (bf16x3 or bf16x6)")
        run_split(args, rank, world, local)
        return

    import torch
    import torch.distributed as dist
    from paper_1609_01490_gb300 import inputs
    from paper_1609_01490_gb300 import tri

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    PRECS = {"fp32": tri.FP32, "bf16x3": tri.BF16X3, "bf16x6": tri.BF16X6}
    prec = PRECS[args.prec]
    x_host = inputs.edm_normal_points(N_PTS, D_FEAT, seed=1609 + rank, dup_frac=DUP)
    P = N_PTS * (N_PTS + 1) // 2
    x = torch.from_numpy(x_host).to(dev)
    out = torch.empty(P, dtype=torch.float32, device=dev)
    ws_bytes = max(tri.tri_edm_workspace_size(N_PTS, D_FEAT, p) for p in PRECS.values())
    ws = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=dev)
    flagged = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    phase_events = []  # (prepare, gram, fixup) event pairs recorded inside the timed region

    def step(map_id, pr=prec, record=False):
        if pr == tri.FP32:
            # the FP32 comparison arm in its fastest measured shape: 8 x 8 pairs per
            # thread at high d (compute-bound), 4 x 4 at low d (store-bound)
            tri.tri_edm(x, out, map=map_id, rho=16, reg=8 if D_FEAT >= 32 else 4, prec=pr)
            return
        if not record:
            tri.tri_edm(x, out, map=map_id, prec=pr, workspace=ws, n_flagged=flagged)
            return
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        tri.tri_edm_prepare(x, pr, ws)
        ev[1].record(stream)
        tri.tri_edm_gram(N_PTS, D_FEAT, out, map_id, pr, ws)
        ev[2].record(stream)
        tri.tri_edm_fixup(x, out, pr, ws, flagged)
        ev[3].record(stream)
        phase_events.append(ev)

    def timed(fn, k, w, sampler=None):
        for _ in range(w):
            fn()
        barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.mark_begin()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(k):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        if sampler:
            sampler.mark_end()
        barrier()
        return ev0.elapsed_time(ev1) / k  # ms per step

    # ---- headline: lambda map, timed region with clock sampling
    sampler = ClockSampler(local)
    for _ in range(args.warmup):
        step(tri.MAP_LAMBDA)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    ms_lambda = timed(lambda: step(tri.MAP_LAMBDA, record=True), args.steps, 0, sampler)
    clocks = sampler.stop()
    ms_step = max_over_ranks([ms_lambda], world, dev)[0]
    value = job_rate(world, P, ms_step)
    n_flagged = int(flagged.item())
    phases = None
    if phase_events:
        tot = [0.0, 0.0, 0.0]
        for ev in phase_events:
            for q in range(3):
                tot[q] += ev[q].elapsed_time(ev[q + 1])
        phases = {"prepare_ms": tot[0] / len(phase_events), "gram_ms": tot[1] / len(phase_events),
                  "fixup_ms": tot[2] / len(phase_events)}

    # ---- bounding box on the same input (the paper's I = t_BB / t_lambda)
    # (every timed leg warms up with the headline's W >= 3 steps)
    ms_bb = float("nan") if args.no_arms else timed(lambda: step(tri.MAP_BB), max(3, args.steps // 2), args.warmup)
    # ---- the FP32 direct-difference path on the same input, for comparison
    if prec == tri.FP32:
        ms_fp32 = ms_step
    else:
        ms_fp32 = float("nan") if args.no_arms else timed(lambda: step(tri.MAP_LAMBDA, tri.FP32), 3,
                                                              args.warmup)
    ms_bb, ms_fp32 = max_over_ranks([ms_bb, ms_fp32], world, dev)
    # ---- the paper's comparison of maps at its own sizes (outside the timed region)
    paper = None if args.no_arms else paper_comparison(tri, inputs, dev, stream)

    # ---- roofline of the dominant kernel
    peaks, peak_src = load_peaks()
    clk = float(peaks.get("sm_max_mhz", 2070.0))
    if prec == tri.FP32:
        flops = 3.0 * D_FEAT * P  # sub, mul, add per feature and pair
        achieved = flops / (ms_step * 1e-3) / 1e12
        peak = NUM_SMS * FP32_LANES_PER_SM * 2 * clk * 1e6 / 1e12
        roof = {"bound": "alu", "kernel": f"edm_kernel<lambda,16,{8 if D_FEAT >= 32 else 4}>", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": f"152 SMs x 128 FP32 lanes x 2 flop x {clk:.0f} MHz (derived)"}
        roof_alt = None
    else:
        nprod = 6 if prec == tri.BF16X6 else 3
        planes = 3 if prec == tri.BF16X6 else 2
        dp = -(-D_FEAT // 64) * 64
        t_gram = phases["gram_ms"] * 1e-3
        # algorithmic bytes: the packed FP32 triangle written once, the planes and norms read once
        nbytes = 4.0 * P + planes * N_PTS * dp * 2 + 4 * N_PTS
        hbm = nbytes / t_gram / 1e9
        # algorithmic tensor work: every pair i >= j once, 2 flop per
        # multiply-add over the K-padded features, for each kept plane product
        flops = 2.0 * dp * nprod * P
        tflop = flops / t_gram / 1e12
        traffic = NCU_TRAFFIC.get((args.prec, N_PTS, D_FEAT))
        roof_hbm = {"bound": "hbm", "kernel": f"gram_kernel<lambda,{planes}>", "achieved": hbm,
                    "peak": float(peaks["hbm_gbs"]), "unit": "GB/s", "frac": hbm / float(peaks["hbm_gbs"]),
                    "traffic": traffic, "algorithmic_bytes": nbytes,
                    "peak_source": f"hbm_gbs of {peak_src}"}
        roof_tc = {"bound": "tensor", "kernel": f"gram_kernel<lambda,{planes}>", "achieved": tflop,
                   "peak": float(peaks["bf16_tflops"]), "unit": "TFLOP/s",
                   "frac": tflop / float(peaks["bf16_tflops"]), "traffic": traffic,
                   "flops": flops, "flops_note": "N(N+1)/2 pairs x 2 x K(padded) x plane products",
                   "peak_source": f"bf16_tflops (burst) of {peak_src}"}
        roof, roof_alt = (roof_hbm, roof_tc) if roof_hbm["frac"] >= roof_tc["frac"] else (roof_tc, roof_hbm)

    # ---- end to end through host buffers: tri_edm_host (pinned H2D of x, banded
    # compute with each band's D2H overlapping the next band; FP32: copies around tri_edm)
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(x_host).pin_memory()
        oh = torch.empty(P, dtype=torch.float32).pin_memory()

        if prec == tri.FP32:
            def e2e_step():
                x.copy_(xh, non_blocking=True)
                step(tri.MAP_LAMBDA)
                oh.copy_(out, non_blocking=True)
        else:
            def e2e_step():
                tri.tri_edm_host(xh, oh, x, out, ws, map=tri.MAP_LAMBDA, prec=prec, n_flagged=flagged)

        ms_e2e = max_over_ranks([timed(e2e_step, max(2, min(args.steps, 5)), args.warmup)], world, dev)[0]
        # the same steps one by one (the host link is shared with the machine's
        # other jobs: a slow step shows here rather than only in the mean)
        step_ms = []
        for _ in range(3):
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record(stream)
            e2e_step()
            eb.record(stream)
            eb.synchronize()
            step_ms.append(ea.elapsed_time(eb))
        # the same device-to-host copy alone on this machine (it bounds the step):
        # in the 16 row bands of ~512 MB that tri_edm_host copies, and as one
        # 8.59 GB copy (shared hosts have given ~90 to ~195 GB/s for the latter)
        nb = 16
        edges = [0] + [min(P, int(P * (k + 1) / nb)) for k in range(nb)]

        def banded():
            for a, b in zip(edges[:-1], edges[1:]):
                oh[a:b].copy_(out[a:b], non_blocking=True)
        ms_copy = timed(banded, 2, args.warmup)
        ms_copy1 = timed(lambda: oh.copy_(out, non_blocking=True), 2, args.warmup)
        e2e = {"value": job_rate(world, P, ms_e2e), "ms_per_step": ms_e2e,
               "d2h_copy_alone_gbs": oh.numel() * 4 / (ms_copy * 1e-3) / 1e9,
               "d2h_single_copy_gbs": oh.numel() * 4 / (ms_copy1 * 1e-3) / 1e9,
               "single_steps_ms": step_ms, "copy_alone_ms": ms_copy,
               "unit": "pairs/s", "h2d_bytes_per_step": xh.numel() * 4,
               "d2h_bytes_per_step": oh.numel() * 4,
               "path": "tri_edm_host" if prec != tri.FP32 else "copies around tri_edm"}
        del oh, xh

    line = {
        "metric": "pairs/s", "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "bf16x3": "bf16", "bf16x6": "bf16"}[args.prec],
        "data": "synthetic",
        "config": headline_config(args.prec),
        "bb": {"ms_per_step": ms_bb, "value": job_rate(world, P, ms_bb), "I_bb_over_lambda": ms_bb / ms_step},
        "fp32_lambda": {"ms_per_step": ms_fp32, "value": job_rate(world, P, ms_fp32),
                        "speedup_of_headline": ms_fp32 / ms_step},
        "paper_maps": paper,
        "clocks": clocks,
        "gpu_launches": args.steps * (1 if prec == tri.FP32 else 3),
        "roofline": roof,
        "roofline_other": roof_alt,
        "phases": phases,
        "n_flagged": n_flagged if prec != tri.FP32 else None,
        "peaks": {"source": peak_src},
    }
    if e2e:
        line["e2e"] = e2e
    if rank == 0 and not args.no_cpu:
        rate, thr, sample = cpu_oracle_sample(x_host)
        line["cpu_baseline"] = {"value": rate, "unit": "pairs/s", "cores": thr, "kind": "oracle", "sample": sample,
                                "host_cores": host_cores()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
