"""Autotuner: time every (map, rho) candidate of a kernel at a given size and
keep the fastest.

Each candidate runs on the same seeded input; times are medians of CUDA-event
measurements after warm-up launches.  Results are cached in a JSON file
(``TRI_TUNE_CACHE``, default ``~/.cache/tri_autotune.json``) keyed by the GPU
name, kernel and size, so a sweep is paid once per configuration.  The
exhaustive sweep is also the ground truth the learned selector is judged
against (``selector.py``).

Kernels and their candidate maps:
  edm: lambda, lambda on P_Delta, BB, RB, REC, UTM (Section 4.2), FP32 direct
       differences, 4 x 4 pairs per thread (reg = 4)
  ca:  lambda, lambda on P_Delta, BB, RB, REC (one Life step)
  at:  tetrahedral lambda, BB (Axilrod-Teller energy)
REC is skipped where the block count is not a power of two.

The batched EDM (many uneven triangles in one persistent launch, lambda on
each instance's blocks) has one map and is tuned over its tile instead:
rho in {8, 16, 32} threads per side times reg x reg pairs per thread
(``tune_batched``).
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics
import time

import numpy as np
import torch

from . import inputs
from . import tri

KERNELS = ("edm", "ca", "at")
RHOS = (8, 16, 32)
MAPS = {
    "edm": (tri.MAP_LAMBDA, tri.MAP_LAMBDA_PDELTA, tri.MAP_BB, tri.MAP_RB, tri.MAP_REC, tri.MAP_UTM),
    "ca": (tri.MAP_LAMBDA, tri.MAP_LAMBDA_PDELTA, tri.MAP_BB, tri.MAP_RB, tri.MAP_REC),
    "at": (tri.MAP_LAMBDA, tri.MAP_BB),
}


def _cache_path() -> str:
    return os.environ.get("TRI_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "tri_autotune.json"))


def _key(kernel: str, n: int, d: int) -> str:
    return f"{torch.cuda.get_device_name()}|{kernel}|{n}|{d}"


def cand_name(map_id: int, rho: int) -> str:
    return f"{tri.MAP_NAMES[map_id]}/{rho}"


def applicable(kernel: str, map_id: int, n: int, rho: int, d: int = 1) -> bool:
    """Whether a candidate can run at this size (REC needs 2^k block rows)."""
    if map_id == tri.MAP_REC:
        side = {"edm": 4 * rho, "ca": 4 * rho, "at": rho}[kernel]
        m = -(-n // side)
        return m & (m - 1) == 0
    return True


class _Workload:
    """Device buffers for one (kernel, n, d) and a launcher per candidate."""

    def __init__(self, kernel: str, n: int, d: int, seed: int):
        dev = torch.device("cuda")
        self.kernel, self.n, self.d = kernel, n, d
        if kernel == "edm":
            self.x = torch.from_numpy(inputs.edm_normal_points(n, d, seed=seed)).to(dev)
            self.out = torch.empty(n * (n + 1) // 2, dtype=torch.float32, device=dev)
        elif kernel == "ca":
            ld = -(-n // 16) * 16
            self.a = torch.from_numpy(inputs.ca_grid(n, seed=seed, ld=ld)).to(dev)
            self.b = torch.zeros_like(self.a)
        elif kernel == "at":
            self.p = torch.from_numpy(inputs.at_points(n, seed=seed)).to(dev)
            self.e = torch.zeros(1, dtype=torch.float64, device=dev)
            ws = max(tri.tet_at_workspace_size(n, r, m) for r in RHOS for m in MAPS["at"])
            self.ws = torch.empty(ws // 8 + 1, dtype=torch.float64, device=dev)
        else:
            raise ValueError(kernel)

    def launch(self, map_id: int, rho: int):
        if self.kernel == "edm":
            tri.tri_edm(self.x, self.out, map=map_id, rho=rho, reg=0)
        elif self.kernel == "ca":
            tri.tri_ca_step(self.a, self.b, self.n, map=map_id, rho=rho)
        else:
            tri.tet_at_energy(self.p, self.e, 1.0, map_id, rho, self.ws)


def time_candidate(work: _Workload, map_id: int, rho: int, reps: int = 5, warmup: int = 2) -> float:
    """Median milliseconds of one launch of the candidate (CUDA events)."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        work.launch(map_id, rho)
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        work.launch(map_id, rho)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return float(statistics.median(times))


def tune(kernel: str, n: int, d: int = 1, reps: int = 5, seed: int = 1610, use_cache: bool = True,
         rhos=RHOS, maps=None) -> dict:
    """{candidate name: median ms} for every applicable candidate."""
    key = _key(kernel, n, d)
    cache = load_cache() if use_cache else {}
    if key in cache:
        return cache[key]
    work = _Workload(kernel, n, d, seed)
    res = {}
    for m in (maps or MAPS[kernel]):
        for r in rhos:
            if applicable(kernel, m, n, r, d):
                res[cand_name(m, r)] = time_candidate(work, m, r, reps)
    del work
    torch.cuda.empty_cache()
    if use_cache:
        cache[key] = res
        save_cache(cache)
    return res


def best(kernel: str, n: int, d: int = 1, **kw):
    """(map id, rho, ms) of the fastest candidate."""
    res = tune(kernel, n, d, **kw)
    name = min(res, key=res.get)
    mname, rho = name.split("/")
    inv = {v: k for k, v in tri.MAP_NAMES.items()}
    return inv[mname], int(rho), res[name]


# (rho, reg) tiles of the batched launch: reg x reg pairs per thread, 8 x 8 only with rho <= 16
BATCHED_TILES = tuple((r, g) for r in RHOS for g in (1, 2, 4, 8) if not (g == 8 and r > 16))


class _Batched:
    """Device buffers of one batch (instances of sizes `sizes`, d features each)."""

    def __init__(self, sizes, d: int, seed: int):
        dev = torch.device("cuda")
        sizes = np.asarray(sizes, dtype=np.uint32)
        x, pt_off = inputs.batched_points(sizes, d, seed=seed)
        tri_len = sizes.astype(np.int64) * (sizes.astype(np.int64) + 1) // 2
        out_off = np.zeros(len(sizes), dtype=np.uint64)
        out_off[1:] = np.cumsum(tri_len)[:-1]
        self.x = torch.from_numpy(x).to(dev)
        self.pt_off = torch.from_numpy(pt_off.view(np.int64)).to(dev)
        self.n_k = torch.from_numpy(sizes.astype(np.int32)).to(dev)
        self.out_off = torch.from_numpy(out_off.view(np.int64)).to(dev)
        self.out = torch.empty(max(int(tri_len.sum()), 1), dtype=torch.float32, device=dev)
        self.ws = torch.empty(tri.tri_edm_batched_workspace_size(len(sizes)) // 8 + 1, dtype=torch.int64, device=dev)

    def launch(self, rho: int, reg: int):
        tri.tri_edm_batched(self.x, self.pt_off, self.n_k, self.out, self.out_off, rho=rho, reg=reg,
                            workspace=self.ws)


def tune_batched(sizes, d: int, reps: int = 5, seed: int = 1609, use_cache: bool = True,
                 tiles=BATCHED_TILES) -> dict:
    """{"rho/reg": median ms} of the batched launch over every tile, on one
    seeded batch of instances of the given sizes."""
    sizes = np.asarray(sizes, dtype=np.uint32)
    digest = hashlib.sha1(sizes.tobytes()).hexdigest()[:16]
    key = f"{torch.cuda.get_device_name()}|batched|{len(sizes)}|{digest}|{d}"
    cache = load_cache() if use_cache else {}
    if key in cache:
        return cache[key]
    work = _Batched(sizes, d, seed)
    stream = torch.cuda.current_stream()
    res = {}
    for rho, reg in tiles:
        for _ in range(2):
            work.launch(rho, reg)
        times = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            work.launch(rho, reg)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        res[f"{rho}/{reg}"] = float(statistics.median(times))
    del work
    torch.cuda.empty_cache()
    if use_cache:
        cache[key] = res
        save_cache(cache)
    return res


def best_batched(sizes, d: int, **kw):
    """(rho, reg, ms) of the fastest tile of the batched launch."""
    res = tune_batched(sizes, d, **kw)
    name = min(res, key=res.get)
    rho, reg = (int(v) for v in name.split("/"))
    return rho, reg, res[name]


def load_cache(path: str | None = None) -> dict:
    path = path or _cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str | None = None) -> None:
    path = path or _cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


# Sizes of the selector sweep: EDM over N and d, the Life step over n, the
# triplet energy over N.
SWEEP = ([("edm", n, d) for n in (1024, 2048, 4096, 8192, 16384, 32768, 65536) for d in (3, 64, 128)]
         + [("ca", n, 1) for n in (2048, 4096, 8192, 16384, 32768)]
         + [("at", n, 3) for n in (256, 512, 768, 1024, 1280, 1536)])


def sweep(configs=SWEEP, reps: int = 5, log=None) -> dict:
    """Exhaustive timing of every candidate of every configuration.

    Returns {"gpu": name, "reps": reps, "groups": {"kernel|n|d": {cand: ms}}}."""
    out = {"gpu": torch.cuda.get_device_name(), "reps": reps, "groups": {}}
    for kernel, n, d in configs:
        t0 = time.perf_counter()
        out["groups"][f"{kernel}|{n}|{d}"] = tune(kernel, n, d, reps=reps, use_cache=False)
        if log:
            log(f"{kernel} n={n} d={d}: {len(out['groups'][f'{kernel}|{n}|{d}'])} candidates "
                f"in {time.perf_counter() - t0:.1f} s")
    return out
