"""GPU: bench.py's modes run to completion on small cases and print the line
the measurement contract asks for (the headline on a 4096-point triangle,
the split over ranks at one rank, a profiling case)."""
import json
import os
import subprocess
import sys

import pytest

from gpu_util import dev

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args):
    dev()
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_headline_line_keys():
    d = _bench("--n", "4096", "--d", "128", "--steps", "3", "--warmup", "3", "--no-cpu")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "clocks", "gpu_launches", "e2e"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["gpu_launches"] == 9
    assert d["value"] > 0 and d["roofline"]["frac"] > 0
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in d["roofline"], k
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in d["e2e"], k
    assert d["e2e"]["d2h_bytes_per_step"] == 4 * 4096 * 4097 // 2
    for k in ("sm_mhz", "sm_max_mhz", "reasons"):
        assert k in d["clocks"], k
    assert set(d["paper_maps"]) >= {"edm_n2048_d3_rho16_reg1", "life_n16384_step_rho32", "life_n16384_100steps_run",
                                    "at_energy_n1536_rho32", "edm_batched_1000_d64"}


def test_split_at_one_rank():
    d = _bench("--split", "--n", "4096", "--d", "64", "--steps", "3", "--warmup", "3", "--no-e2e")
    assert d["scaling"] == "strong" and d["band"]["rows"] == [0, 4096] and d["band"]["pairs"] == 4096 * 4097 // 2


def test_profile_case():
    d = _bench("--profile", "life")
    assert d == {"profile_case": "life", "ok": True}
