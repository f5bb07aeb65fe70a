"""The C ABI library builds, loads and exports every entry point of include/tri.h (no GPU calls)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tri.h")).read()
    return sorted(set(re.findall(r"^TRI_API\s+[\w\s\*]*?\b((?:tri|tet)_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1609_01490_gb300 import build
    build.build()
    return build.LIB


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("tri_map_launch", "tri_edm", "tri_ca_step", "tet_map", "tet_at_energy", "tri_edm_batched",
                 "tri_mlp_grad", "tri_lambda_verify"):
        assert must in names


def test_exports_match_header(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(_declared()) <= exported
    # nothing but the declared entry points leaks out of the library
    assert {e for e in exported if e.startswith(("tri_", "tet_"))} == set(_declared())


def test_binding_loads_without_gpu(lib):
    pytest.importorskip("torch")
    from paper_1609_01490_gb300 import tri
    assert tri.tri_version() == 10000
    assert set(tri.EXPORTS) >= set(_declared())
    assert tri.tri_edm_workspace_size(100, 3, tri.FP32) == 0
    assert tri.tet_at_workspace_size(96, 8) == 8 * (12 * 13 * 14 // 6)
    assert tri.tri_edm_batched_workspace_size(10) >= 8 * 11
    with pytest.raises(tri.TriError):
        tri.tet_at_workspace_size(96, 7)


def test_host_side_argument_errors(lib):
    # argument checks run on the host before any launch, so they need no GPU
    import ctypes
    L = ctypes.CDLL(lib)
    L.tri_map_launch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    dummy = ctypes.c_void_p(16)
    assert L.tri_map_launch(0, 1, 100, 7, 1, 0, dummy, None) == 1          # rho 7
    assert L.tri_map_launch(0, 1, 0, 16, 1, 0, dummy, None) == 1           # n = 0
    assert L.tri_map_launch(0, 1, 100, 16, 1, 0, None, None) == 1          # null out
    assert L.tri_map_launch(9, 1, 100, 16, 1, 0, dummy, None) == 1         # unknown map
    assert L.tri_map_launch(3, 1, 100, 16, 1, 0, dummy, None) == 2         # REC needs 2^k blocks
    assert L.tri_map_launch(0, 1, 4000000, 8, 1, 0, dummy, None) == 2      # > 2^32 blocks
    L.tri_ca_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_size_t,
                              ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p]
    assert L.tri_ca_step(dummy, dummy, 64, 64, 8, 12, 0, 16, None) == 1   # aliasing
    assert L.tri_ca_step(ctypes.c_void_p(4096), ctypes.c_void_p(1 << 20), 64, 60, 8, 12, 0, 16, None) == 1  # ld
    L.tri_status_string.restype = ctypes.c_char_p
    assert b"TRI_ERANGE" in L.tri_status_string(2)


def test_host_side_argument_errors_of_the_later_calls(lib):
    # every one of these is rejected on the host before any CUDA call
    import ctypes
    L = ctypes.CDLL(lib)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    dummy = vp(4096)
    L.tri_collide.argtypes = [vp, vp, u32, u32, i32, u32, u32, vp, vp, u64, vp, vp]
    assert L.tri_collide(dummy, dummy, 100, 3, 0, 16, 0, None, None, 0, None, None) == 1     # no n_pairs
    assert L.tri_collide(dummy, dummy, 100, 4, 0, 16, 0, None, None, 0, dummy, None) == 1    # dim 4
    assert L.tri_collide(dummy, dummy, 100, 3, 0, 16, 2, None, None, 0, dummy, None) == 1    # reg 2
    assert L.tri_collide(dummy, dummy, 100, 3, 0, 32, 8, None, None, 0, dummy, None) == 1    # 8 x 8 at rho 32
    assert L.tri_collide(dummy, dummy, 100, 3, 6, 16, 0, None, None, 0, dummy, None) == 1    # tetrahedral map
    assert L.tri_collide(dummy, dummy, 100, 3, 0, 16, 0, None, None, 5, dummy, None) == 1    # cap, no list
    # block counts beyond the map's range are refused before the device is touched, also
    # where n + tile - 1 would wrap around 2^32
    assert L.tri_collide(dummy, dummy, 0xFFFFFFF0, 3, 0, 16, 0, None, None, 0, dummy, None) == 2  # lambda
    assert L.tri_collide(dummy, dummy, 65535 * 128 + 1, 3, 1, 16, 0, None, None, 0, dummy, None) == 2  # BB
    assert L.tri_collide(dummy, dummy, 100000, 3, 4, 16, 0, None, None, 0, dummy, None) == 2  # UTM threads
    assert L.tri_collide(dummy, dummy, 300, 3, 3, 16, 0, None, None, 0, dummy, None) == 2    # REC, 3 rows
    L.tet_map_ex.argtypes = [i32, u32, u32, i32, vp, vp]
    assert L.tet_map_ex(2, 100, 16, 1, dummy, None) == 1     # RB is not a tetrahedral map
    assert L.tet_map_ex(6, 100, 12, 1, dummy, None) == 1     # rho 12
    assert L.tet_map_ex(6, 8 * 2953, 8, 1, dummy, None) == 2  # 2953 layers exceed 2^32 blocks
    L.tri_map_first_error.argtypes = [i32, i32, u64, u64, u64, vp, vp]
    assert L.tri_map_first_error(0, 0, 0, 0, 10, None, None) == 1          # no result word
    assert L.tri_map_first_error(0, 0, 0, 0, (1 << 32) + 1, dummy, None) == 2
    assert L.tri_map_first_error(4, 0, 1000, 0, 1000 * 999 // 2 + 1, dummy, None) == 2
    assert L.tri_map_first_error(1, 0, 0, 0, 10, dummy, None) == 1          # BB has no printed formula
    L.tri_peak_probe.argtypes = [i32, u32, u32, vp, vp, vp]
    assert L.tri_peak_probe(3, 1, 1, dummy, dummy, None) == 1
    L.tet_at_workspace_size.argtypes = [u32, u32, i32, ctypes.POINTER(ctypes.c_size_t)]
    n = ctypes.c_size_t(0)
    assert L.tet_at_workspace_size(96, 16, 6, ctypes.byref(n)) == 0 and n.value == 8 * (6 * 7 * 8 // 6)


def test_host_side_argument_errors_of_tri_ca_run(lib):
    # rejected on the host before any CUDA call: null or misaligned buffers, a
    # leading dimension below n or not a multiple of 16, steps = 0, rule masks
    # past 8 neighbours, a map without a 2-D block grid, overlapping buffers and
    # a missing scratch when more than one pass is needed (over 16 steps for
    # Conway's rule at rho = 32, over 1 otherwise)
    import ctypes
    L = ctypes.CDLL(lib)
    vp, u32, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int
    L.tri_ca_run.argtypes = [vp, vp, vp, u32, ctypes.c_size_t, u32, u32, i32, u32, u32, vp]
    n, ld = 200, 208
    span = (n - 1) * ld + n
    a, b, c = 1 << 20, 1 << 24, 1 << 28  # 16-byte aligned, far apart: never dereferenced
    life = (8, 12)
    assert L.tri_ca_run(None, vp(b), vp(c), n, ld, *life, 0, 32, 3, None) == 1            # null in
    assert L.tri_ca_run(vp(a), None, vp(c), n, ld, *life, 0, 32, 3, None) == 1            # null out
    assert L.tri_ca_run(vp(a), vp(b), vp(c), 0, ld, *life, 0, 32, 3, None) == 1           # n = 0
    assert L.tri_ca_run(vp(a), vp(b), vp(c), n, ld, *life, 0, 32, 0, None) == 1           # steps = 0
    assert L.tri_ca_run(vp(a), vp(b), vp(c), n, ld, *life, 0, 12, 3, None) == 1           # rho 12
    assert L.tri_ca_run(vp(a), vp(b), vp(c), n, 192, *life, 0, 32, 3, None) == 1          # ld < n
    assert L.tri_ca_run(vp(a), vp(b), vp(c), n, 200, *life, 0, 32, 3, None) == 1          # ld % 16
    assert L.tri_ca_run(vp(a + 4), vp(b), vp(c), n, ld, *life, 0, 32, 3, None) == 1       # misaligned in
    assert L.tri_ca_run(vp(a), vp(b), vp(c), n, ld, 1 << 9, 12, 0, 32, 3, None) == 1      # birth past 8
    assert L.tri_ca_run(vp(a), vp(b), vp(c), n, ld, *life, 4, 32, 3, None) == 1           # UTM
    assert L.tri_ca_run(vp(a), vp(a + span - 16), vp(c), n, ld, *life, 0, 32, 3, None) == 1  # out overlaps in
    assert L.tri_ca_run(vp(a), vp(b), None, n, ld, *life, 0, 32, 17, None) == 1           # 2 passes, no scratch
    assert L.tri_ca_run(vp(a), vp(b), vp(b + 16), n, ld, *life, 0, 32, 17, None) == 1     # scratch overlaps out
    assert L.tri_ca_run(vp(a), vp(b), None, n, ld, *life, 0, 16, 2, None) == 1            # rho 16 steps one at a time
    assert L.tri_ca_run(vp(a), vp(b), None, n, ld, 8 | 64, 12, 0, 32, 2, None) == 1       # another rule, likewise
