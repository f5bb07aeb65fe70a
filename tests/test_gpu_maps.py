"""GPU: every map covers its triangular (or tetrahedral) domain exactly once,
and lambda is exact for every omega < 2^32 (Section 3.1, 4.1, 4.2, 6)."""
import math

import numpy as np
import pytest

from gpu_util import dev, tri

pytestmark = pytest.mark.gpu

MAPS = ["LAMBDA", "LAMBDA_PDELTA", "BB", "RB", "REC", "UTM"]


def _count(t, map_id, sq, n, rho, diag):
    import torch
    size = n * (n + 1) // 2 if diag else n * (n - 1) // 2
    out = torch.zeros(max(size, 1) + 64, dtype=torch.int32, device=dev())
    t.tri_map_launch(map_id, sq, n, rho, diag, t.BODY_COUNT, out)
    torch.cuda.synchronize()
    c = out.cpu().numpy()
    return c[:size], c[size:]


@pytest.mark.parametrize("mapname", MAPS)
@pytest.mark.parametrize("rho", [8, 16, 32])
@pytest.mark.parametrize("diag", [True, False])
def test_map_covers_triangle_once(mapname, rho, diag):
    t = tri()
    map_id = getattr(t, "MAP_" + mapname)
    for n in (1, 2, 3, rho - 1, rho, rho + 1, 5 * rho + 3, 37, 1000, 4096):
        if mapname == "REC":
            m = -(-(n - (0 if diag else 1)) // rho)
            if m < 1 or m & (m - 1):
                continue
        counts, guard = _count(t, map_id, t.SQRT_R, n, rho, diag)
        assert np.all(counts == 1), (mapname, n, rho, diag, np.unique(counts))
        assert np.all(guard == 0)


@pytest.mark.parametrize("sq", ["SQRT_X", "SQRT_R", "SQRT_N"])
def test_lambda_sqrt_variants_cover(sq):
    t = tri()
    for n, rho, diag in [(4096, 8, True), (3001, 16, False), (30720, 32, True)]:
        counts, _ = _count(t, t.MAP_LAMBDA, getattr(t, sq), n, rho, diag)
        assert np.all(counts == 1)


@pytest.mark.parametrize("sq", ["SQRT_X", "SQRT_R", "SQRT_N"])
@pytest.mark.parametrize("diag", [True, False])
def test_lambda_exact_for_every_omega_below_2_32(orc, sq, diag):
    import torch
    t = tri()
    res = torch.zeros(6, dtype=torch.int64, device=dev())
    t.tri_lambda_verify(getattr(t, sq), diag, 0, 1 << 32, res)
    torch.cuda.synchronize()
    got = [int(v) & (2 ** 64 - 1) for v in res.cpu().tolist()]
    assert got[0] == 0, f"{got[0]} omegas violate T(i) <= omega < T(i+1)"
    cs = orc.lambda_checksums(1 << 32, with_diag=diag)
    for k, key in enumerate(["sum_i", "sum_j", "sum_ii", "sum_jj", "sum_ij"], start=1):
        assert got[k] == cs[key] % 2 ** 64, key


def test_lambda_block_enumeration_matches_oracle(orc):
    # element level with rho = 8 and n = 8m puts block (bi, bj) at elements
    # [8bi, 8bi+8) x [8bj, 8bj+8): the set of blocks the map launches is the
    # oracle's enumeration of m rows, each exactly once
    t = tri()
    m = 300
    counts, _ = _count(t, t.MAP_LAMBDA, t.SQRT_R, 8 * m, 8, True)
    oi, oj = orc.lambda_enum(m)
    assert len(oi) == m * (m + 1) // 2
    corner = oi.astype(np.int64) * 8
    idx = corner * (corner + 1) // 2 + oj.astype(np.int64) * 8
    assert np.all(counts[idx] == 1) and np.all(counts == 1)


def test_dummy_and_sentinel_bodies_run():
    import torch
    t = tri()
    out = torch.zeros(4, dtype=torch.int32, device=dev())
    for m in (t.MAP_LAMBDA, t.MAP_BB, t.MAP_RB, t.MAP_REC, t.MAP_UTM, t.MAP_LAMBDA_PDELTA):
        t.tri_map_launch(m, t.SQRT_R, 4096, 16, True, t.BODY_SENTINEL, out)
    torch.cuda.synchronize()
    assert int(out[0]) == 0
    t.tri_map_launch(t.MAP_LAMBDA, t.SQRT_R, 4096, 16, True, t.BODY_DUMMY, out)
    torch.cuda.synchronize()
    assert 0 <= int(out[0]) <= 2 * 4095


@pytest.mark.parametrize("mapname", ["LAMBDA", "TET_TABLE", "BB"])
@pytest.mark.parametrize("rho", [8, 16, 32])
def test_tet_map_covers_strict_triplets(rho, mapname):
    # the closed-form cubic, the layer table (Section 7) and the m^3 box each
    # cover every strict triplet exactly once
    import torch
    t = tri()
    map_id = getattr(t, "MAP_" + mapname)
    for n in (1, 2, 3, 4, 17, rho + 1, 100, 300, 8 * rho + 5):
        size = math.comb(n, 3)
        out = torch.zeros(size + 64, dtype=torch.int32, device=dev())
        if mapname == "LAMBDA":
            t.tet_map(n, rho, t.BODY_COUNT, out)
        else:
            t.tet_map_ex(map_id, n, rho, t.BODY_COUNT, out)
        torch.cuda.synchronize()
        c = out.cpu().numpy()
        assert np.all(c[:size] == 1) and np.all(c[size:] == 0), (n, rho)


def test_tet_block_layers_match_oracle(orc):
    # with rho = 8, n = 8m: block (L, R, C) owns triplets with i in [8L, 8L+8),
    # j in [8R, ..), k in [8C, ..); every oracle block of the m-tetrahedron that
    # contains a strict triplet is launched once
    import torch
    t = tri()
    m = 20
    n = 8 * m
    out = torch.zeros(math.comb(n, 3), dtype=torch.int32, device=dev())
    t.tet_map(n, 8, t.BODY_COUNT, out)
    torch.cuda.synchronize()
    c = out.cpu().numpy()
    assert np.all(c == 1)
    L, R, C = orc.tet_enum(m)
    assert len(L) == m * (m + 1) * (m + 2) // 6


def test_tet_map_ex_arguments():
    import torch
    t = tri()
    out = torch.zeros(8, dtype=torch.int32, device=dev())
    for args in ((t.MAP_RB, 100, 16, t.BODY_SENTINEL), (t.MAP_TET_TABLE, 100, 7, t.BODY_SENTINEL),
                 (t.MAP_TET_TABLE, 100, 16, 9)):
        with pytest.raises(t.TriError):
            t.tet_map_ex(*args, out)
    # 2952 layers of blocks is the last count below 2^32 blocks; one more is out of range
    with pytest.raises(t.TriError):
        t.tet_map_ex(t.MAP_TET_TABLE, 8 * 2953, 8, t.BODY_SENTINEL, out)


def _first_error(t, map_id, sq, n_items, begin, end):
    import torch
    fb = torch.full((1,), -1, dtype=torch.int64, device=dev())  # all ones: no failure seen
    t.tri_map_first_error(map_id, sq, n_items, begin, end, fb)
    torch.cuda.synchronize()
    v = int(fb.item()) & (2 ** 64 - 1)
    return None if v == 2 ** 64 - 1 else v


def _exact_rows(w):
    r = ((np.sqrt(8.0 * w.astype(np.float64) + 1.0) - 1.0) // 2).astype(np.int64)
    r -= (r * (r + 1) // 2 > w)
    r += ((r + 1) * (r + 2) // 2 <= w)
    return r


def test_printed_lambda_x_first_error_matches_cpu():
    # Section 4.1's lambda_X taken as printed (FP32 sqrtf, no correction): the
    # GPU's first wrong omega below 2^32 is the first one a step-by-step FP32
    # emulation on the host finds (2 w is exact, the sum and the root round
    # once each, as fmaf and sqrtf do)
    t = tri()
    fx = _first_error(t, t.MAP_LAMBDA, t.SQRT_X, 0, 0, 1 << 32)
    assert fx is not None and fx < 200_000_000
    first = None
    for a in range(0, fx + 1, 1 << 24):
        w = np.arange(a, min(fx + 1, a + (1 << 24)), dtype=np.int64)
        x = np.float32(2.0) * w.astype(np.float32) + np.float32(0.25)
        row = np.floor(np.sqrt(x) - np.float32(0.5)).astype(np.int64)
        bad = np.nonzero(row != _exact_rows(w))[0]
        if len(bad):
            first = int(w[bad[0]])
            break
    assert first == fx


def test_printed_formulas_first_errors_run():
    # the eps variants and UTM as printed: every range call succeeds; UTM is
    # exact for 1000 items (its discriminant stays below 2^24)
    t = tri()
    for sq in (t.SQRT_R, t.SQRT_N):
        f = _first_error(t, t.MAP_LAMBDA, sq, 0, 0, 1 << 32)
        assert f is None or 0 < f < (1 << 32)
    assert _first_error(t, t.MAP_UTM, t.SQRT_X, 1000, 0, 1000 * 999 // 2) is None
    with pytest.raises(t.TriError):
        _first_error(t, t.MAP_UTM, t.SQRT_X, 1000, 0, 1000 * 999 // 2 + 1)
    with pytest.raises(t.TriError):
        _first_error(t, t.MAP_BB, t.SQRT_X, 0, 0, 10)
