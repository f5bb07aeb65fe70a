"""GPU: collision detection of N spheres (Section 5, test 3) is bit-exact
against the oracle under every map, tile shape and dimension: the number of
colliding pairs, every per-sphere count, and the pair set (the kernel lists
pairs in no particular order, so both lists are sorted before comparing).
Both sides take the FP32 test s <= (r_i + r_j)^2 with the same operations,
so there is no tolerance."""
import ctypes

import numpy as np
import pytest

from gpu_util import dev, tri
from paper_1609_01490_gb300 import inputs

pytestmark = pytest.mark.gpu
CONFIGS = [(8, 1), (8, 4), (8, 8), (16, 1), (16, 4), (16, 8), (32, 1), (32, 4)]


def _run(c, r, map_id=None, rho=16, reg=0, cap=None, want_count=True):
    import torch
    t = tri()
    D = dev()
    n = c.shape[0]
    cd = torch.from_numpy(np.ascontiguousarray(c)).to(D)
    rd = torch.from_numpy(np.ascontiguousarray(r)).to(D)
    npairs = torch.full((1,), 12345, dtype=torch.int64, device=D)
    count = torch.full((n,), 7, dtype=torch.int32, device=D) if want_count else None
    cap = 10 * n + 64 if cap is None else cap  # above the pair count of every workload here
    pairs = torch.zeros((cap, 2), dtype=torch.int32, device=D) if cap > 0 else None
    t.tri_collide(cd, rd, npairs, count=count, pairs=pairs, map=t.MAP_LAMBDA if map_id is None else map_id,
                  rho=rho, reg=reg)
    torch.cuda.synchronize()
    tot = int(npairs.item())
    cnt = count.cpu().numpy().astype(np.uint32) if want_count else None
    pl = pairs[:min(tot, cap)].cpu().numpy().astype(np.int64) if cap > 0 else np.zeros((0, 2), np.int64)
    return tot, cnt, pl


def _sorted_pairs(pl, n):
    key = np.sort(pl[:, 0] * n + pl[:, 1])
    return key // n, key % n


def _check(orc, c, r, **kw):
    n = c.shape[0]
    cnt_ref, pi, pj = orc.collide_counts(c, r)
    tot, cnt, pl = _run(c, r, **kw)
    assert tot == len(pi)
    np.testing.assert_array_equal(cnt, cnt_ref)
    gi, gj = _sorted_pairs(pl, n)
    np.testing.assert_array_equal(gi, pi)
    np.testing.assert_array_equal(gj, pj)
    return tot


@pytest.mark.parametrize("mapname", ["LAMBDA", "LAMBDA_PDELTA", "BB", "RB", "REC", "UTM"])
@pytest.mark.parametrize("dim", [1, 2, 3])
def test_collide_bit_exact(orc, mapname, dim):
    t = tri()
    map_id = getattr(t, "MAP_" + mapname)
    total = 0
    for rho, reg in CONFIGS:
        S = rho * reg
        for n in (1, 2, S - 1, S + 3, 2 * S, 4 * S, 700):
            if mapname == "REC":
                m = -(-n // S)
                if m & (m - 1):
                    continue
            # denser than the bench workload so that small cases collide
            c, r = inputs.spheres(n, dim, kappa=12.0, seed=n * 7 + rho + reg + dim)
            total += _check(orc, c, r, map_id=map_id, rho=rho, reg=reg)
    assert total > 1000


@pytest.mark.parametrize("dim", [1, 3])
def test_collide_touching_lattice(orc, dim):
    # exact ties: lattice spheres touch their axis neighbours (distance h = 2 r)
    import itertools
    k = 12 if dim == 3 else 300
    pts = np.array(list(itertools.product(range(k), repeat=dim)))
    c = (pts / 16.0).astype(np.float32)
    r = np.full(len(pts), 1 / 32, dtype=np.float32)
    for map_id in (tri().MAP_LAMBDA, tri().MAP_BB, tri().MAP_UTM):
        for rho, reg in ((16, 4), (8, 1), (16, 8)):
            tot = _check(orc, c, r, map_id=map_id, rho=rho, reg=reg)
            assert tot == dim * k ** (dim - 1) * (k - 1)


def test_collide_edge_cases(orc):
    t = tri()
    # coincident zero-radius spheres all touch
    c = np.full((130, 3), 0.5, dtype=np.float32)
    tot, cnt, _ = _run(c, np.zeros(130, np.float32), cap=130 * 129 // 2)
    assert tot == 130 * 129 // 2 and np.all(cnt == 129)
    # list overflow: the total is still exact, the list holds cap distinct true pairs
    c, r = inputs.spheres(3000, 3, kappa=10.0, seed=3)
    _, pi, pj = orc.collide_counts(c, r)
    cap = len(pi) // 3
    tot, cnt, pl = _run(c, r, cap=cap)
    assert tot == len(pi) and len(pl) == cap
    truth = set(zip(pi.tolist(), pj.tolist()))
    got = set(map(tuple, pl.tolist()))
    assert len(got) == cap and got <= truth
    # counts alone, list alone
    tot2, cnt2, _ = _run(c, r, cap=0)
    assert tot2 == len(pi)
    tot3, cnt3, pl3 = _run(c, r, cap=len(pi) + 10, want_count=False)
    assert tot3 == len(pi) and cnt3 is None and len(pl3) == len(pi)
    # n = 0 zeroes the pair count
    import torch
    z = torch.full((1,), 99, dtype=torch.int64, device=dev())
    t.tri_collide(torch.zeros((0, 3), device=dev()), torch.zeros(0, device=dev()), z)
    assert int(z.item()) == 0


def test_collide_argument_errors():
    import torch
    t = tri()
    D = dev()
    c = torch.zeros((10, 3), device=D)
    r = torch.zeros(10, device=D)
    np_ = torch.zeros(1, dtype=torch.int64, device=D)
    for kw in (dict(rho=7), dict(reg=2), dict(rho=32, reg=8), dict(map=9)):
        with pytest.raises(t.TriError):
            t.tri_collide(c, r, np_, **kw)
    with pytest.raises(t.TriError):
        t.tri_collide(torch.zeros((10, 4), device=D), r, np_)
    with pytest.raises(t.TriError):  # REC needs a power-of-two block count: 300 spheres in tiles of 64 -> 5
        t.tri_collide(torch.zeros((300, 3), device=D), torch.zeros(300, device=D), np_, map=t.MAP_REC)
    L = ctypes.CDLL(t.LIB_PATH).tri_collide
    L.restype = ctypes.c_int
    vp = ctypes.c_void_p
    L.argtypes = [vp, vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32, vp, vp,
                  ctypes.c_uint64, vp, vp]
    assert L(c.data_ptr(), r.data_ptr(), 10, 3, 0, 16, 4, None, None, 0, None, None) == t.TRI_EINVAL
    assert L(c.data_ptr(), r.data_ptr(), 10, 3, 0, 16, 4, None, None, 5, np_.data_ptr(), None) == t.TRI_EINVAL
    assert L(c.data_ptr(), r.data_ptr(), 10, 0, 0, 16, 4, None, None, 0, np_.data_ptr(), None) == t.TRI_EINVAL


@pytest.mark.parametrize("dim", [1, 3])
def test_collide_full_size(orc, dim):
    # the bench's workload: 65,536 spheres, about 4 contacts each, lambda with
    # 16 x 16 threads of 8 x 8 pairs (the default); every pair of the 2^31 tested
    n = 65536
    c, r = inputs.spheres(n, dim)
    tot = _check(orc, c, r, map_id=tri().MAP_LAMBDA, rho=16, reg=0, cap=4 * n)
    assert 3.0 * n / 2 < tot < 4.5 * n / 2
