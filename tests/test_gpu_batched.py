"""GPU: one persistent launch over many uneven EDM triangles matches the
oracle instance by instance (relative error <= 1e-5, exact zeros kept)."""
import numpy as np
import pytest

from gpu_util import dev, rel_err, tri
from paper_1609_01490_gb300 import inputs

pytestmark = pytest.mark.gpu


def _batched(t, sizes, d, rho, reg, seed=5):
    import torch
    x, pt_off = inputs.batched_points(sizes, d, seed=seed)
    tri_len = sizes.astype(np.int64) * (sizes.astype(np.int64) + 1) // 2
    out_off = np.zeros(len(sizes), dtype=np.uint64)
    out_off[1:] = np.cumsum(tri_len)[:-1]
    total = int(tri_len.sum())
    D = dev()
    out = torch.full((total + 64,), -3.0, dtype=torch.float32, device=D)
    ws = torch.empty(t.tri_edm_batched_workspace_size(len(sizes)) // 8 + 1, dtype=torch.int64, device=D)
    t.tri_edm_batched(torch.from_numpy(x).to(D), torch.from_numpy(pt_off.view(np.int64)).to(D),
                      torch.from_numpy(sizes.astype(np.int32)).to(D), out,
                      torch.from_numpy(out_off.view(np.int64)).to(D), rho=rho, reg=reg, workspace=ws)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.all(o[total:] == -3.0)
    return x, pt_off, out_off, o


@pytest.mark.parametrize("rho,reg", [(8, 1), (16, 1), (16, 4), (32, 2)])
def test_batched_matches_oracle(orc, rho, reg):
    t = tri()
    sizes = inputs.batched_sizes(40, lo=1, hi=400, seed=rho * 10 + reg)
    sizes[3] = 0
    sizes[7] = 1
    d = 17
    x, pt_off, out_off, o = _batched(t, sizes, d, rho, reg)
    for k, nk in enumerate(sizes):
        if nk == 0:
            continue
        xk = x[int(pt_off[k]): int(pt_off[k]) + nk]
        got = o[int(out_off[k]): int(out_off[k]) + nk * (nk + 1) // 2]
        assert rel_err(got, orc.edm_packed(xk)) <= 1e-5, k


@pytest.mark.parametrize("rho,reg", [(16, 8), (32, 4), (8, 2)])
def test_batched_pipelined_ragged_features(orc, rho, reg):
    # d = 70: two full 32-feature passes and a 6-feature tail, copied in while
    # the previous pass is computed; instances of 0 and 1 points among them
    t = tri()
    sizes = inputs.batched_sizes(30, lo=1, hi=500, seed=rho + reg)
    sizes[2] = 0
    sizes[5] = 1
    x, pt_off, out_off, o = _batched(t, sizes, 70, rho, reg, seed=11)
    for k, nk in enumerate(sizes):
        nk = int(nk)
        if nk == 0:
            continue
        xk = x[int(pt_off[k]): int(pt_off[k]) + nk]
        got = o[int(out_off[k]): int(out_off[k]) + nk * (nk + 1) // 2]
        assert rel_err(got, orc.edm_packed(xk)) <= 1e-5, (rho, reg, k)


ALL_TILES = [(8, 1), (8, 2), (8, 4), (8, 8), (16, 1), (16, 2), (16, 4), (16, 8), (32, 1), (32, 2), (32, 4)]


@pytest.mark.parametrize("d", [17, 70])
@pytest.mark.parametrize("rho,reg", ALL_TILES)
def test_batched_every_tile_shape(orc, rho, reg, d):
    # instance sizes q S + r (S = rho reg, q = 0, 1, 2) with r stepping through
    # 1 .. S, so that an instance's last row block holds every count of live
    # row groups and its diagonal blocks are both full and ragged; d = 17 is
    # one plain pass, d = 70 the pipelined passes with a 6-feature tail
    t = tri()
    S = rho * reg
    sizes = np.array([S * (k % 3) + r for k, r in enumerate(range(1, S + 1, max(1, rho // 2)))], dtype=np.int64)
    x, pt_off, out_off, o = _batched(t, sizes, d, rho, reg, seed=rho * 100 + reg + d)
    for k, nk in enumerate(sizes):
        nk = int(nk)
        xk = x[int(pt_off[k]): int(pt_off[k]) + nk]
        got = o[int(out_off[k]): int(out_off[k]) + nk * (nk + 1) // 2]
        assert rel_err(got, orc.edm_packed(xk)) <= 1e-5, (rho, reg, d, k, nk)


def test_batched_thousand_instances_every_pair(orc):
    # the 1000-instance batch (N log-uniform in [64, 8192], d = 64, seed 1609):
    # every pair of every instance against the FP64 oracle, at rho = 16 with
    # 8 x 8 pairs per thread (the tuned launch the bench times) and rho = 32
    # with 4 x 4
    t = tri()
    sizes = inputs.batched_sizes(1000, seed=1609)
    tiles = ((16, 8), (32, 4))
    runs = [_batched(t, sizes, 64, rho, reg, seed=1609) for rho, reg in tiles]
    x, pt_off, out_off, _ = runs[0]
    for k, nk in enumerate(sizes):
        nk = int(nk)
        ref = orc.edm_packed(x[int(pt_off[k]): int(pt_off[k]) + nk])
        for tile, (_, _, _, o) in zip(tiles, runs):
            got = o[int(out_off[k]): int(out_off[k]) + nk * (nk + 1) // 2]
            assert rel_err(got, ref) <= 1e-5, (tile, k)
