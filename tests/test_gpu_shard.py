"""GPU: the ranks' shares of a split, run one after another on one GPU.

- Life in row bands: each emulated rank holds its own grid whose rows outside
  its band are junk, receives its two halo rows from the neighbouring ranks'
  buffers before every step and steps its band with tri_ca_step_rows; the
  bands assemble tri_ca_step's grid bit for bit, and the step writes no row
  outside its band.
- The Axilrod-Teller energy: each block range's energy matches the oracle's
  energy of the same blocks (1e-5 of their sum of |term|), and the ranges of
  every partition add up to tet_at_energy's result (1e-12 of the sum of
  |term|; only the order of the FP64 additions differs).
- The batched EDM: the ranks' launches over their instances write the same
  bytes as one launch over the batch.
"""
import numpy as np
import pytest

from gpu_util import dev, tri
from paper_1609_01490_gb300 import inputs

pytestmark = pytest.mark.gpu


def _full_life(t, g, n, steps, rho):
    import torch
    a = torch.from_numpy(g).to(dev())
    b = a.clone()
    for _ in range(steps):
        t.tri_ca_step(a, b, n, map=t.MAP_LAMBDA, rho=rho)
        a, b = b, a
    torch.cuda.synchronize()
    return a.cpu().numpy()


def _banded_life(t, g, n, steps, rho, world):
    import torch
    bands = [t.tri_ca_partition(n, rho, world, r) for r in range(world)]

    def owner(row):
        return next(r for r, (b0, b1) in enumerate(bands) if b0 <= row < b1)

    rng = np.random.default_rng(world)
    bufs = []
    for r, (b0, b1) in enumerate(bands):
        junk = rng.integers(0, 256, size=g.shape, dtype=np.uint8)
        a = junk.copy()
        a[b0:b1] = g[b0:b1]
        bufs.append([torch.from_numpy(a).to(dev()), torch.from_numpy(junk).to(dev())])
    for _ in range(steps):
        # halo rows from the owners' current buffers (every rank's step of the
        # previous round has been enqueued on the same stream before)
        for r, (b0, b1) in enumerate(bands):
            if b0 >= b1:
                continue
            if b0 > 0:
                bufs[r][0][b0 - 1].copy_(bufs[owner(b0 - 1)][0][b0 - 1])
            if b1 < n:
                bufs[r][0][b1].copy_(bufs[owner(b1)][0][b1])
        for r, (b0, b1) in enumerate(bands):
            before = bufs[r][1].clone()
            t.tri_ca_step_rows(bufs[r][0], bufs[r][1], n, b0, b1, rho=rho)
            after = bufs[r][1]
            # nothing outside the band's rows is written
            assert torch.equal(before[:b0], after[:b0]) and torch.equal(before[b1:], after[b1:])
        for r in range(world):
            bufs[r].reverse()
    torch.cuda.synchronize()
    out = np.zeros_like(g)
    for r, (b0, b1) in enumerate(bands):
        out[b0:b1] = bufs[r][0][b0:b1].cpu().numpy()
    return out, bands


@pytest.mark.parametrize("rho", [8, 16, 32])
@pytest.mark.parametrize("world", [2, 3, 5])
def test_life_bands_match_the_whole_grid(rho, world):
    t = tri()
    S = 4 * rho
    for n in (S + 1, 3 * S + 5, 1000):
        g = inputs.ca_grid(n, seed=n + world, ld=-(-n // 16) * 16)
        ref = _full_life(t, g, n, 7, rho)
        got, bands = _banded_life(t, g, n, 7, rho, world)
        assert np.array_equal(np.tril(got[:, :n]), np.tril(ref[:, :n])), (rho, world, n, bands)


def test_life_bands_n16384():
    # the full-size grid in four bands, 10 steps, at the bench's rho = 32
    t = tri()
    n = 16384
    g = inputs.ca_grid(n, seed=1609)
    ref = _full_life(t, g, n, 10, 32)
    got, bands = _banded_life(t, g, n, 10, 32, 4)
    assert all(b1 > b0 for b0, b1 in bands)
    assert np.array_equal(np.tril(got), np.tril(ref))


def test_life_band_errors():
    import torch
    t = tri()
    n = 200
    a = torch.zeros((n, 208), dtype=torch.uint8, device=dev())
    b = torch.zeros_like(a)
    for r0, r1 in [(1, 64), (0, 65), (64, 32), (0, 201), (192, 201)]:
        with pytest.raises(t.TriError) as e:
            t.tri_ca_step_rows(a, b, n, r0, r1, rho=16)
        assert e.value.status == t.TRI_EINVAL
    t.tri_ca_step_rows(a, b, n, 64, 64, rho=16)  # empty band
    t.tri_ca_step_rows(a, b, n, 200, 200, rho=16)  # empty band at the end of the grid (partition's last ranks)
    t.tri_ca_step_rows(a, b, n, 192, 200, rho=16)  # ragged last band
    torch.cuda.synchronize()


def _range_energy(t, xyz, w0, w1, rho, map_id, nu=1.0):
    import torch
    e = torch.full((1,), -1.0, dtype=torch.float64, device=dev())
    ws = torch.empty(max(1, w1 - w0), dtype=torch.float64, device=dev())
    t.tet_at_energy_range(xyz, e, w0, w1, nu=nu, map=map_id, rho=rho, workspace=ws)
    torch.cuda.synchronize()
    return float(e.item())


@pytest.mark.parametrize("rho", [8, 16, 32])
def test_at_ranges_match_the_oracle_and_add_up(orc, rho):
    import torch
    t = tri()
    for n in (3, 100, 301):
        p = inputs.at_points(n, seed=1610 + n)
        xyz = torch.from_numpy(p).to(dev())
        _, scale = orc.at_energy(p, nu=0.7)
        whole = torch.zeros(1, dtype=torch.float64, device=dev())
        ws = torch.empty(t.tet_at_workspace_size(n, rho, t.MAP_LAMBDA) // 8 + 1, dtype=torch.float64,
                         device=dev())
        t.tet_at_energy(xyz, whole, 0.7, t.MAP_LAMBDA, rho, ws)
        whole = float(whole.item())
        for ranks in (1, 2, 3, 7):
            for map_id in (t.MAP_LAMBDA, t.MAP_TET_TABLE):
                total = 0.0
                for r in range(ranks):
                    w0, w1 = t.tet_at_partition(n, rho, ranks, r)
                    got = _range_energy(t, xyz, w0, w1, rho, map_id, nu=0.7)
                    ref, rscale = orc.at_energy_blocks(p, rho, w0, w1, nu=0.7)
                    assert abs(got - ref) <= 1e-5 * rscale + 1e-300, (n, rho, ranks, r)
                    total += got
                assert abs(total - whole) <= 1e-12 * scale + 1e-300, (n, rho, ranks, map_id)


def test_at_range_n1536_four_ranks(orc):
    import torch
    t = tri()
    n, rho = 1536, 32
    p = inputs.at_points(n, seed=1610)
    xyz = torch.from_numpy(p).to(dev())
    ref, scale = orc.at_energy(p)
    total = sum(_range_energy(t, xyz, *t.tet_at_partition(n, rho, 4, r), rho, t.MAP_TET_TABLE) for r in range(4))
    assert abs(total - ref) <= 1e-5 * scale


def test_at_range_errors():
    import torch
    t = tri()
    xyz = torch.zeros((50, 3), dtype=torch.float32, device=dev())
    e = torch.zeros(1, dtype=torch.float64, device=dev())
    ws = torch.empty(64, dtype=torch.float64, device=dev())
    m = -(-50 // 8)
    Tm = m * (m + 1) * (m + 2) // 6
    for w0, w1, mp in [(5, 4, t.MAP_LAMBDA), (0, Tm + 1, t.MAP_LAMBDA), (0, 4, t.MAP_BB)]:
        with pytest.raises(t.TriError) as err:
            t.tet_at_energy_range(xyz, e, w0, w1, map=mp, rho=8, workspace=ws)
        assert err.value.status == t.TRI_EINVAL
    with pytest.raises(t.TriError) as err:
        t.tet_at_energy_range(xyz, e, 0, Tm, map=t.MAP_LAMBDA, rho=8, workspace=ws[:Tm - 1])
    assert err.value.status == t.TRI_ENOSPACE
    assert _range_energy(t, xyz, 7, 7, 8, t.MAP_LAMBDA) == 0.0


@pytest.mark.parametrize("d", [17, 70])
@pytest.mark.parametrize("rho,reg", [(16, 8), (32, 4), (8, 2)])
def test_batched_shards_write_the_batch(rho, reg, d):
    import torch
    from paper_1609_01490_gb300 import shard
    t = tri()
    sizes = inputs.batched_sizes(60, lo=1, hi=700, seed=rho + reg + d)
    sizes[4] = 0
    x, pt_off = inputs.batched_points(sizes, d, seed=3)
    tl = sizes.astype(np.int64) * (sizes.astype(np.int64) + 1) // 2
    oo = np.zeros(len(sizes), dtype=np.uint64)
    oo[1:] = np.cumsum(tl)[:-1]
    D = dev()
    xd = torch.from_numpy(x).to(D)
    ptd = torch.from_numpy(pt_off.view(np.int64)).to(D)
    nkd = torch.from_numpy(sizes.astype(np.int32)).to(D)
    ood = torch.from_numpy(oo.view(np.int64)).to(D)
    ws = torch.empty(t.tri_edm_batched_workspace_size(len(sizes)) // 8 + 1, dtype=torch.int64, device=D)
    whole = torch.full((int(tl.sum()),), -1.0, device=D)
    t.tri_edm_batched(xd, ptd, nkd, whole, ood, rho=rho, reg=reg, workspace=ws)
    for world in (1, 2, 3, 4):
        out = torch.full_like(whole, -1.0)
        ranges = [shard.batched_sharded(xd, ptd, nkd, sizes, out, ood, r, world, rho=rho, reg=reg, workspace=ws)
                  for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == len(sizes)
        torch.cuda.synchronize()
        assert torch.equal(out, whole), (world, ranges)
