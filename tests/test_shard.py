"""CPU: the splits of the batched EDM, the cellular automaton and the
Axilrod-Teller energy across ranks (host code of libtri.so and the
torch.distributed driver in shard.py, no GPU).

- The partitions are contiguous, disjoint, in rank order, cover their domain
  and are balanced to within one unit of work.
- The oracle's block-range energy is pinned: each block's energy is the sum of
  the three-point energies of its triplets, the block found through
  tet_enum's order, and ranges that partition the blocks add up to the whole.
- gloo ranks run shard.py's drivers with the oracle standing in for the GPU
  (a rank's grid is poisoned outside its band and halo rows) and reach the
  oracle's single-process results: the Life grid after 12 steps exactly, the
  energy to 1e-12 of the sum of |term|.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def t():
    pytest.importorskip("torch")
    from paper_1609_01490_gb300 import build
    build.build()
    from paper_1609_01490_gb300 import tri
    return tri


def T(i):
    return i * (i + 1) // 2


def T3(i):
    return i * (i + 1) * (i + 2) // 6


# ------------------------------------------------------------ partitions ----
@pytest.mark.parametrize("n", [1, 31, 32, 33, 500, 4096, 16384, 20001])
@pytest.mark.parametrize("rho", [8, 32])
@pytest.mark.parametrize("ranks", [1, 2, 3, 5, 8])
def test_ca_partition_whole_block_rows_balanced(t, n, rho, ranks):
    S = 4 * rho
    m = -(-n // S)
    bands = [t.tri_ca_partition(n, rho, ranks, r) for r in range(ranks)]
    assert bands[0][0] == 0 and bands[-1][1] == n
    for (b0, b1), nxt in zip(bands, bands[1:] + [None]):
        assert b0 <= b1
        assert b0 % S == 0 or b0 == n
        assert b1 % S == 0 or b1 == n
        if nxt is not None:
            assert nxt[0] == b1
    tiles = [T(-(-b1 // S)) - T(-(-b0 // S)) for b0, b1 in bands]
    assert sum(tiles) == T(m)
    for k in tiles:
        assert abs(k - T(m) / ranks) <= m  # within one block row of an equal share


@pytest.mark.parametrize("n", [1, 7, 100, 1536, 4000])
@pytest.mark.parametrize("rho", [8, 16, 32])
@pytest.mark.parametrize("ranks", [1, 2, 3, 7, 8])
def test_at_partition_equal_block_ranges(t, n, rho, ranks):
    m = -(-n // rho)
    rng = [t.tet_at_partition(n, rho, ranks, r) for r in range(ranks)]
    assert rng[0][0] == 0 and rng[-1][1] == T3(m)
    for (w0, w1), nxt in zip(rng, rng[1:] + [None]):
        assert w1 - w0 in (T3(m) // ranks, T3(m) // ranks + 1)
        if nxt is not None:
            assert nxt[0] == w1


@pytest.mark.parametrize("ranks", [1, 2, 3, 8, 40])
@pytest.mark.parametrize("rho,reg", [(16, 8), (32, 4), (8, 1)])
def test_batched_partition_whole_instances(t, ranks, rho, reg):
    from paper_1609_01490_gb300 import inputs
    sizes = inputs.batched_sizes(200, lo=1, hi=3000, seed=7)
    sizes[5] = 0
    S = rho * reg
    blocks = np.array([T(-(-int(s) // S)) for s in sizes])
    parts = [t.tri_edm_batched_partition(sizes, rho, reg, ranks, r) for r in range(ranks)]
    assert parts[0][0] == 0 and parts[-1][1] == len(sizes)
    for (k0, k1), nxt in zip(parts, parts[1:] + [None]):
        assert k0 <= k1
        if nxt is not None:
            assert nxt[0] == k1
    total = blocks.sum()
    for k0, k1 in parts:
        assert abs(blocks[k0:k1].sum() - total / ranks) <= blocks.max()


def test_partition_argument_errors(t):
    for call, args in [(t.tri_ca_partition, (100, 8, 0, 0)), (t.tri_ca_partition, (100, 8, 2, 2)),
                       (t.tri_ca_partition, (100, 12, 2, 0)), (t.tet_at_partition, (100, 8, 0, 0)),
                       (t.tet_at_partition, (100, 8, 3, 3)), (t.tet_at_partition, (100, 7, 1, 0))]:
        with pytest.raises(t.TriError) as e:
            call(*args)
        assert e.value.status == t.TRI_EINVAL
    with pytest.raises(t.TriError) as e:
        t.tet_at_partition(2954 * 32, 32, 2, 0)  # T3(2954) >= 2^32 blocks
    assert e.value.status == t.TRI_ERANGE
    for args in [([10, 20], 16, 8, 0, 0), ([10, 20], 16, 8, 2, 2), ([10, 20], 32, 8, 1, 0),
                 ([10, 20], 16, 3, 1, 0)]:
        with pytest.raises(t.TriError) as e:
            t.tri_edm_batched_partition(*args)
        assert e.value.status == t.TRI_EINVAL
    assert t.tri_edm_batched_partition([], 16, 8, 3, 1) == (0, 0)


# ------------------------------------------------------ oracle pins ----
def test_at_energy_blocks_is_the_sum_of_its_triplets():
    import oracle
    rng = np.random.default_rng(11)
    n, rho = 19, 4
    p = (rng.random((n, 3)) * 2.5).astype(np.float32)
    L, R, C = oracle.tet_enum(-(-n // rho))
    number = {(int(a), int(b), int(c)): w for w, (a, b, c) in enumerate(zip(L, R, C))}
    per_block = np.zeros(len(L))
    for i in range(n):
        for j in range(i):
            for k in range(j):
                e, _ = oracle.at_energy(p[[k, j, i]])  # one triplet
                per_block[number[(i // rho, j // rho, k // rho)]] += e
    for w in range(len(L)):
        e, _ = oracle.at_energy_blocks(p, rho, w, w + 1)
        assert abs(e - per_block[w]) <= 1e-12 * max(1.0, abs(per_block[w])), w


def test_at_energy_blocks_ranges_add_up():
    import oracle
    from paper_1609_01490_gb300 import inputs
    p = inputs.at_points(150, seed=5)
    rho = 8
    Tm = T3(-(-150 // rho))
    whole, asum = oracle.at_energy(p)
    assert oracle.at_energy_blocks(p, rho, 0, Tm) == (whole, asum)  # same terms, same order
    edges = [0, 1, 37, 38, 400, Tm - 1, Tm]
    parts = [oracle.at_energy_blocks(p, rho, a, b)[0] for a, b in zip(edges, edges[1:])]
    assert abs(sum(parts) - whole) <= 1e-12 * asum
    assert oracle.at_energy_blocks(p, rho, 5, 5) == (0.0, 0.0)


# --------------------------------------------------------- gloo ranks ----
def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _ca_rank(rank, world, port, n, rho, steps, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1609_01490_gb300 import inputs, shard, tri
    g0 = inputs.ca_grid(n, seed=1609)
    b0, b1 = tri.tri_ca_partition(n, rho, world, rank)
    # this rank holds only its band: every other row is junk
    junk = np.random.default_rng(100 + rank).integers(0, 2, size=g0.shape, dtype=np.uint8)
    a = junk.copy()
    a[b0:b1] = g0[b0:b1]
    a, b = torch.from_numpy(a), torch.from_numpy(junk.copy())

    def step_rows(src, dst, r0, r1):
        # rows r0 .. r1 - 1 of one oracle step depend on rows r0 - 1 .. r1 only
        dst[r0:r1] = torch.from_numpy(oracle.ca_step(src.numpy())[r0:r1])

    a, band = shard.ca_run_bands(a, b, n, steps, rank, world, rho=rho, step_rows=step_rows)
    rows = a[band[0]:band[1]].clone()
    got = [None] * world
    dist.all_gather_object(got, (band, rows.numpy()))
    if rank == 0:
        ref = oracle.ca_run(g0, steps)
        whole = np.concatenate([r for _, r in got])
        ok = whole.shape == ref.shape and bool(np.array_equal(np.tril(whole), np.tril(ref)))
        q.put((rank, ok, [bd for bd, _ in got]))
    else:
        q.put((rank, None, None))
    dist.barrier()
    dist.destroy_process_group()


def _at_rank(rank, world, port, n, rho, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1609_01490_gb300 import inputs, shard
    p = inputs.at_points(n, seed=1610)

    def energy_range(xyz, e, w0, w1):
        e[0] = oracle.at_energy_blocks(xyz.numpy(), rho, w0, w1)[0]

    e = shard.at_energy_sharded(torch.from_numpy(p), rank, world, rho=rho, energy_range=energy_range)
    whole, asum = oracle.at_energy(p)
    q.put((rank, abs(float(e.item()) - whole) <= 1e-12 * asum, None))
    dist.barrier()
    dist.destroy_process_group()


def _spawn(target, world, *args):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, *args, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict((r, (ok, extra)) for r, ok, extra in (q.get(timeout=300) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_run_life_in_bands(t, world):
    n, rho, steps = 300, 8, 12  # 32-row block rows: bands of whole block rows
    res = _spawn(_ca_rank, world, n, rho, steps)
    ok, bands = res[0]
    assert ok
    assert all(b1 > b0 for b0, b1 in bands)


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_add_the_energy(t, world):
    res = _spawn(_at_rank, world, 120, 8)
    assert all(ok for ok, _ in res.values())
