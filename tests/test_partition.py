"""CPU: one EDM split across ranks (tri_edm_partition, host code of libtri.so,
no GPU).  The bands are whole 256-row unit rows, disjoint, in rank order and
cover the triangle; their pair counts are within one unit row of an equal
share; and two gloo ranks that each compute their band (here with the FP64
oracle, standing in for the GPU) assemble, on rank 0, exactly the packed
triangle."""
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


@pytest.mark.parametrize("n", [1, 255, 256, 257, 1000, 4096, 20000, 65536, 92681])
@pytest.mark.parametrize("ranks", [1, 2, 3, 4, 7, 8])
def test_partition_covers_in_balanced_bands(t, n, ranks):
    bands = [t.tri_edm_partition(n, ranks, r) for r in range(ranks)]
    assert bands[0][0] == 0 and bands[-1][1] == n
    for (rb, re_, pb, pe), nxt in zip(bands, bands[1:] + [None]):
        assert rb <= re_ and (pb, pe) == (T(rb), T(re_))
        assert (rb % 256 == 0 or rb == n) and (re_ % 256 == 0 or re_ == n)
        if nxt is not None:
            assert nxt[0] == re_  # contiguous, disjoint, in rank order
    total = T(n)
    unit_max = T(n) - T(max(0, n - 256))  # pairs of the largest unit row
    for r, (rb, re_, pb, pe) in enumerate(bands):
        if r > 0:
            # the band starts at the first unit row whose packed offset reaches its share
            share = total * r / ranks
            assert pb >= share or rb == n
            prev = 256 * (-(-rb // 256) - 1)  # the unit row edge before rb
            assert rb == 0 or T(min(n, prev)) < share
        assert abs((pe - pb) - total / ranks) <= unit_max


def test_partition_argument_errors(t):
    for args in [(100, 0, 0), (100, 2, 2)]:
        with pytest.raises(t.TriError) as e:
            t.tri_edm_partition(*args)
        assert e.value.status == t.TRI_EINVAL
    with pytest.raises(t.TriError) as e:
        t.tri_edm_partition(92682, 2, 0)
    assert e.value.status == t.TRI_ERANGE


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, d, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1609_01490_gb300 import inputs, tri
    x = inputs.edm_normal_points(n, d, seed=1609, dup_frac=0.01)
    rb, re_, pb, pe = tri.tri_edm_partition(n, world, rank)
    band = torch.from_numpy(oracle.edm_rows(x, rb, re_))
    assert band.numel() == pe - pb
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([band.numel()], dtype=torch.int64))
    # gloo gathers equal sizes: pad each band to the largest, trim on rank 0
    top = max(int(s.item()) for s in sizes)
    padded = torch.zeros(top, dtype=torch.float64)
    padded[:band.numel()] = band
    if rank == 0:
        parts = [torch.empty(top, dtype=torch.float64) for _ in sizes]
        dist.gather(padded, parts, dst=0)
        whole = torch.cat([p[:int(s.item())] for p, s in zip(parts, sizes)]).numpy()
        q.put((rank, bool(np.array_equal(whole, oracle.edm_packed(x))), [int(s.item()) for s in sizes]))
    else:
        dist.gather(padded, None, dst=0)
        q.put((rank, None, None))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_assemble_the_triangle(t):
    import torch.multiprocessing as mp
    n, d, world = 1500, 16, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, d, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict((r, (ok, sz)) for r, ok, sz in (q.get(timeout=180) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ok, sizes = res[0]
    assert ok and sum(sizes) == T(n) and min(sizes) > 0
