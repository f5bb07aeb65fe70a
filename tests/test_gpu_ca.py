"""GPU: the triangular Life step is bit-exact against the oracle under every
block map, including ragged sizes, the diagonal and the untouched upper triangle."""
import numpy as np
import pytest

from gpu_util import dev, tri
from paper_1609_01490_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run(t, g, n, steps, map_id, rho, birth=None, survive=None):
    import torch
    a = torch.from_numpy(g).to(dev())
    b = a.clone()
    kw = {}
    if birth is not None:
        kw = dict(birth_mask=birth, survive_mask=survive)
    for s in range(steps):
        src, dst = (a, b) if s % 2 == 0 else (b, a)
        t.tri_ca_step(src, dst, n, map=map_id, rho=rho, **kw)
    torch.cuda.synchronize()
    return (a if steps % 2 == 0 else b).cpu().numpy()


@pytest.mark.parametrize("mapname", ["LAMBDA", "LAMBDA_PDELTA", "BB", "RB", "REC"])
@pytest.mark.parametrize("rho", [8, 16, 32])
def test_ca_bit_exact(orc, mapname, rho):
    t = tri()
    map_id = getattr(t, "MAP_" + mapname)
    S = 4 * rho
    for n in (1, 2, 5, S - 1, S, S + 3, 2 * S, 4 * S, 257):
        if mapname == "REC":
            m = -(-n // S)
            if m & (m - 1):
                continue
        ld = -(-n // 16) * 16 + (16 if n % 3 == 0 else 0)
        g = inputs.ca_grid(n, seed=n + rho, ld=ld)
        iu = np.triu_indices(n, 1)
        g[iu] = 5                         # bytes above the diagonal are outside the domain
        got = _run(t, g, n, 9, map_id, rho)
        ref = orc.ca_run(g, 9)
        assert np.array_equal(got, ref), (mapname, rho, n)
        assert np.all(got[iu] == 5)


def test_ca_other_rule_and_patterns(orc):
    t = tri()
    n = 96
    g = np.zeros((n, n), dtype=np.uint8)
    glider = [(10, 2), (11, 3), (12, 1), (12, 2), (12, 3)]
    for i, j in glider:
        g[i, j] = 1
    got = _run(t, g, n, 40, t.MAP_LAMBDA, 8)
    assert {(int(a), int(b)) for a, b in zip(*np.nonzero(got))} == {(i + 10, j + 10) for i, j in glider}
    g = inputs.ca_grid(200, seed=3, ld=208)
    # HighLife (B36/S23) and a rule with births on 0 neighbours
    for birth, survive in [((1 << 3) | (1 << 6), (1 << 2) | (1 << 3)), (1, 1 << 8)]:
        got = _run(t, g, 200, 3, t.MAP_LAMBDA, 16, birth, survive)
        assert np.array_equal(got, orc.ca_run(g, 3, birth, survive))


def test_ca_rejects_unaligned_buffers():
    # rows are read and written 16 bytes at a time: both buffers must be 16-byte aligned
    import torch
    t = tri()
    a = torch.zeros(64 * 48 + 16, dtype=torch.uint8, device=dev())
    b = torch.zeros_like(a)
    with pytest.raises(t.TriError) as e:
        t.tri_ca_step(a[4:4 + 64 * 48].view(48, 64), b[:64 * 48].view(48, 64), 48)
    assert e.value.status == t.TRI_EINVAL


def test_ca_n16384_one_step(orc):
    # the n = 16384 triangle (134,225,920 cells) of the Life workload: one step, every cell
    t = tri()
    n = 16384
    g = inputs.ca_grid(n, seed=1609)
    ref = orc.ca_step(g)
    # rho = 32 is the tile the bench's Life row times; rho = 16 beside it
    for m, rho in ((t.MAP_LAMBDA, 32), (t.MAP_BB, 32), (t.MAP_RB, 32), (t.MAP_LAMBDA, 16), (t.MAP_BB, 16)):
        got = _run(t, g, n, 1, m, rho)
        assert np.array_equal(got, ref), (m, rho)


def test_ca_hundred_steps(orc):
    t = tri()
    n = 1000
    g = inputs.ca_grid(n, seed=1609, ld=1008)
    ref = orc.ca_run(g, 100)
    for m, rho in ((t.MAP_LAMBDA, 16), (t.MAP_BB, 16), (t.MAP_LAMBDA, 32), (t.MAP_RB, 8)):
        assert np.array_equal(_run(t, g, n, 100, m, rho), ref)


def test_ca_n16384_hundred_steps(orc):
    # the Life workload as configured: the n = 16384 triangle, Bernoulli(0.5)
    # cells, 100 synchronous steps, every cell bit-exact after the last step,
    # under lambda and the bounding box at the tile the bench times (rho = 32)
    t = tri()
    n = 16384
    g = inputs.ca_grid(n, seed=1609)
    ref = orc.ca_run(g, 100)
    for m in (t.MAP_LAMBDA, t.MAP_BB):
        got = _run(t, g, n, 100, m, 32)
        assert np.array_equal(got, ref), m
