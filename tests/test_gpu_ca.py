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
        # the same 100 steps in passes of up to 16 steps (tri_ca_run)
        assert np.array_equal(_run_fused(t, g, n, 100, m, 32), ref), ("run", m)


def _run_fused(t, g, n, steps, map_id, rho, birth=None, survive=None):
    import torch
    D = dev()
    a = torch.from_numpy(g).to(D)
    out = a.clone()        # the bytes outside the domain must come back unchanged
    scratch = torch.full_like(a, 7)
    kw = {}
    if birth is not None:
        kw = dict(birth_mask=birth, survive_mask=survive)
    t.tri_ca_run(a, out, n, steps, scratch=scratch, map=map_id, rho=rho, **kw)
    torch.cuda.synchronize()
    assert torch.equal(a.cpu(), torch.from_numpy(g))  # the input is only read
    return out.cpu().numpy()


@pytest.mark.parametrize("mapname", ["LAMBDA", "LAMBDA_PDELTA", "BB", "RB", "REC"])
def test_ca_run_fused_matches_the_oracle(orc, mapname):
    # Conway's rule at rho = 32 runs up to 16 steps per pass: step counts below,
    # at and across a pass, sizes around the 128-cell tile and sizes with tiles
    # whose 16-cell halo lies wholly inside the domain (n >= 1000), a padded leading
    # dimension and junk above the diagonal (outside the domain)
    t = tri()
    map_id = getattr(t, "MAP_" + mapname)
    for n in (1, 5, 127, 128, 129, 300, 1000, 1024, 2500):
        m = -(-n // 128)
        if mapname == "REC" and m & (m - 1):
            continue
        ld = -(-n // 16) * 16 + (16 if n % 3 == 0 else 0)
        g = inputs.ca_grid(n, seed=n + 3, ld=ld)
        g[np.triu_indices(n, 1)] = 5
        g[:, n:] = 9
        for steps in (1, 3, 8, 15, 16, 17, 33):
            got = _run_fused(t, g, n, steps, map_id, 32)
            assert np.array_equal(got, orc.ca_run(g, steps)), (mapname, n, steps)


def test_ca_run_any_nonzero_byte_is_alive(orc):
    # a cell is alive when its byte is non-zero: live cells carry bytes with
    # every bit pattern that the byte-to-bit packing must map to 1 (0x01, 0x7F,
    # 0x80, 0x81, 0xFF and random ones), in tiles inside the domain and on its
    # edges, for one step, one pass and across passes
    t = tri()
    rng = np.random.default_rng(1609)
    for n in (300, 1000):
        g = inputs.ca_grid(n, seed=n + 11, ld=-(-n // 16) * 16)
        live = g != 0
        vals = rng.choice(np.array([0x01, 0x7F, 0x80, 0x81, 0xFF, 0x10, 0x02, 0x40], dtype=np.uint8), size=g.shape)
        rnd = rng.integers(1, 256, size=g.shape, dtype=np.uint8)
        vals = np.where(rng.random(g.shape) < 0.5, vals, rnd)
        g = np.where(live, vals, 0).astype(np.uint8)
        for map_id in (t.MAP_LAMBDA, t.MAP_BB):
            for steps in (1, 16, 17):
                got = _run_fused(t, g, n, steps, map_id, 32)
                assert np.array_equal(got, orc.ca_run(g, steps)), (n, map_id, steps)


def test_ca_run_other_rules_and_tiles(orc):
    # rules other than Conway's and tiles other than rho = 32 step one launch at a time
    t = tri()
    n = 300
    g = inputs.ca_grid(n, seed=11, ld=304)
    highlife = ((1 << 3) | (1 << 6), (1 << 2) | (1 << 3))
    for rho, rule in ((16, None), (8, None), (32, highlife), (16, highlife)):
        b, s_ = rule if rule else (None, None)
        got = _run_fused(t, g, n, 11, t.MAP_LAMBDA, rho, b, s_)
        ref = orc.ca_run(g, 11, *rule) if rule else orc.ca_run(g, 11)
        assert np.array_equal(got, ref), (rho, rule)


def test_ca_run_errors():
    import torch
    t = tri()
    n = 200
    a = torch.zeros((n, 208), dtype=torch.uint8, device=dev())
    b, c = torch.zeros_like(a), torch.zeros_like(a)
    cases = [dict(steps=0, scratch=c), dict(steps=17, scratch=None), dict(steps=17, scratch=a),
             dict(steps=3, scratch=c, map=t.MAP_UTM)]
    for kw in cases:
        with pytest.raises(t.TriError) as e:
            t.tri_ca_run(a, b, n, **kw)
        assert e.value.status == t.TRI_EINVAL, kw
    with pytest.raises(t.TriError) as e:
        t.tri_ca_run(a, a, n, 3)  # out is in
    assert e.value.status == t.TRI_EINVAL
    t.tri_ca_run(a, b, n, 16)  # one pass: no scratch needed
    torch.cuda.synchronize()
