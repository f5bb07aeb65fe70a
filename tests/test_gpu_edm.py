"""GPU: FP32 EDM under every map against the FP64 oracle, element by element
(Section 5, test 2), plus the full-size workloads on sampled pairs.

Tolerance: relative error <= 1e-5 per distance.  Direct differences in FP32
round each of the d differences, squares and sums once, so the relative error
of d^2 is at most about (d+2)*2^-24 (7.7e-6 at d = 128) and that of d about half
of it; exact zeros (diagonal, duplicated points) must come out exactly 0.
"""
import numpy as np
import pytest

from gpu_util import dev, rel_err, tri
from paper_1609_01490_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _edm(t, x, map_id, rho, reg, guard=64):
    import torch
    n = x.shape[0]
    size = n * (n + 1) // 2
    out = torch.full((size + guard,), -7.0, dtype=torch.float32, device=dev())
    t.tri_edm(torch.from_numpy(x).to(dev()), out, map=map_id, rho=rho, reg=reg)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.all(o[size:] == -7.0), "store past the packed triangle"
    return o[:size]


@pytest.mark.parametrize("mapname", ["LAMBDA", "LAMBDA_PDELTA", "BB", "RB", "REC", "UTM"])
@pytest.mark.parametrize("rho,reg", [(8, 1), (16, 1), (32, 1), (8, 4), (16, 2), (16, 4), (32, 4), (8, 8), (16, 8)])
def test_edm_fp32_all_maps(orc, mapname, rho, reg):
    t = tri()
    map_id = getattr(t, "MAP_" + mapname)
    S = rho * reg
    for n, d in [(1, 3), (2, 1), (S - 1, 3), (S + 1, 4), (3 * S + 5, 33), (2 * S + 3, 100), (300, 128), (1024, 3)]:
        if mapname == "REC":
            m = -(-n // S)
            if m & (m - 1):
                continue
        x = inputs.edm_normal_points(n, d, seed=n * 31 + d, dup_frac=0.02)
        got = _edm(t, x, map_id, rho, reg)
        assert rel_err(got, orc.edm_packed(x)) <= TOL, (mapname, n, d, rho, reg)


def test_edm_n2048_d3_every_pair(orc):
    # N = 2048 points in [0,1)^3, rho = 16: every one of the 2,098,176 pairs, lambda and BB
    t = tri()
    x = inputs.edm_uniform_points(2048, 3, seed=1609)
    ref = orc.edm_packed(x)
    for m in (t.MAP_LAMBDA, t.MAP_BB):
        got = _edm(t, x, m, 16, 1)
        assert len(got) == 2_098_176
        assert rel_err(got, ref) <= TOL


def test_edm_large_sampled(orc):
    # N = 65536, d = 128 with 1% duplicated rows: the launch the bench times for
    # the FP32 path, checked on 200k sampled pairs plus every duplicated pair
    import torch
    t = tri()
    n, d = 65536, 128
    x = inputs.edm_normal_points(n, d, seed=1609, dup_frac=0.01)
    out = torch.empty(n * (n + 1) // 2, dtype=torch.float32, device=dev())
    xd = torch.from_numpy(x).to(dev())
    t.tri_edm(xd, out, map=t.MAP_LAMBDA, rho=16, reg=4)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    pi = rng.integers(0, n, 200_000)
    pj = (rng.random(200_000) * (pi + 1)).astype(np.int64)
    dup = inputs.duplicate_pairs(x)
    pi = np.concatenate([pi, dup[:, 0], np.arange(0, n, 997)])
    pj = np.concatenate([pj, dup[:, 1], np.arange(0, n, 997)])
    idx = torch.from_numpy(pi * (pi + 1) // 2 + pj).to(dev())
    got = out[idx].cpu().numpy()
    assert rel_err(got, orc.edm_pairs(x, pi, pj)) <= TOL
    assert len(dup) >= 600


def test_edm_rejects_bad_arguments():
    import torch
    t = tri()
    x = torch.zeros(10, 3, device=dev())
    out = torch.zeros(55, device=dev())
    with pytest.raises(t.TriError):
        t.tri_edm(x, out, rho=12)
    with pytest.raises(t.TriError):
        t.tri_edm(x, out, reg=3)
    with pytest.raises(t.TriError):  # 8 x 8 pairs per thread needs rho <= 16
        t.tri_edm(x, out, rho=32, reg=8)
    with pytest.raises(t.TriError):  # REC needs a power-of-two block count: 40 points / 8 = 5
        t.tri_edm(torch.zeros(40, 3, device=dev()), torch.zeros(820, device=dev()), map=t.MAP_REC, rho=8, reg=1)
