"""GPU: tensor-core EDM (tcgen05, split BF16, FP64 recompute of flagged pairs)
against the FP64 oracle, element by element.

Tolerance: relative error <= 1e-5 per distance for the three-plane split
(BF16X6), exact zeros for the diagonal and duplicated points.  The bound
behind it: the split is exact, the dropped products are below 2^-23 |x_i||x_j|
in sum, and 48 FP32 accumulation steps add at most 48*2^-23 of the magnitude
sum, so |error of d^2| <= 6.2e-6 (|x_i|^2 + |x_j|^2); pairs whose estimate of
d^2 is below tau = 0.3125 (|x_i|^2 + |x_j|^2) are recomputed in FP64, which
leaves every other pair within 6.2e-6 / (2 * 0.3125) ~ 1e-5.  The two-plane
split (BF16X3) carries no such guarantee; its measured error is checked
against 1e-4.
"""
import numpy as np
import pytest

from gpu_util import dev, rel_err, tri
from paper_1609_01490_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run(t, x, prec, map_id, guard=64):
    import torch
    n, d = x.shape
    size = n * (n + 1) // 2
    D = dev()
    out = torch.full((size + guard,), -7.0, dtype=torch.float32, device=D)
    ws = torch.empty(t.tri_edm_workspace_size(n, d, prec), dtype=torch.uint8, device=D)
    nf = torch.zeros(1, dtype=torch.int64, device=D)
    t.tri_edm(torch.from_numpy(x).to(D), out, map=map_id, prec=prec, workspace=ws, n_flagged=nf)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.all(o[size:] == -7.0), "store past the packed triangle"
    status = int(ws[8:12].view(torch.int32).item())
    assert status == 0, f"device status {status}"
    return o[:size], int(nf.item())


@pytest.mark.parametrize("prec,tol", [("BF16X6", 1e-5), ("BF16X3", 1e-4)])
@pytest.mark.parametrize("mapname", ["LAMBDA", "BB"])
def test_tc_edm_small(orc, prec, tol, mapname):
    t = tri()
    p = getattr(t, prec)
    m = getattr(t, "MAP_" + mapname)
    cases = [(1, 3), (5, 3), (128, 64), (129, 17), (300, 128), (1000, 100), (777, 64)]
    if prec == "BF16X3":
        cases.append((260, 256))  # four 64-wide K chunks: the BF16X3 limit
    else:
        cases.append((200, 192))  # three 64-wide K chunks: the BF16X6 limit
    for n, d in cases:
        x = inputs.edm_normal_points(n, d, seed=n + d, dup_frac=0.02)
        got, nflag = _run(t, x, p, m)
        ref = orc.edm_packed(x)
        err = rel_err(got, ref)
        assert err <= tol, (prec, mapname, n, d, err)
        assert nflag >= len(inputs.duplicate_pairs(x))


def test_tc_edm_uniform_low_d(orc):
    # few features in [0,1): large norms relative to distances -> many flags
    t = tri()
    x = inputs.edm_uniform_points(2048, 3, seed=1609)
    got, nflag = _run(t, x, t.BF16X6, t.MAP_LAMBDA)
    assert rel_err(got, orc.edm_packed(x)) <= 1e-5
    assert nflag > 0


def test_tc_edm_list_overflow_falls_back_to_scan(orc):
    # 1500 identical points: every pair is flagged, 1,124,250 > the list's 2^20
    t = tri()
    x = np.repeat(inputs.edm_normal_points(1, 40, seed=3), 1500, axis=0)
    x[::97] += 0.5
    got, nflag = _run(t, x, t.BF16X6, t.MAP_LAMBDA)
    assert nflag > 1 << 20
    assert rel_err(got, orc.edm_packed(x)) <= 1e-5


def test_tc_edm_full_size_sampled(orc):
    # N = 65536, d = 128, 1% duplicated rows: the launch the bench times
    import torch
    t = tri()
    n, d = 65536, 128
    x = inputs.edm_normal_points(n, d, seed=1609, dup_frac=0.01)
    D = dev()
    out = torch.empty(n * (n + 1) // 2, dtype=torch.float32, device=D)
    xd = torch.from_numpy(x).to(D)
    rng = np.random.default_rng(0)
    dup = inputs.duplicate_pairs(x)
    pi = rng.integers(0, n, 300_000)
    pj = (rng.random(300_000) * (pi + 1)).astype(np.int64)
    # plus whole tiles on the diagonal and at the far corner
    ti, tj = np.tril_indices(256)
    pi = np.concatenate([pi, dup[:, 0], ti, n - 256 + ti, n - 256 + ti])
    pj = np.concatenate([pj, dup[:, 1], tj, n - 256 + tj, tj])
    ref = orc.edm_pairs(x, pi, pj)
    idx = torch.from_numpy(pi * (pi + 1) // 2 + pj).to(D)
    for prec, tol in ((t.BF16X6, 1e-5), (t.BF16X3, 1e-4)):
        ws = torch.empty(t.tri_edm_workspace_size(n, d, prec), dtype=torch.uint8, device=D)
        nf = torch.zeros(1, dtype=torch.int64, device=D)
        t.tri_edm(xd, out, map=t.MAP_LAMBDA, prec=prec, workspace=ws, n_flagged=nf)
        torch.cuda.synchronize()
        assert int(ws[8:12].view(torch.int32).item()) == 0
        assert rel_err(out[idx].cpu().numpy(), ref) <= tol, prec
        assert int(nf.item()) >= len(dup)


def test_tc_phases_and_errors():
    import torch
    t = tri()
    D = dev()
    x = torch.from_numpy(inputs.edm_normal_points(200, 64, seed=9)).to(D)
    out = torch.empty(200 * 201 // 2, device=D)
    need = t.tri_edm_workspace_size(200, 64, t.BF16X6)
    small = torch.empty(need - 256, dtype=torch.uint8, device=D)
    with pytest.raises(t.TriError) as e:
        t.tri_edm(x, out, prec=t.BF16X6, workspace=small)
    assert e.value.status == t.TRI_ENOSPACE
    with pytest.raises(t.TriError):
        t.tri_edm(x, out, map=t.MAP_RB, prec=t.BF16X6,
                  workspace=torch.empty(need, dtype=torch.uint8, device=D))
    # d = 193 (BF16X6) and d = 257 (BF16X3) exceed the resident-operand limits
    for dd, pr in ((193, t.BF16X6), (257, t.BF16X3)):
        with pytest.raises(t.TriError) as e:
            xx = torch.zeros(10, dd, device=D)
            t.tri_edm(xx, torch.empty(55, device=D), prec=pr,
                      workspace=torch.empty(t.tri_edm_workspace_size(10, dd, pr), dtype=torch.uint8, device=D))
        assert e.value.status == t.TRI_ERANGE
    # the three phases called one by one give the same bytes as tri_edm
    ws = torch.empty(need, dtype=torch.uint8, device=D)
    a = torch.empty_like(out)
    t.tri_edm(x, a, prec=t.BF16X6, workspace=ws)
    b = torch.empty_like(out)
    t.tri_edm_prepare(x, t.BF16X6, ws)
    t.tri_edm_gram(200, 64, b, t.MAP_LAMBDA, t.BF16X6, ws)
    t.tri_edm_fixup(x, b, t.BF16X6, ws)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("bands", [0, 1, 5])
def test_tc_edm_host_matches_device_path(bands):
    # host buffers in and out, banded compute overlapped with the copies: the
    # same bytes as tri_edm on device buffers, flags included
    import torch
    t = tri()
    D = dev()
    n, d = 3000, 64
    x = inputs.edm_normal_points(n, d, seed=77, dup_frac=0.02)
    size = n * (n + 1) // 2
    for prec in (t.BF16X6, t.BF16X3):
        ws = torch.empty(t.tri_edm_workspace_size(n, d, prec), dtype=torch.uint8, device=D)
        ref = torch.empty(size, device=D)
        nf_ref = torch.zeros(1, dtype=torch.int64, device=D)
        t.tri_edm(torch.from_numpy(x).to(D), ref, prec=prec, workspace=ws, n_flagged=nf_ref)
        xh = torch.from_numpy(x).pin_memory()
        oh = torch.full((size,), -1.0).pin_memory()
        xd = torch.empty(n, d, device=D)
        od = torch.empty(size, device=D)
        nf = torch.zeros(1, dtype=torch.int64, device=D)
        t.tri_edm_host(xh, oh, xd, od, ws, prec=prec, bands=bands, n_flagged=nf)
        torch.cuda.synchronize()
        assert int(ws[8:12].view(torch.int32).item()) == 0
        assert torch.equal(oh, ref.cpu()), (prec, bands)
        assert torch.equal(od, ref)
        assert int(nf.item()) == int(nf_ref.item()) > 0


def test_tc_edm_host_list_overflow_per_band(orc):
    # every pair flagged (identical points): each band falls back to scanning its own rows
    import torch
    t = tri()
    D = dev()
    x = np.repeat(inputs.edm_normal_points(1, 40, seed=3), 1500, axis=0)
    x[::97] += 0.5
    n, d = x.shape
    size = n * (n + 1) // 2
    ws = torch.empty(t.tri_edm_workspace_size(n, d, t.BF16X6), dtype=torch.uint8, device=D)
    xh = torch.from_numpy(x).pin_memory()
    oh = torch.zeros(size).pin_memory()
    nf = torch.zeros(1, dtype=torch.int64, device=D)
    t.tri_edm_host(xh, oh, torch.empty(n, d, device=D), torch.empty(size, device=D), ws, prec=t.BF16X6, bands=4,
                   n_flagged=nf)
    torch.cuda.synchronize()
    assert int(nf.item()) > 1 << 20
    assert rel_err(oh.numpy(), orc.edm_packed(x)) <= 1e-5


def test_tc_edm_host_errors():
    import torch
    t = tri()
    D = dev()
    xh = torch.zeros(10, 4).pin_memory()
    ws = torch.empty(t.tri_edm_workspace_size(10, 4, t.BF16X6), dtype=torch.uint8, device=D)
    with pytest.raises(t.TriError) as e:  # FP32 has no host-buffer path
        t.tri_edm_host(xh, torch.zeros(55).pin_memory(), torch.empty(10, 4, device=D), torch.empty(55, device=D), ws,
                       prec=t.FP32)
    assert e.value.status == t.TRI_EINVAL
    with pytest.raises(ValueError):  # host buffers must be host tensors
        t.tri_edm_host(xh.to(D), torch.zeros(55), torch.empty(10, 4, device=D), torch.empty(55, device=D), ws)
