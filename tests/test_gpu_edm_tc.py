"""GPU: tensor-core EDM (tcgen05, split BF16, FP64 recompute of flagged pairs)
against the FP64 oracle, element by element.

Tolerance: relative error <= 1e-5 per distance for the three-plane split
(BF16X6), exact zeros for the diagonal and duplicated points.  The bound
behind it: the split is exact, the dropped products are below 2^-23 |x_i||x_j|
in sum, and each of the 24 FP32 accumulation steps per 64-wide K chunk adds at
most 2^-23 of the magnitude sum, so |error of d^2| <= (2 + 24 nkc) 2^-23
(|x_i|^2 + |x_j|^2) for nkc = ceil(d / 64) chunks; pairs whose estimate of d^2
is below tau = (2 + 24 nkc) 2^-23 / 1.96e-5 times (|x_i|^2 + |x_j|^2) are
recomputed in FP64, which leaves every other pair within 1e-5.  The two-plane
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
        cases.append((260, 320))  # five 64-wide K chunks: the BF16X3 limit
    else:
        cases.append((200, 192))  # three 64-wide K chunks: the BF16X6 limit
    for n, d in cases:
        x = inputs.edm_normal_points(n, d, seed=n + d, dup_frac=0.02)
        got, nflag = _run(t, x, p, m)
        ref = orc.edm_packed(x)
        err = rel_err(got, ref)
        assert err <= tol, (prec, mapname, n, d, err)
        assert nflag >= len(inputs.duplicate_pairs(x))


def test_tc_edm_near_cancellation_d192(orc):
    # d = 192 (three K chunks, the BF16X6 limit), large norms: pairs that
    # differ in one coordinate by a few ulps (the flag path must decide them),
    # and pairs spread over d^2 / (|x_i|^2 + |x_j|^2) in [0.3, 0.7], around the
    # flag threshold (0.45 at three chunks), where unflagged pairs sit closest
    # to the error bound
    t = tri()
    n, d = 600, 192
    rng = np.random.default_rng(192)
    base = (rng.standard_normal((n // 3, d)) * 50.0).astype(np.float32)
    x = np.empty((n, d), dtype=np.float32)
    x[0::3] = base
    near = base.copy()
    k = rng.integers(0, d, n // 3)
    rows = np.arange(n // 3)
    near[rows, k] = np.nextafter(near[rows, k], np.float32(np.inf))
    near[rows, (k + 1) % d] = np.nextafter(np.nextafter(near[rows, (k + 1) % d], np.float32(-np.inf)),
                                           np.float32(-np.inf))
    x[1::3] = near
    # ratio r = d^2 / (|a|^2 + |b|^2) for b = c a + s z (z orthogonal to a, |z| = |a|):
    # r = ((1 - c)^2 + s^2) / (1 + c^2 + s^2); c = sqrt(1 - s^2) keeps |b| = |a|,
    # so r = 1 - c, spread over [0.3, 0.7]
    z = rng.standard_normal((n // 3, d))
    a = base.astype(np.float64)
    z -= (np.sum(z * a, axis=1) / np.sum(a * a, axis=1))[:, None] * a
    z *= (np.linalg.norm(a, axis=1) / np.linalg.norm(z, axis=1))[:, None]
    c = 1.0 - np.linspace(0.3, 0.7, n // 3)
    sn = np.sqrt(1.0 - c * c)
    x[2::3] = (c[:, None] * a + sn[:, None] * z).astype(np.float32)
    got, nflag = _run(t, x, t.BF16X6, t.MAP_LAMBDA)
    ref = orc.edm_packed(x)
    assert rel_err(got, ref) <= 1e-5
    assert nflag >= n // 3


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


def test_edm_largest_triangle(orc):
    # n = 92681, the largest n whose packed triangle stays below 2^32 entries
    # (4,294,930,221 distances, 17.2 GB): the tensor-core path (BF16X6) and
    # the FP32 path (lambda, 4 x 4 pairs per thread) on sampled pairs, whole
    # blocks at the first rows, the diagonal and the far corner, the pairs
    # around packed offsets 2^31 and 2^32 - 1, every duplicated pair, and
    # guard words past the end
    import torch
    t = tri()
    n, d = 92681, 64
    size = n * (n + 1) // 2
    assert size < 1 << 32 and (n + 1) * (n + 2) // 2 >= 1 << 32
    x = inputs.edm_normal_points(n, d, seed=92681, dup_frac=0.001)
    D = dev()
    xd = torch.from_numpy(x).to(D)
    rng = np.random.default_rng(7)
    pi = rng.integers(0, n, 200_000)
    pj = (rng.random(200_000) * (pi + 1)).astype(np.int64)
    ti, tj = np.tril_indices(300)
    last = np.arange(n - 300, n)
    ci, cj = np.repeat(last, 512), np.tile(np.arange(512), 300)   # far corner: the last 300 rows, columns 0..511
    di, dj = np.repeat(last, 300), (last[:, None] - np.arange(300)[None, :]).ravel()  # last rows at the diagonal
    # the packed offsets around 2^31 and the end of the triangle
    extra = []
    for w0 in (1 << 31, size - 1):
        for w in range(w0 - 600, w0 + 600):
            if 0 <= w < size:
                i = (int(np.sqrt(8 * w + 1)) - 1) // 2
                while i * (i + 1) // 2 > w:
                    i -= 1
                while (i + 1) * (i + 2) // 2 <= w:
                    i += 1
                extra.append((i, w - i * (i + 1) // 2))
    ei, ej = np.array(extra, dtype=np.int64).T
    dup = inputs.duplicate_pairs(x)
    pi = np.concatenate([pi, ti, ci, di, ei, dup[:, 0]])
    pj = np.concatenate([pj, tj, cj, dj, ej, dup[:, 1]])
    ref = orc.edm_pairs(x, pi, pj)
    idx = torch.from_numpy(pi * (pi + 1) // 2 + pj).to(D)
    out = torch.full((size + 64,), -7.0, dtype=torch.float32, device=D)
    ws = torch.empty(t.tri_edm_workspace_size(n, d, t.BF16X6), dtype=torch.uint8, device=D)
    nf = torch.zeros(1, dtype=torch.int64, device=D)
    t.tri_edm(xd, out, map=t.MAP_LAMBDA, prec=t.BF16X6, workspace=ws, n_flagged=nf)
    torch.cuda.synchronize()
    assert int(ws[8:12].view(torch.int32).item()) == 0
    assert torch.all(out[size:] == -7.0)
    assert rel_err(out[idx].cpu().numpy(), ref) <= 1e-5
    assert int(nf.item()) >= len(dup)
    out[:size].fill_(-1.0)
    t.tri_edm(xd, out, map=t.MAP_LAMBDA, rho=16, reg=4, prec=t.FP32)
    torch.cuda.synchronize()
    assert torch.all(out[size:] == -7.0)
    assert rel_err(out[idx].cpu().numpy(), ref) <= 1e-5


def _full_compare(orc, x, outs, bands=16):
    """Every pair of the packed triangle of each host array in `outs` against
    the FP64 oracle, in row bands of equal pair count.  Returns, per array,
    the maximum and the 99.99th percentile relative error (from a histogram
    of log10 errors at 0.001 resolution), the exact zeros of the reference and
    whether the array matched them all.  The comparison runs on several host
    threads (numpy releases the interpreter lock in its loops)."""
    import concurrent.futures as cf
    import os
    n = x.shape[0]
    edges = [0] + [min(n, int(np.ceil(n * np.sqrt(b / bands)))) for b in range(1, bands)] + [n]
    bins = np.linspace(-12.0, -2.0, 10001)

    def part(o, ref, p0, a, b):
        r = ref[a:b]
        got = o[p0 + a:p0 + b].astype(np.float64)
        z = r == 0
        zok = bool(np.all(got[z] == 0.0))
        nz = ~z
        rel = np.abs(got[nz] - r[nz]) / r[nz]
        pos = rel > 0
        h = np.histogram(np.log10(rel[pos]), bins=bins)[0]
        return (float(rel.max()) if rel.size else 0.0, h, int(rel.size - np.count_nonzero(pos)), zok,
                int(np.count_nonzero(z)))

    st = [{"max": 0.0, "hist": np.zeros(len(bins) - 1, dtype=np.int64), "under": 0, "zeros_ok": True}
          for _ in outs]
    zeros = 0
    step = 1 << 23
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        for r0, r1 in zip(edges[:-1], edges[1:]):
            if r1 <= r0:
                continue
            ref = orc.edm_rows(x, r0, r1)
            p0 = r0 * (r0 + 1) // 2
            for oi, (o, s) in enumerate(zip(outs, st)):
                for mx, h, under, zok, nzero in ex.map(lambda ab: part(o, ref, p0, *ab),
                                                       [(a, min(a + step, len(ref))) for a in range(0, len(ref), step)]):
                    s["max"] = max(s["max"], mx)
                    s["hist"] += h
                    s["under"] += under
                    s["zeros_ok"] &= zok
                    if oi == 0:
                        zeros += nzero
    total = n * (n + 1) // 2 - zeros
    res = []
    for s in st:
        # the error that 0.01% of the nonzero pairs exceed (upper edge of its bin)
        need = int(np.ceil(1e-4 * total))
        c = np.cumsum(s["hist"][::-1])
        k = int(np.searchsorted(c, need))
        p9999 = 10.0 ** bins[len(bins) - 1 - k] if k < len(c) else 0.0
        res.append({"max_rel": s["max"], "p99_99_rel": p9999, "exact_zero_pairs": zeros,
                    "zeros_ok": s["zeros_ok"], "exact_pairs": s["under"]})
    return res


def test_tc_edm_full_triangle_every_pair(orc):
    # the launch the bench times (N = 65536, d = 128, 1% duplicated rows, seed
    # 1609): all 2,147,516,416 pairs of the BF16X6 and BF16X3 triangles against
    # the FP64 oracle, with the per-result error stated (pytest -s prints it)
    import json
    import torch
    t = tri()
    n, d = 65536, 128
    x = inputs.edm_normal_points(n, d, seed=1609, dup_frac=0.01)
    D = dev()
    xd = torch.from_numpy(x).to(D)
    out = torch.empty(n * (n + 1) // 2, dtype=torch.float32, device=D)
    hosts, flags = [], []
    for prec in (t.BF16X6, t.BF16X3):
        ws = torch.empty(t.tri_edm_workspace_size(n, d, prec), dtype=torch.uint8, device=D)
        nf = torch.zeros(1, dtype=torch.int64, device=D)
        t.tri_edm(xd, out, map=t.MAP_LAMBDA, prec=prec, workspace=ws, n_flagged=nf)
        torch.cuda.synchronize()
        assert int(ws[8:12].view(torch.int32).item()) == 0
        hosts.append(out.cpu().numpy())
        flags.append(int(nf.item()))
        del ws
    del out, xd
    torch.cuda.empty_cache()
    res = _full_compare(orc, x, hosts)
    for r, nf, name in zip(res, flags, ("bf16x6", "bf16x3")):
        r["n_flagged"] = nf
        print(f"full-triangle error {name}: " + json.dumps(r))
    assert res[0]["zeros_ok"] and res[1]["zeros_ok"]
    assert res[0]["max_rel"] <= 1e-5, res[0]
    assert res[1]["max_rel"] <= 1e-4, res[1]
    assert flags[0] >= len(inputs.duplicate_pairs(x))


@pytest.mark.parametrize("prec", ["BF16X6", "BF16X3"])
def test_tc_gram_wait_limit_runs_out_cleanly(orc, prec):
    # The Gram kernel's waits between its roles (copy, MMA, epilogue) are
    # bounded.  The workspace word at byte 40 shortens that bound (here to
    # 1 ns): the waits give up, both CTAs of every pair stop, drain the copies
    # and MMAs in flight, free their tensor memory and return, and the status
    # word (int at byte 8) reads TRI_ETIMEOUT.  The same workspace then gives
    # the right triangle on a normal call (tri_edm_prepare clears the header).
    import torch
    t = tri()
    p = getattr(t, prec)
    D = dev()
    n, d = 1000, 100
    x = inputs.edm_normal_points(n, d, seed=41, dup_frac=0.02)
    xd = torch.from_numpy(x).to(D)
    size = n * (n + 1) // 2
    out = torch.full((size + 64,), -7.0, dtype=torch.float32, device=D)
    ws = torch.empty(t.tri_edm_workspace_size(n, d, p), dtype=torch.uint8, device=D)
    for _ in range(2):
        t.tri_edm_prepare(xd, p, ws)
        ws[40:48].view(torch.int64).fill_(1)
        t.tri_edm_gram(n, d, out, t.MAP_LAMBDA, p, ws)
        assert t.tri_sync_status(ws[8:12].view(torch.int32)) == t.TRI_ETIMEOUT
    assert torch.all(out[size:] == -7.0)
    nf = torch.zeros(1, dtype=torch.int64, device=D)
    t.tri_edm(xd, out, map=t.MAP_LAMBDA, prec=p, workspace=ws, n_flagged=nf)
    assert t.tri_sync_status(ws[8:12].view(torch.int32)) == t.TRI_OK
    o = out.cpu().numpy()
    assert np.all(o[size:] == -7.0)
    assert rel_err(o[:size], orc.edm_packed(x)) <= (1e-5 if prec == "BF16X6" else 1e-4)


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
    # d = 193 (BF16X6) and d = 321 (BF16X3) exceed the resident-operand limits
    for dd, pr in ((193, t.BF16X6), (321, t.BF16X3)):
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


@pytest.mark.parametrize("ranks", [1, 3, 8])
def test_tc_edm_rows_bands_assemble_the_triangle(ranks):
    # one triangle split across ranks (tri_edm_partition): each rank's band,
    # computed by tri_edm_rows into its own buffer, holds the same bytes as
    # that range of tri_edm's output (the ranks run here one after another)
    import torch
    t = tri()
    D = dev()
    n, d = 3000, 64
    x = inputs.edm_normal_points(n, d, seed=78, dup_frac=0.02)
    xd = torch.from_numpy(x).to(D)
    size = n * (n + 1) // 2
    for prec in (t.BF16X6, t.BF16X3):
        ws = torch.empty(t.tri_edm_workspace_size(n, d, prec), dtype=torch.uint8, device=D)
        ref = torch.empty(size, device=D)
        t.tri_edm(xd, ref, prec=prec, workspace=ws)
        parts = []
        for r in range(ranks):
            rb, re_, pb, pe = t.tri_edm_partition(n, ranks, r)
            band = torch.full((pe - pb + 16,), -5.0, device=D)
            t.tri_edm_rows(xd, rb, re_, band, prec=prec, workspace=ws)
            torch.cuda.synchronize()
            assert int(ws[8:12].view(torch.int32).item()) == 0
            assert torch.all(band[pe - pb:] == -5.0), "store past the band"
            parts.append(band[:pe - pb])
        assert torch.equal(torch.cat(parts), ref), (prec, ranks)


def test_tc_edm_rows_errors():
    import torch
    t = tri()
    D = dev()
    x = torch.zeros(600, 8, device=D)
    ws = torch.empty(t.tri_edm_workspace_size(600, 8, t.BF16X6), dtype=torch.uint8, device=D)
    band = torch.empty(600 * 601 // 2, device=D)
    for rb, re_ in ((100, 256), (0, 300), (256, 601), (300, 200)):  # not on unit rows / past n / reversed
        with pytest.raises(t.TriError) as e:
            t.tri_edm_rows(x, rb, re_, band, workspace=ws)
        assert e.value.status == t.TRI_EINVAL
    t.tri_edm_rows(x, 600, 600, band, workspace=ws)  # an empty band is allowed
    torch.cuda.synchronize()


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
