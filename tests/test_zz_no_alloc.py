"""GPU: tet_at_energy_noalloc, the workspace-free variant of tet_at_energy for
callers that cannot allocate device memory (their memory belongs to another
allocator, or they must not trigger cudaMalloc's implicit synchronisation).

It is called straight through the C ABI and must give the same energy as
tet_at_energy, bit for bit, on several calls in a row (each on other points,
with no more partials than the call before, so stale partials from an earlier
call would show); the last energy is also held to the AT tolerance of the
FP64 oracle, |E - E_ref| <= 1e-5 * sum |term|.  This file sorts last so that
a run that stops at the first failure has run every other test first.
"""
import ctypes

import pytest

import oracle

from gpu_util import dev, tri
from paper_1609_01490_gb300 import inputs

pytestmark = pytest.mark.gpu


def _c_noalloc(t):
    fn = ctypes.CDLL(t.LIB_PATH).tet_at_energy_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_double, ctypes.c_void_p, ctypes.c_int,
                   ctypes.c_uint32, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def _with_workspace(t, p_dev, n, nu, map_id, rho):
    import torch
    e = torch.zeros(1, dtype=torch.float64, device=dev())
    ws = torch.empty(t.tet_at_workspace_size(n, rho, map_id) // 8 + 1, dtype=torch.float64, device=dev())
    t.tet_at_energy(p_dev, e, nu, map_id, rho, ws)
    torch.cuda.synchronize()
    return float(e.item())


def test_noalloc_matches_workspace_entry_point():
    # Calls in a row on different points, each with no more block partials
    # than the call before, so that a read of partials left by an earlier
    # call would change the energy.  The two entry points run the same kernels
    # in the same order on the same inputs, so the energies agree bit for bit.
    import torch
    t = tri()
    fn = _c_noalloc(t)
    stream = torch.cuda.current_stream().cuda_stream
    # (n, rho, map, seed): partial counts 260,130 (the array's edge at rho = 32),
    # 152,096, 152,096, 117,480
    cases = [(3680, 32, t.MAP_TET_TABLE, 1610), (1536, 16, t.MAP_LAMBDA, 1611),
             (1536, 16, t.MAP_LAMBDA, 1612), (700, 8, t.MAP_BB, 1613)]
    for n, rho, map_id, seed in cases:
        p = inputs.at_points(n, seed=seed)
        pd = torch.from_numpy(p).to(dev())
        ref = _with_workspace(t, pd, n, 0.9, map_id, rho)
        e = torch.full((1,), float("nan"), dtype=torch.float64, device=dev())
        st = fn(pd.data_ptr(), n, 0.9, e.data_ptr(), map_id, rho, stream)
        assert st == t.TRI_OK, t.TriError("tet_at_energy_noalloc", st)
        torch.cuda.synchronize()
        got = float(e.item())
        assert got == ref, (n, rho, map_id, got, ref)
    # and within the AT tolerance of the FP64 oracle on the last points
    eref, scale = oracle.at_energy(p, nu=0.9)
    assert abs(got - eref) <= 1e-5 * scale


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    t = tri()
    fn = _c_noalloc(t)
    pd = torch.zeros(2000, 3, dtype=torch.float32, device=dev())
    e = torch.zeros(1, dtype=torch.float64, device=dev())
    # 2000 points at rho = 8: 250 block rows, T_250 = 2,635,500 partials > 262,144
    assert fn(pd.data_ptr(), 2000, 1.0, e.data_ptr(), t.MAP_LAMBDA, 8, None) == t.TRI_ENOSPACE
    assert fn(pd.data_ptr(), 1840, 1.0, e.data_ptr(), t.MAP_LAMBDA, 16, None) == t.TRI_OK
    assert fn(pd.data_ptr(), 1841, 1.0, e.data_ptr(), t.MAP_LAMBDA, 16, None) == t.TRI_ENOSPACE
    pd = torch.zeros(3681, 3, dtype=torch.float32, device=dev())
    assert fn(pd.data_ptr(), 3681, 1.0, e.data_ptr(), t.MAP_TET_TABLE, 32, None) == t.TRI_ENOSPACE
    torch.cuda.synchronize()
