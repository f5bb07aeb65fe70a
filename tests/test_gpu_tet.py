"""GPU: Axilrod-Teller triplet energy over the tetrahedral domain against the
FP64 oracle.  Tolerance |E - E_ref| <= 1e-5 * sum |term|: terms change sign, so
the error is measured against the magnitude sum; each FP32 term carries a
relative error of a few 2^-24, the per-thread FP32 sums have at most 32 terms
and the FP32 warp sums five more levels."""
import numpy as np
import pytest

from gpu_util import dev, tri
from paper_1609_01490_gb300 import inputs

pytestmark = pytest.mark.gpu


def _energy(t, p, map_id, rho, nu=1.0):
    import torch
    e = torch.zeros(1, dtype=torch.float64, device=dev())
    ws = torch.empty(t.tet_at_workspace_size(p.shape[0], rho, map_id) // 8 + 1, dtype=torch.float64,
                     device=dev())
    t.tet_at_energy(torch.from_numpy(p).to(dev()), e, nu, map_id, rho, ws)
    torch.cuda.synchronize()
    return float(e.item())


@pytest.mark.parametrize("rho", [8, 16, 32])
def test_at_energy_small(orc, rho):
    t = tri()
    for n in (1, 2, 3, 4, 5, 17, rho + 3, 100, 301):
        p = inputs.at_points(n, seed=1610 + n)
        ref, scale = orc.at_energy(p, nu=0.7)
        for m in (t.MAP_LAMBDA, t.MAP_BB):
            got = _energy(t, p, m, rho, nu=0.7)
            assert abs(got - ref) <= 1e-5 * scale + 1e-300, (n, rho, m, got, ref)


def test_at_energy_closed_form_tetrahedron():
    t = tri()
    p = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float32)
    got = _energy(t, p, t.MAP_LAMBDA, 8)
    assert got == pytest.approx(4 * 1.375 / (2 * np.sqrt(2.0)) ** 9, rel=1e-6)


def test_at_energy_n1536_largest(orc):
    t = tri()
    p = inputs.at_points(1536, seed=1610)
    ref, scale = orc.at_energy(p)
    a = _energy(t, p, t.MAP_LAMBDA, 16)
    b = _energy(t, p, t.MAP_BB, 16)
    assert a == b                         # same partials, same order
    assert abs(a - ref) <= 1e-5 * scale
    # rho = 32, the tile the bench's AT row times: layer table, cubic root and box agree bit for bit
    c = _energy(t, p, t.MAP_TET_TABLE, 32)
    assert c == _energy(t, p, t.MAP_LAMBDA, 32) == _energy(t, p, t.MAP_BB, 32)
    assert abs(c - ref) <= 1e-5 * scale


@pytest.mark.parametrize("rho", [8, 16, 32])
def test_at_energy_layer_table_is_bit_identical(rho):
    # the layer table finds the same blocks as the cubic root, so every
    # partial and the fixed-order sum are the same bits
    t = tri()
    for n in (3, 50, rho * 9 + 1, 700):
        p = inputs.at_points(n, seed=77 + n)
        assert _energy(t, p, t.MAP_TET_TABLE, rho) == _energy(t, p, t.MAP_LAMBDA, rho), (n, rho)
