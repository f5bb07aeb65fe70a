"""The hot path split across processes, one per GPU (torch.distributed: NCCL
between GPUs; the tests run the same code over gloo on CPU tensors).

Every split follows lambda's numbering: block rows [R0, R1) of a triangle are
the block numbers [T(R0), T(R1)), so a band of rows is one contiguous range of
work and, for the packed outputs, of memory.

- The Euclidean distance map: ``tri_edm_partition`` bands, each rank computing
  its rows with ``tri_edm_rows``; nothing is exchanged.
- A batch of triangles: ``batched_sharded``, whole instances per rank from
  ``tri_edm_batched_partition``; nothing is exchanged.
- A cellular automaton: ``ca_run_bands``, row bands from ``tri_ca_partition``
  stepped with ``tri_ca_step_rows``, with one halo row swapped with each
  neighbouring band before every step.
- The Axilrod-Teller energy: ``at_energy_sharded``, a tetrahedral block range
  per rank from ``tet_at_partition`` summed by ``tet_at_energy_range``, then
  one FP64 all-reduce.

The compute runs in libtri.so; this module only decides who computes what and
moves the halo rows and the partial energy.  A rank leaves these calls only
between steps, with none of its transfers in flight.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import tri


def _owners(bands):
    """Row -> rank over non-empty bands [(row_begin, row_end), ...] in rank order."""
    def owner(row: int) -> int:
        for r, (b0, b1) in enumerate(bands):
            if b0 <= row < b1:
                return r
        raise ValueError(f"row {row} lies in no band")
    return owner


def ca_halo_exchange(grid, n: int, band, bands, group=None) -> None:
    """Swap the halo rows of this rank's band [b0, b1) with the ranks owning
    rows b0 - 1 and b1: send rows b0 and b1 - 1, receive rows b0 - 1 and b1
    (each a whole row of the row-major grid, leading dimension included)."""
    b0, b1 = band
    if b0 >= b1:
        return
    owner = _owners(bands)
    ops = []
    if b0 > 0:
        peer = owner(b0 - 1)
        ops += [dist.P2POp(dist.isend, grid[b0], peer, group), dist.P2POp(dist.irecv, grid[b0 - 1], peer, group)]
    if b1 < n:
        peer = owner(b1)
        ops += [dist.P2POp(dist.isend, grid[b1 - 1], peer, group), dist.P2POp(dist.irecv, grid[b1], peer, group)]
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


def ca_run_bands(a, b, n: int, steps: int, rank: int, world: int, rho: int = 32, birth: int = tri.LIFE_BIRTH,
                 survive: int = tri.LIFE_SURVIVE, group=None, step_rows=None):
    """`steps` steps of the automaton on this rank's band of the n x n grid.

    a holds the current grid (at least this rank's band), b is scratch of the
    same shape; both are row-major uint8 [n][ld].  Returns (grid, band): the
    buffer holding the final state of rows band[0] .. band[1] - 1.
    step_rows(src, dst, row_begin, row_end) computes one step of the band;
    the default is tri_ca_step_rows on the current stream.
    """
    bands = [tri.tri_ca_partition(n, rho, world, r) for r in range(world)]
    band = bands[rank]
    if step_rows is None:
        def step_rows(src, dst, r0, r1):
            tri.tri_ca_step_rows(src, dst, n, r0, r1, birth, survive, rho)
    # the first point-to-point call of a group must involve every rank
    dist.barrier(group=group)
    for _ in range(steps):
        ca_halo_exchange(a, n, band, bands, group)
        step_rows(a, b, band[0], band[1])
        a, b = b, a
    return a, band


def at_energy_sharded(xyz, rank: int, world: int, rho: int = 32, map: int = tri.MAP_TET_TABLE, nu: float = 1.0,
                      group=None, energy_range=None):
    """The Axilrod-Teller energy of all n points, each rank summing its block
    range; every rank returns the total (an FP64 tensor of one element).
    energy_range(xyz, energy, w0, w1) writes the range's energy into `energy`;
    the default is tet_at_energy_range with a workspace of w1 - w0 doubles."""
    n = xyz.shape[0]
    w0, w1 = tri.tet_at_partition(n, rho, world, rank)
    energy = torch.zeros(1, dtype=torch.float64, device=xyz.device)
    if energy_range is None:
        ws = torch.empty(max(1, w1 - w0), dtype=torch.float64, device=xyz.device)

        def energy_range(p, e, a, b):
            tri.tet_at_energy_range(p, e, a, b, nu=nu, map=map, rho=rho, workspace=ws)
    energy_range(xyz, energy, w0, w1)
    dist.all_reduce(energy, op=dist.ReduceOp.SUM, group=group)
    return energy


def batched_sharded(x_cat, pt_off, n_k, n_k_host, out_cat, out_off, rank: int, world: int, rho: int = 16,
                    reg: int = 8, workspace=None):
    """This rank's instances [k_begin, k_end) of a batched EDM, computed with
    tri_edm_batched on its slices of pt_off, n_k and out_off (device tensors;
    n_k_host the same sizes on the host).  Returns (k_begin, k_end)."""
    kb, ke = tri.tri_edm_batched_partition(n_k_host, rho, reg, world, rank)
    if ke > kb:
        tri.tri_edm_batched(x_cat, pt_off[kb:ke], n_k[kb:ke], out_cat, out_off[kb:ke], rho=rho, reg=reg,
                            workspace=workspace)
    return kb, ke
