"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds no arithmetic of the method itself: it only draws numbers.
Every value comes from one counter-based generator, splitmix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the k-th
output for seed s is the splitmix64 finaliser applied to s + (k+1)*0x9E3779B97F4A7C15
(mod 2^64).  Inputs are generated on the host and uploaded, so both sides of a
parity test see identical bytes.

Workload shapes follow the paper's tests (Section 5: EDM over points with a
few features, shared-memory style neighbourhood work) and the extensions the
library ships (high-dimensional EDM with duplicated points, batched uneven
triangles, a triangular cellular automaton, tetrahedral triplets).
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """k-th splitmix64 output for every k in ``idx`` (uint64 array)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx.astype(np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_f32(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """U[0,1) in FP32: the top 24 bits of each draw times 2^-24 (exact)."""
    z = splitmix64(seed, np.arange(offset, offset + count, dtype=np.uint64))
    return ((z >> np.uint64(40)).astype(np.float64) * 2.0 ** -24).astype(np.float32)


def uniform_f64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """U[0,1) in FP64 from the top 53 bits of each draw."""
    z = splitmix64(seed, np.arange(offset, offset + count, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def normal_f32(seed: int, count: int) -> np.ndarray:
    """N(0,1) by Box-Muller in FP64 (draws 2k and 2k+1 feed value k), rounded to FP32."""
    u = uniform_f64(seed, 2 * count)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)).astype(np.float32)


def edm_uniform_points(n: int, d: int, seed: int = 1609) -> np.ndarray:
    """n points in [0,1)^d, FP32, row-major [n][d] (the paper's EDM test, Section 5)."""
    return uniform_f32(seed, n * d).reshape(n, d)


def edm_normal_points(n: int, d: int, seed: int = 1609, dup_frac: float = 0.0) -> np.ndarray:
    """n points drawn N(0,1) in FP32, row-major [n][d].

    With ``dup_frac`` > 0, floor(dup_frac*n) destination rows (chosen without
    replacement) are overwritten by copies of randomly chosen non-destination
    rows, which plants exact-zero distances (the cancellation cases of a Gram
    formulation).
    """
    x = normal_f32(seed, n * d).reshape(n, d)
    ndup = int(math.floor(dup_frac * n))
    if ndup > 0:
        keys = splitmix64(seed ^ 0x5DEECE66D, np.arange(n, dtype=np.uint64))
        order = np.argsort(keys, kind="stable")
        dest = np.sort(order[:ndup])
        rest = np.sort(order[ndup:])
        pick = splitmix64(seed ^ 0xB5297A4D, np.arange(ndup, dtype=np.uint64)) % np.uint64(len(rest))
        src = rest[pick.astype(np.int64)]
        x[dest] = x[src]
    return x


def duplicate_pairs(x: np.ndarray) -> np.ndarray:
    """All (i, j), i > j, whose rows are bitwise identical (for checks of exact zeros)."""
    view = np.ascontiguousarray(x).view(np.dtype((np.void, x.dtype.itemsize * x.shape[1]))).ravel()
    order = np.argsort(view, kind="stable")
    out = []
    s = 0
    for t in range(1, len(order) + 1):
        if t == len(order) or view[order[t]] != view[order[s]]:
            grp = np.sort(order[s:t])
            for a in range(len(grp)):
                for b in range(a):
                    out.append((int(grp[a]), int(grp[b])))
            s = t
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def ca_grid(n: int, seed: int = 1609, ld: int | None = None) -> np.ndarray:
    """uint8 [n][ld] grid: cells j <= i Bernoulli(0.5) (low bit of draw i*n+j), others 0."""
    ld = n if ld is None else ld
    g = np.zeros((n, ld), dtype=np.uint8)
    rows = max(1, (1 << 22) // max(n, 1))
    for r0 in range(0, n, rows):
        r1 = min(n, r0 + rows)
        idx = (np.arange(r0, r1, dtype=np.uint64)[:, None] * np.uint64(n)
               + np.arange(n, dtype=np.uint64)[None, :])
        bits = (splitmix64(seed, idx) & np.uint64(1)).astype(np.uint8)
        g[r0:r1, :n] = np.tril(bits, k=r0)
    return g


def at_points(n: int, seed: int = 1610) -> np.ndarray:
    """n points uniform in [0,L)^3 with L = n^(1/3) (unit density), FP32 [n][3]."""
    side = n ** (1.0 / 3.0)
    return (uniform_f64(seed, 3 * n) * side).astype(np.float32).reshape(n, 3)


def batched_sizes(count: int, lo: int = 64, hi: int = 8192, seed: int = 1609) -> np.ndarray:
    """Instance sizes floor(exp(U(ln lo, ln hi))) for a batch of uneven triangles."""
    u = uniform_f64(seed ^ 0x3C6EF372, count)
    return np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


def batched_points(sizes: np.ndarray, d: int, seed: int = 1609):
    """Concatenated N(0,1) FP32 points for a batch plus per-instance point offsets.

    Returns (x_cat [sum(sizes)][d], pt_off [count] row offsets into x_cat).
    """
    sizes = np.asarray(sizes, dtype=np.int64)
    pt_off = np.zeros(len(sizes), dtype=np.uint64)
    pt_off[1:] = np.cumsum(sizes)[:-1].astype(np.uint64)
    x = normal_f32(seed, int(sizes.sum()) * d).reshape(-1, d)
    return x, pt_off


def sphere_radius_max(n: int, dim: int, kappa: float) -> float:
    """Upper end a of the radius distribution U[0, a) that gives about kappa
    contacts per sphere among n uniform centres in the unit box (boundary
    effects ignored): two spheres meet when their centres lie within
    r_i + r_j, a ball of volume V_dim(r_i + r_j); with E[(r_i + r_j)^3] =
    3a^3/2, E[(r_i + r_j)^2] = 7a^2/6 and E[r_i + r_j] = a the expected count
    is (n-1) E[V_dim] = kappa."""
    if dim == 1:  # V = 2 s
        return kappa / (2.0 * (n - 1))
    if dim == 2:  # V = pi s^2
        return math.sqrt(kappa / ((n - 1) * math.pi * 7.0 / 6.0))
    return (kappa / ((n - 1) * (4.0 / 3.0) * math.pi * 1.5)) ** (1.0 / 3.0)  # V = 4/3 pi s^3


def spheres(n: int, dim: int = 3, kappa: float = 4.0, seed: int = 1611):
    """n spheres in the unit box (Section 5, test 3): centres U[0,1)^dim, FP32
    row-major [n][dim]; radii U[0, a) in FP32 with a from sphere_radius_max,
    about kappa contacts per sphere."""
    c = uniform_f32(seed, n * dim).reshape(n, dim)
    a = sphere_radius_max(max(n, 2), dim, kappa)
    r = (uniform_f64(seed ^ 0x2545F491, n) * a).astype(np.float32)
    return c, r
