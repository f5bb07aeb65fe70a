"""CPU oracle for the triangular-domain maps and workloads.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg import this package; the library itself never does.
It shares no code with the CUDA path.  The heavy loops live in ``oracle.c``
(FP64, plain nested loops); the small pieces below are numpy/Python written
straight from the definitions they cite.

Paper: Navarro, Bustos, Hitschfeld, "A Non-linear GPU Thread Map for
Triangular Domains" (arXiv 1609.01490).

Parity status per function (which pin ties it to something outside itself):
  lambda_enum / tet_enum    pinned: worked examples of Section 3.1, closed
                            forms of Eq. eq_gmap and of the cubic in Section 6,
                            block counts m(m+1)/2 and T_m.
  edm_rows / edm_pairs      pinned: exact-zero duplicates, 1-D and lattice
                            closed forms, symmetry/translation invariants,
                            the triangle inequality.
  ca_step / ca_run          pinned: Life still lifes, oscillators and a glider
                            inside the triangle, plus a pure-Python brute force.
  at_energy                 pinned: equilateral, collinear and right-isosceles
                            closed forms; invariance under rigid motion and
                            permutation.
  at_energy_blocks          pinned: each block's energy equals the sum of the
                            three-point energies of its triplets, found through
                            tet_enum's order; the whole range gives at_energy.
  collide_*                 pinned: exact integer brute force on inputs where
                            FP32 is exact, a touching lattice (closed-form
                            neighbour counts), an interval sweep in 1-D,
                            coincident and isolated spheres.
  mlp_*                     pinned: central finite differences of the loss, a
                            hand-solved one-unit network, the sign property of
                            the first Adam step.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    """Load (building first if needed) the compiled oracle."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i64, u32p = ctypes.c_int64, ctypes.POINTER(ctypes.c_uint32)
        vp = ctypes.c_void_p
        L.orc_threads.restype = ctypes.c_int
        L.orc_lambda_enum.argtypes = [i64, ctypes.c_int, vp, vp]
        L.orc_lambda_enum.restype = i64
        L.orc_tet_enum.argtypes = [i64, vp, vp, vp]
        L.orc_tet_enum.restype = i64
        L.orc_edm_rows.argtypes = [vp, i64, i64, i64, i64, vp]
        L.orc_edm_pairs.argtypes = [vp, i64, vp, vp, i64, vp]
        L.orc_ca_step.argtypes = [vp, vp, i64, i64, ctypes.c_uint32, ctypes.c_uint32]
        L.orc_ca_run.argtypes = [vp, vp, i64, i64, ctypes.c_uint32, ctypes.c_uint32, i64]
        L.orc_at_energy.argtypes = [vp, i64, ctypes.c_double, vp]
        L.orc_at_energy.restype = ctypes.c_double
        L.orc_at_energy_blocks.argtypes = [vp, i64, ctypes.c_double, i64, i64, i64, vp]
        L.orc_at_energy_blocks.restype = ctypes.c_double
        L.orc_collide_rows.argtypes = [vp, vp, i64, i64, i64, vp]
        L.orc_collide_pairs.argtypes = [vp, vp, i64, i64, i64, vp, vp, vp]
        L.orc_collide_count_of.argtypes = [vp, vp, i64, i64, vp, i64, vp]
        del u32p
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    """Host threads the compiled oracle uses (OpenMP's maximum)."""
    return int(lib().orc_threads())


# ---------------------------------------------------------------- maps ----
def lambda_enum(m: int, with_diag: bool = True):
    """Block omega -> (i, j) by walking the enumeration matrix of Section 3.1."""
    cnt = m * (m + 1) // 2 if with_diag else m * (m - 1) // 2
    oi = np.empty(cnt, dtype=np.uint32)
    oj = np.empty(cnt, dtype=np.uint32)
    got = lib().orc_lambda_enum(m, 1 if with_diag else 0, _p(oi), _p(oj))
    assert got == cnt
    return oi, oj


def tet_enum(m: int):
    """Block omega -> (layer, row, col), layer >= row >= col (Section 6)."""
    cnt = m * (m + 1) * (m + 2) // 6
    a = np.empty(cnt, dtype=np.uint32)
    b = np.empty(cnt, dtype=np.uint32)
    c = np.empty(cnt, dtype=np.uint32)
    got = lib().orc_tet_enum(m, _p(a), _p(b), _p(c))
    assert got == cnt
    return a, b, c


def lambda_checksums(w_end: int, with_diag: bool = True):
    """Sums of i, j, i*i, j*j and i*j over omega in [0, w_end), row by row.

    Walks the rows of the enumeration matrix (Section 3.1): row i holds the
    omegas [T(i), T(i+1)) with j = 0..i (strict form: [T(i-1), T(i)) with
    j = 0..i-1).  Python integers, so exact for any w_end.
    """
    si = sj = sii = sjj = sij = 0
    w = 0
    i = 0 if with_diag else 1
    while w < w_end:
        width = i + 1 if with_diag else i
        cnt = min(width, w_end - w)  # j = 0 .. cnt-1 in this row
        s1 = cnt * (cnt - 1) // 2
        s2 = (cnt - 1) * cnt * (2 * cnt - 1) // 6
        si += i * cnt
        sii += i * i * cnt
        sj += s1
        sjj += s2
        sij += i * s1
        w += cnt
        i += 1
    return {"sum_i": si, "sum_j": sj, "sum_ii": sii, "sum_jj": sjj, "sum_ij": sij}


# ----------------------------------------------------------------- EDM ----
def edm_rows(x: np.ndarray, r0: int = 0, r1: int | None = None) -> np.ndarray:
    """FP64 distances of the pairs (i, j), r0 <= i < r1, j <= i, packed by row."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n, d = x.shape
    r1 = n if r1 is None else r1
    out = np.empty(r1 * (r1 + 1) // 2 - r0 * (r0 + 1) // 2, dtype=np.float64)
    lib().orc_edm_rows(_p(x), n, d, r0, r1, _p(out))
    return out


def edm_packed(x: np.ndarray) -> np.ndarray:
    """FP64 distances of every pair i >= j, packed i(i+1)/2 + j."""
    return edm_rows(x, 0, None)


def edm_pairs(x: np.ndarray, pi: np.ndarray, pj: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    pi = np.ascontiguousarray(pi, dtype=np.int64)
    pj = np.ascontiguousarray(pj, dtype=np.int64)
    out = np.empty(len(pi), dtype=np.float64)
    lib().orc_edm_pairs(_p(x), x.shape[1], _p(pi), _p(pj), len(pi), _p(out))
    return out


# ------------------------------------------------------------------ CA ----
LIFE_BIRTH = 1 << 3
LIFE_SURVIVE = (1 << 2) | (1 << 3)


def ca_step(grid: np.ndarray, birth: int = LIFE_BIRTH, survive: int = LIFE_SURVIVE) -> np.ndarray:
    g = np.ascontiguousarray(grid, dtype=np.uint8)
    out = g.copy()
    lib().orc_ca_step(_p(g), _p(out), g.shape[0], g.shape[1], birth, survive)
    return out


def ca_run(grid: np.ndarray, steps: int, birth: int = LIFE_BIRTH, survive: int = LIFE_SURVIVE) -> np.ndarray:
    a = np.ascontiguousarray(grid, dtype=np.uint8).copy()
    b = a.copy()
    lib().orc_ca_run(_p(a), _p(b), a.shape[0], a.shape[1], birth, survive, steps)
    return a if steps % 2 == 0 else b


# ------------------------------------------------------------------ AT ----
def at_energy(p: np.ndarray, nu: float = 1.0):
    """(E, sum |term|) of the Axilrod-Teller energy over all triplets i > j > k."""
    p = np.ascontiguousarray(p, dtype=np.float32)
    a = np.zeros(1, dtype=np.float64)
    e = lib().orc_at_energy(_p(p), p.shape[0], float(nu), _p(a))
    return float(e), float(a[0])


def at_energy_blocks(p: np.ndarray, rho: int, w0: int, w1: int, nu: float = 1.0):
    """(E, sum |term|) over the triplets whose tetrahedral block (i / rho, j /
    rho, k / rho) has a number in [w0, w1) of the order of tet_enum (Section 6)."""
    p = np.ascontiguousarray(p, dtype=np.float32)
    a = np.zeros(1, dtype=np.float64)
    e = lib().orc_at_energy_blocks(_p(p), p.shape[0], float(nu), int(rho), int(w0), int(w1), _p(a))
    return float(e), float(a[0])


# ------------------------------------------------------------- collide ----
def _spheres(c: np.ndarray, r: np.ndarray):
    c = np.ascontiguousarray(c, dtype=np.float32)
    if c.ndim == 1:
        c = c[:, None]
    r = np.ascontiguousarray(r, dtype=np.float32)
    assert r.shape == (c.shape[0],)
    return c, r


def collide_pairs(c: np.ndarray, r: np.ndarray, r0: int = 0, r1: int | None = None):
    """Colliding pairs (i, j), i > j, r0 <= i < r1, in increasing (i, j)
    (Section 5, test 3; the FP32 test s <= (r_i + r_j)^2 of oracle.c)."""
    c, r = _spheres(c, r)
    n, dim = c.shape
    r1 = n if r1 is None else r1
    hits = np.zeros(max(r1 - r0, 0), dtype=np.int64)
    if r1 > r0:
        lib().orc_collide_rows(_p(c), _p(r), dim, r0, r1, _p(hits))
    off = np.concatenate([[0], np.cumsum(hits)]).astype(np.int64)
    pi = np.empty(int(off[-1]), dtype=np.uint32)
    pj = np.empty(int(off[-1]), dtype=np.uint32)
    if len(pi):
        lib().orc_collide_pairs(_p(c), _p(r), dim, r0, r1, _p(off), _p(pi), _p(pj))
    return pi, pj


def collide_counts(c: np.ndarray, r: np.ndarray):
    """(per-sphere collision counts, pairs i, pairs j) over all pairs."""
    c, r = _spheres(c, r)
    pi, pj = collide_pairs(c, r)
    n = c.shape[0]
    cnt = np.bincount(pi, minlength=n) + np.bincount(pj, minlength=n)
    return cnt.astype(np.uint32), pi, pj


def collide_count_of(c: np.ndarray, r: np.ndarray, idx) -> np.ndarray:
    """Collision counts of the listed spheres alone, each against all others."""
    c, r = _spheres(c, r)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(len(idx), dtype=np.int64)
    lib().orc_collide_count_of(_p(c), _p(r), c.shape[0], c.shape[1], _p(idx), len(idx), _p(out))
    return out


# ----------------------------------------------------------------- MLP ----
# A two-hidden-layer perceptron y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 with
# mean-squared-error loss and the Adam update (Kingma and Ba, 2015).  The flat
# parameter vector holds W1 [H1][F], b1 [H1], W2 [H2][H1], b2 [H2], W3 [H2],
# b3 [1] in that order, row-major.
def mlp_sizes(f: int, h1: int = 64, h2: int = 64):
    return [(h1, f), (h1,), (h2, h1), (h2,), (1, h2), (1,)]


def mlp_unpack(theta: np.ndarray, f: int, h1: int = 64, h2: int = 64):
    out, o = [], 0
    for s in mlp_sizes(f, h1, h2):
        k = int(np.prod(s))
        out.append(np.asarray(theta[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return out


def mlp_nparams(f: int, h1: int = 64, h2: int = 64) -> int:
    return sum(int(np.prod(s)) for s in mlp_sizes(f, h1, h2))


def mlp_forward(theta, X, h1: int = 64, h2: int = 64) -> np.ndarray:
    X = np.asarray(X, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = mlp_unpack(theta, X.shape[1], h1, h2)
    a1 = np.maximum(X @ W1.T + b1, 0.0)
    a2 = np.maximum(a1 @ W2.T + b2, 0.0)
    return (a2 @ W3.T + b3)[:, 0]


def mlp_loss(theta, X, y, h1: int = 64, h2: int = 64) -> float:
    r = mlp_forward(theta, X, h1, h2) - np.asarray(y, dtype=np.float64)
    return float(np.mean(r * r))


def mlp_grad(theta, X, y, h1: int = 64, h2: int = 64):
    """(loss, gradient of the loss w.r.t. the flat parameters) by the chain rule."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    B = X.shape[0]
    W1, b1, W2, b2, W3, b3 = mlp_unpack(theta, X.shape[1], h1, h2)
    z1 = X @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    out = (a2 @ W3.T + b3)[:, 0]
    r = out - y
    loss = float(np.mean(r * r))
    g_out = (2.0 / B) * r                   # dL/dout
    gW3 = g_out[None, :] @ a2               # [1][H2]
    gb3 = np.array([g_out.sum()])
    g_a2 = g_out[:, None] * W3              # [B][H2]
    g_z2 = g_a2 * (z2 > 0)
    gW2 = g_z2.T @ a1
    gb2 = g_z2.sum(axis=0)
    g_a1 = g_z2 @ W2
    g_z1 = g_a1 * (z1 > 0)
    gW1 = g_z1.T @ X
    gb1 = g_z1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam_step(theta, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma and Ba, Algorithm 1); t counts from 1."""
    theta = np.asarray(theta, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ----------------------------------------------------------- selector ----
def regret(times: dict, pick: dict) -> float:
    """Mean of t(pick)/t(best) - 1 over the groups in ``pick``.

    ``times[group][candidate]`` is a measured time; ``pick[group]`` a candidate.
    """
    r = []
    for gkey, cand in pick.items():
        tbl = times[gkey]
        best = min(tbl.values())
        r.append(tbl[cand] / best - 1.0)
    return float(np.mean(r)) if r else math.nan
