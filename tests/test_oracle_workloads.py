"""Pins of the oracle's workloads (EDM, cellular automaton, triplet energy,
MLP cost model) against closed forms, invariants and brute force (no GPU)."""
import math

import numpy as np
import pytest

from paper_1609_01490_gb300 import inputs


# ------------------------------------------------------------------ EDM ----
def test_edm_one_dimensional_integers(orc):
    # d = 1, x_i = i: d_ij = |i - j| exactly
    x = np.arange(50, dtype=np.float32)[:, None]
    out = orc.edm_packed(x)
    i, j = np.tril_indices(50)
    np.testing.assert_array_equal(out, (i - j).astype(np.float64))


def test_edm_lattice_hypot(orc):
    # d = 2 integer lattice: d_ij = hypot(dx, dy); d = 3 Pythagorean quadruple 1,2,2 -> 3
    rng = np.random.default_rng(5)
    x = rng.integers(-20, 20, size=(40, 2)).astype(np.float32)
    out = orc.edm_packed(x)
    i, j = np.tril_indices(40)
    ref = np.array([math.hypot(float(x[a, 0] - x[b, 0]), float(x[a, 1] - x[b, 1])) for a, b in zip(i, j)])
    np.testing.assert_allclose(out, ref, rtol=1e-15, atol=0)
    y = np.array([[0, 0, 0], [1, 2, 2], [3, 6, 6]], dtype=np.float32)
    np.testing.assert_array_equal(orc.edm_packed(y), [0, 3, 0, 9, 6, 0])


def test_edm_duplicates_and_diagonal_exact_zero(orc):
    x = inputs.edm_normal_points(300, 16, seed=3, dup_frac=0.05)
    out = orc.edm_packed(x)
    dup = inputs.duplicate_pairs(x)
    assert len(dup) >= 15
    assert np.all(out[dup[:, 0] * (dup[:, 0] + 1) // 2 + dup[:, 1]] == 0.0)
    diag = np.arange(300)
    assert np.all(out[diag * (diag + 1) // 2 + diag] == 0.0)
    assert np.count_nonzero(out == 0.0) == len(dup) + 300


def test_edm_invariants(orc):
    # coordinates on a 2^-16 grid, so that adding 2.0 is exact in FP32
    x = (np.round(inputs.edm_uniform_points(120, 5, seed=11) * 65536.0) / 65536.0).astype(np.float32)
    out = orc.edm_packed(x)
    # translation by an exactly representable shift leaves every distance unchanged
    np.testing.assert_array_equal(orc.edm_packed(x + np.float32(2.0)), out)
    # triangle inequality on all triples of the first 40 points
    D = np.zeros((40, 40))
    i, j = np.tril_indices(40)
    D[i, j] = out[i * (i + 1) // 2 + j]
    D = D + D.T
    # D[a, b] <= D[a, c] + D[c, b], laid out as [a, b, c]
    assert np.all(D[:, :, None] <= D[:, None, :] + D.T[None, :, :] + 1e-12)
    # pair list and row bands agree with the whole packed triangle
    pi = np.array([0, 5, 119, 77], dtype=np.int64)
    pj = np.array([0, 2, 118, 3], dtype=np.int64)
    np.testing.assert_array_equal(orc.edm_pairs(x, pi, pj), out[pi * (pi + 1) // 2 + pj])
    band = orc.edm_rows(x, 30, 61)
    np.testing.assert_array_equal(band, out[30 * 31 // 2: 61 * 62 // 2])


# ------------------------------------------------------------------- CA ----
def _place(n, cells, ld=None):
    g = np.zeros((n, n if ld is None else ld), dtype=np.uint8)
    for i, j in cells:
        assert j <= i
        g[i, j] = 1
    return g


def _alive(g):
    return {(int(a), int(b)) for a, b in zip(*np.nonzero(g))}


def _brute_life(g):
    # plain Python: the triangle {0 <= j <= i < n}, Moore neighbourhood, B3/S23
    n = g.shape[0]
    live = {(i, j) for i in range(n) for j in range(i + 1) if g[i, j]}
    out = g.copy()
    for i in range(n):
        for j in range(i + 1):
            c = sum((i + a, j + b) in live for a in (-1, 0, 1) for b in (-1, 0, 1) if (a, b) != (0, 0))
            out[i, j] = 1 if (c == 3 or (c == 2 and (i, j) in live)) else 0
    return out


def test_ca_still_life_and_blinker(orc):
    block = [(20, 5), (20, 6), (21, 5), (21, 6)]
    g = _place(40, block)
    assert _alive(orc.ca_run(g, 7)) == set(block)
    blink = [(30, 9), (30, 10), (30, 11)]
    g = _place(40, blink)
    g1 = orc.ca_step(g)
    assert _alive(g1) == {(29, 10), (30, 10), (31, 10)}
    assert _alive(orc.ca_step(g1)) == set(blink)


def test_ca_glider_moves_down_the_triangle(orc):
    # a glider heading towards +i, +j keeps i - j fixed and so stays inside
    glider = [(10, 2), (11, 3), (12, 1), (12, 2), (12, 3)]
    g = _place(60, glider)
    for gen in range(1, 6):
        g = orc.ca_run(g, 4)
        assert _alive(g) == {(i + gen, j + gen) for i, j in glider}


def test_ca_diagonal_edge_and_upper_triangle(orc):
    # a blinker lying on the diagonal loses the cells that would fall above it
    g = _place(10, [(5, 4), (5, 5)])
    g1 = orc.ca_step(g)
    assert _alive(g1) == set()
    # random grids against plain-Python brute force, including the diagonal
    for seed in range(4):
        g = inputs.ca_grid(13, seed=seed)
        np.testing.assert_array_equal(orc.ca_step(g), _brute_life(g))
    # cells above the diagonal are never written and count as dead
    g = inputs.ca_grid(16, seed=9)
    poison = g.copy()
    iu = np.triu_indices(16, 1)
    poison[iu] = 7
    out = orc.ca_step(poison)
    np.testing.assert_array_equal(out[iu], 7)
    np.testing.assert_array_equal(np.tril(out), np.tril(orc.ca_step(g)))


def test_ca_birth_survive_masks(orc):
    # B1/S (every dead cell with exactly one neighbour is born; nothing survives)
    g = _place(9, [(4, 2)])
    out = orc.ca_step(g, birth=1 << 1, survive=0)
    assert _alive(out) == {(3, 1), (3, 2), (3, 3), (4, 1), (4, 3), (5, 1), (5, 2), (5, 3)}


# ------------------------------------------------------------------- AT ----
def test_at_closed_forms(orc):
    r = 1.25
    eq = np.array([[0, 0, 0], [r, 0, 0], [r / 2, r * math.sqrt(3) / 2, 0]], dtype=np.float32)
    e, a = orc.at_energy(eq)
    # equilateral: cos 60 deg at each vertex; FP32 coordinates perturb r^9 by ~1e-6
    assert e == pytest.approx(1.375 / r ** 9, rel=3e-6)
    col = np.array([[0, 0, 0], [r, 0, 0], [2 * r, 0, 0]], dtype=np.float32)
    e, a = orc.at_energy(col, nu=2.0)
    assert e == pytest.approx(2.0 * -0.25 / r ** 9, rel=1e-12)  # collinear: cos 0, 0, 180
    assert a == pytest.approx(abs(e))
    rt = np.array([[0, 0, 0], [r, 0, 0], [0, r, 0]], dtype=np.float32)
    e, _ = orc.at_energy(rt)
    assert e == pytest.approx(1.0 / (2.0 * math.sqrt(2.0) * r ** 9), rel=1e-12)  # right isosceles
    # regular tetrahedron of edge s: four equilateral faces
    s = math.sqrt(2.0)
    tet = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float32)
    e, _ = orc.at_energy(tet)
    assert e == pytest.approx(4 * 1.375 / (2 * s) ** 9, rel=1e-12)


def test_at_invariants(orc):
    # coordinates on a 2^-12 grid so that the shift below is exact in FP32
    p = (np.round(inputs.at_points(30, seed=4) * 4096.0) / 4096.0).astype(np.float32)
    e, a = orc.at_energy(p)
    assert a >= abs(e) > 0
    perm = p[np.random.default_rng(1).permutation(30)]
    assert orc.at_energy(perm)[0] == pytest.approx(e, rel=1e-12)
    q = (p.astype(np.float64)[:, [1, 2, 0]] + 0.5).astype(np.float32)  # axis cycle + exact shift
    assert orc.at_energy(q)[0] == pytest.approx(e, rel=1e-12)
    # three points: the energy is that one triangle's term
    e3, _ = orc.at_energy(p[:3])
    e4, _ = orc.at_energy(p[:4])
    parts = [orc.at_energy(p[list(t)])[0] for t in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))]
    assert e4 == pytest.approx(sum(parts), rel=1e-12)
    assert e3 == parts[0]


# ------------------------------------------------------------------ MLP ----
def test_mlp_gradient_finite_differences(orc):
    rng = np.random.default_rng(0)
    F, H1, H2, B = 14, 8, 6, 9
    theta = rng.normal(size=orc.mlp_nparams(F, H1, H2)) * 0.5
    X = rng.normal(size=(B, F))
    y = rng.normal(size=B)
    loss, g = orc.mlp_grad(theta, X, y, H1, H2)
    assert loss == pytest.approx(orc.mlp_loss(theta, X, y, H1, H2))
    h = 1e-6
    for k in range(len(theta)):
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        fd = (orc.mlp_loss(tp, X, y, H1, H2) - orc.mlp_loss(tm, X, y, H1, H2)) / (2 * h)
        assert fd == pytest.approx(g[k], rel=1e-5, abs=1e-7)


def test_mlp_hand_solved(orc):
    # one unit per layer: y = w3 relu(w2 relu(w1 . x + b1) + b2) + b3
    theta = np.array([2.0, -1.0, 0.5, 3.0, -2.0, 4.0, 1.5, 0.25])  # W1[1][2], b1, W2, b2, W3, b3
    X = np.array([[1.0, 1.0], [0.0, 1.0], [-3.0, 0.0]])
    # x=(1,1): z1 = 2 - 1 + 0.5 = 1.5; z2 = 3*1.5 - 2 = 2.5; y = 4*2.5 + 1.5 = 11.5
    # x=(0,1): z1 = -0.5 -> 0;        z2 = -2 -> 0;          y = 1.5
    # x=(-3,0): z1 = -5.5 -> 0;       y = 1.5
    np.testing.assert_allclose(orc.mlp_forward(theta, X, 1, 1), [11.5, 1.5, 1.5])
    assert orc.mlp_loss(theta, X, [11.5, 1.5, 2.5], 1, 1) == pytest.approx(1.0 / 3.0)


def test_adam_first_step_is_sign(orc):
    # with zero moments, the bias-corrected first step is lr * g / (|g| + eps)
    g = np.array([3.0, -0.5, 1e-3, -7.0])
    th, m, v = orc.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), rtol=1e-4)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_regret(orc):
    times = {"a": {"x": 1.0, "y": 2.0}, "b": {"x": 3.0, "y": 1.5}}
    assert orc.regret(times, {"a": "x", "b": "y"}) == 0.0
    assert orc.regret(times, {"a": "y", "b": "x"}) == pytest.approx((1.0 + 1.0) / 2)
