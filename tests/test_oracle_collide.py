"""Pins of the collision oracle (Section 5, test 3), no GPU.

The oracle decides s = sum_k (c_i,k - c_j,k)^2 <= (r_i + r_j)^2 in FP32.  On
inputs that are multiples of 2^-10 in [0, 1) every one of those FP32
operations is exact (differences have at most 10 significant bits, squares
20, sums of three 22, (r_i + r_j)^2 22), so there the oracle must agree pair
for pair with exact integer arithmetic, with other algorithms (an interval
sweep in 1-D) and with closed forms (a touching lattice).  Invariants cover
general FP32 inputs.
"""
import itertools

import numpy as np
import pytest

import oracle

Q = 1024  # grid 2^-10


def _grid_spheres(n, dim, rmax_q, seed):
    rng = np.random.default_rng(seed)
    ci = rng.integers(0, Q, size=(n, dim))
    ri = rng.integers(0, rmax_q, size=n)
    return ci, ri, (ci / Q).astype(np.float32), (ri / Q).astype(np.float32)


def _exact_pairs(ci, ri):
    """Brute force in integers: sum of squared differences <= (r_i + r_j)^2."""
    n = len(ri)
    out = set()
    for i in range(n):
        d2 = ((ci[:i] - ci[i]) ** 2).sum(axis=1)
        rr = (ri[:i] + ri[i]) ** 2
        for j in np.nonzero(d2 <= rr)[0]:
            out.add((i, int(j)))
    return out


@pytest.mark.parametrize("dim,rmax_q", [(1, 3), (2, 40), (3, 90)])
def test_exact_brute_force_on_grid(dim, rmax_q):
    ci, ri, c, r = _grid_spheres(400, dim, rmax_q, seed=dim)
    want = _exact_pairs(ci, ri)
    cnt, pi, pj = oracle.collide_counts(c, r)
    got = set(zip(pi.tolist(), pj.tolist()))
    assert len(want) > 20 and got == want
    ref = np.zeros(len(ri), dtype=np.int64)
    for i, j in want:
        ref[i] += 1
        ref[j] += 1
    np.testing.assert_array_equal(cnt, ref)
    # increasing (i, j) order, i > j
    assert np.all(pi > pj)
    key = pi.astype(np.int64) * len(ri) + pj
    assert np.all(np.diff(key) > 0)


def test_touching_and_missing_by_one_ulp_of_the_grid():
    # 3-4-5 triangle: centres 5u apart, radii summing to exactly 5u touch; one
    # grid step less misses
    u = 8
    ci = np.array([[512, 512, 512], [512 + 3 * u, 512 + 4 * u, 512], [100, 100, 100],
                   [100, 100 + 3 * u, 100 + 4 * u]])
    ri = np.array([2 * u, 3 * u, 2 * u, 3 * u - 1])
    c, r = (ci / Q).astype(np.float32), (ri / Q).astype(np.float32)
    cnt, pi, pj = oracle.collide_counts(c, r)
    assert set(zip(pi.tolist(), pj.tolist())) == {(1, 0)}
    np.testing.assert_array_equal(cnt, [1, 1, 0, 0])


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_touching_lattice(dim):
    # k^dim lattice of spacing h = 1/8, radius h/2: each sphere touches its axis
    # neighbours only (diagonal neighbours are h sqrt(2) apart); total
    # dim k^(dim-1) (k - 1) contacts.  Radius h/2 - 2^-12 gives none.
    k = 5
    pts = np.array(list(itertools.product(range(k), repeat=dim)))
    c = (pts / 8.0).astype(np.float32)
    r = np.full(len(pts), 1 / 16, dtype=np.float32)
    cnt, pi, pj = oracle.collide_counts(c, r)
    assert len(pi) == dim * k ** (dim - 1) * (k - 1)
    interior = ((pts > 0) & (pts < k - 1)).sum(axis=1)
    edge = dim - interior
    np.testing.assert_array_equal(cnt, 2 * interior + edge)
    d = np.abs(pts[pi].astype(np.int64) - pts[pj]).sum(axis=1)
    assert np.all(d == 1)
    cnt0, pi0, _ = oracle.collide_counts(c, np.full(len(pts), 1 / 16 - 2 ** -12, dtype=np.float32))
    assert len(pi0) == 0 and not cnt0.any()


def test_interval_sweep_1d():
    # in 1-D two spheres collide iff the closed intervals [x - r, x + r]
    # overlap; a sweep over the sorted left ends finds those pairs without
    # testing every pair
    ci, ri, c, r = _grid_spheres(3000, 1, 2, seed=11)
    lo, hi = ci[:, 0] - ri, ci[:, 0] + ri
    order = sorted(range(len(ri)), key=lambda t: (lo[t], t))
    active, want = [], set()
    for t in order:
        active = [a for a in active if hi[a] >= lo[t]]
        for a in active:
            want.add((max(a, t), min(a, t)))
        active.append(t)
    _, pi, pj = oracle.collide_counts(c, r)
    assert len(want) > 100 and set(zip(pi.tolist(), pj.tolist())) == want


def test_coincident_isolated_and_tiny():
    # coincident centres with radius 0 touch (distance 0 <= 0): every pair
    c = np.full((7, 3), 0.25, dtype=np.float32)
    cnt, pi, _ = oracle.collide_counts(c, np.zeros(7, dtype=np.float32))
    assert len(pi) == 21 and np.all(cnt == 6)
    # distinct centres with radius 0: none, and a sphere never meets itself
    c = (np.arange(30, dtype=np.float32)[:, None] / 32).repeat(3, axis=1)
    cnt, pi, _ = oracle.collide_counts(c, np.zeros(30, dtype=np.float32))
    assert len(pi) == 0 and not cnt.any()
    for n in (0, 1):
        cnt, pi, _ = oracle.collide_counts(np.zeros((n, 3), np.float32), np.ones(n, np.float32))
        assert len(pi) == 0 and len(cnt) == n


def test_invariants_on_general_fp32():
    rng = np.random.default_rng(5)
    n = 700
    c = rng.random((n, 3), dtype=np.float32)
    r = (rng.random(n, dtype=np.float32) * np.float32(0.06)).astype(np.float32)
    cnt, pi, pj = oracle.collide_counts(c, r)
    pairs = set(zip(pi.tolist(), pj.tolist()))
    assert cnt.sum() == 2 * len(pi) and len(pi) > 50
    # the test is symmetric in i and j: relabelling the spheres relabels the pairs
    perm = rng.permutation(n)
    _, qi, qj = oracle.collide_counts(c[perm], r[perm])
    mapped = {(max(int(perm[a]), int(perm[b])), min(int(perm[a]), int(perm[b]))) for a, b in zip(qi, qj)}
    assert mapped == pairs
    # scaling centres and radii by 2 scales every FP32 step exactly
    _, si, sj = oracle.collide_counts(c * np.float32(2), r * np.float32(2))
    assert set(zip(si.tolist(), sj.tolist())) == pairs
    # row ranges concatenate to the whole list; single-sphere counts agree
    a_i, a_j = oracle.collide_pairs(c, r, 0, 300)
    b_i, b_j = oracle.collide_pairs(c, r, 300, n)
    np.testing.assert_array_equal(np.concatenate([a_i, b_i]), pi)
    np.testing.assert_array_equal(np.concatenate([a_j, b_j]), pj)
    idx = np.array([0, 1, 299, 300, n - 1])
    np.testing.assert_array_equal(oracle.collide_count_of(c, r, idx), cnt[idx])


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_sphere_workload_contact_rate(dim):
    # the workload recipe: radii U[0, a) with (n - 1) E[V_dim(r_i + r_j)] = kappa
    # gives about kappa contacts per sphere (fewer near the box walls)
    from paper_1609_01490_gb300 import inputs
    n, kappa = 20000, 4.0
    c, r = inputs.spheres(n, dim, kappa=kappa, seed=11)
    assert c.shape == (n, dim) and c.dtype == np.float32 and r.dtype == np.float32
    assert float(r.min()) >= 0.0 and float(r.max()) < inputs.sphere_radius_max(n, dim, kappa)
    cnt, _, _ = oracle.collide_counts(c, r)
    assert 0.85 * kappa < cnt.mean() <= 1.02 * kappa
