"""Pins of the oracle's block enumerations against the paper (no GPU).

Section 3.1: the enumeration matrix D (Eq. eq_matrix_indexing), the closed
form of lambda (Eq. eq_gmap), its worked examples, and the strict-triangle
variant (Eq. eq_theorem_nodiag).  Section 4.2: the rectangular box and the
recursive partition as read, and the upper-triangular map as printed, read
1-indexed.  Section 6: tetrahedral numbers and the cubic whose
root gives the layer of a block.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _closed_form_diag(w: np.ndarray):
    # Eq. eq_gmap typed as printed: i = floor(sqrt(1/4 + 2w) - 1/2), j = w - i(i+1)/2.
    # FP64 is exact here: 8w+1 < 2^53 and sqrt is correctly rounded.
    wf = w.astype(np.float64)
    i = np.floor(np.sqrt(0.25 + 2.0 * wf) - 0.5).astype(np.int64)
    j = w.astype(np.int64) - i * (i + 1) // 2
    return i, j


def test_worked_examples(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "lambda_worked_examples.txt"))
            if l.strip() and not l.startswith("#")]
    oi, oj = orc.lambda_enum(8)
    for w, i, j in rows:
        assert (oi[int(w)], oj[int(w)]) == (int(i), int(j))
    # non-linearity: g(4) + g(3) = (4,1) != g(7) = (3,1)
    s = (int(oi[4]) + int(oi[3]), int(oj[4]) + int(oj[3]))
    assert s == (4, 1) and s != (int(oi[7]), int(oj[7]))


def test_enumeration_matrix(orc):
    lines = [l.strip() for l in open(os.path.join(GOLDEN, "enumeration_matrix.txt"))
             if l.strip() and not l.startswith("#")]
    oi, oj = orc.lambda_enum(3)
    for l in lines:
        if l.startswith("m "):
            _, m, first, last = l.split()
            m, first, last = int(m), int(first), int(last)
            ai, aj = orc.lambda_enum(m)
            assert len(ai) == m * (m + 1) // 2 == last + 1
            assert ai[first] == m - 1 and aj[first] == 0
            assert ai[last] == m - 1 and aj[last] == m - 1
            assert ai[first - 1] == m - 2
        else:
            r, nums = l.split(":")
            for c, w in enumerate(nums.split()):
                assert (oi[int(w)], oj[int(w)]) == (int(r), c)


@pytest.mark.parametrize("m", [1, 2, 3, 17, 128, 4096])
def test_enum_matches_closed_form(orc, m):
    oi, oj = orc.lambda_enum(m)
    assert len(oi) == m * (m + 1) // 2          # m(m+1)/2 blocks suffice (Section 3.1)
    i, j = _closed_form_diag(np.arange(len(oi), dtype=np.int64))
    np.testing.assert_array_equal(oi, i)
    np.testing.assert_array_equal(oj, j)
    # bijection onto {0 <= j <= i < m}
    assert np.all(oj <= oi) and np.all(oi < m)
    flat = oi.astype(np.int64) * m + oj
    assert len(np.unique(flat)) == len(flat)


@pytest.mark.parametrize("m", [2, 3, 50, 1000])
def test_nodiag_enum(orc, m):
    oi, oj = orc.lambda_enum(m, with_diag=False)
    assert len(oi) == m * (m - 1) // 2
    w = np.arange(len(oi), dtype=np.int64)
    # Eq. eq_theorem_nodiag: i = floor(sqrt(1/4 + 2w) + 1/2).  The printed
    # j = w - i(i+1)/2 is negative at w = 0; the row of i starts at i(i-1)/2.
    i = np.floor(np.sqrt(0.25 + 2.0 * w) + 0.5).astype(np.int64)
    j = w - i * (i - 1) // 2
    np.testing.assert_array_equal(oi, i)
    np.testing.assert_array_equal(oj, j)
    assert np.all(oj < oi)
    if m >= 4:
        assert [(int(a), int(b)) for a, b in zip(oi[:4], oj[:4])] == [(1, 0), (2, 0), (2, 1), (3, 0)]
    assert int(w[0] - i[0] * (i[0] + 1) // 2) == -1   # the printed j fails at omega = 0


def test_bounds_and_waste():
    # P_Delta of Section 3.1: m' = ceil(sqrt(m(m+1)/2)) per side covers the triangle;
    # the threads wasted are rho(rho-1)/2 * ceil(n/rho) (diagonal blocks' upper halves).
    for n, rho in [(2048, 16), (1000, 8), (30720, 32), (65536, 16)]:
        m = -(-n // rho)
        mp = math.isqrt(m * (m + 1) // 2)
        mp += mp * mp < m * (m + 1) // 2
        assert mp * mp >= m * (m + 1) // 2 > (mp - 1) ** 2
        if n % rho == 0:
            in_domain = n * (n + 1) // 2
            launched = (m * (m + 1) // 2) * rho * rho
            assert launched - in_domain == rho * (rho - 1) // 2 * m


def test_improvement_bound():
    # Eq. eq_I: I = 2 beta m^2 / (tau (m^2 + m)) tends to 2 beta / tau and stays in (0, 2)
    for k in [1.0, 1.2, 2.5]:
        vals = [2.0 * m * m / (k * (m * m + m)) for m in (1, 10, 1000, 10 ** 6)]
        assert all(0 < v < 2 for v in vals)
        assert abs(vals[-1] - 2.0 / k) < 1e-5


def _utm_printed(N: int, k: int):
    # Section 4.2's upper-triangular map over N items, 1-indexed pairs a < b:
    # a = floor(((2N + 1) - sqrt((2N - 1)^2 - 8k)) / 2), b = (a + 1) + k - (a - 1)(2N - a) / 2,
    # evaluated exactly: floor((2N + 1 - sqrt(D)) / 2) = floor((2N + 1 - ceil(sqrt(D))) / 2)
    # for integer D >= 0, since no integer lies strictly between sqrt(D) and its ceiling.
    D = (2 * N - 1) ** 2 - 8 * k
    r = math.isqrt(D)
    c = r if r * r == D else r + 1
    a = (2 * N + 1 - c) // 2
    b = (a + 1) + k - (a - 1) * (2 * N - a) // 2
    return a, b


def test_utm_reading_hand_values_and_bijection():
    # reading of Section 4.2: the printed formula is 1-indexed.  By hand for
    # N = 4: k = 0 .. 5 -> (1,2), (1,3), (1,4), (2,3), (2,4), (3,4).
    assert [_utm_printed(4, k) for k in range(6)] == [(1, 2), (1, 3), (1, 4), (2, 3), (2, 4), (3, 4)]
    # over N items it enumerates every pair a < b once, row by row; with
    # N = n + 1 and (i, j) = (b - 2, a - 1) that is the triangle 0 <= j <= i < n
    for n in (1, 2, 3, 7, 64, 299):
        N = n + 1
        pairs = [_utm_printed(N, k) for k in range(N * (N - 1) // 2)]
        assert pairs == [(a, b) for a in range(1, N + 1) for b in range(a + 1, N + 1)]
        tri = sorted((b - 2, a - 1) for a, b in pairs)
        assert tri == [(i, j) for i in range(n) for j in range(i + 1)]
    # the last k gives the last pair
    N = 10
    a, b = _utm_printed(N, N * (N - 1) // 2 - 1)
    assert (a, b) == (N - 1, N)


def _rb_blocks(m: int):
    # reading of Section 4.2's rectangular box at block level: a grid of m
    # columns and (m + 1) / 2 rows (odd m) or m / 2 + 1 rows (even m, whose last
    # row is used only for t_x < m / 2); block (t_x, t_y) is (m - t_y - 1,
    # m - t_x - 1) for t_x >= t_y and (t_y - 1, t_x) below.  Returns the used
    # blocks and the grid's block count.
    rows = (m + 1) // 2 if m % 2 else m // 2 + 1
    used = []
    for ty in range(rows):
        for tx in range(m):
            if m % 2 == 0 and ty == rows - 1 and tx >= m // 2:
                continue
            used.append((m - ty - 1, m - tx - 1) if tx >= ty else (ty - 1, tx))
    return used, rows * m


@pytest.mark.parametrize("m", [1, 2, 3, 4, 7, 8, 33, 64, 101])
def test_rb_reading_tiles_the_triangle(m):
    used, launched = _rb_blocks(m)
    assert sorted(used) == [(i, j) for i in range(m) for j in range(i + 1)]
    # every grid block is used for odd m; even m wastes the last row's m / 2
    assert launched - len(used) == (0 if m % 2 else m // 2)


def _rec_blocks(k: int):
    # reading of Section 4.2's recursive partition (details deferred by the
    # paper): m = 2^k block rows; level 0 is the m diagonal blocks; level l =
    # 1 .. k holds 2^(k - l) squares of side 2^(l - 1), square s covering block
    # rows [s 2^l + 2^(l - 1), (s + 1) 2^l) and columns [s 2^l, s 2^l + 2^(l - 1)).
    m = 1 << k
    levels = [[(i, i) for i in range(m)]]
    for lev in range(1, k + 1):
        side, step = 1 << (lev - 1), 1 << lev
        levels.append([(r, c) for s in range(m >> lev)
                       for r in range(s * step + side, (s + 1) * step)
                       for c in range(s * step, s * step + side)])
    return m, levels


@pytest.mark.parametrize("k", [0, 1, 2, 3, 6])
def test_rec_reading_tiles_the_triangle(k):
    m, levels = _rec_blocks(k)
    allb = [b for lev in levels for b in lev]
    assert sorted(allb) == [(i, j) for i in range(m) for j in range(i + 1)]
    # each level above the first has half the squares of the one below it
    squares = [m >> lev for lev in range(1, k + 1)]
    assert all(a == 2 * b for a, b in zip(squares, squares[1:]))
    assert len(levels) == k + 1


@pytest.mark.parametrize("m", [1, 2, 5, 24])
def test_tet_enum(orc, m):
    a, b, c = orc.tet_enum(m)
    assert len(a) == m * (m + 1) * (m + 2) // 6 == math.comb(m + 2, 3)  # T_m (Section 6)
    assert np.all((c <= b) & (b <= a) & (a < m))
    flat = (a.astype(np.int64) * m + b) * m + c
    assert len(np.unique(flat)) == len(flat)
    # layer = integer part of the real root of x^3 + 3x^2 + 2x - 6w = 0, via the
    # paper's closed form (Section 6) for w >= 1, and 0 at w = 0
    for w in range(len(a)):
        if w == 0:
            x = 0.0
        else:
            s = math.sqrt(729.0 * w * w - 3.0) + 27.0 * w
            x = s ** (1 / 3) / 3 ** (2 / 3) + 1.0 / (3 ** (1 / 3) * s ** (1 / 3)) - 1.0
            assert abs(x ** 3 + 3 * x * x + 2 * x - 6 * w) < 1e-6 * max(1, w)
        assert a[w] <= x + 1e-7 and x < a[w] + 1
        # then the 2-D map on w - T_layer gives (row, col)
        w2 = w - int(a[w]) * (int(a[w]) + 1) * (int(a[w]) + 2) // 6
        r = int(math.floor(math.sqrt(0.25 + 2 * w2) - 0.5))
        assert (b[w], c[w]) == (r, w2 - r * (r + 1) // 2)


@pytest.mark.parametrize("n", [3, 4, 10, 37])
def test_strict_triplets_from_layers(n):
    # layers L = 0..n-3 hold (L+1)(L+2)/2 strict triplets: the total is C(n,3)
    assert sum((L + 1) * (L + 2) // 2 for L in range(n - 2)) == math.comb(n, 3)


def test_lambda_checksums(orc):
    # row-walk checksums agree with direct sums over the enumeration
    for m, diag in [(60, True), (60, False)]:
        oi, oj = orc.lambda_enum(m, with_diag=diag)
        for w_end in (0, 1, 7, len(oi) // 3, len(oi)):
            cs = orc.lambda_checksums(w_end, with_diag=diag)
            i = oi[:w_end].astype(object)
            j = oj[:w_end].astype(object)
            assert cs["sum_i"] == sum(i) and cs["sum_j"] == sum(j)
            assert cs["sum_ii"] == sum(i * i) and cs["sum_jj"] == sum(j * j)
            assert cs["sum_ij"] == sum(i * j)
