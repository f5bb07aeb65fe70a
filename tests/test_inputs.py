"""The seeded input generators shared by the oracle and the CUDA path (no GPU):
splitmix64 against the output sequence of its published definition (Steele,
Lea and Flood, OOPSLA 2014; state 0, increment 0x9E3779B97F4A7C15), and the
shape, range and structure of every workload recipe."""
import math

import numpy as np

from paper_1609_01490_gb300 import inputs


def test_splitmix64_reference_sequence():
    got = inputs.splitmix64(0, np.arange(4, dtype=np.uint64))
    assert [int(v) for v in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
                                     0xF88BB8A8724C81EC]
    # counter-based: any index can be drawn on its own
    assert int(inputs.splitmix64(0, np.array([3], dtype=np.uint64))[0]) == 0xF88BB8A8724C81EC


def test_uniform_draws_are_exact_and_in_range():
    u = inputs.uniform_f32(1609, 100000)
    assert u.dtype == np.float32 and float(u.min()) >= 0.0 and float(u.max()) < 1.0
    # top 24 bits times 2^-24: every value is a multiple of 2^-24
    assert np.all((u.astype(np.float64) * 2 ** 24) % 1 == 0)
    assert abs(float(u.mean()) - 0.5) < 0.005
    # offsets continue the same stream
    np.testing.assert_array_equal(inputs.uniform_f32(1609, 10, offset=5), u[5:15])


def test_normal_draws():
    z = inputs.normal_f32(1609, 200000).astype(np.float64)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_edm_duplicates_are_planted():
    x = inputs.edm_normal_points(2000, 8, seed=3, dup_frac=0.01)
    pairs = inputs.duplicate_pairs(x)
    assert len(pairs) >= 20  # floor(1% of 2000) rows copied from other rows
    assert np.all(pairs[:, 0] > pairs[:, 1])
    assert all(np.array_equal(x[i], x[j]) for i, j in pairs)


def test_ca_grid_structure():
    n, ld = 300, 304
    g = inputs.ca_grid(n, seed=5, ld=ld)
    assert g.shape == (n, ld) and g.dtype == np.uint8
    assert not np.triu(g[:, :n], 1).any() and not g[:, n:].any()
    live = g[np.tril_indices(n)]
    assert set(np.unique(live)) <= {0, 1} and abs(float(live.mean()) - 0.5) < 0.02


def test_at_points_unit_density():
    p = inputs.at_points(1000, seed=1610)
    side = 1000 ** (1 / 3)
    assert p.shape == (1000, 3) and float(p.min()) >= 0.0 and float(p.max()) < side


def test_batched_sizes_log_uniform():
    s = inputs.batched_sizes(1000, seed=1609)
    assert s.min() >= 64 and s.max() < 8192
    # log-uniform: the median sits near the geometric mean of the range
    assert abs(math.log(float(np.median(s))) - 0.5 * (math.log(64) + math.log(8192))) < 0.2
    x, off = inputs.batched_points(s[:5], 4, seed=1)
    assert x.shape == (int(s[:5].sum()), 4) and int(off[0]) == 0 and int(off[1]) == int(s[0])


def test_sphere_radius_closed_forms():
    # a = kappa / (2 (n - 1)) in 1-D; (n - 1) pi (7/6) a^2 = kappa in 2-D; (n - 1) 2 pi a^3 = kappa in 3-D
    n, k = 1001, 4.0
    assert math.isclose(inputs.sphere_radius_max(n, 1, k), k / 2000)
    assert math.isclose((n - 1) * math.pi * 7 / 6 * inputs.sphere_radius_max(n, 2, k) ** 2, k)
    assert math.isclose((n - 1) * 2 * math.pi * inputs.sphere_radius_max(n, 3, k) ** 3, k)
