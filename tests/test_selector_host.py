"""Host logic of the selector (no GPU): features, candidates, the split and
the committed GB300 sweep table."""
import json
import math
import os

import numpy as np
import pytest

pytest.importorskip("torch")
TABLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1609_01490_gb300", "data",
                     "gb300_sweep.json")


@pytest.fixture(scope="module")
def sel():
    from paper_1609_01490_gb300 import build
    build.build()
    from paper_1609_01490_gb300 import selector
    return selector


def test_features_and_blocks(sel):
    from paper_1609_01490_gb300 import tri
    f = sel.features("edm", 2048, 3, tri.MAP_LAMBDA, 16)
    assert f.shape == (sel.NFEAT,) and np.all(np.isfinite(f))
    assert f[0] == 11 and f[2] == 4 and f[4] == 1 and f[7] == 1
    # launched blocks (tiles of 4 rho = 64 points): lambda m(m+1)/2, BB m^2, RB m (m/2 + 1) for
    # even m (Section 3.1, 4.2)
    assert sel._blocks("edm", 2048, 3, tri.MAP_LAMBDA, 16) == 32 * 33 / 2
    assert sel._blocks("edm", 2048, 3, tri.MAP_BB, 16) == 32 * 32
    assert sel._blocks("edm", 2048, 3, tri.MAP_RB, 16) == 32 * 17
    assert sel._blocks("at", 256, 3, tri.MAP_LAMBDA, 16) == 16 * 17 * 18 / 6
    assert math.isclose(sel._blocks("edm", 2048, 3, tri.MAP_UTM, 16), 2049 * 2048 / 2 / 256)


def test_candidates(sel):
    from paper_1609_01490_gb300 import tri
    assert len(sel.candidates("edm", 2048, 3)) == 18
    # REC only where the block count is a power of two: 1000 points in tiles of 32, 64 and 128
    # give 32, 16 and 8 block rows (all powers of two); 1100 points give 35, 18 and 9 (none)
    assert len(sel.candidates("edm", 1000, 3)) == 18
    assert len(sel.candidates("edm", 1100, 3)) == 15
    assert len(sel.candidates("at", 300, 3)) == 6
    assert all(m in (tri.MAP_LAMBDA, tri.MAP_BB) for m, _ in sel.candidates("at", 300, 3))


def test_committed_sweep_table(sel):
    table = json.load(open(TABLE))
    assert table["reps"] >= 5 and "GB300" in table["gpu"]
    groups = table["groups"]
    assert len(groups) == 32
    n_runs = sum(len(v) for v in groups.values()) * table["reps"]
    assert n_runs >= 2000
    for gkey, tbl in groups.items():
        kernel, n, d = gkey.split("|")
        assert set(tbl) == {sel.autotune_name(m, r) for m, r in sel.candidates(kernel, int(n), int(d))}
        assert all(v > 0 for v in tbl.values())
    train, held = sel.split_groups(table)
    assert sorted(train + held) == sorted(groups) and len(held) == round(0.2 * len(groups))
    assert sel.split_groups(table) == (train, held)


def test_library_features_match_selector(sel):
    # tri_select_features (host code in the library) and the trainer's features
    # list the same candidates in the same order with the same values
    from paper_1609_01490_gb300 import tri
    for kernel in ("edm", "ca", "at"):
        for n, d in ((2048, 3), (1000, 1), (4096, 128), (65536, 3), (96, 8)):
            X, maps, rhos = tri.tri_select_features(sel.KERNELS.index(kernel), n, d)
            cands = sel.candidates(kernel, n, d)
            assert list(zip(maps, rhos)) == cands
            ref = np.stack([sel.features(kernel, n, d, m, r) for m, r in cands]).astype(np.float32)
            np.testing.assert_allclose(X, ref, rtol=1e-6, atol=1e-6)
    with pytest.raises(tri.TriError):
        tri.tri_select_features(7, 100, 3)
    with pytest.raises(tri.TriError):
        tri.tri_select_features(0, 0, 3)
    assert tri.tri_select_workspace_size(64, 64) >= 1280
