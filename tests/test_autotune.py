"""Host logic of the autotuner (paper_1104_5497_gb300/autotune.py): the calibration
sample, the choice among timed candidates, the cache, and the options it hands back."""
import numpy as np

from paper_1104_5497_gb300 import autotune as A
import paper_1104_5497_gb300.nphc as N_


def test_calibration_paths_spread_over_the_whole_range():
    p = A.calibration_paths(4 ** 9, 65536)
    assert len(p) == 65536 and len(np.unique(p)) == 65536
    assert p[0] == 0 and p[-1] < 4 ** 9 and p[-1] > 4 ** 9 - 8
    assert np.all(np.diff(p) == 4)
    assert np.array_equal(A.calibration_paths(100, 1000), np.arange(100))


def test_pick_fastest_and_ties_keep_the_first_listed():
    assert A.pick({0: 10.0, 7: 9.5, 6: 9.9}) == 7
    assert A.pick({2: 5.0, 1: 5.0, 3: 6.0}) == 2
    assert A.LIST_CANDIDATES[0] == 2 and A.FP32_CANDIDATES[0] == 0   # the defaults first


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "autotune.json")
    assert A.load_cache(path) == {}
    k = A.cache_key(10, "GPU X", 152)
    A.store_cache(path, k, dict(blocks_per_sm=7, list_blocks_per_sm=2))
    A.store_cache(path, A.cache_key(8, "GPU X", 152), dict(blocks_per_sm=6, list_blocks_per_sm=1))
    d = A.load_cache(path)
    assert d[k] == dict(blocks_per_sm=7, list_blocks_per_sm=2) and len(d) == 2
    open(path, "w").write("{not json")
    assert A.load_cache(path) == {}


def test_apply_copies_the_options():
    o = N_.nphc_options()
    o.tol_sol, o.h_max, o.gamma_re, o.blocks_per_sm = 1e-10, 0.05, 0.3, 0
    t = A.apply(o, dict(blocks_per_sm=5, list_blocks_per_sm=3))
    assert (t.blocks_per_sm, t.list_blocks_per_sm) == (5, 3)
    assert (t.tol_sol, t.h_max, t.gamma_re) == (1e-10, 0.05, 0.3)
    assert o.blocks_per_sm == 0 and o.list_blocks_per_sm == 0
