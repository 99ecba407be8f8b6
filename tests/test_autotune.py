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


def test_candidates_list_the_defaults_first():
    assert A.STEP_CANDIDATES[0] == (3, 1e-5)
    assert A.THREADS_PER_PATH[0] == 0 and set(A.THREADS_PER_PATH) == {0, 1}


def test_apply_sets_threads_per_path_and_step_control():
    o = N_.nphc_options()
    o.max_newton_fp32, o.eps_fp32, o.threads_per_path = 3, 1e-5, 0
    t = A.apply(o, dict(blocks_per_sm=0, list_blocks_per_sm=0, threads_per_path=1,
                        max_newton_fp32=2, eps_fp32=3e-5))
    assert (t.threads_per_path, t.max_newton_fp32, t.eps_fp32) == (1, 2, 3e-5)
    assert (o.threads_per_path, o.max_newton_fp32, o.eps_fp32) == (0, 3, 1e-5)


def test_step_gate_compares_classes_and_certified_points():
    z = np.array([[1 + 1j, 2.0], [3.0, 4.0], [5.0, 6.0]])
    cls = np.array([N_.END_REAL, N_.END_NONE, N_.END_NONREAL])
    a = dict(cls=cls, z=z)
    assert A.same_certified(a, dict(cls=cls.copy(), z=z + 1e-12))
    z2 = z.copy()
    z2[1] += 5.0                      # an uncertified endpoint may move
    assert A.same_certified(a, dict(cls=cls, z=z2))
    z3 = z.copy()
    z3[2, 0] += 1e-6                  # a certified one may not
    assert not A.same_certified(a, dict(cls=cls, z=z3))
    c2 = cls.copy()
    c2[0] = N_.END_SINGULAR           # nor may a class change
    assert not A.same_certified(a, dict(cls=c2, z=z))
