"""Pins for the randomized KD-forest oracle (Sec. 4.2) against things other than itself."""
import numpy as np
import pytest

from conftest import golden
from paper_1512_01655_gb300 import synth


def test_splitmix64_published_vector(oracle_mod):
    # First five outputs of SplitMix64 seeded with 1234567, as published with
    # the generator's reference implementation (Steele, Lea, Flood 2014; Vigna).
    expect = [6457827717110365317, 3203168211198807973, 9817491932198370423,
              4593380528125082431, 16408922859458223821]
    assert [oracle_mod.splitmix64_at(1234567, c) for c in range(1, 6)] == expect


def test_golden_1d_tree_and_search(oracle_mod):
    g = golden("forest_1d.json")
    X = np.array(g["x"], np.float32)[:, None]
    f = oracle_mod.forest_build(X, trees=1, top_var_dims=5, leaf_size=1, seed=3)
    assert f["depth"] == 3
    assert f["split_val"][0].tolist() == g["split_val"]
    assert np.all(f["split_dim"] == 0)
    assert f["perm"][0].tolist() == g["perm"] and f["leaf_ofs"].tolist() == g["leaf_ofs"]
    for case in g["cases"]:
        idx, d2, ev = oracle_mod.forest_query(X, f, case["k"], case["checks"],
                                              queries=[g["query"]])
        assert idx[0].tolist() == case["idx"], case
        assert d2[0].tolist() == case["d2"], case
        assert ev[0] == case["evaluated"], case


def test_leaf_offsets_are_the_halving_rule(oracle_mod):
    for N, leaf in [(1, 1), (3, 1), (8, 1), (1000, 1), (1000, 7), (70000, 16)]:
        h = oracle_mod.forest_depth(N, leaf)
        assert -(-N // (1 << h)) <= leaf and (h == 0 or -(-N // (1 << (h - 1))) > leaf)
        ofs = oracle_mod.forest_leaf_offsets(N, h)
        sizes = np.diff(ofs)
        assert ofs[0] == 0 and ofs[-1] == N and sizes.min() >= 0 and sizes.max() <= leaf


@pytest.mark.parametrize("N,D,T,V,leaf,seed", [(300, 6, 3, 5, 1, 11), (257, 2, 2, 5, 4, 5),
                                               (500, 40, 4, 5, 8, 2), (64, 3, 1, 1, 1, 0)])
def test_tree_structure(oracle_mod, N, D, T, V, leaf, seed):
    X = synth.gaussian_mixture(N, D, n_centres=3, seed=seed)
    f = oracle_mod.forest_build(X, trees=T, top_var_dims=V, leaf_size=leaf, seed=seed)
    h = f["depth"]
    ofs = f["leaf_ofs"]
    nV = min(V, D)
    for t in range(T):
        perm = f["perm"][t]
        assert np.array_equal(np.sort(perm), np.arange(N))
        for l in range(h):
            for m in range(1 << l):
                v = (1 << l) - 1 + m
                lo, hi = ofs[m << (h - l)], ofs[(m + 1) << (h - l)]
                pts = perm[lo:hi]
                n = hi - lo
                dim = f["split_dim"][t, v]
                sv = f["split_val"][t, v]
                if n == 0:
                    continue
                var = X[pts].astype(np.float64).var(axis=0)
                order = np.lexsort((np.arange(D), -var))
                top = order[:nV]
                r = oracle_mod.splitmix64_at(seed, (t << 32) + v + 1)
                assert dim == top[r % nV], (t, v)
                vals = X[pts, dim]
                # the left child holds the first ceil(n/2) points in (value, index)
                # order, the right child the rest (children re-sort their halves later,
                # so only this partition survives in the final permutation) ...
                nl = (n + 1) // 2
                left, right = pts[:nl], pts[nl:]
                if n >= 2:
                    lmax = max(zip(X[left, dim].tolist(), left.tolist()))
                    rmin = min(zip(X[right, dim].tolist(), right.tolist()))
                    assert lmax < rmin
                    # ... and the split value is the float midpoint of the two
                    assert sv == np.float32(0.5) * (np.float32(lmax[0]) + np.float32(rmin[0]))
                    assert lmax[0] <= sv <= rmin[0]
                else:
                    assert np.isinf(sv)


def test_full_budget_gives_exact_knn(oracle_mod):
    X = synth.gaussian_mixture(400, 10, seed=8)
    f = oracle_mod.forest_build(X, trees=2, top_var_dims=5, leaf_size=3, seed=1)
    ex_idx, ex_d2 = oracle_mod.knn_exact(X, 25)
    idx, d2, ev = oracle_mod.forest_query(X, f, 25, checks=399, qcap=4096)
    assert np.array_equal(idx, ex_idx) and np.array_equal(d2, ex_d2)
    assert np.all(ev == 399)


def test_budget_only_extends_the_visit(oracle_mod):
    # No pruning: the visiting order does not depend on checks (at a fixed queue
    # capacity), so per row the evaluated set grows with the budget and rho_i can
    # only rise (Eq. 9).
    X = synth.gaussian_mixture(800, 24, seed=4)
    k = 30
    f = oracle_mod.forest_build(X, trees=3, top_var_dims=5, leaf_size=1, seed=9)
    ex_idx, _ = oracle_mod.knn_exact(X, k)
    prev = None
    for checks in [1, 32, 64, 128, 256, 799]:
        idx, d2, ev = oracle_mod.forest_query(X, f, k, checks, qcap=4096)
        assert np.all(ev == max(checks, k))
        rho_i, rho = oracle_mod.precision(idx, ex_idx)
        if prev is not None:
            assert np.all(rho_i >= prev)
        prev = rho_i
    assert np.all(prev == 1.0)


def test_greedy_setting_is_the_floor(oracle_mod):
    # T = 1, L = 1 is the paper's lowest-precision setting (Sec. 4.4).
    X = synth.gaussian_mixture(1000, 32, seed=12)
    k = 30
    ex_idx, _ = oracle_mod.knn_exact(X, k)
    f1 = oracle_mod.forest_build(X, trees=1, top_var_dims=5, leaf_size=1, seed=2)
    f4 = oracle_mod.forest_build(X, trees=4, top_var_dims=5, leaf_size=1, seed=2)
    greedy = oracle_mod.precision(oracle_mod.forest_query(X, f1, k, 1)[0], ex_idx)[1]
    for f, checks in [(f1, 128), (f4, 64), (f4, 256)]:
        rho = oracle_mod.precision(oracle_mod.forest_query(X, f, k, checks)[0], ex_idx)[1]
        assert rho >= greedy


def test_results_are_true_distances_of_evaluated_points(oracle_mod):
    X = synth.gaussian_mixture(300, 5, seed=3)
    f = oracle_mod.forest_build(X, trees=2, top_var_dims=5, leaf_size=2, seed=4)
    idx, d2, _ = oracle_mod.forest_query(X, f, 10, 40)
    ref = ((X[:, None, :].astype(np.float64) - X[idx].astype(np.float64)) ** 2).sum(-1)
    assert np.array_equal(ref, d2)
    assert np.all(np.diff(d2, axis=1) >= 0)
    assert not np.any(idx == np.arange(300)[:, None])


def test_golden_two_identical_trees_bounded_queue(oracle_mod):
    """Two identical trees and a queue of capacity 4 (hand-derived): pins which
    entry a full queue drops, the (tree, node) order of equal keys, and that a
    point found in the second tree is not evaluated again."""
    g = golden("forest_1d.json")
    t = g["two_identical_trees"]
    X = np.array(g["x"], np.float32)[:, None]
    f = oracle_mod.forest_build(X, trees=t["trees"], top_var_dims=5, leaf_size=1, seed=3)
    for case in t["cases"]:
        idx, d2, ev = oracle_mod.forest_query(X, f, case["k"], case["checks"], qcap=case["queue_cap"],
                                              queries=[g["query"]])
        assert idx[0].tolist() == case["idx"], case
        assert d2[0].tolist() == case["d2"], case
        assert ev[0] == case["evaluated"], case


def test_golden_two_distinct_trees(oracle_mod):
    """Two different trees in 2-D (hand-derived): the split choice among the
    top-V dimensions, the initial descents of both trees before the first pop,
    the cross-tree order of equal keys, evictions from a queue of capacity 4 and
    the completion of a queue that runs dry."""
    g = golden("forest_2tree.json")
    X = np.array(g["points"], np.float32)
    f = oracle_mod.forest_build(X, trees=g["trees"], top_var_dims=g["top_var_dims"], leaf_size=1,
                                seed=g["seed"])
    assert f["split_dim"].tolist() == g["split_dim"]
    assert f["split_val"].tolist() == g["split_val"]
    assert f["perm"].tolist() == g["perm"]
    for case in g["cases"]:
        idx, d2, ev = oracle_mod.forest_query(X, f, case["k"], case["checks"], qcap=case["queue_cap"],
                                              queries=[g["query"]])
        assert idx[0].tolist() == case["idx"], case
        assert d2[0].tolist() == case["d2"], case
        assert ev[0] == case["evaluated"], case
