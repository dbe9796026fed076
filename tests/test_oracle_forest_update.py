"""Pins for adding points to and removing points from the forest (Sec. 5.3.1,
Sec. 5.3.2): the tree structure stays, a new point sits in the leaf its descent
reaches, and the search over the updated forest is still the forest search."""
import numpy as np
import pytest

from paper_1512_01655_gb300 import synth


def descend_leaves(forest, X, t):
    # numpy restatement of the descent rule: value below the split -> left child
    h = forest["depth"]
    n_int = (1 << h) - 1
    sd = np.asarray(forest["split_dim"]).reshape(forest["trees"], n_int)[t]
    sv = np.asarray(forest["split_val"]).reshape(forest["trees"], n_int)[t]
    v = np.zeros(X.shape[0], np.int64)
    for _ in range(h):
        go_left = X[np.arange(X.shape[0]), sd[v]] < sv[v]
        v = np.where(go_left, 2 * v + 1, 2 * v + 2)
    return v - n_int


def buckets(forest, t):
    ofs = np.asarray(forest["leaf_ofs"])
    ofs = ofs[t] if ofs.ndim == 2 else ofs
    perm = np.asarray(forest["perm"])[t]
    return [perm[ofs[m]:ofs[m + 1]] for m in range(ofs.shape[0] - 1)]


@pytest.fixture(scope="module")
def grown(oracle_mod):
    X = synth.gaussian_mixture(1700, 12, seed=17)
    f0 = oracle_mod.forest_build(X[:1500], trees=3, top_var_dims=5, leaf_size=1, seed=4)
    f1 = oracle_mod.forest_insert(f0, X, 1500)
    return X, f0, f1


def test_inserted_points_sit_where_their_descent_ends(oracle_mod, grown):
    X, f0, f1 = grown
    for t in range(3):
        b0, b1 = buckets(f0, t), buckets(f1, t)
        leaf_of = descend_leaves(f1, X, t)
        seen = np.zeros(1700, np.int64)
        for m, (old, new) in enumerate(zip(b0, b1)):
            assert np.array_equal(new[:len(old)], old)  # old points first, unchanged
            added = new[len(old):]
            assert np.all(added >= 1500) and np.all(np.diff(added) > 0)  # index order
            assert np.all(leaf_of[added] == m)
            seen[new] += 1
        assert np.all(seen == 1)  # every point once per tree


def test_full_budget_search_after_insertion_is_exact(oracle_mod, grown):
    X, _, f1 = grown
    idx, d2, ev = oracle_mod.forest_query(X, f1, 20, checks=1700)
    e_idx, e_d2 = oracle_mod.knn_exact(X, 20)
    assert np.array_equal(idx, e_idx) and np.allclose(d2, e_d2, rtol=0, atol=0)


def test_shared_and_per_tree_offsets_search_alike(oracle_mod, grown):
    X, f0, _ = grown
    per_tree = dict(f0, leaf_ofs=np.ascontiguousarray(np.broadcast_to(f0["leaf_ofs"], (3, len(f0["leaf_ofs"])))))
    a = oracle_mod.forest_query(X[:1500], f0, 15, checks=200)
    b = oracle_mod.forest_query(X[:1500], per_tree, 15, checks=200)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_delete_undoes_insert(oracle_mod, grown):
    _, f0, f1 = grown
    back = oracle_mod.forest_delete(f1, np.arange(1500, 1700))
    assert np.array_equal(back["perm"], f0["perm"])
    for t in range(3):
        assert np.array_equal(back["leaf_ofs"][t], f0["leaf_ofs"])


def test_delete_renumbers_and_keeps_order(oracle_mod, grown):
    X, f0, _ = grown
    gone = np.arange(3, 1500, 7)
    f2 = oracle_mod.forest_delete(f0, gone)
    keep = np.setdiff1d(np.arange(1500), gone)
    newid = -np.ones(1500, np.int64)
    newid[keep] = np.arange(keep.size)
    for t in range(3):
        for old, new in zip(buckets(f0, t), buckets(f2, t)):
            assert np.array_equal(new, newid[old][newid[old] >= 0])
    # the reduced forest still searches the reduced corpus exactly at full budget
    Xr = X[:1500][keep]
    idx, _, _ = oracle_mod.forest_query(Xr, f2, 10, checks=keep.size)
    assert np.array_equal(idx, oracle_mod.knn_exact(Xr, 10)[0])


def test_update_rejects_bad_lists(oracle_mod, grown):
    _, f0, _ = grown
    with pytest.raises(Exception):
        oracle_mod.forest_delete(f0, np.array([5, 5]))
    with pytest.raises(Exception):
        oracle_mod.forest_delete(f0, np.array([1500]))
