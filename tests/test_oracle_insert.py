"""Pins of the oracle's insertion of new points (Eq. 11, Sec. 5.3.1): a
hand-derived case with ties at d_i^Max and an absent entry, and the property
that inserting into exact neighbourhoods gives the exact neighbourhoods of the
grown set (checked against numpy brute force)."""
import numpy as np

from conftest import golden


def as_d2(rows):
    return np.array([[np.inf if v is None else v for v in r] for r in rows], np.float64)


def test_insert_hand_derived_case(oracle_mod):
    g = golden("insert_1d.json")
    X = np.array(g["X"], np.float32)
    idx, d2, ch = oracle_mod.insert(X, g["n_old"], np.array(g["idx_in"], np.int32), as_d2(g["d2_in"]))
    assert idx.tolist() == g["idx_out"]
    assert np.array_equal(d2, as_d2(g["d2_out"]))
    assert ch.tolist() == g["changed"]


def brute_knn(X, rows, k):
    """k nearest of each listed row among all rows of X (self excluded), in
    (d2, index) order; FP64 direct differences."""
    Xd = X.astype(np.float64)
    out_i, out_d = [], []
    for r in rows:
        d = ((Xd - Xd[r]) ** 2).sum(axis=1)
        d[r] = np.inf
        order = np.lexsort((np.arange(len(d)), d))[:k]
        out_i.append(order)
        out_d.append(d[order])
    return np.array(out_i, np.int32), np.array(out_d)


def test_insert_into_exact_neighbourhoods_is_exact():
    # integer coordinates: exact distances with many ties, so the tie rules count
    import oracle
    rng = np.random.default_rng(41)
    n_old, B, D, k = 300, 90, 5, 10
    X = rng.integers(0, 12, size=(n_old + B, D)).astype(np.float32)
    i0, d0 = brute_knn(X[:n_old], range(n_old), k)
    idx, d2, ch = oracle.insert(X, n_old, i0, d0)
    ie, de = brute_knn(X, range(n_old), k)
    assert np.array_equal(idx, ie)
    assert np.array_equal(d2, de)
    assert np.array_equal(ch, (idx != i0).any(axis=1))
    assert ch.any() and not ch.all()


def test_insert_nothing_new_and_rows_without_neighbours():
    import oracle
    X = np.arange(12, dtype=np.float32).reshape(6, 2)
    i0, d0 = brute_knn(X, range(6), 3)
    idx, d2, ch = oracle.insert(X, 6, i0, d0)  # no new rows
    assert np.array_equal(idx, i0) and np.array_equal(d2, d0) and not ch.any()
    # a row whose entries are all absent has no d_i^Max: it takes no point
    i1 = np.full((2, 3), -1, np.int32)
    d1 = np.full((2, 3), np.inf)
    idx, d2, ch = oracle.insert(X[:4], 2, i1, d1)
    assert (idx == -1).all() and np.isinf(d2).all() and not ch.any()
