"""Pins for the exact-kNN oracle (Eq. 8, Sec. 3.1) against things other than itself."""
import numpy as np
import pytest

from conftest import golden
from paper_1512_01655_gb300 import synth


def brute_force(X, k, queries=None):
    """Full FP64 distance matrix by direct differences + a stable lexicographic
    sort on (distance, index): the library-routine form of Eq. 8."""
    X = X.astype(np.float64)
    q = np.arange(X.shape[0]) if queries is None else np.asarray(queries)
    D2 = ((X[q, None, :] - X[None, :, :]) ** 2).sum(-1)
    D2[np.arange(q.shape[0]), q] = np.inf
    order = np.lexsort((np.broadcast_to(np.arange(X.shape[0]), D2.shape), D2), axis=1)[:, :k]
    return order.astype(np.int32), np.take_along_axis(D2, order, 1)


@pytest.mark.parametrize("N,D,k,seed", [(50, 1, 5, 0), (120, 3, 10, 1), (300, 17, 40, 2),
                                        (91, 64, 90, 3), (257, 8, 90, 4)])
def test_matches_numpy_brute_force(oracle_mod, N, D, k, seed):
    X = synth.gaussian_mixture(N, D, n_centres=4, seed=seed)
    idx, d2 = oracle_mod.knn_exact(X, k)
    ref_idx, ref_d2 = brute_force(X, k)
    assert np.array_equal(idx, ref_idx)
    assert np.allclose(d2, ref_d2, rtol=1e-12, atol=0)


def test_integer_data_with_ties(oracle_mod):
    # Small integer coordinates give many exactly tied distances; the tie rule
    # (distance, index) must match the stable numpy ordering.
    rng = np.random.default_rng(7)
    X = rng.integers(0, 3, size=(200, 4)).astype(np.float32)
    idx, d2 = oracle_mod.knn_exact(X, 30)
    ref_idx, ref_d2 = brute_force(X, 30)
    assert np.array_equal(idx, ref_idx)
    assert np.array_equal(d2, ref_d2)


def test_lattice_golden(oracle_mod):
    g = golden("knn_lattice.json")
    n = g["grid"]
    X = np.array([[a, b] for a in range(n) for b in range(n)], np.float32)
    for case in g["cases"]:
        idx, d2 = oracle_mod.knn_exact(X, case["k"], queries=[case["query"]])
        assert idx[0].tolist() == case["idx"]
        assert d2[0].tolist() == case["d2"]


def test_duplicates_are_neighbours_self_excluded(oracle_mod):
    X = np.zeros((10, 3), np.float32)
    X[5:] = 1.0
    idx, d2 = oracle_mod.knn_exact(X, 4)
    # point 0's four nearest are the other zero points 1..4 at distance 0
    assert idx[0].tolist() == [1, 2, 3, 4] and d2[0].tolist() == [0, 0, 0, 0]
    for i in range(10):
        assert i not in idx[i]


def test_query_subset_equals_full_rows(oracle_mod):
    X = synth.gaussian_mixture(400, 12, seed=5)
    idx, d2 = oracle_mod.knn_exact(X, 20)
    q = np.array([3, 399, 0, 17, 17], np.int32)
    qi, qd = oracle_mod.knn_exact(X, 20, queries=q)
    assert np.array_equal(qi, idx[q]) and np.array_equal(qd, d2[q])


def test_rejects_bad_arguments(oracle_mod):
    X = np.zeros((5, 2), np.float32)
    with pytest.raises(ValueError):
        oracle_mod.knn_exact(X, 5)          # k > N - 1
    with pytest.raises(ValueError):
        oracle_mod.knn_exact(X, 2, queries=[7])


def test_cross_matches_numpy_brute_force(oracle_mod):
    # Eq. 8 across two point sets: no point is excluded; ties by index
    Xq = synth.gaussian_mixture(70, 6, n_centres=3, seed=6)
    Xc = synth.gaussian_mixture(130, 6, n_centres=3, seed=7)
    Xc[10] = Xq[3]  # a corpus point equal to a query: distance 0, kept
    idx, d2 = oracle_mod.knn_cross(Xq, Xc, 12)
    D2 = ((Xq.astype(np.float64)[:, None, :] - Xc.astype(np.float64)[None, :, :]) ** 2).sum(-1)
    order = np.lexsort((np.broadcast_to(np.arange(130), D2.shape), D2), axis=1)[:, :12]
    assert np.array_equal(idx, order)
    assert np.allclose(d2, np.take_along_axis(D2, order, 1), rtol=1e-12, atol=0)
    assert idx[3, 0] == 10 and d2[3, 0] == 0.0


def test_cross_against_itself_is_the_exact_knn_plus_self(oracle_mod):
    X = synth.gaussian_mixture(200, 9, n_centres=4, seed=8)
    c_idx, c_d2 = oracle_mod.knn_cross(X, X, 21)
    e_idx, e_d2 = oracle_mod.knn_exact(X, 20)
    assert np.array_equal(c_idx[:, 0], np.arange(200)) and np.all(c_d2[:, 0] == 0.0)
    assert np.array_equal(c_idx[:, 1:], e_idx) and np.array_equal(c_d2[:, 1:], e_d2)
