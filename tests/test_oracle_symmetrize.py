"""Pins for the symmetrisation oracle (Eq. 2 / Eq. 10)."""
import numpy as np

from conftest import golden
from paper_1512_01655_gb300 import synth


def test_golden_three_points(oracle_mod):
    g = golden("symmetrize_3pt.json")
    rp, col, val = oracle_mod.symmetrize(np.array(g["idx"]), np.array(g["P"]))
    assert rp.tolist() == g["row_ptr"] and col.tolist() == g["col"]
    assert np.allclose(val, g["val"], rtol=1e-15)


def test_matches_dense_transpose(oracle_mod):
    # Dense restatement: scatter the conditional rows into an N x N matrix and
    # add its transpose (a library transpose), divided by 2N.
    X = synth.gaussian_mixture(300, 10, seed=2)
    idx, d2 = oracle_mod.knn_exact(X, 20)
    P, _, _, _ = oracle_mod.calibrate(d2, 6.0)
    N = X.shape[0]
    C = np.zeros((N, N))
    C[np.repeat(np.arange(N), 20), idx.ravel()] = P.ravel()
    S = (C + C.T) / (2 * N)
    rp, col, val = oracle_mod.symmetrize(idx, P)
    dense = np.zeros((N, N))
    rows = np.repeat(np.arange(N), np.diff(rp))
    dense[rows, col] = val
    assert np.allclose(dense, S, rtol=1e-14, atol=0)
    assert np.array_equal(np.sort(np.flatnonzero(dense)), np.sort(np.flatnonzero(S)))


def test_invariants(oracle_mod):
    X = synth.gaussian_mixture(500, 8, seed=9)
    k = 30
    idx, d2 = oracle_mod.knn_exact(X, k)
    P, _, _, _ = oracle_mod.calibrate(d2, 10.0)
    rp, col, val = oracle_mod.symmetrize(idx, P)
    N = X.shape[0]
    nnz = rp[-1]
    assert N * k <= nnz <= 2 * N * k
    assert abs(val.sum() - 1.0) < 1e-12
    rows = np.repeat(np.arange(N), np.diff(rp))
    assert np.all(rows != col)
    for i in range(N):
        c = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c) > 0)
    # P == P^T entry by entry, bit for bit
    fwd = dict(zip(zip(rows.tolist(), col.tolist()), val.tolist()))
    for (i, j), v in fwd.items():
        assert fwd[(j, i)] == v
