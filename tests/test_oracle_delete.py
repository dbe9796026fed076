"""Oracle pins for deletion (Sec. 5.3.2) and for absent neighbours (index -1,
distance +inf) in the bisection (Eq. 3, Eq. 4), the symmetrisation (Eq. 2) and
the precision (Eq. 9)."""
import numpy as np
import pytest

import oracle
from paper_1512_01655_gb300 import synth


def _state(N=400, D=10, k=12, mu=4.0, seed=3):
    X = synth.gaussian_mixture(N, D, seed=seed)
    idx, d2 = oracle.knn_exact(X, k)
    P, beta, _, _ = oracle.calibrate(d2, mu)
    return X, idx, d2, P, beta, np.ones(N)


def test_calibrate_absent_entries_equal_the_shorter_row():
    # +inf distances are outside N_i: the row calibrates as its finite prefix
    rng = np.random.default_rng(1)
    d = np.sort(rng.random((50, 20)) * 10.0, axis=1)
    short = d[:, :14]
    padded = np.concatenate([short, np.full((50, 6), np.inf)], axis=1)
    Ps, bs, ps, _ = oracle.calibrate(short, 5.0)
    Pp, bp, pp, _ = oracle.calibrate(padded, 5.0)
    assert np.array_equal(Pp[:, :14], Ps) and np.all(Pp[:, 14:] == 0.0)
    assert np.array_equal(bp, bs) and np.array_equal(pp, ps)
    # no neighbour at all
    P0, b0, p0, it0 = oracle.calibrate(np.full((2, 5), np.inf), 2.0)
    assert np.all(P0 == 0.0) and np.all(b0 == 0.0) and np.all(p0 == 0.0) and np.all(it0 == 0)


def test_delete_keeps_exact_prefixes_of_the_reduced_set():
    X, idx, d2, P, beta, rho = _state()
    N, k = X.shape[0], idx.shape[1]
    rng = np.random.default_rng(2)
    rows = np.sort(rng.choice(N, 37, replace=False))
    Xn, i2, dd2, P2, b2, r2 = oracle.delete(X, rows, k, 4.0, idx, d2, P, beta, rho)
    keep = np.setdiff1d(np.arange(N), rows)
    assert np.array_equal(Xn, X[keep])
    # from scratch on the reduced set: every row's remaining entries are the
    # first k - r of its exact list there (the points it lost are gone and
    # nothing closer appeared); rows that lost nothing equal it
    e_idx, e_d2 = oracle.knn_exact(Xn, k)
    dead = np.zeros(N, bool)
    dead[rows] = True
    removed = dead[idx[keep]].sum(axis=1)
    assert removed.sum() > 0
    for n in range(len(keep)):
        c = k - removed[n]
        assert np.array_equal(i2[n, :c], e_idx[n, :c])
        assert np.array_equal(dd2[n, :c], e_d2[n, :c])
        assert np.all(i2[n, c:] == -1) and np.all(np.isinf(dd2[n, c:]))
        assert np.all(P2[n, c:] == 0.0)
    assert np.array_equal(r2, 1.0 - removed / k)


def test_delete_recalibrates_over_the_remaining_neighbours():
    X, idx, d2, P, beta, rho = _state(mu=4.0)
    _, i2, dd2, P2, b2, r2 = oracle.delete(X, [0, 1, 2, 50, 51], idx.shape[1], 4.0, idx, d2, P,
                                          beta, rho, tol=1e-12)
    valid = i2 >= 0
    assert np.allclose(np.where(valid, P2, 0.0).sum(axis=1), 1.0, atol=1e-12)
    # entropy from the probabilities themselves: ln(perplexity)
    with np.errstate(divide="ignore", invalid="ignore"):
        H = -np.where(P2 > 0, P2 * np.log(P2), 0.0).sum(axis=1)
    assert np.allclose(H, np.log(4.0), atol=1e-9)


def test_delete_nothing_and_rho_floor():
    X, idx, d2, P, beta, rho = _state()
    Xn, i2, dd2, P2, b2, r2 = oracle.delete(X, [], idx.shape[1], 4.0, idx, d2, P, beta, rho)
    assert np.array_equal(Xn, X) and np.array_equal(i2, idx) and np.array_equal(dd2, d2)
    assert np.allclose(P2, P, atol=1e-9) and np.array_equal(r2, rho)
    # rho never drops below zero
    _, i3, _, _, _, r3 = oracle.delete(X, np.arange(0, 400, 2), idx.shape[1], 4.0, idx, d2, P, beta,
                                       np.zeros(400))
    assert np.all(r3 == 0.0)


def test_delete_rejects_bad_lists():
    X, idx, d2, P, beta, rho = _state(N=100)
    for bad in ([3, 3], [100], [-1]):
        with pytest.raises(ValueError):
            oracle.delete(X, bad, idx.shape[1], 4.0, idx, d2, P, beta, rho)


def test_symmetrize_and_precision_skip_absent_entries():
    X, idx, d2, P, beta, rho = _state(N=300)
    _, i2, _, P2, _, _ = oracle.delete(X, [7, 8, 9], idx.shape[1], 4.0, idx, d2, P, beta, rho)
    N = i2.shape[0]
    rp, col, val = oracle.symmetrize(i2, P2)
    assert abs(val.sum() - 1.0) < 1e-12          # every row's P sums to one
    assert rp[-1] == col.shape[0]
    r = np.repeat(np.arange(N), np.diff(rp))
    assert np.all(col >= 0) and np.all(r != col)
    # an absent entry never matches, also against another absent entry
    rho_i, _ = oracle.precision(i2, i2)
    assert np.array_equal(rho_i, (i2 >= 0).sum(axis=1) / i2.shape[1])
