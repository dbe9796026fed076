"""Pins for the precision (Eq. 9) and refinement (Sec. 4.3) oracles."""
import numpy as np

from conftest import golden
from paper_1512_01655_gb300 import synth


def test_precision_golden(oracle_mod):
    g = golden("precision_example.json")
    rho_i, rho = oracle_mod.precision(np.array(g["approx"]), np.array(g["exact"]))
    assert np.allclose(rho_i, g["rho_i"]) and abs(rho - g["rho"]) < 1e-15


def test_precision_identity_and_order_free(oracle_mod):
    rng = np.random.default_rng(1)
    e = np.stack([rng.permutation(1000)[:90] for _ in range(20)]).astype(np.int32)
    a = np.stack([rng.permutation(r) for r in e]).astype(np.int32)
    rho_i, rho = oracle_mod.precision(a, e)
    assert np.all(rho_i == 1.0) and rho == 1.0


def test_refine_equals_full_recompute_rows(oracle_mod):
    X = synth.gaussian_mixture(600, 16, seed=6)
    k = 45
    full_idx, full_d2 = oracle_mod.knn_exact(X, k)
    full_P, full_b, _, _ = oracle_mod.calibrate(full_d2, 15.0)
    # start from a deliberately wrong state: every row's neighbours shifted
    idx = np.ascontiguousarray(np.roll(full_idx, 1, axis=0))
    d2 = np.ascontiguousarray(np.roll(full_d2, 1, axis=0))
    P = np.ascontiguousarray(np.roll(full_P, 1, axis=0))
    beta = np.roll(full_b, 1).copy()
    rho = np.full(600, 0.25)
    sub = np.array([5, 100, 599, 5, 42], np.int32)
    before = idx.copy()
    oracle_mod.refine(X, sub, k, 15.0, idx, d2, P, beta, rho)
    s = np.unique(sub)
    assert np.array_equal(idx[s], full_idx[s]) and np.array_equal(d2[s], full_d2[s])
    assert np.array_equal(P[s], full_P[s]) and np.array_equal(beta[s], full_b[s])
    assert np.all(rho[s] == 1.0)
    others = np.setdiff1d(np.arange(600), s)
    assert np.array_equal(idx[others], before[others]) and np.all(rho[others] == 0.25)
