"""Pins for the beta-bisection oracle (Eq. 3, Eq. 4; normaliser over N_i, Eq. 8)."""
import numpy as np
import pytest
from scipy.optimize import brentq
from scipy.special import xlogy

from conftest import golden
from paper_1512_01655_gb300 import synth


def test_golden_closed_cases(oracle_mod):
    for case in golden("calibrate_closed.json")["cases"]:
        d2 = np.array([case["d2"]])
        P, beta, perp, _ = oracle_mod.calibrate(d2, case["perplexity"])
        assert np.allclose(P[0], case["P"], rtol=0, atol=1e-10), case["name"]
        if case["beta"] is not None:
            assert abs(beta[0] - case["beta"]) < 1e-9 * case["beta"]
            assert abs(perp[0] - case["perplexity"]) < 1e-9


def two_level_entropy(beta, m, k, delta):
    """Shannon entropy -sum p ln p of m neighbours at shift 0 and k-m at shift delta."""
    u = np.exp(-beta * delta)
    Z = m + (k - m) * u
    p0, p1 = 1.0 / Z, u / Z
    return -(m * xlogy(p0, p0) + (k - m) * xlogy(p1, p1))


@pytest.mark.parametrize("m,k,delta,mu", [(1, 90, 3.0, 30.0), (5, 90, 0.25, 30.0),
                                          (10, 90, 100.0, 30.0), (2, 9, 1.0, 3.0)])
def test_two_level_against_root_finder(oracle_mod, m, k, delta, mu):
    a = 7.0
    d2 = np.array([[a] * m + [a + delta] * (k - m)])
    P, beta, perp, _ = oracle_mod.calibrate(d2, mu)
    b_star = brentq(lambda b: two_level_entropy(b, m, k, delta) - np.log(mu), 1e-12, 1e6,
                    xtol=1e-15, rtol=1e-15)
    assert abs(beta[0] - b_star) <= 1e-8 * b_star
    u = np.exp(-b_star * delta)
    Z = m + (k - m) * u
    assert np.allclose(P[0, :m], 1.0 / Z, atol=1e-10)
    assert np.allclose(P[0, m:], u / Z, atol=1e-10)


def test_rows_sum_to_one_and_hit_perplexity(oracle_mod):
    X = synth.gaussian_mixture(1000, 16, seed=3)
    _, d2 = oracle_mod.knn_exact(X, 90)
    P, beta, perp, iters = oracle_mod.calibrate(d2, 30.0)
    assert np.all(np.abs(P.sum(1) - 1.0) < 1e-12)
    assert np.all(np.abs(perp - 30.0) <= 1e-5)
    # perplexity recomputed from P with Eq. 4's base-2 form, independently
    H2 = -(P * np.log2(np.where(P > 0, P, 1.0))).sum(1)
    assert np.all(np.abs(2.0 ** H2 - 30.0) <= 1e-5)
    assert np.all(beta > 0) and np.all(iters < 200)


def test_probabilities_fall_with_distance(oracle_mod):
    rng = np.random.default_rng(0)
    d2 = np.sort(rng.uniform(1, 50, size=(50, 90)), axis=1)
    P, _, _, _ = oracle_mod.calibrate(d2, 30.0)
    assert np.all(np.diff(P, axis=1) <= 1e-15)


def test_small_perplexity_concentrates_on_nearest(oracle_mod):
    d2 = np.array([[1.0, 2.0, 3.0, 4.0, 5.0, 6.0]])
    P, _, perp, _ = oracle_mod.calibrate(d2, 1.001)
    assert P[0, 0] > 0.999 and abs(perp[0] - 1.001) < 1e-6


def test_shift_invariance(oracle_mod):
    # Adding a constant to all distances of a row multiplies every exp term of
    # Eq. 3 by the same factor, which cancels in p_{j|i}.
    rng = np.random.default_rng(4)
    d2 = np.sort(rng.uniform(0, 10, size=(20, 30)), axis=1)
    P1, b1, _, _ = oracle_mod.calibrate(d2, 10.0)
    P2, b2, _, _ = oracle_mod.calibrate(d2 + 1000.0, 10.0)
    assert np.allclose(P1, P2, atol=1e-9) and np.allclose(b1, b2, rtol=1e-9)


def test_rows_at_most_perplexity_neighbours_are_uniform(oracle_mod):
    # over n present neighbours H <= ln n, with equality only at beta = 0, so a
    # target ln(mu) >= ln n is met only in the limit beta -> 0: P = 1/n on N_i
    rng = np.random.default_rng(4)
    d2 = np.sort(rng.uniform(0.5, 9.0, size=(3, 8)), axis=1)
    d2[1, 5:] = np.inf   # 5 present
    d2[2, 3:] = np.inf   # 3 present
    for mu in (5.0, 6.5):
        P, beta, perp, _ = oracle_mod.calibrate(d2, mu)
        assert np.all(P[1, :5] == 0.2) and np.all(P[1, 5:] == 0.0) and beta[1] == 0.0
        assert np.all(P[2, :3] == 1.0 / 3) and beta[2] == 0.0 and perp[2] == 3.0
    # the limit: just below mu = n the bisection's row tends to the uniform one
    dev = []
    for eps in (1e-2, 1e-4, 1e-6):
        P, beta, _, _ = oracle_mod.calibrate(d2[1:2], 5.0 - eps)
        assert beta[0] > 0
        dev.append(np.abs(P[0, :5] - 0.2).max())
    assert dev[0] > dev[1] > dev[2] and dev[2] < 1e-2
