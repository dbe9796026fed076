"""Pins of the oracle's density view and approximation map (Eq. 12, Eq. 13,
Sec. 5.2.2) against closed forms and invariances of the definitions."""
import math

import numpy as np

import oracle


def g(d, h):
    return math.exp(-d * d / (2 * h * h)) / (2 * math.pi * h * h)


def test_single_point_closed_form():
    Y = np.array([[0.25, -0.5]], np.float32)
    # 5 x 5 pixels of side 0.5 centred on the point
    f, s, a, al = oracle.kde(Y, 0.25 - 1.25, -0.5 - 1.25, 0.5, 5, 5, 0.7, cutoff=0)
    for y in range(5):
        for x in range(5):
            d = math.hypot((x - 2) * 0.5, (y - 2) * 0.5)
            assert abs(f[y, x] - g(d, 0.7)) <= 1e-15
    assert np.all(s == 0.0) and np.all(a == 1.0) and np.all(al == 0.0)


def test_unit_mass():
    # the kernel density integrates to one: midpoint sum over +-8 h
    rng = np.random.default_rng(5)
    Y = rng.normal(0.0, 0.3, size=(7, 2)).astype(np.float32)
    h, px = 0.4, 0.05
    n = int(round(2 * (8 * h + 1.5) / px))
    f, _, _, _ = oracle.kde(Y, -(8 * h + 1.5), -(8 * h + 1.5), px, n, n, h, cutoff=0)
    assert abs(f.sum() * px * px - 1.0) < 1e-6


def test_selected_share_and_precision_mean():
    Y = np.array([[-2.0, 0.0], [2.0, 0.0]], np.float32)
    sel = np.array([1, 0], np.uint8)
    rho = np.array([0.2, 1.0], np.float32)
    # pixel centres at x = -2, 0, 2 on y = 0
    f, s, a, al = oracle.kde(Y, -3.0, -1.0, 2.0, 3, 1, 1.0, cutoff=0, k=2.0, rho=rho, selected=sel)
    ga, gb = g(0.0, 1.0), g(4.0, 1.0)
    assert abs(s[0, 1] - 0.5) < 1e-15  # the midpoint sees both equally
    assert abs(s[0, 0] - ga / (ga + gb)) < 1e-15
    assert abs(s[0, 2] - gb / (ga + gb)) < 1e-15
    r0 = float(np.float32(0.2))  # rho is held in float32
    assert abs(a[0, 1] - (r0 + 1.0) / 2) < 1e-15
    assert abs(a[0, 0] - (r0 * ga + gb) / (ga + gb)) < 1e-15
    assert np.allclose(al, 1.0 - a ** 2, rtol=0, atol=1e-15)
    assert np.allclose(f[0], [(ga + gb) / 2, (2 * g(2.0, 1.0)) / 2, (ga + gb) / 2], rtol=1e-14)


def test_constant_precision_and_lens():
    rng = np.random.default_rng(6)
    Y = rng.normal(size=(50, 2)).astype(np.float32)
    rho = np.full(50, 0.3, np.float32)
    _, s, a, al = oracle.kde(Y, -3.0, -3.0, 0.25, 24, 24, 0.5, cutoff=0, k=3.0, rho=rho)
    assert np.allclose(a, np.float32(0.3), rtol=1e-12)
    assert np.allclose(al, 1.0 - np.float64(np.float32(0.3)) ** 3, rtol=1e-12)
    assert np.all(s == 0.0)


def test_cutoff_excludes_far_points():
    Y = np.array([[0.0, 0.0]], np.float32)
    # pixel centres at distance 3.9 h (kept) and 4.1 h (dropped), cutoff 4
    f, s, a, _ = oracle.kde(Y, 3.8, -0.1, 0.2, 2, 1, 1.0, cutoff=4.0)
    # pixel centres are FP32 values (one rounding of x0 + (x + 0.5) pixel)
    cx = float(np.float32(np.float64(np.float32(0.5)) * np.float32(0.2) + np.float32(3.8)))
    cy = float(np.float32(np.float64(np.float32(0.5)) * np.float32(0.2) + np.float32(-0.1)))
    assert abs(f[0, 0] - g(math.hypot(cx, cy), 1.0)) < 1e-15
    assert f[0, 1] == 0.0 and s[0, 1] == 0.0 and a[0, 1] == 1.0


def test_translation_permutation_and_scale():
    rng = np.random.default_rng(7)
    # coordinates on a 1/1024 grid, so that shifting and doubling them is exact
    Y = (np.round(rng.normal(size=(40, 2)) * 1024) / 1024).astype(np.float32)
    rho = rng.random(40).astype(np.float32)
    sel = (rng.random(40) < 0.4).astype(np.uint8)
    base = oracle.kde(Y, -2.5, -2.0, 0.125, 40, 32, 0.6, cutoff=3.0, rho=rho, selected=sel)
    t = np.array([1.5, -0.75], np.float32)  # exactly representable shift
    moved = oracle.kde(Y + t, -2.5 + 1.5, -2.0 - 0.75, 0.125, 40, 32, 0.6, cutoff=3.0, rho=rho,
                       selected=sel)
    for u, v in zip(base, moved):
        assert np.allclose(u, v, rtol=1e-12, atol=1e-15)
    p = rng.permutation(40)
    perm = oracle.kde(Y[p], -2.5, -2.0, 0.125, 40, 32, 0.6, cutoff=3.0, rho=rho[p], selected=sel[p])
    for u, v in zip(base, perm):
        assert np.allclose(u, v, rtol=1e-12, atol=1e-15)
    c = 2.0  # scaling the plane by c scales the density by 1/c^2, the shares not at all
    sc = oracle.kde(Y * c, -2.5 * c, -2.0 * c, 0.125 * c, 40, 32, 0.6 * c, cutoff=3.0, rho=rho,
                    selected=sel)
    assert np.allclose(sc[0] * c * c, base[0], rtol=1e-12)
    for u, v in zip(base[1:], sc[1:]):
        assert np.allclose(u, v, rtol=1e-12, atol=1e-15)
