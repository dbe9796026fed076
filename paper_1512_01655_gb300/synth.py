"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random data; it holds none of the method's arithmetic
and is shared by the tests, the smoke check and the benchmark. The paper's
datasets (MNIST, TIMIT, the IMU stream; Sec. 4.4, Sec. 8) are not available, so
these mixtures stand in for their shapes:

* ``gaussian_mixture``: the small parity workload, N=2000, D=64, ten isotropic
  Gaussians (sigma 1) around centres drawn from N(0, 5^2 I).
* ``sparse_prototypes``: MNIST-shaped, N=70000, D=784, integer values in
  [0, 255] with about 80% zeros: ten sparse prototypes (20% support, values
  U(64, 255)); a sample keeps each support dimension with probability 0.95,
  switches on 2% of the other dimensions, and takes
  clip(round(prototype + N(0, 40^2)), 0, 255) on its active dimensions.
* ``gamma_clusters``: TIMIT-scale N, N=10^6, D=128, non-negative features in
  50 clusters: cluster m has a scale vector s_m ~ U(0.5, 2)^D and
  x_d = s_{m,d} * Gamma(2, 1).
* ``refine_subsets``: sizes log-uniform in [lo, hi], members drawn from one to
  three clusters (a brushed selection, Sec. 5.1.1).
* ``lognormal_clusters``: the IMU-stream-shaped serving workload (Sec. 8 of the
  paper streams IMU records): D = 50, 30 clusters, mu_{m,d} ~ N(0, 1),
  x_d = exp(mu_{m,d} + N(0, 1)).
* ``embedding_2d``: a stand-in for a 2-D tSNE layout of labelled points (the
  optimiser is not part of this library): cluster m centred on a circle of
  radius 10 at angle 2 pi m / M, points spread N(0, diag(s_x^2, s_y^2)) with
  s ~ U(0.5, 1.5) per cluster and axis.
"""
import numpy as np


def gaussian_mixture(N=2000, D=64, n_centres=10, centre_sigma=5.0, sigma=1.0, seed=1,
                     return_labels=False):
    rng = np.random.default_rng(seed)
    centres = rng.normal(0.0, centre_sigma, size=(n_centres, D))
    labels = rng.integers(0, n_centres, size=N)
    X = centres[labels] + rng.normal(0.0, sigma, size=(N, D))
    X = X.astype(np.float32)
    return (X, labels) if return_labels else X


def sparse_prototypes(N=70000, D=784, n_protos=10, support=0.20, keep=0.95, extra=0.02,
                      noise=40.0, seed=2, return_labels=False, chunk=8192):
    rng = np.random.default_rng(seed)
    proto_val = rng.uniform(64.0, 255.0, size=(n_protos, D))
    proto_sup = rng.random(size=(n_protos, D)) < support
    labels = rng.integers(0, n_protos, size=N)
    X = np.empty((N, D), np.float32)
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        lab = labels[s:e]
        active = (proto_sup[lab] & (rng.random(size=(e - s, D)) < keep)) | \
                 (rng.random(size=(e - s, D)) < extra)
        v = np.clip(np.rint(proto_val[lab] + rng.normal(0.0, noise, size=(e - s, D))), 0, 255)
        X[s:e] = np.where(active, v, 0.0).astype(np.float32)
    return (X, labels) if return_labels else X


def gamma_clusters(N=1_000_000, D=128, n_clusters=50, shape=2.0, seed=3, return_labels=False,
                   chunk=65536):
    rng = np.random.default_rng(seed)
    scales = rng.uniform(0.5, 2.0, size=(n_clusters, D))
    labels = rng.integers(0, n_clusters, size=N)
    X = np.empty((N, D), np.float32)
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        X[s:e] = (scales[labels[s:e]] * rng.gamma(shape, 1.0, size=(e - s, D))).astype(np.float32)
    return (X, labels) if return_labels else X


def refine_subsets(labels, n_subsets, lo=200, hi=20000, seed=4):
    """Brushed selections: each subset draws its size log-uniformly in [lo, hi]
    and its members uniformly from the points of one to three random clusters."""
    rng = np.random.default_rng(seed)
    labels = np.asarray(labels)
    n_cl = int(labels.max()) + 1
    members = [np.flatnonzero(labels == c) for c in range(n_cl)]
    out = []
    for _ in range(n_subsets):
        size = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        cl = rng.choice(n_cl, size=int(rng.integers(1, 4)), replace=False)
        pool = np.concatenate([members[c] for c in cl])
        size = min(size, pool.shape[0])
        out.append(np.sort(rng.choice(pool, size=size, replace=False)).astype(np.int32))
    return out


def sample_rows(N, n, seed=11):
    """A seeded sorted sample of n distinct row indices."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(N, size=min(n, N), replace=False)).astype(np.int32)


def embedding_2d(labels, seed=6):
    """A seeded 2-D layout of labelled points: cluster m on a circle of radius
    10 at angle 2 pi m / M, anisotropic Gaussian spread U(0.5, 1.5) per axis."""
    rng = np.random.default_rng(seed)
    labels = np.asarray(labels)
    M = int(labels.max()) + 1
    ang = 2 * np.pi * np.arange(M) / M
    centres = np.stack([10 * np.cos(ang), 10 * np.sin(ang)], axis=1)
    spread = rng.uniform(0.5, 1.5, size=(M, 2))
    Y = centres[labels] + spread[labels] * rng.normal(size=(labels.shape[0], 2))
    return Y.astype(np.float32)


def lognormal_clusters(N, D=50, n_clusters=30, seed=5, return_labels=False, chunk=262144):
    """Log-normal features in clusters: x_d = exp(mu_{m,d} + N(0, 1)), mu ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    mu = rng.normal(size=(n_clusters, D))
    labels = rng.integers(0, n_clusters, size=N)
    X = np.empty((N, D), np.float32)
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        X[s:e] = np.exp(mu[labels[s:e]] + rng.normal(size=(e - s, D))).astype(np.float32)
    return (X, labels) if return_labels else X
