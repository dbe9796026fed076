"""Adding points to and removing points from the forest on the GPU (Sec. 5.3.1,
Sec. 5.3.2) against the oracle: the buckets bit for bit, and the search over
the updated buckets with the oracle's visiting order."""
import numpy as np
import pytest
import torch

import oracle
from conftest import forest_parity
from paper_1512_01655_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def at():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1512_01655_gb300 as pkg
    return pkg


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def same_buckets(b, o):
    g = {a: v.cpu().numpy() for a, v in b.arrays().items()}
    assert np.array_equal(g["perm"], o["perm"])
    assert np.array_equal(g["leaf_ofs"], o["leaf_ofs"])
    sizes = np.diff(o["leaf_ofs"], axis=1)
    assert b.max_bucket == sizes.max()


def same_search(at, Xd, X, f, b, o, k, checks, exact):
    idx, d2, ev = at.atsne_forest_query(Xd, f, k, checks=checks, buckets=b)
    at.atsne_check()
    _, o_ev = forest_parity(idx.cpu().numpy(), d2.cpu().numpy(), X, o, k, checks, exact=exact)
    assert np.array_equal(ev.cpu().numpy(), o_ev)  # identical visiting order


@pytest.mark.parametrize("kind", ["gauss", "bytes"])
def test_insert_delete_and_search_match_oracle(at, kind):
    if kind == "gauss":
        X = synth.gaussian_mixture(2200, 16, seed=23)
    else:
        X = synth.sparse_prototypes(N=2200, D=784, seed=5)
    Xd = to_dev(X)
    f = at.atsne_forest_build(Xd[:1800].contiguous(), trees=3, leaf_size=1, seed=6)
    o = oracle.forest_build(X[:1800], trees=3, top_var_dims=5, leaf_size=1, seed=6)
    # two insertions: from the built forest, then from the first one's buckets
    b1 = at.atsne_forest_insert(Xd[:2000].contiguous(), f, 1800)
    o1 = oracle.forest_insert(o, X[:2000], 1800)
    same_buckets(b1, o1)
    b2 = at.atsne_forest_insert(Xd, f, 2000, buckets=b1)
    o2 = oracle.forest_insert(o1, X, 2000)
    same_buckets(b2, o2)
    same_search(at, Xd, X, f, b2, o2, 20, 300, kind == "bytes")
    # a deletion from the updated buckets, then the search over the reduced corpus
    gone = np.arange(0, 2200, 11).astype(np.int32)
    b3 = at.atsne_forest_delete(f, to_dev(gone), buckets=b2)
    at.atsne_check()
    o3 = oracle.forest_delete(o2, gone)
    same_buckets(b3, o3)
    keep = np.setdiff1d(np.arange(2200), gone)
    Xr = X[keep]
    same_search(at, to_dev(Xr), Xr, f, b3, o3, 20, 300, kind == "bytes")


def test_delete_from_the_built_forest_and_edge_cases(at):
    X = synth.gaussian_mixture(1000, 8, seed=24)
    Xd = to_dev(X)
    f = at.atsne_forest_build(Xd, trees=2, leaf_size=1, seed=2)
    o = oracle.forest_build(X, trees=2, top_var_dims=5, leaf_size=1, seed=2)
    gone = np.array([0, 17, 999], np.int32)
    b = at.atsne_forest_delete(f, to_dev(gone))
    at.atsne_check()
    same_buckets(b, oracle.forest_delete(o, gone))
    # nothing added, nothing removed: the forest's own buckets
    b0 = at.atsne_forest_insert(Xd, f, 1000)
    same_buckets(b0, oracle.forest_insert(o, X, 1000))
    b00 = at.atsne_forest_delete(f, to_dev(np.zeros(0, np.int32)))
    at.atsne_check()
    same_buckets(b00, oracle.forest_delete(o, np.zeros(0, np.int32)))
    # a row listed twice is reported through the status word
    at.atsne_forest_delete(f, to_dev(np.array([4, 4], np.int32)))
    with pytest.raises(at.AtsneError):
        at.atsne_check()


def test_search_flags_a_bucket_bound_below_the_largest_bucket(at):
    """The search sizes each query's point list by the bucket bound it is
    given; a bound below the largest bucket (a stale value) is reported through
    the status word instead of writing past a list."""
    X = synth.gaussian_mixture(1200, 8, seed=25)
    Xd = to_dev(X)
    f = at.atsne_forest_build(Xd[:1000].contiguous(), trees=2, leaf_size=1, seed=3)
    b = at.atsne_forest_insert(Xd, f, 1000)
    at.atsne_check()
    assert b.max_bucket >= 2
    at.atsne_forest_query(Xd, f, 10, checks=64, buckets=b)
    at.atsne_check()
    stale = at.ForestBuckets(b.buf, f, b.N, b.max_bucket - 1)
    at.atsne_forest_query(Xd, f, 10, checks=64, buckets=stale)
    with pytest.raises(at.AtsneError):
        at.atsne_check()
    # the library stays usable: the right bound searches cleanly again
    at.atsne_forest_query(Xd, f, 10, checks=64, buckets=b)
    at.atsne_check()


def test_many_identical_points_share_a_bucket_in_index_order(at):
    # identical rows all descend to the same leaf of every tree: thousands of
    # new points in one bucket, placed in index order as the oracle places them
    base = synth.gaussian_mixture(1800, 16, seed=29)
    dup = np.repeat(base[:2], [2500, 700], axis=0)
    X = np.ascontiguousarray(np.concatenate([base, dup]).astype(np.float32))
    Xd = to_dev(X)
    f = at.atsne_forest_build(Xd[:1800].contiguous(), trees=2, leaf_size=1, seed=8)
    o = oracle.forest_build(X[:1800], trees=2, top_var_dims=5, leaf_size=1, seed=8)
    b = at.atsne_forest_insert(Xd, f, 1800)
    at.atsne_check()
    same_buckets(b, oracle.forest_insert(o, X, 1800))
