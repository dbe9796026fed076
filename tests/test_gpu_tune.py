"""The autotuner of the exact tensor-core kNN's column split: it records a
split per shape, later calls of the shape use it, and results never depend on
it (exact neighbourhoods, Eq. 8, against the oracle)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1512_01655_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def at():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1512_01655_gb300 as pkg
    yield pkg
    pkg.atsne_tune_clear()


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_tuned_split_gives_the_same_neighbours(at, precision):
    X = synth.gaussian_mixture(9000, 48, seed=21)
    Xd = to_dev(X)
    k = 30
    rows = np.sort(np.random.default_rng(2).choice(9000, 700, replace=False)).astype(np.int32)
    q = to_dev(rows)
    at.atsne_tune_clear()
    o = at.knn_opts(precision=precision)
    ws_knn = at.workspace_bytes(at.OP_KNN, 9000, 48, k, 700, o)
    assert at.workspace_bytes(at.OP_TUNE_KNN, 9000, 48, k, 700, o) >= ws_knn
    i0, d0 = at.atsne_knn(Xd, k, queries=q, opts=o)
    splits, ms = at.atsne_tune_knn(Xd, k, queries=q, opts=o)
    assert splits >= 1 and ms > 0.0
    i1, d1 = at.atsne_knn(Xd, k, queries=q, opts=o)
    at.atsne_check()
    assert torch.equal(i0, i1) and torch.equal(d0, d1)
    o_idx, o_d2 = oracle.knn_exact(X, k + 1, queries=rows)
    clear = (o_d2[:, k] - o_d2[:, k - 1]) / o_d2[:, k] > 1e-4
    g = i1.cpu().numpy()
    for r in np.flatnonzero(clear):
        assert set(g[r]) == set(o_idx[r, :k])
    at.atsne_tune_clear()


def test_tuned_batch_refinement_equals_untuned(at):
    X, labels = synth.gaussian_mixture(12000, 32, seed=22, return_labels=True)
    subs = synth.refine_subsets(labels, 6, lo=50, hi=600, seed=3)
    lists = to_dev(np.concatenate(subs))
    N, k, mu = 12000, 30, 10.0
    Xd = to_dev(X)
    outs = []
    for tune in (False, True):
        at.atsne_tune_clear()
        if tune:
            rows_max = min(N, int(lists.numel()))
            splits, _ = at.atsne_tune_knn(Xd, k, queries=torch.arange(rows_max, dtype=torch.int32,
                                                                        device=DEV), precision="fp32")
            assert splits >= 1
        idx, d2 = at.atsne_knn(Xd, k, method="forest", trees=2, checks=64, seed=1)
        P, beta = at.atsne_calibrate_P(d2, mu)
        rho = torch.zeros(N, dtype=torch.float32, device=DEV)
        at.atsne_refine_batch(Xd, lists, mu, idx, d2, P, beta, rho)
        at.atsne_check()
        outs.append([t.cpu() for t in (idx, d2, P, beta, rho)])
    at.atsne_tune_clear()
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def test_tuner_rejects_the_forest(at):
    Xd = to_dev(synth.gaussian_mixture(500, 8, seed=1))
    with pytest.raises(at.AtsneError) as e:
        at.atsne_tune_knn(Xd, 10, method="forest")
    assert e.value.status == at.ATSNE_EUNSUPPORTED
