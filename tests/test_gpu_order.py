"""The exact kNN of a large point set against itself runs with its rows and
columns grouped by nearest centroid (each row tile streams its own groups'
columns first). The order changes only the work of the streaming filter: the
lists must equal those of the same rows asked for as a query list (which keeps
the natural order), and the oracle's (Eq. 8)."""
import numpy as np
import pytest
import torch

from paper_1512_01655_gb300 import synth
from test_gpu_parity import knn_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def at():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1512_01655_gb300 as pkg
    assert torch.cuda.is_available()
    return pkg


def _data(N, D, seed):
    X = synth.gaussian_mixture(N, D, n_centres=40, centre_sigma=3.0, seed=seed)
    return X


@pytest.mark.parametrize("N", [70000, 66001])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_ordered_lists_equal_query_lists_and_oracle(at, N, precision):
    X = _data(N, 48, seed=41)
    Xd = torch.from_numpy(X).cuda()
    k = 30
    idx, d2 = at.atsne_knn(Xd, k, precision=precision)
    rows = synth.sample_rows(N, 1500, seed=42)
    q = torch.from_numpy(rows.astype(np.int32)).cuda()
    qi, qd = at.atsne_knn(Xd, k, queries=q, precision=precision)
    at.atsne_check()
    gi, gd = idx.cpu().numpy()[rows], d2.cpu().numpy()[rows]
    # certified exact in both orders, distances in the one summation order
    assert np.array_equal(gi, qi.cpu().numpy())
    assert np.array_equal(gd, qd.cpu().numpy())
    sub = rows[:64]
    knn_parity(idx.cpu().numpy()[sub], d2.cpu().numpy()[sub], X, k, queries=sub)


@pytest.mark.parametrize("precision", ["bf16_approx", "fp8"])
def test_ordered_approximate_modes_match_query_lists(at, precision):
    # without a certificate the k best of the top-4k keys are returned; the
    # top-4k key set is the same in any column order up to keys that tie at
    # its boundary, so the lists agree up to a recall of 0.999
    N = 70000
    X = _data(N, 48, seed=43)
    Xd = torch.from_numpy(X).cuda()
    k = 30
    idx, _ = at.atsne_knn(Xd, k, precision=precision)
    rows = synth.sample_rows(N, 1500, seed=44)
    q = torch.from_numpy(rows.astype(np.int32)).cuda()
    qi, _ = at.atsne_knn(Xd, k, queries=q, precision=precision)
    at.atsne_check()
    a, b = idx.cpu().numpy()[rows], qi.cpu().numpy()
    agree = np.mean([len(np.intersect1d(a[i], b[i])) / k for i in range(len(rows))])
    assert agree >= 0.999
