"""The no-allocation refinement entry point (atsne_refine_subset_noalloc).

It serves callers that cannot allocate device memory while they refine, such
as a render callback of an interactive view that must not stall on cudaMalloc,
or a program with a fixed device-memory budget. Through the C ABI it must
give the same rows as the workspace-based atsne_refine_subset, on two calls in
a row that share the library's fixed scratch. Collected last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1512_01655_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def at():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1512_01655_gb300 as pkg
    assert torch.cuda.is_available()
    return pkg


def start_state(X, k, mu):
    f = oracle.forest_build(X, trees=1, top_var_dims=5, leaf_size=1, seed=3)
    idx, d2, _ = oracle.forest_query(X, f, k, 1)
    P, beta, _, _ = oracle.calibrate(d2, mu)
    return idx, d2.astype(np.float32), P.astype(np.float32), beta.astype(np.float32)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def test_noalloc_matches_workspace_refine_twice(at):
    N, D, k, mu = 3000, 48, 60, 20.0
    X = synth.gaussian_mixture(N, D, seed=31)
    idx0, d20, P0, b0 = start_state(X, k, mu)
    Xd = to_dev(X)
    subsets = [np.unique(synth.sample_rows(N, 700, seed=5)),
               np.concatenate([synth.sample_rows(N, 1500, seed=6), [7, 7]]).astype(np.int32)]
    for sub in subsets:
        sd = to_dev(sub.astype(np.int32))
        ref = [to_dev(a) for a in (idx0, d20, P0, b0)] + [torch.zeros(N, device="cuda:0")]
        at.atsne_refine_subset(Xd, sd, mu, *ref)
        got = [to_dev(a) for a in (idx0, d20, P0, b0)] + [torch.zeros(N, device="cuda:0")]
        at.atsne_refine_subset_noalloc(Xd, sd, mu, *got)
        at.atsne_check()
        # the two paths rank by FP32 distances summed in different orders, so rows
        # compare as index sets wherever the k-th/(k+1)-th gap is clear (1e-4)
        gi, ri = got[0].cpu().numpy(), ref[0].cpu().numpy()
        _, od = oracle.knn_exact(X, k + 1, queries=np.unique(sub))
        gap = (od[:, k] - od[:, k - 1]) / od[:, k]
        rows = np.unique(sub)
        for r, g in zip(rows, gap):
            if g > 1e-4:
                assert set(gi[r]) == set(ri[r]), r
        assert np.array_equal(np.delete(gi, rows, 0), np.delete(ri, rows, 0))
        assert (got[1] - ref[1]).abs().max().item() <= 1e-5 * max(1.0, ref[1].abs().max().item())
        assert (got[2] - ref[2]).abs().max().item() <= 1e-5
        assert (got[3] - ref[3]).abs().max().item() <= 1e-5 * ref[3].abs().max().item()
        assert torch.equal(got[4], ref[4])


def test_noalloc_rejects_oversized_selection(at):
    N, D, k = 3000, 8, 10
    X = to_dev(synth.gaussian_mixture(N, D, seed=2))
    sub = to_dev(np.arange(at.REFINE_NOALLOC_MAX_ROWS + 1, dtype=np.int32))
    idx = torch.zeros((N, k), dtype=torch.int32, device="cuda:0")
    d2 = torch.zeros((N, k), device="cuda:0")
    P = torch.zeros((N, k), device="cuda:0")
    with pytest.raises(at.AtsneError) as ei:
        at.atsne_refine_subset_noalloc(X, sub, 3.0, idx, d2, P)
    assert ei.value.status == at.ATSNE_ENOMEM
    assert "fixed scratch" in str(ei.value)
