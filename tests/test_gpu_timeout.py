"""Failure detection of the tensor-core kNN on the GPU: a bounded pipeline
wait that runs out (here made to by a limit of one nanosecond) is reported
through the device status word as ATSNE_ETIMEOUT, without a fault or a hang,
and the library stays usable: the next call, with the default limit, is
exact."""
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
    return pkg


@pytest.mark.parametrize("precision", ["fp32", "bf16_approx"])
def test_expired_pipeline_wait_is_reported_and_the_library_recovers(at, precision):
    X = synth.gaussian_mixture(20000, 64, seed=3)
    Xd = torch.from_numpy(X).to("cuda:0")
    at.atsne_check()  # nothing pending
    at.set_wait_limit(1)  # every wait that is not already satisfied runs out
    try:
        at.atsne_knn(Xd, 30, precision=precision)
        with pytest.raises(at.AtsneError) as ei:
            at.atsne_check()
        assert ei.value.status == at.ATSNE_ETIMEOUT
    finally:
        at.set_wait_limit(0)
    idx, d2 = at.atsne_knn(Xd, 30, precision=precision)
    at.atsne_check()
    rows = synth.sample_rows(X.shape[0], 16, seed=5)
    o_idx, _ = oracle.knn_exact(X, 30, queries=rows)
    g = idx.cpu().numpy()[rows]
    assert np.mean([len(set(g[r]) & set(o_idx[r])) / 30 for r in range(len(rows))]) >= 0.999
