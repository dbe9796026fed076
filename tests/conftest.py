import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.lib()
    return oracle


def forest_parity(gi, gd, X, o, k, checks, qcap=None, rows=None, exact=False):
    """GPU forest lists against the oracle's search over the same forest. Both
    visit the same points in the same order (the evaluated counts are compared
    by the callers), so they select from the same points: with exact distances
    (integer data, the byte path) the lists are identical; otherwise the index
    sets are identical on every row whose k-th/(k+1)-th distance among the
    evaluated points differs by more than 1e-4 (relative), and every distance
    is within 1e-5 (relative) of the oracle's."""
    import oracle
    o_idx, o_d2, o_ev = oracle.forest_query(X, o, k, checks, qcap=qcap, queries=rows)
    if exact:
        assert np.array_equal(gi, o_idx)
        assert np.array_equal(gd.astype(np.float64), o_d2)
        return o_idx, o_ev
    # the (k+1)-th evaluated point, from a search with one more neighbour that
    # visits the same points (same budget); a row that evaluated exactly k
    # points returns all of them
    o1_idx, o1_d2, o1_ev = oracle.forest_query(X, o, k + 1, checks, qcap=qcap, queries=rows)
    same_visit = o1_ev == o_ev
    for r in range(gi.shape[0]):
        if o_ev[r] <= k:
            clear = True
        elif same_visit[r] and o1_idx[r, k] >= 0:
            dk, dn = o_d2[r, k - 1], o1_d2[r, k]
            clear = (dn - dk) > 1e-4 * max(dn, 1e-300)
        else:
            clear = False
        if clear:
            assert set(gi[r]) == set(o_idx[r]), r
    scale = np.maximum(np.abs(o_d2), 1e-30)
    err = np.abs(gd.astype(np.float64) - o_d2) / scale
    assert np.all((err <= 1e-5) | (np.abs(gd - o_d2) <= 1e-5)), err.max()
    return o_idx, o_ev

