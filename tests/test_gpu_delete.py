"""Deletion of points (Sec. 5.3.2) and absent neighbours on the GPU against the
oracle: the compacted state, the bisection over the remaining neighbours, the
symmetrised P, and insertion filling the holes a deletion left."""
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
    return pkg


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _state(at, N, D, k, mu, seed):
    X = synth.gaussian_mixture(N, D, seed=seed)
    Xd = to_dev(X)
    idx, d2 = at.atsne_knn(Xd, k)
    P, beta = at.atsne_calibrate_P(d2, mu)
    rho = torch.rand(N, device=DEV, generator=torch.Generator(device=DEV).manual_seed(seed))
    return X, Xd, idx, d2, P, beta, rho


@pytest.mark.parametrize("N,D,k,R", [(3000, 16, 30, 150), (1200, 40, 90, 1), (800, 8, 12, 700)])
def test_delete_matches_oracle(at, N, D, k, R):
    mu = min(10.0, k / 3)
    X, Xd, idx, d2, P, beta, rho = _state(at, N, D, k, mu, seed=N + R)
    rows = np.sort(np.random.default_rng(R).choice(N, R, replace=False)).astype(np.int32)
    # the oracle from the same starting state
    s0 = [t.cpu().numpy() for t in (idx, d2, P, beta, rho)]
    Xo, io, do, Po, bo, ro = oracle.delete(X, rows, k, mu, s0[0], s0[1].astype(np.float64),
                                           s0[2].astype(np.float64), s0[3].astype(np.float64),
                                           s0[4].astype(np.float64))
    n = at.atsne_delete_rows(Xd, to_dev(rows), mu, idx, d2, P, beta, rho)
    at.atsne_check()
    assert n == N - R == Xo.shape[0]
    assert np.array_equal(Xd[:n].cpu().numpy(), Xo)
    assert np.array_equal(idx[:n].cpu().numpy(), io)
    gd = d2[:n].cpu().numpy()
    assert np.array_equal(np.isinf(gd), np.isinf(do))
    assert np.array_equal(gd[np.isfinite(gd)].astype(np.float64), do[np.isfinite(do)])
    assert np.abs(rho[:n].cpu().numpy() - ro).max() <= 1e-6
    assert np.abs(P[:n].cpu().numpy() - Po).max() <= 1e-5
    live = bo > 0
    assert np.allclose(beta[:n].cpu().numpy()[live], bo[live], rtol=1e-3)


def test_calibrate_with_absent_entries(at):
    rng = np.random.default_rng(3)
    d = np.sort(rng.random((400, 32)) * 5.0, axis=1).astype(np.float32)
    cut = rng.integers(3, 33, 400)
    for r, c in enumerate(cut):
        d[r, c:] = np.inf
    d[7] = np.inf  # no neighbour at all
    P, beta = at.atsne_calibrate_P(to_dev(d), 2.5)
    at.atsne_check()
    o_P, o_b, _, _ = oracle.calibrate(d.astype(np.float64), 2.5)
    assert np.abs(P.cpu().numpy() - o_P).max() <= 1e-5
    assert np.all(P.cpu().numpy()[np.isinf(d)] == 0.0) and beta[7].item() == 0.0


def test_symmetrize_after_delete(at):
    X, Xd, idx, d2, P, beta, rho = _state(at, 2000, 12, 20, 6.0, seed=5)
    rows = to_dev(np.arange(0, 2000, 17).astype(np.int32))
    n = at.atsne_delete_rows(Xd, rows, 6.0, idx, d2, P, beta, rho)
    rp, col, val = at.atsne_symmetrize(idx[:n].contiguous(), P[:n].contiguous())
    at.atsne_check()
    o_rp, o_col, o_val = oracle.symmetrize(idx[:n].cpu().numpy(), P[:n].cpu().numpy().astype(np.float64))
    assert np.array_equal(rp.cpu().numpy(), o_rp) and np.array_equal(col.cpu().numpy(), o_col)
    assert np.abs(val.cpu().numpy() - o_val).max() * n <= 1e-5


def test_insertion_after_a_deletion(at):
    # serving: a deletion request, then an insertion. An existing row takes the
    # k smallest of its remaining entries and the new points strictly closer
    # than its d_i^Max, the farthest neighbour left in N_i (Eq. 11); in a row
    # with holes such points fill them. The new rows are exact over the corpus
    # now present.
    from paper_1512_01655_gb300.serve import Request, Server
    Xall = synth.gaussian_mixture(3000, 16, seed=31)
    k = 30
    srv = Server(Xall[:2000], capacity=3000, k=k, perplexity=10.0, precision="fp32", slots=2)
    e_idx, e_d2 = srv.idx[:2000].cpu().numpy(), srv.d2[:2000].cpu().numpy()  # the initial lists
    gone = np.arange(0, 2000, 9).astype(np.int32)
    new = Xall[2000:2600]
    srv.run([Request(0, "delete", 0.0, rows=gone), Request(1, "insert", 0.0, points=new)])
    at.atsne_check()
    keep = np.setdiff1d(np.arange(2000), gone)
    Xf = np.concatenate([Xall[keep], new])
    N, n0 = srv.N, len(keep)
    assert N == Xf.shape[0] and np.array_equal(srv.X[:N].cpu().numpy(), Xf)
    g_idx = srv.idx[:N].cpu().numpy()
    # expected lists of the kept rows
    newid = -np.ones(2000, np.int64)
    newid[keep] = np.arange(n0)
    c_idx, c_d2 = oracle.knn_cross(Xall[keep], new, k)
    ok = checked = 0
    for r, i in enumerate(keep):
        rem = [(d, newid[j]) for d, j in zip(e_d2[i], e_idx[i]) if newid[j] >= 0]
        dmax = rem[-1][0] if rem else np.inf
        if np.isfinite(dmax) and any(abs(d - dmax) <= 1e-5 * dmax for d in c_d2[r]):
            continue  # a new point at d_i^Max within rounding: either side is right
        merged = sorted(rem + [(d, n0 + j) for d, j in zip(c_d2[r], c_idx[r]) if d < dmax])
        if len(merged) > k and merged[k][0] - merged[k - 1][0] <= 1e-5 * merged[k][0]:
            continue  # a near tie at the k-th place
        checked += 1
        row = g_idx[r]
        ok += (set(row[row >= 0]) == set(j for _, j in merged[:k])
               and int((row < 0).sum()) == k - min(k, len(merged)))
    assert checked > 0.9 * n0 and ok == checked
    # rows that lost neighbours and got every hole filled by closer new points
    lost = np.array([(newid[e_idx[i]] < 0).any() for i in keep])
    assert (lost & (g_idx[:n0] >= 0).all(1)).sum() > 0
    # the new rows: exact over the present corpus
    o_idx, o_d2 = oracle.knn_exact(Xf, k + 1, queries=np.arange(n0, N))
    clear = (o_d2[:, k] - o_d2[:, k - 1]) / o_d2[:, k] > 1e-4
    for r in np.flatnonzero(clear):
        assert set(g_idx[n0 + r]) == set(o_idx[r, :k])


def test_delete_edge_cases(at):
    mu, k = 4.0, 12
    X, Xd, idx, d2, P, beta, rho = _state(at, 500, 8, k, mu, seed=9)
    before = [t.clone() for t in (Xd, idx, d2, P, beta, rho)]
    # nothing deleted: the state stays, its Gaussians calibrated again (the same)
    n = at.atsne_delete_rows(Xd, to_dev(np.zeros(0, np.int32)), mu, idx, d2, P, beta, rho)
    at.atsne_check()
    assert n == 500
    for a, b in zip((Xd, idx, d2, P, beta, rho), before):
        assert torch.equal(a, b)
    # a row listed twice is refused through the status word
    n = at.atsne_delete_rows(Xd, to_dev(np.array([3, 3], np.int32)), mu, idx, d2, P, beta, rho)
    with pytest.raises(at.AtsneError):
        at.atsne_check()
    # every row deleted: nothing remains
    X, Xd, idx, d2, P, beta, rho = _state(at, 300, 8, k, mu, seed=10)
    n = at.atsne_delete_rows(Xd, to_dev(np.arange(300, dtype=np.int32)), mu, idx, d2, P, beta, rho)
    at.atsne_check()
    assert n == 0
    # more rows than the state holds: refused on the host
    with pytest.raises(at.AtsneError):
        at.atsne_delete_rows(Xd, to_dev(np.arange(301, dtype=np.int32) % 300), mu, idx, d2, P, beta,
                             rho, N=300)


def test_update_is_a_deletion_then_an_insertion(at):
    # Sec. 5.3.3: a changed point is removed and added again. An "update"
    # request equals a deletion request followed by an insertion request.
    from paper_1512_01655_gb300.serve import Request, Server
    Xall = synth.gaussian_mixture(2500, 12, seed=41)
    rows = np.array([5, 9, 300, 1999], np.int32)
    new = Xall[2000:2004]
    a = Server(Xall[:2000], capacity=2100, k=20, perplexity=6.0, precision="fp32", slots=2)
    b = Server(Xall[:2000], capacity=2100, k=20, perplexity=6.0, precision="fp32", slots=2)
    a.run([Request(0, "update", 0.0, rows=rows, points=new),
           Request(1, "insert", 0.0, points=Xall[2004:2050])])
    b.run([Request(0, "delete", 0.0, rows=rows), Request(1, "insert", 0.0, points=new),
           Request(2, "insert", 0.0, points=Xall[2004:2050])])
    at.atsne_check()
    assert a.N == b.N == 2046
    for t in ("X", "idx", "d2", "P", "beta", "rho"):
        assert torch.equal(getattr(a, t)[:a.N], getattr(b, t)[:b.N]), t
    keep = np.setdiff1d(np.arange(2000), rows)
    assert np.array_equal(a.X[:a.N].cpu().numpy(), np.concatenate([Xall[keep], Xall[2000:2050]]))
