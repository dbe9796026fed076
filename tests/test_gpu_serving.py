"""Serving (insertion, Eq. 11 / Sec. 5.3.1; refinement, Sec. 4.3): the
primitives against the oracle, the served state against the oracle's exact
neighbourhoods of the grown corpus, and the same state whether requests run
alone or overlapped in the mix."""
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


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp32_cuda"])
def test_knn_cross_matches_oracle(at, precision):
    rng = np.random.default_rng(21)
    Xq = synth.gaussian_mixture(700, 24, seed=22)
    Xc = synth.gaussian_mixture(1500, 24, seed=23)
    for k in (1, 17, 90):
        idx, d2 = at.atsne_knn_cross(to_dev(Xq), to_dev(Xc), k, precision=precision)
        at.atsne_check()
        o_idx, o_d2 = oracle.knn_cross(Xq, Xc, k + 1 if k < 1500 else k)
        g_idx, g_d2 = idx.cpu().numpy(), d2.cpu().numpy()
        gap = (o_d2[:, k] - o_d2[:, k - 1]) / o_d2[:, k]
        clear = gap > 1e-4
        for r in np.flatnonzero(clear):
            assert set(g_idx[r]) == set(o_idx[r, :k]), r
        assert np.allclose(g_d2, o_d2[:, :k], rtol=1e-5, atol=1e-5)
    _ = rng


def test_merge_neighbors_rule(at):
    # rows of 6 sorted neighbours; candidates enter only when strictly closer
    # than the farthest, ties go to the listed (smaller) index
    k = 6
    d = np.array([[1, 2, 3, 4, 5, 6], [1, 2, 3, 4, 5, 6], [1, 1, 1, 1, 1, 1]], np.float32)
    i = np.array([[10, 11, 12, 13, 14, 15], [10, 11, 12, 13, 14, 15], [1, 2, 3, 4, 5, 6]], np.int32)
    cd = np.array([[0.5, 3.5, 9.0], [6.0, 7.0, 8.0], [0.5, 1.0, 1.0]], np.float32)
    ci = np.array([[0, 1, 2], [0, 1, 2], [0, 1, 2]], np.int32)
    idx, d2 = to_dev(i), to_dev(d)
    ch = at.atsne_merge_neighbors(idx, d2, to_dev(ci), to_dev(cd), 100).cpu().numpy()
    assert list(ch) == [1, 0, 1]
    assert idx.cpu().numpy().tolist() == [[100, 10, 11, 12, 101, 13], [10, 11, 12, 13, 14, 15],
                                          [100, 1, 2, 3, 4, 5]]
    assert d2.cpu().numpy().tolist()[0] == [0.5, 1, 2, 3, 3.5, 4]
    # random rows against numpy's k smallest of the union
    rng = np.random.default_rng(24)
    R, k, kc = 300, 20, 7
    d = np.sort(rng.random((R, k)).astype(np.float32), axis=1)
    i = rng.permutation(R * k).reshape(R, k).astype(np.int32)
    cd = np.sort(rng.random((R, kc)).astype(np.float32) * 0.8, axis=1)
    ci = np.tile(np.arange(kc, dtype=np.int32), (R, 1))
    idx, d2 = to_dev(i), to_dev(d)
    at.atsne_merge_neighbors(idx, d2, to_dev(ci), to_dev(cd), 10**6)
    for r in range(R):
        pairs = sorted(list(zip(d[r], i[r])) + list(zip(cd[r], ci[r] + 10**6)))[:k]
        assert idx.cpu().numpy()[r].tolist() == [p[1] for p in pairs]


@pytest.mark.parametrize("kind", ["integer", "gauss"])
def test_insertion_matches_oracle(at, kind):
    """Eq. 11 through the library's insertion primitives (d_i^Max of each row,
    the radius search among the new points, the merge) against oracle.insert,
    on rows with and without absent entries."""
    if kind == "integer":  # exact FP32 distances: the lists must be identical
        X = np.random.default_rng(43).integers(0, 16, size=(2600, 8)).astype(np.float32)
    else:
        X = synth.gaussian_mixture(2600, 24, seed=44)
    n_old, k = 2000, 30
    i0, d0 = oracle.knn_exact(X[:n_old], k)
    holes = np.arange(0, n_old, 7)  # absent entries, as a deletion leaves them
    i0[holes, -3:] = -1
    d0[holes, -3:] = np.inf
    d0 = d0.astype(np.float32).astype(np.float64)  # the state the library holds
    oi, od, och = oracle.insert(X, n_old, i0, d0)
    Xd, idx, d2 = to_dev(X), to_dev(i0), to_dev(d0.astype(np.float32))
    radius = at.atsne_row_dmax(d2)
    cand = at.atsne_knn_cross(Xd[:n_old], Xd[n_old:], min(k, X.shape[0] - n_old), radius_d2=radius)
    ch = at.atsne_merge_neighbors(idx, d2, cand[0], cand[1], n_old)
    at.atsne_check()
    gi, gd, gch = idx.cpu().numpy(), d2.cpu().numpy(), ch.cpu().numpy().astype(bool)
    if kind == "integer":
        assert np.array_equal(gi, oi)
        assert np.array_equal(gd.astype(np.float64), od)
        assert np.array_equal(gch, och)
        return
    # continuous data: where FP32 cannot decide as FP64 does (a new point within
    # 1e-4 of d_i^Max, or a k-th/(k+1)-th tie in the merged list) rows may differ
    Xo = X.astype(np.float64)
    dnew = ((Xo[:n_old, None, :] - Xo[None, n_old:, :]) ** 2).sum(-1)
    checked = 0
    for r in range(n_old):
        present = d0[r][i0[r] >= 0]
        dmax = present.max()
        if (np.abs(dnew[r] - dmax) <= 1e-4 * dmax).any():
            continue
        u = np.sort(np.concatenate([present, dnew[r][dnew[r] < dmax]]))
        if len(u) > k and (u[k] - u[k - 1]) <= 1e-4 * u[k]:
            continue
        assert set(gi[r]) == set(oi[r]), r
        assert gch[r] == och[r], r
        m = oi[r] >= 0
        assert np.allclose(gd[r][m], od[r][m], rtol=1e-5, atol=1e-5), r
        checked += 1
    assert checked > 0.95 * n_old
    assert och.any()


def _requests(at, X0, extra, seed):
    from paper_1512_01655_gb300.serve import Request
    rng = np.random.default_rng(seed)
    reqs, n, pos = [], X0.shape[0], 0
    for rid, size in enumerate([400, 250, 600, 300, 500]):
        if rid % 2 == 0:
            reqs.append(Request(rid, "insert", 0.0, points=extra[pos:pos + size]))
            n += size
            pos += size
        else:
            reqs.append(Request(rid, "refine", 0.0, rows=np.sort(rng.choice(n, size, replace=False)).astype(np.int32)))
    return reqs, pos


def test_served_state_is_the_exact_state_of_the_grown_corpus(at):
    from paper_1512_01655_gb300.serve import Server
    Xall = synth.gaussian_mixture(3500, 16, seed=25)
    X0, extra = Xall[:2000], Xall[2000:]
    srv = Server(X0, capacity=3500, k=30, perplexity=10.0, precision="fp32", slots=3)
    reqs, used = _requests(at, X0, extra, seed=26)
    srv.run(reqs)
    at.atsne_check()
    N = srv.N
    assert N == 2000 + used
    Xf = Xall[:N]
    assert np.array_equal(srv.X[:N].cpu().numpy(), Xf)
    o_idx, o_d2 = oracle.knn_exact(Xf, 31)
    g_idx, g_d2 = srv.idx[:N].cpu().numpy(), srv.d2[:N].cpu().numpy()
    clear = (o_d2[:, 30] - o_d2[:, 29]) / o_d2[:, 30] > 1e-4
    bad = [r for r in np.flatnonzero(clear) if set(g_idx[r]) != set(o_idx[r, :30])]
    assert not bad, bad[:5]
    assert np.allclose(g_d2, o_d2[:, :30], rtol=1e-5, atol=1e-4)
    o_P, _, _, _ = oracle.calibrate(o_d2[:, :30], 10.0)
    same = np.all(np.sort(g_idx, 1) == np.sort(o_idx[:, :30], 1), axis=1)
    gP = srv.P[:N].cpu().numpy()
    for r in np.flatnonzero(same)[::7]:
        assert np.abs(gP[r][np.argsort(g_idx[r])] - o_P[r][np.argsort(o_idx[r, :30])]).max() <= 1e-5
    assert np.all(srv.rho[:N].cpu().numpy() == 1.0)


def test_same_state_alone_and_in_the_mix(at):
    from paper_1512_01655_gb300.serve import Server
    Xall = synth.gaussian_mixture(3500, 16, seed=27)
    X0, extra = Xall[:2000], Xall[2000:]
    states = []
    for slots, spread in ((1, None), (4, 0.0), (3, 0.003)):
        srv = Server(X0, capacity=3500, k=30, perplexity=10.0, precision="bf16", slots=slots)
        reqs, _ = _requests(at, X0, extra, seed=28)
        if slots == 1:  # alone: each request admitted after the previous one finished
            served = []
            for r in reqs:
                s, _ = srv.run([r])
                served += s
        else:  # in the mix: all at once, or arriving a few ms apart
            for j, r in enumerate(reqs):
                r.arrival = 0.0 if not spread else j * spread
            served, summary = srv.run(reqs)
            assert summary["requests"] == len(reqs)
        at.atsne_check()
        N = srv.N
        states.append([t[:N].cpu().numpy() for t in (srv.X, srv.idx, srv.d2, srv.P, srv.beta, srv.rho)])
    for other in states[1:]:
        for a, b in zip(states[0], other):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp32_cuda"])
def test_knn_cross_radius_keeps_exactly_the_points_inside(at, precision):
    Xq = synth.gaussian_mixture(800, 24, seed=31)
    Xc = synth.gaussian_mixture(1200, 24, seed=32)
    k = 40
    o_idx, o_d2 = oracle.knn_cross(Xq, Xc, k)
    # radii between the 5th and 30th nearest distances, some rows with none inside
    rng = np.random.default_rng(33)
    pick = rng.integers(5, 30, size=800)
    rad = o_d2[np.arange(800), pick].astype(np.float32) * np.float32(0.999)
    rad[::17] = 0.0
    idx, d2 = at.atsne_knn_cross(to_dev(Xq), to_dev(Xc), k, precision=precision, radius_d2=to_dev(rad))
    at.atsne_check()
    g_idx, g_d2 = idx.cpu().numpy(), d2.cpu().numpy()
    for r in range(800):
        inside = o_idx[r][o_d2[r] < rad[r] * (1 - 1e-5)]
        maybe = o_idx[r][o_d2[r] < rad[r] * (1 + 1e-5)]
        got = g_idx[r][g_idx[r] >= 0]
        assert set(inside) <= set(got) <= set(maybe), r
        assert np.all(np.isinf(g_d2[r][g_idx[r] < 0]))
        assert np.all(g_d2[r][g_idx[r] >= 0] < rad[r])


def _oracle_serve(X0, extra, reqs, k, trees, checks, seed):
    """The oracle's account of a served session with a resident forest: the
    initial rows exact; an insertion adds the points to the forest's buckets
    (Sec. 5.3.1), gives them the forest search's neighbourhoods over the
    updated buckets, and updates the existing rows by Eq. 11; a refinement makes
    the listed rows exact (Sec. 4.3)."""
    idx, d2 = oracle.knn_exact(X0, k)
    f = oracle.forest_build(X0, trees=trees, top_var_dims=5, leaf_size=1, seed=seed)
    X = X0
    for r in reqs:
        n = X.shape[0]
        if r.kind == "insert":
            Xg = np.concatenate([X, r.points])
            f = oracle.forest_insert(f, Xg, n)
            ni, nd, _ = oracle.forest_query(Xg, f, k, checks, queries=np.arange(n, Xg.shape[0], dtype=np.int32))
            idx, d2, _ = oracle.insert(Xg, n, idx, d2)
            idx, d2, X = np.concatenate([idx, ni]), np.concatenate([d2, nd]), Xg
        else:
            ri, rd = oracle.knn_exact(X, k, queries=r.rows)
            idx[r.rows], d2[r.rows] = ri, rd
    return X, idx, d2


def test_forest_serving_state_matches_the_oracle(at):
    """Serving with the KD-forest resident: integer data (exact distances on
    both sides), so the served lists equal the oracle's bit for bit."""
    from paper_1512_01655_gb300.serve import Server
    rng = np.random.default_rng(41)
    Xall = rng.integers(0, 24, size=(3500, 12)).astype(np.float32)
    X0, extra = Xall[:2000], Xall[2000:]
    srv = Server(X0, capacity=3500, k=20, perplexity=6.0, precision="fp32", slots=3, forest_trees=3,
                 checks=150, seed=9)
    reqs, used = _requests(at, X0, extra, seed=42)
    srv.run(reqs)
    at.atsne_check()
    N = srv.N
    oX, o_idx, o_d2 = _oracle_serve(X0, extra, _requests(at, X0, extra, seed=42)[0], 20, 3, 150, 9)
    assert N == oX.shape[0]
    assert np.array_equal(srv.idx[:N].cpu().numpy(), o_idx)
    assert np.array_equal(srv.d2[:N].cpu().numpy().astype(np.float64), o_d2)
    # inserted rows carry the forest's estimated precision until refined
    assert 0.0 < srv.rho_forest <= 1.0
    # the resident CSR P is the symmetrisation of the served state
    rp, col, val = srv.csr()
    e_rp, e_col, e_val = at.atsne_symmetrize(srv.idx[:N], srv.P[:N])
    assert torch.equal(rp, e_rp) and torch.equal(col, e_col) and torch.equal(val, e_val)


def test_forest_serving_same_state_alone_and_in_the_mix(at):
    from paper_1512_01655_gb300.serve import Server
    Xall = synth.gaussian_mixture(3500, 16, seed=43)
    X0, extra = Xall[:2000], Xall[2000:]
    states = []
    for slots, spread in ((1, None), (4, 0.0), (3, 0.003)):
        srv = Server(X0, capacity=3500, k=30, perplexity=10.0, precision="fp32", slots=slots, forest_trees=2,
                     checks=128)
        reqs, _ = _requests(at, X0, extra, seed=44)
        if slots == 1:
            for r in reqs:
                srv.run([r])
        else:
            for j, r in enumerate(reqs):
                r.arrival = 0.0 if not spread else j * spread
            srv.run(reqs)
        at.atsne_check()
        N = srv.N
        b = srv.buckets.arrays()
        states.append([t[:N].cpu().numpy() for t in (srv.X, srv.idx, srv.d2, srv.P, srv.beta, srv.rho)] +
                      [b["perm"].cpu().numpy(), b["leaf_ofs"].cpu().numpy()] +
                      [t.cpu().numpy() for t in srv.csr()])
    for other in states[1:]:
        for a, c in zip(states[0], other):
            assert np.array_equal(a, c)
