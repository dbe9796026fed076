"""GPU parity: every kernel of the library against the FP64 oracle on the same
seeded inputs, element by element (idx bit-exact where the k-th/(k+1)-th gap
exceeds 1e-4 relative; P within 1e-5 absolute; N*p_ij within 1e-5)."""
import numpy as np
import pytest
import torch

import oracle
from conftest import forest_parity
from paper_1512_01655_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def at():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1512_01655_gb300 as pkg
    assert torch.cuda.is_available()
    return pkg


DEV = "cuda:0"
PRECISIONS = ["fp32", "bf16", "fp32_cuda"]


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def knn_parity(g_idx, g_d2, X, k, queries=None, rtol=1e-5, exact_lists=True):
    """Compare GPU kNN rows with the oracle's. exact_lists: the lists equal the
    oracle's, index for index on every row (near ties are settled in FP64 as
    the oracle orders them). Always: index sets identical on rows whose
    k-th/(k+1)-th gap exceeds 1e-4 relative; elsewhere every point strictly
    inside the k-th distance (by 1e-4) is present; distances per position."""
    N = X.shape[0]
    kk = min(k + 1, N - 1)
    o_idx, o_d2 = oracle.knn_exact(X, kk, queries=queries)
    if exact_lists:
        diff = np.flatnonzero((g_idx != o_idx[:, :k]).any(axis=1))
        assert diff.size == 0, "lists differ from the oracle's on %d rows, first %d" % (diff.size, diff[0])
    dk = o_d2[:, k - 1]
    if kk > k:
        dn = o_d2[:, kk - 1]
        gap = (dn - dk) / np.maximum(dn, 1e-300)
    else:  # k = N - 1: every other point is a neighbour
        gap = np.full_like(dk, np.inf)
    clear = gap > 1e-4
    bad = [r for r in np.flatnonzero(clear) if set(g_idx[r]) != set(o_idx[r, :k])]
    assert not bad, "index sets differ on %d clear rows, first %d" % (len(bad), bad[0])
    for r in np.flatnonzero(~clear):
        inside = o_idx[r, :k][o_d2[r, :k] < dk[r] * (1 - 1e-4)]
        assert set(inside) <= set(g_idx[r]), r
    scale = np.maximum(np.abs(o_d2[:, :k]), 1e-30)
    err = np.abs(g_d2.astype(np.float64) - o_d2[:, :k]) / scale
    assert np.all((err <= rtol) | (np.abs(g_d2 - o_d2[:, :k]) <= 1e-5)), err.max()
    assert np.all(np.diff(g_d2, axis=1) >= 0)
    return clear.mean()


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("N,D,k,seed", [(2000, 64, 90, 1), (91, 1, 90, 2), (100, 3, 10, 3),
                                        (257, 17, 40, 4), (777, 784, 90, 5), (130, 128, 33, 6),
                                        (1000, 200, 90, 7)])
def test_knn_exact_continuous(at, N, D, k, seed, precision):
    X = synth.gaussian_mixture(N, D, seed=seed)
    idx, d2 = at.atsne_knn(to_dev(X), k, precision=precision)
    frac = knn_parity(idx.cpu().numpy(), d2.cpu().numpy(), X, k)
    assert frac > 0.5  # most rows have a clear k-th/(k+1)-th gap, so the exact check bites


@pytest.mark.parametrize("precision", PRECISIONS)
def test_knn_exact_integer_data_bit_exact(at, precision):
    # integer-valued data: FP32 sums of squared integer differences below 2^24
    # are exact, so distances and the (d2, index) order match the oracle exactly.
    X = synth.sparse_prototypes(N=3000, D=784, seed=7)
    idx, d2 = at.atsne_knn(to_dev(X), 90, precision=precision)
    o_idx, o_d2 = oracle.knn_exact(X, 90)
    assert np.array_equal(idx.cpu().numpy(), o_idx)
    assert np.array_equal(d2.cpu().numpy().astype(np.float64), o_d2)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_knn_query_list_and_duplicates(at, precision):
    X = synth.gaussian_mixture(500, 24, seed=8)
    X[10] = X[20]  # an exact duplicate pair
    q = np.array([20, 10, 0, 499, 20], np.int32)
    idx, d2 = at.atsne_knn(to_dev(X), 30, queries=to_dev(q), precision=precision)
    knn_parity(idx.cpu().numpy(), d2.cpu().numpy(), X, 30, queries=q)
    assert idx[0, 0].item() == 10 and d2[0, 0].item() == 0.0
    assert np.array_equal(idx[0].cpu().numpy(), idx[4].cpu().numpy())


@pytest.mark.parametrize("precision", PRECISIONS)
def test_knn_all_identical_points(at, precision):
    # every key ties: no row can be certified, all fall back to the CUDA cores
    X = np.ones((1200, 5), np.float32)
    idx, d2 = at.atsne_knn(to_dev(X), 20, precision=precision)
    o_idx, _ = oracle.knn_exact(X, 20)
    assert np.array_equal(idx.cpu().numpy(), o_idx)  # ties broken by index
    assert torch.all(d2 == 0)


def test_knn_tensor_rows_that_fail_the_certificate_fall_back(at):
    # one BF16 pass with the smallest candidate budget on continuous data: many
    # rows cannot be certified and are recomputed; the result is still exact
    X = synth.gaussian_mixture(3000, 96, seed=9)
    idx, d2 = at.atsne_knn(to_dev(X), 60, precision="bf16", rerank_k=60)
    knn_parity(idx.cpu().numpy(), d2.cpu().numpy(), X, 60)


def test_knn_many_tiles_query_list(at):
    # more than one 128-row query tile and a ragged last corpus tile
    X = synth.gaussian_mixture(5000, 70, seed=10)
    q = synth.sample_rows(5000, 700, seed=3)
    idx, d2 = at.atsne_knn(to_dev(X), 90, queries=to_dev(q))
    knn_parity(idx.cpu().numpy(), d2.cpu().numpy(), X, 90, queries=q)


@pytest.mark.parametrize("N,D,k,mu,seed", [(2000, 64, 90, 30.0, 1), (300, 10, 30, 10.0, 2),
                                           (150, 3, 12, 4.0, 3)])
def test_calibrate_matches_oracle(at, N, D, k, mu, seed):
    X = synth.gaussian_mixture(N, D, seed=seed)
    _, o_d2 = oracle.knn_exact(X, k)
    d2_32 = o_d2.astype(np.float32)
    P, beta = at.atsne_calibrate_P(to_dev(d2_32), mu)
    o_P, o_beta, o_perp, _ = oracle.calibrate(d2_32.astype(np.float64), mu)
    Pg = P.cpu().numpy().astype(np.float64)
    assert np.abs(Pg - o_P).max() <= 1e-5
    assert np.abs(Pg.sum(1) - 1).max() <= 1e-5
    assert np.abs(beta.cpu().numpy() / o_beta - 1).max() <= 1e-3


def test_calibrate_wide_and_degenerate_rows(at):
    rng = np.random.default_rng(5)
    # MNIST-like magnitudes (d2 ~ 1e5..1e6), an equidistant row, a row with
    # 40 neighbours tied at the minimum (perplexity 30 unreachable)
    d2 = np.sort(rng.uniform(2e5, 9e5, size=(64, 90)), axis=1)
    d2[5] = 12345.0
    d2[6, :40] = 100.0
    d2[6, 40:] = np.linspace(200, 900, 50)
    d2 = d2.astype(np.float32)
    P, _ = at.atsne_calibrate_P(to_dev(d2), 30.0)
    o_P, _, _, _ = oracle.calibrate(d2.astype(np.float64), 30.0)
    Pg = P.cpu().numpy()
    assert np.abs(Pg - o_P).max() <= 1e-5
    assert np.allclose(Pg[5], 1 / 90, atol=1e-7)


def dense_from_csr(rp, col, val, N):
    M = np.zeros((N, N))
    rows = np.repeat(np.arange(N), np.diff(rp))
    M[rows, col] = val
    return M


@pytest.mark.parametrize("N,D,k,mu,seed", [(2000, 64, 90, 30.0, 1), (400, 8, 25, 8.0, 2)])
def test_symmetrize_matches_oracle(at, N, D, k, mu, seed):
    X = synth.gaussian_mixture(N, D, seed=seed)
    o_idx, o_d2 = oracle.knn_exact(X, k)
    o_P, _, _, _ = oracle.calibrate(o_d2, mu)
    P32 = o_P.astype(np.float32)
    rp, col, val = at.atsne_symmetrize(to_dev(o_idx), to_dev(P32))
    at.atsne_check()
    e_rp, e_col, e_val = oracle.symmetrize(o_idx, P32.astype(np.float64))
    assert np.array_equal(rp.cpu().numpy(), e_rp)
    assert np.array_equal(col.cpu().numpy(), e_col)
    assert np.abs(val.cpu().numpy().astype(np.float64) - e_val).max() * N <= 1e-5
    g = dense_from_csr(rp.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy(), N)
    assert np.array_equal(g, g.T)  # bit-exact symmetry
    assert abs(g.sum() - 1.0) <= 1e-5


def test_symmetrize_hub_rows_longer_than_a_warp_sort(at):
    # every row lists points 0..9 first: those ten rows receive ~N reverse
    # entries each, exercising the one-CTA-per-long-row sort
    N, k = 3000, 16
    rng = np.random.default_rng(3)
    idx = np.empty((N, k), np.int32)
    for i in range(N):
        hubs = [h for h in range(10) if h != i]
        rest = rng.choice(np.setdiff1d(np.arange(10, N), [i]), size=k - len(hubs), replace=False)
        idx[i] = np.concatenate([hubs, rest])
    P = rng.random((N, k))
    P /= P.sum(1, keepdims=True)
    P32 = P.astype(np.float32)
    rp, col, val = at.atsne_symmetrize(to_dev(idx), to_dev(P32))
    e_rp, e_col, e_val = oracle.symmetrize(idx, P32.astype(np.float64))
    assert np.array_equal(rp.cpu().numpy(), e_rp) and np.array_equal(col.cpu().numpy(), e_col)
    assert np.abs(val.cpu().numpy() - e_val).max() * N <= 1e-5
    assert e_rp[1] - e_rp[0] > 1024


def forest_compare(at, X, trees, leaf, seed, V=5):
    f = at.atsne_forest_build(to_dev(X), trees=trees, leaf_size=leaf, seed=seed, top_var_dims=V)
    g = {a: b.cpu().numpy() for a, b in f.arrays().items() if a != "depth"}
    o = oracle.forest_build(X, trees=trees, top_var_dims=V, leaf_size=leaf, seed=seed)
    assert f.arrays()["depth"] == o["depth"]
    assert np.array_equal(g["leaf_ofs"], o["leaf_ofs"])
    assert np.array_equal(g["split_dim"], o["split_dim"])
    assert np.array_equal(g["split_val"], o["split_val"])
    assert np.array_equal(g["perm"], o["perm"])
    return f, o


@pytest.mark.parametrize("N,D,T,leaf,seed", [(2000, 64, 4, 1, 1), (1000, 17, 2, 8, 2),
                                             (5000, 32, 3, 4, 3), (9000, 8, 1, 1, 4)])
def test_forest_build_matches_oracle(at, N, D, T, leaf, seed):
    X = synth.gaussian_mixture(N, D, seed=seed)
    forest_compare(at, X, T, leaf, seed)


def test_forest_build_integer_data(at):
    X = synth.sparse_prototypes(N=6000, D=784, seed=9)
    forest_compare(at, X, 4, 1, 11)


@pytest.mark.parametrize("N,D,T,leaf,checks,seed", [(2000, 64, 4, 1, 256, 1),
                                                    (1500, 20, 2, 4, 90, 2),
                                                    (3000, 784, 4, 1, 512, 3),
                                                    (800, 10, 1, 1, 1, 4)])
def test_forest_query_matches_oracle(at, N, D, T, leaf, checks, seed):
    X = (synth.sparse_prototypes(N=N, D=D, seed=seed) if D == 784
         else synth.gaussian_mixture(N, D, seed=seed))
    k = 90 if N > 1000 else 30
    f, o = forest_compare(at, X, T, leaf, seed)
    idx, d2, ev = at.atsne_forest_query(to_dev(X), f, k, checks=checks)
    gi = idx.cpu().numpy()
    o_idx, o_ev = forest_parity(gi, d2.cpu().numpy(), X, o, k, checks, exact=(D == 784))
    assert np.array_equal(ev.cpu().numpy(), o_ev)          # identical visiting order
    e_idx, _ = oracle.knn_exact(X, k)
    rho_g = oracle.precision(gi, e_idx)[1]
    rho_o = oracle.precision(o_idx, e_idx)[1]
    assert abs(rho_g - rho_o) <= 1e-3


@pytest.mark.parametrize("name", ["forest_1d", "forest_2tree"])
def test_forest_golden_cases_on_the_gpu(at, name):
    """The hand-derived forest cases (split choices, the queue's order across
    trees, evictions from a small queue, completion of a queue that runs dry)
    through the library's build and search."""
    from conftest import golden
    g = golden(name + ".json")
    if name == "forest_1d":
        X = np.array(g["x"], np.float32)[:, None]
        build = dict(trees=g["two_identical_trees"]["trees"], top_var_dims=5, seed=3)
        cases = g["two_identical_trees"]["cases"]
    else:
        X = np.array(g["points"], np.float32)
        build = dict(trees=g["trees"], top_var_dims=g["top_var_dims"], seed=g["seed"])
        cases = g["cases"]
    Xd = to_dev(X)
    f = at.atsne_forest_build(Xd, leaf_size=1, **build)
    q = to_dev(np.array([g["query"]], np.int32))
    for case in cases:
        idx, d2, ev = at.atsne_forest_query(Xd, f, case["k"], checks=case["checks"], queries=q,
                                            queue_cap=case["queue_cap"])
        at.atsne_check()
        assert idx.cpu().numpy()[0].tolist() == case["idx"], case
        assert d2.cpu().numpy()[0].tolist() == case["d2"], case
        assert int(ev.cpu().numpy()[0]) == case["evaluated"], case

def test_forest_full_budget_is_exact(at):
    X = synth.gaussian_mixture(600, 12, seed=5)
    f = at.atsne_forest_build(to_dev(X), trees=2, leaf_size=2, seed=1)
    idx, d2, ev = at.atsne_forest_query(to_dev(X), f, 20, checks=599, queue_cap=4096)
    # the forest's distances are FP32: near ties keep their FP32 order
    knn_parity(idx.cpu().numpy(), d2.cpu().numpy(), X, 20, exact_lists=False)
    assert torch.all(ev == 599)


def test_forest_query_cutoff_is_exact(at):
    # In all-rows mode most queries search under a cut-off taken from seed
    # queries (pushes above it skipped, a search that runs dry repeated without
    # it); a query list searches without one. Both give the same lists bit for
    # bit; 30000 queries are several waves of warps, so most queries start after
    # their seeds have finished and take the cut-off.
    X = synth.sparse_prototypes(N=30000, D=784, seed=12)
    Xd = to_dev(X)
    f = at.atsne_forest_build(Xd, trees=4, leaf_size=1, seed=3)
    a = at.atsne_forest_query(Xd, f, 90, checks=1024)
    rows = torch.arange(X.shape[0], dtype=torch.int32, device=DEV)
    b = at.atsne_forest_query(Xd, f, 90, checks=1024, queries=rows)
    at.atsne_check()
    for u, v in zip(a, b):
        assert torch.equal(u, v)
    # a small queue (evictions decide what is popped) and a multi-point leaf
    for leaf, qcap in ((1, 128), (4, 256)):
        f = at.atsne_forest_build(Xd, trees=2, leaf_size=leaf, seed=4)
        a = at.atsne_forest_query(Xd, f, 90, checks=512, queue_cap=qcap)
        b = at.atsne_forest_query(Xd, f, 90, checks=512, queue_cap=qcap, queries=rows)
        for u, v in zip(a, b):
            assert torch.equal(u, v)


@pytest.mark.parametrize("spoil", [None, 100.5, 300.0, -1.0])
def test_byte_paths_follow_the_data(at, spoil):
    # The forest build and search read a byte copy of X only when every value is
    # an integer in [0, 255] (a device flag); one value outside that set sends
    # the whole call to the FP32 kernels. Either way the forest equals the
    # oracle's and the search visits the same points.
    X = synth.sparse_prototypes(N=4000, D=784, seed=14)
    if spoil is not None:
        X = X.copy()
        X[1234, 300] = spoil
    f, o = forest_compare(at, X, 4, 1, 5)
    idx, d2, ev = at.atsne_forest_query(to_dev(X), f, 90, checks=512)
    at.atsne_check()
    # integer data (the byte path) compare exactly; a fractional value (the FP32
    # path) by the gap rule; a value above 255 or below 0 is integer too, and its
    # FP32 sums stay exact
    _, o_ev = forest_parity(idx.cpu().numpy(), d2.cpu().numpy(), X, o, 90, 512, exact=spoil != 100.5)
    assert np.array_equal(ev.cpu().numpy(), o_ev)
    # the exact path on the same data (one tensor pass when every value is exact in BF16)
    e_idx, e_d2 = at.atsne_knn(to_dev(X), 90)
    knn_parity(e_idx.cpu().numpy(), e_d2.cpu().numpy(), X, 90)


def test_forest_mnist_shaped_full_size_sampled(at):
    # the benchmark's forest launch (N=70000, D=784, T=4, V=5, checks=1024,
    # queue 512): the forest compared whole, the search on 64 sampled rows the
    # oracle runs one by one (same visiting order: same evaluated counts)
    X = synth.sparse_prototypes(seed=2)
    Xd = to_dev(X)
    f, o = forest_compare(at, X, 4, 1, 7)
    idx, d2, ev = at.atsne_forest_query(Xd, f, 90, checks=1024)
    at.atsne_check()
    rows = synth.sample_rows(X.shape[0], 64, seed=23)
    # integer data: the sampled lists equal the oracle's bit for bit
    _, o_ev = forest_parity(idx.cpu().numpy()[rows], d2.cpu().numpy()[rows], X, o, 90, 1024, rows=rows,
                            exact=True)
    assert np.array_equal(ev.cpu().numpy()[rows], o_ev)


def test_knn_forest_method_matches_build_then_query(at):
    X = synth.gaussian_mixture(1200, 16, seed=6)
    Xd = to_dev(X)
    a_idx, a_d2 = at.atsne_knn(Xd, 30, method="forest", trees=3, checks=200, seed=4)
    f = at.atsne_forest_build(Xd, trees=3, seed=4)
    b_idx, b_d2, _ = at.atsne_forest_query(Xd, f, 30, checks=200)
    assert torch.equal(a_idx, b_idx) and torch.equal(a_d2, b_d2)


def test_precision_matches_oracle(at):
    rng = np.random.default_rng(2)
    e = np.stack([rng.permutation(5000)[:90] for _ in range(700)]).astype(np.int32)
    a = e.copy()
    for r in range(700):
        m = rng.integers(0, 91)
        a[r, :m] = rng.permutation(np.setdiff1d(np.arange(5000, 9000), []))[:m]
    rho_i, rho = at.atsne_knn_precision(to_dev(a), to_dev(e))
    o_rho_i, o_rho = oracle.precision(a, e)
    assert np.allclose(rho_i.cpu().numpy(), o_rho_i, atol=1e-7)
    assert abs(rho - o_rho) < 1e-12


def test_refine_matches_oracle(at):
    N, D, k, mu = 1500, 32, 45, 15.0
    X = synth.gaussian_mixture(N, D, seed=12)
    f_o = oracle.forest_build(X, trees=1, top_var_dims=5, leaf_size=1, seed=3)
    a_idx, a_d2, _ = oracle.forest_query(X, f_o, k, 1)   # a low-precision start (T=1, L=1)
    a_P, a_beta, _, _ = oracle.calibrate(a_d2, mu)
    sub = np.array([0, 7, 7, 1499, 600, 42], np.int32)
    idx, d2 = to_dev(a_idx), to_dev(a_d2.astype(np.float32))
    P, beta = to_dev(a_P.astype(np.float32)), to_dev(a_beta.astype(np.float32))
    rho = torch.full((N,), 0.1, device=DEV)
    at.atsne_refine_subset(to_dev(X), to_dev(sub), mu, idx, d2, P, beta, rho)
    at.atsne_check()
    o = dict(idx=a_idx.copy(), d2=a_d2.copy(), P=a_P.copy(), beta=a_beta.copy(),
             rho=np.full(N, 0.1))
    oracle.refine(X, sub, k, mu, o["idx"], o["d2"], o["P"], o["beta"], o["rho"])
    s = np.unique(sub)
    gi = idx.cpu().numpy()
    knn_parity(gi[s], d2.cpu().numpy()[s], X, k, queries=s)
    assert np.abs(P.cpu().numpy()[s] - o["P"][s]).max() <= 1e-5
    assert np.allclose(rho.cpu().numpy(), o["rho"])
    others = np.setdiff1d(np.arange(N), s)
    assert np.array_equal(gi[others], a_idx[others])


def test_non_finite_input_is_reported(at):
    X = synth.gaussian_mixture(300, 8, seed=1)
    X[17, 3] = np.nan
    at.atsne_knn(to_dev(X), 10)
    with pytest.raises(at.AtsneError) as ei:
        at.atsne_check()
    assert ei.value.status == at.ATSNE_EINVAL
    at.atsne_check()  # the status word was cleared


def test_out_of_range_subset_is_reported(at):
    X = synth.gaussian_mixture(300, 8, seed=1)
    idx, d2 = at.atsne_knn(to_dev(X), 10)
    P, beta = at.atsne_calibrate_P(d2, 3.0)
    at.atsne_refine_subset(to_dev(X), to_dev(np.array([5, 300], np.int32)), 3.0, idx, d2, P, beta)
    with pytest.raises(at.AtsneError):
        at.atsne_check()


def test_misaligned_workspace_is_refused(at):
    import ctypes
    X = to_dev(synth.gaussian_mixture(300, 8, seed=1))
    o = at.knn_opts()
    n = at.workspace_bytes(at.OP_KNN, 300, 8, 10, 0, o)
    ws = torch.empty(n + 256, dtype=torch.uint8, device=X.device)
    idx = torch.empty((300, 10), dtype=torch.int32, device=X.device)
    d2 = torch.empty((300, 10), dtype=torch.float32, device=X.device)
    rc = at.lib().atsne_knn(at._p(X), 300, 8, None, 0, 10, ctypes.byref(o), at._p(idx), at._p(d2),
                            ctypes.c_void_p(ws.data_ptr() + 16), n, at._stream(None))
    assert rc == at.ATSNE_EINVAL


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_mnist_shaped_full_size_sampled(at, precision):
    # full-size workload (N=70000, D=784): the launch the benchmark times,
    # checked on 48 sampled rows the oracle computes one by one, and P/CSR by
    # properties that hold at any size.
    X = synth.sparse_prototypes(seed=2)
    Xd = to_dev(X)
    idx, d2 = at.atsne_knn(Xd, 90, precision=precision)
    rows = synth.sample_rows(X.shape[0], 48, seed=21)
    o_idx, o_d2 = oracle.knn_exact(X, 90, queries=rows)
    assert np.array_equal(idx.cpu().numpy()[rows], o_idx)
    assert np.array_equal(d2.cpu().numpy()[rows].astype(np.float64), o_d2)
    P, beta = at.atsne_calibrate_P(d2, 30.0)
    o_P, _, _, _ = oracle.calibrate(o_d2, 30.0)
    assert np.abs(P.cpu().numpy()[rows] - o_P).max() <= 1e-5
    rp, col, val = at.atsne_symmetrize(idx, P)
    at.atsne_check()
    rp, col, val = rp.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()
    N = X.shape[0]
    assert N * 90 <= rp[-1] <= 2 * N * 90 and rp[-1] == col.shape[0]
    assert abs(val.astype(np.float64).sum() - 1.0) < 1e-5
    r = np.repeat(np.arange(N), np.diff(rp))
    assert np.all(r != col)
    starts = rp[:-1]
    d = np.diff(col)
    inner = np.ones(col.shape[0] - 1, bool)
    inner[starts[1:] - 1] = False
    assert np.all(d[inner] > 0)
    # symmetric: the transposed entries are the same entries with the same bits
    key = r.astype(np.int64) * N + col
    key_t = col.astype(np.int64) * N + r
    perm = np.argsort(key_t)
    assert np.array_equal(key_t[perm], key)
    assert np.array_equal(val[perm], val)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_gamma_clusters_full_size_sampled(at, precision):
    # the TIMIT-scale workload at full size (N=10^6, D=128, continuous
    # Gamma-distributed features in 50 clusters): all rows on the tensor cores,
    # 48 sampled rows checked against the oracle one by one, their P rows too.
    X = synth.gamma_clusters(seed=3)
    Xd = to_dev(X)
    idx, d2 = at.atsne_knn(Xd, 90, precision=precision)
    at.atsne_check()
    rows = synth.sample_rows(X.shape[0], 48, seed=31)
    g_idx, g_d2 = idx.cpu().numpy()[rows], d2.cpu().numpy()[rows]
    knn_parity(g_idx, g_d2, X, 90, queries=rows)
    P, beta = at.atsne_calibrate_P(d2, 30.0)
    o_idx, o_d2 = oracle.knn_exact(X, 90, queries=rows)
    o_P, _, _, _ = oracle.calibrate(o_d2, 30.0)
    # P rows are compared where the index sets agree, which knn_parity requires
    # of every row with a clear k-th/(k+1)-th gap
    same = np.all(np.sort(g_idx, 1) == np.sort(o_idx, 1), axis=1)
    g_P = P.cpu().numpy()[rows]
    for r in np.flatnonzero(same):  # compared by neighbour index (near ties may swap places)
        gp = g_P[r][np.argsort(g_idx[r])]
        op = o_P[r][np.argsort(o_idx[r])]
        assert np.abs(gp - op).max() <= 1e-5, r


def _refine_state(at, X, k, perp):
    Xd = to_dev(X)
    idx, d2 = at.atsne_knn(Xd, k, method="forest", trees=2, checks=64)
    P, beta = at.atsne_calibrate_P(d2, perp)
    return Xd, [idx, d2, P, beta, torch.zeros(X.shape[0], dtype=torch.float32, device=DEV)]


def test_refine_batch_equals_refining_each_selection(at):
    X, labels = synth.gaussian_mixture(3000, 32, seed=8, return_labels=True)
    Xd, base = _refine_state(at, X, 30, 10.0)
    subs = synth.refine_subsets(labels, 6, lo=128, hi=700, seed=9)  # overlapping brushes
    a = [t.clone() for t in base]
    for sub in subs:
        at.atsne_refine_subset(Xd, to_dev(sub), 10.0, *a)
    b = [t.clone() for t in base]
    cnt = at.atsne_refine_batch(Xd, [to_dev(s) for s in subs], 10.0, *b)
    at.atsne_check()
    union = np.unique(np.concatenate(subs))
    assert int(cnt.item()) == union.size
    ai, bi = a[0].cpu().numpy(), b[0].cpu().numpy()
    assert np.array_equal(ai, bi)
    for x, y in zip(a[1:], b[1:]):
        assert torch.allclose(x, y, rtol=1e-6, atol=1e-7)
    untouched = np.setdiff1d(np.arange(X.shape[0]), union)
    assert np.array_equal(bi[untouched], base[0].cpu().numpy()[untouched])
    assert np.all(b[4].cpu().numpy()[union] == 1.0)
    knn_parity(bi[union], b[1].cpu().numpy()[union], X, 30, queries=union)


def test_refine_batch_replays_from_a_cuda_graph(at):
    X, labels = synth.gaussian_mixture(3000, 32, seed=8, return_labels=True)
    Xd, base = _refine_state(at, X, 30, 10.0)
    subs = synth.refine_subsets(labels, 5, lo=40, hi=900, seed=10)
    lists = to_dev(np.concatenate(subs))
    eager = [t.clone() for t in base]
    at.atsne_refine_batch(Xd, lists, 10.0, *eager)
    at.atsne_check()
    state = [t.clone() for t in base]
    ws = torch.empty(at.workspace_bytes(at.OP_REFINE_BATCH, 3000, 32, 30, lists.shape[0]),
                     dtype=torch.uint8, device=DEV)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        cnt = at.atsne_refine_batch(Xd, lists, 10.0, *state, workspace=ws)
    for t, b0 in zip(state, base):  # capture records without running; reset to the base
        t.copy_(b0)
    g.replay()
    torch.cuda.synchronize()
    at.atsne_check()
    assert int(cnt.item()) == np.unique(np.concatenate(subs)).size
    for x, y in zip(eager, state):
        assert torch.equal(x, y)


def test_refine_batch_edge_cases(at):
    X, labels = synth.gaussian_mixture(500, 8, seed=12, return_labels=True)
    Xd, base = _refine_state(at, X, 10, 3.0)
    st = [t.clone() for t in base]
    cnt = at.atsne_refine_batch(Xd, [], 3.0, *st)  # nothing listed: nothing changes
    assert int(cnt.item()) == 0
    for x, y in zip(st, base):
        assert torch.equal(x, y)
    rep = np.array([7, 7, 7, 3, 499, 3], np.int32)  # duplicates, small batch (CUDA-core path)
    cnt = at.atsne_refine_batch(Xd, to_dev(rep), 3.0, *st)
    at.atsne_check()
    assert int(cnt.item()) == 3
    knn_parity(st[0].cpu().numpy()[[3, 7, 499]], st[1].cpu().numpy()[[3, 7, 499]], X, 10,
               queries=np.array([3, 7, 499], np.int32))
    with pytest.raises(at.AtsneError):
        at.atsne_refine_batch(Xd, to_dev(np.array([1, 500], np.int32)), 3.0, *st)
        at.atsne_check()


def test_refine_batch_full_size_sampled(at):
    # the batched-refinement workload at full size: a 500000 x 256 corpus of 100
    # Gaussian clusters and 512 brushed selections of 200..20000 points, refined
    # in one call; 32 sampled rows of the union checked against the oracle.
    X, labels = synth.gaussian_mixture(500_000, 256, n_centres=100, centre_sigma=4.0, seed=4,
                                       return_labels=True)
    Xd = to_dev(X)
    N, k = X.shape[0], 90
    subs = synth.refine_subsets(labels, 512, lo=200, hi=20000, seed=4)
    union = np.unique(np.concatenate(subs))
    idx = torch.zeros((N, k), dtype=torch.int32, device=DEV)
    d2 = torch.zeros((N, k), dtype=torch.float32, device=DEV)
    P = torch.zeros((N, k), dtype=torch.float32, device=DEV)
    beta = torch.zeros(N, dtype=torch.float32, device=DEV)
    rho = torch.zeros(N, dtype=torch.float32, device=DEV)
    cnt = at.atsne_refine_batch(Xd, [to_dev(s) for s in subs], 30.0, idx, d2, P, beta, rho)
    at.atsne_check()
    assert int(cnt.item()) == union.size
    rows = union[synth.sample_rows(union.size, 32, seed=41)]
    knn_parity(idx.cpu().numpy()[rows], d2.cpu().numpy()[rows], X, k, queries=rows.astype(np.int32))
    assert np.all(rho.cpu().numpy()[union] == 1.0)
    outside = np.setdiff1d(np.arange(N), union)
    if outside.size:
        assert not idx.cpu().numpy()[outside].any()


@pytest.mark.parametrize("cutoff", [4.0, 0.0])
def test_kde_map_matches_oracle(at, cutoff):
    labels = np.random.default_rng(13).integers(0, 6, size=3000)
    Y = synth.embedding_2d(labels, seed=13)
    rng = np.random.default_rng(14)
    rho = rng.random(3000).astype(np.float32)
    sel = (labels == 2).astype(np.uint8)
    x0, y0, px, W, H, h = -13.0, -12.0, 0.25, 104, 90, 0.6
    g = at.atsne_kde_map(to_dev(Y), x0, y0, px, W, H, h, cutoff=cutoff, lens_k=2.0,
                         rho=to_dev(rho), selected=to_dev(sel))
    o = oracle.kde(Y, x0, y0, px, W, H, h, cutoff=cutoff, k=2.0, rho=rho, selected=sel)
    gf, gs, ga, gal = [t.cpu().numpy().astype(np.float64) for t in g]
    of, os_, oa, oal = o
    assert np.all(np.abs(gf - of) <= 1e-5 * np.abs(of) + 1e-12)
    # shares compared where the density is not vanishing (FP32 sums of tiny terms)
    live = of > 1e-9
    assert live.mean() > 0.3
    for u, v in ((gs, os_), (ga, oa), (gal, oal)):
        assert np.abs(u - v)[live].max() <= 1e-5
    dead = of == 0.0
    assert np.all(gs[dead] == 0.0) and np.all(ga[dead] == 1.0)


def test_kde_map_edges(at):
    Y = to_dev(np.array([[0.0, 0.0]], np.float32))
    f, s, a, al = at.atsne_kde_map(Y, -0.5, -0.5, 1.0, 1, 1, 1.0, cutoff=0.0)  # no rho, no selection
    assert abs(f.item() - 1 / (2 * np.pi)) < 1e-6 and s.item() == 0.0 and a.item() == 1.0
    assert al.item() == 0.0
    for bad in (dict(h=0.0), dict(cutoff=-1.0), dict(width=0)):
        kw = dict(x0=0.0, y0=0.0, pixel=1.0, width=4, height=4, h=1.0, cutoff=4.0)
        kw.update(bad)
        with pytest.raises(at.AtsneError):
            at.atsne_kde_map(Y, kw["x0"], kw["y0"], kw["pixel"], kw["width"], kw["height"], kw["h"],
                             cutoff=kw["cutoff"])


def _sq_dists(X, rows, idx):
    Xd = X.astype(np.float64)
    return np.stack([((Xd[idx[i]] - Xd[r]) ** 2).sum(1) for i, r in enumerate(rows)])


@pytest.mark.parametrize("kind", ["mnist", "gauss"])
def test_knn_fp8_rerank_recall_and_exact_distances(at, kind):
    # FP8 (E4M3, per-row scale) keys select 4k candidates, re-ranked in FP32:
    # approximate, so the test measures recall against the oracle, and checks
    # that every returned distance is the FP32 direct difference of its pair.
    if kind == "mnist":
        X = synth.sparse_prototypes(N=6000, seed=2)
    else:
        X = synth.gaussian_mixture(4000, 64, seed=1)
    idx, d2 = at.atsne_knn(to_dev(X), 90, precision="fp8")
    at.atsne_check()
    rows = synth.sample_rows(X.shape[0], 200, seed=51)
    o_idx, o_d2 = oracle.knn_exact(X, 90, queries=rows)
    g_idx, g_d2 = idx.cpu().numpy()[rows], d2.cpu().numpy()[rows]
    recall = np.mean([len(set(g_idx[i]) & set(o_idx[i])) / 90 for i in range(len(rows))])
    print("fp8 recall", kind, recall)
    assert recall >= 0.99
    exact = _sq_dists(X, rows, g_idx)
    assert np.all(np.abs(g_d2 - exact) <= 1e-5 * exact + 1e-3)
    assert np.all(np.diff(g_d2, axis=1) >= 0)
    assert np.all(g_idx != rows[:, None])


@pytest.mark.parametrize("kind", ["gamma", "gauss"])
def test_knn_bf16_approx_recall_and_exact_distances(at, kind):
    # BF16 keys select 4k candidates, re-ranked in FP32, without a certificate:
    # recall against the oracle, and every returned distance the FP32 direct
    # difference of its pair. Gamma-distributed features (wide norms) are the
    # case where the certified BF16 mode sends most rows to the CUDA cores.
    if kind == "gamma":
        X = synth.gamma_clusters(N=20000, D=128, seed=3)
    else:
        X = synth.gaussian_mixture(4000, 64, seed=1)
    rows = synth.sample_rows(X.shape[0], 300, seed=52)
    idx, d2 = at.atsne_knn(to_dev(X), 90, queries=to_dev(rows.astype(np.int32)), precision="bf16_approx")
    at.atsne_check()
    o_idx, o_d2 = oracle.knn_exact(X, 90, queries=rows)
    g_idx, g_d2 = idx.cpu().numpy(), d2.cpu().numpy()
    recall = np.mean([len(set(g_idx[i]) & set(o_idx[i])) / 90 for i in range(len(rows))])
    print("bf16 approx recall", kind, recall)
    assert recall >= 0.999
    exact = _sq_dists(X, rows, g_idx)
    assert np.all(np.abs(g_d2 - exact) <= 1e-5 * exact + 1e-3)
    assert np.all(np.diff(g_d2, axis=1) >= 0)
    assert np.all(g_idx != rows[:, None])


@pytest.mark.parametrize("k", [20, 128])
def test_knn_bf16_approx_rerank_set_sizes_and_tie_order(at, k):
    # The re-rank set holds the 4k best keys: at k = 20 the merge sorts sets of
    # 128 entries in registers, at k = 128 sets of more than 512 entries in
    # shared memory (k = 90 elsewhere sorts 512 in registers). Half the rows
    # appear twice, so many distances are exactly equal; both sorts order them
    # by index, as Eq. 8's (d^2, index) order does.
    X = synth.sparse_prototypes(N=6000, seed=5)
    X = np.ascontiguousarray(np.concatenate([X, X[:3000]]))
    rows = synth.sample_rows(X.shape[0], 200, seed=54)
    idx, d2 = at.atsne_knn(to_dev(X), k, queries=to_dev(rows.astype(np.int32)), precision="bf16_approx")
    at.atsne_check()
    o_idx, _ = oracle.knn_exact(X, k, queries=rows)
    g_idx, g_d2 = idx.cpu().numpy(), d2.cpu().numpy()
    recall = np.mean([len(set(g_idx[i]) & set(o_idx[i])) / k for i in range(len(rows))])
    assert recall >= 0.999
    exact = _sq_dists(X, rows, g_idx)
    assert np.all(np.abs(g_d2 - exact) <= 1e-5 * exact + 1e-3)
    same = g_d2[:, 1:] == g_d2[:, :-1]
    assert same.any()
    assert np.all(np.diff(g_d2, axis=1) >= 0)
    assert np.all((g_idx[:, 1:] > g_idx[:, :-1]) | ~same)
    assert np.all(g_idx != rows[:, None])
