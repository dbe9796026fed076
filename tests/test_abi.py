"""The C ABI library loads and exports every symbol include/atsne.h declares;
host-side argument validation (no device work) behaves as documented."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1512_01655_gb300 as at
    return at


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "atsne.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(atsne_[A-Za-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    syms = declared_symbols()
    assert "atsne_knn" in syms and "atsne_refine_subset" in syms
    lib = ctypes.CDLL(L.LIB_PATH)
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing
    assert sorted(L.EXPORTED) == syms


def test_defaults_and_workspace_sizes(L):
    o = L.knn_opts()
    assert (o.method, o.trees, o.top_var_dims, o.leaf_size) == (L.KNN_EXACT, 4, 5, 1)
    assert L.workspace_bytes(L.OP_CALIBRATE, 1000, 64, 90) == 0
    sym = L.workspace_bytes(L.OP_SYMMETRIZE, 70000, 784, 90)
    assert sym >= 70000 * 90 * 8
    fo = L.knn_opts(method="forest", checks=256)
    fb = L.workspace_bytes(L.OP_KNN, 70000, 784, 90, 0, fo)
    assert fb > 70000 * 4 * 4


def test_forest_layout_matches_depth_rule(L, oracle_mod):
    for N, leaf in [(2000, 1), (70000, 8), (3, 1)]:
        lay = L.ForestLayout()
        o = L.knn_opts(method="forest", leaf_size=leaf, trees=3)
        assert L.lib().atsne_forest_layout(N, 16, ctypes.byref(o), ctypes.byref(lay)) == 0
        assert lay.depth == oracle_mod.forest_depth(N, leaf)
        assert lay.n_internal == (1 << lay.depth) - 1
        assert lay.off_perm % 256 == 0 and lay.bytes >= lay.off_leaf_ofs + 4 * ((1 << lay.depth) + 1)


@pytest.mark.parametrize("N,D,k", [(1, 4, 1), (10, 0, 3), (10, 4, 10), (10, 4, 0)])
def test_bad_sizes_rejected_on_host(L, N, D, k):
    lib = L.lib()
    fake = ctypes.c_void_p(256)  # never dereferenced: validation fails first
    rc = lib.atsne_knn(fake, N, D, None, 0, k, None, fake, fake, None, 0, None)
    assert rc == L.ATSNE_EINVAL
    assert lib.atsne_last_error()


def test_calibrate_rejects_bad_perplexity(L):
    lib = L.lib()
    fake = ctypes.c_void_p(256)
    assert lib.atsne_calibrate_P(fake, 10, 9, 9.5, 0.0, 0, fake, None, None) == L.ATSNE_EINVAL
    assert lib.atsne_calibrate_P(fake, 10, 9, 0.0, 0.0, 0, fake, None, None) == L.ATSNE_EINVAL
    assert b"perplexity" in lib.atsne_last_error()


def test_forest_option_validation(L):
    lib = L.lib()
    fake = ctypes.c_void_p(256)
    for bad in [dict(trees=0), dict(top_var_dims=9), dict(checks=0), dict(leaf_size=0),
                dict(queue_cap=1)]:
        o = L.knn_opts(method="forest", **bad)
        rc = lib.atsne_knn(fake, 100, 4, None, 0, 5, ctypes.byref(o), fake, fake, None, 0, None)
        assert rc == L.ATSNE_EINVAL, bad


def test_workspace_too_small_is_enomem(L):
    lib = L.lib()
    fake = ctypes.c_void_p(256)
    rc = lib.atsne_symmetrize(fake, fake, 100, 5, fake, fake, fake, None, fake, 16, None)
    assert rc == L.ATSNE_ENOMEM


def test_tuner_workspace_and_host_checks(L):
    lib = L.lib()
    fake = ctypes.c_void_p(256)
    for prec in ("fp32", "bf16", "bf16_approx", "fp8"):
        o = L.knn_opts(precision=prec)
        for N, D, S in [(70000, 784, 0), (500000, 256, 2000), (20000, 50, 300)]:
            # the tuner's workspace holds the largest candidate, the rule's among them
            assert L.workspace_bytes(L.OP_TUNE_KNN, N, D, 90, S, o) >= L.workspace_bytes(L.OP_KNN, N, D, 90, S, o)
    fo = L.knn_opts(method="forest")
    assert L.workspace_bytes(L.OP_TUNE_KNN, 1000, 16, 10, 0, fo) == 0
    splits, ms = ctypes.c_int32(0), ctypes.c_float(0)
    rc = lib.atsne_tune_knn(fake, 1000, 16, None, 0, 10, ctypes.byref(fo), fake, fake, fake, 1 << 20, None,
                            ctypes.byref(splits), ctypes.byref(ms))
    assert rc == L.ATSNE_EUNSUPPORTED
    o = L.knn_opts()
    rc = lib.atsne_tune_knn(fake, 1000, 16, None, 0, 10, ctypes.byref(o), fake, fake, fake, 16, None,
                            ctypes.byref(splits), ctypes.byref(ms))
    assert rc == L.ATSNE_ENOMEM and b"tune" in lib.atsne_last_error()


def test_delete_and_row_dmax_host_checks(L):
    lib = L.lib()
    fake = ctypes.c_void_p(256)
    # more rows than the state holds, a perplexity not below k
    assert lib.atsne_delete_rows(fake, 11, fake, 10, 4, 5, 2.0, fake, fake, fake, None, None, fake, 1 << 20,
                                 None) == L.ATSNE_EINVAL
    assert lib.atsne_delete_rows(fake, 1, fake, 10, 4, 5, 5.0, fake, fake, fake, None, None, fake, 1 << 20,
                                 None) == L.ATSNE_EINVAL
    assert lib.atsne_row_dmax(fake, -1, 5, fake, None) == L.ATSNE_EINVAL
    assert lib.atsne_row_dmax(None, 0, 5, None, None) == L.ATSNE_OK  # nothing to do


def test_forest_update_rejects_overlapping_buckets(L):
    """buckets_out may not share a byte with buckets_in (the copy would race
    with its source): equal bases and a partial overlap are both refused on the
    host, before any device work."""
    lib = L.lib()
    N_built, D, trees = 1000, 8, 2
    o = L.knn_opts(method="forest", trees=trees, leaf_size=1)
    lay = L.ForestLayout()
    assert lib.atsne_forest_layout(N_built, D, ctypes.byref(o), ctypes.byref(lay)) == 0
    n_in = lib.atsne_forest_buckets_bytes(N_built, lay.depth, trees)
    n_out = lib.atsne_forest_buckets_bytes(N_built + 100, lay.depth, trees)
    mb = ctypes.c_int32(0)
    base = 1 << 20  # fake, 256-byte aligned addresses: never dereferenced
    for out in (base, base + 256 * ((n_in // 2) // 256), base - 256 * ((n_out // 2) // 256)):
        rc = lib.atsne_forest_insert(ctypes.c_void_p(base), N_built, N_built, N_built + 100, D, ctypes.byref(o),
                                     ctypes.c_void_p(1 << 30), ctypes.c_void_p(base), ctypes.c_void_p(out), n_out,
                                     ctypes.byref(mb), ctypes.c_void_p(1 << 31), 1 << 30, None)
        assert rc == L.ATSNE_EINVAL and b"overlap" in lib.atsne_last_error(), out
