"""CPU tests of the C ABI (library loads, every declared symbol is exported, host-side errors) and
of the host analysis (nested dissection, update sets, operation-count model). No GPU needed."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1702_05167_gb300 import hsc, workloads as W
from treecheck import _check_tree, _handle, _tree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not os.path.exists(hsc.lib_path()):
        from paper_1702_05167_gb300 import build
        build.build()
    hsc.load()


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w\*\s]+?\b(hsc_\w+)\s*\(", txt, flags=re.M))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    names = declared_symbols()
    assert {"hsc_create", "hsc_analyze", "hsc_solve", "hsc_destroy", "hsc_last_error"} <= set(names)
    out = subprocess.run(["nm", "-D", "--defined-only", hsc.lib_path()], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (hsc_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = hsc.load()
    for n in names:
        assert hasattr(L, n)


def test_rejects_non_symmetric_h():
    dev = W.cubic_device((3, 3, 3), seed=0)
    val = dev.val.copy()
    val[1] += 0.5        # breaks H = H^T
    with pytest.raises(hsc.HSCError) as ei:
        hsc.hsc_create(dev.n, 1, dev.rowptr, dev.col, val, dev.contact_ptr, dev.contact_sites, dev.dims)
    assert ei.value.code == hsc.HSC_ERR_NOT_SYMMETRIC


def test_rejects_bad_arguments_and_state():
    dev = W.cubic_device((3, 3, 3), seed=0)
    with pytest.raises(hsc.HSCError) as ei:
        hsc.hsc_create(dev.n, 1, dev.rowptr, dev.col, dev.val, dev.contact_ptr, dev.contact_sites,
                       (3, 3, 4))
    assert ei.value.code == hsc.HSC_ERR_ARG
    h = _handle(dev)
    sr, sl = W.self_energies(dev, 1)
    out = np.zeros((1, dev.n), np.complex128)
    with pytest.raises(hsc.HSCError) as ei:    # solve before analyze
        hsc.hsc_solve(h, np.array([0.1]), 1e-6, sr, sl, hsc.HSC_FP64, None, out, out.copy(), None, None)
    assert ei.value.code == hsc.HSC_ERR_STATE
    with pytest.raises(hsc.HSCError):
        hsc.hsc_analyze(h, 0)
    hsc.hsc_destroy(h)


@pytest.mark.parametrize("dims,orb,leaf,geo", [((8, 8, 8), 1, 4, True), ((9, 5, 7), 1, 3, True),
                                               ((6, 3, 2), 3, 2, True), ((7, 6, 5), 1, 2, False),
                                               ((17, 1, 1), 1, 1, True)])
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_tree_partitions_and_update_sets_are_exact(dims, orb, leaf, geo, variant):
    """Every unknown is owned once; no H entry joins two unrelated clusters (separation); each U_i
    is exactly the set of ancestor unknowns adjacent to the subtree of i (Section 2.2). Holds for
    the plain tree and both alternate trees (cuts below the root shifted)."""
    dev = W.cubic_device(dims, seed=1) if orb == 1 else W.wire_device(dims, orb=orb, seed=1)
    st, cl = _tree(dev, leaf, geo, variant)
    _check_tree(dev, cl)
    for i, (info, own, upd) in enumerate(cl):
        assert info.lesser == int(bool(np.isin(own, dev.contact_unknowns()).any()) or
                                  any(cl[c][0].lesser for c in info.child if c >= 0))


def _dense_edges(dev, contacts):
    """The coupling a DENSE self-energy block adds: every pair of unknowns of each contact."""
    cu, cid = dev.contact_unknowns(), dev.contact_of_unknown()
    out = []
    for c in contacts:
        u = cu[cid == c]
        out += [(a, b) for a in u for b in u if a != b]
    return out


@pytest.mark.parametrize("dims,orb,leaf,geo,dense", [((8, 8, 8), 1, 4, True, (0, 1)),
                                                     ((9, 5, 7), 1, 3, True, (0,)),
                                                     ((6, 4, 4), 1, 2, True, (1,)),
                                                     ((5, 3, 2), 2, 2, True, (0, 1)),
                                                     ((7, 6, 5), 1, 2, False, (0, 1)),
                                                     ((2, 3, 3), 1, 2, True, (0, 1))])
@pytest.mark.parametrize("variant", [0, 2])
def test_dense_contacts_become_one_cluster_each_on_top(dims, orb, leaf, geo, dense, variant):
    """Section 3.1.2's DENSE self-energy couples all unknowns of a contact: with the contact marked
    dense, its unknowns form one cluster, the dense contacts are chained at the top of the tree
    (the last one is the root), and the tree stays exact for the graph with those couplings."""
    dev = W.cubic_device(dims, seed=1) if orb == 1 else W.wire_device(dims, orb=orb, seed=1)
    st, cl = _tree(dev, leaf, geo, variant, dense)
    _check_tree(dev, cl, _dense_edges(dev, dense))
    cu, cid = dev.contact_unknowns(), dev.contact_of_unknown()
    nc = len(cl)
    for k, c in enumerate(reversed(dense)):
        info, own, upd = cl[nc - 1 - k]
        assert set(own.tolist()) == set(cu[cid == c].tolist())
        assert info.child[1] == -1


def test_dense_end_faces_keep_the_geometric_interior_and_fill_the_interior_root():
    """Both end planes of a cube dense: below them the interior box is dissected as before (its
    root is the x = mid plane) and, after the interior is eliminated, that plane is coupled to both
    faces: its update set is exactly the two faces."""
    dims = (10, 6, 6)
    dev = W.cubic_device(dims, seed=0)
    st, cl = _tree(dev, 3, True, 0, (0, 1))
    nc = len(cl)
    inner = cl[nc - 3]
    face = dims[1] * dims[2]
    assert inner[0].parent == nc - 2 and cl[nc - 2][0].parent == nc - 1
    xs = np.unique(inner[1] // face)
    assert len(xs) == 1 and xs[0] == (1 + dims[0] - 2) // 2
    assert inner[0].m == 2 * face and cl[nc - 2][0].m == face and cl[nc - 1][0].m == 0


def test_a_dense_contact_that_is_not_an_end_plane_falls_back_to_graph_bisection():
    dev = W.cubic_device((6, 5, 4), seed=2)
    half = W.face_sites(dev.dims, 0)[:7]
    dev2 = W.Device(dims=dev.dims, orb=1, rowptr=dev.rowptr, col=dev.col, val=dev.val,
                    contact_ptr=np.array([0, len(half)], np.int64), contact_sites=half.astype(np.int32),
                    gamma=np.array([0.5]))
    st, cl = _tree(dev2, 2, True, 0, (0,))
    _check_tree(dev2, cl, _dense_edges(dev2, (0,)))
    assert set(cl[-1][1].tolist()) == set(half.tolist())


def test_set_contact_dense_checks_arguments_and_requires_a_new_analysis():
    dev = W.cubic_device((4, 4, 4), seed=0)
    h = _handle(dev)
    hsc.hsc_analyze(h, 2)
    for c, v in ((2, 1), (-1, 1), (0, 2)):
        with pytest.raises(hsc.HSCError) as ei:
            hsc._check(h, hsc.load().hsc_set_contact_dense(h, c, v))
        assert ei.value.code == hsc.HSC_ERR_ARG
    hsc.hsc_set_contact_dense(h, 0)
    sr, sl = W.self_energies(dev, 1)
    out = np.zeros((1, dev.n), np.complex128)
    with pytest.raises(hsc.HSCError) as ei:
        hsc.hsc_solve(h, np.array([0.1]), 1e-6, sr, sl, hsc.HSC_FP64, None, out, out.copy(), None, None)
    assert ei.value.code == hsc.HSC_ERR_STATE
    hsc.hsc_destroy(h)


@pytest.mark.parametrize("dims,leaf,geo", [((32, 32, 32), 8, True), ((12, 9, 7), 3, True),
                                           ((9, 8, 7), 2, False)])
def test_alternate_trees_share_the_root_and_move_the_leaves(dims, leaf, geo):
    """The alternate separator trees keep the root separator (so the coupling entries across it
    stay in the selected pattern) and change the leaf clusters (different isolated blocks); shown
    on the plain geometric tree, whose deeper cuts run along every axis."""
    dev = W.cubic_device(dims, seed=2)
    trees = [_tree(dev, leaf, geo, v, ordering=2 if geo else None)[1] for v in (0, 1, 2, 3, 4)]
    roots = [set(t[-1][1].tolist()) for t in trees]
    assert all(r == roots[0] for r in roots)
    leaves = [{frozenset(own.tolist()) for info, own, _ in t if info.child[0] < 0 and info.child[1] < 0}
              for t in trees]
    assert all(leaves[a] != leaves[b] for a in range(5) for b in range(a))


def test_operation_count_follows_table_1_cube_slope():
    """Table 1: the HSC-extension costs O(N^6) on an N^3 cube; the model's log-log slope between
    N = 24 and N = 48 (leaves <= 8) must be close to 6 (and far from RGF's 7)."""
    f = []
    Ns = [24, 32, 40, 48]
    for N in Ns:
        st, _ = _tree(W.cubic_device((N, N, N), seed=0), 8)
        f.append(st.flops_gr + st.flops_gl)
    slope = np.polyfit(np.log(Ns), np.log(f), 1)[0]
    assert 5.3 < slope < 6.5, slope


def test_solve_dense_checks_its_arguments_on_the_host():
    """hsc_solve_dense needs a dense contact in the analysed tree and the block arrays that go with
    the diagonal ones; all checked before any device work."""
    dev = W.cubic_device((4, 3, 3), seed=0)
    sr, sl = W.self_energies(dev, 1)
    out = np.zeros((1, dev.n), np.complex128)
    E = np.array([0.2])
    blk = np.zeros((1, 2 * 9 * 9), np.complex128)
    h = _handle(dev)
    hsc.hsc_analyze(h, 2)
    with pytest.raises(hsc.HSCError) as ei:     # no dense contact
        hsc.hsc_solve_dense(h, E, 1e-6, sr, sl, blk, blk, hsc.HSC_FP64, None, out, out.copy(), None, None)
    assert ei.value.code == hsc.HSC_ERR_ARG and "dense" in str(ei.value)
    hsc.hsc_set_contact_dense(h, 0)
    hsc.hsc_set_contact_dense(h, 1)
    with pytest.raises(hsc.HSCError) as ei:     # not analysed since
        hsc.hsc_solve_dense(h, E, 1e-6, sr, sl, blk, blk, hsc.HSC_FP64, None, out, out.copy(), None, None)
    assert ei.value.code == hsc.HSC_ERR_STATE
    hsc.hsc_analyze(h, 2)
    for r, l, lsig in ((None, blk, sl), (blk, None, sl), (blk, blk, None)):
        with pytest.raises(hsc.HSCError) as ei:
            hsc.hsc_solve_dense(h, E, 1e-6, sr, lsig, r, l, hsc.HSC_FP64, None, out, out.copy(), None, None)
        assert ei.value.code == hsc.HSC_ERR_ARG
    hsc.hsc_destroy(h)


def test_dense_contacts_keep_the_cube_slope():
    """Section 3.1.2: DENSE self-energies make the HSC-extension slower but leave its asymptotic
    operation count unchanged. With both end planes dense the model's log-log slope between N = 24
    and N = 40 stays near 6, at a bounded multiple of the diagonal case."""
    Ns = [24, 32, 40]
    f, g = [], []
    for N in Ns:
        dev = W.cubic_device((N, N, N), seed=0)
        st, _ = _tree(dev, 8)
        st_d, _ = _tree(dev, 8, dense=(0, 1))
        f.append(st.flops_gr + st.flops_gl)
        g.append(st_d.flops_gr + st_d.flops_gl)
    slope = np.polyfit(np.log(Ns), np.log(g), 1)[0]
    assert 5.3 < slope < 6.5, slope
    assert all(1.2 < b / a < 3.0 for a, b in zip(f, g))


def test_graph_ordering_option_matches_a_handle_without_grid_dims():
    """HSC_OPT_ORDERING = 1 makes the next analysis ignore grid_dims: the same tree as a handle
    created without them, and exact for any variant."""
    dev = W.cubic_device((9, 8, 7), seed=3)
    h = _handle(dev, True)
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_ORDERING) == 0
    hsc.hsc_set_option(h, hsc.HSC_OPT_ORDERING, 1)
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_ORDERING) == 1
    st = hsc.hsc_analyze(h, 2)
    cl = [hsc.hsc_cluster(h, i) for i in range(st.n_clusters)]
    with pytest.raises(hsc.HSCError) as ei:
        hsc.hsc_set_option(h, hsc.HSC_OPT_ORDERING, 3)
    assert ei.value.code == hsc.HSC_ERR_ARG
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_TREE_FORM) == 2
    hsc.hsc_destroy(h)
    st2, cl2 = _tree(dev, 2, geometric=False)
    assert st.n_clusters == st2.n_clusters and st.flops_gr == st2.flops_gr
    assert all(np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2]) for a, b in zip(cl, cl2))
    _check_tree(dev, cl)


def test_degenerate_chain_tree():
    """A 1D chain with leaves of one site: every cluster is one unknown and every update set has at
    most two entries (the separator structure that makes HSC coincide with RGF, Section 2.2)."""
    st, cl = _tree(W.chain_device(31), 1, ordering=2)
    assert st.max_n == 1 and st.max_m <= 2


def test_scba_rejects_uncovered_sites_and_bad_parameters():
    """hsc_scba needs a self-energy slot on every unknown and sane loop parameters; both are
    checked on the host before any device work."""
    E = np.array([0.1])
    for dev, ok in ((W.cubic_device((4, 4, 4), seed=0), False),
                    (W.with_scattering_contact(W.cubic_device((4, 4, 4), seed=0)), True)):
        h = _handle(dev)
        hsc.hsc_analyze(h, 2)
        ncs = len(dev.contact_unknowns())
        sr = np.zeros((1, ncs), np.complex128)
        out = np.zeros((1, dev.n), np.complex128)
        for d0, mix, tol, it in ((-0.1, 0.5, 1e-8, 10), (0.1, 0.0, 1e-8, 10), (0.1, 1.5, 1e-8, 10),
                                 (0.1, 0.5, -1.0, 10), (0.1, 0.5, 1e-8, 0)):
            with pytest.raises(hsc.HSCError) as ei:
                hsc.hsc_scba(h, E, 1e-6, sr, sr.copy(), d0, mix, tol, it, hsc.HSC_FP64, out, out.copy())
            assert ei.value.code == hsc.HSC_ERR_ARG
        if not ok:
            with pytest.raises(hsc.HSCError) as ei:
                hsc.hsc_scba(h, E, 1e-6, sr, sr.copy(), 0.1, 0.5, 1e-8, 10, hsc.HSC_FP64, out, out.copy())
            assert ei.value.code == hsc.HSC_ERR_ARG and "cover every site" in str(ei.value)
        hsc.hsc_destroy(h)


def test_options_round_trip_and_reject_bad_values():
    dev = W.cubic_device((4, 4, 4), seed=0)
    h = _handle(dev)
    hsc.hsc_analyze(h, 2)
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_GJ_PANEL) == 16
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_GJ_WIDE) == 128
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_LEAF) == 2
    hsc.hsc_set_option(h, hsc.HSC_OPT_GJ_PANEL, 8)
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_GJ_PANEL) == 8
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_RESOLVE_DIGITS) == 10
    hsc.hsc_set_option(h, hsc.HSC_OPT_FP64_ENGINE, 2)
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_FP64_ENGINE) == 2
    hsc.hsc_set_option(h, hsc.HSC_OPT_RESOLVE_DIGITS, 8)
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_RESOLVE_DIGITS) == 8
    hsc.hsc_set_option(h, hsc.HSC_OPT_GJ_WIDE, 0)
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_GJ_WIDE) == 0
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_LEAF_BAND) == 1
    hsc.hsc_set_option(h, hsc.HSC_OPT_LEAF_BAND, 0)
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_LEAF_BAND) == 0
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_LEAF_SPARSE) == 1
    hsc.hsc_set_option(h, hsc.HSC_OPT_LEAF_SPARSE, 0)
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_LEAF_SPARSE) == 0
    for opt, val in ((hsc.HSC_OPT_GJ_PANEL, 0), (hsc.HSC_OPT_GJ_PANEL, 65), (99, 1),
                     (hsc.HSC_OPT_FP64_ENGINE, 3), (hsc.HSC_OPT_RESOLVE_DIGITS, 16),
                     (hsc.HSC_OPT_TREE_VARIANT, 5), (hsc.HSC_OPT_GJ_WIDE, -1), (hsc.HSC_OPT_GJ_WIDE, 513),
                     (hsc.HSC_OPT_TREE_FORM, 1), (hsc.HSC_OPT_LEAF_BAND, 2), (hsc.HSC_OPT_LEAF_BAND, -1),
                     (hsc.HSC_OPT_LEAF_SPARSE, 2)):
        with pytest.raises(hsc.HSCError) as ei:
            hsc.hsc_set_option(h, opt, val)
        assert ei.value.code == hsc.HSC_ERR_ARG
    with pytest.raises(hsc.HSCError):
        hsc.hsc_solve_batch([], 0.05, hsc.HSC_FP64)
    hsc.hsc_destroy(h)


def test_binding_rejects_buffers_of_the_wrong_kind_before_the_call():
    """A host array given for device I/O (or a float32 array) would be read as something else by the
    library; the binding refuses it before any C call."""
    import torch
    dev = W.cubic_device((3, 3, 3), seed=0)
    h = _handle(dev)
    hsc.hsc_analyze(h, 2)
    sr, sl = W.self_energies(dev, 1)
    out = np.zeros((1, dev.n), np.complex128)
    E = np.array([0.1])
    with pytest.raises(ValueError):
        hsc.hsc_solve(h, E, 1e-6, sr, sl, hsc.HSC_FP64, None, out, out.copy(), None, None, io_on_device=True)
    with pytest.raises(TypeError):
        hsc.hsc_solve(h, E.astype(np.float32), 1e-6, sr, sl, hsc.HSC_FP64, None, out, out.copy(), None, None)
    with pytest.raises(ValueError):
        hsc.hsc_scba(h, torch.from_numpy(E), 1e-6, sr, sl, 0.1, 0.5, 1e-8, 3, hsc.HSC_FP64, out, out.copy(),
                     io_on_device=True)
    with pytest.raises(TypeError):
        hsc.hsc_solve(h, torch.from_numpy(E).float(), 1e-6, sr, sl, hsc.HSC_FP64, None, out, out.copy(),
                      None, None)
    hsc.hsc_destroy(h)
    blocks = torch.zeros(2 * 4 * 4 * 2, dtype=torch.float64)   # host memory: refused for device I/O
    with pytest.raises(ValueError):
        hsc.hsc_block_inverse_noalloc(4, 2, blocks, blocks)
    with pytest.raises(ValueError):
        hsc.hsc_block_inverse_noalloc(4, 2, None, None)


FLOPS_CC = (427439805056.0, 272819044952.0)   # model flops per energy, contact-connected 32^3 tree


def test_metric_workload_tree_is_unchanged():
    """The 32^3 workload's trees (leaf_max 8) and their models, the figures the measurements use:
    the default contact-connected tree (x cut once, 15/16 x 8 x 8 leaves): 63 clusters over 6
    levels; the plain geometric tree (8^3 leaves): 127 clusters over 7 levels, 179.5 + 189.6 GFLOP
    per energy."""
    dev = W.cubic_device((32, 32, 32), seed=0)
    h = _handle(dev)
    st = hsc.hsc_analyze(h, 8)
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_TREE_FORM) == 1
    assert (st.n_clusters, st.n_heights, st.n_depths, st.max_n, st.max_m) == (63, 6, 6, 1024, 1024)
    assert abs(st.flops_gr - FLOPS_CC[0]) <= 1.0 and abs(st.flops_gl - FLOPS_CC[1]) <= 1.0
    hsc.hsc_set_option(h, hsc.HSC_OPT_ORDERING, 2)
    st = hsc.hsc_analyze(h, 8)
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_TREE_FORM) == 0
    hsc.hsc_destroy(h)
    assert (st.n_clusters, st.n_heights, st.n_depths, st.max_n, st.max_m) == (127, 7, 7, 1024, 1024)
    assert abs(st.flops_gr - 179528180960.0) <= 1.0 and abs(st.flops_gl - 189624310312.0) <= 1.0


def test_contact_connected_tree_keeps_every_box_on_a_contact_face():
    """Contact-connected dissection (the default for contacts on the end planes x = 0 and
    x = Nx-1): the root is the one x plane; every other cluster is a y or z cut or a leaf box
    spanning half the device in x, so each of them holds sites of an end plane; the tree is exact.
    An elongated device keeps the plain form (model cost above 3x)."""
    for dims, leaf in (((12, 9, 7), 3), ((9, 8, 8), 4), ((16, 5, 11), 2)):
        dev = W.cubic_device(dims, seed=1)
        st, cl = _tree(dev, leaf)
        _check_tree(dev, cl)
        Nx, Ny, Nz = dims
        x_of = lambda own: own // (Ny * Nz)   # noqa: E731  (one orbital per site)
        root = cl[-1][1]
        assert len(set(x_of(root).tolist())) == 1 and len(root) == Ny * Nz
        for info, own, upd in cl[:-1]:
            xs = set(x_of(own).tolist())
            assert 0 in xs or Nx - 1 in xs, (dims, info.n)
            if info.child[0] < 0:
                assert max(np.ptp((own % (Ny * Nz)) // Nz), np.ptp(own % Nz)) < leaf
    wire = W.wire_device((64, 12, 12), orb=2, seed=0)
    h = _handle(wire)
    hsc.hsc_analyze(h, 4)
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_TREE_FORM) == 0
    hsc.hsc_destroy(h)


def test_binding_constants_match_the_header():
    """Every enumerator of include/*.h (status codes, precisions, options) has the same value in the
    Python binding, so a call through either passes the same integer."""
    consts = {}
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", f)).read(), flags=re.S)
            for body in re.findall(r"\benum\b[^{]*\{(.*?)\}", txt, flags=re.S):
                for name, val in re.findall(r"\b(HSC_\w+)\s*=\s*(-?\d+)", body):
                    consts[name] = int(val)
    assert {"HSC_OK", "HSC_ERR_TIMEOUT", "HSC_FP64", "HSC_MIXED", "HSC_OPT_LEAF_SPARSE"} <= set(consts)
    for name, val in consts.items():
        assert getattr(hsc, name) == val, name


def test_binding_argument_counts_match_the_header():
    """Every function the binding declares (ctypes argtypes) takes as many arguments as its
    prototype in include/*.h: a dropped or extra argument would shift every later one."""
    protos = {}
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", f)).read(), flags=re.S)
            txt = re.sub(r"//[^\n]*", "", txt)
            for name, params in re.findall(r"\b(hsc_\w+)\s*\(([^;{}]*?)\)\s*;", txt, flags=re.S):
                p = params.strip()
                protos[name] = 0 if p in ("", "void") else p.count(",") + 1
    L = hsc.load()
    checked = 0
    for name, n in protos.items():
        at = getattr(L, name).argtypes
        if at is not None:
            assert len(at) == n, (name, len(at), n)
            checked += 1
    assert checked >= 15
