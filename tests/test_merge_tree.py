"""Merged cluster trees (hsc_set_merge): the analysis stays exact, pass-through clusters keep the tree
binary, the recurrences over merged trees reproduce Eqs. 1-2, and merging the high-growth clusters
recovers the digits an isolated level costs at small eta. CPU only."""
import numpy as np
import pytest

from hsc_emulator import selected, tree
from oracle import dense
from paper_1702_05167_gb300 import hsc, workloads as W
from treecheck import _check_tree, _handle


def _merged(dev, leaf, merge, geo=True, dense_contacts=()):
    h = _handle(dev, geo)
    for c in dense_contacts:
        hsc.hsc_set_contact_dense(h, c)
    st0 = hsc.hsc_analyze(h, leaf)
    base = [hsc.hsc_cluster(h, i) for i in range(st0.n_clusters)]
    hsc.hsc_set_merge(h, merge)
    st = hsc.hsc_analyze(h, leaf)
    cl = [hsc.hsc_cluster(h, i) for i in range(st.n_clusters)]
    hsc.hsc_destroy(h)
    return base, cl


def _separators(base):
    return [i for i, (info, _, _) in enumerate(base) if info.child[0] >= 0 and info.parent >= 0]


@pytest.mark.parametrize("geo", [True, False])
def test_merged_trees_are_exact_and_binary(geo):
    dev = W.cubic_device((9, 7, 6), seed=1)
    h = _handle(dev, geo)
    st = hsc.hsc_analyze(h, 2)
    base = [hsc.hsc_cluster(h, i) for i in range(st.n_clusters)]
    hsc.hsc_destroy(h)
    rng = np.random.default_rng(0)
    seps = _separators(base)
    leaves = [i for i, (info, _, _) in enumerate(base) if info.child[0] < 0]
    for merge in ([seps[0]], list(rng.choice(seps, 4, replace=False)), list(rng.choice(leaves, 6, replace=False)),
                  list(rng.choice(seps, 3, replace=False)) + list(rng.choice(leaves, 3, replace=False))):
        merge = [int(m) for m in merge]
        _, cl = _merged(dev, 2, merge, geo)
        _check_tree(dev, cl)
        for info, own, upd in cl:
            assert info.child[0] >= 0 or info.child[1] < 0
            if info.n == 0:      # pass-through: two children, updates handed on
                assert info.child[0] >= 0 and info.child[1] >= 0
        # every merged cluster's unknowns now live with its parent's (or a further merged ancestor's)
        owner = {}
        for i, (info, own, upd) in enumerate(cl):
            for u in own:
                owner[int(u)] = i
        for m in merge:
            p = base[m][0].parent
            while p in merge:
                p = base[p][0].parent
            assert {owner[int(u)] for u in base[m][1]} == {owner[int(base[p][1][0])]}


def test_merging_a_separator_creates_pass_through_clusters():
    dev = W.cubic_device((8, 8, 8), seed=2)
    h = _handle(dev)
    st = hsc.hsc_analyze(h, 2)
    base = [hsc.hsc_cluster(h, i) for i in range(st.n_clusters)]
    hsc.hsc_destroy(h)
    sep = next(i for i in _separators(base) if base[base[i][0].parent][0].parent >= 0)
    _, cl = _merged(dev, 2, [sep])
    assert sum(info.n == 0 for info, _, _ in cl) == 1 and len(cl) == len(base)
    _check_tree(dev, cl)


def test_merge_list_errors():
    dev = W.cubic_device((4, 4, 4), seed=0)
    h = _handle(dev)
    st = hsc.hsc_analyze(h, 2)
    for bad in ([st.n_clusters - 1], [st.n_clusters + 5]):
        hsc.hsc_set_merge(h, bad)
        with pytest.raises(hsc.HSCError) as ei:
            hsc.hsc_analyze(h, 2)
        assert ei.value.code == hsc.HSC_ERR_ARG
    with pytest.raises(hsc.HSCError) as ei:
        hsc.hsc_set_merge(h, [-1])
    assert ei.value.code == hsc.HSC_ERR_ARG
    hsc.hsc_set_merge(h, [])
    assert hsc.hsc_analyze(h, 2).n_clusters == st.n_clusters
    hsc.hsc_destroy(h)


def test_recurrences_over_merged_trees_reproduce_the_definition():
    dev = W.cubic_device((7, 5, 4), seed=4)
    h = _handle(dev)
    st = hsc.hsc_analyze(h, 2)
    base = [hsc.hsc_cluster(h, i) for i in range(st.n_clusters)]
    hsc.hsc_destroy(h)
    merge = [int(m) for m in np.random.default_rng(3).choice(_separators(base), 3, replace=False)]
    _, cl = _merged(dev, 2, merge, dense_contacts=())
    sr, sl = W.self_energies(dev, 1)
    idx = dev.contact_unknowns()
    A = dense.system_matrix(dev.to_scipy().toarray(), 0.3, 0.05, dense.embed_diag(dev.n, idx, sr[0]))
    L = dense.embed_diag(dev.n, idx, sl[0])
    G, P = selected(A, L, [(np.asarray(o, np.int64), np.asarray(u, np.int64)) for _, o, u in cl])
    Gd = dense.retarded(A)
    Pd = dense.lesser(Gd, L)
    assert np.abs(np.diag(G) - np.diag(Gd)).max() <= 1e-11 * np.abs(np.diag(Gd)).max()
    assert np.abs(np.diag(P) - np.diag(Pd)).max() <= 1e-11 * np.abs(np.diag(Pd)).max()


def test_merging_high_growth_clusters_recovers_the_lost_digits():
    """12^3, leaves <= 3, eta = 1e-6, E = -1.1: an isolated level costs the plain tree ~4e-3 of
    diag G^r; merging the clusters whose D_i^{-1} growth exceeds 30x the median (the library's own
    merged tree) brings it below 1e-6 for about the same flops."""
    dev = W.cubic_device((12, 12, 12), seed=0)
    sr, sl = W.self_energies(dev, 1)
    idx = dev.contact_unknowns()
    A = dense.system_matrix(dev.to_scipy().toarray(), -1.1, 1e-6, dense.embed_diag(dev.n, idx, sr[0]))
    L = dense.embed_diag(dev.n, idx, sl[0])
    gd = np.diag(np.linalg.inv(A))
    h = _handle(dev)
    hsc.hsc_set_option(h, hsc.HSC_OPT_ORDERING, 2)   # the plain geometric tree, which meets the level
    st = hsc.hsc_analyze(h, 3)
    base = tree(h, st.n_clusters)
    parents = [hsc.hsc_cluster(h, i, want_sets=False)[0].parent for i in range(st.n_clusters)]
    stats = {}
    G, _ = selected(A, L, base, stats)
    e0 = np.abs(np.diag(G) - gd).max() / np.abs(gd).max()
    g = np.array(stats["cluster_growth"])
    merge = [i for i in range(len(g)) if g[i] > 30 * np.median(g) and parents[i] >= 0]
    hsc.hsc_set_merge(h, merge)
    st2 = hsc.hsc_analyze(h, 3)
    cl = tree(h, st2.n_clusters)
    hsc.hsc_destroy(h)
    G2, _ = selected(A, L, cl)
    e1 = np.abs(np.diag(G2) - gd).max() / np.abs(gd).max()
    assert e0 > 1e-4 and e1 < 1e-6 and 0 < len(merge) < 20
    assert (st2.flops_gr + st2.flops_gl) < 1.1 * (st.flops_gr + st.flops_gl)
