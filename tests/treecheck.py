"""Helpers shared by the analysis tests: build a handle's cluster tree and check it exactly
against the coupling graph (partition, separation, update sets). No GPU."""
import numpy as np

from paper_1702_05167_gb300 import hsc


def _handle(dev, geometric=True):
    return hsc.hsc_create(dev.n, dev.orb, dev.rowptr, dev.col, dev.val, dev.contact_ptr,
                          dev.contact_sites, dev.dims if geometric else None)


def _tree(dev, leaf, geometric=True, variant=0, dense=(), ordering=None):
    h = _handle(dev, geometric)
    if ordering is not None:
        hsc.hsc_set_option(h, hsc.HSC_OPT_ORDERING, ordering)
    if variant:
        hsc.hsc_set_option(h, hsc.HSC_OPT_TREE_VARIANT, variant)
    for c in dense:
        hsc.hsc_set_contact_dense(h, c)
    st = hsc.hsc_analyze(h, leaf)
    cl = [hsc.hsc_cluster(h, i) for i in range(st.n_clusters)]
    hsc.hsc_destroy(h)
    return st, cl


def _check_tree(dev, cl, extra_edges=()):
    """Every unknown owned once; no coupling (H entries and extra_edges) joins two unrelated
    clusters; each U_i is exactly the set of ancestor unknowns adjacent to the subtree of i."""
    nc = len(cl)
    owner = np.full(dev.n, -1)
    for i, (info, own, upd) in enumerate(cl):
        assert np.all(owner[own] == -1)
        owner[own] = i
    assert np.all(owner >= 0)
    parent = [info.parent for info, _, _ in cl]
    assert parent[-1] == -1 and all(p > i for i, p in enumerate(parent[:-1]))
    anc = [set() for _ in range(nc)]
    for i in range(nc - 1, -1, -1):
        if parent[i] >= 0:
            anc[i] = anc[parent[i]] | {parent[i]}
    sub = [set() for _ in range(nc)]
    for i in range(nc):
        sub[i].add(i)
        for a in anc[i]:
            sub[a].add(i)
    H = dev.to_scipy().tocoo()
    pairs = list(zip(H.row, H.col)) + list(extra_edges)
    for a, b in pairs:
        ca, cb = owner[a], owner[b]
        assert ca == cb or ca in anc[cb] or cb in anc[ca]
    adj = [set() for _ in range(dev.n)]
    for a, b in pairs:
        if a != b:
            adj[a].add(b)
    for i, (info, own, upd) in enumerate(cl):
        dom = set(np.nonzero(np.isin(owner, list(sub[i])))[0])
        boundary = set()
        for u in dom:
            boundary |= adj[u]
        boundary -= dom
        assert set(upd.tolist()) == boundary
        assert all(owner[u] in anc[i] for u in upd)
        assert info.m == len(upd) and info.n == len(own)
    return owner
