"""Degenerate sub-trees (HSC_OPT_MAX_CLUSTER, Section 3.4): clusters larger than the limit become
chains of pieces; the trees stay exact and the recurrences over them reproduce Eqs. 1-2. CPU only."""
import numpy as np
import pytest

from hsc_emulator import selected, tree
from oracle import dense
from paper_1702_05167_gb300 import hsc, workloads as W
from treecheck import _check_tree, _handle


def _dense_blocks_device(sizes=(40, 40, 24), seed=0):
    """A DNA-like stand-in: dense all-to-all blocks (random symmetric couplings) joined by a few
    bonds, contacts on the first and last block's first sites; no grid."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    n = sum(sizes)
    H = np.zeros((n, n))
    off = 0
    starts = []
    for m in sizes:
        B = rng.normal(scale=0.3, size=(m, m))
        H[off:off + m, off:off + m] = B + B.T
        starts.append(off)
        off += m
    for k in range(len(sizes) - 1):
        a, b = starts[k] + sizes[k] - 1, starts[k + 1]
        for j in range(3):
            H[a - j, b + j] = H[b + j, a - j] = -1.0
    M = sp.csr_matrix(H.astype(np.complex128))
    M.sort_indices()
    left = np.arange(0, 4, dtype=np.int32)
    right = np.arange(n - 4, n, dtype=np.int32)
    return W.Device(dims=(n, 1, 1), orb=1, rowptr=M.indptr.astype(np.int64), col=M.indices.astype(np.int32),
                    val=M.data.astype(np.complex128), contact_ptr=np.array([0, 4, 8], np.int64),
                    contact_sites=np.concatenate([left, right]), gamma=np.array([0.5, 0.5]))


def _split_tree(dev, K, geo=False, leaf=3, merge=()):
    h = _handle(dev, geo)
    hsc.hsc_set_option(h, hsc.HSC_OPT_MAX_CLUSTER, K)
    assert hsc.hsc_get_option(h, hsc.HSC_OPT_MAX_CLUSTER) == K
    if merge:
        hsc.hsc_analyze(h, leaf)
        hsc.hsc_set_merge(h, list(merge))
    st = hsc.hsc_analyze(h, leaf)
    cl = [hsc.hsc_cluster(h, i) for i in range(st.n_clusters)]
    em = tree(h, st.n_clusters)
    hsc.hsc_destroy(h)
    return st, cl, em


@pytest.mark.parametrize("K", [8, 16, 25])
def test_dense_blocks_become_chains_of_bounded_pieces(K):
    dev = _dense_blocks_device()
    st0, cl0, _ = _split_tree(dev, 0)
    assert max(info.n for info, _, _ in cl0) > K          # bisection leaves a dense block whole
    st, cl, em = _split_tree(dev, K)
    assert max(info.n for info, _, _ in cl) <= K
    _check_tree(dev, cl)
    sr, sl = W.self_energies(dev, 1)
    idx = dev.contact_unknowns()
    A = dense.system_matrix(dev.to_scipy().toarray(), 0.2, 0.05, dense.embed_diag(dev.n, idx, sr[0]))
    L = dense.embed_diag(dev.n, idx, sl[0])
    G, P = selected(A, L, em)
    Gd = dense.retarded(A)
    Pd = dense.lesser(Gd, L)
    assert np.abs(np.diag(G) - np.diag(Gd)).max() <= 1e-11 * np.abs(np.diag(Gd)).max()
    assert np.abs(np.diag(P) - np.diag(Pd)).max() <= 1e-11 * np.abs(np.diag(Pd)).max()


def test_split_with_merges_and_on_a_cube_stays_exact():
    dev = W.cubic_device((8, 6, 5), seed=3)
    st, cl, _ = _split_tree(dev, 12, geo=True, leaf=3, merge=(0, 5))
    assert max(info.n for info, _, _ in cl) <= 12
    _check_tree(dev, cl)


def test_dense_contacts_are_not_split():
    dev = W.cubic_device((6, 5, 4), seed=1)
    h = _handle(dev)
    hsc.hsc_set_contact_dense(h, 0)
    hsc.hsc_set_option(h, hsc.HSC_OPT_MAX_CLUSTER, 6)
    st = hsc.hsc_analyze(h, 2)
    cl = [hsc.hsc_cluster(h, i) for i in range(st.n_clusters)]
    hsc.hsc_destroy(h)
    assert cl[-1][0].n == 20 and all(info.n <= 6 for info, _, _ in cl[:-1])
    with pytest.raises(hsc.HSCError):
        h = _handle(dev)
        try:
            hsc.hsc_set_option(h, hsc.HSC_OPT_MAX_CLUSTER, -1)
        finally:
            hsc.hsc_destroy(h)
