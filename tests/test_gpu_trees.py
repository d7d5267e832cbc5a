"""GPU parity on the cluster trees that the analysis options build beyond plain nested dissection:
merged trees (hsc_set_merge: a cluster eliminated together with its parent, pass-through clusters
with no own unknowns keeping the tree binary), the degenerate chains of HSC_OPT_MAX_CLUSTER
(Section 3.4: an oversized cluster split into a chain of pieces, each the parent of the previous),
and both together. Every solve goes through the C ABI and is compared element by element with the
dense definition (Eqs. 1-2) at eta = 0.05, where the block elimination's growth is bounded, so
any indexing mistake in the assembly, gather, fold or downward pass over such clusters shows up as
an O(1) difference."""
import numpy as np
import pytest

from oracle import dense
from paper_1702_05167_gb300 import hsc, workloads as W
from test_chain_split import _dense_blocks_device
from treecheck import _check_tree, _handle

pytestmark = pytest.mark.gpu
TOL = 1e-10
ETA = 0.05


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hsc.load()


def _relerr(x, ref):
    return np.abs(x - ref).max() / np.abs(ref).max()


def _solve_and_check(dev, h, E, f=(1.0, 0.0), pairs=None):
    sr, sl = W.self_energies(dev, len(E), f)
    n_E, n = len(E), dev.n
    dgr = np.zeros((n_E, n), np.complex128)
    dgl = np.zeros((n_E, n), np.complex128)
    pgr = np.zeros((n_E, len(pairs)), np.complex128) if pairs is not None else None
    pgl = np.zeros_like(pgr) if pairs is not None else None
    hsc.hsc_solve(h, np.ascontiguousarray(E, np.float64), ETA, sr, sl, hsc.HSC_FP64, pairs, dgr, dgl, pgr, pgl)
    Hd = dev.to_scipy().toarray()
    for k in range(n_E):
        G, Gl = dense.solve(Hd, E[k], ETA, dev.contact_unknowns(), sr[k], sl[k])
        assert _relerr(dgr[k], np.diag(G)) <= TOL, k
        assert _relerr(dgl[k], np.diag(Gl)) <= TOL, k
        if pairs is not None:
            assert _relerr(pgr[k], G[pairs[:, 0], pairs[:, 1]]) <= TOL, k
            assert _relerr(pgl[k], Gl[pairs[:, 0], pairs[:, 1]]) <= TOL, k


def _tree(h, leaf):
    st = hsc.hsc_analyze(h, leaf)
    return st, [hsc.hsc_cluster(h, i) for i in range(st.n_clusters)]


@pytest.mark.parametrize("kind", ["separators", "leaves", "mixed"])
def test_merged_trees_match_dense(kind):
    dev = W.cubic_device((9, 7, 6), W=1.0, seed=1)
    h = _handle(dev)
    _, base = _tree(h, 2)
    seps = [i for i, (info, _, _) in enumerate(base) if info.child[0] >= 0 and info.parent >= 0]
    leaves = [i for i, (info, _, _) in enumerate(base) if info.child[0] < 0]
    rng = np.random.default_rng({"separators": 0, "leaves": 1, "mixed": 2}[kind])
    merge = {"separators": list(rng.choice(seps, 4, replace=False)),
             "leaves": list(rng.choice(leaves, 6, replace=False)),
             "mixed": list(rng.choice(seps, 3, replace=False)) + list(rng.choice(leaves, 3, replace=False))}[kind]
    hsc.hsc_set_merge(h, [int(m) for m in merge])
    st, cl = _tree(h, 2)
    _check_tree(dev, cl)
    if kind != "leaves":
        assert any(info.n == 0 for info, _, _ in cl)      # pass-through clusters are exercised
    _solve_and_check(dev, h, np.array([-2.3, 0.15, 1.8]), f=(1.0, 0.4), pairs=W.plane_pairs(dev, 4))
    hsc.hsc_destroy(h)


@pytest.mark.parametrize("K", [8, 16])
def test_chain_split_dense_blocks_match_dense(K):
    """The DNA-like stand-in (dense all-to-all blocks joined by a few bonds, graph ordering): every
    cluster larger than K sites becomes a chain of pieces of at most K."""
    dev = _dense_blocks_device()
    h = _handle(dev, geometric=False)
    hsc.hsc_set_option(h, hsc.HSC_OPT_MAX_CLUSTER, K)
    st, cl = _tree(h, 3)
    assert max(info.n for info, _, _ in cl) <= K
    _solve_and_check(dev, h, np.array([-0.7, 0.2, 1.1]))
    hsc.hsc_destroy(h)


def test_chain_split_with_merges_on_a_cube_matches_dense():
    dev = W.cubic_device((8, 6, 5), W=1.0, seed=3)
    h = _handle(dev)
    hsc.hsc_set_option(h, hsc.HSC_OPT_MAX_CLUSTER, 12)
    hsc.hsc_analyze(h, 3)
    hsc.hsc_set_merge(h, [0, 5])
    st, cl = _tree(h, 3)
    assert max(info.n for info, _, _ in cl) <= 12
    _check_tree(dev, cl)
    _solve_and_check(dev, h, np.array([-1.4, 0.6]), pairs=W.plane_pairs(dev, 3))
    hsc.hsc_destroy(h)
