"""Leaf clusters. Column bands (HSC_OPT_LEAF_BAND): the downward products of a leaf cluster form its G_ii and
G^<_ii blocks only on the column band, per block of <= 128 rows, that spans the entries read
afterwards (diagonal, the residual check's H neighbours, requested pairs inside the block, and every
column of a lesser leaf's contact rows). On the FP64-emulation engine each computed entry is the
same exact digit sum rounded once, so the outputs must equal those of whole blocks bit for bit;
both against the dense definition (Eqs. 1-2) at eta = 0.05. Sparse coupling blocks
(HSC_OPT_LEAF_SPARSE): a leaf's X = D^{-1} A_iU and Schur update from the H pattern of A_iU, in FP64,
against the dense block products and the dense definition."""
import numpy as np
import pytest

from oracle import dense
from paper_1702_05167_gb300 import hsc, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hsc.load()


def _leaf_pairs(dev, s, count, seed):
    """Pairs (u, v) with both unknowns in one leaf cluster and far apart in its local order (outside
    any band the diagonal and the H neighbours alone would give)."""
    rng = np.random.default_rng(seed)
    cl = [hsc.hsc_cluster(s.h, i) for i in range(s.stats.n_clusters)]
    parents = {info.parent for info, _, _ in cl}
    leaves = [np.asarray(own) for i, (info, own, _) in enumerate(cl) if i not in parents and len(own) > 1]
    out = []
    for k in range(count):
        own = leaves[rng.integers(len(leaves))]
        a, b = rng.choice(len(own), 2, replace=False)
        out.append((own[min(a, b)], own[max(a, b)]))
    return np.array(out, dtype=np.int32)


def _solve(dev, leaf, band, pairs, E, sr, sl, engine=2, sparse=1):
    s = hsc.Solver(dev, leaf)
    hsc.hsc_set_option(s.h, hsc.HSC_OPT_FP64_ENGINE, engine)
    hsc.hsc_set_option(s.h, hsc.HSC_OPT_LEAF_BAND, band)
    hsc.hsc_set_option(s.h, hsc.HSC_OPT_LEAF_SPARSE, sparse)
    out = s.solve(E, 0.05, sr, sl, pairs=pairs)
    res = hsc.hsc_residual(s.h, len(E))
    return s, out, res


@pytest.mark.parametrize("dims,leaf", [((15, 16, 16), 8), ((9, 7, 8), 3)])
def test_leaf_bands_equal_whole_blocks_bitwise(dims, leaf):
    dev = W.cubic_device(dims, W=1.0, seed=5)
    E = np.array([-1.3, 0.45])
    sr, sl = W.self_energies(dev, len(E))
    s0 = hsc.Solver(dev, leaf)
    pairs = np.concatenate([W.plane_pairs(dev, dims[0] // 2), _leaf_pairs(dev, s0, 40, 1)])
    s0.close()
    sb, ob, rb = _solve(dev, leaf, 1, pairs, E, sr, sl)
    sf, of, rf = _solve(dev, leaf, 0, pairs, E, sr, sl)
    for a, b in zip(ob, of):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(rb, rf)
    Hd = dev.to_scipy().toarray()
    for k in range(len(E)):
        G, Gl = dense.solve(Hd, E[k], 0.05, dev.contact_unknowns(), sr[k], sl[k])
        for x, ref in ((ob[0][k], np.diag(G)), (ob[1][k], np.diag(Gl)),
                       (ob[2][k], G[pairs[:, 0], pairs[:, 1]]), (ob[3][k], Gl[pairs[:, 0], pairs[:, 1]])):
            assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()
    sb.close()
    sf.close()


def test_new_pairs_inside_leaves_rebuild_the_bands():
    """A second solve on the same handle asking for other pairs inside leaf blocks: the schedule is
    rebuilt so that the bands cover them; the results equal a whole-block solve."""
    dims = (12, 10, 9)
    dev = W.cubic_device(dims, W=1.0, seed=8)
    E = np.array([0.3])
    sr, sl = W.self_energies(dev, 1)
    s = hsc.Solver(dev, 4)
    hsc.hsc_set_option(s.h, hsc.HSC_OPT_FP64_ENGINE, 2)
    p1 = _leaf_pairs(dev, s, 10, 2)
    p2 = _leaf_pairs(dev, s, 25, 3)
    s.solve(E, 0.05, sr, sl, pairs=p1)
    got = s.solve(E, 0.05, sr, sl, pairs=p2)
    _, ref, _ = _solve(dev, 4, 0, p2, E, sr, sl)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
    s.close()


def test_leaf_bands_with_dense_contact_blocks():
    """DENSE lead blocks on both end planes (the contact rows of the leaves are read whole by the
    lesser products): banded and whole-block solves agree bit for bit, diag and face pairs."""
    from oracle import lead
    dims, t, eta = (8, 6, 5), -1.0, 0.05
    dev = W.cubic_device(dims, t=t, W=1.0, seed=9)
    E = np.array([-0.45, 1.3])
    H00, H01 = W.cubic_lead(dims, t=t)
    tau = t * np.eye(H00.shape[0])
    S = [lead.contact_self_energy(e, eta, H00, H01, tau) for e in E]
    ncs = len(dev.contact_unknowns())
    nu = ncs // 2
    zr = np.zeros((len(E), ncs), np.complex128)
    dr = np.zeros((len(E), 2 * nu * nu), np.complex128)
    dl = np.zeros_like(dr)
    for k in range(len(E)):
        dr[k, :nu * nu] = S[k].ravel()
        dr[k, nu * nu:] = S[k].ravel()
        dl[k, :nu * nu] = (1j * lead.broadening(S[k])).ravel()
    right = W.face_sites(dims, dims[0] - 1).astype(np.int32)
    a, b = np.meshgrid(right, right, indexing="ij")
    pairs = np.stack([a.ravel(), b.ravel()], axis=1).astype(np.int32)
    outs = []
    for band in (1, 0):
        h = hsc.hsc_create(dev.n, dev.orb, dev.rowptr, dev.col, dev.val, dev.contact_ptr, dev.contact_sites,
                           dev.dims)
        hsc.hsc_set_contact_dense(h, 0)
        hsc.hsc_set_contact_dense(h, 1)
        hsc.hsc_analyze(h, 2)
        hsc.hsc_set_option(h, hsc.HSC_OPT_FP64_ENGINE, 2)
        hsc.hsc_set_option(h, hsc.HSC_OPT_LEAF_BAND, band)
        o = [np.zeros((len(E), dev.n), np.complex128), np.zeros((len(E), dev.n), np.complex128),
             np.zeros((len(E), len(pairs)), np.complex128), np.zeros((len(E), len(pairs)), np.complex128)]
        hsc.hsc_solve_dense(h, E, eta, zr, zr.copy(), dr, dl, hsc.HSC_FP64, pairs, *o)
        hsc.hsc_destroy(h)
        outs.append(o)
    for x, y in zip(*outs):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("dims,leaf", [((15, 16, 16), 8), ((9, 7, 8), 3), ((12, 10, 9), 4)])
def test_sparse_leaf_couplings_against_dense_products(dims, leaf):
    """X and the Schur update of every leaf from A_iU's H pattern (FP64 gathers) against the dense
    block products of the same tree: diag G^r, diag G^<, coupling and in-leaf pairs within 1e-12
    of each other, both within 1e-10 of the dense definition; residuals within 1e-12 absolute."""
    dev = W.cubic_device(dims, W=1.0, seed=12)
    E = np.array([-2.1, 0.6])
    sr, sl = W.self_energies(dev, len(E))
    s0 = hsc.Solver(dev, leaf)
    pairs = np.concatenate([W.plane_pairs(dev, dims[0] // 2), _leaf_pairs(dev, s0, 30, 4)])
    s0.close()
    ss, osp, rsp = _solve(dev, leaf, 1, pairs, E, sr, sl, engine=0, sparse=1)
    sd, odn, rdn = _solve(dev, leaf, 1, pairs, E, sr, sl, engine=0, sparse=0)
    for a, b in zip(osp, odn):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    assert np.abs(rsp - rdn).max() <= 1e-12
    Hd = dev.to_scipy().toarray()
    for k in range(len(E)):
        G, Gl = dense.solve(Hd, E[k], 0.05, dev.contact_unknowns(), sr[k], sl[k])
        for x, ref in ((osp[0][k], np.diag(G)), (osp[1][k], np.diag(Gl)),
                       (osp[2][k], G[pairs[:, 0], pairs[:, 1]]), (osp[3][k], Gl[pairs[:, 0], pairs[:, 1]])):
            assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()
    ss.close()
    sd.close()


def test_banded_inversion_with_pivots_below_the_diagonal():
    """Weak disorder at E ~ 0: the leaves' diagonal entries (E - eps_i, |eps_i| <= 0.1) are small
    against the hopping, so partial pivoting takes most pivots from rows below the diagonal, up to
    the bandwidth. The banded Gauss-Jordan (HSC_OPT_LEAF_SPARSE = 1) must still give the dense
    definition at 1e-10 and the dense-block path within 1e-12."""
    dims = (14, 9, 9)
    dev = W.cubic_device(dims, W=0.2, seed=21)
    E = np.array([0.0, 0.05, -0.03])
    sr, sl = W.self_energies(dev, len(E))
    pairs = W.plane_pairs(dev, dims[0] // 2)
    ss, osp, _ = _solve(dev, 4, 1, pairs, E, sr, sl, engine=0, sparse=1)
    sd, odn, _ = _solve(dev, 4, 1, pairs, E, sr, sl, engine=0, sparse=0)
    for a, b in zip(osp, odn):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    Hd = dev.to_scipy().toarray()
    for k in range(len(E)):
        G, Gl = dense.solve(Hd, E[k], 0.05, dev.contact_unknowns(), sr[k], sl[k])
        for x, ref in ((osp[0][k], np.diag(G)), (osp[1][k], np.diag(Gl)), (osp[2][k], G[pairs[:, 0], pairs[:, 1]])):
            assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()
    ss.close()
    sd.close()
