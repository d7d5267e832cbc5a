"""The implemented recurrences over the library's own trees reproduce Eqs. 1-2, on the CPU:
diagonal contacts, DENSE lead self-energies on the top-chain contact clusters, an alternate tree,
and the graph-ordered G-BN-G stand-in; and the LU form of the recurrences for a Hermitian,
non-symmetric H (no library solve yet). See hsc_emulator for what this does and does not show."""
import numpy as np
import pytest

from hsc_emulator import selected, tree
from oracle import dense, lead
from paper_1702_05167_gb300 import hsc, workloads as W
from treecheck import _handle

ETA = 0.05


def _run(dev, leaf, E, sigma, sless, geo=True, dense_contacts=(), variant=0):
    h = _handle(dev, geo)
    if variant:
        hsc.hsc_set_option(h, hsc.HSC_OPT_TREE_VARIANT, variant)
    for c in dense_contacts:
        hsc.hsc_set_contact_dense(h, c)
    st = hsc.hsc_analyze(h, leaf)
    cl = tree(h, st.n_clusters)
    hsc.hsc_destroy(h)
    A = dense.system_matrix(dev.to_scipy().toarray(), E, ETA, sigma)
    G, P = selected(A, sless, cl)
    Gd = dense.retarded(A)
    Pd = dense.lesser(Gd, sless)
    return G, P, Gd, Pd, cl


def _close(G, P, Gd, Pd, pairs):
    assert np.abs(np.diag(G) - np.diag(Gd)).max() <= 1e-11 * np.abs(np.diag(Gd)).max()
    assert np.abs(np.diag(P) - np.diag(Pd)).max() <= 1e-11 * np.abs(np.diag(Pd)).max()
    a, b = pairs[:, 0], pairs[:, 1]
    assert np.abs(G[a, b] - Gd[a, b]).max() <= 1e-11 * np.abs(Gd[a, b]).max()
    assert np.abs(P[a, b] - Pd[a, b]).max() <= 1e-11 * np.abs(Pd[a, b]).max()


def _h_pairs(dev):
    H = dev.to_scipy().tocoo()
    off = H.row != H.col
    return np.stack([H.row[off], H.col[off]], axis=1)


@pytest.mark.parametrize("variant", [0, 3])
def test_diagonal_contacts(variant):
    dev = W.cubic_device((7, 5, 4), seed=4)
    sr, sl = W.self_energies(dev, 1)
    idx = dev.contact_unknowns()
    G, P, Gd, Pd, _ = _run(dev, 2, 0.4, dense.embed_diag(dev.n, idx, sr[0]),
                           dense.embed_diag(dev.n, idx, sl[0]), variant=variant)
    _close(G, P, Gd, Pd, _h_pairs(dev))


@pytest.mark.parametrize("E", [-1.7, 0.6])
def test_dense_lead_self_energies_on_the_top_chain(E):
    """Both end planes carry full lead self-energy blocks (left lead filled): with the contacts
    marked dense, the recurrences over the chained tree give G^r and G^< exactly, including a
    dense, anti-Hermitian L_ii at the chain clusters."""
    dims, t = (7, 4, 3), -1.0
    dev = W.cubic_device(dims, t=t, seed=5)
    H00, H01 = W.cubic_lead(dims, t=t)
    S = lead.contact_self_energy(E, ETA, H00, H01, t * np.eye(H00.shape[0]))
    left, right = W.face_sites(dims, 0), W.face_sites(dims, dims[0] - 1)
    sigma = lead.embed_blocks(dev.n, [(left, S), (right, S)])
    sless = lead.embed_blocks(dev.n, [(left, 1j * lead.broadening(S))])
    G, P, Gd, Pd, cl = _run(dev, 2, E, sigma, sless, dense_contacts=(0, 1))
    assert set(cl[-1][0].tolist()) == set(right.tolist()) and set(cl[-2][0].tolist()) == set(left.tolist())
    _close(G, P, Gd, Pd, _h_pairs(dev))


def test_graph_ordered_gbng_stack():
    dev = W.gbng_device(8, 6, 4, W=0.3, seed=6)
    sr, sl = W.self_energies(dev, 1)
    idx = dev.contact_unknowns()
    G, P, Gd, Pd, _ = _run(dev, 2, -0.8, dense.embed_diag(dev.n, idx, sr[0]),
                           dense.embed_diag(dev.n, idx, sl[0]), geo=False)
    _close(G, P, Gd, Pd, _h_pairs(dev))


@pytest.mark.parametrize("z_form", [False, True])
@pytest.mark.parametrize("phi,E,leaf", [(0.13, 0.4, 2), (0.21, -1.6, 3)])
def test_lu_form_for_a_hermitian_non_symmetric_h(phi, E, leaf, z_form):
    """A magnetic device (Peierls phases: H Hermitian, H != H^T) on the tree of the same lattice
    without field (same pattern): the LU form of the recurrences gives G^r and G^< of Eqs. 1-2 on
    every selected block, with the lesser fold term by term or as Z - Z^dagger, while the
    complex-symmetric recurrences (Y = X^T) do not."""
    from hsc_emulator import selected_general
    dims = (7, 5, 4)
    dev = W.magnetic_cubic_device(dims, phi, seed=7)
    plain = W.cubic_device(dims, seed=7)
    Hp, Hm = plain.to_scipy(), dev.to_scipy()
    assert (abs(Hp) != 0).toarray().tolist() == (abs(Hm) != 0).toarray().tolist()
    h = _handle(plain, True)
    st = hsc.hsc_analyze(h, leaf)
    cl = tree(h, st.n_clusters)
    hsc.hsc_destroy(h)
    sr, sl = W.self_energies(dev, 1)
    idx = dev.contact_unknowns()
    A = dense.system_matrix(Hm.toarray(), E, ETA, dense.embed_diag(dev.n, idx, sr[0]))
    Lm = dense.embed_diag(dev.n, idx, sl[0])
    Gd = dense.retarded(A)
    Pd = dense.lesser(Gd, Lm)
    G, P = selected_general(A, Lm, cl, z_form)
    _close(G, P, Gd, Pd, _h_pairs(dev))
    for I, U in cl:   # the column blocks too
        if not len(U):
            continue
        assert np.abs(G[np.ix_(U, I)] - Gd[np.ix_(U, I)]).max() <= 1e-11 * np.abs(Gd).max()
        assert np.abs(P[np.ix_(U, I)] - Pd[np.ix_(U, I)]).max() <= 1e-11 * np.abs(Pd).max()
    Gs, _ = selected(A, Lm, cl)
    assert np.abs(np.diag(Gs) - np.diag(Gd)).max() > 1e-3 * np.abs(np.diag(Gd)).max()
