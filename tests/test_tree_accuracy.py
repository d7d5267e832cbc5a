"""Accuracy of the cluster trees at small eta, on the CPU: the library's own trees (hsc_analyze) run
through the FP64 recurrences it implements (tests/hsc_emulator.py, numpy) against the dense
definition of Eqs. 1-2. The plain geometric tree has interior clusters whose blocks carry only eta;
one with a level close to E costs the downward step of Eq. 4 digits in proportion to
||D_i^{-1}||^2. The default contact-connected tree (x cut once, at the root) keeps a share of a
contact face in every cluster below the root and does not lose them."""
import numpy as np

from hsc_emulator import selected, tree
from oracle import dense
from paper_1702_05167_gb300 import hsc, workloads as W
from treecheck import _handle


def _errors(dev, leaf, ordering, energies, eta=1e-6):
    h = _handle(dev)
    hsc.hsc_set_option(h, hsc.HSC_OPT_ORDERING, ordering)
    st = hsc.hsc_analyze(h, leaf)
    form = hsc.hsc_get_option(h, hsc.HSC_OPT_TREE_FORM)
    cl = tree(h, st.n_clusters)
    hsc.hsc_destroy(h)
    sr, sl = W.self_energies(dev, 1)
    idx = dev.contact_unknowns()
    Hd = dev.to_scipy().toarray()
    out, growth = [], []
    for E in energies:
        A = dense.system_matrix(Hd, E, eta, dense.embed_diag(dev.n, idx, sr[0]))
        L = dense.embed_diag(dev.n, idx, sl[0])
        G = dense.retarded(A)
        gd, pd = np.diag(G), np.diag(dense.lesser(G, L))
        stats = {}
        Gs, Ps = selected(A, L, cl, stats)
        out.append(max(np.abs(np.diag(Gs) - gd).max() / np.abs(gd).max(),
                       np.abs(np.diag(Ps) - pd).max() / np.abs(pd).max()))
        growth.append(stats["growth"])
    return form, np.array(out)


def test_contact_connected_tree_keeps_the_digits_the_plain_tree_loses():
    """12^3 cube, leaves 3, eta = 1e-6: at E = -1.1 an interior cluster of the plain tree has a level
    close to E and diag G^r / G^< lose ~3e-3; the contact-connected tree stays within 1e-10 at
    every energy checked."""
    dev = W.cubic_device((12, 12, 12), seed=0)
    E = np.array([-1.1, -3.3, 0.45, 2.7])
    form_p, ep = _errors(dev, 3, 2, E)
    form_c, ec = _errors(dev, 3, 0, E)
    assert (form_p, form_c) == (0, 1)
    assert ep[0] > 1e-4, ep
    assert ec.max() <= 1e-10, ec
