"""CPU experiment: per energy, the diag G^r error of the FP64 recurrences (hsc_emulator) over the
library's own tree at small eta against the dense inverse, next to the two a-posteriori signals the
library records: the residual max_u |(A G^r - I)_uu| (hsc_residual) and the growth max |D_i^{-1}|
(hsc_growth).

    python tests/error_predictors.py --n 16 --leaf 2 --energies 16
"""
import argparse
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from hsc_emulator import selected, tree          # noqa: E402
from oracle import dense                          # noqa: E402
from paper_1702_05167_gb300 import hsc, workloads as W   # noqa: E402
from treecheck import _handle                     # noqa: E402


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=16)
    p.add_argument("--leaf", type=int, default=2)
    p.add_argument("--energies", type=int, default=16)
    p.add_argument("--eta", type=float, default=1e-6)
    a = p.parse_args()
    hsc.load()
    dev = W.cubic_device((a.n, a.n, a.n), seed=0)
    Hs = dev.to_scipy()
    Hd = Hs.toarray()
    idx = dev.contact_unknowns()
    sr, sl = W.self_energies(dev, 1)
    h = _handle(dev, True)
    st = hsc.hsc_analyze(h, a.leaf)
    cl = tree(h, st.n_clusters)
    hsc.hsc_destroy(h)
    coo = Hs.tocoo()
    off = coo.row != coo.col
    rr, cc = coo.row[off], coo.col[off]
    print("      E     error  residual    growth  residual*growth^2")
    for E in np.linspace(-5.5, 5.5, a.energies):
        A = dense.system_matrix(Hd, E, a.eta, dense.embed_diag(dev.n, idx, sr[0]))
        L = dense.embed_diag(dev.n, idx, sl[0])
        gd = np.diag(np.linalg.inv(A))
        stats = {}
        G, _ = selected(A, L, cl, stats)
        err = np.abs(np.diag(G) - gd).max() / np.abs(gd).max()
        r = np.diag(A) * np.diag(G) - 1.0
        np.add.at(r, rr, A[rr, cc] * G[cc, rr])
        res, g = np.abs(r).max(), stats["growth"]
        print(f"{E:+7.2f}  {err:8.1e}  {res:8.1e}  {g:8.1e}  {res * g * g:8.1e}")


if __name__ == "__main__":
    main()
