"""CPU experiment: accuracy of the FP64 recurrences (hsc_emulator) over several cluster trees of one
cubic device at small eta, against the dense inverse.

    python tests/tree_accuracy.py --n 16 --energies 16 --trees geo:4:0 graph:4:0 geo:2:0 geo:8:0 geo:4:1

A tree is ordering:leaf_max:variant (ordering geo or graph; variant 0..4 = HSC_OPT_TREE_VARIANT).
Prints, per tree, the model flops and the median / max over the energies (linspace(-5.5, 5.5)) of
max_u |G_uu - G_uu(dense)| / max_u |G_uu(dense)|."""
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
    p.add_argument("--energies", type=int, default=16)
    p.add_argument("--eta", type=float, default=1e-6)
    p.add_argument("--trees", nargs="+", default=["geo:4:0", "graph:4:0"])
    a = p.parse_args()
    hsc.load()
    dev = W.cubic_device((a.n, a.n, a.n), seed=0)
    Hd = dev.to_scipy().toarray()
    idx = dev.contact_unknowns()
    sr, sl = W.self_energies(dev, 1)
    trees = {}
    for spec in a.trees:
        order, leaf, var = spec.split(":")
        h = _handle(dev, order == "geo")
        if int(var):
            hsc.hsc_set_option(h, hsc.HSC_OPT_TREE_VARIANT, int(var))
        st = hsc.hsc_analyze(h, int(leaf))
        trees[spec] = (tree(h, st.n_clusters), st.flops_gr + st.flops_gl)
        hsc.hsc_destroy(h)
    err = {spec: [] for spec in a.trees}
    for E in np.linspace(-5.5, 5.5, a.energies):
        A = dense.system_matrix(Hd, E, a.eta, dense.embed_diag(dev.n, idx, sr[0]))
        L = dense.embed_diag(dev.n, idx, sl[0])
        gd = np.diag(np.linalg.inv(A))
        for spec in a.trees:
            G, _ = selected(A, L, trees[spec][0])
            err[spec].append(np.abs(np.diag(G) - gd).max() / np.abs(gd).max())
    for spec in a.trees:
        e = np.array(err[spec])
        print(f"{spec:12s} {trees[spec][1] / 1e9:8.3f} GFLOP  median {np.median(e):.1e}  max {e.max():.1e}"
              f"  above 1e-8: {(e > 1e-8).sum()}  above 1e-4: {(e > 1e-4).sum()}")


if __name__ == "__main__":
    main()
