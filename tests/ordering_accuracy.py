"""CPU experiment: accuracy of the FP64 recurrences (hsc_emulator) over the geometric and the graph
nested-dissection trees at eta = 1e-6, against the dense inverse, on a cubic device.

    python tests/ordering_accuracy.py --n 16 --leaf 4 --energies 16

Prints, per ordering, the model flops and the median / max of max_u |G_uu - G_uu(dense)| /
max_u |G_uu(dense)| over the energies (linspace(-5.5, 5.5))."""
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
    p.add_argument("--leaf", type=int, default=4)
    p.add_argument("--energies", type=int, default=16)
    p.add_argument("--eta", type=float, default=1e-6)
    a = p.parse_args()
    hsc.load()
    dev = W.cubic_device((a.n, a.n, a.n), seed=0)
    Hd = dev.to_scipy().toarray()
    idx = dev.contact_unknowns()
    sr, sl = W.self_energies(dev, 1)
    trees, flops = {}, {}
    for geo in (True, False):
        h = _handle(dev, geo)
        st = hsc.hsc_analyze(h, a.leaf)
        trees[geo], flops[geo] = tree(h, st.n_clusters), st.flops_gr + st.flops_gl
        hsc.hsc_destroy(h)
    err = {True: [], False: []}
    for E in np.linspace(-5.5, 5.5, a.energies):
        A = dense.system_matrix(Hd, E, a.eta, dense.embed_diag(dev.n, idx, sr[0]))
        L = dense.embed_diag(dev.n, idx, sl[0])
        gd = np.diag(np.linalg.inv(A))
        for geo in (True, False):
            G, _ = selected(A, L, trees[geo])
            err[geo].append(np.abs(np.diag(G) - gd).max() / np.abs(gd).max())
    for geo in (True, False):
        e = np.array(err[geo])
        print(f"{'geometric' if geo else 'graph':9s} {flops[geo] / 1e9:8.3f} GFLOP  median {np.median(e):.1e}"
              f"  max {e.max():.1e}  above 1e-8: {(e > 1e-8).sum()}  above 1e-4: {(e > 1e-4).sum()}")


if __name__ == "__main__":
    main()
