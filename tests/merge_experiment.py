"""CPU experiment: re-solve by merging, into their parents, the clusters whose D_i^{-1} shows growth
far above the median (the delayed-pivot idea at cluster granularity), on the library's own tree at
small eta; errors of diag G^r against the dense inverse before and after, and the model-flop ratio.

    python tests/merge_experiment.py --n 16 --leaf 2 --energies 16 [--leaves-only]
"""
import argparse
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from hsc_emulator import selected, update_sets    # noqa: E402
from oracle import dense                          # noqa: E402
from paper_1702_05167_gb300 import hsc, workloads as W   # noqa: E402
from treecheck import _handle                     # noqa: E402


def flops(cl):
    return sum(8 * (len(o) ** 2 * (len(o) + len(u)) + 2 * len(o) * len(u) ** 2 + len(o) ** 2 * len(u))
               for o, u in cl)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=16)
    p.add_argument("--leaf", type=int, default=2)
    p.add_argument("--energies", type=int, default=16)
    p.add_argument("--eta", type=float, default=1e-6)
    p.add_argument("--factor", type=float, default=30.0, help="merge where growth > factor x median")
    p.add_argument("--leaves-only", action="store_true")
    a = p.parse_args()
    hsc.load()
    dev = W.cubic_device((a.n, a.n, a.n), seed=0)
    Hs = dev.to_scipy()
    Hd = Hs.toarray()
    idx = dev.contact_unknowns()
    sr, sl = W.self_energies(dev, 1)
    h = _handle(dev, True)
    st = hsc.hsc_analyze(h, a.leaf)
    infos = [hsc.hsc_cluster(h, i) for i in range(st.n_clusters)]
    hsc.hsc_destroy(h)
    owns = [np.asarray(o, np.int64) for _, o, _ in infos]
    parent = [inf.parent for inf, _, _ in infos]
    leaf = [inf.child[0] < 0 and inf.child[1] < 0 for inf, _, _ in infos]
    base = [(o, np.asarray(u, np.int64)) for (_, o, u), o in zip(infos, owns)]
    for E in np.linspace(-5.5, 5.5, a.energies):
        A = dense.system_matrix(Hd, E, a.eta, dense.embed_diag(dev.n, idx, sr[0]))
        L = dense.embed_diag(dev.n, idx, sl[0])
        gd = np.diag(np.linalg.inv(A))
        stats = {}
        G, _ = selected(A, L, base, stats)
        e0 = np.abs(np.diag(G) - gd).max() / np.abs(gd).max()
        if e0 < 1e-8:
            continue
        g = np.array(stats["cluster_growth"])
        flag = [i for i in range(len(owns)) if g[i] > a.factor * np.median(g) and parent[i] >= 0
                and (leaf[i] or not a.leaves_only)]
        target = list(range(len(owns)))
        for i in flag:
            target[i] = parent[i]

        def root(i):
            while target[i] != i:
                i = target[i]
            return i
        groups = {}
        for i in range(len(owns)):
            groups.setdefault(root(i), []).append(i)
        merged = update_sets([np.concatenate([owns[j] for j in sorted(groups[k])]) for k in sorted(groups)], Hs)
        G2, _ = selected(A, L, merged)
        e1 = np.abs(np.diag(G2) - gd).max() / np.abs(gd).max()
        print(f"E {E:+.2f}: error {e0:.1e} (growth {g.max():.0e}) -> {len(flag)} clusters merged: {e1:.1e}"
              f"  (model flops x{flops(merged) / flops(base):.2f})")


if __name__ == "__main__":
    main()
