"""Writes tests/golden/tiny_8x8x8.txt from the dense oracle (Eq. 1-2) on the seeded 8x8x8 workload.

The paper prints no worked numerical example, so this fixture is not a paper value: it freezes the
oracle's own output (and the seeded generator feeding it) so that an accidental change to either is
caught. Run from the repository root: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import dense  # noqa: E402
from paper_1702_05167_gb300 import workloads as W  # noqa: E402


def compute():
    cfg = W.tiny()
    dev = cfg["dev"]
    sr, sl = W.self_energies(dev, 1, cfg["f"])
    G, Gl = dense.solve(dev.to_scipy().toarray(), cfg["energies"][0], cfg["eta"],
                        dev.contact_unknowns(), sr[0], sl[0])
    return np.diag(G), np.diag(Gl)


if __name__ == "__main__":
    gr, gl = compute()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_8x8x8.txt")
    with open(out, "w") as f:
        f.write("# 8x8x8 workload (workloads.tiny): E = 0.3 eV, eta = 1e-6, leaves <= 4\n")
        f.write("# columns: unknown, Re G^r_uu, Im G^r_uu, Re G^<_uu, Im G^<_uu (dense oracle)\n")
        for u in range(len(gr)):
            f.write(f"{u} {gr[u].real:.17e} {gr[u].imag:.17e} {gl[u].real:.17e} {gl[u].imag:.17e}\n")
    print("wrote", out)
