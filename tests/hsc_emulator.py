"""Test helper: the selected-inversion recurrences that the library implements (Algorithm 1, and
Algorithm 2 with the lesser front folded from both sides), written in numpy over a cluster tree
read back from the library's analysis (hsc_cluster). Full dense work arrays, read and written only
on the blocks the recurrences name. It checks the analysis plus the recurrences on the CPU (for
instance with DENSE contact blocks); it is not the oracle and makes no parity claim for the GPU."""
import numpy as np

from paper_1702_05167_gb300 import hsc


def tree(h, n_clusters):
    """(own unknowns in local order, update set) of every cluster, in postorder."""
    out = []
    for i in range(n_clusters):
        info, own, upd = hsc.hsc_cluster(h, i)
        out.append((np.asarray(own, np.int64), np.asarray(upd, np.int64)))
    return out


def selected(A, L, clusters, stats=None):
    """Upward elimination in postorder, then downward selected inversion root first.

    A: dense complex-symmetric system matrix; L: dense anti-Hermitian Sigma^<; clusters: list of
    (own unknowns in local order, update set U_i) in postorder. Returns dense G, P holding the
    selected blocks of G^r and G^< (zeros elsewhere). If stats is a dict, stats["growth"] receives
    the largest |Re| + |Im| of any D_i^{-1} entry (what hsc_growth records) and
    stats["cluster_growth"] that value per cluster.
    """
    Aw, Lw = A.astype(np.complex128).copy(), L.astype(np.complex128).copy()
    fac = []
    for I, U in clusters:
        Dinv = np.linalg.inv(Aw[np.ix_(I, I)])
        if stats is not None:
            g = float((np.abs(Dinv.real) + np.abs(Dinv.imag)).max()) if Dinv.size else 0.0
            stats["growth"] = max(stats.get("growth", 0.0), g)
            stats.setdefault("cluster_growth", []).append(g)
        X = Dinv @ Aw[np.ix_(I, U)]
        Lii, LiU = Lw[np.ix_(I, I)].copy(), Lw[np.ix_(I, U)].copy()
        if len(U):
            Aw[np.ix_(U, U)] -= Aw[np.ix_(I, U)].T @ X                  # S_i += -A_iU^T X
            T = 0.5 * Lii @ X.conj() - LiU                               # lesser fold
            Z = X.T @ T
            Lw[np.ix_(U, U)] += Z - Z.conj().T
        fac.append((Dinv, X, Lii, LiU))
    n = A.shape[0]
    G = np.zeros((n, n), np.complex128)
    P = np.zeros((n, n), np.complex128)
    for (I, U), (Dinv, X, Lii, LiU) in reversed(list(zip(clusters, fac))):
        Guu, Puu = G[np.ix_(U, U)], P[np.ix_(U, U)]
        GiU = -X @ Guu
        Gii = Dinv - X @ GiU.T
        N_ii = Lii @ Gii.conj() + LiU @ GiU.T.conj()
        N_iU = Lii @ GiU.conj() + LiU @ Guu.conj()
        W_ii, W_iU = Dinv @ N_ii, Dinv @ N_iU
        PiU = W_iU - X @ Puu
        Pii = W_ii + X @ PiU.conj().T
        G[np.ix_(I, I)], G[np.ix_(I, U)], G[np.ix_(U, I)] = Gii, GiU, GiU.T
        P[np.ix_(I, I)], P[np.ix_(I, U)], P[np.ix_(U, I)] = Pii, PiU, -PiU.conj().T
    return G, P


def update_sets(owns, H):
    """Exact update sets for clusters given as own-unknown lists in elimination order (children
    before parents), by symbolic elimination: a cluster absorbs the pending boundary of every earlier
    cluster that reaches it. For trees the analysis does not build (merged clusters)."""
    n = H.shape[0]
    owner = np.empty(n, int)
    for i, o in enumerate(owns):
        owner[o] = i
    coo = H.tocoo()
    adj = [set() for _ in range(n)]
    for a, b in zip(coo.row, coo.col):
        if a != b:
            adj[a].add(b)
    reach, taken = [], [False] * len(owns)
    for i, own in enumerate(owns):
        dom = set(own.tolist())
        ext = set()
        for u in own:
            ext |= adj[u]
        for j in range(i):
            if not taken[j] and reach[j] & dom:
                taken[j] = True
                ext |= reach[j]
        reach.append({u for u in ext - dom if owner[u] > i})
    return [(np.asarray(own, np.int64), np.array(sorted(r, key=lambda u: (owner[u], u)), dtype=np.int64))
            for own, r in zip(owns, reach)]
