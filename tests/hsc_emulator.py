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


def selected_general(A, L, clusters, z_form=False):
    """The same two passes for a general (not complex-symmetric) A, e.g. a Hermitian H with Peierls
    phases: the LU form, with a left factor beside the right one and column blocks of G beside the
    row blocks. Upward, per cluster: D^{-1}; X = D^{-1} A_iU; Y = A_Ui D^{-1}; S_UU -= A_Ui X; and
    the lesser fold L_UU += Y L_ii Y^dagger - Y L_iU - L_Ui Y^dagger (the congruence by the
    elimination [[I, 0], [-Y, I]], which keeps G^< = A^{-1} L A^{-dagger} on the reduced system).
    Downward: G_iU = -X G_UU, G_Ui = -G_UU Y, G_ii = D^{-1} - X G_Ui; N_i. = L_i. (G^dagger)_.
    restricted to i and U; P_iU = D^{-1} N_iU - X P_UU, P_ii = D^{-1} N_ii - X P_Ui with
    P_Ui = -P_iU^dagger. For a symmetric A, Y = X^T and this is `selected`. (With L anti-Hermitian
    the fold equals Z - Z^dagger, Z = Y (L_ii Y^dagger / 2 - L_iU): `selected`'s form with Y for
    X^T; written out term by term unless z_form.)"""
    Aw, Lw = A.astype(np.complex128).copy(), L.astype(np.complex128).copy()
    fac = []
    for I, U in clusters:
        Dinv = np.linalg.inv(Aw[np.ix_(I, I)])
        X = Dinv @ Aw[np.ix_(I, U)]
        Y = Aw[np.ix_(U, I)] @ Dinv
        Lii, LiU, LUi = Lw[np.ix_(I, I)].copy(), Lw[np.ix_(I, U)].copy(), Lw[np.ix_(U, I)].copy()
        if len(U):
            Aw[np.ix_(U, U)] -= Aw[np.ix_(U, I)] @ X
            if z_form:
                Z = Y @ (0.5 * Lii @ Y.conj().T - LiU)
                Lw[np.ix_(U, U)] += Z - Z.conj().T
            else:
                Lw[np.ix_(U, U)] += Y @ Lii @ Y.conj().T - Y @ LiU - LUi @ Y.conj().T
        fac.append((Dinv, X, Y, Lii, LiU))
    n = A.shape[0]
    G = np.zeros((n, n), np.complex128)
    P = np.zeros((n, n), np.complex128)
    for (I, U), (Dinv, X, Y, Lii, LiU) in reversed(list(zip(clusters, fac))):
        Guu, Puu = G[np.ix_(U, U)], P[np.ix_(U, U)]
        GiU, GUi = -X @ Guu, -Guu @ Y
        Gii = Dinv - X @ GUi
        N_ii = Lii @ Gii.conj().T + LiU @ GiU.conj().T
        N_iU = Lii @ GUi.conj().T + LiU @ Guu.conj().T
        PiU = Dinv @ N_iU - X @ Puu
        Pii = Dinv @ N_ii + X @ PiU.conj().T
        G[np.ix_(I, I)], G[np.ix_(I, U)], G[np.ix_(U, I)] = Gii, GiU, GUi
        P[np.ix_(I, I)], P[np.ix_(I, U)], P[np.ix_(U, I)] = Pii, PiU, -PiU.conj().T
    return G, P
