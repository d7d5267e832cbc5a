"""Recursive Green's function (RGF) sweep for block-tridiagonal A, complex128. Test infrastructure only.

This is the paper's comparison method (Section 2.1): the unknowns are grouped into layers orthogonal
to the transport direction, ordered one layer at a time, so that A(E) = (E + i eta) I - H - Sigma^r is
block tridiagonal.

* First pass (left to right, the "fold" of Section 2.1): the block LDL^T factorisation of Eq. 3,
  D_1 = A_11, D_n = A_nn - A_{n,n-1} D_{n-1}^{-1} A_{n-1,n}; gL_n = D_n^{-1} is the left-connected
  Green's function.
* Second pass (right to left, the "extract"): Eq. 4, G = (I - L^T) G + D^{-1} L^{-1}, read block by
  block: G_NN = gL_N, G_{n,n+1} = -gL_n A_{n,n+1} G_{n+1,n+1},
  G_{n+1,n} = -G_{n+1,n+1} A_{n+1,n} gL_n, G_nn = gL_n - gL_n A_{n,n+1} G_{n+1,n}.
* G^< (Eq. 2, G^< = G^r Sigma^< G^r^dagger) with Sigma^< non-zero only in the first and last layers
  (the contacts) needs only the first and last block columns of G^r:
  G^<_{ab} = G_{a,1} Sigma^<_1 G_{b,1}^dagger + G_{a,N} Sigma^<_N G_{b,N}^dagger.
  G_{n,N} follows from the extract relation of Eq. 4 (G_{n,N} = -gL_n A_{n,n+1} G_{n+1,N}), and
  G_{n,1} from the mirror-image sweep (right-connected gR_n, G_{n,1} = -gR_n A_{n,n-1} G_{n-1,1}).

Outputs: diag G^r, diag G^<, and for requested layer indices n the coupling blocks G^r_{n,n+1} and
G^<_{n,n+1} (all in the layer-ordered unknown numbering).
"""
import numpy as np


def layer_blocks(H, layer_size):
    """Split a block-tridiagonal sparse H (scipy CSR, n = N*layer_size) into dense blocks.

    Returns (Hd, Hu, Hl): lists of diagonal blocks H_nn, upper blocks H_{n,n+1}, lower H_{n+1,n}.
    Raises ValueError if H couples non-adjacent layers.
    """
    n = H.shape[0]
    if n % layer_size:
        raise ValueError("n is not a multiple of the layer size")
    N = n // layer_size
    coo = H.tocoo()
    if np.any(np.abs(coo.row // layer_size - coo.col // layer_size) > 1):
        raise ValueError("H is not block tridiagonal in the given layering")
    Hd, Hu, Hl = [], [], []
    for k in range(N):
        s = slice(k * layer_size, (k + 1) * layer_size)
        Hd.append(H[s, s].toarray().astype(np.complex128))
        if k + 1 < N:
            t = slice((k + 1) * layer_size, (k + 2) * layer_size)
            Hu.append(H[s, t].toarray().astype(np.complex128))
            Hl.append(H[t, s].toarray().astype(np.complex128))
    return Hd, Hu, Hl


def sweep(H, layer_size, E, eta, contact_idx, sigma_r_vals, sigma_less_vals, coupling_layers=(),
          dense_r=None, dense_l=None):
    """Selected G^r and G^< at one energy by RGF (Section 2.1, Eqs. 3-4 and Eq. 2).

    H: scipy sparse n x n; contact_idx/sigma_*_vals: diagonal self-energies (they must lie in the
    first and last layers); coupling_layers: layer indices n for which G_{n,n+1} blocks are returned.
    dense_r, dense_l: optional (first-layer block, last-layer block) of a DENSE Sigma^r / Sigma^<
    (Section 3.1.2), layer-local numbering, added to the diagonal ones; they need two layers or more.
    Returns dict(diag_gr, diag_gl, coupling_gr={n: block}, coupling_gl={n: block}).
    """
    n = H.shape[0]
    Ls = layer_size
    N = n // Ls
    contact_idx = np.asarray(contact_idx, dtype=np.int64)
    lay = contact_idx // Ls
    if np.any((lay != 0) & (lay != N - 1)):
        raise ValueError("contacts must lie in the first or last layer")
    sr = np.zeros(n, dtype=np.complex128)
    sl = np.zeros(n, dtype=np.complex128)
    np.add.at(sr, contact_idx, sigma_r_vals)
    np.add.at(sl, contact_idx, sigma_less_vals)

    Hd, Hu, Hl = layer_blocks(H, Ls)
    eye = np.eye(Ls, dtype=np.complex128)
    z = E + 1j * eta
    # A blocks (Eq. 1): A_nn = z I - H_nn - Sigma^r_n, A_{n,n+1} = -H_{n,n+1}, A_{n+1,n} = -H_{n+1,n}
    Ad = [z * eye - Hd[k] - np.diag(sr[k * Ls:(k + 1) * Ls]) for k in range(N)]
    if (dense_r is not None or dense_l is not None) and N < 2:
        raise ValueError("dense contact blocks need at least two layers")
    if dense_r is not None:
        Ad[0] = Ad[0] - dense_r[0]
        Ad[N - 1] = Ad[N - 1] - dense_r[1]
    Au = [-h for h in Hu]
    Al = [-h for h in Hl]

    # first pass, left to right: D_n (Eq. 3) and gL_n = D_n^{-1}
    gL = [None] * N
    gL[0] = np.linalg.inv(Ad[0])
    for k in range(1, N):
        gL[k] = np.linalg.inv(Ad[k] - Al[k - 1] @ gL[k - 1] @ Au[k - 1])
    # mirror sweep, right to left: right-connected gR_n (needed for the first block column)
    gR = [None] * N
    gR[N - 1] = np.linalg.inv(Ad[N - 1])
    for k in range(N - 2, -1, -1):
        gR[k] = np.linalg.inv(Ad[k] - Au[k] @ gR[k + 1] @ Al[k])

    # second pass, right to left (Eq. 4)
    diag_gr = np.empty(n, dtype=np.complex128)
    Gnn = [None] * N
    Gnn[N - 1] = gL[N - 1]
    coupling_gr = {}
    for k in range(N - 2, -1, -1):
        Gk_k1 = -gL[k] @ Au[k] @ Gnn[k + 1]          # G_{n,n+1}
        Gk1_k = -Gnn[k + 1] @ Al[k] @ gL[k]          # G_{n+1,n}
        Gnn[k] = gL[k] - gL[k] @ Au[k] @ Gk1_k       # G_nn
        if k in coupling_layers:
            coupling_gr[k] = Gk_k1
    for k in range(N):
        diag_gr[k * Ls:(k + 1) * Ls] = np.diag(Gnn[k])

    # block columns 1 and N of G^r (Eq. 4 and its mirror image), then G^< (Eq. 2)
    s1 = sl[:Ls]
    sN = sl[(N - 1) * Ls:]
    colN = [None] * N
    colN[N - 1] = Gnn[N - 1]
    for k in range(N - 2, -1, -1):
        colN[k] = -gL[k] @ Au[k] @ colN[k + 1]
    col1 = [None] * N
    col1[0] = Gnn[0]
    for k in range(1, N):
        col1[k] = -gR[k] @ Al[k - 1] @ col1[k - 1]
    diag_gl = np.empty(n, dtype=np.complex128)
    coupling_gl = {}
    if dense_l is None:
        for k in range(N):
            a, b = col1[k], colN[k]
            diag_gl[k * Ls:(k + 1) * Ls] = ((np.abs(a) ** 2) @ s1) + ((np.abs(b) ** 2) @ sN) \
                if N > 1 else (np.abs(a) ** 2) @ s1
        for k in coupling_layers:
            coupling_gl[k] = (col1[k] * s1) @ col1[k + 1].conj().T + (colN[k] * sN) @ colN[k + 1].conj().T
    else:   # Sigma^<_1, Sigma^<_N full blocks: G^<_ab = G_a1 S_1 G_b1^dagger + G_aN S_N G_bN^dagger
        S1 = np.diag(s1) + dense_l[0]
        SN = np.diag(sN) + dense_l[1]
        for k in range(N):
            a, b = col1[k], colN[k]
            diag_gl[k * Ls:(k + 1) * Ls] = np.einsum("ij,jk,ik->i", a, S1, a.conj()) + \
                np.einsum("ij,jk,ik->i", b, SN, b.conj())
        for k in coupling_layers:
            coupling_gl[k] = col1[k] @ S1 @ col1[k + 1].conj().T + colN[k] @ SN @ colN[k + 1].conj().T
    return dict(diag_gr=diag_gr, diag_gl=diag_gl, coupling_gr=coupling_gr, coupling_gl=coupling_gl)
