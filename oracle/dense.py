"""Dense definition of G^r and G^< (Eq. 1 and Eq. 2), complex128. Test infrastructure only.

A(E) = (E + i eta) I - H - Sigma^r            (Eq. 1; eta is the usual positive infinitesimal)
G^r  = A^{-1}                                 (Eq. 1)
G^<  = G^r Sigma^< (G^r)^dagger               (Eq. 2)

Sigma^r and Sigma^< are diagonal here (the "SPARSE" self-energy of Section 3.1.1): they are given as
values on a list of unknowns and embedded into an n x n diagonal matrix.
"""
import numpy as np


def embed_diag(n, idx, vals):
    """Diagonal n x n matrix with vals on the unknowns idx (Section 3.1.1, SPARSE self-energy)."""
    d = np.zeros(n, dtype=np.complex128)
    np.add.at(d, np.asarray(idx, dtype=np.int64), np.asarray(vals, dtype=np.complex128))
    return np.diag(d)


def system_matrix(H, E, eta, sigma_r):
    """A = (E + i eta) I - H - Sigma^r (Eq. 1). H and sigma_r are dense n x n arrays."""
    H = np.asarray(H, dtype=np.complex128)
    n = H.shape[0]
    return (E + 1j * eta) * np.eye(n, dtype=np.complex128) - H - sigma_r


def retarded(A):
    """G^r = A^{-1} (Eq. 1), by LAPACK (LU with partial pivoting)."""
    return np.linalg.inv(A)


def lesser(G, sigma_less):
    """G^< = G^r Sigma^< (G^r)^dagger (Eq. 2)."""
    return G @ sigma_less @ G.conj().T


def solve(H, E, eta, contact_idx, sigma_r_vals, sigma_less_vals):
    """Full G^r and G^< at one energy for diagonal contact self-energies (Eqs. 1-2).

    H: dense n x n; contact_idx: unknowns carrying self-energy; sigma_*_vals: values on them.
    Returns (G, Gl) as dense complex128 n x n matrices.
    """
    H = np.asarray(H, dtype=np.complex128)
    n = H.shape[0]
    A = system_matrix(H, E, eta, embed_diag(n, contact_idx, sigma_r_vals))
    G = retarded(A)
    Gl = lesser(G, embed_diag(n, contact_idx, sigma_less_vals))
    return G, Gl
