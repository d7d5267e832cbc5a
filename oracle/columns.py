"""Single columns of G^r by sparse direct solves, complex128. Test infrastructure only.

For a sampled unknown a, the column G^r e_a solves A x = e_a with A = (E + i eta) I - H - Sigma^r
(Eq. 1). Because A is complex symmetric (H = H^T, diagonal Sigma^r), G^r = (G^r)^T, so the same x is
also row a of G^r, and Eq. 2 with a diagonal Sigma^< gives
    G^<_aa = sum_c G^r_ac Sigma^<_cc conj(G^r_ac).
This reaches any sampled diagonal entry at full problem size, one unknown at a time. The sparse LU
(SuperLU through scipy) is a library primitive used as-is.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def system_matrix(H, E, eta, contact_idx, sigma_r_vals):
    """Sparse A = (E + i eta) I - H - Sigma^r (Eq. 1)."""
    n = H.shape[0]
    d = np.full(n, E + 1j * eta, dtype=np.complex128)
    np.subtract.at(d, np.asarray(contact_idx, dtype=np.int64), np.asarray(sigma_r_vals))
    return (sp.diags(d) - H.astype(np.complex128)).tocsc()


def sampled(H, E, eta, contact_idx, sigma_r_vals, sigma_less_vals, rows, pairs=()):
    """G^r_aa and G^<_aa for a in rows, plus G^r_ab for (a, b) in pairs, at one energy.

    Returns (gr[len(rows)], gl[len(rows)], gr_pairs[len(pairs)]).
    """
    A = system_matrix(H, E, eta, contact_idx, sigma_r_vals)
    lu = spla.splu(A, permc_spec="MMD_AT_PLUS_A")
    rows = np.asarray(rows, dtype=np.int64)
    contact_idx = np.asarray(contact_idx, dtype=np.int64)
    sl = np.asarray(sigma_less_vals, dtype=np.complex128)
    n = A.shape[0]
    gr = np.empty(len(rows), dtype=np.complex128)
    gl = np.empty(len(rows), dtype=np.complex128)
    for k, a in enumerate(rows):
        e = np.zeros(n, dtype=np.complex128)
        e[a] = 1.0
        x = lu.solve(e)
        gr[k] = x[a]
        xc = x[contact_idx]
        gl[k] = np.sum(xc * sl * xc.conj())
    gp = np.empty(len(pairs), dtype=np.complex128)
    for k, (a, b) in enumerate(pairs):
        e = np.zeros(n, dtype=np.complex128)
        e[b] = 1.0
        gp[k] = lu.solve(e)[a]
    return gr, gl, gp
