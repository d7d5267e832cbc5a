"""Open-boundary (DENSE) contact self-energies, complex128. Test infrastructure only.

Section 3.1.2 replaces the diagonal contact self-energy by a dense block on the contact layer to
model open boundaries, without saying how the block is obtained. The reading here: the contact is
a semi-infinite lead that continues the device's cross-section, with layer Hamiltonian H00 and
coupling H01 from one lead layer to the next one further out; the device layer couples to the
lead's surface layer through tau. With transposes throughout (H complex symmetric, Eq. 3):

    Sigma^r = tau g_s tau^T,    g_s = (z - H00 - H01 g_s H01^T)^{-1},   z = E + i eta,

g_s being the surface Green's function of the lead. It is computed by the decimation of Lopez Sancho,
Lopez Sancho and Rubio (J. Phys. F 15, 851, 1985): every step eliminates every other layer of the
remaining chain, so the effective couplings shrink doubly exponentially once eta damps them.
The broadening is Gamma = i (Sigma^r - Sigma^r^dagger) and the lesser self-energy i f Gamma.

What pins it: the semi-infinite chain's closed form; the mode decomposition of a uniform lead into
independent chains; the surface block of a long finite lead inverted by brute force; and the
integer channel count of a perfect wire (tests/test_lead_oracle.py).
"""
import numpy as np


def surface_gf(E, eta, H00, H01, tol=1e-14, max_iter=200):
    """Retarded surface Green's function of a semi-infinite lead (Lopez Sancho-Rubio decimation).

    H00: layer Hamiltonian (complex symmetric); H01: coupling from a layer to the next one outward;
    the coupling back is H01^T. Raises if the couplings have not vanished after max_iter steps.
    """
    H00 = np.asarray(H00, dtype=np.complex128)
    H01 = np.asarray(H01, dtype=np.complex128)
    n = H00.shape[0]
    zI = (E + 1j * eta) * np.eye(n, dtype=np.complex128)
    eps_s = H00.copy()      # renormalised surface layer
    eps = H00.copy()        # renormalised bulk layer
    fwd = H01.copy()        # effective coupling outward
    back = H01.T.copy()     # effective coupling inward
    scale = 1.0 + np.abs(H01).max()
    for _ in range(max_iter):
        g = np.linalg.inv(zI - eps)
        fgb = fwd @ g @ back
        eps_s = eps_s + fgb
        eps = eps + fgb + back @ g @ fwd
        fwd = fwd @ g @ fwd
        back = back @ g @ back
        if max(np.abs(fwd).max(), np.abs(back).max()) <= tol * scale:
            return np.linalg.inv(zI - eps_s)
    raise RuntimeError("decimation did not converge (eta too small for max_iter?)")


def contact_self_energy(E, eta, H00, H01, tau):
    """Sigma^r = tau g_s tau^T on the device's contact layer (Section 3.1.2, DENSE self-energy)."""
    tau = np.asarray(tau, dtype=np.complex128)
    return tau @ surface_gf(E, eta, H00, H01) @ tau.T


def broadening(sigma_r):
    """Gamma = i (Sigma^r - Sigma^r^dagger), Hermitian positive semi-definite."""
    return 1j * (sigma_r - sigma_r.conj().T)


def embed_blocks(n, blocks):
    """Dense n x n matrix with each (unknown index list, block) of `blocks` added on its rows and
    columns: the dense self-energy of every contact layer placed in the device's numbering."""
    S = np.zeros((n, n), dtype=np.complex128)
    for idx, B in blocks:
        idx = np.asarray(idx, dtype=np.int64)
        S[np.ix_(idx, idx)] += B
    return S
