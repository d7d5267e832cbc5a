"""Self-consistent local elastic dephasing around Eqs. 1-2, complex128. Test infrastructure only.

Section 1 splits Sigma^r of Eq. 1 into a contact part and a part for scattering mechanisms, but the
paper fixes no scattering model. The model written out here is local elastic dephasing in the
self-consistent Born approximation: a delta-correlated scattering potential of strength d0 (eV^2)
gives, on every unknown u,

    Sigma^r_scatt,uu = d0 G^r_uu,        Sigma^<_scatt,uu = d0 G^<_uu = i d0 Im G^<_uu,

with G^r and G^< from Eqs. 1-2 evaluated with Sigma = Sigma_contact + Sigma_scatt. G^< is
anti-Hermitian when Sigma^< is (Algorithm 2 relies on it: its downward pass sets the transposed
block to minus the adjoint), so its diagonal is purely imaginary and the lesser self-energy keeps
only that part: a real part would be rounding (or conditioning) error with no physical meaning, fed
back as a Hermitian component that the selected-inversion recurrences do not carry. The fixed point
is reached by linear mixing, all energies together:

    S_0 = 0;  solve with Sigma_contact + S_k  ->  G_k;
    F_k = (d0 diag G^r_k, i d0 Im diag G^<_k);
    delta_k = max |F_k - S_k| / max |F_k|   (over energies, unknowns, retarded and lesser; 0 if F = 0);
    stop when delta_k <= tol or after max_iter solves, else S_{k+1} = S_k + mix (F_k - S_k).

What pins it (no worked example in the paper): a single site has closed forms for both fixed points
(a quadratic for G^r, a linear equation for G^<); at the fixed point every unknown exchanges no
current with the scattering self-energy, so the contact currents balance up to the eta leak; with
d0 = 0 the loop is the plain solve of ``dense``.
"""
import numpy as np

from . import dense


def scba(H, energies, eta, contact_idx, sigma_r_vals, sigma_less_vals, d0, mix, tol, max_iter):
    """Dense SCBA loop with local elastic dephasing (Section 1, Eq. 1 scattering self-energy).

    H: dense n x n; energies: [n_E]; contact_idx: unknowns of the contact self-energies;
    sigma_r_vals, sigma_less_vals: [n_E, len(contact_idx)] contact parts.
    Returns dict(gr, gl: [n_E, n] diagonals of the last solve; iters: solves made; delta: the last
    delta_k; sr, sl: [n_E, n] the scattering self-energies that last solve used).
    """
    H = np.asarray(H, dtype=np.complex128)
    n = H.shape[0]
    energies = np.asarray(energies, dtype=np.float64)
    n_E = len(energies)
    s_r = np.zeros((n_E, n), dtype=np.complex128)
    s_l = np.zeros((n_E, n), dtype=np.complex128)
    for k in range(max_iter):
        gr = np.empty((n_E, n), dtype=np.complex128)
        gl = np.empty((n_E, n), dtype=np.complex128)
        for e, E in enumerate(energies):
            sig_r = dense.embed_diag(n, contact_idx, sigma_r_vals[e]) + np.diag(s_r[e])
            sig_l = dense.embed_diag(n, contact_idx, sigma_less_vals[e]) + np.diag(s_l[e])
            G = dense.retarded(dense.system_matrix(H, E, eta, sig_r))
            gr[e] = np.diag(G)
            gl[e] = np.diag(dense.lesser(G, sig_l))
        f_r, f_l = d0 * gr, 1j * d0 * gl.imag
        diff = max(np.abs(f_r - s_r).max(), np.abs(f_l - s_l).max())
        scale = max(np.abs(f_r).max(), np.abs(f_l).max())
        delta = diff / scale if scale > 0 else 0.0
        if delta <= tol or k == max_iter - 1:
            return dict(gr=gr, gl=gl, iters=k + 1, delta=delta, sr=s_r, sl=s_l)
        s_r = s_r + mix * (f_r - s_r)
        s_l = s_l + mix * (f_l - s_l)
    raise ValueError("max_iter must be >= 1")


def single_site(E, eta, eps, gamma, f, d0):
    """Closed-form fixed point of one site (onsite eps, one contact of broadening gamma filled to f).

    G^r = 1 / (z - d0 G^r) with z = E + i eta - eps + i gamma/2, i.e. d0 G^2 - z G + 1 = 0: the two
    roots multiply to 1/d0 > 0, so exactly one has Im G < 0 (the retarded one). G^< = |G|^2 (i f gamma
    + d0 G^<) gives G^< = i f gamma |G|^2 / (1 - d0 |G|^2).
    """
    z = E + 1j * eta - eps + 0.5j * gamma
    if d0 == 0:
        g = 1.0 / z
    else:
        r = np.sqrt(z * z - 4.0 * d0 + 0j)
        roots = [(z - r) / (2.0 * d0), (z + r) / (2.0 * d0)]
        g = min(roots, key=lambda x: x.imag)
    gl = 1j * f * gamma * abs(g) ** 2 / (1.0 - d0 * abs(g) ** 2)
    return g, gl


def currents(gr, gl, sr, sl, contact_idx, gamma, f, eta):
    """Currents into the device per energy (Section 1 observables, diagonal self-energies).

    With A = -2 Im G^r_uu (spectral function), Gn = Im G^<_uu (G^< = i Gn on the diagonal) and, for a
    diagonal self-energy, broadening Gamma_u = -2 Im Sigma^r_uu and in-scattering Im Sigma^<_uu, the
    current a terminal injects through unknown u is (in-scattering) A_uu - Gamma_u Gn_uu.
    gamma, f: per entry of contact_idx. Returns dict with 'contact' [n_E, len(contact_idx)] (per
    contact unknown; sum the entries of one contact for its current),
    'scatt' [n_E, n] (per unknown, into the scattering self-energy sr / sl), 'eta' [n_E] (the leak
    of the i eta term, broadening 2 eta, no in-scattering). The three sum to zero for any sr, sl.
    """
    A = -2.0 * gr.imag
    gn = gl.imag
    idx = np.asarray(contact_idx, dtype=np.int64)
    g = np.asarray(gamma, dtype=np.float64)
    fc = np.asarray(f, dtype=np.float64)
    i_c = g[None, :] * (fc[None, :] * A[:, idx] - gn[:, idx])
    i_s = sl.imag * A - (-2.0 * sr.imag) * gn
    i_eta = -2.0 * eta * gn.sum(axis=1)
    return dict(contact=i_c, scatt=i_s, eta=i_eta)
