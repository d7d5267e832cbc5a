"""Pins of the open-boundary (DENSE) contact self-energy oracle: closed form, mode decomposition,
brute force and the channel count of a perfect wire. CPU only."""
import numpy as np
import pytest

from oracle import dense, lead
from paper_1702_05167_gb300 import workloads as W


def _chain_closed_form(E, eta, eps0, t):
    """Semi-infinite chain: t^2 g^2 - (z - eps0) g + 1 = 0; the roots multiply to 1/t^2 > 0, so
    exactly one has Im g < 0 (the retarded one)."""
    z = E + 1j * eta - eps0
    r = np.sqrt(z * z - 4 * t * t + 0j)
    return min([(z - r) / (2 * t * t), (z + r) / (2 * t * t)], key=lambda x: x.imag)


@pytest.mark.parametrize("E", [-2.5, -1.2, 0.0, 0.7, 1.9, 2.6])
def test_semi_infinite_chain_matches_the_closed_form(E):
    eta, eps0, t = 1e-9, 0.1, -1.0
    g = lead.surface_gf(E, eta, np.array([[eps0]]), np.array([[t]]))[0, 0]
    ref = _chain_closed_form(E, eta, eps0, t)
    assert abs(g - ref) <= 1e-10 * abs(ref) and g.imag <= 0


def test_uniform_lead_decomposes_into_transverse_modes():
    """H01 = t I commutes with H00, so the lead is a set of independent chains with onsite energies
    the eigenvalues of H00: g_s = Psi diag(g_chain(E - e_m)) Psi^T. The energies keep >= 0.2 eV
    from every mode's band edge e_m +- 2|t| (the square-root edge amplifies rounding)."""
    H00, H01 = W.cubic_lead((1, 4, 3), t=-1.0)
    e, psi = np.linalg.eigh(H00.real)
    for E in (-4.5, -2.4, -0.7, 0.6, 2.4):
        assert np.abs(np.abs(E - e) - 2.0).min() >= 0.15
        g = lead.surface_gf(E, 1e-9, H00, H01)
        ref = psi @ np.diag([_chain_closed_form(E, 1e-9, em, -1.0) for em in e]) @ psi.T
        assert np.abs(g - ref).max() <= 1e-9 * np.abs(ref).max()
        assert np.abs(g - g.T).max() <= 1e-10 * np.abs(g).max()


def test_surface_block_of_a_long_finite_lead():
    """Brute force: for a two-orbital lead whose inter-layer coupling is not symmetric, the
    surface block of the inverse of a long finite block-tridiagonal stack converges to g_s
    (eta damps the far end exponentially)."""
    rng = np.random.default_rng(5)
    H00 = rng.normal(size=(2, 2))
    H00 = H00 + H00.T
    H01 = rng.normal(size=(2, 2))
    eta, L = 0.05, 600
    for E in (-1.0, 0.3, 2.0):
        g = lead.surface_gf(E, eta, H00, H01)
        A = np.zeros((2 * L, 2 * L), dtype=np.complex128)
        for k in range(L):
            A[2 * k:2 * k + 2, 2 * k:2 * k + 2] = (E + 1j * eta) * np.eye(2) - H00
            if k + 1 < L:
                A[2 * k:2 * k + 2, 2 * k + 2:2 * k + 4] = -H01
                A[2 * k + 2:2 * k + 4, 2 * k:2 * k + 2] = -H01.T
        ref = np.linalg.inv(A)[:2, :2]
        assert np.abs(g - ref).max() <= 1e-9 * np.abs(ref).max()


def test_broadening_is_hermitian_positive():
    H00, H01 = W.cubic_lead((1, 3, 3), t=-1.0)
    for E in (-2.0, 0.5):
        S = lead.contact_self_energy(E, 1e-9, H00, H01, H01)
        G = lead.broadening(S)
        assert np.abs(G - G.conj().T).max() <= 1e-13
        assert np.linalg.eigvalsh(G).min() >= -1e-10


@pytest.mark.parametrize("E", [-4.6, -2.9, -0.35, 0.8, 3.3, 5.1])
def test_perfect_wire_transmits_one_per_open_channel(E):
    """A clean device between two leads that continue it: T(E) = Tr[Gamma_L G Gamma_R G^dagger]
    equals the number of transverse modes m with |E - e_m| < 2|t|, e_m = 2t cos(pi k/(Ny+1)) +
    2t cos(pi l/(Nz+1)) (the cross-section's eigenvalues in closed form)."""
    dims, t, eta = (6, 4, 3), -1.0, 1e-10
    dev = W.cubic_device(dims, t=t, W=0.0, seed=0)
    H = dev.to_scipy().toarray()
    H00, H01 = W.cubic_lead(dims, t=t)
    tau = t * np.eye(H00.shape[0])
    left, right = W.face_sites(dims, 0), W.face_sites(dims, dims[0] - 1)
    S = lead.contact_self_energy(E, eta, H00, H01, tau)
    G = dense.retarded(dense.system_matrix(H, E, eta, lead.embed_blocks(dev.n, [(left, S), (right, S)])))
    gl = lead.broadening(S)
    glr = G[np.ix_(left, right)]
    T = np.trace(gl @ glr @ gl @ glr.conj().T).real
    k = np.arange(1, dims[1] + 1)
    l = np.arange(1, dims[2] + 1)
    em = (2 * t * np.cos(np.pi * k / (dims[1] + 1)))[:, None] + (2 * t * np.cos(np.pi * l / (dims[2] + 1)))[None, :]
    open_channels = int((np.abs(E - em) < 2 * abs(t)).sum())
    assert abs(T - open_channels) <= 1e-6


@pytest.mark.parametrize("E", [-2.7, -0.9, 0.4, 1.8])
def test_rgf_with_dense_contacts_matches_the_dense_definition(E):
    """The RGF sweep with DENSE first/last-layer self-energies (lead surface Green's functions)
    against Eqs. 1-2 written out with the same blocks embedded: diag G^r, diag G^< and the
    coupling blocks of two layer pairs."""
    from oracle import rgf
    dims, t, eta = (5, 3, 4), -1.0, 1e-6
    dev = W.cubic_device(dims, t=t, W=1.0, seed=6)
    Hs = dev.to_scipy()
    H00, H01 = W.cubic_lead(dims, t=t)
    tau = t * np.eye(H00.shape[0])
    S = lead.contact_self_energy(E, eta, H00, H01, tau)
    Sl = 1j * lead.broadening(S)          # left lead filled (f = 1), right lead empty
    Z = np.zeros_like(S)
    Ls = dims[1] * dims[2]
    out = rgf.sweep(Hs, Ls, E, eta, [], [], [], coupling_layers=(1, 3), dense_r=(S, S), dense_l=(Sl, Z))
    left, right = W.face_sites(dims, 0), W.face_sites(dims, dims[0] - 1)
    A = dense.system_matrix(Hs.toarray(), E, eta, lead.embed_blocks(dev.n, [(left, S), (right, S)]))
    G = dense.retarded(A)
    Gl = dense.lesser(G, lead.embed_blocks(dev.n, [(left, Sl)]))
    assert np.abs(out["diag_gr"] - np.diag(G)).max() <= 1e-11 * np.abs(np.diag(G)).max()
    assert np.abs(out["diag_gl"] - np.diag(Gl)).max() <= 1e-11 * np.abs(np.diag(Gl)).max()
    for k in (1, 3):
        a, b = slice(k * Ls, (k + 1) * Ls), slice((k + 1) * Ls, (k + 2) * Ls)
        assert np.abs(out["coupling_gr"][k] - G[a, b]).max() <= 1e-11 * np.abs(G[a, b]).max()
        assert np.abs(out["coupling_gl"][k] - Gl[a, b]).max() <= 1e-11 * np.abs(Gl[a, b]).max()
