"""Pins for the CPU oracle: each check ties it to something other than itself.

* open-chain spectral sum (eigenvectors sqrt(2/(N+1)) sin(k i pi/(N+1))) -- pins Eq. 1's signs;
* Usmani's continuant formula for the inverse of a tridiagonal matrix -- pins Eq. 1 with
  self-energies and disorder, and the RGF sweep of Section 2.1 at layer size 1;
* the optical-theorem sum rule at eta = 0, -2 Im G^r = G^r Gamma G^r^dagger, and Im G^< = G Gamma G^dagger
  for f = 1 everywhere -- pins Eq. 2 (placement of Sigma^< and of the adjoint);
* complex symmetry G^r = (G^r)^T and anti-Hermiticity of G^< (the relations used by Algorithms 1-2);
* Caroli transmission against the lesser-function form, and against |G_1N|^2 Gamma^2 on a chain;
* RGF against the dense definition on small 3D grids (including several orbitals per site);
* sparse single-column solves against the dense definition;
* the density of states of a closed chain against its sum of Lorentzians over the closed-form
  eigenvalues.
"""
import numpy as np
import pytest

from oracle import dense, rgf, columns, observables
from paper_1702_05167_gb300 import workloads as W


def _dense_H(dev):
    return dev.to_scipy().toarray()


def _solve_dense(dev, E, eta, f=(1.0, 0.0)):
    sr, sl = W.self_energies(dev, 1, f)
    return dense.solve(_dense_H(dev), E, eta, dev.contact_unknowns(), sr[0], sl[0])


# ---- closed forms for the 1D chain ---------------------------------------------------------

def usmani_inverse(a, b):
    """Inverse of the symmetric tridiagonal matrix with diagonal a and constant off-diagonal b,
    by Usmani's continuants: theta_0 = 1, theta_1 = a_1, theta_k = a_k theta_{k-1} - b^2 theta_{k-2};
    phi_{N+1} = 1, phi_N = a_N, phi_k = a_k phi_{k+1} - b^2 phi_{k+2};
    T^{-1}_ij = (-b)^{j-i} theta_{i-1} phi_{j+1} / theta_N for i <= j (1-based)."""
    N = len(a)
    th = np.zeros(N + 1, dtype=complex)
    th[0] = 1.0
    th[1] = a[0]
    for k in range(2, N + 1):
        th[k] = a[k - 1] * th[k - 1] - b * b * th[k - 2]
    ph = np.zeros(N + 2, dtype=complex)
    ph[N + 1] = 1.0
    ph[N] = a[N - 1]
    for k in range(N - 1, 0, -1):
        ph[k] = a[k - 1] * ph[k + 1] - b * b * ph[k + 2]
    G = np.zeros((N, N), dtype=complex)
    for i in range(1, N + 1):
        for j in range(i, N + 1):
            G[i - 1, j - 1] = (-b) ** (j - i) * th[i - 1] * ph[j + 1] / th[N]
            G[j - 1, i - 1] = G[i - 1, j - 1]
    return G


def test_open_chain_spectral_sum():
    """Clean open chain (no contacts): G = sum_k psi_k psi_k^T / (z - 2 t cos(k pi/(N+1)))."""
    N, t, E, eta = 11, -1.0, 0.37, 0.05
    dev = W.chain_device(N, t=t, gamma=0.0)
    G, _ = _solve_dense(dev, E, eta)
    k = np.arange(1, N + 1)
    i = np.arange(1, N + 1)
    psi = np.sqrt(2.0 / (N + 1)) * np.sin(np.outer(i, k) * np.pi / (N + 1))   # [site, mode]
    ek = 2 * t * np.cos(k * np.pi / (N + 1))
    Gs = (psi / (E + 1j * eta - ek)) @ psi.T
    np.testing.assert_allclose(G, Gs, rtol=0, atol=1e-13 * np.abs(Gs).max())


@pytest.mark.parametrize("seed", [0, 1])
def test_chain_usmani_dense_and_rgf(seed):
    """Disordered chain with wide-band end contacts: dense and RGF against Usmani's formula."""
    rng = np.random.default_rng(seed)
    N, t, gam, E, eta = 17, -1.0, 0.5, 0.3, 1e-6
    eps = rng.uniform(-0.5, 0.5, N)
    dev = W.chain_device(N, t=t, eps=eps, gamma=gam)
    a = (E + 1j * eta) - eps.astype(complex)
    a[0] += 0.5j * gam        # -Sigma^r = +i Gamma/2 on the end sites
    a[-1] += 0.5j * gam
    Gu = usmani_inverse(a, -t)
    G, Gl = _solve_dense(dev, E, eta)
    np.testing.assert_allclose(G, Gu, rtol=0, atol=1e-12 * np.abs(Gu).max())
    # transmission of a chain: T = Gamma_L Gamma_R |G_1N|^2
    T_closed = gam * gam * abs(Gu[0, -1]) ** 2
    T_dense = observables.transmission_from_lesser(np.diag(Gl), np.array([N - 1]), np.array([gam]))
    assert abs(T_dense - T_closed) <= 1e-12 * max(1.0, T_closed)
    # RGF with one site per layer is a scalar recursion; compare with the closed form too
    sr, sl = W.self_energies(dev, 1)
    out = rgf.sweep(dev.to_scipy(), 1, E, eta, dev.contact_unknowns(), sr[0], sl[0],
                    coupling_layers=(3, 8))
    np.testing.assert_allclose(out["diag_gr"], np.diag(Gu), rtol=1e-11)
    assert abs(out["coupling_gr"][3][0, 0] - Gu[3, 4]) <= 1e-11 * abs(Gu[3, 4])
    gl_closed = 1j * gam * np.abs(Gu[:, 0]) ** 2      # f_L = 1, f_R = 0
    np.testing.assert_allclose(out["diag_gl"], gl_closed, rtol=1e-10, atol=1e-14)


def test_sum_rule_eta_zero():
    """At eta = 0: -2 Im diag G^r = diag(G Gamma G^dagger); with f = 1 on every contact,
    Im diag G^< = -2 Im diag G^r as well (Eq. 2)."""
    dev = W.cubic_device((4, 3, 3), W=1.0, seed=3, gamma=0.7)
    G, Gl = _solve_dense(dev, E=0.41, eta=0.0, f=(1.0, 1.0))
    n = dev.n
    Gam = np.zeros(n)
    Gam[dev.contact_unknowns()] = dev.gamma[dev.contact_of_unknown()]
    lhs = -2 * np.imag(np.diag(G))
    rhs = np.real(np.diag((G * Gam) @ G.conj().T))
    np.testing.assert_allclose(lhs, rhs, rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(np.imag(np.diag(Gl)), lhs, rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(np.real(np.diag(Gl)), 0, atol=1e-12)


def test_symmetry_and_positivity():
    dev = W.cubic_device((5, 4, 3), W=1.0, seed=7)
    G, Gl = _solve_dense(dev, E=-0.2, eta=1e-6)
    np.testing.assert_allclose(G, G.T, atol=1e-12 * np.abs(G).max())
    np.testing.assert_allclose(Gl, -Gl.conj().T, atol=1e-12 * np.abs(Gl).max())
    assert np.all(-np.imag(np.diag(G)) > 0)
    assert np.all(np.imag(np.diag(Gl)) >= -1e-14)


def test_caroli_equals_lesser_transmission():
    dev = W.cubic_device((6, 3, 4), W=1.0, seed=2)
    G, Gl = _solve_dense(dev, E=0.3, eta=1e-6)
    cu = dev.contact_unknowns()
    cid = dev.contact_of_unknown()
    L, R = cu[cid == 0], cu[cid == 1]
    gL = np.full(len(L), dev.gamma[0])
    gR = np.full(len(R), dev.gamma[1])
    T1 = observables.transmission_caroli(G, L, gL, R, gR)
    T2 = observables.transmission_from_lesser(np.diag(Gl), R, gR)
    assert abs(T1 - T2) <= 1e-10 * max(T1, 1e-300)
    assert 0 <= T1 <= len(L) + 1e-9      # at most one per open channel


@pytest.mark.parametrize("dims,orb", [((6, 3, 4), 1), ((5, 2, 3), 3)])
def test_rgf_matches_dense(dims, orb):
    """RGF sweep (Section 2.1) against the dense definition: diag G^r, diag G^<, coupling blocks."""
    dev = W.cubic_device(dims, W=1.0, seed=5) if orb == 1 else W.wire_device(dims, orb=orb, seed=5)
    E, eta = 0.25, 1e-6
    G, Gl = _solve_dense(dev, E, eta)
    sr, sl = W.self_energies(dev, 1)
    Ls = dims[1] * dims[2] * orb
    out = rgf.sweep(dev.to_scipy(), Ls, E, eta, dev.contact_unknowns(), sr[0], sl[0],
                    coupling_layers=(0, dims[0] // 2))
    sc = np.abs(np.diag(G)).max()
    np.testing.assert_allclose(out["diag_gr"], np.diag(G), rtol=0, atol=1e-11 * sc)
    np.testing.assert_allclose(out["diag_gl"], np.diag(Gl), rtol=0, atol=1e-11 * np.abs(np.diag(Gl)).max())
    for k in (0, dims[0] // 2):
        s, t = slice(k * Ls, (k + 1) * Ls), slice((k + 1) * Ls, (k + 2) * Ls)
        np.testing.assert_allclose(out["coupling_gr"][k], G[s, t], atol=1e-11 * sc)
        np.testing.assert_allclose(out["coupling_gl"][k], Gl[s, t], atol=1e-11 * np.abs(Gl).max())


def test_sparse_columns_match_dense():
    dev = W.cubic_device((5, 4, 4), W=1.0, seed=9)
    E, eta = -1.1, 1e-6
    G, Gl = _solve_dense(dev, E, eta)
    sr, sl = W.self_energies(dev, 1)
    rows = np.array([0, 7, 33, 79])
    pairs = [(16, 32), (40, 41)]
    gr, gl, gp = columns.sampled(dev.to_scipy(), E, eta, dev.contact_unknowns(), sr[0], sl[0],
                                 rows, pairs)
    np.testing.assert_allclose(gr, np.diag(G)[rows], rtol=1e-11)
    np.testing.assert_allclose(gl, np.diag(Gl)[rows], rtol=1e-10, atol=1e-15)
    np.testing.assert_allclose(gp, [G[a, b] for a, b in pairs], rtol=1e-11)


def test_oracle_detects_planted_mistakes():
    """A transposed (not adjoint) G^< or a flipped Sigma^r sign fails the pins above."""
    dev = W.cubic_device((4, 3, 3), W=1.0, seed=3, gamma=0.7)
    Hd = _dense_H(dev)
    cu = dev.contact_unknowns()
    sr, sl = W.self_energies(dev, 1, (1.0, 1.0))
    A = dense.system_matrix(Hd, 0.41, 0.0, dense.embed_diag(dev.n, cu, sr[0]))
    G = dense.retarded(A)
    wrong = G @ dense.embed_diag(dev.n, cu, sl[0]) @ G.T        # transpose instead of adjoint
    lhs = -2 * np.imag(np.diag(G))
    assert np.max(np.abs(np.imag(np.diag(wrong)) - lhs)) > 1e-3
    A2 = dense.system_matrix(Hd, 0.41, 0.0, dense.embed_diag(dev.n, cu, -sr[0]))   # sign flip
    G2 = dense.retarded(A2)
    Gam = np.zeros(dev.n)
    Gam[cu] = 0.7
    rhs2 = np.real(np.diag((G2 * Gam) @ G2.conj().T))
    assert np.max(np.abs(-2 * np.imag(np.diag(G2)) - rhs2)) > 1e-3


def test_dos_is_the_lorentzian_sum_of_the_closed_chain():
    """DOS(E) = -(1/pi) sum_n Im G^r_nn of a closed chain (no contacts, hopping t) equals
    (1/pi) sum_k eta / ((E - e_k)^2 + eta^2) with the closed-form levels e_k = 2 t cos(k pi / (N + 1)):
    pins observables.dos (sign, 1/pi, imaginary part) independently of any inverse routine."""
    N, t, eta = 17, -1.0, 0.07
    H = t * (np.eye(N, k=1) + np.eye(N, k=-1))
    ek = 2 * t * np.cos(np.arange(1, N + 1) * np.pi / (N + 1))
    for E in (-1.3, 0.0, 0.55, 1.9):
        G = dense.retarded(dense.system_matrix(H, E, eta, np.zeros((N, N))))
        ref = np.sum(eta / ((E - ek) ** 2 + eta ** 2)) / np.pi
        assert abs(observables.dos(np.diag(G)) - ref) <= 1e-12 * ref
        assert abs(-np.sum(np.real(np.diag(G))) / np.pi - ref) > 1e-3 * ref   # the real part would not do
