"""Pins of the oracle for a general Hermitian H (the "next" row of non-symmetric H, e.g. a magnetic
field): gauge invariance of the diagonals, two-terminal reciprocity, RGF = dense. CPU only."""
import numpy as np
import pytest

from oracle import dense, observables, rgf
from paper_1702_05167_gb300 import workloads as W

DIMS, ETA = (6, 4, 3), 1e-6


def _solve(dev, E):
    H = dev.to_scipy().toarray()
    sr, sl = W.self_energies(dev, 1)
    return dense.solve(H, E, ETA, dev.contact_unknowns(), sr[0], sl[0])


def test_the_magnetic_device_is_hermitian_and_not_symmetric():
    H = W.magnetic_cubic_device(DIMS, 0.13, seed=2).to_scipy().toarray()
    assert np.abs(H - H.conj().T).max() == 0.0
    assert np.abs(H - H.T).max() > 0.1


@pytest.mark.parametrize("E", [-2.2, 0.35, 1.7])
def test_diagonals_are_gauge_invariant(E):
    """A gauge transformation H -> U H U^dagger, U = diag(exp(i theta_s)), changes no diagonal of
    G^r or G^< when the self-energies are diagonal; an oracle that took a transpose where Eq. 2
    has an adjoint would break it."""
    dev = W.magnetic_cubic_device(DIMS, 0.13, seed=2)
    th = np.random.default_rng(3).uniform(0, 2 * np.pi, dev.n)
    U = np.exp(1j * th)
    Hs = dev.to_scipy()
    Hg = Hs.multiply(U[:, None]).multiply(U.conj()[None, :]).tocsr()
    Hg.sort_indices()
    dev_g = W.Device(dims=dev.dims, orb=1, rowptr=Hg.indptr.astype(np.int64), col=Hg.indices.astype(np.int32),
                     val=Hg.data.astype(np.complex128), contact_ptr=dev.contact_ptr,
                     contact_sites=dev.contact_sites, gamma=dev.gamma)
    G, Gl = _solve(dev, E)
    Gg, Glg = _solve(dev_g, E)
    assert np.abs(np.diag(Gg) - np.diag(G)).max() <= 1e-12 * np.abs(np.diag(G)).max()
    assert np.abs(np.diag(Glg) - np.diag(Gl)).max() <= 1e-12 * np.abs(np.diag(Gl)).max()


@pytest.mark.parametrize("E", [-1.9, 0.6])
def test_transmission_obeys_onsager_reciprocity(E):
    """H(-phi) = H(phi)^T, so G(-phi) = G(phi)^T and T_{L->R}(phi) = T_{R->L}(-phi) exactly, at any
    eta. The two-terminal T(phi) = T(-phi) holds only up to the eta absorption (a third terminal,
    O(eta |G|^2)); the field does change T."""
    T = {}
    for phi in (0.0, 0.13, -0.13):
        dev = W.magnetic_cubic_device(DIMS, phi, seed=2)
        cu, cid = dev.contact_unknowns(), dev.contact_of_unknown()
        L, R = cu[cid == 0], cu[cid == 1]
        gL, gR = np.full(len(L), dev.gamma[0]), np.full(len(R), dev.gamma[1])
        G, _ = _solve(dev, E)
        T[phi] = (observables.transmission_caroli(G, L, gL, R, gR),     # L -> R
                  observables.transmission_caroli(G, R, gR, L, gL))     # R -> L
    assert abs(T[0.13][0] - T[-0.13][1]) <= 1e-12 * T[0.13][0]
    assert abs(T[0.13][0] - T[-0.13][0]) <= 1e-5 * T[0.13][0]
    assert abs(T[0.13][0] - T[0.0][0]) > 1e-3 * T[0.0][0]


@pytest.mark.parametrize("E", [-2.4, 0.9])
def test_rgf_matches_the_dense_definition_for_hermitian_h(E):
    dev = W.magnetic_cubic_device(DIMS, 0.21, seed=4)
    Hs = dev.to_scipy()
    sr, sl = W.self_energies(dev, 1)
    Ls = DIMS[1] * DIMS[2]
    out = rgf.sweep(Hs, Ls, E, ETA, dev.contact_unknowns(), sr[0], sl[0], coupling_layers=(2,))
    G, Gl = _solve(dev, E)
    assert np.abs(out["diag_gr"] - np.diag(G)).max() <= 1e-11 * np.abs(np.diag(G)).max()
    assert np.abs(out["diag_gl"] - np.diag(Gl)).max() <= 1e-11 * np.abs(np.diag(Gl)).max()
    a, b = slice(2 * Ls, 3 * Ls), slice(3 * Ls, 4 * Ls)
    assert np.abs(out["coupling_gr"][2] - G[a, b]).max() <= 1e-11 * np.abs(G[a, b]).max()
    assert np.abs(out["coupling_gl"][2] - Gl[a, b]).max() <= 1e-11 * np.abs(Gl[a, b]).max()
