"""Pins of the SCBA oracle (local elastic dephasing around Eqs. 1-2): closed forms of a single
site, the current balance that the fixed point enforces, and the d0 = 0 reduction. CPU only."""
import numpy as np
import pytest

from oracle import dense, scba
from paper_1702_05167_gb300 import workloads as W


@pytest.mark.parametrize("E,eps,d0", [(0.3, 0.0, 0.05), (-0.7, 0.2, 0.3), (1.9, -0.4, 1.0),
                                      (0.0, 0.0, 2.5)])
def test_single_site_matches_the_closed_form(E, eps, d0):
    eta, gamma, f = 1e-6, 0.5, 1.0
    out = scba.scba(np.array([[eps]]), [E], eta, [0], np.array([[-0.5j * gamma]]),
                    np.array([[1j * f * gamma]]), d0, 0.5, 1e-14, 5000)
    g, gl = scba.single_site(E, eta, eps, gamma, f, d0)
    assert out["delta"] <= 1e-14
    assert abs(out["gr"][0, 0] - g) <= 1e-12 * abs(g)
    assert abs(out["gl"][0, 0] - gl) <= 1e-12 * abs(gl)
    assert g.imag < 0 and gl.imag > 0


def test_closed_form_is_the_fixed_point():
    """The closed-form roots satisfy the defining equations themselves (checks single_site)."""
    E, eta, eps, gamma, f, d0 = 0.4, 1e-6, 0.1, 0.5, 1.0, 0.7
    g, gl = scba.single_site(E, eta, eps, gamma, f, d0)
    z = E + 1j * eta - eps + 0.5j * gamma
    assert abs(g - 1.0 / (z - d0 * g)) <= 1e-14
    assert abs(gl - abs(g) ** 2 * (1j * f * gamma + d0 * gl)) <= 1e-14


def _small():
    dev = W.cubic_device((4, 3, 3), seed=3)
    H = dev.to_scipy().toarray()
    idx = dev.contact_unknowns()
    cid = dev.contact_of_unknown()
    E = np.array([-1.3, 0.2, 2.1])
    sr, sl = W.self_energies(dev, len(E))
    return dev, H, idx, cid, E, sr, sl


def test_zero_dephasing_is_the_plain_solve():
    dev, H, idx, cid, E, sr, sl = _small()
    out = scba.scba(H, E, 1e-6, idx, sr, sl, 0.0, 0.5, 1e-12, 50)
    assert out["iters"] == 1
    for e in range(len(E)):
        G, Gl = dense.solve(H, E[e], 1e-6, idx, sr[e], sl[e])
        assert np.array_equal(out["gr"][e], np.diag(G)) and np.array_equal(out["gl"][e], np.diag(Gl))


def test_fixed_point_conserves_current():
    """Every terminal current balances for any scattering self-energy (a trace identity); at the
    fixed point the scattering self-energy takes in and gives back the same current at every
    unknown, so the contacts' currents balance with the eta leak alone. Two iterations in, the
    scattering currents are still far from zero (the check discriminates)."""
    dev, H, idx, cid, E, sr, sl = _small()
    gam = dev.gamma[cid]
    f = np.array([1.0, 0.0])[cid]
    eta = 1e-6
    for iters, tol in ((2, 0.0), (400, 1e-13)):
        out = scba.scba(H, E, eta, idx, sr, sl, 0.2, 0.6, tol, iters)
        cur = scba.currents(out["gr"], out["gl"], out["sr"], out["sl"], idx, gam, f, eta)
        i_l = cur["contact"][:, cid == 0].sum(axis=1)
        i_r = cur["contact"][:, cid == 1].sum(axis=1)
        total = i_l + i_r + cur["scatt"].sum(axis=1) + cur["eta"]
        assert np.all(np.abs(total) <= 1e-12 * np.abs(i_l))
        assert np.all(i_l > 0) and np.all(i_r < 0)
        worst = np.abs(cur["scatt"]).max(axis=1) / np.abs(i_l)
        if iters == 2:
            assert worst.min() > 1e-3
        else:
            assert out["delta"] <= 1e-13 and out["iters"] < 400
            assert worst.max() <= 1e-10
            assert np.all(np.abs(i_l + i_r + cur["eta"]) <= 1e-10 * np.abs(i_l))


def test_dephasing_makes_a_clean_chain_ohmic():
    """A clean chain is ballistic (T = 1 inside the band, whatever its length); with dephasing its
    resistance 1/I_L grows linearly with the length, the textbook signature of the model."""
    d0, eta, E = 0.05, 1e-9, 0.0
    res = []
    Ns = [8, 16, 24, 32]
    for N in Ns:
        dev = W.chain_device(N, gamma=2.0)     # gamma = 2|t|: reflectionless leads at E = 0
        H = dev.to_scipy().toarray()
        idx = dev.contact_unknowns()
        cid = dev.contact_of_unknown()
        sr, sl = W.self_energies(dev, 1)
        out = scba.scba(H, [E], eta, idx, sr, sl, d0, 0.7, 1e-13, 2000)
        cur = scba.currents(out["gr"], out["gl"], out["sr"], out["sl"], idx, dev.gamma[cid],
                            np.array([1.0, 0.0])[cid], eta)
        res.append(1.0 / cur["contact"][0, cid == 0].sum())
        clean = scba.scba(H, [E], eta, idx, sr, sl, 0.0, 0.7, 1e-13, 5)
        cur0 = scba.currents(clean["gr"], clean["gl"], clean["sr"], clean["sl"], idx,
                             dev.gamma[cid], np.array([1.0, 0.0])[cid], eta)
        assert abs(cur0["contact"][0, cid == 0].sum() - 1.0) <= 1e-6
    slope, icpt = np.polyfit(Ns, res, 1)
    fit = slope * np.array(Ns) + icpt
    assert slope > 0 and np.abs(fit - res).max() <= 0.02 * (res[-1] - res[0])
