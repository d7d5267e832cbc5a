"""Host logic of the learned energy grid, on the CPU with an analytic stand-in for the surrogate:
grid placement by equal quantiles of the trapezoid error density, the disorder features and the
trapezoid integrals."""
import numpy as np
import pytest

from paper_1702_05167_gb300 import learned as LG, workloads as W


class _Analytic:
    """predict() in the surrogate's output layout: columns (log10 T, DOS) at the rows' energies."""

    def __init__(self, T, D):
        self.T, self.D = T, D

    def predict(self, X):
        E = X[:, 0]
        return np.column_stack([np.log10(self.T(E)), self.D(E)])


FEATS = np.zeros(LG.N_FEATURES)


def test_flat_spectra_give_the_uniform_grid():
    """With constant T and DOS the error density is the floor alone: equal quantiles of a
    constant are the uniform grid, endpoints included."""
    sur = _Analytic(lambda E: 0.5 + 0.0 * E, lambda E: 1.0 + 0.0 * E)
    E = LG.adaptive_grid(sur, FEATS, 33, fine=4097, window=(-2.0, 2.0))
    assert np.allclose(E, np.linspace(-2.0, 2.0, 33), atol=1e-9)


def test_linear_spectra_stay_nearly_uniform():
    """A linear DOS and transmission have no curvature; their discrete second derivatives are
    rounding noise, which the range-based normalisation keeps small (normalised by their own mean,
    the noise would be scaled to O(1) and placed as structure)."""
    sur = _Analytic(lambda E: 0.3 + 0.1 * (E + 2.0), lambda E: 1.0 + 0.25 * E)
    E = LG.adaptive_grid(sur, FEATS, 33, fine=4097, window=(-2.0, 2.0))
    assert np.abs(E - np.linspace(-2.0, 2.0, 33)).max() <= 0.02 * (4.0 / 32)


def test_points_equidistribute_the_density_and_crowd_at_a_resonance():
    """A Lorentzian transmission peak: consecutive points enclose equal integrals of
    rho = |T''|^(1/3)/mean + |D''|^(1/3)/mean + floor, so they crowd where T bends."""
    g, e0 = 0.05, 0.3
    sur = _Analytic(lambda E: g * g / ((E - e0) ** 2 + g * g) + 1e-3, lambda E: 1.0 + 0.0 * E)
    n, fine, win = 65, 16385, (-3.0, 3.0)
    E = LG.adaptive_grid(sur, FEATS, n, fine=fine, window=win)
    assert len(E) == n and E[0] == win[0] and E[-1] == win[1] and np.all(np.diff(E) > 0)
    Ef = np.linspace(win[0], win[1], fine)
    h = Ef[1] - Ef[0]
    T = sur.T(Ef)
    a = np.abs(np.gradient(np.gradient(T, h), h)) ** (1 / 3)
    rho = a / max(a.mean(), (np.ptp(T) / 36.0) ** (1 / 3)) + 1.0   # the DOS is flat: its term vanishes
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (rho[1:] + rho[:-1]) * h)])
    mass = np.diff(np.interp(E, Ef, cdf))
    assert np.abs(mass / mass.mean() - 1.0).max() <= 1e-6
    near = np.abs(E - e0) < 3 * g
    assert np.diff(E)[near[:-1] & near[1:]].max() < 0.5 * (win[1] - win[0]) / (n - 1)


def test_features_of_a_clean_device_and_their_scaling():
    """Constant onsite energy c: the mean is c and every central moment vanishes. Scaling the
    onsite energies by s scales every feature by s (k-th roots of k-th moments are homogeneous of
    degree one, signs kept)."""
    dev = W.cubic_device((5, 4, 3), W=0.0, seed=0)
    f0 = LG.disorder_features(dev)
    assert f0.shape == (LG.N_FEATURES,) and np.allclose(f0, 0.0, atol=1e-15)
    dev1 = W.cubic_device((5, 4, 3), W=1.0, seed=3)
    dev2 = W.cubic_device((5, 4, 3), W=2.0, seed=3)
    f1, f2 = LG.disorder_features(dev1), LG.disorder_features(dev2)
    assert np.allclose(f2, 2.0 * f1, rtol=1e-12, atol=1e-15)
    assert f1[1] > 0 and f1[8] > 0


@pytest.mark.parametrize("k", [0, 1])
def test_trapezoid_integrals_are_exact_for_linear_integrands(k):
    E = np.sort(np.random.default_rng(k).uniform(-1.0, 2.0, 40))
    lin = 3.0 * E - 0.5
    got = LG.integrals(E, lin, lin, lin)
    exact = 1.5 * (E[-1] ** 2 - E[0] ** 2) - 0.5 * (E[-1] - E[0])
    assert abs(got["int_DOS_dE"] - exact) <= 1e-12 * abs(exact)
    assert abs(got["current_int_T_dE"] - exact) <= 1e-12 * abs(exact)
    assert abs(got["electrons_int_ImGless_dE_over_2pi"] - exact / (2 * np.pi)) <= 1e-12 * abs(exact)
