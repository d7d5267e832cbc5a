"""Observables from Green's functions (Section 1, the quantities NEGF evaluates). Test infrastructure.

With A = (E + i eta) I - H - Sigma^r, Gamma_c = i (Sigma^r_c - Sigma^r_c^dagger) and
Sigma^< = i sum_c f_c Gamma_c:
* density of states   DOS(E) = -(1/pi) sum_n Im G^r_nn;
* transmission        T(E) = Tr[Gamma_R G^r Gamma_L G^r^dagger]   (Caroli form, from the full G^r);
  with f_L = 1, f_R = 0 this equals sum_{m in R} Gamma_m Im G^<_mm (from the diagonal of G^<).
"""
import numpy as np


def dos(diag_gr):
    return -np.sum(np.imag(diag_gr)) / np.pi


def transmission_caroli(G, left_idx, gamma_left, right_idx, gamma_right):
    """Tr[Gamma_R G Gamma_L G^dagger] from a dense G^r and diagonal broadenings."""
    Grl = G[np.ix_(right_idx, left_idx)]
    return float(np.real(np.sum((gamma_right[:, None] * Grl) * (Grl.conj() * gamma_left[None, :]))))


def transmission_from_lesser(diag_gl, right_idx, gamma_right):
    """sum_{m in R} Gamma_m Im G^<_mm, valid for f_L = 1 and f_R = 0."""
    return float(np.sum(gamma_right * np.imag(diag_gl[right_idx])))
