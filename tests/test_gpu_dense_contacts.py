"""GPU parity of hsc_solve_dense: DENSE contact self-energy blocks (Section 3.1.2) from semi-infinite
leads that continue the device's cross-section (Sigma^r = tau g_s tau^T, oracle/lead.py), added to the
fronts of the contact clusters (chained on top of the dissection of the remaining sites).

* A disordered 8 x 6 x 5 device with lead blocks on both end planes: diag G^r, diag G^< and the
  x = 3/4 coupling blocks against the RGF sweep with the same dense first/last-layer blocks, at
  eta = 0.05 (1e-10), with the left lead filled and the right one empty.
* A perfect wire (6 x 4 x 3, no disorder) between two such leads: the transmission read from the
  GPU's G^< block on the right face, T = Tr[Gamma_R (-i G^<_RR)], equals the number of open
  transverse channels (closed-form cross-section energies) up to O(eta).
"""
import numpy as np
import pytest

from oracle import dense, lead, rgf
from paper_1702_05167_gb300 import hsc, workloads as W
from treecheck import _handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hsc.load()


def _dense_handle(dev, leaf):
    h = _handle(dev)
    hsc.hsc_set_contact_dense(h, 0)
    hsc.hsc_set_contact_dense(h, 1)
    st = hsc.hsc_analyze(h, leaf)
    return h, st


def _blocks(dims, t, E, eta):
    H00, H01 = W.cubic_lead(dims, t=t)
    tau = t * np.eye(H00.shape[0])
    S = [lead.contact_self_energy(e, eta, H00, H01, tau) for e in E]
    return S


def _solve(dev, h, E, eta, S, pairs):
    """hsc_solve_dense with zero diagonal self-energies, the lead blocks on both faces, the left
    lead filled (Sigma^< = i Gamma_L) and the right one empty."""
    nE, n = len(E), dev.n
    ncs = len(dev.contact_unknowns())
    nu = ncs // 2
    zr = np.zeros((nE, ncs), np.complex128)
    dr = np.zeros((nE, 2 * nu * nu), np.complex128)
    dl = np.zeros_like(dr)
    for k in range(nE):
        dr[k, :nu * nu] = S[k].ravel()
        dr[k, nu * nu:] = S[k].ravel()
        dl[k, :nu * nu] = (1j * lead.broadening(S[k])).ravel()
    dgr = np.zeros((nE, n), np.complex128)
    dgl = np.zeros((nE, n), np.complex128)
    pgr = np.zeros((nE, len(pairs)), np.complex128)
    pgl = np.zeros((nE, len(pairs)), np.complex128)
    hsc.hsc_solve_dense(h, np.asarray(E, np.float64), eta, zr, zr.copy(), dr, dl, hsc.HSC_FP64, pairs,
                        dgr, dgl, pgr, pgl)
    return dgr, dgl, pgr, pgl


def test_dense_lead_blocks_match_rgf():
    dims, t, eta = (8, 6, 5), -1.0, 0.05
    dev = W.cubic_device(dims, t=t, W=1.0, seed=9)
    E = np.array([-2.6, -0.45, 1.3])
    S = _blocks(dims, t, E, eta)
    h, st = _dense_handle(dev, 3)
    pairs = W.plane_pairs(dev, 3)
    dgr, dgl, pgr, pgl = _solve(dev, h, E, eta, S, pairs)
    hsc.hsc_destroy(h)
    Ls = dims[1] * dims[2]
    u, v = pairs[:, 0] - 3 * Ls, pairs[:, 1] - 4 * Ls
    rel = lambda x, r: np.abs(x - r).max() / np.abs(r).max()
    for k in range(len(E)):
        Sl = 1j * lead.broadening(S[k])
        out = rgf.sweep(dev.to_scipy(), Ls, E[k], eta, [], [], [], coupling_layers=(3,),
                        dense_r=(S[k], S[k]), dense_l=(Sl, np.zeros_like(Sl)))
        errs = [rel(dgr[k], out["diag_gr"]), rel(dgl[k], out["diag_gl"]),
                rel(pgr[k], out["coupling_gr"][3][u, v]), rel(pgl[k], out["coupling_gl"][3][u, v])]
        print(f"dense leads 8x6x5 E={E[k]:+.2f}: " + " ".join(f"{e:.1e}" for e in errs))
        assert max(errs) <= 1e-10


def test_perfect_wire_transmits_one_per_open_channel_on_the_gpu():
    dims, t, eta = (6, 4, 3), -1.0, 1e-8
    dev = W.cubic_device(dims, t=t, W=0.0, seed=0)
    E = np.array([-4.6, -2.9, -0.35, 0.8, 3.3])
    S = _blocks(dims, t, E, eta)
    right = W.face_sites(dims, dims[0] - 1).astype(np.int32)
    a, b = np.meshgrid(right, right, indexing="ij")
    pairs = np.stack([a.ravel(), b.ravel()], axis=1).astype(np.int32)
    h, st = _dense_handle(dev, 2)
    _, _, _, pgl = _solve(dev, h, E, eta, S, pairs)
    hsc.hsc_destroy(h)
    k = np.arange(1, dims[1] + 1)
    l = np.arange(1, dims[2] + 1)
    em = (2 * t * np.cos(np.pi * k / (dims[1] + 1)))[:, None] + (2 * t * np.cos(np.pi * l / (dims[2] + 1)))[None, :]
    nr = len(right)
    for q in range(len(E)):
        Pr = pgl[q].reshape(nr, nr)
        T = float(np.real(np.trace(lead.broadening(S[q]) @ (-1j * Pr))))
        channels = int((np.abs(E[q] - em) < 2 * abs(t)).sum())
        print(f"perfect wire E={E[q]:+.2f}: T = {T:.9f}, open channels {channels}")
        assert abs(T - channels) <= 2e-6
