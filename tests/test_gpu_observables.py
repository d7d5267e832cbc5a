"""GPU parity of hsc_observables (the per-energy observables of Section 1 that the learned energy
grid is trained on) against the CPU oracle: the density of states from diag G^r, the Caroli
transmission Tr[Gamma_R G^r Gamma_L G^r^dagger] from the dense inverse, and the lesser trace
sum_u Im G^<_uu from the dense G^< (Eq. 2), on 8^3 and 12^3 devices at eta = 0.05 and 1e-6."""
import numpy as np
import pytest

from oracle import dense, observables
from paper_1702_05167_gb300 import hsc, workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no GPU")
    return t


@pytest.mark.parametrize("dims,leaf,eta", [((8, 8, 8), 4, 0.05), ((12, 12, 12), 4, 1e-6)])
def test_observables_match_the_dense_oracle(torch, dims, leaf, eta):
    dev = W.cubic_device(dims, W=1.0, seed=5)
    E = np.array([-2.2, -0.3, 0.8, 3.1])
    sr, sl = W.self_energies(dev, len(E), (1.0, 0.0))
    s = hsc.Solver(dev, leaf)
    dv = torch.device("cuda")
    tE = torch.from_numpy(E).to(dv)
    tsr = torch.from_numpy(sr.view(np.float64)).to(dv)
    tsl = torch.from_numpy(sl.view(np.float64)).to(dv)
    ogr = torch.zeros((len(E), 2 * dev.n), dtype=torch.float64, device=dv)
    ogl = torch.zeros_like(ogr)
    stream = torch.cuda.current_stream().cuda_stream
    hsc.hsc_solve(s.h, tE, eta, tsr, tsl, hsc.HSC_FP64, None, ogr, ogl, None, None, stream=stream,
                  io_on_device=True)
    out = torch.zeros((len(E), 3), dtype=torch.float64, device=dv)
    hsc.hsc_observables(s.h, ogr, ogl, tsr, 1, out, stream=stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    s.close()
    Hd = dev.to_scipy().toarray()
    cid = dev.contact_of_unknown()
    idx = dev.contact_unknowns()
    gamma = -2.0 * sr.imag
    for k in range(len(E)):
        G, Gl = dense.solve(Hd, E[k], eta, idx, sr[k], sl[k])
        left, right = idx[cid == 0], idx[cid == 1]
        ref = [observables.dos(np.diag(G)),
               observables.transmission_caroli(G, left, gamma[k][cid == 0], right, gamma[k][cid == 1]),
               float(np.sum(np.imag(np.diag(Gl))))]
        for q in range(3):
            assert abs(got[k, q] - ref[q]) <= TOL * max(abs(ref[q]), 1e-300) + 1e-13, (k, q, got[k, q], ref[q])
