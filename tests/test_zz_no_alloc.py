"""The allocation-free block inversion entry point (hsc_block_inverse_noalloc).

It exists for callers that cannot allocate device memory while they run -- for instance an
application whose memory pool already holds the free device memory, so that a cudaMalloc would
fail, or a latency-bound loop that cannot take cudaMalloc/cudaFree's implicit synchronisation. Its
scratch is a fixed device array shared by all calls, so every check below makes two calls in a row
(the second one runs on the scratch the first one left behind). The results are compared with the
regular entry point (with the whole 4x4x4 device in a single cluster, hsc_solve's requested entries
are the full inverse of A(E)) and with LAPACK's inverse (numpy.linalg.inv) at the documented limits,
at an order that is not a multiple of the 16-wide panel, in place, and on a singular block.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1702_05167_gb300 import hsc, workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    return torch


def _blocks(n, batch, seed):
    """Well-conditioned complex blocks: Ginibre / sqrt(n) + 2.5 I (spectrum in |z - 2.5| <= 1)."""
    rng = np.random.default_rng(seed)
    g = (rng.standard_normal((batch, n, n)) + 1j * rng.standard_normal((batch, n, n))) / np.sqrt(2 * n)
    return g + 2.5 * np.eye(n)[None]


def _invert(torch, A, in_place=False):
    batch, n, _ = A.shape
    tA = torch.from_numpy(A.view(np.float64)).cuda()
    out = tA if in_place else torch.full_like(tA, float("nan"))
    hsc.hsc_block_inverse_noalloc(n, batch, tA, out, stream=torch.cuda.current_stream().cuda_stream)
    return out.cpu().numpy().view(np.complex128).reshape(batch, n, n)


def _rel(got, ref):
    return max(np.abs(got[k] - ref[k]).max() / np.abs(ref[k]).max() for k in range(len(ref)))


def test_noalloc_block_inverse_matches_hsc_solve_twice():
    torch = _torch()
    dev = W.cubic_device((4, 4, 4), W=1.0, seed=2)
    n = dev.n
    E = np.array([-1.2, 0.3, 2.1])
    eta = 0.05
    sr, sl = W.self_energies(dev, len(E))
    s = hsc.Solver(dev, 4, ordering=2)   # plain geometric dissection: one 64-site leaf, no cut
    assert s.stats.n_clusters == 1
    a, b = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pairs = np.stack([a.ravel(), b.ravel()], axis=1).astype(np.int32)
    _, _, pgr, _ = s.solve(E, eta, sr, sl, pairs=pairs)
    s.close()
    ref = pgr.reshape(len(E), n, n)

    Hd = dev.to_scipy().toarray()
    cu = dev.contact_unknowns()
    A = np.empty((len(E), n, n), dtype=np.complex128)
    for k in range(len(E)):
        A[k] = (E[k] + 1j * eta) * np.eye(n) - Hd
        A[k][cu, cu] -= sr[k]
    for call in range(2):
        got = _invert(torch, A)
        assert _rel(got, ref) <= TOL, call
        assert _rel(got, np.linalg.inv(A)) <= TOL, call


@pytest.mark.parametrize("n,batch", [(50, 5), (1000, 8), (1024, 8), (32, 256)])
def test_noalloc_matches_lapack_inverse(n, batch):
    """Against numpy.linalg.inv: a ragged final panel (50, 1000), the largest order (1024 x 8 =
    8192 rows) and the largest batch (256 blocks of 32)."""
    torch = _torch()
    A = _blocks(n, batch, seed=n + batch)
    ref = np.linalg.inv(A)
    for call in range(2):
        got = _invert(torch, A)
        assert _rel(got, ref) <= TOL, (call, _rel(got, ref))


def test_noalloc_in_place():
    torch = _torch()
    A = _blocks(50, 5, seed=7)
    ref = np.linalg.inv(A)
    for call in range(2):
        assert _rel(_invert(torch, A, in_place=True), ref) <= TOL, call


def test_noalloc_singular_block_is_reported_and_the_next_call_is_clean():
    torch = _torch()
    A = _blocks(50, 5, seed=11)
    A[3, 17, :] = 0.0          # one block with a zero row: a zero pivot, reported by the host-read flag
    with pytest.raises(hsc.HSCError) as ei:
        _invert(torch, A)
    assert ei.value.code == hsc.HSC_ERR_SINGULAR
    B = _blocks(50, 5, seed=12)   # the flag is cleared at the start of each call
    assert _rel(_invert(torch, B), np.linalg.inv(B)) <= TOL


def test_noalloc_setup_call_and_limits():
    torch = _torch()
    hsc.hsc_block_inverse_noalloc(64, 0, None, None)          # set-up only
    t = torch.zeros(2, dtype=torch.float64, device="cuda")
    for n, batch in ((2048, 1), (1024, 9), (16, 257)):   # rejected before any GPU work
        code = hsc.load().hsc_block_inverse_noalloc(n, batch, hsc._ptr(t), hsc._ptr(t), None)
        assert code == hsc.HSC_ERR_ARG, (n, batch, code)
    with pytest.raises(ValueError):   # the binding refuses a buffer smaller than batch * n * n values
        hsc.hsc_block_inverse_noalloc(16, 2, t, t)
