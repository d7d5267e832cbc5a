"""The allocation-free block inversion entry point (hsc_block_inverse_noalloc).

It exists for callers that cannot allocate device memory while they run -- for instance an
application whose memory pool already holds the free device memory, so that a cudaMalloc would
fail, or a latency-bound loop that cannot take cudaMalloc/cudaFree's implicit synchronisation. Its
scratch is a fixed device array shared by all calls, so this test checks two calls in a row (the
second one runs on the scratch the first one left behind) against the regular entry point: with the
whole 4x4x4 device in a single cluster, hsc_solve's requested entries are the full inverse of A(E).
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1702_05167_gb300 import hsc, workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10


def test_noalloc_block_inverse_matches_hsc_solve_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    dev = W.cubic_device((4, 4, 4), W=1.0, seed=2)
    n = dev.n
    E = np.array([-1.2, 0.3, 2.1])
    eta = 0.05
    sr, sl = W.self_energies(dev, len(E))
    s = hsc.Solver(dev, 4)
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
    tA = torch.from_numpy(A.view(np.float64)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = torch.full_like(tA, float("nan"))
        hsc.hsc_block_inverse_noalloc(n, len(E), tA, out, stream=stream)
        got = out.cpu().numpy().view(np.complex128).reshape(len(E), n, n)
        for k in range(len(E)):
            err = np.abs(got[k] - ref[k]).max() / np.abs(ref[k]).max()
            assert err <= TOL, (call, k, err)


def test_noalloc_rejects_sizes_beyond_its_limit():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    t = torch.zeros(2, device="cuda")
    with pytest.raises(hsc.HSCError) as ei:
        hsc.hsc_block_inverse_noalloc(2048, 1, t, t)
    assert ei.value.code == hsc.HSC_ERR_ARG
