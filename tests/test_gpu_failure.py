"""Failure detection without faulting the GPU: a bounded device wait on a flag that nothing sets
expires and is reported as HSC_ERR_TIMEOUT; the context stays usable afterwards."""
import ctypes

import numpy as np
import pytest

from paper_1702_05167_gb300 import hsc, workloads as W
from oracle import dense

pytestmark = pytest.mark.gpu


def test_bounded_wait_expires_and_context_survives():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    L = hsc.load()
    L.hsc_debug_wait_timeout.argtypes = [ctypes.c_double]
    L.hsc_debug_wait_timeout.restype = ctypes.c_int
    assert L.hsc_debug_wait_timeout(0.05) == hsc.HSC_ERR_TIMEOUT
    assert "expired" in hsc.hsc_last_error()
    assert L.hsc_debug_wait_timeout(5.0) == hsc.HSC_ERR_ARG       # refuses long waits
    dev = W.cubic_device((5, 4, 4), seed=1)                        # the GPU still solves correctly
    sr, sl = W.self_energies(dev, 1)
    s = hsc.Solver(dev, 2)
    dgr, _, _, _ = s.solve(np.array([0.4]), 0.05, sr, sl)
    s.close()
    G, _ = dense.solve(dev.to_scipy().toarray(), 0.4, 0.05, dev.contact_unknowns(), sr[0], sl[0])
    assert np.abs(dgr[0] - np.diag(G)).max() / np.abs(np.diag(G)).max() <= 1e-10
