"""The dense oracle still reproduces the frozen 8x8x8 fixture written by tests/golden/make_golden.py."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def test_oracle_matches_frozen_fixture():
    ref = np.loadtxt(os.path.join(HERE, "golden", "tiny_8x8x8.txt"))
    gr, gl = make_golden.compute()
    np.testing.assert_allclose(gr, ref[:, 1] + 1j * ref[:, 2], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(gl, ref[:, 3] + 1j * ref[:, 4], rtol=1e-12, atol=1e-14)
