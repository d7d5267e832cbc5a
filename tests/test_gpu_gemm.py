"""Both GEMM engines of the solve (FP64 tensor pipe; tcgen05 3xTF32) against numpy complex128, on
ragged shapes spanning several tiles and every operand-op combination the solve uses."""
import ctypes

import numpy as np
import pytest

from paper_1702_05167_gb300 import hsc

pytestmark = pytest.mark.gpu
OPS = [(0, 0), (1, 0), (0, 1), (0, 2), (0, 3)]
SHAPES = [(1, 1, 1), (5, 7, 3), (64, 64, 16), (130, 257, 33), (128, 128, 128), (300, 200, 517),
          (70, 90, 0)]


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    L = hsc.load()
    L.hsc_debug_gemm.argtypes = [ctypes.c_int32] * 6 + [ctypes.c_void_p, ctypes.c_int32,
                                                         ctypes.c_void_p, ctypes.c_int32,
                                                         ctypes.c_void_p, ctypes.c_int32,
                                                         ctypes.c_void_p, ctypes.c_int32] + \
        [ctypes.c_double] * 4 + [ctypes.c_void_p]
    L.hsc_debug_gemm.restype = ctypes.c_int
    return L


def op(X, o):
    return [X, X.T, X.conj(), X.conj().T][o]


def run(L, engine, oa, ob, M, N, K, seed):
    import torch
    rng = np.random.default_rng(seed)
    cplx = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    A = cplx(M, K) if oa in (0, 2) else cplx(K, M)
    B = cplx(K, N) if ob in (0, 2) else cplx(N, K)
    Dm = cplx(M, N)
    alpha, beta = -0.7 + 0.2j, 0.5 - 1.5j
    ref = alpha * (op(A, oa) @ op(B, ob)) + beta * Dm
    dv = torch.device("cuda")
    tA = torch.from_numpy(np.ascontiguousarray(A).view(np.float64)).to(dv)
    tB = torch.from_numpy(np.ascontiguousarray(B).view(np.float64)).to(dv)
    tD = torch.from_numpy(np.ascontiguousarray(Dm).view(np.float64)).to(dv)
    tC = torch.full((M, 2 * N), float("nan"), dtype=torch.float64, device=dv)
    code = L.hsc_debug_gemm(engine, oa, ob, M, N, K, tA.data_ptr(), A.shape[1], tB.data_ptr(),
                            B.shape[1], tC.data_ptr(), N, tD.data_ptr(), N, alpha.real, alpha.imag,
                            beta.real, beta.imag, None)
    assert code == 0, hsc.hsc_last_error()
    C = tC.cpu().numpy().view(np.complex128)
    scale = np.abs(alpha) * np.abs(op(A, oa)) @ np.abs(op(B, ob)) + np.abs(beta * Dm)
    return np.max(np.abs(C - ref) / scale)


@pytest.mark.parametrize("oa,ob", OPS)
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_fp64_engine(lib, oa, ob, M, N, K):
    """3M products: the imaginary part is a difference of products, bounded by ~eps K (|Ar|+|Ai|)
    (|Br|+|Bi|); asserted at 1e-13 of |alpha||A||B| + |beta D| componentwise."""
    assert run(lib, 0, oa, ob, M, N, K, M + N + K) <= 1e-13


@pytest.mark.parametrize("oa,ob", OPS)
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_fp64_engine_four_products(lib, oa, ob, M, N, K):
    assert run(lib, 3, oa, ob, M, N, K, M + N + K) <= 1e-14


@pytest.mark.parametrize("oa,ob", OPS)
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_tcgen05_packed_engine(lib, oa, ob, M, N, K):
    """Operands packed once into TF32 tile images and streamed with bulk async copies."""
    err = run(lib, 2, oa, ob, M, N, K, M + N + K)
    assert err <= 2e-6, err


@pytest.mark.parametrize("oa,ob", OPS)
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_tcgen05_3xtf32_engine(lib, oa, ob, M, N, K):
    """Componentwise error relative to |alpha| |A||B| + |beta D|: 3xTF32 products keep ~22
    significant bits; FP32 accumulation adds ~K * 2^-24."""
    err = run(lib, 1, oa, ob, M, N, K, M + N + K)
    assert err <= 2e-6, err
