"""The GEMM engines of the solve (FP64 tensor pipe; FP64 emulation on the BF16 tensor cores;
tcgen05 3xTF32) against numpy complex128, on ragged shapes spanning several tiles and every
operand-op combination the solve uses."""
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


@pytest.mark.parametrize("oa,ob", OPS)
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_fp64_emulation_engine(lib, oa, ob, M, N, K):
    """Eight balanced base-128 digits on the BF16 tensor cores: per K value and real product the
    error is below 2^-54.5 times the row and column scales (at most 8x the complex maxima's powers
    of two), so at FP64 level of |A||B|."""
    err = run(lib, 4, oa, ob, M, N, K, M + N + K)
    assert err <= 1e-13, err


def _emulated(L, A, B, oa=0, ob=0):
    import torch
    M, K = A.shape if oa == 0 else A.shape[::-1]
    N = B.shape[1] if ob == 0 else B.shape[0]
    dv = torch.device("cuda")
    tA = torch.from_numpy(np.ascontiguousarray(A, dtype=np.complex128).view(np.float64)).to(dv)
    tB = torch.from_numpy(np.ascontiguousarray(B, dtype=np.complex128).view(np.float64)).to(dv)
    tC = torch.full((M, 2 * N), float("nan"), dtype=torch.float64, device=dv)
    code = L.hsc_debug_gemm(4, oa, ob, M, N, K, tA.data_ptr(), A.shape[1], tB.data_ptr(), B.shape[1],
                            tC.data_ptr(), N, None, 0, 1.0, 0.0, 0.0, 0.0, None)
    assert code == 0, hsc.hsc_last_error()
    return tC.cpu().numpy().view(np.complex128)


@pytest.mark.parametrize("K", [1, 128, 517, 2048])
def test_fp64_emulation_exact_on_short_integers(lib, K):
    """Entries with at most 5 significant bits fit the first slice: the product is then computed
    exactly (integer slice products, FP32 accumulation exact below 2^24), equal to numpy's."""
    rng = np.random.default_rng(K)
    A = rng.integers(-15, 16, (70, K)) + 1j * rng.integers(-15, 16, (70, K))
    B = rng.integers(-15, 16, (K, 90)) + 1j * rng.integers(-15, 16, (K, 90))
    C = _emulated(lib, A, B)
    assert np.array_equal(C, A @ B)


@pytest.mark.parametrize("K", [200, 384, 1000])
def test_fp64_emulation_full_digits(lib, K):
    """x = sum_s d_s 2^(-7 s) with balanced base-128 digits d = (63, ..., 63, 60) (53 significant
    bits, in [1/4, 1/2), so its row scale is 1): every digit product on diagonal 9 is ~63^2 and the
    FP32 accumulators meet their largest partial sums (8 pairs, 12.2e6 over 384 K values, below
    2^24). The result must be K times the kept diagonals (s + r <= 9) up to the FP64 rounding of
    the drain; a lost unit in the accumulator of diagonal d would add 2^(-7 d) per chunk."""
    from fractions import Fraction
    t = [63] * 7 + [60]
    xf = sum(Fraction(t[s - 1], 2 ** (7 * s)) for s in range(1, 9))
    x = float(xf)
    assert Fraction(x) == xf and 0.25 <= x < 0.5
    pairs = [(s, r) for s in range(1, 9) for r in range(1, 9)]
    term = lambda s, r: Fraction(t[s - 1] * t[r - 1], 2 ** (7 * (s + r)))
    kept = sum(term(s, r) for s, r in pairs if s + r <= 9)
    assert kept + sum(term(s, r) for s, r in pairs if s + r >= 10) == xf ** 2
    assert sum(t[s - 1] * t[8 - s] for s in range(1, 9)) * 384 < 2 ** 24   # diagonal 9, one chunk
    A = np.full((130, K), x, dtype=np.complex128)
    B = np.full((K, 70), x, dtype=np.complex128)
    C = _emulated(lib, A, B)
    assert np.all(C.imag == 0.0)
    assert np.max(np.abs(C.real - float(K * kept))) <= K * 2.0 ** -50


def _scheme_scales(X, axis):
    """The emulation's power-of-two scale of each row (axis 1) or column (axis 0): one for the three
    real operands re, im and re + im, 4 times the power of two at or below their largest |entry|."""
    m = np.maximum(np.maximum(np.abs(X.real), np.abs(X.imag)), np.abs(X.real + X.imag)).max(axis=axis)
    return np.where(m > 0, 2.0 ** (np.floor(np.log2(np.where(m > 0, m, 1))) + 2), 0.0)


@pytest.mark.parametrize("K", [128, 700])
def test_fp64_emulation_within_row_dynamic_range(lib, K):
    """Entries of one row of A (and of one column of B) spanning 2^-40 .. 1: the emulation keeps 56
    bits relative to each row's and column's scale (sigma_i, tau_j: powers of two above twice the
    row's or column's largest real or imaginary part), so per K value and real product its error is
    below 2^-54.5 sigma_i tau_j, and the imaginary part of the complex product carries three real
    products: |C - AB| <= 3 K 2^-54.5 sigma_i tau_j plus the final rounding (the documented bound;
    a componentwise K u |A||B| bound does not hold for entries far below their row's maximum,
    which keep fewer bits). K = 128 runs the four-product form (two real products per part, the
    scales from re and im alone, at most those of the three-product form), K = 700 the 3M form."""
    rng = np.random.default_rng(11)
    M, N = 96, 80
    mag = lambda *sh: 2.0 ** rng.uniform(-40, 0, sh)
    A = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))) * mag(M, K)
    B = (rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))) * mag(K, N)
    C = _emulated(lib, A, B)
    ref = A @ B
    bound = 3 * K * 2.0 ** -54.5 * _scheme_scales(A, 1)[:, None] * _scheme_scales(B, 0)[None, :] + \
        2.0 ** -52 * np.abs(ref)
    assert np.all(np.abs(C.real - ref.real) <= bound) and np.all(np.abs(C.imag - ref.imag) <= bound)


def test_fp64_emulation_row_scaling(lib):
    """Rows of A and columns of B spanning 2^-300 .. 2^300: each gets its own power-of-two scale,
    so the error stays relative to the row and column maxima."""
    rng = np.random.default_rng(7)
    M, N, K = 96, 80, 300
    A = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))) * 2.0 ** rng.integers(-300, 300, (M, 1))
    B = (rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))) * 2.0 ** rng.integers(-300, 300, (1, N))
    C = _emulated(lib, A, B)
    ref = A @ B
    bound = K * np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(B), axis=0)[None, :] * 2.0 ** -46
    assert np.all(np.abs(C - ref) <= bound)


def _emulated_ab(L, A, B, Dm, alpha, beta, inplace=False):
    """C = alpha A B + beta D on the emulation engine (op N, N); D may be C itself (in place)."""
    import torch
    M, K = A.shape
    N = B.shape[1]
    dv = torch.device("cuda")
    tA = torch.from_numpy(np.ascontiguousarray(A, dtype=np.complex128).view(np.float64)).to(dv)
    tB = torch.from_numpy(np.ascontiguousarray(B, dtype=np.complex128).view(np.float64)).to(dv)
    tD = torch.from_numpy(np.ascontiguousarray(Dm, dtype=np.complex128).view(np.float64)).to(dv)
    tC = tD if inplace else torch.full((M, 2 * N), float("nan"), dtype=torch.float64, device=dv)
    code = L.hsc_debug_gemm(4, 0, 0, M, N, K, tA.data_ptr(), K, tB.data_ptr(), N, tC.data_ptr(), N,
                            tD.data_ptr(), N, alpha.real, alpha.imag, beta.real, beta.imag, None)
    assert code == 0, hsc.hsc_last_error()
    return tC.cpu().numpy().view(np.complex128)


@pytest.mark.parametrize("alpha,beta", [(1, 1), (-1, 1), (1, -1), (-1, -1), (0.5, -1), (-2, 0.25),
                                        (1, 0), (-0.5, 0), (0.7, 1), (1, 0.3 + 0.1j)])
@pytest.mark.parametrize("M,N,K", [(5, 7, 3), (130, 257, 33), (300, 200, 517)])
def test_fp64_emulation_alpha_beta(lib, alpha, beta, M, N, K):
    """alpha = +-2^k with beta = 0 or +-2^k (every product of the solve) takes the integer epilogue:
    beta D is folded into the exact sums in the product's units and the result rounded once; other
    alpha, beta take the FP64 epilogue. Both at 1e-13 of |alpha||A||B| + |beta D| componentwise,
    also with C aliasing D."""
    rng = np.random.default_rng(M * N + K)
    cplx = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    A, B, Dm = cplx(M, K), cplx(K, N), cplx(M, N)
    alpha, beta = complex(alpha), complex(beta)
    ref = alpha * (A @ B) + beta * Dm
    scale = np.abs(alpha) * np.abs(A) @ np.abs(B) + np.abs(beta * Dm)
    for inplace in (False, True):
        C = _emulated_ab(lib, A, B, Dm, alpha, beta, inplace)
        assert np.max(np.abs(C - ref) / scale) <= 1e-13


def test_fp64_emulation_integer_epilogue_is_one_rounding(lib):
    """Small integers: alpha A B + beta D is an exact double, and the integer epilogue (one rounding
    of the whole expression) must return it bit for bit, for every sign combination and a power-of-
    two alpha; D entries of 2^40 sit far above the product's units and still fold in exactly."""
    rng = np.random.default_rng(5)
    M, N, K = 140, 70, 300
    ints = lambda *s: rng.integers(-15, 16, s) + 1j * rng.integers(-15, 16, s)
    A, B = ints(M, K), ints(K, N)
    Dm = ints(M, N) * 2.0 ** rng.integers(0, 41, (M, N))
    for alpha, beta in ((1, 1), (-1, 1), (1, -1), (-1, -1), (0.5, -1), (-4, 0.5)):
        alpha, beta = complex(alpha), complex(beta)
        C = _emulated_ab(lib, A, B, Dm, alpha, beta)
        assert np.array_equal(C, alpha * (A @ B) + beta * Dm)


def test_fp64_emulation_epilogue_fallbacks(lib):
    """Elements the integer epilogue cannot fold take the FP64 one: D far above the product's
    range (|D| = 2^200 times the row and column scales), an all-zero row of A or column of B (zero
    scale: C = beta D exactly), and non-finite D (inf propagates); tiny and subnormal D fold in with
    a rounding at 2^-63 of the scales."""
    rng = np.random.default_rng(9)
    M, N, K = 130, 66, 200
    cplx = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    A, B, Dm = cplx(M, K), cplx(K, N), cplx(M, N)
    A[7, :] = 0
    B[:, 40] = 0
    Dm[3, :8] *= 2.0 ** 200
    Dm[5, 10:20] = 5e-310 - 3e-320j
    Dm[9, 30:34] *= 2.0 ** -600
    Dm[11, 50] = np.inf
    alpha, beta = complex(-1), complex(1)
    with np.errstate(invalid="ignore"):
        ref = alpha * (A @ B) + beta * Dm
        C = _emulated_ab(lib, A, B, Dm, alpha, beta)
    assert np.isposinf(C[11, 50].real)
    assert np.array_equal(C[7], beta * Dm[7]) and np.array_equal(C[:, 40], beta * Dm[:, 40])
    fin = np.isfinite(ref)
    scale = np.abs(A) @ np.abs(B) + np.abs(Dm)
    assert np.max(np.abs(C[fin] - ref[fin]) / scale[fin]) <= 1e-13
    assert np.max(np.abs(C[3, :8] - ref[3, :8]) / np.abs(ref[3, :8])) <= 2.0 ** -52
