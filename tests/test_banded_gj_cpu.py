"""The two facts the banded Gauss-Jordan of the leaf blocks relies on, checked on the CPU with plain
Gauss-Jordan elimination (partial pivoting, largest |re| + |im|, as the panel kernels) on banded
complex-symmetric matrices whose small diagonal forces most pivots from below the diagonal:

* rows at positions >= k + b (b the bandwidth) are untouched until pivot k: no earlier pivot
  changes them and no earlier row interchange involves them;
* after its pivot step, pivot row j has no non-zero beyond column j + 2b.

So the panel of columns [k0, k0 + w) needs rows < k0 + w + b only, and the products of a wide panel
[k1, k1 + W) rows < k1 + W + b and columns < k1 + W + 2b; the inverse is unchanged (it equals
numpy's). No GPU."""
import numpy as np
import pytest


def _banded(n, b, seed, diag_scale):
    rng = np.random.default_rng(seed)
    A = np.zeros((n, n), complex)
    for d in range(1, b + 1):
        v = rng.standard_normal(n - d) + 1j * rng.standard_normal(n - d)
        v *= rng.random(n - d) < 0.6          # a sparse band, as a stencil's
        A += np.diag(v, d) + np.diag(v, -d)   # complex symmetric
    A += np.diag(diag_scale * (rng.standard_normal(n) + 1j * rng.standard_normal(n)))
    return A


def _gauss_jordan(A, b):
    """In-place Gauss-Jordan inverse with row interchanges; returns the inverse and, per step k,
    the largest row position changed by the step and the last non-zero column of the pivot row."""
    M = A.copy()
    n = len(M)
    perm = np.arange(n)
    touched, reach = [], []
    swaps = 0
    for k in range(n):
        p = k + int(np.argmax(np.abs(M[k:, k].real) + np.abs(M[k:, k].imag)))
        touched_k = p if p != k else -1
        if p != k:
            swaps += 1
            M[[k, p]] = M[[p, k]]
            perm[[k, p]] = perm[[p, k]]
        inv = 1.0 / M[k, k]
        M[k] *= inv
        M[k, k] = inv
        f = M[:, k].copy()
        f[k] = 0.0
        rows = np.nonzero(f)[0]
        if len(rows):
            touched_k = max(touched_k, int(rows.max()))
        M[rows] -= np.outer(f[rows], M[k])
        M[rows, k] = -f[rows] * inv
        nz = np.nonzero(M[k, k + 1:])[0]
        reach.append(int(k + 1 + nz.max()) if len(nz) else k)
        touched.append(touched_k)
    # undo the interchanges on the columns: inverse = M P
    Z = np.empty_like(M)
    Z[:, perm] = M
    return Z, touched, reach, swaps


@pytest.mark.parametrize("n,b,scale,seed", [(120, 8, 0.05, 1), (200, 16, 0.02, 2), (96, 12, 0.1, 3)])
def test_rows_beyond_the_band_stay_untouched_and_pivot_rows_end_within_2b(n, b, scale, seed):
    A = _banded(n, b, seed, scale)
    Z, touched, reach, swaps = _gauss_jordan(A, b)
    np.testing.assert_allclose(Z, np.linalg.inv(A), rtol=0, atol=1e-9 * np.abs(Z).max())
    for k in range(n):
        assert touched[k] < k + b + 1          # step k changes rows <= k + b only
        assert reach[k] <= k + 2 * b           # pivot row k ends at column k + 2b
    # row interchanges did happen (the small diagonal makes the test meaningful)
    assert swaps > n // 4


def test_deferred_rows_take_the_wide_panels_transform():
    """The deferral of the rows above a wide panel: after Gauss-Jordan with partial pivoting over the
    wide panel's columns [k1, k1 + W) (rows >= k1 eligible as pivots), the pivot rows (positions
    k1..k1 + W - 1) hold P^{-1} in those columns, P the pivot block, and a row above the wide panel
    that was left out of the eliminations becomes, from its values x there and y elsewhere:
    wide-panel part x T and other columns y + x T R, with T = -P^{-1} and R the pivot rows' other
    columns before the wide panel: the product the trailing step forms. Checked against running the
    same eliminations on that row."""
    rng = np.random.default_rng(4)
    n, k1, W = 40, 12, 8
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A[k1:, k1:k1 + W] *= 0.1 * (rng.random((n - k1, W)) < 0.5) + 0.05   # pivots from below
    M = A.copy()
    full = A.copy()   # the same steps applied to every row
    for j in range(k1, k1 + W):
        p = j + int(np.argmax(np.abs(full[j:, j].real) + np.abs(full[j:, j].imag)))
        full[[j, p]] = full[[p, j]]
        M[[j, p]] = M[[p, j]]
        inv = 1.0 / full[j, j]
        full[j] *= inv
        full[j, j] = inv
        f = full[:, j].copy()
        f[j] = 0.0
        full -= np.outer(f, full[j])
        full[:, j] = -f * inv
        full[j, j] = inv
    P = M[k1:k1 + W, k1:k1 + W]        # the pivot block (rows in their final order)
    Pinv = np.linalg.inv(P)
    np.testing.assert_allclose(full[k1:k1 + W, k1:k1 + W], Pinv, atol=1e-10 * np.abs(Pinv).max())
    T = -full[k1:k1 + W, k1:k1 + W]
    cols = np.r_[0:k1, k1 + W:n]
    R = M[k1:k1 + W][:, cols]            # the pivot rows' other columns before the wide panel
    for r in range(k1):                  # rows above: never pivots
        x, y = A[r, k1:k1 + W], A[r, cols]
        np.testing.assert_allclose(full[r, k1:k1 + W], x @ T, atol=1e-10 * np.abs(full[r]).max())
        np.testing.assert_allclose(full[r, cols], y + x @ T @ R, atol=1e-10 * np.abs(full[r]).max())
