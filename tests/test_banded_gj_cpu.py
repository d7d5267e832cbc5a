"""The two facts the banded Gauss-Jordan of the leaf blocks relies on, checked on the CPU with plain
Gauss-Jordan elimination (partial pivoting, largest |re| + |im|, as the panel kernels) on banded
complex-symmetric matrices whose small diagonal forces most pivots from below the diagonal:

* rows at positions >= k + b (b the bandwidth) are untouched until pivot k: no earlier pivot
  changes them and no earlier row interchange involves them;
* after its pivot step, pivot row j has no non-zero beyond column j + 2b.

So the panel of columns [k0, k0 + w) needs rows < k0 + w + b only, and the products of a wide panel
[k1, k1 + W) rows < k1 + W + b and columns < k1 + W + 2b; the inverse is unchanged (it equals
numpy's). With outermost diagonals that dominate, both bounds are attained.

Then the rows above a wide panel, left out of its nested panels: they take the wide panel's
transform T = -P^{-1} in its trailing product. And the whole leaf-block schedule (nested panels,
band limits, deferred rows, ragged last panels) against plain Gauss-Jordan after every wide panel.
No GPU."""
import numpy as np
import pytest


def _banded(n, b, seed, diag_scale, edge=0.0):
    """Complex-symmetric, bandwidth b. edge > 0 adds entries of modulus edge..2 edge on the outermost
    diagonals, so that most pivots come from b rows below and the bounds below are attained."""
    rng = np.random.default_rng(seed)
    A = np.zeros((n, n), complex)
    for d in range(1, b + 1):
        v = rng.standard_normal(n - d) + 1j * rng.standard_normal(n - d)
        v *= rng.random(n - d) < 0.6          # a sparse band, as a stencil's
        A += np.diag(v, d) + np.diag(v, -d)   # complex symmetric
    A += np.diag(diag_scale * (rng.standard_normal(n) + 1j * rng.standard_normal(n)))
    if edge:
        v = edge * (1 + rng.random(n - b)) * np.exp(2j * np.pi * rng.random(n - b))
        A += np.diag(v, b) + np.diag(v, -b)
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


@pytest.mark.parametrize("n,b,scale,seed,edge", [(120, 8, 0.05, 1, 0.0), (200, 16, 0.02, 2, 0.0),
                                                  (96, 12, 0.1, 3, 0.0), (120, 6, 0.05, 3, 10.0)])
def test_rows_beyond_the_band_stay_untouched_and_pivot_rows_end_within_2b(n, b, scale, seed, edge):
    A = _banded(n, b, seed, scale, edge)
    Z, touched, reach, swaps = _gauss_jordan(A, b)
    np.testing.assert_allclose(Z, np.linalg.inv(A), rtol=0, atol=1e-9 * np.abs(Z).max())
    for k in range(n):
        assert touched[k] < k + b + 1          # step k changes rows <= k + b only
        assert reach[k] <= k + 2 * b           # pivot row k ends at column k + 2b
    # row interchanges did happen (the small diagonal makes the test meaningful)
    assert swaps > n // 4
    if edge:   # both bounds attained
        assert max(touched[k] - k for k in range(n)) == b
        assert sum(reach[k] == k + 2 * b for k in range(n)) > n // 2


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


def _panel_gj(X, k0, w, lo, hi):
    """Unblocked Gauss-Jordan over columns [k0, k0 + w) of rows [lo, hi) (pivot search over rows
    j..hi-1), row interchanges applied to whole rows of X. Returns the finished panel block: the
    pivot rows (positions k0..k0 + w - 1) hold P^{-1}, the other rows -x P^{-1}."""
    S = X[lo:hi, k0:k0 + w].copy()
    for jj in range(w):
        j = k0 + jj
        p = j + int(np.argmax(np.abs(S[j - lo:, jj].real) + np.abs(S[j - lo:, jj].imag)))
        if p != j:
            X[[j, p]] = X[[p, j]]
            S[[j - lo, p - lo]] = S[[p - lo, j - lo]]
        inv = 1.0 / S[j - lo, jj]
        S[j - lo] *= inv
        S[j - lo, jj] = inv
        f = S[:, jj].copy()
        f[j - lo] = 0.0
        S -= np.outer(f, S[j - lo])
        S[:, jj] = -f * inv
        S[j - lo, jj] = inv
    return S


def _apply(X, Mt, rows, cols, k0, w, R):
    """X[rows, cols] = (0 on the pivot rows, else X) + Mt R, R the pivot rows' columns cols with the
    identity in the panel's own columns (those of X taken as 0): the trailing product of a panel."""
    C = X[np.ix_(rows, cols)].copy()
    piv = (rows >= k0) & (rows < k0 + w)
    C[piv] = 0.0
    C[:, (cols >= k0) & (cols < k0 + w)] = 0.0
    X[np.ix_(rows, cols)] = C + Mt @ R


def _nested_banded_deferred_gj(A, nb, W, b):
    """The leaf-block schedule: panels of nb inside wide panels of W. A nested panel works on rows
    [k1, k0 + w + b) (b = 0: all rows from k1) and the wide panel's columns; the wide panel's
    trailing product on rows [k1, k1 + W + b) and columns [0, k1 + W + 2b); the rows above k1 take
    (their wide-panel part) x (-P^{-1} R) in that product. Yields the state after each wide panel."""
    X = A.copy()
    n = len(X)
    for k1 in range(0, n, W):
        wo = min(W, n - k1)
        wide = np.arange(k1, k1 + wo)
        x_above = X[:k1, k1:k1 + wo].copy()       # the rows above: untouched until the wide product
        for k0 in range(k1, k1 + wo, nb):
            w = min(nb, k1 + wo - k0)
            hi = min(n, k0 + w + b) if b else n
            S = _panel_gj(X, k0, w, k1, hi)
            R = X[np.ix_(np.arange(k0, k0 + w), wide)].copy()
            R[:, k0 - k1:k0 - k1 + w] = np.eye(w)
            _apply(X, S, np.arange(k1, hi), wide, k0, w, R)
        # the wide panel's trailing product, K = wo
        mr = min(n, k1 + wo + b) if b else n
        nc = min(n, k1 + wo + 2 * b) if b else n
        cols = np.arange(nc)
        Mt = X[k1:mr, k1:k1 + wo].copy()          # P^{-1} on the pivot rows, -x P^{-1} below
        R = X[np.ix_(np.arange(k1, k1 + wo), cols)].copy()
        R[:, k1:k1 + wo] = np.eye(wo)
        if b:   # pivot rows end within 2b of their column: nothing beyond nc
            assert not np.any(X[k1:k1 + wo, nc:])
        Bp = -Mt[:wo] @ R                         # T R, T = -P^{-1}
        _apply(X, Mt, np.arange(k1, mr), cols, k1, wo, R)
        if k1:
            X[:k1, k1:k1 + wo] = 0.0
            X[:k1, :nc] += x_above @ Bp
        yield k1 + wo, X


@pytest.mark.parametrize("n,b,nb,W,scale,seed,edge", [(200, 8, 16, 64, 0.05, 5, 0.0), (150, 6, 16, 48, 0.02, 6, 0.0),
                                                       (130, 0, 16, 64, 0.3, 7, 0.0), (97, 12, 8, 32, 0.1, 8, 0.0),
                                                       (200, 6, 16, 64, 0.05, 9, 10.0), (161, 5, 16, 48, 0.05, 10, 10.0)])
def test_nested_banded_deferred_schedule_is_exact(n, b, nb, W, scale, seed, edge):
    """The composition of the three restrictions (banded rows and columns, nested panels on the
    wide panel's columns, rows above each wide panel deferred to its trailing product) gives, after
    every wide panel, the state of plain Gauss-Jordan over the same columns, and at the end the
    inverse (ragged last panels included; b = 0 is a dense block)."""
    A = _banded(n, b, seed, scale, edge) if b else (
        np.random.default_rng(seed).standard_normal((n, n)) + 1j * np.random.default_rng(seed + 1).standard_normal((n, n)))
    ref = A.copy()
    perm = np.arange(n)
    done = 0
    for upto, X in _nested_banded_deferred_gj(A, nb, W, b):
        for k in range(done, upto):   # plain in-place Gauss-Jordan, whole rows
            p = k + int(np.argmax(np.abs(ref[k:, k].real) + np.abs(ref[k:, k].imag)))
            ref[[k, p]] = ref[[p, k]]
            perm[[k, p]] = perm[[p, k]]
            inv = 1.0 / ref[k, k]
            ref[k] *= inv
            ref[k, k] = inv
            f = ref[:, k].copy()
            f[k] = 0.0
            ref -= np.outer(f, ref[k])
            ref[:, k] = -f * inv
            ref[k, k] = inv
        done = upto
        np.testing.assert_allclose(X, ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    Z = np.empty_like(X)
    Z[:, perm] = X   # undo the interchanges on the columns
    np.testing.assert_allclose(Z, np.linalg.inv(A), rtol=0, atol=1e-9 * np.abs(Z).max())
