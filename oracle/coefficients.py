"""B-spline coefficients C from cell-centre samples sigma (Sec. 2.3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper references:
  * Eq. (eqnSigmaB) - interpolation condition sigma(x_i, y_j) = sum C B B at cell centres.
  * Sec. 2.3, k = 1, 2: C_ij = sigma_ij (the normalised spline is 1 at its own centre and
    0 at every other centre).
  * Eq. (sigmaW) - for k = 3, sigma_ij = z_{i,j-1} + 6 z_ij + z_{i,j+1} with
    z_ij = (C_{i-1,j} + 6 C_ij + C_{i+1,j}) / 64.
  * Eq. (z_system) - tridiag(1,6,1) z = sigma along j, one system per i.
  * Eq. (C_system) - (1/64) tridiag(1,6,1) C = z along i, one system per j.
  * Isolated boundary condition C_ij = 0 outside the grid: the tridiagonal systems are the
    truncated ones (first and last rows keep only two entries).
  * Orders 4 and 5 (the paper calls the extension straightforward, Sec. 2.2 and Sec. 2.3):
    the same interpolation condition, sum_i' C_i' b_k(i - i') = s_i along each axis with
    C = 0 outside, whose stencil is b_k at the integer offsets: (1, 4, 1)/6 for k = 4
    (knots at cell centres) and (1, 76, 230, 76, 1)/384 for k = 5 (knots at faces).  One
    banded solve along y, then one along x, by plain Gaussian elimination.

Array convention: sigma has shape (Nx, Ny), index [i, j] <-> (x_i, y_j); axis 0 is x.
"""
from __future__ import annotations

import numpy as np

from .bspline import values_at_integers


def thomas(sub: float, diag: float, sup: float, rhs: np.ndarray) -> np.ndarray:
    """Plain Thomas algorithm (Gaussian elimination without pivoting) for a constant
    tridiagonal Toeplitz matrix tridiag(sub, diag, sup), solved along axis 0 of rhs.

    Every other axis of rhs is an independent system (vectorised, not fused).
    """
    rhs = np.asarray(rhs, dtype=np.float64)
    n = rhs.shape[0]
    cp = np.zeros(n)
    dp = np.zeros_like(rhs)
    cp[0] = sup / diag
    dp[0] = rhs[0] / diag
    for i in range(1, n):
        denom = diag - sub * cp[i - 1]
        cp[i] = sup / denom
        dp[i] = (rhs[i] - sub * dp[i - 1]) / denom
    x = np.zeros_like(rhs)
    x[n - 1] = dp[n - 1]
    for i in range(n - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    return x


def stencil(k: int) -> list[float]:
    """b_k at the integer offsets -h..h (h = (k - 1) // 2): row i of the 1-D interpolation
    matrix holds stencil[d + h] in column i + d."""
    v = values_at_integers(k)
    h = (k - 1) // 2
    return [v.get(d, 0.0) for d in range(-h, h + 1)]


def banded_solve(st: list[float], rhs: np.ndarray) -> np.ndarray:
    """Gaussian elimination without pivoting for the truncated banded Toeplitz matrix of
    stencil st (rows near the ends lose the entries that fall outside), along axis 0 of
    rhs.  The matrices here are strictly diagonally dominant, so no pivoting is needed."""
    rhs = np.array(rhs, dtype=np.float64)
    n = rhs.shape[0]
    h = (len(st) - 1) // 2
    band = np.tile(np.asarray(st, dtype=np.float64), (n, 1))  # band[i, d + h] = A[i, i + d]
    for i in range(n):
        for d in range(-h, h + 1):
            if not 0 <= i + d < n:
                band[i, d + h] = 0.0
    for i in range(n):
        piv = band[i, h]
        for r in range(1, h + 1):
            if i + r >= n:
                break
            f = band[i + r, h - r] / piv
            for d in range(0, h + 1):
                band[i + r, h - r + d] -= f * band[i, h + d]
            rhs[i + r] -= f * rhs[i]
    x = np.zeros_like(rhs)
    for i in range(n - 1, -1, -1):
        acc = rhs[i].copy()
        for d in range(1, h + 1):
            if i + d < n:
                acc -= band[i, h + d] * x[i + d]
        x[i] = acc / band[i, h]
    return x


def bspline_coefficients(sigma: np.ndarray, k: int) -> np.ndarray:
    """C from sigma at order k (Sec. 2.3)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    if k in (1, 2):
        return sigma.copy()
    if k in (4, 5):
        st = stencil(k)
        z = banded_solve(st, sigma.T).T  # along j (axis 1), one system per row i
        return banded_solve(st, z)       # along i (axis 0), one system per column j
    if k != 3:
        raise ValueError("order must be 1 to 5")
    # Eq. (z_system): along j (axis 1), one system per row i.
    z = thomas(1.0, 6.0, 1.0, sigma.T).T
    # Eq. (C_system): (1/64) tridiag(1,6,1) C = z along i (axis 0), one system per column j.
    c = thomas(1.0, 6.0, 1.0, 64.0 * z)
    return c


def apply_interpolation(c: np.ndarray, k: int) -> np.ndarray:
    """Forward map C -> sigma at the cell centres (Eq. sigmaW for k = 3, identity below),
    with C = 0 outside the grid.  Used to check a coefficient solve by its residual."""
    c = np.asarray(c, dtype=np.float64)
    if k in (1, 2):
        return c.copy()
    if k in (4, 5):
        st = stencil(k)
        h = (k - 1) // 2
        nx, ny = c.shape
        p = np.pad(c, h)
        z = sum(st[d + h] * p[h + d:h + d + nx, :] for d in range(-h, h + 1))
        return sum(st[d + h] * z[:, h + d:h + d + ny] for d in range(-h, h + 1))
    p = np.pad(c, 1)
    z = (p[:-2, 1:-1] + 6.0 * p[1:-1, 1:-1] + p[2:, 1:-1]) / 64.0
    q = np.pad(z, ((0, 0), (1, 1)))
    return q[:, :-2] + 6.0 * q[:, 1:-1] + q[:, 2:]


def adjoint_coefficients(gc: np.ndarray, k: int) -> np.ndarray:
    """Transpose of sigma -> C.  The map is the product of the x and y solves with
    symmetric matrices (64 T_x^{-1} T_y^{-1} for k = 3, the banded ones for k = 4, 5), so
    its transpose is the same pair of solves."""
    return bspline_coefficients(gc, k)
