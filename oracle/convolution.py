"""Discrete force convolution F_ij = G sum C_{i'j'} w_{i-i', j-j'} (Eq. eqnF) and its
transpose.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Two evaluations of the same exact discrete result:
  * ``forces_direct``: the double sum of Eq. (eqnF) written out (O(Nx^2 Ny^2)), for small
    grids;
  * ``forces_fft``: the same linear convolution through the convolution theorem (Sec. 4.1,
    one forward transform of C and two inverse transforms), with C and the tables placed
    on a zero-padded 2Nx x 2Ny periodic grid.  Circular convolution of period
    P >= 2N - 1 equals the linear one on the cropped window; offset +-N (index N) is never
    reached and is set to zero.  pocketfft in FP64 is the library primitive: numpy's
    (one thread), or scipy's when a thread count is given (the same transforms over the
    rows and columns of the padded arrays, spread over host threads).

Array convention: shape (Nx, Ny), axis 0 is x.  Tables are the full arrays of
``kernel_tables`` (shape (2Nx-1, 2Ny-1), index [m + Nx - 1, n + Ny - 1]).
"""
from __future__ import annotations

import numpy as np

from .coefficients import adjoint_coefficients, bspline_coefficients
from .kernel_tables import kernel_tables, potential_table


def forces_direct(c: np.ndarray, wx: np.ndarray, wy: np.ndarray, G: float = 1.0):
    """Eq. (eqnF) as a literal double sum over source cells, one output cell at a time."""
    nx, ny = c.shape
    fx = np.zeros((nx, ny))
    fy = np.zeros((nx, ny))
    for i in range(nx):
        for j in range(ny):
            # offsets m = i - i' for i' = 0..nx-1 -> table rows (i - i') + nx - 1
            rows = slice(i + nx - 1, i - 1 if i > 0 else None, -1)
            cols = slice(j + ny - 1, j - 1 if j > 0 else None, -1)
            fx[i, j] = np.sum(c * wx[rows, cols])
            fy[i, j] = np.sum(c * wy[rows, cols])
    return G * fx, G * fy


def place_periodic(w: np.ndarray, px: int, py: int) -> np.ndarray:
    """Table on the periodic P_x x P_y grid: entry (m, n) at (m mod P_x, n mod P_y)."""
    mx = (w.shape[0] + 1) // 2
    my = (w.shape[1] + 1) // 2
    out = np.zeros((px, py))
    ms = np.arange(-(mx - 1), mx) % px
    ns = np.arange(-(my - 1), my) % py
    out[np.ix_(ms, ns)] = w
    return out


def spectra(wx: np.ndarray, wy: np.ndarray, px: int, py: int):
    """Forward transforms of the placed tables (Sec. 4.1, convolution theorem)."""
    return (np.fft.rfft2(place_periodic(wx, px, py)),
            np.fft.rfft2(place_periodic(wy, px, py)))


def _fft2(workers):
    """(rfft2, irfft2) of the library: numpy's for workers None, else scipy's on that many
    host threads."""
    if workers is None:
        return np.fft.rfft2, np.fft.irfft2
    import scipy.fft as sf
    return (lambda a, s: sf.rfft2(a, s=s, workers=workers)), (lambda a, s: sf.irfft2(a, s=s, workers=workers))


def forces_fft(c: np.ndarray, wx: np.ndarray, wy: np.ndarray, G: float = 1.0, spec=None, workers=None):
    """Same result as ``forces_direct`` via zero-padded FFTs (1 forward + 2 inverse)."""
    nx, ny = c.shape
    px, py = 2 * nx, 2 * ny
    if spec is None:
        spec = spectra(wx, wy, px, py)
    rfft2, irfft2 = _fft2(workers)
    chat = rfft2(c, s=(px, py))
    fx = irfft2(chat * spec[0], s=(px, py))[:nx, :ny]
    fy = irfft2(chat * spec[1], s=(px, py))[:nx, :ny]
    return G * fx, G * fy


def correlate_fft(gx: np.ndarray, gy: np.ndarray, wx: np.ndarray, wy: np.ndarray,
                  G: float = 1.0, spec=None):
    """Transpose of C -> (F^x, F^y): dL/dC_{i'j'} = G sum_ij (gx_ij w^x_{i-i',j-j'} +
    gy_ij w^y_{i-i',j-j'}), i.e. a correlation with the same tables."""
    nx, ny = gx.shape
    px, py = 2 * nx, 2 * ny
    if spec is None:
        spec = spectra(wx, wy, px, py)
    gxh = np.fft.rfft2(gx, s=(px, py))
    gyh = np.fft.rfft2(gy, s=(px, py))
    out = np.fft.irfft2(gxh * np.conj(spec[0]) + gyh * np.conj(spec[1]), s=(px, py))[:nx, :ny]
    return G * out


def correlate_direct(gx, gy, wx, wy, G: float = 1.0):
    """The transpose as a literal double sum (small grids)."""
    nx, ny = gx.shape
    out = np.zeros((nx, ny))
    for ip in range(nx):
        for jp in range(ny):
            rows = slice(nx - 1 - ip, 2 * nx - 1 - ip)
            cols = slice(ny - 1 - jp, 2 * ny - 1 - jp)
            out[ip, jp] = np.sum(gx * wx[rows, cols]) + np.sum(gy * wy[rows, cols])
    return G * out


def potential_direct(c: np.ndarray, wphi: np.ndarray, G: float = 1.0):
    """Phi_ij = -G sum_{i'j'} C_{i'j'} w^phi(i - i', j - j') as a literal double sum."""
    nx, ny = c.shape
    out = np.zeros((nx, ny))
    for i in range(nx):
        for j in range(ny):
            rows = slice(i + nx - 1, i - 1 if i > 0 else None, -1)
            cols = slice(j + ny - 1, j - 1 if j > 0 else None, -1)
            out[i, j] = np.sum(c * wphi[rows, cols])
    return -G * out


def potential_fft(c: np.ndarray, wphi: np.ndarray, G: float = 1.0):
    """The same through zero-padded FFTs (one forward transform of C, one inverse)."""
    nx, ny = c.shape
    px, py = 2 * nx, 2 * ny
    spec = np.fft.rfft2(place_periodic(wphi, px, py))
    return -G * np.fft.irfft2(np.fft.rfft2(c, s=(px, py)) * spec, s=(px, py))[:nx, :ny]


class Solver:
    """The oracle's whole force solve for one grid: tables once, then sigma -> forces.

    Sec. 4.2: the tables (and their transforms) are computed once and reused.
    """

    def __init__(self, nx: int, ny: int, k: int, dx: float, dy: float, G: float = 1.0):
        self.nx, self.ny, self.k = nx, ny, k
        self.dx, self.dy, self.G = dx, dy, G
        self.wx, self.wy = kernel_tables(k, nx, ny, dx, dy)
        self._spec = None

    @property
    def spec(self):
        if self._spec is None:
            self._spec = spectra(self.wx, self.wy, 2 * self.nx, 2 * self.ny)
        return self._spec

    def coefficients(self, sigma):
        return bspline_coefficients(sigma, self.k)

    def forces(self, sigma, method: str = "fft", workers=None):
        """workers: host threads of the FFTs (None: numpy's single-threaded pocketfft)."""
        c = self.coefficients(sigma)
        if method == "direct":
            return forces_direct(c, self.wx, self.wy, self.G)
        return forces_fft(c, self.wx, self.wy, self.G, self.spec, workers)

    def forces_at(self, sigma, points):
        """F^x, F^y at a few output cells, each one by its own literal sum (any size)."""
        c = self.coefficients(sigma)
        nx, ny = self.nx, self.ny
        fx, fy = [], []
        for i, j in points:
            rows = slice(i + nx - 1, i - 1 if i > 0 else None, -1)
            cols = slice(j + ny - 1, j - 1 if j > 0 else None, -1)
            fx.append(self.G * np.sum(c * self.wx[rows, cols]))
            fy.append(self.G * np.sum(c * self.wy[rows, cols]))
        return np.array(fx), np.array(fy)

    def potential(self, sigma, method: str = "fft"):
        """Phi at the cell centres (the potential kernel's table is built on first use)."""
        if getattr(self, "_wphi", None) is None:
            self._wphi = potential_table(self.k, self.nx, self.ny, self.dx, self.dy)
        c = self.coefficients(sigma)
        if method == "direct":
            return potential_direct(c, self._wphi, self.G)
        return potential_fft(c, self._wphi, self.G)

    def adjoint(self, gx, gy, method: str = "fft"):
        """dL/dsigma for L = sum(gx F^x + gy F^y)."""
        if method == "direct":
            gc = correlate_direct(gx, gy, self.wx, self.wy, self.G)
        else:
            gc = correlate_fft(gx, gy, self.wx, self.wy, self.G, self.spec)
        return adjoint_coefficients(gc, self.k)
