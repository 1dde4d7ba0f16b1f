"""Error norms and orders of accuracy (Sec. 3, Eqs. oneNormErr, twoNormErr, inftyNormErr).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Reading of the norms: the printed formulas divide by N^2, but the printed values of
Tables 4-9 are reproduced exactly only by the cell-area weighting
L1 = sum dx dy |e|, L2 = (sum dx dy e^2)^(1/2), Linf = max |e| (on [-1, 1]^2 this is 4x
and 2x the 1/N^2 forms).  ``paper_norms`` returns the area-weighted forms; the literal
1/N^2 forms are ``mean_norms``.  Orders: O = log2(L_{N_p} / L_{N_{p+1}}) (Sec. 3.1).
"""
from __future__ import annotations

import numpy as np


def paper_norms(err: np.ndarray, dx: float, dy: float) -> tuple[float, float, float]:
    e = np.abs(np.asarray(err, dtype=np.float64))
    return float(np.sum(e) * dx * dy), float(np.sqrt(np.sum(e * e) * dx * dy)), float(np.max(e))


def mean_norms(err: np.ndarray) -> tuple[float, float, float]:
    e = np.abs(np.asarray(err, dtype=np.float64))
    return float(np.mean(e)), float(np.sqrt(np.mean(e * e))), float(np.max(e))


def orders(values) -> list[float]:
    v = list(values)
    return [float(np.log2(v[p] / v[p + 1])) for p in range(len(v) - 1)]


def rel_l2(fx, fy, fx_ref, fy_ref) -> float:
    """Relative L2 error of the pair (F^x, F^y) over all cells, one number per form."""
    num = np.sum((np.asarray(fx, np.float64) - fx_ref) ** 2) + np.sum((np.asarray(fy, np.float64) - fy_ref) ** 2)
    den = np.sum(np.asarray(fx_ref, np.float64) ** 2) + np.sum(np.asarray(fy_ref, np.float64) ** 2)
    return float(np.sqrt(num / den))
