"""Linear-decay spatial filter on element centroids (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper, Section 2.4: weights decay linearly with the distance between element
centroids up to rmin; the filter is the sparse product H . dc.  The paper
prints no normalisation or density weighting.  Reading taken here (the
classic sensitivity filter that the SIMP/OC literature pairs with OC):

    H_ei  = max(0, rmin - ||c_e - c_i||)      (weight 0 at distance rmin)
    Hs_e  = sum_i H_ei                        (over in-grid elements only,
                                               i.e. normalised at the boundary)
    dc~_e = sum_i H_ei x_i dc_i / (Hs_e max(1e-3, x_e))

Density filter: x~ = H x / Hs, with chain rule dc_e = sum_i H_ie dc_i / Hs_i.
Where passive elements i are pinned after filtering (x~_i = 0 or 1), x~_i
does not depend on x, so their terms drop out of the chain rule.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

GAMMA = 1e-3


def centroids(nelx, nely, nelz) -> np.ndarray:
    k, j, i = np.meshgrid(np.arange(nelz), np.arange(nely), np.arange(nelx), indexing="ij")
    return np.stack([i.ravel() + 0.5, j.ravel() + 0.5, k.ravel() + 0.5], axis=1)


def filter_matrix_bruteforce(nelx, nely, nelz, rmin) -> sp.csr_matrix:
    """O(nel^2) pairwise distances.  Tiny grids only."""
    c = centroids(nelx, nely, nelz)
    d = np.sqrt(((c[:, None, :] - c[None, :, :]) ** 2).sum(-1))
    w = np.maximum(0.0, rmin - d)
    return sp.csr_matrix(w)


def stencil_offsets(rmin):
    """Integer offsets (di, dj, dk) with positive weight rmin - |d|."""
    R = int(np.ceil(rmin)) - 1 if float(rmin).is_integer() else int(np.floor(rmin))
    out = []
    for dk in range(-R, R + 1):
        for dj in range(-R, R + 1):
            for di in range(-R, R + 1):
                w = rmin - np.sqrt(di * di + dj * dj + dk * dk)
                if w > 0:
                    out.append((di, dj, dk, w))
    return out


def filter_matrix(nelx, nely, nelz, rmin) -> sp.csr_matrix:
    """H by an O(nel * S) loop over stencil offsets (S = stencil size)."""
    nel = nelx * nely * nelz
    k, j, i = np.meshgrid(np.arange(nelz), np.arange(nely), np.arange(nelx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    rows, cols, vals = [], [], []
    for di, dj, dk, w in stencil_offsets(rmin):
        ii, jj, kk = i + di, j + dj, k + dk
        ok = (ii >= 0) & (ii < nelx) & (jj >= 0) & (jj < nely) & (kk >= 0) & (kk < nelz)
        e = np.flatnonzero(ok)
        rows.append(e)
        cols.append(ii[ok] + nelx * (jj[ok] + nely * kk[ok]))
        vals.append(np.full(e.size, w))
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(nel, nel)).tocsr()


def row_sums(H) -> np.ndarray:
    return np.asarray(H.sum(axis=1)).ravel()


def sensitivity_filter(H, Hs, x, dc) -> np.ndarray:
    return (H @ (x * dc)) / (Hs * np.maximum(GAMMA, x))


def density_filter(H, Hs, x) -> np.ndarray:
    return (H @ x) / Hs


def density_filter_chain(H, Hs, dc, passive=None) -> np.ndarray:
    """d/dx of a function of the filtered field, given its gradient dc with
    respect to the filtered field.  Elements whose filtered value is pinned
    (passive != 0) contribute nothing."""
    g = dc / Hs
    if passive is not None:
        g = np.where(np.asarray(passive) != 0, 0.0, g)
    return H.T @ g


def _shift_sum(nelx, nely, nelz, rmin, v):
    """sum over in-grid stencil neighbours i of H_ei v_i, for every e."""
    V = v.reshape(nelz, nely, nelx)
    out = np.zeros_like(V)
    for di, dj, dk, w in stencil_offsets(rmin):
        # out[k, j, i] += w * V[k+dk, j+dj, i+di] where in range
        ks = slice(max(0, -dk), nelz - max(0, dk))
        js = slice(max(0, -dj), nely - max(0, dj))
        is_ = slice(max(0, -di), nelx - max(0, di))
        ks2 = slice(max(0, dk), nelz - max(0, -dk))
        js2 = slice(max(0, dj), nely - max(0, -dj))
        is2 = slice(max(0, di), nelx - max(0, -di))
        out[ks, js, is_] += w * V[ks2, js2, is2]
    return out.reshape(-1)


def sensitivity_filter_stencil(nelx, nely, nelz, rmin, x, dc) -> np.ndarray:
    """Same as ``sensitivity_filter`` without forming H (large grids)."""
    Hs = _shift_sum(nelx, nely, nelz, rmin, np.ones(nelx * nely * nelz))
    return _shift_sum(nelx, nely, nelz, rmin, x * dc) / (Hs * np.maximum(GAMMA, x))


def row_sums_stencil(nelx, nely, nelz, rmin) -> np.ndarray:
    return _shift_sum(nelx, nely, nelz, rmin, np.ones(nelx * nely * nelz))
