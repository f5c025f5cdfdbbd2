"""Oracle: the orthonormal 2-D Haar transform Omega (mu = Omega beta, Eq. 1.2).

TEST INFRASTRUCTURE ONLY.  Shares no code with the CUDA path.

The paper uses a level-L Haar discrete wavelet transform (Results section) and
does not state its normalisation; this oracle takes the orthonormal one, so
Omega^T = Omega^{-1}.  A coefficient at level l (1..L) belongs to a block of
2^l x 2^l pixels; its basis function is +-2^-l on that block:

  approximation (level L only):      +1 everywhere
  detail "h" (type 0):  +1 on the half with the lower y, -1 on the upper half
  detail "v" (type 1):  +1 on the half with the lower x, -1 on the upper half
  detail "d" (type 2):  the product of the two signs

Coefficient vector layout (length nx*ny): the level-L approximations
(ny>>L, nx>>L) row-major, then for l = L, L-1, ..., 1 the planes h_l, v_l,
d_l, each (ny>>l, nx>>l) row-major.

Two independent codings are given: the level-by-level butterfly
(`analysis`/`synthesis`) and the explicit basis matrix built from the
definition above (`basis_matrix`).  The tests pin them against each other
and against orthonormality and perfect reconstruction.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def layout(nx: int, ny: int, L: int):
    """List of planes (level, type, offset, rows, cols); type -1 = approximation."""
    if nx % (1 << L) or ny % (1 << L):
        raise ValueError("image sides must be divisible by 2^L")
    planes = []
    off = 0
    r, c = ny >> L, nx >> L
    planes.append((L, -1, off, r, c))
    off += r * c
    for l in range(L, 0, -1):
        r, c = ny >> l, nx >> l
        for t in range(3):
            planes.append((l, t, off, r, c))
            off += r * c
    assert off == nx * ny
    return planes


def analysis(img: np.ndarray, L: int) -> np.ndarray:
    """beta = Omega^T mu, level by level."""
    ny, nx = img.shape
    a = np.asarray(img, dtype=np.float64)
    det = {}
    for l in range(1, L + 1):
        ll, lh = a[0::2, 0::2], a[0::2, 1::2]     # (y lo, x lo), (y lo, x hi)
        hl, hh = a[1::2, 0::2], a[1::2, 1::2]     # (y hi, x lo), (y hi, x hi)
        det[l] = ((ll + lh - hl - hh) / 2.0,      # h: + on lower y
                  (ll - lh + hl - hh) / 2.0,      # v: + on lower x
                  (ll - lh - hl + hh) / 2.0)      # d
        a = (ll + lh + hl + hh) / 2.0
    out = [a.ravel()]
    for l in range(L, 0, -1):
        out.extend(p.ravel() for p in det[l])
    return np.concatenate(out)


def synthesis(beta: np.ndarray, nx: int, ny: int, L: int) -> np.ndarray:
    """mu = Omega beta, level by level."""
    planes = layout(nx, ny, L)
    beta = np.asarray(beta, dtype=np.float64)
    lvl, _, off, r, c = planes[0]
    a = beta[off:off + r * c].reshape(r, c)
    k = 1
    for l in range(L, 0, -1):
        h, v, d = (beta[planes[k + t][2]:planes[k + t][2] + planes[k + t][3] * planes[k + t][4]]
                   .reshape(planes[k + t][3], planes[k + t][4]) for t in range(3))
        k += 3
        out = np.empty((2 * a.shape[0], 2 * a.shape[1]))
        out[0::2, 0::2] = (a + h + v + d) / 2.0
        out[0::2, 1::2] = (a + h - v - d) / 2.0
        out[1::2, 0::2] = (a - h + v - d) / 2.0
        out[1::2, 1::2] = (a - h - v + d) / 2.0
        a = out
    return a


def coefficient_info(nx: int, ny: int, L: int):
    """Per coefficient: level, type (-1 approx, 0 h, 1 v, 2 d), block bx, by."""
    N = nx * ny
    level = np.empty(N, dtype=np.int64)
    typ = np.empty(N, dtype=np.int64)
    bx = np.empty(N, dtype=np.int64)
    by = np.empty(N, dtype=np.int64)
    for l, t, off, r, c in layout(nx, ny, L):
        yy, xx = np.meshgrid(np.arange(r), np.arange(c), indexing="ij")
        sl = slice(off, off + r * c)
        level[sl], typ[sl], bx[sl], by[sl] = l, t, xx.ravel(), yy.ravel()
    return level, typ, bx, by


def basis_matrix(nx: int, ny: int, L: int) -> sp.csc_matrix:
    """Omega (pixels x coefficients) from the definition of the basis functions."""
    rows, cols, vals = [], [], []
    for l, t, off, r, c in layout(nx, ny, L):
        s = 1 << l
        half = s >> 1
        # local pixel offsets inside one block, and the block origins
        oy, ox = np.meshgrid(np.arange(s), np.arange(s), indexing="ij")
        ylo, xlo = (oy < half).ravel(), (ox < half).ravel()
        if t == -1:
            sign = np.ones(s * s)
        elif t == 0:
            sign = np.where(ylo, 1.0, -1.0)
        elif t == 1:
            sign = np.where(xlo, 1.0, -1.0)
        else:
            sign = np.where(ylo, 1.0, -1.0) * np.where(xlo, 1.0, -1.0)
        by, bx = np.meshgrid(np.arange(r), np.arange(c), indexing="ij")
        by, bx = by.ravel(), bx.ravel()
        iy = by[:, None] * s + oy.ravel()[None, :]
        ix = bx[:, None] * s + ox.ravel()[None, :]
        rows.append((iy * nx + ix).ravel())
        cols.append(np.repeat(off + by * c + bx, s * s))
        vals.append(np.tile(sign / s, r * c))
    N = nx * ny
    return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N))
