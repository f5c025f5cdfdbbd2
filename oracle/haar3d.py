"""Oracle: the orthonormal 3-D Haar transform (Eq. 1.2 for a volume).

TEST INFRASTRUCTURE ONLY.  Shares no code with the CUDA path.

A level-l coefficient (l = 1..L) belongs to a block of 2^l x 2^l x 2^l
voxels and its basis function is +-2^(-3l/2) on the block.  Its type t =
0..7 is a bit mask of the axes along which it differences (x = 1, y = 2,
z = 4): on the block's child octant (cx, cy, cz) (0 = lower half, 1 = upper
half of each axis) the sign is the product of (-1)^c over the axes in t.
t = 0 is the approximation (level L only); t = 1..7 are the seven details.

Coefficient vector layout (length nx*ny*nz): the level-L approximations
((nz>>L), (ny>>L), (nx>>L)) z-major, then for l = L, ..., 1 the detail
planes t = 1..7 in that order, each (nz>>l, ny>>l, nx>>l).

Two codings: the level-by-level butterfly (analysis / synthesis) and the
explicit basis matrix from the definition above; the tests pin them
against each other and against orthonormality.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

S3 = 2.0 * np.sqrt(2.0)
OCTANTS = list(itertools.product((0, 1), repeat=3))   # (cz, cy, cx)


def layout(nx: int, ny: int, nz: int, L: int):
    """Planes (level, type, offset, (gz, gy, gx)); type 0 = approximation."""
    for n in (nx, ny, nz):
        if n % (1 << L):
            raise ValueError("volume sides must be divisible by 2^L")
    planes = []
    g = (nz >> L, ny >> L, nx >> L)
    off = 0
    planes.append((L, 0, off, g))
    off += int(np.prod(g))
    for l in range(L, 0, -1):
        g = (nz >> l, ny >> l, nx >> l)
        for t in range(1, 8):
            planes.append((l, t, off, g))
            off += int(np.prod(g))
    assert off == nx * ny * nz
    return planes


def _sign(t, cz, cy, cx):
    s = 1.0
    if t & 1 and cx:
        s = -s
    if t & 2 and cy:
        s = -s
    if t & 4 and cz:
        s = -s
    return s


def analysis(vol: np.ndarray, L: int) -> np.ndarray:
    nz, ny, nx = vol.shape
    a = np.asarray(vol, dtype=np.float64)
    det = {}
    for l in range(1, L + 1):
        ch = {(cz, cy, cx): a[cz::2, cy::2, cx::2] for cz, cy, cx in OCTANTS}
        out = []
        for t in range(8):
            acc = sum(_sign(t, cz, cy, cx) * ch[(cz, cy, cx)] for cz, cy, cx in OCTANTS)
            out.append(acc / S3)
        det[l] = out[1:]
        a = out[0]
    res = [a.ravel()]
    for l in range(L, 0, -1):
        res.extend(p.ravel() for p in det[l])
    return np.concatenate(res)


def synthesis(beta: np.ndarray, nx: int, ny: int, nz: int, L: int) -> np.ndarray:
    planes = layout(nx, ny, nz, L)
    beta = np.asarray(beta, dtype=np.float64)
    _, _, off, g = planes[0]
    a = beta[off:off + int(np.prod(g))].reshape(g)
    k = 1
    for l in range(L, 0, -1):
        coefs = [a]
        for t in range(1, 8):
            _, _, off, g = planes[k]
            coefs.append(beta[off:off + int(np.prod(g))].reshape(g))
            k += 1
        out = np.empty(tuple(2 * s for s in a.shape))
        for cz, cy, cx in OCTANTS:
            out[cz::2, cy::2, cx::2] = sum(_sign(t, cz, cy, cx) * coefs[t] for t in range(8)) / S3
        a = out
    return a


def basis_matrix(nx: int, ny: int, nz: int, L: int) -> sp.csc_matrix:
    """Omega (voxels x coefficients) from the definition of the basis."""
    rows, cols, vals = [], [], []
    for l, t, off, (gz, gy, gx) in layout(nx, ny, nz, L):
        s = 1 << l
        h = s >> 1
        oz, oy, ox = np.meshgrid(np.arange(s), np.arange(s), np.arange(s), indexing="ij")
        sign = np.ones(oz.shape)
        if t & 1:
            sign = sign * np.where(ox >= h, -1.0, 1.0)
        if t & 2:
            sign = sign * np.where(oy >= h, -1.0, 1.0)
        if t & 4:
            sign = sign * np.where(oz >= h, -1.0, 1.0)
        bz, by, bx = np.meshgrid(np.arange(gz), np.arange(gy), np.arange(gx), indexing="ij")
        bz, by, bx = bz.ravel(), by.ravel(), bx.ravel()
        iz = bz[:, None] * s + oz.ravel()[None, :]
        iy = by[:, None] * s + oy.ravel()[None, :]
        ix = bx[:, None] * s + ox.ravel()[None, :]
        rows.append(((iz * ny + iy) * nx + ix).ravel())
        cols.append(np.repeat(off + (bz * gy + by) * gx + bx, s ** 3))
        vals.append(np.tile(sign.ravel() / s ** 1.5, gz * gy * gx))
    N = nx * ny * nz
    return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


def coefficient_info(nx: int, ny: int, nz: int, L: int):
    N = nx * ny * nz
    level = np.empty(N, dtype=np.int64)
    typ = np.empty(N, dtype=np.int64)
    bx = np.empty(N, dtype=np.int64)
    by = np.empty(N, dtype=np.int64)
    bz = np.empty(N, dtype=np.int64)
    for l, t, off, (gz, gy, gx) in layout(nx, ny, nz, L):
        zz, yy, xx = np.meshgrid(np.arange(gz), np.arange(gy), np.arange(gx), indexing="ij")
        sl = slice(off, off + gz * gy * gx)
        level[sl], typ[sl], bx[sl], by[sl], bz[sl] = l, t, xx.ravel(), yy.ravel(), zz.ravel()
    return level, typ, bx, by, bz
