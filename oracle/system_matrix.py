"""Oracle: the system matrix H of the forward model, FP64.

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the
benchmark).  Shares no code with the CUDA path.

Sec. II (Introduction): q(mu)(y) = I0(y) exp(-sum_x h(y|x) mu(x)) with
h(y|x) the length of the intersection of ray path y with voxel x.  H is built
explicitly, row by row, by Siddon's method (oracle/siddon.c) and stored as a
scipy CSR matrix with rows y = view * n_bins + bin and columns
x = iy * nx + ix.

Scan convention (restated here independently of the other modules): view k
has angle theta_k = angle0 + k * angle_span / n_views, e = (cos, sin),
u = (-sin, cos); bin b lies at u_b = (b - (n_bins - 1)/2) * bin_pitch on the
detector axis u.  Parallel beam: the ray is the line through u_b u with
direction e.  Flat-detector fan beam: the segment from the source SOD e to
-(SDD - SOD) e + u_b u.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import scipy.sparse as sp

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        for name in ("or_siddon_counts", "or_siddon_fill"):
            getattr(_lib, name).restype = None
    return _lib


def ray_segments(g) -> np.ndarray:
    """(n_rays, 4) array of segment endpoints (x1, y1, x2, y2), 2-D scans."""
    th = g.angle0 + np.arange(g.n_views, dtype=np.float64) * (g.angle_span / g.n_views)
    e = np.stack([np.cos(th), np.sin(th)], axis=1)            # (V, 2)
    u = np.stack([-np.sin(th), np.cos(th)], axis=1)
    ub = (np.arange(g.n_bins, dtype=np.float64) - 0.5 * (g.n_bins - 1)) * g.bin_pitch
    seg = np.empty((g.n_views, g.n_bins, 4))
    if g.kind == 0:
        reach = 2.0 * math.hypot(g.nx * g.vx, g.ny * g.vy) + 10.0
        mid = ub[None, :, None] * u[:, None, :]               # (V, B, 2)
        seg[..., 0:2] = mid + reach * e[:, None, :]
        seg[..., 2:4] = mid - reach * e[:, None, :]
    elif g.kind == 1:
        seg[..., 0:2] = (g.sod * e)[:, None, :]
        seg[..., 2:4] = (-(g.sdd - g.sod) * e)[:, None, :] + ub[None, :, None] * u[:, None, :]
    else:
        raise ValueError("2-D scan expected")
    return seg.reshape(-1, 4)


def siddon_matrix(seg: np.ndarray, shape, size) -> sp.csr_matrix:
    """CSR matrix of intersection lengths of segments with a voxel grid.

    seg: (R, 2*dims) endpoints; shape: (nx, ny[, nz]); size: voxel edge lengths.
    """
    lib = _load()
    dims = len(shape)
    seg = np.ascontiguousarray(seg, dtype=np.float64)
    R = seg.shape[0]
    n = (ctypes.c_int * 3)(*list(shape) + [1] * (3 - dims))
    v = (ctypes.c_double * 3)(*list(size) + [1.0] * (3 - dims))
    counts = np.zeros(R, dtype=np.int64)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int64)
    lib.or_siddon_counts(ctypes.c_int(dims), ctypes.c_int64(R), seg.ctypes.data_as(dp), n, v,
                         counts.ctypes.data_as(ip))
    rowptr = np.zeros(R + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    cols = np.zeros(int(rowptr[-1]), dtype=np.int64)
    vals = np.zeros(int(rowptr[-1]), dtype=np.float64)
    lib.or_siddon_fill(ctypes.c_int(dims), ctypes.c_int64(R), seg.ctypes.data_as(dp), n, v,
                       rowptr.ctypes.data_as(ip), cols.ctypes.data_as(ip), vals.ctypes.data_as(dp))
    N = int(np.prod(shape))
    return sp.csr_matrix((vals, cols, rowptr), shape=(R, N))


def ray_segments_cone(g) -> np.ndarray:
    """(n_rays, 6) segments of a circular cone-beam scan: from the source
    SOD e (z = 0) to the flat-detector point -(SDD - SOD) e + u_b u + v_r z,
    v_r = (r - (n_rows - 1)/2) * row_pitch; rays indexed
    (view * n_rows + row) * n_bins + bin."""
    th = g.angle0 + np.arange(g.n_views, dtype=np.float64) * (g.angle_span / g.n_views)
    ub = (np.arange(g.n_bins, dtype=np.float64) - 0.5 * (g.n_bins - 1)) * g.bin_pitch
    vr = (np.arange(g.n_rows, dtype=np.float64) - 0.5 * (g.n_rows - 1)) * g.row_pitch
    seg = np.zeros((g.n_views, g.n_rows, g.n_bins, 6))
    c = np.cos(th)[:, None, None]
    s = np.sin(th)[:, None, None]
    seg[..., 0] = g.sod * c
    seg[..., 1] = g.sod * s
    seg[..., 3] = -(g.sdd - g.sod) * c - ub[None, None, :] * s
    seg[..., 4] = -(g.sdd - g.sod) * s + ub[None, None, :] * c
    seg[..., 5] = vr[None, :, None]
    return seg.reshape(-1, 6)


def system_matrix(g) -> sp.csr_matrix:
    """H for a 2-D scan (rays x pixels) or a cone-beam scan (rays x voxels)."""
    if g.kind == 2:
        return siddon_matrix(ray_segments_cone(g), (g.nx, g.ny, g.nz), (g.vx, g.vy, g.vz))
    return siddon_matrix(ray_segments(g), (g.nx, g.ny), (g.vx, g.vy))
