"""Seeded synthetic inputs: scan geometries, baggage phantoms and Poisson counts.

This module is shared by the CUDA path's callers (benchmark, smoke check) and
the CPU oracle's tests.  It holds none of the reconstruction method's
arithmetic (no system matrix, no wavelet transform, no AM update): it only
describes scans, draws phantoms and simulates transmission counts.

Counts are simulated from the *continuous* phantom: the line integral of the
painter-ordered union of ellipses/rectangles along each ray is computed in
closed form (ray/ellipse quadratic, ray/rectangle slab), then
d ~ Poisson(I0 exp(-integral)).  This is a different discretisation from the
voxel model h(y|x) the method reconstructs with, so the data are not an
"inverse crime".

Ray convention (the same convention is restated, in independent code, by the
oracle and by the CUDA library): view k has angle
theta_k = angle0 + k * angle_span / n_views, e = (cos, sin), u = (-sin, cos);
bin b sits at u_b = (b - (n_bins - 1) / 2) * bin_pitch on the detector axis u.
Parallel beam: the ray is the line {u_b u + t e}.  Fan beam (flat detector):
the ray runs from the source SOD e to the detector point
-(SDD - SOD) e + u_b u.  Rays are indexed y = k * n_bins + b.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

PARALLEL2D = 0
FAN2D_FLAT = 1
CONE3D_FLAT_CIRCULAR = 2


@dataclasses.dataclass
class Geometry:
    """Scan geometry; the field list mirrors the C struct wam_geometry."""
    kind: int
    nx: int
    ny: int
    nz: int = 1
    vx: float = 1.0
    vy: float = 1.0
    vz: float = 1.0
    n_views: int = 1
    angle0: float = 0.0
    angle_span: float = math.pi
    n_bins: int = 1
    n_rows: int = 1
    bin_pitch: float = 1.0
    row_pitch: float = 1.0
    sod: float = 0.0
    sdd: float = 0.0

    @property
    def n_pixels(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_rays(self) -> int:
        return self.n_views * self.n_bins * self.n_rows


@dataclasses.dataclass
class Shape:
    """One object of a painter-ordered phantom (later objects overwrite)."""
    kind: str          # "ellipse" or "rect"
    cx: float
    cy: float
    a: float           # semi-axis along the rotated x axis (mm)
    b: float           # semi-axis along the rotated y axis (mm)
    psi: float         # rotation (rad)
    mu: float          # attenuation (1/mm)


@dataclasses.dataclass
class Problem:
    name: str
    geom: Geometry
    shapes: List[Shape]
    I0: float
    d: np.ndarray              # counts, float64 [n_views][n_bins]
    mu_true: np.ndarray        # 4x4-supersampled raster of the phantom, [ny][nx]
    line_integrals: np.ndarray  # exact integrals of the continuous phantom


# ---------------------------------------------------------------------------
# geometries of the workloads
# ---------------------------------------------------------------------------

def geom_parallel64() -> Geometry:
    """64x64 at 1 mm; 90 views over 180 deg; 96 bins at 1 mm."""
    return Geometry(kind=PARALLEL2D, nx=64, ny=64, vx=1.0, vy=1.0, n_views=90,
                    angle0=0.0, angle_span=math.pi, n_bins=96, bin_pitch=1.0)


def geom_fan(n: int, n_views: int, n_bins: int, bin_pitch: float = 1.2,
             sod: float = 1000.0, sdd: float = 1500.0, pixel: float = 1.0) -> Geometry:
    """Fan beam over 360 deg with a flat detector."""
    return Geometry(kind=FAN2D_FLAT, nx=n, ny=n, vx=pixel, vy=pixel, n_views=n_views,
                    angle0=0.0, angle_span=2.0 * math.pi, n_bins=n_bins,
                    bin_pitch=bin_pitch, sod=sod, sdd=sdd)


def geom_fan512() -> Geometry:
    """512x512 at 1 mm; 720 views over 360 deg; 1024 bins x 1.2 mm; SOD 1000, SDD 1500."""
    return geom_fan(512, 720, 1024)


def geom_fan256() -> Geometry:
    """256x256 at 1 mm; 360 views; 512 bins x 1.2 mm."""
    return geom_fan(256, 360, 512)


# ---------------------------------------------------------------------------
# ray endpoints (data simulation only)
# ---------------------------------------------------------------------------

def _ray_segments_2d(g: Geometry):
    k = np.arange(g.n_views, dtype=np.float64)
    th = g.angle0 + k * g.angle_span / g.n_views
    ex, ey = np.cos(th)[:, None], np.sin(th)[:, None]
    ux, uy = -ey, ex
    ub = ((np.arange(g.n_bins, dtype=np.float64) - (g.n_bins - 1) / 2.0) * g.bin_pitch)[None, :]
    if g.kind == PARALLEL2D:
        T = 2.0 * math.hypot(g.nx * g.vx, g.ny * g.vy) + 10.0
        x1, y1 = ub * ux + T * ex, ub * uy + T * ey
        x2, y2 = ub * ux - T * ex, ub * uy - T * ey
    elif g.kind == FAN2D_FLAT:
        x1 = np.broadcast_to(g.sod * ex, (g.n_views, g.n_bins))
        y1 = np.broadcast_to(g.sod * ey, (g.n_views, g.n_bins))
        x2 = -(g.sdd - g.sod) * ex + ub * ux
        y2 = -(g.sdd - g.sod) * ey + ub * uy
    else:
        raise ValueError("2-D geometry expected")
    return [np.ascontiguousarray(np.broadcast_to(a, (g.n_views, g.n_bins))).ravel()
            for a in (x1, y1, x2, y2)]


# ---------------------------------------------------------------------------
# painter-ordered line integrals of the continuous phantom
# ---------------------------------------------------------------------------

def _shape_intervals(shapes: List[Shape], x1, y1, dx, dy):
    """Entry/exit parameters (t in [0,1] along P1 + t (P2-P1)) of every ray
    with every shape; empty intervals get t0 = t1 = 0."""
    R, K = x1.shape[0], len(shapes)
    t0 = np.zeros((R, K))
    t1 = np.zeros((R, K))
    for k, s in enumerate(shapes):
        c, sn = math.cos(s.psi), math.sin(s.psi)
        px = c * (x1 - s.cx) + sn * (y1 - s.cy)
        py = -sn * (x1 - s.cx) + c * (y1 - s.cy)
        qx = c * dx + sn * dy
        qy = -sn * dx + c * dy
        if s.kind == "ellipse":
            A = (qx / s.a) ** 2 + (qy / s.b) ** 2
            B = 2.0 * (px * qx / s.a ** 2 + py * qy / s.b ** 2)
            C = (px / s.a) ** 2 + (py / s.b) ** 2 - 1.0
            disc = B * B - 4.0 * A * C
            ok = disc > 0.0
            sq = np.sqrt(np.where(ok, disc, 0.0))
            lo = np.where(ok, (-B - sq) / (2.0 * A), 0.0)
            hi = np.where(ok, (-B + sq) / (2.0 * A), 0.0)
        else:
            lo = np.full(R, -np.inf)
            hi = np.full(R, np.inf)
            for p, q, h in ((px, qx, s.a), (py, qy, s.b)):
                with np.errstate(divide="ignore", invalid="ignore"):
                    ta = (-h - p) / q
                    tb = (h - p) / q
                par = q == 0.0
                inside = np.abs(p) < h
                ta = np.where(par, np.where(inside, -np.inf, np.inf), ta)
                tb = np.where(par, np.where(inside, np.inf, -np.inf), tb)
                lo = np.maximum(lo, np.minimum(ta, tb))
                hi = np.minimum(hi, np.maximum(ta, tb))
        lo = np.clip(lo, 0.0, 1.0)
        hi = np.clip(hi, 0.0, 1.0)
        empty = hi <= lo
        t0[:, k] = np.where(empty, 0.0, lo)
        t1[:, k] = np.where(empty, 0.0, hi)
    return t0, t1


def painter_line_integrals(shapes: List[Shape], x1, y1, x2, y2, chunk: int = 4096, device=None) -> np.ndarray:
    """Integral of mu along each segment, where mu at a point is the value of
    the last shape (in list order) containing it, 0 outside all shapes.
    device: evaluate with torch on that device instead (large scans)."""
    R = x1.shape[0]
    out = np.zeros(R)
    if not shapes:
        return out
    if device is not None:
        # the same computation through the 3-D routine with z = 0 and
        # infinitely tall prisms / cylinders along z
        shapes3 = []
        for s in shapes:
            if s.kind == "ellipse":
                shapes3.append(Shape3("ellipsoid", s.cx, s.cy, 0.0, s.a, s.b, 1e9, s.psi, mu=s.mu))
            else:
                shapes3.append(Shape3("box", s.cx, s.cy, 0.0, s.a, s.b, 1e9, s.psi, mu=s.mu))
        seg = np.stack([x1, y1, np.zeros_like(x1), x2, y2, np.zeros_like(x2)], axis=1)
        return painter_line_integrals_3d(shapes3, seg, chunk=65536, device=device)
    mus = np.array([s.mu for s in shapes])
    K = len(shapes)
    for r0 in range(0, R, chunk):
        sl = slice(r0, min(R, r0 + chunk))
        dx, dy = x2[sl] - x1[sl], y2[sl] - y1[sl]
        length = np.hypot(dx, dy)
        t0, t1 = _shape_intervals(shapes, x1[sl], y1[sl], dx, dy)
        pts = np.sort(np.concatenate([t0, t1], axis=1), axis=1)
        mid = 0.5 * (pts[:, 1:] + pts[:, :-1])
        seg = pts[:, 1:] - pts[:, :-1]
        cover = (t0[:, None, :] <= mid[:, :, None]) & (mid[:, :, None] < t1[:, None, :])
        # index of the last covering shape; -1 when none covers
        rev = cover[:, :, ::-1]
        anyc = rev.any(axis=2)
        top = K - 1 - rev.argmax(axis=2)
        val = np.where(anyc, mus[top], 0.0)
        out[sl] = (seg * val).sum(axis=1) * length
    return out


def rasterize(shapes: List[Shape], g: Geometry, ss: int = 4) -> np.ndarray:
    """Pixel averages of the painter-ordered phantom from ss x ss point samples."""
    ox = -0.5 * g.nx * g.vx
    oy = -0.5 * g.ny * g.vy
    sub = (np.arange(ss) + 0.5) / ss
    xs = ox + (np.arange(g.nx)[:, None] + sub[None, :]).ravel() * g.vx
    ys = oy + (np.arange(g.ny)[:, None] + sub[None, :]).ravel() * g.vy
    X, Y = np.meshgrid(xs, ys)
    img = np.zeros_like(X)
    for s in shapes:
        c, sn = math.cos(s.psi), math.sin(s.psi)
        px = c * (X - s.cx) + sn * (Y - s.cy)
        py = -sn * (X - s.cx) + c * (Y - s.cy)
        if s.kind == "ellipse":
            inside = (px / s.a) ** 2 + (py / s.b) ** 2 < 1.0
        else:
            inside = (np.abs(px) < s.a) & (np.abs(py) < s.b)
        img[inside] = s.mu
    return img.reshape(g.ny, ss, g.nx, ss).mean(axis=(1, 3))


# ---------------------------------------------------------------------------
# phantoms
# ---------------------------------------------------------------------------

def phantom_water_metal() -> List[Shape]:
    """Water disk (mu 0.02/mm, r 28 mm) holding two metal disks (0.5/mm, r 3 mm)."""
    return [Shape("ellipse", 0.0, 0.0, 28.0, 28.0, 0.0, 0.02),
            Shape("ellipse", -12.0, 0.0, 3.0, 3.0, 0.0, 0.5),
            Shape("ellipse", 12.0, 0.0, 3.0, 3.0, 0.0, 0.5)]


def phantom_bag(seed: int, half_width: float, n_min: int = 20, n_max: int = 40) -> List[Shape]:
    """Seeded baggage phantom: 20-40 ellipses/rectangles (50/50), rotation
    U[0, pi); plastic U(0.01, 0.03) (p 0.5), liquid 0.02 (p 0.3), both with
    semi-axes U(8, 60) mm; metal U(0.3, 0.8) (p 0.2) with semi-axes U(2, 12) mm.
    Sizes scale with half_width / 256 mm.  Every object lies inside the disk
    of radius 0.96 half_width.  Painter order: non-metal first, then metal."""
    rng = np.random.Generator(np.random.PCG64(seed))
    scale = half_width / 256.0
    n = int(rng.integers(n_min, n_max + 1))
    shapes = []
    for _ in range(n):
        kind = "ellipse" if rng.random() < 0.5 else "rect"
        m = rng.random()
        if m < 0.5:
            mu = float(rng.uniform(0.01, 0.03)); lo, hi, metal = 8.0, 60.0, False
        elif m < 0.8:
            mu = 0.02; lo, hi, metal = 8.0, 60.0, False
        else:
            mu = float(rng.uniform(0.3, 0.8)); lo, hi, metal = 2.0, 12.0, True
        a = float(rng.uniform(lo, hi)) * scale
        b = float(rng.uniform(lo, hi)) * scale
        psi = float(rng.uniform(0.0, math.pi))
        reach = 0.96 * half_width - max(a, b) * (math.sqrt(2.0) if kind == "rect" else 1.0)
        r = reach * math.sqrt(float(rng.random()))
        ang = float(rng.uniform(0.0, 2.0 * math.pi))
        shapes.append((metal, Shape(kind, r * math.cos(ang), r * math.sin(ang), a, b, psi, mu)))
    return [s for metal, s in shapes if not metal] + [s for metal, s in shapes if metal]


def simulate(name: str, g: Geometry, shapes: List[Shape], I0: float, seed: int,
             ss: int = 4, device=None) -> Problem:
    """Poisson counts d ~ Poisson(I0 exp(-line integral)) with a seeded PCG64."""
    x1, y1, x2, y2 = _ray_segments_2d(g)
    li = painter_line_integrals(shapes, x1, y1, x2, y2, device=device)
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.poisson(I0 * np.exp(-li)).astype(np.float64).reshape(g.n_views, g.n_bins)
    return Problem(name, g, shapes, float(I0), d, rasterize(shapes, g, ss),
                   li.reshape(g.n_views, g.n_bins))


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------

SEED_BASE = 1508


def problem_parallel64(seed: int = SEED_BASE + 0) -> Problem:
    """2-D parallel beam, 64x64, water disk with two metal disks, I0 = 1e4."""
    return simulate("parallel64", geom_parallel64(), phantom_water_metal(), 1e4, seed)


def problem_fan512(seed: int = SEED_BASE + 1) -> Problem:
    """2-D fan beam, 512x512, 720 views x 1024 bins, baggage phantom, I0 = 1e5."""
    g = geom_fan512()
    return simulate("fan512", g, phantom_bag(seed, 256.0), 1e5, seed)


def problem_fan(n: int, n_views: int, n_bins: int, I0: float, seed: int,
                bin_pitch: Optional[float] = None, device=None, sod: float = 1000.0,
                sdd: float = 1500.0) -> Problem:
    """A fan-beam bag of any size; the detector covers the image's circumcircle."""
    if bin_pitch is None:
        # half-width of the shadow of the circumscribed circle, x1.03 margin
        r = n * math.sqrt(0.5)
        half = sdd * r / math.sqrt(sod ** 2 - r * r) * 1.03
        bin_pitch = 2.0 * half / n_bins
    g = geom_fan(n, n_views, n_bins, bin_pitch=bin_pitch, sod=sod, sdd=sdd)
    return simulate("fan%d" % n, g, phantom_bag(seed, 0.5 * n), I0, seed, device=device)


def batch_bags(n_bags: int = 32, seed0: int = SEED_BASE + 4, device=None, sizes=(256, 768),
               views=(360, 1440), bins=(512, 1536)) -> List[Problem]:
    """Seeded bags of uneven size: side U{256..768} in steps of 16 (1 mm
    pixels), views U{360..1440}, bins U{512..1536}, I0 log-uniform in
    [1e4, 1e5]; bag i uses seed seed0 + i.  SOD 1000 mm, SDD 1600 mm, so the
    detector stays outside the largest image's circumcircle (543 mm)."""
    out = []
    for i in range(n_bags):
        rng = np.random.Generator(np.random.PCG64(seed0 + i))
        n = int(rng.integers(sizes[0] // 16, sizes[1] // 16 + 1)) * 16
        V = int(rng.integers(views[0], views[1] + 1))
        B = int(rng.integers(bins[0], bins[1] + 1))
        I0 = float(10.0 ** rng.uniform(4.0, 5.0))
        out.append(problem_fan(n, V, B, I0, seed0 + i, device=device, sdd=1600.0))
    return out


def small_problem(nx: int, ny: int, n_views: int, n_bins: int, kind: int = FAN2D_FLAT,
                  I0: float = 1e4, seed: int = 7, pixel: float = 1.0) -> Problem:
    """Small seeded cases for tests (any nx, ny; the detector covers the image)."""
    half = 0.5 * min(nx, ny) * pixel
    shapes = phantom_bag(seed, half, 6, 12)
    r = 0.5 * math.hypot(nx, ny) * pixel
    if kind == PARALLEL2D:
        g = Geometry(kind=PARALLEL2D, nx=nx, ny=ny, vx=pixel, vy=pixel, n_views=n_views,
                     angle0=0.1, angle_span=math.pi, n_bins=n_bins,
                     bin_pitch=2.0 * r * 1.02 / n_bins)
    else:
        sod, sdd = 4.0 * r + 20.0, 6.0 * r + 30.0
        half_det = sdd * r / math.sqrt(sod * sod - r * r) * 1.02
        g = Geometry(kind=FAN2D_FLAT, nx=nx, ny=ny, vx=pixel, vy=pixel, n_views=n_views,
                     angle0=0.05, angle_span=2.0 * math.pi, n_bins=n_bins,
                     bin_pitch=2.0 * half_det / n_bins, sod=sod, sdd=sdd)
    return simulate("small", g, shapes, I0, seed)


# ---------------------------------------------------------------------------
# 3-D circular cone beam
# ---------------------------------------------------------------------------
# Ray (view k, row r, bin b): from the source SOD e (z = 0) to the detector
# point -(SDD - SOD) e + u_b u + v_r z_hat, u_b as above and
# v_r = (r - (n_rows - 1) / 2) * row_pitch.  Ray index (k * n_rows + r) *
# n_bins + b; voxel index (iz * ny + iy) * nx + ix.

def geom_cone(nx: int, ny: int, nz: int, voxel: float, n_views: int, n_rows: int, n_bins: int,
              row_pitch: float, bin_pitch: float, sod: float = 1000.0, sdd: float = 1500.0) -> Geometry:
    return Geometry(kind=CONE3D_FLAT_CIRCULAR, nx=nx, ny=ny, nz=nz, vx=voxel, vy=voxel, vz=voxel,
                    n_views=n_views, angle0=0.0, angle_span=2.0 * math.pi, n_bins=n_bins, n_rows=n_rows,
                    bin_pitch=bin_pitch, row_pitch=row_pitch, sod=sod, sdd=sdd)


def geom_cone256() -> Geometry:
    """256x256x128 at 1.5 mm; 900 views; 64 rows x 5 mm, 768 channels x 1.2 mm."""
    return geom_cone(256, 256, 128, 1.5, 900, 64, 768, 5.0, 1.2)


@dataclasses.dataclass
class Shape3:
    """One object of a painter-ordered 3-D phantom."""
    kind: str          # "ellipsoid", "box" (both rotated by psi about z) or "rod"
    cx: float
    cy: float
    cz: float
    a: float           # semi-axes (ellipsoid, box); rod: radius
    b: float
    c: float           # rod: half-length
    psi: float = 0.0
    axis: tuple = (0.0, 0.0, 1.0)   # rod axis (unit)
    mu: float = 0.0


def ray_segments_3d(g: Geometry) -> np.ndarray:
    """(n_rays, 6) endpoints (x1, y1, z1, x2, y2, z2) of a cone-beam scan."""
    k = np.arange(g.n_views, dtype=np.float64)
    th = g.angle0 + k * g.angle_span / g.n_views
    c, s = np.cos(th)[:, None, None], np.sin(th)[:, None, None]
    ub = ((np.arange(g.n_bins) - (g.n_bins - 1) / 2.0) * g.bin_pitch)[None, None, :]
    vr = ((np.arange(g.n_rows) - (g.n_rows - 1) / 2.0) * g.row_pitch)[None, :, None]
    shape = (g.n_views, g.n_rows, g.n_bins)
    out = np.empty(shape + (6,))
    out[..., 0] = np.broadcast_to(g.sod * c, shape)
    out[..., 1] = np.broadcast_to(g.sod * s, shape)
    out[..., 2] = 0.0
    out[..., 3] = np.broadcast_to(-(g.sdd - g.sod) * c - ub * s, shape)
    out[..., 4] = np.broadcast_to(-(g.sdd - g.sod) * s + ub * c, shape)
    out[..., 5] = np.broadcast_to(vr, shape)
    return out.reshape(-1, 6)


def _intervals_3d(shapes, P1, D, xp):
    """Entry/exit t in [0, 1] of every ray P1 + t D with every shape."""
    R = P1.shape[0]
    if xp is np:
        t0 = np.zeros((R, len(shapes)), dtype=P1.dtype)
        t1 = np.zeros((R, len(shapes)), dtype=P1.dtype)
    else:
        t0 = xp.zeros((R, len(shapes)), dtype=P1.dtype, device=P1.device)
        t1 = xp.zeros((R, len(shapes)), dtype=P1.dtype, device=P1.device)
    for k, sh in enumerate(shapes):
        px, py, pz = P1[:, 0] - sh.cx, P1[:, 1] - sh.cy, P1[:, 2] - sh.cz
        if sh.kind == "rod":
            w = sh.axis
            pa = px * w[0] + py * w[1] + pz * w[2]
            da = D[:, 0] * w[0] + D[:, 1] * w[1] + D[:, 2] * w[2]
            qx, qy, qz = px - pa * w[0], py - pa * w[1], pz - pa * w[2]
            ex, ey, ez = D[:, 0] - da * w[0], D[:, 1] - da * w[1], D[:, 2] - da * w[2]
            A = ex * ex + ey * ey + ez * ez
            B = 2.0 * (qx * ex + qy * ey + qz * ez)
            C = qx * qx + qy * qy + qz * qz - sh.a * sh.a
            disc = B * B - 4.0 * A * C
            ok = (disc > 0.0) & (A > 0.0)
            sq = xp.sqrt(xp.where(ok, disc, 0.0))
            Asafe = xp.where(ok, A, 1.0)
            lo = xp.where(ok, (-B - sq) / (2.0 * Asafe), 0.0)
            hi = xp.where(ok, (-B + sq) / (2.0 * Asafe), 0.0)
            inside_par = (~ok) & (A == 0.0) & (C < 0.0)
            lo = xp.where(inside_par, -1e30, lo)
            hi = xp.where(inside_par, 1e30, hi)
            # end caps: |pa + t da| <= half-length
            dsafe = xp.where(da == 0.0, 1.0, da)
            ta = (-sh.c - pa) / dsafe
            tb = (sh.c - pa) / dsafe
            cin = xp.abs(pa) < sh.c
            ta2 = xp.where(da == 0.0, xp.where(cin, -1e30, 1e30), xp.minimum(ta, tb))
            tb2 = xp.where(da == 0.0, xp.where(cin, 1e30, -1e30), xp.maximum(ta, tb))
            lo = xp.maximum(lo, ta2)
            hi = xp.minimum(hi, tb2)
            hi = xp.where(ok | inside_par, hi, lo)
        else:
            cc, sn = math.cos(sh.psi), math.sin(sh.psi)
            rx = cc * px + sn * py
            ry = -sn * px + cc * py
            dx = cc * D[:, 0] + sn * D[:, 1]
            dy = -sn * D[:, 0] + cc * D[:, 1]
            rz, dz = pz, D[:, 2]
            if sh.kind == "ellipsoid":
                A = (dx / sh.a) ** 2 + (dy / sh.b) ** 2 + (dz / sh.c) ** 2
                B = 2.0 * (rx * dx / sh.a ** 2 + ry * dy / sh.b ** 2 + rz * dz / sh.c ** 2)
                C = (rx / sh.a) ** 2 + (ry / sh.b) ** 2 + (rz / sh.c) ** 2 - 1.0
                disc = B * B - 4.0 * A * C
                ok = disc > 0.0
                sq = xp.sqrt(xp.where(ok, disc, 0.0))
                lo = xp.where(ok, (-B - sq) / (2.0 * A), 0.0)
                hi = xp.where(ok, (-B + sq) / (2.0 * A), 0.0)
            else:
                lo = xp.full_like(rx, -1e30)
                hi = xp.full_like(rx, 1e30)
                for p_, q_, h_ in ((rx, dx, sh.a), (ry, dy, sh.b), (rz, dz, sh.c)):
                    qs = xp.where(q_ == 0.0, 1.0, q_)
                    ta = (-h_ - p_) / qs
                    tb = (h_ - p_) / qs
                    inside = xp.abs(p_) < h_
                    ta2 = xp.where(q_ == 0.0, xp.where(inside, -1e30, 1e30), xp.minimum(ta, tb))
                    tb2 = xp.where(q_ == 0.0, xp.where(inside, 1e30, -1e30), xp.maximum(ta, tb))
                    lo = xp.maximum(lo, ta2)
                    hi = xp.minimum(hi, tb2)
        lo = xp.clip(lo, 0.0, 1.0)
        hi = xp.clip(hi, 0.0, 1.0)
        empty = hi <= lo
        t0[:, k] = xp.where(empty, 0.0, lo)
        t1[:, k] = xp.where(empty, 0.0, hi)
    return t0, t1


def painter_line_integrals_3d(shapes, seg, chunk: int = 20000, device=None) -> np.ndarray:
    """Line integrals of a painter-ordered 3-D phantom along segments
    (n, 6); numpy, or torch on `device` (plumbing for large scans)."""
    R = seg.shape[0]
    out = np.zeros(R)
    if not shapes:
        return out
    if device is None:
        xp = np
        mus = np.array([s.mu for s in shapes])
    else:
        import torch as xp
        mus = xp.tensor([s.mu for s in shapes], dtype=xp.float64, device=device)
    K = len(shapes)
    for r0 in range(0, R, chunk):
        sl = slice(r0, min(R, r0 + chunk))
        if device is None:
            P1 = seg[sl, :3]
            D = seg[sl, 3:] - P1
        else:
            s_ = xp.tensor(seg[sl], dtype=xp.float64, device=device)
            P1 = s_[:, :3]
            D = s_[:, 3:] - P1
        length = (D * D).sum(1) ** 0.5
        t0, t1 = _intervals_3d(shapes, P1, D, xp)
        if device is None:
            pts = np.sort(np.concatenate([t0, t1], axis=1), axis=1)
        else:
            pts = xp.sort(xp.cat([t0, t1], dim=1), dim=1).values
        mid = 0.5 * (pts[:, 1:] + pts[:, :-1])
        segl = pts[:, 1:] - pts[:, :-1]
        cover = (t0[:, None, :] <= mid[:, :, None]) & (mid[:, :, None] < t1[:, None, :])
        if device is None:
            rev = cover[:, :, ::-1]
            anyc = rev.any(axis=2)
            top = K - 1 - rev.argmax(axis=2)
            val = np.where(anyc, mus[top], 0.0)
            out[sl] = (segl * val).sum(axis=1) * length
        else:
            idx = xp.arange(K, device=device)
            top = xp.where(cover, idx, -1).max(dim=2).values
            val = xp.where(top >= 0, mus[top.clamp(min=0)], xp.zeros((), dtype=xp.float64, device=device))
            out[sl] = ((segl * val).sum(dim=1) * length).cpu().numpy()
    return out


def phantom_bag3d(seed: int, radius: float, zhalf: float, n_min: int = 20, n_max: int = 40,
                  rods: tuple = (2, 6)) -> List[Shape3]:
    """Seeded 3-D bag: 20-40 boxes/ellipsoids (50/50, rotated about z) inside
    a cylinder of the given radius and half-height, materials as in the 2-D
    bag (sizes scaled by radius / 170 mm), then 2-6 metal rods (radius
    2-6 mm, length 40-150 mm, random direction).  Painter order: non-metal,
    metal objects, rods."""
    rng = np.random.Generator(np.random.PCG64(seed))
    scale = radius / 170.0
    n = int(rng.integers(n_min, n_max + 1))
    objs = []
    for _ in range(n):
        kind = "ellipsoid" if rng.random() < 0.5 else "box"
        m = rng.random()
        if m < 0.5:
            mu = float(rng.uniform(0.01, 0.03)); lo, hi, metal = 8.0, 60.0, False
        elif m < 0.8:
            mu = 0.02; lo, hi, metal = 8.0, 60.0, False
        else:
            mu = float(rng.uniform(0.3, 0.8)); lo, hi, metal = 2.0, 12.0, True
        a, b = (float(rng.uniform(lo, hi)) * scale for _ in range(2))
        c = min(float(rng.uniform(lo, hi)) * scale, 0.9 * zhalf)
        psi = float(rng.uniform(0.0, math.pi))
        ext = max(a, b) * (math.sqrt(2.0) if kind == "box" else 1.0)
        rr = max(0.0, 0.96 * radius - ext) * math.sqrt(float(rng.random()))
        ang = float(rng.uniform(0.0, 2.0 * math.pi))
        cz = float(rng.uniform(-1.0, 1.0)) * max(0.0, 0.96 * zhalf - c)
        objs.append((metal, Shape3(kind, rr * math.cos(ang), rr * math.sin(ang), cz, a, b, c, psi, mu=mu)))
    shapes = [s for metal, s in objs if not metal] + [s for metal, s in objs if metal]
    for _ in range(int(rng.integers(rods[0], rods[1] + 1))):
        rad = float(rng.uniform(2.0, 6.0)) * scale
        half = 0.5 * float(rng.uniform(40.0, 150.0)) * scale
        w = rng.standard_normal(3)
        w /= np.linalg.norm(w)
        reach = max(0.0, 0.96 * radius - half - rad)
        rr = reach * math.sqrt(float(rng.random()))
        ang = float(rng.uniform(0.0, 2.0 * math.pi))
        zr = max(0.0, 0.96 * zhalf - half * abs(w[2]) - rad)
        cz = float(rng.uniform(-1.0, 1.0)) * zr
        shapes.append(Shape3("rod", rr * math.cos(ang), rr * math.sin(ang), cz, rad, rad, half,
                             axis=tuple(float(x) for x in w), mu=float(rng.uniform(0.3, 0.8))))
    return shapes


def rasterize3d(shapes, g: Geometry, ss: int = 2) -> np.ndarray:
    """Voxel averages of the painter-ordered phantom from ss^3 samples."""
    sub = (np.arange(ss) + 0.5) / ss
    ax = [(-0.5 * n * v + (np.arange(n)[:, None] + sub[None, :]).ravel() * v)
          for n, v in ((g.nx, g.vx), (g.ny, g.vy), (g.nz, g.vz))]
    out = np.zeros((g.nz, g.ny, g.nx))
    Y, X = np.meshgrid(ax[1], ax[0], indexing="ij")
    for kz in range(g.nz):
        acc = np.zeros((g.ny * ss, g.nx * ss))
        for j in range(ss):
            Z = ax[2][kz * ss + j]
            img = np.zeros_like(X)
            for sh in shapes:
                px, py, pz = X - sh.cx, Y - sh.cy, Z - sh.cz
                if sh.kind == "rod":
                    w = sh.axis
                    pa = px * w[0] + py * w[1] + pz * w[2]
                    d2 = px * px + py * py + pz * pz - pa * pa
                    inside = (d2 < sh.a * sh.a) & (np.abs(pa) < sh.c)
                else:
                    cc, sn = math.cos(sh.psi), math.sin(sh.psi)
                    rx, ry = cc * px + sn * py, -sn * px + cc * py
                    if sh.kind == "ellipsoid":
                        inside = (rx / sh.a) ** 2 + (ry / sh.b) ** 2 + (pz / sh.c) ** 2 < 1.0
                    else:
                        inside = (np.abs(rx) < sh.a) & (np.abs(ry) < sh.b) & (abs(pz) < sh.c)
                img[inside] = sh.mu
            acc += img
        out[kz] = (acc / ss).reshape(g.ny, ss, g.nx, ss).mean(axis=(1, 3))
    return out


def simulate3d(name: str, g: Geometry, shapes, I0: float, seed: int, device=None,
               raster: bool = True) -> Problem:
    seg = ray_segments_3d(g)
    li = painter_line_integrals_3d(shapes, seg, device=device)
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.poisson(I0 * np.exp(-li)).astype(np.float64).reshape(g.n_views, g.n_rows * g.n_bins)
    mu = rasterize3d(shapes, g) if raster else np.zeros((0,))
    return Problem(name, g, shapes, float(I0), d, mu, li.reshape(g.n_views, g.n_rows * g.n_bins))


def problem_cone256(seed: int = SEED_BASE + 2, device=None) -> Problem:
    """3-D cone beam: 256x256x128 at 1.5 mm, 900 views, 64 x 768, I0 = 5e4."""
    g = geom_cone256()
    return simulate3d("cone256", g, phantom_bag3d(seed, 170.0, 90.0), 5e4, seed, device=device, raster=False)


def small_problem3d(nx: int, ny: int, nz: int, n_views: int, n_rows: int, n_bins: int,
                    I0: float = 1e4, seed: int = 7, voxel: float = 1.0) -> Problem:
    """Small seeded cone-beam cases for tests; the detector covers the volume."""
    r = 0.5 * math.hypot(nx, ny) * voxel
    zh = 0.5 * nz * voxel
    sod, sdd = 4.0 * r + 20.0, 6.0 * r + 30.0
    half_det = sdd * r / math.sqrt(sod * sod - r * r) * 1.02
    half_row = sdd * zh / (sod - r) * 1.02
    g = geom_cone(nx, ny, nz, voxel, n_views, n_rows, n_bins, 2.0 * half_row / n_rows, 2.0 * half_det / n_bins,
                  sod=sod, sdd=sdd)
    g.angle0 = 0.05
    shapes = phantom_bag3d(seed, 0.45 * min(nx, ny) * voxel, 0.45 * nz * voxel, 4, 8, rods=(1, 2))
    return simulate3d("small3d", g, shapes, I0, seed)
