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


def painter_line_integrals(shapes: List[Shape], x1, y1, x2, y2, chunk: int = 4096) -> np.ndarray:
    """Integral of mu along each segment, where mu at a point is the value of
    the last shape (in list order) containing it, 0 outside all shapes."""
    R = x1.shape[0]
    out = np.zeros(R)
    if not shapes:
        return out
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
             ss: int = 4) -> Problem:
    """Poisson counts d ~ Poisson(I0 exp(-line integral)) with a seeded PCG64."""
    x1, y1, x2, y2 = _ray_segments_2d(g)
    li = painter_line_integrals(shapes, x1, y1, x2, y2)
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
                bin_pitch: Optional[float] = None) -> Problem:
    """A fan-beam bag of any size; the detector covers the image's circumcircle."""
    if bin_pitch is None:
        # half-width of the shadow of the circumscribed circle, x1.03 margin
        r = n * math.sqrt(0.5)
        half = 1500.0 * r / math.sqrt(1000.0 ** 2 - r * r) * 1.03
        bin_pitch = 2.0 * half / n_bins
    g = geom_fan(n, n_views, n_bins, bin_pitch=bin_pitch)
    return simulate("fan%d" % n, g, phantom_bag(seed, 0.5 * n), I0, seed)


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
