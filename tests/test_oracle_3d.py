"""Pins of the oracle's 3-D parts: cone-beam intersection lengths, the
orthonormal 3-D Haar transform, the 3-D tree rule and Algorithm 1 in both
3-D modes (3-D Haar, and 2-D Haar per z-slice with the z-summed criterion of
the Results section)."""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import am, haar3d
from oracle import system_matrix as smx
from paper_1508_04458_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_cube_diagonal_and_axis_chords():
    # a 1x1x1 voxel at the origin: the body diagonal is sqrt(3) long inside it;
    # a ray along x through the interior crosses 1 mm
    seg = np.array([[-2.0, -2.0, -2.0, 2.0, 2.0, 2.0], [-3.0, 0.2, -0.1, 3.0, 0.2, -0.1]])
    H = smx.siddon_matrix(seg, (1, 1, 1), (1.0, 1.0, 1.0)).toarray()
    np.testing.assert_allclose(H[:, 0], [math.sqrt(3.0), 1.0], atol=1e-14)


def test_cone_row_sums_are_box_chords():
    p = I.small_problem3d(12, 10, 6, 9, 5, 17)
    g = p.geom
    H = smx.system_matrix(g)
    seg = smx.ray_segments_cone(g)
    lo = np.array([-0.5 * g.nx * g.vx, -0.5 * g.ny * g.vy, -0.5 * g.nz * g.vz])
    want = []
    for s in seg:
        d = s[3:] - s[:3]
        t0, t1 = 0.0, 1.0
        for k in range(3):
            a1, a2 = (lo[k] - s[k]) / d[k] if d[k] else -np.inf, (-lo[k] - s[k]) / d[k] if d[k] else np.inf
            t0, t1 = max(t0, min(a1, a2)), min(t1, max(a1, a2))
        want.append(max(0.0, t1 - t0) * np.linalg.norm(d))
    np.testing.assert_allclose(np.asarray(H.sum(axis=1)).ravel(), want, atol=1e-12)
    assert (np.array(want) > 0).mean() > 0.5


def test_brute_force_4x4x4():
    rng = np.random.default_rng(3)
    n = 4
    nsamp = 200000
    for _ in range(8):
        dvec = rng.standard_normal(3)
        dvec /= np.linalg.norm(dvec)
        p0 = rng.uniform(-1.5, 1.5, 3)
        s = np.concatenate([p0 - 5 * dvec, p0 + 5 * dvec])
        h = smx.siddon_matrix(s[None, :], (n, n, n), (1.0, 1.0, 1.0)).toarray()[0]
        t = (np.arange(nsamp) + 0.5) / nsamp
        pts = s[:3][None, :] + t[:, None] * (s[3:] - s[:3])[None, :]
        idx = np.floor(pts + 2).astype(int)
        ok = np.all((idx >= 0) & (idx < n), axis=1)
        step = 10.0 / nsamp
        est = np.bincount((idx[ok, 2] * n + idx[ok, 1]) * n + idx[ok, 0], minlength=n ** 3) * step
        assert np.max(np.abs(est - h)) < 3 * step


def test_haar3d_hand_example_and_orthonormality():
    g = json.load(open(os.path.join(GOLD, "haar3d_2x2x2.json")))
    vol = np.array(g["volume"])
    b = haar3d.analysis(vol, 1)
    np.testing.assert_allclose(b, g["coefficients"], atol=1e-12)
    for nx, ny, nz, L in [(4, 4, 4, 2), (8, 4, 8, 2), (16, 8, 8, 3)]:
        O = haar3d.basis_matrix(nx, ny, nz, L)
        assert abs(O.T @ O - sp.identity(nx * ny * nz)).max() < 1e-14
        x = np.random.default_rng(nx).standard_normal((nz, ny, nx))
        np.testing.assert_allclose(O.T @ x.ravel(), haar3d.analysis(x, L), atol=1e-12)
        np.testing.assert_allclose(haar3d.synthesis(haar3d.analysis(x, L), nx, ny, nz, L), x, atol=1e-12)


def test_expand3d_rule():
    nx = ny = nz = 8
    L = 2
    S = np.zeros((nz, ny, nx))
    S[1, 2, 6] = 10.0     # block (bz 0, by 0, bx 1) at level 2
    S[6, 5, 1] = 3.0      # block (1, 1, 0)
    S[7, 7, 7] = 0.5      # below 0.1 * max
    t = am.expand3d(am.empty_tree3d(nx, ny, nz, L), S, 0.1)
    assert set(zip(*np.nonzero(t[1]))) == {(0, 0, 1), (1, 1, 0)} and not t[0].any()
    t = am.expand3d(t, S, 0.1)
    assert set(zip(*np.nonzero(t[0]))) == {(0, 1, 3), (3, 2, 0)}
    t2 = am.expand3d(t, S, 0.1)
    assert all(np.array_equal(a, b) for a, b in zip(t, t2))


def test_per_slice_mode_uses_the_z_sum():
    # a feature in one slice only: the shared tree expands where the sum over
    # slices is large, for every slice
    nx = ny = 8
    nz = 4
    L = 2
    S = np.zeros((nz, ny, nx))
    S[2, 1, 1] = 4.0
    S[:, 6, 6] = 1.5      # sum 6 > 4
    t = am.expand(am.empty_tree(nx, ny, L), S.sum(axis=0), 0.9)
    assert t[1][1, 1] and not t[1][0, 0]


@pytest.mark.parametrize("mode", ["3d", "slices"])
def test_monotone_decrease_3d_modes(mode):
    p = I.small_problem3d(16, 16, 8, 20, 6, 24, seed=9)
    H = smx.system_matrix(p.geom)
    if mode == "3d":
        r = am.wavelet_am3d(H, p.d, p.I0, 16, 16, 8, 2, 12, expand_at=(3, 6), taus=(0.1, -1.0))
    else:
        r = am.wavelet_am(H, p.d, p.I0, 16, 16, 2, 12, expand_at=(3, 6), taus=(0.1, -1.0), nz=8)
    assert np.all(np.diff(r.cost) <= 1e-12 * r.cost[:-1])
    assert r.n_active[-1] > r.n_active[0]
    a = am.wavelet_am3d(H, p.d, p.I0, 16, 16, 8, 0, 4)
    b = am.plain_am(H, p.d, p.I0, 4)
    np.testing.assert_allclose(a.beta, b.beta, rtol=1e-12, atol=1e-15)


def test_analytic_3d_bag_integrals_against_point_sampling():
    # the cone-beam data's closed-form integrals (ray/ellipsoid, ray/box,
    # ray/cylinder-rod intervals, painter order on the ray) against midpoint
    # sampling of the painter-ordered 3-D phantom along random segments
    rng = np.random.default_rng(22)
    shapes = I.phantom_bag3d(8, 60.0, 40.0, n_min=8, n_max=12)
    n_rays, h, length = 40, 0.004, 200.0
    P = rng.uniform(-30, 30, (n_rays, 3))
    D = rng.normal(size=(n_rays, 3))
    D /= np.linalg.norm(D, axis=1, keepdims=True)
    seg = np.concatenate([P - 0.5 * length * D, P + 0.5 * length * D], axis=1)
    got = I.painter_line_integrals_3d(shapes, seg)
    t = (np.arange(int(length / h)) + 0.5) * h
    bound = 2 * len(shapes) * h * 1.0 + 1e-9
    for k in range(n_rays):
        X, Y, Z = (seg[k, i] + t * D[k, i] for i in range(3))
        val = np.zeros_like(t)
        for sh in shapes:
            px, py, pz = X - sh.cx, Y - sh.cy, Z - sh.cz
            if sh.kind == "rod":
                w = sh.axis
                pa = px * w[0] + py * w[1] + pz * w[2]
                inside = (px * px + py * py + pz * pz - pa * pa < sh.a * sh.a) & (np.abs(pa) < sh.c)
            else:
                c, s = math.cos(sh.psi), math.sin(sh.psi)
                rx, ry = c * px + s * py, -s * px + c * py
                if sh.kind == "ellipsoid":
                    inside = (rx / sh.a) ** 2 + (ry / sh.b) ** 2 + (pz / sh.c) ** 2 < 1.0
                else:
                    inside = (np.abs(rx) < sh.a) & (np.abs(ry) < sh.b) & (np.abs(pz) < sh.c)
            val[inside] = sh.mu
        assert abs(got[k] - val.sum() * h) <= bound, (k, got[k], val.sum() * h)
    assert np.count_nonzero(got) > n_rays // 2


@pytest.mark.parametrize("vox", [(15, 4, 9), (3, 16, 2)])
def test_cone_hot_voxel_shadow_placement(vox):
    # The cone-beam scan convention, pinned without the oracle's own ray code:
    # the source at SOD e in the plane z = 0, the flat detector through
    # -(SDD - SOD) e spanned by u = (-sin, cos, 0) and z.  By similar triangles
    # a point with a = <P, e>, w = <P, u> and height z meets the detector at
    # (u, v) = SDD (w, z) / (SOD - a).  One hot voxel off centre in x, y and z:
    # at view 0 and a quarter turn later, the rays (row, bin) that cross it are
    # exactly those whose detector point lies inside the convex hull of its
    # eight projected corners.  A detector at -SDD, a flipped row or bin axis,
    # or a half-pitch shift of the row or bin centres moves this set.
    from scipy.spatial import Delaunay
    ix, iy, iz = vox
    nx, ny, nz, sod, sdd = 20, 20, 12, 50.0, 120.0
    g = I.Geometry(kind=I.CONE3D_FLAT_CIRCULAR, nx=nx, ny=ny, nz=nz, n_views=4, angle0=0.0,
                   angle_span=2 * math.pi, n_bins=401, n_rows=201, bin_pitch=0.5, row_pitch=0.5,
                   sod=sod, sdd=sdd)
    vol = np.zeros((nz, ny, nx))
    vol[iz, iy, ix] = 1.0
    proj = (smx.system_matrix(g) @ vol.ravel()).reshape(4, g.n_rows, g.n_bins)
    x0, y0, z0 = -0.5 * nx + ix, -0.5 * ny + iy, -0.5 * nz + iz
    corners = [(x0 + i, y0 + j, z0 + k) for i in (0, 1) for j in (0, 1) for k in (0, 1)]
    ub = (np.arange(g.n_bins) - 0.5 * (g.n_bins - 1)) * g.bin_pitch
    vr = (np.arange(g.n_rows) - 0.5 * (g.n_rows - 1)) * g.row_pitch
    V, U = np.meshgrid(vr, ub, indexing="ij")
    pts = np.stack([U.ravel(), V.ravel()], 1)
    for k in (0, 1):                                   # theta = 0 and pi/2
        th = k * math.pi / 2
        c, s = math.cos(th), math.sin(th)
        shadow = []
        for x, y, z in corners:
            a, w = x * c + y * s, -x * s + y * c
            shadow.append((sdd * w / (sod - a), sdd * z / (sod - a)))
        shadow = np.array(shadow)
        hull = Delaunay(shadow)
        cen = shadow.mean(axis=0)
        # shrink / grow the hull about its centre to keep rays on its edge out
        inside = hull.find_simplex(cen + (pts - cen) / (1 - 1e-6)) >= 0
        near = hull.find_simplex(cen + (pts - cen) / (1 + 1e-6)) >= 0
        got = proj[k].ravel() > 0
        assert inside.sum() >= 9
        assert np.all(got[inside]), k
        assert not np.any(got & ~near), k
