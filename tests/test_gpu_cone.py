"""GPU parity of the 3-D circular cone-beam path through the C-ABI against the
FP64 oracle: H and H^T, plain AM on voxels, Algorithm 1 with the 3-D Haar
tree and with the per-slice 2-D Haar tree (z-summed criterion), and sampled
rays of the full-size 256x256x128 projector.  FP32 bounds as in the 2-D
parity tests (RMS <= 1e-5, max <= 1e-4 of max |ref| for single operators,
1e-4 relative for iterates); trees bit-exact.  The FP32 cost's error is
first order, sum |d - q| |dp|, about constant in absolute terms while the cost
falls, so cost histories are bounded by 1e-4 relative plus 2e-5 of the
initial cost."""
import numpy as np
import pytest

from oracle import am
from oracle import system_matrix as smx
from paper_1508_04458_gb300 import inputs as I

from gpu_helpers import cuda, tree_to_masks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1508_04458_gb300 import wam  # noqa: E402

FP32_MAX, FP32_RMS = 1e-4, 1e-5


def _close(got, want, what):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    scale = np.max(np.abs(want))
    e = np.abs(got - want)
    assert e.max() <= FP32_MAX * scale, "%s: max %.3e" % (what, e.max() / scale)
    assert np.sqrt(np.mean(e * e)) <= FP32_RMS * scale, "%s: rms %.3e" % (what, np.sqrt(np.mean(e * e)) / scale)


def _case(nx=20, ny=16, nz=12, V=24, R=7, B=33, seed=5):
    p = I.small_problem3d(nx, ny, nz, V, R, B, seed=seed)
    return p, smx.system_matrix(p.geom)


def test_cone_project_backproject():
    p, H = _case()
    g = p.geom
    ctx = wam.Context(g)
    rng = np.random.default_rng(1)
    mu = rng.random(H.shape[1])
    s = rng.random(H.shape[0])
    mu_d, s_d = cuda(mu, torch.float32), cuda(s, torch.float32)
    p_d = torch.empty(H.shape[0], dtype=torch.float32, device="cuda")
    g_d = torch.empty(H.shape[1], dtype=torch.float32, device="cuda")
    st = wam.current_stream()
    ctx.check(wam.wam_project(ctx.h, wam.ptr(mu_d), wam.ptr(p_d), st))
    ctx.check(wam.wam_backproject(ctx.h, wam.ptr(s_d), wam.ptr(g_d), st))
    torch.cuda.synchronize()
    _close(p_d.cpu().numpy(), H @ mu.astype(np.float32).astype(np.float64), "H mu")
    _close(g_d.cpu().numpy(), H.T @ s.astype(np.float32).astype(np.float64), "H^T s")
    # 2-D-only step calls are refused on a cone context
    assert wam.wam_z0(ctx.h, 1, 0, 0, st) == wam.WAM_ERR_ARG


def test_cone_plain_am():
    p, H = _case(seed=6)
    ref = am.plain_am(H, p.d, p.I0, 12)
    ctx = wam.Context(p.geom)
    ctx.set_data(p.d.astype(np.float32), p.I0)
    mu, hist, _, st = ctx.reconstruct(0, 12, full_am=True)
    assert st == wam.WAM_OK
    rel = np.linalg.norm(mu.astype(np.float64) - ref.mu) / np.linalg.norm(ref.mu)
    assert rel <= 1e-4, rel
    np.testing.assert_allclose(hist, ref.cost, rtol=1e-4, atol=2e-5 * ref.cost[0])


def test_cone_wavelet_am_3d_haar():
    p, H = _case(nx=16, ny=16, nz=8, V=24, R=6, B=29, seed=7)
    L, J, ea, tau = 2, 14, (3, 7), (0.1, -1.0)
    ref = am.wavelet_am3d(H, p.d, p.I0, 16, 16, 8, L, J, expand_at=ea, taus=tau)
    ctx = wam.Context(p.geom)
    ctx.set_data(p.d.astype(np.float32), p.I0)
    mu, hist, masks, st = ctx.reconstruct(L, J, ea, tau, dims=3)
    assert st == wam.WAM_OK
    want = np.concatenate([ref.tree[l - 1].astype(np.uint8).ravel() for l in range(L, 0, -1)])
    np.testing.assert_array_equal(masks, want)
    rel = np.linalg.norm(mu.astype(np.float64) - ref.mu.ravel()) / np.linalg.norm(ref.mu)
    assert rel <= 1e-4, rel
    np.testing.assert_allclose(hist, ref.cost, rtol=1e-4, atol=2e-5 * ref.cost[0])


def test_cone_wavelet_am_per_slice():
    # the paper's own 3-D setting: 2-D Haar on every z-slice, one tree,
    # the criterion summed over slices
    p, H = _case(nx=16, ny=16, nz=6, V=24, R=6, B=29, seed=8)
    L, J, ea, tau = 2, 14, (3, 7), (0.1, 0.05)
    ref = am.wavelet_am(H, p.d, p.I0, 16, 16, L, J, expand_at=ea, taus=tau, nz=6)
    ctx = wam.Context(p.geom)
    ctx.set_data(p.d.astype(np.float32), p.I0)
    mu, hist, masks, st = ctx.reconstruct(L, J, ea, tau, dims=2, zsum=True)
    assert st == wam.WAM_OK
    np.testing.assert_array_equal(masks, tree_to_masks(ref.tree, L))
    rel = np.linalg.norm(mu.astype(np.float64) - ref.mu.ravel()) / np.linalg.norm(ref.mu)
    assert rel <= 1e-4, rel
    np.testing.assert_allclose(hist, ref.cost, rtol=1e-4, atol=2e-5 * ref.cost[0])


def test_cone256_projector_sampled_rays():
    # the full 256x256x128, 900-view, 64x768 scan: sampled rays of H mu
    g = I.geom_cone256()
    ctx = wam.Context(g)
    rng = np.random.default_rng(2)
    mu = rng.random((g.nz, g.ny, g.nx)).astype(np.float32) * 0.03
    mu_d = torch.from_numpy(mu.ravel()).cuda()
    M = g.n_views * g.n_rows * g.n_bins
    p_d = torch.empty(M, dtype=torch.float32, device="cuda")
    ctx.check(wam.wam_project(ctx.h, wam.ptr(mu_d), wam.ptr(p_d), wam.current_stream()))
    torch.cuda.synchronize()
    rays = rng.choice(M, 300, replace=False)
    seg = smx.ray_segments_cone(g)[rays]
    Hs = smx.siddon_matrix(seg, (g.nx, g.ny, g.nz), (g.vx, g.vy, g.vz))
    ref = Hs @ mu.ravel().astype(np.float64)
    got = p_d.cpu().numpy()[rays].astype(np.float64)
    assert np.max(np.abs(got - ref)) <= FP32_MAX * np.max(np.abs(ref))
