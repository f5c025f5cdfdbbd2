"""GPU parity with rectangular pixels (vy != vx): the projector pair, the
split back-projection of Eq. 1.10, Z0 of Eq. 1.61 and the forward over a tree,
against the FP64 oracle's exact chords on the same geometry.  The back-
projector measures lengths in units of a block's half-width, so the pixel's
aspect ratio enters through its direction table; these cases pin that path."""
import dataclasses

import numpy as np
import pytest

from oracle import am, haar
from oracle import system_matrix as smx
from paper_1508_04458_gb300 import inputs as I

from gpu_helpers import cuda, random_tree, tree_to_masks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1508_04458_gb300 import wam  # noqa: E402

FP32_MAX, FP32_RMS = 1e-4, 1e-5
CASES = {
    # name: (nx, ny, views, bins, kind, L, vy / vx)
    "fan80x48_flat": (80, 48, 37, 131, I.FAN2D_FLAT, 3, 0.6),
    "par64_tall": (64, 64, 30, 97, I.PARALLEL2D, 3, 1.7),
}


def _close(got, want, rel, what):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = max(np.max(np.abs(want)), 1e-300)
    err = np.max(np.abs(got - want)) / scale
    bound = FP32_MAX if rel is None else rel
    assert err <= bound, "%s: max error %.3e of max |ref| (bound %.1e)" % (what, err, bound)
    if rel is None:
        rms = np.sqrt(np.mean((got - want) ** 2)) / scale
        assert rms <= FP32_RMS, "%s: rms error %.3e of max |ref| (bound %.1e)" % (what, rms, FP32_RMS)


def _case(name, seed=5):
    nx, ny, V, B, kind, L, ry = CASES[name]
    p = I.small_problem(nx, ny, V, B, kind=kind, seed=seed)
    # the same scan with pixels ry times as tall (the detector still covers
    # the image for ry <= 1; for ry > 1 the bins are widened to cover it)
    g = dataclasses.replace(p.geom, vy=p.geom.vx * ry,
                            bin_pitch=p.geom.bin_pitch * max(1.0, ry))
    return p, g, smx.system_matrix(g), L


@pytest.mark.parametrize("name", list(CASES))
def test_aniso_project_backproject(name):
    p, g, H, _ = _case(name)
    ctx = wam.Context(g)
    rng = np.random.default_rng(1)
    mu = rng.random(g.nx * g.ny)
    s = rng.random(g.n_views * g.n_bins)
    for dt, rel, proj, back in ((torch.float32, None, wam.wam_project, wam.wam_backproject),
                                (torch.float64, 1e-10, wam.wam_project_f64, wam.wam_backproject_f64)):
        mu_d, s_d = cuda(mu, dt), cuda(s, dt)
        p_d = torch.empty(g.n_views * g.n_bins, dtype=dt, device="cuda")
        g_d = torch.empty(g.nx * g.ny, dtype=dt, device="cuda")
        ctx.check(proj(ctx.h, wam.ptr(mu_d), wam.ptr(p_d), wam.current_stream()))
        ctx.check(back(ctx.h, wam.ptr(s_d), wam.ptr(g_d), wam.current_stream()))
        torch.cuda.synchronize()
        _close(p_d.cpu().numpy(), H @ mu, rel, "H mu (%s)" % dt)
        _close(g_d.cpu().numpy(), H.T @ s, rel, "H^T s (%s)" % dt)
    ctx.close()


@pytest.mark.parametrize("name", list(CASES))
def test_aniso_split_backprojection_z0_forward(name):
    p, g, H, L = _case(name)
    nx, ny = g.nx, g.ny
    ctx = wam.Context(g)
    ctx.set_data(p.d.astype(np.float32), p.I0)
    rng = np.random.default_rng(7)
    tree = random_tree(nx, ny, L, rng, p=0.6)
    masks = tree_to_masks(tree, L)
    act = am.active_mask(tree, nx, ny, L)
    Phi = (H @ haar.basis_matrix(nx, ny, L)).tocsc()
    st = wam.current_stream()
    m_d = cuda(masks)

    # a4: bhat+- of a positive qhat, split by the sign of phi
    q = (p.I0 * np.exp(-rng.random(g.n_views * g.n_bins))).astype(np.float32)
    q_d = cuda(q)
    bp_d = torch.empty(nx * ny, dtype=torch.float64, device="cuda")
    bm_d = torch.empty_like(bp_d)
    ctx.check(wam.wam_split_backproject(ctx.h, L, wam.ptr(m_d), wam.ptr(q_d), wam.ptr(bp_d), wam.ptr(bm_d), st))
    q64 = q.astype(np.float64)
    bp_ref = Phi.maximum(0).T @ q64
    bm_ref = Phi.minimum(0).T @ q64
    bp_ref[~act] = 0.0
    bm_ref[~act] = 0.0
    torch.cuda.synchronize()
    bp, bm = bp_d.cpu().numpy(), bm_d.cpu().numpy()
    _close(np.concatenate([bp, bm]), np.concatenate([bp_ref, bm_ref]), None, "bhat+-")
    assert np.all(bp >= 0) and np.all(bm <= 0)
    assert np.all(bp[~act] == 0) and np.all(bm[~act] == 0)

    # a5: Z0 over the active set
    z_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.check(wam.wam_z0(ctx.h, L, wam.ptr(m_d), wam.ptr(z_d), st))
    z_ref = float(np.max(np.asarray(abs(Phi[:, act]).sum(axis=1))))
    assert abs(float(z_d) - z_ref) <= FP32_MAX * z_ref

    # a2+a3: qhat of an image constant on the tree's leaves
    beta = rng.normal(0.0, 0.01, nx * ny)
    nA = (nx >> L) * (ny >> L)
    beta[:nA] = rng.uniform(0.05, 0.3, nA)
    beta[~act] = 0.0
    mu = haar.basis_matrix(nx, ny, L) @ beta
    mu32 = cuda(mu, torch.float32)
    qf_d = torch.empty(g.n_views * g.n_bins, dtype=torch.float32, device="cuda")
    cost_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.check(wam.wam_forward(ctx.h, L, wam.ptr(m_d), wam.ptr(mu32), wam.ptr(qf_d), wam.ptr(cost_d), st))
    torch.cuda.synchronize()
    q_ref = p.I0 * np.exp(-(H @ mu32.cpu().numpy().astype(np.float64)))
    _close(qf_d.cpu().numpy(), q_ref, None, "qhat")
    ctx.close()
