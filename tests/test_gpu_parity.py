"""GPU parity: every step of the hot path, called through the C-ABI, against
the FP64 oracle on the same seeded inputs.  Sizes span several CTA tiles and
end in ragged tails (bins not a multiple of 128, block lists not a multiple
of 128 threads, image sides not powers of two).

Tolerances.  FP32 path: a ray's position is held to ~4 ulp of the scan's
coordinates (|x| up to the source distance), i.e. an offset eps of a few
1e-7 of that radius.  A chord through a pixel changes by eps / sin(psi) for a
ray at angle psi to a pixel edge, so the rare rays that graze an edge carry
errors up to ~1e-4 of a chord while the bulk carries ~1e-6.  Single
operators are therefore bounded by RMS <= 1e-5 and max <= 1e-4 relative to
the largest reference entry.  FP64 path: max <= 1e-10.  Integer outputs
(tree masks) bit-exact.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import am, haar
from oracle import system_matrix as smx
from paper_1508_04458_gb300 import inputs as I

from gpu_helpers import cuda, random_tree, tree_to_masks, masks_to_tree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1508_04458_gb300 import wam  # noqa: E402  (fails loudly without libwam)

CASES = {
    # name: (nx, ny, views, bins, kind, L)
    "fan80x48": (80, 48, 37, 131, I.FAN2D_FLAT, 3),
    "par64": (64, 64, 30, 97, I.PARALLEL2D, 3),
    "fan96": (96, 96, 45, 150, I.FAN2D_FLAT, 4),
}


def _case(name, seed=3):
    nx, ny, V, B, kind, L = CASES[name]
    p = I.small_problem(nx, ny, V, B, kind=kind, seed=seed)
    H = smx.system_matrix(p.geom)
    return p, H, L


def _stream():
    return wam.current_stream()


FP32_MAX, FP32_RMS = 1e-4, 1e-5


def _close(got, want, rel, what):
    """rel = None: the FP32 bounds (RMS and max); else max error <= rel."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = max(np.max(np.abs(want)), 1e-300)
    err = np.max(np.abs(got - want)) / scale
    bound = FP32_MAX if rel is None else rel
    assert err <= bound, "%s: max error %.3e of max |ref| (bound %.1e)" % (what, err, bound)
    if rel is None:
        rms = np.sqrt(np.mean((got - want) ** 2)) / scale
        assert rms <= FP32_RMS, "%s: rms error %.3e of max |ref| (bound %.1e)" % (what, rms, FP32_RMS)


@pytest.mark.parametrize("name", list(CASES))
def test_project_and_backproject(name):
    p, H, _ = _case(name)
    g = p.geom
    ctx = wam.Context(g)
    rng = np.random.default_rng(1)
    mu = rng.random(g.nx * g.ny)
    s = rng.random(g.n_views * g.n_bins)
    ref_p = H @ mu
    ref_g = H.T @ s
    for dt, rel, proj, back in ((torch.float32, None, wam.wam_project, wam.wam_backproject),
                                (torch.float64, 1e-10, wam.wam_project_f64, wam.wam_backproject_f64)):
        mu_d, s_d = cuda(mu, dt), cuda(s, dt)
        p_d = torch.empty(g.n_views * g.n_bins, dtype=dt, device="cuda")
        g_d = torch.empty(g.nx * g.ny, dtype=dt, device="cuda")
        ctx.check(proj(ctx.h, wam.ptr(mu_d), wam.ptr(p_d), _stream()))
        ctx.check(back(ctx.h, wam.ptr(s_d), wam.ptr(g_d), _stream()))
        torch.cuda.synchronize()
        _close(p_d.cpu().numpy(), ref_p, rel, "H mu (%s)" % dt)
        _close(g_d.cpu().numpy(), ref_g, rel, "H^T s (%s)" % dt)
    ctx.close()


def test_adjoint_fp64_on_gpu():
    p, H, _ = _case("fan80x48")
    g = p.geom
    ctx = wam.Context(g)
    rng = np.random.default_rng(2)
    x = cuda(rng.random(g.nx * g.ny), torch.float64)
    y = cuda(rng.random(g.n_views * g.n_bins), torch.float64)
    hx = torch.empty_like(y)
    hty = torch.empty_like(x)
    ctx.check(wam.wam_project_f64(ctx.h, wam.ptr(x), wam.ptr(hx), _stream()))
    ctx.check(wam.wam_backproject_f64(ctx.h, wam.ptr(y), wam.ptr(hty), _stream()))
    a, b = float(torch.dot(hx, y)), float(torch.dot(x, hty))
    assert abs(a - b) <= 1e-12 * abs(a)


@pytest.mark.parametrize("L", [1, 3])
def test_haar(L):
    nx, ny = 80, 48
    g = I.Geometry(kind=I.PARALLEL2D, nx=nx, ny=ny, n_views=4, n_bins=8, bin_pitch=20.0)
    ctx = wam.Context(g)
    rng = np.random.default_rng(L)
    x = rng.standard_normal(nx * ny)
    xd = cuda(x, torch.float64)
    b = torch.empty_like(xd)
    back = torch.empty_like(xd)
    ctx.check(wam.wam_haar(ctx.h, L, wam.ptr(xd), wam.ptr(b), 0, _stream()))
    ctx.check(wam.wam_haar(ctx.h, L, wam.ptr(b), wam.ptr(back), 1, _stream()))
    np.testing.assert_allclose(b.cpu().numpy(), haar.analysis(x.reshape(ny, nx), L), rtol=0, atol=1e-13)
    np.testing.assert_allclose(back.cpu().numpy(), x, rtol=0, atol=1e-13)


@pytest.mark.parametrize("name", ["fan80x48", "fan96"])
def test_synthesize_forward_split_z0(name):
    p, H, L = _case(name)
    g = p.geom
    nx, ny = g.nx, g.ny
    ctx = wam.Context(g)
    ctx.set_data(p.d.astype(np.float32), p.I0)
    rng = np.random.default_rng(7)
    tree = random_tree(nx, ny, L, rng, p=0.6)
    masks = tree_to_masks(tree, L)
    act = am.active_mask(tree, nx, ny, L)
    beta = rng.normal(0.0, 0.01, nx * ny)
    beta[: (nx >> L) * (ny >> L)] = rng.uniform(0.05, 0.3, (nx >> L) * (ny >> L))
    beta[~act] = 0.0
    Om = haar.basis_matrix(nx, ny, L)
    Phi = (H @ Om).tocsc()
    st = _stream()
    m_d = cuda(masks)
    b_d = cuda(beta, torch.float64)

    # a1: synthesis over the tree (inactive entries set to garbage must be ignored)
    beta_junk = beta.copy()
    beta_junk[~act] = 1e3
    mu_d = torch.empty(nx * ny, dtype=torch.float32, device="cuda")
    # every device input is held by a name until the kernels have run: a
    # temporary freed early would be recycled by torch's allocator
    junk_d = cuda(beta_junk, torch.float64)
    ctx.check(wam.wam_synthesize(ctx.h, L, wam.ptr(m_d), wam.ptr(junk_d), wam.ptr(mu_d), st))
    mu_ref = Om @ beta
    _close(mu_d.cpu().numpy(), mu_ref, 1e-6, "synthesis")

    # a2+a3: qhat and cost from the leaf projection
    q_d = torch.empty(g.n_views * g.n_bins, dtype=torch.float32, device="cuda")
    cost_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    mu32 = cuda(mu_ref, torch.float32)
    ctx.check(wam.wam_forward(ctx.h, L, wam.ptr(m_d), wam.ptr(mu32), wam.ptr(q_d), wam.ptr(cost_d), st))
    pr = H @ mu32.cpu().numpy().astype(np.float64)
    q_ref = p.I0 * np.exp(-pr)
    torch.cuda.synchronize()
    failures = []

    def soft(fn, *a):
        try:
            fn(*a)
        except AssertionError as e:
            failures.append(str(e))

    qg = q_d.cpu().numpy().astype(np.float64)
    soft(_close, qg, q_ref, None, "qhat")
    c_ref = am.idiv(p.d, p.I0, pr)
    # first order: dI = sum_y (1 - d/q) dq = sum_y (q - d) dp; dp from the qhat error
    dp = np.abs(qg - q_ref) / q_ref
    cbound = 2.0 * np.sum(np.abs(q_ref - p.d.ravel()) * dp) + 1e-9 * c_ref
    if not abs(float(cost_d) - c_ref) <= cbound:
        failures.append("cost %.9e vs %.9e (bound %.3e)" % (float(cost_d), c_ref, cbound))

    # a4: split back-projection of qhat
    qh = q_ref.astype(np.float32)
    bp_d = torch.empty(nx * ny, dtype=torch.float64, device="cuda")
    bm_d = torch.empty(nx * ny, dtype=torch.float64, device="cuda")
    qh_d = cuda(qh)
    ctx.check(wam.wam_split_backproject(ctx.h, L, wam.ptr(m_d), wam.ptr(qh_d), wam.ptr(bp_d),
                                        wam.ptr(bm_d), st))
    q64 = qh.astype(np.float64)
    bp_ref = Phi.maximum(0).T @ q64
    bm_ref = Phi.minimum(0).T @ q64
    bp_ref[~act] = 0.0
    bm_ref[~act] = 0.0
    torch.cuda.synchronize()
    bp, bm = bp_d.cpu().numpy(), bm_d.cpu().numpy()
    soft(_close, np.concatenate([bp, bm]), np.concatenate([bp_ref, bm_ref]), None, "bhat+-")
    if not (np.all(bp[~act] == 0) and np.all(bm[~act] == 0)):
        failures.append("inactive bhat not zero")
    if not (np.all(bp >= 0) and np.all(bm <= 0)):
        failures.append("bhat signs")

    # a5: Z0
    z_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.check(wam.wam_z0(ctx.h, L, wam.ptr(m_d), wam.ptr(z_d), st))
    z_ref = float(np.max(np.asarray(abs(Phi[:, act]).sum(axis=1))))
    if not abs(float(z_d) - z_ref) <= FP32_MAX * z_ref:
        failures.append("Z0 %.9e vs %.9e" % (float(z_d), z_ref))

    # a6: the update on the same b, bhat+-, Z0 (FP64 arithmetic on both sides)
    bvec = Phi.T @ p.d.ravel()
    beta_d = cuda(beta, torch.float64)
    bv_d, bpr_d, bmr_d = (cuda(x, torch.float64) for x in (bvec, bp_ref, bm_ref))
    z0r_d = cuda(np.array([z_ref]), torch.float64)
    ctx.check(wam.wam_update(ctx.h, L, wam.ptr(m_d), wam.ptr(bv_d), wam.ptr(bpr_d), wam.ptr(bmr_d),
                             wam.ptr(z0r_d), 30.0, wam.ptr(beta_d), st))
    torch.cuda.synchronize()
    new_ref = beta.copy()
    new_ref[act] += am.am_root(bvec[act], bp_ref[act], bm_ref[act], z_ref)
    soft(np.testing.assert_allclose, beta_d.cpu().numpy(), new_ref, 1e-12, 1e-15)
    ctx.close()
    assert not failures, "\n".join(failures)


@pytest.mark.parametrize("tau", [0.1, 0.3, -1.0])
def test_expand_bit_exact(tau):
    nx, ny, L = 80, 48, 3
    g = I.Geometry(kind=I.PARALLEL2D, nx=nx, ny=ny, n_views=4, n_bins=8, bin_pitch=20.0)
    ctx = wam.Context(g)
    rng = np.random.default_rng(5)
    tree = random_tree(nx, ny, L, rng, p=0.4)
    S = rng.random((ny, nx)).astype(np.float32) ** 3
    want = am.expand(tree, S.astype(np.float64), tau)
    m_in = cuda(tree_to_masks(tree, L))
    m_out = torch.empty_like(m_in)
    S_d = cuda(S.ravel())
    ctx.check(wam.wam_expand(ctx.h, L, wam.ptr(S_d), tau, wam.ptr(m_in), wam.ptr(m_out), _stream()))
    got = masks_to_tree(m_out.cpu().numpy(), nx, ny, L)
    for l in range(L):
        np.testing.assert_array_equal(got[l], want[l])


def test_plain_am_fp64_parallel64():
    # the 64x64 parallel-beam, plain-AM FP64 workload (water + 2 metal disks, 20 iterations)
    p = I.problem_parallel64()
    H = smx.system_matrix(p.geom)
    ref = am.plain_am(H, p.d, p.I0, 20, shape=(64, 64))
    ctx = wam.Context(p.geom)
    ctx.set_data(p.d.astype(np.float32), p.I0)
    mu, hist, _, st = ctx.reconstruct(0, 20, precision=64, full_am=True)
    assert st == wam.WAM_OK
    rel = np.linalg.norm(mu - ref.mu.ravel()) / np.linalg.norm(ref.mu)
    assert rel <= 1e-10, rel
    np.testing.assert_allclose(hist, ref.cost, rtol=1e-10)


@pytest.mark.parametrize("precision,bound", [(64, 1e-9), (32, 1e-4)])
def test_wavelet_am_matches_oracle(precision, bound):
    p, H, L = _case("fan96", seed=9)
    g = p.geom
    sched = dict(expand_at=(4, 8, 12, 16), tau=(0.1, 0.03, 0.01, -1.0))
    ref = am.wavelet_am(H, p.d, p.I0, g.nx, g.ny, L, 24, **{"expand_at": sched["expand_at"],
                                                              "taus": sched["tau"]})
    ctx = wam.Context(g)
    ctx.set_data(p.d.astype(np.float32), p.I0)
    mu, hist, masks, st = ctx.reconstruct(L, 24, sched["expand_at"], sched["tau"], precision=precision)
    assert st == wam.WAM_OK
    got_tree = masks_to_tree(masks, g.nx, g.ny, L)
    for l in range(L):
        np.testing.assert_array_equal(got_tree[l], ref.tree[l])
    rel = np.linalg.norm(mu.astype(np.float64) - ref.mu.ravel()) / np.linalg.norm(ref.mu)
    assert rel <= bound, rel
    np.testing.assert_allclose(hist, ref.cost, rtol=bound)


def test_plain_am_fp32_matches_oracle():
    p, H, _ = _case("fan80x48")
    ref = am.plain_am(H, p.d, p.I0, 30)
    ctx = wam.Context(p.geom)
    ctx.set_data(p.d.astype(np.float32), p.I0)
    mu, hist, _, st = ctx.reconstruct(0, 30, full_am=True)
    assert st == wam.WAM_OK
    rel = np.linalg.norm(mu.astype(np.float64) - ref.mu) / np.linalg.norm(ref.mu)
    assert rel <= 1e-4, rel
    # the cost is a sum of ~M terms each carrying the FP32 projection error:
    # 1e-4 relative, the same bound as mu
    np.testing.assert_allclose(hist, ref.cost, rtol=1e-4)


def test_errors_are_reported():
    g = I.Geometry(kind=I.PARALLEL2D, nx=48, ny=40, n_views=4, n_bins=8, bin_pitch=20.0)
    ctx = wam.Context(g)
    with pytest.raises(wam.WamError) as e:
        ctx.reconstruct(3, 2)
    assert e.value.status == wam.WAM_ERR_STATE
    ctx.set_data(np.ones((4, 8), np.float32), 10.0)
    with pytest.raises(wam.WamError) as e:
        ctx.reconstruct(4, 2)                       # 40 not divisible by 16
    assert e.value.status == wam.WAM_ERR_ARG
    with pytest.raises(wam.WamError) as e:
        ctx.set_data(-np.ones((4, 8), np.float32), 10.0)
    assert e.value.status == wam.WAM_ERR_ARG
    bad = I.Geometry(kind=I.FAN2D_FLAT, nx=64, ny=64, n_views=4, n_bins=8, bin_pitch=1.0, sod=10.0, sdd=20.0)
    with pytest.raises(wam.WamError):
        wam.Context(bad)
