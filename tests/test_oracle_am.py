"""Pins of the oracle's Algorithm 1 (unregularised wavelet AM) and plain AM:
the closed-form root against bracketing on Eq. 1.9, the surrogate of Eq. 1.8
majorising the cost, closed-form fixed points, the textbook AM log-ratio,
monotone decrease (Summary: guaranteed decrease at every iteration), the
expansion rule of the Results section, and Phi = H Omega against closed-form
chords through the children of a Haar block."""
import json
import math
import os

import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp
import scipy.stats as st

from oracle import am, haar
from oracle import system_matrix as smx
from paper_1508_04458_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def eq19(delta, b, bp, bm, Z0):
    return b - bp * math.exp(-Z0 * delta) - bm * math.exp(Z0 * delta)


def test_root_matches_bracketing_on_eq19():
    rng = np.random.default_rng(0)
    n = 400
    b = rng.standard_normal(n) * 10.0 ** rng.uniform(-2, 3, n)
    bp = rng.uniform(0, 1, n) * 10.0 ** rng.uniform(-2, 3, n)
    bm = -rng.uniform(0, 1, n) * 10.0 ** rng.uniform(-2, 3, n)
    bm[::5] = 0.0                       # approximation-like coefficients
    Z0 = 37.5
    got = am.am_root(b, bp, bm, Z0)
    for i in range(n):
        if bm[i] == 0.0 and b[i] <= 0.0:
            assert got[i] == pytest.approx(am.CLAMP / Z0)
            continue
        ref = so.brentq(eq19, -am.CLAMP / Z0, am.CLAMP / Z0, args=(b[i], bp[i], bm[i], Z0),
                        xtol=1e-300, rtol=1e-15, maxiter=500) \
            if np.sign(eq19(-am.CLAMP / Z0, b[i], bp[i], bm[i], Z0)) != \
            np.sign(eq19(am.CLAMP / Z0, b[i], bp[i], bm[i], Z0)) else None
        if ref is None:
            assert abs(got[i]) == pytest.approx(am.CLAMP / Z0)
        else:
            assert got[i] == pytest.approx(ref, rel=1e-10, abs=1e-13)


def test_root_degenerate_cases():
    Z0 = 2.0
    # nothing sees the coefficient
    assert am.am_root([0.0], [0.0], [0.0], Z0)[0] == 0.0
    # only negative weights: u = bm / b
    assert am.am_root([-3.0], [0.0], [-1.5], Z0)[0] == pytest.approx(-math.log(0.5) / Z0)
    # minimiser at +infinity (b <= 0, no negative part) and -infinity
    assert am.am_root([-1.0], [2.0], [0.0], Z0)[0] == pytest.approx(am.CLAMP / Z0)
    assert am.am_root([1.0], [0.0], [-2.0], Z0)[0] == pytest.approx(-am.CLAMP / Z0)
    # plain AM: bm = 0 gives the log-ratio
    assert am.am_root([2.0], [5.0], [0.0], Z0)[0] == pytest.approx(math.log(5.0 / 2.0) / Z0)


def test_idiv_is_poisson_log_likelihood_ratio():
    # Sec. II: minimising I(d||q) is maximising the Poisson log-likelihood;
    # I(d||q) = log P(d | mean d) - log P(d | mean q)
    rng = np.random.default_rng(1)
    q = rng.uniform(0.5, 50, 300)
    d = rng.poisson(q).astype(float)
    d[:7] = 0.0
    I0 = 60.0
    p = np.log(I0 / q)
    ll = st.poisson.logpmf(d, q).sum()
    ll_sat = st.poisson.logpmf(d, np.where(d > 0, d, 1e-300)).sum()
    assert am.idiv(d, I0, p) == pytest.approx(ll_sat - ll, rel=1e-10)
    assert am.idiv(d[d > 0], I0, np.log(I0 / d[d > 0])) == pytest.approx(0.0, abs=1e-9)


def _small(kind=I.FAN2D_FLAT, nx=32, ny=24, V=30, B=41, seed=7):
    p = I.small_problem(nx, ny, V, B, kind=kind, seed=seed)
    return p, smx.system_matrix(p.geom)


def test_single_pixel_fixed_point():
    # one 1x1 mm pixel, rays through it with h = 1 (horizontal and vertical
    # lines through its interior); equal counts d: the ML estimate is
    # mu* = ln(I0 / d) / h, reached by AM in one step (Z0 = 1)
    seg = np.array([[-2.0, y, 2.0, y] for y in (-0.3, 0.0, 0.2)] +
                   [[x, -2.0, x, 2.0] for x in (-0.4, 0.1)])
    H = smx.siddon_matrix(seg, (1, 1), (1.0, 1.0))
    np.testing.assert_allclose(H.toarray().ravel(), 1.0)
    I0, dbar = 1000.0, 250.0
    r = am.plain_am(H, np.full(5, dbar), I0, 3)
    assert r.beta[0] == pytest.approx(math.log(I0 / dbar), rel=1e-14)
    assert r.cost[-1] == pytest.approx(0.0, abs=1e-9)


def test_plain_am_first_step_is_textbook_log_ratio():
    # Omega = I: mu1 = mu0 + (1/Z0) ln(H^T qhat / H^T d) with qhat = I0 at mu0 = 0,
    # Z0 = max_y sum_x h(y|x) = the longest chord through the image
    p, H = _small(kind=I.PARALLEL2D)
    r = am.plain_am(H, p.d, p.I0, 1)
    ones = np.full(H.shape[0], p.I0)
    b = H.T @ p.d.ravel()
    bq = H.T @ ones
    seen = b > 0
    Z0 = np.max(np.asarray(H.sum(axis=1)))
    np.testing.assert_allclose(r.beta[seen], np.log(bq[seen] / b[seen]) / Z0, rtol=1e-12)
    g = p.geom
    lo = (-0.5 * g.nx * g.vx, -0.5 * g.ny * g.vy)
    # the longest chord of any ray through the image rectangle (slab clipping)
    best = 0.0
    for s in smx.ray_segments(g):
        d = s[2:] - s[:2]
        t0, t1 = 0.0, 1.0
        for k in range(2):
            if d[k] != 0:
                a1, a2 = (lo[k] - s[k]) / d[k], (-lo[k] - s[k]) / d[k]
                t0, t1 = max(t0, min(a1, a2)), min(t1, max(a1, a2))
        best = max(best, max(0.0, t1 - t0) * np.linalg.norm(d))
    assert r.z0[0] == pytest.approx(best, rel=1e-12)


def test_wavelet_am_with_no_levels_is_plain_am():
    p, H = _small()
    a = am.plain_am(H, p.d, p.I0, 6)
    w = am.wavelet_am(H, p.d, p.I0, p.geom.nx, p.geom.ny, 0, 6)
    np.testing.assert_allclose(w.beta, a.beta, rtol=1e-12, atol=1e-15)


def _surrogate(Ps, b_s, beta_hat, beta, qhat, Z0):
    """F^(beta) of Eq. 1.8 up to the constant: sum_z b beta + sum_y qhat *
    [sum_z r exp(-(phi/r)(beta - beta_hat)) + (1 - sum_z r)], r = |phi|/Z0."""
    P = Ps.toarray()
    r = np.abs(P) / Z0
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(r > 0, P / np.where(r > 0, r, 1.0), 0.0)
    ex = r * np.exp(-ratio * (beta - beta_hat)[None, :])
    return b_s @ beta + qhat @ (ex.sum(axis=1) + 1.0 - r.sum(axis=1))


def test_surrogate_majorises_and_update_minimises_it():
    p, H = _small(nx=16, ny=16, V=20, B=29)
    nx, ny, L = 16, 16, 2
    Om = haar.basis_matrix(nx, ny, L)
    Phi = (H @ Om).tocsc()
    d = p.d.ravel()
    b = Phi.T @ d
    tree = am.empty_tree(nx, ny, L)
    tree[1][0, 1] = tree[1][1, 1] = True
    tree[0][0, 2] = True
    act = am.active_mask(tree, nx, ny, L)
    Ps = Phi[:, act]
    rng = np.random.default_rng(2)
    beta_hat = rng.normal(0.0, 0.05, act.sum())
    beta_hat[: (nx >> L) * (ny >> L)] = 0.08
    qhat = p.I0 * np.exp(-(Ps @ beta_hat))
    Z0 = float(np.max(np.asarray(abs(Ps).sum(axis=1))))

    def F(beta):  # the cost minus its beta-independent constant
        return b[act] @ beta + np.sum(p.I0 * np.exp(-(Ps @ beta)))

    Fh = _surrogate(Ps, b[act], beta_hat, beta_hat, qhat, Z0)
    assert Fh == pytest.approx(F(beta_hat), rel=1e-12)
    for _ in range(20):
        beta = beta_hat + rng.normal(0, 0.02, beta_hat.size)
        assert _surrogate(Ps, b[act], beta_hat, beta, qhat, Z0) >= F(beta) - 1e-9 * abs(F(beta))
    delta, cost, z0 = am.am_step(Ps, b[act], beta_hat, d, p.I0)
    assert z0 == pytest.approx(Z0)
    new = beta_hat + delta
    # the update is the surrogate's minimiser: no coordinate move lowers it
    s0 = _surrogate(Ps, b[act], beta_hat, new, qhat, Z0)
    for k in rng.choice(new.size, 25, replace=False):
        for h in (1e-4, -1e-4):
            e = new.copy()
            e[k] += h
            assert _surrogate(Ps, b[act], beta_hat, e, qhat, Z0) >= s0 - 1e-9 * abs(s0)
    assert F(new) <= F(beta_hat)


@pytest.mark.parametrize("kind", [I.PARALLEL2D, I.FAN2D_FLAT])
def test_monotone_decrease_with_expansions(kind):
    p, H = _small(kind=kind, nx=32, ny=32, V=36, B=49, seed=11)
    r = am.wavelet_am(H, p.d, p.I0, 32, 32, 3, 30, expand_at=(5, 10, 20), taus=(0.1, 0.03, -1.0))
    assert np.all(np.diff(r.cost) <= 1e-12 * r.cost[:-1])
    assert r.n_active[0] == 16 and r.n_active[-1] > r.n_active[0]
    assert len(r.trees) == 3
    a = am.plain_am(H, p.d, p.I0, 30)
    assert np.all(np.diff(a.cost) <= 1e-12 * a.cost[:-1])


def test_noiseless_block_constant_object_is_recovered():
    # data consistent with a block-constant mu_true (in the span of the
    # level-L approximations): coarse AM drives mu towards mu_true and the
    # surrogate gradient b - bhat+ - bhat- towards 0
    nx = ny = 16
    L = 2
    g = I.Geometry(kind=I.PARALLEL2D, nx=nx, ny=ny, n_views=24, angle0=0.1,
                   angle_span=math.pi, n_bins=31, bin_pitch=0.8)
    H = smx.system_matrix(g)
    rng = np.random.default_rng(4)
    blocks = rng.uniform(0.01, 0.05, (ny >> L, nx >> L))
    mu_true = np.kron(blocks, np.ones((1 << L, 1 << L)))
    I0 = 1e4
    d = I0 * np.exp(-(H @ mu_true.ravel()))
    r1 = am.wavelet_am(H, d, I0, nx, ny, L, 20)
    r2 = am.wavelet_am(H, d, I0, nx, ny, L, 200)
    e1 = np.linalg.norm(r1.mu - mu_true)
    e2 = np.linalg.norm(r2.mu - mu_true)
    assert e2 < 0.5 * e1 and e2 < 0.05 * np.linalg.norm(mu_true)
    assert r2.cost[-1] < 1e-4 * r2.cost[0]


def test_expansion_golden():
    g = json.load(open(os.path.join(GOLD, "expand_8x8.json")))
    ny, nx = g["shape"]
    L = g["L"]
    S = np.zeros((ny, nx))
    for y, x, v in g["S_nonzero"]:
        S[y, x] = v
    tree = am.empty_tree(nx, ny, L)
    for step in g["after_step"]:
        tree = am.expand(tree, S, g["tau"])
        for lev, key in ((2, "level2"), (1, "level1")):
            want = np.zeros_like(tree[lev - 1])
            for by, bx in step[key]:
                want[by, bx] = True
            np.testing.assert_array_equal(tree[lev - 1], want)


def test_phi_equals_child_chords():
    # phi(y|z) for a level-l detail = 2^-l sum_k s_k chord(y, child_k): the
    # children are 2^(l-1)-pixel squares; chords by slab clipping
    p, H = _small(nx=32, ny=32, V=12, B=45)
    g = p.geom
    nx, ny, L = 32, 32, 3
    Phi = (H @ haar.basis_matrix(nx, ny, L)).tocsc()
    seg = smx.ray_segments(g)
    ox, oy = -0.5 * nx, -0.5 * ny

    def chord(s, x0, y0, w):
        d = s[2:] - s[:2]
        t0, t1 = 0.0, 1.0
        for k, (lo, hi) in enumerate(((x0, x0 + w), (y0, y0 + w))):
            if d[k] == 0:
                if not lo <= s[k] < hi:
                    return 0.0
                continue
            a1, a2 = (lo - s[k]) / d[k], (hi - s[k]) / d[k]
            t0, t1 = max(t0, min(a1, a2)), min(t1, max(a1, a2))
        return max(0.0, t1 - t0) * np.linalg.norm(d)

    level, typ, bx, by = haar.coefficient_info(nx, ny, L)
    rng = np.random.default_rng(9)
    for z in rng.choice(nx * ny, 60, replace=False):
        l, t = int(level[z]), int(typ[z])
        s = 1 << l
        h = s // 2
        x0, y0 = ox + bx[z] * s, oy + by[z] * s
        col = Phi[:, z].toarray().ravel()
        for y in range(0, H.shape[0], 7):
            c = [chord(seg[y], x0 + i * h, y0 + j * h, h) for j in (0, 1) for i in (0, 1)]
            # c = [ylo-xlo, ylo-xhi, yhi-xlo, yhi-xhi]
            if t == -1:
                want = sum(c) / s
            elif t == 0:
                want = (c[0] + c[1] - c[2] - c[3]) / s
            elif t == 1:
                want = (c[0] - c[1] + c[2] - c[3]) / s
            else:
                want = (c[0] - c[1] - c[2] + c[3]) / s
            assert col[y] == pytest.approx(want, abs=1e-12)


# ---------------------------------------------------------------------------
# ordered subsets
# ---------------------------------------------------------------------------

def test_view_subsets_partition_interleaved():
    subs = am.view_subsets(10, 3)
    assert [list(x) for x in subs] == [[0, 3, 6, 9], [1, 4, 7], [2, 5, 8]]
    assert sorted(np.concatenate(am.view_subsets(37, 4)).tolist()) == list(range(37))


def test_one_subset_is_algorithm_1():
    p = I.small_problem(16, 16, 12, 25, seed=81)
    H = smx.system_matrix(p.geom)
    kw = dict(expand_at=(2, 4), taus=(0.1, -1.0))
    ref = am.wavelet_am(H, p.d, p.I0, 16, 16, 2, 6, **kw)
    os1 = am.os_wavelet_am(H, p.d, p.I0, 16, 16, 2, 6, 1, p.geom.n_bins, **kw)
    np.testing.assert_allclose(os1.beta, ref.beta, rtol=0, atol=1e-14 * np.abs(ref.beta).max())
    np.testing.assert_allclose(os1.cost, ref.cost, rtol=1e-14)
    for t1, t2 in zip(os1.tree, ref.tree):
        np.testing.assert_array_equal(t1, t2)


def test_each_subset_step_decreases_its_own_cost_and_subset_z0_is_bounded():
    p = I.small_problem(16, 16, 12, 25, seed=82)
    H = smx.system_matrix(p.geom)
    r = am.os_wavelet_am(H, p.d, p.I0, 16, 16, 2, 5, 4, p.geom.n_bins, expand_at=(2,), taus=(0.05,))
    # a sub-step minimises a majoriser of the subset's own I-divergence (Eq. 1.8 on the subset)
    assert np.all(r.sub_cost[:, :, 1] <= r.sub_cost[:, :, 0] * (1 + 1e-12))
    # Z0 of a subset is a max over fewer rays than the full Z0 of the same tree
    Phi = (H @ haar.basis_matrix(16, 16, 2)).tocsr()
    act = am.active_mask(am.empty_tree(16, 16, 2), 16, 16, 2)
    z_full = np.max(np.asarray(abs(Phi[:, act]).sum(axis=1)).ravel())
    assert np.all(r.z0[0] <= z_full * (1 + 1e-15)) and np.isclose(r.z0[0].max(), z_full, rtol=1e-15)


def test_os_single_pixel_reaches_the_fixed_point_in_one_sub_step():
    # one pixel, every ray of the same length h and the same counts: the first
    # sub-step lands on mu* = ln(I0 / d) / h, later sub-steps stay there
    h, I0, dv, n = 3.0, 1e4, 2500.0, 12
    H = sp.csr_matrix(np.full((n, 1), h))
    r = am.os_wavelet_am(H, np.full(n, dv), I0, 1, 1, 0, 3, 3, 1)
    assert abs(r.beta[0] - np.log(I0 / dv) / h) <= 1e-14


def test_nonneg_plain_am_minimises_the_surrogate_over_nonnegative_images():
    # low counts, so that unconstrained AM drives background pixels negative
    p, H = _small(nx=16, ny=16, V=20, B=29, seed=11)
    rng = np.random.default_rng(12)
    I0 = 30.0
    d = rng.poisson(I0 * np.exp(-p.line_integrals.ravel())).astype(np.float64)
    free = am.plain_am(H, d, I0, 30)
    assert free.mu.min() < -1e-4
    nn = am.plain_am(H, d, I0, 30, nonneg=True)
    assert nn.mu.min() >= 0.0
    assert np.all(np.diff(nn.cost) <= 1e-12 * nn.cost[:-1])
    # the oracle's clamped step from an iterate with pixels at the bound equals
    # the minimiser over mu >= 0 of the surrogate of Eq. 1.8 (Omega = I), found
    # by a generic bounded quasi-Newton search on the surrogate's own formula
    Hc = H.tocsc()
    b = Hc.T @ d
    mu_hat = am.plain_am(H, d, I0, 12, nonneg=True).mu
    assert np.sum(mu_hat == 0.0) > 0
    delta, _, Z0 = am.am_step(Hc, b, mu_hat, d, I0)
    step = np.maximum(mu_hat + delta, 0.0)
    qhat = I0 * np.exp(-(Hc @ mu_hat))
    Hd = H.toarray()
    r = Hd / Z0

    def F(mu):
        ex = r * np.exp(-Z0 * (mu - mu_hat)[None, :])
        val = b @ mu + qhat @ (ex.sum(axis=1) + 1.0 - r.sum(axis=1))
        grad = b - Z0 * (qhat @ ex)
        return val, grad

    res = so.minimize(F, mu_hat, jac=True, method="L-BFGS-B", bounds=[(0.0, None)] * mu_hat.size,
                      options=dict(ftol=1e-15, gtol=1e-12, maxiter=5000))
    np.testing.assert_allclose(res.x, step, atol=2e-6 * max(1.0, np.abs(step).max()))
    assert np.any((step == 0.0) & (mu_hat + delta < 0.0))   # the bound is active somewhere


# ---------------------------------------------------------------------------
# the L1-penalised step (Eq. 1.1 with R = l1 norm of the detail coefficients)
# ---------------------------------------------------------------------------

def _penalised_1d(delta, b, bp, bm, Z0, beta_hat, lam):
    """The one-coefficient surrogate of Eq. 1.8 (up to a constant) plus the
    penalty: b D + (bp exp(-Z0 D) - bm exp(Z0 D)) / Z0 + lam |beta_hat + D|;
    its derivative in D is Eq. 1.9 plus lam sign(beta_hat + D)."""
    return b * delta + (bp * math.exp(-Z0 * delta) - bm * math.exp(Z0 * delta)) / Z0 + lam * abs(beta_hat + delta)


def test_l1_root_minimises_the_penalised_surrogate():
    rng = np.random.default_rng(12)
    n = 300
    Z0 = 20.0
    b = rng.standard_normal(n) * 10.0 ** rng.uniform(-1, 2, n)
    bp = rng.uniform(0.1, 1, n) * 10.0 ** rng.uniform(-1, 2, n)
    bm = -rng.uniform(0.1, 1, n) * 10.0 ** rng.uniform(-1, 2, n)
    beta_hat = rng.normal(0, 0.05, n)
    beta_hat[::7] = 0.0
    lam = 10.0 ** rng.uniform(-2, 2, n)
    got = am.am_root_l1(b, bp, bm, Z0, beta_hat, lam, clamp=np.inf)
    for i in range(n):
        f = lambda x: _penalised_1d(x, b[i], bp[i], bm[i], Z0, beta_hat[i], lam[i])
        ref = so.minimize_scalar(f, bounds=(-3.0, 3.0), method="bounded",
                                 options={"xatol": 1e-13, "maxiter": 2000}).x
        assert f(got[i]) <= f(ref) + 1e-10 * (1 + abs(f(ref)))
        # the kink: beta lands exactly on 0 when neither one-sided root is admissible
        if abs(beta_hat[i] + got[i]) < 1e-300:
            assert beta_hat[i] + got[i] == 0.0
    # lam = 0 is the unpenalised root of Eq. 1.9
    np.testing.assert_allclose(am.am_root_l1(b, bp, bm, Z0, beta_hat, 0.0), am.am_root(b, bp, bm, Z0),
                               rtol=1e-14, atol=1e-300)


def test_l1_root_soft_threshold_at_zero():
    # from beta_hat = 0 with |g(0)| = |b - bp - bm| <= lam the coefficient stays 0
    Z0 = 5.0
    b, bp, bm = np.array([1.0, 1.0, 1.0]), np.array([0.8, 0.8, 0.8]), np.array([-0.1, -0.1, -0.1])
    g0 = 1.0 - 0.8 + 0.1
    d = am.am_root_l1(b, bp, bm, Z0, 0.0, np.array([g0 * 1.01, g0 * 0.5, 0.0]))
    assert d[0] == 0.0
    assert d[1] < 0.0 and d[1] > d[2]          # shrunk toward 0 relative to the unpenalised step


def test_penalised_wavelet_am_decreases_its_objective():
    p, H = _small(nx=32, ny=32, V=36, B=53)
    L = 3
    for lam in (1.0, 30.0):
        r = am.wavelet_am(H, p.d, p.I0, 32, 32, L, 14, expand_at=(3, 6, 9), taus=(0.1, 0.03, -1.0), lam=lam)
        assert np.all(np.diff(r.cost) <= 1e-12 * r.cost[:-1])
        # the reported objective is the data term plus the penalty of the same beta
        Phi = H @ haar.basis_matrix(32, 32, L)
        want = am.idiv(p.d, p.I0, Phi @ r.beta) + lam * am.l1_details(r.beta, 32, 32, L)
        assert r.cost[-1] == pytest.approx(want, rel=1e-12)
    r0 = am.wavelet_am(H, p.d, p.I0, 32, 32, L, 6, expand_at=(3,), taus=(0.1,), lam=0.0)
    r1 = am.wavelet_am(H, p.d, p.I0, 32, 32, L, 6, expand_at=(3,), taus=(0.1,))
    assert np.array_equal(r0.beta, r1.beta)
    # a penalty larger than every detail gradient keeps every detail at 0
    big = am.wavelet_am(H, p.d, p.I0, 32, 32, L, 8, expand_at=(2,), taus=(-1.0,), lam=1e12)
    _, typ, _, _ = haar.coefficient_info(32, 32, L)
    assert np.all(big.beta[typ >= 0] == 0.0)
