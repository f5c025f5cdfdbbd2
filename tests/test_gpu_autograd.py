"""Differentiation through the method on the GPU (torch.autograd over the
C-ABI) against the FP64 oracle: the projector Phi = H Omega and its adjoint,
the I-divergence + lambda L1(details) gradient, and 10 unrolled AM steps
differentiated with respect to the starting coefficients (per-step
checkpoints), checked against oracle values and FP64 finite differences."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import am, haar
from oracle import system_matrix as smx
from paper_1508_04458_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1508_04458_gb300 import wam  # noqa: E402
from paper_1508_04458_gb300.autograd import AMUnroll, IDivLoss, Operators, PhiProject  # noqa: E402

FP32_MAX, FP32_RMS = 1e-4, 1e-5


def _close(got, want, what, mx=FP32_MAX, rms=FP32_RMS):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    scale = np.max(np.abs(want))
    e = np.abs(got - want)
    assert e.max() <= mx * scale, "%s: max %.3e" % (what, e.max() / scale)
    assert np.sqrt(np.mean(e * e)) <= rms * scale, "%s: rms" % what


def _setup(nx=32, ny=32, V=24, B=45, L=2, seed=13):
    p = I.small_problem(nx, ny, V, B, seed=seed)
    H = smx.system_matrix(p.geom)
    Phi = (H @ haar.basis_matrix(nx, ny, L)).tocsr()
    ctx = wam.Context(p.geom)
    ctx.set_data(p.d.astype(np.float32), p.I0)
    return p, Phi, ctx, Operators(ctx, L)


def _beta(p, L, rng):
    nx, ny = p.geom.nx, p.geom.ny
    nA = (nx >> L) * (ny >> L)
    b = rng.normal(0.0, 0.004, nx * ny)
    b[:nA] = rng.uniform(0.01, 0.04, nA) * (1 << L)
    return b, nA


def _oracle_loss(Phi, p, beta, lam, nA):
    return am.idiv(p.d, p.I0, Phi @ beta) + lam * np.sum(np.abs(beta[nA:]))


def test_projector_function_and_adjoint():
    p, Phi, ctx, ops = _setup()
    rng = np.random.default_rng(1)
    beta, _ = _beta(p, 2, rng)
    bt = torch.tensor(beta, dtype=torch.float32, device="cuda", requires_grad=True)
    pr = PhiProject.apply(bt, ops)
    _close(pr.detach().cpu().numpy(), Phi @ beta.astype(np.float32).astype(np.float64), "Phi beta")
    w = rng.random(Phi.shape[0])
    (pr * torch.tensor(w, dtype=torch.float32, device="cuda")).sum().backward()
    _close(bt.grad.cpu().numpy(), Phi.T @ w.astype(np.float32).astype(np.float64), "Phi^T w")


@pytest.mark.parametrize("lam", [0.0, 5.0])
def test_idiv_loss_gradient(lam):
    p, Phi, ctx, ops = _setup()
    L = 2
    rng = np.random.default_rng(2)
    beta, nA = _beta(p, L, rng)
    beta = beta.astype(np.float32).astype(np.float64)
    bt = torch.tensor(beta, dtype=torch.float32, device="cuda", requires_grad=True)
    loss = IDivLoss.apply(bt, ops, lam)
    loss.backward()
    ref = _oracle_loss(Phi, p, beta, lam, nA)
    assert abs(float(loss.detach()) - ref) <= 1e-5 * ref
    q = p.I0 * np.exp(-(Phi @ beta))
    g_ref = Phi.T @ (p.d.ravel() - q)
    g_ref[nA:] += lam * np.sign(beta[nA:])
    g = bt.grad.cpu().numpy()
    _close(g, g_ref, "dL/dbeta")
    # FP64 finite differences of the oracle's loss along random directions
    for _ in range(3):
        dvec = rng.standard_normal(beta.size)
        eps = 1e-6 / np.linalg.norm(dvec) * np.linalg.norm(beta)
        fd = (_oracle_loss(Phi, p, beta + eps * dvec, lam, nA) -
              _oracle_loss(Phi, p, beta - eps * dvec, lam, nA)) / (2 * eps)
        assert abs(float(g @ dvec) - fd) <= 1e-3 * abs(fd) + 1e-6 * np.abs(g).sum()


def test_unrolled_am_gradient():
    p, Phi, ctx, ops = _setup(nx=32, ny=32, V=24, B=45, L=2, seed=17)
    L, steps, lam = 2, 10, 2.0
    rng = np.random.default_rng(3)
    beta0, nA = _beta(p, L, rng)
    beta0 = beta0.astype(np.float32).astype(np.float64)
    d = torch.tensor(p.d.ravel(), dtype=torch.float32, device="cuda")
    ops.setup(d)

    # oracle: 10 AM steps of Algorithm 1 on the full tree (every coefficient active)
    Pc = Phi.tocsc()
    b = Pc.T @ p.d.ravel()

    def unroll(b0):
        x = b0.copy()
        for _ in range(steps):
            delta, _, _ = am.am_step(Pc, b, x, p.d.ravel(), p.I0)
            x = x + delta
        return x

    def loss_of(b0):
        return _oracle_loss(Phi, p, unroll(b0), lam, nA)

    b10_ref = unroll(beta0)
    bt = torch.tensor(beta0, dtype=torch.float32, device="cuda", requires_grad=True)
    b10 = AMUnroll.apply(bt, ops, steps)
    rel = np.linalg.norm(b10.detach().cpu().numpy() - b10_ref) / np.linalg.norm(b10_ref)
    assert rel <= 1e-4, rel
    loss = IDivLoss.apply(b10, ops, lam)
    loss.backward()
    g = bt.grad.cpu().numpy()
    assert np.all(np.isfinite(g))
    for _ in range(3):
        dvec = rng.standard_normal(beta0.size)
        eps = 1e-5 / np.linalg.norm(dvec) * np.linalg.norm(beta0)
        fd = (loss_of(beta0 + eps * dvec) - loss_of(beta0 - eps * dvec)) / (2 * eps)
        assert abs(float(g @ dvec) - fd) <= 2e-3 * abs(fd) + 1e-5 * np.abs(g).sum(), (float(g @ dvec), fd)


def test_batch_of_eight_256():
    # the differentiation workload's shape: 256x256 fan beam, 360 views x 512 bins, batch 8
    prob = I.problem_fan(256, 360, 512, 1e5, seed=1511)
    L = 4
    ctx = wam.Context(prob.geom)
    ctx.set_data(prob.d.astype(np.float32), prob.I0)
    ops = Operators(ctx, L)
    rng = np.random.default_rng(4)
    betas = np.stack([_beta(prob, L, rng)[0] for _ in range(8)]).astype(np.float32)
    bt = torch.tensor(betas, device="cuda", requires_grad=True)
    losses = IDivLoss.apply(bt, ops, 1.0)
    assert losses.shape == (8,)
    losses.sum().backward()
    # every item equals its single-item evaluation, bit for bit (deterministic kernels)
    for k in (0, 5):
        bk = torch.tensor(betas[k], device="cuda", requires_grad=True)
        lk = IDivLoss.apply(bk, ops, 1.0)
        lk.backward()
        assert float(lk.detach()) == float(losses[k].detach())
        assert torch.equal(bk.grad, bt.grad[k])
    # sampled oracle check of the gradient on a subset of coefficients:
    # dI/dbeta_z = sum_y phi(y|z) (d - q)(y), rows of H built view by view
    g = prob.geom
    nx = ny = 256
    Om = haar.basis_matrix(nx, ny, L)
    zs = rng.choice(nx * ny, 12, replace=False)
    beta = betas[0].astype(np.float64)
    mu = (Om @ beta)
    seg = smx.ray_segments(g)
    acc = np.zeros(zs.size)
    for v0 in range(0, g.n_views, 60):
        rows = slice(v0 * g.n_bins, (v0 + 60) * g.n_bins)
        Hc = smx.siddon_matrix(seg[rows], (nx, ny), (g.vx, g.vy))
        r = prob.d.ravel()[rows] - prob.I0 * np.exp(-(Hc @ mu))
        acc += (Hc @ Om[:, zs]).T @ r
    nA = (nx >> L) * (ny >> L)
    acc += np.where(zs >= nA, 1.0 * np.sign(beta[zs]), 0.0)
    got = bt.grad[0].cpu().numpy()[zs]
    scale = np.max(np.abs(bt.grad[0].cpu().numpy()))
    assert np.max(np.abs(got - acc)) <= FP32_MAX * scale


def test_precompute_b_against_oracle():
    # a0 (Eq. 1.6): b = Phi^T d from the context's data, FP64 output
    p, Phi, ctx, ops = _setup(seed=19)
    ops.setup(torch.tensor(p.d.ravel(), dtype=torch.float32, device="cuda"))
    want = Phi.T @ p.d.ravel().astype(np.float32).astype(np.float64)
    _close(ops._b.cpu().numpy(), want, "b = Phi^T d")


def test_projector_batch_matches_items():
    # the batch calls give each item's single-call result, bit for bit
    p, Phi, ctx, ops = _setup(seed=23)
    rng = np.random.default_rng(5)
    betas = np.stack([_beta(p, 2, rng)[0] for _ in range(3)]).astype(np.float32)
    bt = torch.tensor(betas, device="cuda", requires_grad=True)
    pr = PhiProject.apply(bt, ops)
    w = torch.tensor(rng.random(pr.shape), dtype=torch.float32, device="cuda")
    (pr * w).sum().backward()
    for k in range(3):
        assert torch.equal(pr[k].detach(), ops.phi(bt[k].detach()))
        assert torch.equal(bt.grad[k], ops.phi_t(w[k]))
    _close(pr[1].detach().cpu().numpy(), Phi @ betas[1].astype(np.float64), "Phi beta (batch)")
    empty = ops.phi_batch(torch.zeros(0, ops.N, device="cuda"))
    assert empty.shape == (0, ops.M)


def test_one_step_vjp_against_oracle_jacobian():
    # the transposed Jacobian of one full-tree AM step, applied to gbar,
    # against FP64 central differences of the oracle's step
    p, Phi, ctx, ops = _setup(nx=32, ny=32, V=24, B=45, L=2, seed=29)
    rng = np.random.default_rng(6)
    beta, _ = _beta(p, 2, rng)
    beta = beta.astype(np.float32).astype(np.float64)
    ops.setup(torch.tensor(p.d.ravel(), dtype=torch.float32, device="cuda"))
    Pc = Phi.tocsc()
    b = Pc.T @ p.d.ravel()

    def step(x):
        delta, _, _ = am.am_step(Pc, b, x, p.d.ravel(), p.I0)
        return x + delta

    gbar = rng.standard_normal(beta.size).astype(np.float32)
    got = ops.am_step_vjp(torch.tensor(beta, device="cuda"),
                          torch.tensor(gbar, device="cuda")).cpu().numpy().astype(np.float64)
    for _ in range(3):
        dvec = rng.standard_normal(beta.size)
        eps = 1e-6 / np.linalg.norm(dvec) * np.linalg.norm(beta)
        jd = (step(beta + eps * dvec) - step(beta - eps * dvec)) / (2 * eps)
        want = float(gbar.astype(np.float64) @ jd)
        assert abs(float(got @ dvec) - want) <= 2e-3 * abs(want) + 1e-5 * np.abs(got).sum(), (float(got @ dvec), want)
