"""GPU parity of the regularised method (Eq. 1.1 with lambda R(mu) =
lambda * the l1 norm of the detail coefficients; wam_schedule.lambda)
against the FP64 oracle (am.wavelet_am with lam, am.am_root_l1):

* the penalised step of one coefficient (wam_am_delta with lambda) against
  am_root_l1: FP64 to 1e-12 (1 + |Z0 Delta|), FP32 within the bound of the
  unpenalised FP32 root, 5e-7 (1 + |Z0 Delta|) (the kink decision compares
  two such roots with -Z0 beta, continuous across it); beta = 0 exactly
  where the oracle puts it there;
* Algorithm 1 with the penalty on a fan-beam case with four expansions:
  mu within 1e-4 (FP32) / 1e-9 (FP64), the history of
  I(d || qhat) + lambda sum |beta_detail| within 1e-4 / 1e-9 and
  non-increasing, trees bit-exact, and every detail coefficient that the
  oracle sets to exactly 0 is exactly 0 on the GPU (FP64);
* a penalty above every detail gradient keeps every detail at 0;
* checkpoint / resume with lambda is bit-exact, and a resume with another
  lambda is refused; lambda with plain AM, or negative, is refused.
"""
import numpy as np
import pytest

from oracle import am, haar
from oracle import system_matrix as smx
from paper_1508_04458_gb300 import inputs as I

from gpu_helpers import masks_to_tree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1508_04458_gb300 import wam  # noqa: E402

NX, NY, V, B, L, J = 96, 80, 45, 150, 3, 20
EXP, TAU = (3, 6, 10, 14), (0.1, 0.03, 0.01, -1.0)
CLAMP = 30.0


@pytest.fixture(scope="module")
def case():
    p = I.small_problem(NX, NY, V, B, seed=9)
    return p, smx.system_matrix(p.geom)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("precision", [64, 32])
def test_penalised_root_against_oracle(precision):
    rng = np.random.default_rng(31)
    n = 100000
    z0 = 412.5
    scale = 10.0 ** rng.uniform(-6, 4, n)
    bp = (scale * rng.random(n)).astype(np.float32).astype(np.float64)
    bm = (-scale * 10.0 ** rng.uniform(-3, 3, n) * rng.random(n)).astype(np.float32).astype(np.float64)
    b = ((bp + bm) * (1 + 10.0 ** rng.uniform(-6, 0, n) * rng.choice([-1, 1], n))).astype(np.float32)
    b = b.astype(np.float64)
    beta = rng.normal(0, 1e-3, n) * (rng.random(n) < 0.8)
    lam = scale * 10.0 ** rng.uniform(-3, 1, n)
    lam_one = float(np.median(lam))
    want = am.am_root_l1(b, bp, bm, z0, beta, lam_one, CLAMP)
    tb, tp, tm, tbeta = _dev(b), _dev(bp), _dev(bm), _dev(beta)
    delta = torch.empty_like(tb)
    rc = wam.wam_am_delta(n, wam.ptr(tb), wam.ptr(tp), wam.ptr(tm), wam.ptr(tbeta), lam_one, z0, CLAMP, precision,
                          wam.ptr(delta), 0, wam.current_stream())
    assert rc == wam.WAM_OK
    got = delta.cpu().numpy()
    err = np.abs(got - want) * z0
    tw = np.abs(want) * z0
    bound = (1e-12 if precision == 64 else 5e-7) * (1.0 + tw)
    worst = int(np.argmax(err / bound))
    assert np.all(err <= bound), (err[worst], bound[worst], b[worst], bp[worst], bm[worst], beta[worst])
    zero_ref = beta + want == 0.0
    assert zero_ref.sum() > 100                     # the kink is exercised
    if precision == 64:
        np.testing.assert_array_equal(beta[zero_ref] + got[zero_ref], 0.0)


@pytest.mark.parametrize("precision", [32, 64])
def test_penalised_reconstruction_against_oracle(case, precision):
    p, H = case
    lam = 1000.0                  # zeroes about a fifth of the active details on this scan
    ref = am.wavelet_am(H, p.d, p.I0, NX, NY, L, J, expand_at=EXP, taus=TAU, lam=lam)
    ctx = wam.Context(p.geom)
    ctx.set_data(p.d.astype(np.float32), p.I0)
    mu, hist, masks, st = ctx.reconstruct(L, J, EXP, TAU, precision=precision, lam=lam)
    assert st == wam.WAM_OK, st
    tree = masks_to_tree(masks, NX, NY, L)
    for l in range(L):
        np.testing.assert_array_equal(tree[l], ref.tree[l])
    tol = 1e-4 if precision == 32 else 1e-9
    rel = np.linalg.norm(mu.astype(np.float64).ravel() - ref.mu.ravel()) / np.linalg.norm(ref.mu)
    assert rel <= tol, rel
    np.testing.assert_allclose(hist, ref.cost, rtol=tol)
    assert np.all(np.diff(hist) <= (1e-6 if precision == 32 else 1e-11) * hist[:-1])
    # the penalty acts: fewer nonzero details than the unpenalised run's
    free = am.wavelet_am(H, p.d, p.I0, NX, NY, L, J, expand_at=EXP, taus=TAU)
    _, typ, _, _ = haar.coefficient_info(NX, NY, L)
    assert np.count_nonzero(ref.beta[typ >= 0]) < 0.9 * np.count_nonzero(free.beta[typ >= 0])
    ctx.close()


def test_huge_penalty_keeps_details_at_zero(case):
    p, H = case
    ctx = wam.Context(p.geom)
    ctx.set_data(p.d.astype(np.float32), p.I0)
    mu, hist, masks, st = ctx.reconstruct(L, 8, (2,), (-1.0,), precision=64, lam=1e12)
    ref = am.wavelet_am(H, p.d, p.I0, NX, NY, L, 8, expand_at=(2,), taus=(-1.0,), lam=1e12)
    # mu is then block-constant on the 8x8 approximation blocks
    blocks = mu.reshape(NY // 8, 8, NX // 8, 8)
    assert np.all(blocks == blocks[:, :1, :, :1])
    np.testing.assert_allclose(mu.ravel(), ref.mu.ravel(), rtol=1e-9, atol=1e-12)
    ctx.close()


def test_penalised_resume_and_refusals(case, tmp_path):
    p, _ = case
    lam = 1000.0

    def ctx():
        c = wam.Context(p.geom)
        c.set_data(p.d.astype(np.float32), p.I0)
        return c

    a = ctx()
    mu_full, h_full, m_full, _ = a.reconstruct(L, J, EXP, TAU, lam=lam)
    a.reconstruct(L, 8, EXP, TAU, lam=lam)
    path = str(tmp_path / "l1.ckpt")
    a.checkpoint(path)
    b = ctx()
    b.resume(path)
    mu, h, m, _ = b.reconstruct(L, J, EXP, TAU, lam=lam)
    np.testing.assert_array_equal(mu, mu_full)
    np.testing.assert_array_equal(h, h_full)
    np.testing.assert_array_equal(m, m_full)
    c = ctx()
    c.resume(path)
    with pytest.raises(wam.WamError) as e:
        c.reconstruct(L, J, EXP, TAU, lam=1.0)
    assert e.value.status == wam.WAM_ERR_STATE
    for kw in (dict(full_am=True), dict(lam=-1.0)):
        lam_kw = kw.pop("lam", 1.0)
        with pytest.raises(wam.WamError) as e:
            a.reconstruct(0 if kw else L, 4, lam=lam_kw, **kw)
        assert e.value.status == wam.WAM_ERR_ARG
    for x in (a, b, c):
        x.close()
