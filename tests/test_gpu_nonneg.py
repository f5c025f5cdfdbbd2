"""Plain AM kept nonnegative (wam_schedule.nonneg): each pixel's (voxel's)
step ends at mu = 0, the exact minimiser of the separable surrogate over
mu >= 0, as the oracle's plain_am(nonneg=True) does (pinned on the CPU against
a bounded minimisation of the surrogate).  GPU against the oracle on
low-count scans where unconstrained AM goes negative: 2-D pixel quads and odd
sides (single pixels) in FP32 and FP64, and the 3-D voxel basis; a Haar tree
is refused; a checkpoint keeps the flag (resume bit-exact, a mismatch
refused)."""
import numpy as np
import pytest

from oracle import am
from oracle import system_matrix as smx
from paper_1508_04458_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1508_04458_gb300 import wam  # noqa: E402


def _lowcount(p, I0=30.0, seed=0):
    rng = np.random.default_rng(seed)
    return rng.poisson(I0 * np.exp(-p.line_integrals.ravel())).astype(np.float32), I0


def _check(mu, hist, ref, bound, what):
    mu = np.asarray(mu, np.float64).ravel()
    assert mu.min() >= 0.0, what
    rel = np.linalg.norm(mu - ref.mu.ravel()) / np.linalg.norm(ref.mu)
    assert rel <= bound, (what, rel)
    atol = (2e-5 if bound > 1e-6 else 1e-12) * ref.cost[0]
    np.testing.assert_allclose(hist, ref.cost, rtol=bound, atol=atol)


@pytest.mark.parametrize("nx,ny", [(32, 24), (31, 25)])
@pytest.mark.parametrize("precision", [32, 64])
def test_nonneg_plain_am_2d(nx, ny, precision):
    p = I.small_problem(nx, ny, 24, 45, seed=nx + ny)
    d, I0 = _lowcount(p, seed=nx)
    H = smx.system_matrix(p.geom)
    assert am.plain_am(H, d, I0, 15).mu.min() < 0.0      # the bound matters here
    ref = am.plain_am(H, d, I0, 15, nonneg=True)
    ctx = wam.Context(p.geom)
    ctx.set_data(d, I0)
    mu, hist, _, st = ctx.reconstruct(0, 15, full_am=True, precision=precision, nonneg=True)
    assert st == wam.WAM_OK
    _check(mu, hist, ref, 1e-4 if precision == 32 else 1e-10, "%dx%d FP%d" % (nx, ny, precision))


def test_nonneg_plain_am_cone():
    p = I.small_problem3d(20, 16, 12, 24, 7, 33, seed=8)
    d, I0 = _lowcount(p, I0=20.0, seed=3)
    H = smx.system_matrix(p.geom)
    assert am.plain_am(H, d, I0, 10).mu.min() < 0.0
    ref = am.plain_am(H, d, I0, 10, nonneg=True)
    ctx = wam.Context(p.geom)
    ctx.set_data(d, I0)
    mu, hist, _, st = ctx.reconstruct(0, 10, full_am=True, nonneg=True)
    assert st == wam.WAM_OK
    _check(mu, hist, ref, 1e-4, "cone")


def test_nonneg_refused_with_a_haar_tree():
    p = I.small_problem(32, 32, 12, 45, seed=5)
    ctx = wam.Context(p.geom)
    ctx.set_data(p.d.astype(np.float32), p.I0)
    with pytest.raises(wam.WamError) as e:
        ctx.reconstruct(2, 4, (2,), (0.1,), nonneg=True)
    assert e.value.status == wam.WAM_ERR_ARG


def test_nonneg_resume(tmp_path):
    p = I.small_problem(32, 24, 24, 45, seed=9)
    d, I0 = _lowcount(p, seed=4)

    def ctx():
        c = wam.Context(p.geom)
        c.set_data(d, I0)
        return c

    mu_ref, h_ref, _, _ = ctx().reconstruct(0, 12, full_am=True, nonneg=True, device_out=True)
    a = ctx()
    a.reconstruct(0, 5, full_am=True, nonneg=True)
    path = str(tmp_path / "nn.ckpt")
    a.checkpoint(path)
    b = ctx()
    b.resume(path)
    with pytest.raises(wam.WamError) as e:
        b.reconstruct(0, 12, full_am=True, nonneg=False)
    assert e.value.status == wam.WAM_ERR_STATE
    mu_b, h_b, _, _ = b.reconstruct(0, 12, full_am=True, nonneg=True, device_out=True)
    assert torch.equal(mu_b, mu_ref) and torch.equal(h_b, h_ref)
