"""Ordered subsets of views (n_subsets > 1) through the C-ABI against the
oracle's os_wavelet_am: uneven subsets (37 views), the wavelet tree with
expansions and plain AM, FP32 (iterate 1e-4 relative, cost 1e-4 + 2e-5 of the
initial cost, trees bit-exact) and FP64 (1e-9); a resumed run is bit-exact;
the calls that cannot take subsets refuse them."""
import numpy as np
import pytest

from oracle import am
from oracle import system_matrix as smx
from paper_1508_04458_gb300 import inputs as I

from gpu_helpers import tree_to_masks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1508_04458_gb300 import wam  # noqa: E402


def _ctx(p):
    c = wam.Context(p.geom)
    c.set_data(p.d.astype(np.float32), p.I0)
    return c


@pytest.mark.parametrize("S,precision,bound", [(3, 32, 1e-4), (4, 32, 1e-4), (4, 64, 1e-9)])
def test_os_wavelet_am_matches_oracle(S, precision, bound):
    p = I.small_problem(80, 48, 37, 131, seed=91)
    L, J, ea, tau = 3, 10, (3, 6), (0.1, -1.0)
    ref = am.os_wavelet_am(smx.system_matrix(p.geom), p.d, p.I0, 80, 48, L, J, S, p.geom.n_bins,
                           expand_at=ea, taus=tau)
    mu, hist, masks, st = _ctx(p).reconstruct(L, J, ea, tau, precision=precision, n_subsets=S)
    assert st in (wam.WAM_OK, wam.WAM_WARN_NONMONOTONE)
    rel = np.linalg.norm(mu.astype(np.float64) - ref.mu.ravel()) / np.linalg.norm(ref.mu)
    assert rel <= bound, rel
    np.testing.assert_array_equal(masks, tree_to_masks(ref.tree, L))
    atol = (2e-5 if precision == 32 else 1e-10) * ref.cost[0]
    np.testing.assert_allclose(hist, ref.cost, rtol=bound, atol=atol)


def test_os_plain_am_matches_oracle():
    p = I.small_problem(64, 64, 30, 97, kind=I.PARALLEL2D, seed=92)
    ref = am.os_wavelet_am(smx.system_matrix(p.geom), p.d, p.I0, 64, 64, 0, 8, 5, p.geom.n_bins)
    mu, hist, _, _ = _ctx(p).reconstruct(0, 8, full_am=True, n_subsets=5)
    rel = np.linalg.norm(mu.astype(np.float64) - ref.mu.ravel()) / np.linalg.norm(ref.mu)
    assert rel <= 1e-4, rel
    np.testing.assert_allclose(hist, ref.cost, rtol=1e-4, atol=2e-5 * ref.cost[0])


def test_os_resume_is_bit_exact(tmp_path):
    p = I.small_problem(80, 48, 37, 131, seed=93)
    kw = dict(levels=3, expand_at=(3, 6), tau=(0.1, -1.0), n_subsets=4, device_out=True)
    mu_ref, h_ref, m_ref, _ = _ctx(p).reconstruct(n_iters=10, **kw)
    a = _ctx(p)
    a.reconstruct(n_iters=4, **kw)
    path = str(tmp_path / "os.ckpt")
    a.checkpoint(path)
    b = _ctx(p)
    b.resume(path)
    with pytest.raises(wam.WamError):
        b.reconstruct(n_iters=10, **dict(kw, n_subsets=3))      # another subset count
    mu_b, h_b, m_b, _ = b.reconstruct(n_iters=10, **kw)
    assert torch.equal(mu_b, mu_ref) and torch.equal(h_b, h_ref) and torch.equal(m_b, m_ref)


def test_os_refusals():
    p = I.small_problem(32, 32, 12, 45, seed=94)
    c = _ctx(p)
    with pytest.raises(wam.WamError):
        c.reconstruct(2, 4, n_subsets=13)                        # more subsets than views
    with pytest.raises(wam.WamError):
        sc, keep = wam.schedule(2, 4, n_subsets=2)
        ptrs = (wam._P * 1)(c.h)
        st = wam.wam_reconstruct_batch(ptrs, 1, wam.ctypes.byref(sc), None, None, 1, 0, wam.current_stream())
        c.check(st)
    q = I.small_problem3d(16, 16, 8, 12, 4, 29, seed=95)
    cone = _ctx(q)
    with pytest.raises(wam.WamError):
        cone.reconstruct(2, 4, (2,), (0.1,), dims=3, n_subsets=2)
