"""Algorithm 1 at the scale and with the schedule the benchmark times,
against the FP64 oracle iterate for iterate: a 256 x 256 fan-beam bag at
1 mm (360 views x 512 bins spanning the image's shadow, SOD 1000, SDD 1500,
I0 = 1e5), L = 4, 100 iterations, expansions after 8, 16, 32, 64 with
tau = 0.1, 0.03, 0.01 and finally every leaf -- the benchmark's
reconstruction on a quarter of its pixels and half of its views, where the
oracle's explicit Phi = H Omega (1.1e8 nonzeros) still fits and runs in
about half a minute.

Bounds: relative L2 error of mu <= 1e-4 (FP32 bulk), every I-divergence of
the history within 1e-4 relative, the trees after each expansion bit-exact
(the criterion S > tau max S decides on the synthesised image, which agrees
to ~1e-6, far from every pixel's distance to the threshold on this scan), and
the FP64 path (precision 64) within 1e-9.
"""
import numpy as np
import pytest

from oracle import am
from oracle import system_matrix as smx
from paper_1508_04458_gb300 import inputs as I

from gpu_helpers import masks_to_tree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1508_04458_gb300 import wam  # noqa: E402

N, V, B, L, J = 256, 360, 512, 4, 100
EXPAND_AT = (8, 16, 32, 64)
TAU = (0.1, 0.03, 0.01, -1.0)


@pytest.fixture(scope="module")
def case():
    p = I.problem_fan(N, V, B, 1e5, I.SEED_BASE + 3)
    H = smx.system_matrix(p.geom)
    ref = am.wavelet_am(H, p.d, p.I0, N, N, L, J, expand_at=EXPAND_AT, taus=TAU)
    return p, ref


@pytest.mark.parametrize("precision", [32, 64])
def test_fan256_bench_schedule_against_oracle(case, precision):
    p, ref = case
    ctx = wam.Context(p.geom)
    ctx.set_data(p.d.astype(np.float32), p.I0)
    mu, hist, masks, st = ctx.reconstruct(L, J, EXPAND_AT, TAU, precision=precision)
    torch.cuda.synchronize()
    assert st == wam.WAM_OK, st
    tree = masks_to_tree(masks, N, N, L)
    for l in range(L):
        np.testing.assert_array_equal(tree[l], ref.tree[l], err_msg="level %d" % (l + 1))
    rel = np.linalg.norm(mu.astype(np.float64).ravel() - ref.mu.ravel()) / np.linalg.norm(ref.mu)
    tol = 1e-4 if precision == 32 else 1e-9
    assert rel <= tol, "mu relative error %.3e" % rel
    np.testing.assert_allclose(hist, ref.cost, rtol=tol)
    ctx.close()
