"""Batched multiresolution AM over bags of uneven size (one CUDA graph per
tree epoch: every bag on its own stream branch, or five multi-bag kernels
with persistent forward and back-projection CTAs on a work queue) against
the per-bag loop, bit for bit, and the oracle; the autotuner."""
import numpy as np
import pytest

from oracle import am
from oracle import system_matrix as smx
from paper_1508_04458_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1508_04458_gb300 import autotune, wam  # noqa: E402

SCHED = dict(levels=3, n_iters=16, expand_at=(3, 6, 10), tau=(0.1, 0.03, -1.0))


def _bags():
    shapes = [(64, 64, 40, 97), (80, 48, 37, 131), (96, 96, 45, 150), (48, 64, 33, 70), (112, 80, 51, 160)]
    return [I.small_problem(nx, ny, V, B, seed=20 + i) for i, (nx, ny, V, B) in enumerate(shapes)]


def test_batch_equals_per_bag_loop_bit_for_bit():
    bags = _bags()
    ctxs = []
    for p in bags:
        c = wam.Context(p.geom)
        c.set_data(p.d.astype(np.float32), p.I0)
        ctxs.append(c)
    singles = [c.reconstruct(SCHED["levels"], SCHED["n_iters"], SCHED["expand_at"], SCHED["tau"], device_out=True)
               for c in ctxs]
    for use_graph in (True, False):
        mus, hists, st = wam.reconstruct_batch(ctxs, SCHED["levels"], SCHED["n_iters"], SCHED["expand_at"],
                                               SCHED["tau"], use_graph=use_graph)
        assert st == wam.WAM_OK
        for (mu1, h1, _, _), mu2, h2 in zip(singles, mus, hists):
            assert torch.equal(mu1, mu2)
            assert torch.equal(h1, h2)
    # the persistent multi-bag kernels run the same bodies and sums in the same
    # order, compiled into other kernels: they agree to FP32 rounding
    mus, hists, st = wam.reconstruct_batch(ctxs, SCHED["levels"], SCHED["n_iters"], SCHED["expand_at"],
                                           SCHED["tau"], use_graph=wam.BATCH_PERSISTENT)
    assert st == wam.WAM_OK
    for (mu1, h1, _, _), mu2, h2 in zip(singles, mus, hists):
        assert float((mu1 - mu2).norm() / mu1.norm()) <= 1e-5
        assert float(((h1 - h2).abs() / h1.abs()).max()) <= 1e-5
        assert torch.equal(h1[0], h2[0])                 # the first cost (beta = 0) is the same sum
    # one bag of the batch against the oracle
    p = bags[2]
    ref = am.wavelet_am(smx.system_matrix(p.geom), p.d, p.I0, p.geom.nx, p.geom.ny, SCHED["levels"],
                        SCHED["n_iters"], expand_at=SCHED["expand_at"], taus=SCHED["tau"])
    rel = np.linalg.norm(mus[2].cpu().numpy() - ref.mu.ravel()) / np.linalg.norm(ref.mu)
    assert rel <= 1e-4, rel


def test_batch_rejects_bad_input():
    p = _bags()[0]
    c = wam.Context(p.geom)
    with pytest.raises(wam.WamError):
        wam.reconstruct_batch([c], 3, 4)          # no data
    c.set_data(p.d.astype(np.float32), p.I0)
    with pytest.raises(wam.WamError):
        wam.reconstruct_batch([c, c], 3, 4)       # same context twice


def test_autotuner(tmp_path):
    p = I.problem_fan(128, 180, 256, 1e5, seed=31)
    ctx = wam.Context(p.geom)
    ctx.set_data(p.d.astype(np.float32), p.I0)
    ref, _, _, _ = ctx.reconstruct(4, 12, (2, 4, 6, 8), (0.1, 0.03, 0.01, -1.0), device_out=True)
    cache = str(tmp_path / "tune.json")
    best = autotune.tune(ctx, cache=cache)
    assert best["back_ctas_per_sm"] in autotune.CANDIDATES and best["fwd_stage_rows"] in autotune.STAGE_ROWS
    # cached on the second call, same answer
    assert autotune.tune(ctx, cache=cache) == best
    mu, _, _, _ = ctx.reconstruct(4, 12, (2, 4, 6, 8), (0.1, 0.03, 0.01, -1.0), device_out=True)
    # the back-projector knob only reorders fixed partial sums: results agree to FP32 rounding
    assert float((mu - ref).norm() / ref.norm()) <= 1e-5
    # the forward's tile height changes nothing that is computed
    ctx.check(wam.wam_set_tuning(ctx.h, wam.WAM_TUNE_BACK_CTAS_PER_SM, 32.0))
    outs = []
    for rows in autotune.STAGE_ROWS:
        ctx.check(wam.wam_set_tuning(ctx.h, wam.WAM_TUNE_FWD_STAGE_ROWS, float(rows)))
        outs.append(ctx.reconstruct(4, 12, (2, 4, 6, 8), (0.1, 0.03, 0.01, -1.0), device_out=True)[:2])
    for mu_r, h_r in outs[1:]:
        assert torch.equal(mu_r, outs[0][0]) and torch.equal(h_r, outs[0][1])
    with pytest.raises(wam.WamError):
        ctx.check(wam.wam_set_tuning(ctx.h, wam.WAM_TUNE_FWD_STAGE_ROWS, 8.0))
