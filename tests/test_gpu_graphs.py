"""wam_reconstruct replays the iteration of each tree epoch as a CUDA graph
(the default, WAM_TUNE_GRAPHS = 1): the image, the cost history and the tree
are bit for bit those of direct launches (WAM_TUNE_GRAPHS = 0), in FP32 and
FP64, multiresolution and plain AM, from a fresh start and from a resumed
checkpoint, and the kernel count the library reports is the same (a replay
counts the kernels it runs)."""
import numpy as np
import pytest

from paper_1508_04458_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1508_04458_gb300 import wam  # noqa: E402

SCHED = dict(levels=3, n_iters=14, expand_at=(3, 6, 10), tau=(0.1, 0.03, -1.0))


def _ctx(p, graphs):
    c = wam.Context(p.geom)
    c.set_data(p.d.astype(np.float32), p.I0)
    c.check(wam.wam_set_tuning(c.h, wam.WAM_TUNE_GRAPHS, float(graphs)))
    return c


def _run(c, **kw):
    torch.cuda.synchronize()
    n0 = wam.kernel_launches()
    mu, h, m, st = c.reconstruct(device_out=True, **kw)
    torch.cuda.synchronize()
    assert st in (wam.WAM_OK, wam.WAM_WARN_NONMONOTONE)
    return mu, h, m, wam.kernel_launches() - n0


@pytest.mark.parametrize("precision,full", [(32, False), (64, False), (32, True)])
def test_graph_replay_matches_direct_launches(precision, full):
    p = I.small_problem(80, 48, 37, 131, seed=41)
    kw = dict(levels=0, n_iters=9, full_am=True) if full else dict(SCHED)
    outs = [_run(_ctx(p, g), precision=precision, **kw) for g in (1, 0)]
    (mu_g, h_g, m_g, n_g), (mu_d, h_d, m_d, n_d) = outs
    assert torch.equal(mu_g, mu_d) and torch.equal(h_g, h_d)
    if not full:
        assert torch.equal(m_g, m_d)
    assert n_g == n_d > 0


def test_graph_replay_after_resume(tmp_path):
    p = I.small_problem(80, 48, 37, 131, seed=41)
    a = _ctx(p, 1)
    _run(a, precision=32, **dict(SCHED, n_iters=7))
    path = str(tmp_path / "cut.ckpt")
    a.checkpoint(path)
    res = []
    for g in (1, 0):
        b = _ctx(p, g)
        b.resume(path)
        res.append(_run(b, precision=32, **SCHED))
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
    assert res[0][3] == res[1][3]
