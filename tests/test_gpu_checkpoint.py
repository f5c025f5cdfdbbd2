"""Checkpoint and resume through the C-ABI: a run cut after j iterations,
written with wam_checkpoint, loaded into a fresh context with wam_resume and
continued, ends bit for bit where the uninterrupted run ends (image, whole
cost history, tree), in FP32 and FP64, plain AM, a cut at an expansion, with
a non-default back-projector tuning, and in both cone-beam modes.  The file
decodes with the host reader to the run's own history and tree.  Refusals:
nothing to checkpoint, a corrupt file, other data, a schedule that does not
continue the checkpoint's, a batch with a pending state."""
import numpy as np
import pytest

from paper_1508_04458_gb300 import checkpoint as ck
from paper_1508_04458_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1508_04458_gb300 import wam  # noqa: E402

SCHED = dict(levels=3, expand_at=(3, 6, 10), tau=(0.1, 0.03, -1.0))
J = 16


def _ctx(p, tuning=None):
    c = wam.Context(p.geom)
    c.set_data(p.d.astype(np.float32), p.I0)
    if tuning is not None:
        c.check(wam.wam_set_tuning(c.h, wam.WAM_TUNE_BACK_CTAS_PER_SM, tuning))
    return c


def _run(c, n, **kw):
    mu, h, m, st = c.reconstruct(n_iters=n, device_out=True, **kw)
    assert st in (wam.WAM_OK, wam.WAM_WARN_NONMONOTONE)
    return mu, h, m


@pytest.mark.parametrize("cut,precision,tuning", [(6, 32, None), (10, 32, None), (7, 64, None), (5, 32, 8.0)])
def test_resume_is_bit_exact(tmp_path, cut, precision, tuning):
    p = I.small_problem(80, 48, 37, 131, seed=41)
    mu_ref, h_ref, m_ref = _run(_ctx(p, tuning), J, precision=precision, **SCHED)
    a = _ctx(p, tuning)
    _, h_a, m_a = _run(a, cut, precision=precision, **SCHED)
    path = str(tmp_path / "run.ckpt")
    a.checkpoint(path)
    rec = ck.read(path)
    assert rec["iters_done"] == cut and rec["precision"] == precision
    assert rec["expansions_done"] == sum(e <= cut for e in SCHED["expand_at"])
    np.testing.assert_array_equal(rec["hist"], h_a.cpu().numpy())
    np.testing.assert_array_equal(rec["masks"], m_a.cpu().numpy())
    np.testing.assert_array_equal(rec["hist"], h_ref.cpu().numpy()[: cut + 1])
    b = _ctx(p)                                   # default tuning: the file sets it
    b.resume(path)
    mu_b, h_b, m_b = _run(b, J, precision=precision, **SCHED)
    assert torch.equal(mu_b, mu_ref) and torch.equal(h_b, h_ref) and torch.equal(m_b, m_ref)


def test_resume_plain_am(tmp_path):
    p = I.small_problem(64, 64, 30, 97, kind=I.PARALLEL2D, seed=42)
    mu_ref, h_ref, _ = _run(_ctx(p), 12, levels=0, full_am=True)
    a = _ctx(p)
    _run(a, 5, levels=0, full_am=True)
    path = str(tmp_path / "am.ckpt")
    a.checkpoint(path)
    b = _ctx(p)
    b.resume(path)
    mu_b, h_b, _ = _run(b, 12, levels=0, full_am=True)
    assert torch.equal(mu_b, mu_ref) and torch.equal(h_b, h_ref)


@pytest.mark.parametrize("dims,zsum", [(3, False), (2, True)])
def test_resume_cone(tmp_path, dims, zsum):
    p = I.small_problem3d(16, 16, 8, 24, 6, 29, seed=43)
    kw = dict(levels=2, expand_at=(3, 7), tau=(0.1, -1.0), dims=dims, zsum=zsum)
    mu_ref, h_ref, m_ref = _run(_ctx(p), 12, **kw)
    a = _ctx(p)
    _run(a, 5, **kw)
    path = str(tmp_path / "cone.ckpt")
    a.checkpoint(path)
    b = _ctx(p)
    b.resume(path)
    mu_b, h_b, m_b = _run(b, 12, **kw)
    assert torch.equal(mu_b, mu_ref) and torch.equal(h_b, h_ref) and torch.equal(m_b, m_ref)


def test_refusals(tmp_path):
    p = I.small_problem(80, 48, 37, 131, seed=44)
    a = _ctx(p)
    path = str(tmp_path / "x.ckpt")
    assert wam.wam_checkpoint(a.h, path.encode()) == wam.WAM_ERR_STATE      # nothing ran yet
    _run(a, 6, **SCHED)
    a.checkpoint(path)
    raw = bytearray(open(path, "rb").read())
    bad = str(tmp_path / "bad.ckpt")
    raw[len(raw) // 2] ^= 1
    open(bad, "wb").write(bytes(raw))
    b = _ctx(p)
    assert wam.wam_resume(b.h, bad.encode()) == wam.WAM_ERR_IO
    assert wam.wam_resume(b.h, str(tmp_path / "missing").encode()) == wam.WAM_ERR_IO
    other = _ctx(I.small_problem(80, 48, 37, 131, seed=45))
    assert wam.wam_resume(other.h, path.encode()) == wam.WAM_ERR_STATE    # other data
    b.resume(path)
    with pytest.raises(wam.WamError) as e:                                 # another tau
        b.reconstruct(3, J, (3, 6, 10), (0.2, 0.03, -1.0))
    assert e.value.status == wam.WAM_ERR_STATE
    with pytest.raises(wam.WamError) as e:                                 # a batch
        wam.reconstruct_batch([b], 3, J, SCHED["expand_at"], SCHED["tau"])
    assert e.value.status == wam.WAM_ERR_STATE
    mu_ref, h_ref, _ = _run(_ctx(p), J, **SCHED)
    mu_b, h_b, _ = _run(b, J, **SCHED)                                     # the state stayed pending
    assert torch.equal(mu_b, mu_ref) and torch.equal(h_b, h_ref)
