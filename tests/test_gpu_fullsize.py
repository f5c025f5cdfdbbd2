"""The fan-beam workload at full size (512x512, 720 views x 1024 bins), in the
launch configuration the benchmark times, against the FP64 oracle on sampled
outputs and against properties that hold at any size:

* H mu on 400 sampled rays (the oracle builds those rows only);
* H^T s on 48 sampled pixels (the oracle builds H in chunks of 60 views and
  keeps the sampled columns);
* Algorithm 1 with the benchmark's schedule (L = 4, 100 iterations,
  expansions after 8, 16, 32, 64 with tau 0.1, 0.03, 0.01, every leaf),
  with the forward's image band staged in shared memory or not: a
  finite, non-increasing I-divergence history (each AM step minimises a
  separable majoriser, Eq. 1.8-1.9, so the exact cost cannot rise; the FP32
  projections allow a 1e-6 relative rise), a valid tree, and bit-identical
  results on a second run (every reduction has a fixed order) and with
  every staged tile height.

FP32 bounds as in the small-case parity tests: max <= 1e-4 and RMS <= 1e-5 of
the largest reference entry.  At this size the rays that graze a pixel edge
(angle psi ~ 4e-4 rad to it) sit at the FP32 limit: a ray held to ~1e-5 mm
moves its crossing by 1e-5 / psi ~ 0.03 mm, so the few worst rays of the
737,280 reach ~1e-4 of the largest ray sum; a random sample of 400 carries
~1e-6.
"""
import numpy as np
import pytest

from oracle import system_matrix as smx
from paper_1508_04458_gb300 import inputs as I

from gpu_helpers import masks_to_tree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1508_04458_gb300 import wam  # noqa: E402

FP32_MAX, FP32_RMS = 1e-4, 1e-5


def _close(got, want, what):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    scale = np.max(np.abs(want))
    e = np.abs(got - want)
    assert e.max() <= FP32_MAX * scale, "%s: max %.3e" % (what, e.max() / scale)
    assert np.sqrt(np.mean(e * e)) <= FP32_RMS * scale, "%s: rms %.3e" % (what, np.sqrt(np.mean(e * e)) / scale)


def test_fan512_projector_sampled():
    g = I.geom_fan512()
    ctx = wam.Context(g)
    rng = np.random.default_rng(11)
    mu = rng.random(g.nx * g.ny).astype(np.float32) * 0.03
    M = g.n_views * g.n_bins
    s = rng.random(M).astype(np.float32)
    mu_d = torch.from_numpy(mu).cuda()
    s_d = torch.from_numpy(s).cuda()
    p_d = torch.empty(M, dtype=torch.float32, device="cuda")
    b_d = torch.empty(g.nx * g.ny, dtype=torch.float32, device="cuda")
    st = wam.current_stream()
    ctx.check(wam.wam_project(ctx.h, wam.ptr(mu_d), wam.ptr(p_d), st))
    ctx.check(wam.wam_backproject(ctx.h, wam.ptr(s_d), wam.ptr(b_d), st))
    torch.cuda.synchronize()
    seg = smx.ray_segments(g)
    rays = rng.choice(M, 400, replace=False)
    Hs = smx.siddon_matrix(seg[rays], (g.nx, g.ny), (g.vx, g.vy))
    _close(p_d.cpu().numpy()[rays], Hs @ mu.astype(np.float64), "H mu (sampled rays)")
    zs = rng.choice(g.nx * g.ny, 48, replace=False)
    acc = np.zeros(zs.size)
    for v0 in range(0, g.n_views, 60):
        rows = slice(v0 * g.n_bins, (v0 + 60) * g.n_bins)
        Hc = smx.siddon_matrix(seg[rows], (g.nx, g.ny), (g.vx, g.vy)).tocsc()
        acc += Hc[:, zs].T @ s[rows].astype(np.float64)
    _close(b_d.cpu().numpy()[zs], acc, "H^T s (sampled pixels)")


def test_fan512_multires_schedule():
    p = I.problem_fan(512, 720, 1024, 1e5, seed=1509, device="cuda")
    d = p.d if isinstance(p.d, np.ndarray) else p.d.float().cpu().numpy()
    ctx = wam.Context(p.geom)
    ctx.set_data(d.astype(np.float32), p.I0)
    sched = (4, 100, (8, 16, 32, 64), (0.1, 0.03, 0.01, -1.0))
    mu1, h1, m1, st = ctx.reconstruct(*sched, precision=32, device_out=True)
    assert st == wam.WAM_OK
    mu2, h2, m2, _ = ctx.reconstruct(*sched, precision=32, device_out=True)
    assert torch.equal(mu1, mu2) and torch.equal(h1, h2) and torch.equal(m1, m2)
    # the forward with its image band staged in shared memory (every tile
    # height) walks and sums exactly as the unstaged one
    for rows in (16, 24, 32):
        ctx.check(wam.wam_set_tuning(ctx.h, wam.WAM_TUNE_FWD_STAGE_ROWS, float(rows)))
        mu3, h3, m3, _ = ctx.reconstruct(*sched, precision=32, device_out=True)
        assert torch.equal(mu1, mu3) and torch.equal(h1, h3) and torch.equal(m1, m3), rows
    ctx.check(wam.wam_set_tuning(ctx.h, wam.WAM_TUNE_FWD_STAGE_ROWS, 0.0))
    h = h1.cpu().numpy()
    assert np.all(np.isfinite(h))
    assert np.all(h[1:] <= h[:-1] * (1 + 1e-6)), np.max(h[1:] / h[:-1])
    assert h[-1] < 0.1 * h[0]
    # the grown tree is a tree: a block's details are active only under an
    # active parent, and the root level (L = 4) is fully active after the
    # first expansion with tau < 0 at the latest
    tree = masks_to_tree(m1.cpu().numpy(), 512, 512, 4)
    for l in range(1, 4):
        parent = np.kron(tree[l], np.ones((2, 2), dtype=bool))
        assert not np.any(tree[l - 1] & ~parent), l
    assert tree[3].all()
