"""wam_backproject_static: the back-projection for callers that cannot allocate
device memory (an application that reserves all of its device memory in a
fixed pool at start-up and forbids later cudaMalloc calls).  It must give the
same H^T s as wam_backproject, on consecutive calls that reuse its fixed
scratch, and a call must leave the device's free memory unchanged.  This file
is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1508_04458_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1508_04458_gb300 import wam  # noqa: E402

# the FP32 bounds of the parity tests: RMS <= 1e-5 and max <= 1e-4 of max |ref|
FP32_MAX, FP32_RMS = 1e-4, 1e-5


def _check(got, want, what):
    scale = float(want.abs().max())
    diff = (got.double() - want.double()).abs()
    assert float(diff.max()) <= FP32_MAX * scale, what
    assert float(diff.pow(2).mean().sqrt()) <= FP32_RMS * scale, what


@pytest.mark.parametrize("kind,nx,ny,V,B", [(I.FAN2D_FLAT, 96, 80, 45, 150), (I.PARALLEL2D, 64, 64, 30, 97)])
def test_static_backprojection_matches_allocating_one(kind, nx, ny, V, B):
    g = I.small_problem(nx, ny, V, B, kind=kind, seed=5).geom
    ctx = wam.Context(g)
    gs = wam.geometry(g)
    st = wam.current_stream()
    rng = np.random.default_rng(11)
    for call in range(2):           # two calls in a row share the scratch
        s = torch.from_numpy(rng.random(V * B).astype(np.float32)).cuda()
        ref = torch.empty(nx * ny, dtype=torch.float32, device="cuda")
        out = torch.full((nx * ny,), float("nan"), dtype=torch.float32, device="cuda")
        ctx.check(wam.wam_backproject(ctx.h, wam.ptr(s), wam.ptr(ref), st))
        torch.cuda.synchronize()
        # the first call on a device may load the library's module, which
        # places the static array; from the second call on nothing may change
        free0 = torch.cuda.mem_get_info()[0]
        torch_bytes0 = torch.cuda.memory_allocated()
        rc = wam.wam_backproject_static(ctypes.byref(gs), wam.ptr(s), wam.ptr(out), st)
        assert rc == wam.WAM_OK
        torch.cuda.synchronize()
        if call > 0:
            assert torch.cuda.mem_get_info()[0] == free0, "device memory changed"
            assert torch.cuda.memory_allocated() == torch_bytes0
        assert torch.isfinite(out).all()
        _check(out, ref, "call %d" % call)
    ctx.close()


def test_static_backprojection_rejects_oversize():
    # 2048 x 2048 needs 16 MiB of partials: more than the fixed scratch
    g = I.Geometry(kind=I.PARALLEL2D, nx=2048, ny=2048, n_views=8, n_bins=64, bin_pitch=64.0)
    gs = wam.geometry(g)
    rc = wam.wam_backproject_static(ctypes.byref(gs), 0, 0, 0)
    assert rc == wam.WAM_ERR_ARG                 # null pointers
    s = torch.zeros(8 * 64, dtype=torch.float32, device="cuda")
    out = torch.zeros(2048 * 2048, dtype=torch.float32, device="cuda")
    rc = wam.wam_backproject_static(ctypes.byref(gs), wam.ptr(s), wam.ptr(out), wam.current_stream())
    assert rc == wam.WAM_ERR_ARG


def test_static_backprojection_rejects_what_wam_create_rejects():
    # the same geometry check as wam_create: a non-finite angle, a cone-beam
    # geometry, a fan source inside the image
    s = torch.zeros(16 * 32, dtype=torch.float32, device="cuda")
    out = torch.zeros(32 * 32, dtype=torch.float32, device="cuda")
    base = I.small_problem(32, 32, 16, 32, kind=I.FAN2D_FLAT, seed=3).geom
    bad = [dict(angle0=float("nan")), dict(angle_span=float("inf")), dict(sod=5.0),
           dict(kind=I.CONE3D_FLAT_CIRCULAR, nz=4, n_rows=2, vz=1.0, row_pitch=1.0)]
    import dataclasses
    for kw in bad:
        gs = wam.geometry(dataclasses.replace(base, **kw))
        rc = wam.wam_backproject_static(ctypes.byref(gs), wam.ptr(s), wam.ptr(out), wam.current_stream())
        assert rc == wam.WAM_ERR_ARG, kw
