"""GPU parity of the AM step of Eq. 1.9, the root the reconstruction's update
kernel applies to every active coefficient (k_update: FP32 on normalised
inputs in an FP32 run, FP64 in an FP64 run), called through wam_am_delta on
extreme (b, bhat+, bhat-) triples against the oracle's FP64 root.

Bound of the FP32 root.  The inputs are divided by m = max(|b|, bhat+,
-bhat-), so no square or product overflows or loses range.  The root
u = (b + sqrt(b^2 - 4 bhat+ bhat-)) / (2 bhat+) (or its conjugate form for
b < 0) adds only terms of one sign (bhat+ >= 0 >= bhat-), so u carries about
4 roundings (relative 2.4e-7), i.e. an absolute 2.4e-7 in t = Z0 Delta =
-ln u; logf adds an ulp of t and the product with the FP32 1/Z0 two more
roundings of the result (3e-7 |t| together).  The test enforces
|Z0 Delta_32 - Z0 Delta_64| <= 5e-7 (1 + |Z0 Delta_64|), about twice that
estimate (an FP32 emulation of the same arithmetic over these triples peaks
at 0.41 of the bound).  The FP64 root must agree to 1e-12 (1 + |t|).
The inputs are FP32-representable, since in an FP32 run bhat+- are FP32 sums.
"""
import numpy as np
import pytest

from oracle import am

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1508_04458_gb300 import wam  # noqa: E402

CLAMP = 30.0


def _triples(n, seed):
    rng = np.random.default_rng(seed)
    scale = 10.0 ** rng.uniform(-15, 5, n)            # 20 decades of ray weight
    ratio = 10.0 ** rng.uniform(-6, 6, n)             # |bhat-| / bhat+ over 12 decades
    bp = scale * rng.random(n)
    bm = -scale * ratio * rng.random(n)
    pick = rng.random(n)
    near = (bp + bm) * (1 + 10.0 ** rng.uniform(-7, 0, n) * rng.choice([-1, 1], n))   # small steps
    b = np.where(pick < 0.5, near, scale * rng.uniform(-3, 3, n))
    # the degenerate cases of the root (Eq. 1.9 has a closed form only generically)
    s = 1e3
    special = np.array([
        (0.0, 0.0, 0.0),            # seen by no ray: Delta = 0
        (-2 * s, 0.0, -s),          # bhat+ = 0, b < 0: u = bhat- / b
        (2 * s, 0.0, -s),           # bhat+ = 0, b >= 0: minimiser at -infinity, clamped
        (0.0, 0.0, -s),             # the same with zero counts
        (2 * s, s, 0.0),            # bhat- = 0: u = b / bhat+
        (-s, s, 0.0),               # bhat- = 0, b < 0: minimiser at +infinity, clamped
        (0.0, s, 0.0),              # zero counts, bhat- = 0: clamped
        (0.0, s, -4 * s),           # zero counts: u = sqrt(-bhat- / bhat+) = 2
        (0.0, 1e-40, -1e-40),       # denormal float sums (q-hat underflowing behind metal)
        (1e-41, 3e-41, -2e-41),
        (1e-30, 1e-38, -1e-38),
        (5e12, 1e13, -1e12),        # large sums
        (1.0, 1.0 + 1e-7, -1e-7),   # a step at the rounding level
        (1e5, 1e-12, 0.0),          # a step beyond the clamp
    ])
    b = np.concatenate([b, special[:, 0]])
    bp = np.concatenate([bp, special[:, 1]])
    bm = np.concatenate([bm, special[:, 2]])
    f32 = lambda x: x.astype(np.float32).astype(np.float64)
    return f32(b), f32(bp), f32(bm)


def _run(b, bp, bm, z0, precision):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    tb, tp, tm = dev(b), dev(bp), dev(bm)
    delta = torch.empty_like(tb)
    hit = torch.empty(len(b), dtype=torch.int32, device="cuda")
    rc = wam.wam_am_delta(len(b), wam.ptr(tb), wam.ptr(tp), wam.ptr(tm), 0, 0.0, z0, CLAMP, precision,
                          wam.ptr(delta), wam.ptr(hit), wam.current_stream())
    assert rc == wam.WAM_OK
    torch.cuda.synchronize()
    return delta.cpu().numpy(), hit.cpu().numpy()


@pytest.mark.parametrize("z0", [723.4, 4.9e-2, 3.1e3])
def test_fp32_root_of_the_reconstruction_against_oracle(z0):
    b, bp, bm = _triples(200000, seed=int(z0 * 10))
    want = am.am_root(b, bp, bm, z0, CLAMP) * z0          # t = Z0 Delta, FP64
    got, hit = _run(b, bp, bm, z0, 32)
    t = got * z0
    err = np.abs(t - want)
    bound = 5e-7 * (1.0 + np.abs(want))
    worst = int(np.argmax(err / bound))
    assert np.all(err <= bound), (err[worst], bound[worst], b[worst], bp[worst], bm[worst])
    # steps at the clamp are flagged (away from the clamp's rounding band)
    clear = np.abs(np.abs(want) - CLAMP) > 1e-3
    np.testing.assert_array_equal(hit[clear], (np.abs(want[clear]) >= CLAMP).astype(np.int32))
    assert (np.abs(want) >= CLAMP).sum() >= 5          # the clamp is exercised
    assert np.all(got[-14] == 0.0)                     # no ray weight: no step


@pytest.mark.parametrize("z0", [723.4, 4.9e-2])
def test_fp64_root_against_oracle(z0):
    b, bp, bm = _triples(50000, seed=7)
    want = am.am_root(b, bp, bm, z0, CLAMP) * z0
    got, _ = _run(b, bp, bm, z0, 64)
    assert np.all(np.abs(got * z0 - want) <= 1e-12 * (1.0 + np.abs(want)))


def test_root_rejects_bad_arguments():
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = wam.ptr(x)
    st = wam.current_stream()
    assert wam.wam_am_delta(4, p, p, p, 0, 0.0, 0.0, CLAMP, 32, p, 0, st) == wam.WAM_ERR_ARG     # Z0 = 0
    assert wam.wam_am_delta(4, p, p, p, 0, 0.0, 1.0, CLAMP, 16, p, 0, st) == wam.WAM_ERR_ARG     # precision
    assert wam.wam_am_delta(4, 0, p, p, 0, 0.0, 1.0, CLAMP, 32, p, 0, st) == wam.WAM_ERR_ARG     # null
    assert wam.wam_am_delta(4, p, p, p, 0, 1.0, 1.0, CLAMP, 32, p, 0, st) == wam.WAM_ERR_ARG     # no beta
    assert wam.wam_am_delta(4, p, p, p, p, -1.0, 1.0, CLAMP, 32, p, 0, st) == wam.WAM_ERR_ARG    # lambda < 0
    assert wam.wam_am_delta(0, 0, 0, 0, 0, 0.0, 1.0, CLAMP, 32, 0, 0, st) == wam.WAM_OK          # empty
