"""Pins of the oracle's readings of the points the paper leaves open that set
how fast Algorithm 1 converges (oracle/readings.py): the Haar normalisation
("Level 3 Haar", Results section), the update subset Z_s^(j) of Algorithm 1
(footnote to Eq. 1.61: fixed or varied over iterations, every voxel
represented) and the expansion schedule.

* With the defaults the reading runner is Algorithm 1 (am.wavelet_am) bit for
  bit.
* Under every reading the surrogate of Eq. 1.8, built with Z0 over the
  iteration's own Z_s^(j), majorises the cost and touches it at beta-hat, and
  the cost never rises (the paper's guarantee).
* The per-level contraction rates that explain the measured time to target
  (the design notes' table): in the orthonormal basis the surrogate allows
  about the same contraction at every level, while plain AM's surrogate
  allows twice as much per coarser level for the same basis function.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import am, haar, readings as R
from oracle import system_matrix as smx
from paper_1508_04458_gb300 import inputs as I

SCHED = ((3, 6, 9), (0.1, 0.03, -1.0))


@pytest.fixture(scope="module")
def case():
    p = I.small_problem(32, 32, 40, 61, seed=4)
    return p, smx.system_matrix(p.geom)


def test_defaults_are_algorithm_1(case):
    p, H = case
    a = am.wavelet_am(H, p.d, p.I0, 32, 32, 3, 14, expand_at=SCHED[0], taus=SCHED[1])
    b = R.wavelet_am_reading(H, p.d, p.I0, 32, 32, 3, 14, expand_at=SCHED[0], taus=SCHED[1])
    assert np.array_equal(a.beta, b.beta) and np.array_equal(a.cost, b.cost)


@pytest.mark.parametrize("norm,subsets", [("equal", "tree"), ("orthonormal", "alternate"),
                                          ("orthonormal", "levels"), ("equal", "levels")])
def test_every_reading_decreases_the_cost(case, norm, subsets):
    p, H = case
    r = R.wavelet_am_reading(H, p.d, p.I0, 32, 32, 3, 20, expand_at=SCHED[0], taus=SCHED[1], norm=norm,
                             subsets=subsets)
    assert np.all(np.diff(r.cost) <= 1e-12 * r.cost[:-1])
    assert r.cost[-1] < 0.5 * r.cost[0]


def test_subset_surrogate_majorises_with_its_own_z0(case):
    # Eq. 1.8 on Z_s = approximations + the level-1 details only, equal
    # amplitudes; the coefficients outside Z_s stay fixed and enter qhat
    p, H = case
    nx = ny = 32
    L = 2
    W = R.level_weights(nx, ny, L, "equal")
    Phi = (H @ (haar.basis_matrix(nx, ny, L) @ sp.diags(W))).tocsc()
    level, typ, _, _ = haar.coefficient_info(nx, ny, L)
    rng = np.random.default_rng(8)
    beta_hat = rng.normal(0.0, 0.003, nx * ny)
    beta_hat[typ < 0] = 0.02
    zs = (typ < 0) | ((level == 1) & (typ >= 0))
    Ps = Phi[:, zs].toarray()
    rest = Phi[:, ~zs] @ beta_hat[~zs]
    d = p.d.ravel()
    b = Phi.T @ d
    Z0 = float(np.max(np.abs(Ps).sum(axis=1)))
    assert Z0 < float(np.max(np.abs(Phi.toarray()).sum(axis=1)))
    qhat = p.I0 * np.exp(-(Ps @ beta_hat[zs] + rest))

    def F(beta_s):
        return b[zs] @ beta_s + np.sum(p.I0 * np.exp(-(Ps @ beta_s + rest)))

    def surrogate(beta_s):
        r = np.abs(Ps) / Z0
        with np.errstate(divide="ignore", invalid="ignore"):
            ratio = np.where(r > 0, Ps / np.where(r > 0, r, 1.0), 0.0)
        ex = r * np.exp(-ratio * (beta_s - beta_hat[zs])[None, :])
        return b[zs] @ beta_s + qhat @ (ex.sum(axis=1) + 1.0 - r.sum(axis=1))

    assert surrogate(beta_hat[zs]) == pytest.approx(F(beta_hat[zs]), rel=1e-12)
    for _ in range(10):
        x = beta_hat[zs] + rng.normal(0, 0.002, zs.sum())
        assert surrogate(x) >= F(x) - 1e-9 * abs(F(x))
    A = am.active_columns(Phi[:, zs])
    delta, _, z0 = R.am_step_offset(A, b[zs], Phi @ beta_hat, d, p.I0)
    assert z0 == pytest.approx(Z0)
    assert F(beta_hat[zs] + delta) <= F(beta_hat[zs])


def test_mode_rates_flat_in_the_wavelet_basis_doubling_for_plain_am():
    p = I.small_problem(64, 64, 60, 96, seed=4)
    H = smx.system_matrix(p.geom)
    pl = am.plain_am(H, p.d, p.I0, 30)
    q = p.I0 * np.exp(-(H @ pl.mu.ravel()))
    r = R.mode_rates(H, q, 64, 64, 3, n_per_level=60)["levels"]
    wav = [r[l]["wavelet"] for l in (1, 2, 3)]
    pix = [r[l]["pixel"] for l in (1, 2, 3, 4)]
    assert max(wav) / min(wav) < 1.2                       # the same rate at every detail level
    assert all(1.6 < pix[k + 1] / pix[k] < 3.2 for k in range(3))   # about 2x per coarser level
    assert all(r[l]["wavelet"] < r[l]["pixel"] for l in (1, 2, 3, 4))
