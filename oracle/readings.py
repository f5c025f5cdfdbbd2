"""Oracle: readings of the points the paper leaves open that change how fast
Algorithm 1 converges, and the experiment that compares them with plain AM.

TEST INFRASTRUCTURE ONLY (tests and this module's own experiment).  Shares
no code with the CUDA path.

The paper fixes the method (Eq. 1.8-1.10, Algorithm 1) but not
  * the normalisation of the Haar basis ("Level 3 Haar", Results section):
    the amplitude alpha_l of a level-l basis function on its 2^l x 2^l block.
    Orthonormal is alpha_l = 2^-l; "equal" is alpha_l = 1 (the unnormalised
    box functions).  Scaling a column of Omega scales its column of Phi and so
    its share r(z|y) = |phi(y|z)| / Z0 of the convex decomposition (Eq. 1.61);
  * the update subset Z_s^(j) (the footnote to Eq. 1.61: a subset of the
    wavelet domain chosen for update, which "can be fixed or be varied over
    iterations", with every voxel represented at any iteration).  Algorithm 1
    takes Z_s^(j) as an input per iteration; its Z0^(j) is the max over rays of
    the row sums over Z_s^(j) only;
  * the expansion schedule (the paper's: 3 levels, expansions after
    iterations 64, 128, 256 of 300 with factor 0.1).

wavelet_am_reading() runs Algorithm 1 under any combination of these
readings; with the defaults it is am.wavelet_am.  mode_rates() measures,
per level, the per-iteration contraction of one coefficient's error that the
separable surrogate allows, next to what plain AM's surrogate allows for the
same basis function seen as an image (both are Rayleigh quotients of the
cost's curvature over the surrogate's, see its docstring).
"""
from __future__ import annotations

import json
import sys
from typing import Callable, Optional, Sequence

import numpy as np
import scipy.sparse as sp

from . import am, haar


def level_weights(nx: int, ny: int, L: int, norm: str) -> np.ndarray:
    """Column scale of Omega per coefficient: 1 for the orthonormal basis,
    2^l for equal-amplitude (alpha_l = 1) basis functions of level l (the
    approximations are level L)."""
    level, typ, _, _ = haar.coefficient_info(nx, ny, L)
    if norm == "orthonormal":
        return np.ones(nx * ny)
    if norm == "equal":
        return np.ldexp(1.0, level)
    raise ValueError(norm)


def subset_rule(kind: str, L: int) -> Optional[Callable]:
    """Z_s^(j) inside the tree's active set, as a function of (j, level, typ,
    active) -> bool mask.  The level-L approximations stay in every subset,
    so every voxel is represented at every iteration (the footnote's
    condition).
      "tree"      : the whole tree (Algorithm 1 as run in the Results section)
      "alternate" : the whole tree on even j; on odd j the approximations and
                    the finest active detail level
      "levels"    : the approximations and one detail level, cycling over
                    the active levels from the coarsest to the finest"""
    if kind == "tree":
        return None

    def rule(j, level, typ, act):
        det = act & (typ >= 0)
        levels = sorted(set(level[det].tolist()), reverse=True)     # coarse -> fine
        keep = act & (typ < 0)
        if not levels:
            return act
        if kind == "alternate":
            if j % 2 == 0:
                return act
            return keep | (det & (level == levels[-1]))
        if kind == "levels":
            return keep | (det & (level == levels[j % len(levels)]))
        raise ValueError(kind)
    return rule


def wavelet_am_reading(H: sp.spmatrix, d, I0, nx: int, ny: int, L: int, n_iter: int,
                       expand_at: Sequence[int] = (), taus: Sequence[float] = (), norm: str = "orthonormal",
                       subsets: str = "tree", tree0=None) -> am.AMResult:
    """Algorithm 1 (2-D) under the given readings.  beta lives in the scaled
    basis Omega W (W = level_weights); mu = Omega W beta.  Per iteration j the
    update set is Z_s^(j) = subset_rule(...) of the tree's active set; qhat
    uses every active coefficient (the inactive ones are 0 and the ones left
    out of Z_s^(j) keep their values), Z0^(j) is Eq. 1.61 over Z_s^(j), and
    only Z_s^(j) is updated.  Expansions follow am.expand on mu."""
    d = np.asarray(d, dtype=np.float64).ravel()
    W = level_weights(nx, ny, L, norm)
    Omega = (haar.basis_matrix(nx, ny, L) @ sp.diags(W)).tocsc()
    Phi = (H @ Omega).tocsc()
    b = Phi.T @ d
    level, typ, _, _ = haar.coefficient_info(nx, ny, L)
    rule = subset_rule(subsets, L)
    beta = np.zeros(nx * ny)
    tree = [t.copy() for t in tree0] if tree0 is not None else am.empty_tree(nx, ny, L)
    sched = dict(zip(expand_at, taus))
    costs, z0s, nact = [], [], []
    cache = {}
    for j in range(n_iter):
        act = am.active_mask(tree, nx, ny, L)
        zs = act if rule is None else rule(j, level, typ, act)
        key = zs.tobytes()
        if key not in cache:                              # one per (tree epoch, subset)
            cache[key] = am.active_columns(Phi[:, zs])
        A = cache[key]
        p = Phi[:, act] @ beta[act]
        delta, cost, Z0 = am_step_offset(A, b[zs], p, d, I0)
        costs.append(cost)
        z0s.append(Z0)
        nact.append(int(zs.sum()))
        beta[zs] += delta
        if (j + 1) in sched:
            tree = am.expand(tree, (Omega @ beta).reshape(ny, nx), sched[j + 1])
            cache = {}
    costs.append(am.idiv(d, I0, Phi @ beta))
    return am.AMResult(beta, (Omega @ beta).reshape(ny, nx), np.array(costs), np.array(z0s), tree, [],
                       np.array(nact))


def am_step_offset(A: am.ActiveColumns, b_s, p, d, I0):
    """am.am_step with the line integrals p of the whole current image given
    (the coefficients outside Z_s^(j) contribute to qhat but are not
    updated)."""
    q = np.broadcast_to(np.asarray(I0, dtype=np.float64), p.shape) * np.exp(-p)
    cost = am.idiv(d, I0, p)
    bp = A.Pplus.T @ q
    bm = A.Pminus.T @ q
    return am.am_root(b_s, bp, bm, A.Z0), cost, A.Z0


def mode_rates(H: sp.spmatrix, q: np.ndarray, nx: int, ny: int, L: int, norm: str = "orthonormal",
               n_per_level: int = 200, seed: int = 0) -> dict:
    """Per level l, the median over sampled level-l detail coefficients z of

      wavelet: phi_z^T Q phi_z / (Z0 |phi_z|^T qhat)      (Z0 of the full tree)
      pixel  : psi_z^T H^T Q H psi_z / (Z0_pix sum_x psi_z(x)^2 (H^T qhat)(x))

    with Q = diag(qhat) and psi_z = Omega e_z the basis function as an image.
    Each is the factor by which one AM iteration can shrink an error along
    that direction, to first order: the cost's curvature along it over the
    separable surrogate's (Eq. 1.8 for the wavelet basis; the same equation
    with Omega = I for plain AM, whose surrogate is diagonal in the pixels).
    The approximation coefficients are reported as level L + 1."""
    rng = np.random.default_rng(seed)
    W = level_weights(nx, ny, L, norm)
    Omega = (haar.basis_matrix(nx, ny, L) @ sp.diags(W)).tocsc()
    Phi = (H @ Omega).tocsc()
    Hc = H.tocsc()
    z0w = am._row_abs_max(Phi)
    z0p = am._row_abs_max(Hc)
    htq = Hc.T @ q
    level, typ, _, _ = haar.coefficient_info(nx, ny, L)
    out = {}
    for l in range(1, L + 2):
        sel = np.nonzero((level == l) & (typ >= 0))[0] if l <= L else np.nonzero(typ < 0)[0]
        pick = rng.choice(sel, size=min(n_per_level, sel.size), replace=False)
        rw, rp = [], []
        for z in pick:
            phi = Phi[:, z].toarray().ravel()
            den = z0w * float(np.abs(phi) @ q)
            if den <= 0:
                continue
            rw.append(float(phi * phi @ q) / den)
            psi = Omega[:, z].toarray().ravel()
            rp.append(float(phi * phi @ q) / (z0p * float(psi * psi @ htq)))
        out[l] = {"wavelet": float(np.median(rw)), "pixel": float(np.median(rp)), "n": len(rw)}
    return {"z0_wavelet_full_tree": z0w, "z0_pixel": z0p, "levels": out}


def experiment(n: int = 128, views: int = 180, bins: int = 256, n_plain: int = 100, factor: int = 3,
               seed: int = 1515):
    """Iterations each reading needs to reach plain AM's cost after k
    iterations (k = 10, 20, 50, 100), on a seeded fan-beam bag."""
    from . import system_matrix as smx
    from paper_1508_04458_gb300 import inputs as I
    p = I.problem_fan(n, views, bins, 1e5, seed)
    H = smx.system_matrix(p.geom)
    plain = am.plain_am(H, p.d, p.I0, n_plain)
    targets = {k: plain.cost[k] * (1 + 1e-3) for k in (10, 20, 50, n_plain)}
    J = factor * n_plain
    s = J / 100.0
    bench_sched = (tuple(int(round(e * s)) for e in (8, 16, 32, 64)), (0.1, 0.03, 0.01, -1.0))
    paper_sched = (tuple(int(round(e * J / 300)) for e in (64, 128, 256)), (0.1, 0.1, 0.1))
    full_tree = lambda L: [np.ones((n >> l, n >> l), dtype=bool) for l in range(1, L + 1)]
    runs = {
        "A1 as printed (orthonormal, tree, adaptive tau, L=4)": dict(L=4, sched=bench_sched),
        "paper schedule (L=3, tau 0.1 at 64/128/256 of 300)": dict(L=3, sched=paper_sched),
        "equal-amplitude levels (alpha_l = 1)": dict(L=4, sched=bench_sched, norm="equal"),
        "Z_s alternating: tree / finest level": dict(L=4, sched=bench_sched, subsets="alternate"),
        "Z_s cycling over levels": dict(L=4, sched=bench_sched, subsets="levels"),
        "full tree from the start (L=4)": dict(L=4, sched=((), ()), tree0=full_tree(4)),
        "full tree from the start (L=1)": dict(L=1, sched=((), ()), tree0=full_tree(1)),
    }
    res = {"problem": "fan %dx%d, %d views x %d bins, I0 1e5, seed %d" % (n, n, views, bins, seed),
           "plain_am": {k: float(plain.cost[k]) for k in targets}, "readings": {}}
    for name, r in runs.items():
        out = wavelet_am_reading(H, p.d, p.I0, n, n, r["L"], J, expand_at=r["sched"][0], taus=r["sched"][1],
                                 norm=r.get("norm", "orthonormal"), subsets=r.get("subsets", "tree"),
                                 tree0=r.get("tree0"))
        hit = {}
        for k, t in targets.items():
            j = np.nonzero(out.cost <= t)[0]
            hit[k] = int(j[0]) if j.size else None
        res["readings"][name] = {"iters_to_plain_cost_after": hit, "final_cost": float(out.cost[-1]),
                                 "monotone": bool(np.all(np.diff(out.cost) <= 1e-12 * out.cost[:-1]))}
    q = p.I0 * np.exp(-(H @ plain.mu.ravel()))
    res["mode_rates_at_plain_am_%d" % n_plain] = {nm: mode_rates(H, q, n, n, 4, norm=nm)
                                                 for nm in ("orthonormal", "equal")}
    return res


if __name__ == "__main__":
    kw = {}
    if len(sys.argv) > 1:
        kw["n"] = int(sys.argv[1])
    print(json.dumps(experiment(**kw), indent=1))
