"""Oracle: unregularised wavelet alternating minimisation (Algorithm 1) and the
plain pixel-domain AM it reduces to, in FP64 with explicit sparse matrices.

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the
benchmark).  Shares no code with the CUDA path.

Each step follows the paper's definitions literally, with scipy.sparse
products as the only library primitive:

  Phi = H Omega                                       (Sec. II, after Eq. 1.4)
  b(z) = sum_y d(y) phi(y|z)                           (Eq. 1.6, for all z)
  per iteration j (Algorithm 1):
    qhat(y) = I0(y) exp(-sum_{z in Zs} phi(y|z) beta(z))
    Z0 = max_y sum_{z in Zs} |phi(y|z)|                (Eq. 1.61)
    bhat+(z) = sum_{y: phi>0} qhat phi,  bhat-(z) = sum_{y: phi<0} qhat phi   (Eq. 1.10)
    beta(z) <- the zero of Eq. 1.9 in beta(z)          (closed form, see am_root)
  I-divergence I(d||q) = sum d log(d/q) - d + q        (Sec. II footnote)

Readings where the paper is silent (each also listed in the design notes):
  * beta^(0) = 0 (mu = 0, qhat = I0).
  * The active set Zs is a tree: the level-L approximations are always
    active; the three level-l details of a block are active when that block
    is "expanded".  Inactive coefficients stay 0.
  * Expansion (Results section): after the iterations listed in expand_at
    have completed, the image mu = Omega beta is formed, S = mu (summed over
    z-slices in the per-slice 3-D mode), and every pixel with S > tau * max S
    expands its current leaf one level (the leaf is the finest block on the
    pixel's path from level L whose details are inactive).  tau < 0 expands
    every leaf.  The comparison is made in FP64 on the given S.
  * Degenerate roots and the clamp |Z0 delta| <= 30 (see am_root).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np
import scipy.sparse as sp

from . import haar

CLAMP = 30.0


# ---------------------------------------------------------------------------
# cost
# ---------------------------------------------------------------------------

def idiv(d: np.ndarray, I0, p: np.ndarray) -> float:
    """I(d || q) with q = I0 exp(-p), written with log q = log I0 - p so that
    an underflowed q never enters a logarithm; 0 log 0 = 0."""
    d = np.asarray(d, dtype=np.float64).ravel()
    p = np.asarray(p, dtype=np.float64).ravel()
    I0 = np.broadcast_to(np.asarray(I0, dtype=np.float64), d.shape)
    q = I0 * np.exp(-p)
    pos = d > 0
    logterm = np.zeros_like(d)
    logterm[pos] = d[pos] * (np.log(d[pos]) - np.log(I0[pos]) + p[pos])
    return float(np.sum(logterm - d + q))


# ---------------------------------------------------------------------------
# the closed-form coordinate update
# ---------------------------------------------------------------------------

def am_root(b, bp, bm, Z0: float, clamp: float = CLAMP) -> np.ndarray:
    """Delta = beta~ - betahat solving Eq. 1.9 = 0:
        b - bp exp(-Z0 Delta) - bm exp(Z0 Delta) = 0,  bp >= 0 >= bm.
    With u = exp(-Z0 Delta) this is bp u^2 - b u + bm = 0, whose positive root
    is taken in the cancellation-free form for the sign of b.  Cases:
      bp > 0, b >= 0 : u = (b + sqrt(b^2 - 4 bp bm)) / (2 bp)
      bp > 0, b <  0 : u = 2 bm / (b - sqrt(b^2 - 4 bp bm))
      bp = 0, b <  0, bm < 0 : u = bm / b
      bp = 0, otherwise      : Delta = 0 when bm = 0 (nothing to update);
                               the minimiser is at -infinity when bm < 0 <= b
    u = 0 or u = infinity (minimiser at +-infinity) is clamped to
    |Z0 Delta| <= clamp; any step between 0 and the 1-D minimiser keeps the
    surrogate's decrease."""
    b = np.asarray(b, dtype=np.float64)
    bp = np.asarray(bp, dtype=np.float64)
    bm = np.asarray(bm, dtype=np.float64)
    u = np.empty_like(b)
    zero = np.zeros_like(b, dtype=bool)
    with np.errstate(divide="ignore", invalid="ignore"):
        disc = np.sqrt(b * b - 4.0 * bp * bm)
        c1 = (bp > 0) & (b >= 0)
        c2 = (bp > 0) & (b < 0)
        c3 = (bp == 0) & (bm < 0) & (b < 0)
        c4 = (bp == 0) & (bm < 0) & (b >= 0)
        c5 = (bp == 0) & (bm == 0)
        u[c1] = (b[c1] + disc[c1]) / (2.0 * bp[c1])
        u[c2] = 2.0 * bm[c2] / (b[c2] - disc[c2])
        u[c3] = bm[c3] / b[c3]
        u[c4] = np.inf
        u[c5] = 1.0
        zero |= c5
        t = -np.log(u)                     # = Z0 * Delta
    t = np.clip(t, -clamp, clamp)
    t[zero] = 0.0
    return t / Z0


def am_root_l1(b, bp, bm, Z0: float, beta_hat, lam, clamp: float = CLAMP) -> np.ndarray:
    """Delta minimising the one-coefficient surrogate of Eq. 1.8 plus an L1
    penalty lam |beta_hat + Delta| (Eq. 1.1 with R = the l1 norm of the detail
    coefficients, the wavelet-domain roughness penalty the Summary names).

    The surrogate's derivative in Delta is g(Delta) = b - bp exp(-Z0 Delta)
    - bm exp(Z0 Delta) (Eq. 1.9), increasing; the penalised problem is convex
    with a kink at Delta0 = -beta_hat, where beta becomes 0.  Its minimiser:
      g(Delta) + lam = 0  (the root with b + lam) if that root lies beyond Delta0,
      g(Delta) - lam = 0  (the root with b - lam) if that root lies before Delta0,
      Delta0 otherwise (beta is set to 0).
    The decision uses the unclamped roots; the result is then clamped to
    |Z0 Delta| <= clamp (a step between 0 and the minimiser of a convex
    function still lowers it).  lam = 0 gives am_root."""
    b = np.asarray(b, dtype=np.float64)
    lam = np.broadcast_to(np.asarray(lam, dtype=np.float64), b.shape)
    beta_hat = np.broadcast_to(np.asarray(beta_hat, dtype=np.float64), b.shape)
    up = am_root(b + lam, bp, bm, 1.0, np.inf)          # Z0 Delta for g = -lam
    dn = am_root(b - lam, bp, bm, 1.0, np.inf)          # Z0 Delta for g = +lam
    t0 = -Z0 * beta_hat
    kink = ~(up > t0) & ~(dn < t0)
    t = np.where(up > t0, up, np.where(dn < t0, dn, t0))
    # at the kink beta becomes exactly 0 (unless the clamp stops the step short)
    return np.where(kink & (np.abs(t0) <= clamp), -beta_hat, np.clip(t, -clamp, clamp) / Z0)


def l1_details(beta, nx: int, ny: int, L: int, act=None) -> float:
    """sum over the detail coefficients of |beta| (the penalty of am_root_l1)."""
    _, typ, _, _ = haar.coefficient_info(nx, ny, L)
    sel = typ >= 0
    return float(np.sum(np.abs(np.asarray(beta)[sel])))


# ---------------------------------------------------------------------------
# the wavelet tree
# ---------------------------------------------------------------------------

def empty_tree(nx: int, ny: int, L: int) -> List[np.ndarray]:
    """tree[l-1][by, bx] is True when the level-l block's details are active."""
    return [np.zeros((ny >> l, nx >> l), dtype=bool) for l in range(1, L + 1)]


def active_mask(tree: List[np.ndarray], nx: int, ny: int, L: int) -> np.ndarray:
    level, typ, bx, by = haar.coefficient_info(nx, ny, L)
    act = typ == -1
    for l in range(1, L + 1):
        sel = (level == l) & (typ >= 0)
        act[sel] = tree[l - 1][by[sel], bx[sel]]
    return act


def leaf_levels(tree: List[np.ndarray], nx: int, ny: int, L: int) -> np.ndarray:
    """Level of the leaf block holding each pixel ([ny, nx])."""
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    lev = np.full((ny, nx), L, dtype=np.int64)
    descending = np.ones((ny, nx), dtype=bool)
    for l in range(L, 0, -1):
        exp_l = tree[l - 1][iy >> l, ix >> l]
        descending &= exp_l
        lev[descending] = l - 1
    return lev


def expand(tree: List[np.ndarray], S: np.ndarray, tau: float) -> List[np.ndarray]:
    """One expansion step on the criterion image S ([ny, nx]); the leaf of each
    selected pixel is read from the tree before the step."""
    ny, nx = S.shape
    L = len(tree)
    S64 = np.asarray(S, dtype=np.float64)
    if tau < 0:
        sel = np.ones_like(S64, dtype=bool)
    else:
        sel = S64 > float(tau) * float(S64.max())
    lev = leaf_levels(tree, nx, ny, L)
    new = [t.copy() for t in tree]
    iy, ix = np.nonzero(sel & (lev >= 1))
    for l in range(1, L + 1):
        m = lev[iy, ix] == l
        new[l - 1][iy[m] >> l, ix[m] >> l] = True
    return new


# ---------------------------------------------------------------------------
# the iterations
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class AMResult:
    beta: np.ndarray
    mu: np.ndarray
    cost: np.ndarray                  # I(d||qhat^(j)), j = 0..n_iter
    z0: np.ndarray                    # Z0 used at each iteration
    tree: Optional[List[np.ndarray]]
    trees: list                       # tree after each expansion
    n_active: np.ndarray


def _row_abs_max(Ps: sp.spmatrix) -> float:
    return float(np.max(np.asarray(abs(Ps).sum(axis=1)).ravel()))


@dataclasses.dataclass
class ActiveColumns:
    """The columns of Phi active in one tree epoch, with the quantities of
    Algorithm 1 that depend on them alone: Z0 (Eq. 1.61, a max over rays of
    the row sums of |phi|) and the positive and negative parts of phi whose
    products with qhat give bhat+ and bhat- (Eq. 1.10).  Built once per
    epoch; every iteration of the epoch reuses them (the same numbers an
    iteration would form from scratch)."""
    P: sp.csc_matrix
    Pplus: sp.csc_matrix
    Pminus: sp.csc_matrix
    Z0: float


def active_columns(Ps: sp.spmatrix) -> ActiveColumns:
    Ps = sp.csc_matrix(Ps)
    return ActiveColumns(Ps, Ps.maximum(0).tocsc(), Ps.minimum(0).tocsc(), _row_abs_max(Ps))


def am_step(A, b_s, beta_s, d, I0):
    """One AM iteration on the active columns A (an ActiveColumns, or a
    matrix of Phi's active columns); returns (Delta, cost, Z0)."""
    if not isinstance(A, ActiveColumns):
        A = active_columns(A)
    p = A.P @ beta_s
    q = np.broadcast_to(np.asarray(I0, dtype=np.float64), p.shape) * np.exp(-p)
    cost = idiv(d, I0, p)
    bp = A.Pplus.T @ q
    bm = A.Pminus.T @ q
    return am_root(b_s, bp, bm, A.Z0), cost, A.Z0


def wavelet_am(H: sp.spmatrix, d, I0, nx: int, ny: int, L: int, n_iter: int,
               expand_at: Sequence[int] = (), taus: Sequence[float] = (),
               tree0: Optional[List[np.ndarray]] = None, nz: int = 1, lam: float = 0.0) -> AMResult:
    """Algorithm 1 with the tree schedule; nz > 1 runs the per-slice 2-D Haar
    mode (one tree shared by all slices, criterion summed over slices).

    lam > 0 (2-D only): the regularised problem of Eq. 1.1 with
    lam R(mu) = lam * sum over the detail coefficients of |beta|; every detail
    coefficient takes the penalised step am_root_l1, the approximations the
    plain one, and the cost history holds I(d || qhat) + lam * sum |beta_det|,
    which then decreases at every iteration."""
    d = np.asarray(d, dtype=np.float64).ravel()
    Om2 = haar.basis_matrix(nx, ny, L)
    Omega = sp.block_diag([Om2] * nz, format="csc") if nz > 1 else Om2
    Phi = (H @ Omega).tocsc()
    b = Phi.T @ d                                        # Eq. 1.6, all z
    N = nx * ny
    beta = np.zeros(N * nz)
    tree = [t.copy() for t in tree0] if tree0 is not None else empty_tree(nx, ny, L)
    costs, z0s, trees, nact = [], [], [], []
    sched = dict(zip(expand_at, taus))
    if lam > 0 and nz > 1:
        raise ValueError("the penalised step is defined for 2-D images")
    _, typ, _, _ = haar.coefficient_info(nx, ny, L)
    det = typ >= 0
    pen = (lambda be: lam * float(np.sum(np.abs(be[det])))) if lam > 0 else (lambda be: 0.0)
    A = None
    for j in range(n_iter):
        act = np.tile(active_mask(tree, nx, ny, L), nz)
        if A is None:                                    # a new tree epoch
            A = active_columns(Phi[:, act])
        if lam > 0:
            p_ = A.P @ beta[act]
            q_ = np.broadcast_to(np.asarray(I0, dtype=np.float64), p_.shape) * np.exp(-p_)
            cost = idiv(d, I0, p_) + pen(beta)
            Z0 = A.Z0
            bp_, bm_ = A.Pplus.T @ q_, A.Pminus.T @ q_
            delta = np.where(det[act], am_root_l1(b[act], bp_, bm_, Z0, beta[act], lam),
                             am_root(b[act], bp_, bm_, Z0))
        else:
            delta, cost, Z0 = am_step(A, b[act], beta[act], d, I0)
        costs.append(cost)
        z0s.append(Z0)
        nact.append(int(act.sum()))
        beta[act] += delta
        if (j + 1) in sched:
            mu = (Omega @ beta).reshape(nz, ny, nx)
            tree = expand(tree, mu.sum(axis=0), sched[j + 1])
            trees.append([t.copy() for t in tree])
            A = None
    costs.append(idiv(d, I0, Phi @ beta) + pen(beta))
    mu = (Omega @ beta).reshape(nz, ny, nx) if nz > 1 else (Omega @ beta).reshape(ny, nx)
    return AMResult(beta, mu, np.array(costs), np.array(z0s), tree, trees, np.array(nact))


def plain_am(H: sp.spmatrix, d, I0, n_iter: int, shape=None, nonneg: bool = False) -> AMResult:
    """O'Sullivan-Benac AM: Algorithm 1 with Omega = I and every pixel active.

    nonneg: keep mu >= 0 by ending each pixel's step at mu = 0 where the
    unconstrained step would cross it.  With Omega = I the surrogate of
    Eq. 1.8 is a sum of one-dimensional convex functions, one per pixel, so
    this clamp is its exact minimiser over mu >= 0 and the decrease guarantee
    holds.  Algorithm 1 itself is unconstrained (the default); the paper's
    problem statement (Eq. 1.3) asks for a nonnegative image."""
    d = np.asarray(d, dtype=np.float64).ravel()
    Hc = H.tocsc()
    b = Hc.T @ d
    A = active_columns(Hc)
    mu = np.zeros(H.shape[1])
    costs, z0s = [], []
    for _ in range(n_iter):
        delta, cost, Z0 = am_step(A, b, mu, d, I0)
        costs.append(cost)
        z0s.append(Z0)
        mu += delta
        if nonneg:
            mu = np.maximum(mu, 0.0)
    costs.append(idiv(d, I0, Hc @ mu))
    out = mu.reshape(shape) if shape is not None else mu
    return AMResult(mu, out, np.array(costs), np.array(z0s), None, [], np.array([H.shape[1]] * n_iter))


# ---------------------------------------------------------------------------
# ordered subsets (the paper's Conclusion combines the method with ordered
# subsets; the combination is read here as: a sub-iteration is one step of
# Algorithm 1 on the rays of one subset of views)
# ---------------------------------------------------------------------------

def view_subsets(n_views: int, n_subsets: int) -> List[np.ndarray]:
    """Subset s holds the views k with k mod S = s (interleaved, so every
    subset spans the whole angular range)."""
    return [np.arange(s, n_views, n_subsets) for s in range(n_subsets)]


@dataclasses.dataclass
class OSResult:
    beta: np.ndarray
    mu: np.ndarray
    cost: np.ndarray                  # full I(d||qhat) at the start of each outer iteration, and at the end
    z0: np.ndarray                    # [n_iter, S]: Z0 of each sub-iteration (max over its subset's rays)
    sub_cost: np.ndarray              # [n_iter, S, 2]: the subset's own I-divergence before / after its step
    tree: Optional[List[np.ndarray]]


def os_wavelet_am(H: sp.spmatrix, d, I0, nx: int, ny: int, L: int, n_iter: int, n_subsets: int, n_bins: int,
                  expand_at: Sequence[int] = (), taus: Sequence[float] = ()) -> OSResult:
    """Algorithm 1 with ordered subsets of views.  Each outer iteration visits
    the subsets in order s = 0..S-1; sub-iteration s is one step of Algorithm 1
    restricted to the rays y of subset s: b_s(z) = sum_{y in s} d(y) phi(y|z)
    (Eq. 1.6 on the subset), qhat and bhat+- over those rays (Eq. 1.10), and
    Z0_s = max over those rays of sum_{z in Zs} |phi(y|z)| (Eq. 1.61), which
    keeps the convex decomposition valid for the subset's surrogate.  The tree
    grows after the listed outer iterations.  S = 1 is Algorithm 1."""
    d = np.asarray(d, dtype=np.float64).ravel()
    I0a = np.broadcast_to(np.asarray(I0, dtype=np.float64), d.shape)
    Omega = haar.basis_matrix(nx, ny, L)
    Phi = (H @ Omega).tocsr()
    n_views = Phi.shape[0] // n_bins
    rows = [(k[:, None] * n_bins + np.arange(n_bins)[None, :]).ravel() for k in view_subsets(n_views, n_subsets)]
    Phis = [Phi[r].tocsc() for r in rows]
    bs = [P.T @ d[r] for P, r in zip(Phis, rows)]
    beta = np.zeros(nx * ny)
    tree = empty_tree(nx, ny, L)
    sched = dict(zip(expand_at, taus))
    costs, z0s, subc = [], np.zeros((n_iter, n_subsets)), np.zeros((n_iter, n_subsets, 2))
    for j in range(n_iter):
        costs.append(idiv(d, I0a, Phi @ beta))
        act = active_mask(tree, nx, ny, L)
        for s_ in range(n_subsets):
            Ps = Phis[s_][:, act]
            ds, Is = d[rows[s_]], I0a[rows[s_]]
            delta, c_before, Z0 = am_step(Ps, bs[s_][act], beta[act], ds, Is)
            beta[act] += delta
            z0s[j, s_] = Z0
            subc[j, s_] = (c_before, idiv(ds, Is, Ps @ beta[act]))
        if (j + 1) in sched:
            tree = expand(tree, (Omega @ beta).reshape(ny, nx), sched[j + 1])
    costs.append(idiv(d, I0a, Phi @ beta))
    return OSResult(beta, (Omega @ beta).reshape(ny, nx), np.array(costs), z0s, subc, tree)


# ---------------------------------------------------------------------------
# 3-D Haar trees (volume blocks of 2^l voxels per side, seven details each)
# ---------------------------------------------------------------------------

def empty_tree3d(nx: int, ny: int, nz: int, L: int) -> List[np.ndarray]:
    """tree[l-1][bz, by, bx] is True when the level-l block's 7 details are active."""
    return [np.zeros((nz >> l, ny >> l, nx >> l), dtype=bool) for l in range(1, L + 1)]


def active_mask3d(tree, nx: int, ny: int, nz: int, L: int) -> np.ndarray:
    from . import haar3d
    level, typ, bx, by, bz = haar3d.coefficient_info(nx, ny, nz, L)
    act = typ == 0
    for l in range(1, L + 1):
        sel = (level == l) & (typ > 0)
        act[sel] = tree[l - 1][bz[sel], by[sel], bx[sel]]
    return act


def leaf_levels3d(tree, nx: int, ny: int, nz: int, L: int) -> np.ndarray:
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lev = np.full((nz, ny, nx), L, dtype=np.int64)
    descending = np.ones((nz, ny, nx), dtype=bool)
    for l in range(L, 0, -1):
        descending &= tree[l - 1][iz >> l, iy >> l, ix >> l]
        lev[descending] = l - 1
    return lev


def expand3d(tree, S: np.ndarray, tau: float):
    """The expansion rule on a volume S ([nz, ny, nx])."""
    nz, ny, nx = S.shape
    L = len(tree)
    S64 = np.asarray(S, dtype=np.float64)
    sel = np.ones_like(S64, dtype=bool) if tau < 0 else S64 > float(tau) * float(S64.max())
    lev = leaf_levels3d(tree, nx, ny, nz, L)
    new = [t.copy() for t in tree]
    iz, iy, ix = np.nonzero(sel & (lev >= 1))
    for l in range(1, L + 1):
        m = lev[iz, iy, ix] == l
        new[l - 1][iz[m] >> l, iy[m] >> l, ix[m] >> l] = True
    return new


def wavelet_am3d(H: sp.spmatrix, d, I0, nx: int, ny: int, nz: int, L: int, n_iter: int,
                 expand_at: Sequence[int] = (), taus: Sequence[float] = ()) -> AMResult:
    """Algorithm 1 with a 3-D Haar basis and a 3-D tree (criterion S = mu)."""
    from . import haar3d
    d = np.asarray(d, dtype=np.float64).ravel()
    Omega = haar3d.basis_matrix(nx, ny, nz, L)
    Phi = (H @ Omega).tocsc()
    b = Phi.T @ d
    beta = np.zeros(nx * ny * nz)
    tree = empty_tree3d(nx, ny, nz, L)
    costs, z0s, trees, nact = [], [], [], []
    sched = dict(zip(expand_at, taus))
    A = None
    for j in range(n_iter):
        act = active_mask3d(tree, nx, ny, nz, L)
        if A is None:                                    # a new tree epoch
            A = active_columns(Phi[:, act])
        delta, cost, Z0 = am_step(A, b[act], beta[act], d, I0)
        costs.append(cost)
        z0s.append(Z0)
        nact.append(int(act.sum()))
        beta[act] += delta
        if (j + 1) in sched:
            tree = expand3d(tree, (Omega @ beta).reshape(nz, ny, nx), sched[j + 1])
            trees.append([t.copy() for t in tree])
            A = None
    costs.append(idiv(d, I0, Phi @ beta))
    return AMResult(beta, (Omega @ beta).reshape(nz, ny, nx), np.array(costs), np.array(z0s), tree, trees,
                    np.array(nact))
