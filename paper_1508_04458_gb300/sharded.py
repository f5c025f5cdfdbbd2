"""Algorithm 1 with the scan's views partitioned over ranks (one GPU per
rank, torch.distributed; NCCL on GPUs).

Every quantity of an iteration that sums over rays splits by views: the
back-projected data b = Phi^T d (Eq. 1.6), the split back-projections
bhat+ and bhat- (Eq. 1.10) and the I-divergence.  A rank owning views
[v0, v0 + n) computes its partial sums with its own scan, and one all-reduce
(sum) per iteration completes them.  Z0 = max over rays of sum_z |phi(y|z)|
(Eq. 1.61) is a max over rays, each complete on the rank owning its view: a
max all-reduce at each tree change.  The update (Eq. 1.9), the synthesis and
the tree growth read only these reduced values and the replicated beta, so
every rank keeps an identical copy of beta and of the tree without further
exchange.

The arithmetic of each step runs in a backend with the interface of
WamSteps (libwam's step-level calls on the rank's GPU); this module only
orders the steps and the exchanges.  Results equal the single-GPU
reconstruction up to the order of the FP32 partial sums.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import torch


def view_block(n_views: int, world: int, rank: int):
    """Contiguous, balanced block of views of `rank`: (first view, count)."""
    if world < 1 or not 0 <= rank < world or n_views < world:
        raise ValueError("need 0 <= rank < world <= n_views")
    base, extra = divmod(n_views, world)
    v0 = rank * base + min(rank, extra)
    return v0, base + (1 if rank < extra else 0)


def shard_geometry(geom, v0: int, n: int):
    """The scan of views v0 .. v0 + n - 1 of `geom` as a geometry of its own
    (view k at angle0 + k * angle_span / n_views, so the block keeps the
    spacing angle_span / n_views)."""
    step = geom.angle_span / geom.n_views
    return dataclasses.replace(geom, angle0=geom.angle0 + v0 * step, angle_span=n * step, n_views=n)


def shard_rows(d, geom, v0: int, n: int):
    """The rows of a full sinogram [n_views, ...] that belong to the block."""
    per_view = len(d.reshape(-1)) // geom.n_views
    return d.reshape(-1)[v0 * per_view:(v0 + n) * per_view]


class Comm:
    """Sum and max across the ranks of a process group (no-ops for one rank)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1

    def sum_(self, t: torch.Tensor) -> torch.Tensor:
        if self.world > 1:
            self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t

    def max_(self, t: torch.Tensor) -> torch.Tensor:
        if self.world > 1:
            self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return t


class WamSteps:
    """The steps of one iteration on the views of one rank, through libwam's
    step-level C-ABI calls on the current CUDA device (FP64 coefficients,
    FP32 images and sinograms).  d: this rank's counts as a [n, B] array."""

    def __init__(self, geom, d, I0, levels: int):
        from . import wam
        self.wam = wam
        self.ctx = wam.Context(geom)
        self.ctx.set_data(d, I0)
        self.L = levels
        self.N = geom.nx * geom.ny
        self.M = geom.n_views * geom.n_bins
        self.mb = self.ctx.mask_bytes(levels)
        self.d = torch.as_tensor(d, dtype=torch.float32).reshape(-1).cuda()
        self.dev = self.d.device

    def _chk(self, st):
        return self.ctx.check(st)

    def empty_masks(self):
        return torch.zeros(max(1, self.mb), dtype=torch.uint8, device=self.dev)

    def b_partial(self):
        w, s = self.wam, self.wam.current_stream()
        g = torch.empty(self.N, dtype=torch.float32, device=self.dev)
        self._chk(w.wam_backproject(self.ctx.h, w.ptr(self.d), w.ptr(g), s))
        g64 = g.double()
        b = torch.empty(self.N, dtype=torch.float64, device=self.dev)
        self._chk(w.wam_haar(self.ctx.h, self.L, w.ptr(g64), w.ptr(b), 0, s))
        torch.cuda.current_stream().synchronize()
        return b

    def z0(self, masks):
        w = self.wam
        z = torch.empty(1, dtype=torch.float64, device=self.dev)
        self._chk(w.wam_z0(self.ctx.h, self.L, w.ptr(masks), w.ptr(z), w.current_stream()))
        return z

    def synthesize(self, masks, beta):
        w = self.wam
        mu = torch.empty(self.N, dtype=torch.float32, device=self.dev)
        self._chk(w.wam_synthesize(self.ctx.h, self.L, w.ptr(masks), w.ptr(beta), w.ptr(mu), w.current_stream()))
        return mu

    def forward(self, masks, mu):
        w = self.wam
        q = torch.empty(self.M, dtype=torch.float32, device=self.dev)
        cost = torch.empty(1, dtype=torch.float64, device=self.dev)
        self._chk(w.wam_forward(self.ctx.h, self.L, w.ptr(masks), w.ptr(mu), w.ptr(q), w.ptr(cost),
                                w.current_stream()))
        return q, cost

    def split_backproject(self, masks, q):
        w = self.wam
        bp = torch.empty(self.N, dtype=torch.float64, device=self.dev)
        bm = torch.empty(self.N, dtype=torch.float64, device=self.dev)
        self._chk(w.wam_split_backproject(self.ctx.h, self.L, w.ptr(masks), w.ptr(q), w.ptr(bp), w.ptr(bm),
                                          w.current_stream()))
        return bp, bm

    def update(self, masks, b, bp, bm, z0, clamp, beta):
        w = self.wam
        self._chk(w.wam_update(self.ctx.h, self.L, w.ptr(masks), w.ptr(b), w.ptr(bp), w.ptr(bm), w.ptr(z0),
                               clamp, w.ptr(beta), w.current_stream()))

    def expand(self, mu, tau, masks):
        w = self.wam
        out = torch.empty_like(masks)
        self._chk(w.wam_expand(self.ctx.h, self.L, w.ptr(mu), float(tau), w.ptr(masks), w.ptr(out),
                               w.current_stream()))
        return out


@dataclasses.dataclass
class ShardedResult:
    beta: torch.Tensor        # FP64 coefficients (identical on every rank)
    mu: torch.Tensor          # final image
    cost: list                # I(d || qhat^(j)), j = 0..n_iters, summed over all views
    masks: torch.Tensor       # final tree
    z0: list                  # Z0 of each tree epoch


def reconstruct_sharded(steps, n_iters: int, expand_at: Sequence[int] = (), taus: Sequence[float] = (),
                        clamp: float = 30.0, comm: Optional[Comm] = None) -> ShardedResult:
    """Algorithm 1 from beta = 0 with the tree grown after the iterations in
    expand_at (thresholds taus), every sum over rays completed across ranks."""
    comm = comm or Comm()
    if list(expand_at) != sorted(set(expand_at)) or len(expand_at) != len(taus):
        raise ValueError("expand_at must be increasing, one tau each")
    sched = dict(zip(expand_at, taus))
    masks = steps.empty_masks()
    b = comm.sum_(steps.b_partial())                                    # a0, Eq. 1.6
    beta = torch.zeros_like(b)
    z0 = comm.max_(steps.z0(masks))                                      # a5, Eq. 1.61
    z0s = [float(z0.item())]
    cost = []
    N = b.numel()
    for j in range(n_iters):
        mu = steps.synthesize(masks, beta)                               # a1
        q, c = steps.forward(masks, mu)                                  # a2, a3
        bp, bm = steps.split_backproject(masks, q)                       # a4, Eq. 1.10
        red = comm.sum_(torch.cat([bp, bm, c.reshape(1).to(bp.dtype)]))  # the one exchange
        cost.append(red[-1:].clone())
        steps.update(masks, b, red[:N].contiguous(), red[N:2 * N].contiguous(), z0, clamp, beta)   # a6
        if (j + 1) in sched:                                             # a7, replicated
            mu = steps.synthesize(masks, beta)
            masks = steps.expand(mu, sched[j + 1], masks)
            z0 = comm.max_(steps.z0(masks))
            z0s.append(float(z0.item()))
    mu = steps.synthesize(masks, beta)
    _, c = steps.forward(masks, mu)
    cost.append(comm.sum_(c.reshape(1).to(torch.float64).clone()))
    return ShardedResult(beta, mu, torch.cat(cost).cpu().tolist(), masks, z0s)
