"""torch.autograd Functions over libwam (argument marshalling only).

* `PhiProject`: p = Phi beta = H Omega beta on the full L-level Haar basis;
  its hand-written backward is the back-projector, Phi^T g.
* `IDivLoss`: L(beta) = I(d || I0 exp(-Phi beta)) + lambda sum |beta_detail|
  and its gradient Phi^T (d - qhat) + lambda sign(beta_detail) from one
  fused call.
* `AMUnroll`: n steps of the AM update (Algorithm 1 on the full tree, fixed
  Z0), differentiable with respect to the starting coefficients.  Only the
  iterates are kept (per-step checkpoints); the backward recomputes qhat and
  bhat+- of each step and applies the transposed Jacobian of the step:
  gbar <- gbar - Phi^T Q (Phi+ (D+ gbar) + Phi- (D- gbar)), with Q = diag(qhat),
  Phi+- the positive / negative parts of Phi and D+- the derivatives of the
  root of Eq. 1.9 with respect to bhat+-.

Inputs are CUDA float32 tensors in the coefficient layout of include/wam.h;
a leading batch dimension goes to the library's batch calls in one call
each.  Every numeric step (b = Phi^T d, the step's transposed Jacobian
including its identity term) runs in libwam's kernels on the current stream.
"""
from __future__ import annotations

import torch

from . import wam


def _st():
    return wam.current_stream()


class Operators:
    """A wam.Context plus the Haar levels of the coefficient vectors."""

    def __init__(self, ctx: "wam.Context", levels: int):
        self.ctx = ctx
        self.levels = levels
        g = ctx.geom
        self.N = g.nx * g.ny
        self.M = g.n_views * g.n_bins
        self._masks = None
        self._b = None
        self._z0 = None

    # ---- linear operators -------------------------------------------------
    def phi(self, beta: torch.Tensor) -> torch.Tensor:
        p = torch.empty(self.M, dtype=torch.float32, device=beta.device)
        beta = beta.contiguous()
        self.ctx.check(wam.wam_project_coef(self.ctx.h, self.levels, wam.ptr(beta), wam.ptr(p), _st()))
        return p

    def phi_t(self, s: torch.Tensor) -> torch.Tensor:
        g = torch.empty(self.N, dtype=torch.float32, device=s.device)
        s = s.contiguous()
        self.ctx.check(wam.wam_backproject_coef(self.ctx.h, self.levels, wam.ptr(s), wam.ptr(g), _st()))
        return g

    def phi_batch(self, beta: torch.Tensor) -> torch.Tensor:
        beta = beta.contiguous()
        p = torch.empty(beta.shape[0], self.M, dtype=torch.float32, device=beta.device)
        self.ctx.check(wam.wam_project_coef_batch(self.ctx.h, self.levels, beta.shape[0], wam.ptr(beta), wam.ptr(p),
                                                  _st()))
        return p

    def phi_t_batch(self, s: torch.Tensor) -> torch.Tensor:
        s = s.contiguous()
        g = torch.empty(s.shape[0], self.N, dtype=torch.float32, device=s.device)
        self.ctx.check(wam.wam_backproject_coef_batch(self.ctx.h, self.levels, s.shape[0], wam.ptr(s), wam.ptr(g),
                                                      _st()))
        return g

    def loss_grad(self, beta: torch.Tensor, lam: float):
        beta = beta.contiguous()
        loss = torch.empty(1, dtype=torch.float64, device=beta.device)
        grad = torch.empty(self.N, dtype=torch.float32, device=beta.device)
        self.ctx.check(wam.wam_idiv_grad(self.ctx.h, self.levels, wam.ptr(beta), float(lam), wam.ptr(loss),
                                         wam.ptr(grad), 0, _st()))
        return loss, grad

    # ---- pieces of one AM step on the full tree ---------------------------
    def masks(self, device):
        if self._masks is None:
            n = self.ctx.mask_bytes(self.levels)
            self._masks = torch.ones(max(1, n), dtype=torch.uint8, device=device)
        return self._masks

    def setup(self, d: torch.Tensor):
        """b = Phi^T d in FP64 (the precompute of Algorithm 1, from the context's
        data) and Z0 of the full tree."""
        dev = d.device
        m = self.masks(dev)
        self._b = torch.empty(self.N, dtype=torch.float64, device=dev)
        self.ctx.check(wam.wam_precompute_b(self.ctx.h, self.levels, wam.ptr(self._b), _st()))
        self._z0 = torch.empty(1, dtype=torch.float64, device=dev)
        self.ctx.check(wam.wam_z0(self.ctx.h, self.levels, wam.ptr(m), wam.ptr(self._z0), _st()))

    def qhat_split(self, beta64: torch.Tensor):
        """qhat at beta and its split back-projections bhat+, bhat-."""
        dev = beta64.device
        m = self.masks(dev)
        mu = torch.empty(self.N, dtype=torch.float32, device=dev)
        q = torch.empty(self.M, dtype=torch.float32, device=dev)
        cost = torch.empty(1, dtype=torch.float64, device=dev)
        self.ctx.check(wam.wam_synthesize(self.ctx.h, self.levels, wam.ptr(m), wam.ptr(beta64), wam.ptr(mu), _st()))
        self.ctx.check(wam.wam_forward(self.ctx.h, self.levels, wam.ptr(m), wam.ptr(mu), wam.ptr(q), wam.ptr(cost),
                                       _st()))
        bp = torch.empty(self.N, dtype=torch.float64, device=dev)
        bm = torch.empty_like(bp)
        self.ctx.check(wam.wam_split_backproject(self.ctx.h, self.levels, wam.ptr(m), wam.ptr(q), wam.ptr(bp),
                                                 wam.ptr(bm), _st()))
        return q, bp, bm

    def am_step(self, beta64: torch.Tensor, clamp: float = 30.0) -> torch.Tensor:
        """One AM update of every coefficient (in place on an FP64 copy)."""
        _, bp, bm = self.qhat_split(beta64)
        out = beta64.clone()
        m = self.masks(beta64.device)
        self.ctx.check(wam.wam_update(self.ctx.h, self.levels, wam.ptr(m), wam.ptr(self._b), wam.ptr(bp),
                                      wam.ptr(bm), wam.ptr(self._z0), clamp, wam.ptr(out), _st()))
        return out

    def am_step_vjp(self, beta64: torch.Tensor, gbar: torch.Tensor, clamp: float = 30.0) -> torch.Tensor:
        """The transposed Jacobian of one AM step at beta applied to gbar (one
        library call)."""
        gbar = gbar.contiguous()
        out = torch.empty_like(gbar)
        self.ctx.check(wam.wam_am_step_vjp(self.ctx.h, self.levels, wam.ptr(beta64.contiguous()), wam.ptr(self._b),
                                           wam.ptr(self._z0), clamp, wam.ptr(gbar), wam.ptr(out), _st()))
        return out

    def loss_grad_batch(self, beta: torch.Tensor, lam: float):
        """wam_idiv_grad over the rows of beta ([n, N]) in one call."""
        beta = beta.contiguous()
        n = beta.shape[0]
        loss = torch.empty(n, dtype=torch.float64, device=beta.device)
        grad = torch.empty_like(beta)
        self.ctx.check(wam.wam_idiv_grad_batch(self.ctx.h, self.levels, n, wam.ptr(beta), float(lam), wam.ptr(loss),
                                               wam.ptr(grad), _st()))
        return loss, grad


class PhiProject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, beta, ops: Operators):
        ctx.ops = ops
        b = beta.detach().float()
        return ops.phi(b) if b.dim() == 1 else ops.phi_batch(b.reshape(b.shape[0], -1))

    @staticmethod
    def backward(ctx, gp):
        g = gp.float()
        return (ctx.ops.phi_t(g) if g.dim() == 1 else ctx.ops.phi_t_batch(g.reshape(g.shape[0], -1))), None


class IDivLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, beta, ops: Operators, lam: float):
        b = beta.detach().float()
        if b.dim() == 1:
            loss, grad = ops.loss_grad(b, lam)
            ctx.save_for_backward(grad)
            return loss[0]
        loss, grad = ops.loss_grad_batch(b.reshape(b.shape[0], -1), lam)
        ctx.save_for_backward(grad.reshape(b.shape))
        return loss

    @staticmethod
    def backward(ctx, gl):
        grad, = ctx.saved_tensors
        gl = gl.to(torch.float32)
        return (gl.reshape(-1, *([1] * (grad.dim() - 1))) * grad if grad.dim() > 1 else gl * grad), None, None


class AMUnroll(torch.autograd.Function):
    @staticmethod
    def forward(ctx, beta0, ops: Operators, n_steps: int):
        if beta0.dim() != 1:
            raise ValueError("AMUnroll takes one coefficient vector")
        b = beta0.detach().to(torch.float64).contiguous()
        checkpoints = [b]
        for _ in range(n_steps):
            b = ops.am_step(b)
            checkpoints.append(b)
        ctx.ops = ops
        ctx.checkpoints = checkpoints[:-1]
        return b.float()

    @staticmethod
    def backward(ctx, gbar):
        g = gbar.float().contiguous()
        for b in reversed(ctx.checkpoints):
            g = ctx.ops.am_step_vjp(b, g)
        return g, None, None
