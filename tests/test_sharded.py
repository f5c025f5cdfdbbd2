"""The view-sharded driver on CPU ranks: two gloo processes, each with the
views of its block and a stand-in backend doing each step with the oracle's
FP64 arithmetic, reproduce the single-process oracle run of Algorithm 1
(iterates, cost history, tree, Z0 per epoch) to FP64 rounding; both ranks
hold the same beta bit for bit.  Plus the view partition itself."""
import math
import os
import socket

import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import am, haar
from oracle import system_matrix as smx
from paper_1508_04458_gb300 import inputs as I
from paper_1508_04458_gb300 import sharded

from gpu_helpers import masks_to_tree, tree_to_masks

NX, NY, V, B, L, J = 32, 32, 24, 45, 2, 10
EXPAND_AT, TAUS = (3, 6), (0.1, -1.0)


class OracleSteps:
    """One rank's steps with the oracle's arithmetic (CPU, FP64)."""

    def __init__(self, geom, d, I0, levels):
        self.nx, self.ny, self.L = geom.nx, geom.ny, levels
        self.H = smx.system_matrix(geom).tocsr()
        self.Om = haar.basis_matrix(self.nx, self.ny, levels)
        self.Phi = (self.H @ self.Om).tocsc()
        self.d = np.asarray(d, np.float64).ravel()
        self.I0 = I0
        self.mb = sum((self.nx >> l) * (self.ny >> l) for l in range(1, levels + 1))

    def _act(self, masks):
        return am.active_mask(masks_to_tree(masks.numpy(), self.nx, self.ny, self.L), self.nx, self.ny, self.L)

    def empty_masks(self):
        return torch.zeros(self.mb, dtype=torch.uint8)

    def b_partial(self):
        return torch.from_numpy(self.Phi.T @ self.d)

    def z0(self, masks):
        Ps = self.Phi[:, self._act(masks)]
        return torch.tensor([float(np.max(np.asarray(abs(Ps).sum(axis=1)).ravel()))], dtype=torch.float64)

    def synthesize(self, masks, beta):
        x = beta.numpy().copy()
        x[~self._act(masks)] = 0.0
        return torch.from_numpy(self.Om @ x)

    def forward(self, masks, mu):
        p = self.H @ mu.numpy()
        q = self.I0 * np.exp(-p)
        return torch.from_numpy(q), torch.tensor([am.idiv(self.d, self.I0, p)], dtype=torch.float64)

    def split_backproject(self, masks, q):
        act = self._act(masks)
        Ps = self.Phi[:, act]
        bp, bm = np.zeros(self.Phi.shape[1]), np.zeros(self.Phi.shape[1])
        bp[act] = Ps.maximum(0).T @ q.numpy()
        bm[act] = Ps.minimum(0).T @ q.numpy()
        return torch.from_numpy(bp), torch.from_numpy(bm)

    def update(self, masks, b, bp, bm, z0, clamp, beta):
        act = self._act(masks)
        x = beta.numpy()
        x[act] += am.am_root(b.numpy()[act], bp.numpy()[act], bm.numpy()[act], float(z0.item()), clamp)

    def expand(self, mu, tau, masks):
        tree = am.expand(masks_to_tree(masks.numpy(), self.nx, self.ny, self.L),
                         mu.numpy().reshape(self.ny, self.nx), tau)
        return torch.from_numpy(tree_to_masks(tree, self.L))


def _problem():
    return I.small_problem(NX, NY, V, B, seed=61)


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _problem()
        v0, n = sharded.view_block(p.geom.n_views, world, rank)
        steps = OracleSteps(sharded.shard_geometry(p.geom, v0, n), sharded.shard_rows(p.d, p.geom, v0, n), p.I0, L)
        r = sharded.reconstruct_sharded(steps, J, EXPAND_AT, TAUS)
        np.savez(out % rank, beta=r.beta.numpy(), cost=np.array(r.cost), masks=r.masks.numpy(), z0=np.array(r.z0))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_cpu_ranks_match_the_oracle(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "rank%d.npz")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    r0, r1 = np.load(out % 0), np.load(out % 1)
    np.testing.assert_array_equal(r0["beta"], r1["beta"])
    np.testing.assert_array_equal(r0["masks"], r1["masks"])
    p = _problem()
    ref = am.wavelet_am(smx.system_matrix(p.geom), p.d, p.I0, NX, NY, L, J, expand_at=EXPAND_AT, taus=TAUS)
    assert np.linalg.norm(r0["beta"] - ref.beta) <= 1e-10 * np.linalg.norm(ref.beta)
    np.testing.assert_allclose(r0["cost"], ref.cost, rtol=1e-10)
    np.testing.assert_array_equal(r0["masks"], tree_to_masks(ref.tree, L))
    # Z0 of each tree epoch: the first and one after each expansion
    epochs = [0] + list(EXPAND_AT)
    np.testing.assert_allclose(r0["z0"], [ref.z0[e] for e in epochs], rtol=1e-12)


def test_view_blocks():
    for nv, world in [(720, 1), (720, 8), (37, 4), (5, 5)]:
        blocks = [sharded.view_block(nv, world, r) for r in range(world)]
        assert blocks[0][0] == 0 and sum(n for _, n in blocks) == nv
        assert all(blocks[k][0] + blocks[k][1] == blocks[k + 1][0] for k in range(world - 1))
        assert max(n for _, n in blocks) - min(n for _, n in blocks) <= 1
    with pytest.raises(ValueError):
        sharded.view_block(3, 4, 0)
    g = I.geom_fan512()
    s = sharded.shard_geometry(g, 180, 90)
    assert s.n_views == 90 and math.isclose(s.angle0, 180 * 2 * math.pi / 720)
    assert math.isclose(s.angle_span / s.n_views, g.angle_span / g.n_views)


class FailingSteps(OracleSteps):
    """A rank whose forward step fails at its third call (a host-side fault)."""

    calls = 0

    def forward(self, masks, mu):
        FailingSteps.calls += 1
        if FailingSteps.calls == 3:
            raise RuntimeError("injected step failure")
        return super().forward(masks, mu)


def _worker_fail(rank, world, port, out):
    import datetime
    import time
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    p = _problem()
    v0, n = sharded.view_block(p.geom.n_views, world, rank)
    cls = FailingSteps if rank == 1 else OracleSteps
    steps = cls(sharded.shard_geometry(p.geom, v0, n), sharded.shard_rows(p.d, p.geom, v0, n), p.I0, L)
    t0 = time.monotonic()
    try:
        sharded.reconstruct_sharded(steps, J, EXPAND_AT, TAUS)
        outcome = "finished"
    except Exception as e:   # the failure as each rank sees it
        outcome = type(e).__name__ + ": " + str(e)[:200]
    with open(out % rank, "w") as f:
        f.write("%s\n%.1f\n" % (outcome, time.monotonic() - t0))
    if rank == 1:
        os._exit(0)          # the failed rank leaves without its remaining collectives
    dist.destroy_process_group()


def test_a_failing_rank_ends_the_others_collective_with_an_error(tmp_path):
    # rank 1's third forward raises and the rank leaves; rank 0 learns of it
    # from its next all-reduce, which fails (peer gone, or the 10 s process-
    # group timeout) instead of waiting forever
    import torch.multiprocessing as mp
    out = str(tmp_path / "rank%d.txt")
    mp.spawn(_worker_fail, args=(2, _free_port(), out), nprocs=2, join=True)
    r0 = open(out % 0).read().split("\n")
    r1 = open(out % 1).read().split("\n")
    assert r1[0].startswith("RuntimeError: injected step failure")
    assert r0[0] != "finished", r0
    assert float(r0[1]) < 60.0
