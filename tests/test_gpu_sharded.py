"""The view-sharded driver on the GPU through libwam's step-level calls:
one rank, and two ranks emulated on one GPU by two host threads whose
exchanges meet at a barrier (every sum taken in rank order, so both ranks
see the same values; no kernel waits on another), against the FP64 oracle
with the FP32 bounds of the other end-to-end tests (iterate 1e-4 relative,
cost 1e-4 relative + 2e-5 of the initial cost) and the tree bit-exact."""
import threading

import numpy as np
import pytest

from oracle import am
from oracle import system_matrix as smx
from paper_1508_04458_gb300 import inputs as I
from paper_1508_04458_gb300 import sharded

from gpu_helpers import tree_to_masks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

L, J, EXPAND_AT, TAUS = 3, 14, (3, 7), (0.1, -1.0)


class ThreadComm:
    """Sum / max across threads standing in for ranks."""

    def __init__(self, rank, shared):
        self.rank, self.sh = rank, shared
        self.world = len(shared["slots"])

    def _all(self, t, op):
        sh = self.sh
        sh["slots"][self.rank] = t
        sh["bar"].wait()
        acc = sh["slots"][0].clone()
        for k in range(1, self.world):
            acc = op(acc, sh["slots"][k])
        sh["bar"].wait()
        t.copy_(acc)
        return t

    def sum_(self, t):
        return self._all(t, torch.add)

    def max_(self, t):
        return self._all(t, torch.maximum)


def _check(p, res):
    ref = am.wavelet_am(smx.system_matrix(p.geom), p.d, p.I0, p.geom.nx, p.geom.ny, L, J,
                        expand_at=EXPAND_AT, taus=TAUS)
    mu = res.mu.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(mu - ref.mu.ravel()) <= 1e-4 * np.linalg.norm(ref.mu)
    np.testing.assert_allclose(res.cost, ref.cost, rtol=1e-4, atol=2e-5 * ref.cost[0])
    np.testing.assert_array_equal(res.masks.cpu().numpy(), tree_to_masks(ref.tree, L))


def test_one_rank():
    p = I.small_problem(80, 48, 37, 131, seed=71)
    steps = sharded.WamSteps(p.geom, p.d.astype(np.float32), p.I0, L)
    _check(p, sharded.reconstruct_sharded(steps, J, EXPAND_AT, TAUS))


def test_two_ranks_on_one_gpu():
    p = I.small_problem(80, 48, 37, 131, seed=72)
    world = 2
    shared = {"slots": [None] * world, "bar": threading.Barrier(world)}
    steps = []
    for r in range(world):
        v0, n = sharded.view_block(p.geom.n_views, world, r)
        steps.append(sharded.WamSteps(sharded.shard_geometry(p.geom, v0, n),
                                      sharded.shard_rows(p.d.astype(np.float32), p.geom, v0, n), p.I0, L))
    out, errs = [None] * world, []

    def run(r):
        try:
            out[r] = sharded.reconstruct_sharded(steps[r], J, EXPAND_AT, TAUS, comm=ThreadComm(r, shared))
        except Exception as e:  # pragma: no cover
            errs.append(e)
            shared["bar"].abort()

    th = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errs, errs
    torch.cuda.synchronize()
    assert torch.equal(out[0].beta, out[1].beta)
    _check(p, out[0])
