"""Shared helpers of the GPU tests: tree masks in the C-ABI layout, tensors."""
import numpy as np


def tree_to_masks(tree, L):
    """Oracle tree (tree[l-1] bool [gh, gw]) -> C-ABI bytes (levels L..1)."""
    return np.concatenate([tree[l - 1].astype(np.uint8).ravel() for l in range(L, 0, -1)]) \
        if L > 0 else np.zeros(0, np.uint8)


def masks_to_tree(masks, nx, ny, L):
    out = [None] * L
    off = 0
    for l in range(L, 0, -1):
        n = (nx >> l) * (ny >> l)
        out[l - 1] = masks[off:off + n].reshape(ny >> l, nx >> l).astype(bool)
        off += n
    return out


def random_tree(nx, ny, L, rng, p=0.5):
    """A random valid tree: a block may expand only if its parent did."""
    tree = [np.zeros((ny >> l, nx >> l), dtype=bool) for l in range(1, L + 1)]
    for l in range(L, 0, -1):
        r = rng.random((ny >> l, nx >> l)) < p
        if l < L:
            parent = np.kron(tree[l], np.ones((2, 2), dtype=bool))
            r &= parent
        tree[l - 1] = r
    return tree


def cuda(a, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda().contiguous()
