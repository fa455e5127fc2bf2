"""Helpers for the GPU tests: move synthetic inputs to the device and wrap
the library handles so they are released."""
from __future__ import annotations

import contextlib

import numpy as np


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


@contextlib.contextmanager
def gpu_graph(g, ground=0):
    """(ctx, tree, device CSR tensors) for a synth.Graph."""
    import paper_1911_04382_gb300 as G
    ctx = G.grass_ctx_create()
    rp, col, val = dev(g.rowptr), dev(g.col), dev(g.val)
    tree = None
    try:
        tree = G.grass_build_tree(ctx, rp, col, val, ground)
        yield ctx, tree, (rp, col, val)
    finally:
        if tree:
            G.grass_tree_destroy(tree)
        G.grass_ctx_destroy(ctx)


def tree_mask(ctx, tree, m):
    import torch
    import paper_1911_04382_gb300 as G
    out = torch.empty(m, dtype=torch.uint8, device="cuda")
    G.grass_tree_edges(ctx, tree, out)
    return host(out)
