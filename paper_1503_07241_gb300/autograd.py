"""torch.autograd.Function around the weighted-PageRank forward and its adjoint.

    x = WeightedPageRank.apply(w, graph, r, steps, ckpt_every)

`w` is a CUDA float32 tensor of edge weights in the graph's CSR edge order
(gm_graph_get_edges); the returned `x` is x^steps.  The backward pass runs the
hand-written adjoint kernels (reverse SpMV + edge gradient, recomputed from
checkpoints) -- no autograd tape is built through the supersteps.
"""
from __future__ import annotations

import torch


class WeightedPageRank(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, graph, r=0.15, steps=30, ckpt_every=5):
        if not (w.is_cuda and w.dtype == torch.float32 and w.is_contiguous()):
            raise ValueError("w must be a contiguous CUDA float32 tensor")
        ctx.graph = graph
        return graph.wpagerank_forward(w.detach(), r, steps, ckpt_every)

    @staticmethod
    def backward(ctx, grad_x):
        return ctx.graph.wpagerank_backward(grad_x.float()), None, None, None, None
