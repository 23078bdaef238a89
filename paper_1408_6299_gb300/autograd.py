"""The state solve as a differentiable PyTorch operation.

``transport(m0, v, op)`` returns m_1 = m(t=1) of dm/dt + grad m . v = 0 with
m(0) = m0 (Eq. first-order-forward) on the GPU. Its backward pass is the
adjoint solve of the library (Eq. first-order-adjoint run backward from
lambda_1 = -dL/dm_1), which returns dL/dv = int b_l lambda grad m dt and
dL/dm0 = -lambda_0. With the discrete quadrature (the default of
:func:`make_transport`) both are the exact derivatives of the Heun-discretised
map, so they agree with finite differences to rounding.

When the stored state of all n_t + 1 time nodes would exceed the memory budget,
the operator keeps every K-th state and recomputes the others in the backward
pass (time checkpointing).
"""
from __future__ import annotations

import torch

from . import lib


def make_transport(n, n_t, n_c=1, memory_budget_bytes=None, quadrature=lib.REG_QUAD_DISCRETE, stream=None):
    """A library context for differentiable transport on grid n with n_t steps.

    The regulariser arguments of the context do not enter the transport; they
    are fixed to H1 and beta = 1. Checkpointing is chosen so that the stored
    state gradients fit memory_budget_bytes (default: a quarter of the free
    device memory).
    """
    n = tuple(int(k) for k in n)
    d = len(n)
    N = 1
    for k in n:
        N *= k
    if memory_budget_bytes is None:
        free, _ = torch.cuda.mem_get_info()
        memory_budget_bytes = free // 4
    per_node = 2 * d * N * 8  # state gradient and stage gradient, double precision
    ckpt = 0
    if (n_t + 1) * per_node > memory_budget_bytes:
        for K in range(1, n_t + 1):
            if n_t % K == 0 and (K + 1) * per_node + (n_t // K + 1) * N * 8 <= memory_budget_bytes:
                ckpt = K
        if ckpt == 0:
            ckpt = 1
    return lib.Registration(n, n_t, n_c, 1.0, lib.REG_H1, False, lib.REG_FP64, ckpt, stream=stream,
                            quadrature=quadrature)


class TransportFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m0, v, op):
        m0c = m0.detach().contiguous()
        vc = v.detach().contiguous()
        m1 = torch.empty_like(m0c)
        op.transport(vc, m0c, m1)
        ctx.save_for_backward(m0c, vc)
        ctx.op = op
        return m1

    @staticmethod
    def backward(ctx, G):
        m0, v = ctx.saved_tensors
        gv = torch.empty_like(v) if ctx.needs_input_grad[1] else None
        gm = torch.empty_like(m0) if ctx.needs_input_grad[0] else None
        ctx.op.transport_adjoint(v, m0, G.contiguous(), gv, gm)
        return gm, gv, None


def transport(m0: torch.Tensor, v: torch.Tensor, op: lib.Registration) -> torch.Tensor:
    """m_1 of the transport of m0 (shape n) by the velocity coefficients v
    (shape (n_c, d, *n)); float64 CUDA tensors."""
    return TransportFn.apply(m0, v, op)
