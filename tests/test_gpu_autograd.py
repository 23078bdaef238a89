"""The differentiable transport (torch.autograd.Function over the CUDA state
and adjoint solves) on the 64^3 Stokes workload with n_c = 3 Chebyshev
coefficients and n_t = 32: central finite differences (h = 1e-6, FP64) along 20
seeded directions, agreement with the oracle's discrete-adjoint gradient, and
exactness in the template (the map is linear in m0)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1408_6299_gb300 import autograd as AG
from paper_1408_6299_gb300 import synth
from gpu_util import cuda, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload():
    c = synth.stokes_3d(64)
    op = AG.make_transport(c["n"], c["n_t"], c["n_c"])
    W = np.random.default_rng(9).standard_normal(c["n"])
    return c, op, W


def loss(m1, W):
    return (m1 * W).sum() + 0.5 * (m1 ** 2).sum()


def test_gradient_matches_central_differences_on_20_directions(workload):
    c, op, W = workload
    v = cuda(c["v_true"]).requires_grad_(True)
    m0 = cuda(c["mT"])
    Wt = cuda(W)
    L = loss(AG.transport(m0, v, op), Wt)
    (gv,) = torch.autograd.grad(L, v)
    eps = 1e-6
    errs = []
    for k in range(20):
        w = cuda(np.random.default_rng(200 + k).standard_normal(c["v_true"].shape))
        with torch.no_grad():
            lp = loss(AG.transport(m0, v + eps * w, op), Wt)
            lm = loss(AG.transport(m0, v - eps * w, op), Wt)
        fd = float((lp - lm) / (2 * eps))
        an = float((gv * w).sum())
        errs.append(abs(fd - an) / abs(an))
    assert max(errs) < 1e-6, errs


def test_gradient_matches_oracle(workload):
    c, op, W = workload
    v = cuda(c["v_true"]).requires_grad_(True)
    m0 = cuda(c["mT"]).requires_grad_(True)
    m1 = AG.transport(m0, v, op)
    Gt = cuda(W) + m1.detach()  # dL/dm1 of loss()
    gv, gm0 = torch.autograd.grad(loss(m1, cuda(W)), (v, m0))
    P = O.Problem(c["n"], c["n_t"], c["n_c"], 1.0, 1, False, dto=True)
    G = host(Gt)
    m1o = P.state(c["v_true"], c["mT"])[-1]
    g, _ = P.gradient(c["v_true"], c["mT"], m1o - G)  # lambda_1 = -G
    f = g - P.reg_apply(c["v_true"])
    assert rel(host(gv), f) < 1e-10
    assert rel(host(gm0), -P.adjoint(c["v_true"], -G)[0]) < 1e-10


def test_template_gradient_is_exact(workload):
    c, op, W = workload
    v = cuda(c["v_true"])
    m0 = cuda(c["mT"]).requires_grad_(True)
    Wt = cuda(W)
    (gm,) = torch.autograd.grad((AG.transport(m0, v, op) * Wt).sum(), m0)
    dm = cuda(np.random.default_rng(5).standard_normal(c["n"]))
    with torch.no_grad():
        lin = float((AG.transport(dm, v, op) * Wt).sum())  # the map is linear in m0
    assert abs(lin - float((gm * dm).sum())) < 1e-11 * abs(lin)


@pytest.fixture(scope="module")
def checkpointed():
    """The same workload with a memory budget (100 MB) below the stored state of
    all 33 time nodes (about 415 MB at 64^3): the operator keeps every K-th
    state and recomputes the others in the backward pass."""
    c = synth.stokes_3d(64)
    op = AG.make_transport(c["n"], c["n_t"], c["n_c"], memory_budget_bytes=100 << 20)
    W = np.random.default_rng(9).standard_normal(c["n"])
    return c, op, W


def test_checkpointed_backward_matches_differences_and_oracle(checkpointed):
    c, op, W = checkpointed
    assert 0 < op.ckpt_every < c["n_t"] and c["n_t"] % op.ckpt_every == 0
    v = cuda(c["v_true"]).requires_grad_(True)
    m0 = cuda(c["mT"]).requires_grad_(True)
    Wt = cuda(W)
    m1 = AG.transport(m0, v, op)
    gv, gm0 = torch.autograd.grad(loss(m1, Wt), (v, m0))
    eps = 1e-6
    errs = []
    for k in range(20):
        w = cuda(np.random.default_rng(200 + k).standard_normal(c["v_true"].shape))
        with torch.no_grad():
            lp = loss(AG.transport(m0, v + eps * w, op), Wt)
            lm = loss(AG.transport(m0, v - eps * w, op), Wt)
        fd = float((lp - lm) / (2 * eps))
        an = float((gv * w).sum())
        errs.append(abs(fd - an) / abs(an))
    assert max(errs) < 1e-6, errs
    P = O.Problem(c["n"], c["n_t"], c["n_c"], 1.0, 1, False, dto=True)
    G = W + host(m1.detach())
    m1o = P.state(c["v_true"], c["mT"])[-1]
    g, _ = P.gradient(c["v_true"], c["mT"], m1o - G)
    assert rel(host(gv), g - P.reg_apply(c["v_true"])) < 1e-10
    assert rel(host(gm0), -P.adjoint(c["v_true"], -G)[0]) < 1e-10
