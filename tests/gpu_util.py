"""Helpers shared by the GPU tests: marshal numpy inputs to CUDA tensors and
back, and build matching library/oracle problems from a workload dict."""
import numpy as np

from oracle import oracle as O
from paper_1408_6299_gb300 import lib


def cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def empty(shape):
    import torch
    return torch.empty(shape, dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def relmax(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def pair(c, precision=lib.REG_FP64, ckpt=0, quad=0, n_t=None, beta=None):
    """(library context, oracle problem) for workload dict c."""
    nt = n_t or c["n_t"]
    b = beta if beta is not None else c["beta"]
    R = lib.Registration(c["n"], nt, c["n_c"], b, c["reg"], c["stokes"], precision, ckpt, quadrature=quad)
    P = O.Problem(c["n"], nt, c["n_c"], b, c["reg"], c["stokes"], dto=bool(quad))
    return R, P
