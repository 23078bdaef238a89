"""Parity at the benchmark's full size: the 256^3 random-field Gauss-Newton
matvec in the launch configuration bench.py times (state checkpoints every 8
steps, n_t doubled from 64 until CFL <= 0.2, i.e. 128), mixed precision and
FP64, against one full oracle matvec on the host cores (about 70 GB of host
memory and a few minutes on 16 cores)."""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1408_6299_gb300 import lib, synth
from gpu_util import cuda, empty, host, rel, relmax

pytestmark = pytest.mark.gpu


def host_mem_available():
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable:"):
                return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return 0


@pytest.mark.skipif(host_mem_available() < 100 * 2 ** 30, reason="needs about 100 GB of host memory for the oracle")
def test_256_matvec_mixed_and_fp64_against_oracle():
    c = synth.random_3d(256)
    v, mT, vt = cuda(c["v_true"]), cuda(c["mT"]), cuda(c["vt"])
    n_t = 64
    while True:
        probe = lib.Registration(c["n"], n_t, 1, c["beta"], c["reg"], False)
        cfl = probe.cfl(v)
        probe.close()
        if cfl <= 0.2:
            break
        n_t *= 2
    assert n_t == 128
    out = {}
    for prec in (lib.REG_MIXED, lib.REG_FP64):
        R = lib.Registration(c["n"], n_t, 1, c["beta"], c["reg"], False, prec, 8)
        mR = empty(c["n"])
        R.transport(v, mT, mR)
        R.set_images(mT, mR)
        R.linearize(v)
        H = empty((1, 3) + c["n"])
        R.hessvec(vt, H)
        out[prec] = host(H)
        R.close()
        torch.cuda.empty_cache()
    P = O.Problem(c["n"], n_t, 1, c["beta"], c["reg"], False)
    ref = P.hessvec(c["v_true"], c["mT"], c["vt"])
    assert rel(out[lib.REG_FP64], ref) < 1e-10
    assert rel(out[lib.REG_MIXED], ref) < 1e-5
    assert relmax(out[lib.REG_MIXED], ref) < 1e-4
