"""reg_precond_noalloc: the preconditioner for callers that cannot allocate.

Some callers cannot call cudaMalloc when they need the operator (another
runtime owns all device memory through its own pool, a memory budget fixed at
start-up, loops that must not allocate after initialisation). The entry
point works in a fixed device array instead. These checks compare it with
reg_precond through the C ABI on two calls in a row (the second call finds
the first call's leftovers in the shared array), check that a repeated call
takes no device memory, and that sizes beyond the fixed capacity are
rejected with a clear message. The file is named to run last.
"""
import numpy as np
import pytest

from paper_1408_6299_gb300 import lib
from gpu_util import cuda, empty, host, rel

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the tolerance of the other Fourier-diagonal operator checks

CASES = [((32, 32), 1, 1e-2, lib.REG_H1, 11), ((16, 8, 32), 3, 3e-3, lib.REG_H2, 12)]


def reference(n, nc, beta, reg, r):
    R = lib.Registration(n, 4, nc, beta, reg)
    out = empty(r.shape)
    R.precond(cuda(r), out)
    R.close()
    return host(out)


def test_noalloc_matches_reg_precond_on_consecutive_calls():
    import torch
    results = []
    for n, nc, beta, reg, seed in CASES:
        r = np.random.default_rng(seed).standard_normal((nc, len(n)) + n)
        z = empty(r.shape)
        lib.precond_noalloc(n, nc, beta, reg, cuda(r), z)
        torch.cuda.synchronize()
        results.append((host(z), reference(n, nc, beta, reg, r)))
    for z, ref in results:
        assert rel(z, ref) < TOL


def test_repeat_call_takes_no_device_memory_and_is_stable():
    import torch
    n, nc, beta, reg, seed = CASES[1]
    r = cuda(np.random.default_rng(seed).standard_normal((nc, len(n)) + n))
    z1, z2 = empty(r.shape), empty(r.shape)
    lib.precond_noalloc(n, nc, beta, reg, r, z1)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    lib.precond_noalloc(n, nc, beta, reg, r, z2)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    assert torch.equal(z1, z2)


def test_sizes_beyond_the_fixed_scratch_are_rejected():
    n = (128, 128, 128)
    r = empty((1, 3) + n)
    with pytest.raises(lib.RegError) as e:
        lib.precond_noalloc(n, 1, 1e-2, lib.REG_H1, r, r)
    assert e.value.status == lib.REG_EINVAL
    assert "capacity" in str(e.value)
