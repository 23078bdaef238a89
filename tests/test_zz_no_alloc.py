"""reg_precond_noalloc: the preconditioner for callers that cannot allocate.

Some callers cannot call cudaMalloc when they need the operator (another
runtime owns all device memory through its own pool, a memory budget fixed at
start-up, loops that must not allocate after initialisation). The entry
point works in a fixed device array instead. These checks compare it with
reg_precond through the C ABI on two calls in a row (the second call finds
the first call's leftovers in the shared array), check that a repeated call
takes no device memory, and that sizes beyond the fixed capacity are
rejected with a clear message. Further cases reach the end of the array (the
largest admissible spectra, 512-point rows, n_c = 16) and run a large, a
small and again the large problem in a row, where stale spectra of the large
call lie beyond the small call's extent. The file is named to run last.
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


def test_capacity_boundary_at_64_cubed():
    # n_c*d*N/2 <= 2,095,040: at 64^3 (d = 3, N/2 = 131072) n_c = 5 fits and n_c = 6 does not
    import torch
    n = (64, 64, 64)
    r = np.random.default_rng(21).standard_normal((5, 3) + n)
    z = empty(r.shape)
    lib.precond_noalloc(n, 5, 1e-2, lib.REG_H1, cuda(r), z)
    torch.cuda.synchronize()
    assert rel(host(z), reference(n, 5, 1e-2, lib.REG_H1, r)) < TOL
    big = empty((6, 3) + n)
    with pytest.raises(lib.RegError) as e:
        lib.precond_noalloc(n, 6, 1e-2, lib.REG_H1, big, big)
    assert e.value.status == lib.REG_EINVAL and "capacity" in str(e.value)


def test_large_small_large_and_the_largest_tables():
    # 512^2 with n_c = 7 (H2) fills 1,835,008 of the 2,095,040 spectral slots;
    # 8 x 512 with n_c = 16 uses the 512-point tables and the largest Gram inverse
    import torch
    seq = [((512, 512), 7, 1e-3, lib.REG_H2, 31), ((16, 8, 32), 3, 3e-3, lib.REG_H2, 32),
           ((512, 512), 7, 1e-3, lib.REG_H2, 31), ((8, 512), 16, 1e-2, lib.REG_H1, 33)]
    outs = []
    for n, nc, beta, reg, seed in seq:
        r = np.random.default_rng(seed).standard_normal((nc, len(n)) + n)
        z = empty(r.shape)
        lib.precond_noalloc(n, nc, beta, reg, cuda(r), z)
        torch.cuda.synchronize()
        outs.append(host(z))
        assert rel(outs[-1], reference(n, nc, beta, reg, r)) < TOL, (n, nc)
    assert np.array_equal(outs[0], outs[2])


def test_tensor_of_another_device_is_refused_without_a_launch():
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    n = (16, 16)
    torch.cuda.set_device(0)
    r1 = torch.zeros((1, 2) + n, dtype=torch.float64, device="cuda:1")
    z0 = empty((1, 2) + n)
    L = lib.load()
    arr = (lib.ctypes.c_int64 * 2)(*n)
    st = L.reg_precond_noalloc(2, arr, 1, 1e-2, lib.REG_H1, r1.data_ptr(), z0.data_ptr(), None)
    assert st == lib.REG_EINVAL
