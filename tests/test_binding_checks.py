"""The Python binding refuses arrays of the wrong size before any library call.

The C ABI takes plain pointers, so the library cannot know how many values an
array holds; an undersized array would be read or written past its end by the
kernels. The binding checks every array against the count the call implies
(N for images, n_c*d*N for coefficient vectors) and raises ValueError first.
These checks run on CPU: the library object is replaced by one whose every
function fails the test if it is reached.
"""
import numpy as np
import pytest

from paper_1408_6299_gb300 import lib


class _Unreachable:
    def __getattr__(self, name):
        def fail(*a, **k):
            raise AssertionError(f"library function {name} was called")
        return fail


def fake_context(n=(8, 16), n_c=2):
    R = object.__new__(lib.Registration)
    R.L = _Unreachable()
    R.n, R.d, R.n_c, R.n_t, R.ckpt_every, R.ctx = tuple(n), len(n), n_c, 4, 0, None
    return R


def test_addr_counts_elements():
    a = np.zeros(12)
    assert lib._addr(a, 12)[0] == a.ctypes.data
    with pytest.raises(ValueError):
        lib._addr(a, 13)
    with pytest.raises(TypeError):
        lib._addr(np.zeros(12, dtype=np.float32), 12)


def test_undersized_arrays_are_refused_before_the_library():
    R = fake_context()
    N, ncdN = 8 * 16, 2 * 2 * 8 * 16
    short = np.zeros(ncdN - 1)
    with pytest.raises(ValueError):
        R.hessvec(short, np.zeros(ncdN))
    with pytest.raises(ValueError):
        R.hessvec(np.zeros(ncdN), short)
    with pytest.raises(ValueError):
        R.gradient(np.zeros(ncdN), np.zeros(N))
    with pytest.raises(ValueError):
        R.set_images(np.zeros(N), np.zeros(N - 1))
    with pytest.raises(ValueError):
        R.transport(np.zeros(ncdN), np.zeros(N), np.zeros(2 * N))
    with pytest.raises(ValueError):
        R.transport_adjoint(np.zeros(ncdN), np.zeros(N), np.zeros(N), np.zeros(N), None)
    with pytest.raises(ValueError):
        R.displacement(np.zeros(ncdN), np.zeros(N))
    with pytest.raises(ValueError):
        R.precond(np.zeros(N), np.zeros(ncdN))
    with pytest.raises(ValueError):
        R.solve(np.zeros(ncdN + 1))


def test_noalloc_and_batched_arrays_are_checked():
    with pytest.raises(ValueError):
        lib.precond_noalloc((8, 8), 2, 1e-2, lib.REG_H1, np.zeros(2 * 2 * 64 - 2), np.zeros(2 * 2 * 64))
    p = dict(n=(8, 8), n_t=4, n_c=1, beta=1e-2, mT=np.zeros(64), mR=np.zeros(64), v=np.zeros(64))
    with pytest.raises(ValueError):
        lib._problem_array([p])
