"""Failure detection without a GPU fault: the bounded waits of the TMA column
pass give up, count the timeout and let the host fail the call. A probe
kernel waits on an mbarrier that nothing completes; the context stays usable
afterwards."""
import numpy as np
import pytest

from paper_1408_6299_gb300 import lib, synth
from gpu_util import cuda, empty

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_is_counted():
    assert lib.selftest_copy_timeout() == 1
    assert lib.selftest_copy_timeout() == 1  # cleared on read, counted again


def test_library_still_works_after_a_timeout():
    lib.selftest_copy_timeout()
    c = synth.sinusoid_2d(32)
    R = lib.Registration(c["n"], 4, 1, c["beta"], c["reg"], False, lib.REG_FP64)
    m1 = empty(c["n"])
    R.transport(cuda(c["v_true"]), cuda(c["mT"]), m1)
    assert np.isfinite(m1.cpu().numpy()).all()
