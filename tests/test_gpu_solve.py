"""Inexact Gauss-Newton-Krylov solves (Alg. 1) on the GPU.

The 3D Stokes scheme with n_c = 3 Chebyshev coefficients reaches the relative
gradient reduction 1e-2 with a divergence-free iterate (to rounding); det F_1
of App. D Eq. def-grad stays within 1e-4 of one there, the remaining deviation
being the spatial aliasing of the pseudospectral F-equation (it does not
shrink with the time step). A smaller Stokes problem matches the oracle's
solve iterate by iterate."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1408_6299_gb300 import lib, synth
from gpu_util import cuda, host, pair, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [lib.REG_MIXED, lib.REG_FP64])
def test_stokes_3d_solve_reaches_tolerance_with_unit_jacobian(precision):
    c = synth.stokes_3d(64)
    R = lib.Registration(c["n"], c["n_t"], c["n_c"], c["beta"], c["reg"], c["stokes"], precision)
    P = O.Problem(c["n"], c["n_t"], c["n_c"], c["beta"], c["reg"], c["stokes"])
    mR = P.state(c["v_true"], c["mT"])[-1]
    R.set_images(cuda(c["mT"]), cuda(mR))
    v = cuda(np.zeros(R.coef_shape()))
    rep = R.solve(v, grad_rtol=1e-2, detF_substeps=16)
    assert rep["status"] == 0
    assert rep["g_inf"] <= 1e-2 * rep["g0_inf"]
    assert rep["J"] < rep["J0"]
    dmin, dmax = rep["detF"][0], rep["detF"][1]
    assert abs(dmin - 1) < 1e-4 and abs(dmax - 1) < 1e-4, rep["detF"]
    # the iterate stays divergence-free (pressure elimination, Sec. 3.3.4)
    div = np.zeros(c["n"])
    Pg = O.Problem(c["n"], 2)
    for l in range(c["n_c"]):
        div = np.maximum(div, np.abs(Pg.div(host(v)[l])))
    assert div.max() < 1e-10 * np.abs(host(v)).max()


def test_small_stokes_solve_matches_oracle():
    c = synth.stokes_3d(16, n_t=8, n_c=2)
    R, P = pair(c)
    mR = P.state(c["v_true"], c["mT"])[-1]
    R.set_images(cuda(c["mT"]), cuda(mR))
    v = cuda(np.zeros(R.coef_shape()))
    rep = R.solve(v, grad_rtol=1e-2)
    vo, repo = P.solve(c["mT"], mR, grad_rtol=1e-2)
    assert rep["status"] == 0 and repo["status"] == 0
    assert (rep["outer"], rep["pcg_iters"], rep["ls_trials"]) == (repo["outer"], repo["pcg_iters"], repo["ls_trials"])
    assert rel(host(v), vo) < 1e-8
