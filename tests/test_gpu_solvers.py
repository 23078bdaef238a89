"""The outer-loop variants of Sec. 3.2-3.3.5 on the GPU against the oracle,
iterate by iterate: the Picard iteration (Eq. picard) with and without the
step memory alpha~, the C1-C5 stopping set (Eq. stopping-criteria), CFL step
halving, and their combinations with GN-PCG and N-PCG."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1408_6299_gb300 import lib, synth
from gpu_util import cuda, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def prob():
    c = synth.sinusoid_2d(32)
    mR = O.Problem(c["n"], 16).state(c["v_true"], c["mT"])[-1]  # not reachable exactly with n_t = 8
    return c, mR


def run_both(c, mR, hessian=lib.REG_HESS_GN, **kw):
    R = lib.Registration(c["n"], 8, 1, c["beta"], c["reg"], False, lib.REG_FP64, hessian=hessian)
    P = O.Problem(c["n"], 8, 1, c["beta"], c["reg"], False)
    R.set_images(cuda(c["mT"]), cuda(mR))
    v = cuda(np.zeros(R.coef_shape()))
    gkw = dict(kw)
    okw = dict(kw)
    if "picard" in kw:
        gkw["method"] = lib.REG_METHOD_PICARD if gkw.pop("picard") else lib.REG_METHOD_KRYLOV
    if "step_memory" in gkw:
        gkw["step_memory"] = int(gkw["step_memory"])
    rep = R.solve(v, **gkw)
    vo, repo = P.solve(c["mT"], mR, newton=hessian == lib.REG_HESS_NEWTON, **okw)
    return host(v), rep, vo, repo


CASES = [
    dict(picard=True, grad_rtol=1e-3, max_outer=100),
    dict(picard=True, step_memory=False, grad_rtol=1e-3, max_outer=100),
    dict(picard=True, grad_rtol=1e-3, max_outer=100, cfl_max=0.25),
    dict(stop_rule=1, tau_J=1e-3, max_outer=100),
    dict(stop_rule=1, tau_J=1e-4, max_outer=100, picard=True),
    dict(stop_rule=1, tau_J=1e-3, max_outer=2),  # C5 ends it
]


@pytest.mark.parametrize("kw", CASES, ids=[str(i) for i in range(len(CASES))])
def test_outer_variants_match_oracle(prob, kw):
    c, mR = prob
    v, rep, vo, repo = run_both(c, mR, **kw)
    assert rep["status"] == repo["status"], (rep["status"], repo["status"])
    for k in ("outer", "pcg_iters", "ls_trials", "stop_flags", "cfl_halvings"):
        assert rep[k] == repo[k], (k, rep[k], repo[k])
    assert rep["alpha_mem"] == repo["alpha_mem"]
    assert rel(v, vo) < 1e-8
    assert abs(rep["J"] - repo["J"]) <= 1e-10 * repo["J"]
    for k in ("J_prev", "dv_inf", "v_inf"):
        assert abs(rep[k] - repo[k]) <= 1e-8 * max(abs(repo[k]), 1e-30), k
    if kw.get("cfl_max"):
        assert rep["cfl_halvings"] > 0 and rep["cfl"] <= kw["cfl_max"]


def test_newton_with_stopping_set(prob):
    c, mR = prob
    v, rep, vo, repo = run_both(c, mR, hessian=lib.REG_HESS_NEWTON, stop_rule=1, tau_J=1e-4, max_outer=50)
    assert rep["status"] == 0 and (rep["stop_flags"] & 7) == 7
    assert (rep["outer"], rep["pcg_iters"], rep["stop_flags"]) == (repo["outer"], repo["pcg_iters"], repo["stop_flags"])
    assert rel(v, vo) < 1e-8


def test_c4_at_a_stationary_start(prob):
    c, _ = prob
    R = lib.Registration(c["n"], 8, 1, c["beta"], c["reg"], False, lib.REG_FP64)
    R.set_images(cuda(c["mT"]), cuda(c["mT"]))
    v = cuda(np.zeros(R.coef_shape()))
    rep = R.solve(v, stop_rule=lib.REG_STOP_C1C5)
    assert rep["status"] == 0 and rep["outer"] == 0 and rep["stop_flags"] & 8 and rep["g_inf"] == 0.0


def test_bad_options_are_rejected(prob):
    c, mR = prob
    R = lib.Registration(c["n"], 8, 1, c["beta"], c["reg"], False, lib.REG_FP64)
    R.set_images(cuda(c["mT"]), cuda(mR))
    v = cuda(np.zeros(R.coef_shape()))
    for bad in (dict(method=5), dict(stop_rule=3), dict(stop_rule=1, tau_J=0.0)):
        with pytest.raises(lib.RegError) as e:
            R.solve(v, **bad)
        assert e.value.status == lib.REG_EINVAL
    with pytest.raises(TypeError):
        R.solve(v, not_an_option=1)
