"""Lockstep batched solves (reg_solve_lockstep): problems of one shape stacked
into one context and iterated together must take, problem by problem, the
iterates of their own single-problem solve, and match the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1408_6299_gb300 import lib, synth
from gpu_util import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    pairs = synth.batch_2d(count=7, seed=77, sizes=(32, 64), ratio=(4, 3), n_t=8)
    for p in pairs:  # references not reachable exactly with the problems' n_t = 8
        p["mR"] = O.Problem(p["n"], 16).state(p["v_true"], p["mT"])[-1]
    return pairs


def problems_of(pairs):
    return [dict(n=p["n"], n_t=p["n_t"], n_c=1, beta=p["beta"], reg=1, stokes=False, mT=p["mT"], mR=p["mR"],
                 v=np.zeros((1, 2) + tuple(p["n"]))) for p in pairs]


def single(p, precision, **opts):
    R = lib.Registration(p["n"], p["n_t"], 1, p["beta"], 1, False, precision)
    R.set_images(p["mT"], p["mR"])
    v = np.zeros((1, 2) + tuple(p["n"]))
    rep = R.solve(v, **opts)
    return v, rep


@pytest.mark.parametrize("opts", [dict(grad_rtol=1e-3), dict(method=lib.REG_METHOD_PICARD, grad_rtol=1e-2, max_outer=200),
                                  dict(stop_rule=lib.REG_STOP_C1C5, tau_J=1e-4)], ids=["gn", "picard", "c1c5"])
def test_lockstep_equals_single_solves_fp64(batch, opts):
    probs = problems_of(batch)
    reps = lib.solve_lockstep(probs, lib.REG_FP64, **opts)
    for p, q, r in zip(batch, probs, reps):
        v1, r1 = single(p, lib.REG_FP64, **opts)
        for k in ("outer", "pcg_iters", "ls_trials", "status", "stop_flags"):
            assert r[k] == r1[k], (k, r[k], r1[k], p["n"], p["beta"])
        assert rel(q["v"], v1) < 1e-9
        assert abs(r["J"] - r1["J"]) <= 1e-11 * r1["J"]


def test_lockstep_matches_oracle(batch):
    probs = problems_of(batch)
    reps = lib.solve_lockstep(probs, lib.REG_FP64, grad_rtol=1e-3)
    for p, q, r in list(zip(batch, probs, reps))[:3]:
        P = O.Problem(p["n"], p["n_t"], 1, p["beta"], 1, False)
        vo, ro = P.solve(p["mT"], p["mR"], grad_rtol=1e-3)
        assert (r["outer"], r["pcg_iters"]) == (ro["outer"], ro["pcg_iters"])
        assert rel(q["v"], vo) < 1e-8


def test_lockstep_mixed_precision_and_stack_limit(batch):
    probs = problems_of(batch)
    reps = lib.solve_lockstep(probs, lib.REG_MIXED, grad_rtol=1e-2)
    probs2 = problems_of(batch)
    reps2 = lib.solve_lockstep(probs2, lib.REG_MIXED, max_stack=2, grad_rtol=1e-2)
    for p, q, r, q2, r2 in zip(batch, probs, reps, probs2, reps2):
        v1, r1 = single(p, lib.REG_MIXED, grad_rtol=1e-2)
        assert r["status"] == 0 and r["g_inf"] <= 1e-2 * r["g0_inf"]
        assert r["outer"] == r1["outer"] and r2["outer"] == r1["outer"]
        # the stacked FP32 sweeps may pick other column-pass variants than a single
        # problem: agreement to the mixed path's tolerance
        assert rel(q["v"], v1) < 1e-5 and rel(q2["v"], v1) < 1e-5


def test_lockstep_rejects_invalid_problems(batch):
    probs = problems_of(batch[:2])
    probs[1]["beta"] = -1.0
    with pytest.raises(lib.RegError) as e:
        lib.solve_lockstep(probs, lib.REG_FP64)
    assert e.value.status == lib.REG_EINVAL


def test_lockstep_restacks_running_problems():
    # 12 pairs of one shape: once half of them have stopped the stack is
    # rebuilt from the running ones; every problem still takes its own iterates
    pairs = synth.batch_2d(count=12, seed=78, sizes=(32,), ratio=(1,), n_t=8)
    for i, p in enumerate(pairs):
        p["mR"] = O.Problem(p["n"], 16).state((0.5 + 0.1 * i) * p["v_true"], p["mT"])[-1]
    probs = problems_of(pairs)
    reps = lib.solve_lockstep(probs, lib.REG_FP64, grad_rtol=1e-4)
    outers = []
    for p, q, r in zip(pairs, probs, reps):
        v1, r1 = single(p, lib.REG_FP64, grad_rtol=1e-4)
        for k in ("outer", "pcg_iters", "ls_trials", "status"):
            assert r[k] == r1[k], (k, r[k], r1[k])
        assert rel(q["v"], v1) < 1e-9
        assert abs(r["J"] - r1["J"]) <= 1e-11 * r1["J"] and abs(r["dist_rel"] - r1["dist_rel"]) <= 1e-9
        outers.append(r["outer"])
    assert len(set(outers)) > 1  # the problems stop at different iterations


@pytest.mark.parametrize("precision", [lib.REG_FP64, lib.REG_MIXED])
def test_device_driven_loops_take_the_host_loops_iterates(batch, precision, monkeypatch):
    # the PCG and line-search loops as conditional CUDA graphs take every
    # decision the host-driven loops take, problem by problem
    probs = problems_of(batch)
    monkeypatch.setenv("REG_LOCKSTEP_GRAPHS", "1")
    dev = lib.solve_lockstep(probs, precision, grad_rtol=1e-3)
    monkeypatch.setenv("REG_LOCKSTEP_GRAPHS", "0")
    probs_h = problems_of(batch)
    host = lib.solve_lockstep(probs_h, precision, grad_rtol=1e-3)
    for a, b, qa, qb in zip(dev, host, probs, probs_h):
        assert a["device_loops"] == 1 and b["device_loops"] == 0
        for k in ("status", "outer", "pcg_iters", "matvecs", "n_pde", "ls_trials"):
            assert a[k] == b[k], (k, a[k], b[k])
        assert rel(qa["v"], qb["v"]) < 1e-12
