"""Batched solves (reg_solve_batched) and CUDA-graph replay of the matvec.

Pairs of the seeded batch workload (2D blobs of uneven size) solved
concurrently must give the same iterates, iteration counts and line-search
trials as one-at-a-time solves (same arithmetic, only scheduled differently);
a context with its own stream replays its matvec as a CUDA graph and must
reproduce the direct launches bit for bit."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1408_6299_gb300 import lib, synth
from gpu_util import cuda, empty, host, rel

pytestmark = pytest.mark.gpu


def cfl_nt(n, speed=0.3, nt=16, bound=0.2):
    while speed * n / (2 * np.pi * nt) > bound:
        nt *= 2
    return nt


def make_pairs(count, sizes, seed):
    pairs = synth.batch_2d(count=count, seed=seed, sizes=sizes)
    for p in pairs:
        p["n_t"] = cfl_nt(p["n"][0])
        P = O.Problem(p["n"], p["n_t"], 1, p["beta"], 1, False)
        p["mR"] = P.state(p["v_true"], p["mT"])[-1]
    return pairs


def as_problems(pairs):
    return [dict(n=p["n"], n_t=p["n_t"], n_c=1, beta=p["beta"], reg=lib.REG_H1, stokes=False, mT=cuda(p["mT"]),
                 mR=cuda(p["mR"]), v=cuda(np.zeros((1, 2) + p["n"]))) for p in pairs]


def test_batched_matches_single_solves():
    pairs = make_pairs(6, (32, 64), 7)
    probs = as_problems(pairs)
    reps = lib.solve_batched(probs, precision=lib.REG_FP64, workers=3, grad_rtol=1e-2)
    for p, pb, rb in zip(pairs, probs, reps):
        R = lib.Registration(p["n"], p["n_t"], 1, p["beta"], lib.REG_H1, False, lib.REG_FP64)
        R.set_images(cuda(p["mT"]), cuda(p["mR"]))
        v = cuda(np.zeros((1, 2) + p["n"]))
        r1 = R.solve(v, grad_rtol=1e-2)
        assert (rb["outer"], rb["pcg_iters"], rb["ls_trials"]) == (r1["outer"], r1["pcg_iters"], r1["ls_trials"])
        assert rel(host(pb["v"]), host(v)) < 1e-12
        assert rb["status"] == 0 and rb["g_inf"] <= 1e-2 * rb["g0_inf"]


def test_mixed_batch_reaches_tolerance():
    pairs = make_pairs(8, (64, 128), 8)
    probs = as_problems(pairs)
    reps = lib.solve_batched(probs, precision=lib.REG_MIXED, workers=4, grad_rtol=1e-2)
    for r in reps:
        assert r["status"] == 0 and r["g_inf"] <= 1e-2 * r["g0_inf"]


@pytest.mark.parametrize("precision", [lib.REG_FP64, lib.REG_MIXED])
def test_graph_replay_matches_direct_launches(precision):
    c = synth.stokes_3d(16, n_t=6, n_c=2)
    P = O.Problem(c["n"], c["n_t"], c["n_c"], c["beta"], c["reg"], c["stokes"])
    mR = P.state(c["v_true"], c["mT"])[-1]
    stream = torch.cuda.Stream()
    out = []
    for s in (None, stream.cuda_stream):
        R = lib.Registration(c["n"], c["n_t"], c["n_c"], c["beta"], c["reg"], c["stokes"], precision, 2, stream=s)
        R.set_images(cuda(c["mT"]), cuda(mR))
        R.linearize(cuda(c["v_true"]))
        H = empty(R.coef_shape())
        for k in range(3):  # first call captures the graph, later calls replay it
            d = cuda(np.random.default_rng(k).standard_normal(R.coef_shape()))
            torch.cuda.synchronize()
            R.hessvec(d, H)
        out.append(H.clone())
        R.close()
    assert torch.equal(out[0], out[1])
