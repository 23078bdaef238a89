#!/usr/bin/env python
"""Gauss-Newton Hessian matvecs/s on the 256^3 random-field registration workload.

Workload (one step = one Hessian matvec, Alg. 2 of Mang & Biros): 256^3 grid,
H2 regularisation, beta = 1e-3, stationary velocity (n_c = 1), state
checkpoints every 8 steps recomputed in both sweeps, single precision
transport sweeps with double precision outer vectors (REG_MIXED). The number
of Heun steps starts at the workload's n_t = 64 and is doubled until the CFL
number is at most eps_CFL = 0.2 (Sec. 3.3.1); for this velocity that gives
n_t = 128. At n_t = 64 (CFL 0.25) Heun amplifies the highest Fourier modes by
about 1.6x per step, so single precision rounding noise grows without bound;
that configuration is still timed and reported under "as_configured".
Inputs are seeded synthetic fields (paper_1408_6299_gb300.synth.random_3d):
a unit-variance template band-limited to |k| <= 48, a smooth velocity of max
speed 0.5 (|k| <= 8) and a unit-speed direction. Every field is 64-128 MB,
well above the 129 MB L2 in aggregate per step (the state checkpoints alone
are 580 MB), so no explicit L2 flush is done.

One process per GPU (torchrun); with several GPUs every rank runs its own
replica of the workload (the solver does not shard) and value counts the
matvecs of all ranks over the slowest rank's time.

--impl reference times the CPU oracle (oracle/) on the same workload. A full
oracle matvec at n_t = 128 takes minutes, so each step is a bounded sample: one
oracle matvec on the 256^3 grid with n_t = 2, timed as it runs (ms_per_step is
that sample's time). value is the rate of full matvecs extrapolated linearly
in n_t from that sample and one n_t = 1 run (the line says so). With
--cpu-full the reference arm instead times one whole n_t = 128 oracle matvec
(steps = 1), the measurement that checks the extrapolation.

Other workloads: --workload batch (the 256-pair 2D batch, sharded across
ranks), --workload profile (set up the matvec, run one warm-up and one
measured matvec and print the launch counts SETUP/WARM/MEAS that ncu skips and
captures), --workload stability --sweep-nt 64,88,128 (per n_t: CFL number and
mixed-vs-FP64 difference of the matvec).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Hessian matvecs/s at 256^3 (FP32-Krylov vs FP64) and solve time to rel-grad 1e-2"
UNIT = "matvecs/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=256)
    p.add_argument("--n_t", type=int, default=64, help="starting n_t (doubled until CFL <= cfl)")
    p.add_argument("--cfl", type=float, default=0.2)
    p.add_argument("--as-configured-steps", type=int, default=2)
    p.add_argument("--store-all-steps", type=int, default=2)
    p.add_argument("--newton-steps", type=int, default=2)
    p.add_argument("--ckpt", type=int, default=8)
    p.add_argument("--fp64-steps", type=int, default=1)
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-solves", action="store_true")
    p.add_argument("--workload", default="matvec", choices=["matvec", "batch", "profile", "stability"])
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"], help="--workload profile only")
    p.add_argument("--sweep-nt", default="64,88,96,128", help="--workload stability: n_t values")
    p.add_argument("--cpu-full", action="store_true", help="--impl reference: one whole oracle matvec")
    p.add_argument("--pairs", type=int, default=256)
    p.add_argument("--batch-sample", type=int, default=256)
    p.add_argument("--batch-mode", default="lockstep", choices=["lockstep", "executor"])
    p.add_argument("--max-stack", type=int, default=0, help="problems per lockstep stack (0: one per shape)")
    p.add_argument("--workers", type=int, default=8)
    return p.parse_args()


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_traffic(kind):
    """Per-launch DRAM bytes of `kind` from the committed ncu summary, if the
    kernel sources are unchanged since it was taken (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    ent = d.get(kind)
    if not ent:
        return None
    src = os.path.join(ROOT, ent["source"])
    if not os.path.exists(src):
        return None
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if h != ent.get("source_sha256_16"):
        return None
    return float(ent["dram_bytes_per_launch"])


# ----------------------------------------------------------------------------
# oracle timing (CPU baseline and the reference arm)
# ----------------------------------------------------------------------------
def oracle_matvec_seconds(c, n_t):
    from oracle import oracle as O
    P = O.Problem(c["n"], n_t, c["n_c"], c["beta"], c["reg"], c["stokes"])
    t = time.perf_counter()
    P.hessvec(c["v_true"], c["mT"], c["vt"])
    return time.perf_counter() - t


def oracle_extrapolated(c, n_t, t1=None, reps=1):
    """seconds of one full n_t-step oracle matvec from runs with 1 and 2 steps"""
    if t1 is None:
        t1 = oracle_matvec_seconds(c, 1)
    t2s = [oracle_matvec_seconds(c, 2) for _ in range(reps)]
    t2 = statistics.median(t2s)
    per_step = max(t2 - t1, 1e-9)
    return t1 + (n_t - 1) * per_step, t1, t2s


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1408_6299_gb300 import synth
    c = synth.random_3d(args.n, n_t=args.n_t)
    n_t = args.n_t
    P = O.Problem(c["n"], n_t, c["n_c"], c["beta"], c["reg"], c["stokes"])
    cfl = P.cfl(c["v_true"])
    while cfl > args.cfl:
        n_t *= 2
        cfl /= 2
    cores = O.num_threads()
    base = {"impl": "reference", "metric": METRIC, "unit": UNIT, "n_gpus": args.gpus, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"random-field {args.n}^3 H2 beta=1e-3 n_c=1 n_t={n_t} GN matvec (CPU oracle)",
                       "grid": [args.n] * 3, "n_t": n_t}}
    if args.cpu_full:
        t = oracle_matvec_seconds(c, n_t)
        value = 1.0 / t
        sample = f"one whole oracle GN matvec on the {args.n}^3 grid with n_t={n_t}, measured"
        line = dict(base, value=value, steps=1, warmup=0, ms_per_step=1000.0 * t)
    else:
        t1 = oracle_matvec_seconds(c, 1)
        for _ in range(max(0, args.warmup - 1)):
            oracle_matvec_seconds(c, 2)
        t2s = [oracle_matvec_seconds(c, 2) for _ in range(args.steps)]
        t2 = statistics.median(t2s)
        T = t1 + (n_t - 1) * max(t2 - t1, 1e-9)
        value = 1.0 / T
        sample = (f"each step: one oracle GN matvec on the {args.n}^3 grid with n_t=2 ({t2:.2f} s median, the "
                  f"step's measured time); value extrapolated to n_t={n_t} as t1 + {n_t - 1}*(t2 - t1) with "
                  f"t1 = {t1:.2f} s (n_t=1)")
        line = dict(base, value=value, steps=args.steps, warmup=args.warmup, ms_per_step=1000.0 * t2,
                    extrapolated_ms_per_matvec=1000.0 * T)
    line["cpu_baseline"] = {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    line["e2e"] = {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# solve time to rel-grad 1e-2 (Alg. 1) on the 128^2 and 64^3 workloads
# ----------------------------------------------------------------------------
def solve_times():
    import numpy as np
    import torch

    from paper_1408_6299_gb300 import lib, synth

    out = {}
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    for c, precs in ((synth.blobs_2d(128), ("mixed", "fp64")), (synth.stokes_3d(64), ("mixed",))):
        mT = dev(c["mT"])
        for pname in precs:
            prec = lib.REG_MIXED if pname == "mixed" else lib.REG_FP64
            R = lib.Registration(c["n"], c["n_t"], c["n_c"], c["beta"], c["reg"], c["stokes"], prec)
            mR = torch.empty(c["n"], dtype=torch.float64, device="cuda")
            R.transport(dev(c["v_true"]), mT, mR)  # reference image by the library's own state solve
            R.set_images(mT, mR)
            v = torch.zeros(R.coef_shape(), dtype=torch.float64, device="cuda")
            R.solve(v.clone(), grad_rtol=1e-2)  # warm-up (allocations, tables)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = R.solve(v, grad_rtol=1e-2)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            ent = {"seconds": sec, "outer": rep["outer"], "pcg_iters": rep["pcg_iters"], "n_pde": rep["n_pde"],
                   "grad_rel": rep["g_inf"] / rep["g0_inf"], "J_rel": rep["J"] / rep["J0"],
                   "status": rep["status"]}
            if c["stokes"]:
                t0 = time.perf_counter()
                st = R.detF_refined(v, 4, 2)
                ent["detF_min_max"] = st[:2]
                ent["detF_seconds"] = time.perf_counter() - t0
                ent["detF_eval"] = "Eq. def-grad on the grid refined 2x per axis, 4 n_t Heun steps (after the solve)"
                ent["detF_min_max_unrefined"] = R.detF(v, 4)[:2]
            out[f"{c['name']}-{pname}"] = ent
            R.close()
    return out


# ----------------------------------------------------------------------------
# batched 2D pairs (uneven sizes 64^2/128^2/256^2 at 4:2:1, H1, n_c = 1)
# ----------------------------------------------------------------------------
def batch_pairs(count):
    import numpy as np

    from paper_1408_6299_gb300 import synth
    pairs = synth.batch_2d(count=count)
    for p in pairs:
        nt = 16  # doubled until the CFL number of the workload's max speed 0.3 is <= 0.2
        while 0.3 * p["n"][0] / (2 * np.pi * nt) > 0.2:
            nt *= 2
        p["n_t"] = nt
    return pairs


MAX_STACK = 0  # problems per lockstep stack (0: one stack per shape)


def solve_pairs(pairs, workers, mode="lockstep"):
    """reference images by the library's own transport, then one batched solve
    (mode "lockstep": reg_solve_lockstep; "executor": reg_solve_batched with
    `workers` threads); returns (seconds of the solve call, reports)"""
    import numpy as np
    import torch

    from paper_1408_6299_gb300 import lib
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    probs, ctxs = [], {}
    for p in pairs:
        key = (p["n"], p["n_t"], p["beta"])
        if key not in ctxs:
            ctxs[key] = lib.Registration(p["n"], p["n_t"], 1, p["beta"], lib.REG_H1, False, lib.REG_FP64)
        mT = dev(p["mT"])
        mR = torch.empty(p["n"], dtype=torch.float64, device="cuda")
        ctxs[key].transport(dev(p["v_true"]), mT, mR)
        probs.append(dict(n=p["n"], n_t=p["n_t"], n_c=1, beta=p["beta"], reg=lib.REG_H1, stokes=False, mT=mT,
                          mR=mR, v=torch.zeros((1, 2) + p["n"], dtype=torch.float64, device="cuda")))
    for R in ctxs.values():
        R.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if mode == "lockstep":
        reps = lib.solve_lockstep(probs, precision=lib.REG_MIXED, max_stack=MAX_STACK, grad_rtol=1e-2)
    else:
        reps = lib.solve_batched(probs, precision=lib.REG_MIXED, workers=workers, grad_rtol=1e-2)
    torch.cuda.synchronize()
    return time.perf_counter() - t0, reps


def batch_sample(count, workers):
    pairs = batch_pairs(count)
    # warm-up: the autotuner's trials for every stack size, tables, graph capture
    solve_pairs(pairs[:min(4, count)], workers, "executor")
    solve_pairs(pairs, workers, "lockstep")
    tl, reps = solve_pairs(pairs, workers, "lockstep")
    os.environ["REG_LOCKSTEP_GRAPHS"] = "0"  # the same lockstep solve with host-driven loops
    th, _ = solve_pairs(pairs, workers, "lockstep")
    del os.environ["REG_LOCKSTEP_GRAPHS"]
    tb, repb = solve_pairs(pairs, workers, "executor")
    ts, _ = solve_pairs(pairs, 1, "executor")
    ok = sum(1 for r in reps if r["status"] == 0 and r["g_inf"] <= 1e-2 * r["g0_inf"])
    by_shape = {}  # each shape's stack solved alone (lockstep, device-driven loops)
    for n in sorted({p["n"] for p in pairs}):
        grp = [p for p in pairs if p["n"] == n]
        tg, rg = solve_pairs(grp, workers, "lockstep")
        by_shape["x".join(map(str, n))] = {
            "pairs": len(grp), "n_t": grp[0]["n_t"], "seconds": tg,
            "mean_outer": sum(r["outer"] for r in rg) / len(grp),
            "mean_matvecs": sum(r["matvecs"] for r in rg) / len(grp),
            "max_matvecs": max(r["matvecs"] for r in rg)}
    return {"pairs": count, "lockstep_solves_per_s": count / tl, "lockstep_by_shape": by_shape,
            "lockstep_device_loops": sum(r["device_loops"] for r in reps),
            "lockstep_host_loops_solves_per_s": count / th, "executor_solves_per_s": count / tb,
            "executor_workers": workers, "sequential_solves_per_s": count / ts, "speedup_vs_sequential": ts / tl,
            "converged": ok, "mean_outer": sum(r["outer"] for r in reps) / count,
            "mean_matvecs": sum(r["matvecs"] for r in reps) / count,
            "same_outer_as_executor": sum(1 for a, b in zip(reps, repb) if a["outer"] == b["outer"])}


def run_batch(args):
    """--workload batch: the full batch, problems sharded across ranks"""
    import torch

    from paper_1408_6299_gb300.shard import partition
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pairs = batch_pairs(args.pairs)
    mine = [pairs[i] for i in partition([p["n"][0] ** 2 * p["n_t"] for p in pairs], world)[rank]]
    solve_pairs(mine[:4], args.workers, args.batch_mode)
    if dist is not None:
        dist.barrier()
    t, reps = solve_pairs(mine, args.workers, args.batch_mode)
    if dist is not None:
        tt = torch.tensor([t], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    if rank == 0:
        print(json.dumps({"metric": "batched 2D registration solves/s (rel-grad 1e-2)", "value": args.pairs / t,
                          "unit": "solves/s", "n_gpus": world, "higher_is_better": True, "scaling": "strong",
                          "data": "synthetic", "dtype": "f32",
                          "config": {"workload": f"{args.pairs} 2D pairs 64^2/128^2/256^2 at 4:2:1, H1, n_c=1",
                                     "mode": args.batch_mode, "workers_per_gpu": args.workers}}), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# helpers for ncu captures and the Heun stability table (profiles/)
# ----------------------------------------------------------------------------
def matvec_context(c, n_t, prec, ckpt):
    import numpy as np
    import torch

    from paper_1408_6299_gb300 import lib
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    v, mT = dev(c["v_true"]), dev(c["mT"])
    R = lib.Registration(c["n"], n_t, 1, c["beta"], c["reg"], c["stokes"], prec, ckpt)
    mR = torch.empty(c["n"], dtype=torch.float64, device="cuda")
    R.transport(v, mT, mR)
    R.set_images(mT, mR)
    R.linearize(v)
    return R, v, dev(c["vt"])


def run_profile(args):
    """one warm-up and one measured matvec; prints the launch counts to skip
    (SETUP + WARM) and to capture (MEAS) with ncu"""
    import torch

    from paper_1408_6299_gb300 import lib, synth
    c = synth.random_3d(args.n)
    prec = lib.REG_MIXED if args.precision == "mixed" else lib.REG_FP64
    R, v, vt = matvec_context(c, args.n_t, prec, args.ckpt)
    H = torch.empty((1, 3) + c["n"], dtype=torch.float64, device="cuda")
    l0 = lib.launch_count()
    R.hessvec(vt, H)
    l1 = lib.launch_count()
    R.hessvec(vt, H)
    l2 = lib.launch_count()
    torch.cuda.synchronize()
    print(f"SETUP={l0} WARM={l1 - l0} MEAS={l2 - l1}", flush=True)


def run_stability(args):
    """per n_t: CFL number and relative 2-norm difference of the mixed and FP64 matvecs"""
    import torch

    from paper_1408_6299_gb300 import lib, synth
    c = synth.random_3d(args.n)
    for n_t in [int(x) for x in args.sweep_nt.split(",")]:
        out = {}
        for prec in (lib.REG_FP64, lib.REG_MIXED):
            R, v, vt = matvec_context(c, n_t, prec, args.ckpt)
            H = torch.empty((1, 3) + c["n"], dtype=torch.float64, device="cuda")
            R.hessvec(vt, H)
            out[prec] = H
            cfl = R.cfl(v)
            R.close()
        err = float(torch.linalg.vector_norm(out[1] - out[0]) / torch.linalg.vector_norm(out[0]))
        print(f"n_t={n_t} cfl={cfl:.4f} mixed_vs_fp64={err:.3e} "
              f"norm_fp64={float(torch.linalg.vector_norm(out[0])):.6e} "
              f"norm_mixed={float(torch.linalg.vector_norm(out[1])):.6e}", flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    from paper_1408_6299_gb300 import lib, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    c = synth.random_3d(args.n, n_t=args.n_t)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    shape = (c["n_c"], 3) + c["n"]
    v, mT, vt = dev(c["v_true"]), dev(c["mT"]), dev(c["vt"])
    nt_cfg = args.n_t
    n_t = nt_cfg
    while True:
        probe = lib.Registration(c["n"], n_t, c["n_c"], c["beta"], c["reg"], c["stokes"], lib.REG_FP64, 0)
        cfl = probe.cfl(v)
        probe.close()
        if cfl <= args.cfl:
            break
        n_t *= 2
    cfl_cfg = cfl * n_t / nt_cfg
    R = lib.Registration(c["n"], n_t, c["n_c"], c["beta"], c["reg"], c["stokes"], lib.REG_MIXED, args.ckpt)
    mR = torch.empty(c["n"], dtype=torch.float64, device="cuda")
    R.transport(v, mT, mR)
    R.set_images(mT, mR)
    g = torch.empty(shape, dtype=torch.float64, device="cuda")
    R.gradient(v, g)  # linearisation point of the matvecs (stored state)
    Hv = torch.empty_like(g)
    for _ in range(args.warmup):
        R.hessvec(vt, Hv)
    # one profiled matvec to find the dominant kernel kind
    R.profile_begin()
    R.hessvec(vt, Hv)
    prof_all = R.profile_end()
    dominant = max(prof_all, key=lambda k: prof_all[k]["ms"])
    kind_idx = lib.KIND_NAMES.index(dominant)

    clocks = ClockSampler(local)
    clocks.start()
    l0 = lib.launch_count()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    R.profile_begin(1 << kind_idx)
    e0.record()
    for _ in range(args.steps):
        R.hessvec(vt, Hv)
    e1.record()
    torch.cuda.synchronize()
    barrier()
    prof = R.profile_end()[dominant]
    launches = lib.launch_count() - l0
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * args.steps / (ms / 1000.0)

    # end to end through the C ABI with host buffers (copies inside the timed region)
    vt_h = torch.empty(shape, dtype=torch.float64, pin_memory=True)
    vt_h.copy_(vt.cpu())
    Hv_h = torch.empty(shape, dtype=torch.float64, pin_memory=True)
    R.hessvec(vt_h, Hv_h)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        R.hessvec(vt_h, Hv_h)
    e2e_s = time.perf_counter() - t0
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    nbytes = int(np.prod(shape)) * 8
    e2e = {"value": world * args.e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes}

    # plain FP64 GPU form (same checkpointing), for the FP32-vs-FP64 comparison
    fp64 = None
    if args.fp64_steps > 0:
        R64 = lib.Registration(c["n"], n_t, c["n_c"], c["beta"], c["reg"], c["stokes"], lib.REG_FP64, args.ckpt)
        R64.set_images(mT, mR)
        R64.linearize(v)
        H64 = torch.empty_like(g)
        R64.hessvec(vt, H64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.fp64_steps):
            R64.hessvec(vt, H64)
        torch.cuda.synchronize()
        fp64_s = (time.perf_counter() - t0) / args.fp64_steps
        mixed_err = float(torch.linalg.vector_norm(Hv - H64) / torch.linalg.vector_norm(H64))
        # the FP64 form against both of its roofs: HBM and the measured FP64 FMA rate
        R64.profile_begin()
        R64.hessvec(vt, H64)
        p64 = R64.profile_end()
        dom64 = max(p64, key=lambda k: p64[k]["ms"])
        k64 = p64[dom64]
        peak64 = lib.fp64_peak_gflops()
        hbm_peak, _ = measured_peaks()
        fl_rate = k64["flops"] / (k64["ms"] / 1000.0) / 1e9 if k64["ms"] > 0 else 0.0
        by_rate = k64["bytes"] / (k64["ms"] / 1000.0) / 1e9 if k64["ms"] > 0 else 0.0
        fp64 = {"value": 1.0 / fp64_s, "unit": UNIT, "mixed_vs_fp64_rel_err": mixed_err,
                "roofline": {"kernel": dom64, "share_of_matvec": k64["ms"] / max(sum(x["ms"] for x in p64.values()), 1e-9),
                             "fp64_gflops_achieved": fl_rate, "fp64_gflops_peak": peak64,
                             "fp64_frac": fl_rate / peak64 if peak64 > 0 else None,
                             "fp64_peak_source": "measured live (reg_fp64_peak: FMA chains, CUDA events)",
                             "hbm_gbs_achieved": by_rate, "hbm_frac": by_rate / hbm_peak,
                             "flops_counted": "FFT butterflies, twiddles, multipliers and packing (radix-plan counts)"}}
        R64.close()

    # the same matvec with the whole state trajectory stored (no recomputation)
    store_all = None
    if args.store_all_steps > 0:
        Rs = lib.Registration(c["n"], n_t, c["n_c"], c["beta"], c["reg"], c["stokes"], lib.REG_MIXED, 0)
        Rs.set_images(mT, mR)
        Rs.linearize(v)
        Hs = torch.empty_like(g)
        Rs.hessvec(vt, Hs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.store_all_steps):
            Rs.hessvec(vt, Hs)
        torch.cuda.synchronize()
        ts = (time.perf_counter() - t0) / args.store_all_steps
        store_all = {"value": 1.0 / ts, "unit": UNIT, "ckpt_every": 0,
                     "rel_diff_vs_ckpt": float(torch.linalg.vector_norm(Hs - Hv) / torch.linalg.vector_norm(Hv))}
        Rs.close()
        torch.cuda.empty_cache()

    # the full Newton matvec (N-PCG) in the headline configuration
    newton = None
    if args.newton_steps > 0:
        Rn = lib.Registration(c["n"], n_t, c["n_c"], c["beta"], c["reg"], c["stokes"], lib.REG_MIXED, args.ckpt,
                              hessian=lib.REG_HESS_NEWTON)
        Rn.set_images(mT, mR)
        Rn.linearize(v)
        Hn = torch.empty_like(g)
        Rn.hessvec(vt, Hn)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.newton_steps):
            Rn.hessvec(vt, Hn)
        torch.cuda.synchronize()
        tn = (time.perf_counter() - t0) / args.newton_steps
        newton = {"value": 1.0 / tn, "unit": UNIT, "ckpt_every": args.ckpt,
                  "note": "same point as the headline (m_R = m_1 there, so the result equals Gauss-Newton)"}
        Rn.close()
        torch.cuda.empty_cache()

    # the workload's own n_t (unstable at the top modes in single precision)
    as_cfg = None
    if args.as_configured_steps > 0 and n_t != nt_cfg:
        Rc = lib.Registration(c["n"], nt_cfg, c["n_c"], c["beta"], c["reg"], c["stokes"], lib.REG_MIXED, args.ckpt)
        Rc.set_images(mT, mR)
        Rc.linearize(v)
        Hc = torch.empty_like(g)
        Rc.hessvec(vt, Hc)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.as_configured_steps):
            Rc.hessvec(vt, Hc)
        torch.cuda.synchronize()
        tc = (time.perf_counter() - t0) / args.as_configured_steps
        as_cfg = {"n_t": nt_cfg, "cfl": cfl_cfg, "value": 1.0 / tc, "unit": UNIT,
                  "mixed_result_norm_over_stable_norm": float(torch.linalg.vector_norm(Hc) /
                                                              torch.linalg.vector_norm(Hv))}
        Rc.close()

    peak, peak_src = measured_peaks()
    achieved = prof["bytes"] / (prof["ms"] / 1000.0) / 1e9 if prof["ms"] > 0 else 0.0
    traffic = kernel_traffic(dominant)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": dominant,
                "peak_source": f"{peak_src} (hbm_gbs)", "launches": prof["launches"],
                "bytes_per_launch": prof["bytes"] / max(prof["launches"], 1),
                "share_of_matvec": prof_all[dominant]["ms"] / max(sum(v["ms"] for v in prof_all.values()), 1e-9)}

    solves = solve_times() if not args.no_solves else None
    batch = batch_sample(args.batch_sample, args.workers) if (args.batch_sample > 0 and rank == 0) else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        T, t1, t2s = oracle_extrapolated(c, n_t)
        cpu = {"value": 1.0 / T, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle", "extrapolated": True,
               "sample": f"oracle GN matvec on the {args.n}^3 grid measured with n_t=1 ({t1:.1f} s) and n_t=2 "
                         f"({t2s[0]:.1f} s); the n_t={n_t} matvec is extrapolated linearly in n_t as "
                         f"t1 + {n_t - 1}*(t2 - t1) = {T:.1f} s (bench.py --impl reference --cpu-full measures one)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"random-field {args.n}^3 H2 beta=1e-3 n_c=1 n_t={n_t} GN matvec, "
                                   f"state checkpoints every {args.ckpt}",
                       "grid": [args.n] * 3, "n_t": n_t, "n_t_rule": f"doubled from {nt_cfg} until CFL <= {args.cfl}",
                       "cfl": cfl, "ckpt_every": args.ckpt,
                       "precision": "mixed (f32 sweeps; body force accumulated as a compensated f32 pair; "
                                    "f64 tail and Krylov vectors)",
                       "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}"},
            "clocks": ck, "gpu_launches": launches, "roofline": roofline, "e2e": e2e, "fp64": fp64,
            "store_all": store_all, "newton": newton, "as_configured": as_cfg, "solve_to_rel_grad_1e-2": solves, "batch_2d": batch, "cpu_baseline": cpu,
            "kernel_ms_per_matvec": {k: round(v["ms"], 3) for k, v in prof_all.items()},
            # every kernel kind of the profiled matvec: algorithmic bytes / event-timed duration
            "roofline_by_kind": {k: {"ms": round(v["ms"], 3), "launches": v["launches"],
                                     "GB_per_s": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1),
                                     "frac": round(v["bytes"] / (v["ms"] / 1e3) / 1e9 / peak, 4)}
                                 for k, v in prof_all.items() if v["ms"] > 0 and v["bytes"] > 0},
        }
        print(json.dumps(line), flush=True)
    R.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    global MAX_STACK
    args = parse()
    MAX_STACK = args.max_stack
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "profile":
        run_profile(args)
    elif args.workload == "stability":
        run_stability(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
