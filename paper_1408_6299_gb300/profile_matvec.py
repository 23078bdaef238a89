"""Profiling helper for the Gauss-Newton matvec on the random-field workload.

    python -m paper_1408_6299_gb300.profile_matvec --n 256 --n_t 128
        sets up the workload, runs one warm-up and one measured matvec and
        prints SETUP=<launches> WARM=<launches> MEAS=<launches>, the kernel
        launch counts to skip and capture with ncu (-s SETUP+WARM -c MEAS).

    python -m paper_1408_6299_gb300.profile_matvec --n 256 --sweep-nt 64,88,96,128
        for each n_t prints the CFL number and the relative 2-norm difference
        between the mixed-precision and the FP64 matvec (Heun stability check).
"""
import argparse
import sys

import numpy as np


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=256)
    p.add_argument("--n_t", type=int, default=128)
    p.add_argument("--ckpt", type=int, default=8)
    p.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    p.add_argument("--sweep-nt", default="")
    a = p.parse_args(argv)

    import torch

    from . import lib, synth

    c = synth.random_3d(a.n)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    v, mT, vt = dev(c["v_true"]), dev(c["mT"]), dev(c["vt"])
    shape = (1, 3) + c["n"]

    def context(n_t, prec):
        R = lib.Registration(c["n"], n_t, 1, c["beta"], c["reg"], c["stokes"], prec, a.ckpt)
        mR = torch.empty(c["n"], dtype=torch.float64, device="cuda")
        R.transport(v, mT, mR)
        R.set_images(mT, mR)
        R.linearize(v)
        return R

    if a.sweep_nt:
        for n_t in [int(x) for x in a.sweep_nt.split(",")]:
            out = {}
            for prec in (lib.REG_FP64, lib.REG_MIXED):
                R = context(n_t, prec)
                H = torch.empty(shape, dtype=torch.float64, device="cuda")
                R.hessvec(vt, H)
                out[prec] = H
                cfl = R.cfl(v)
                R.close()
            err = float(torch.linalg.vector_norm(out[1] - out[0]) / torch.linalg.vector_norm(out[0]))
            print(f"n_t={n_t} cfl={cfl:.4f} mixed_vs_fp64={err:.3e} "
                  f"norm_fp64={float(torch.linalg.vector_norm(out[0])):.6e} "
                  f"norm_mixed={float(torch.linalg.vector_norm(out[1])):.6e}", flush=True)
        return 0

    R = context(a.n_t, lib.REG_MIXED if a.precision == "mixed" else lib.REG_FP64)
    H = torch.empty(shape, dtype=torch.float64, device="cuda")
    l0 = lib.launch_count()
    R.hessvec(vt, H)
    l1 = lib.launch_count()
    R.hessvec(vt, H)
    l2 = lib.launch_count()
    torch.cuda.synchronize()
    print(f"SETUP={l0} WARM={l1 - l0} MEAS={l2 - l1}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
