"""CPU timing of the FP64 oracle in the style of the paper's own measurements
(Sec. 4): sequential AQS (Eq. 12) against Algorithm 1 run with P host threads
(one chain per thread), on the stored N = 256 glass, dgamma = 1e-4, 200
steps.  Test infrastructure: the oracle is slow by design, so these figures
are context for the method's parallel speed-up on CPU threads, not a target.

Usage: python tests/oracle_cpu_scaling.py [--steps 200] [--P 4 8] [--K 1 10]
Prints one markdown table (wall-clock seconds, speed-up over sequential,
passes, rejections) with the host's core count and CPU model.
"""
import argparse
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2507_20802_gb300 import synthetic as syn  # noqa: E402


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--P", type=int, nargs="+", default=[4, 8])
    ap.add_argument("--K", type=int, nargs="+", default=[1, 10])
    ap.add_argument("--dgamma", type=float, default=1e-4)
    args = ap.parse_args()
    oracle.build()
    g = dict(np.load(os.path.join(ROOT, "tests", "golden", "glass_2d_n256_s0.npz")))
    pot = oracle.make_potential(2, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    fp = oracle.make_fire(**syn.FIRE)
    t0 = time.perf_counter()
    seq = oracle.aqs(pot, fp, g["x"], g["types"], g["H"], args.dgamma, args.steps)
    t_seq = time.perf_counter() - t0
    assert seq["status"] == 0
    rows = [("sequential (Eq. 12)", 1, "-", t_seq, 1.0, "-", "-", "-")]
    for K in args.K:
        for P in args.P:
            t0 = time.perf_counter()
            r = oracle.parallel(pot, fp, g["x"], g["types"], g["H"], args.dgamma, K, P,
                                args.steps, eq_tol=1e-6, n_threads=P)
            dt = time.perf_counter() - t0
            assert r["status"] == 0
            rej = int(np.sum(r["log_eq"] == 0))
            same = np.allclose(r["E"], seq["E"], rtol=1e-9)
            rows.append((f"Algorithm 1, P = {P}, K = {K}", P, K, dt, t_seq / dt,
                         int(r["iterations"]), rej, "yes" if same else "no"))
    print(f"host: {os.cpu_count()} cores, {cpu_model()}; N = 256 glass (seed 0), "
          f"dgamma = {args.dgamma}, {args.steps} steps, FP64 all-pairs oracle\n")
    print("| run | threads | K | wall s | speed-up | passes | rejections | energies = sequential |")
    print("|---|---:|---:|---:|---:|---:|---:|---|")
    for name, thr, K, dt, sp, it, rej, same in rows:
        print(f"| {name} | {thr} | {K} | {dt:.1f} | {sp:.2f} | {it} | {rej} | {same} |")


if __name__ == "__main__":
    main()
