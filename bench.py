"""Benchmark: converged AQS strain steps per second of two-level parallel
stepping (Algorithm 1) on one GB300, with FIRE minimisation in mixed precision.

Workload (one "step" = one pass of Algorithm 1's while loop: level I, P batched
level-II chains of K fine AQS steps each, the equality tests and r_star <- r_q):
  2D binary Lennard-Jones glass, 65:35 A:B, N = 4096, number density 1.2,
  shifted-force cutoff 2.5 sigma_ab, uniform random start (seed = rank)
  quenched on the GPU to |F|max < 1e-10 (untimed set-up), simple shear
  dgamma = 1e-4, K = 10, P = 16, every step converged to |F|max < 1e-10 (FP64).
  Inputs are synthetic (seeded) and stand in for the paper's melt-quenched
  samples.

Reported (one JSON line on rank 0):
  value    accepted fine strain steps / s, device-timed (CUDA events on the
           library's stream) over the K timed passes, L2 flushed between passes
  e2e      the same metric through the public C ABI with host buffers:
           host -> device positions, the pass, device -> host positions and
           per-step observables, all inside the timed region
  roofline the persistent minimiser kernel (FP32 pipe; its FP64 work noted)
  cpu_baseline  the FP64 oracle on the host cores: complete converged AQS
           steps of the N = 256 glass (the small configuration of this
           workload; the all-pairs oracle cannot finish an N = 4096 step in
           the time a benchmark run allows)
  fp64_sequential_gpu_baseline  plain sequential AQS with the same kernels in
           FP64 mode, one replica, no batching: 20 steps sampled at four
           points of the timed strain window
  clocks   SM clocks and throttle reasons sampled during the timed region

``--impl reference`` times the oracle instead (the CPU program this project is
checked against): each step is one converged AQS step of the N = 256 glass.
``--workload oracle-threads`` reproduces the paper's own kind of measurement
with the oracle on host threads (sequential AQS against Algorithm 1 with one
chain per thread).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ATOMS, P_CHAINS, K_FINE, DGAMMA, GAMMA_END = 4096, 16, 10, 1e-4, 0.2
METRIC = "converged AQS strain steps/s (two-level parallel stepping, |F|max<1e-10)"
UNIT = "steps/s"
# Algorithmic flops of the method per list entry (one atom looking at one
# neighbour) of a 2D shifted-force LJ force-and-energy evaluation, FMA = 2:
#   separation d = (q_j - q_i) + image offset   4
#   r^2, cutoff test                            4
#   u = 1/r^2, u^3, u^4, u^7, r^-1              6
#   phi = A u^7 + B u^4 + C r^-1                5
#   F_i += phi d                                4
#   U_sf = e12 u^6 - e6 u^3 - Uc - (r - rc) dUc 7
# = 30.  (The kernel's own mixed-precision formulation, F_ref + dF by exact
# divided differences, executes about 62 FP32 flops per visit; that count is
# reported beside it as "kernel_flop_per_visit".)
FLOP32_PER_PAIR = 30
KERNEL_FLOP32_PER_VISIT = 62
FLOP64_PER_PAIR = 32
# DRAM bytes (read + write) of the dominant kernel from one ncu capture each
# (--set full, clocks unlocked), for the roofline's "traffic"; a capture is
# valid only for the kernel version it was taken on (None: not captured on
# the current kernel).
#   Algorithm 1 (2D, N = 4096): one level-II chain launch, per barrier mode of
#   the chains (thread-block clusters, or one cooperative launch with grid
#   barriers); the kernel runs from L2, and its DRAM traffic is the working
#   set read once per launch
TRAFFIC_CFG1_PER_LAUNCH = {"cluster": 10_614_016, "grid_barrier": 11_797_504}
#   3D (N = 65536), per replica-iteration of the timed launch (6 replicas x
#   200 iterations: 35.88 GB read + 0.45 GB written; a capture of only the
#   two DRAM counters)
TRAFFIC_3D_PER_REPLICA_ITER = 30_277_000

CONFIG = {"workload": "2D binary LJ glass (65:35, rho=1.2), N=4096, Algorithm 1 with P=16 "
                      "chains of K=10 fine steps, dgamma=1e-4, FIRE to |F|max<1e-10, mixed "
                      "precision", "n_atoms": N_ATOMS, "P": P_CHAINS, "K": K_FINE,
          "dgamma": DGAMMA, "gamma_end": GAMMA_END, "precision": "mixed",
          "l2": "flushed (256 MiB write) between timed passes"}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.path = os.path.join(tempfile.gettempdir(), f"aqs_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200",
                                          "-i", str(self.gpu)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [v.strip() for v in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def fp32_peak_tflops():
    """FP32 peak of the device from its unit counts: SMs (queried) x 128 FP32
    lanes x 2 flop (FMA) x the maximum SM clock (measured peaks file, else
    nvidia-smi, else 2.07 GHz)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = _peaks().get("sm_max_mhz")
    if not mhz:
        try:
            out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm",
                                  "--format=csv,noheader,nounits", "-i", "0"],
                                 capture_output=True, text=True, timeout=20).stdout
            mhz = float(out.split()[0])
        except Exception:
            mhz = 2070.0
    return sms * 128 * 2 * float(mhz) * 1e6 / 1e12, sms, float(mhz)


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def host_desc():
    return {"nproc": os.cpu_count(), "cpu": cpu_model(), "machine": platform.machine()}


def combine_ranks(secs, units, device):
    """Whole-job figures over the ranks (weak scaling, one glass per rank):
    the sum of the units every rank processed and the slowest rank's time.
    Returns (units, seconds); a single process returns its own figures."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(units), float(secs)
    tt = torch.tensor([float(secs), float(units)], device=device, dtype=torch.float64)
    mx = tt.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    return float(tt[1]), float(mx[0])


def oracle_steps(n_steps=None, budget_s=None, dgamma=DGAMMA):
    """Complete converged AQS steps (Eq. 12: affine dgamma, then FIRE to
    |F|max < 1e-10) of the FP64 all-pairs oracle on one host core, from the
    stored N = 256 glass (the small configuration of this workload).  Runs
    n_steps steps, or steps one at a time until budget_s seconds are used (at
    least two).  Returns (steps, seconds, FIRE iterations)."""
    import oracle
    from paper_2507_20802_gb300 import synthetic as syn
    oracle.build()
    g = np.load(os.path.join(ROOT, "tests", "golden", "glass_2d_n256_s0.npz"))
    x, t, H = g["x"], g["types"], g["H"]
    pot = oracle.make_potential(2, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    fp = oracle.make_fire(**syn.FIRE)
    steps, secs, iters = 0, 0.0, 0
    while True:
        t0 = time.perf_counter()
        r = oracle.aqs(pot, fp, x, t, H, dgamma, 1)
        secs += time.perf_counter() - t0
        assert r["status"] == 0
        x, H = r["x"], r["H"]
        steps += 1
        iters += int(r["iters"][0])
        if n_steps is not None and steps >= n_steps:
            break
        if budget_s is not None and secs >= budget_s and steps >= 2:
            break
    return steps, secs, iters


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    per_step = []
    for i in range(args.warmup + args.steps):
        n, dt, it = oracle_steps(n_steps=1)
        if i >= args.warmup:
            per_step.append((dt, it))
    secs = sum(d for d, _ in per_step)
    value = len(per_step) / secs
    sample = ("each step: one complete AQS step (dgamma=1e-4, FIRE to |F|max<1e-10, %d FIRE "
              "iterations on average) of the FP64 all-pairs oracle on the N=256 glass, one host "
              "core; the N=4096 glass of this workload costs (4096/256)^2 = 256x more per "
              "iteration in this O(N^2) oracle and ~10x more iterations per step"
              % round(np.mean([i for _, i in per_step])))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / max(1, len(per_step)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": CONFIG,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample, "host": host_desc()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_oracle_threads(args):
    """The paper's own kind of measurement (Sec. 4) with the FP64 oracle on
    this machine's host cores: sequential AQS (Eq. 12) against Algorithm 1
    with one level-II chain per POSIX thread, on the stored N = 256 glass,
    dgamma = 1e-4.  Prints one line with a row per (P, K): wall seconds,
    speed-up over sequential, passes, rejections, and whether the energies
    equal the sequential run's."""
    import oracle
    from paper_2507_20802_gb300 import synthetic as syn
    oracle.build()
    g = np.load(os.path.join(ROOT, "tests", "golden", "glass_2d_n256_s0.npz"))
    pot = oracle.make_potential(2, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    fp = oracle.make_fire(**syn.FIRE)
    n = args.oracle_steps
    t0 = time.perf_counter()
    seq = oracle.aqs(pot, fp, g["x"], g["types"], g["H"], DGAMMA, n)
    t_seq = time.perf_counter() - t0
    assert seq["status"] == 0
    rows = []
    for K in args.oracle_K:
        for P in args.oracle_P:
            if P > (os.cpu_count() or 1):
                continue
            t0 = time.perf_counter()
            r = oracle.parallel(pot, fp, g["x"], g["types"], g["H"], DGAMMA, K, P, n,
                                eq_tol=1e-6, n_threads=P)
            dt = time.perf_counter() - t0
            assert r["status"] == 0
            rows.append({"P": P, "K": K, "threads": P, "wall_s": dt, "speedup": t_seq / dt,
                         "passes": int(r["iterations"]),
                         "rejections": int(np.sum(r["log_eq"] == 0)),
                         "energies_equal_sequential": bool(np.allclose(r["E"], seq["E"],
                                                                       rtol=1e-9))})
    best = max((r["speedup"] for r in rows), default=1.0)
    line = {"metric": "Algorithm 1 speed-up over sequential AQS, FP64 oracle on host threads",
            "value": best, "unit": "x", "n_gpus": 0, "steps": n, "warmup": 0,
            "ms_per_step": 1e3 * t_seq / n, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "N=256 2D binary LJ glass (seed 0), dgamma=1e-4, %d steps, "
                                   "FP64 all-pairs oracle, one chain per POSIX thread" % n},
            "host": host_desc(), "sequential_s": t_seq, "rows": rows,
            "paper": "2.02-6.33x average speed-up at 4-32 threads (CPU, hardware not stated)"}
    print(json.dumps(line), flush=True)
    return 0


def _line(metric, value, unit, args, ms, config, extra):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
         "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
         "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": config}
    d.update(extra)
    print(json.dumps(d), flush=True)


def run_seeds(args):
    """Metric 1 over several glasses: for seeds 0..n-1 the FP64-quenched glass,
    one warm-up pass (autotuning the chains) and `steps` timed passes of
    Algorithm 1; prints one line with the per-seed values, their mean and
    standard deviation (device time, same workload as the default line)."""
    import torch
    from paper_2507_20802_gb300 import aqs as A, synthetic as syn
    torch.cuda.set_device(0)
    vals, accepted_all, ms_all = [], [], 0.0
    for seed in range(args.seeds):
        x, t, H = syn.random_glass_start(N_ATOMS, 2, seed=seed)
        g = A.System(x, t, H[None], [N_ATOMS], syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR,
                     precision=A.AQS_FP64)
        q = g.minimize(A.fire_params(max_iter=2_000_000))[0]
        assert q["status"] == 0, q
        xq, Hq = g.positions(), g.box()
        g.close()
        s = A.System(xq, t, Hq[None], [N_ATOMS], syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR,
                     precision=A.AQS_MIXED)
        if args.autotune > 0:
            s.set_autotune(args.autotune)
        s.set_launch_budget(args.launch_budget)
        n_total = int(round(GAMMA_END / DGAMMA))
        done = 0

        def one_pass():
            nonlocal done
            r = s.parallel_step(DGAMMA, K_FINE, P_CHAINS, max(1, n_total - done),
                                max_iterations=1)
            done += r["accepted"]
            return r
        for _ in range(max(1, args.warmup)):
            one_pass()
        acc, ms = 0, 0.0
        for _ in range(args.steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = one_pass()
            e1.record()
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            acc += r["accepted"]
        vals.append(acc / (ms / 1e3))
        accepted_all.append(acc)
        ms_all += ms
        s.close()
    v = np.array(vals)
    config = dict(CONFIG, seeds=list(range(args.seeds)),
                  l2="not flushed (seed statistics; the default line flushes)")
    _line(METRIC + ", mean over glasses", float(v.mean()), UNIT, args,
          ms_all / max(1, args.seeds * args.steps), config,
          {"per_seed": [float(a) for a in v], "std": float(v.std(ddof=1)) if len(v) > 1 else 0.0,
           "accepted_per_seed": accepted_all,
           "note": "one warm-up pass then the timed passes, each glass from the same strain"})


def run_warm(args):
    """The learned warm start's kernels at the inference size of the warm-start
    workload (32 replicas x 16384 atoms = 524288 per-atom rows): BF16
    tensor-core MLP forward (66 -> 128 -> 128 -> 128 -> 2), fused forward +
    backward + AdamW training step on 65536-row batches, and the FP64
    neighbour-shell features of the same 524288 atoms.  value = inference rows/s."""
    import torch
    from paper_2507_20802_gb300 import aqs as A, synthetic as syn
    torch.cuda.set_device(0)
    R, n = 32, 16384
    rows = R * n
    flop_fwd = 2 * (66 * 128 + 2 * 128 * 128 + 128 * 2)  # algorithmic, per row
    g = torch.Generator(device="cpu").manual_seed(0)
    feat = (torch.randn((rows, A.WARM_IN), generator=g) * 0.5).to(torch.bfloat16).cuda()
    feat[:, 66:] = 0
    target = torch.randn((rows, 2), generator=g).cuda()
    out = torch.zeros((rows, 2), dtype=torch.float32, device="cuda")
    w = A.Warm(seed=1)
    l0 = A.aqs_launch_count()

    def timed(fn, reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    for _ in range(max(3, args.warmup)):
        w.predict(feat, out)
    with Clocks(0) as clk:
        t_fwd = timed(lambda: w.predict(feat, out), max(1, args.steps) * 4)
        batch = 65536
        k = [0]

        def step():
            i = k[0] % (rows // batch)
            k[0] += 1
            w.train_step(feat[i * batch:(i + 1) * batch], target[i * batch:(i + 1) * batch], 1e-3)
        step()
        t_train = timed(step, max(1, args.steps) * 4)
        # features of 32 replicas of a 16384-atom 2D configuration
        xs, ts, Hs = [], [], []
        for r in range(R):
            x, t, H = syn.random_glass_start(n, 2, seed=2000 + r)
            xs.append(x); ts.append(t); Hs.append(H)
        sy = A.System(np.concatenate(xs), np.concatenate(ts), np.stack(Hs), [n] * R,
                      syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR, precision=A.AQS_MIXED)
        fb = torch.zeros((rows, A.WARM_IN), dtype=torch.bfloat16, device="cuda")
        sy.warm_features(fb)
        t_feat = timed(lambda: sy.warm_features(fb), max(1, args.steps))
    peak = _peaks().get("bf16_tflops", 1900.0)
    fwd_tf = rows * flop_fwd / t_fwd / 1e12
    train_tf = 3 * batch * flop_fwd / t_train / 1e12
    config = {"workload": "learned warm start: MLP 66->128->128->128->2 (BF16, FP32 accumulate) "
                          "on 524288 per-atom rows (32 x 16384 atoms), training on 65536-row "
                          "batches, FP64 32-neighbour features", "rows": rows,
              "train_batch": batch, "l2": "inputs (84 MB of BF16 features) resident; not flushed"}
    _line("warm-start inference rows/s", rows / t_fwd, "rows/s", args, 1e3 * t_fwd, config,
          {"gpu_launches": A.aqs_launch_count() - l0, "clocks": clk.summary(),
           "roofline": {"bound": "tensor", "achieved": fwd_tf, "peak": peak, "unit": "TFLOP/s",
                        "frac": fwd_tf / peak, "traffic": None,
                        "note": "algorithmic 82944 flop per row; mma.sync BF16 (not tcgen05); "
                                "peak = measured cuBLAS bf16 burst"},
           "detail": {"train_step_ms": 1e3 * t_train, "train_rows_per_s": batch / t_train,
                      "train_tflops": train_tf, "train_frac": train_tf / peak,
                      "features_ms": 1e3 * t_feat, "features_rows_per_s": rows / t_feat}})


def run_warm_eval(args):
    """The learned warm start at the scale of its workload.  Training data come
    from the method itself: 16 N = 4096 glasses (seeds 100..115, mixed-
    precision GPU quench), `warm_collect` over 4 AQS steps of dgamma = 1e-4
    (features of each minimum, the non-affine displacement per unit strain of
    the next step as target): 262 144 per-atom rows, the last step held out.
    Evaluation on 8 held-out glasses of N = 16384 (seeds 0..7, one batched
    system): `steps` sequential AQS steps with the gated learned start against
    the plain affine start from the same minima (Algorithm 1 does not take the
    learned start).  value = FIRE iterations of the plain run / those of the
    learned run (above 1: the learned start saves iterations); the detail
    gives both runs' iterations per step and steps/s (device time), the steps
    that kept the learned start, and how far the two runs' energies and event
    steps agree."""
    import torch
    from paper_2507_20802_gb300 import aqs as A, synthetic as syn
    torch.cuda.set_device(0)
    dg = 1e-4

    def glasses(n, seeds):
        xs, ts, Hs = [], [], []
        for sd in seeds:
            x, t, H = syn.random_glass_start(n, 2, seed=sd)
            xs.append(x); ts.append(t); Hs.append(H)
        g = A.System(np.concatenate(xs), np.concatenate(ts), np.stack(Hs), [n] * len(seeds),
                     syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR, precision=A.AQS_MIXED)
        q = g.minimize(A.fire_params(max_iter=args.quench_iters))
        assert all(r["status"] == 0 for r in q), [r["status"] for r in q]
        return g, np.concatenate(ts), max(r["iters"] for r in q)

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        e1.synchronize()
        return out, e0.elapsed_time(e1) / 1e3

    l0 = A.aqs_launch_count()
    # ---- training data: 16 x 4096 atoms, 4 steps
    n_tr, g_tr, st_tr = 4096, 16, 4
    tr, _, q_tr = glasses(n_tr, range(100, 100 + g_tr))
    rows_step = n_tr * g_tr
    F = torch.zeros((st_tr * rows_step, A.WARM_IN), dtype=torch.bfloat16, device="cuda")
    T = torch.zeros((st_tr * rows_step, 2), dtype=torch.float32, device="cuda")
    _, t_collect = timed(lambda: tr.warm_collect(dg, st_tr, F, T))
    tr.close()
    n_train = (st_tr - 1) * rows_step
    w = A.Warm(seed=1)
    batch, iters = 65536, args.warm_train_iters
    losses = []

    def train():
        for it in range(iters):
            i = it % (n_train // batch)
            lr = 2e-3 if it < (2 * iters) // 3 else 5e-4
            losses.append(w.train_step(F[i * batch:(i + 1) * batch], T[i * batch:(i + 1) * batch],
                                       lr))
    _, t_train = timed(train)
    held, _ = w.loss_grad(F[n_train:], T[n_train:])
    base = 0.5 * float((T[n_train:] ** 2).sum(dim=1).mean())
    del F, T
    # ---- evaluation: 8 held-out glasses of 16384 atoms
    n_ev, g_ev = 16384, 8
    plain, t_ev, q_ev = glasses(n_ev, range(g_ev))
    x0 = np.concatenate([plain.positions(r) for r in range(g_ev)])
    H0 = np.stack([plain.box(r) for r in range(g_ev)])
    warm = A.System(x0, t_ev, H0, [n_ev] * g_ev, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR,
                    precision=A.AQS_MIXED)
    steps = max(1, args.steps)
    with Clocks(0) as clk:
        rp, t_plain = timed(lambda: plain.run_sequential(dg, steps))
        rw, t_warm = timed(lambda: warm.run_sequential_warm(w, dg, steps))
    it_p, it_w = int(rp["iters"].sum()), int(rw["iters"].sum())
    e_dev = float(np.max(np.abs(rw["E"] - rp["E"]) / np.abs(rp["E"])))
    ev_same = bool(np.array_equal(rw["D"] > 1e-2, rp["D"] > 1e-2))
    config = {"workload": "learned warm start: MLP trained on 4 AQS steps of 16 N=4096 2D glasses "
                          "(seeds 100-115, 262144 rows, last step held out); sequential AQS "
                          "dgamma=1e-4 on 8 held-out N=16384 glasses (seeds 0-7), gated learned "
                          "start vs plain affine start, mixed precision",
              "train_glasses": g_tr, "train_atoms": n_tr, "train_rows": n_train,
              "eval_glasses": g_ev, "eval_atoms": n_ev, "steps": steps, "dgamma": dg,
              "l2": "working set on chip / L2; not flushed"}
    _line("FIRE-iteration gain of the learned warm start (plain / learned)", it_p / max(1, it_w),
          "x", args, 1e3 * (t_plain + t_warm), config,
          {"gpu_launches": A.aqs_launch_count() - l0, "clocks": clk.summary(),
           "detail": {"fire_iters_per_glass_step_plain": it_p / (steps * g_ev),
                      "fire_iters_per_glass_step_learned": it_w / (steps * g_ev),
                      "glass_steps_per_s_plain": steps * g_ev / t_plain,
                      "glass_steps_per_s_learned": steps * g_ev / t_warm,
                      "learned_start_kept": int(rw["used"].sum()), "glass_steps": steps * g_ev,
                      "max_rel_energy_diff": e_dev, "same_event_steps": ev_same,
                      "train_loss_first_last": [losses[0], losses[-1]], "train_iters": iters,
                      "held_out_loss": held, "zero_prediction_loss": base,
                      "collect_s": t_collect, "train_s": t_train,
                      "quench_iters_max": {"train": q_tr, "eval": q_ev}}})
    plain.close()
    warm.close()


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(path)) if os.path.exists(path) else {}


def run_batch64(args):
    """64 independent 2D glasses of log-uniform size in [1024, 16384] (sizes
    from stream seed 2, glass r from seed 1000 + r), plain AQS dgamma = 5e-5,
    all in one batched system (per-replica convergence, concurrent launches
    for the different cluster sizes).  value = glass-steps / s."""
    import torch
    from paper_2507_20802_gb300 import aqs as A, synthetic as syn
    torch.cuda.set_device(0)
    sizes = syn.log_uniform_sizes(64, 1024, 16384, seed=2)
    xs, ts, Hs = [], [], []
    for r, n in enumerate(sizes):
        x, t, H = syn.random_glass_start(int(n), 2, seed=1000 + r)
        xs.append(x); ts.append(t); Hs.append(H)
    # the glasses are FP64 quenches (independent of the mixed path's rounding)
    g = A.System(np.concatenate(xs), np.concatenate(ts), np.stack(Hs), sizes, syn.LJ_SIGMA,
                 syn.LJ_EPS, syn.RC_FACTOR, precision=A.AQS_FP64)
    res = g.minimize(A.fire_params(max_iter=2_000_000))
    quench = int(max(q["iters"] for q in res))
    xq = np.concatenate([g.positions(r) for r in range(64)])
    Hq = np.stack([g.box(r) for r in range(64)])
    g.close()
    s = A.System(xq, np.concatenate(ts), Hq, sizes, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR,
                 precision=A.AQS_MIXED)
    for _ in range(args.warmup):
        s.run_sequential(5e-5, 1)
    A.aqs_reset_kernel_stats()
    A.aqs_set_kernel_timing(True)
    l0 = A.aqs_launch_count()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        e0.record()
        out = s.run_sequential(5e-5, args.steps)
        e1.record()
        e1.synchronize()
    st = A.aqs_get_kernel_stats()
    A.aqs_set_kernel_timing(False)
    secs = e0.elapsed_time(e1) / 1e3
    value = 64 * args.steps / secs
    kern_s = st["kernel_ms"] / 1e3
    achieved = st["pairs32"] * FLOP32_PER_PAIR / kern_s / 1e12 if kern_s else 0.0
    peak32, n_sm, mhz = fp32_peak_tflops()
    config = {"workload": "64 independent 2D binary LJ glasses, N log-uniform in [1024, 16384] "
                          "(sum %d), plain AQS dgamma=5e-5, batched mixed precision" % int(sizes.sum()),
              "n_glasses": 64, "atoms_total": int(sizes.sum()), "dgamma": 5e-5,
              "l2": "working set on chip / L2; not flushed"}
    _line("converged AQS glass-steps/s (64 glasses batched)", value, "glass-steps/s", args,
          1e3 * secs / max(1, args.steps), config,
          {"gpu_launches": A.aqs_launch_count() - l0, "clocks": clk.summary(),
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak32,
                        "unit": "TFLOP/s", "frac": achieved / peak32, "traffic": None,
                        "flop_per_list_entry": FLOP32_PER_PAIR,
                        "peak_note": "FP32 peak derived: %d SMs x 128 lanes x 2 x %.0f MHz"
                                     % (n_sm, mhz)},
           "detail": {"fire_iters_per_step_mean": float(out["iters"].mean()),
                      "fire_iters_per_step_max": int(out["iters"].max()), "quench_iters_max": quench,
                      "slowest_glass": {"index": int(np.argmax(out["iters"].sum(axis=0))),
                                        "n_atoms": int(sizes[int(np.argmax(out["iters"].sum(axis=0)))]),
                                        "iters_per_step": out["iters"][:, int(np.argmax(out["iters"].sum(axis=0)))].tolist(),
                                        "D_per_step": out["D"][:, int(np.argmax(out["iters"].sum(axis=0)))].tolist()},
                      "glass_quench": "FP64",
                      "cluster_sizes": sorted({s.cluster_size(r) for r in range(64)})}})


def run_glass3d(args):
    """3D binary LJ glass (80:20, N = 65536, density 1.2), the level-II fine
    steps of Algorithm 1: replica i is the quenched glass after (i + 1) fine
    shear steps of 5e-5, and the replicas are minimised together for a bounded
    number of FIRE iterations (the regime where AQS spends its iterations:
    small displacements from a converged state).  value = FIRE iterations / s
    summed over the replicas; the roofline reports the force kernel's streamed
    list and position bytes against HBM."""
    import torch
    from paper_2507_20802_gb300 import aqs as A, synthetic as syn
    torch.cuda.set_device(0)
    n, P, K, dg = 65536, args.replicas3d, 20, 5e-5
    x, t, H = syn.random_glass_start(n, 3, seed=0)
    s = A.System(x, t, H[None], [n], syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR,
                 precision=A.AQS_MIXED)
    q = s.minimize(A.fire_params(max_iter=args.quench_iters), check_status=False)[0]
    xq, Hq = s.positions(), s.box()
    s.close()
    b = A.System(np.tile(xq, (P, 1)), np.tile(t, P), np.tile(Hq[None], (P, 1, 1)), [n] * P,
                 syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR, precision=A.AQS_MIXED)
    b.shear((np.arange(P) + 1) * dg)
    nb = b.mean_neighbours(0)
    budget = args.iters3d
    b.minimize(A.fire_params(max_iter=50), check_status=False)  # warm-up
    A.aqs_reset_kernel_stats()
    A.aqs_set_kernel_timing(True)
    l0 = A.aqs_launch_count()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        torch.cuda.nvtx.range_push("glass3d_timed")
        e0.record()
        res = b.minimize(A.fire_params(max_iter=budget), check_status=False)
        e1.record()
        e1.synchronize()
        torch.cuda.nvtx.range_pop()
    st = A.aqs_get_kernel_stats()
    A.aqs_set_kernel_timing(False)
    secs = e0.elapsed_time(e1) / 1e3
    iters = sum(r["iters"] for r in res)
    kern_s = st["kernel_ms"] / 1e3
    # algorithmic bytes of the FP32 force evaluations: 4 B per list entry
    # (the lists, ~0.4 GB per replica set, stream from HBM) plus 28 B per atom
    # (its 16-byte position record and 12-byte FP32 force); neighbour records
    # are gathered from cell-sorted storage and are not counted
    algo_bytes = 4.0 * st["pairs32"] + 28.0 * n * st["evals32"]
    gbs = algo_bytes / kern_s / 1e9 if kern_s else 0.0
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    config = {"workload": "3D binary LJ glass (80:20, rho=1.2), N=65536: %d replicas, replica i "
                          "the quenched glass after i+1 fine shear steps of dgamma=5e-5, minimised "
                          "as one batch for a bounded number of FIRE iterations, mixed precision"
                          % P,
              "n_atoms": n, "replicas": P, "dgamma": dg, "fire_iterations_budget": budget,
              "l2": "working set (~%d MB of lists) exceeds L2" % int(4 * nb * n * P / 1e6)}
    _line("FIRE iterations/s (3D, %d x 65536 atoms)" % P, iters / secs, "iterations/s", args,
          1e3 * secs, config,
          {"gpu_launches": A.aqs_launch_count() - l0, "clocks": clk.summary(),
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                        "frac": gbs / peak,
                        "traffic": (TRAFFIC_3D_PER_REPLICA_ITER * iters / max(1, st["launches"])
                                    if TRAFFIC_3D_PER_REPLICA_ITER else None),
                        "note": "algorithmic bytes = 4 per list entry visited + 28 per atom per FP32 evaluation"},
           "detail": {"mean_neighbours": nb, "quench_iters": q["iters"],
                      "quench_fmax": q["fmax"], "fp32_evals": st["evals32"],
                      "fp64_evals": st["evals64"], "rebuilds_in_kernel": st["rebuilds"],
                      "cluster_size": b.cluster_size(0), "staging": b.staging(0)}})


def run_sweep(args):
    """The paper's experiment (Sec. 4) on the GPU: its S/L glass model (N =
    400, density 1), simple shear dgamma = 1/200 for 200 steps (gamma = 1),
    for every glass j (seeds 0..n-1, FP64 GPU quench of the seeded start) the
    run time C_S of sequential AQS and C_(P,K) of Algorithm 1 for P in
    {4, 8, 16, 32} and K in {1, 2, 6, 10, 14, 16}; speed-up S_j = C_S / C_(P,K),
    and its mean mu and standard deviation sigma over the glasses (the paper's
    definitions).  Every run's final configuration is checked to equal the
    sequential one (1e-6 sigma), as the paper reports for its runs.  Mixed
    precision, device time.  value = mu at (P, K) = (32, 10)."""
    import torch
    from paper_2507_20802_gb300 import aqs as A, synthetic as syn
    torch.cuda.set_device(0)
    n, dg, steps = 400, 1.0 / 200.0, 200
    Ps, Ks = args.sweep_P, args.sweep_K

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        e1.synchronize()
        return out, e0.elapsed_time(e1) / 1e3

    def mi(a, b, H):
        d = a - b
        for c in (1, 0):
            d -= np.round(d[:, c] / H[c, c])[:, None] * H[:, c][None, :]
        d -= d.mean(axis=0)
        return float(np.sqrt((d * d).sum(1)).max())

    S = {(P, K): [] for P in Ps for K in Ks}
    seq_s, all_equal, rej = [], True, {}
    l0 = A.aqs_launch_count()
    with Clocks(0) as clk:
        for seed in range(args.sweep_seeds):
            x, t, H = syn.random_glass_start(n, 2, seed, fraction_a=syn.SL_FRACTION_S,
                                             density=syn.SL_DENSITY)
            g = A.System(x, t, H[None], [n], syn.SL_SIGMA, syn.SL_EPS, syn.RC_FACTOR,
                         precision=A.AQS_FP64)
            assert g.minimize(A.fire_params(max_iter=2_000_000))[0]["status"] == 0
            xq, Hq = g.positions(), g.box()
            g.close()

            def mk():
                return A.System(xq, t, Hq[None], [n], syn.SL_SIGMA, syn.SL_EPS, syn.RC_FACTOR,
                                precision=A.AQS_MIXED)
            s0 = mk()
            s0.run_sequential(dg, 2)  # warm-up of this glass's launch path
            s0.close()
            s0 = mk()
            _, cs = timed(lambda: s0.run_sequential(dg, steps))
            x_seq, H_seq = s0.positions(), s0.box()
            s0.close()
            seq_s.append(cs)
            for P in Ps:
                for K in Ks:
                    sp = mk()
                    r, cp = timed(lambda: sp.parallel_step(dg, K, P, steps))
                    all_equal = all_equal and mi(sp.positions(), x_seq, H_seq) < 1e-6
                    rej[(P, K)] = rej.get((P, K), 0) + int(r["rejections"])
                    sp.close()
                    S[(P, K)].append(cs / cp)
    table = []
    for P in Ps:
        for K in Ks:
            v = np.array(S[(P, K)])
            table.append({"P": P, "K": K, "mu": float(v.mean()), "sigma": float(v.std()),
                          "S": [float(a) for a in v], "rejections": rej[(P, K)]})
    head = next((r for r in table if r["P"] == 32 and r["K"] == 10), table[-1])
    config = {"workload": "the paper's S/L glass (N=400, density 1), dgamma=1/200, 200 steps, "
                          "%d glasses (seeds 0..%d, FP64 GPU quench), mixed precision, "
                          "P in %s, K in %s" % (args.sweep_seeds, args.sweep_seeds - 1, Ps, Ks),
              "l2": "working set on chip; not flushed"}
    _line("Algorithm 1 speed-up mu over sequential AQS (the paper's mu, P=%d, K=%d)"
          % (head["P"], head["K"]), head["mu"], "x", args, 1e3 * float(np.mean(seq_s)), config,
          {"gpu_launches": A.aqs_launch_count() - l0, "clocks": clk.summary(),
           "sigma": head["sigma"], "all_final_configurations_equal": all_equal,
           "sequential_s": [float(a) for a in seq_s], "table": table,
           "paper": "mu 2.02 (P=4, K=1) to 6.33 (P=32, K=10), CPU threads, hardware not stated"})


def run_tune_table(args):
    """The launch-configuration table of the benchmark's level-II chains: the
    N = 4096 glass (FP64 GPU quench of seed 0) in 16 replicas at the level-I
    strains i K dgamma, minimised and sheared one fine step, then the
    autotuner's time per FIRE iteration for every cluster size (and the
    staging modes at the best one), with one thread per atom and with the
    split force phase allowed; also for a single replica (the sequential
    AQS shape).  Prints one line."""
    import torch
    from paper_2507_20802_gb300 import aqs as A, synthetic as syn
    torch.cuda.set_device(0)
    x, t, H = syn.random_glass_start(N_ATOMS, 2, seed=0)
    g = A.System(x, t, H[None], [N_ATOMS], syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR,
                 precision=A.AQS_FP64)
    assert g.minimize(A.fire_params(max_iter=2_000_000))[0]["status"] == 0
    xq, Hq = g.positions(), g.box()
    g.close()
    rows = []
    for R in (P_CHAINS, 1):
        s = A.System(np.tile(xq, (R, 1)), np.tile(t, R), np.tile(Hq[None], (R, 1, 1)),
                     [N_ATOMS] * R, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR,
                     precision=A.AQS_MIXED)
        s.shear(np.arange(R) * K_FINE * DGAMMA)
        s.minimize()
        s.shear(np.full(R, DGAMMA))
        if R == P_CHAINS:
            occ = {m: {c: s.max_active_clusters(c, m) for c in range(1, 17)}
                   for m in (-1, 0, 1, 2, 3)}
            rows.append({"max_active_clusters_by_staging_and_C": occ})
        for gb in (False, True):
            s.set_grid_barrier(gb)
            for tpa in ((1, 2, 0) if not gb else (1,)):
                s.set_threads_per_atom(tpa)
                C, mode, msC, msM = s.autotune(iters=args.tune_iters)
                rows.append({"replicas": R, "grid_barrier": gb,
                             "threads_per_atom": {1: "1", 2: "2", 0: "tuned"}[tpa],
                             "chosen_threads_per_atom": s.threads_per_atom(), "best_C": C,
                             "staging": mode,
                             "us_per_iter_by_C": {c: round(v * 1e3, 2) for c, v in msC.items()},
                             "us_per_iter_by_staging": {m: round(v * 1e3, 2)
                                                        for m, v in msM.items()}})
        s.close()
    print(json.dumps({"metric": "minimiser time per FIRE iteration by launch configuration",
                      "unit": "us", "config": CONFIG, "iters_per_candidate": args.tune_iters,
                      "rows": rows}), flush=True)


def quench_3d(A, syn, n, seed, max_iter):
    """The 3D glass of the cfg3 workload: seeded random start, mixed-precision
    GPU FIRE quench (status and iterations returned; not converged when the
    budget runs out)."""
    x, t, H = syn.random_glass_start(n, 3, seed=seed)
    s = A.System(x, t, H[None], [n], syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR,
                 precision=A.AQS_MIXED)
    q = s.minimize(A.fire_params(max_iter=max_iter), check_status=False)[0]
    xq, Hq = s.positions(), s.box()
    s.close()
    return xq, t, Hq, q


def run_cfg3(args):
    """Algorithm 1 in 3D (80:20 binary LJ glass, N = 65536, density 1.2): P = 32
    chains of K = 20 fine steps of dgamma = 5e-5, every step converged to
    |F|max < 1e-10 (FP64 test), mixed precision; `steps` passes after
    `warmup` passes, from the quenched glass.  value = accepted fine steps /
    s (device time).  The plain FP64 sequential GPU AQS on the same glass
    (same kernels in FP64 mode, one replica) runs `baseline_steps` steps
    from the r_star reached."""
    import torch
    from paper_2507_20802_gb300 import aqs as A, synthetic as syn
    torch.cuda.set_device(0)
    n, P, K, dg = 65536, 32, 20, 5e-5
    t0 = time.perf_counter()
    xq, t, Hq, q = quench_3d(A, syn, n, 0, args.quench_iters)
    quench_s = time.perf_counter() - t0
    assert q["status"] == 0, q
    s = A.System(xq, t, Hq[None], [n], syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR,
                 precision=A.AQS_MIXED)
    s.set_launch_budget(args.launch_budget)
    n_total = int(round(0.15 / dg))
    done = 0

    def one_pass():
        nonlocal done
        r = s.parallel_step(dg, K, P, max(1, n_total - done), max_iterations=1)
        done += r["accepted"]
        return r
    for _ in range(args.warmup):
        one_pass()
    A.aqs_reset_kernel_stats()
    A.aqs_set_kernel_timing(True)
    l0 = A.aqs_launch_count()
    acc, ms, rej, passes = 0, 0.0, 0, []
    with Clocks(0) as clk:
        for _ in range(args.steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = one_pass()
            e1.record()
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            acc += r["accepted"]
            rej += r["rejections"]
            passes.append({"accepted": int(r["accepted"]), "ms": e0.elapsed_time(e1),
                           "fire_iters_total": int(r["fire_iters_total"]),
                           "first_failed_chain": int(r["log_i"][r["log_eq"] == 0][0])
                           if np.any(r["log_eq"] == 0) else None})
    st = A.aqs_get_kernel_stats()
    A.aqs_set_kernel_timing(False)
    value = acc / (ms / 1e3)
    base = None
    if args.baseline_steps > 0:
        b = A.System(s.positions(), t, s.box()[None], [n], syn.LJ_SIGMA, syn.LJ_EPS,
                     syn.RC_FACTOR, precision=A.AQS_FP64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ob = b.run_sequential(dg, args.baseline_steps)
        e1.record()
        e1.synchronize()
        bs = e0.elapsed_time(e1) / 1e3
        base = {"value": args.baseline_steps / bs, "unit": UNIT, "steps": args.baseline_steps,
                "fire_iters_per_step": float(ob["iters"].mean()),
                "speedup_of_value": value / (args.baseline_steps / bs),
                "cluster_size": b.cluster_size()}
        b.close()
    kern_s = st["kernel_ms"] / 1e3
    algo_bytes = 4.0 * st["pairs32"] + 28.0 * n * st["evals32"]
    gbs = algo_bytes / kern_s / 1e9 if kern_s else 0.0
    peak = _peaks().get("hbm_gbs", 6800.0)
    config = {"workload": "3D binary LJ glass (80:20, rho=1.2), N=65536, Algorithm 1 with P=32 "
                          "chains of K=20 fine steps, dgamma=5e-5, FIRE to |F|max<1e-10, mixed "
                          "precision", "n_atoms": n, "P": P, "K": K, "dgamma": dg,
              "l2": "lists of the chains (~1 GB) exceed L2"}
    _line(METRIC + " (3D)", value, UNIT, args, ms / max(1, args.steps), config,
          {"gpu_launches": A.aqs_launch_count() - l0, "clocks": clk.summary(),
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                        "frac": gbs / peak, "traffic": None,
                        "note": "algorithmic bytes = 4 per list entry visited + 28 per atom per "
                                "FP32 evaluation, over all minimiser launches of the passes"},
           "fp64_sequential_gpu_baseline": base,
           "detail": {"accepted_steps": acc, "rejections": rej, "passes": passes,
                      "quench_iters": q["iters"], "quench_s": quench_s,
                      "fire_iters_per_step": float(np.mean([p["fire_iters_total"] for p in passes]))
                      / max(1, acc / max(1, len(passes))),
                      "fp32_evals": st["evals32"], "fp64_evals": st["evals64"]}})


def force_3d_line(A, syn, quench_iters, replicas, iters):
    """Force-kernel bandwidth on the 3D workload for the default line: the
    cfg3 glass (partially quenched within `quench_iters`), `replicas` copies at
    the level-II fine steps, `iters` FIRE iterations each, timed by CUDA
    events in the library."""
    n, dg = 65536, 5e-5
    xq, t, Hq, q = quench_3d(A, syn, n, 0, quench_iters)
    b = A.System(np.tile(xq, (replicas, 1)), np.tile(t, replicas),
                 np.tile(Hq[None], (replicas, 1, 1)), [n] * replicas, syn.LJ_SIGMA, syn.LJ_EPS,
                 syn.RC_FACTOR, precision=A.AQS_MIXED)
    b.shear((np.arange(replicas) + 1) * dg)
    b.minimize(A.fire_params(max_iter=50), check_status=False)
    A.aqs_reset_kernel_stats()
    A.aqs_set_kernel_timing(True)
    b.minimize(A.fire_params(max_iter=iters), check_status=False)
    st = A.aqs_get_kernel_stats()
    A.aqs_set_kernel_timing(False)
    b.close()
    kern_s = st["kernel_ms"] / 1e3
    algo_bytes = 4.0 * st["pairs32"] + 28.0 * n * st["evals32"]
    gbs = algo_bytes / kern_s / 1e9 if kern_s else 0.0
    peak = _peaks().get("hbm_gbs", 6800.0)
    return {"kernel": "k_minimize<3,mixed> (lean launch)", "bound": "hbm", "achieved": gbs,
            "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "workload": "3D glass N=65536 (quench budget %d iterations, fmax %.2g), %d replicas "
                        "at fine steps of 5e-5, %d FIRE iterations each"
                        % (quench_iters, q["fmax"], replicas, iters),
            "algorithmic_bytes": "4 per list entry visited + 28 per atom per FP32 evaluation",
            "kernel_ms": st["kernel_ms"], "fp32_evals": st["evals32"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=20.0,
                    help="host-core budget of the oracle CPU baseline (whole steps)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--baseline-steps", type=int, default=20)
    ap.add_argument("--workload", choices=["cfg1", "batch64", "glass3d", "cfg3", "warm",
                                           "warm-eval", "oracle-threads", "sweep", "tune-table"],
                    default="cfg1")
    ap.add_argument("--tune-iters", type=int, default=500)
    ap.add_argument("--sweep-seeds", type=int, default=4)
    ap.add_argument("--sweep-P", type=int, nargs="+", default=[4, 8, 16, 32])
    ap.add_argument("--sweep-K", type=int, nargs="+", default=[1, 2, 6, 10, 14, 16])
    ap.add_argument("--no-force3d", action="store_true",
                    help="skip the 3D force-kernel bandwidth figure of the default line")
    ap.add_argument("--oracle-steps", type=int, default=60)
    ap.add_argument("--oracle-P", type=int, nargs="+", default=[4, 8, 16])
    ap.add_argument("--oracle-K", type=int, nargs="+", default=[1, 10])
    ap.add_argument("--k-max", type=int, default=0,
                    help="> K: dynamic K up to this chain length (default: fixed K = 10)")
    ap.add_argument("--seeds", type=int, default=0,
                    help="> 0: Metric 1 over glasses of seeds 0..n-1 (mean and std)")
    ap.add_argument("--launch-budget", type=int, default=2048,
                    help="FIRE iterations per persistent launch")
    ap.add_argument("--grid-barrier", action="store_true",
                    help="the chains in one cooperative launch with global-memory barriers")
    ap.add_argument("--autotune", type=int, default=300,
                    help="FIRE iterations per autotuner candidate (0: size rule only)")
    ap.add_argument("--quench-iters", type=int, default=400000)
    ap.add_argument("--iters3d", type=int, default=2000)
    ap.add_argument("--warm-train-iters", type=int, default=600)
    ap.add_argument("--replicas3d", type=int, default=32)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.seeds > 0:
        return run_seeds(args) or 0
    if args.workload == "batch64":
        return run_batch64(args) or 0
    if args.workload == "warm":
        return run_warm(args) or 0
    if args.workload == "warm-eval":
        return run_warm_eval(args) or 0
    if args.workload == "glass3d":
        return run_glass3d(args) or 0
    if args.workload == "oracle-threads":
        return run_oracle_threads(args) or 0
    if args.workload == "cfg3":
        return run_cfg3(args) or 0
    if args.workload == "sweep":
        return run_sweep(args) or 0
    if args.workload == "tune-table":
        return run_tune_table(args) or 0

    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2507_20802_gb300 import aqs as A, synthetic as syn

    # ---------------- set-up (untimed): seeded start, quench on the GPU
    # the glass is the FP64 quench of the seeded start, so that it does not
    # depend on how the mixed-precision path rounds
    x, t, H = syn.random_glass_start(N_ATOMS, 2, seed=rank)
    g = A.System(x, t, H[None], [N_ATOMS], syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR,
                 precision=A.AQS_FP64)
    q = g.minimize(A.fire_params(max_iter=2_000_000))[0]
    assert q["status"] == 0, q
    xq, Hq = g.positions(), g.box()
    g.close()
    s = A.System(xq, t, Hq[None], [N_ATOMS], syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR,
                 precision=A.AQS_MIXED)
    if args.grid_barrier:
        s.set_grid_barrier(True)
    if args.autotune > 0:
        # the chains tune cluster size and staging during the first (untimed)
        # warm-up pass
        s.set_autotune(args.autotune)
    s.set_launch_budget(args.launch_budget)
    fire = A.fire_params()
    n_total = int(round(GAMMA_END / DGAMMA))
    done = 0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    k_cur = [K_FINE]  # chain length of the next pass (changes only with --k-max)

    def one_pass():
        nonlocal done
        remaining = n_total - done if n_total > done else P_CHAINS * K_FINE
        torch.cuda.nvtx.range_push("aqs_pass")  # lets a profiler select the passes
        r = s.parallel_step(DGAMMA, k_cur[0], P_CHAINS, remaining, fire=fire, max_iterations=1,
                            K_max=args.k_max)
        k_cur[0] = r["K_next"]
        torch.cuda.nvtx.range_pop()
        done += r["accepted"]
        return r

    for _ in range(args.warmup):
        one_pass()

    # ---------------- timed passes (device time)
    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize()

    A.aqs_reset_kernel_stats()
    A.aqs_set_kernel_timing(True)
    launches0 = A.aqs_launch_count()
    gpu_index = int((os.environ.get("CUDA_VISIBLE_DEVICES") or str(local)).split(",")[0]) \
        if (os.environ.get("CUDA_VISIBLE_DEVICES") or "").split(",")[0].isdigit() else local
    accepted, dev_ms, wall, iters, rej, stopped = 0, 0.0, 0.0, [], 0, 0
    # r_star at four evenly spaced passes of the timed window: the FP64
    # sequential baseline starts from these states (read back between passes,
    # outside the device-timed region)
    snap_at = sorted({int(k * args.steps / 4) for k in range(4)})
    snaps = []
    barrier()
    with Clocks(gpu_index) as clk:
        for ip in range(args.steps):
            if rank == 0 and not args.no_baseline and ip in snap_at:
                snaps.append((s.positions(), s.box()))
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            w0 = time.perf_counter()
            e0.record()
            r = one_pass()
            e1.record()
            e1.synchronize()
            wall += time.perf_counter() - w0
            dev_ms += e0.elapsed_time(e1)
            accepted += r["accepted"]
            rej += r["rejections"]
            stopped += r["chains_stopped"]
            iters.extend(r["iters"].tolist())
    barrier()
    gpu_launches = A.aqs_launch_count() - launches0
    A.aqs_set_kernel_timing(False)
    st = A.aqs_get_kernel_stats()
    clocks = clk.summary()

    total_steps, secs = combine_ranks(dev_ms / 1e3, accepted, "cuda")
    value = total_steps / secs

    # ---------------- end to end through the C ABI with host buffers
    n_e2e = max(1, args.e2e_steps)
    pin = torch.empty((N_ATOMS, 2), dtype=torch.float64).pin_memory()
    A.aqs_get_positions(s.h, 0, pin.numpy())
    e2e_steps, e2e_wall = 0, 0.0
    h2d = d2h = 0
    for _ in range(n_e2e):
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        A.aqs_set_positions(s.h, 0, pin.numpy())           # host -> device
        r = one_pass()                                      # the pass (host result arrays)
        A.aqs_get_positions(s.h, 0, pin.numpy())           # device -> host
        torch.cuda.synchronize()
        e2e_wall += time.perf_counter() - w0
        e2e_steps += r["accepted"]
        h2d = pin.numel() * 8
        d2h = pin.numel() * 8 + r["accepted"] * (8 + 8 + 8 + 8 + 1)
    e2e_value = e2e_steps * ws / e2e_wall

    # ---------------- roofline of the persistent minimiser kernel
    kern_s = st["kernel_ms"] / 1e3
    flop32 = st["pairs32"] * FLOP32_PER_PAIR
    flop64 = st["pairs64"] * FLOP64_PER_PAIR
    achieved = flop32 / kern_s / 1e12 if kern_s > 0 else 0.0
    peak32, n_sm, mhz = fp32_peak_tflops()
    chain_mode = "grid_barrier" if s.grid_barrier(chains=True) == 1 else "cluster"
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak32,
                "unit": "TFLOP/s", "frac": achieved / peak32,
                "flop_per_list_entry": FLOP32_PER_PAIR,
                "kernel_flop_per_visit": KERNEL_FLOP32_PER_VISIT,
                "traffic": TRAFFIC_CFG1_PER_LAUNCH[chain_mode],
                "traffic_note": "DRAM bytes of one captured level-II chain launch (the L2-resident "
                                "working set, read once per launch), %s kernel" % chain_mode,
                "kernel": "k_minimize<2,mixed>",
                "barrier_mode": chain_mode,
                "kernel_share_of_step": kern_s / secs if secs > 0 else None,
                "fp64_tflops": flop64 / kern_s / 1e12 if kern_s > 0 else 0.0,
                "launches": st["launches"], "avg_launch_ms": st["kernel_ms"] / max(1, st["launches"]),
                "pair_visits_fp32": st["pairs32"], "pair_visits_fp64": st["pairs64"],
                "peak_note": "FP32 peak derived: %d SMs (queried) x 128 lanes x 2 x %.0f MHz"
                             % (n_sm, mhz)}

    # ---------------- plain FP64 sequential GPU AQS on the same glass (the
    # denominator of the speed-up target): same kernels in FP64 mode, one
    # replica, no batching, no warm start; baseline_steps steps split over the
    # four r_star states taken across the timed window
    base = None
    if rank == 0 and not args.no_baseline and snaps:
        per = max(1, -(-args.baseline_steps // len(snaps)))
        bsec, bsteps, bits, csize = 0.0, 0, 0, 0
        for xs_, Hs_ in snaps:
            b = A.System(xs_, t, Hs_[None], [N_ATOMS], syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR,
                         precision=A.AQS_FP64)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ob = b.run_sequential(DGAMMA, per)
            e1.record()
            e1.synchronize()
            bsec += e0.elapsed_time(e1) / 1e3
            bsteps += per
            bits += int(ob["iters"].sum())
            csize = b.cluster_size()
            b.close()
        # the same comparison at equal work: the FP64 time per iteration times
        # the FIRE iterations per accepted step of the timed region
        t_it64 = bsec / max(1, bits)
        mean_acc = float(np.mean(iters)) if iters else float("nan")
        same = 1.0 / (mean_acc * t_it64)
        bval = bsteps / bsec
        base = {"value": bval, "unit": UNIT, "steps": bsteps,
                "sample": "%d steps from each of %d r_star states taken at timed passes %s"
                          % (per, len(snaps), snap_at),
                "fire_iters_per_step": bits / bsteps,
                "us_per_fp64_iteration": 1e6 * t_it64,
                "same_steps_value": same,
                "same_steps_note": "FP64 time per iteration x FIRE iterations per accepted step "
                                   "of the timed region",
                "cluster_size": csize,
                "occupancy_note": "one replica of %d atoms fills one cluster of %d CTAs, i.e. "
                                  "%d of %d SMs: sequential AQS cannot use the rest"
                                  % (N_ATOMS, csize, csize, n_sm),
                "speedup_of_value": value / bval,
                "speedup_same_steps": value / same}

    # ---------------- the force kernel's HBM bandwidth on the 3D workload
    force3d = None
    if rank == 0 and not args.no_force3d:
        force3d = force_3d_line(A, syn, 20000, 32, 500)

    # ---------------- CPU baseline (oracle, rank 0, N = 1 only)
    cpu = None
    mean_iters = float(np.mean(iters)) if iters else float("nan")
    if rank == 0 and ws == 1 and not args.no_cpu:
        nst, dt, oit = oracle_steps(budget_s=args.cpu_seconds)
        cpu = {"value": nst / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "%d complete AQS steps (dgamma=1e-4, FIRE to |F|max<1e-10, %d FIRE "
                         "iterations per step) of the FP64 all-pairs oracle on the N=256 glass "
                         "in %.1f s on one host core; an N=4096 step of this workload costs "
                         "about 256x more per iteration in the O(N^2) oracle" % (nst, oit / nst, dt),
               "host": host_desc()}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": dev_ms / max(1, args.steps), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic", "config": CONFIG,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": int(gpu_launches), "clocks": clocks, "roofline": roofline,
                "cpu_baseline": cpu,
                "fp64_sequential_gpu_baseline": base,
                "force_kernel_3d": force3d,
                "detail": {"accepted_steps": int(total_steps), "rejections": rej,
                           "chains_stopped_early": stopped, "autotune_iters": args.autotune,
                           "launch_budget": args.launch_budget, "k_max": args.k_max,
                           "wall_s": wall, "fire_iters_per_step": mean_iters,
                           "fp32_evals": st["evals32"], "fp64_evals": st["evals64"],
                           "rebuilds_in_kernel": st["rebuilds"],
                           "glass_quench_iters": q["iters"], "glass_quench": "FP64"}}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
