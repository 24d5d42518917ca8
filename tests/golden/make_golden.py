"""Writes the stored expected values under tests/golden/ -- calls only the
oracle (and the seeded input generators).

Each file is an .npz of FP64/int arrays:

* glass_<d>d_n<N>_s<seed>.npz -- seeded random start (uniform positions,
  exact species counts) FIRE-quenched by the oracle to |F|max < 1e-10:
  the inherent structure every trajectory test starts from.
* aqs_2d_n256_s0.npz -- sequential AQS (Eq. 12) from glass_2d_n256_s0,
  simple shear dgamma = 1e-4, 200 steps: per-step energy, stress, FIRE
  iterations, non-affine displacement D_k, final positions and cell.
* par_2d_n256_s<seed>.npz -- Algorithm 1 from that glass at the paper's
  increment dgamma = 1/200 (Sec. 4) with K = 3, P = 4, 30 steps: per-step
  observables, decision log, final positions.
* pardynk_2d_n256_s0.npz -- the same Algorithm-1 run with dynamic K
  (K_max = 12): chain length per pass, decisions, observables.
* par_2d_n1024_s0.npz -- Algorithm 1 at the benchmark's shape, reduced:
  the N = 1024 glass, dgamma = 1e-4, K = 10, P = 4, 400 steps (to
  gamma = 0.04): per-step observables, decision log, final positions.
* aqs_3d_n2048_s0.npz -- ten sequential AQS steps of the 3D glass,
  dgamma = 5e-5.
* hist_2d_n256_s0.npz -- AQS under a deformation history on the N = 256
  glass: 40 pull-push increments F = [[1, 2e-4], [1.5e-4, 1]] (Sec. 2.2),
  then 40 increments of F^-1 (a strain cycle, Sec. 5): the history, per-step
  observables, final positions, stored and laboratory cells.
* parhist_2d_n256_s0.npz -- Algorithm 1 under the pull-push history
  F = [[1, 4e-3], [3e-3, 1]], K = 3, P = 4, 24 steps: decision log and
  per-step observables.
* glass_sl_n400_s0.npz, aqs_sl_n400_s0.npz -- the paper's S/L glass (N = 400,
  density 1, Sec. 2.2) quenched by the oracle, and 20 sequential AQS steps
  of the paper's increment dgamma = 1/200 (Sec. 4).
* aqs_sl_n400_s0_g1.npz -- the paper's whole protocol on that glass: 200
  steps of dgamma = 1/200 to gamma = 1 (Sec. 2.2, Fig. 2b).

Usage: python tests/golden/make_golden.py [name ...]   (default: all)
"""
import os
import sys
import time
from multiprocessing import get_context

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2507_20802_gb300 import synthetic as syn  # noqa: E402


def _pot(dim):
    return oracle.make_potential(dim, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)


def _fire():
    return oracle.make_fire(**syn.FIRE)


def glass(dim, n, seed):
    name = f"glass_{dim}d_n{n}_s{seed}.npz"
    path = os.path.join(HERE, name)
    if os.path.exists(path):
        return dict(np.load(path))
    x, t, H = syn.random_glass_start(n, dim, seed)
    r = oracle.fire(_pot(dim), _fire(), x, t, H)
    assert r["status"] == 0, r["status"]
    out = dict(x=r["x"], types=t, H=H, E=r["E"], iters=r["iters"], fmax=r["fmax"])
    np.savez(path, **out)
    return out


def job_glass2d256():
    glass(2, 256, 0)


def job_glass2d1024():
    glass(2, 1024, 0)


def job_aqs2d256():
    g = glass(2, 256, 0)
    r = oracle.aqs(_pot(2), _fire(), g["x"], g["types"], g["H"], 1e-4, 200)
    assert r["status"] == 0
    np.savez(os.path.join(HERE, "aqs_2d_n256_s0.npz"), dgamma=1e-4, n_steps=200, **r)


def job_par2d256():
    g = glass(2, 256, 0)
    dg, K, P, n = 5e-3, 3, 4, 30
    r = oracle.parallel(_pot(2), _fire(), g["x"], g["types"], g["H"], dg, K, P, n, eq_tol=1e-6,
                        n_threads=4)
    assert r["status"] == 0
    np.savez(os.path.join(HERE, "par_2d_n256_s0.npz"), dgamma=dg, K=K, P=P, n_steps=n,
             eq_tol=1e-6, **r)


def job_pardynk2d256():
    g = glass(2, 256, 0)
    dg, K, P, n, K_max = 5e-3, 3, 4, 30, 12
    r = oracle.parallel(_pot(2), _fire(), g["x"], g["types"], g["H"], dg, K, P, n, eq_tol=1e-6,
                        n_threads=4, K_max=K_max)
    assert r["status"] == 0
    np.savez(os.path.join(HERE, "pardynk_2d_n256_s0.npz"), dgamma=dg, K=K, P=P, n_steps=n,
             K_max=K_max, eq_tol=1e-6, **r)


def job_par2d1024():
    g = glass(2, 1024, 0)
    dg, K, P, n = 1e-4, 10, 4, 400
    r = oracle.parallel(_pot(2), _fire(), g["x"], g["types"], g["H"], dg, K, P, n, eq_tol=1e-6,
                        n_threads=4)
    assert r["status"] == 0
    np.savez(os.path.join(HERE, "par_2d_n1024_s0.npz"), dgamma=dg, K=K, P=P, n_steps=n,
             eq_tol=1e-6, **r)


def job_aqs3d2048():
    g = glass(3, 2048, 0)
    r = oracle.aqs(_pot(3), _fire(), g["x"], g["types"], g["H"], 5e-5, 10)
    assert r["status"] == 0
    np.savez(os.path.join(HERE, "aqs_3d_n2048_s0.npz"), dgamma=5e-5, n_steps=10, **r)


def job_hist2d256():
    g = glass(2, 256, 0)
    F = np.array([[1.0, 2e-4], [1.5e-4, 1.0]])
    hist = np.concatenate([np.tile(F, (40, 1, 1)), np.tile(np.linalg.inv(F), (40, 1, 1))])
    r = oracle.aqs_history(_pot(2), _fire(), g["x"], g["types"], g["H"], hist)
    assert r["status"] == 0
    np.savez(os.path.join(HERE, "hist_2d_n256_s0.npz"), F_steps=hist, n_steps=len(hist), **r)


def job_parhist2d256():
    g = glass(2, 256, 0)
    K, P, n = 3, 4, 24
    hist = np.tile(np.array([[1.0, 4e-3], [3e-3, 1.0]]), (n, 1, 1))
    r = oracle.parallel(_pot(2), _fire(), g["x"], g["types"], g["H"], 0.0, K, P, n, eq_tol=1e-6,
                        n_threads=4, F_steps=hist)
    assert r["status"] == 0
    np.savez(os.path.join(HERE, "parhist_2d_n256_s0.npz"), F_steps=hist, K=K, P=P, n_steps=n,
             eq_tol=1e-6, **r)


def _pot_sl():
    return oracle.make_potential(2, syn.SL_SIGMA, syn.SL_EPS, syn.RC_FACTOR)


def glass_sl(n, seed):
    path = os.path.join(HERE, f"glass_sl_n{n}_s{seed}.npz")
    if os.path.exists(path):
        return dict(np.load(path))
    x, t, H = syn.random_glass_start(n, 2, seed, fraction_a=syn.SL_FRACTION_S,
                                     density=syn.SL_DENSITY)
    r = oracle.fire(_pot_sl(), _fire(), x, t, H)
    assert r["status"] == 0, r["status"]
    out = dict(x=r["x"], types=t, H=H, E=r["E"], iters=r["iters"], fmax=r["fmax"])
    np.savez(path, **out)
    return out


def job_aqssl400():
    g = glass_sl(400, 0)
    r = oracle.aqs(_pot_sl(), _fire(), g["x"], g["types"], g["H"], 1.0 / 200.0, 20)
    assert r["status"] == 0
    np.savez(os.path.join(HERE, "aqs_sl_n400_s0.npz"), dgamma=1.0 / 200.0, n_steps=20, **r)


def job_aqssl400full():
    g = glass_sl(400, 0)
    r = oracle.aqs(_pot_sl(), _fire(), g["x"], g["types"], g["H"], 1.0 / 200.0, 200)
    assert r["status"] == 0
    np.savez(os.path.join(HERE, "aqs_sl_n400_s0_g1.npz"), dgamma=1.0 / 200.0, n_steps=200, **r)


JOBS = {k[4:]: v for k, v in globals().items() if k.startswith("job_")}


def _run(name):
    t0 = time.time()
    JOBS[name]()
    return name, time.time() - t0


if __name__ == "__main__":
    oracle.build()
    names = sys.argv[1:] or list(JOBS)
    with get_context("spawn").Pool(min(len(names), os.cpu_count() or 1)) as pool:
        for name, dt in pool.imap_unordered(_run, names):
            print(f"{name}: {dt:.1f} s", flush=True)
