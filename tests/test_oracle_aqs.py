"""Pins of the oracle's AQS protocol (Eq. 12) and of Algorithm 1 (Sec. 3)
against the properties the paper proves or states (no GPU):

* the decision rule reproduces the worked 15-step, 3-thread example (Sec. 3.5);
* the parallel trajectory equals the sequential one at every accepted step
  (Sec. 3.6, Sec. 4: "all final configurations were equal");
* finite termination within ceil(N_steps / K) passes, and the best case of
  ceil(N_steps / (P K)) passes when every prediction is right (Sec. 3.7);
* repeating a run gives exactly the same outcome (Sec. 3.6), with or without
  threads.
"""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def small_glass(orc, syn):
    pot = orc.make_potential(2, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    fp = orc.make_fire(**syn.FIRE)
    x, t, H = syn.random_glass_start(64, 2, seed=23)
    q = orc.fire(pot, fp, x, t, H)
    assert q["status"] == 0
    return pot, fp, q["x"], t, H


def test_decision_rule_worked_example(orc):
    """P = 3 threads, K = 5, 15 steps (Fig. 4 / Sec. 3.5)."""
    K = [5, 5, 5]
    assert orc.alg1_decide(K, [0, 1, 1]) == (15, -1)   # both checks pass: accept all
    assert orc.alg1_decide(K, [0, 0, 1]) == (5, 1)     # r_5 != r_5|r^c_5: restart from r_5
    assert orc.alg1_decide(K, [0, 1, 0]) == (10, 2)    # second check fails: keep up to r_10
    assert orc.alg1_decide([5], [0]) == (5, -1)        # single chain (last window)
    assert orc.alg1_decide([4, 4, 2], [0, 1, 1]) == (10, -1)  # shortened last chain


def test_parallel_equals_sequential_with_rejections(orc, small_glass):
    pot, fp, x0, t, H = small_glass
    dg, K, P, n = 5e-3, 3, 4, 30  # the paper's increment 1/200 (Sec. 4)
    seq = orc.aqs(pot, fp, x0, t, H, dg, n)
    par = orc.parallel(pot, fp, x0, t, H, dg, K, P, n, eq_tol=1e-6)
    assert seq["status"] == 0 and par["status"] == 0
    # equal minima at every accepted step: same energy, same final state
    np.testing.assert_allclose(par["E"], seq["E"], rtol=1e-9)
    np.testing.assert_allclose(par["tau"], seq["tau"], rtol=1e-6, atol=1e-8)
    assert orc.max_rel_disp(par["x"], seq["x"], seq["H"]) < 1e-6
    np.testing.assert_allclose(par["H"], seq["H"], rtol=1e-13)
    # the same plastic events (non-affine jump larger than 0.01 sigma)
    assert np.array_equal(par["D"] > 1e-2, seq["D"] > 1e-2)
    # termination bound and at least one rejection at this large K P dgamma
    assert par["iterations"] <= math.ceil(n / K)
    assert np.any(par["log_eq"] == 0), "workload chosen to show a rejection"
    # every logged test value sits far from the threshold on either side
    m = par["log_m"]
    assert np.all((m < 1e-8) | (m > 1e-4))


def test_parallel_best_case_on_lattice(orc, syn):
    pot = orc.make_potential(2, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    fp = orc.make_fire(**syn.FIRE)
    x, t, H = syn.triangular_lattice(8, 8)
    K, P, n = 2, 3, 13
    par = orc.parallel(pot, fp, x, t, H, 1e-3, K, P, n, eq_tol=1e-6)
    assert par["status"] == 0
    assert par["iterations"] == math.ceil(n / (P * K))
    assert np.all(par["log_eq"] == 1)
    assert par["fire_iters_total"] == 0
    assert par["H"][0, 1] == pytest.approx(n * 1e-3 * H[1, 1], rel=1e-12)


def test_parallel_is_deterministic_and_thread_independent(orc, small_glass):
    pot, fp, x0, t, H = small_glass
    a = orc.parallel(pot, fp, x0, t, H, 2e-3, 3, 4, 12, eq_tol=1e-6, n_threads=1)
    b = orc.parallel(pot, fp, x0, t, H, 2e-3, 3, 4, 12, eq_tol=1e-6, n_threads=4)
    for k in ["x", "E", "tau", "iters", "D", "log_eq", "log_m"]:
        assert np.array_equal(a[k], b[k]), k


def test_sequential_aqs_elastic_step_is_small(orc, small_glass):
    pot, fp, x0, t, H = small_glass
    r = orc.aqs(pot, fp, x0, t, H, 1e-5, 2)
    assert r["status"] == 0
    # non-affine response is linear in the increment for an elastic step
    r2 = orc.aqs(pot, fp, x0, t, H, 2e-5, 1)
    assert r2["D"][0] == pytest.approx(2 * r["D"][0], rel=0.05)
