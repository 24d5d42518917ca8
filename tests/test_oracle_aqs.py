"""Pins of the oracle's AQS protocol (Eq. 12) and of Algorithm 1 (Sec. 3)
against the properties the paper proves or states (no GPU):

* the decision rule reproduces the worked 15-step, 3-thread example (Sec. 3.5);
* the parallel trajectory equals the sequential one at every accepted step
  (Sec. 3.6; the paper's runs in Sec. 4 ended in identical configurations);
* finite termination within ceil(N_steps / K) passes, and the best case of
  ceil(N_steps / (P K)) passes when every prediction is right (Sec. 3.7);
* a repeated run gives an identical result (Sec. 3.6), with or without
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


def _check_k_rule(par, K0, K_max, P):
    """The recorded chain length of every pass follows the dynamic-K rule."""
    Ks = list(par["K_pass"])
    assert Ks[0] == K0
    for p in range(1, len(Ks)):
        sel = par["log_iter"] == p - 1
        fails = par["log_i"][sel][par["log_eq"][sel] == 0]
        if len(fails) == 0:
            assert Ks[p] == min(K_max, 2 * Ks[p - 1]), (p, Ks)
        else:
            q = int(fails[0]) * Ks[p - 1]  # chains 0..i-1 accepted (none shortened here)
            assert Ks[p] == max(1, -(-q // P)), (p, Ks, q)


def test_dynamic_k_keeps_the_sequential_trajectory(orc, small_glass):
    """Any chain-length schedule reproduces sequential AQS (Algorithm 1 is
    exact); with rejections the schedule shrinks and grows by the rule."""
    pot, fp, x0, t, H = small_glass
    dg, K, P, n = 5e-3, 3, 4, 30
    seq = orc.aqs(pot, fp, x0, t, H, dg, n)
    par = orc.parallel(pot, fp, x0, t, H, dg, K, P, n, eq_tol=1e-6, K_max=12)
    assert par["status"] == 0
    np.testing.assert_allclose(par["E"], seq["E"], rtol=1e-9)
    assert orc.max_rel_disp(par["x"], seq["x"], seq["H"]) < 1e-6
    assert np.array_equal(par["D"] > 1e-2, seq["D"] > 1e-2)
    assert np.any(par["log_eq"] == 0)
    # all but the last pass are full windows, so the rule can be checked exactly
    full = dict(par)
    full["K_pass"] = par["K_pass"][:-1]
    _check_k_rule(full, K, 12, P)
    # K_max <= K is the fixed schedule
    fixed = orc.parallel(pot, fp, x0, t, H, dg, K, P, n, eq_tol=1e-6, K_max=K)
    ref = orc.parallel(pot, fp, x0, t, H, dg, K, P, n, eq_tol=1e-6)
    assert np.array_equal(fixed["E"], ref["E"]) and np.all(fixed["K_pass"] == K)


def test_dynamic_k_doubles_on_the_lattice(orc, syn):
    """No plastic events on the lattice: K doubles every pass up to K_max."""
    pot = orc.make_potential(2, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    fp = orc.make_fire(**syn.FIRE)
    x, t, H = syn.triangular_lattice(8, 8)
    par = orc.parallel(pot, fp, x, t, H, 1e-3, 1, 2, 40, eq_tol=1e-6, K_max=8)
    assert par["status"] == 0
    assert list(par["K_pass"]) == [1, 2, 4, 8, 8, 8][:len(par["K_pass"])]
    assert par["H"][0, 1] == pytest.approx(40 * 1e-3 * H[1, 1], rel=1e-12)


def test_lattice_steps_have_zero_nonaffine_displacement(orc, syn):
    """Every atom of the perfect triangular lattice is an inversion centre, so
    the sheared lattice is again a minimum: the minimiser does not move and
    D_k, measured against the affinely mapped previous minimum F r_{k-1}, is
    zero at every step.  Measured against r_{k-1} instead, D_k would be about
    dgamma L_y / 2 (7e-3 here)."""
    pot = orc.make_potential(2, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    fp = orc.make_fire(**syn.FIRE)
    x, t, H = syn.triangular_lattice(8, 8)
    r = orc.aqs(pot, fp, x, t, H, 2e-3, 10)
    assert r["status"] == 0
    assert np.all(r["iters"] == 0)
    assert np.all(r["D"] < 1e-12), r["D"]


def test_equality_test_uses_the_shared_strain_cell(orc, syn):
    """Incoming and outgoing minima of a test are compared at their common
    strain i K dgamma (Sec. 3.4), so the minimum image must use that cell.
    With chain ends wrapped into the cell, an atom that crossed the y face
    carries the tilt of that strain; in a later cell the image would be off by
    K dgamma L_y.  On the lattice every prediction is right (Sec. 3.7), with
    or without wrapping."""
    pot = orc.make_potential(2, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    fp = orc.make_fire(**syn.FIRE)
    x, t, H = syn.triangular_lattice(8, 8)
    x = x + np.array([0.0, 0.5 * H[1, 1]])  # half of the atoms outside the cell in y
    K, P, n = 2, 3, 13
    for wrap in (False, True):
        par = orc.parallel(pot, fp, x, t, H, 1e-3, K, P, n, eq_tol=1e-6, wrap_ends=wrap)
        assert par["status"] == 0
        assert np.all(par["log_eq"] == 1) and np.all(par["log_m"] < 1e-12), par["log_m"]
        assert par["iterations"] == math.ceil(n / (P * K))
    # the same comparison made directly: a wrapped copy is equal in its own
    # cell and unequal in the cell K steps later
    xa, Ha = orc.affine_shear(x, H, K * 1e-3)
    xw = orc.wrap(xa, Ha)
    assert orc.max_rel_disp(xw, xa, Ha) < 1e-12
    _, Hb = orc.affine_shear(xa, Ha, K * 1e-3)
    assert orc.max_rel_disp(xw, xa, Hb) > 1e-3


def test_wrapped_chain_ends_keep_decisions_on_a_glass(orc, small_glass):
    """Wrapping chain ends (positions are defined modulo the cell) changes no
    decision and no accepted step on a glass with rejections."""
    pot, fp, x0, t, H = small_glass
    x0 = x0 + np.array([0.3 * H[0, 0], 0.5 * H[1, 1]])
    dg, K, P, n = 5e-3, 3, 4, 30
    a = orc.parallel(pot, fp, x0, t, H, dg, K, P, n, eq_tol=1e-6)
    b = orc.parallel(pot, fp, x0, t, H, dg, K, P, n, eq_tol=1e-6, wrap_ends=True)
    assert a["status"] == 0 and b["status"] == 0
    assert np.any(a["log_eq"] == 0)
    assert np.array_equal(a["log_eq"], b["log_eq"]) and np.array_equal(a["log_i"], b["log_i"])
    np.testing.assert_allclose(b["E"], a["E"], rtol=1e-12)
    assert orc.max_rel_disp(a["x"], b["x"], a["H"]) < 1e-9


def test_wrap_moves_atoms_by_lattice_vectors_into_the_cell(orc, syn):
    """orc_wrap: fractional coordinates end in [0, 1) and every shift is an
    integer combination of the cell's columns."""
    H = np.array([[5.0, 1.7], [0.0, 4.0]])
    x = (syn.uniform(31, 200).reshape(100, 2) - 0.5) * 30.0
    w = orc.wrap(x, H)
    s = np.linalg.solve(H, w.T).T
    assert np.all(s >= -1e-12) and np.all(s < 1.0 + 1e-12)
    m = np.linalg.solve(H, (x - w).T).T
    np.testing.assert_allclose(m, np.round(m), atol=1e-9)
