"""Pins of the oracle's general deformation histories (pure, or pull-push,
shear of Sec. 2.2; cyclic protocols named in Sec. 5), against facts fixed by
the geometry and by the simple-shear path already pinned:

* a history of simple-shear matrices reproduces orc_aqs bit for bit, and
  Algorithm 1 under it reproduces orc_parallel;
* the upper-triangular frame undoes a rigid rotation exactly, and a
  pull-push increment keeps every separation vector's length |F d|;
* volume after k pull-push steps is V0 det(F)^k;
* a Bravais lattice stays force-free under any affine map: zero FIRE
  iterations and zero non-affine displacement at every step;
* a small elastic cycle (forward, then the inverse increments) returns the
  lattice cell and a glass's configuration to where they started;
* Algorithm 1 under a pull-push history reproduces the sequential history
  step by step, with rejections.
"""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def setup(orc, syn):
    pot = orc.make_potential(2, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    fp = orc.make_fire(**syn.FIRE)
    x, t, H = syn.random_glass_start(64, 2, seed=23)
    q = orc.fire(pot, fp, x, t, H)
    assert q["status"] == 0
    return pot, fp, q["x"], t, H


def pull_push(a, b, n):
    return np.tile(np.array([[1.0, a], [b, 1.0]]), (n, 1, 1))


def mi_disp(a, b, H):
    d = np.asarray(a, float) - np.asarray(b, float)
    for c in reversed(range(H.shape[0])):
        d -= np.round(d[:, c] / H[c, c])[:, None] * H[:, c][None, :]
    d -= d.mean(axis=0)
    return float(np.sqrt((d * d).sum(axis=1)).max())


def test_simple_shear_history_is_orc_aqs(orc, setup):
    pot, fp, x, t, H = setup
    dg, n = 2e-3, 6
    a = orc.aqs(pot, fp, x, t, H, dg, n)
    F = np.tile(np.array([[1.0, dg], [0.0, 1.0]]), (n, 1, 1))
    b = orc.aqs_history(pot, fp, x, t, H, F)
    for k in ("x", "H", "E", "tau", "iters", "D"):
        assert np.array_equal(a[k], b[k]), k


def test_triangularise_undoes_a_rigid_rotation(orc, syn):
    x, t, H = syn.random_glass_start(50, 2, seed=4)
    H = H.copy()
    H[0, 1] = 0.3 * H[1, 1]
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    xr, Hr = orc.triangularise(x @ R.T, R @ H)
    np.testing.assert_allclose(Hr, H, rtol=0, atol=1e-13)
    np.testing.assert_allclose(xr, x, rtol=0, atol=1e-12)


def test_pull_push_step_keeps_lengths_and_scales_volume(orc, syn):
    x, t, H = syn.random_glass_start(40, 2, seed=6)
    a, b = 0.02, 0.015
    F = np.array([[1.0, a], [b, 1.0]])
    x1, H1, L1 = orc.deform(x, H, F)
    assert H1[1, 0] == 0.0 and H1[0, 0] > 0 and H1[1, 1] > 0
    np.testing.assert_allclose(L1, F @ H, rtol=1e-15)  # the laboratory cell
    # every separation vector (no images) keeps its length F d
    i, j = np.triu_indices(len(x), 1)
    np.testing.assert_allclose(np.linalg.norm(x1[i] - x1[j], axis=1),
                               np.linalg.norm((x[i] - x[j]) @ F.T, axis=1), rtol=1e-13)
    # the cell's columns keep their lengths and their angle
    np.testing.assert_allclose(np.linalg.norm(H1, axis=0), np.linalg.norm(F @ H, axis=0),
                               rtol=1e-13)
    xk, Hk, Lk = x, H, H
    for _ in range(7):
        xk, Hk, Lk = orc.deform(xk, Hk, F, Lk)
    assert orc.volume(Hk) == pytest.approx(orc.volume(H) * (1 - a * b) ** 7, rel=1e-13)


def test_lattice_is_force_free_under_pull_push(orc, syn):
    pot = orc.make_potential(2, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    fp = orc.make_fire(**syn.FIRE)
    x, t, H = syn.triangular_lattice(8, 8)
    r = orc.aqs_history(pot, fp, x, t, H, pull_push(2e-3, 1.5e-3, 8))
    assert r["status"] == 0
    assert np.all(r["iters"] == 0) and np.all(r["D"] < 1e-12)


def test_elastic_cycle_returns(orc, syn, setup):
    """Forward pull-push increments, then their inverses in reverse order:
    the lattice cell comes back to rounding, and a glass driven elastically
    returns to its starting minimum."""
    a, b, n = 4e-4, 3e-4, 5
    F = np.array([[1.0, a], [b, 1.0]])
    Fi = np.linalg.inv(F)
    hist = np.concatenate([np.tile(F, (n, 1, 1)), np.tile(Fi, (n, 1, 1))])
    pot = orc.make_potential(2, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    fp = orc.make_fire(**syn.FIRE)
    xl, tl, Hl = syn.triangular_lattice(8, 8)
    r = orc.aqs_history(pot, fp, xl, tl, Hl, hist)
    np.testing.assert_allclose(r["H"], Hl, atol=1e-12)
    _, _, x, t, H = setup
    r = orc.aqs_history(setup[0], setup[1], x, t, H, hist)
    assert r["status"] == 0 and np.all(r["D"] < 1e-2)
    np.testing.assert_allclose(r["H"], H, atol=1e-12)
    assert mi_disp(r["x"], x, H) < 1e-6


def test_parallel_under_pull_push_equals_sequential(orc, setup):
    pot, fp, x, t, H = setup
    n, K, P = 24, 3, 4
    hist = pull_push(4e-3, 3e-3, n)
    seq = orc.aqs_history(pot, fp, x, t, H, hist)
    par = orc.parallel(pot, fp, x, t, H, 0.0, K, P, n, eq_tol=1e-6, F_steps=hist)
    assert seq["status"] == 0 and par["status"] == 0
    np.testing.assert_allclose(par["E"], seq["E"], rtol=1e-9)
    assert np.array_equal(par["D"] > 1e-2, seq["D"] > 1e-2)
    assert mi_disp(par["x"], seq["x"], seq["H"]) < 1e-6
    np.testing.assert_allclose(par["H"], seq["H"], rtol=1e-13)
    assert np.any(par["log_eq"] == 0), "history chosen to show a rejection"
    m = par["log_m"]
    assert np.all((m < 1e-8) | (m > 1e-4))
