"""Deformation histories on the GPU (pull-push shear of Sec. 2.2, a strain
cycle as named in Sec. 5) against the FP64 oracle's stored runs.

The library keeps every cell upper triangular and stores the configuration
in the Gram-Schmidt frame of the laboratory cell; the oracle does the same by
its own arithmetic, so stored positions, stored cells and frames are compared
directly.  Tolerances as for simple shear: E/N 1e-9 (FP64) / 1e-6 (mixed),
positions 1e-6 sigma, identical events and Algorithm-1 decisions."""
import ctypes as C

import numpy as np
import pytest

from conftest import load_golden

pytestmark = pytest.mark.gpu
EV_THR = 1e-2


@pytest.fixture(scope="module")
def A():
    from paper_2507_20802_gb300 import aqs
    aqs.lib()
    return aqs


@pytest.fixture(scope="module")
def glass256():
    return load_golden("glass_2d_n256_s0.npz")


def mi_disp(a, b, H):
    d = np.asarray(a, float) - np.asarray(b, float)
    for c in reversed(range(H.shape[0])):
        d -= np.round(d[:, c] / H[c, c])[:, None] * H[:, c][None, :]
    d -= d.mean(axis=0)
    return float(np.sqrt((d * d).sum(axis=1)).max())


def make(A, syn, g, prec):
    return A.System(g["x"], g["types"], g["H"][None], [len(g["x"])], syn.LJ_SIGMA, syn.LJ_EPS,
                    syn.RC_FACTOR, precision=prec)


def test_one_increment_matches_oracle_map(A, orc, syn, glass256):
    F = np.array([[1.0, 3e-3], [2e-3, 1.0]])
    s = make(A, syn, glass256, A.AQS_FP64)
    s.deform(F)
    xo, Ho, Lo = orc.deform(glass256["x"], glass256["H"], F)
    np.testing.assert_allclose(s.box(), Ho, rtol=0, atol=1e-13)
    np.testing.assert_allclose(s.frame() @ s.box(), Lo, rtol=0, atol=1e-13)
    assert mi_disp(s.positions(), xo, Ho) < 1e-12
    # forces of the deformed configuration equal the oracle's in the stored frame
    E, Fg, _ = s.energy_forces()
    pot = orc.make_potential(2, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    Eo, Fo, _ = orc.energy_forces(pot, xo, glass256["types"], Ho)
    assert E == pytest.approx(Eo, rel=1e-11)
    assert np.abs(Fg - Fo).max() < 1e-9
    s.close()


def test_simple_shear_history_equals_sequential(A, syn, glass256):
    gold = load_golden("aqs_2d_n256_s0.npz")
    n = 30
    F = np.tile(np.array([[1.0, float(gold["dgamma"])], [0.0, 1.0]]), (n, 1, 1))
    s = make(A, syn, glass256, A.AQS_FP64)
    out = s.run_history(F)
    np.testing.assert_allclose(out["E"][:, 0], gold["E"][:n], rtol=1e-9)
    assert np.array_equal(out["D"][:, 0] > EV_THR, gold["D"][:n] > EV_THR)
    assert np.array_equal(s.frame(), np.eye(2))
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pull_push_cycle_matches_golden(A, syn, glass256, prec):
    gold = load_golden("hist_2d_n256_s0.npz")
    P = A.AQS_FP64 if prec == "fp64" else A.AQS_MIXED
    s = make(A, syn, glass256, P)
    out = s.run_history(gold["F_steps"])
    rel = 1e-9 if prec == "fp64" else 1e-6
    np.testing.assert_allclose(out["E"][:, 0], gold["E"], rtol=rel)
    np.testing.assert_allclose(out["tau"][:, 0], gold["tau"], rtol=1e-6, atol=1e-7)
    assert np.array_equal(out["D"][:, 0] > EV_THR, gold["D"] > EV_THR)
    np.testing.assert_allclose(s.box(), gold["H"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(s.frame() @ s.box(), gold["Hlab"], rtol=0, atol=1e-12)
    assert mi_disp(s.positions(), gold["x"], gold["H"]) < 1e-6
    # a later simple-shear step still works from the rotated frame
    s.shear(1e-4)
    assert s.minimize()[0]["status"] == 0
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_parallel_stepping_under_pull_push_matches_golden(A, syn, glass256, prec):
    gold = load_golden("parhist_2d_n256_s0.npz")
    P = A.AQS_FP64 if prec == "fp64" else A.AQS_MIXED
    s = make(A, syn, glass256, P)
    r = s.parallel_step(0.0, int(gold["K"]), int(gold["P"]), int(gold["n_steps"]),
                        eq_tol=float(gold["eq_tol"]), F_steps=gold["F_steps"])
    assert np.array_equal(r["log_i"], gold["log_i"])
    assert np.array_equal(r["log_eq"], gold["log_eq"])
    assert r["iterations"] == int(gold["iterations"])
    rel = 1e-9 if prec == "fp64" else 1e-6
    np.testing.assert_allclose(r["E"], gold["E"], rtol=rel)
    assert np.array_equal(r["D"] > EV_THR, gold["D"] > EV_THR)
    np.testing.assert_allclose(s.box(), gold["H"], rtol=0, atol=1e-12)
    assert mi_disp(s.positions(), gold["x"], gold["H"]) < 1e-6
    s.close()


def test_history_beyond_the_minimum_image_rule_is_refused(A, syn, glass256):
    s = make(A, syn, glass256, A.AQS_FP64)
    x0, H0 = s.positions(), s.box()
    F = np.tile(np.array([[1.0, 0.0], [0.0, 0.8]]), (6, 1, 1))  # compress y by 0.8^6
    st = A.lib().aqs_run_history(s.h, C.byref(A.fire_params()),
                                 np.ascontiguousarray(F).ctypes.data_as(C.POINTER(C.c_double)),
                                 C.c_int64(6), None, None, None, None)
    assert st == A.AQS_ERR_BOX_TOO_SMALL
    assert np.array_equal(s.box(), H0) and mi_disp(s.positions(), x0, H0) == 0.0
    s.close()
