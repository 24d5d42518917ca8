"""Status codes of the C ABI and the equality call, exercised through the
library on the GPU.

* Every failure the host can provoke comes back as an aqs_status (never an
  abort): a cell too small for the cutoff, non-finite positions (host and
  device buffers), a minimisation that runs out of iterations, a list
  capacity that is too small (the library grows it and the result is the
  oracle's), a shear beyond the minimum-image rule, and NaN forces raised
  inside the persistent kernel (reported through its status word).
* aqs_compare_configs, the equality test of Eq. 20, against the oracle's
  measure and against properties the measure must have: zero under a uniform
  translation and under whole-cell wraps (also in a sheared cell), and
  delta (1 - 1/N) for one atom moved by delta.
"""
import ctypes as C

import numpy as np
import pytest

from conftest import load_golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    from paper_2507_20802_gb300 import aqs
    aqs.lib()
    return aqs


@pytest.fixture(scope="module")
def glass256():
    return load_golden("glass_2d_n256_s0.npz")


def _create(A, syn, x, t, H, prec=None, **kw):
    """aqs_create_system through the C ABI; returns (status, handle)."""
    x = np.ascontiguousarray(x, dtype=np.float64) if not hasattr(x, "data_ptr") else x
    t = np.ascontiguousarray(t, dtype=np.int32) if not hasattr(t, "data_ptr") else t
    n = np.array([len(t)], dtype=np.int64)
    box = np.ascontiguousarray(H, dtype=np.float64)
    d = A.aqs_system_desc()
    d.dim, d.n_replicas = H.shape[0], 1
    d.n_atoms = n.ctypes.data_as(C.POINTER(C.c_int64))
    d.box = box.ctypes.data_as(C.POINTER(C.c_double))
    d.pos = A._ptr(x)
    d.types = A._ptr(t)
    d.pot = A.make_potential(syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    d.precision = A.AQS_FP64 if prec is None else prec
    d.skin = kw.get("skin", 0.3)
    d.nlist_capacity = kw.get("nlist_capacity", 0)
    h = C.c_void_p()
    st = A.lib().aqs_create_system(C.byref(d), C.byref(h))
    return st, h


def mi_disp(a, b, H):
    d = np.asarray(a, float) - np.asarray(b, float)
    for c in reversed(range(H.shape[0])):
        n = np.round(d[:, c] / H[c, c])
        d -= n[:, None] * H[:, c][None, :]
    d -= d.mean(axis=0)
    return float(np.sqrt((d * d).sum(axis=1)).max())


# ------------------------------------------------------------ status codes
def test_box_too_small_is_reported(A, syn):
    x, t, H = syn.random_glass_start(16, 2, seed=1)  # L = 3.65 < 3 (rc + skin)
    st, h = _create(A, syn, x, t, H)
    assert st == A.AQS_ERR_BOX_TOO_SMALL and not h.value
    assert b"width" in A.lib().aqs_last_error()


def test_nonfinite_positions_are_refused(A, syn, glass256):
    torch = pytest.importorskip("torch")
    x, t, H = glass256["x"].copy(), glass256["types"], glass256["H"]
    bad = x.copy()
    bad[17, 1] = np.nan
    st, h = _create(A, syn, bad, t, H)
    assert st == A.AQS_ERR_NONFINITE and not h.value
    bad[17, 1] = np.inf
    st, h = _create(A, syn, torch.tensor(bad, device="cuda"), t, H)
    assert st == A.AQS_ERR_NONFINITE and not h.value
    # set_positions refuses them and leaves the replica as it was
    s = A.System(x, t, H[None], [len(x)], syn.LJ_SIGMA, syn.LJ_EPS, precision=A.AQS_FP64)
    assert A.lib().aqs_set_positions(s.h, 0, A._ptr(np.ascontiguousarray(bad))) == \
        A.AQS_ERR_NONFINITE
    assert mi_disp(s.positions(), x, H) == 0.0
    s.close()


def test_nan_forces_inside_the_kernel_are_reported(A, syn, glass256):
    """Two atoms on the same spot give infinite pair terms; the persistent
    kernel reports AQS_ERR_NONFINITE through its status word and the context
    stays usable (a later system on the same device works)."""
    x, t, H = glass256["x"].copy(), glass256["types"], glass256["H"]
    x[5] = x[4]
    for prec in (A.AQS_FP64, A.AQS_MIXED):
        s = A.System(x, t, H[None], [len(x)], syn.LJ_SIGMA, syn.LJ_EPS, precision=prec)
        res = s.minimize(check_status=False)[0]
        assert res["status"] == A.AQS_ERR_NONFINITE
        s.close()
    s = A.System(glass256["x"], t, H[None], [len(x)], syn.LJ_SIGMA, syn.LJ_EPS,
                 precision=A.AQS_FP64)
    assert s.minimize()[0]["status"] == A.AQS_OK
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_iteration_limit_then_resume_matches_oracle(A, orc, syn, glass256, prec):
    """max_iter = 10 ends the minimisation with AQS_ERR_NOT_CONVERGED (call
    status and replica status); a second call restarts FIRE from the
    positions reached and lands on the minimum the oracle's FIRE reaches from
    those same positions."""
    x, t, H = glass256["x"], glass256["types"], glass256["H"]
    P = A.AQS_FP64 if prec == "fp64" else A.AQS_MIXED
    s = A.System(x, t, H[None], [len(x)], syn.LJ_SIGMA, syn.LJ_EPS, precision=P)
    s.shear(2e-3)
    st, res = A.aqs_minimize(s.h, A.fire_params(max_iter=10), 1)
    assert st == A.AQS_ERR_NOT_CONVERGED and res[0].status == A.AQS_ERR_NOT_CONVERGED
    assert res[0].iters == 10 and res[0].fmax > 1e-10
    mid = s.positions()
    r = s.minimize()[0]
    pot = orc.make_potential(2, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    ro = orc.fire(pot, orc.make_fire(**syn.FIRE), mid, t, s.box())
    assert r["status"] == 0 and ro["status"] == 0
    rel = 1e-9 if prec == "fp64" else 1e-6
    assert r["E"] / len(x) == pytest.approx(ro["E"] / len(x), rel=rel)
    assert mi_disp(s.positions(), ro["x"], s.box()) < 1e-6
    s.close()


def test_small_list_capacity_grows_and_keeps_the_golden_trajectory(A, syn, glass256):
    """nlist_capacity = 8 is far below the ~28 neighbours per atom: the list
    overflows, the library grows it and rebuilds, and the first 20 steps of
    the stored 200-step oracle run are reproduced."""
    gold = load_golden("aqs_2d_n256_s0.npz")
    x, t, H = glass256["x"], glass256["types"], glass256["H"]
    s = A.System(x, t, H[None], [len(x)], syn.LJ_SIGMA, syn.LJ_EPS, precision=A.AQS_FP64,
                 nlist_capacity=8)
    assert s.mean_neighbours() > 8
    out = s.run_sequential(float(gold["dgamma"]), 20)
    np.testing.assert_allclose(out["E"][:, 0], gold["E"][:20], rtol=1e-9)
    assert np.array_equal(out["D"][:, 0] > 1e-2, gold["D"][:20] > 1e-2)
    s.close()


def test_shear_beyond_the_minimum_image_rule_is_refused(A, syn, glass256):
    x, t, H = glass256["x"], glass256["types"], glass256["H"]
    s = A.System(x, t, H[None], [len(x)], syn.LJ_SIGMA, syn.LJ_EPS, precision=A.AQS_FP64)
    st = A.lib().aqs_affine_shear(s.h, np.array([5.0]).ctypes.data_as(C.POINTER(C.c_double)))
    assert st == A.AQS_ERR_BOX_TOO_SMALL
    assert np.array_equal(s.box(), H)  # nothing applied
    st = A.lib().aqs_affine_shear(s.h, np.array([np.nan]).ctypes.data_as(C.POINTER(C.c_double)))
    assert st == A.AQS_ERR_INVALID_ARG
    s.close()


# ------------------------------------------------------------ equality (Eq. 20)
def _compare(A, sa, sb, tol):
    return A.aqs_compare_configs(sa.h, 0, sb.h, 0, tol)


def test_compare_configs_matches_oracle_and_its_invariants(A, orc, syn, glass256):
    x, t, H = glass256["x"], glass256["types"], glass256["H"]
    n = len(x)
    # a sheared cell, so that a wrap across the y face carries the tilt
    xs, Hs = orc.affine_shear(x, H, 0.05)
    base = A.System(xs, t, Hs[None], [n], syn.LJ_SIGMA, syn.LJ_EPS, precision=A.AQS_FP64)
    # 1. uniform translation, then every atom wrapped into the cell
    shift = np.array([0.37, -2.21])
    moved = orc.wrap(xs + shift, Hs)
    assert np.any(np.abs(moved - xs - shift)[:, 1] > 1.0)  # some atoms crossed the y face
    b = A.System(moved, t, Hs[None], [n], syn.LJ_SIGMA, syn.LJ_EPS, precision=A.AQS_FP64)
    m, eq = _compare(A, base, b, 1e-6)
    assert m < 1e-12 and eq
    # 2. one atom moved by delta: max deviation from the mean shift is delta (1 - 1/N)
    delta = 1e-3
    one = xs.copy()
    one[100, 0] += delta
    c = A.System(one, t, Hs[None], [n], syn.LJ_SIGMA, syn.LJ_EPS, precision=A.AQS_FP64)
    m, eq = _compare(A, base, c, 1e-6)
    assert m == pytest.approx(delta * (1.0 - 1.0 / n), rel=1e-9) and not eq
    m2, eq2 = _compare(A, base, c, 1e-2)
    assert m2 == m and eq2
    # 3. a random perturbation of every atom: the oracle's measure, element for
    # element the same definition
    rnd = xs + 0.03 * (syn.uniform(77, xs.size).reshape(xs.shape) - 0.5)
    d = A.System(rnd, t, Hs[None], [n], syn.LJ_SIGMA, syn.LJ_EPS, precision=A.AQS_FP64)
    m, _ = _compare(A, d, base, 1e-6)
    assert m == pytest.approx(orc.max_rel_disp(rnd, xs, Hs), rel=1e-12, abs=1e-15)
    # symmetric in its arguments
    m_ba, _ = _compare(A, base, d, 1e-6)
    assert m_ba == pytest.approx(m, rel=1e-12)
    # 4. sizes must agree
    small = A.System(xs[:200], t[:200], Hs[None], [200], syn.LJ_SIGMA, syn.LJ_EPS,
                     precision=A.AQS_FP64)
    st = A.lib().aqs_compare_configs(base.h, 0, small.h, 0, C.c_double(1e-6),
                                     C.byref(C.c_double()), C.byref(C.c_int()))
    assert st == A.AQS_ERR_INVALID_ARG
    for s in (base, b, c, d, small):
        s.close()
