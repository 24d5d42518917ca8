"""GPU checks of the launch configuration: staging modes and the autotuner.

* every staging mode (where list rows and neighbour records are read from)
  gives bitwise identical trajectories, with list rebuilds inside the kernel;
* tuning times every feasible cluster size and staging mode and leaves
  positions, boxes and results untouched (bitwise equal configuration);
* a system that tunes before each minimisation still reproduces the oracle's
  stored AQS trajectory and Algorithm-1 decision log.
"""
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
        n = np.round(d[:, c] / H[c, c])
        d -= n[:, None] * H[:, c][None, :]
    d -= d.mean(axis=0)
    return float(np.sqrt((d * d).sum(axis=1)).max())


def test_autotune_times_candidates_and_keeps_configuration(A, syn, glass256):
    x, t, H = glass256["x"], glass256["types"], glass256["H"]
    R = 4
    s = A.System(np.tile(x, (R, 1)), np.tile(t, R), np.tile(H[None], (R, 1, 1)), [len(x)] * R,
                 syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR, precision=A.AQS_MIXED)
    s.shear(np.arange(R) * 1e-3)
    before = [s.positions(r) for r in range(R)]
    boxes = [s.box(r) for r in range(R)]
    best, mode, ms, ms_mode = s.autotune(iters=64)
    # 256 atoms: at least 32 atoms per CTA allows C = 1..8, all feasible
    assert sorted(ms) == list(range(1, 9)), ms
    assert all(v > 0 for v in ms.values())
    assert all(s.cluster_size(r) == best for r in range(R))
    # every staging mode fits at 32..256 atoms per CTA and was timed
    assert sorted(ms_mode) == [0, 1, 2, 3], ms_mode
    fastest = min(min(ms.values()), min(ms_mode.values()))
    if mode >= 0:
        assert ms_mode[mode] == fastest
        assert s.staging(0) == mode
    else:
        assert ms[best] == fastest
    for r in range(R):
        assert np.array_equal(s.positions(r), before[r])
        assert np.array_equal(s.box(r), boxes[r])
    # the tuned system minimises to the same minimum as a default one
    ref = A.System(np.tile(x, (R, 1)), np.tile(t, R), np.tile(H[None], (R, 1, 1)), [len(x)] * R,
                   syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR, precision=A.AQS_MIXED)
    ref.shear(np.arange(R) * 1e-3)
    a = s.minimize()
    b = ref.minimize()
    for r in range(R):
        assert a[r]["E"] == pytest.approx(b[r]["E"], rel=1e-12)
        assert mi_disp(s.positions(r), ref.positions(r), s.box(r)) < 1e-6


def test_autotuned_sequential_aqs_matches_golden(A, syn, glass256):
    gold = load_golden("aqs_2d_n256_s0.npz")
    x, t, H = glass256["x"], glass256["types"], glass256["H"]
    s = A.System(x, t, H[None], [len(x)], syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR,
                 precision=A.AQS_FP64)
    s.set_autotune(32)
    n = int(gold["n_steps"])
    out = s.run_sequential(float(gold["dgamma"]), n)
    np.testing.assert_allclose(out["E"][:, 0], gold["E"], rtol=1e-9)
    assert np.array_equal(out["D"][:, 0] > EV_THR, gold["D"] > EV_THR)
    assert mi_disp(s.positions(), gold["x"], gold["H"]) < 1e-6


def test_autotuned_parallel_stepping_matches_golden(A, syn, glass256):
    gold = load_golden("par_2d_n256_s0.npz")
    x, t, H = glass256["x"], glass256["types"], glass256["H"]
    s = A.System(x, t, H[None], [len(x)], syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR,
                 precision=A.AQS_MIXED)
    s.set_autotune(32)
    r = s.parallel_step(float(gold["dgamma"]), int(gold["K"]), int(gold["P"]),
                        int(gold["n_steps"]), eq_tol=float(gold["eq_tol"]))
    assert np.array_equal(r["log_i"], gold["log_i"])
    assert np.array_equal(r["log_eq"], gold["log_eq"])
    assert np.array_equal(r["log_iter"], gold["log_iter"])
    np.testing.assert_allclose(r["E"], gold["E"], rtol=1e-6)
    assert np.array_equal(r["D"] > EV_THR, gold["D"] > EV_THR)
    assert mi_disp(s.positions(), gold["x"], gold["H"]) < 1e-6


@pytest.mark.parametrize("dim", [2, 3])
def test_staging_modes_give_identical_trajectories(A, syn, dim):
    """Shear steps large enough to trip the Verlet skin (rebuilds inside the
    kernel) on one cluster of 16 CTAs; modes 0..3 read identical values, so
    energies, iteration counts and positions must agree bitwise."""
    if dim == 2:
        g = load_golden("glass_2d_n1024_s0.npz")
        dg, steps = 5e-3, 4
    else:
        g = load_golden("glass_3d_n2048_s0.npz")
        dg, steps = 2e-3, 3
    x, t, H = g["x"], g["types"], g["H"]
    out = {}
    for mode in range(4):
        s = A.System(x, t, H[None], [len(x)], syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR,
                     precision=A.AQS_MIXED, cluster_size=16)
        s.set_staging(mode)
        assert s.staging(0) == mode
        r = s.run_sequential(dg, steps)
        out[mode] = (r, s.positions())
    r0, x0 = out[0]
    assert r0["D"].max() > 0.0
    for mode in (1, 2, 3):
        r, xm = out[mode]
        assert np.array_equal(r["E"], r0["E"]), mode
        assert np.array_equal(r["iters"], r0["iters"]), mode
        assert np.array_equal(xm, x0), mode


def test_staging_rejects_unknown_modes(A, syn, glass256):
    x, t, H = glass256["x"], glass256["types"], glass256["H"]
    s = A.System(x, t, H[None], [len(x)], syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    with pytest.raises(A.AqsError):
        s.set_staging(4)
    s.set_staging(-1)
