"""Grid-barrier launches (aqs_set_grid_barrier: one cooperative launch, no
thread-block clusters, per-replica barriers in global memory) reproduce the
stored oracle runs to the tolerances of the cluster launches: the 200-step
AQS run and Algorithm 1 on the N = 256 glass in both precisions, several
replicas of one launch, and the 3D N = 2048 run (lean launches)."""
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


def mi_disp(a, b, H):
    d = np.asarray(a, float) - np.asarray(b, float)
    for c in reversed(range(H.shape[0])):
        d -= np.round(d[:, c] / H[c, c])[:, None] * H[:, c][None, :]
    d -= d.mean(axis=0)
    return float(np.sqrt((d * d).sum(axis=1)).max())


def make(A, syn, g, prec, R=1, **kw):
    x, t, H = g["x"], g["types"], g["H"]
    s = A.System(np.tile(x, (R, 1)), np.tile(t, R), np.tile(H[None], (R, 1, 1)), [len(x)] * R,
                 syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR, precision=prec, **kw)
    s.set_grid_barrier(True)
    assert s.grid_barrier() == 1 and s.grid_barrier(chains=True) == -1  # no chains yet
    return s


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_grid_barrier_trajectory_matches_golden(A, syn, prec):
    g = load_golden("glass_2d_n256_s0.npz")
    gold = load_golden("aqs_2d_n256_s0.npz")
    P = A.AQS_FP64 if prec == "fp64" else A.AQS_MIXED
    s = make(A, syn, g, P, R=3)  # three replicas in one cooperative launch
    out = s.run_sequential(float(gold["dgamma"]), int(gold["n_steps"]))
    rel = 1e-9 if prec == "fp64" else 1e-6
    for r in range(3):
        np.testing.assert_allclose(out["E"][:, r], gold["E"], rtol=rel)
        assert np.array_equal(out["D"][:, r] > EV_THR, gold["D"] > EV_THR)
        assert mi_disp(s.positions(r), gold["x"], gold["H"]) < 1e-6
    assert s.cluster_size(0) > 1
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_grid_barrier_parallel_stepping_matches_golden(A, syn, prec):
    g = load_golden("glass_2d_n256_s0.npz")
    gold = load_golden("par_2d_n256_s0.npz")
    P = A.AQS_FP64 if prec == "fp64" else A.AQS_MIXED
    s = make(A, syn, g, P)
    r = s.parallel_step(float(gold["dgamma"]), int(gold["K"]), int(gold["P"]),
                        int(gold["n_steps"]), eq_tol=float(gold["eq_tol"]))
    assert s.grid_barrier(chains=True) == 1  # the chains inherit the fixed mode
    assert np.array_equal(r["log_eq"], gold["log_eq"])
    assert np.array_equal(r["log_i"], gold["log_i"])
    rel = 1e-9 if prec == "fp64" else 1e-6
    np.testing.assert_allclose(r["E"], gold["E"], rtol=rel)
    assert mi_disp(s.positions(), gold["x"], gold["H"]) < 1e-6
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_grid_barrier_3d_matches_golden(A, syn, prec):
    g = load_golden("glass_3d_n2048_s0.npz")
    gold = load_golden("aqs_3d_n2048_s0.npz")
    P = A.AQS_FP64 if prec == "fp64" else A.AQS_MIXED
    s = make(A, syn, g, P)
    n = min(4, int(gold["n_steps"]))
    out = s.run_sequential(float(gold["dgamma"]), n)
    rel = 1e-9 if prec == "fp64" else 1e-6
    np.testing.assert_allclose(out["E"][:, 0], gold["E"][:n], rtol=rel)
    np.testing.assert_allclose(out["D"][:, 0], gold["D"][:n], rtol=1e-3)
    s.close()
