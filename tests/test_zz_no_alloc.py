"""GPU check of aqs_energy_forces_noalloc, the entry point for callers that
must not allocate device memory (see include/aqs.h).

It is compared through the C ABI with the regular path (a system created with
aqs_create_system, evaluated by aqs_energy_forces) on two configurations in a
row, so that the second call runs on scratch left over from the first.  The
tolerances are those of the FP64 force parity tests.  This file sorts last so
that a run stopping at the first failure has run every other test before it."""
import ctypes as C

import numpy as np
import pytest

from conftest import load_golden

pytestmark = pytest.mark.gpu


def _regular(A, syn, x, t, H):
    s = A.System(x, t, H[None], [len(x)], syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR,
                 precision=A.AQS_FP64)
    E, F, tau = s.energy_forces()
    s.close()
    return E, F, tau


def _noalloc(A, torch, syn, x, t, H):
    dim = H.shape[0]
    pos = torch.tensor(x, dtype=torch.float64, device="cuda")
    typ = torch.tensor(t, dtype=torch.int32, device="cuda")
    out_f = torch.full_like(pos, float("nan"))
    out_e = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    box = np.ascontiguousarray(H, dtype=np.float64)
    pot = A.make_potential(syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    st = A.lib().aqs_energy_forces_noalloc(dim, len(x), C.c_void_p(pos.data_ptr()),
                                           C.c_void_p(typ.data_ptr()),
                                           box.ctypes.data_as(C.POINTER(C.c_double)),
                                           C.byref(pot), C.c_void_p(out_f.data_ptr()),
                                           C.c_void_p(out_e.data_ptr()), None)
    assert st == A.AQS_OK
    torch.cuda.synchronize()
    e, tau = out_e.cpu().numpy()
    return float(e), out_f.cpu().numpy(), float(tau)


def _check_cases(A, torch, syn, cases):
    for x, t, H in cases:
        E, F, tau = _regular(A, syn, x, t, H)
        En, Fn, taun = _noalloc(A, torch, syn, x, t, H)
        scale = max(1.0, np.abs(F).max())
        assert En == pytest.approx(E, rel=1e-11, abs=1e-9)
        assert np.abs(Fn - F).max() <= 1e-11 * scale
        assert taun == pytest.approx(tau, rel=1e-10, abs=1e-10)


def test_noalloc_energy_forces_match_regular_path_twice():
    torch = pytest.importorskip("torch")
    from paper_2507_20802_gb300 import aqs as A, synthetic as syn
    g = load_golden("glass_2d_n256_s0.npz")
    cases = [(g["x"], g["types"], g["H"])]
    x2, t2, H2 = syn.random_glass_start(1000, 2, seed=3)  # larger, ragged, huge forces
    H2 = H2.copy()
    H2[0, 1] = 0.03 * H2[1, 1]
    cases.append((x2, t2, H2))
    _check_cases(A, torch, syn, cases)


def test_noalloc_3d_tilted_glass_and_full_scratch():
    """The 3D kernel on the stored 3D glass with an xy tilt, then the largest
    size the fixed scratch takes (65 536 atoms: every slot of the array is
    written and read), then the 3D glass again on the scratch the large call
    left behind."""
    torch = pytest.importorskip("torch")
    from paper_2507_20802_gb300 import aqs as A, synthetic as syn
    g = load_golden("glass_3d_n2048_s0.npz")
    H3 = g["H"].copy()
    H3[0, 1] = 0.02 * H3[1, 1]
    x4, t4, H4 = syn.random_glass_start(65536, 2, seed=5)
    _check_cases(A, torch, syn, [(g["x"], g["types"], H3), (x4, t4, H4),
                                 (g["x"], g["types"], H3)])


def test_noalloc_rejects_tilts_outside_xy():
    """The 3D width test and minimum image assume the only tilt is H[0][1];
    an xz or yz tilt is refused before anything is launched."""
    pytest.importorskip("torch")
    from paper_2507_20802_gb300 import aqs as A, synthetic as syn
    pot = A.make_potential(syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    for k in (2, 5):
        box = np.eye(3) * 20.0
        box.flat[k] = 1.0
        box = np.ascontiguousarray(box)
        st = A.lib().aqs_energy_forces_noalloc(3, 100, C.c_void_p(1), C.c_void_p(1),
                                               box.ctypes.data_as(C.POINTER(C.c_double)),
                                               C.byref(pot), C.c_void_p(1), C.c_void_p(1), None)
        assert st == A.AQS_ERR_INVALID_ARG


def test_noalloc_rejects_sizes_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    from paper_2507_20802_gb300 import aqs as A, synthetic as syn
    pot = A.make_potential(syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    box = np.eye(2) * 300.0
    n = 65537
    st = A.lib().aqs_energy_forces_noalloc(2, n, C.c_void_p(1), C.c_void_p(1),
                                           box.ctypes.data_as(C.POINTER(C.c_double)),
                                           C.byref(pot), C.c_void_p(1), C.c_void_p(1), None)
    assert st == A.AQS_ERR_INVALID_ARG
