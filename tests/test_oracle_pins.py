"""Pins of the FP64 oracle against facts fixed by the paper and by
mathematics (no GPU).  Each test is chosen so that a plausible mistake in the
oracle (a dropped term, a wrong sign, a transposed index) fails it:

* textbook LJ values and the shifted-force structure (Sec. 2.2, Eq. 13);
* forces = -gradient of the energy by central finite differences (Eq. 6);
* Newton's third law (net force zero);
* stress = (1/V) dE/dgamma along the simple-shear path (Eq. 16, Fig. 2b);
* minimum image = brute-force search over periodic images (Sec. 2.1);
* affine maps compose, F(a) F(b) = F(a + b) (Eqs. 1-3, 16; Sec. 3.2);
* a perfect triangular lattice has zero force before and after shear;
* FIRE lands on the dimer minimum and lowers the energy; CG (the paper's
  minimiser, Sec. 2.1) lands on the same minimum.
"""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def pot2(orc, syn):
    return orc.make_potential(2, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)


@pytest.fixture(scope="module")
def pot3(orc, syn):
    return orc.make_potential(3, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)


def _jiggled_lattice(syn, seed=3, amp=0.05):
    x, t, H = syn.triangular_lattice(8, 8)
    u = syn.uniform(900 + seed, x.size).reshape(x.shape) - 0.5
    t = (syn.uniform(950 + seed, len(t)) < 0.35).astype(np.int32)
    return x + amp * u, t, H


def _jiggled_cubic(syn, seed=3, amp=0.08, m=6, density=0.6):
    a = (1.0 / density) ** (1.0 / 3.0)
    g = np.arange(m) * a
    x = np.array(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1).T
    u = syn.uniform(700 + seed, x.size).reshape(x.shape) - 0.5
    t = (syn.uniform(750 + seed, len(x)) < 0.2).astype(np.int32)
    return x + amp * u, t, np.eye(3) * (m * a)


# ----------------------------------------------------------------- pair term
@pytest.mark.parametrize("sig,eps", [(1.0, 1.0), (0.8, 1.5), (0.88, 0.5)])
def test_pair_textbook_points(orc, sig, eps):
    """Plain LJ is 0 at r = sigma and has its minimum -eps at 2^(1/6) sigma.
    The shifted-force term only adds a linear function c0 + c1 r, and its
    slope is -U'(rc) = -du(r_min); so the difference u(sigma) - u(r_min) must
    be eps + (sigma - r_min) du(r_min)."""
    rc = 2.5 * sig
    rm = 2.0 ** (1.0 / 6.0) * sig
    u_s, _ = orc.pair_sflj(sig * sig, sig, eps, rc)
    u_m, du_m = orc.pair_sflj(rm * rm, sig, eps, rc)
    assert u_s - u_m == pytest.approx(eps + (sig - rm) * du_m, rel=1e-13, abs=1e-14)
    # U'(rc) of plain LJ is small and positive (attractive tail): du(r_min) = -U'(rc) < 0
    assert du_m < 0.0


@pytest.mark.parametrize("sig,eps", [(1.0, 1.0), (0.8, 1.5)])
def test_pair_cutoff_continuity(orc, sig, eps):
    """U_sf(rc) = 0 and F_sf(rc) = 0, approaching as O(d^2) and O(d)."""
    rc = 2.5 * sig
    for d in [1e-4, 1e-5, 1e-6, 1e-7]:
        u, du = orc.pair_sflj((rc - d) ** 2, sig, eps, rc)
        assert abs(u) < 1.0 * d * d
        assert abs(du) < 1.0 * d
    u, du = orc.pair_sflj(rc * rc, sig, eps, rc)
    assert u == 0.0 and du == 0.0
    # ratios confirm the orders: halving d quarters u and halves du
    u1, du1 = orc.pair_sflj((rc - 1e-3) ** 2, sig, eps, rc)
    u2, du2 = orc.pair_sflj((rc - 5e-4) ** 2, sig, eps, rc)
    assert u1 / u2 == pytest.approx(4.0, rel=2e-3)
    assert du1 / du2 == pytest.approx(2.0, rel=2e-3)


def test_pair_derivative_fd(orc):
    sig, eps, rc = 0.8, 1.5, 2.0
    for r in [0.7, 0.85, 1.0, 1.5, 1.9]:
        h = 1e-6
        up, _ = orc.pair_sflj((r + h) ** 2, sig, eps, rc)
        um, _ = orc.pair_sflj((r - h) ** 2, sig, eps, rc)
        _, du = orc.pair_sflj(r * r, sig, eps, rc)
        assert (up - um) / (2 * h) == pytest.approx(du, rel=1e-7, abs=1e-9)


# --------------------------------------------------------------- all pairs
@pytest.mark.parametrize("dim", [2, 3])
def test_forces_are_minus_gradient(orc, syn, dim, pot2, pot3):
    pot = pot2 if dim == 2 else pot3
    if dim == 2:
        x, t, H = _jiggled_lattice(syn)
        H = H.copy()
        H[0, 1] = 0.07 * H[1, 1]  # sheared cell
    else:
        x, t, H = _jiggled_cubic(syn, seed=7)
    E, F, _ = orc.energy_forces(pot, x, t, H)
    h = 1e-6
    rng_idx = list(range(0, len(x), max(1, len(x) // 12)))
    worst = 0.0
    for i in rng_idx:
        for c in range(dim):
            xp = x.copy(); xp[i, c] += h
            xm = x.copy(); xm[i, c] -= h
            Ep, _, _ = orc.energy_forces(pot, xp, t, H)
            Em, _, _ = orc.energy_forces(pot, xm, t, H)
            g = -(Ep - Em) / (2 * h)
            worst = max(worst, abs(g - F[i, c]) / max(1.0, abs(F[i, c])))
    assert worst < 1e-6


@pytest.mark.parametrize("dim", [2, 3])
def test_newton_third_law(orc, syn, dim, pot2, pot3):
    pot = pot2 if dim == 2 else pot3
    x, t, H = (_jiggled_lattice(syn) if dim == 2 else _jiggled_cubic(syn, seed=2))
    _, F, _ = orc.energy_forces(pot, x, t, H)
    assert np.linalg.norm(F.sum(axis=0)) < 1e-12 * max(1.0, np.abs(F).max())


@pytest.mark.parametrize("dim", [2, 3])
def test_stress_is_energy_strain_derivative(orc, syn, dim, pot2, pot3):
    """tau = (1/V) dE/dgamma along the simple-shear affine path."""
    pot = pot2 if dim == 2 else pot3
    x, t, H = (_jiggled_lattice(syn) if dim == 2 else _jiggled_cubic(syn, seed=5))
    E, _, tau = orc.energy_forces(pot, x, t, H)
    h = 1e-6
    xp, Hp = orc.affine_shear(x, H, h)
    xm, Hm = orc.affine_shear(x, H, -h)
    Ep, _, _ = orc.energy_forces(pot, xp, t, Hp)
    Em, _, _ = orc.energy_forces(pot, xm, t, Hm)
    dEdg = (Ep - Em) / (2 * h)
    assert tau == pytest.approx(dEdg / orc.volume(H), rel=1e-6, abs=1e-9)


# ---------------------------------------------------------------- geometry
@pytest.mark.parametrize("dim,tilt", [(2, 0.0), (2, 0.2), (2, -0.15), (3, 0.1)])
def test_min_image_matches_brute_force(orc, syn, dim, tilt):
    L = np.array([7.0, 6.0, 5.5][:dim])
    H = np.diag(L)
    H[0, 1] = tilt * L[1]
    r = orc.half_min_width(H)
    u = syn.uniform(77, 400 * dim).reshape(400, dim)
    d = (u - 0.5) * 4.0 * L[None, :]
    mi = orc.min_image(H, d)
    rng = range(-2, 3)
    checked = 0
    for k in range(len(d)):
        best = None
        for n in np.array(np.meshgrid(*([list(rng)] * dim))).reshape(dim, -1).T:
            cand = d[k] + H @ n
            if best is None or np.dot(cand, cand) < np.dot(best, best):
                best = cand
        if np.linalg.norm(best) < r:  # the rule is exact inside half the width
            assert np.allclose(mi[k], best, atol=1e-12)
            checked += 1
    assert checked > 20


def test_affine_maps_compose(orc, syn):
    x, t, H = syn.random_glass_start(100, 2, seed=1)
    xa, Ha = orc.affine_shear(x, H, 1e-3)
    xb, Hb = orc.affine_shear(xa, Ha, 2e-3)
    xc, Hc = orc.affine_shear(x, H, 3e-3)
    assert np.allclose(xb, xc, rtol=0, atol=1e-13 * H[0, 0])
    assert np.allclose(Hb, Hc, rtol=0, atol=1e-14 * H[0, 0])
    assert Hc[0, 1] == pytest.approx(3e-3 * H[1, 1], rel=1e-14)
    # level I (Sec. 3.2): F^(i K dg) equals i*K fine maps
    xs, Hs = x, H
    for _ in range(10):
        xs, Hs = orc.affine_shear(xs, Hs, 1e-4)
    xl, Hl = orc.affine_shear(x, H, 10 * 1e-4)
    assert np.allclose(xs, xl, rtol=0, atol=1e-12 * H[0, 0])
    # the general map with F = [[1, g], [0, 1]] is the same operation
    xg, Hg = orc.affine_map(x, H, np.array([[1.0, 3e-3], [0.0, 1.0]]))
    assert np.array_equal(xg, xc) and np.array_equal(Hg, Hc)


def test_max_rel_disp_invariances(orc, syn):
    x, t, H = syn.random_glass_start(200, 2, seed=4)
    assert orc.max_rel_disp(x, x, H) == 0.0
    # uniform translation and whole-cell wraps are invisible
    shift = np.array([0.3, -0.7])
    y = x + shift
    y[::7] += H[:, 0]
    y[::5] -= H[:, 1]
    assert orc.max_rel_disp(y, x, H) < 1e-12
    # one atom moved by delta (mean removal shrinks it by 1/N)
    z = x.copy()
    z[17] += np.array([1e-3, 0.0])
    assert orc.max_rel_disp(z, x, H) == pytest.approx(1e-3 * (1 - 1 / 200), rel=1e-9)


# ---------------------------------------------------------------- lattice
def test_triangular_lattice_has_zero_force_under_shear(orc, syn, pot2):
    fp = orc.make_fire(**syn.FIRE)
    x, t, H = syn.triangular_lattice()
    E0, F0, tau0 = orc.energy_forces(pot2, x, t, H)
    assert np.abs(F0).max() < 1e-10 and abs(tau0) < 1e-12
    for g in [1e-4, 1e-3, 5e-3]:
        xs, Hs = orc.affine_shear(x, H, g)
        r = orc.fire(pot2, fp, xs, t, Hs)
        assert r["status"] == 0 and r["iters"] == 0  # already a minimum
        assert orc.max_rel_disp(r["x"], xs, Hs) == 0.0
    # all sites equivalent: per-atom energy is the same everywhere, which
    # also shows as E/N independent of the lattice size
    x2, t2, H2 = syn.triangular_lattice(8, 8)
    E2, _, _ = orc.energy_forces(pot2, x2, t2, H2)
    assert E2 / 64 == pytest.approx(E0 / 256, rel=1e-12)


# ---------------------------------------------------------------- minimisers
def test_fire_dimer_lands_on_pair_minimum(orc, syn):
    """Two A atoms: FIRE must stop at the root of U_sf'(r) = 0."""
    pot = orc.make_potential(2, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    H = np.eye(2) * 12.0
    x = np.array([[3.0, 3.0], [4.3, 3.4]])
    t = np.array([0, 0], np.int32)
    r = orc.fire(pot, orc.make_fire(**syn.FIRE), x, t, H)
    assert r["status"] == 0
    d = np.linalg.norm(r["x"][1] - r["x"][0])
    lo, hi = 1.0, 1.3  # bisection on the oracle's pair derivative
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        _, du = orc.pair_sflj(mid * mid, 1.0, 1.0, 2.5)
        lo, hi = (mid, hi) if du < 0 else (lo, mid)
    assert d == pytest.approx(0.5 * (lo + hi), abs=1e-10)
    # slightly beyond the plain-LJ minimum 2^(1/6): removing the tail force
    # U'(rc) > 0 leaves less attraction
    assert 2 ** (1 / 6) < d < 1.13


def test_fire_lowers_energy_and_converges(orc, syn, pot2):
    fp = orc.make_fire(**syn.FIRE)
    x, t, H = _jiggled_lattice(syn, seed=9, amp=0.2)
    E0, _, _ = orc.energy_forces(pot2, x, t, H)
    r = orc.fire(pot2, fp, x, t, H, trace_cap=200000)
    assert r["status"] == 0 and r["fmax"] < 1e-10
    assert r["E"] <= E0
    et, rt = r["e_trace"], r["reset_trace"]
    # reading of "monotone energy" for the inertial FIRE: every velocity reset
    # happens at an energy no higher than the start
    assert np.all(et[:len(rt)][rt == 1] <= E0)
    assert et[-1] == pytest.approx(r["E"])


def test_cg_is_monotone_and_agrees_with_fire(orc, syn, pot2):
    fp = orc.make_fire(**syn.FIRE)
    x, t, H = _jiggled_lattice(syn, seed=11, amp=0.1)
    f = orc.fire(pot2, fp, x, t, H)
    c = orc.cg(pot2, x, t, H, 1e-9, 50000, trace_cap=60000)
    assert np.all(np.diff(c["e_trace"]) < 0)
    # CG stalls where energy differences fall below FP64 resolution; near
    # the minimum |x - x*| ~ |F| / lambda_min
    assert c["fmax"] < 1e-4
    assert orc.max_rel_disp(f["x"], c["x"], H) < 1e-4


def test_fire_reports_nonfinite(orc, syn, pot2):
    x, t, H = _jiggled_lattice(syn)
    x[1] = x[0]  # zero distance -> infinite force
    r = orc.fire(pot2, orc.make_fire(**syn.FIRE), x, t, H)
    assert r["status"] == 5


def test_box_too_small_is_rejected(orc, syn, pot2):
    x, t, H = syn.random_glass_start(16, 2, seed=0)  # L = 3.65 < 2 * 2.5
    with pytest.raises(RuntimeError):
        orc.energy_forces(pot2, x, t, H)
