"""Pins of the oracle's pointwise functions (CPU only).

Each test checks the oracle against something other than itself: numpy's
linear algebra, textbook flat-space physics carried to a curved metric by a
coordinate transformation (tests/flatspace.py), hand-computed reconstruction
values, closed-form limits, and brute-force root scans.
"""
import numpy as np
import pytest

import oracle
from tests import flatspace as fs


# ------------------------------------------------------------- metric

def test_metric_inverse_matches_numpy():
    rng = np.random.default_rng(1)
    for _ in range(50):
        A = fs.random_A(rng)
        g6, _ = fs.metric_of(A)
        gi6, sg = oracle.metric_inverse(g6)
        g = np.array([[g6[0], g6[1], g6[2]], [g6[1], g6[3], g6[4]],
                      [g6[2], g6[4], g6[5]]])
        assert np.allclose(fs.g6_of(np.linalg.inv(g)), gi6, rtol=1e-13, atol=1e-13)
        assert abs(sg - np.sqrt(np.linalg.det(g))) < 1e-13 * sg


# ------------------------------------------------ conserved vector and fluxes

@pytest.mark.parametrize("seed", range(6))
def test_flux_and_cons_equal_transformed_textbook(seed):
    """Eqs. conserved_dens/tau/S and the flux column of Eq. GRRMHD_flux_form
    (with Ohm's law for the charge flux) in a constant curved metric with lapse
    and shift equal the textbook flat-space values transformed as tensor
    densities: U_x = T(U_flat), F_x = alpha T(F_flat) - beta U_x."""
    rng = np.random.default_rng(seed)
    gam_eos = [2.0, 4.0 / 3.0, 5.0 / 3.0][seed % 3]
    sigma = [0.0, 3.0, 1e4][seed % 3]
    for _ in range(20):
        prim = fs.random_flat_prim(rng, gam_eos)
        A = fs.random_A(rng)
        alpha = rng.uniform(0.5, 1.5)
        beta = rng.uniform(-0.3, 0.3, 3)
        g6, _ = fs.metric_of(A)
        U0, F0 = fs.textbook(prim, gam_eos, sigma)
        Ux = fs.transform_cons(U0, A)
        Fx = fs.transform_flux(F0, A)
        px = fs.transform_prim(prim, A)
        cons = oracle.prim2con(px, alpha, beta, g6, gam_eos)
        scale = np.abs(Ux).max()
        assert np.allclose(cons, Ux, rtol=1e-12, atol=1e-12 * scale), (cons - Ux)
        for d in range(3):
            F, U = oracle.flux(d, px, alpha, beta, g6, sigma, gam_eos)
            expect = alpha * Fx[d] - beta[d] * Ux
            fscale = max(np.abs(expect).max(), 1.0)
            assert np.allclose(F, expect, rtol=1e-11, atol=1e-11 * fscale), (d, F - expect)


def test_stress_reading_distinguishes_sqrt_gamma():
    """The undensitised stress reading of Eq. conserved_Sij: for a fluid at
    rest the S_i flux in direction i is alpha sqrt(gamma) p delta (not
    alpha gamma p)."""
    prim = np.zeros(14)
    prim[0], prim[1] = 1.0, 0.7
    g6 = np.array([4.0, 0, 0, 4.0, 0, 4.0])      # sqrt(gamma) = 8
    F, _ = oracle.flux(0, prim, 1.3, (0, 0, 0), g6, 0.0, 2.0)
    assert abs(F[1] - 1.3 * 8.0 * 0.7) < 1e-14


# ------------------------------------------------------------- HLLE

def test_hlle_consistent_state_gives_physical_flux():
    rng = np.random.default_rng(7)
    for _ in range(30):
        A = fs.random_A(rng)
        prim = fs.transform_prim(fs.random_flat_prim(rng), A)
        g6, _ = fs.metric_of(A)
        alpha, beta = rng.uniform(0.5, 1.5), rng.uniform(-0.3, 0.3, 3)
        for d in range(3):
            F = oracle.hlle(d, prim, prim, alpha, beta, g6, 2.0, 2.0)
            Fp, _ = oracle.flux(d, prim, alpha, beta, g6, 2.0, 2.0)
            assert np.allclose(F, Fp, rtol=1e-13, atol=1e-13 * np.abs(Fp).max())


def test_hlle_flat_is_rusanov_with_unit_speed():
    rng = np.random.default_rng(8)
    for _ in range(10):
        pL, pR = fs.random_flat_prim(rng), fs.random_flat_prim(rng)
        UL, FL = fs.textbook(pL, 2.0, 1.0)
        UR, FR = fs.textbook(pR, 2.0, 1.0)
        for d in range(3):
            F = oracle.hlle(d, pL, pR, sigma=1.0, gamma_eos=2.0)
            expect = 0.5 * (FL[d] + FR[d]) - 0.5 * (UR - UL)
            assert np.allclose(F, expect, rtol=1e-12, atol=1e-12 * np.abs(expect).max())


def test_hlle_upwinds_when_shift_exceeds_light_speed():
    """lambda_+- = +-sqrt(gamma^dd) - beta^d/alpha both > 0 => F = F_L."""
    rng = np.random.default_rng(9)
    pL, pR = fs.random_flat_prim(rng), fs.random_flat_prim(rng)
    beta = np.array([-2.5, 0.0, 0.0])
    F = oracle.hlle(0, pL, pR, 1.0, beta, (1, 0, 0, 1, 0, 1), 0.0, 2.0)
    FL, _ = oracle.flux(0, pL, 1.0, beta, (1, 0, 0, 1, 0, 1), 0.0, 2.0)
    assert np.allclose(F, FL, rtol=1e-14, atol=1e-14)


# ------------------------------------------------------------- reconstruction

def test_tvd_hand_values():
    u = np.array([0.0, 0.0, 1.0, 3.0, 4.0, 4.0, 4.0])
    # face between u[2]=1 and u[3]=3
    uL, uR = oracle.recon_line(0, u)          # minmod
    assert uL[2] == 1.5 and uR[2] == 2.5
    uL, uR = oracle.recon_line(1, u)          # MC2
    assert uL[2] == 1.75 and uR[2] == 2.25


@pytest.mark.parametrize("method", [0, 1])
def test_tvd_exact_on_linear_and_flat_at_extrema(method):
    i = np.arange(12, dtype=float)
    u = 0.3 + 1.7 * i
    uL, uR = oracle.recon_line(method, u)
    ok = ~np.isnan(uL)
    assert np.allclose(uL[ok], (0.3 + 1.7 * (i + 0.5))[ok], rtol=0, atol=1e-13)
    assert np.allclose(uR[ok], (0.3 + 1.7 * (i + 0.5))[ok], rtol=0, atol=1e-13)
    u = np.array([0, 0, 0, 1, 0, 0, 0, 0], dtype=float)  # extremum at 3
    uL, uR = oracle.recon_line(method, u)
    assert uL[3] == 1.0 and uR[2] == 1.0


def _cell_avg(poly, x0, x1):
    P = np.polyint(poly)
    return (np.polyval(P, x1) - np.polyval(P, x0)) / (x1 - x0)


def test_weno5_exact_for_quadratic_cell_averages():
    h = 0.1
    edges = np.arange(13) * h
    poly = np.array([0.7, -1.3, 2.1])
    u = _cell_avg(poly, edges[:-1], edges[1:])
    uL, uR = oracle.recon_line(2, u)
    ok = ~np.isnan(uL)
    exact = np.polyval(poly, edges[1:])
    assert np.allclose(uL[ok], exact[ok], atol=1e-13)
    assert np.allclose(uR[ok], exact[ok], atol=1e-13)


def test_weno5_fifth_order_on_smooth_monotone_data():
    errs = []
    for n in (40, 80, 160):
        h = 0.5 / n
        edges = np.arange(n + 1) * h
        f = lambda x: np.sin(np.pi * x)  # monotone on [0, 0.5]
        F = lambda x: -np.cos(np.pi * x) / np.pi
        u = (F(edges[1:]) - F(edges[:-1])) / h
        uL, uR = oracle.recon_line(2, u)
        ok = ~np.isnan(uL)
        errs.append(np.abs(uL[ok] - f(edges[1:])[ok]).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > 4.5, (errs, rates)


def test_weno5_no_new_extrema_at_a_step():
    u = np.where(np.arange(20) < 10, 1.0, 0.0)
    uL, uR = oracle.recon_line(2, u)
    ok = ~np.isnan(uL)
    assert (uL[ok] >= -1e-6).all() and (uL[ok] <= 1 + 1e-6).all()
    assert (uR[ok] >= -1e-6).all() and (uR[ok] <= 1 + 1e-6).all()
    # upwind side is kept at the jump
    assert abs(uL[9] - 1.0) < 1e-6 and abs(uR[9]) < 1e-6


# ------------------------------------------------------------- implicit E

def _flat_implicit(Estar, B, v, cs):
    """Solve E - E* + cs W (E + v x B - (v.E) v) = 0 with numpy (flat)."""
    W = 1.0 / np.sqrt(1.0 - v @ v)
    C = cs * W
    M = (1.0 + C) * np.eye(3) - C * np.outer(v, v)
    return np.linalg.solve(M, Estar - C * np.cross(v, B))


@pytest.mark.parametrize("cs", [0.0, 0.3, 30.0, 3e5])
def test_implicit_E_matches_linear_solve_in_transformed_frame(cs):
    """Eq. 3D_NR: the oracle's Newton solve in a curved frame equals the
    numpy solution of the flat-space linear system, transformed."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        v = rng.standard_normal(3)
        v *= rng.uniform(0, 0.9) / np.linalg.norm(v)
        B, Estar = rng.standard_normal(3), rng.standard_normal(3)
        E = _flat_implicit(Estar, B, v, cs)
        A = fs.random_A(rng)
        g6, sg = fs.metric_of(A)
        alpha = rng.uniform(0.5, 1.5)
        c = 0.37
        sigma = cs / (alpha * c)      # proper-time coefficient alpha c sigma = cs
        J = np.linalg.det(A)
        Ex = oracle.implicit_E(A @ Estar / J, A @ B / J, A @ v, alpha, g6, sigma, c)
        assert np.allclose(Ex, A @ E / J, rtol=1e-12, atol=1e-12 * np.abs(A @ E / J).max())


def test_implicit_E_limits():
    rng = np.random.default_rng(12)
    v = np.array([0.3, -0.2, 0.5])
    B = rng.standard_normal(3)
    Estar = rng.standard_normal(3)
    # sigma = 0: no change
    assert np.array_equal(oracle.implicit_E(Estar, B, v, sigma=0.0, c=1.0), Estar)
    # ideal limit: E -> -v x B with an O(1/(c sigma)) remainder
    for cs in (1e6, 1e9):
        E = oracle.implicit_E(Estar, B, v, sigma=cs, c=1.0)
        assert np.abs(E + np.cross(v, B)).max() < 10.0 / cs


# ------------------------------------------------------------- recovery

def _manufactured(rng, gam_eos, cs, curved=True):
    """A known state and the stage input (D, S, tau, calB, calE*) whose joint
    implicit-E + recovery root it is.  For stiff coefficients the field is
    near-ideal, E = -v x B + O(1/cs), as it is after any stiff stage; with an
    O(1) non-ideal part at cs >> 1 the joint system has several roots."""
    prim = fs.random_flat_prim(rng, gam_eos, vmax=0.9)
    v, B = prim[2:5], prim[8:11]
    if cs > 10.0:
        prim[5:8] = -np.cross(v, B) + rng.standard_normal(3) * np.linalg.norm(B) / cs
    U, _ = fs.textbook(prim, gam_eos)
    E = prim[5:8]
    W = 1.0 / np.sqrt(1.0 - v @ v)
    # calE* such that calE is the implicit root: E* = E + cs W (E + vxB - (v.E)v)
    Estar = E + cs * W * (E + np.cross(v, B) - (v @ E) * v)
    A = fs.random_A(rng) if curved else np.eye(3)
    alpha = rng.uniform(0.5, 1.5) if curved else 1.0
    g6, _ = fs.metric_of(A)
    Ux = fs.transform_cons(U, A)
    J = np.linalg.det(A)
    Ustar = Ux.copy()
    Ustar[8:11] = A @ Estar / J
    return prim, A, alpha, g6, Ux, Ustar


@pytest.mark.parametrize("gam_eos", [2.0, 4.0 / 3.0])
def test_con2prim_round_trip_fixed_E(gam_eos):
    """Sec. III.B recovery with calE fixed inverts prim->con (1e-13)."""
    rng = np.random.default_rng(21)
    P = oracle.make_params(gamma_eos=gam_eos, rho_atmo=1e-14)
    for _ in range(300):
        prim, A, alpha, g6, Ux, _ = _manufactured(rng, gam_eos, 0.0)
        px = fs.transform_prim(prim, A)
        guess = px.copy()
        guess[1] *= 1.0 + 0.05 * rng.standard_normal()
        guess[2:5] *= 1.0 + 0.02 * rng.standard_normal()
        out, cout, it, st = oracle.con2prim(P, Ux, 0, 0.0, 0.0, guess, alpha, g6)
        assert st in (0, 1, 4)
        scale = np.abs(px).max()
        assert np.allclose(out, px, rtol=1e-12, atol=1e-12 * scale), (out - px, st, it)
        assert np.array_equal(cout, Ux)


@pytest.mark.parametrize("cs", [0.1, 10.0, 1e3, 1e6])
def test_con2prim_round_trip_implicit(cs):
    """Joint implicit-E + recovery (Sec. III.A-B): from (D, S, tau, calB,
    calE*) built around a known state, the recovery returns that state and its
    calE."""
    rng = np.random.default_rng(22)
    P = oracle.make_params(gamma_eos=2.0, rho_atmo=1e-14)
    fails = 0
    for _ in range(200):
        prim, A, alpha, g6, Ux, Ustar = _manufactured(rng, 2.0, cs)
        px = fs.transform_prim(prim, A)
        c = 0.25
        sigma = cs / (alpha * c)
        guess = px.copy()
        guess[1] *= 1.0 + 0.02 * rng.standard_normal()
        guess[2:5] *= 1.0 + 0.01 * rng.standard_normal()
        out, cout, it, st = oracle.con2prim(P, Ustar, 1, c, sigma, guess, alpha, g6)
        if st in (2, 3):
            fails += 1
            continue
        scale = np.abs(px).max()
        assert np.allclose(out, px, rtol=1e-11, atol=1e-11 * scale), (out - px, st, it)
        assert np.allclose(cout[8:11], Ux[8:11], rtol=1e-11, atol=1e-11 * np.abs(Ux).max())
    assert fails == 0


def test_con2prim_resets_unphysical_state_to_atmosphere():
    """A state with tau too small for its momentum has no root: the recovery
    reports failure and returns the atmosphere (rho_atmo, v = 0,
    p = K rho_atmo^Gamma) with calB kept."""
    P = oracle.make_params(gamma_eos=2.0, rho_atmo=1e-6, K_atmo=100.0)
    cons = np.zeros(14)
    cons[0], cons[1], cons[4] = 1.0, 5.0, 0.01
    cons[5] = 0.2
    guess = np.zeros(14)
    guess[0], guess[1] = 1.0, 1.0
    out, cout, it, st = oracle.con2prim(P, cons, 0, 0.0, 0.0, guess)
    assert st == 2
    assert out[0] == 1e-6 and out[1] == 100.0 * 1e-12 and not out[2:5].any()
    assert out[8] == 0.2
    assert cout[0] == 1e-6 and cout[1] == 0.0


def _hard_cases():
    import os
    d = np.load(os.path.join(os.path.dirname(__file__), "golden", "recovery_hard_cases.npz"))
    return {k: d[k] for k in d.files}


def test_pressure_bracket_recovers_states_where_newton_stalls():
    """Stage inputs from the magnetised blast front (tests/golden, written by
    make_recovery_cases.py from the oracle) on which the paper iteration and
    the kernel's 4D Newton fail: the bracket finds a root, checked independently by
    re-forming D, S_i, tau from the returned primitives and re-solving the
    implicit field (Eq. 3D_NR) at the returned velocity."""
    d = _hard_cases()
    gam = float(d["gamma_eos"])
    P = oracle.make_params(gamma_eos=gam, rho_atmo=1e-10)
    for i in range(d["cons"].shape[1]):
        cin, guess = d["cons"][:, i], d["guess"][:, i]
        out, cout, it, st = oracle.con2prim(P, cin, 1, float(d["c"]), float(d["sigma"]), guess)
        assert st == 4, st
        # the returned calE solves the stage equation at the returned v
        E = oracle.implicit_E(cin[8:11], cin[5:8], out[2:5], sigma=float(d["sigma"]),
                              c=float(d["c"]))
        assert np.allclose(E, cout[8:11], rtol=1e-12, atol=1e-15)
        # and prim -> con of the returned state gives back D, S_i, tau
        U = oracle.prim2con(out, 1.0, (0, 0, 0), (1, 0, 0, 1, 0, 1), gam)
        scale = cin[4] + cin[0] + out[1]
        assert np.abs(U[:5] - cin[:5]).max() < 1e-12 * scale


@pytest.mark.parametrize("D_over_floor", [0.5, 0.999])
def test_con2prim_density_below_the_floor_is_atmosphere_at_once(D_over_floor):
    """rho = D / (W sqrt(gamma)) <= D / sqrt(gamma): when D / sqrt(gamma) is
    below the floor rho_atmo (1 + atmo_tol) every root is below it, so the
    recovery returns the atmosphere without iterating (status 3, 0
    iterations), calE of the implicit solve at v = 0 = calE*/(1 + c alpha sigma)
    and calB kept; just above the floor it iterates as usual."""
    P = oracle.make_params(gamma_eos=2.0, rho_atmo=1e-6, K_atmo=100.0, atmo_tol=1e-2)
    g6 = (1.21, 0.0, 0.0, 1.21, 0.0, 1.21)       # sqrt(gamma) = 1.331
    sg = 1.331
    floor = 1e-6 * 1.01
    cons = np.zeros(14)
    cons[0] = D_over_floor * floor * sg
    cons[1], cons[4] = 1e-7, 2e-5
    cons[5], cons[8] = 0.02, 0.03
    guess = np.zeros(14)
    guess[0], guess[1] = 1e-6, 1e-10
    c, sigma, alpha = 0.05, 20.0, 0.9
    out, cout, it, st = oracle.con2prim(P, cons, 1, c, sigma, guess, alpha=alpha, g6=g6)
    assert st == 3 and it == 0
    assert out[0] == 1e-6 and out[1] == 100.0 * 1e-12 and not out[2:5].any()
    assert abs(cout[8] - 0.03 / (1.0 + c * alpha * sigma)) <= 1e-15
    assert abs(out[8] - 0.02 / sg) <= 1e-15
    # above the floor the same state is iterated (it need not converge)
    cons[0] = 1.5 * floor * sg
    _, _, it2, st2 = oracle.con2prim(P, cons, 1, c, sigma, guess, alpha=alpha, g6=g6)
    assert it2 > 0
