"""Pins of the oracle's whole-step behaviour (CPU only): closed forms,
invariants and the paper's analytic test solutions."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

G_IMEX = 1.0 - 1.0 / math.sqrt(2.0)


def _metric(wl):
    a, b, g, K = wl.metric_arrays()
    return oracle.Metric(a.ravel(), b.reshape(3, -1), g.reshape(6, -1), K.reshape(6, -1))


def _init(wl):
    m = _metric(wl)
    prim = np.ascontiguousarray(wl.prim.copy())
    cons = oracle.prim2con_grid(wl.params, m, prim)
    return m, prim, cons


def _run(wl, nsteps, dt=None):
    m, prim, cons = _init(wl)
    sf = None if wl.sigma_profile is None else wl.sigma_profile.ravel()
    st, stats = oracle.step(wl.params, m, cons, prim, wl.dt if dt is None else dt,
                            nsteps, sigma_field=sf)
    return st, stats, prim, cons


def _uniform(n, prim0, sigma, gamma_eos=2.0, bc=0):
    P = W.base_params((n, 1, 1), (0, 0, 0), (0.1, 0.1, 0.1), (bc, bc, bc), "mc2",
                      gamma_eos, sigma)
    prim = np.zeros((14, 1, 1, n))
    prim[:] = np.asarray(prim0)[:, None, None, None]
    return W.Workload("uniform", P, prim, 0.05, 1)


def imex_amplification(z):
    """IMEX-SSP2(2,2,2) (Table imex) applied to dE/dt = -lambda E, z = lambda dt."""
    e1 = 1.0 / (1.0 + G_IMEX * z)
    e2 = (1.0 - (1.0 - 2.0 * G_IMEX) * z * e1) / (1.0 + G_IMEX * z)
    return 1.0 - 0.5 * z * (e1 + e2)


@pytest.mark.parametrize("z", [1e-3, 0.1, 1.0, 10.0, 1e3, 1e6])
def test_imex_stages_reproduce_closed_form_relaxation(z):
    """Uniform state at rest with E parallel to B: only the stiff term acts,
    dcalE/dt = -sigma calE, so one step multiplies calE by R(z) exactly, while
    D, S_i, tau stay fixed (energy moves from the field to the fluid)."""
    prim0 = np.zeros(14)
    prim0[0], prim0[1] = 1.0, 1.0
    prim0[5:8] = [0.06, 0.08, 0.0]
    prim0[8:11] = [0.3, 0.4, 0.0]
    wl = _uniform(4, prim0, sigma=z / 0.05)
    m, prim, cons = _init(wl)
    c0 = cons.copy()
    st, _ = oracle.step(wl.params, m, cons, prim, 0.05, 1)
    assert st == 0
    R = imex_amplification(z)
    assert np.allclose(cons[8:11], R * c0[8:11], rtol=1e-13, atol=1e-16)
    for f in (0, 1, 2, 3, 4):
        assert np.allclose(cons[f], c0[f], rtol=1e-14, atol=1e-16)
    assert (prim[1] > 1.0).all() or z < 1e-2      # Ohmic heating


@pytest.mark.parametrize("model,extra,factor", [
    (2, dict(sigma_exp=0.5), 2.0),                 # sigma0 D^(1/2), D = 4
    (2, dict(sigma_exp=-1.0), 0.25),               # sigma0 / D
    (3, dict(D_atmo=1.0), 0.5625),                 # sigma0 (1 - 1/4)^2
    (3, dict(D_atmo=8.0), 0.0),                    # D below D_atmo: no conduction
])
def test_density_dependent_conductivity_closed_form(model, extra, factor):
    """Conductivity models of Eqs. sigma_evol and dynamo_sigma on a uniform
    state at rest with D = rho = 4: the stiff relaxation of calE is the
    closed form above with sigma = factor * sigma0."""
    prim0 = np.zeros(14)
    prim0[0], prim0[1] = 4.0, 1.0
    prim0[5:8] = [0.06, 0.08, 0.0]
    prim0[8:11] = [0.3, 0.4, 0.0]
    sigma0, dt = 40.0, 0.05
    wl = _uniform(4, prim0, sigma=sigma0)
    wl.params.update(sigma_model=model, **extra)
    m, prim, cons = _init(wl)
    c0 = cons.copy()
    st, _ = oracle.step(wl.params, m, cons, prim, dt, 1)
    assert st == 0
    R = imex_amplification(factor * sigma0 * dt)
    assert np.allclose(cons[8:11], R * c0[8:11], rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("model,extra", [(2, dict(sigma_exp=0.7)), (3, dict(D_atmo=1.3))])
def test_density_dependent_conductivity_uses_conserved_density(model, extra):
    """A uniform flow keeps D = rho W uniform for the whole step, so the
    density-dependent models must equal the uniform model with sigma0
    replaced by its value at that D (computed here from rho and v); rho in
    place of D would change sigma by W^0.7 or through D_atmo/D."""
    prim0 = np.zeros(14)
    prim0[0], prim0[1] = 2.0, 0.5
    prim0[2:5] = [0.3, -0.2, 0.4]
    prim0[5:8] = [0.05, 0.02, -0.03]
    prim0[8:11] = [0.2, 0.3, -0.1]
    W_lor = 1.0 / math.sqrt(1.0 - float(np.dot(prim0[2:5], prim0[2:5])))
    D = prim0[0] * W_lor
    sigma0, dt = 30.0, 0.05
    if model == 2:
        sig = sigma0 * D ** extra["sigma_exp"]
    else:
        sig = sigma0 * (1.0 - extra["D_atmo"] / D) ** 2
    out = []
    for params in (dict(sigma_model=model, **extra), dict(sigma_model=0, sigma0=sig)):
        wl = _uniform(4, prim0, sigma=sigma0)
        wl.params.update(params)
        m, prim, cons = _init(wl)
        st, _ = oracle.step(wl.params, m, cons, prim, dt, 1)
        assert st == 0
        out.append(cons.copy())
    assert np.allclose(out[0], out[1], rtol=1e-12, atol=1e-15)
    # and sigma matters here: the unscaled uniform model differs
    wl = _uniform(4, prim0, sigma=sigma0)
    m, prim, cons = _init(wl)
    oracle.step(wl.params, m, cons, prim, dt, 1)
    assert not np.allclose(out[0][8:11], cons[8:11], rtol=1e-6)


def test_imex_amplification_is_second_order_and_l_stable():
    for z in (1e-2, 5e-3):
        assert abs(imex_amplification(z) - math.exp(-z)) < 0.1 * z ** 3
    assert abs(imex_amplification(1e12)) < 1e-11


def _smooth_periodic(n, recon, sigma, seed=3):
    rng = np.random.default_rng(seed)
    P = W.base_params((n, n, n), (0, 0, 0), (1.0 / n,) * 3, (0, 0, 0), recon, 5.0 / 3.0,
                      sigma)
    X, Y, Z = W.cell_centres(P["n"], P["x0"], P["dx"])
    prim = np.zeros((14,) + X.shape)
    tp = 2 * np.pi

    def wave(a):
        k = rng.integers(1, 3, 3)
        ph = rng.uniform(0, tp)
        return a * np.sin(tp * (k[0] * X + k[1] * Y + k[2] * Z) + ph)

    prim[0] = 1.0 + wave(0.2)
    prim[1] = 0.5 + wave(0.1)
    for i in range(3):
        prim[2 + i] = wave(0.2)
        prim[5 + i] = wave(0.1)
        prim[8 + i] = 0.5 + wave(0.2)
    prim[11] = wave(0.01)
    prim[12] = wave(0.01)
    prim[13] = wave(0.05)
    return W.Workload("smooth", P, prim, 0.25 / n, 1)


@pytest.mark.parametrize("recon", ["minmod", "mc2", "weno5"])
def test_conservation_periodic_flat(recon):
    """Flat periodic grid: D, S_i, tau, calB^i and Q have no source terms in
    Eq. GRRMHD_flux_form, so their totals are conserved to rounding."""
    wl = _smooth_periodic(8, recon, sigma=50.0)
    m, prim, cons = _init(wl)
    tot0 = cons.reshape(14, -1).sum(axis=1)
    st, stats = oracle.step(wl.params, m, cons, prim, wl.dt, 2)
    assert st == 0 and stats["c2p_failures"] == 0
    tot1 = cons.reshape(14, -1).sum(axis=1)
    scale = np.abs(cons).reshape(14, -1).sum(axis=1)
    for f in (0, 1, 2, 3, 4, 5, 6, 7, 13):
        assert abs(tot1[f] - tot0[f]) < 1e-13 * scale[f], (f, tot1[f] - tot0[f])


def _pressure_only_curved(n):
    """Fluid at rest, uniform p, alpha = 1, beta = 0, K = 0, conformally flat
    gamma_ij = psi4 delta_ij varying along x."""
    dx = 1.0 / n
    P = W.base_params((n, 1, 1), (0, 0, 0), (dx, dx, dx), (0, 0, 0), "mc2", 2.0, 0.0)
    x = (np.arange(n) + 0.5) * dx
    psi4 = 1.0 + 0.3 * np.sin(2 * np.pi * x)
    g = np.zeros((6, 1, 1, n))
    g[0] = g[3] = g[5] = psi4
    prim = np.zeros((14, 1, 1, n))
    prim[0], prim[1] = 1.0, 0.8
    wl = W.Workload("pconst", P, prim, 0.1 * dx, 1, alpha=np.ones((1, 1, n)),
                    beta=np.zeros((3, 1, 1, n)), gamma=g, K=np.zeros((6, 1, 1, n)))
    return wl


def test_static_pressure_in_curved_space_is_balanced_to_second_order():
    """With the undensitised stress, -d_k(alpha sqrt(g) p delta^k_i) +
    (alpha sqrt(g)/2) p gamma^{jk} d_i gamma_jk vanishes in the continuum
    (d_i sqrt(g) = sqrt(g)/2 gamma^{jk} d_i gamma_jk); the discrete residual is
    O(dx^2).  D and tau have exactly zero right-hand side."""
    errs = []
    for n in (16, 32, 64):
        wl = _pressure_only_curved(n)
        m, prim, cons = _init(wl)
        r = oracle.rhs(wl.params, m, prim)
        assert np.abs(r[0]).max() == 0.0 and np.abs(r[4]).max() < 1e-14
        errs.append(np.abs(r[1]).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[0] < 0.05 and rates.min() > 1.8, (errs, rates)


def test_zero_conductivity_decouples_fields_from_fluid():
    """sigma = 0, Q = 0: E, B, Phi, Psi follow vacuum Maxwell whatever the
    fluid does (Sec. IV.A, sigma0 = 0 limit)."""
    wl1 = _smooth_periodic(6, "mc2", sigma=0.0, seed=5)
    wl1.prim[13] = 0.0
    wl2 = _smooth_periodic(6, "mc2", sigma=0.0, seed=5)
    wl2.prim[13] = 0.0
    wl2.prim[0] *= 1.5
    wl2.prim[2:5] *= -0.5
    outs = []
    for wl in (wl1, wl2):
        st, _, prim, cons = _run(wl, 3)
        assert st == 0
        outs.append(cons)
    for f in (5, 6, 7, 8, 9, 10, 11, 12, 13):
        assert np.array_equal(outs[0][f], outs[1][f]), f


def test_current_sheet_follows_resistive_diffusion():
    """Sec. IV.C: B^y(x, t) = B0 erf(x sqrt(sigma)/(2 sqrt(t))), sigma = 100,
    p = 50, rho = 1, minmod, outflow; from t = 1 to t = 2.  The error shrinks
    with resolution."""
    errs = []
    for n in (60, 120):
        wl = W.current_sheet(n=n)
        nsteps = int(round(1.0 / wl.dt))
        st, _, prim, _ = _run(wl, nsteps)
        assert st == 0
        x = wl.params["x0"][0] + (np.arange(n) + 0.5) * wl.params["dx"][0]
        exact = np.array([math.erf(xx * 10.0 / (2.0 * math.sqrt(2.0))) for xx in x])
        errs.append(np.abs(prim[9, 0, 0] - exact).max())
    assert errs[1] < 0.02 and errs[1] < 0.6 * errs[0], errs


def test_alfven_wave_returns_after_one_period():
    """Sec. IV.D: sigma = 1e6, MC2, periodic; after t = L/v_A = 2 the wave is
    back; the error against the initial data shrinks with resolution."""
    errs = []
    for n in (32, 64):
        wl = W.alfven_1d(n=n)
        assert abs(wl.extra["vA"] - 0.5) < 1e-4
        st, _, prim, _ = _run(wl, wl.nsteps)
        assert st == 0
        errs.append(np.abs(prim[9] - wl.prim[9]).mean())
    assert errs[1] < 0.5 * errs[0] and errs[1] < 0.1, errs


def test_ideal_limit_after_the_implicit_stage():
    """Large sigma: the implicit stage solved jointly with the recovery puts
    the field on the ideal-MHD manifold, E + v x B = O(1/(sigma dt))
    (Sec. II.D: Ohm's law recovers ideal MHD as sigma grows)."""
    res = []
    for sigma in (1e4, 1e6):
        wl = W.alfven_1d(n=32, sigma=sigma)
        st, _, prim, cons = _run(wl, 2)
        P = oracle.make_params(**wl.params)
        worst = 0.0
        for i in range(32):
            out, _, _, s = oracle.con2prim(P, cons[:, 0, 0, i], 1, G_IMEX * wl.dt, sigma,
                                           prim[:, 0, 0, i])
            assert s in (0, 1, 4)
            v, E, B = out[2:5], out[5:8], out[8:11]
            worst = max(worst, np.abs(E + np.cross(v, B)).max())
        res.append(worst)
    assert res[1] < 1e-4 and res[1] < 0.02 * res[0], res


def test_literal_face_ohm_current_is_stiff_in_the_charge_flux():
    """Evidence for the reading of the charge flux: evaluating Ohm's law at
    the reconstructed face states makes Q grow in proportion to sigma (here
    the smooth Alfven wave), while the stage current keeps it bounded."""
    qmax = {}
    for mode in (0, 1):
        for sigma in (1e2, 1e6):
            wl = W.alfven_1d(n=32, sigma=sigma)
            wl.params["qflux_mode"] = mode
            st, _, prim, _ = _run(wl, 3)
            qmax[mode, sigma] = np.abs(prim[13]).max()
    assert qmax[1, 1e6] > 1e3 * qmax[1, 1e2]
    assert qmax[0, 1e6] < 0.02 and qmax[0, 1e2] < 0.02, qmax


@pytest.mark.parametrize("curved", [False, True])
def test_gauss_law_charge_converges_to_evolved_charge(curved):
    """Charge from Gauss's law (the Sec. IV.E variant) against the evolved
    charge: on data that satisfy the constraint q = nabla_i E^i, Ampere's law
    and charge conservation keep it satisfied, so the two runs agree in the
    continuum and their difference must shrink at second order.  A missing
    sqrt(gamma), a sign or a factor in the Gauss charge would leave an O(1)
    difference (the curved case has E . grad ln sqrt(gamma) ~ q)."""
    d = []
    for n in (32, 64):
        runs = []
        for mode in (0, 2):
            wl = W.gauss_smooth(n, curved, mode)
            nsteps = int(round(0.25 / wl.dt))
            st, _, prim, cons = _run(wl, nsteps)
            assert st == 0
            runs.append(prim)
        d.append(np.abs(runs[0][13] - runs[1][13]).mean() / np.abs(runs[0][13]).mean())
    assert d[1] < 0.03 and d[0] / d[1] > 3.0, d


def test_gauss_law_charge_totals_vanish_on_a_periodic_grid():
    """sum_cells d_i calE^i telescopes to zero on a periodic grid."""
    wl = W.gauss_smooth(16, True, 2)
    st, _, prim, cons = _run(wl, 3)
    assert st == 0
    assert abs(cons[13].sum()) < 1e-13 * np.abs(cons[13]).sum()


def test_z_uniform_blast_equals_its_plane():
    """The cylindrical explosion does not depend on z and has outflow faces:
    the z-face fluxes of identical neighbours are identical, their difference
    is exactly zero, so every z-layer of a 3D run equals the 2D run of one
    layer bit for bit (used to check the 64^3 configuration against a 64^2
    oracle run for its 100 steps)."""
    import workloads as W
    from tests.helpers import run_oracle
    _, _, p3, c3 = run_oracle(W.cyl_blast(n=12, nz=5), 4)
    _, _, p2, c2 = run_oracle(W.cyl_blast(n=12, nz=1), 4)
    for k in range(5):
        assert np.array_equal(c3[:, k], c2[:, 0]) and np.array_equal(p3[:, k], p2[:, 0])
