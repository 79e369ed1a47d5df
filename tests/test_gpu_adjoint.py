"""The discrete adjoint (rmhd_adjoint_forward / rmhd_adjoint_backward)
against central finite differences of the oracle's step and against the
oracle's FP64 tangent-linear model (oracle.tangent_step).

Loss L = sum_cells (B^y(t_N) - B^y_target)^2 dx^3 of the primitives after N
steps; dL/dP^N = 2 (B^y - B^y_target) dx^3 in the B^y row.  The adjoint's
<dL/dP^0, u> for seeded smooth directions u (a relative change of about h
in every field) and dL/dlog sigma0 are compared with central differences
computed by the oracle alone, to 1e-6 relative.  The differences are
Richardson-extrapolated over h = 1e-6 and h/2: the WENO5 weights (epsilon =
1e-6) make the third derivatives large enough that a plain central
difference at h = 1e-6 is off by up to ~1e-4; the extrapolated one is not.
TVD limiters are checked on curved states where no neighbouring
difference comes near zero: at a limiter kink a central difference is not
the derivative of the branch the step takes (and that the adjoint takes)."""
import numpy as np
import pytest

import workloads as W
from tests.helpers import make_solver, oracle_metric

pytestmark = pytest.mark.gpu

import oracle

H = 1e-6
TOL = 1e-6


def _oracle_final(wl, prim0, nsteps, sigma0=None):
    P = dict(wl.params)
    if sigma0 is not None:
        P["sigma0"] = sigma0
    m = oracle_metric(wl)
    prim = np.ascontiguousarray(prim0.copy())
    cons = oracle.prim2con_grid(P, m, prim)
    sf = None if wl.sigma_profile is None else wl.sigma_profile.ravel()
    st, _ = oracle.step(P, m, cons, prim, wl.dt, nsteps, sigma_field=sf)
    assert st == 0
    return prim


def _loss(prim, target, dV):
    return float(np.sum((prim[9] - target) ** 2) * dV)


def _smooth_modes(shape, rng, kmax=2, kmin=0):
    """A seeded smooth field: a few random low Fourier modes on the grid
    (wavenumbers kmin..kmax along every active axis)."""
    nz, ny, nx = shape
    z, y, x = [(np.arange(n) + 0.5) / n for n in (nz, ny, nx)]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    out = np.zeros(shape)
    for _ in range(4):
        k = rng.integers(kmin, kmax + 1, 3) * np.array([nz > 1, ny > 1, nx > 1])
        ph = rng.uniform(0, 2 * np.pi)
        out += rng.standard_normal() * np.sin(2 * np.pi * (k[0] * Z + k[1] * Y + k[2] * X) + ph)
    return out


def _directions(prim0, rng, ndir):
    """Seeded smooth directions, each field scaled to its local magnitude
    (so that h u is a relative change of about h everywhere): the first
    ones confined to one field group, the rest on all 14 fields."""
    groups = [(0, 2), (2, 5), (5, 11), (11, 14)]
    mag = np.abs(prim0) + 0.01 * np.abs(prim0).reshape(14, -1).max(axis=1)[:, None, None, None]
    mag += 1e-3 * np.abs(prim0[8:11]).max()
    dirs = []
    for q in range(ndir):
        u = np.stack([_smooth_modes(prim0.shape[1:], rng) for _ in range(14)]) * mag
        if q < len(groups):
            keep = np.zeros(14, bool)
            keep[groups[q][0]:groups[q][1]] = True
            u[~keep] = 0.0
        dirs.append(u)
    return dirs


def _generic_smooth(curved, recon="mc2"):
    """2D periodic state on which every field varies along both axes, so that
    no neighbouring difference vanishes: the TVD limiters have a kink there,
    where a central difference is not the derivative of the frozen branch."""
    wl = W.gauss_smooth(12, curved=curved, qflux_mode=0)
    rng = np.random.default_rng(23)
    amp = {0: 0.1, 1: 0.1, 2: 0.05, 3: 0.05, 4: 0.05, 5: 0.01, 6: 0.01, 7: 0.01, 8: 0.05,
           9: 0.05, 10: 0.05, 11: 0.01, 12: 0.01, 13: 0.01}
    for f, a in amp.items():
        wl.prim[f] += a * _smooth_modes(wl.shape, rng, kmax=2, kmin=1)
    wl.params["recon"] = W.RECON[recon]
    return wl


def _general_metric(recon):
    """The generic 2D state on a smooth static metric with lapse, shift,
    off-diagonal gamma_ij and K_ij (every metric term of the flux and the
    sources is exercised)."""
    wl = _generic_smooth(False, recon)
    rng = np.random.default_rng(31)
    shp = wl.shape
    alpha = 1.0 + 0.1 * _smooth_modes(shp, rng, kmax=1)
    beta = np.stack([0.05 * _smooth_modes(shp, rng, kmax=1) for _ in range(3)])
    gamma = np.zeros((6,) + shp)
    for a, diag in enumerate((True, False, False, True, False, True)):
        gamma[a] = (1.0 if diag else 0.0) + 0.05 * _smooth_modes(shp, rng, kmax=1)
    K = np.stack([0.02 * _smooth_modes(shp, rng, kmax=1) for _ in range(6)])
    wl.alpha, wl.beta, wl.gamma, wl.K = alpha, beta, gamma, K
    return wl


def _blast_weno5():
    wl = W.cyl_blast(n=16, nz=1, L=1.5)
    wl.params["recon"] = W.RECON["weno5"]
    return wl


CASES = {
    # smooth periodic wave, WENO5, the stiff and the resistive regimes
    "alfven_s1e3": lambda: W.alfven_diag(n=8, sigma=1e3),
    "alfven_s10": lambda: W.alfven_diag(n=8, sigma=10.0),
    # MC2 on flat and curved static metrics
    "generic_mc2_flat": lambda: _generic_smooth(False),
    "generic_mc2_curved": lambda: _generic_smooth(True),
    # minmod, curved
    "generic_minmod_curved": lambda: _generic_smooth(True, "minmod"),
    # outflow boundaries, blast profile, WENO5
    "blast_weno5": _blast_weno5,
    # lapse, shift, off-diagonal 3-metric, extrinsic curvature
    "general_metric_weno5": lambda: _general_metric("weno5"),
    "general_metric_mc2": lambda: _general_metric("mc2"),
    # conductivity models: sigma0 x profile, sigma0 D^(1/2), sigma0 (1 - D_atmo/D)^2
    "sigma_profile": lambda: _with_sigma(_generic_smooth(True, "weno5"), 1),
    "sigma_powD": lambda: _with_sigma(_generic_smooth(True, "weno5"), 2, sigma_exp=0.5),
    "sigma_atmo": lambda: _with_sigma(_generic_smooth(True, "weno5"), 3, D_atmo=0.3),
}


def _with_sigma(wl, model, **extra):
    wl.params.update(sigma_model=model, **extra)
    if model == 1:
        rng = np.random.default_rng(41)
        wl.sigma_profile = 1.0 + 0.5 * np.tanh(_smooth_modes(wl.shape, rng, kmax=1))
    return wl


@pytest.mark.parametrize("name,nsteps,every", [("alfven_s1e3", 6, 4), ("alfven_s10", 6, 2),
                                               ("generic_mc2_curved", 5, 3),
                                               ("generic_minmod_curved", 4, 1),
                                               ("blast_weno5", 4, 3),
                                               ("general_metric_weno5", 4, 2),
                                               ("general_metric_mc2", 4, 2),
                                               ("sigma_profile", 4, 2), ("sigma_powD", 4, 2),
                                               ("sigma_atmo", 4, 2)])
def test_adjoint_matches_oracle_finite_differences(name, nsteps, every):
    wl = CASES[name]()
    dx = wl.params["dx"]
    dV = dx[0] * dx[1] * dx[2]
    rng = np.random.default_rng(17)
    prim0 = wl.prim
    target = np.roll(prim0[9], 1, axis=-1) * 0.9
    s = make_solver(wl)
    s.adjoint_forward(wl.dt, nsteps, every)
    PN = s.get_prims()
    lam = np.zeros_like(PN)
    lam[9] = 2.0 * (PN[9] - target) * dV
    grad, gls = s.adjoint_backward(np.ascontiguousarray(lam))
    # the recording is reusable: a second backward gives the same result
    grad2, gls2 = s.adjoint_backward(np.ascontiguousarray(lam))
    s.close()
    assert np.isfinite(grad).all()
    # fixed summation order: bit for bit
    assert np.array_equal(grad2, grad) and gls2 == gls

    adj, fd = [], []
    for u in _directions(prim0, rng, 8):
        fd.append(_richardson(lambda h: _loss(_oracle_final(wl, prim0 + h * u, nsteps),
                                              target, dV)))
        adj.append(float(np.sum(grad * u)))
    adj, fd = np.array(adj), np.array(fd)
    # each direction relative to its own derivative, but at least to 1e-2 of
    # the largest: the oracle's extrapolated differences carry an absolute
    # error of ~1e-12 (its recovery stops at a tolerance of 1e-14 on the
    # change of the iterate, divided by h = 1e-6), which is 1e-6 of a
    # directional derivative a thousand times smaller than the largest one
    rel = np.abs(adj - fd) / np.maximum(np.abs(fd), 1e-2 * np.abs(fd).max())
    print(name, "directional derivatives: adjoint vs oracle FD, max rel", rel.max())
    assert rel.max() < TOL, (name, adj, fd, rel)

    s0 = wl.params["sigma0"]
    fds = _richardson(lambda h: _loss(_oracle_final(wl, prim0, nsteps, s0 * np.exp(h)),
                                      target, dV))
    print(name, "dL/dlog sigma0: adjoint", gls, "oracle FD", fds)
    assert abs(gls - fds) <= TOL * abs(fds), (name, gls, fds)


def _richardson(L, h=H):
    """(4 D(h/2) - D(h)) / 3 with D the central difference of L at 0."""
    d1 = (L(h) - L(-h)) / (2 * h)
    d2 = (L(h / 2) - L(-h / 2)) / h
    return (4.0 * d2 - d1) / 3.0


def test_flat_kernels_and_identity_metric_give_the_same_adjoint():
    """The flat specialisation against the general kernels on the identity
    metric: same trajectory, same gradient up to rounding (this also covers
    flat TVD states, where limiter kinks make finite differences useless)."""
    wl = CASES["generic_mc2_flat"]()
    dx = wl.params["dx"]
    dV = dx[0] * dx[1] * dx[2]
    target = np.roll(wl.prim[9], 1, axis=-1) * 0.9
    out = []
    for identity in (False, True):
        s = make_solver(wl)
        if identity:
            shp = wl.shape
            g = np.zeros((6,) + shp)
            g[0] = g[3] = g[5] = 1.0
            s.set_metric(np.ones(shp), np.zeros((3,) + shp), g, np.zeros((6,) + shp))
            s.set_prims(np.ascontiguousarray(wl.prim))
        s.adjoint_forward(wl.dt, 5, 2)
        PN = s.get_prims()
        lam = np.zeros_like(PN)
        lam[9] = 2.0 * (PN[9] - target) * dV
        out.append((PN,) + s.adjoint_backward(lam))
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.abs(out[0][1] - out[1][1]).max() <= 1e-13 * np.abs(out[1][1]).max()
    assert abs(out[0][2] - out[1][2]) <= 1e-13 * abs(out[1][2])


def test_adjoint_of_the_resistive_alfven_inverse_problem():
    """The spec style check on the GPU alone: 32^3 Alfven cube, WENO5,
    sigma = 1e3, 60 steps with checkpoints every 10, target B^y from the same
    initial data evolved with sigma = 2e3; 32 seeded directions and
    d/dlog sigma0 against Richardson central differences of rmhd_step."""
    wl = W.alfven_diag(n=32, sigma=1e3)
    nsteps = 60
    dx = wl.params["dx"]
    dV = dx[0] * dx[1] * dx[2]
    s = make_solver(wl, sigma0=2e3)
    s.step(wl.dt, nsteps)
    target = s.get_prims()[9].copy()
    s.close()

    def L(prim0, sigma0=1e3):
        sv = make_solver(wl, sigma0=sigma0)
        sv.set_prims(np.ascontiguousarray(prim0))
        sv.step(wl.dt, nsteps)
        p = sv.get_prims()
        sv.close()
        return _loss(p, target, dV)

    s = make_solver(wl)
    s.adjoint_forward(wl.dt, nsteps, 10)
    PN = s.get_prims()
    lam = np.zeros_like(PN)
    lam[9] = 2.0 * (PN[9] - target) * dV
    grad, gls = s.adjoint_backward(lam)
    s.close()
    rng = np.random.default_rng(2510)
    adj, fd = [], []
    for u in _directions(wl.prim, rng, 32):
        fd.append(_richardson(lambda h: L(wl.prim + h * u)))
        adj.append(float(np.sum(grad * u)))
    adj, fd = np.array(adj), np.array(fd)
    # each direction relative to its own derivative, but at least to 1e-2 of
    # the largest: the oracle's extrapolated differences carry an absolute
    # error of ~1e-12 (its recovery stops at a tolerance of 1e-14 on the
    # change of the iterate, divided by h = 1e-6), which is 1e-6 of a
    # directional derivative a thousand times smaller than the largest one
    rel = np.abs(adj - fd) / np.maximum(np.abs(fd), 1e-2 * np.abs(fd).max())
    fds = _richardson(lambda h: L(wl.prim, 1e3 * np.exp(h)))
    print("32^3 Alfven, 60 steps: max rel over 32 directions", rel.max(),
          "dL/dlog sigma0", gls, fds)
    assert rel.max() < TOL, (adj, fd, rel)
    assert abs(gls - fds) <= TOL * abs(fds)


def test_adjoint_matches_the_oracle_tangent_linear():
    """The adjoint inverse problem's setup (Alfven cube, WENO5, sigma = 1e3,
    60 steps with checkpoints every 10, loss = sum (B^y - B^y_target)^2 dx^3,
    target from the same initial data at sigma = 2e3) on a 16^3 grid, against
    the oracle's own FP64 tangent-linear model (oracle.tangent_step: forward-
    mode differentiation of the oracle's step): the adjoint's <dL/dP^0, u>
    for six seeded smooth directions and dL/dlog sigma0 equal
    <dL/dP^N, dP^N(u)> of the tangent-linear run, within 1e-6.  The target
    and the loss's dL/dP^N are the oracle's own."""
    wl = W.alfven_diag(n=16, sigma=1e3)
    nsteps = 60
    dx = wl.params["dx"]
    dV = dx[0] * dx[1] * dx[2]
    target = _oracle_final(wl, wl.prim, nsteps, sigma0=2e3)[9]
    s = make_solver(wl)
    s.adjoint_forward(wl.dt, nsteps, 10)
    PN = s.get_prims()
    lam = np.zeros_like(PN)
    lam[9] = 2.0 * (PN[9] - target) * dV
    grad, gls = s.adjoint_backward(lam)
    s.close()
    m = oracle_metric(wl)
    rng = np.random.default_rng(2510)
    adj, tlm = [], []
    for u in _directions(wl.prim, rng, 6):
        st, _, pN, dpN = oracle.tangent_step(wl.params, m, wl.prim, u, wl.dt, nsteps)
        assert st == 0
        tlm.append(float(np.sum(2.0 * (pN[9] - target) * dV * dpN[9])))
        adj.append(float(np.sum(grad * u)))
    adj, tlm = np.array(adj), np.array(tlm)
    rel = np.abs(adj - tlm) / np.maximum(np.abs(tlm), 1e-2 * np.abs(tlm).max())
    st, _, pN, ds = oracle.tangent_step(wl.params, m, wl.prim, np.zeros_like(wl.prim), wl.dt,
                                        nsteps, dlog_sigma0=1.0)
    tls = float(np.sum(2.0 * (pN[9] - target) * dV * ds[9]))
    print("16^3 Alfven, 60 steps: adjoint vs oracle tangent-linear, max rel", rel.max(),
          "dL/dlog sigma0", gls, tls)
    assert rel.max() < TOL, (adj, tlm, rel)
    assert abs(gls - tls) <= TOL * abs(tls), (gls, tls)


def test_adjoint_leaves_the_state_and_rejects_unsupported_paths():
    wl = W.alfven_diag(n=8, sigma=1e3)
    s = make_solver(wl)
    s.adjoint_forward(wl.dt, 3, 2)
    p_fwd = s.get_prims()
    s.adjoint_backward(np.zeros((14,) + wl.shape))
    assert np.array_equal(s.get_prims(), p_fwd)
    s.close()
    import paper_2510_18968_b300 as R
    for over in (dict(precision=1), dict(qflux_mode=1)):
        s = make_solver(wl, **over)
        with pytest.raises(R.RMHDError):
            s.adjoint_forward(wl.dt, 2, 1)
        s.close()
    s = make_solver(wl)
    with pytest.raises(R.RMHDError):
        s.adjoint_backward(np.zeros((14,) + wl.shape))
    s.close()


def test_autograd_function_gives_the_adjoint_gradient():
    import torch
    import paper_2510_18968_b300 as R
    wl = W.alfven_diag(n=8, sigma=1e3)
    s = make_solver(wl)
    P0 = torch.tensor(wl.prim, dtype=torch.float64, device="cuda", requires_grad=True)
    ls = torch.tensor(np.log(wl.params["sigma0"]), dtype=torch.float64, requires_grad=True)
    PN = R.evolve_function().apply(P0, ls, s, wl.dt, 4, 2)
    loss = (PN[9] ** 2).sum()
    loss.backward()
    lam = np.zeros((14,) + wl.shape)
    lam[9] = 2.0 * PN[9].detach().cpu().numpy()
    g, gls = s.adjoint_backward(lam)
    s.close()
    assert np.abs(P0.grad.cpu().numpy() - g).max() <= 1e-12 * np.abs(g).max()
    assert abs(float(ls.grad) - gls) <= 1e-12 * abs(gls)


def test_full_tape_gives_the_same_gradient_bit_for_bit():
    """checkpoint_every = 0 keeps every step's states instead of re-running
    segments; the reverse sweep sees the same states, so the gradient is
    identical."""
    wl = W.alfven_diag(n=8, sigma=1e3)
    dV = np.prod(wl.params["dx"])
    out = []
    for every in (0, 3, 1):
        s = make_solver(wl)
        s.adjoint_forward(wl.dt, 7, every)
        PN = s.get_prims()
        lam = np.zeros_like(PN)
        lam[9] = 2.0 * PN[9] * dV
        out.append(s.adjoint_backward(lam))
        s.close()
    for g, ls in out[1:]:
        assert np.array_equal(g, out[0][0]) and ls == out[0][1]
