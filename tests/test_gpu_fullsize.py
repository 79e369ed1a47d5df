"""Parity at the full benchmark sizes, in the benchmark's launch configuration.

The oracle cannot step a 256^3 grid in seconds, but one step of a cell only
depends on the cells within two reconstruction stencils (one per explicit
stage; the recoveries are pointwise).  So for sampled cells the oracle runs
the same step on a small box cut around the cell (wide enough that its
boundary is outside that range of dependence) and its centre must equal the
GPU result of the full-size run."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.helpers import make_solver, state_error

pytestmark = pytest.mark.gpu

RADIUS = {0: 2, 1: 2, 2: 3}   # cells one explicit stage reaches, per reconstruction


def _cut(a, centre, half, periodic):
    """Box of a (..., nz, ny, nx) around centre = (k, j, i)."""
    idx = []
    for d, c in enumerate(centre):
        n = a.shape[-3 + d]
        r = np.arange(c - half, c + half + 1)
        idx.append(np.mod(r, n) if periodic else r)
    return a[..., idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :]]


def _oracle_centre(wl, centre, half):
    periodic = wl.params["bc"][0] == W.BC_PERIODIC
    prim = np.ascontiguousarray(_cut(wl.prim, centre, half, periodic))
    a, b, g, K = wl.metric_arrays()
    sub = dict(wl.params, n=(2 * half + 1,) * 3)
    m = oracle.Metric(_cut(a, centre, half, periodic).ravel(),
                      _cut(b, centre, half, periodic).reshape(3, -1),
                      _cut(g, centre, half, periodic).reshape(6, -1),
                      _cut(K, centre, half, periodic).reshape(6, -1))
    sf = None
    if wl.sigma_profile is not None:
        sf = np.ascontiguousarray(_cut(wl.sigma_profile, centre, half, periodic)).ravel()
    cons = oracle.prim2con_grid(sub, m, prim)
    oracle.step(sub, m, cons, prim, wl.dt, 1, sigma_field=sf)
    return cons[:, half, half, half], prim[:, half, half, half]


def _samples(wl, rng, n, margin, active_field=None):
    shape = wl.shape
    picks = []
    if active_field is not None:
        # half of the samples where the state varies (blast front, star)
        cand = np.argwhere(active_field)
        cand = cand[(cand >= margin).all(axis=1) & (cand < np.array(shape) - margin).all(axis=1)]
        picks += [tuple(c) for c in cand[rng.choice(len(cand), n // 2, replace=False)]]
    while len(picks) < n:
        picks.append(tuple(int(rng.integers(margin, s - margin)) for s in shape))
    return picks


@pytest.mark.parametrize("name", ["cyl_blast_256", "alfven_128", "lane_emden_192"])
def test_one_step_at_full_size_matches_oracle_on_samples(name):
    rng = np.random.default_rng(7)
    if name == "cyl_blast_256":
        wl = W.cyl_blast(n=256)
        X, Y, _ = W.cell_centres(wl.params["n"], wl.params["x0"], wl.params["dx"])
        r = np.sqrt(X * X + Y * Y)
        active = (r > 0.6) & (r < 1.2)
    elif name == "alfven_128":
        wl = W.alfven_diag(n=128, sigma=1e4)
        active = None
    else:
        wl = W.lane_emden_star(n=192)
        X, Y, Z = W.cell_centres(wl.params["n"], wl.params["x0"], wl.params["dx"])
        r = np.sqrt(X * X + Y * Y + Z * Z)
        active = (r > 6.0) & (r < 8.5)
    half = 2 * RADIUS[wl.params["recon"]] + 1
    s = make_solver(wl)
    s.step(wl.dt, 1)
    cons_g, prim_g = s.get_cons(), s.get_prims()
    s.close()
    picks = _samples(wl, rng, 24, half + 1, active)
    co = np.zeros((14, len(picks)))
    po = np.zeros((14, len(picks)))
    cg = np.zeros_like(co)
    pg = np.zeros_like(po)
    for q, c in enumerate(picks):
        co[:, q], po[:, q] = _oracle_centre(wl, c, half)
        cg[:, q] = cons_g[(slice(None),) + c]
        pg[:, q] = prim_g[(slice(None),) + c]
    # scales from the full GPU state (field maxima over the grid)
    dx = wl.params["dx"]
    full_scale_c = np.abs(cons_g).reshape(14, -1).max(axis=1)[:, None]
    full_scale_p = np.abs(prim_g).reshape(14, -1).max(axis=1)[:, None]
    ec = state_error(np.concatenate([cg, full_scale_c], axis=1),
                     np.concatenate([co, full_scale_c], axis=1), "cons", dx)
    ep = state_error(np.concatenate([pg, full_scale_p], axis=1),
                     np.concatenate([po, full_scale_p], axis=1), "prim", dx)
    assert ec.max() < 1e-12, (name, ec)
    assert ep.max() < 1e-12, (name, ep)


@pytest.mark.parametrize("scheme", [1, 3])
def test_general_imex_form_at_full_size_matches_oracle_on_samples(scheme):
    """The 256^3 blast with SSP2(3,3,2) / SSP3(4,3,3), one step: three face
    flux evaluations lie on the longest chain of a step (F of stages 1-3 or
    2-4), so the oracle's box reaches three stencils."""
    rng = np.random.default_rng(9)
    wl = W.cyl_blast(n=256)
    wl.params["imex"] = scheme
    X, Y, _ = W.cell_centres(wl.params["n"], wl.params["x0"], wl.params["dx"])
    r = np.sqrt(X * X + Y * Y)
    active = (r > 0.6) & (r < 1.2)
    half = 3 * RADIUS[wl.params["recon"]] + 1
    s = make_solver(wl)
    s.step(wl.dt, 1)
    cons_g, prim_g = s.get_cons(), s.get_prims()
    s.close()
    picks = _samples(wl, rng, 16, half + 1, active)
    full_scale_c = np.abs(cons_g).reshape(14, -1).max(axis=1)[:, None]
    full_scale_p = np.abs(prim_g).reshape(14, -1).max(axis=1)[:, None]
    dx = wl.params["dx"]
    for c in picks:
        co, po = _oracle_centre(wl, c, half)
        cg = cons_g[(slice(None),) + c][:, None]
        pg = prim_g[(slice(None),) + c][:, None]
        ec = state_error(np.concatenate([cg, full_scale_c], axis=1),
                         np.concatenate([co[:, None], full_scale_c], axis=1), "cons", dx)
        ep = state_error(np.concatenate([pg, full_scale_p], axis=1),
                         np.concatenate([po[:, None], full_scale_p], axis=1), "prim", dx)
        assert ec.max() < 1e-12, (c, ec)
        assert ep.max() < 1e-12, (c, ep)


def test_full_size_conservation_periodic():
    """Property at any size: the periodic 128^3 Alfven wave conserves D, S_i,
    tau, calB^i and Q to rounding over 5 steps (no sources in flat space)."""
    wl = W.alfven_diag(n=128, sigma=1e6)
    s = make_solver(wl)
    c0 = s.get_cons().reshape(14, -1).sum(axis=1)
    s.step(wl.dt, 5)
    c1 = s.get_cons()
    s.close()
    tot = c1.reshape(14, -1).sum(axis=1)
    scale = np.abs(c1).reshape(14, -1).sum(axis=1)
    for f in (0, 1, 2, 3, 4, 5, 6, 7, 13):
        assert abs(tot[f] - c0[f]) < 1e-12 * scale[f], (f, tot[f] - c0[f])


@pytest.mark.parametrize("name", ["cyl_blast_256", "alfven_128", "lane_emden_192"])
def test_mixed_precision_l1_error_at_full_size(name):
    """Mixed path against the FP64 path after 10 steps: relative L1 per
    field, vector components against their vector's scale, cleaning scalars
    and charge against their source fields.

    The star's primitive velocities are left out of the bound: in its
    low-density surface layer both precisions fail the same recoveries and
    reset the same atmosphere cells, decisions that rounding can flip, and
    the velocities of that layer then differ at O(1e-2) in L1 (the conserved
    momentum, which the step evolves, stays within the bound)."""
    from tests.helpers import state_l1
    wl = {"cyl_blast_256": lambda: W.cyl_blast(n=256),
          "alfven_128": lambda: W.alfven_diag(n=128, sigma=1e4),
          "lane_emden_192": lambda: W.lane_emden_star(n=192)}[name]()
    out = {}
    for prec in (0, 1):
        s = make_solver(wl, precision=prec)
        s.step(wl.dt, 10)
        out[prec] = (s.get_cons(), s.get_prims())
        s.close()
    dx = wl.params["dx"]
    ec = state_l1(out[1][0], out[0][0], "cons", dx, vector_scale=True)
    ep = state_l1(out[1][1], out[0][1], "prim", dx, vector_scale=True)
    print(name, "mixed-vs-FP64 L1 per conserved field:", np.array2string(ec, precision=2))
    print(name, "  own-scale:", np.array2string(state_l1(out[1][0], out[0][0], "cons", dx),
                                                 precision=2))
    print(name, "mixed-vs-FP64 L1 per primitive field:", np.array2string(ep, precision=2))
    assert ec.max() < 1e-5, (name, ec)
    keep = [f for f in range(14) if not (name == "lane_emden_192" and 2 <= f <= 4)]
    assert ep[keep].max() < 1e-5, (name, ep)


def test_long_blast_run_keeps_its_mirror_symmetry():
    """100 steps of the 256^3 blast (FP64 path): finite, and the mirror
    symmetries of the initial data kept to rounding (the run has recoveries
    that fail and are reset to the atmosphere after ~20 steps; those
    decisions come out mirror-symmetric too).  The
    resistive system is invariant under reflections (E polar, B axial) and
    under the global sign flip of (E, B, q, psi, phi), since the fluid sees
    only products of the fields.  With B = (0.1, 0, 0): x -> -x with E polar
    and B axial leaves the data unchanged; y -> -y does so combined with the
    sign flip (E axial, B polar)."""
    wl = W.cyl_blast(n=256)
    s = make_solver(wl)
    fails = s.step(wl.dt, 100)
    p = s.get_prims()
    s.close()
    assert np.isfinite(p).all()
    # odd fields under each symmetry (arrays are (field, z, y, x))
    odd_x = [2, 5, 9, 10, 12]          # v^x; E^x; B^y, B^z; phi (div B, pseudoscalar)
    odd_y = [3, 5, 7, 9, 11, 13]       # v^y; E^x, E^z; B^y; psi, q (flip of E)
    # components against their vector's magnitude (v^z, E^x, E^y, B^z vanish
    # in this z-uniform problem up to rounding), potentials against the fields
    scale = np.abs(p).reshape(14, -1).max(axis=1)
    for lo, hi in ((2, 5), (5, 8), (8, 11)):
        scale[lo:hi] = scale[lo:hi].max()
    scale[11:14] = np.maximum(scale[11:14], scale[5:11].max())
    for axis, odd in ((3, odd_x), (2, odd_y)):
        sign = np.ones(14)
        sign[odd] = -1.0
        mirror = sign[:, None, None, None] * np.flip(p, axis=axis)
        err = np.abs(p - mirror).reshape(14, -1).max(axis=1) / np.maximum(scale, 1e-300)
        assert err.max() < 1e-9, (axis, err)
