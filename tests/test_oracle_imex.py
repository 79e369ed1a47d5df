"""Oracle pins for the IMEX-RK tableaux (Sec. III.A, Table imex; the other
SSP schemes the paper lists in Sec. I).

* Each tableau has the structure of the general IMEX form (explicit part
  strictly lower triangular, implicit part diagonally implicit), satisfies
  the order conditions of a partitioned Runge-Kutta method of its order
  (explicit, implicit and coupling conditions), and is L-stable.  A wrong
  coefficient breaks one of these: they fix the remembered values of the
  published tableaux independently of the code that applies them.
* Scheme 0 is the paper's printed Table imex.
* The stepper applies the implicit tableau exactly: a uniform plasma at rest
  with B = 0 and Q = 0 has no flux and no explicit source for calE, and the
  stiff Ohm term is -sigma calE, so one step multiplies calE by the
  stability function R(-sigma dt) = 1 - sigma dt w^T (I + sigma dt A)^{-1} 1
  of the implicit tableau, for any sigma dt.
* The general form run with Table imex equals the literal equations
  (U^(1), U^(2), IMEX3) to rounding.
* A smooth problem on a fixed grid converges in dt at the scheme's order."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.helpers import oracle_metric, state_error

ORDER = {0: 2, 1: 2, 2: 2, 3: 3}
EXPLICIT_ORDER = {0: 2, 1: 2, 2: 3, 3: 3}   # order of At, wt alone


def _c(At, A):
    return At.sum(axis=1), A.sum(axis=1)


@pytest.mark.parametrize("scheme", [0, 1, 2, 3])
def test_tableau_structure_and_order_conditions(scheme):
    At, wt, A, w = oracle.imex_tableau(scheme)
    s = len(wt)
    assert np.all(np.triu(At) == 0.0)                 # explicit
    assert np.all(np.triu(A, 1) == 0.0)               # diagonally implicit
    assert np.all(np.diag(A) > 0.0)                   # every stage has an implicit solve
    assert np.all(At >= 0.0) and np.all(wt >= 0.0)    # SSP explicit part
    ct, c = _c(At, A)
    cs = (ct, c)
    bs = (wt, w)
    tol = 1e-12
    for b in bs:
        assert abs(b.sum() - 1.0) < tol
        for cy in cs:
            assert abs(b @ cy - 0.5) < tol
    if ORDER[scheme] >= 3:
        # the coefficients are published to 14 digits
        tol3 = 1e-12
        for b in bs:
            for cy in cs:
                for cz in cs:
                    assert abs(b @ (cy * cz) - 1.0 / 3.0) < tol3
            for Ay in (At, A):
                for cz in cs:
                    assert abs(b @ Ay @ cz - 1.0 / 6.0) < tol3
    else:
        # a second-order scheme misses at least one third-order condition
        third = [wt @ (ct * ct) - 1 / 3, wt @ At @ ct - 1 / 6, w @ (c * c) - 1 / 3,
                 w @ A @ c - 1 / 6]
        assert max(abs(v) for v in third) > 1e-3
    # L-stability: R(z) -> 1 - w^T A^{-1} 1 = 0 as z -> -inf
    assert abs(1.0 - w @ np.linalg.solve(A, np.ones(s))) < 1e-12


def test_scheme0_is_table_imex():
    """The paper's printed SSP2(2,2,2) tableau, gamma = 1 - 1/sqrt(2)."""
    g = 1.0 - 1.0 / np.sqrt(2.0)
    At, wt, A, w = oracle.imex_tableau(0)
    assert np.array_equal(At, [[0.0, 0.0], [1.0, 0.0]])
    assert np.array_equal(wt, [0.5, 0.5]) and np.array_equal(w, [0.5, 0.5])
    assert np.allclose(A, [[g, 0.0], [1.0 - 2.0 * g, g]], rtol=0, atol=1e-16)


def _stability(scheme, z):
    """R(z) = 1 + z w^T (I - z A)^{-1} 1 of the implicit tableau."""
    _, _, A, w = oracle.imex_tableau(scheme)
    s = len(w)
    return 1.0 + z * (w @ np.linalg.solve(np.eye(s) - z * A, np.ones(s)))


def _uniform_E_state(n=(3, 1, 1)):
    prim = np.zeros((14, n[2], n[1], n[0]))
    prim[0], prim[1] = 1.0, 1.0
    prim[5], prim[6], prim[7] = 0.3, -0.2, 0.5
    return prim


@pytest.mark.parametrize("scheme", [0, 1, 2, 3])
@pytest.mark.parametrize("z", [0.1, 1.0, 10.0, 1e3, 1e6])
def test_stiff_decay_follows_the_stability_function(scheme, z):
    dt, nsteps = 0.01, 3
    prim = _uniform_E_state()
    params = W.base_params((3, 1, 1), (0, 0, 0), (0.1, 0.1, 0.1), (0, 0, 0), "minmod",
                           2.0, z / dt, imex=scheme)
    m = oracle.Metric.flat(prim.shape[1:])
    cons = oracle.prim2con_grid(params, m, prim)
    E0 = cons[8:11].copy()
    st, _ = oracle.step(params, m, cons, prim, dt, nsteps)
    assert st == 0
    want = _stability(scheme, -z) ** nsteps * E0
    assert np.abs(cons[8:11] - want).max() <= 1e-12 * np.abs(E0).max()
    assert np.abs(prim[2:5]).max() == 0.0       # the plasma stays at rest


@pytest.mark.parametrize("case", ["alfven_diag", "blast_curved", "shocktube_sigma", "gauss"])
def test_general_form_reduces_to_the_literal_ssp222(case):
    if case == "alfven_diag":
        wl = W.alfven_diag(n=8, sigma=1e3)
    elif case == "blast_curved":
        wl = W.cyl_blast(n=12)
    elif case == "shocktube_sigma":
        wl = W.shocktube_sigma(n=64)
    else:
        wl = W.gauss_smooth(8, curved=True)
    out = []
    for general in (False, True):
        m = oracle_metric(wl)
        prim = np.ascontiguousarray(wl.prim.copy())
        cons = oracle.prim2con_grid(wl.params, m, prim)
        sf = None if wl.sigma_profile is None else wl.sigma_profile.ravel()
        st, _ = oracle.step(wl.params, m, cons, prim, wl.dt, 3, sigma_field=sf,
                            general_form=general)
        assert st in (0, -4)
        out.append((cons, prim))
    dx = wl.params["dx"]
    assert state_error(out[1][0], out[0][0], "cons", dx).max() < 1e-12
    assert state_error(out[1][1], out[0][1], "prim", dx).max() < 1e-12


def _alfven_at(scheme, sigma, dt, t_end=0.25):
    wl = W.alfven_1d(n=32, sigma=sigma, recon="weno5")
    params = dict(wl.params, imex=scheme)
    m = oracle_metric(wl)
    prim = np.ascontiguousarray(wl.prim.copy())
    cons = oracle.prim2con_grid(params, m, prim)
    nsteps = int(round(t_end / dt))
    st, _ = oracle.step(params, m, cons, prim, dt, nsteps)
    assert st == 0
    return cons


@pytest.mark.parametrize("scheme", [0, 1, 2, 3])
@pytest.mark.parametrize("sigma", [0.0, 20.0])
def test_temporal_order_on_a_smooth_wave(scheme, sigma):
    """Large-amplitude circularly polarised Alfven wave, 32 cells, WENO5,
    fixed grid: differences between runs at dt, dt/2, dt/4, dt/8 shrink by
    2^p (sigma = 0: the explicit tableau alone, whose order is 3 for the
    SSP3(3,3) part of SSP3(3,3,2); sigma = 20, sigma dt up to 0.16: both
    tableaux and their coupling, the scheme's order)."""
    dt0 = 1.0 / 128.0
    runs = [_alfven_at(scheme, sigma, dt0 / 2 ** k) for k in range(4)]
    diffs = [np.abs(runs[k] - runs[k + 1]).max() for k in range(3)]
    rates = [np.log2(diffs[k] / diffs[k + 1]) for k in range(2)]
    p = EXPLICIT_ORDER[scheme] if sigma == 0.0 else ORDER[scheme]
    assert rates[-1] > p - 0.15, (scheme, sigma, diffs, rates)
    assert rates[-1] < p + 0.6, (scheme, sigma, diffs, rates)
