"""The oracle's tangent-linear model (oracle/tangent.h: the oracle's C source
compiled on tangent numbers, the recovery's derivative from the implicit-
function theorem at its root) pinned on the CPU:

* its values are the plain oracle's, bit for bit (same FP64 operations);
* its directional derivatives of the primitives after K steps, and of a
  loss of them, equal Richardson-extrapolated central differences of the
  plain oracle (h = 1e-6 and h/2) on smooth states, for directions in the
  initial primitives and in log sigma0;
* it is linear in the direction (a seed twice as large gives exactly twice
  the derivative).
States with TVD limiters are curved and smooth along both axes, so that no
neighbouring difference comes near zero: at a limiter kink a central
difference is not the derivative of the branch taken."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.helpers import oracle_metric, run_oracle
from tests.test_gpu_adjoint import (_blast_weno5, _directions, _general_metric,
                                    _generic_smooth, _richardson, _smooth_modes)

CASES = {
    "alfven_s1e3": lambda: W.alfven_diag(n=8, sigma=1e3),
    "alfven_s10": lambda: W.alfven_diag(n=8, sigma=10.0),
    "generic_mc2_curved": lambda: _generic_smooth(True, "mc2"),
    "general_metric_weno5": lambda: _general_metric("weno5"),
    "blast_weno5": _blast_weno5,
    "star_weno5": lambda: W.lane_emden_star(n=12),
}


def _plain(wl, prim0, K, sigma0=None):
    P = dict(wl.params)
    if sigma0 is not None:
        P["sigma0"] = sigma0
    m = oracle_metric(wl)
    prim = np.ascontiguousarray(prim0.copy())
    cons = oracle.prim2con_grid(P, m, prim)
    sf = None if wl.sigma_profile is None else wl.sigma_profile.ravel()
    st, _ = oracle.step(P, m, cons, prim, wl.dt, K, sigma_field=sf)
    return prim


def _tangent(wl, prim0, u, K, dls=0.0):
    sf = None if wl.sigma_profile is None else wl.sigma_profile.ravel()
    st, stats, pN, dpN = oracle.tangent_step(wl.params, oracle_metric(wl), prim0, u, wl.dt, K,
                                             sigma_field=sf, dlog_sigma0=dls)
    return st, stats, pN, dpN


@pytest.mark.parametrize("name", ["alfven_s1e3", "generic_mc2_curved", "star_weno5"])
def test_tangent_build_computes_the_oracle_values(name):
    wl = CASES[name]()
    _, _, p0, _ = run_oracle(wl, 3)
    rng = np.random.default_rng(3)
    _, _, p1, _ = _tangent(wl, wl.prim, rng.standard_normal(wl.prim.shape), 3, dls=0.5)
    assert np.array_equal(p0, p1)


@pytest.mark.parametrize("name,K", [("alfven_s1e3", 4), ("alfven_s10", 4),
                                    ("generic_mc2_curved", 3), ("general_metric_weno5", 3),
                                    ("blast_weno5", 3)])
def test_tangent_matches_oracle_finite_differences(name, K):
    """Directions and the functional lam . P^K are smooth (low Fourier modes
    scaled to each field's magnitude), so that the extrapolated differences
    are accurate to well below 1e-6; the blast's stiff cells are recovered
    by the pressure bracket, whose derivative comes from the implicit-
    function theorem like every other recovery's."""
    wl = CASES[name]()
    prim0 = wl.prim
    rng = np.random.default_rng(29)
    lam = np.stack([_smooth_modes(prim0.shape[1:], rng) for _ in range(14)])
    lam /= np.abs(prim0).reshape(14, -1).max(axis=1)[:, None, None, None] + 1e-3
    tl, fd = [], []
    for u in _directions(prim0, rng, 5):
        st, stats, _, dpN = _tangent(wl, prim0, u, K)
        assert st == 0
        tl.append(float(np.sum(lam * dpN)))
        fd.append(_richardson(lambda h: float(np.sum(lam * _plain(wl, prim0 + h * u, K)))))
    tl, fd = np.array(tl), np.array(fd)
    rel = np.abs(tl - fd) / np.maximum(np.abs(fd), 1e-2 * np.abs(fd).max())
    assert rel.max() < 1e-6, (name, tl, fd, rel)
    if wl.params.get("sigma0", 0.0) > 0.0:
        s0 = wl.params["sigma0"]
        _, _, _, ds = _tangent(wl, prim0, np.zeros_like(prim0), K, dls=1.0)
        # h = 1e-4 in log sigma0: the recovery's stopping tolerance makes the
        # loss noisy at ~1e-14 / h, and the loss is smooth in sigma0 on this
        # scale (Richardson over 1e-3 ... 3e-5 agrees to 1e-9)
        fds = _richardson(lambda h: float(np.sum(lam * _plain(wl, prim0, K, s0 * np.exp(h)))),
                          h=1e-4)
        assert abs(np.sum(lam * ds) - fds) <= 1e-6 * abs(fds), (name, np.sum(lam * ds), fds)


def test_tangent_is_linear_in_the_direction():
    wl = CASES["alfven_s1e3"]()
    rng = np.random.default_rng(8)
    u = _directions(wl.prim, rng, 5)[-1]
    _, _, _, d1 = _tangent(wl, wl.prim, u, 3)
    _, _, _, d2 = _tangent(wl, wl.prim, 2.0 * u, 3)
    # derivative parts are linear in the seed; a factor of two is exact
    assert np.array_equal(d2, 2.0 * d1)
