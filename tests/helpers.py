"""Shared helpers for the parity tests: run a workload through the oracle or
through the CUDA library, and compare fields."""
import numpy as np

import oracle
import workloads as W


def oracle_metric(wl):
    a, b, g, K = wl.metric_arrays()
    return oracle.Metric(a.ravel(), b.reshape(3, -1), g.reshape(6, -1), K.reshape(6, -1))


def run_oracle(wl, nsteps, dt=None, params=None):
    m = oracle_metric(wl)
    prim = np.ascontiguousarray(wl.prim.copy())
    P = dict(wl.params if params is None else params)
    cons = oracle.prim2con_grid(P, m, prim)
    sf = None if wl.sigma_profile is None else wl.sigma_profile.ravel()
    st, stats = oracle.step(P, m, cons, prim, wl.dt if dt is None else dt, nsteps,
                            sigma_field=sf)
    return st, stats, prim, cons


def make_solver(wl, params=None, **over):
    import paper_2510_18968_b300 as R
    P = dict(wl.params if params is None else params)
    P.update(over)
    s = R.Solver(P)
    if wl.alpha is not None:
        a, b, g, K = wl.metric_arrays()
        s.set_metric(np.ascontiguousarray(a), np.ascontiguousarray(b),
                     np.ascontiguousarray(g), np.ascontiguousarray(K))
    if wl.sigma_profile is not None:
        s.set_sigma(np.ascontiguousarray(wl.sigma_profile))
    s.set_prims(np.ascontiguousarray(wl.prim))
    return s


def run_gpu(wl, nsteps, dt=None, **over):
    s = make_solver(wl, **over)
    fails = s.step(wl.dt if dt is None else dt, nsteps)
    prim, cons = s.get_prims(), s.get_cons()
    stats = s.stats()
    s.close()
    return fails, stats, prim, cons


def rel_linf(a, b):
    """Per-field max|a-b| / max|b| (fields cross zero; see the tolerance
    definition in the design notes).  Fields that are identically zero in b
    are compared absolutely against 1e-300."""
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    den = np.maximum(np.abs(b).max(axis=1), 1e-300)
    return np.abs(a - b).max(axis=1) / den


def rel_l1(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return np.abs(a - b).sum(axis=1) / np.maximum(np.abs(b).sum(axis=1), 1e-300)


def state_error(a, b, kind, dx):
    """Per-field relative L-inf error of a grid state, max|a-b| / scale_f.

    scale_f = max|b_f| for the fluid and field variables.  The cleaning
    scalars and the charge start from zero in smooth flows and grow only from
    discrete divergence errors, so their own maximum is not the scale of the
    rounding they carry; for them the scale is that of the field that sources
    them (Phi, phi ~ B; Psi, psi ~ E; Q, q ~ E / dx), or their own maximum if
    larger."""
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    mx = np.abs(b).max(axis=1)
    scale = mx.copy()
    if kind == "cons":      # D Sx Sy Sz tau Bx By Bz Ex Ey Ez Phi Psi Q
        Bm, Em = mx[5:8].max(), mx[8:11].max()
        floors = {11: Bm, 12: Em, 13: Em / min(dx)}
    else:                   # rho p vx vy vz Ex Ey Ez Bx By Bz psi phi q
        Bm, Em = mx[8:11].max(), mx[5:8].max()
        floors = {11: Em, 12: Bm, 13: Em / min(dx)}
    if kind == "prim":
        # velocities are fractions of c: one recovered from a near-cancelling
        # S - E x B is compared in absolute units of 1e-3 c when smaller
        for f in (2, 3, 4):
            floors[f] = 1e-3
    for f, fl in floors.items():
        scale[f] = max(scale[f], fl)
    return np.abs(a - b).max(axis=1) / np.maximum(scale, 1e-300)


def state_l1(a, b, kind, dx, vector_scale=False):
    """Per-field relative L1 error with the same scales as state_error.

    vector_scale: each Cartesian component of S, v, B and E is measured
    against the largest of its vector's three component scales, so that a
    component that vanishes in the exact solution (E^z of a static poloidal
    field) is not compared against its own discretisation noise."""
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    l1 = np.abs(b).mean(axis=1)
    scale = l1.copy()
    if kind == "cons":
        Bm, Em = l1[5:8].max(), l1[8:11].max()
        floors = {11: Bm, 12: Em, 13: Em / min(dx)}
        vectors = ((1, 4), (5, 8), (8, 11))
    else:
        Bm, Em = l1[8:11].max(), l1[5:8].max()
        floors = {11: Em, 12: Bm, 13: Em / min(dx)}
        vectors = ((2, 5), (5, 8), (8, 11))
    for f, fl in floors.items():
        scale[f] = max(scale[f], fl)
    if vector_scale:
        for lo, hi in vectors:
            scale[lo:hi] = l1[lo:hi].max()
    return np.abs(a - b).mean(axis=1) / np.maximum(scale, 1e-300)
