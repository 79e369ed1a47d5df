"""FP64 CPU oracle for one IMEX-RK step of resistive GRMHD.

TEST INFRASTRUCTURE ONLY.  This package restates, in plain C called through
ctypes, what arXiv:2510.18968 (Sec. II-III) computes: primitive->conserved map
(Eqs. conserved_dens/tau/S), fluxes and sources (Eq. GRRMHD_flux_form), Ohm's
law (Eq. Ohm_law), HLLE with light-speed bounds (Sec. III), TVD/WENO5
reconstruction, the IMEX-SSP2(2,2,2) stages (Table imex, Eq. IMEX3) or the
general IMEX-RK form with another of the paper's SSP tableaux, and the
implicit-E + 1D recovery (Sec. III.B).  It shares no code with the CUDA
library and never imports it.  Only tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline / reference legs may use it.

Array conventions: grid fields are interior-only, float64, shape
(nfields, nz, ny, nx) (x fastest).  Primitive order: rho, p, vx, vy, vz,
Ex, Ey, Ez, Bx, By, Bz, psi, phi, q.  Conserved order: D, Sx, Sy, Sz, tau,
Bx, By, Bz, Ex, Ey, Ez, Phi, Psi, Q (densitised).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_DP = ctypes.POINTER(ctypes.c_double)


class _Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("dx", ctypes.c_double * 3),
        ("bc", ctypes.c_int * 3),
        ("recon", ctypes.c_int),
        ("gamma_eos", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("sigma_model", ctypes.c_int),
        ("sigma0", ctypes.c_double),
        ("sigma_exp", ctypes.c_double),
        ("D_atmo", ctypes.c_double),
        ("rho_atmo", ctypes.c_double),
        ("K_atmo", ctypes.c_double),
        ("atmo_tol", ctypes.c_double),
        ("c2p_tol", ctypes.c_double),
        ("c2p_maxit", ctypes.c_int),
        ("c2p_wmax", ctypes.c_double),
        ("qflux_mode", ctypes.c_int),
        ("imex", ctypes.c_int),
    ]


DEFAULTS = dict(n=(1, 1, 1), dx=(1.0, 1.0, 1.0), bc=(0, 0, 0), recon=0,
                gamma_eos=2.0, kappa=1.0, sigma_model=0, sigma0=0.0,
                sigma_exp=0.0, D_atmo=0.0, rho_atmo=1e-10, K_atmo=100.0,
                atmo_tol=1e-2, c2p_tol=1e-14, c2p_maxit=100, c2p_wmax=100.0,
                qflux_mode=0, imex=0)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(_Params)
        i, d = ctypes.c_int, ctypes.c_double
        L.orc_metric_inverse.argtypes = [_DP, _DP, _DP]
        L.orc_prim2con.argtypes = [_DP, d, _DP, _DP, d, _DP]
        L.orc_flux.argtypes = [i, _DP, d, _DP, _DP, d, d, _DP, _DP]
        L.orc_hlle.argtypes = [i, _DP, _DP, d, _DP, _DP, d, d, _DP]
        L.orc_recon_line.argtypes = [i, i, _DP, _DP, _DP]
        L.orc_implicit_E.argtypes = [_DP, _DP, _DP, d, _DP, d, d, _DP]
        L.orc_implicit_E.restype = i
        L.orc_con2prim.argtypes = [P, _DP, i, d, d, d, _DP, _DP, _DP, _DP,
                                   ctypes.POINTER(i)]
        L.orc_con2prim.restype = i
        L.orc_con2prim_batch.argtypes = [P, ctypes.c_long, _DP, i, d, _DP, _DP, _DP, _DP,
                                         _DP, _DP, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_rhs.argtypes = [P, _DP, _DP, _DP, _DP, _DP, _DP, _DP, _DP]
        L.orc_prim2con_grid.argtypes = [P, _DP, _DP, _DP, _DP, _DP]
        L.orc_step.argtypes = [P, _DP, _DP, _DP, _DP, _DP, _DP, _DP, d, i,
                               ctypes.POINTER(ctypes.c_longlong)]
        L.orc_step.restype = i
        L.orc_step_tableau.argtypes = L.orc_step.argtypes
        L.orc_step_tableau.restype = i
        L.orc_imex_tableau.argtypes = [i, _DP, _DP, _DP, _DP]
        L.orc_imex_tableau.restype = i
        L.orc_set_status_buffer.argtypes = [ctypes.c_void_p]
        L.orc_set_fail_buffer.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p]
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


def _arr(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n, (a.shape, n)
    return a


def make_params(**kw):
    p = dict(DEFAULTS)
    # grid origin and the GPU precision switch do not enter the oracle's
    # arithmetic (it is always FP64 and position-free)
    kw = {k: v for k, v in kw.items() if k not in ("x0", "precision")}
    unknown = set(kw) - set(DEFAULTS)
    if unknown:
        raise KeyError(f"unknown oracle parameters {sorted(unknown)}")
    p.update(kw)
    s = _Params()
    s.n[:] = [int(v) for v in p["n"]]
    s.dx[:] = [float(v) for v in p["dx"]]
    s.bc[:] = [int(v) for v in p["bc"]]
    for k in ("recon", "sigma_model", "c2p_maxit", "qflux_mode", "imex"):
        setattr(s, k, int(p[k]))
    for k in ("gamma_eos", "kappa", "sigma0", "sigma_exp", "D_atmo", "rho_atmo",
              "K_atmo", "atmo_tol", "c2p_tol", "c2p_wmax"):
        setattr(s, k, float(p[k]))
    return s


# ------------------------------------------------------------ pointwise

def metric_inverse(g6):
    g6 = _arr(g6, 6)
    gi = np.zeros(6)
    sg = ctypes.c_double()
    lib().orc_metric_inverse(_ptr(g6), _ptr(gi), ctypes.byref(sg))
    return gi, sg.value


def prim2con(prim, alpha=1.0, beta=(0, 0, 0), g6=(1, 0, 0, 1, 0, 1), gamma_eos=2.0):
    prim, beta, g6 = _arr(prim, 14), _arr(beta, 3), _arr(g6, 6)
    out = np.zeros(14)
    lib().orc_prim2con(_ptr(prim), float(alpha), _ptr(beta), _ptr(g6),
                       float(gamma_eos), _ptr(out))
    return out


def flux(d, prim, alpha=1.0, beta=(0, 0, 0), g6=(1, 0, 0, 1, 0, 1), sigma=0.0,
         gamma_eos=2.0):
    prim, beta, g6 = _arr(prim, 14), _arr(beta, 3), _arr(g6, 6)
    F, U = np.zeros(14), np.zeros(14)
    lib().orc_flux(int(d), _ptr(prim), float(alpha), _ptr(beta), _ptr(g6),
                   float(sigma), float(gamma_eos), _ptr(F), _ptr(U))
    return F, U


def hlle(d, primL, primR, alpha=1.0, beta=(0, 0, 0), g6=(1, 0, 0, 1, 0, 1),
         sigma=0.0, gamma_eos=2.0):
    pL, pR = _arr(primL, 14), _arr(primR, 14)
    beta, g6 = _arr(beta, 3), _arr(g6, 6)
    F = np.zeros(14)
    lib().orc_hlle(int(d), _ptr(pL), _ptr(pR), float(alpha), _ptr(beta),
                   _ptr(g6), float(sigma), float(gamma_eos), _ptr(F))
    return F


def recon_line(method, u):
    """Face states of a 1D line: uL[i], uR[i] at the face between u[i], u[i+1]
    (NaN where the stencil leaves the array)."""
    u = _arr(u)
    n = u.size
    uL, uR = np.zeros(n), np.zeros(n)
    lib().orc_recon_line(int(method), n, _ptr(u), _ptr(uL), _ptr(uR))
    return uL, uR


def implicit_E(Estar, Bcons, v, alpha=1.0, g6=(1, 0, 0, 1, 0, 1), sigma=0.0, c=0.0):
    Estar, Bcons, v, g6 = _arr(Estar, 3), _arr(Bcons, 3), _arr(v, 3), _arr(g6, 6)
    out = np.zeros(3)
    ok = lib().orc_implicit_E(_ptr(Estar), _ptr(Bcons), _ptr(v), float(alpha),
                              _ptr(g6), float(sigma), float(c), _ptr(out))
    if not ok:
        raise FloatingPointError("singular implicit-E system")
    return out


def con2prim(params, cons, implicit, c, sigma, guess, alpha=1.0,
             g6=(1, 0, 0, 1, 0, 1)):
    """Returns (prim, cons_out, iterations, status)."""
    P = params if isinstance(params, _Params) else make_params(**params)
    cons, guess, g6 = _arr(cons, 14), _arr(guess, 14), _arr(g6, 6)
    prim, cout = np.zeros(14), np.zeros(14)
    it = ctypes.c_int()
    st = lib().orc_con2prim(ctypes.byref(P), _ptr(cons), int(implicit), float(c),
                            float(sigma), float(alpha), _ptr(g6), _ptr(guess),
                            _ptr(prim), _ptr(cout), ctypes.byref(it))
    return prim, cout, it.value, st


def con2prim_batch(params, cons, implicit, c, sigma, guess, alpha, g6):
    """orc_con2prim on n points: cons, guess (n, 14), sigma, alpha (n,),
    g6 (n, 6).  Returns (prim, cons_out, iterations, status)."""
    P = params if isinstance(params, _Params) else make_params(**params)
    cons, guess = _arr(cons), _arr(guess)
    n = cons.shape[0]
    sigma, alpha, g6 = _arr(sigma, n), _arr(alpha, n), _arr(g6, 6 * n)
    assert cons.shape == (n, 14) and guess.shape == (n, 14)
    prim, cout = np.zeros((n, 14)), np.zeros((n, 14))
    it, st = np.zeros(n, np.int32), np.zeros(n, np.int32)
    lib().orc_con2prim_batch(ctypes.byref(P), n, _ptr(cons), int(implicit), float(c),
                             _ptr(sigma), _ptr(alpha), _ptr(g6), _ptr(guess), _ptr(prim),
                             _ptr(cout), it.ctypes.data, st.ctypes.data)
    return prim, cout, it, st


# ------------------------------------------------------------ grid

class Metric:
    """Static 3+1 metric on the interior grid (shape (nz, ny, nx) per field)."""

    def __init__(self, alpha, beta, gamma, K):
        self.alpha = _arr(alpha)
        self.beta = _arr(beta)
        self.gamma = _arr(gamma)
        self.K = _arr(K)

    @classmethod
    def flat(cls, shape):
        N = int(np.prod(shape))
        g = np.zeros((6, N))
        g[0] = g[3] = g[5] = 1.0
        return cls(np.ones(N), np.zeros((3, N)), g, np.zeros((6, N)))


def _grid_params(params, shape_zyx):
    p = dict(params)
    p.setdefault("n", (shape_zyx[2], shape_zyx[1], shape_zyx[0]))
    return make_params(**p)


def prim2con_grid(params, metric, prim):
    prim = _arr(prim)
    P = _grid_params(params, prim.shape[1:])
    cons = np.zeros_like(prim)
    lib().orc_prim2con_grid(ctypes.byref(P), _ptr(metric.alpha), _ptr(metric.beta),
                            _ptr(metric.gamma), _ptr(prim), _ptr(cons))
    return cons


def rhs(params, metric, prim, sigma_field=None, J=None):
    """Non-stiff right-hand side F(U) of the stage whose primitives are prim.
    J (3, ...) is the cell-centred stage current used in the charge flux;
    None evaluates Ohm's law at the face states instead."""
    prim = _arr(prim)
    P = _grid_params(params, prim.shape[1:])
    out = np.zeros_like(prim)
    sf = None if sigma_field is None else _arr(sigma_field)
    Jc = None if J is None else _arr(J)
    lib().orc_rhs(ctypes.byref(P), _ptr(metric.alpha), _ptr(metric.beta),
                  _ptr(metric.gamma), _ptr(metric.K), _ptr(sf), _ptr(prim), _ptr(Jc),
                  _ptr(out))
    return out


STAT_NAMES = ("c2p_calls", "c2p_iterations", "c2p_fallbacks", "c2p_failures",
              "atmo_floor_resets", "c2p_max_iterations", "nan")


IMEX_SCHEMES = {0: "SSP2(2,2,2)", 1: "SSP2(3,3,2)", 2: "SSP3(3,3,2)", 3: "SSP3(4,3,3)"}


def imex_tableau(scheme):
    """(At, wt, A, w) of an IMEX scheme (Sec. III.A), trimmed to its stages."""
    At, A = np.zeros(16), np.zeros(16)
    wt, w = np.zeros(4), np.zeros(4)
    s = lib().orc_imex_tableau(int(scheme), _ptr(At), _ptr(wt), _ptr(A), _ptr(w))
    if not s:
        raise KeyError(f"unknown IMEX scheme {scheme}")
    return (At.reshape(4, 4)[:s, :s].copy(), wt[:s].copy(),
            A.reshape(4, 4)[:s, :s].copy(), w[:s].copy())


FAIL_REC = 39   # doubles per failed-recovery record (rmhd_oracle.h ORC_FAIL_REC)


def step(params, metric, cons, prim, dt, nsteps=1, sigma_field=None,
         status_out=None, general_form=False, fail_out=None):
    """Advance (cons, prim) in place by nsteps IMEX-RK steps with the
    tableau params["imex"] (0: SSP2(2,2,2), Table imex, through its literal
    equations; others, or general_form=True, through the general form).
    Returns (status, stats dict).  status 0 ok, -4 recovery failures were
    reset to atmosphere, -5 non-finite conserved values."""
    assert cons.dtype == np.float64 and prim.dtype == np.float64
    assert cons.flags["C_CONTIGUOUS"] and prim.flags["C_CONTIGUOUS"]
    P = _grid_params(params, prim.shape[1:])
    stats = (ctypes.c_longlong * 8)()
    sf = None if sigma_field is None else _arr(sigma_field)
    if status_out is not None:
        assert status_out.dtype == np.int32 and status_out.size == 3 * prim[0].size
        lib().orc_set_status_buffer(status_out.ctypes.data)
    if fail_out is not None:
        # fail_out: dict with "buf" (cap x FAIL_REC float64) and "count" (int64[1])
        lib().orc_set_fail_buffer(fail_out["buf"].ctypes.data, fail_out["buf"].shape[0],
                                  fail_out["count"].ctypes.data)
    fn = lib().orc_step_tableau if general_form else lib().orc_step
    st = fn(ctypes.byref(P), _ptr(metric.alpha), _ptr(metric.beta),
                        _ptr(metric.gamma), _ptr(metric.K), _ptr(sf), _ptr(cons),
                        _ptr(prim), float(dt), int(nsteps), stats)
    if status_out is not None:
        lib().orc_set_status_buffer(None)
    if fail_out is not None:
        lib().orc_set_fail_buffer(None, 0, None)
    return st, dict(zip(STAT_NAMES, list(stats)[:7]))


# ------------------------------------------------------- tangent-linear model

_tlib = None


class _TL(ctypes.Structure):
    """One tangent number passed by value (value, derivative)."""
    _fields_ = [("v", ctypes.c_double), ("d", ctypes.c_double)]


def tangent_lib():
    """The tangent-linear build of the oracle (the same C source on tangent
    numbers: value and directional derivative, oracle/tangent.h)."""
    global _tlib
    if _tlib is None:
        L = ctypes.CDLL(_build.build_tangent())
        P = ctypes.POINTER(_Params)
        v = ctypes.c_void_p
        L.orc_prim2con_grid.argtypes = [P, v, v, v, v, v]
        L.orc_step.argtypes = [P, v, v, v, v, v, v, v, _TL, ctypes.c_int,
                               ctypes.POINTER(ctypes.c_longlong)]
        L.orc_step.restype = ctypes.c_int
        L.orc_set_tangent_log_sigma0.argtypes = [ctypes.c_double]
        _tlib = L
    return _tlib


def _tl(value, deriv=None):
    """A tangent array: (..., 2) float64, value and derivative interleaved."""
    value = np.asarray(value, dtype=np.float64)
    out = np.zeros(value.shape + (2,))
    out[..., 0] = value
    if deriv is not None:
        out[..., 1] = deriv
    return out


def tangent_step(params, metric, prim, dprim, dt, nsteps, sigma_field=None, dlog_sigma0=0.0):
    """Tangent-linear model of nsteps IMEX-SSP2(2,2,2) steps (forward-mode
    differentiation of the oracle's step, branches as the values take them):
    from the primitives prim and a direction dprim of them (and dlog_sigma0
    of log sigma0), returns (status, stats, prim^N, dprim^N), dprim^N the
    derivative of the final primitives along that direction.  The initial
    conserved state is formed from prim (and its derivative from dprim)."""
    L = tangent_lib()
    prim = _arr(prim)
    P = _grid_params(params, prim.shape[1:])
    tp = np.ascontiguousarray(_tl(prim, dprim))
    tc = np.zeros_like(tp)
    ta, tb = _tl(metric.alpha), _tl(metric.beta)
    tg, tk = _tl(metric.gamma), _tl(metric.K)
    tsf = None if sigma_field is None else _tl(sigma_field)
    p = lambda a: None if a is None else a.ctypes.data
    L.orc_prim2con_grid(ctypes.byref(P), p(ta), p(tb), p(tg), p(tp), p(tc))
    stats = (ctypes.c_longlong * 8)()
    L.orc_set_tangent_log_sigma0(float(dlog_sigma0))
    try:
        st = L.orc_step(ctypes.byref(P), p(ta), p(tb), p(tg), p(tk), p(tsf), p(tc), p(tp),
                        _TL(float(dt), 0.0), int(nsteps), stats)
    finally:
        L.orc_set_tangent_log_sigma0(0.0)
    return st, dict(zip(STAT_NAMES, list(stats)[:7])), tp[..., 0].copy(), tp[..., 1].copy()
