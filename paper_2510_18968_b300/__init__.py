"""Python binding of the B300 resistive-GRMHD IMEX step library (librmhd.so).

Argument marshalling only: every step of the method runs in the CUDA kernels
behind the C ABI of include/rmhd.h.  Host numpy arrays are passed with
on_device = 0; CUDA torch tensors (float64, contiguous, on the current device)
with on_device = 1.  There is no CPU fallback: if the library cannot be
loaded, importing it raises.

Array layout (as in the C ABI): float64 structure of arrays, interior cells,
shape (nfields, nz, ny, nx), x fastest.  Primitives: rho, p, v^x..z, E^x..z,
B^x..z, psi, phi, q.  Conserved (densitised): D, S_x..z, tau, B^x..z,
E^x..z, Phi, Psi, Q.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librmhd.so")

RMHD_OK, RMHD_EINVAL, RMHD_ECUDA, RMHD_ENOMEM, RMHD_EC2P, RMHD_ENAN = 0, -1, -2, -3, -4, -5
ERROR_NAMES = {0: "RMHD_OK", -1: "RMHD_EINVAL", -2: "RMHD_ECUDA", -3: "RMHD_ENOMEM",
               -4: "RMHD_EC2P", -5: "RMHD_ENAN"}
PREC_FP64, PREC_MIXED = 0, 1


class RMHDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("x0", ctypes.c_double * 3),
        ("dx", ctypes.c_double * 3),
        ("bc", ctypes.c_int * 3),
        ("recon", ctypes.c_int),
        ("precision", ctypes.c_int),
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
        ("c2p_first_pass", ctypes.c_int),
        ("imex", ctypes.c_int),
    ]


EXPORTS = ("rmhd_default_params", "rmhd_create", "rmhd_set_metric", "rmhd_set_sigma",
           "rmhd_set_prims", "rmhd_step", "rmhd_get_prims", "rmhd_get_cons",
           "rmhd_set_state", "rmhd_set_cons", "rmhd_state_layer_bytes", "rmhd_get_state_layers",
           "rmhd_set_state_layers", "rmhd_get_stats", "rmhd_step_profiled", "rmhd_rhs", "rmhd_con2prim_points",
           "rmhd_con2prim_points_noalloc", "rmhd_set_sigma0", "rmhd_adjoint_forward",
           "rmhd_adjoint_backward", "rmhd_test_rcp64", "rmhd_test_mm3", "rmhd_test_mm3f",
           "rmhd_test_tile_copies", "rmhd_test_tile_copy_launches", "rmhd_test_bracket_points",
           "rmhd_last_error", "rmhd_destroy")

_lib = None


def load(build_if_missing=True):
    """Load librmhd.so (building it with nvcc if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if not build_if_missing:
            raise ImportError(f"{LIB_PATH} is missing; run paper_2510_18968_b300/build.py")
        from . import build as _b
        _b.build()
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER(Params)
    L.rmhd_default_params.argtypes = [P]
    L.rmhd_default_params.restype = None
    L.rmhd_create.argtypes = [P, vp, ctypes.POINTER(vp)]
    L.rmhd_set_metric.argtypes = [vp, vp, vp, vp, vp, i]
    L.rmhd_set_sigma.argtypes = [vp, vp, i]
    L.rmhd_set_prims.argtypes = [vp, vp, i]
    L.rmhd_step.argtypes = [vp, d, i, ctypes.POINTER(ctypes.c_longlong)]
    L.rmhd_get_prims.argtypes = [vp, vp, i]
    L.rmhd_get_cons.argtypes = [vp, vp, i]
    L.rmhd_set_state.argtypes = [vp, vp, vp, i]
    L.rmhd_set_cons.argtypes = [vp, vp, i]
    L.rmhd_state_layer_bytes.argtypes = [vp]
    L.rmhd_get_state_layers.argtypes = [vp, i, i, vp, i]
    L.rmhd_set_state_layers.argtypes = [vp, i, i, vp, i]
    L.rmhd_get_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.rmhd_step_profiled.argtypes = [vp, d, i, ctypes.POINTER(ctypes.c_double)]
    L.rmhd_rhs.argtypes = [vp, vp, vp, vp, i]
    L.rmhd_con2prim_points.argtypes = [P, i, vp, vp, vp, vp, vp, i, d, vp, vp, vp, vp, vp]
    L.rmhd_con2prim_points_noalloc.argtypes = [P, i, vp, vp, vp, vp, vp, i, d, vp, vp, vp, vp,
                                               vp]
    L.rmhd_set_sigma0.argtypes = [vp, d]
    L.rmhd_adjoint_forward.argtypes = [vp, d, i, i]
    L.rmhd_adjoint_backward.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_double), i,
                                        ctypes.POINTER(ctypes.c_double)]
    L.rmhd_test_rcp64.argtypes = [vp, vp, ctypes.c_longlong, vp]
    L.rmhd_test_mm3.argtypes = [vp, vp, vp, vp, ctypes.c_longlong, vp]
    L.rmhd_test_mm3f.argtypes = [vp, vp, vp, vp, ctypes.c_longlong, vp]
    L.rmhd_test_tile_copies.argtypes = [ctypes.c_int]
    L.rmhd_test_tile_copies.restype = ctypes.c_int
    L.rmhd_test_tile_copy_launches.argtypes = []
    L.rmhd_test_tile_copy_launches.restype = ctypes.c_longlong
    L.rmhd_test_bracket_points.argtypes = [P, i, vp, vp, vp, i, d, i, vp, vp, vp]
    L.rmhd_last_error.argtypes = [vp]
    L.rmhd_last_error.restype = ctypes.c_char_p
    L.rmhd_destroy.argtypes = [vp]
    for name in EXPORTS:
        if name not in ("rmhd_default_params", "rmhd_last_error"):
            getattr(L, name).restype = i
    L.rmhd_state_layer_bytes.restype = ctypes.c_longlong
    _lib = L
    return L


def make_params(**kw):
    """rmhd_params from the library defaults updated with kw (workload dicts
    from the workloads module are accepted as they are)."""
    L = load()
    p = Params()
    L.rmhd_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k in ("n", "bc"):
            getattr(p, k)[:] = [int(x) for x in v]
        elif k in ("x0", "dx"):
            getattr(p, k)[:] = [float(x) for x in v]
        elif k in ("recon", "precision", "sigma_model", "c2p_maxit", "qflux_mode",
                   "c2p_first_pass", "imex"):
            setattr(p, k, int(v))
        elif k in ("gamma_eos", "kappa", "sigma0", "sigma_exp", "D_atmo", "rho_atmo",
                   "K_atmo", "atmo_tol", "c2p_tol", "c2p_wmax"):
            setattr(p, k, float(v))
        else:
            raise KeyError(f"unknown parameter {k}")
    return p


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, nelem=None):
    """(pointer, on_device) for a float64 numpy array or CUDA torch tensor."""
    if a is None:
        return None, 0
    if _is_torch(a):
        import torch
        if not a.is_cuda:
            a = a.numpy()
        else:
            if a.dtype != torch.float64 or not a.is_contiguous():
                raise TypeError("device arrays must be contiguous float64 CUDA tensors")
            if nelem is not None and a.numel() != nelem:
                raise ValueError(f"expected {nelem} elements, got {a.numel()}")
            return a.data_ptr(), 1
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
        raise TypeError("host arrays must be C-contiguous float64 numpy arrays")
    if nelem is not None and a.size != nelem:
        raise ValueError(f"expected {nelem} elements, got {a.size}")
    return a.ctypes.data, 0


def _raw_ptr(a, nbytes):
    """(pointer, on_device) of a contiguous buffer of exactly nbytes bytes:
    a CUDA torch tensor or a host numpy array of any dtype."""
    if _is_torch(a):
        if not a.is_contiguous() or a.numel() * a.element_size() != nbytes:
            raise ValueError(f"need a contiguous buffer of {nbytes} bytes")
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda)
    if not a.flags["C_CONTIGUOUS"] or a.nbytes != nbytes:
        raise ValueError(f"need a contiguous buffer of {nbytes} bytes")
    return a.ctypes.data_as(ctypes.c_void_p), 0


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


class Solver:
    """One grid, one state, one CUDA stream (rmhd_create ... rmhd_destroy)."""

    def __init__(self, params, stream=None):
        self.L = load()
        self.params = params if isinstance(params, Params) else make_params(**params)
        self.shape = (self.params.n[2], self.params.n[1], self.params.n[0])
        self.N = int(np.prod(self.shape))
        h = ctypes.c_void_p()
        rc = self.L.rmhd_create(ctypes.byref(self.params), _stream_ptr(stream), ctypes.byref(h))
        if rc:
            raise RMHDError(rc, self.L.rmhd_last_error(None).decode())
        self.h = h

    def _check(self, rc, soft_ok=()):
        if rc and rc not in soft_ok:
            raise RMHDError(rc, self.L.rmhd_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.L.rmhd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- set-up
    def set_metric(self, alpha=None, beta=None, gamma=None, K=None):
        if alpha is None:
            return self._check(self.L.rmhd_set_metric(self.h, None, None, None, None, 0))
        pa, da = _ptr(alpha, self.N)
        pb, _ = _ptr(beta, 3 * self.N)
        pg, _ = _ptr(gamma, 6 * self.N)
        pk, _ = _ptr(K, 6 * self.N)
        return self._check(self.L.rmhd_set_metric(self.h, pa, pb, pg, pk, da))

    def set_sigma(self, profile=None):
        p, d = _ptr(profile, self.N)
        return self._check(self.L.rmhd_set_sigma(self.h, p, d))

    def set_prims(self, prim):
        p, d = _ptr(prim, 14 * self.N)
        return self._check(self.L.rmhd_set_prims(self.h, p, d))

    def set_cons(self, cons):
        """Restore from the conserved variables alone (primitives recovered
        on the device); returns RMHD_EC2P (soft) when cells were reset to the
        atmosphere."""
        pc, d = _ptr(cons, 14 * self.N)
        return self._check(self.L.rmhd_set_cons(self.h, pc, d), soft_ok=(RMHD_EC2P,))

    # ---- z-slab decomposition: raw state of a range of z-layers
    def state_layer_bytes(self):
        return int(self.L.rmhd_state_layer_bytes(self.h))

    def get_state_layers(self, k0, nk, out):
        """Pack the state of interior z-layers [k0, k0 + nk) into `out`
        (a contiguous CUDA torch tensor or host numpy array of
        nk * state_layer_bytes() bytes)."""
        p, d = _raw_ptr(out, nk * self.state_layer_bytes())
        return self._check(self.L.rmhd_get_state_layers(self.h, int(k0), int(nk), p, d))

    def set_state_layers(self, k0, nk, buf):
        p, d = _raw_ptr(buf, nk * self.state_layer_bytes())
        return self._check(self.L.rmhd_set_state_layers(self.h, int(k0), int(nk), p, d))

    def set_state(self, cons, prim):
        pc, d = _ptr(cons, 14 * self.N)
        pp, _ = _ptr(prim, 14 * self.N)
        return self._check(self.L.rmhd_set_state(self.h, pc, pp, d))

    # ---- stepping
    def step(self, dt, nsteps=1, sync=True):
        """Returns the number of recoveries reset to the atmosphere (sync) or
        None (async)."""
        if not sync:
            self._check(self.L.rmhd_step(self.h, float(dt), int(nsteps), None))
            return None
        fails = ctypes.c_longlong()
        self._check(self.L.rmhd_step(self.h, float(dt), int(nsteps), ctypes.byref(fails)),
                    soft_ok=(RMHD_EC2P,))
        return fails.value

    PROFILE_GROUPS = ("stage1_recovery", "ghost_fill", "flux_stage2", "stage2_rhs_recovery",
                      "flux_final", "final_rhs_recovery")

    def step_profiled(self, dt, nsteps=1):
        """Step with CUDA events between kernel groups; returns ms per group."""
        ms = (ctypes.c_double * 6)()
        self._check(self.L.rmhd_step_profiled(self.h, float(dt), int(nsteps), ms))
        return dict(zip(self.PROFILE_GROUPS, list(ms)))

    # ---- read-out
    def get_prims(self, out=None):
        out = np.empty((14,) + self.shape) if out is None else out
        p, d = _ptr(out, 14 * self.N)
        self._check(self.L.rmhd_get_prims(self.h, p, d))
        return out

    def get_cons(self, out=None):
        out = np.empty((14,) + self.shape) if out is None else out
        p, d = _ptr(out, 14 * self.N)
        self._check(self.L.rmhd_get_cons(self.h, p, d))
        return out

    def stats(self):
        s = (ctypes.c_longlong * 8)()
        self._check(self.L.rmhd_get_stats(self.h, s))
        names = ("c2p_calls", "c2p_iterations", "c2p_fallbacks", "c2p_failures",
                 "atmo_floor_resets", "c2p_max_iterations", "nan", "steps")
        return dict(zip(names, list(s)))

    # ---- adjoint
    def set_sigma0(self, sigma0):
        return self._check(self.L.rmhd_set_sigma0(self.h, float(sigma0)))

    def adjoint_forward(self, dt, nsteps, checkpoint_every=10):
        """nsteps steps from the current state, recorded for adjoint_backward."""
        return self._check(self.L.rmhd_adjoint_forward(self.h, float(dt), int(nsteps),
                                                       int(checkpoint_every)))

    ADJOINT_GROUPS = ("recompute", "adjoint_flux", "adjoint_sources", "adjoint_stages")

    def adjoint_backward(self, lam_prims, out=None, profile=False):
        """(dL/dP^0, dL/dlog sigma0) for lam_prims = dL/dP^N (14, nz, ny, nx);
        with profile=True also a dict of CUDA-event ms per kernel group."""
        if out is None:
            if _is_torch(lam_prims) and lam_prims.is_cuda:
                import torch
                out = torch.empty_like(lam_prims)
            else:
                out = np.empty((14,) + self.shape)
        pl, d = _ptr(lam_prims, 14 * self.N)
        po, d2 = _ptr(out, 14 * self.N)
        if d != d2:
            raise TypeError("lam_prims and out must both be host or both be device arrays")
        ls = ctypes.c_double()
        ms = (ctypes.c_double * 4)() if profile else None
        self._check(self.L.rmhd_adjoint_backward(self.h, pl, po, ctypes.byref(ls), d, ms))
        if profile:
            return out, ls.value, dict(zip(self.ADJOINT_GROUPS, list(ms)))
        return out, ls.value

    def rhs(self, prim, J=None, out=None):
        out = np.empty((14,) + self.shape) if out is None else out
        pp, d = _ptr(prim, 14 * self.N)
        pj, _ = _ptr(J, 3 * self.N)
        po, _ = _ptr(out, 14 * self.N)
        self._check(self.L.rmhd_rhs(self.h, pp, pj, po, d))
        return out


def con2prim_points(params, cons, guess, alpha, gamma, sigma, implicit, c, stream=None,
                    out=None, noalloc=False):
    """Pointwise recovery on CUDA torch tensors (cons/guess (14, n), alpha (n,),
    gamma (6, n), sigma (n,)).  Returns (prim, cons_out, iters, status).
    noalloc=True calls rmhd_con2prim_points_noalloc, the variant that uses
    the library's built-in work list instead of allocating; pass preallocated
    outputs in `out` = (prim, cons_out, iters, status) to allocate nothing
    here either."""
    import torch
    L = load()
    P = params if isinstance(params, Params) else make_params(**params)
    n = int(alpha.numel())
    dev = alpha.device
    if out is None:
        prim = torch.empty((14, n), dtype=torch.float64, device=dev)
        cout = torch.empty((14, n), dtype=torch.float64, device=dev)
        iters = torch.empty(n, dtype=torch.int32, device=dev)
        status = torch.empty(n, dtype=torch.int32, device=dev)
    else:
        prim, cout, iters, status = out
    args = [_ptr(x, m)[0] for x, m in ((cons, 14 * n), (guess, 14 * n), (alpha, n),
                                        (gamma, 6 * n), (sigma, n))]
    fn = L.rmhd_con2prim_points_noalloc if noalloc else L.rmhd_con2prim_points
    rc = fn(ctypes.byref(P), n, *args, int(implicit), float(c), prim.data_ptr(),
            cout.data_ptr(), iters.data_ptr(), status.data_ptr(), _stream_ptr(stream))
    if rc:
        raise RMHDError(rc, L.rmhd_last_error(None).decode())
    return prim, cout, iters, status


def evolve_function():
    """torch.autograd.Function: (P^0, log sigma0) -> P^N through nsteps FP64
    steps; backward is the library's discrete adjoint.

        P_N = evolve_function().apply(P0, log_sigma0, solver, dt, nsteps, every)

    P0: CUDA float64 tensor (14, nz, ny, nx); log_sigma0: 0-d tensor."""
    import torch

    class Evolve(torch.autograd.Function):
        @staticmethod
        def forward(ctx, P0, log_sigma0, solver, dt, nsteps, every):
            solver.set_sigma0(float(torch.exp(log_sigma0.detach())))
            solver.set_prims(P0.detach().contiguous())
            solver.adjoint_forward(dt, nsteps, every)
            ctx.solver = solver
            ctx.sigma_device = log_sigma0.device
            out = torch.empty_like(P0)
            solver.get_prims(out=out)
            return out

        @staticmethod
        def backward(ctx, grad_out):
            g, ls = ctx.solver.adjoint_backward(grad_out.contiguous())
            return (g, torch.tensor(ls, dtype=torch.float64, device=ctx.sigma_device), None,
                    None, None, None)

    return Evolve
