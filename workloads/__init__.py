"""Seeded synthetic inputs (initial primitives, static metric, conductivity).

This module only builds inputs.  It holds none of the step's arithmetic and is
shared by the oracle tests, the CUDA parity tests and the benchmark.  Each
generator returns a ``Workload`` whose arrays are float64, interior-only,
shape (nfields, nz, ny, nx), x fastest.

The initial data follow the paper's test problems (arXiv:2510.18968 Sec. IV)
as modified by the benchmark configurations:
  * Brio-Wu shocktube, Sec. IV.A (variant with B^x = 0.5, B^y = +-1), and
    the section's own shocktube with conductivity sigma0 D^gamma_sigma;
  * circularly polarised Alfven wave, Sec. IV.D, Eqs. Bi, vyvz, Alf_vel,
    rotated onto the (1,1,1) diagonal of a periodic cube;
  * cylindrical explosion, Sec. IV.B (log-linear taper of rho and p);
  * static weak-field star: an n=1 Lane-Emden density with its Newtonian
    potential Phi, alpha = 1 + Phi, gamma_ij = (1 - 2 Phi) delta_ij, and a
    poloidal field from A_phi ~ max(p - 0.04 p_max, 0) (Sec. IV.E vector
    potential with power 1), conductivity blended by tanh at the surface;
  * self-similar current sheet, Sec. IV.C (B^y = B0 erf(x sqrt(sigma)/(2 sqrt(t))));
  * a smooth 2D periodic state on the Gauss constraint q = nabla_i E^i, flat
    or conformally flat, for the Gauss's-law charge variant of Sec. IV.E.
"""
from dataclasses import dataclass, field
from math import erf, pi, sqrt
from typing import Optional

import numpy as np

SEED = 2510189

PRIM_NAMES = ("rho", "p", "vx", "vy", "vz", "Ex", "Ey", "Ez", "Bx", "By", "Bz",
              "psi", "phi", "q")
CONS_NAMES = ("D", "Sx", "Sy", "Sz", "tau", "Bx", "By", "Bz", "Ex", "Ey", "Ez",
              "Phi", "Psi", "Q")

RECON = {"minmod": 0, "mc2": 1, "weno5": 2}
BC_PERIODIC, BC_OUTFLOW = 0, 1


@dataclass
class Workload:
    name: str
    params: dict
    prim: np.ndarray                      # (14, nz, ny, nx)
    dt: float
    nsteps: int
    alpha: Optional[np.ndarray] = None    # (nz, ny, nx); None = flat metric
    beta: Optional[np.ndarray] = None     # (3, nz, ny, nx)
    gamma: Optional[np.ndarray] = None    # (6, nz, ny, nx) xx,xy,xz,yy,yz,zz
    K: Optional[np.ndarray] = None        # (6, nz, ny, nx)
    sigma_profile: Optional[np.ndarray] = None  # (nz, ny, nx), sigma = sigma0*profile
    extra: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.prim.shape[1:]

    @property
    def ncells(self):
        return int(np.prod(self.shape))

    def metric_arrays(self):
        """(alpha, beta, gamma, K) as float64 arrays, flat metric filled in."""
        shp = self.shape
        if self.alpha is None:
            alpha = np.ones(shp)
            beta = np.zeros((3,) + shp)
            gamma = np.zeros((6,) + shp)
            gamma[0] = gamma[3] = gamma[5] = 1.0
            K = np.zeros((6,) + shp)
            return alpha, beta, gamma, K
        return self.alpha, self.beta, self.gamma, self.K


def base_params(n, x0, dx, bc, recon, gamma_eos, sigma0, **kw):
    p = dict(n=tuple(int(v) for v in n), x0=tuple(float(v) for v in x0),
             dx=tuple(float(v) for v in dx), bc=tuple(int(v) for v in bc),
             recon=RECON[recon] if isinstance(recon, str) else int(recon),
             gamma_eos=float(gamma_eos), kappa=1.0, sigma_model=0,
             sigma0=float(sigma0), sigma_exp=0.0, D_atmo=0.0,
             rho_atmo=1e-10, K_atmo=100.0, atmo_tol=1e-2, c2p_tol=1e-14, c2p_maxit=100,
             c2p_wmax=100.0, qflux_mode=0)
    p.update(kw)
    return p


def cell_centres(n, x0, dx):
    """Cell-centre coordinates (z, y, x) meshes for the interior grid."""
    xs = [x0[d] + (np.arange(n[d]) + 0.5) * dx[d] for d in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return X, Y, Z


def _empty_prim(shape):
    return np.zeros((14,) + tuple(shape))


def alfven_speed(rho, p, gamma_eos, B0, eta):
    """v_A of a circularly polarised Alfven wave, Eq. Alf_vel (h = rho(1+eps)+p)."""
    h = rho + gamma_eos / (gamma_eos - 1.0) * p
    a = 2.0 * B0 ** 2 / (h + B0 ** 2 * (1.0 + eta ** 2))
    b = 2.0 * eta * B0 ** 2 / (h + B0 ** 2 * (1.0 + eta ** 2))
    return sqrt(a / (1.0 + sqrt(1.0 - b * b)))


# ------------------------------------------------------------------ configs

def brio_wu(n=400, sigma=1e5, cfl=0.5, nsteps=320, axis=0):
    """1D relativistic Brio-Wu shocktube on [-0.5, 0.5], Gamma=2, outflow,
    minmod + HLLE; left (rho,p,Bx,By)=(1,1,0.5,1), right (0.125,0.1,0.5,-1)."""
    nn = [1, 1, 1]
    nn[axis] = n
    dx = 1.0 / n
    x0 = [-0.5 if d == axis else -0.5 * dx for d in range(3)]
    dxs = [dx] * 3
    P = base_params(nn, x0, dxs, [BC_OUTFLOW] * 3, "minmod", 2.0, sigma)
    X, Y, Z = cell_centres(nn, x0, dxs)
    s = (X, Y, Z)[axis]
    prim = _empty_prim(X.shape)
    left = s < 0.0
    prim[0] = np.where(left, 1.0, 0.125)
    prim[1] = np.where(left, 1.0, 0.1)
    # B along the shock normal 0.5, transverse +-1 (rotated with the axis)
    prim[8 + axis] = 0.5
    prim[8 + (axis + 1) % 3] = np.where(left, 1.0, -1.0)
    return Workload("brio_wu_%d" % n, P, prim, cfl * dx, nsteps)


def shocktube_sigma(n=400, sigma0=1e6, sigma_exp=12.0, cfl=0.25, t_end=0.4):
    """Sec. IV.A shocktube with the conductivity of Eq. sigma_evol,
    sigma = sigma0 D^sigma_exp: left (rho, p, B^y) = (1, 1, 0.5), right
    (0.125, 0.1, -0.5), B^x = 0, E = 0, Gamma = 2, minmod, outflow, on
    [-0.5, 0.5] with CFL 0.25 to t = 0.4."""
    dx = 1.0 / n
    nn, x0, dxs = [n, 1, 1], [-0.5, -0.5 * dx, -0.5 * dx], [dx] * 3
    P = base_params(nn, x0, dxs, [BC_OUTFLOW] * 3, "minmod", 2.0, sigma0,
                    sigma_model=2, sigma_exp=sigma_exp)
    X, _, _ = cell_centres(nn, x0, dxs)
    prim = _empty_prim(X.shape)
    left = X < 0.0
    prim[0] = np.where(left, 1.0, 0.125)
    prim[1] = np.where(left, 1.0, 0.1)
    prim[9] = np.where(left, 0.5, -0.5)
    dt = cfl * dx
    return Workload("shocktube_sigma_D%g" % sigma_exp, P, prim, dt, int(round(t_end / dt)))


def alfven_diag(n=128, sigma=1e6, eta=0.1, B0=1.0, gamma_eos=4.0 / 3.0,
                cfl=0.125, nsteps=200, noise=1e-6, recon="weno5", seed=SEED):
    """Circularly polarised Alfven wave travelling along (1,1,1) in the
    periodic cube [-0.5,0.5]^3 (Eqs. Bi, vyvz, Alf_vel rotated)."""
    dx = 1.0 / n
    nn, x0, dxs = [n] * 3, [-0.5] * 3, [dx] * 3
    P = base_params(nn, x0, dxs, [BC_PERIODIC] * 3, recon, gamma_eos, sigma)
    X, Y, Z = cell_centres(nn, x0, dxs)
    nhat = np.array([1.0, 1.0, 1.0]) / sqrt(3.0)
    e1 = np.array([1.0, -1.0, 0.0]) / sqrt(2.0)
    e2 = np.array([1.0, 1.0, -2.0]) / sqrt(6.0)
    phase = 2.0 * pi * (X + Y + Z)
    vA = alfven_speed(1.0, 1.0, gamma_eos, B0, eta)
    rng = np.random.default_rng(seed)
    prim = _empty_prim(X.shape)
    prim[0] = 1.0 + noise * rng.standard_normal(X.shape)
    prim[1] = 1.0
    Bt = [eta * B0 * (np.cos(phase) * e1[i] + np.sin(phase) * e2[i]) for i in range(3)]
    B = [B0 * nhat[i] + Bt[i] for i in range(3)]
    v = [-(vA / B0) * Bt[i] for i in range(3)]
    E = [-(v[1] * B[2] - v[2] * B[1]), -(v[2] * B[0] - v[0] * B[2]),
         -(v[0] * B[1] - v[1] * B[0])]
    for i in range(3):
        prim[2 + i] = v[i]
        prim[5 + i] = E[i]
        prim[8 + i] = B[i]
    return Workload("alfven_diag_%d_s%.0e" % (n, sigma), P, prim, cfl * dx, nsteps,
                    extra=dict(vA=vA))


def alfven_1d(n=100, sigma=1e6, eta=1.0, B0=1.1547, gamma_eos=2.0, cfl=0.25,
              recon="mc2", t_final=2.0):
    """Paper's 1D CP Alfven wave on [-0.5, 0.5], rho = p = 1 (Sec. IV.D)."""
    dx = 1.0 / n
    nn, x0, dxs = [n, 1, 1], [-0.5, -0.5 * dx, -0.5 * dx], [dx] * 3
    P = base_params(nn, x0, dxs, [BC_PERIODIC] * 3, recon, gamma_eos, sigma)
    X, _, _ = cell_centres(nn, x0, dxs)
    vA = alfven_speed(1.0, 1.0, gamma_eos, B0, eta)
    k = 2.0 * pi
    prim = _empty_prim(X.shape)
    prim[0] = 1.0
    prim[1] = 1.0
    By = eta * B0 * np.cos(k * X)
    Bz = eta * B0 * np.sin(k * X)
    prim[8] = B0
    prim[9] = By
    prim[10] = Bz
    prim[3] = -vA / B0 * By
    prim[4] = -vA / B0 * Bz
    # E = -v x B = (0, vA Bz, -vA By) with v = -(vA/B0)(0, By, Bz), Bx = B0
    prim[6] = vA * Bz
    prim[7] = -vA * By
    dt = cfl * dx
    nsteps = int(round(t_final / dt))
    return Workload("alfven_1d_%d" % n, P, prim, dt, nsteps, extra=dict(vA=vA))


def cyl_blast(n=256, sigma=1e3, cfl=0.25, nsteps=100, rho_in=1e-2, p_in=1.0,
              rho_out=1e-4, p_out=3e-5, Bx=0.1, r_in=0.8, r_out=1.0,
              gamma_eos=4.0 / 3.0, recon="mc2", L=6.0, nz=None):
    """Cylindrical explosion (axis z) in [-L, L]^3, Sec. IV.B density/pressure
    profile with log-linear taper between r_in and r_out, uniform B^x."""
    nz = n if nz is None else nz
    dx = 2.0 * L / n
    nn = [n, n, nz]
    x0 = [-L, -L, -0.5 * nz * dx]
    dxs = [dx] * 3
    P = base_params(nn, x0, dxs, [BC_OUTFLOW] * 3, recon, gamma_eos, sigma)
    X, Y, _ = cell_centres(nn, x0, dxs)
    r = np.sqrt(X * X + Y * Y)

    def taper(vin, vout):
        t = ((r_out - r) * np.log(vout) + (r - r_in) * np.log(vin)) / (r_out - r_in)
        return np.where(r <= r_in, vin, np.where(r >= r_out, vout, np.exp(t)))

    prim = _empty_prim(X.shape)
    prim[0] = taper(rho_in, rho_out)
    prim[1] = taper(p_in, p_out)
    prim[8] = Bx
    return Workload("cyl_blast_%d" % n, P, prim, cfl * dx, nsteps)


def lane_emden_star(n=192, L=12.0, R=8.0, rho_c=1.28e-3, K=100.0, gamma_eos=2.0,
                    rho_atmo=1e-10, sigma0=1e6, width=0.25, Bmax=1e-3, cfl=0.125,
                    nsteps=500, recon="weno5"):
    """Static weak-field star in [-L, L]^3 (stand-in for the TOV test of
    Sec. IV.E): n=1 Lane-Emden density, alpha = 1+Phi, gamma_ij=(1-2Phi)delta,
    poloidal B from A_phi = A_b varpi^2 max(p - 0.04 p_max, 0), sigma blended
    by tanh at the surface."""
    dx = 2.0 * L / n
    nn, x0, dxs = [n] * 3, [-L] * 3, [dx] * 3
    P = base_params(nn, x0, dxs, [BC_OUTFLOW] * 3, recon, gamma_eos, sigma0,
                    sigma_model=1, rho_atmo=rho_atmo, K_atmo=K)
    X, Y, Z = cell_centres(nn, x0, dxs)
    r = np.sqrt(X * X + Y * Y + Z * Z)
    xi = pi * r / R
    sinc = np.where(xi > 0, np.sin(xi) / np.where(xi > 0, xi, 1.0), 1.0)
    inside = r < R
    rho = np.where(inside, np.maximum(rho_c * sinc, rho_atmo), rho_atmo)
    p = K * rho ** 2
    M = 4.0 * rho_c * R ** 3 / pi
    Phi = np.where(inside, -(4.0 * rho_c * R * R / pi) * (1.0 + sinc),
                   -M / np.maximum(r, 1e-300))
    alpha = 1.0 + Phi
    psi4 = 1.0 - 2.0 * Phi
    gamma = np.zeros((6,) + X.shape)
    gamma[0] = gamma[3] = gamma[5] = psi4
    beta = np.zeros((3,) + X.shape)
    Kc = np.zeros((6,) + X.shape)
    # vector potential A = A_b max(p - p_cut, 0) (-y, x, 0); B^i = eta^{ijk} d_j A_k / sqrt(g)
    p_cut = 0.04 * p.max()
    amp = np.maximum(p - p_cut, 0.0)
    Ax, Ay = -Y * amp, X * amp
    dAy_dx = np.gradient(Ay, dx, axis=2)
    dAx_dy = np.gradient(Ax, dx, axis=1)
    dAy_dz = np.gradient(Ay, dx, axis=0)
    dAx_dz = np.gradient(Ax, dx, axis=0)
    sg = psi4 ** 1.5
    Bx = -dAy_dz / sg
    By = dAx_dz / sg
    Bz = (dAy_dx - dAx_dy) / sg
    bmag = np.sqrt(Bx * Bx + By * By + Bz * Bz).max()
    scale = Bmax / bmag if bmag > 0 else 0.0
    prim = _empty_prim(X.shape)
    prim[0] = rho
    prim[1] = p
    prim[8], prim[9], prim[10] = Bx * scale, By * scale, Bz * scale
    profile = 0.5 * (1.0 - np.tanh((r - R) / width))
    return Workload("lane_emden_%d" % n, P, prim, cfl * dx, nsteps, alpha=alpha,
                    beta=beta, gamma=gamma, K=Kc, sigma_profile=profile)


def current_sheet(n=600, sigma=100.0, L=1.5, B0=1.0, p=50.0, rho=1.0, t0=1.0,
                  cfl=0.25, gamma_eos=2.0):
    """Self-similar current sheet, Sec. IV.C: B^y = B0 erf(x sqrt(sigma)/(2 sqrt(t0)))."""
    dx = 2.0 * L / n
    nn, x0, dxs = [n, 1, 1], [-L, -0.5 * dx, -0.5 * dx], [dx] * 3
    P = base_params(nn, x0, dxs, [BC_OUTFLOW] * 3, "minmod", gamma_eos, sigma)
    X, _, _ = cell_centres(nn, x0, dxs)
    prim = _empty_prim(X.shape)
    prim[0] = rho
    prim[1] = p
    prim[9] = B0 * np.vectorize(erf)(X * sqrt(sigma) / (2.0 * sqrt(t0)))
    return Workload("current_sheet_%d" % n, P, prim, cfl * dx, 0,
                    extra=dict(t0=t0, B0=B0))


# ------------------------------------------------------------------ random states

def gauss_smooth(n, curved=False, qflux_mode=2):
    """2D periodic smooth state with q = (1/sqrt(g)) d_i(sqrt(g) E^i) exactly
    (analytic derivatives) and a divergence-free densitised B."""
    dx = 1.0 / n
    P = base_params((n, n, 1), (0, 0, 0), (dx, dx, dx), (0, 0, 0), "mc2", 2.0, 20.0,
                    qflux_mode=qflux_mode)
    x = (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(x, x, indexing="xy")
    X, Y = X[None], Y[None]
    tp, e0 = 2.0 * np.pi, 0.05
    prim = np.zeros((14, 1, n, n))
    prim[0] = 1.0 + 0.2 * np.sin(tp * (X + Y))
    prim[1] = 1.0
    prim[2], prim[3] = 0.1 * np.sin(tp * Y), 0.1 * np.cos(tp * X)
    prim[5], prim[6] = e0 * np.sin(tp * X), e0 * np.cos(tp * Y)
    q = tp * e0 * (np.cos(tp * X) - np.sin(tp * Y))
    sg = np.ones_like(X)
    kw = {}
    if curved:
        psi4 = 1.0 + 0.2 * np.sin(tp * X) * np.cos(tp * Y)
        dpx = 0.2 * tp * np.cos(tp * X) * np.cos(tp * Y)
        dpy = -0.2 * tp * np.sin(tp * X) * np.sin(tp * Y)
        sg = psi4 ** 1.5
        q = q + 1.5 * (prim[5] * dpx + prim[6] * dpy) / psi4   # + E . grad ln sqrt(g)
        g = np.zeros((6, 1, n, n))
        g[0] = g[3] = g[5] = psi4
        kw = dict(alpha=np.ones((1, n, n)), beta=np.zeros((3, 1, n, n)), gamma=g,
                  K=np.zeros((6, 1, n, n)))
    prim[8] = (0.3 + 0.1 * np.cos(tp * Y)) / sg
    prim[9] = (0.2 + 0.1 * np.sin(tp * X)) / sg
    prim[13] = q
    return Workload("gauss", P, prim, 0.25 * dx, 1, **kw)


def random_metric(rng, npts, strength=0.3):
    """Random positive-definite 3-metrics gamma = I + strength*sym(A), lapse in
    [0.6, 1.2], shift |beta| < 0.2."""
    A = rng.uniform(-1, 1, (npts, 3, 3))
    S = 0.5 * (A + np.transpose(A, (0, 2, 1)))
    g = np.eye(3)[None] + strength * S
    # make sure it is positive definite: add a multiple of I if needed
    w = np.linalg.eigvalsh(g)
    g += np.maximum(0.2 - w.min(axis=1), 0)[:, None, None] * np.eye(3)[None]
    g6 = np.stack([g[:, 0, 0], g[:, 0, 1], g[:, 0, 2], g[:, 1, 1], g[:, 1, 2],
                   g[:, 2, 2]])
    alpha = rng.uniform(0.6, 1.2, npts)
    beta = rng.uniform(-0.2, 0.2, (3, npts))
    return alpha, beta, g6


def random_prims(rng, npts, g6=None, wmax=5.0, mag_range=(1e-3, 1e2),
                 rho_range=(1e-4, 1.0), p_over_rho=(1e-3, 1.0)):
    """Random physical primitive states: W <= wmax, magnetisation
    B^2/p log-uniform in mag_range, E comparable to v x B plus a random part."""
    rho = np.exp(rng.uniform(np.log(rho_range[0]), np.log(rho_range[1]), npts))
    p = rho * np.exp(rng.uniform(np.log(p_over_rho[0]), np.log(p_over_rho[1]), npts))
    if g6 is None:
        g = np.broadcast_to(np.eye(3), (npts, 3, 3))
    else:
        g = np.empty((npts, 3, 3))
        idx = [(0, 0, 0), (1, 0, 1), (2, 0, 2), (3, 1, 1), (4, 1, 2), (5, 2, 2)]
        for a, i, j in idx:
            g[:, i, j] = g6[a]
            g[:, j, i] = g6[a]
    # velocity with |v| from W in [1, wmax]
    W = np.exp(rng.uniform(0, np.log(wmax), npts))
    vmag = np.sqrt(1.0 - 1.0 / W ** 2)
    dirn = rng.standard_normal((npts, 3))
    norm = np.sqrt(np.einsum("ni,nij,nj->n", dirn, g, dirn))
    v = dirn / norm[:, None] * vmag[:, None]
    bdir = rng.standard_normal((npts, 3))
    bn = np.sqrt(np.einsum("ni,nij,nj->n", bdir, g, bdir))
    mag = np.exp(rng.uniform(np.log(mag_range[0]), np.log(mag_range[1]), npts))
    B = bdir / bn[:, None] * np.sqrt(mag * p)[:, None]
    # E near the ideal value -v x B (flat cross product of contravariant parts
    # is only a template here) plus a random 10% part
    E = -np.cross(v, B) + 0.1 * rng.standard_normal((npts, 3)) * np.sqrt(mag * p)[:, None]
    prim = np.zeros((14, npts))
    prim[0], prim[1] = rho, p
    prim[2:5] = v.T
    prim[5:8] = E.T
    prim[8:11] = B.T
    prim[11:14] = 0.1 * rng.standard_normal((3, npts))
    return prim
