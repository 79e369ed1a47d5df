"""Pin of the oracle's source terms and flux divergence against the covariant
equations they come from, with nothing shared with the oracle.

The right-hand side of Eq. GRRMHD_flux_form, -d_k F^k + S, is the time
derivative of the conserved vector.  Here that time derivative is built
independently at one point x0 of a smooth analytic state in a smooth analytic
metric with lapse, shift, off-diagonal 3-metric and extrinsic curvature:

* fluid rows (D, S_j, tau) from the 4-dimensional conservation laws
  nabla_mu (rho u^mu) = 0 and nabla_mu T^{mu nu} = 0 (Sec. II.C), by direct
  tensor algebra on the 4-metric of Eq. 3plus1_metric, its Christoffel
  symbols and T^{mu nu} = fluid + Faraday (Sec. II.B-C);
* field rows (calB, calE, Phi, Psi, calQ) from the covariant 3+1 Maxwell
  system of Sec. II.B (the equations for E^i, psi, B^i, phi and q with
  Lie derivatives along the shift, spatial covariant derivatives and K),
  densitised with d_t sqrt(gamma) = sqrt(gamma) (-alpha K + D_i beta^i).

The extrinsic curvature is an input of the step, so the spacetime is the one
in which d_t gamma_ij = -2 alpha K_ij + D_i beta_j + D_j beta_i (the ADM
definition of K_ij); the time derivatives of lapse and shift are free (gauge)
and must drop out, which the test checks.  Spatial derivatives of the
analytic expressions are taken by 8th-order central differences with a step
far below the grid spacing.

The oracle's right-hand side at the cell centred on x0 (WENO5, sigma = 0, so
that Ohm's law is the advective current Q v) must converge to the exact
value at second order in the grid spacing in every one of the 14 rows: a
dropped term, a wrong sign or a transposed index in a source would leave an
O(1) difference.  A second test does the same for a fluid in hydrostatic
equilibrium in the Rindler lapse alpha = 1 + g x, where the exact time
derivative is zero.
"""
import itertools

import numpy as np
import pytest

import oracle

GAM = 5.0 / 3.0
KAPPA = 0.7
X0 = np.array([0.13, -0.21, 0.07])

LC3 = np.zeros((3, 3, 3))
for (i, j, k), s in (((0, 1, 2), 1), ((1, 2, 0), 1), ((2, 0, 1), 1),
                     ((0, 2, 1), -1), ((2, 1, 0), -1), ((1, 0, 2), -1)):
    LC3[i, j, k] = s


def _perm_sign(p):
    p = list(p)
    s = 1
    for i in range(len(p)):
        for j in range(i + 1, len(p)):
            if p[i] > p[j]:
                s = -s
    return s


LC4 = np.zeros((4, 4, 4, 4))
for p in itertools.permutations(range(4)):
    LC4[p] = _perm_sign(p)


# ------------------------------------------------------------ the fields

def metric_fields(x):
    """alpha, beta^i, gamma_ij (3x3), K_ij (3x3) at the point x."""
    X, Y, Z = x
    alpha = 1.0 + 0.15 * np.sin(1.3 * X + 0.4 * Y - 0.2 * Z + 0.3)
    beta = 0.12 * np.array([np.sin(0.9 * Y + 0.5 * Z), np.cos(1.1 * X - 0.3 * Z),
                            np.sin(0.7 * X + 0.8 * Y + 0.1)])
    g = np.eye(3) + 0.1 * np.array([
        [np.sin(X + 0.2), 0.5 * np.cos(Y - Z), 0.3 * np.sin(X + Z)],
        [0.0, np.cos(0.8 * Y + 0.1), 0.4 * np.sin(X - Y)],
        [0.0, 0.0, np.sin(0.6 * Z + X)]])
    g = np.triu(g) + np.triu(g, 1).T
    K = 0.08 * np.array([
        [np.cos(X + Y), 0.6 * np.sin(Z), 0.2 * np.cos(X - Z)],
        [0.0, np.sin(Y + 0.3), 0.5 * np.cos(X + 2 * Z)],
        [0.0, 0.0, np.cos(Z - Y)]])
    K = np.triu(K) + np.triu(K, 1).T
    return alpha, beta, g, K


def prim_fields(x):
    """rho, p, v^i, E^i, B^i, psi, phi, q (contravariant, undensitised)."""
    X, Y, Z = x
    rho = 1.0 + 0.2 * np.sin(X + 2 * Y + 0.1)
    p = 0.6 + 0.15 * np.cos(1.2 * X - Z)
    v = np.array([0.25 * np.sin(Y + Z), 0.2 * np.cos(X + 0.5), -0.15 * np.sin(X - Y)])
    E = np.array([0.3 * np.cos(Z), 0.2 * np.sin(X + Y), 0.25 * np.cos(Y - 0.2)])
    B = np.array([0.8 + 0.2 * np.sin(Y), 0.4 * np.cos(X + Z), -0.3 * np.sin(Z + 0.4)])
    psi = 0.1 * np.sin(X + Y + Z)
    phi = 0.12 * np.cos(X - 2 * Y)
    q = 0.2 * np.sin(2 * X + Z)
    return rho, p, v, E, B, psi, phi, q


def d_num(f, x, k, h=2e-3):
    """d f / d x^k at x by an 8th-order central difference."""
    c = (4 / 5, -1 / 5, 4 / 105, -1 / 280)
    e = np.zeros(3)
    e[k] = 1.0
    acc = 0.0
    for m, cm in enumerate(c, start=1):
        acc = acc + cm * (np.asarray(f(x + m * h * e)) - np.asarray(f(x - m * h * e)))
    return acc / h


def grad(f, x):
    return np.array([d_num(f, x, k) for k in range(3)])


# ----------------------------------------------------- 4-metric and tensors

def four_metric(x):
    alpha, beta, g, _ = metric_fields(x)
    bl = g @ beta
    G = np.zeros((4, 4))
    G[0, 0] = -alpha ** 2 + bl @ beta
    G[0, 1:] = G[1:, 0] = bl
    G[1:, 1:] = g
    return G


def christoffel3(x):
    """Gamma^i_jk of gamma_ij at x."""
    g = metric_fields(x)[2]
    dg = np.array([d_num(lambda y: metric_fields(y)[2], x, k) for k in range(3)])  # dg[k,i,j]
    gi = np.linalg.inv(g)
    return 0.5 * (np.einsum("il,jlk->ijk", gi, dg) + np.einsum("il,klj->ijk", gi, dg)
                  - np.einsum("il,ljk->ijk", gi, dg))


def gamma_dot(x):
    """d_t gamma_ij = -2 alpha K_ij + D_i beta_j + D_j beta_i."""
    alpha, beta, g, K = metric_fields(x)
    dbl = np.array([d_num(lambda y: metric_fields(y)[2] @ metric_fields(y)[1], x, k)
                    for k in range(3)])          # dbl[i, j] = d_i beta_j
    Chr = christoffel3(x)
    bl = g @ beta
    Db = dbl - np.einsum("kij,k->ij", Chr, bl)   # D_i beta_j
    return -2.0 * alpha * K + Db + Db.T


def four_metric_dt(x, adot, bdot):
    """d_t g_{mu nu} at t = 0 for lapse and shift changing at rates adot,
    bdot (gauge) and the 3-metric changing by gamma_dot."""
    alpha, beta, g, _ = metric_fields(x)
    gd = gamma_dot(x)
    Gd = np.zeros((4, 4))
    Gd[0, 0] = -2.0 * alpha * adot + beta @ gd @ beta + 2.0 * beta @ g @ bdot
    Gd[0, 1:] = Gd[1:, 0] = gd @ beta + g @ bdot
    Gd[1:, 1:] = gd
    return Gd


def christoffel4(x, adot, bdot):
    G = four_metric(x)
    dG = np.zeros((4, 4, 4))      # dG[mu, a, b] = d_mu g_ab
    dG[0] = four_metric_dt(x, adot, bdot)
    for k in range(3):
        dG[1 + k] = d_num(four_metric, x, k)
    Gi = np.linalg.inv(G)
    return 0.5 * (np.einsum("ls,msn->lmn", Gi, dG) + np.einsum("ls,nsm->lmn", Gi, dG)
                  - np.einsum("ls,smn->lmn", Gi, dG))


def stress_tensor(x, eta_sign=1.0, prims=prim_fields):
    """T^{mu nu} (perfect fluid + Faraday, Sec. II.C), rho u^mu, and the
    4-metric at x.  eta_sign fixes the orientation eta^{0123} = eta_sign."""
    alpha, beta, g, _ = metric_fields(x)
    rho, p, v, E, B, _, _, _ = prims(x)
    G = four_metric(x)
    Gi = np.linalg.inv(G)
    W = 1.0 / np.sqrt(1.0 - v @ g @ v)
    u = np.concatenate([[W / alpha], W * (v - beta / alpha)])
    h = rho + GAM * p / (GAM - 1.0)               # rho (1 + eps) + p
    T = h * np.outer(u, u) + p * Gi
    sqrtmg = alpha * np.sqrt(np.linalg.det(g))
    eps_up = eta_sign * LC4 / sqrtmg                # epsilon^{mu nu a b}
    n_up = np.concatenate([[1.0 / alpha], -beta / alpha])
    n_dn = np.array([-alpha, 0.0, 0.0, 0.0])
    E4, B4 = np.concatenate([[0.0], E]), np.concatenate([[0.0], B])
    B4_dn = G @ B4
    F = (np.outer(n_up, E4) - np.outer(E4, n_up)
         + np.einsum("mnab,a,b->mn", eps_up, B4_dn, n_dn))
    F_dn = G @ F @ G
    # T_EM^{mu nu} = F^{mu a} F^{nu}_a - 1/4 g^{mu nu} F_{ab} F^{ab}
    Tem = np.einsum("ma,nb,ab->mn", F, F, G) - 0.25 * Gi * np.einsum("ab,ab->", F_dn, F)
    return T + Tem, rho * u, G


def paper_conserved(x):
    """D, S_i, tau of Eqs. conserved_dens, conserved_S, conserved_tau."""
    alpha, beta, g, _ = metric_fields(x)
    rho, p, v, E, B, _, _, _ = prim_fields(x)
    sg = np.sqrt(np.linalg.det(g))
    W = 1.0 / np.sqrt(1.0 - v @ g @ v)
    h = rho + GAM * p / (GAM - 1.0)
    E2, B2 = E @ g @ E, B @ g @ B
    S = sg * (h * W * W * (g @ v) + sg * np.einsum("ijk,j,k->i", LC3, E, B))
    tau = sg * (h * W * W - p + 0.5 * (E2 + B2)) - sg * rho * W
    return sg * rho * W, S, tau


def eta_sign_of_paper():
    """The orientation of the 4D Levi-Civita symbol for which the Eulerian
    momentum density of T^{mu nu} is the paper's S_i (Poynting E x B)."""
    x = X0
    alpha = metric_fields(x)[0]
    sg = np.sqrt(np.linalg.det(metric_fields(x)[2]))
    _, S, _ = paper_conserved(x)
    for s in (1.0, -1.0):
        T, _, G = stress_tensor(x, s)
        Smom = sg * alpha * (T @ G)[0, 1:]           # sqrt(gamma) alpha T^t_i
        if np.allclose(Smom, S, rtol=1e-12, atol=1e-12):
            return s
    raise AssertionError("no orientation reproduces Eq. conserved_S")


def exact_fluid_rhs(x, eta_sign, adot=0.0, bdot=(0.0, 0.0, 0.0), prims=prim_fields):
    """d_t (D, S_j, tau) from nabla_mu (rho u^mu) = 0 and nabla_mu T^{mu nu} = 0:
      d_t D = -d_i (sqrt(-g) rho u^i)
      d_t S_j = -d_i (sqrt(-g) T^i_j) + 1/2 sqrt(-g) T^{ab} d_j g_ab
      d_t (sqrt(gamma) n_a n_b T^ab) = -d_i (sqrt(-g) alpha T^{it})
                 + sqrt(-g) (T^{mu t} d_mu alpha - alpha Gamma^t_{ab} T^{ab})."""
    bdot = np.asarray(bdot, float)

    def sqrtmg(y):
        al, _, g, _ = metric_fields(y)
        return al * np.sqrt(np.linalg.det(g))

    def mass_flux(y):
        T, J, G = stress_tensor(y, eta_sign, prims)
        return sqrtmg(y) * J[1:]

    def mom_flux(y):          # sqrt(-g) T^i_j   [i, j]
        T, J, G = stress_tensor(y, eta_sign, prims)
        return sqrtmg(y) * (T @ G)[1:, 1:]

    def en_flux(y):           # sqrt(-g) alpha T^{it}
        T, J, G = stress_tensor(y, eta_sign, prims)
        return sqrtmg(y) * metric_fields(y)[0] * T[1:, 0]

    T, J, G = stress_tensor(x, eta_sign, prims)
    sq = sqrtmg(x)
    dD = -sum(d_num(lambda y: mass_flux(y)[k], x, k) for k in range(3))
    dS = np.zeros(3)
    for j in range(3):
        div = sum(d_num(lambda y: mom_flux(y)[k, j], x, k) for k in range(3))
        dgj = d_num(four_metric, x, j)
        dS[j] = -div + 0.5 * sq * np.einsum("ab,ab->", T, dgj)
    alpha = metric_fields(x)[0]
    dalpha = np.concatenate([[adot], grad(lambda y: metric_fields(y)[0], x)])
    Chr4 = christoffel4(x, adot, bdot)
    div = sum(d_num(lambda y: en_flux(y)[k], x, k) for k in range(3))
    dEn = -div + sq * (T[:, 0] @ dalpha - alpha * np.einsum("ab,ab->", Chr4[0], T))
    return dD, dS, dEn - dD


def exact_field_rhs(x, prims=prim_fields):
    """d_t (calB^i, calE^i, Phi, Psi, calQ) from the 3+1 Maxwell system of
    Sec. II.B with sigma = 0 (J^i = q v^i):
      (d_t - L_beta) E^i - eps^{ijk} D_j (alpha B_k) + alpha gamma^{ij} D_j psi
          = alpha K E^i - alpha J^i
      (d_t - L_beta) B^i + eps^{ijk} D_j (alpha E_k) + alpha gamma^{ij} D_j phi
          = alpha K B^i
      (d_t - L_beta) psi + alpha D_i E^i = alpha q - alpha kappa psi
      (d_t - L_beta) phi + alpha D_i B^i = -alpha kappa phi
      (d_t - L_beta) q + D_i (alpha J^i) = alpha K q
    and d_t (sqrt(gamma) X) = sqrt(gamma) d_t X + X d_t sqrt(gamma)."""
    def sg_of(y):
        return np.sqrt(np.linalg.det(metric_fields(y)[2]))

    alpha, beta, g, K = metric_fields(x)
    rho, p, v, E, B, psi, phi, q = prims(x)
    sg = sg_of(x)
    gi = np.linalg.inv(g)
    Ktr = np.einsum("ij,ij->", gi, K)
    dbeta = np.array([d_num(lambda y: metric_fields(y)[1], x, k) for k in range(3)])  # [k, i]

    def vec_grad(idx):
        return np.array([d_num(lambda y: prims(y)[idx], x, k) for k in range(3)])  # [k, i]

    dE, dB = vec_grad(3), vec_grad(4)
    dpsi = grad(lambda y: prims(y)[5], x)
    dphi = grad(lambda y: prims(y)[6], x)
    dq = grad(lambda y: prims(y)[7], x)

    def low(y, idx):
        al, _, gg, _ = metric_fields(y)
        return al * (gg @ prims(y)[idx])

    # eps^{ijk} d_j (alpha X_k): antisymmetry removes the connection
    curl_aB = np.einsum("ijk,jk->i", LC3, np.array([d_num(lambda y: low(y, 4), x, j)
                                                    for j in range(3)])) / sg
    curl_aE = np.einsum("ijk,jk->i", LC3, np.array([d_num(lambda y: low(y, 3), x, j)
                                                    for j in range(3)])) / sg
    divE = sum(d_num(lambda y: sg_of(y) * prims(y)[3][k], x, k) for k in range(3)) / sg
    divB = sum(d_num(lambda y: sg_of(y) * prims(y)[4][k], x, k) for k in range(3)) / sg
    divaJ = sum(d_num(lambda y: sg_of(y) * metric_fields(y)[0] * prims(y)[7] * prims(y)[2][k],
                      x, k) for k in range(3)) / sg
    divbeta = sum(d_num(lambda y: sg_of(y) * metric_fields(y)[1][k], x, k) for k in range(3)) / sg
    dt_sg = sg * (-alpha * Ktr + divbeta)

    LbE = beta @ dE - E @ dbeta
    LbB = beta @ dB - B @ dbeta
    Et = LbE + curl_aB - alpha * gi @ dpsi + alpha * Ktr * E - alpha * q * v
    Bt = LbB - curl_aE - alpha * gi @ dphi + alpha * Ktr * B
    psit = beta @ dpsi - alpha * divE + alpha * q - alpha * KAPPA * psi
    phit = beta @ dphi - alpha * divB - alpha * KAPPA * phi
    qt = beta @ dq - divaJ + alpha * Ktr * q
    dens = lambda Xt, X: sg * Xt + X * dt_sg
    return dens(Bt, B), dens(Et, E), dens(phit, phi), dens(psit, psi), dens(qt, q)


def exact_rhs(eta_sign, adot=0.0, bdot=(0.0, 0.0, 0.0)):
    dD, dS, dtau = exact_fluid_rhs(X0, eta_sign, adot, bdot)
    dB, dE, dPhi, dPsi, dQ = exact_field_rhs(X0)
    return np.concatenate([[dD], dS, [dtau], dB, dE, [dPhi], [dPsi], [dQ]])


# ----------------------------------------------------------- the oracle

def oracle_rhs_at_centre(h, metric_fn=metric_fields, prims=prim_fields, recon=2):
    """The oracle's F(U) at the centre cell of a 7^3 grid of spacing h whose
    centre cell sits at X0 (every stencil point is inside the grid)."""
    n = 7
    idx = np.arange(n) - 3
    pts = [(X0[0] + i * h, X0[1] + j * h, X0[2] + k * h)
           for k in idx for j in idx for i in idx]
    N = n ** 3
    alpha, beta, g6, K6, prim = (np.zeros(N), np.zeros((3, N)), np.zeros((6, N)),
                                 np.zeros((6, N)), np.zeros((14, N)))
    for c, x in enumerate(pts):
        x = np.array(x)
        a, b, g, K = metric_fn(x)
        alpha[c], beta[:, c] = a, b
        g6[:, c] = [g[0, 0], g[0, 1], g[0, 2], g[1, 1], g[1, 2], g[2, 2]]
        K6[:, c] = [K[0, 0], K[0, 1], K[0, 2], K[1, 1], K[1, 2], K[2, 2]]
        rho, p, v, E, B, psi, phi, q = prims(x)
        prim[:, c] = np.concatenate([[rho, p], v, E, B, [psi, phi, q]])
    m = oracle.Metric(alpha, beta, g6, K6)
    P = dict(n=(n, n, n), dx=(h, h, h), bc=(1, 1, 1), recon=recon, gamma_eos=GAM, kappa=KAPPA,
             sigma0=0.0, qflux_mode=1)
    out = oracle.rhs(P, m, prim.reshape(14, n, n, n))
    return out.reshape(14, N)[:, N // 2]


ROWS = ["D", "S_x", "S_y", "S_z", "tau", "B^x", "B^y", "B^z", "E^x", "E^y", "E^z",
        "Phi", "Psi", "Q"]


def test_levi_civita_orientation_and_conserved_vector():
    """With the orientation that reproduces Eq. conserved_S, the projections
    of T^{mu nu} also give Eq. conserved_tau and D = sqrt(-g) rho u^t."""
    s = eta_sign_of_paper()
    T, J, G = stress_tensor(X0, s)
    alpha, _, g, _ = metric_fields(X0)
    sg = np.sqrt(np.linalg.det(g))
    D, S, tau = paper_conserved(X0)
    assert abs(alpha * sg * J[0] - D) < 1e-13 * D
    assert abs(sg * alpha ** 2 * T[0, 0] - D - tau) < 1e-12 * (tau + D)


def test_gauge_rates_of_lapse_and_shift_drop_out():
    """The time derivatives of lapse and shift do not enter the evolution of
    the conserved fluid variables (a check of the 4D machinery itself)."""
    s = eta_sign_of_paper()
    a = exact_fluid_rhs(X0, s)
    b = exact_fluid_rhs(X0, s, adot=0.37, bdot=(0.2, -0.5, 0.11))
    for u, w in zip(a, b):
        assert np.allclose(u, w, rtol=1e-10, atol=1e-11)


def test_oracle_rhs_converges_to_the_covariant_time_derivative():
    """Every row of the oracle's -d_k F^k + S converges at second order to
    the time derivative given by the covariant equations (curved metric with
    lapse, shift, off-diagonal gamma_ij, K_ij; nonzero cleaning scalars,
    charge and damping)."""
    exact = exact_rhs(eta_sign_of_paper())
    hs = (0.04, 0.02, 0.01)
    errs = np.array([np.abs(oracle_rhs_at_centre(h) - exact) for h in hs])
    # scale of each row: its exact value or, if that is small, the largest
    # row of its group
    scale = np.maximum(np.abs(exact), 0.05 * np.abs(exact).max())
    rel = errs / scale
    ratio = rel[:-1] / np.maximum(rel[1:], 1e-300)
    for r in range(14):
        assert rel[-1, r] < 2e-3, (ROWS[r], rel[:, r])
        # second order: the error falls ~4x per halving of h
        assert ratio[-1, r] > 3.0 or rel[-1, r] < 1e-7, (ROWS[r], rel[:, r], ratio[:, r])


# ------------------------------------------- hydrostatic Rindler slicing

G_RINDLER = 0.4
RHO_H = 1.0
C_H = 2.0


def rindler_metric(x):
    return 1.0 + G_RINDLER * x[0], np.zeros(3), np.eye(3), np.zeros((3, 3))


def rindler_prims(x):
    """Static fluid in alpha = 1 + g x with d_x p = -(e + p) d_x ln alpha,
    e + p = rho + Gamma p / (Gamma - 1) at constant rho:
    rho + a p = C alpha^{-a}, a = Gamma / (Gamma - 1)."""
    a = GAM / (GAM - 1.0)
    al = 1.0 + G_RINDLER * x[0]
    p = (C_H * al ** (-a) - RHO_H) / a
    z = np.zeros(3)
    return RHO_H, p, z, z, z, 0.0, 0.0, 0.0


def test_hydrostatic_fluid_in_rindler_lapse_is_static_to_second_order():
    """Exact equilibrium: the oracle's right-hand side of S_x (pressure
    gradient against the lapse gradient, each O(1)) vanishes at second order
    and every other row stays at the reconstruction's rounding-to-jump level."""
    x = X0
    a = GAM / (GAM - 1.0)
    al = 1.0 + G_RINDLER * x[0]
    p = (C_H * al ** (-a) - RHO_H) / a
    term = (RHO_H + a * p) * G_RINDLER / al      # size of each balancing term
    errs = []
    for h in (0.04, 0.02, 0.01):
        r = oracle_rhs_at_centre(h, rindler_metric, rindler_prims)
        # tau moves only by the HLLE dissipation of the 5th-order jump
        # between the reconstructed pressures at a face
        assert np.abs(np.delete(r, 1)).max() < 1e-6 * term
        errs.append(abs(r[1]) / term)
    assert errs[-1] < 1e-4 and errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs
