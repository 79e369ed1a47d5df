"""Independent flat-space physics and coordinate transformations for the pins.

Nothing here is taken from the oracle.  The flat-space quantities are the
textbook special-relativistic ones: the perfect-fluid stress-energy tensor
T^{mu nu} = (e + p) u^mu u^nu + p eta^{mu nu}; electromagnetic energy density
(E^2 + B^2)/2, Poynting momentum E x B and Maxwell stress
T^{ij} = -E^i E^j - B^i B^j + delta^{ij}(E^2 + B^2)/2; Maxwell's equations in
conservation form with the cleaning scalars (dt B + curl E + grad phi = 0,
dt E - curl B + grad psi = -J, dt phi + div B = ..., dt psi + div E = ...)
and the relativistic Ohm's law J = q v + W sigma (E + v x B - (v.E) v).

A curved (constant) metric is produced from flat space by a linear change of
spatial coordinates x = A y (gamma_ij = (A^-T A^-1)_ij, sqrt(gamma) = 1/det A),
a constant lapse (proper time = alpha t) and a constant shift
(x' = x - beta t).  Conserved densities, their fluxes and vectors transform as
tensor densities; the fluxes pick up alpha F - beta^k U.  Comparing the oracle
in the curved frame with the transformed textbook values checks every index
position, sqrt(gamma) factor and Levi-Civita convention of the 3+1 formulas.
"""
import numpy as np

LC = np.zeros((3, 3, 3))
LC[0, 1, 2] = LC[1, 2, 0] = LC[2, 0, 1] = 1.0
LC[0, 2, 1] = LC[2, 1, 0] = LC[1, 0, 2] = -1.0


def textbook(prim, gamma_eos, sigma=0.0):
    """Flat-space conserved vector U (14) and fluxes F[k] (3 x 14)."""
    rho, p = prim[0], prim[1]
    v, E, B = prim[2:5], prim[5:8], prim[8:11]
    psi, phi, q = prim[11], prim[12], prim[13]
    W = 1.0 / np.sqrt(1.0 - v @ v)
    u = W * np.concatenate([[1.0], v])
    e = rho + p / (gamma_eos - 1.0)           # rest-mass + internal energy
    eta_inv = np.diag([-1.0, 1.0, 1.0, 1.0])
    T = (e + p) * np.outer(u, u) + p * eta_inv
    Tem = np.zeros((4, 4))
    Tem[0, 0] = 0.5 * (E @ E + B @ B)
    Tem[0, 1:] = Tem[1:, 0] = np.cross(E, B)
    Tem[1:, 1:] = (-np.outer(E, E) - np.outer(B, B)
                   + 0.5 * np.eye(3) * (E @ E + B @ B))
    T = T + Tem
    D = rho * u[0]
    U = np.zeros(14)
    U[0] = D
    U[1:4] = T[0, 1:]
    U[4] = T[0, 0] - D
    U[5:8] = B
    U[8:11] = E
    U[11] = phi
    U[12] = psi
    U[13] = q
    J = q * v + W * sigma * (E + np.cross(v, B) - (v @ E) * v)
    F = np.zeros((3, 14))
    for k in range(3):
        F[k, 0] = rho * u[1 + k]
        F[k, 1:4] = T[1 + k, 1:]
        F[k, 4] = T[0, 1 + k] - rho * u[1 + k]
        # flux of B^i in direction k: eps_{ikj} E_j + delta_ik phi
        F[k, 5:8] = np.einsum("ij,j->i", LC[:, k, :], E) + np.eye(3)[k] * phi
        F[k, 8:11] = -np.einsum("ij,j->i", LC[:, k, :], B) + np.eye(3)[k] * psi
        F[k, 11] = B[k]
        F[k, 12] = E[k]
        F[k, 13] = J[k]
    return U, F


def g6_of(g):
    return np.array([g[0, 0], g[0, 1], g[0, 2], g[1, 1], g[1, 2], g[2, 2]])


def metric_of(A):
    """3-metric (6 comps) of the coordinates x = A y, and sqrt(gamma)."""
    Ai = np.linalg.inv(A)
    g = Ai.T @ Ai
    return g6_of(g), 1.0 / np.linalg.det(A)


def transform_prim(prim, A):
    out = prim.copy()
    for s in (slice(2, 5), slice(5, 8), slice(8, 11)):
        out[s] = A @ prim[s]
    return out


def transform_cons(U, A):
    """Densitised conserved vector under x = A y (det A > 0)."""
    J = np.linalg.det(A)
    Ai = np.linalg.inv(A)
    out = U / J
    out[1:4] = Ai.T @ U[1:4] / J          # covector density
    out[5:8] = A @ U[5:8] / J             # vector densities
    out[8:11] = A @ U[8:11] / J
    return out


def transform_flux(F, A):
    """F[k, comp] flat -> curved: direction index is a vector index."""
    J = np.linalg.det(A)
    Ai = np.linalg.inv(A)
    out = np.einsum("kl,lc->kc", A, F) / J
    # S_i: mixed tensor density F^k_i -> A F A^-1
    out[:, 1:4] = A @ F[:, 1:4] @ Ai / J
    # B^i, E^i: F^{k i} -> A F A^T
    out[:, 5:8] = A @ F[:, 5:8] @ A.T / J
    out[:, 8:11] = A @ F[:, 8:11] @ A.T / J
    return out


def random_A(rng, strength=0.4):
    while True:
        A = np.eye(3) + strength * rng.uniform(-1, 1, (3, 3))
        if np.linalg.det(A) > 0.3:
            return A


def random_flat_prim(rng, gamma_eos=2.0, vmax=0.8, scale=1.0):
    prim = np.zeros(14)
    prim[0] = rng.uniform(0.1, 2.0)
    prim[1] = rng.uniform(0.05, 2.0)
    d = rng.standard_normal(3)
    prim[2:5] = d / np.linalg.norm(d) * rng.uniform(0, vmax)
    prim[5:8] = scale * rng.standard_normal(3) * 0.5
    prim[8:11] = scale * rng.standard_normal(3)
    prim[11:14] = rng.standard_normal(3) * 0.3
    return prim


# ------------------------------------------- many points at once (vectorised)

def random_prims(rng, n, gamma_eos=2.0, vmax=0.8, scale=1.0):
    """n random flat-space primitive states (rows), as random_flat_prim."""
    prim = np.zeros((n, 14))
    prim[:, 0] = rng.uniform(0.1, 2.0, n)
    prim[:, 1] = rng.uniform(0.05, 2.0, n)
    d = rng.standard_normal((n, 3))
    prim[:, 2:5] = d / np.linalg.norm(d, axis=1)[:, None] * rng.uniform(0, vmax, n)[:, None]
    prim[:, 5:8] = scale * rng.standard_normal((n, 3)) * 0.5
    prim[:, 8:11] = scale * rng.standard_normal((n, 3))
    prim[:, 11:14] = rng.standard_normal((n, 3)) * 0.3
    return prim


def textbook_cons_many(prim, gamma_eos):
    """Flat-space conserved vectors of n states (rows): D = rho W,
    S = (e + p) W^2 v + E x B, tau = (e + p) W^2 - p + (E^2 + B^2)/2 - D."""
    rho, p = prim[:, 0], prim[:, 1]
    v, E, B = prim[:, 2:5], prim[:, 5:8], prim[:, 8:11]
    W = 1.0 / np.sqrt(1.0 - np.einsum("ni,ni->n", v, v))
    w = (rho + p / (gamma_eos - 1.0) + p) * W * W
    U = np.zeros_like(prim)
    U[:, 0] = rho * W
    U[:, 1:4] = w[:, None] * v + np.cross(E, B)
    U[:, 4] = w - p + 0.5 * (np.einsum("ni,ni->n", E, E) + np.einsum("ni,ni->n", B, B)) - U[:, 0]
    U[:, 5:8] = B
    U[:, 8:11] = E
    U[:, 11] = prim[:, 12]
    U[:, 12] = prim[:, 11]
    U[:, 13] = prim[:, 13]
    return U


def random_A_many(rng, n, strength=0.4):
    A = np.eye(3) + strength * rng.uniform(-1, 1, (n, 3, 3))
    bad = np.linalg.det(A) <= 0.3
    while bad.any():
        A[bad] = np.eye(3) + strength * rng.uniform(-1, 1, (int(bad.sum()), 3, 3))
        bad = np.linalg.det(A) <= 0.3
    return A


def metric_of_many(A):
    Ai = np.linalg.inv(A)
    g = np.einsum("nki,nkj->nij", Ai, Ai)
    g6 = np.stack([g[:, 0, 0], g[:, 0, 1], g[:, 0, 2], g[:, 1, 1], g[:, 1, 2], g[:, 2, 2]], 1)
    return g6, 1.0 / np.linalg.det(A)


def transform_prim_many(prim, A):
    out = prim.copy()
    for s in (slice(2, 5), slice(5, 8), slice(8, 11)):
        out[:, s] = np.einsum("nij,nj->ni", A, prim[:, s])
    return out


def transform_cons_many(U, A):
    J = np.linalg.det(A)
    Ai = np.linalg.inv(A)
    out = U / J[:, None]
    out[:, 1:4] = np.einsum("nji,nj->ni", Ai, U[:, 1:4]) / J[:, None]
    out[:, 5:8] = np.einsum("nij,nj->ni", A, U[:, 5:8]) / J[:, None]
    out[:, 8:11] = np.einsum("nij,nj->ni", A, U[:, 8:11]) / J[:, None]
    return out
