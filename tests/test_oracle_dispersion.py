"""Oracle pin: linear resistive Alfven waves in flat space.

Small transverse perturbations (v^y, B^y, E^z) of a uniform plasma at rest
with B = B0 x-hat obey Faraday's and Ampere's laws (Eqs. B_evol, E_evol),
the y-momentum equation with the Lorentz force J^z B0, and the resistive
Ohm law J^z = sigma (E^z - v^y B0) (Eq. Ohm with Gamma = 1 to first
order).  A plane wave exp(i(kx - omega t)) then requires

    omega^3 + i sigma (1 + a) omega^2 - k^2 omega - i sigma a k^2 = 0,
    a = B0^2 / h,  h = rho + Gamma_eos/(Gamma_eos - 1) p,

whose roots tend to the relativistic Alfven branch omega^2 = k^2 B0^2/(h + B0^2)
as sigma -> inf and to light waves omega = +-k as sigma -> 0.  Each test
starts the oracle on one eigenvector of this system and measures omega from
the phase and decay of the Fourier coefficient of B^y; the measured value
must converge to the analytic root as the grid is refined.  A dropped source
term, a wrong sign in the v x B term or a wrong enthalpy moves the root by
O(1), far outside the discretisation error checked here."""
import numpy as np
import pytest

import workloads as W
from tests.helpers import run_oracle

K_WAVE = 2.0 * np.pi
B0, RHO, P, GAM = 1.0, 1.0, 1.0, 4.0 / 3.0
H = RHO + GAM / (GAM - 1.0) * P


def dispersion_roots(k, sigma):
    a = B0 * B0 / H
    return np.roots([1.0, 1j * sigma * (1.0 + a), -k * k, -1j * sigma * a * k * k])


def forward_root(sigma):
    """Root travelling in +x that decays least."""
    r = [w for w in dispersion_roots(K_WAVE, sigma) if w.real > 1e-8]
    return max(r, key=lambda z: z.imag)


def measured_omega(n, sigma, recon="weno5", t_end=0.375, amp=1e-6):
    w = forward_root(sigma)
    dx = 1.0 / n
    params = W.base_params((n, 1, 1), (0.0, 0.0, 0.0), (dx, dx, dx), (0, 0, 0), recon,
                           GAM, sigma)
    x = (np.arange(n) + 0.5) * dx
    e = amp * np.exp(1j * K_WAVE * x)
    b = -K_WAVE / w * e                               # Faraday
    v = -B0 * (w * w - K_WAVE ** 2) / (H * w * w) * e  # Ampere + momentum
    prim = np.zeros((14, 1, 1, n))
    prim[0], prim[1], prim[8] = RHO, P, B0
    prim[3, 0, 0], prim[9, 0, 0], prim[7, 0, 0] = v.real, b.real, e.real
    dt = 0.25 * dx
    nsteps = int(round(t_end / dt))
    wl = W.Workload("linear_alfven", params, prim, dt, nsteps)
    st, _, pr, _ = run_oracle(wl, nsteps)
    assert st == 0
    c0 = np.sum(b.real * np.exp(-1j * K_WAVE * x))
    c1 = np.sum(pr[9, 0, 0] * np.exp(-1j * K_WAVE * x))
    # |Re omega| t < pi keeps the complex logarithm on its principal branch
    return w, 1j * np.log(c1 / c0) / (nsteps * dt)


def test_cubic_limits():
    """The cubic itself: ideal and vacuum limits."""
    vA = B0 / np.sqrt(H + B0 * B0)
    w = dispersion_roots(K_WAVE, 1e7)
    assert np.min(np.abs(w - K_WAVE * vA)) < 1e-5 * K_WAVE
    w = dispersion_roots(K_WAVE, 0.0)
    assert np.min(np.abs(w - K_WAVE)) < 1e-12


@pytest.mark.parametrize("sigma", [0.0, 3.0, 10.0])
def test_oracle_resistive_alfven_dispersion(sigma):
    """Second-order convergence of the measured omega to the analytic root
    (sigma = 3: damped light-like branch; sigma = 10: damped Alfven branch;
    sigma = 0: undamped light wave, omega = k)."""
    w, w32 = measured_omega(32, sigma)
    _, w64 = measured_omega(64, sigma)
    e32, e64 = abs(w32 - w), abs(w64 - w)
    assert e64 < 2e-3 * abs(w), (sigma, w, w64)
    assert 3.0 < e32 / e64 < 5.5, (sigma, e32, e64)
