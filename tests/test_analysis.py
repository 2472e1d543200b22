"""Post-processing (Sec. 2.3, Eqs. 7-12, 36) against closed forms: an exponential
VAC gives back its velocity, relaxation time and mean free path; a saturating MSD
gives back xi; an exponential conductance gives back the fitted xi."""
import numpy as np

from paper_1705_01387_gb300 import analysis as A


def test_exponential_vac_recovers_tau_and_mfp():
    """C_vv = v^2 exp(-t/tau) (Eq. 7) integrates to sigma(t) = rho v^2 tau (1 - exp(-t/tau)),
    whose maximum is the semiclassical rho v^2 tau (Eq. 8)."""
    rho, v, tau = np.array([0.3, 0.1]), np.array([1.2, 2.0]), np.array([0.8, 2.5])
    t = np.linspace(0, 60, 2001)
    vac = rho[None] * v[None] ** 2 * np.exp(-t[:, None] / tau[None])
    sigma = rho[None] * v[None] ** 2 * tau[None] * (1 - np.exp(-t[:, None] / tau[None]))
    out = A.semiclassical(rho, vac, sigma)
    assert np.allclose(out["velocity"], v, rtol=1e-12)
    assert np.allclose(out["tau"], tau, rtol=1e-8)
    assert np.allclose(out["mfp"], v * tau, rtol=1e-8)
    assert np.allclose(out["diffusivity"], v ** 2 * tau, rtol=1e-8)


def test_propagation_and_localisation_length():
    rho = np.array([0.5])
    t = np.linspace(0.1, 200, 400)
    xi = 7.0
    dx2 = (np.pi * xi) ** 2 * (1 - np.exp(-t / 5.0)) ** 2  # L = 2 sqrt(dX^2) -> 2 pi xi
    L = A.propagation_length(rho, rho[None] * dx2[:, None])
    assert np.allclose(L[:, 0], 2 * np.sqrt(dx2))
    assert abs(A.xi_saturation(L)[0] - xi) < 1e-6


def test_xi_fit_exponential_conductance():
    """g = sigma W / L = g0 exp(-L / 2 xi) (Eq. 36) fitted over a chosen L range."""
    L = np.linspace(1, 80, 50)
    xi = 12.5
    sigma = 3.0 * np.exp(-L / (2 * xi)) * L
    assert abs(A.xi_fit(L, sigma) - xi) < 1e-9
    assert abs(A.xi_fit(L, sigma, L_range=(10, 40)) - xi) < 1e-9
