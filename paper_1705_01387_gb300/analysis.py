"""Host post-processing of reconstructed DOS, VAC and MSD (Sec. 2.3), the role the
paper gives to its plotting scripts: semiclassical conductivity, relaxation time,
mean free path, propagation length and localisation length.

Inputs are the library's reconstructed arrays: ``dos`` [NE] = rho(E) (Eq. 25),
``vac`` [Nt, NE] = rho C_vv(E, t_k) (Eq. 26, rows t_0 = 0 .. t_{Nt-1}),
``msd`` [Nt, NE] = rho dX^2(E, t_k) (Eq. 27, rows t_1 .. t_Nt), and running
conductivities ``sigma`` [Nt, NE] (Eqs. 2, 5).  Units hbar = e = 1.
"""
from __future__ import annotations

import numpy as np


def group_velocity(dos, vac):
    """v_x(E) = sqrt(C_vv(E, 0)) with C_vv = (rho C_vv) / rho (Sec. 5.1)."""
    dos = np.asarray(dos, np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.sqrt(np.maximum(np.asarray(vac, np.float64)[0] / dos, 0.0))


def semiclassical(dos, vac, sigma):
    """sigma_sc(E) = max_t sigma(E, t) (Sec. 5.1), tau = sigma_sc / (rho v^2) (Eq. 8),
    lambda = v tau (Eq. 9), D = v^2 tau (Eq. 10).  Returns a dict of [NE] arrays."""
    dos = np.asarray(dos, np.float64)
    v = group_velocity(dos, vac)
    sig_sc = np.max(np.asarray(sigma, np.float64), axis=0)
    with np.errstate(invalid="ignore", divide="ignore"):
        tau = sig_sc / (dos * v * v)
    return {"sigma_sc": sig_sc, "velocity": v, "tau": tau, "mfp": v * tau, "diffusivity": v * v * tau}


def propagation_length(dos, msd):
    """L(E, t) = 2 sqrt(dX^2(E, t)) with dX^2 = (rho dX^2) / rho (Eq. 11); [Nt, NE]."""
    dos = np.asarray(dos, np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        return 2.0 * np.sqrt(np.maximum(np.asarray(msd, np.float64) / dos[None, :], 0.0))


def xi_saturation(L):
    """xi(E) = lim_t L(E, t) / 2 pi (Eq. 12), taken at the last time row."""
    return np.asarray(L, np.float64)[-1] / (2.0 * np.pi)


def xi_fit(L, sigma, width: float = 1.0, L_range=None):
    """Fit ln g = c - L / (2 xi) with g(E, L) = sigma(E, L) * width / L (Eq. 36) for
    one energy: L and sigma are the [Nt] columns at that energy; L_range = (lo, hi)
    selects the rows used.  Returns xi."""
    L = np.asarray(L, np.float64)
    g = np.asarray(sigma, np.float64) * width / L
    m = np.isfinite(g) & (g > 0) & (L > 0)
    if L_range is not None:
        m &= (L >= L_range[0]) & (L <= L_range[1])
    if m.sum() < 2:
        return float("nan")
    slope, _ = np.polyfit(L[m], np.log(g[m]), 1)
    return float(-1.0 / (2.0 * slope))
