"""Runs in the form of the paper's program (Sec. 4): a model in the input form
(neighbour list, hoppings, on-site energies, bond x-displacements, length and
volume), an energy grid, the time steps (step sizes, not cumulative times) and
the keywords of its parameter file in; per random vector the density of states
rho(E), rho(E) C_vv(E, t) for the VAC rows and rho(E) dX^2(E, t) for the MSD
rows out, one row per vector (per vector and time step), as the paper's output
files hold them; the running conductivities follow from the rows by
``sigma_vac`` and ``sigma_msd``.

Orchestration only: every number comes from the library's kernels behind the
gqt_* calls (moments, evolution, reconstruction, time integration).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import (GQT_FP32_ACC64, GQT_FP64, gqt_build_hamiltonian, gqt_dos_moments, gqt_kpm_reconstruct,
               gqt_msd_init, gqt_msd_moments, gqt_random_phase, gqt_sigma_msd, gqt_sigma_vac, gqt_vac_init,
               gqt_vac_moments)


@dataclasses.dataclass
class Params:
    """The keywords of the paper's parameter file, with its defaults: whether to
    compute the VAC and the MSD rows, the number of random vectors N_r (1), the
    number of Chebyshev moments N_m (1000) and the energy scale dE (10) with
    H/dE inside [-1, 1]."""
    calculate_vac: bool = False
    calculate_msd: bool = False
    number_of_random_vectors: int = 1
    number_of_moments: int = 1000
    energy_max: float = 10.0


def run(lattice, energies, params: Params, time_steps=None, seed: int = 1705013870, precision: int = GQT_FP64,
        device: str = "cuda") -> dict:
    """DOS for every run, VAC and MSD rows as the keywords ask.  Random vector r
    is stream r of ``seed`` (the library's random-phase generator).  Returns
    numpy arrays: ``dos`` [N_r][NE], ``vac`` and ``msd`` [N_r * N_t][NE] (the N_t
    rows of vector 0 first), and ``time_steps``."""
    if (params.calculate_vac or params.calculate_msd) and time_steps is None:
        raise ValueError("time_steps are needed for the VAC or MSD rows")
    ham = gqt_build_hamiltonian(lattice, params.energy_max, precision)
    M = int(params.number_of_moments)
    E = torch.as_tensor(np.asarray(energies, np.float64), device=device)
    dts = None if time_steps is None else np.asarray(time_steps, np.float64)
    cd = torch.complex128 if precision == GQT_FP64 else torch.complex64
    n_over_omega = ham.n / ham.volume
    out = {"dos": [], "vac": [], "msd": [], "time_steps": dts}

    def rows(mu):
        rec = torch.empty((mu.shape[0], E.numel()), dtype=torch.float64, device=device)
        gqt_kpm_reconstruct(mu.contiguous(), E, params.energy_max, n_over_omega, rec)
        return rec.cpu().numpy()

    for r in range(int(params.number_of_random_vectors)):
        phi = torch.empty((ham.n, 1), dtype=cd, device=device)
        gqt_random_phase(ham, seed, 1, phi, first_vector=r)
        mu = torch.empty((1, 1, M), dtype=torch.float64, device=device)
        gqt_dos_moments(ham, phi, 1, M, mu)
        out["dos"].append(rows(mu.view(1, M))[0])
        if params.calculate_vac:
            a, b = torch.empty_like(phi), torch.empty_like(phi)
            gqt_vac_init(ham, phi, a, b, 1)
            vac = torch.empty((dts.size, 1, 1, M), dtype=torch.float64, device=device)
            gqt_vac_moments(ham, a, b, 1, dts, M, vac)
            out["vac"].append(rows(vac.view(dts.size, M)))
        if params.calculate_msd:
            p, px = torch.empty_like(phi), torch.empty_like(phi)
            gqt_msd_init(ham, phi, p, px, 1)
            msd = torch.empty((dts.size, 1, 1, M), dtype=torch.float64, device=device)
            gqt_msd_moments(ham, p, px, 1, dts, M, msd)
            out["msd"].append(rows(msd.view(dts.size, M)))
    out["dos"] = np.stack(out["dos"])
    for k in ("vac", "msd"):
        out[k] = np.concatenate(out[k]) if out[k] else None
    return out


def sigma_vac(vac_rows, time_steps, device: str = "cuda") -> np.ndarray:
    """Running conductivity from the rows of one vector, rho C_vv [N_t][NE] at
    t_0 = 0 .. t_{N_t - 1}: the time integral by the trapezoid rule (library call)."""
    v = torch.as_tensor(np.ascontiguousarray(vac_rows, np.float64), device=device)
    s = torch.empty_like(v)
    gqt_sigma_vac(v, np.asarray(time_steps, np.float64), s)
    return s.cpu().numpy()


def sigma_msd(msd_rows, time_steps, device: str = "cuda") -> np.ndarray:
    """Running conductivity from the rows of one vector, rho dX^2 [N_t][NE] at
    t_1 .. t_{N_t}: half the time derivative at the step midpoints (library call)."""
    v = torch.as_tensor(np.ascontiguousarray(msd_rows, np.float64), device=device)
    s = torch.empty_like(v)
    gqt_sigma_msd(v, np.asarray(time_steps, np.float64), s)
    return s.cpu().numpy()


__all__ = ["Params", "run", "sigma_vac", "sigma_msd", "GQT_FP64", "GQT_FP32_ACC64"]
