"""GPUQT-style runs through the driver (the paper's parameter-file keywords in;
per random vector the DOS, rho C_vv and rho dX^2 rows out, Sec. 4) on the GPU:
every row equals the oracle's reconstruction of the oracle's moments for the
same seeded vectors (1e-10 normalised), and the running conductivities the
oracle's time integral and derivative (1e-9)."""
import numpy as np
import pytest

import gqt_synth as S
import oracle as O

torch = pytest.importorskip("torch")
g = pytest.importorskip("paper_1705_01387_gb300")
from paper_1705_01387_gb300 import driver  # noqa: E402

pytestmark = pytest.mark.gpu


def nerr(x, y):
    return float(np.max(np.abs(np.asarray(x) - np.asarray(y))) / max(float(np.max(np.abs(y))), 1e-300))


@pytest.mark.parametrize("precision", [g.GQT_FP64])
def test_driver_rows_match_oracle(precision):
    lat = S.honeycomb(16, 12, -2.7, 1.0, seed=71)
    dE = S.energy_scale_rule(3, -2.7, 1.0)
    params = driver.Params(calculate_vac=True, calculate_msd=True, number_of_random_vectors=2, number_of_moments=64,
                           energy_max=dE)
    E = np.linspace(-8.0, 8.0, 41)
    dts = np.array([0.2, 0.4, 0.4])
    seed = 99
    out = driver.run(lat, E, params, time_steps=dts, seed=seed, precision=precision)
    assert out["dos"].shape == (2, E.size) and out["vac"].shape == (2 * dts.size, E.size)
    h = O.Hamiltonian(lat, dE)
    nO = lat.n / lat.volume
    Np = [O.np_rule(dE * t, 64) for t in dts]
    for r in range(2):
        phi = S.random_phase(lat.n, 1, seed=seed, first_vector=r)[:, 0]
        dos = O.kpm_reconstruct(h.dos_moments(phi, 64).real, E, dE, nO)[0]
        vac = O.kpm_reconstruct(h.vac_moments(phi, dts, Np, 64), E, dE, nO)
        msd = O.kpm_reconstruct(h.msd_moments(phi, dts, Np, 64), E, dE, nO)
        rows = slice(r * dts.size, (r + 1) * dts.size)
        assert nerr(out["dos"][r], dos) < 1e-10
        assert nerr(out["vac"][rows], vac) < 1e-10
        assert nerr(out["msd"][rows], msd) < 1e-10
        assert nerr(driver.sigma_vac(out["vac"][rows], dts), O.sigma_vac(vac, dts)) < 1e-9
        assert nerr(driver.sigma_msd(out["msd"][rows], dts), O.sigma_msd(msd, dts)) < 1e-9


def test_driver_dos_only():
    """Without the VAC and MSD keywords only the DOS rows come back, and no time
    steps are needed."""
    lat = S.square(20, 17, -1.0, 2.0, seed=72)
    dE = S.energy_scale_rule(4, -1.0, 2.0)
    out = driver.run(lat, np.linspace(-3, 3, 13), driver.Params(number_of_moments=32, energy_max=dE))
    assert out["dos"].shape == (1, 13) and out["vac"] is None and out["msd"] is None
    phi = S.random_phase(lat.n, 1, seed=1705013870)[:, 0]
    ref = O.kpm_reconstruct(O.Hamiltonian(lat, dE).dos_moments(phi, 32).real, np.linspace(-3, 3, 13), dE,
                            lat.n / lat.volume)[0]
    assert nerr(out["dos"][0], ref) < 1e-10
