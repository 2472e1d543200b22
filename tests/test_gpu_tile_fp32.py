"""Temporal blocking of the FP32 multi-vector moment rows (k_cheb2_honey_wv):
two Chebyshev orders (Eq. 21) per launch on FP32-storage honeycomb handles with
R = 2, 4, 8 or 16 random vectors, the precision workload's form (R = 8, 1%
vacancies).  Through the C ABI, the DOS, VAC and MSD rows must match

  - the serial FP64 oracle within the FP32-storage bounds (1e-5 normalised on
    DOS moments, 1e-4 on VAC and MSD rows), for the first and last vector;
  - the same handle with one order per launch within 1e-10: the blocked kernel
    computes the chains with the same fused multiply-adds in the same order, so
    only the split of the FP64 moment sums over CTAs differs;

and the blocked kernel must actually have run (profile families 12 and 13).
"""
import numpy as np
import pytest

import gqt_synth as S
import oracle as O

torch = pytest.importorskip("torch")
g = pytest.importorskip("paper_1705_01387_gb300")

pytestmark = pytest.mark.gpu


def nerr(x, y):
    x = np.asarray(x)
    y = np.asarray(y)
    return float(np.max(np.abs(x - y)) / max(float(np.max(np.abs(y))), 1e-300))


def _blocked_launches(fn):
    g.gqt_profile_start()
    fn()
    torch.cuda.synchronize()
    _, n = g.gqt_profile_stop(14)
    return int(n[12] + n[13])


MODELS = {
    "honeycomb64x32": lambda: (S.honeycomb(64, 32, -2.7, 2.0, seed=23), S.energy_scale_rule(3, -2.7, 2.0)),
    "honeycomb64x40_vac": lambda: (S.honeycomb(64, 40, -2.7, 0.5, seed=24, vacancy_frac=0.01),
                                   S.energy_scale_rule(3, -2.7, 0.5)),
    "honeycomb64x32_phases": lambda: (S.with_random_bond_phases(S.honeycomb(64, 32, -2.7, 2.0, seed=25), 26),
                                      S.energy_scale_rule(3, -2.7, 2.0)),
}


def _rows(lat, dE, R, M, tiling, phi, dts, Np):
    ham = g.gqt_build_hamiltonian(lat, dE, g.GQT_FP32_ACC64)
    g.gqt_set_temporal_blocking(ham, tiling)
    d = torch.from_numpy(phi.astype(np.complex64)).cuda()
    dos = np.empty((1, R, M))
    vac = np.empty((1, 1, R, M))
    msd = np.empty((1, 1, R, M))
    a, b, p, px = (torch.empty_like(d) for _ in range(4))
    g.gqt_vac_init(ham, d, a, b, R)
    g.gqt_msd_init(ham, d, p, px, R)

    def run():
        g.gqt_dos_moments(ham, d, R, M, dos)
        g.gqt_vac_moments(ham, a, b, R, dts, M, vac, Np=Np)
        g.gqt_msd_moments(ham, p, px, R, dts, M, msd, Np=Np)

    n = _blocked_launches(run)
    return n, dos[0], vac[0, 0], msd[0, 0]


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("R", [2, 4, 8, 16])
@pytest.mark.parametrize("M", [1, 3, 4, 9, 130])
def test_blocked_fp32_rows_match_oracle_and_single_order(name, R, M):
    lat, dE = MODELS[name]()
    phi = S.random_phase(lat.n, R, seed=100 + M)
    dts = np.array([0.5])
    Np = [O.np_rule(dE * 0.5, 64)]
    n_on, *on = _rows(lat, dE, R, M, True, phi, dts, Np)
    n_off, *off = _rows(lat, dE, R, M, False, phi, dts, Np)
    steps = (M + 1) // 2
    assert (n_on > 0) == (steps >= 3) and n_off == 0, (n_on, n_off)
    for k in range(3):
        assert nerr(on[k], off[k]) < 1e-10, k
    h = O.Hamiltonian(lat, dE)
    # the oracle takes the vectors as stored (complex64 rounded to complex128)
    ph = phi.astype(np.complex64).astype(np.complex128)
    for r in (0, R - 1):
        assert nerr(on[0][r], h.dos_moments(ph[:, r], M).real) < 1e-5
        assert nerr(on[1][r], h.vac_moments(ph[:, r], dts, Np, M)[0]) < 1e-4
        assert nerr(on[2][r], h.msd_moments(ph[:, r], dts, Np, M)[0]) < 1e-4


BANDS = {
    # one band (R = 8: 32 cells): the halo wraps round on both sides; the fewest rows
    "honeycomb32x4_R8": (32, 4, 8),
    # 32 bands x several segments of rows (R = 8)
    "honeycomb1024x300_R8": (1024, 300, 8),
    # R = 16: bands of 16 cells, more bands (512) than resident CTAs, so the band
    # rows are cut into equal ranges that cross band ends
    "honeycomb8192x4_R16": (8192, 4, 16),
    # R = 2: bands of 128 cells with 256 threads
    "honeycomb256x9_R2": (256, 9, 2),
}


@pytest.mark.parametrize("name", list(BANDS))
def test_blocked_fp32_band_geometry(name):
    """Band walk of the FP32 blocked kernel at the edges of its geometry: nine
    moments (the first order, two blocked passes) of DOS, VAC and MSD rows equal
    the single-order kernels within 1e-10 and the oracle within the FP32 bounds."""
    L1, L2, R = BANDS[name]
    lat = S.honeycomb(L1, L2, -2.7, 2.0, seed=L1 + L2, vacancy_frac=0.005)
    dE = S.energy_scale_rule(3, -2.7, 2.0)
    M = 9
    phi = S.random_phase(lat.n, R, seed=L2)
    dts = np.array([0.5])
    Np = [O.np_rule(dE * 0.5, 64)]
    n_on, *on = _rows(lat, dE, R, M, True, phi, dts, Np)
    n_off, *off = _rows(lat, dE, R, M, False, phi, dts, Np)
    assert n_on > 0 and n_off == 0, (n_on, n_off)
    for k in range(3):
        assert nerr(on[k], off[k]) < 1e-10, k
    ph = phi.astype(np.complex64).astype(np.complex128)
    ref = O.Hamiltonian(lat, dE).dos_moments(ph[:, R - 1], M).real
    assert nerr(on[0][R - 1], ref) < 1e-5


def test_blocked_fp32_not_applicable_runs_single_order():
    """Where the blocked walk does not apply the single-order kernels run, with the
    same results: a honeycomb lattice whose L1 = 36 no band width divides (R = 8
    takes bands of 32, 16 or 8 cells), R = 32 (no blocked lane layout) and R = 1."""
    lat = S.honeycomb(36, 24, -2.7, 2.0, seed=16)
    dE = S.energy_scale_rule(3, -2.7, 2.0)
    cases = [(lat, 8), (S.honeycomb(64, 8, -2.7, 2.0, seed=17), 32), (S.honeycomb(64, 8, -2.7, 2.0, seed=18), 1)]
    for lt, R in cases:
        phi = S.random_phase(lt.n, R, seed=5)
        n_on, *on = _rows(lt, dE, R, 20, True, phi, np.array([0.5]), [O.np_rule(dE * 0.5, 64)])
        assert n_on == 0, (lt.n, R)
        ph = phi.astype(np.complex64).astype(np.complex128)
        assert nerr(on[0][0], O.Hamiltonian(lt, dE).dos_moments(ph[:, 0], 20).real) < 1e-5
