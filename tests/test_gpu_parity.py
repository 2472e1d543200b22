"""Parity of the CUDA path (through the C ABI) with the serial FP64 oracle.

Same seeded inputs on both sides; sizes span several CTAs and a ragged tail.
FP64 tolerance: 1e-10 relative for moments (normalised L-infinity,
max_n |d mu_n| / max_n |mu_n|) and 1e-9 for sigma; FP32-storage tolerances are
stated per test.
"""
import math

import numpy as np
import pytest

import gqt_synth as S
import oracle as O

torch = pytest.importorskip("torch")
g = pytest.importorskip("paper_1705_01387_gb300")

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def nerr(x, y):
    x = np.asarray(x)
    y = np.asarray(y)
    return float(np.max(np.abs(x - y)) / max(float(np.max(np.abs(y))), 1e-300))


def dev(a, fp64=True):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to(torch.complex128 if fp64 else torch.complex64).cuda()


MODELS = {
    "honeycomb32x32": lambda: (S.honeycomb(32, 32, -2.7, 1.0, seed=S.BASE_SEED), S.energy_scale_rule(3, -2.7, 1.0)),
    "honeycomb37x23_phases": lambda: (S.with_random_bond_phases(S.honeycomb(37, 23, -2.7, 2.0, seed=3), 4),
                                      S.energy_scale_rule(3, -2.7, 2.0)),
    "square41x29": lambda: (S.square(41, 29, -1.0, 4.0, seed=5), S.energy_scale_rule(4, -1.0, 4.0)),
    "cubic13": lambda: (S.cubic(13, -1.0, 16.5, seed=7), S.energy_scale_rule(6, -1.0, 16.5)),
    "chain5001": lambda: (S.chain(5001, -1.0, 4.0, seed=9), S.energy_scale_rule(2, -1.0, 4.0)),
}


@pytest.fixture(scope="module")
def models():
    return {k: f() for k, f in MODELS.items()}


def test_random_phase_matches_generator():
    lat, dE = MODELS["honeycomb37x23_phases"]()
    ham = g.gqt_build_hamiltonian(lat, dE)
    for R in (1, 8):
        phi = torch.empty((lat.n, R), dtype=torch.complex128, device="cuda")
        g.gqt_random_phase(ham, 1234, R, phi, first_vector=3)
        ref = S.random_phase(lat.n, R, seed=1234, first_vector=3)
        assert np.max(np.abs(phi.cpu().numpy() - ref)) < 1e-15


@pytest.mark.parametrize("name", list(MODELS))
def test_dos_moments_fp64(models, name):
    lat, dE = models[name]
    ham = g.gqt_build_hamiltonian(lat, dE)
    phi = S.random_phase(lat.n, 1, seed=11)
    M = 300
    mu = np.empty((1, 1, M))
    g.gqt_dos_moments(ham, dev(phi), 1, M, mu)
    ref = O.Hamiltonian(lat, dE).dos_moments(phi[:, 0], M)
    assert nerr(mu.reshape(M), ref) < TOL64


def test_cheb_moments_complex_l_neq_r(models):
    lat, dE = models["honeycomb37x23_phases"]
    ham = g.gqt_build_hamiltonian(lat, dE)
    assert not ham.hop_real
    ph = S.random_phase(lat.n, 2, seed=12)
    M = 200
    mu = np.empty((1, 1, M, 2))
    g.gqt_cheb_moments(ham, dev(ph[:, :1]), dev(ph[:, 1:]), 1, M, mu)
    ref = O.Hamiltonian(lat, dE).cheb_moments(ph[:, 0], ph[:, 1], M)
    got = mu[..., 0] + 1j * mu[..., 1]
    assert nerr(got.reshape(M), ref) < TOL64


@pytest.mark.parametrize("name", ["honeycomb37x23_phases", "square41x29", "cubic13"])
@pytest.mark.parametrize("sign", [1, -1])
def test_evolve_fp64(models, name, sign):
    lat, dE = models[name]
    ham = g.gqt_build_hamiltonian(lat, dE)
    psi = S.random_phase(lat.n, 1, seed=13)
    dt = 0.7
    Np = O.np_rule(dE * dt, 64)
    d = dev(psi)
    norm = np.empty(1)
    g.gqt_evolve(ham, d, 1, dt, sign, Np, norm=norm)
    ref = O.Hamiltonian(lat, dE).evolve(psi[:, 0], dt, sign, Np)
    assert nerr(d.cpu().numpy()[:, 0], ref) < TOL64
    assert abs(norm[0] - 1.0) < 1e-12


@pytest.mark.parametrize("name", ["honeycomb37x23_phases", "square41x29"])
def test_commutator_evolve_fp64(models, name):
    lat, dE = models[name]
    ham = g.gqt_build_hamiltonian(lat, dE)
    psi = S.random_phase(lat.n, 1, seed=14)
    dt = 0.9
    Np = O.np_rule(dE * dt, 64)
    out = torch.empty((lat.n, 1), dtype=torch.complex128, device="cuda")
    g.gqt_commutator_evolve(ham, dev(psi), out, 1, dt, Np)
    ref = O.Hamiltonian(lat, dE).commutator_evolve(psi[:, 0], dt, Np)
    assert nerr(out.cpu().numpy()[:, 0], ref) < TOL64


def test_velocity_fp64(models):
    lat, dE = models["honeycomb37x23_phases"]
    ham = g.gqt_build_hamiltonian(lat, dE)
    x = S.random_phase(lat.n, 1, seed=15)
    y = torch.empty((lat.n, 1), dtype=torch.complex128, device="cuda")
    g.gqt_apply_velocity(ham, dev(x), y, 1)
    ref = O.Hamiltonian(lat, dE).apply_v(x[:, 0])
    assert nerr(y.cpu().numpy()[:, 0], ref) < 1e-13


def _c1():
    w = S.config(0)
    lat = S.build_lattice(w.lattice_args, w.seed)
    return w, lat


def test_vac_msd_config1_fp64():
    """Honeycomb 32x32 (N = 2048), M = 512, 10 steps of dt = 1 hbar/|t|: VAC and MSD moments."""
    w, lat = _c1()
    dE = w.energy_scale
    ham = g.gqt_build_hamiltonian(lat, dE)
    phi = S.random_phase(lat.n, 1, seed=w.seed)
    dts = np.full(w.n_steps, w.dt)
    Np = [O.np_rule(dE * d, 64) for d in dts]
    h = O.Hamiltonian(lat, dE)
    a, b = torch.empty((lat.n, 1), dtype=torch.complex128, device="cuda"), torch.empty((lat.n, 1), dtype=torch.complex128, device="cuda")
    d = dev(phi)
    g.gqt_vac_init(ham, d, a, b, 1)
    vac = np.empty((w.n_steps, 1, 1, w.M))
    g.gqt_vac_moments(ham, a, b, 1, dts, w.M, vac, Np=Np)
    ref = h.vac_moments(phi[:, 0], dts, Np, w.M)
    assert nerr(vac.reshape(w.n_steps, w.M), ref) < TOL64
    p, px = torch.empty_like(a), torch.empty_like(a)
    g.gqt_msd_init(ham, d, p, px, 1)
    msd = np.empty((w.n_steps, 1, 1, w.M))
    g.gqt_msd_moments(ham, p, px, 1, dts, w.M, msd, Np=Np)
    refm = h.msd_moments(phi[:, 0], dts, Np, w.M)
    assert nerr(msd.reshape(w.n_steps, w.M), refm) < TOL64
    # reconstruction and running conductivity on 1001 energies
    E = w.energies
    nO = lat.n / lat.volume
    for rows, refrows, sig_fn, osig in ((vac, ref, g.gqt_sigma_vac, O.sigma_vac), (msd, refm, g.gqt_sigma_msd, O.sigma_msd)):
        mu_d = torch.from_numpy(rows.reshape(w.n_steps, w.M)).cuda()
        out = torch.empty((w.n_steps, E.size), dtype=torch.float64, device="cuda")
        g.gqt_kpm_reconstruct(mu_d, torch.from_numpy(E).cuda(), dE, nO, out)
        r_ref = O.kpm_reconstruct(refrows, E, dE, nO)
        assert nerr(out.cpu().numpy(), r_ref) < TOL64
        sig = torch.empty_like(out)
        sig_fn(out, dts, sig)
        s_ref = osig(r_ref, dts)
        assert nerr(sig.cpu().numpy(), s_ref) < 1e-9


def test_kpm_reconstruct_same_moments():
    """Reconstruction alone, on identical moments: GPU vs oracle (Eqs. 25-27, 31)."""
    rng = np.random.default_rng(0)
    rows, M = 7, 777
    mu = rng.standard_normal((rows, M)) / (1 + np.arange(M))
    E = np.linspace(-9.5, 9.5, 1001)
    dE = 9.03
    out = torch.empty((rows, E.size), dtype=torch.float64, device="cuda")
    g.gqt_kpm_reconstruct(torch.from_numpy(mu).cuda(), torch.from_numpy(E).cuda(), dE, 0.77, out)
    ref = O.kpm_reconstruct(mu, E, dE, 0.77)
    got = out.cpu().numpy()
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    m = ~np.isnan(ref)
    assert nerr(got[m], ref[m]) < 1e-12


def test_fp32_storage_error_is_small(models):
    """FP32 H~ and vectors with FP64 accumulation: DOS moments within 1e-5 (normalised) of the FP64 oracle."""
    lat, dE = models["honeycomb32x32"]
    ham = g.gqt_build_hamiltonian(lat, dE, g.GQT_FP32_ACC64)
    phi = S.random_phase(lat.n, 1, seed=11)
    M = 300
    mu = np.empty((1, 1, M))
    g.gqt_dos_moments(ham, dev(phi, False), 1, M, mu)
    ref = O.Hamiltonian(lat, dE).dos_moments(phi[:, 0], M)
    assert nerr(mu.reshape(M), ref) < 1e-5


@pytest.mark.parametrize("R", [2, 8, 32])
def test_batched_vectors_match_single(models, R):
    lat, dE = models["square41x29"]
    ham = g.gqt_build_hamiltonian(lat, dE)
    ph = S.random_phase(lat.n, R, seed=21)
    M = 128
    mu = np.empty((1, R, M))
    g.gqt_dos_moments(ham, dev(ph), R, M, mu)
    h = O.Hamiltonian(lat, dE)
    for r in range(0, R, max(1, R // 4)):
        assert nerr(mu[0, r], h.dos_moments(ph[:, r], M)) < TOL64


def test_ragged_segments_match_separate_builds():
    parts = [S.cubic(L, -1.0, 16.5, seed=30 + q) for q, L in enumerate((5, 7, 4, 6))]
    blk = S.block_diagonal(parts)
    dE = S.energy_scale_rule(6, -1.0, 16.5)
    ham = g.gqt_build_hamiltonian(blk, dE)
    assert ham.nseg == 4
    phi = torch.empty((blk.n, 1), dtype=torch.complex128, device="cuda")
    g.gqt_random_phase(ham, 77, 1, phi)
    M = 100
    mu = np.empty((4, 1, M))
    g.gqt_dos_moments(ham, phi, 1, M, mu)
    ph = phi.cpu().numpy()[:, 0]
    for q, p in enumerate(parts):
        o = blk.seg_offsets[q]
        seg_phi = ph[o:o + p.n]
        assert abs(np.linalg.norm(seg_phi) - 1.0) < 1e-14
        ref = O.Hamiltonian(p, dE).dos_moments(seg_phi, M)
        assert nerr(mu[q, 0], ref) < TOL64


def test_energy_scale_too_small_is_erange():
    lat = S.honeycomb(16, 16, -2.7, 1.0, seed=1)
    ham = g.gqt_build_hamiltonian(lat, 4.0)  # spectrum reaches 8.6 > 4
    phi = dev(S.random_phase(lat.n, 1, seed=1))
    mu = np.empty((1, 1, 200))
    with pytest.raises(g.GqtError) as e:
        g.gqt_dos_moments(ham, phi, 1, 200, mu)
    assert e.value.status == g.GQT_ERANGE


def test_non_hermitian_input_is_einval():
    lat = S.square(5, 5, -1.0, 0.0)
    lat.hop[3, 0] = -1.5
    with pytest.raises(g.GqtError) as e:
        g.gqt_build_hamiltonian(lat, 5.0)
    assert e.value.status == g.GQT_EINVAL
    lat = S.square(5, 5, -1.0, 0.0)
    lat.nb_idx[2, 1] = 999
    with pytest.raises(g.GqtError) as e:
        g.gqt_build_hamiltonian(lat, 5.0)
    assert e.value.status == g.GQT_EINVAL


@pytest.mark.parametrize("M", [1, 2, 3, 4, 5, 301])
def test_dos_moment_counts_edge_cases(models, M):
    """l = r moments use two moments per recursion step; odd and tiny M must still
    give exactly M moments equal to the plain recursion's."""
    lat, dE = models["square41x29"]
    ham = g.gqt_build_hamiltonian(lat, dE)
    phi = S.random_phase(lat.n, 1, seed=31)
    mu = np.full((1, 1, M), np.nan)
    g.gqt_dos_moments(ham, dev(phi), 1, M, mu)
    ref = O.Hamiltonian(lat, dE).dos_moments(phi[:, 0], M)
    assert nerr(mu.reshape(M), ref) < TOL64


def test_fp32_vac_msd_error_table(models):
    """FP32 storage with FP64 accumulation on VAC and MSD rows: normalised error vs the
    FP64 oracle below 1e-4 (stated bound for these lengths)."""
    lat, dE = models["honeycomb32x32"]
    ham = g.gqt_build_hamiltonian(lat, dE, g.GQT_FP32_ACC64)
    phi = S.random_phase(lat.n, 1, seed=41)
    dts = np.full(3, 1 / 2.7)
    Np = [O.np_rule(dE * d, 64) for d in dts]
    M = 256
    d = dev(phi, False)
    a, b = torch.empty_like(d), torch.empty_like(d)
    g.gqt_vac_init(ham, d, a, b, 1)
    vac = np.empty((3, 1, 1, M))
    g.gqt_vac_moments(ham, a, b, 1, dts, M, vac, Np=Np)
    p, px = torch.empty_like(d), torch.empty_like(d)
    g.gqt_msd_init(ham, d, p, px, 1)
    msd = np.empty((3, 1, 1, M))
    g.gqt_msd_moments(ham, p, px, 1, dts, M, msd, Np=Np)
    h = O.Hamiltonian(lat, dE)
    assert nerr(vac.reshape(3, M), h.vac_moments(phi[:, 0], dts, Np, M)) < 1e-4
    assert nerr(msd.reshape(3, M), h.msd_moments(phi[:, 0], dts, Np, M)) < 1e-4
