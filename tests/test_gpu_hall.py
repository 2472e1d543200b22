"""Hall conductivity (Kubo-Bastin moments and sigma_xy) through the C ABI against
the serial FP64 oracle, whose Kubo-Bastin functions are pinned in
test_oracle_pins.py (eigenbasis closed form, mirror symmetry, closed-form
integrals, the Haldane Chern plateau against the eigenstate Kubo sum)."""
import math

import numpy as np
import pytest

import gqt_synth as S
import oracle as O

torch = pytest.importorskip("torch")
g = pytest.importorskip("paper_1705_01387_gb300")

pytestmark = pytest.mark.gpu


def nerr(x, y):
    return float(np.max(np.abs(np.asarray(x) - np.asarray(y))) / max(float(np.max(np.abs(y))), 1e-300))


def _model(name):
    if name == "haldane":
        lat = S.haldane(5, 4, -1.0, 0.2, math.pi / 3, 0.1, 0.5, seed=3)
        return lat, 1.05 * (3 + 6 * 0.2 + 0.1 + 0.25)
    if name == "square_phases":
        return S.with_random_bond_phases(S.square(7, 6, -1.0, 1.0, seed=4), 8), 5.0
    if name == "honeycomb_phases":
        return S.with_random_bond_phases(S.honeycomb(6, 5, -2.7, 1.0, seed=5), 9), S.energy_scale_rule(3, -2.7, 1.0)
    if name == "honeycomb_real":
        return S.honeycomb(7, 5, -2.7, 1.0, seed=6), S.energy_scale_rule(3, -2.7, 1.0)
    raise ValueError(name)


def _gpu_lambda(lat, dE, ph, M, a, b):
    ham = g.gqt_build_hamiltonian(lat, dE)
    lam = torch.empty((M, M), dtype=torch.complex128, device="cuda")
    g.gqt_kb_moments(ham, torch.from_numpy(ph).cuda(), ph.shape[1], M, a, b, lam)
    return lam


@pytest.mark.parametrize("name", ["haldane", "square_phases", "honeycomb_phases", "honeycomb_real"])
@pytest.mark.parametrize("M,R", [(1, 1), (2, 2), (17, 3), (70, 1)])
@pytest.mark.parametrize("pair", ["xy", "yx", "xx"])
def test_kb_moments_match_oracle(name, M, R, pair):
    lat, dE = _model(name)
    ph = S.random_phase(lat.n, R, seed=31)
    d = {"x": (0, lat.dx), "y": (1, lat.dy)}
    (a, da), (b, db) = d[pair[0]], d[pair[1]]
    got = _gpu_lambda(lat, dE, ph, M, a, b).cpu().numpy()
    ref = O.Hamiltonian(lat, dE).kb_moments(da, db, ph, M)
    assert nerr(got, ref) < 1e-10


def test_kb_moments_split_contraction():
    """N R large enough that the contraction is split across CTAs (deterministic
    sum of the splits): same moments as the oracle, and bit-identical on repeat."""
    lat = S.haldane(23, 19, -1.0, 0.15, math.pi / 2, 0.0, 1.0, seed=7)
    dE = 1.05 * (3 + 6 * 0.15 + 0.5)
    ph = S.random_phase(lat.n, 2, seed=32)
    M = 64
    first = _gpu_lambda(lat, dE, ph, M, 0, 1).cpu().numpy()
    again = _gpu_lambda(lat, dE, ph, M, 0, 1).cpu().numpy()
    ref = O.Hamiltonian(lat, dE).kb_moments(lat.dx, lat.dy, ph, M)
    assert nerr(first, ref) < 1e-10
    assert np.array_equal(first, again)


@pytest.mark.parametrize("kernel", [0, 1])
def test_kubo_bastin_matches_oracle(kernel):
    rng = np.random.default_rng(5)
    M, dE, area = 37, 3.7, 12.5
    lam = (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))) / (1 + np.arange(M))[None, :]
    E = np.linspace(-0.95 * dE, 0.9 * dE, 1201)
    sig = torch.empty(E.size, dtype=torch.float64, device="cuda")
    g.gqt_kubo_bastin(torch.from_numpy(lam).cuda(), torch.from_numpy(E).cuda(), dE, area, sig, kernel=kernel)
    ref = O.kubo_bastin(lam, E, dE, area, kernel)
    assert nerr(sig.cpu().numpy(), ref) < 1e-10


def test_haldane_chern_plateau_on_gpu():
    """Haldane model, 8 x 8 cells, exact trace (the site basis as the vectors),
    M = 256: sigma_xy in the gap is the Chern number 1 (the oracle's pin against
    the eigenstate Kubo sum), and equals the oracle's reconstruction."""
    lat = S.haldane(8, 8, -1.0, 0.15, math.pi / 2, 0.0, 0.0)
    dE = 1.05 * (3.0 + 6 * 0.15)
    basis = np.eye(lat.n, dtype=np.complex128)
    M = 256
    lam = _gpu_lambda(lat, dE, basis, M, 0, 1)
    E = np.linspace(-0.97 * dE, 0.0, 3001)
    sig = torch.empty(E.size, dtype=torch.float64, device="cuda")
    g.gqt_kubo_bastin(lam, torch.from_numpy(E).cuda(), dE, lat.volume, sig)
    s = sig.cpu().numpy()
    assert abs(s[-1] - 1.0) < 1e-2
    ref = O.kubo_bastin(O.Hamiltonian(lat, dE).kb_moments(lat.dx, lat.dy, basis, M), E, dE, lat.volume)
    assert nerr(s, ref) < 1e-9


def test_kb_moments_full_size_lattice():
    """The Hall workload's lattice (Haldane 512 x 512 cells, N = 524,288, W = 1)
    at M = 64: every moment equals the oracle's (the same kernels and split
    contraction as at M = 1024, with one 64 x 64 output tile)."""
    lat = S.haldane(512, 512, -1.0, 0.15, math.pi / 2, 0.0, 1.0, seed=1705013875)
    dE = 1.05 * (3 + 6 * 0.15 + 0.5)
    ph = S.random_phase(lat.n, 1, seed=1705013875)
    M = 64
    got = _gpu_lambda(lat, dE, ph, M, 0, 1).cpu().numpy()
    ref = O.Hamiltonian(lat, dE).kb_moments(lat.dx, lat.dy, ph, M)
    assert nerr(got, ref) < 1e-10


def test_hall_argument_errors():
    lat, dE = _model("haldane")
    ph = torch.from_numpy(S.random_phase(lat.n, 1, seed=1)).cuda()
    lam = torch.empty((8, 8), dtype=torch.complex128, device="cuda")
    h32 = g.gqt_build_hamiltonian(lat, dE, g.GQT_FP32_ACC64)
    with pytest.raises(g.GqtError) as e:
        g.gqt_kb_moments(h32, ph.to(torch.complex64), 1, 8, 0, 1, lam)
    assert e.value.status == g.GQT_EINVAL
    no_dy = S.Lattice("no_dy", lat.n, lat.max_nb, lat.nb_count, lat.nb_idx, lat.hop, lat.onsite, lat.dx,
                      lat.length_x, lat.volume)
    with pytest.raises(g.GqtError) as e:
        g.gqt_kb_moments(g.gqt_build_hamiltonian(no_dy, dE), ph, 1, 8, 0, 1, lam)
    assert e.value.status == g.GQT_EINVAL
    g.gqt_kb_moments(g.gqt_build_hamiltonian(no_dy, dE), ph, 1, 8, 0, 0, lam)  # x only: fine
    blk = S.block_diagonal([lat, lat])
    with pytest.raises(g.GqtError) as e:
        g.gqt_kb_moments(g.gqt_build_hamiltonian(blk, dE), torch.from_numpy(S.random_phase(blk.n, 1)).cuda(), 1, 8,
                         0, 1, lam)
    assert e.value.status == g.GQT_EINVAL
    with pytest.raises(g.GqtError) as e:
        g.gqt_set_kb_contraction(g.gqt_build_hamiltonian(lat, dE), 2)
    assert e.value.status == g.GQT_EINVAL
    sig = torch.empty(3, dtype=torch.float64, device="cuda")
    for bad in ([0.1, 0.0, 0.2], [-dE, 0.0, 0.1]):
        with pytest.raises(g.GqtError) as e:
            g.gqt_kubo_bastin(lam, torch.tensor(bad, dtype=torch.float64, device="cuda"), dE, lat.volume, sig)
        assert e.value.status == g.GQT_EINVAL


def _gpu_lambda_tc(lat, dE, ph, M, a, b):
    ham = g.gqt_build_hamiltonian(lat, dE)
    g.gqt_set_kb_contraction(ham, 1)
    lam = torch.empty((M, M), dtype=torch.complex128, device="cuda")
    g.gqt_kb_moments(ham, torch.from_numpy(ph).cuda(), ph.shape[1], M, a, b, lam)
    return lam


@pytest.mark.parametrize("name", ["haldane", "square_phases", "honeycomb_real"])
@pytest.mark.parametrize("M,R", [(1, 1), (17, 2), (70, 1), (130, 3), (300, 1)])
@pytest.mark.parametrize("pair", ["xy", "yx", "xx"])
def test_kb_moments_tensor_core_contraction(name, M, R, pair):
    """Split-TF32 contraction on the tcgen05 tensor cores (three products per pair,
    FP32 accumulation per split, FP64 sum of splits): within 1e-5 of the oracle
    (normalised by the largest moment), including partial 128 x 256 tiles and
    contraction lengths N R that are not a multiple of the 8-site chunk."""
    lat, dE = _model(name)
    ph = S.random_phase(lat.n, R, seed=33)
    d = {"x": (0, lat.dx), "y": (1, lat.dy)}
    (a, da), (b, db) = d[pair[0]], d[pair[1]]
    got = _gpu_lambda_tc(lat, dE, ph, M, a, b).cpu().numpy()
    ref = O.Hamiltonian(lat, dE).kb_moments(da, db, ph, M)
    err = nerr(got, ref)
    assert err < 1e-5, err


def test_haldane_chern_plateau_tensor_core():
    """The exact-trace Haldane plateau (M = 256, 8 x 8 cells) through the tensor-core
    contraction: sigma_xy within 1e-4 of the FP64 contraction's at every energy."""
    lat = S.haldane(8, 8, -1.0, 0.15, math.pi / 2, 0.0, 0.0)
    dE = 1.05 * (3.0 + 6 * 0.15)
    basis = np.eye(lat.n, dtype=np.complex128)
    M = 256
    E = torch.from_numpy(np.linspace(-0.97 * dE, 0.0, 3001)).cuda()
    out = {}
    for name, lam in (("tc", _gpu_lambda_tc(lat, dE, basis, M, 0, 1)),
                      ("fp64", _gpu_lambda(lat, dE, basis, M, 0, 1))):
        sig = torch.empty(E.numel(), dtype=torch.float64, device="cuda")
        g.gqt_kubo_bastin(lam, E, dE, lat.volume, sig)
        out[name] = sig.cpu().numpy()
    assert abs(out["tc"][-1] - 1.0) < 1e-2
    diff = float(np.max(np.abs(out["tc"] - out["fp64"])))
    assert diff < 1e-4, diff


def test_tensor_core_wait_timeout_then_recovers():
    """Failure detection of the bounded device waits: with a wait limit of 0 polls every
    mbarrier wait of the tensor-core contraction's pipeline gives up at once (a wait
    that runs out, with no copy withheld and nothing faulted); the issuing thread then
    drains the copies it issued with the fixed drain limit, frees tensor memory, and
    the call returns GQT_ETIMEOUT.  With the default limit restored, the next call on
    the same handle matches the oracle to the contraction's 1e-5 bound."""
    lat = S.haldane(23, 19, -1.0, 0.15, math.pi / 2, 0.0, 1.0, seed=7)
    dE = 1.05 * (3 + 6 * 0.15 + 0.5)
    ph = S.random_phase(lat.n, 1, seed=35)
    M = 256
    ham = g.gqt_build_hamiltonian(lat, dE)
    g.gqt_set_kb_contraction(ham, 1)
    r = torch.from_numpy(ph).cuda()
    lam = torch.empty((M, M), dtype=torch.complex128, device="cuda")
    g.gqt_set_wait_limit(ham, 0)
    with pytest.raises(g.GqtError) as ei:
        g.gqt_kb_moments(ham, r, 1, M, 0, 1, lam)
    assert ei.value.status == g.GQT_ETIMEOUT
    assert "drain" not in str(ei.value)  # the drain collected every copy in flight
    with pytest.raises(g.GqtError):
        g.gqt_set_wait_limit(ham, -1)
    g.gqt_set_wait_limit(ham, 1 << 24)
    g.gqt_kb_moments(ham, r, 1, M, 0, 1, lam)
    ref = O.Hamiltonian(lat, dE).kb_moments(lat.dx, lat.dy, ph, M)
    err = nerr(lam.cpu().numpy(), ref)
    assert err < 1e-5, err


def test_kb_moments_tensor_core_full_size_lattice():
    """Tensor-core contraction on the 512 x 512 Haldane lattice (N = 524,288) at
    M = 64.  Each split accumulates at most 8192 sites' products in FP32, whose
    rounding grows like sqrt(8192) * 2^-24 = 5e-6 of the split's magnitude; the
    bound is 5e-5 of the largest moment (measured: 1.3e-5)."""
    lat = S.haldane(512, 512, -1.0, 0.15, math.pi / 2, 0.0, 1.0, seed=1705013875)
    dE = 1.05 * (3 + 6 * 0.15 + 0.5)
    ph = S.random_phase(lat.n, 1, seed=1705013875)
    M = 64
    got = _gpu_lambda_tc(lat, dE, ph, M, 0, 1).cpu().numpy()
    ref = O.Hamiltonian(lat, dE).kb_moments(lat.dx, lat.dy, ph, M)
    err = nerr(got, ref)
    assert err < 5e-5, err


@pytest.mark.parametrize("kT", [0.0, 0.05, 0.3])
def test_kubo_bastin_fermi_matches_oracle(kT):
    rng = np.random.default_rng(6)
    M, dE, area = 37, 3.7, 12.5
    lam = (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))) / (1 + np.arange(M))[None, :]
    E = np.linspace(-0.95 * dE, 0.9 * dE, 1201)
    mu = np.array([-2.0, -0.5, 0.0, E[600], 1.7])
    sig = torch.empty(mu.size, dtype=torch.float64, device="cuda")
    g.gqt_kubo_bastin_fermi(torch.from_numpy(lam).cuda(), torch.from_numpy(E).cuda(), dE, area,
                            torch.from_numpy(mu).cuda(), kT, sig)
    ref = O.kubo_bastin_fermi(lam, E, dE, area, mu, kT)
    assert nerr(sig.cpu().numpy(), ref) < 1e-10


def test_haldane_plateau_finite_temperature():
    """At kT = 0.02 (gap about 1.7 wide) sigma_xy at the gap centre stays the Chern
    number; well inside the band, temperature changes it."""
    lat = S.haldane(8, 8, -1.0, 0.15, math.pi / 2, 0.0, 0.0)
    dE = 1.05 * (3.0 + 6 * 0.15)
    lam = _gpu_lambda(lat, dE, np.eye(lat.n, dtype=np.complex128), 256, 0, 1)
    E = torch.from_numpy(np.linspace(-0.97 * dE, 0.97 * dE, 4001)).cuda()
    mu = torch.tensor([0.0, -1.9], dtype=torch.float64, device="cuda")
    out = {}
    for kT in (0.0, 0.02, 0.3):
        sig = torch.empty(2, dtype=torch.float64, device="cuda")
        g.gqt_kubo_bastin_fermi(lam, E, dE, lat.volume, mu, kT, sig)
        out[kT] = sig.cpu().numpy()
    assert abs(out[0.02][0] - 1.0) < 1e-2 and abs(out[0.0][0] - 1.0) < 1e-2
    assert abs(out[0.3][1] - out[0.0][1]) > 1e-3


def _gpu_lambda_fp32(lat, dE, ph, M, a, b):
    ham = g.gqt_build_hamiltonian(lat, dE, g.GQT_FP32_ACC64)
    g.gqt_set_kb_contraction(ham, 1)
    lam = torch.empty((M, M), dtype=torch.complex128, device="cuda")
    g.gqt_kb_moments(ham, torch.from_numpy(ph).to(torch.complex64).cuda(), ph.shape[1], M, a, b, lam)
    return lam


@pytest.mark.parametrize("name", ["haldane", "square_phases", "honeycomb_real"])
@pytest.mark.parametrize("M,R", [(17, 1), (70, 2), (130, 1)])
@pytest.mark.parametrize("pair", ["xy", "xx"])
def test_kb_moments_fp32_chains(name, M, R, pair):
    """FP32 storage (H~ and the chains in FP32) with the tensor-core contraction:
    within 1e-5 of the oracle run on the same (FP32-rounded) vectors (measured up
    to 2.4e-6: the chains' FP32 rounding is below the contraction's)."""
    lat, dE = _model(name)
    ph = S.random_phase(lat.n, R, seed=34).astype(np.complex64).astype(np.complex128)
    d = {"x": (0, lat.dx), "y": (1, lat.dy)}
    (a, da), (b, db) = d[pair[0]], d[pair[1]]
    got = _gpu_lambda_fp32(lat, dE, ph, M, a, b).cpu().numpy()
    ref = O.Hamiltonian(lat, dE).kb_moments(da, db, ph, M)
    err = nerr(got, ref)
    assert err < 1e-5, err


def test_haldane_chern_plateau_fp32_chains():
    lat = S.haldane(8, 8, -1.0, 0.15, math.pi / 2, 0.0, 0.0)
    dE = 1.05 * (3.0 + 6 * 0.15)
    basis = np.eye(lat.n, dtype=np.complex128)
    M = 256
    E = torch.from_numpy(np.linspace(-0.97 * dE, 0.0, 3001)).cuda()
    out = {}
    for name, lam in (("fp32", _gpu_lambda_fp32(lat, dE, basis, M, 0, 1)),
                      ("fp64", _gpu_lambda(lat, dE, basis, M, 0, 1))):
        sig = torch.empty(E.numel(), dtype=torch.float64, device="cuda")
        g.gqt_kubo_bastin(lam, E, dE, lat.volume, sig)
        out[name] = sig.cpu().numpy()
    assert abs(out["fp32"][-1] - 1.0) < 1e-2
    diff = float(np.max(np.abs(out["fp32"] - out["fp64"])))
    assert diff < 1e-4, diff  # measured 1.4e-5
