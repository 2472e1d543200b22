"""The paper's two examples (Sec. 5) at reduced size, and long Chebyshev-Bessel
expansions, through the C ABI against the serial FP64 oracle.

Example 2 (the localized 1D chain) takes 30 non-uniform steps up to dt = 100 at
dE = 4.1, i.e. up to N_p = 487 Bessel orders (Eq. 17); these tests take the
library's evolution, commutator evolution and MSD rows through such expansions.
The oracle's long expansions are pinned on the CPU (test_oracle_pins.py: Bessel
values against scipy, the uncapped N_p rule, exp(-i x H~) and the Daleckii-Krein
[X, U] at x = 41 and 410).  Tolerances: 1e-10 normalised on vectors and moments,
1e-9 on sigma, as for the other FP64 parity tests.
"""
import numpy as np
import pytest

import gqt_synth as S
import oracle as O

torch = pytest.importorskip("torch")
g = pytest.importorskip("paper_1705_01387_gb300")
from paper_1705_01387_gb300 import analysis as A  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def nerr(x, y):
    x = np.asarray(x)
    y = np.asarray(y)
    return float(np.max(np.abs(x - y)) / max(float(np.max(np.abs(y))), 1e-300))


def _chain():
    """Example 2's model at reduced length: chain, t = -1, W = 4, dE = 4.1."""
    return S.chain(4001, -1.0, 4.0, seed=S.BASE_SEED + 11), 4.1


EX2_DTS = np.concatenate([np.arange(1, 11) * 0.1, np.arange(1, 11) * 1.0, np.arange(1, 11) * 10.0])


@pytest.mark.parametrize("x", [41.0, 410.0])
def test_long_evolution_matches_oracle(x):
    """U(+-dt) and [X, U(dt)] with N_p = 78 and 487 orders (dt = 10 and 100 at dE = 4.1)
    on two vectors: within 1e-10 of the oracle, |U phi| = 1 to 1e-12."""
    lat, dE = _chain()
    Np = g.gqt_np_rule(x, 4096)
    assert Np == O.np_rule(x, 4096) and Np >= 78
    dt = x / dE
    ham = g.gqt_build_hamiltonian(lat, dE)
    h = O.Hamiltonian(lat, dE)
    R = 2
    phi = S.random_phase(lat.n, R, seed=41)
    for sign in (+1, -1):
        psi = torch.from_numpy(phi.copy()).cuda()
        nrm = np.empty(R)
        g.gqt_evolve(ham, psi, R, dt, sign, Np, norm=nrm)
        got = psi.cpu().numpy()
        for r in range(R):
            ref = h.evolve(phi[:, r], dt, sign, Np)
            assert nerr(got[:, r], ref) < TOL64, (x, sign, r)
        assert np.max(np.abs(nrm - 1.0)) < 1e-12
    psi = torch.from_numpy(phi.copy()).cuda()
    out = torch.empty_like(psi)
    g.gqt_commutator_evolve(ham, psi, out, R, dt, Np)
    got = out.cpu().numpy()
    for r in range(R):
        ref = h.commutator_evolve(phi[:, r], dt, Np)
        assert nerr(got[:, r], ref) < TOL64, (x, r)


def test_example2_localized_chain_reduced():
    """Example 2 (Sec. 5, localized): chain of 4001 sites, W = 4, dE = 4.1, two random
    vectors, M = 500, MSD over the paper's 30 non-uniform steps 0.1..1, 1..10, 10..100
    (N_p from 10 up to 487), DOS; reconstruction on -4..4 step 0.02, sigma_MSD, and the
    propagation length L(E, t) of Eq. 11 from GPU and oracle outputs."""
    lat, dE = _chain()
    ham = g.gqt_build_hamiltonian(lat, dE)
    h = O.Hamiltonian(lat, dE)
    R, M = 2, 500
    dts = EX2_DTS
    Np = [g.gqt_np_rule(dE * d, 4096) for d in dts]
    assert Np == [O.np_rule(dE * d, 4096) for d in dts] and max(Np) == 487
    phi = S.random_phase(lat.n, R, seed=S.BASE_SEED + 11)
    d = torch.from_numpy(phi).cuda()
    dos = np.empty((1, R, M))
    g.gqt_dos_moments(ham, d, R, M, dos)
    p, px = torch.empty_like(d), torch.empty_like(d)
    g.gqt_msd_init(ham, d, p, px, R)
    msd = np.empty((dts.size, 1, R, M))
    g.gqt_msd_moments(ham, p, px, R, dts, M, msd, Np=Np)
    ref_dos = np.array([h.dos_moments(phi[:, r], M).real for r in range(R)])
    ref_msd = np.array([h.msd_moments(phi[:, r], dts, Np, M) for r in range(R)])  # [R, Nt, M]
    assert nerr(dos[0], ref_dos) < TOL64
    for r in range(R):
        assert nerr(msd[:, 0, r], ref_msd[r]) < TOL64, r
    E = np.arange(-200, 201) * 0.02
    nO = lat.n / lat.volume
    Ed = torch.from_numpy(E).cuda()

    def recon(rows):
        out = torch.empty((rows.shape[0], E.size), dtype=torch.float64, device="cuda")
        g.gqt_kpm_reconstruct(torch.from_numpy(np.ascontiguousarray(rows)).cuda(), Ed, dE, nO, out)
        return out

    rd = recon(dos[0].mean(0, keepdims=True))
    rm = recon(msd[:, 0].mean(1))
    sm = torch.empty_like(rm)
    g.gqt_sigma_msd(rm, dts, sm)
    rd_ref = O.kpm_reconstruct(ref_dos.mean(0), E, dE, nO)
    rm_ref = O.kpm_reconstruct(ref_msd.mean(0), E, dE, nO)
    sm_ref = O.sigma_msd(rm_ref, dts)
    assert nerr(rd.cpu().numpy(), rd_ref) < TOL64
    assert nerr(rm.cpu().numpy(), rm_ref) < TOL64
    assert nerr(sm.cpu().numpy(), sm_ref) < 1e-9
    # L = 2 sqrt(rho dX^2 / rho) divides by the DOS, and each energy sums 500
    # moments: normalised noise of 1e-10 on the oracle's moments (the moment
    # tolerance) moves L by up to 2.7e-6 of its largest value where the DOS is above
    # 1% of its maximum (the band tails are left out), so the bound is 1e-5.
    Lg = A.propagation_length(rd.cpu().numpy()[0], rm.cpu().numpy())
    Lo = A.propagation_length(rd_ref[0], rm_ref)
    inner = rd_ref[0] > 1e-2 * rd_ref[0].max()
    m = np.isfinite(Lo) & (Lo > 0) & inner[None, :]
    assert np.array_equal(m, np.isfinite(Lg) & (Lg > 0) & inner[None, :])
    assert nerr(Lg[m], Lo[m]) < 1e-5


def test_example1_diffusive_square_reduced():
    """Example 1 (Sec. 5, diffusive): square lattice 64 x 64, W = 4, dE = 6.1, one
    random vector, M = 1000, DOS, VAC and MSD over 20 steps of 0.2; reconstruction on
    -6..6 step 0.02, sigma_VAC and sigma_MSD, and the semiclassical analysis of
    Sec. 2.3 (sigma_sc, tau, mean free path) from GPU and oracle outputs."""
    lat = S.square(64, 64, -1.0, 4.0, seed=S.BASE_SEED + 10)
    dE = 6.1
    ham = g.gqt_build_hamiltonian(lat, dE)
    h = O.Hamiltonian(lat, dE)
    M, Nt = 1000, 20
    dts = np.full(Nt, 0.2)
    Np = [g.gqt_np_rule(dE * dd, 4096) for dd in dts]
    assert Np == [O.np_rule(dE * dd, 4096) for dd in dts]
    phi = S.random_phase(lat.n, 1, seed=S.BASE_SEED + 10)
    d = torch.from_numpy(phi).cuda()
    dos = np.empty((1, 1, M))
    g.gqt_dos_moments(ham, d, 1, M, dos)
    a, b = torch.empty_like(d), torch.empty_like(d)
    g.gqt_vac_init(ham, d, a, b, 1)
    vac = np.empty((Nt, 1, 1, M))
    g.gqt_vac_moments(ham, a, b, 1, dts, M, vac, Np=Np)
    p, px = torch.empty_like(d), torch.empty_like(d)
    g.gqt_msd_init(ham, d, p, px, 1)
    msd = np.empty((Nt, 1, 1, M))
    g.gqt_msd_moments(ham, p, px, 1, dts, M, msd, Np=Np)
    ref_dos = h.dos_moments(phi[:, 0], M).real
    ref_vac = h.vac_moments(phi[:, 0], dts, Np, M)
    ref_msd = h.msd_moments(phi[:, 0], dts, Np, M)
    assert nerr(dos.reshape(M), ref_dos) < TOL64
    assert nerr(vac.reshape(Nt, M), ref_vac) < TOL64
    assert nerr(msd.reshape(Nt, M), ref_msd) < TOL64
    E = np.arange(-300, 301) * 0.02
    nO = lat.n / lat.volume
    Ed = torch.from_numpy(E).cuda()

    def recon(rows):
        out = torch.empty((rows.shape[0], E.size), dtype=torch.float64, device="cuda")
        g.gqt_kpm_reconstruct(torch.from_numpy(np.ascontiguousarray(rows)).cuda(), Ed, dE, nO, out)
        return out

    rd, rv, rm = recon(dos[0]), recon(vac.reshape(Nt, M)), recon(msd.reshape(Nt, M))
    sv, sm = torch.empty_like(rv), torch.empty_like(rm)
    g.gqt_sigma_vac(rv, dts, sv)
    g.gqt_sigma_msd(rm, dts, sm)
    rd_ref = O.kpm_reconstruct(ref_dos, E, dE, nO)
    rv_ref = O.kpm_reconstruct(ref_vac, E, dE, nO)
    rm_ref = O.kpm_reconstruct(ref_msd, E, dE, nO)
    sv_ref, sm_ref = O.sigma_vac(rv_ref, dts), O.sigma_msd(rm_ref, dts)
    for got, ref in ((rd, rd_ref), (rv, rv_ref), (rm, rm_ref)):
        assert nerr(got.cpu().numpy(), ref) < TOL64
    assert nerr(sv.cpu().numpy(), sv_ref) < 1e-9
    assert nerr(sm.cpu().numpy(), sm_ref) < 1e-9
    inner = (np.abs(E) < 3.5) & (rd_ref[0] > 1e-3 * rd_ref[0].max())
    sc_g = A.semiclassical(rd.cpu().numpy()[0], rv.cpu().numpy(), sv.cpu().numpy())
    sc_o = A.semiclassical(rd_ref[0], rv_ref, sv_ref)
    # energies inside the band where the DOS and velocity are well away from zero;
    # these quantities divide by the DOS and velocity, and normalised noise of 1e-10
    # on the oracle's moments (the moment tolerance) moves them by up to 4.5e-9
    # (sigma_sc, v, tau, mean free path) and 3.4e-8 (L) of their largest values
    for key in ("sigma_sc", "velocity", "tau", "mfp"):
        assert nerr(sc_g[key][inner], sc_o[key][inner]) < 1e-8, key
    Lg = A.propagation_length(rd.cpu().numpy()[0], rm.cpu().numpy())
    Lo = A.propagation_length(rd_ref[0], rm_ref)
    assert nerr(Lg[:, inner], Lo[:, inner]) < 1e-7
