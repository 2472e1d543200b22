"""Edge cases through the C ABI: irregular neighbour lists with padding slots and
neighbour counts outside the specialised set, one-site segments, tiny orders and
expansion lengths, and argument errors returned as status codes."""
import numpy as np
import pytest

import gqt_synth as S
import oracle as O

torch = pytest.importorskip("torch")
g = pytest.importorskip("paper_1705_01387_gb300")

pytestmark = pytest.mark.gpu


def nerr(x, y):
    return float(np.max(np.abs(np.asarray(x) - np.asarray(y))) / max(float(np.max(np.abs(y))), 1e-300))


def random_graph(n, kmax, seed):
    """Random Hermitian model: each undirected bond joins two random sites, complex
    hopping, rows padded to kmax slots (counts 0..kmax), random x-displacements."""
    rng = np.random.default_rng(seed)
    cnt = np.zeros(n, np.int32)
    idx = np.tile(np.arange(n, dtype=np.int32)[:, None], (1, kmax))
    hop = np.zeros((n, kmax), np.complex128)
    dx = np.zeros((n, kmax))
    for _ in range(n * kmax // 3):
        i, j = rng.integers(n, size=2)
        if i == j or cnt[i] >= kmax or cnt[j] >= kmax or j in idx[i, :cnt[i]]:
            continue
        t = rng.normal() + 1j * rng.normal()
        d = rng.normal()
        idx[i, cnt[i]], hop[i, cnt[i]], dx[i, cnt[i]] = j, t, d
        idx[j, cnt[j]], hop[j, cnt[j]], dx[j, cnt[j]] = i, np.conj(t), -d
        cnt[i] += 1
        cnt[j] += 1
    ons = rng.uniform(-1, 1, n)
    lat = S.Lattice("random", n, kmax, cnt, idx, hop, ons, dx, 1.0, float(n))
    dE = 1.05 * float(np.max(np.abs(ons) + np.abs(hop).sum(1)))
    return lat, dE


@pytest.mark.parametrize("kmax", [7, 3])
def test_irregular_neighbour_lists(kmax):
    lat, dE = random_graph(1501, kmax, seed=kmax)
    assert lat.nb_count.min() < kmax  # padding present
    ham = g.gqt_build_hamiltonian(lat, dE)
    phi = S.random_phase(lat.n, 1, seed=3)
    d = torch.from_numpy(phi).cuda()
    h = O.Hamiltonian(lat, dE)
    M = 120
    mu = np.empty((1, 1, M))
    g.gqt_dos_moments(ham, d, 1, M, mu)
    assert nerr(mu.reshape(M), h.dos_moments(phi[:, 0], M)) < 1e-10
    dts = np.array([0.5, 0.3])
    Np = [O.np_rule(dE * x, 64) for x in dts]
    a, b = torch.empty_like(d), torch.empty_like(d)
    g.gqt_vac_init(ham, d, a, b, 1)
    vac = np.empty((2, 1, 1, M))
    g.gqt_vac_moments(ham, a, b, 1, dts, M, vac, Np=Np)
    assert nerr(vac.reshape(2, M), h.vac_moments(phi[:, 0], dts, Np, M)) < 1e-10
    p, px = torch.empty_like(d), torch.empty_like(d)
    g.gqt_msd_init(ham, d, p, px, 1)
    msd = np.empty((2, 1, 1, M))
    g.gqt_msd_moments(ham, p, px, 1, dts, M, msd, Np=Np)
    assert nerr(msd.reshape(2, M), h.msd_moments(phi[:, 0], dts, Np, M)) < 1e-10


@pytest.mark.parametrize("Np", [1, 2, 3])
def test_short_expansions(Np):
    lat = S.square(9, 7, -1.0, 2.0, seed=1)
    dE = S.energy_scale_rule(4, -1.0, 2.0)
    ham = g.gqt_build_hamiltonian(lat, dE)
    psi = S.random_phase(lat.n, 1, seed=2)
    d = torch.from_numpy(psi).cuda()
    g.gqt_set_graphs(ham, False)
    h = O.Hamiltonian(lat, dE)
    # truncated expansions are not unitary: only compare the vectors
    try:
        g.gqt_evolve(ham, d, 1, 0.01, 1, Np)
    except g.GqtError as e:
        assert e.status == g.GQT_ENORM
    assert nerr(d.cpu().numpy()[:, 0], h.evolve(psi[:, 0], 0.01, 1, Np)) < 1e-10
    if Np > 1:
        out = torch.empty_like(d)
        try:
            g.gqt_commutator_evolve(ham, torch.from_numpy(psi).cuda(), out, 1, 0.01, Np)
        except g.GqtError as e:
            assert e.status == g.GQT_ENORM  # truncated U is not unitary
        assert nerr(out.cpu().numpy()[:, 0], h.commutator_evolve(psi[:, 0], 0.01, Np)) < 1e-10


def test_one_site_segments_and_isolated_sites():
    """A block-diagonal batch containing one-site and bond-less realisations."""
    parts = [S.chain(5, -1.0, 1.0, seed=1), S.chain(3, -1.0, 1.0, seed=2)]
    single = S.Lattice("one", 1, 2, np.zeros(1, np.int32), np.zeros((1, 2), np.int32), np.zeros((1, 2), np.complex128),
                       np.array([0.3]), np.zeros((1, 2)), 1.0, 1.0)
    blk = S.block_diagonal(parts + [single])
    ham = g.gqt_build_hamiltonian(blk, 3.0)
    phi = torch.empty((blk.n, 1), dtype=torch.complex128, device="cuda")
    g.gqt_random_phase(ham, 5, 1, phi)
    M = 20
    mu = np.empty((3, 1, M))
    g.gqt_dos_moments(ham, phi, 1, M, mu)
    # the one-site segment: mu_n = cos(n arccos(0.3/3))
    assert np.max(np.abs(mu[2, 0] - np.cos(np.arange(M) * np.arccos(0.1)))) < 1e-13
    for q, p in enumerate(parts):
        o = blk.seg_offsets[q]
        ref = O.Hamiltonian(p, 3.0).dos_moments(phi.cpu().numpy()[o:o + p.n, 0], M)
        assert nerr(mu[q, 0], ref) < 1e-12


def test_argument_errors_are_status_codes():
    lat = S.square(5, 5, -1.0, 1.0, seed=1)
    ham = g.gqt_build_hamiltonian(lat, 5.0)
    phi = torch.zeros((lat.n, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(g.GqtError) as e:
        g.gqt_dos_moments(ham, phi, 3, 10, np.empty(30))  # R = 3 not supported
    assert e.value.status == g.GQT_EINVAL
    phi1 = torch.zeros((lat.n, 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(g.GqtError) as e:
        g.gqt_dos_moments(ham, phi1, 1, 0, np.empty(1))  # M = 0
    assert e.value.status == g.GQT_EINVAL
    with pytest.raises(g.GqtError) as e:
        g.gqt_evolve(ham, phi1, 1, -0.5, 1)  # negative time step
    assert e.value.status == g.GQT_EINVAL
    bad = S.square(5, 5, -1.0, 1.0, seed=1)
    bad.onsite[3] = np.nan
    with pytest.raises(g.GqtError) as e:
        g.gqt_build_hamiltonian(bad, 5.0)
    assert e.value.status == g.GQT_ENAN
    with pytest.raises(g.GqtError) as e:
        g.gqt_build_hamiltonian(None, 5.0, kind=g.GQT_LATTICE_HONEYCOMB, L1=1, L2=4)
    assert e.value.status == g.GQT_EINVAL
