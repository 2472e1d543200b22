"""FP64 moment rows computed on pairs of FP32 numbers (gqt_set_fp64_arith mode 1,
the default for FP64 handles with one vector) through the C ABI.

The kernels k_cheb_pair_df (VAC rows by two recurrences) and k_cheb_dbl_df (l = r
rows: DOS, MSD) keep FP64-sized storage and carry about 48 significant bits in
their arithmetic (hi + lo pairs with error-free sums and products).  They must
meet the FP64 bar: 1e-10 normalised against the serial FP64 oracle, on every
neighbour count they serve (2, 3, 4, 6 slots), real and complex hoppings, tiny
and odd M, several CTAs with a ragged tail, several segments, and at the full
benchmark size against the FP64-pipe mode (gqt_set_fp64_arith mode 0).  The
cluster-resident rows (small systems) are switched off so that the wavefront
kernels run at these sizes.
"""
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


MODELS = {
    "honeycomb37x23": lambda: (S.honeycomb(37, 23, -2.7, 2.0, seed=3), S.energy_scale_rule(3, -2.7, 2.0)),
    "honeycomb37x23_phases": lambda: (S.with_random_bond_phases(S.honeycomb(37, 23, -2.7, 2.0, seed=3), 4),
                                      S.energy_scale_rule(3, -2.7, 2.0)),
    "square41x29": lambda: (S.square(41, 29, -1.0, 4.0, seed=5), S.energy_scale_rule(4, -1.0, 4.0)),
    "cubic13": lambda: (S.cubic(13, -1.0, 16.5, seed=7), S.energy_scale_rule(6, -1.0, 16.5)),
    "chain5001": lambda: (S.chain(5001, -1.0, 4.0, seed=9), S.energy_scale_rule(2, -1.0, 4.0)),
    # real hoppings that are not all equal (bonds to vacancies are zero): the
    # general form, where the others take the one-common-hopping form
    "honeycomb37x23_vac": lambda: (S.honeycomb(37, 23, -2.7, 2.0, seed=4, vacancy_frac=0.02),
                                   S.energy_scale_rule(3, -2.7, 2.0)),
}


def _ham(lat, dE, mode=1):
    ham = g.gqt_build_hamiltonian(lat, dE)
    g.gqt_set_cluster(ham, False)
    g.gqt_set_fp64_arith(ham, mode)
    return ham


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("M", [1, 2, 3, 257])
def test_df_rows_match_oracle(name, M):
    """DOS (l = r), VAC (l != r, two recurrences) and MSD rows of two time steps."""
    lat, dE = MODELS[name]()
    ham = _ham(lat, dE)
    h = O.Hamiltonian(lat, dE)
    phi = S.random_phase(lat.n, 1, seed=M)
    d = torch.from_numpy(phi).cuda()
    dos = np.empty((1, 1, M))
    g.gqt_dos_moments(ham, d, 1, M, dos)
    assert nerr(dos.ravel(), h.dos_moments(phi[:, 0], M).real) < TOL64
    dts = np.array([0.4, 0.7])
    Np = [O.np_rule(dE * t, 64) for t in dts]
    a, b = torch.empty_like(d), torch.empty_like(d)
    g.gqt_vac_init(ham, d, a, b, 1)
    vac = np.empty((2, 1, 1, M))
    g.gqt_vac_moments(ham, a, b, 1, dts, M, vac, Np=Np)
    assert nerr(vac.reshape(2, M), h.vac_moments(phi[:, 0], dts, Np, M)) < TOL64
    p, px = torch.empty_like(d), torch.empty_like(d)
    g.gqt_msd_init(ham, d, p, px, 1)
    msd = np.empty((2, 1, 1, M))
    g.gqt_msd_moments(ham, p, px, 1, dts, M, msd, Np=Np)
    assert nerr(msd.reshape(2, M), h.msd_moments(phi[:, 0], dts, Np, M)) < TOL64


@pytest.mark.parametrize("name", ["honeycomb37x23", "honeycomb37x23_phases", "cubic13"])
def test_df_and_fp64_modes_agree(name):
    """The same rows in both arithmetic modes: within 1e-12 (measured about 2e-15)."""
    lat, dE = MODELS[name]()
    phi = torch.from_numpy(S.random_phase(lat.n, 1, seed=12)).cuda()
    M = 600
    rows = {}
    for mode in (0, 1):
        ham = _ham(lat, dE, mode)
        dos = np.empty((1, 1, M))
        g.gqt_dos_moments(ham, phi, 1, M, dos)
        a, b = torch.empty_like(phi), torch.empty_like(phi)
        g.gqt_vac_init(ham, phi, a, b, 1)
        vac = np.empty((1, 1, 1, M))
        g.gqt_vac_moments(ham, a, b, 1, [0.5], M, vac)
        rows[mode] = (dos.ravel(), vac.ravel())
    for k in range(2):
        assert nerr(rows[1][k], rows[0][k]) < 1e-12


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("dt,sign", [(0.01, 1), (0.05, -1), (0.4, 1), (2.0, -1)])
def test_df_evolution_matches_oracle_and_fp64_pipe(name, dt, sign):
    """U(+-dt) psi (Eq. 17) and [X,U(dt)] psi (Eqs. 18, 22, 24) with the orders on
    pairs of FP32 numbers (mode 1), for expansions of 1, 2, 3 and up to 29 orders,
    on every neighbour count and with complex hoppings: within 1e-10 of the oracle,
    within 1e-13 (U) and 1e-12 ([X,U]) of the FP64-pipe kernels (mode 0), and the
    reported norm within 1e-12 of 1."""
    lat, dE = MODELS[name]()
    h = O.Hamiltonian(lat, dE)
    psi = S.random_phase(lat.n, 1, seed=31)
    rule = O.np_rule(dE * dt, 64)
    for Np in sorted({1, 2, 3, rule}):
        got = {}
        for mode in (1, 0):
            ham = _ham(lat, dE, mode)
            d = torch.from_numpy(psi).cuda()
            norm = np.full(1, np.nan)
            errs = []
            # an expansion cut below the rule fails the norm check (GQT_ENORM) after
            # computing the truncated sum, which is still compared
            try:
                g.gqt_evolve(ham, d, 1, dt, sign, Np, norm=norm)
            except g.GqtError as e:
                errs.append(e.status)
            out = torch.empty_like(d)
            try:
                g.gqt_commutator_evolve(ham, torch.from_numpy(psi).cuda(), out, 1, dt, Np)
            except g.GqtError as e:
                errs.append(e.status)
            got[mode] = (d.cpu().numpy()[:, 0], out.cpu().numpy()[:, 0], norm[0], errs)
        assert got[1][3] == got[0][3], (Np, got[1][3], got[0][3])
        assert (len(got[1][3]) == 0) == (Np >= rule), (Np, rule, got[1][3])
        assert nerr(got[1][0], h.evolve(psi[:, 0], dt, sign, Np)) < TOL64, Np
        assert nerr(got[1][1], h.commutator_evolve(psi[:, 0], dt, Np)) < TOL64, Np
        assert nerr(got[1][0], got[0][0]) < 1e-13, Np
        assert nerr(got[1][1], got[0][1]) < 1e-12, Np
        if Np >= rule:
            assert abs(got[1][2] - 1.0) < 1e-12


def test_df_evolution_runs_on_the_fp32_pipes():
    """Mode 1 handles launch the paired-FP32 evolution orders (profile families 3
    and 4 count the middle orders), and a VAC + MSD step of the bench workload's
    form equals the FP64-pipe mode within 1e-12."""
    lat, dE = MODELS["honeycomb37x23"]()
    phi = torch.from_numpy(S.random_phase(lat.n, 1, seed=33)).cuda()
    M = 64
    rows = {}
    for mode in (1, 0):
        ham = _ham(lat, dE, mode)
        a, b, p, px = (torch.empty_like(phi) for _ in range(4))
        g.gqt_vac_init(ham, phi, a, b, 1)
        g.gqt_msd_init(ham, phi, p, px, 1)
        vac = np.empty((2, 1, 1, M))
        msd = np.empty((2, 1, 1, M))
        g.gqt_profile_start()
        g.gqt_vac_moments(ham, a, b, 1, [0.74, 0.74], M, vac)
        g.gqt_msd_moments(ham, p, px, 1, [0.74, 0.74], M, msd)
        torch.cuda.synchronize()
        _, n = g.gqt_profile_stop(5)
        assert n[3] > 0 and n[4] > 0, n
        rows[mode] = (vac.ravel(), msd.ravel(), a.cpu().numpy(), px.cpu().numpy())
    for k in range(4):
        assert nerr(rows[1][k], rows[0][k]) < 1e-12, k


def test_df_ragged_segments_match_separate_builds():
    """Several segments in one handle (block-diagonal realisations): per-segment DOS
    and VAC moments equal the oracle on each realisation."""
    parts = [S.honeycomb(L1, L2, -2.7, 2.0, seed=40 + q) for q, (L1, L2) in enumerate(((9, 7), (13, 5), (6, 6)))]
    blk = S.block_diagonal(parts)
    dE = S.energy_scale_rule(3, -2.7, 2.0)
    ham = _ham(blk, dE)
    assert ham.nseg == 3
    phi = torch.empty((blk.n, 1), dtype=torch.complex128, device="cuda")
    g.gqt_random_phase(ham, 78, 1, phi)
    M = 129
    mu = np.empty((3, 1, M))
    g.gqt_dos_moments(ham, phi, 1, M, mu)
    a, b = torch.empty_like(phi), torch.empty_like(phi)
    g.gqt_vac_init(ham, phi, a, b, 1)
    vac = np.empty((1, 3, 1, M))
    g.gqt_vac_moments(ham, a, b, 1, [0.3], M, vac)
    ph = phi.cpu().numpy()[:, 0]
    for q, p in enumerate(parts):
        o = blk.seg_offsets[q]
        h = O.Hamiltonian(p, dE)
        assert nerr(mu[q, 0], h.dos_moments(ph[o:o + p.n], M).real) < TOL64
        ref = h.vac_moments(ph[o:o + p.n], [0.3], [O.np_rule(dE * 0.3, 64)], M)
        assert nerr(vac[0, q, 0], ref[0]) < TOL64


def test_df_split_follows_hamiltonian_updates():
    """gqt_update_hamiltonian invalidates the (hi, lo) split of 2H~: moments after an
    update equal the oracle on the updated model."""
    lat, dE = MODELS["square41x29"]()
    ham = _ham(lat, dE)
    phi = torch.from_numpy(S.random_phase(lat.n, 1, seed=3)).cuda()
    M = 200
    mu = np.empty((1, 1, M))
    g.gqt_dos_moments(ham, phi, 1, M, mu)  # builds the split of the first model
    rng = np.random.default_rng(4)
    lat.onsite = rng.uniform(-1.5, 1.5, lat.n)
    lat.hop = lat.hop * 0.9
    g.gqt_update_hamiltonian(ham, lat.onsite, lat.hop)
    g.gqt_dos_moments(ham, phi, 1, M, mu)
    ref = O.Hamiltonian(lat, dE).dos_moments(phi.cpu().numpy()[:, 0], M).real
    assert nerr(mu.ravel(), ref) < TOL64


def test_blocked_rows_follow_hopping_uniformity_through_updates():
    """A honeycomb handle whose hoppings are all equal runs the blocked rows without
    reading a hop array (one product with the common value); an update to unequal
    bond hoppings, and back to equal ones, switches the form on the same handle.
    DOS and VAC rows match the oracle on each model, and the blocked kernel runs."""
    lat, dE = TILED["honeycomb64x32"]()
    ham = _ham(lat, dE)
    phi = S.random_phase(lat.n, 1, seed=8)
    d = torch.from_numpy(phi).cuda()
    M = 40
    dts = np.array([0.4])
    Np = [O.np_rule(dE * 0.4, 64)]
    t0 = lat.hop.copy()
    j = lat.nb_idx
    i = np.arange(lat.n)[:, None]
    models = [t0, t0 * (1.0 + 0.05 * ((i + j) % 7) / 7.0), t0 * 0.9]  # equal, unequal (symmetric), equal
    for q, hop in enumerate(models):
        if q:
            lat.hop = hop
            g.gqt_update_hamiltonian(ham, lat.onsite, lat.hop)
        uniform = g.GQT_FORM_UNIFORM_HOP if q != 1 else 0
        assert ham.forms == g.GQT_FORM_HONEYCOMB | uniform, (q, ham.forms)
        dos = np.empty((1, 1, M))
        vac = np.empty((1, 1, 1, M))
        a, b = torch.empty_like(d), torch.empty_like(d)
        g.gqt_vac_init(ham, d, a, b, 1)

        def run():
            g.gqt_dos_moments(ham, d, 1, M, dos)
            g.gqt_vac_moments(ham, a, b, 1, dts, M, vac, Np=Np)

        assert _tiled_launches(run) > 0, q
        h = O.Hamiltonian(lat, dE)
        assert nerr(dos.ravel(), h.dos_moments(phi[:, 0], M).real) < TOL64, q
        assert nerr(vac.ravel(), h.vac_moments(phi[:, 0], dts, Np, M)[0]) < TOL64, q


def test_storage_forms_reported():
    """gqt_ham_forms: the honeycomb cell layout, one common real hopping (FP64
    handles) and the blocked cubic sweep order, as recognised at build."""
    hc = S.honeycomb(64, 32, -2.7, 2.0, seed=13)
    dE = S.energy_scale_rule(3, -2.7, 2.0)
    assert g.gqt_build_hamiltonian(hc, dE).forms == g.GQT_FORM_HONEYCOMB | g.GQT_FORM_UNIFORM_HOP
    assert g.gqt_build_hamiltonian(hc, dE, g.GQT_FP32_ACC64).forms == g.GQT_FORM_HONEYCOMB
    vac = S.honeycomb(64, 32, -2.7, 2.0, seed=13, vacancy_frac=0.01)
    assert g.gqt_build_hamiltonian(vac, dE).forms == g.GQT_FORM_HONEYCOMB
    ph = S.with_random_bond_phases(hc, 5)
    assert g.gqt_build_hamiltonian(ph, dE).forms == g.GQT_FORM_HONEYCOMB
    cub = g.gqt_build_hamiltonian(None, S.energy_scale_rule(6, -1.0, 16.5), g.GQT_FP64, kind=g.GQT_LATTICE_CUBIC,
                                  L1=64, t=-1.0, W=16.5, seed=3)
    assert cub.forms == g.GQT_FORM_CUBIC_SWEEP | g.GQT_FORM_UNIFORM_HOP
    sq = S.square(41, 29, -1.0, 4.0, seed=5)
    assert g.gqt_build_hamiltonian(sq, S.energy_scale_rule(4, -1.0, 4.0)).forms == g.GQT_FORM_UNIFORM_HOP


def test_df_mode_argument():
    lat, dE = MODELS["chain5001"]()
    ham = g.gqt_build_hamiltonian(lat, dE)
    with pytest.raises(g.GqtError) as e:
        g.gqt_set_fp64_arith(ham, 2)
    assert e.value.status == g.GQT_EINVAL


@pytest.mark.slow
def test_df_full_size_agrees_with_fp64_mode():
    """Honeycomb 4096 x 2048 (N = 16,777,216), the benchmark's rows at M = 3000: DOS,
    one VAC row and one MSD row in both modes agree to 1e-12 of their largest moment
    (measured 2e-15); the FP64 mode is itself oracle-checked at this size on balls of
    the lattice (test_gpu_runtime.py)."""
    ham = g.gqt_build_hamiltonian(None, 9.555, g.GQT_FP64, kind=g.GQT_LATTICE_HONEYCOMB, L1=4096, L2=2048, t=-2.7,
                                  W=2.0, seed=S.BASE_SEED + 1)
    N = 4096 * 2048 * 2
    phi = torch.empty((N, 1), dtype=torch.complex128, device="cuda")
    g.gqt_random_phase(ham, S.BASE_SEED + 1, 1, phi)
    M, dt = 3000, 2.0 / 2.7
    rows = {}
    for mode in (0, 1):
        g.gqt_set_fp64_arith(ham, mode)
        a, b, p, px = (torch.empty_like(phi) for _ in range(4))
        g.gqt_vac_init(ham, phi, a, b, 1)
        g.gqt_msd_init(ham, phi, p, px, 1)
        dos, vac, msd = np.empty((1, 1, M)), np.empty((1, 1, 1, M)), np.empty((1, 1, 1, M))
        g.gqt_dos_moments(ham, phi, 1, M, dos)
        g.gqt_vac_moments(ham, a, b, 1, [dt], M, vac)
        g.gqt_msd_moments(ham, p, px, 1, [dt], M, msd)
        rows[mode] = (dos.ravel(), vac.ravel(), msd.ravel())
    for k in range(3):
        assert nerr(rows[1][k], rows[0][k]) < 1e-12, k
    assert abs(rows[1][0][0] - 1.0) < 1e-13


def _tiled_launches(fn):
    g.gqt_profile_start()
    fn()
    torch.cuda.synchronize()
    _, n = g.gqt_profile_stop(12)
    return int(n[10] + n[11])


TILED = {
    "honeycomb64x32": lambda: (S.honeycomb(64, 32, -2.7, 2.0, seed=13), S.energy_scale_rule(3, -2.7, 2.0)),
    "honeycomb96x48_vac": lambda: (S.honeycomb(96, 48, -2.7, 0.5, seed=14, vacancy_frac=0.01),
                                   S.energy_scale_rule(3, -2.7, 0.5)),
    "honeycomb64x32_phases": lambda: (S.with_random_bond_phases(S.honeycomb(64, 32, -2.7, 2.0, seed=15), 16),
                                      S.energy_scale_rule(3, -2.7, 2.0)),
}


@pytest.mark.parametrize("name", list(TILED))
@pytest.mark.parametrize("M", [1, 3, 4, 5, 6, 9, 130, 257])
def test_tiled_rows_match_oracle_and_single_step(name, M):
    """Temporal blocking (two steps per launch, each CTA walking a band of cells
    down the rows and recomputing its halo) on honeycomb lattices whose L1 the
    bands divide, with disorder, vacancies and complex hoppings, for step counts
    that leave 0 or 1 single steps after the blocked passes: DOS, VAC and MSD
    rows within 1e-10 of the oracle and within 1e-13 of the single-step kernels,
    and the blocked kernel must actually have run."""
    lat, dE = TILED[name]()
    h = O.Hamiltonian(lat, dE)
    phi = S.random_phase(lat.n, 1, seed=M + 1)
    d = torch.from_numpy(phi).cuda()
    dts = np.array([0.5])
    Np = [O.np_rule(dE * 0.5, 64)]
    rows = {}
    for tiling in (True, False):
        ham = _ham(lat, dE)
        g.gqt_set_temporal_blocking(ham, tiling)
        dos = np.empty((1, 1, M))
        vac = np.empty((1, 1, 1, M))
        msd = np.empty((1, 1, 1, M))
        a, b, p, px = (torch.empty_like(d) for _ in range(4))
        g.gqt_vac_init(ham, d, a, b, 1)
        g.gqt_msd_init(ham, d, p, px, 1)

        def run():
            g.gqt_dos_moments(ham, d, 1, M, dos)
            g.gqt_vac_moments(ham, a, b, 1, dts, M, vac, Np=Np)
            g.gqt_msd_moments(ham, p, px, 1, dts, M, msd, Np=Np)

        n_tiled = _tiled_launches(run)
        steps = (M + 1) // 2
        assert (n_tiled > 0) == (tiling and steps >= 3), n_tiled
        rows[tiling] = (dos.ravel(), vac.ravel(), msd.ravel())
    ref = (h.dos_moments(phi[:, 0], M).real, h.vac_moments(phi[:, 0], dts, Np, M)[0],
           h.msd_moments(phi[:, 0], dts, Np, M)[0])
    for k in range(3):
        assert nerr(rows[True][k], ref[k]) < TOL64, k
        assert nerr(rows[True][k], rows[False][k]) < 1e-13, k


def test_tiled_layout_not_recognised_falls_back():
    """A honeycomb lattice whose L1 no band width divides (40 x 24), and a square
    lattice, run the single-step kernels (no blocked launch) and stay exact."""
    for lat, dE in ((S.honeycomb(40, 24, -2.7, 2.0, seed=16), S.energy_scale_rule(3, -2.7, 2.0)),
                    (S.square(41, 29, -1.0, 4.0, seed=5), S.energy_scale_rule(4, -1.0, 4.0))):
        ham = _ham(lat, dE)
        phi = S.random_phase(lat.n, 1, seed=3)
        d = torch.from_numpy(phi).cuda()
        g.gqt_set_temporal_blocking(ham, True)
        mu = np.empty((1, 1, 64))
        assert _tiled_launches(lambda: g.gqt_dos_moments(ham, d, 1, 64, mu)) == 0
        assert nerr(mu.ravel(), O.Hamiltonian(lat, dE).dos_moments(phi[:, 0], 64).real) < TOL64


def test_setting_change_retires_captured_graphs():
    """Switching temporal blocking off and on again on one handle takes effect on
    the next call although the call's pointers and sizes repeat (the captured
    graphs that carried the old choice are retired): blocked launches run, then
    none, then again, with the same moments to 1e-13."""
    lat, dE = TILED["honeycomb64x32"]()
    ham = _ham(lat, dE)
    d = torch.from_numpy(S.random_phase(lat.n, 1, seed=4)).cuda()
    M = 40
    mus, counts = [], []
    for tiling in (True, False, True):
        g.gqt_set_temporal_blocking(ham, tiling)
        mu = np.empty((1, 1, M))
        counts.append(_tiled_launches(lambda: g.gqt_dos_moments(ham, d, 1, M, mu)))
        mus.append(mu.ravel().copy())
    assert counts[0] > 0 and counts[1] == 0 and counts[2] > 0, counts
    assert nerr(mus[1], mus[0]) < 1e-13 and np.array_equal(mus[2], mus[0])


BANDS = {
    # one band of 32 cells: the halo wraps round the periodic boundary on both sides
    "honeycomb32x4": (32, 4),
    "honeycomb32x5": (32, 5),
    # two segments, the second only two rows high
    "honeycomb64x130": (64, 130),
    # 32 bands x 8 segments (the last 104 rows): more work items than CTAs of the
    # two-chain kernel, so a CTA carries its row rings from one item to the next
    "honeycomb1024x1000": (1024, 1000),
    # 64 bands x 5 segments (the last 8 rows): more items than CTAs of either kernel
    "honeycomb2048x520": (2048, 520),
}


@pytest.mark.parametrize("name", list(BANDS))
def test_tiled_band_geometry(name):
    """Band walk of the blocked kernel at the edges of its geometry: a single band,
    the fewest rows, ragged segments and several items per CTA.  Nine moments
    (first order + two blocked passes) of DOS, VAC and MSD rows equal the
    single-step kernels within 1e-13, and the DOS row the oracle within 1e-10."""
    L1, L2 = BANDS[name]
    lat = S.honeycomb(L1, L2, -2.7, 2.0, seed=L1 + L2, vacancy_frac=0.005)
    dE = S.energy_scale_rule(3, -2.7, 2.0)
    M = 9
    phi = S.random_phase(lat.n, 1, seed=L2)
    d = torch.from_numpy(phi).cuda()
    dts = np.array([0.5])
    Np = [O.np_rule(dE * 0.5, 64)]
    rows = {}
    for tiling in (True, False):
        ham = _ham(lat, dE)
        g.gqt_set_temporal_blocking(ham, tiling)
        dos = np.empty((1, 1, M))
        vac = np.empty((1, 1, 1, M))
        msd = np.empty((1, 1, 1, M))
        a, b, p, px = (torch.empty_like(d) for _ in range(4))
        g.gqt_vac_init(ham, d, a, b, 1)
        g.gqt_msd_init(ham, d, p, px, 1)

        def run():
            g.gqt_dos_moments(ham, d, 1, M, dos)
            g.gqt_vac_moments(ham, a, b, 1, dts, M, vac, Np=Np)
            g.gqt_msd_moments(ham, p, px, 1, dts, M, msd, Np=Np)

        n_tiled = _tiled_launches(run)
        assert (n_tiled > 0) == tiling, n_tiled
        rows[tiling] = (dos.ravel(), vac.ravel(), msd.ravel())
    for k in range(3):
        assert nerr(rows[True][k], rows[False][k]) < 1e-13, k
    ref = O.Hamiltonian(lat, dE).dos_moments(phi[:, 0], M).real
    assert nerr(rows[True][0], ref) < TOL64

