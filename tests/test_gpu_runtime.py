"""Runtime features of the library on the GPU: CUDA-graph replay, the autotuner,
launch-shape changes, resumable time loops and full-size sampled parity."""
import numpy as np
import pytest

import gqt_synth as S
import oracle as O

torch = pytest.importorskip("torch")
g = pytest.importorskip("paper_1705_01387_gb300")

pytestmark = pytest.mark.gpu


def nerr(x, y):
    return float(np.max(np.abs(np.asarray(x) - np.asarray(y))) / max(float(np.max(np.abs(y))), 1e-300))


def _c1():
    w = S.config(0)
    return w, S.build_lattice(w.lattice_args, w.seed)


def _vac(ham, phi, dts, M, Np):
    a, b = torch.empty_like(phi), torch.empty_like(phi)
    g.gqt_vac_init(ham, phi, a, b, phi.shape[1])
    out = np.empty((len(dts), ham.nseg, phi.shape[1], M))
    g.gqt_vac_moments(ham, a, b, phi.shape[1], dts, M, out, Np=Np)
    return out


def test_graph_replay_is_bit_identical_to_direct_launches():
    w, lat = _c1()
    ham = g.gqt_build_hamiltonian(lat, w.energy_scale)
    phi = torch.from_numpy(S.random_phase(lat.n, 1, seed=w.seed)).cuda()
    dts = np.full(3, w.dt)
    Np = [g.gqt_np_rule(w.energy_scale * d) for d in dts]
    g.gqt_set_graphs(ham, True)
    first = _vac(ham, phi, dts, 200, Np)
    again = _vac(ham, phi, dts, 200, Np)  # replays the cached graphs
    g.gqt_set_graphs(ham, False)
    direct = _vac(ham, phi, dts, 200, Np)
    assert np.array_equal(first, again) and np.array_equal(first, direct)


def test_autotune_and_launch_shapes_keep_results():
    lat = S.square(61, 47, -1.0, 4.0, seed=5)
    dE = S.energy_scale_rule(4, -1.0, 4.0)
    ham = g.gqt_build_hamiltonian(lat, dE)
    phi = S.random_phase(lat.n, 8, seed=6)
    d = torch.from_numpy(phi).cuda()
    ref = O.Hamiltonian(lat, dE).dos_moments(phi[:, 3], 128)
    thr, bps, var = g.gqt_autotune(ham, 8)
    assert thr in (128, 256, 512) and bps in (0, 2, 4, 8) and var in (0, 1, 2, 3)
    for t, b in ((thr, bps), (128, 2), (512, 8), (256, 4)):
        g.gqt_set_launch(ham, t, b)
        mu = np.empty((1, 8, 128))
        g.gqt_dos_moments(ham, d, 8, 128, mu)
        assert nerr(mu[0, 3], ref) < 1e-10


def test_time_loop_is_resumable():
    """Nt steps in one call equal the same steps split over two calls (state in/out)."""
    w, lat = _c1()
    ham = g.gqt_build_hamiltonian(lat, w.energy_scale)
    phi = torch.from_numpy(S.random_phase(lat.n, 1, seed=3)).cuda()
    dts = np.array([0.3, 0.5, 0.2, 0.4])
    Np = [g.gqt_np_rule(w.energy_scale * d) for d in dts]
    whole = _vac(ham, phi, dts, 64, Np)
    a, b = torch.empty_like(phi), torch.empty_like(phi)
    g.gqt_vac_init(ham, phi, a, b, 1)
    p1 = np.empty((2, 1, 1, 64))
    p2 = np.empty((2, 1, 1, 64))
    g.gqt_vac_moments(ham, a, b, 1, dts[:2], 64, p1, Np=Np[:2])
    g.gqt_vac_moments(ham, a, b, 1, dts[2:], 64, p2, Np=Np[2:])
    assert nerr(np.concatenate([p1, p2]), whole) < 1e-13
    p, px = torch.empty_like(phi), torch.empty_like(phi)
    g.gqt_msd_init(ham, phi, p, px, 1)
    m_all = np.empty((4, 1, 1, 64))
    g.gqt_msd_moments(ham, p, px, 1, dts, 64, m_all, Np=Np)
    g.gqt_msd_init(ham, phi, p, px, 1)
    m1 = np.empty((2, 1, 1, 64))
    m2 = np.empty((2, 1, 1, 64))
    g.gqt_msd_moments(ham, p, px, 1, dts[:2], 64, m1, Np=Np[:2])
    g.gqt_msd_moments(ham, p, px, 1, dts[2:], 64, m2, Np=Np[2:])
    assert nerr(np.concatenate([m1, m2]), m_all) < 1e-13


def _ball_sites(lat, centre, radius):
    """Sites within `radius` hops of `centre`."""
    dist = {centre: 0}
    frontier = [centre]
    for d in range(radius):
        nxt = []
        for i in frontier:
            for k in range(lat.nb_count[i]):
                j = int(lat.nb_idx[i, k])
                if j not in dist:
                    dist[j] = d + 1
                    nxt.append(j)
        frontier = nxt
    return list(dist)


def _ball(lat, centre, radius):
    """Sites within `radius` hops of `centre` and the induced model (same H entries)."""
    sites = np.array(sorted(_ball_sites(lat, centre, radius)))
    pos = {s: q for q, s in enumerate(sites)}
    n, K = sites.size, lat.max_nb
    sub = S.Lattice("ball", n, K, np.zeros(n, np.int32), np.zeros((n, K), np.int32), np.zeros((n, K), np.complex128),
                    lat.onsite[sites].copy(), np.zeros((n, K)), 0.0, 1.0)
    for q, s in enumerate(sites):
        c = 0
        for k in range(lat.nb_count[s]):
            j = int(lat.nb_idx[s, k])
            if j in pos:
                sub.nb_idx[q, c] = pos[j]
                sub.hop[q, c] = lat.hop[s, k]
                sub.dx[q, c] = lat.dx[s, k]
                c += 1
        sub.nb_count[q] = c
        sub.nb_idx[q, c:] = q
    return sub, pos[centre]


@pytest.fixture(scope="module")
def c2():
    """The benchmark's workload: honeycomb 4096 x 2048 (N = 16,777,216), W = 2 eV, FP64."""
    w = S.config(1)
    lat = S.build_lattice(w.lattice_args, w.seed)
    ham = g.gqt_build_hamiltonian(lat, w.energy_scale)
    return w, lat, ham


def _local_start(lat, centre, seed):
    """Unit vector with random phases and magnitudes on the sites within 2 hops of
    `centre` (not an eigenvector of anything, not symmetric under V)."""
    sites = np.array(sorted(_ball_sites(lat, centre, 2)))
    rng = np.random.default_rng(seed)
    v = rng.uniform(0.5, 1.0, sites.size) * np.exp(2j * np.pi * rng.uniform(size=sites.size))
    return sites, v / np.linalg.norm(v)


@pytest.mark.slow
@pytest.mark.parametrize("kind", ["vac", "msd"])
def test_full_size_vac_and_msd_rows_at_benchmark_launch_shape(c2, kind):
    """The VAC row kernel (two recurrences, k_cheb_pair_w) and the MSD row (k_msd_evolve,
    k_cheb_dbl_w) on the full benchmark lattice, launched exactly as the benchmark
    launches them (R = 1, N = 16.8M, every CTA of the wavefront grid), against the
    oracle on a ball of the same lattice.  The start vector lives within 2 hops of a
    sampled site i; two steps of a short dt (N_p = 12) make the second VAC row an
    l != r product (l = V U a, r = U V a).  A row moment after k steps is a closed walk
    from the start support of length <= 2k(N_p - 1) + 2 + n, so the truncated ball of
    radius Nt N_p + M/2 + 4 around i gives exactly the full lattice's values (Eqs. 17,
    18, 22, 29, 30).  Tolerance 1e-10 normalised per row."""
    w, lat, ham = c2
    dE = w.energy_scale
    M, dts = 40, np.array([0.05, 0.05])
    Np = [g.gqt_np_rule(dE * d, 4096) for d in dts]
    assert Np[0] == O.np_rule(dE * dts[0], 4096)
    rng = np.random.default_rng(17 if kind == "vac" else 19)
    for i in rng.choice(lat.n, 2, replace=False):
        sites, v = _local_start(lat, int(i), int(i))
        phi = torch.zeros((lat.n, 1), dtype=torch.complex128, device="cuda")
        phi[torch.from_numpy(sites).cuda(), 0] = torch.from_numpy(v).cuda()
        x, y = torch.empty_like(phi), torch.empty_like(phi)
        got = np.empty((len(dts), 1, 1, M))
        if kind == "vac":
            g.gqt_vac_init(ham, phi, x, y, 1)
            g.gqt_vac_moments(ham, x, y, 1, dts, M, got, Np=Np)
        else:
            g.gqt_msd_init(ham, phi, x, y, 1)
            g.gqt_msd_moments(ham, x, y, 1, dts, M, got, Np=Np)
        radius = len(dts) * max(Np) + M // 2 + 4
        sub, _ = _ball(lat, int(i), radius)
        pos = {s: q for q, s in enumerate(sorted(_ball_sites(lat, int(i), radius)))}
        ps = np.zeros(sub.n, np.complex128)
        for s_, val in zip(sites, v):
            ps[pos[int(s_)]] = val
        h = O.Hamiltonian(sub, dE)
        ref = h.vac_moments(ps, dts, Np, M) if kind == "vac" else h.msd_moments(ps, dts, Np, M)
        for k in range(len(dts)):
            assert nerr(got[k, 0, 0], ref[k]) < 1e-10, (kind, int(i), k)


@pytest.mark.slow
def test_full_size_sampled_local_moments(c2):
    """Honeycomb 4096 x 2048 (N = 16,777,216), FP64, the benchmark's launch shape:
    local moments <e_i|T_m(H~)|e_i> for sampled sites i, m < 40, equal the oracle's on
    the ball of radius 20 around i (closed walks of length m stay within m/2 hops)."""
    w, lat, ham = c2
    dE = w.energy_scale
    M = 40
    rng = np.random.default_rng(5)
    for i in rng.choice(lat.n, 3, replace=False):
        e = torch.zeros((lat.n, 1), dtype=torch.complex128, device="cuda")
        e[int(i), 0] = 1.0
        mu = np.empty((1, 1, M))
        g.gqt_dos_moments(ham, e, 1, M, mu)
        sub, c = _ball(lat, int(i), 20)
        ec = np.zeros(sub.n, np.complex128)
        ec[c] = 1.0
        ref = O.Hamiltonian(sub, dE).dos_moments(ec, M)
        assert nerr(mu.reshape(M), ref) < 1e-10
    # properties at full size: unit norm moments bounded, evolution unitary and reversible
    phi = torch.empty((lat.n, 1), dtype=torch.complex128, device="cuda")
    g.gqt_random_phase(ham, w.seed, 1, phi)
    mu = np.empty((1, 1, 200))
    g.gqt_dos_moments(ham, phi, 1, 200, mu)
    assert abs(mu[0, 0, 0] - 1.0) < 1e-12 and np.all(np.abs(mu) <= 1 + 1e-9)
    psi = phi.clone()
    nrm = np.empty(1)
    g.gqt_evolve(ham, psi, 1, w.dt, 1, 0, norm=nrm)
    g.gqt_evolve(ham, psi, 1, w.dt, -1, 0, norm=nrm)
    assert abs(nrm[0] - 1.0) < 1e-12
    assert float((psi - phi).abs().max()) < 1e-13


def test_forward_then_backward_evolution_on_one_handle():
    """U(-dt) U(+dt) phi = phi with both calls on one handle (distinct cached graphs)."""
    lat = S.honeycomb(40, 30, -2.7, 2.0, seed=8)
    dE = S.energy_scale_rule(3, -2.7, 2.0)
    ham = g.gqt_build_hamiltonian(lat, dE)
    phi = torch.from_numpy(S.random_phase(lat.n, 2, seed=9)).cuda()
    psi = phi.clone()
    for _ in range(2):  # the second round replays both graphs
        g.gqt_evolve(ham, psi, 2, 0.74, 1)
        g.gqt_evolve(ham, psi, 2, 0.74, -1)
    assert float((psi - phi).abs().max()) < 1e-13


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("name", ["chain", "honeycomb", "square", "cubic_fp32"])
def test_moment_kernel_variants_agree_with_oracle(variant, name):
    """Chunk-ordered and wavefront-ordered (one or two elements per thread) moment
    kernels: DOS (l = r) and VAC-type (Re <l|T|r>) moments equal the oracle's."""
    if name == "chain":
        lat, dE, prec = S.chain(3001, -1.0, 4.0, seed=2), 4.2, g.GQT_FP64
    elif name == "honeycomb":
        lat, dE, prec = S.honeycomb(45, 31, -2.7, 1.0, seed=3), S.energy_scale_rule(3, -2.7, 1.0), g.GQT_FP64
    elif name == "square":
        lat, dE, prec = S.with_random_bond_phases(S.square(33, 29, -1.0, 2.0, seed=4), 5), 5.2, g.GQT_FP64
    else:
        lat, dE, prec = S.cubic(15, -1.0, 16.5, seed=6), S.energy_scale_rule(6, -1.0, 16.5), g.GQT_FP32_ACC64
    ham = g.gqt_build_hamiltonian(lat, dE, prec)
    g.gqt_set_variant(ham, variant)
    R = 4
    ph = S.random_phase(lat.n, R, seed=8)
    cd = torch.complex128 if prec == g.GQT_FP64 else torch.complex64
    d = torch.from_numpy(ph).to(cd).cuda()
    M = 97
    mu = np.empty((1, R, M))
    g.gqt_dos_moments(ham, d, R, M, mu)
    h = O.Hamiltonian(lat, dE)
    tol = 1e-10 if prec == g.GQT_FP64 else 2e-5
    for r in (0, 3):
        assert nerr(mu[0, r], h.dos_moments(ph[:, r], M)) < tol
    # VAC row 0: Re <V phi | T_n | V phi>
    vac = _vac(ham, d, np.array([0.5]), M, [O.np_rule(dE * 0.5, 64)])
    for r in (0, 3):
        ref = h.vac_moments(ph[:, r], np.array([0.5]), [O.np_rule(dE * 0.5, 64)], M)[0]
        assert nerr(vac[0, 0, r], ref) < (1e-10 if prec == g.GQT_FP64 else 1e-4)


@pytest.mark.parametrize("name", ["honeycomb32x32", "honeycomb_phases_ragged", "chain", "cubic_fp32"])
def test_cluster_resident_rows_match_oracle(name):
    """Small systems run each moment row as one launch on a thread-block cluster
    (vectors in distributed shared memory); DOS (l = r) and VAC rows equal the
    oracle's, and equal the per-order path (cluster rows switched off)."""
    if name == "honeycomb32x32":
        lat, dE, prec = S.honeycomb(32, 32, -2.7, 1.0, seed=3), S.energy_scale_rule(3, -2.7, 1.0), g.GQT_FP64
    elif name == "honeycomb_phases_ragged":
        lat = S.with_random_bond_phases(S.honeycomb(23, 17, -2.7, 2.0, seed=4), 5)
        dE, prec = S.energy_scale_rule(3, -2.7, 2.0), g.GQT_FP64
    elif name == "chain":
        lat, dE, prec = S.chain(9001, -1.0, 4.0, seed=5), 4.2, g.GQT_FP64
    else:
        lat, dE, prec = S.cubic(12, -1.0, 16.5, seed=6), S.energy_scale_rule(6, -1.0, 16.5), g.GQT_FP32_ACC64
    ham = g.gqt_build_hamiltonian(lat, dE, prec)
    phi = S.random_phase(lat.n, 1, seed=9)
    cd = torch.complex128 if prec == g.GQT_FP64 else torch.complex64
    d = torch.from_numpy(phi).to(cd).cuda()
    M = 257
    h = O.Hamiltonian(lat, dE)
    tol = 1e-10 if prec == g.GQT_FP64 else 2e-5
    Np = [O.np_rule(dE * 0.6, 64)]
    got = {}
    for cl in (True, False):
        g.gqt_set_cluster(ham, cl)
        mu = np.empty((1, 1, M))
        g.gqt_dos_moments(ham, d, 1, M, mu)
        vac = _vac(ham, d, np.array([0.6]), M, Np)
        got[cl] = (mu.reshape(M), vac.reshape(M))
        assert nerr(got[cl][0], h.dos_moments(phi[:, 0], M)) < tol
        assert nerr(got[cl][1], h.vac_moments(phi[:, 0], np.array([0.6]), Np, M)[0]) < (tol if tol < 1e-9 else 1e-4)
    assert nerr(got[True][0], got[False][0]) < tol and nerr(got[True][1], got[False][1]) < tol


def test_update_hamiltonian_equals_fresh_build():
    """New values through gqt_update_hamiltonian give the same moments as a fresh build,
    and replayed graphs see the new values; a non-Hermitian update is rejected."""
    lat1 = S.honeycomb(30, 20, -2.7, 1.0, seed=1)
    lat2 = S.honeycomb(30, 20, -2.7, 2.0, seed=2)
    lat2.hop[:] *= 1.1
    dE = S.energy_scale_rule(3, -2.97, 2.0)
    phi = torch.from_numpy(S.random_phase(lat1.n, 1, seed=3)).cuda()
    ham = g.gqt_build_hamiltonian(lat1, dE)
    M = 100
    mu1 = np.empty((1, 1, M))
    g.gqt_dos_moments(ham, phi, 1, M, mu1)
    g.gqt_update_hamiltonian(ham, lat2.onsite, lat2.hop)
    mu2 = np.empty((1, 1, M))
    g.gqt_dos_moments(ham, phi, 1, M, mu2)  # same graph key, new H values
    fresh = g.gqt_build_hamiltonian(lat2, dE)
    ref = np.empty((1, 1, M))
    g.gqt_dos_moments(fresh, phi, 1, M, ref)
    assert np.max(np.abs(mu2 - ref)) < 1e-13 and np.max(np.abs(mu1 - ref)) > 1e-3
    bad = lat2.hop.copy()
    bad[5, 1] += 0.3
    with pytest.raises(g.GqtError) as e:
        g.gqt_update_hamiltonian(ham, lat2.onsite, bad)
    assert e.value.status == g.GQT_EINVAL


@pytest.mark.parametrize("name,R", [("cubic", 32), ("cubic", 16), ("honeycomb_phases", 8), ("honeycomb_phases", 16),
                                    ("ragged_cubic", 32), ("ragged_honeycomb", 16)])
def test_fp32_multivector_prefetch_matches_oracle(name, R):
    """FP32 multi-vector moment kernels whose lane group per site holds at least K + 1
    lanes fetch the next site's indices, hoppings and diagonal one iteration ahead and
    share them by shuffles.  DOS (l = r, two moments per order) and VAC rows equal
    the oracle's for sampled vectors, including segments whose ends fall inside a
    warp (odd site counts) and complex hoppings."""
    if name == "cubic":
        lat, dE = S.cubic(13, -1.0, 16.5, seed=6), S.energy_scale_rule(6, -1.0, 16.5)
        parts = [lat]
    elif name == "honeycomb_phases":
        lat = S.with_random_bond_phases(S.honeycomb(23, 17, -2.7, 2.0, seed=4), 5)
        dE, parts = S.energy_scale_rule(3, -2.7, 2.0), [lat]
    elif name == "ragged_cubic":
        parts = [S.cubic(L, -1.0, 16.5, seed=40 + q) for q, L in enumerate((5, 7, 3, 6))]
        lat, dE = S.block_diagonal(parts), S.energy_scale_rule(6, -1.0, 16.5)
    else:
        parts = [S.honeycomb(a, b, -2.7, 1.0, seed=50 + q) for q, (a, b) in enumerate(((5, 3), (9, 7), (4, 4)))]
        lat, dE = S.block_diagonal(parts), S.energy_scale_rule(3, -2.7, 1.0)
    ham = g.gqt_build_hamiltonian(lat, dE, g.GQT_FP32_ACC64)
    assert ham.nseg == len(parts)
    ph = S.random_phase(lat.n, R, seed=12)
    if len(parts) > 1:  # unit norm per segment
        for q, p in enumerate(parts):
            o = lat.seg_offsets[q]
            ph[o:o + p.n] *= np.sqrt(lat.n / p.n)
    d = torch.from_numpy(ph).to(torch.complex64).cuda()
    M = 97
    mu = np.empty((len(parts), R, M))
    g.gqt_dos_moments(ham, d, R, M, mu)
    dts = np.array([0.5])
    Np = [O.np_rule(dE * 0.5, 64)]
    vac = _vac(ham, d, dts, M, Np)
    for q, p in enumerate(parts):
        o = 0 if len(parts) == 1 else lat.seg_offsets[q]
        h = O.Hamiltonian(p, dE)
        for r in (0, R // 2 - 1, R - 1):
            seg = ph[o:o + p.n, r]
            assert nerr(mu[q, r], h.dos_moments(seg, M)) < 2e-5
            assert nerr(vac[0, q, r], h.vac_moments(seg, dts, Np, M)[0]) < 1e-4


@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("name,R", [("cubic", 4), ("cubic", 32), ("honeycomb_phases", 8), ("ragged_honeycomb", 16)])
def test_fp64_multivector_tiles_match_oracle(name, R, variant):
    """FP64 storage with 128-thread CTAs runs the multi-vector kernels (two or four
    vectors per lane, interleaved across the site's lane group): DOS and VAC rows
    equal the oracle's to FP64 accuracy for every sampled vector."""
    if name == "cubic":
        parts = [S.cubic(11, -1.0, 16.5, seed=7)]
        dE = S.energy_scale_rule(6, -1.0, 16.5)
    elif name == "honeycomb_phases":
        parts = [S.with_random_bond_phases(S.honeycomb(19, 13, -2.7, 2.0, seed=8), 6)]
        dE = S.energy_scale_rule(3, -2.7, 2.0)
    else:
        parts = [S.honeycomb(a, b, -2.7, 1.0, seed=60 + q) for q, (a, b) in enumerate(((7, 3), (5, 9), (4, 4)))]
        dE = S.energy_scale_rule(3, -2.7, 1.0)
    lat = parts[0] if len(parts) == 1 else S.block_diagonal(parts)
    ham = g.gqt_build_hamiltonian(lat, dE, g.GQT_FP64)
    g.gqt_set_launch(ham, 128, 0)
    g.gqt_set_variant(ham, variant)
    ph = S.random_phase(lat.n, R, seed=13)
    if len(parts) > 1:
        for q, p in enumerate(parts):
            o = lat.seg_offsets[q]
            ph[o:o + p.n] *= np.sqrt(lat.n / p.n)
    d = torch.from_numpy(ph).cuda()
    M = 89
    mu = np.empty((len(parts), R, M))
    g.gqt_dos_moments(ham, d, R, M, mu)
    dts = np.array([0.4])
    Np = [O.np_rule(dE * 0.4, 64)]
    vac = _vac(ham, d, dts, M, Np)
    for q, p in enumerate(parts):
        o = 0 if len(parts) == 1 else lat.seg_offsets[q]
        h = O.Hamiltonian(p, dE)
        for r in sorted({0, 1, R // 2, R - 1}):
            seg = ph[o:o + p.n, r]
            assert nerr(mu[q, r], h.dos_moments(seg, M)) < 1e-10
            assert nerr(vac[0, q, r], h.vac_moments(seg, dts, Np, M)[0]) < 1e-10


@pytest.mark.parametrize("M", [1, 2, 3, 96, 97])
@pytest.mark.parametrize("name,R", [("honeycomb", 1), ("square_phases", 2), ("chain", 1), ("ragged_honeycomb", 1),
                                    ("cubic_fp32", 1), ("cubic_fp32", 8), ("honeycomb_fp32", 16)])
def test_vac_pair_rows_match_oracle(name, R, M):
    """VAC rows by two recurrences (A_k = T_k l, B_k = T_k r; mu_2k = 2 Re <A_k|B_k> -
    mu_0, mu_2k+1 = 2 Re <A_k|B_k+1> - mu_1) equal the oracle's single-recurrence
    moments and the library's own one-recurrence path, for odd and even M."""
    prec = g.GQT_FP64
    if name == "honeycomb":
        parts, dE = [S.honeycomb(29, 21, -2.7, 1.0, seed=3)], S.energy_scale_rule(3, -2.7, 1.0)
    elif name == "square_phases":
        parts, dE = [S.with_random_bond_phases(S.square(27, 23, -1.0, 2.0, seed=4), 9)], 5.2
    elif name == "chain":
        parts, dE = [S.chain(2999, -1.0, 4.0, seed=2)], 4.2
    elif name == "ragged_honeycomb":
        parts = [S.honeycomb(a, b, -2.7, 1.0, seed=70 + q) for q, (a, b) in enumerate(((7, 3), (11, 9), (4, 4)))]
        dE = S.energy_scale_rule(3, -2.7, 1.0)
    elif name == "honeycomb_fp32":  # multi-vector form with the next-site prefetch (G = 8 lanes per site)
        parts = [S.with_random_bond_phases(S.honeycomb(17, 13, -2.7, 1.0, seed=5), 2)]
        dE, prec = S.energy_scale_rule(3, -2.7, 1.0), g.GQT_FP32_ACC64
    else:
        parts, dE, prec = [S.cubic(13, -1.0, 16.5, seed=6)], S.energy_scale_rule(6, -1.0, 16.5), g.GQT_FP32_ACC64
    lat = parts[0] if len(parts) == 1 else S.block_diagonal(parts)
    ham = g.gqt_build_hamiltonian(lat, dE, prec)
    g.gqt_set_cluster(ham, False)
    ph = S.random_phase(lat.n, R, seed=14)
    if len(parts) > 1:
        for q, p in enumerate(parts):
            o = lat.seg_offsets[q]
            ph[o:o + p.n] *= np.sqrt(lat.n / p.n)
    d = torch.from_numpy(ph).to(torch.complex128 if prec == g.GQT_FP64 else torch.complex64).cuda()
    dts = np.array([0.45, 0.3])
    Np = [O.np_rule(dE * x, 64) for x in dts]
    got = {}
    for pair in (True, False):
        g.gqt_set_vac_pair(ham, pair)
        got[pair] = _vac(ham, d, dts, M, Np)
    tol = 1e-10 if prec == g.GQT_FP64 else 1e-4
    for q, p in enumerate(parts):
        o = 0 if len(parts) == 1 else lat.seg_offsets[q]
        h = O.Hamiltonian(p, dE)
        for r in sorted({0, R // 2, R - 1}):
            ref = h.vac_moments(ph[o:o + p.n, r], dts, Np, M)
            for k in range(len(dts)):
                assert nerr(got[True][k, q, r], ref[k]) < tol
                assert nerr(got[False][k, q, r], ref[k]) < tol
    if prec == g.GQT_FP64:
        assert nerr(got[True], got[False]) < 1e-12


@pytest.mark.parametrize("R,prec", [(32, "fp32"), (16, "fp32"), (8, "fp64")])
def test_blocked_sweep_order_cubic(R, prec):
    """Built-in simple-cubic lattice with a power-of-two side (L = 64): the
    multi-vector kernels walk the sites strip by strip (32 y-rows through all z).
    DOS and VAC moments equal the natural order (up to the summation order of the
    dots) and, for sampled vectors, the oracle on the same lattice."""
    L = 64
    p = g.GQT_FP32_ACC64 if prec == "fp32" else g.GQT_FP64
    dE = S.energy_scale_rule(6, -1.0, 16.5)
    ham = g.gqt_build_hamiltonian(None, dE, p, kind=g.GQT_LATTICE_CUBIC, L1=L, t=-1.0, W=16.5, seed=17)
    if prec == "fp64":
        g.gqt_set_launch(ham, 128, 0)  # the multi-vector kernels
    cd = torch.complex64 if prec == "fp32" else torch.complex128
    phi = torch.empty((ham.n, R), dtype=cd, device="cuda")
    g.gqt_random_phase(ham, 5, R, phi)
    M = 40
    dts = np.array([0.4])
    Np = [O.np_rule(dE * 0.4, 64)]
    got = {}
    for order in (True, False):
        g.gqt_set_sweep_order(ham, order)
        mu = np.empty((1, R, M))
        g.gqt_dos_moments(ham, phi, R, M, mu)
        got[order] = (mu, _vac(ham, phi, dts, M, Np))
    tol_same = 1e-5 if prec == "fp32" else 1e-13
    assert nerr(got[True][0], got[False][0]) < tol_same
    assert nerr(got[True][1], got[False][1]) < tol_same
    lat = S.cubic(L, -1.0, 16.5, seed=17)
    h = O.Hamiltonian(lat, dE)
    ph = phi.cpu().numpy().astype(np.complex128)
    tol = 2e-5 if prec == "fp32" else 1e-10
    for r in (0, R - 1):
        assert nerr(got[True][0][0, r], h.dos_moments(ph[:, r], M)) < tol
        assert nerr(got[True][1][0, 0, r], h.vac_moments(ph[:, r], dts, Np, M)[0]) < (1e-4 if prec == "fp32" else 1e-10)
