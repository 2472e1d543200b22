"""Pins of the serial FP64 oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: references come from exact
diagonalisation (numpy eigh on dense matrices built in tests/dense.py),
closed forms (clean periodic graphene and chains), scipy's Bessel functions,
invariants (norm conservation, reversibility, [V,H] = 0 ballistic motion),
the paper's own printed example (cumulative times, tests/golden/) and central
finite differences of the forward oracle for the reverse-mode gradients.
"""
import math
import os

import numpy as np
import pytest
import scipy.special as sp

import gqt_synth as S
import oracle as O
from tests import dense as D

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _model(kind="honeycomb", phases=False, W=1.0, seed=11):
    if kind == "honeycomb":
        lat = S.honeycomb(5, 4, -2.7, W, seed=seed)
        dE = S.energy_scale_rule(3, -2.7, W)
    elif kind == "square":
        lat = S.square(6, 5, -1.0, W, seed=seed)
        dE = S.energy_scale_rule(4, -1.0, W)
    elif kind == "chain":
        lat = S.chain(37, -1.0, W, seed=seed)
        dE = S.energy_scale_rule(2, -1.0, W)
    elif kind == "cubic":
        lat = S.cubic(4, -1.0, W, seed=seed)
        dE = S.energy_scale_rule(6, -1.0, W)
    else:
        raise ValueError(kind)
    if phases:
        lat = S.with_random_bond_phases(lat, seed + 1)
    return lat, dE


MODELS = [("honeycomb", False), ("honeycomb", True), ("square", True), ("chain", False), ("cubic", False)]


@pytest.mark.parametrize("kind,phases", MODELS)
def test_dos_moments_match_exact_diagonalisation(kind, phases):
    """Eq. 28: <phi|T_n(H~)|phi> = sum_a |<a|phi>|^2 cos(n arccos lambda_a)."""
    lat, dE = _model(kind, phases)
    h = O.Hamiltonian(lat, dE)
    phi = S.random_phase(lat.n, 1, seed=5)[:, 0]
    M = 96
    lam, Q = D.eig(D.dense_h(lat, dE))
    assert lam.min() > -1 and lam.max() < 1  # Delta E rule keeps the spectrum inside [-1, 1] (Eq. 19)
    w = np.abs(Q.conj().T @ phi) ** 2
    ref = np.array([np.sum(w * D.cheb_T(n, lam)) for n in range(M)])
    got = h.dos_moments(phi, M)
    assert np.max(np.abs(got - ref)) < 1e-13


def test_general_moments_l_neq_r():
    lat, dE = _model("square", True)
    h = O.Hamiltonian(lat, dE)
    phis = S.random_phase(lat.n, 2, seed=9)
    l, r = phis[:, 0], phis[:, 1]
    lam, Q = D.eig(D.dense_h(lat, dE))
    M = 50
    ref = np.array([l.conj() @ D.fun_of_h(lam, Q, lambda x: D.cheb_T(n, x)) @ r for n in range(M)])
    assert np.max(np.abs(h.cheb_moments(l, r, M) - ref)) < 1e-13


def test_clean_graphene_closed_form():
    """Clean periodic graphene: <A|T_n(H~)|A> = (1/2 L1 L2) sum_k sum_pm T_n(+-|f(k)|/dE),
    f(k) = t (1 + e^{i(k1-k2)} + e^{-i k2}) for the bond set A(c) -> B(c), B(c+a1-a2), B(c-a2)."""
    L1, L2, t = 12, 9, -2.7
    lat = S.honeycomb(L1, L2, t, 0.0)
    dE = S.energy_scale_rule(3, t, 0.0)
    h = O.Hamiltonian(lat, dE)
    k1 = 2 * np.pi * np.arange(L1)[:, None] / L1
    k2 = 2 * np.pi * np.arange(L2)[None, :] / L2
    f = np.abs(t * (1 + np.exp(1j * (k1 - k2)) + np.exp(-1j * k2))).ravel() / dE
    M = 200
    ref = np.array([0.5 * np.mean(D.cheb_T(n, f) + D.cheb_T(n, -f)) for n in range(M)])
    for site in (0, 1, 2 * (3 + L1 * 4) + 1):
        e = np.zeros(lat.n, np.complex128)
        e[site] = 1.0
        assert np.max(np.abs(h.dos_moments(e, M) - ref)) < 1e-13


def test_constant_diagonal_closed_form():
    """H = c I (all hoppings 0): <phi|T_n(H~)|phi> = cos(n arccos(c/dE)) for unit phi."""
    lat = S.chain(31, 0.0, 0.0)
    lat.onsite[:] = 1.7
    dE = 4.0
    h = O.Hamiltonian(lat, dE)
    phi = S.random_phase(lat.n, 1, seed=2)[:, 0]
    n = np.arange(300)
    assert np.max(np.abs(h.dos_moments(phi, 300) - np.cos(n * np.arccos(1.7 / 4.0)))) < 1e-12


def test_moments_bounded_by_norm():
    lat, dE = _model("cubic", W=3.0)
    h = O.Hamiltonian(lat, dE)
    phi = S.random_phase(lat.n, 1, seed=3)[:, 0]
    assert np.all(np.abs(h.dos_moments(phi, 400)) <= 1.0 + 1e-12)


def test_stochastic_trace_converges_to_exact_trace():
    """Eq. 13: the random-phase average approaches Tr T_n / N with error ~ 1/sqrt(N R)."""
    lat = S.honeycomb(8, 8, -2.7, 1.0, seed=4)
    dE = S.energy_scale_rule(3, -2.7, 1.0)
    h = O.Hamiltonian(lat, dE)
    lam, _ = D.eig(D.dense_h(lat, dE))
    M, R = 40, 48
    exact = np.array([np.mean(D.cheb_T(n, lam)) for n in range(M)])
    phis = S.random_phase(lat.n, R, seed=21)
    est = np.mean([h.dos_moments(phis[:, r], M) for r in range(R)], axis=0)
    assert np.max(np.abs(est - exact)) < 5.0 / math.sqrt(lat.n * R)


def test_bessel_against_scipy_and_identity():
    for x in (0.3, 3.344, 7.08, 25.0):
        J = O.bessel(x, 80)
        assert np.max(np.abs(J - sp.jv(np.arange(80), x))) < 1e-14
        assert abs(J[0] + 2 * J[2::2].sum() - 1.0) < 1e-14  # J_0 + 2 sum J_2k = 1


def test_np_rule_values():
    """N_p = 1 + max{m: |J_m(x)| >= 1e-15} (capped at 64), evaluated independently with scipy."""
    for x in (9.03 / 2.7, 9.555 * 2 / 2.7, 8.7675 * 2 / 2.7, 0.5, 12.0):
        m = np.arange(200)
        ref = min(1 + int(np.max(m[np.abs(sp.jv(m, x)) >= 1e-15])), 64)
        assert O.np_rule(x, 64) == ref
    assert O.np_rule(9.03 / 2.7, 64) == 21
    assert O.np_rule(9.555 * 2 / 2.7, 64) == 29
    assert O.np_rule(8.7675 * 2 / 2.7, 64) == 28


@pytest.mark.parametrize("x", [41.0, 410.0])
def test_long_expansions_bessel_and_np_rule(x):
    """The long steps of the paper's localized example (Sec. 5, dt up to 100 with
    dE = 4.1, i.e. x = dE dt up to 410 and N_p = 487 Bessel orders, Eq. 17): the
    oracle's J_m(x) against scipy for every order used, the sum rule
    J_0 + 2 sum J_2k = 1, and N_p = 1 + max{m: |J_m(x)| >= 1e-15} without the cap."""
    m = np.arange(1200)
    ref_np = 1 + int(np.max(m[np.abs(sp.jv(m, x)) >= 1e-15]))
    assert O.np_rule(x, 4096) == ref_np
    J = O.bessel(x, ref_np)
    assert np.max(np.abs(J - sp.jv(np.arange(ref_np), x))) < 5e-14
    assert abs(J[0] + 2 * J[2::2].sum() - 1.0) < 5e-14
    if x == 410.0:
        assert ref_np == 487  # the paper's longest step, dt = 100 at dE = 4.1


@pytest.mark.parametrize("x", [41.0, 410.0])
def test_long_evolution_matches_matrix_exponential(x):
    """Eq. 17 and Eqs. 18, 22, 24 with hundreds of Bessel orders (the localized
    example's steps) on a disordered chain, against exp(-i x H~) and the
    Daleckii-Krein [X, U] from the eigendecomposition."""
    lat = S.chain(61, -1.0, 4.0, seed=21)
    dE = 4.1
    h = O.Hamiltonian(lat, dE)
    psi = S.random_phase(lat.n, 1, seed=22)[:, 0]
    dt = x / dE
    Np = O.np_rule(x, 4096)
    lam, Q = D.eig(D.dense_h(lat, dE))
    for sign in (+1, -1):
        U = D.fun_of_h(lam, Q, lambda l: np.exp(-1j * sign * l * x))
        got = h.evolve(psi, dt, sign, Np)
        assert np.max(np.abs(got - U @ psi)) < 1e-12
        assert abs(np.linalg.norm(got) - 1.0) < 1e-12
    XU = D.frechet(lam, Q, lambda l: np.exp(-1j * l * x), lambda l: -1j * x * np.exp(-1j * l * x),
                   D.dense_xh(lat, dE))
    ref = XU @ psi
    got = h.commutator_evolve(psi, dt, Np)
    assert np.max(np.abs(got - ref)) < 1e-11 * max(1.0, float(np.max(np.abs(ref))))


@pytest.mark.parametrize("kind,phases", MODELS)
@pytest.mark.parametrize("sign", [+1, -1])
def test_evolution_matches_matrix_exponential(kind, phases, sign):
    """Eq. 17 against exp(-+ i H dt) from the eigendecomposition."""
    lat, dE = _model(kind, phases)
    h = O.Hamiltonian(lat, dE)
    psi = S.random_phase(lat.n, 1, seed=8)[:, 0]
    dt = 0.9
    x = dE * dt
    lam, Q = D.eig(D.dense_h(lat, dE))
    U = D.fun_of_h(lam, Q, lambda l: np.exp(-1j * sign * l * x))
    got = h.evolve(psi, dt, sign, O.np_rule(x, 64))
    assert np.max(np.abs(got - U @ psi)) < 1e-13
    assert abs(np.linalg.norm(got) - 1.0) < 1e-13


def test_evolution_is_reversible():
    lat, dE = _model("honeycomb", True)
    h = O.Hamiltonian(lat, dE)
    psi = S.random_phase(lat.n, 1, seed=6)[:, 0]
    Np = O.np_rule(dE * 1.3, 64)
    back = h.evolve(h.evolve(psi, 1.3, +1, Np), 1.3, -1, Np)
    assert np.max(np.abs(back - psi)) < 1e-13


@pytest.mark.parametrize("kind,phases", MODELS)
def test_commutator_matches_daleckii_krein(kind, phases):
    """Eqs. 18, 22, 24 against the Frechet derivative of exp(-i x H~) in the
    direction [X, H~] (Daleckii-Krein), the exact [X, U(dt)] for the slot-defined
    commutator."""
    lat, dE = _model(kind, phases)
    h = O.Hamiltonian(lat, dE)
    psi = S.random_phase(lat.n, 1, seed=12)[:, 0]
    dt = 0.8
    x = dE * dt
    lam, Q = D.eig(D.dense_h(lat, dE))
    XU = D.frechet(lam, Q, lambda l: np.exp(-1j * l * x), lambda l: -1j * x * np.exp(-1j * l * x),
                   D.dense_xh(lat, dE))
    got = h.commutator_evolve(psi, dt, O.np_rule(x, 64))
    assert np.max(np.abs(got - XU @ psi)) < 1e-12


def test_velocity_is_i_commutator():
    """Eq. 34: V = i[H, X] with X diagonal (open chain, where positions exist)."""
    lat = S.chain(9, -1.0, 1.0, seed=3)
    X = np.arange(9, dtype=float)
    # open chain: drop the wrap bonds (0 <-> 8)
    for i in (0, 8):
        for k in range(2):
            if abs(int(lat.nb_idx[i, k]) - i) > 1:
                lat.hop[i, k] = 0.0
    h = O.Hamiltonian(lat, 1.0)
    H = D.dense_h(lat)
    V = 1j * (H @ np.diag(X) - np.diag(X) @ H)
    psi = S.random_phase(9, 1, seed=1)[:, 0]
    assert np.max(np.abs(h.apply_v(psi) - V @ psi)) < 1e-14


def _steps(dE, dts):
    return [O.np_rule(dE * d, 64) for d in dts]


@pytest.mark.parametrize("kind,phases", [("honeycomb", False), ("square", True), ("chain", False)])
def test_vac_moments_match_definition(kind, phases):
    """Eq. 29 at cumulative times t_k = dt_0 + ... + dt_{k-1}, rows t_0 = 0 .. t_{Nt-1}."""
    lat, dE = _model(kind, phases, W=2.0)
    h = O.Hamiltonian(lat, dE)
    phi = S.random_phase(lat.n, 1, seed=14)[:, 0]
    dts = np.array([0.3, 0.5, 0.2, 0.6])
    M = 40
    got = h.vac_moments(phi, dts, _steps(dE, dts), M)
    Ht = D.dense_h(lat, dE)
    lam, Q = D.eig(Ht)
    V = D.dense_v(lat)
    Tn = [D.fun_of_h(lam, Q, lambda x: D.cheb_T(n, x)) for n in range(M)]
    t = np.concatenate([[0.0], np.cumsum(dts)])[: len(dts)]
    for k, tk in enumerate(t):
        U = D.fun_of_h(lam, Q, lambda l: np.exp(-1j * l * dE * tk))
        ref = [np.real(phi.conj() @ U @ V @ Tn[n] @ U.conj().T @ V @ phi) for n in range(M)]
        assert np.max(np.abs(got[k] - ref)) < 1e-12


@pytest.mark.parametrize("kind,phases", [("honeycomb", False), ("square", True), ("chain", False)])
def test_msd_moments_match_definition(kind, phases):
    """Eq. 30 with [X, U(t)] at the cumulative time from Daleckii-Krein; rows t_1 .. t_Nt."""
    lat, dE = _model(kind, phases, W=2.0)
    h = O.Hamiltonian(lat, dE)
    phi = S.random_phase(lat.n, 1, seed=15)[:, 0]
    dts = np.array([0.4, 0.25, 0.7])
    M = 40
    got = h.msd_moments(phi, dts, _steps(dE, dts), M)
    lam, Q = D.eig(D.dense_h(lat, dE))
    Dx = D.dense_xh(lat, dE)
    for k, tk in enumerate(np.cumsum(dts)):
        x = dE * tk
        XU = D.frechet(lam, Q, lambda l: np.exp(-1j * l * x), lambda l: -1j * x * np.exp(-1j * l * x), Dx)
        px = XU @ phi
        ref = [np.real(px.conj() @ D.fun_of_h(lam, Q, lambda y: D.cheb_T(n, y)) @ px) for n in range(M)]
        assert np.max(np.abs(got[k] - ref)) < 1e-12


def test_golden_cumulative_times_and_ballistic_msd():
    """Clean chain: [V, H] = 0, so the VAC moments stay at their t = 0 values and
    the MSD moments are t^2 times them (ballistic motion).  The MSD rows sit at
    the cumulative times of the paper's time-step example (golden file)."""
    steps, cum = [], []
    with open(os.path.join(GOLDEN, "cumulative_times.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                a, b = line.split()
                steps.append(float(a))
                cum.append(float(b))
    t0 = 0.05
    dts = np.array(steps) * t0
    lat = S.chain(41, -1.0, 0.0)
    dE = S.energy_scale_rule(2, -1.0, 0.0)
    h = O.Hamiltonian(lat, dE)
    phi = S.random_phase(lat.n, 1, seed=4)[:, 0]
    M = 30
    Np = _steps(dE, dts)
    vac = h.vac_moments(phi, dts, Np, M)
    msd = h.msd_moments(phi, dts, Np, M)
    assert np.max(np.abs(vac - vac[0][None, :])) < 1e-13
    for k in range(len(dts)):
        assert np.max(np.abs(msd[k] - (np.array(cum[k]) * t0) ** 2 * vac[0])) < 1e-12


def test_vac_time_reversal_real_model():
    """Real H, real phi: Re C^VAC(t) is even in t, so evolving with U(+dt) in place
    of U(-dt) leaves the VAC moments unchanged.  U(+dt) steps are produced by
    conjugating the model's evolution: for real H, U(+dt) psi = conj(U(-dt) conj psi)."""
    lat, dE = _model("honeycomb", False, W=2.0)
    h = O.Hamiltonian(lat, dE)
    phi = np.where(S.uniform(3, 7, lat.n) < 0.5, -1.0, 1.0).astype(np.complex128) / math.sqrt(lat.n)
    dts = np.array([0.5, 0.5, 0.5])
    M = 30
    vac = h.vac_moments(phi, dts, _steps(dE, dts), M)
    # manual U(+dt) version through the oracle's primitives
    a = phi.copy()
    b = h.apply_v(phi)
    for k in range(3):
        l = h.apply_v(a)
        ref = np.real(h.cheb_moments(l, b, M))
        assert np.max(np.abs(ref - vac[k])) < 1e-12
        Np = O.np_rule(dE * dts[k], 64)
        a = h.evolve(a, dts[k], +1, Np)
        b = h.evolve(b, dts[k], +1, Np)


def test_jackson_kernel_properties():
    """Eq. 31: g_0 = 1, 0 <= g_n <= 1 and non-increasing."""
    for M in (10, 512, 3000):
        g = O.jackson(M)
        assert abs(g[0] - 1.0) < 1e-15
        assert np.all(g >= -1e-15) and np.all(g <= 1 + 1e-15) and np.all(np.diff(g) <= 1e-15)


def test_jackson_kernel_autocorrelation_form():
    """Eq. 31 is the closed form of a construction, not a definition of its own: the
    Jackson damping factors are the normalised autocorrelation of the sine window
    a_v = sin(pi (v + 1) / (M + 1)), v = 0..M-1, i.e.
    g_n = sum_{v < M - n} a_v a_{v+n} / sum_v a_v^2 (Weisse et al. 2006, the KPM review the
    paper cites for its kernel).  The window is the optimal one for a positive, minimally
    broadened kernel; evaluating its autocorrelation by direct summation is independent of
    the closed form's trigonometric identities (and of its alpha = 1/(N_m + 1))."""
    for M in (10, 512, 3000):
        v = np.arange(M)
        a = np.sin(np.pi * (v + 1) / (M + 1))
        ref = np.correlate(a, a, mode="full")[M - 1:] / np.dot(a, a)
        assert np.max(np.abs(O.jackson(M) - ref)) < 1e-13


def test_kpm_normalisation_chebyshev_gauss():
    """integral of rho(E) dE = 2 (N/Omega) mu_0: Chebyshev-Gauss quadrature on NE > M nodes is exact."""
    lat, dE = _model("honeycomb", False, W=1.0)
    h = O.Hamiltonian(lat, dE)
    phi = S.random_phase(lat.n, 1, seed=2)[:, 0]
    M, NE = 64, 200
    mu = h.dos_moments(phi, M)
    x = np.cos(np.pi * (np.arange(NE) + 0.5) / NE)
    rho = O.kpm_reconstruct(mu, dE * x, dE, lat.n / lat.volume)[0]
    integral = np.sum(rho * np.sqrt(1 - x ** 2)) * np.pi * dE / NE
    assert abs(integral - 2 * lat.n / lat.volume * mu[0]) < 1e-12


def test_kpm_chain_band_centre():
    """Clean chain DOS (spin 2, per unit length): rho(0) = 2/(pi * 2|t|); Jackson broadening
    of the smooth centre region is O(1/M^2)."""
    L, t = 4001, -1.0
    lat = S.chain(L, t, 0.0)
    dE = 2.05
    h = O.Hamiltonian(lat, dE)
    e = np.zeros(L, np.complex128)
    e[0] = 1.0
    M = 1000
    mu = h.dos_moments(e, M)
    rho = O.kpm_reconstruct(mu, np.array([0.0, 1.0]), dE, L / lat.volume)[0]
    ref = 2.0 / (np.pi * np.sqrt(4 * t * t - np.array([0.0, 1.0]) ** 2))
    assert np.max(np.abs(rho - ref) / ref) < 2e-3
    assert np.isnan(O.kpm_reconstruct(mu[:10], np.array([2.05, -3.0]), dE, 1.0)).all()


def test_kpm_positivity_and_symmetry_bipartite():
    """Jackson damping keeps the DOS of a positive measure non-negative; on a clean
    bipartite lattice the local moments at one site have mu_odd = 0 (odd powers of H
    change sublattice), so the local DOS obeys rho(E) = rho(-E)."""
    lat = S.honeycomb(10, 10, -2.7, 0.0)
    dE = S.energy_scale_rule(3, -2.7, 0.0)
    h = O.Hamiltonian(lat, dE)
    phi = np.zeros(lat.n, np.complex128)
    phi[0] = 1.0
    mu = h.dos_moments(phi, 256)
    assert np.max(np.abs(mu[1::2])) < 1e-14
    E = np.linspace(-8, 8, 321)
    rho = O.kpm_reconstruct(mu, E, dE, lat.n / lat.volume)[0]
    assert rho.min() > -1e-12
    assert np.max(np.abs(rho - rho[::-1])) < 1e-12


def test_sigma_rules():
    """Eq. 2 (trapezoid) and Eq. 5 (finite difference): constant rho C_vv = v gives
    sigma_VAC = v t; rho dX^2 = c t^2 gives sigma_MSD = c t at mid-step."""
    dt = np.array([0.1, 0.2, 0.3, 0.4])
    v = np.full((4, 3), 2.5)
    s = O.sigma_vac(v, dt)
    tv = np.concatenate([[0], np.cumsum(dt)])[:4]
    assert np.allclose(s, 2.5 * tv[:, None], atol=1e-15)
    # rho C_vv linear in t: the trapezoid rule is exact, integral = a t + b t^2 / 2
    lin = (1.5 - 0.7 * tv)[:, None] * np.ones((1, 3))
    assert np.allclose(O.sigma_vac(lin, dt), (1.5 * tv - 0.35 * tv ** 2)[:, None], atol=1e-14)
    tm = np.cumsum(dt)
    m = 3.0 * tm[:, None] ** 2 * np.ones((1, 3))
    sm = O.sigma_msd(m, dt)
    mid = 0.5 * (tm + np.concatenate([[0], tm[:-1]]))
    assert np.allclose(sm, 3.0 * mid[:, None], atol=1e-14)


# ----- reverse-mode gradients (not in the paper; pinned by finite differences and Daleckii-Krein)

def _perturbed(lat, which, i, k, h):
    import copy
    L2 = copy.deepcopy(lat)
    if which == "eps":
        L2.onsite[i] += h
    else:  # Hermitian perturbation of the real part of bond (i,k)
        j = int(lat.nb_idx[i, k])
        kk = [q for q in range(lat.nb_count[j]) if lat.nb_idx[j, q] == i][0]
        L2.hop[i, k] += h
        L2.hop[j, kk] += h
    return L2


def test_cheb_adjoint_matches_daleckii_krein():
    """Gradient of J = Re <l|p(H~)|r>, p = sum coef_m T_m (complex coef): the exact
    derivative is G = Q (P o (Q^+ l r^+ Q)) Q^+ with P the divided differences of p."""
    lat, dE = _model("square", True, W=1.5)
    h = O.Hamiltonian(lat, dE)
    ph = S.random_phase(lat.n, 2, seed=30)
    l, r = ph[:, 0], ph[:, 1]
    M = 25
    coef = np.exp(1j * np.arange(M) * 0.7) / (1.0 + np.arange(M))
    ge, gs, rb = h.cheb_adjoint(l, r, coef)
    lam, Q = D.eig(D.dense_h(lat, dE))

    def p(x):
        return sum(coef[m] * D.cheb_T(m, x) for m in range(M))

    def dp(x):
        th = np.arccos(np.clip(x, -1, 1))
        return sum(coef[m] * m * np.sin(m * th) / np.sin(th) for m in range(1, M))

    # dJ = Re tr(dp r l^+) with dp = Q (P o Q^+ dH~ Q) Q^+; writing dJ = Re sum conj(G_ij) dH~_ij
    # gives G = Q (conj(P) o (Q^+ l r^+ Q)) Q^+.
    F = D.divided_difference(lam, p, dp)
    A = Q.conj().T @ np.outer(l, r.conj()) @ Q  # Q^+ l r^+ Q
    G = Q @ (F.conj() * A) @ Q.conj().T  # sum over a,b of conj(P_ab) ...
    ref_eps = np.real(np.diag(G)) / dE
    assert np.max(np.abs(ge - ref_eps)) < 1e-11
    ref_slot = np.array([[G[i, lat.nb_idx[i, k]] / dE for k in range(lat.max_nb)] for i in range(lat.n)])
    assert np.max(np.abs(gs - ref_slot)) < 1e-11
    # rbar = p(H~)^+ l = Q conj(p(lambda)) Q^+ l
    Pdag = D.fun_of_h(lam, Q, lambda x: np.conj(p(x)))
    assert np.max(np.abs(rb - Pdag @ l)) < 1e-12


def test_vac_loss_gradient_matches_finite_differences():
    """J = sum_k sum_n beta[k,n] C_n^VAC(t_k): adjoint gradient vs central differences
    (h = 1e-6) of the forward oracle for on-site energies and real bond hoppings."""
    lat = S.honeycomb(3, 3, -2.7, 2.0, seed=19)
    dE = S.energy_scale_rule(3, -2.7, 2.0)
    h = O.Hamiltonian(lat, dE)
    phi = S.random_phase(lat.n, 1, seed=40)[:, 0]
    dts = np.array([0.6, 0.4, 0.5])
    Np = _steps(dE, dts)
    M = 20
    beta = np.cos(0.3 * np.arange(M))[None, :] * np.array([1.0, -0.5, 0.8])[:, None]
    J, ge, gs = h.vac_loss_grad(phi, dts, Np, beta)

    def loss(L2):
        return float(np.sum(beta * O.Hamiltonian(L2, dE).vac_moments(phi, dts, Np, M)))

    assert abs(J - loss(lat)) < 1e-13
    eps = 1e-6
    rng = np.random.default_rng(0)
    for i in rng.choice(lat.n, 5, replace=False):
        fd = (loss(_perturbed(lat, "eps", i, 0, eps)) - loss(_perturbed(lat, "eps", i, 0, -eps))) / (2 * eps)
        assert abs(fd - ge[i]) < 1e-7 * max(1.0, abs(fd))
    for i in rng.choice(lat.n, 5, replace=False):
        k = int(rng.integers(3))
        j = int(lat.nb_idx[i, k])
        kk = [q for q in range(3) if lat.nb_idx[j, q] == i][0]
        fd = (loss(_perturbed(lat, "hop", i, k, eps)) - loss(_perturbed(lat, "hop", i, k, -eps))) / (2 * eps)
        an = np.real(gs[i, k] + gs[j, kk])
        assert abs(fd - an) < 1e-7 * max(1.0, abs(fd))


# ---------------------------------------------------------------- Hall (Kubo-Bastin)

def _haldane_small(mass=0.1, W=0.4):
    lat = S.haldane(4, 3, -1.0, 0.2, math.pi / 3, mass, W, seed=21)
    dE = 1.05 * (3 * 1.0 + 6 * 0.2 + abs(mass) + W / 2)
    return lat, dE


@pytest.mark.parametrize("pair", ["xy", "yx", "xx"])
def test_kb_moments_match_exact_trace(pair):
    """Lambda_mn = Tr[v~_a T_m(H~) v~_b T_n(H~)] from the oracle's vector recursions
    with the complete site basis as 'random' vectors equals the eigenbasis
    closed form sum_ab (v_a)_ab T_m(l_b) (v_b)_ba T_n(l_a)."""
    lat, dE = _haldane_small()
    d = {"x": lat.dx, "y": lat.dy}
    da, db = d[pair[0]], d[pair[1]]
    M = 24
    lam = O.Hamiltonian(lat, dE).kb_moments(da, db, np.eye(lat.n), M)
    lamb, Q = D.eig(D.dense_h(lat, dE))
    va = Q.conj().T @ D.dense_vd(lat, da, dE) @ Q
    vb = Q.conj().T @ D.dense_vd(lat, db, dE) @ Q
    T = np.array([D.cheb_T(m, lamb) for m in range(M)])  # [M, N]
    ref = np.einsum("ab,mb,ba,na->mn", va, T, vb, T)
    assert np.max(np.abs(lam - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_kb_moments_vanish_by_mirror_symmetry():
    """Clean square lattice: the mirror x -> -x maps v_x -> -v_x and leaves H and
    v_y unchanged, so the exact trace Lambda^xy vanishes while Lambda^xx does not."""
    lat = S.square(6, 5, -1.0, 0.0)
    dE = 4.2
    h = O.Hamiltonian(lat, dE)
    lxy = h.kb_moments(lat.dx, lat.dy, np.eye(lat.n), 16)
    lxx = h.kb_moments(lat.dx, lat.dx, np.eye(lat.n), 16)
    assert np.max(np.abs(lxx)) > 1.0
    assert np.max(np.abs(lxy)) < 1e-12 * np.max(np.abs(lxx))


def test_kubo_bastin_reconstruction_closed_forms():
    """Single-moment inputs integrate in closed form: Lambda_00 = 1 gives
    F = 2x/(1-x^2)^2 and sigma = (2/Omega)[1/(1-x^2)] from x_0; Lambda_10 = 1
    (no damping) gives F = 2(1+x^2)/(1-x^2)^2 and sigma = (2/Omega)[2x/(1-x^2)],
    and so does Lambda_01 = 1; an imaginary Lambda_10 contributes nothing."""
    M, dE, area = 5, 3.0, 7.5
    E = np.linspace(-0.9 * dE, 0.8 * dE, 20001)
    x = E / dE
    lam = np.zeros((M, M), np.complex128)
    lam[0, 0] = 1.0
    got = O.kubo_bastin(lam, E, dE, area)
    ref = 2.0 / area * (1 / (1 - x ** 2) - 1 / (1 - x[0] ** 2))
    assert np.max(np.abs(got - ref)) < 1e-6 * np.max(np.abs(ref))
    lam[:] = 0.0
    lam[1, 0] = 1.0
    got = O.kubo_bastin(lam, E, dE, area, kernel=1)
    ref = 2.0 / area * (2 * x / (1 - x ** 2) - 2 * x[0] / (1 - x[0] ** 2))
    assert np.max(np.abs(got - ref)) < 1e-6 * np.max(np.abs(ref))
    lam[:] = 0.0
    lam[0, 1] = 1.0  # Gamma_01 = e^{-i th}(x + i sin th) + x^2 = 1 + x^2 as well
    got = O.kubo_bastin(lam, E, dE, area, kernel=1)
    assert np.max(np.abs(got - ref)) < 1e-6 * np.max(np.abs(ref))
    lam[:] = 0.0
    lam[1, 0] = 1j
    assert np.max(np.abs(O.kubo_bastin(lam, E, dE, area, kernel=1))) < 1e-12


@pytest.mark.parametrize("mass,chern", [(0.0, 1.0), (2.0, 0.0)])
def test_kubo_bastin_haldane_chern_plateau(mass, chern):
    """Haldane model (8 x 8 cells, t2 = 0.15, phi = pi/2): in the gap sigma_xy is
    the Chern number (1 in the topological phase, 0 well beyond mass = 3 sqrt3 t2 = 0.78),
    from the eigenstate Kubo (TKNN) sum; the Kubo-Bastin reconstruction from the
    oracle's moments (M = 256, exact trace) agrees within 1e-2."""
    lat = S.haldane(8, 8, -1.0, 0.15, math.pi / 2, mass, 0.0)
    dE = 1.05 * (3.0 + 6 * 0.15 + mass)
    exact = D.tknn_sigma(lat, 0.0, lat.dx, lat.dy)
    assert abs(exact - chern) < 1e-2
    lam = O.Hamiltonian(lat, dE).kb_moments(lat.dx, lat.dy, np.eye(lat.n), 256)
    E = np.linspace(-0.97 * dE, 0.0, 3001)
    sig = O.kubo_bastin(lam, E, dE, lat.volume)
    assert abs(sig[-1] - exact) < 1e-2


def test_kubo_bastin_fermi_limits_and_quadrature():
    """Finite temperature: at kT = 0 on a uniform grid the Fermi-weighted trapezoid
    sum at an interior grid energy mu = E_j equals the zero-temperature integral
    to E_j exactly (the half weight at E = mu splits the last interval evenly); for Lambda_00 = 1,
    F = 2x/(1-x^2)^2 and sigma(mu, T) agrees with an adaptive quadrature of
    (2/Omega) f((dE x - mu)/kT) F(x) (scipy), and rises with mu."""
    from scipy import integrate
    rng = np.random.default_rng(9)
    M, dE, area = 21, 2.5, 4.0
    lam = (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))) / (1 + np.arange(M))[None, :]
    E = np.linspace(-0.9 * dE, 0.9 * dE, 2001)
    zero = O.kubo_bastin(lam, E, dE, area)
    idx = np.array([1, 500, 1000, 1777, 1999])  # interior grid points (an end has one neighbouring interval)
    step = O.kubo_bastin_fermi(lam, E, dE, area, E[idx], 0.0)
    assert np.max(np.abs(step - zero[idx])) <= 1e-12 * np.max(np.abs(zero))
    lam0 = np.zeros((3, 3), np.complex128)
    lam0[0, 0] = 1.0
    E = np.linspace(-0.8 * dE, 0.8 * dE, 40001)
    mus = np.array([-0.6, -0.1, 0.0, 0.3, 1.2])
    kT = 0.05
    got = O.kubo_bastin_fermi(lam0, E, dE, area, mus, kT)
    for q, mu in enumerate(mus):
        f = lambda x: 2.0 / area * 2 * x / (1 - x * x) ** 2 / (1 + np.exp(np.clip((dE * x - mu) / kT, -700, 700)))
        ref, _ = integrate.quad(f, E[0] / dE, E[-1] / dE, points=[mu / dE], limit=400, epsabs=1e-13, epsrel=1e-12)
        assert abs(got[q] - ref) < 1e-6 * (1 + abs(ref))
    assert np.all(np.diff(got[mus > 0]) > 0)  # F > 0 for x > 0: more states filled, larger sigma
