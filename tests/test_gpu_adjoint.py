"""Reverse-mode gradients on the GPU (gqt_vac_loss_grad and the autograd Function)
against the serial FP64 oracle's adjoint (itself pinned by finite differences and
Daleckii-Krein in test_oracle_pins.py) and against central finite differences."""
import numpy as np
import pytest

import gqt_synth as S
import oracle as O

torch = pytest.importorskip("torch")
g = pytest.importorskip("paper_1705_01387_gb300")
from paper_1705_01387_gb300 import autograd as AG  # noqa: E402

pytestmark = pytest.mark.gpu


def nerr(x, y):
    return float(np.max(np.abs(np.asarray(x) - np.asarray(y))) / max(float(np.max(np.abs(y))), 1e-300))


def _run(lat, dE, phi, dts, M, beta, stride=0, prec=None):
    ham = g.gqt_build_hamiltonian(lat, dE, g.GQT_FP64 if prec is None else prec)
    Np = [O.np_rule(dE * d, 64) for d in dts]
    cd = torch.complex128 if prec in (None, g.GQT_FP64) else torch.complex64
    d = torch.from_numpy(phi.reshape(-1, 1)).to(cd).cuda()
    ge = torch.empty(lat.n, dtype=torch.float64, device="cuda")
    gs = torch.empty((lat.n, lat.max_nb, 2), dtype=torch.float64, device="cuda")
    J = g.gqt_vac_loss_grad(ham, d, dts, M, beta, ge, gs, Np=Np, stride=stride)
    gsn = gs.cpu().numpy()
    return J, ge.cpu().numpy(), gsn[..., 0] + 1j * gsn[..., 1], Np


@pytest.mark.parametrize("stride", [0, 3, 7, 1000])
@pytest.mark.parametrize("phases", [False, True])
def test_adjoint_matches_oracle(stride, phases):
    lat = S.honeycomb(7, 5, -2.7, 2.0, seed=19)
    if phases:
        lat = S.with_random_bond_phases(lat, 20)
    dE = S.energy_scale_rule(3, -2.7, 2.0)
    phi = S.random_phase(lat.n, 1, seed=40)[:, 0]
    dts = np.array([0.6, 0.4, 0.5])
    M = 40
    rng = np.random.default_rng(1)
    beta = rng.standard_normal((3, M))
    J, ge, gs, Np = _run(lat, dE, phi, dts, M, beta, stride)
    Jr, ger, gsr = O.Hamiltonian(lat, dE).vac_loss_grad(phi, dts, Np, beta)
    assert abs(J - Jr) <= 1e-10 * abs(Jr)
    assert nerr(ge, ger) < 1e-10
    assert nerr(gs, gsr) < 1e-10


def test_adjoint_fp32_storage_error():
    lat = S.honeycomb(12, 10, -2.7, 2.0, seed=3)
    dE = S.energy_scale_rule(3, -2.7, 2.0)
    phi = S.random_phase(lat.n, 1, seed=4)[:, 0]
    dts = np.array([0.7, 0.7])
    M = 64
    beta = np.cos(0.1 * np.arange(M))[None, :] * np.array([[1.0], [0.5]])
    J, ge, gs, Np = _run(lat, dE, phi, dts, M, beta, prec=g.GQT_FP32_ACC64)
    Jr, ger, gsr = O.Hamiltonian(lat, dE).vac_loss_grad(phi, dts, Np, beta)
    assert abs(J - Jr) <= 1e-4 * abs(Jr)
    assert nerr(ge, ger) < 1e-3 and nerr(gs, gsr) < 1e-3


def _spec(lat, dE, K, M, E, w, seed=7):
    topo = AG.BondTopology.from_lattice(lat)
    phi = torch.from_numpy(S.random_phase(lat.n, 1, seed=seed)).cuda()
    return topo, AG.VacSigmaLossSpec(topo, dE, phi, np.full(K, 2.0 / 2.7), M, torch.from_numpy(E).cuda(),
                                     torch.from_numpy(w).cuda())


def _oracle_loss(lat, dE, spec):
    phi = spec.phi.cpu().numpy()[:, 0]
    dts = np.concatenate([spec.dt, [spec.dt[-1]]])
    Np = [O.np_rule(dE * d, 64) for d in dts]
    vac = O.Hamiltonian(lat, dE).vac_moments(phi, dts, Np, spec.M)
    rho = O.kpm_reconstruct(vac, spec.E.cpu().numpy(), dE, lat.n / lat.volume)
    sig = O.sigma_vac(rho, dts)
    return float(np.sum(spec.w.cpu().numpy() * sig[-1]))


def test_autograd_loss_and_fd():
    """sum_E w(E) sigma_VAC(E, t_K): loss equals the oracle pipeline (moments ->
    reconstruction -> trapezoid) and the autograd gradient matches central differences."""
    lat = S.honeycomb(10, 8, -2.7, 2.0, seed=5)
    dE = S.energy_scale_rule(3, -2.7, 2.0)
    E = np.linspace(-2, 2, 64)
    w = np.exp(-E ** 2 / (2 * 0.5 ** 2))
    topo, spec = _spec(lat, dE, 4, 96, E, w)
    onsite = torch.from_numpy(lat.onsite.copy()).requires_grad_(True)
    hop = torch.full((topo.nbonds,), -2.7, dtype=torch.float64, requires_grad=True)
    L = AG.GqtVacSigmaLoss.apply(onsite, hop, spec)
    L.backward()
    assert abs(float(L) - _oracle_loss(lat, dE, spec)) <= 1e-9 * abs(float(L))
    h = 1e-6
    rng = np.random.default_rng(3)
    for which, vec, grad in (("on", onsite, onsite.grad), ("hop", hop, hop.grad)):
        for q in rng.choice(vec.numel(), 4, replace=False):
            vals = []
            for sgn in (1, -1):
                v = vec.detach().clone()
                v[q] += sgn * h
                args = (v, hop.detach()) if which == "on" else (onsite.detach(), v)
                vals.append(float(AG.GqtVacSigmaLoss.apply(*args, spec)))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - float(grad[q])) <= 1e-6 * max(abs(fd), 1e-3 * float(grad.abs().max()))


@pytest.mark.slow
def test_differentiation_workload_full_size():
    """Honeycomb 256 x 256 (N = 131072), M = 1024, sigma_VAC at t = 50 steps of 2 hbar/|t|
    on 64 energies in [-2, 2] with Gaussian weights: adjoint vs central differences
    (h = 1e-6) on random on-site and bond coordinates."""
    w5 = S.config(4)
    lat = S.build_lattice(w5.lattice_args, w5.seed)
    dE = w5.energy_scale
    E = w5.energies
    wts = np.exp(-E ** 2 / (2 * 0.5 ** 2))
    topo, spec = _spec(lat, dE, w5.n_steps - 1, w5.M, E, wts, seed=w5.seed)
    onsite = torch.from_numpy(lat.onsite.copy()).requires_grad_(True)
    hop = torch.full((topo.nbonds,), -2.7, dtype=torch.float64, requires_grad=True)
    L = AG.GqtVacSigmaLoss.apply(onsite, hop, spec)
    L.backward()
    gmax = max(float(onsite.grad.abs().max()), float(hop.grad.abs().max()))
    h = 1e-6
    rng = np.random.default_rng(11)
    for which, vec, grad in (("on", onsite, onsite.grad), ("hop", hop, hop.grad)):
        for q in rng.choice(vec.numel(), 2, replace=False):
            vals = []
            for sgn in (1, -1):
                v = vec.detach().clone()
                v[q] += sgn * h
                args = (v, hop.detach()) if which == "on" else (onsite.detach(), v)
                vals.append(float(AG.GqtVacSigmaLoss.apply(*args, spec)))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - float(grad[q])) <= 1e-4 * gmax


def test_sigma_vac_loss_weights_linear_form():
    """beta of gqt_sigma_vac_loss_weights turns moments into the loss: for any moments
    mu [K+1][M], sum beta*mu equals sum_E w(E) sigma_VAC(E, t_K) from the oracle's KPM
    reconstruction (Eqs. 26, 31) and trapezoid rule (Eq. 2), with unequal steps."""
    K, M, dE, n_over_omega = 4, 57, 9.3, 0.37
    rng = np.random.default_rng(5)
    mu = rng.standard_normal((K + 1, M)) / (1 + np.arange(M))
    dt = np.array([0.3, 0.7, 0.45, 1.1])
    E = np.linspace(-0.9 * dE, 0.85 * dE, 23)
    w = rng.standard_normal(E.size)
    beta = torch.empty((K + 1, M), dtype=torch.float64, device="cuda")
    g.gqt_sigma_vac_loss_weights(M, torch.from_numpy(E).cuda(), torch.from_numpy(w).cuda(), dE, n_over_omega, dt,
                                 beta)
    got = float(np.sum(beta.cpu().numpy() * mu))
    sig = O.sigma_vac(O.kpm_reconstruct(mu, E, dE, n_over_omega), np.concatenate([dt, [0.0]]))
    want = float(np.sum(w * sig[-1]))
    assert abs(got - want) <= 1e-12 * max(abs(want), float(np.sum(np.abs(w * sig[-1]))))


def test_bond_gradients_gather():
    """Bond gradients are the Hermitian-pair sums of slot gradients; an index outside the
    slot array gives NaN for that bond and leaves the others alone."""
    lat = S.with_random_bond_phases(S.honeycomb(6, 4, -2.7, 2.0, seed=2), 3)
    topo = AG.BondTopology.from_lattice(lat)
    rng = np.random.default_rng(8)
    gs = rng.standard_normal((lat.n, lat.max_nb, 2))
    ia, ib = topo.slot_a.copy(), topo.slot_b.copy()
    ia[5] = lat.n * lat.max_nb  # one past the end
    ib[9] = -1
    gre = torch.empty(topo.nbonds, dtype=torch.float64, device="cuda")
    gim = torch.empty_like(gre)
    g.gqt_bond_gradients(torch.from_numpy(gs).cuda(), torch.from_numpy(ia).cuda(), torch.from_numpy(ib).cuda(), gre,
                         gim)
    gre, gim = gre.cpu().numpy(), gim.cpu().numpy()
    flat = gs.reshape(-1, 2)
    ok = np.ones(topo.nbonds, bool)
    ok[[5, 9]] = False
    assert np.isnan(gre[~ok]).all() and np.isnan(gim[~ok]).all()
    assert np.array_equal(gre[ok], (flat[ia[ok], 0] + flat[ib[ok], 0]))
    assert np.array_equal(gim[ok], (flat[ia[ok], 1] - flat[ib[ok], 1]))
