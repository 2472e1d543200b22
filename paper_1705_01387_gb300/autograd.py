"""torch.autograd.Function over the library's adjoint of the VAC moments.

``GqtVacSigmaLoss.apply(onsite, hop, model)`` returns the loss
L = sum_E w(E) sigma_VAC(E, t_K) -- the running conductivity from the velocity
autocorrelation (Eq. 2, trapezoid rule over rows t_0 = 0 .. t_K) reconstructed by
the kernel polynomial method (Eqs. 26, 31) -- and backpropagates to the on-site
energies (onsite [N]) and the real bond hoppings (hop [nbonds]) through the
library's hand-written adjoint (gqt_vac_loss_grad: reverse three-term recurrence
with sqrt(M) checkpointing).  The energy scale dE is held fixed.

Glue only: Hamiltonian assembly from (onsite, hop) is index bookkeeping on the
host; the moment weights come from gqt_sigma_vac_loss_weights, loss and slot
gradients from gqt_vac_loss_grad and bond gradients from gqt_bond_gradients.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import (GQT_FP64, gqt_bond_gradients, gqt_build_hamiltonian, gqt_np_rule, gqt_sigma_vac_loss_weights,
               gqt_update_hamiltonian, gqt_vac_loss_grad)


@dataclasses.dataclass
class BondTopology:
    """Undirected bonds of a Hermitian neighbour list: bond b joins slot (i, k) and its
    reverse slot (j, kk); ``slot_of_bond`` holds the two flat slot indices i*K + k."""
    n: int
    K: int
    nb_count: np.ndarray
    nb_idx: np.ndarray
    dx: np.ndarray
    volume: float
    length_x: float
    slot_a: np.ndarray
    slot_b: np.ndarray

    @property
    def nbonds(self) -> int:
        return int(self.slot_a.size)

    @staticmethod
    def from_lattice(lat) -> "BondTopology":
        n, K = int(lat.n), int(lat.max_nb)
        idx = np.asarray(lat.nb_idx)
        cnt = np.asarray(lat.nb_count)
        used = np.zeros((n, K), dtype=bool)
        a, b = [], []
        for i in range(n):
            for k in range(cnt[i]):
                if used[i, k]:
                    continue
                j = int(idx[i, k])
                rev = [q for q in range(cnt[j]) if idx[j, q] == i and not used[j, q] and (j != i or q != k)]
                if not rev:
                    raise ValueError("neighbour list is not symmetric")
                used[i, k] = used[j, rev[0]] = True
                a.append(i * K + k)
                b.append(j * K + rev[0])
        return BondTopology(n, K, cnt.astype(np.int32), idx.astype(np.int32), np.asarray(lat.dx, np.float64),
                            float(lat.volume), float(lat.length_x), np.array(a, np.int64), np.array(b, np.int64))

    def lattice(self, onsite: np.ndarray, hop_bonds: np.ndarray):
        hop = np.zeros(self.n * self.K, np.complex128)
        hop[self.slot_a] = hop_bonds
        hop[self.slot_b] = hop_bonds
        return _Lat(self.n, self.K, self.nb_count, self.nb_idx, hop.reshape(self.n, self.K), onsite, self.dx,
                    self.length_x, self.volume)


@dataclasses.dataclass
class _Lat:
    n: int
    max_nb: int
    nb_count: np.ndarray
    nb_idx: np.ndarray
    hop: np.ndarray
    onsite: np.ndarray
    dx: np.ndarray
    length_x: float
    volume: float
    seg_offsets: None = None


@dataclasses.dataclass
class VacSigmaLossSpec:
    """What the loss measures: phi (CUDA [N, 1]), time steps (rows t_0 .. t_K with
    K = len(dt)), M moments, energies E and weights w (CUDA float64), dE."""
    topo: BondTopology
    energy_scale: float
    phi: torch.Tensor
    dt: np.ndarray
    M: int
    E: torch.Tensor
    w: torch.Tensor
    precision: int = GQT_FP64
    stride: int = 0
    _ham: object = dataclasses.field(default=None, repr=False)  # handle reused across evaluations
    _beta: object = dataclasses.field(default=None, repr=False)

    def beta(self):
        """beta[k][n] = c_k * sum_E w(E) d rhoC_vv(E, t_k)/d mu_n (trapezoid weights c_k), on the device."""
        dt = np.asarray(self.dt, np.float64)
        b = torch.empty((dt.size + 1, self.M), dtype=torch.float64, device=self.E.device)
        return gqt_sigma_vac_loss_weights(self.M, self.E, self.w, self.energy_scale, self.topo.n / self.topo.volume,
                                          dt, b)


class GqtVacSigmaLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, onsite: torch.Tensor, hop: torch.Tensor, spec: VacSigmaLossSpec):
        lat = spec.topo.lattice(onsite.detach().cpu().numpy().astype(np.float64),
                                hop.detach().cpu().numpy().astype(np.float64))
        if spec._ham is None:
            spec._ham = gqt_build_hamiltonian(lat, spec.energy_scale, spec.precision)
        else:  # same topology: update values in place (keeps workspace and CUDA graphs)
            gqt_update_hamiltonian(spec._ham, lat.onsite, lat.hop)
        ham = spec._ham
        if spec._beta is None:
            spec._beta = spec.beta()
        beta = spec._beta
        dts = np.concatenate([np.asarray(spec.dt, np.float64), [spec.dt[-1]]])  # Nt = K + 1 rows
        Np = [gqt_np_rule(spec.energy_scale * d, 4096) for d in dts]
        g_on = torch.empty(spec.topo.n, dtype=torch.float64, device=spec.phi.device)
        g_slot = torch.empty((spec.topo.n, spec.topo.K, 2), dtype=torch.float64, device=spec.phi.device)
        loss = gqt_vac_loss_grad(ham, spec.phi, dts, spec.M, beta, g_on, g_slot, Np=Np, stride=spec.stride)
        ia = torch.from_numpy(spec.topo.slot_a).to(g_slot.device)
        ib = torch.from_numpy(spec.topo.slot_b).to(g_slot.device)
        g_hop = torch.empty(spec.topo.nbonds, dtype=torch.float64, device=g_slot.device)
        gqt_bond_gradients(g_slot, ia, ib, g_hop)
        torch.cuda.synchronize(g_slot.device)
        ctx.save_for_backward(g_on.to(onsite.device), g_hop.to(hop.device))
        return torch.tensor(loss, dtype=torch.float64, device=onsite.device)

    @staticmethod
    def backward(ctx, grad):
        g_on, g_hop = ctx.saved_tensors
        return grad * g_on, grad * g_hop, None
