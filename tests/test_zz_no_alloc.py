"""The allocation-free DOS entry point (gqt_dos_moments_noalloc) through the C ABI.

It serves callers that may not call cudaMalloc: their device memory belongs to
another allocator (a framework's caching pool, a fixed budget) that must not be
bypassed, or they sit on latency-critical paths where an allocation would
synchronise the device.  Its scratch lives in a fixed device array inside the
library.  Each case runs two calls in a row with different vectors; each call
must reproduce the regular entry point (gqt_dos_moments) and the serial FP64
oracle, which also shows that leftovers of the first call in the shared array do
not leak into the second.  The cases cover the four instantiations (FP64 and
FP32 storage, real and complex hoppings).  This file is named to be collected
last."""
import ctypes as C

import numpy as np
import pytest

import gqt_synth as S
import oracle as O

torch = pytest.importorskip("torch")
g = pytest.importorskip("paper_1705_01387_gb300")

pytestmark = pytest.mark.gpu

# Normalised L-infinity tolerances (max_n |d mu_n| / max_n |mu_n|): FP64 storage
# 1e-10 against the oracle; FP32 storage 1e-5 against the oracle (the FP32 moment
# bound of the parity tests).  The two entry points run different recursions (the
# regular one the l = r doubling identities, or a cluster-resident row on small
# systems; this one the plain three-term recursion of Eq. 21), so they agree to
# FP64 rounding (1e-12) on FP64 handles and to FP32 storage rounding (1e-5, the
# same bound as against the oracle) on FP32 handles.
TOL = {g.GQT_FP64: 1e-10, g.GQT_FP32_ACC64: 1e-5}
TOL_SAME = {g.GQT_FP64: 1e-12, g.GQT_FP32_ACC64: 1e-5}


def _call(ham, phi, R, M, mu):
    st = torch.cuda.current_stream().cuda_stream
    return g.lib().gqt_dos_moments_noalloc(ham.ptr, C.c_void_p(phi.data_ptr()), R, M, C.c_void_p(mu.data_ptr()),
                                           C.c_void_p(st))


def _nerr(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _lattice(hop):
    if hop == "real":
        return S.honeycomb(32, 32, -2.7, 1.0, seed=S.BASE_SEED), S.energy_scale_rule(3, -2.7, 1.0)
    lat = S.with_random_bond_phases(S.honeycomb(23, 19, -2.7, 2.0, seed=3), 4)  # complex hoppings, N = 874
    return lat, S.energy_scale_rule(3, -2.7, 2.0)


@pytest.mark.parametrize("prec", [g.GQT_FP64, g.GQT_FP32_ACC64], ids=["fp64", "fp32"])
@pytest.mark.parametrize("hop", ["real", "complex"])
@pytest.mark.parametrize("R", [1, 4])
def test_noalloc_matches_regular_entry_point_and_oracle_twice(prec, hop, R):
    lat, dE = _lattice(hop)
    ham = g.gqt_build_hamiltonian(lat, dE, precision=prec)
    orc = O.Hamiltonian(lat, dE)
    M = 512
    ctype = torch.complex128 if prec == g.GQT_FP64 else torch.complex64
    for call in range(2):
        phi_h = S.random_phase(lat.n, R, seed=100 + call)
        phi = torch.from_numpy(phi_h).to(ctype).cuda()
        ref = torch.empty((1, R, M), dtype=torch.float64, device="cuda")
        g.gqt_dos_moments(ham, phi, R, M, ref)
        out = torch.full((1, R, M), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(ham, phi, R, M, out) == g.GQT_OK, g.gqt_last_error()
        torch.cuda.synchronize()
        a, b = out.cpu().numpy()[0], ref.cpu().numpy()[0]
        assert _nerr(a, b) < TOL_SAME[prec]
        # the oracle takes the vector the kernel saw (rounded to FP32 for FP32 storage)
        phi_seen = phi.cpu().to(torch.complex128).numpy()
        for r in range(R):
            mu = orc.dos_moments(phi_seen[:, r], M)
            assert _nerr(a[r], mu.real) < TOL[prec]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lat = S.square(256, 256, -1.0, 1.0, seed=2)
    ham = g.gqt_build_hamiltonian(lat, S.energy_scale_rule(4, -1.0, 1.0))
    phi = torch.zeros((lat.n, 8), dtype=torch.complex128, device="cuda")
    mu = torch.empty((1, 8, 64), dtype=torch.float64, device="cuda")
    assert _call(ham, phi, 8, 64, mu) == g.GQT_EINVAL
    assert "scratch" in g.gqt_last_error()


def test_noalloc_rejects_host_pointers():
    lat, dE = _lattice("real")
    ham = g.gqt_build_hamiltonian(lat, dE)
    phi = torch.from_numpy(S.random_phase(lat.n, 1, seed=1)).cuda()
    mu_dev = torch.empty((1, 1, 16), dtype=torch.float64, device="cuda")
    mu_host = torch.empty((1, 1, 16), dtype=torch.float64)
    phi_host = phi.cpu()
    assert _call(ham, phi, 1, 16, mu_host) == g.GQT_EINVAL
    assert "d_mu" in g.gqt_last_error()
    assert _call(ham, phi_host, 1, 16, mu_dev) == g.GQT_EINVAL
    assert "d_phi" in g.gqt_last_error()
