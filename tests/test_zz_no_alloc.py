"""The allocation-free DOS entry point (gqt_dos_moments_noalloc) against the
regular one (gqt_dos_moments), through the C ABI.

It exists for callers that may not call cudaMalloc (device memory owned by
another allocator, or latency-critical paths where an allocation would
synchronise the device); its scratch lives in a fixed device array inside the
library.  Two calls in a row must each reproduce the regular entry point, which
also shows that leftovers of the first call in the shared array do not leak into
the second.  This file is named to be collected last."""
import ctypes as C

import numpy as np
import pytest

import gqt_synth as S

torch = pytest.importorskip("torch")
g = pytest.importorskip("paper_1705_01387_gb300")

pytestmark = pytest.mark.gpu


def _call(ham, phi, R, M, mu):
    st = torch.cuda.current_stream().cuda_stream
    return g.lib().gqt_dos_moments_noalloc(ham.ptr, C.c_void_p(phi.data_ptr()), R, M, C.c_void_p(mu.data_ptr()),
                                           C.c_void_p(st))


@pytest.mark.parametrize("R", [1, 4])
def test_noalloc_matches_regular_entry_point_twice(R):
    lat = S.honeycomb(32, 32, -2.7, 1.0, seed=S.BASE_SEED)
    dE = S.energy_scale_rule(3, -2.7, 1.0)
    ham = g.gqt_build_hamiltonian(lat, dE)
    M = 512
    ref = torch.empty((1, R, M), dtype=torch.float64, device="cuda")
    for call in range(2):
        phi = torch.from_numpy(S.random_phase(lat.n, R, seed=100 + call)).cuda()
        g.gqt_dos_moments(ham, phi, R, M, ref)
        out = torch.full((1, R, M), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(ham, phi, R, M, out) == g.GQT_OK, g.gqt_last_error()
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < 1e-10


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lat = S.square(256, 256, -1.0, 1.0, seed=2)
    ham = g.gqt_build_hamiltonian(lat, S.energy_scale_rule(4, -1.0, 1.0))
    phi = torch.zeros((lat.n, 8), dtype=torch.complex128, device="cuda")
    mu = torch.empty((1, 8, 64), dtype=torch.float64, device="cuda")
    assert _call(ham, phi, 8, 64, mu) == g.GQT_EINVAL
    assert "scratch" in g.gqt_last_error()
