"""Python binding of libgqt (include/gqt.h): linear-scaling Kubo transport on GB300.

Argument marshalling only.  Every function here has the name of the C entry
point it calls; device vectors are torch tensors (complex128 for a GQT_FP64
handle, complex64 for GQT_FP32_ACC64), laid out [n, R] and contiguous; host
arrays are numpy.  Every computation runs in the library's CUDA kernels: if the
library is missing, importing its functions raises instead of falling back.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB, build

GQT_OK, GQT_EINVAL, GQT_ENOMEM, GQT_ECUDA, GQT_ERANGE, GQT_ENORM, GQT_ENAN, GQT_ETIMEOUT = range(8)
GQT_FP64, GQT_FP32_ACC64 = 0, 1
GQT_LATTICE_CUSTOM, GQT_LATTICE_CHAIN, GQT_LATTICE_SQUARE, GQT_LATTICE_HONEYCOMB, GQT_LATTICE_CUBIC = range(5)
GQT_FORM_HONEYCOMB, GQT_FORM_UNIFORM_HOP, GQT_FORM_CUBIC_SWEEP = 1, 2, 4
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ERANGE", "ENORM", "ENAN", "ETIMEOUT"]


class GqtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class gqt_lattice(C.Structure):
    _fields_ = [("kind", C.c_int), ("L1", C.c_int64), ("L2", C.c_int64), ("L3", C.c_int64), ("t", C.c_double),
                ("W", C.c_double), ("vacancy_frac", C.c_double), ("seed", C.c_uint64), ("n", C.c_int64),
                ("max_nb", C.c_int), ("nb_count", C.c_void_p), ("nb_idx", C.c_void_p), ("hop_re", C.c_void_p),
                ("hop_im", C.c_void_p), ("onsite", C.c_void_p), ("bond_dx", C.c_void_p), ("length_x", C.c_double),
                ("volume", C.c_double), ("bond_dy", C.c_void_p)]


_lib = None
_P, _I, _D, _U64, _I64 = C.c_void_p, C.c_int, C.c_double, C.c_uint64, C.c_int64

_SIGS = {
    "gqt_build_hamiltonian": [C.POINTER(gqt_lattice), _D, _I, _P, _I, C.POINTER(_P)],
    "gqt_free_hamiltonian": [_P],
    "gqt_update_hamiltonian": [_P, _P, _P, _P],
    "gqt_generate_lattice": [C.POINTER(gqt_lattice), _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "gqt_ham_info": [_P, _P, _P, _P, _P, _P, _P],
    "gqt_ham_forms": [_P, _P],
    "gqt_random_phase": [_P, _U64, _I, _I, _P, _P],
    "gqt_cheb_moments": [_P, _P, _P, _I, _I, _P, _P],
    "gqt_dos_moments": [_P, _P, _I, _I, _P, _P],
    "gqt_evolve": [_P, _P, _I, _D, _I, _I, _P, _P],
    "gqt_commutator_evolve": [_P, _P, _P, _I, _D, _I, _P],
    "gqt_apply_velocity": [_P, _P, _P, _I, _P],
    "gqt_vac_init": [_P, _P, _P, _P, _I, _P],
    "gqt_vac_moments": [_P, _P, _P, _I, _P, _P, _I, _I, _P, _P],
    "gqt_msd_init": [_P, _P, _P, _P, _I, _P],
    "gqt_msd_moments": [_P, _P, _P, _I, _P, _P, _I, _I, _P, _P],
    "gqt_kpm_reconstruct": [_P, _I, _I, _P, _I, _D, _D, _I, _P, _P],
    "gqt_kpm_weights": [_I, _P, _I, _P, _D, _D, _I, _P, _P],
    "gqt_kb_moments": [_P, _P, _I, _I, _I, _I, _P, _P],
    "gqt_set_kb_contraction": [_P, _I],
    "gqt_set_wait_limit": [_P, _I],
    "gqt_set_fp64_arith": [_P, _I],
    "gqt_set_temporal_blocking": [_P, _I],
    "gqt_kubo_bastin": [_P, _I, _P, _I, _D, _D, _I, _P, _P],
    "gqt_kubo_bastin_fermi": [_P, _I, _P, _I, _D, _D, _I, _P, _I, _D, _P, _P],
    "gqt_sigma_vac_loss_weights": [_I, _P, _I, _P, _D, _D, _I, _P, _I, _P, _P],
    "gqt_bond_gradients": [_P, _I64, _P, _P, _I, _P, _P, _P],
    "gqt_sigma_vac": [_P, _P, _I, _I, _P, _P],
    "gqt_sigma_msd": [_P, _P, _I, _I, _P, _P],
    "gqt_vac_loss_grad": [_P, _P, _P, _P, _I, _I, _P, _I, _P, _P, _P, _P],
    "gqt_bessel": [_D, _I, _P],
    "gqt_np_rule": [_D, _I],
    "gqt_set_launch": [_P, _I, _I],
    "gqt_autotune": [_P, _I, _P, _P, _P, _P],
    "gqt_set_graphs": [_P, _I],
    "gqt_set_variant": [_P, _I],
    "gqt_set_cluster": [_P, _I],
    "gqt_set_vac_pair": [_P, _I],
    "gqt_set_sweep_order": [_P, _I],
    "gqt_launch_count": [],
    "gqt_profile_start": [],
    "gqt_probe_fp64": [_P, _P],
    "gqt_profile_stop": [_P, _P, _I],
    "gqt_last_error": [],
    "gqt_dos_moments_noalloc": [_P, _P, _I, _I, _P, _P],
}
_RESTYPES = {"gqt_free_hamiltonian": None, "gqt_np_rule": C.c_int, "gqt_launch_count": C.c_uint64,
             "gqt_last_error": C.c_char_p}


def lib():
    """Load libgqt.so (building it first when the sources are newer)."""
    global _lib
    if _lib is None:
        path = LIB
        if not os.path.exists(path) or os.environ.get("GQT_REBUILD") == "1":
            build()
        L = C.CDLL(path)
        for name, args in _SIGS.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.argtypes = args
            fn.restype = _RESTYPES.get(name, C.c_int)
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return [n for n in _SIGS if getattr(lib(), n, None) is not None]


def _check(status: int):
    if status != GQT_OK:
        raise GqtError(status, lib().gqt_last_error().decode())


def _stream(stream):
    if stream is not None:
        return C.c_void_p(stream)
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _state_ptr(t, name="state"):
    """VAC/MSD state vector: a contiguous CUDA tensor, or a contiguous CPU tensor or
    numpy array (pinned or pageable; the library copies it in and out)."""
    import torch
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return C.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray) and t.flags.c_contiguous:
        return C.c_void_p(t.ctypes.data)
    raise ValueError(f"{name} must be a contiguous tensor or numpy array")


def _out_ptr(out):
    """Moment output: a contiguous float64 CUDA tensor or numpy array."""
    import torch
    if isinstance(out, torch.Tensor):
        if out.dtype != torch.float64 or not out.is_contiguous():
            raise ValueError("output tensor must be contiguous float64")
        return C.c_void_p(out.data_ptr())
    if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous):
        raise ValueError("output array must be contiguous float64")
    return C.c_void_p(out.ctypes.data)


class Ham:
    """Owner of a gqt_ham* (freed on garbage collection)."""

    def __init__(self, ptr, keep=()):
        self.ptr = C.c_void_p(ptr)
        n, dE, vol = C.c_int64(), C.c_double(), C.c_double()
        nseg, prec, real = C.c_int(), C.c_int(), C.c_int()
        _check(lib().gqt_ham_info(self.ptr, C.byref(n), C.byref(dE), C.byref(vol), C.byref(nseg), C.byref(prec),
                                  C.byref(real)))
        self.n, self.energy_scale, self.volume = n.value, dE.value, vol.value
        self.nseg, self.precision, self.hop_real = nseg.value, prec.value, bool(real.value)

    @property
    def forms(self) -> int:
        """Bits of GQT_FORM_HONEYCOMB, GQT_FORM_UNIFORM_HOP, GQT_FORM_CUBIC_SWEEP
        (gqt_ham_forms), read when asked (updates can change them)."""
        f = C.c_int()
        _check(lib().gqt_ham_forms(self.ptr, C.byref(f)))
        return f.value

    @property
    def complex_dtype(self):
        import torch
        return torch.complex128 if self.precision == GQT_FP64 else torch.complex64

    def __del__(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value and _lib is not None:
            _lib.gqt_free_hamiltonian(self.ptr)
            self.ptr = None


def _lattice_struct(lattice=None, kind=None, L1=0, L2=0, L3=0, t=-1.0, W=0.0, vacancy_frac=0.0, seed=0):
    s = gqt_lattice()
    keep = []
    if lattice is not None:  # the paper's input form (any object with these attributes)
        s.kind = GQT_LATTICE_CUSTOM
        s.n = int(lattice.n)
        s.max_nb = int(lattice.max_nb)
        arrs = dict(nb_count=np.ascontiguousarray(lattice.nb_count, np.int32),
                    nb_idx=np.ascontiguousarray(lattice.nb_idx, np.int32),
                    hop_re=np.ascontiguousarray(np.real(lattice.hop), np.float64),
                    hop_im=np.ascontiguousarray(np.imag(lattice.hop), np.float64),
                    onsite=np.ascontiguousarray(lattice.onsite, np.float64),
                    bond_dx=np.ascontiguousarray(lattice.dx, np.float64))
        if getattr(lattice, "dy", None) is not None:
            arrs["bond_dy"] = np.ascontiguousarray(lattice.dy, np.float64)
        for k, a in arrs.items():
            keep.append(a)
            setattr(s, k, a.ctypes.data)
        s.length_x = float(lattice.length_x)
        s.volume = float(lattice.volume)
    else:
        s.kind, s.L1, s.L2, s.L3 = int(kind), int(L1), int(L2), int(L3)
        s.t, s.W, s.vacancy_frac, s.seed = float(t), float(W), float(vacancy_frac), int(seed) % (1 << 64)
    return s, keep


def gqt_build_hamiltonian(lattice=None, energy_scale=0.0, precision=GQT_FP64, seg_offsets=None, **kind_args) -> Ham:
    """Build H~ on the current CUDA device: from a lattice in the paper's input form
    (``lattice``) or from a built-in kind (``kind=GQT_LATTICE_..., L1=, L2=, t=, W=, vacancy_frac=, seed=``)."""
    s, keep = _lattice_struct(lattice, **kind_args)
    out = C.c_void_p()
    if seg_offsets is None and lattice is not None and getattr(lattice, "seg_offsets", None) is not None:
        seg_offsets = lattice.seg_offsets
    segp, nseg = None, 0
    if seg_offsets is not None:
        seg = np.ascontiguousarray(seg_offsets, np.int64)
        keep.append(seg)
        segp, nseg = seg.ctypes.data, len(seg) - 1
    _check(lib().gqt_build_hamiltonian(C.byref(s), float(energy_scale), int(precision), segp, nseg, C.byref(out)))
    return Ham(out.value, keep)


def gqt_update_hamiltonian(ham: Ham, onsite, hop):
    """New on-site energies [n] and hoppings [n, max_nb] (complex allowed only on complex
    handles) for an existing handle with the same neighbour list."""
    on = np.ascontiguousarray(onsite, np.float64)
    hop = np.asarray(hop)
    hr = np.ascontiguousarray(np.real(hop), np.float64)
    hi = np.ascontiguousarray(np.imag(hop), np.float64) if np.iscomplexobj(hop) else None
    _check(lib().gqt_update_hamiltonian(ham.ptr, on.ctypes.data, hr.ctypes.data,
                                        None if hi is None else hi.ctypes.data))


def gqt_generate_lattice(kind, L1=0, L2=0, L3=0, t=-1.0, W=0.0, vacancy_frac=0.0, seed=0) -> dict:
    s, _ = _lattice_struct(None, kind, L1, L2, L3, t, W, vacancy_frac, seed)
    n, K = C.c_int64(), C.c_int()
    _check(lib().gqt_generate_lattice(C.byref(s), C.byref(n), C.byref(K), *([None] * 6), None, None))
    n, K = n.value, K.value
    out = dict(nb_count=np.empty(n, np.int32), nb_idx=np.empty((n, K), np.int32), hop_re=np.empty((n, K)),
               hop_im=np.empty((n, K)), onsite=np.empty(n), bond_dx=np.empty((n, K)))
    lx, vol = C.c_double(), C.c_double()
    _check(lib().gqt_generate_lattice(C.byref(s), None, None, *[out[k].ctypes.data for k in
                                                                ("nb_count", "nb_idx", "hop_re", "hop_im", "onsite",
                                                                 "bond_dx")], C.byref(lx), C.byref(vol)))
    out.update(n=n, K=K, length_x=lx.value, volume=vol.value)
    return out


def gqt_random_phase(ham: Ham, seed: int, R: int, phi, first_vector: int = 0, stream=None):
    _check(lib().gqt_random_phase(ham.ptr, int(seed) % (1 << 64), int(first_vector), int(R), _dptr(phi, "phi"),
                                  _stream(stream)))
    return phi


def gqt_cheb_moments(ham: Ham, l, r, R: int, M: int, mu, stream=None):
    """mu: float64 [nseg, R, M, 2] (complex moments as (re, im) pairs)."""
    _check(lib().gqt_cheb_moments(ham.ptr, _dptr(l, "l"), _dptr(r, "r"), int(R), int(M), _out_ptr(mu),
                                  _stream(stream)))
    return mu


def gqt_dos_moments(ham: Ham, phi, R: int, M: int, mu, stream=None):
    _check(lib().gqt_dos_moments(ham.ptr, _dptr(phi, "phi"), int(R), int(M), _out_ptr(mu), _stream(stream)))
    return mu


def gqt_dos_moments_noalloc(ham: Ham, phi, R: int, M: int, mu, stream=None):
    """As gqt_dos_moments, for callers that may not allocate device memory: mu must be a
    float64 CUDA tensor; scratch comes from the library's fixed device array."""
    _check(lib().gqt_dos_moments_noalloc(ham.ptr, _dptr(phi, "phi"), int(R), int(M), _dptr(mu, "mu"),
                                         _stream(stream)))
    return mu


def gqt_evolve(ham: Ham, psi, R: int, dt: float, sign: int, Np: int = 0, norm=None, stream=None):
    nptr = None
    if norm is not None:
        nptr = norm.ctypes.data
    _check(lib().gqt_evolve(ham.ptr, _dptr(psi, "psi"), int(R), float(dt), int(sign), int(Np), nptr, _stream(stream)))
    return psi


def gqt_commutator_evolve(ham: Ham, psi, out, R: int, dt: float, Np: int = 0, stream=None):
    _check(lib().gqt_commutator_evolve(ham.ptr, _dptr(psi, "psi"), _dptr(out, "out"), int(R), float(dt), int(Np),
                                       _stream(stream)))
    return out


def gqt_apply_velocity(ham: Ham, x, y, R: int, stream=None):
    _check(lib().gqt_apply_velocity(ham.ptr, _dptr(x, "x"), _dptr(y, "y"), int(R), _stream(stream)))
    return y


def gqt_vac_init(ham: Ham, phi, a, b, R: int, stream=None):
    _check(lib().gqt_vac_init(ham.ptr, _dptr(phi, "phi"), _dptr(a, "a"), _dptr(b, "b"), int(R), _stream(stream)))


def gqt_msd_init(ham: Ham, phi, p, px, R: int, stream=None):
    _check(lib().gqt_msd_init(ham.ptr, _dptr(phi, "phi"), _dptr(p, "p"), _dptr(px, "px"), int(R), _stream(stream)))


def _steps(dt, Np):
    dt = np.ascontiguousarray(np.atleast_1d(dt), np.float64)
    npp = None
    if Np is not None:
        Np = np.ascontiguousarray(np.broadcast_to(np.asarray(Np, np.int32), dt.shape))
        npp = Np
    return dt, npp


def gqt_vac_moments(ham: Ham, a, b, R: int, dt, M: int, mu, Np=None, stream=None):
    dt, npp = _steps(dt, Np)
    _check(lib().gqt_vac_moments(ham.ptr, _state_ptr(a, "a"), _state_ptr(b, "b"), int(R), dt.ctypes.data,
                                 None if npp is None else npp.ctypes.data, dt.size, int(M), _out_ptr(mu),
                                 _stream(stream)))
    return mu


def gqt_msd_moments(ham: Ham, p, px, R: int, dt, M: int, mu, Np=None, stream=None):
    dt, npp = _steps(dt, Np)
    _check(lib().gqt_msd_moments(ham.ptr, _state_ptr(p, "p"), _state_ptr(px, "px"), int(R), dt.ctypes.data,
                                 None if npp is None else npp.ctypes.data, dt.size, int(M), _out_ptr(mu),
                                 _stream(stream)))
    return mu


def gqt_kpm_reconstruct(mu, E, energy_scale: float, n_over_omega: float, out, kernel: int = 0, stream=None):
    """mu: CUDA float64 [rows, M]; E: CUDA float64 [NE]; out: CUDA float64 [rows, NE]."""
    rows, M = mu.shape
    _check(lib().gqt_kpm_reconstruct(_dptr(mu, "mu"), int(rows), int(M), _dptr(E, "E"), int(E.numel()),
                                     float(energy_scale), float(n_over_omega), int(kernel), _dptr(out, "out"),
                                     _stream(stream)))
    return out


def gqt_kpm_weights(M: int, E, w, energy_scale: float, n_over_omega: float, beta, kernel: int = 0, stream=None):
    """beta[n] = sum_e w[e] d(reconstructed value at E[e]) / d(mu_n); E, w, beta CUDA float64."""
    _check(lib().gqt_kpm_weights(int(M), _dptr(E, "E"), int(E.numel()), _dptr(w, "w"), float(energy_scale),
                                 float(n_over_omega), int(kernel), _dptr(beta, "beta"), _stream(stream)))
    return beta


def gqt_kb_moments(ham: Ham, r, R: int, M: int, alpha: int, beta: int, lam, stream=None):
    """Kubo-Bastin moments Lambda [M, M] (CUDA complex128) of directions alpha, beta
    (0 = x, 1 = y) from R unit vectors r (CUDA [N, R]: complex128 for an FP64
    handle; complex64 for an FP32 handle, which needs gqt_set_kb_contraction(ham, 1))."""
    _check(lib().gqt_kb_moments(ham.ptr, _dptr(r, "r"), int(R), int(M), int(alpha), int(beta), _dptr(lam, "lam"),
                                _stream(stream)))
    return lam


def gqt_set_kb_contraction(ham: Ham, mode: int):
    """0 = FP64 contraction of the Hall moments (default); 1 = split TF32 on the
    tcgen05 tensor cores (Lambda to about 1e-5 of its largest entry)."""
    _check(lib().gqt_set_kb_contraction(ham.ptr, int(mode)))


def gqt_set_fp64_arith(ham: Ham, mode: int):
    """Moment rows of an FP64 handle with one vector: 1 = pairs of FP32 numbers on the
    FP32 pipes (default), 0 = FP64 fused multiply-adds."""
    _check(lib().gqt_set_fp64_arith(ham.ptr, int(mode)))


def gqt_set_temporal_blocking(ham: Ham, enable: bool):
    """Two Chebyshev orders per launch, each CTA walking a band of honeycomb cells
    down the rows (paired-FP32 rows of honeycomb-layout handles; default on)."""
    _check(lib().gqt_set_temporal_blocking(ham.ptr, int(bool(enable))))


def gqt_set_wait_limit(ham: Ham, polls: int):
    """Polls of each bounded device wait of the handle's kernels (default 2**24;
    0 gives up at once); a wait that runs out makes the call return GQT_ETIMEOUT."""
    _check(lib().gqt_set_wait_limit(ham.ptr, int(polls)))


def gqt_kubo_bastin(lam, E, energy_scale: float, area: float, sigma, kernel: int = 0, stream=None):
    """sigma_ab(E) / (e^2/h) (CUDA float64 [NE]) from moments lam (CUDA complex128 [M, M])
    on ascending energies E (CUDA float64 [NE]; E[0] is the lower integration limit)."""
    _check(lib().gqt_kubo_bastin(_dptr(lam, "lam"), int(lam.shape[0]), _dptr(E, "E"), int(E.numel()),
                                 float(energy_scale), float(area), int(kernel), _dptr(sigma, "sigma"),
                                 _stream(stream)))
    return sigma


def gqt_kubo_bastin_fermi(lam, E, energy_scale: float, area: float, mu, kT: float, sigma, kernel: int = 0,
                          stream=None):
    """sigma_ab(mu, T) / (e^2/h) (CUDA float64 [Nmu]) at chemical potentials mu (CUDA float64
    [Nmu]) and temperature kT from moments lam on the ascending energy grid E."""
    _check(lib().gqt_kubo_bastin_fermi(_dptr(lam, "lam"), int(lam.shape[0]), _dptr(E, "E"), int(E.numel()),
                                       float(energy_scale), float(area), int(kernel), _dptr(mu, "mu"),
                                       int(mu.numel()), float(kT), _dptr(sigma, "sigma"), _stream(stream)))
    return sigma


def gqt_sigma_vac_loss_weights(M: int, E, w, energy_scale: float, n_over_omega: float, dt, beta, kernel: int = 0,
                               stream=None):
    """beta [K+1, M] (CUDA float64) of L = sum_E w(E) sigma_VAC(E, t_K) over rows t_0..t_K (dt: K steps)."""
    dt = np.ascontiguousarray(np.atleast_1d(dt), np.float64)
    _check(lib().gqt_sigma_vac_loss_weights(int(M), _dptr(E, "E"), int(E.numel()), _dptr(w, "w"),
                                            float(energy_scale), float(n_over_omega), int(kernel), dt.ctypes.data,
                                            int(dt.size), _dptr(beta, "beta"), _stream(stream)))
    return beta


def gqt_bond_gradients(g_slot, slot_a, slot_b, g_re, g_im=None, stream=None):
    """g_slot: CUDA float64 [n, K, 2]; slot_a/slot_b: CUDA int64 [nbonds]; g_re (g_im): CUDA float64 [nbonds]."""
    _check(lib().gqt_bond_gradients(_dptr(g_slot, "g_slot"), int(g_slot.numel() // 2), _dptr(slot_a, "slot_a"),
                                    _dptr(slot_b, "slot_b"),
                                    int(slot_a.numel()), _dptr(g_re, "g_re"),
                                    None if g_im is None else _dptr(g_im, "g_im"), _stream(stream)))
    return g_re


def gqt_sigma_vac(vac, dt, out, stream=None):
    dt = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, np.float64), (vac.shape[0],)))
    _check(lib().gqt_sigma_vac(_dptr(vac, "vac"), dt.ctypes.data, int(vac.shape[0]), int(vac.shape[1]),
                               _dptr(out, "out"), _stream(stream)))
    return out


def gqt_sigma_msd(msd, dt, out, stream=None):
    dt = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, np.float64), (msd.shape[0],)))
    _check(lib().gqt_sigma_msd(_dptr(msd, "msd"), dt.ctypes.data, int(msd.shape[0]), int(msd.shape[1]),
                               _dptr(out, "out"), _stream(stream)))
    return out


def gqt_vac_loss_grad(ham: Ham, phi, dt, M: int, beta, g_onsite, g_slot, Np=None, stride: int = 0, stream=None):
    """beta: [Nt, M] numpy or CUDA float64; g_onsite: CUDA float64 [n]; g_slot: CUDA float64 [n, K, 2].
    Returns the loss."""
    dt, npp = _steps(dt, Np)
    import torch
    if isinstance(beta, torch.Tensor):
        bptr = _dptr(beta, "beta")
    else:
        beta = np.ascontiguousarray(beta, np.float64)
        bptr = beta.ctypes.data
    loss = C.c_double()
    _check(lib().gqt_vac_loss_grad(ham.ptr, _dptr(phi, "phi"), dt.ctypes.data,
                                   None if npp is None else npp.ctypes.data, dt.size, int(M), bptr,
                                   int(stride), C.byref(loss), _dptr(g_onsite, "g_onsite"), _dptr(g_slot, "g_slot"),
                                   _stream(stream)))
    return loss.value


def gqt_bessel(x: float, count: int) -> np.ndarray:
    J = np.empty(count, np.float64)
    _check(lib().gqt_bessel(float(x), int(count), J.ctypes.data))
    return J


def gqt_np_rule(x: float, cap: int = 64) -> int:
    return int(lib().gqt_np_rule(float(x), int(cap)))


def gqt_set_launch(ham: Ham, threads: int = 0, blocks_per_sm: int = 0):
    _check(lib().gqt_set_launch(ham.ptr, int(threads), int(blocks_per_sm)))


def gqt_set_cluster(ham: Ham, enable: bool):
    _check(lib().gqt_set_cluster(ham.ptr, int(bool(enable))))


def gqt_set_vac_pair(ham: Ham, enable: bool):
    _check(lib().gqt_set_vac_pair(ham.ptr, int(bool(enable))))


def gqt_set_sweep_order(ham: Ham, enable: bool):
    _check(lib().gqt_set_sweep_order(ham.ptr, int(bool(enable))))


def gqt_set_variant(ham: Ham, variant: int):
    _check(lib().gqt_set_variant(ham.ptr, int(variant)))


def gqt_autotune(ham: Ham, R: int, stream=None):
    """Returns (threads, blocks_per_sm, variant) chosen and set on the handle."""
    thr, bps, var = C.c_int(), C.c_int(), C.c_int()
    _check(lib().gqt_autotune(ham.ptr, int(R), C.byref(thr), C.byref(bps), C.byref(var), _stream(stream)))
    return thr.value, bps.value, var.value


def gqt_set_graphs(ham: Ham, enable: bool):
    _check(lib().gqt_set_graphs(ham.ptr, int(bool(enable))))


def gqt_profile_start():
    _check(lib().gqt_profile_start())


def gqt_profile_stop(ncat: int = 5):
    """Returns (ms per family, launches per family) since gqt_profile_start."""
    ms = np.zeros(ncat)
    n = np.zeros(ncat, np.uint64)
    _check(lib().gqt_profile_stop(ms.ctypes.data, n.ctypes.data, int(ncat)))
    return ms, n


def gqt_probe_fp64(stream=None) -> float:
    """Measured FP64 FMA throughput (GFLOP/s) of the current GPU."""
    v = C.c_double()
    _check(lib().gqt_probe_fp64(C.byref(v), _stream(stream)))
    return v.value


def gqt_launch_count() -> int:
    return int(lib().gqt_launch_count())


def gqt_last_error() -> str:
    return lib().gqt_last_error().decode()
