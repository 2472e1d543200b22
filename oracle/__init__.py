"""ctypes front end of the serial FP64 oracle (``gqt_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The GPU library never
imports this package and this package never imports the library.

Arrays are numpy; complex vectors are complex128.  Each wrapper names the
equation of arXiv:1705.01387 it evaluates.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gqt_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "libgqt_oracle.so")
_lock = threading.Lock()
_lib = None

_d = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (portable flags only)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_override_path = None


def use_library(path):
    """Load the oracle from another shared object (a test builds deliberately
    broken copies to show that the pins catch each mistake); None restores the
    regular build."""
    global _lib, _override_path
    with _lock:
        _lib = None
        _override_path = path


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(_override_path or build())
            L.orc_ham_new.restype = C.c_void_p
            L.orc_ham_new.argtypes = [C.c_int64, C.c_int, _i32, _i32, _d, _d, _d, _d, C.c_double]
            L.orc_ham_free.argtypes = [C.c_void_p]
            L.orc_apply_ht.argtypes = [C.c_void_p, _d, _d]
            L.orc_apply_v.argtypes = [C.c_void_p, _d, _d]
            L.orc_cheb_moments.argtypes = [C.c_void_p, _d, _d, C.c_int, _d]
            L.orc_dos_moments.argtypes = [C.c_void_p, _d, C.c_int, _d]
            L.orc_np_rule.restype = C.c_int
            L.orc_np_rule.argtypes = [C.c_double, C.c_int]
            L.orc_bessel.argtypes = [C.c_double, C.c_int, _d]
            L.orc_evolve.argtypes = [C.c_void_p, _d, C.c_double, C.c_int, C.c_int, _d]
            L.orc_commutator_evolve.argtypes = [C.c_void_p, _d, C.c_double, C.c_int, _d]
            _ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
            L.orc_vac_moments.argtypes = [C.c_void_p, _d, _d, _ip, C.c_int, C.c_int, _d, C.c_void_p, C.c_void_p]
            L.orc_msd_moments.argtypes = [C.c_void_p, _d, _d, _ip, C.c_int, C.c_int, _d, C.c_void_p, C.c_void_p]
            L.orc_jackson.argtypes = [C.c_int, _d]
            L.orc_kpm_reconstruct.argtypes = [_d, C.c_int, C.c_int, _d, C.c_int, C.c_double, C.c_double, _d]
            L.orc_sigma_vac.argtypes = [_d, _d, C.c_int, C.c_int, _d]
            L.orc_sigma_msd.argtypes = [_d, _d, C.c_int, C.c_int, _d]
            L.orc_cheb_adjoint.argtypes = [C.c_void_p, _d, _d, _d, C.c_int, _d, _d, C.c_void_p]
            L.orc_vac_loss_grad.restype = C.c_double
            L.orc_vac_loss_grad.argtypes = [C.c_void_p, _d, _d, _ip, C.c_int, C.c_int, _d, _d, _d]
            L.orc_kb_moments.argtypes = [C.c_void_p, _d, _d, _d, C.c_int, C.c_int, _d]
            L.orc_kubo_bastin.argtypes = [_d, C.c_int, _d, C.c_int, C.c_double, C.c_double, C.c_int, _d]
            L.orc_kubo_bastin_fermi.argtypes = [_d, C.c_int, _d, C.c_int, C.c_double, C.c_double, C.c_int, _d,
                                                C.c_int, C.c_double, _d]
            _lib = L
    return _lib


def _cv(x) -> np.ndarray:
    """complex vector -> contiguous float64 view (re, im interleaved)."""
    return np.ascontiguousarray(x, dtype=np.complex128).view(np.float64)


class Hamiltonian:
    """H~ = H / dE of a lattice in the paper's input form (Sec. 4.2, Eqs. 19, 32-34)."""

    def __init__(self, lat, energy_scale: float):
        self.n = int(lat.n)
        self.K = int(lat.max_nb)
        self.energy_scale = float(energy_scale)
        self.lat = lat
        hop = np.ascontiguousarray(lat.hop, dtype=np.complex128)
        self._p = lib().orc_ham_new(self.n, self.K, np.ascontiguousarray(lat.nb_count, np.int32),
                                    np.ascontiguousarray(lat.nb_idx, np.int32).reshape(-1),
                                    np.ascontiguousarray(hop.real).reshape(-1),
                                    np.ascontiguousarray(hop.imag).reshape(-1),
                                    np.ascontiguousarray(lat.onsite, np.float64),
                                    np.ascontiguousarray(lat.dx, np.float64).reshape(-1), self.energy_scale)

    def __del__(self):
        p = getattr(self, "_p", None)
        if p and _lib is not None:
            _lib.orc_ham_free(p)
            self._p = None

    def _vec(self, x):
        x = np.ascontiguousarray(x, dtype=np.complex128).reshape(-1)
        if x.size != self.n:
            raise ValueError("vector length != N")
        return x

    def apply_ht(self, x):
        y = np.empty(self.n, np.complex128)
        lib().orc_apply_ht(self._p, _cv(self._vec(x)), y.view(np.float64))
        return y

    def apply_v(self, x):
        y = np.empty(self.n, np.complex128)
        lib().orc_apply_v(self._p, _cv(self._vec(x)), y.view(np.float64))
        return y

    def cheb_moments(self, l, r, M):
        """mu_m = <l|T_m(H~)|r> (Eqs. 21, 28)."""
        mu = np.empty(M, np.complex128)
        lib().orc_cheb_moments(self._p, _cv(self._vec(l)), _cv(self._vec(r)), M, mu.view(np.float64))
        return mu

    def dos_moments(self, phi, M):
        """C_n^DOS / N (Eq. 28, unit-norm phi)."""
        mu = np.empty(M, np.float64)
        lib().orc_dos_moments(self._p, _cv(self._vec(phi)), M, mu)
        return mu

    def evolve(self, psi, dt, sign, Np):
        """U(sign*dt) psi (Eq. 17)."""
        y = np.empty(self.n, np.complex128)
        lib().orc_evolve(self._p, _cv(self._vec(psi)), float(dt), int(sign), int(Np), y.view(np.float64))
        return y

    def commutator_evolve(self, psi, dt, Np):
        """[X, U(dt)] psi (Eqs. 18, 22, 24)."""
        y = np.empty(self.n, np.complex128)
        lib().orc_commutator_evolve(self._p, _cv(self._vec(psi)), float(dt), int(Np), y.view(np.float64))
        return y

    def _steps(self, dt, Np):
        dt = np.ascontiguousarray(np.atleast_1d(dt), np.float64)
        Np = np.ascontiguousarray(np.atleast_1d(Np), np.int32)
        if Np.size == 1 and dt.size > 1:
            Np = np.full(dt.size, int(Np[0]), np.int32)
        return dt, Np

    def vac_moments(self, phi, dt, Np, M, return_state=False):
        """C_n^VAC(t_k) / N at t_0 = 0 .. t_{Nt-1} (Eq. 29); [Nt, M]."""
        dt, Np = self._steps(dt, Np)
        out = np.empty((dt.size, M), np.float64)
        a = np.empty(self.n, np.complex128)
        b = np.empty(self.n, np.complex128)
        lib().orc_vac_moments(self._p, _cv(self._vec(phi)), dt, Np, dt.size, M, out.reshape(-1),
                              a.ctypes.data, b.ctypes.data)
        return (out, a, b) if return_state else out

    def msd_moments(self, phi, dt, Np, M, return_state=False):
        """C_n^MSD(t_k) / N at t_1 .. t_Nt (Eq. 30); [Nt, M]."""
        dt, Np = self._steps(dt, Np)
        out = np.empty((dt.size, M), np.float64)
        p = np.empty(self.n, np.complex128)
        px = np.empty(self.n, np.complex128)
        lib().orc_msd_moments(self._p, _cv(self._vec(phi)), dt, Np, dt.size, M, out.reshape(-1),
                              p.ctypes.data, px.ctypes.data)
        return (out, p, px) if return_state else out

    def cheb_adjoint(self, l, r, coef):
        """Gradient of Re sum_m coef_m <l|T_m(H~)|r>: (dJ/dU [N], G per slot [N,K], rbar [N])."""
        coef = np.ascontiguousarray(coef, np.complex128)
        ge = np.empty(self.n, np.float64)
        gs = np.empty((self.n, self.K), np.complex128)
        rb = np.empty(self.n, np.complex128)
        lib().orc_cheb_adjoint(self._p, _cv(self._vec(l)), _cv(self._vec(r)), coef.view(np.float64), coef.size,
                               ge, gs.reshape(-1).view(np.float64), rb.ctypes.data)
        return ge, gs, rb

    def vac_loss_grad(self, phi, dt, Np, beta):
        """J = sum_k sum_n beta[k,n] C_n^VAC(t_k)/N and (dJ/dU [N], G per slot [N,K])."""
        dt, Np = self._steps(dt, Np)
        beta = np.ascontiguousarray(beta, np.float64)
        Nt, M = beta.shape
        ge = np.empty(self.n, np.float64)
        gs = np.empty((self.n, self.K), np.complex128)
        J = lib().orc_vac_loss_grad(self._p, _cv(self._vec(phi)), dt, Np, Nt, M, beta.reshape(-1), ge,
                                    gs.reshape(-1).view(np.float64))
        return J, ge, gs


    def kb_moments(self, d_a, d_b, r, M):
        """Kubo-Bastin moments Lambda_mn = Tr[v~_a T_m(H~) v~_b T_n(H~)] (Hall
        conductivity, beyond the paper's Sec. 6 outlook) estimated with the unit
        vectors r [N, R] (site-major); d_a, d_b [N, K] bond displacements of the
        two directions.  Returns complex [M, M]."""
        r = np.ascontiguousarray(np.asarray(r, np.complex128).reshape(self.n, -1).T)
        lam = np.empty((M, M), np.complex128)
        lib().orc_kb_moments(self._p, np.ascontiguousarray(d_a, np.float64).reshape(-1),
                             np.ascontiguousarray(d_b, np.float64).reshape(-1), r.view(np.float64).reshape(-1),
                             r.shape[0], M, lam.view(np.float64).reshape(-1))
        return lam

def np_rule(x: float, cap: int = 64) -> int:
    """N_p = 1 + max{m : |J_m(x)| >= 1e-15}, capped (Sec. 3.2, machine precision)."""
    return int(lib().orc_np_rule(float(x), int(cap)))


def bessel(x: float, count: int) -> np.ndarray:
    J = np.empty(count, np.float64)
    lib().orc_bessel(float(x), int(count), J)
    return J


def jackson(M: int) -> np.ndarray:
    """Jackson damping g_n, n < M (Eq. 31)."""
    g = np.empty(M, np.float64)
    lib().orc_jackson(int(M), g)
    return g


def kpm_reconstruct(mu, E, energy_scale, n_over_omega):
    """rho-weighted reconstruction on energies E (Eqs. 25-27); mu [rows, M] -> [rows, NE]."""
    mu = np.ascontiguousarray(np.atleast_2d(mu), np.float64)
    E = np.ascontiguousarray(E, np.float64)
    out = np.empty((mu.shape[0], E.size), np.float64)
    lib().orc_kpm_reconstruct(mu.reshape(-1), mu.shape[0], mu.shape[1], E, E.size, float(energy_scale),
                              float(n_over_omega), out.reshape(-1))
    return out


def sigma_vac(vac, dt):
    """Running conductivity from the VAC (Eq. 2), trapezoid over rows t_0..t_{Nt-1}."""
    vac = np.ascontiguousarray(vac, np.float64)
    dt = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, np.float64), (vac.shape[0],)))
    out = np.empty_like(vac)
    lib().orc_sigma_vac(vac.reshape(-1), dt, vac.shape[0], vac.shape[1], out.reshape(-1))
    return out


def sigma_msd(msd, dt):
    """Running conductivity from the MSD (Eq. 5), finite difference over rows t_1..t_Nt."""
    msd = np.ascontiguousarray(msd, np.float64)
    dt = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, np.float64), (msd.shape[0],)))
    out = np.empty_like(msd)
    lib().orc_sigma_msd(msd.reshape(-1), dt, msd.shape[0], msd.shape[1], out.reshape(-1))
    return out


def kubo_bastin(lam, E, energy_scale, area, kernel=0):
    """sigma_ab(E_j) / (e^2/h) from Kubo-Bastin moments [M, M] on ascending
    energies E (trapezoid from E_0); kernel 0 = Jackson, 1 = none."""
    lam = np.ascontiguousarray(lam, np.complex128)
    E = np.ascontiguousarray(E, np.float64)
    out = np.empty(E.size, np.float64)
    lib().orc_kubo_bastin(lam.view(np.float64).reshape(-1), lam.shape[0], E, E.size, float(energy_scale),
                          float(area), int(kernel), out)
    return out


def kubo_bastin_fermi(lam, E, energy_scale, area, mu, kT, kernel=0):
    """sigma_ab(mu_j, T) / (e^2/h): the Kubo-Bastin integrand on the ascending grid E
    weighted by the Fermi function 1/(1 + exp((E - mu_j)/kT)) (kT = 0: step)."""
    lam = np.ascontiguousarray(lam, np.complex128)
    E = np.ascontiguousarray(E, np.float64)
    mu = np.ascontiguousarray(np.atleast_1d(mu), np.float64)
    out = np.empty(mu.size, np.float64)
    lib().orc_kubo_bastin_fermi(lam.view(np.float64).reshape(-1), lam.shape[0], E, E.size, float(energy_scale),
                                float(area), int(kernel), mu, mu.size, float(kT), out)
    return out
