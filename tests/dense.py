"""Dense-matrix restatements used to pin the oracle (exact diagonalisation).

Written independently of ``oracle/``: these build H, V and [X,H] as dense numpy
matrices from the paper's input form and evaluate the paper's quantities by
eigendecomposition (numpy.linalg.eigh), which is exact up to rounding.
"""
import numpy as np


def dense_h(lat, scale=1.0):
    """Dense H / scale (Eq. 32): H[i, nb] += hop, H[i, i] = U_i."""
    n = lat.n
    H = np.zeros((n, n), np.complex128)
    for i in range(n):
        H[i, i] += lat.onsite[i]
        for k in range(lat.nb_count[i]):
            H[i, lat.nb_idx[i, k]] += lat.hop[i, k]
    return H / scale


def dense_xh(lat, scale=1.0):
    """Dense [X, H]/scale with [X,H]_mn = (X_m - X_n) H_mn = -dx_mn H_mn."""
    n = lat.n
    D = np.zeros((n, n), np.complex128)
    for i in range(n):
        for k in range(lat.nb_count[i]):
            D[i, lat.nb_idx[i, k]] += -lat.dx[i, k] * lat.hop[i, k]
    return D / scale


def dense_v(lat):
    """V = i [H, X] (Eq. 34), i.e. V_mn = i (X_n - X_m) H_mn."""
    return 1j * _dxh(lat)


def _dxh(lat):
    n = lat.n
    D = np.zeros((n, n), np.complex128)
    for i in range(n):
        for k in range(lat.nb_count[i]):
            D[i, lat.nb_idx[i, k]] += lat.dx[i, k] * lat.hop[i, k]
    return D


def cheb_T(n, x):
    return np.cos(n * np.arccos(np.clip(x, -1.0, 1.0)))


def eig(Ht):
    lam, Q = np.linalg.eigh(Ht)
    return lam, Q


def fun_of_h(lam, Q, f):
    return (Q * f(lam)) @ Q.conj().T


def divided_difference(lam, f, fprime):
    """F_ab = (f(l_a) - f(l_b)) / (l_a - l_b), f'(l_a) when l_a == l_b."""
    la = lam[:, None]
    lb = lam[None, :]
    diff = la - lb
    close = np.abs(diff) < 1e-9
    F = np.where(close, 0.0, (f(la) - f(lb)) / np.where(close, 1.0, diff))
    fp = fprime(0.5 * (la + lb))
    return np.where(close, fp, F)


def frechet(lam, Q, f, fprime, D):
    """Daleckii-Krein: derivative of f(H) in direction D = Q (F o Q^+ D Q) Q^+."""
    F = divided_difference(lam, f, fprime)
    return Q @ (F * (Q.conj().T @ D @ Q)) @ Q.conj().T


def dense_vd(lat, d, scale=1.0):
    """Velocity along the direction with bond displacements d [N, K] (d = dx or
    dy), in units of scale/hbar: V_mn = i d_mn H_mn / scale (i [H, X] / scale)."""
    n = lat.n
    D = np.zeros((n, n), np.complex128)
    for i in range(n):
        for k in range(lat.nb_count[i]):
            D[i, lat.nb_idx[i, k]] += 1j * d[i, k] * lat.hop[i, k]
    return D / scale


def tknn_sigma(lat, mu_f, da, db):
    """Zero-temperature Hall conductivity in units of e^2/h from the eigenstates
    (Kubo formula in the Thouless-Kohmoto-Nightingale-den Nijs form):
    sigma_ab = (4 pi / Omega) sum_{b occupied} sum_{a != b}
    Im[<a|v_a|b><b|v_b|a>] / (E_a - E_b)^2, hbar = 1, v = i [H, X]."""
    H = dense_h(lat)
    w, Q = np.linalg.eigh(H)
    va = Q.conj().T @ dense_vd(lat, da) @ Q
    vb = Q.conj().T @ dense_vd(lat, db) @ Q
    s = 0.0
    for b in np.where(w < mu_f)[0]:
        de = w - w[b]
        m = np.abs(de) > 1e-9
        s += np.sum(np.imag(va[m, b] * vb[b, m]) / de[m] ** 2)
    return 4.0 * np.pi * s / lat.volume
