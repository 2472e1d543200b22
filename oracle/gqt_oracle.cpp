// Serial FP64 oracle for the linear-scaling Kubo method (Fan, Vierimaa, Harju,
// "GPUQT", Comput. Phys. Commun., arXiv:1705.01387).
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
// CPU statement of what the GPU library computes.  Only the test-suite, the
// smoke check and the benchmark's CPU-baseline leg may load it; the library
// never does.  It shares no code, header or constant table with the library.
//
// Every routine follows the paper's equations in the paper's order, with
// std::complex<double> arithmetic and plain loops; the only library primitive
// is std::cyl_bessel_j (C++17 special functions) for the Bessel coefficients.
//
// Conventions (readings of the paper, each pinned by tests):
//  * Input form of Sec. 4.2: row i of the neighbour list has cnt[i] neighbours
//    idx[i*K+k]; hop[i*K+k] = H_{i,idx} (Eq. 32); eps[i] = U_i; dx[i*K+k] =
//    X_idx - X_i as the minimum image (Eqs. 33-34).  hbar = e = 1.
//  * H~ = H / dE and dt~ = dE * dt (Eqs. 19-20).
//  * Random vectors are unit-norm, so every moment here is the paper's C_n / N
//    (Eq. 13 normalises <phi|phi> = N); the factor N returns in the
//    reconstruction prefactor through n_over_omega = N / Omega.
//  * VAC rows are at t_0 = 0 .. t_{Nt-1}; MSD rows at t_1 .. t_Nt.
//
// Parity pins for every function live in the test-suite (exact
// diagonalisation, closed forms, invariants, finite differences).

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

typedef std::complex<double> cplx;

namespace {

struct Ham {
  int64_t n = 0;
  int K = 0;
  std::vector<int32_t> cnt, idx;
  std::vector<cplx> hop;    // unscaled H_{i, idx}
  std::vector<double> eps;  // unscaled U_i
  std::vector<double> dx;   // X_idx - X_i
  double dE = 1.0;
};

// y = H~ x with H~ = H / dE (Eqs. 19, 32).
void apply_Ht(const Ham& h, const cplx* x, cplx* y) {
  for (int64_t i = 0; i < h.n; ++i) {
    cplx s = (h.eps[i] / h.dE) * x[i];
    for (int k = 0; k < h.cnt[i]; ++k) {
      int64_t j = h.idx[i * h.K + k];
      s += (h.hop[i * h.K + k] / h.dE) * x[j];
    }
    y[i] = s;
  }
}

// y = [X, H~] x.  [X, H]_{mn} = (X_m - X_n) H_{mn} = -dx_{mn} H_{mn}.
void apply_XHt(const Ham& h, const cplx* x, cplx* y) {
  for (int64_t i = 0; i < h.n; ++i) {
    cplx s = 0.0;
    for (int k = 0; k < h.cnt[i]; ++k) {
      int64_t j = h.idx[i * h.K + k];
      s += (-h.dx[i * h.K + k]) * (h.hop[i * h.K + k] / h.dE) * x[j];
    }
    y[i] = s;
  }
}

// y = V x with V = (i/hbar) sum (X_n - X_m) H_mn |m><n| (Eq. 34), unscaled H.
void apply_V(const Ham& h, const cplx* x, cplx* y) {
  const cplx I(0.0, 1.0);
  for (int64_t i = 0; i < h.n; ++i) {
    cplx s = 0.0;
    for (int k = 0; k < h.cnt[i]; ++k) {
      int64_t j = h.idx[i * h.K + k];
      s += I * h.dx[i * h.K + k] * h.hop[i * h.K + k] * x[j];
    }
    y[i] = s;
  }
}

cplx dot(int64_t n, const cplx* a, const cplx* b) {  // <a|b>
  cplx s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += std::conj(a[i]) * b[i];
  return s;
}

// mu_m = <l| T_m(H~) |r>, m < M, with T_0 = 1, T_1 = H~ and
// T_m = 2 H~ T_{m-1} - T_{m-2} (Eqs. 21, 23, 28).
void cheb_moments(const Ham& h, const cplx* l, const cplx* r, int M, cplx* mu) {
  const int64_t n = h.n;
  std::vector<cplx> t0(r, r + n), t1(n), t2(n), ht(n);
  if (M > 0) mu[0] = dot(n, l, t0.data());
  if (M > 1) {
    apply_Ht(h, t0.data(), t1.data());
    mu[1] = dot(n, l, t1.data());
  }
  for (int m = 2; m < M; ++m) {
    apply_Ht(h, t1.data(), ht.data());
    for (int64_t i = 0; i < n; ++i) t2[i] = 2.0 * ht[i] - t0[i];
    mu[m] = dot(n, l, t2.data());
    t0.swap(t1);
    t1.swap(t2);
  }
}

// Largest expansion length allowed by the "machine precision" statement
// (Sec. 3.2): N_p = 1 + max{m : |J_m(x)| >= 1e-15}, at most cap.
int np_rule(double x, int cap) {
  int last = 0;
  for (int m = 0; m < cap + 64; ++m)
    if (std::fabs(std::cyl_bessel_j((double)m, x)) >= 1e-15) last = m;
  int np = last + 1;
  return np < cap ? np : cap;
}

// out = U(sign * dt) psi = sum_{m<Np} (2 - delta_m0) (-sign i)^m J_m(dE dt) T_m(H~) psi (Eq. 17).
void evolve(const Ham& h, const cplx* psi, double dt, int sign, int Np, cplx* out) {
  const int64_t n = h.n;
  const double x = h.dE * dt;
  const cplx mi = (sign > 0) ? cplx(0.0, -1.0) : cplx(0.0, 1.0);
  std::vector<cplx> t0(psi, psi + n), t1(n), t2(n), ht(n);
  cplx phase = 1.0;  // (mi)^m
  for (int64_t i = 0; i < n; ++i) out[i] = std::cyl_bessel_j(0.0, x) * t0[i];
  if (Np > 1) {
    apply_Ht(h, t0.data(), t1.data());
    phase *= mi;
    cplx c = 2.0 * phase * std::cyl_bessel_j(1.0, x);
    for (int64_t i = 0; i < n; ++i) out[i] += c * t1[i];
  }
  for (int m = 2; m < Np; ++m) {
    apply_Ht(h, t1.data(), ht.data());
    for (int64_t i = 0; i < n; ++i) t2[i] = 2.0 * ht[i] - t0[i];
    phase *= mi;
    cplx c = 2.0 * phase * std::cyl_bessel_j((double)m, x);
    for (int64_t i = 0; i < n; ++i) out[i] += c * t2[i];
    t0.swap(t1);
    t1.swap(t2);
  }
}

// out = [X, U(dt)] psi = sum_{m<Np} (2 - delta_m0) (-i)^m J_m(dE dt) [X, T_m] psi (Eq. 18),
// with [X,T_0] = 0, [X,T_1] = [X,H~] (Eq. 24) and
// [X,T_m] = 2[X,H~]T_{m-1} + 2H~[X,T_{m-1}] - [X,T_{m-2}] (Eq. 22).
void commutator_evolve(const Ham& h, const cplx* psi, double dt, int Np, cplx* out) {
  const int64_t n = h.n;
  const double x = h.dE * dt;
  const cplx mi(0.0, -1.0);
  std::vector<cplx> u0(psi, psi + n), u1(n), u2(n);  // T_m psi
  std::vector<cplx> w0(n, 0.0), w1(n), w2(n);         // [X, T_m] psi
  std::vector<cplx> a(n), b(n);
  for (int64_t i = 0; i < n; ++i) out[i] = 0.0;  // m = 0 term: [X,T_0] = 0
  if (Np <= 1) return;
  apply_Ht(h, u0.data(), u1.data());
  apply_XHt(h, u0.data(), w1.data());
  cplx phase = mi;
  cplx c = 2.0 * phase * std::cyl_bessel_j(1.0, x);
  for (int64_t i = 0; i < n; ++i) out[i] += c * w1[i];
  for (int m = 2; m < Np; ++m) {
    apply_XHt(h, u1.data(), a.data());
    apply_Ht(h, w1.data(), b.data());
    for (int64_t i = 0; i < n; ++i) w2[i] = 2.0 * a[i] + 2.0 * b[i] - w0[i];
    apply_Ht(h, u1.data(), a.data());
    for (int64_t i = 0; i < n; ++i) u2[i] = 2.0 * a[i] - u0[i];
    phase *= mi;
    c = 2.0 * phase * std::cyl_bessel_j((double)m, x);
    for (int64_t i = 0; i < n; ++i) out[i] += c * w2[i];
    u0.swap(u1);
    u1.swap(u2);
    w0.swap(w1);
    w1.swap(w2);
  }
}

double jackson(int n, int M) {  // Eq. 31, alpha = 1/(N_m + 1)
  const double a = 1.0 / (M + 1.0);
  const double pi = M_PI;
  return (1.0 - n * a) * std::cos(pi * n * a) + a * std::sin(pi * n * a) / std::tan(pi * a);
}

}  // namespace

extern "C" {

struct orc_ham;

orc_ham* orc_ham_new(int64_t n, int K, const int32_t* cnt, const int32_t* idx, const double* hop_re,
                     const double* hop_im, const double* eps, const double* dx, double dE) {
  Ham* h = new Ham;
  h->n = n;
  h->K = K;
  h->cnt.assign(cnt, cnt + n);
  h->idx.assign(idx, idx + n * K);
  h->hop.resize(n * K);
  for (int64_t s = 0; s < n * K; ++s) h->hop[s] = cplx(hop_re[s], hop_im ? hop_im[s] : 0.0);
  h->eps.assign(eps, eps + n);
  h->dx.assign(dx, dx + n * K);
  h->dE = dE;
  return reinterpret_cast<orc_ham*>(h);
}

void orc_ham_free(orc_ham* h) { delete reinterpret_cast<Ham*>(h); }

static const Ham& H(const orc_ham* h) { return *reinterpret_cast<const Ham*>(h); }

// Vectors cross this interface as interleaved (re, im) doubles.
void orc_apply_ht(const orc_ham* h, const double* x, double* y) {
  apply_Ht(H(h), reinterpret_cast<const cplx*>(x), reinterpret_cast<cplx*>(y));
}
void orc_apply_v(const orc_ham* h, const double* x, double* y) {
  apply_V(H(h), reinterpret_cast<const cplx*>(x), reinterpret_cast<cplx*>(y));
}
void orc_cheb_moments(const orc_ham* h, const double* l, const double* r, int M, double* mu) {
  cheb_moments(H(h), reinterpret_cast<const cplx*>(l), reinterpret_cast<const cplx*>(r), M,
               reinterpret_cast<cplx*>(mu));
}
// C_n^DOS = <phi|T_n(H~)|phi> (Eq. 28), real part.
void orc_dos_moments(const orc_ham* h, const double* phi, int M, double* mu) {
  std::vector<cplx> c(M);
  cheb_moments(H(h), reinterpret_cast<const cplx*>(phi), reinterpret_cast<const cplx*>(phi), M, c.data());
  for (int m = 0; m < M; ++m) mu[m] = c[m].real();
}
int orc_np_rule(double x, int cap) { return np_rule(x, cap); }
void orc_bessel(double x, int count, double* J) {
  for (int m = 0; m < count; ++m) J[m] = std::cyl_bessel_j((double)m, x);
}
void orc_evolve(const orc_ham* h, const double* psi, double dt, int sign, int Np, double* out) {
  evolve(H(h), reinterpret_cast<const cplx*>(psi), dt, sign, Np, reinterpret_cast<cplx*>(out));
}
void orc_commutator_evolve(const orc_ham* h, const double* psi, double dt, int Np, double* out) {
  commutator_evolve(H(h), reinterpret_cast<const cplx*>(psi), dt, Np, reinterpret_cast<cplx*>(out));
}

// VAC moments C_n(t_k) = Re <phi|U(t_k) V T_n(H~) U(t_k)^dag V|phi> (Eq. 29) for
// t_k = dt_0 + ... + dt_{k-1}, k < Nt.  With a = U(-t)phi and b = U(-t) V phi the
// moment is Re <V a| T_n |b>; a and b advance by U(-dt_k) (Eq. 17, lower sign).
// Np[k] is the expansion length used for step k.  out is [Nt][M].
// a_io/b_io (may be NULL): on return the states after all Nt evolutions.
void orc_vac_moments(const orc_ham* hh, const double* phi, const double* dt, const int* Np, int Nt, int M,
                     double* out, double* a_io, double* b_io) {
  const Ham& h = H(hh);
  const int64_t n = h.n;
  std::vector<cplx> a(reinterpret_cast<const cplx*>(phi), reinterpret_cast<const cplx*>(phi) + n);
  std::vector<cplx> b(n), l(n), tmp(n), mu(M);
  apply_V(h, a.data(), b.data());
  for (int k = 0; k < Nt; ++k) {
    apply_V(h, a.data(), l.data());
    cheb_moments(h, l.data(), b.data(), M, mu.data());
    for (int m = 0; m < M; ++m) out[(int64_t)k * M + m] = mu[m].real();
    evolve(h, a.data(), dt[k], -1, Np[k], tmp.data());
    a.swap(tmp);
    evolve(h, b.data(), dt[k], -1, Np[k], tmp.data());
    b.swap(tmp);
  }
  if (a_io) std::memcpy(a_io, a.data(), n * sizeof(cplx));
  if (b_io) std::memcpy(b_io, b.data(), n * sizeof(cplx));
}

// MSD moments C_n(t_k) = <phi|[X,U(t_k)]^dag T_n(H~) [X,U(t_k)]|phi> (Eq. 30) at
// t_k = dt_0 + ... + dt_{k-1}, k = 1..Nt (row k-1).  With p = U(t) phi and
// p_X = [X,U(t)] phi, one step is p_X <- [X,U(dt)] p + U(dt) p_X, p <- U(dt) p
// (Eqs. 17, 18).  out is [Nt][M] (real part; the imaginary part vanishes by
// hermiticity).
void orc_msd_moments(const orc_ham* hh, const double* phi, const double* dt, const int* Np, int Nt, int M,
                     double* out, double* p_io, double* px_io) {
  const Ham& h = H(hh);
  const int64_t n = h.n;
  std::vector<cplx> p(reinterpret_cast<const cplx*>(phi), reinterpret_cast<const cplx*>(phi) + n);
  std::vector<cplx> px(n, 0.0), xu(n), upx(n), up(n), mu(M);
  for (int k = 0; k < Nt; ++k) {
    commutator_evolve(h, p.data(), dt[k], Np[k], xu.data());
    evolve(h, px.data(), dt[k], +1, Np[k], upx.data());
    evolve(h, p.data(), dt[k], +1, Np[k], up.data());
    for (int64_t i = 0; i < n; ++i) px[i] = xu[i] + upx[i];
    p.swap(up);
    cheb_moments(h, px.data(), px.data(), M, mu.data());
    for (int m = 0; m < M; ++m) out[(int64_t)k * M + m] = mu[m].real();
  }
  if (p_io) std::memcpy(p_io, p.data(), n * sizeof(cplx));
  if (px_io) std::memcpy(px_io, px.data(), n * sizeof(cplx));
}

void orc_jackson(int M, double* g) {
  for (int n = 0; n < M; ++n) g[n] = jackson(n, M);
}

// Kernel-polynomial reconstruction (Eqs. 25-27 with the Jackson damping of
// Eq. 31): out[r][e] = 2 (N/Omega) / (pi dE sqrt(1 - E~^2))
//                       * sum_n g_n (2 - delta_n0) T_n(E~) mu[r][n],
// E~ = E/dE, T_n(x) = cos(n arccos x).  Energies with |E~| >= 1 give NaN
// (the square root of a negative number the paper warns about).
void orc_kpm_reconstruct(const double* mu, int rows, int M, const double* E, int NE, double dE,
                         double n_over_omega, double* out) {
  std::vector<double> g(M);
  for (int n = 0; n < M; ++n) g[n] = jackson(n, M);
  for (int e = 0; e < NE; ++e) {
    const double x = E[e] / dE;
    for (int r = 0; r < rows; ++r) {
      if (!(std::fabs(x) < 1.0)) {
        out[(int64_t)r * NE + e] = NAN;
        continue;
      }
      double s = 0.0;
      const double th = std::acos(x);
      for (int n = 0; n < M; ++n) s += g[n] * (n == 0 ? 1.0 : 2.0) * std::cos(n * th) * mu[(int64_t)r * M + n];
      out[(int64_t)r * NE + e] = 2.0 * n_over_omega / (M_PI * dE * std::sqrt(1.0 - x * x)) * s;
    }
  }
}

// Running conductivity from the VAC (Eq. 2): sigma(t_k) = integral_0^{t_k} rho C_vv dt,
// trapezoid rule over the rows at t_0 = 0 .. t_{Nt-1}; vac is [Nt][NE], out [Nt][NE].
void orc_sigma_vac(const double* vac, const double* dt, int Nt, int NE, double* out) {
  for (int e = 0; e < NE; ++e) out[e] = 0.0;
  for (int k = 1; k < Nt; ++k)
    for (int e = 0; e < NE; ++e)
      out[(int64_t)k * NE + e] =
          out[(int64_t)(k - 1) * NE + e] +
          0.5 * dt[k - 1] * (vac[(int64_t)(k - 1) * NE + e] + vac[(int64_t)k * NE + e]);
}

// Running conductivity from the MSD (Eq. 5): sigma(t_{k-1/2}) = (1/2) d(rho dX^2)/dt,
// finite difference over the rows at t_1 .. t_Nt with rho dX^2(0) = 0.
void orc_sigma_msd(const double* msd, const double* dt, int Nt, int NE, double* out) {
  for (int k = 0; k < Nt; ++k)
    for (int e = 0; e < NE; ++e) {
      double prev = (k == 0) ? 0.0 : msd[(int64_t)(k - 1) * NE + e];
      out[(int64_t)k * NE + e] = (msd[(int64_t)k * NE + e] - prev) / (2.0 * dt[k]);
    }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Reverse-mode derivatives.  Not part of the paper: they differentiate the
// paper's moments (Eqs. 17, 21, 29, 34) with respect to the Hamiltonian.
//
// For J = Re sum_m <lambda_m| T_m(H~) |r> with u_m = T_m(H~) r, the adjoint
// vectors w_m = lambda_m + 2 H~ w_{m+1} - w_{m+2} (m = M-1..1, w_M = w_{M+1} = 0)
// give dJ = Re sum_ij conj(Gt_ij) dH~_ij with Gt = w_1 u_0^+ + 2 sum_{m>=2} w_m u_{m-1}^+
// and dJ/dr = lambda_0 + H~ w_1 - w_2 (as the vector rbar with dJ = Re <rbar|dr>).
// Gt is only needed on the diagonal and on the neighbour-list slots; with H~ = H/dE
// (dE held fixed) the unscaled derivatives are Gt/dE.
// ---------------------------------------------------------------------------
namespace {

struct Grad {
  std::vector<double> eps;  // dJ/dU_i
  std::vector<cplx> slot;   // G_{i, idx_ik} (unscaled), dJ = Re sum conj(G) dH
};

// lam[m] = coefficient of <.|T_m r>; lam_vec is the common vector; so
// lambda_m = conj(coef[m]) * lam_vec.
void poly_adjoint(const Ham& h, const cplx* coef, int M, const cplx* lam_vec, const cplx* r, Grad& g, cplx* rbar) {
  const int64_t n = h.n;
  std::vector<std::vector<cplx>> u(M, std::vector<cplx>(n));
  for (int64_t i = 0; i < n; ++i) u[0][i] = r[i];
  if (M > 1) apply_Ht(h, u[0].data(), u[1].data());
  std::vector<cplx> ht(n);
  for (int m = 2; m < M; ++m) {
    apply_Ht(h, u[m - 1].data(), ht.data());
    for (int64_t i = 0; i < n; ++i) u[m][i] = 2.0 * ht[i] - u[m - 2][i];
  }
  std::vector<cplx> w1(n, 0.0), w2(n, 0.0), w(n);  // w_{m+1}, w_{m+2}, w_m
  for (int m = M - 1; m >= 1; --m) {
    apply_Ht(h, w1.data(), ht.data());
    const cplx lc = std::conj(coef[m]);
    for (int64_t i = 0; i < n; ++i) w[i] = lc * lam_vec[i] + 2.0 * ht[i] - w2[i];
    const double f = (m == 1 ? 1.0 : 2.0) / h.dE;
    const std::vector<cplx>& up = u[m - 1];
    for (int64_t i = 0; i < n; ++i) {
      g.eps[i] += f * (w[i] * std::conj(up[i])).real();
      for (int k = 0; k < h.cnt[i]; ++k) {
        int64_t j = h.idx[i * h.K + k];
        g.slot[i * h.K + k] += f * w[i] * std::conj(up[j]);
      }
    }
    w2.swap(w1);
    w1.swap(w);
  }
  // now w1 = w_1, w2 = w_2
  if (rbar) {
    apply_Ht(h, w1.data(), ht.data());
    const cplx lc0 = std::conj(coef[0]);
    for (int64_t i = 0; i < n; ++i) rbar[i] = lc0 * lam_vec[i] + (M > 1 ? ht[i] - w2[i] : cplx(0.0));
  }
}

// Contribution of l = V x to dJ given lbar (dJ = Re <lbar|dl>):
// dV_ij = i dx_ij dH_ij, so G_ij += lbar_i (-i dx_ij) conj(x_j).
void velocity_adjoint(const Ham& h, const cplx* lbar, const cplx* x, Grad& g) {
  const cplx mI(0.0, -1.0);
  for (int64_t i = 0; i < h.n; ++i)
    for (int k = 0; k < h.cnt[i]; ++k) {
      int64_t j = h.idx[i * h.K + k];
      g.slot[i * h.K + k] += lbar[i] * mI * h.dx[i * h.K + k] * std::conj(x[j]);
    }
}

void evolve_coefs(double x, int sign, int Np, cplx* c) {  // Eq. 17 coefficients
  const cplx mi = (sign > 0) ? cplx(0.0, -1.0) : cplx(0.0, 1.0);
  cplx phase = 1.0;
  for (int m = 0; m < Np; ++m) {
    c[m] = (m == 0 ? 1.0 : 2.0) * phase * std::cyl_bessel_j((double)m, x);
    phase *= mi;
  }
}

}  // namespace

extern "C" {

// Gradient of J = Re sum_m coef_m <l|T_m(H~)|r> (complex coef, interleaved).
// g_eps [N], g_slot [N*K] complex (interleaved), rbar [N] complex (may be NULL).
void orc_cheb_adjoint(const orc_ham* hh, const double* l, const double* r, const double* coef, int M,
                      double* g_eps, double* g_slot, double* rbar) {
  const Ham& h = H(hh);
  Grad g;
  g.eps.assign(h.n, 0.0);
  g.slot.assign(h.n * h.K, 0.0);
  poly_adjoint(h, reinterpret_cast<const cplx*>(coef), M, reinterpret_cast<const cplx*>(l),
               reinterpret_cast<const cplx*>(r), g, reinterpret_cast<cplx*>(rbar));
  std::memcpy(g_eps, g.eps.data(), h.n * sizeof(double));
  std::memcpy(g_slot, g.slot.data(), h.n * h.K * sizeof(cplx));
}

// Loss J = sum_k sum_n beta[k][n] C_n^VAC(t_k) (Eq. 29 moments, as in
// orc_vac_moments) and its gradient with respect to the unscaled on-site
// energies (g_eps [N]) and the unscaled slot hoppings (g_slot [N*K] complex,
// dJ = Re sum conj(g_slot) dH_slot, every slot treated as independent; the
// velocity operator's dependence on H (Eq. 34) is included, dE is fixed).
double orc_vac_loss_grad(const orc_ham* hh, const double* phi_, const double* dt, const int* Np, int Nt, int M,
                         const double* beta, double* g_eps, double* g_slot) {
  const Ham& h = H(hh);
  const int64_t n = h.n;
  const cplx* phi = reinterpret_cast<const cplx*>(phi_);
  std::vector<std::vector<cplx>> A(Nt, std::vector<cplx>(n)), B(Nt, std::vector<cplx>(n));
  std::vector<cplx> l(n), tmp(n), mu(M);
  for (int64_t i = 0; i < n; ++i) A[0][i] = phi[i];
  apply_V(h, phi, B[0].data());
  double loss = 0.0;
  for (int k = 0; k < Nt; ++k) {
    apply_V(h, A[k].data(), l.data());
    cheb_moments(h, l.data(), B[k].data(), M, mu.data());
    for (int m = 0; m < M; ++m) loss += beta[(int64_t)k * M + m] * mu[m].real();
    if (k + 1 < Nt) {
      evolve(h, A[k].data(), dt[k], -1, Np[k], A[k + 1].data());
      evolve(h, B[k].data(), dt[k], -1, Np[k], B[k + 1].data());
    }
  }
  Grad g;
  g.eps.assign(n, 0.0);
  g.slot.assign(n * h.K, 0.0);
  std::vector<cplx> abar(n, 0.0), bbar(n, 0.0), na(n), nb(n), lbar(n), cb(M);
  std::vector<cplx> ones(M);
  for (int k = Nt - 1; k >= 0; --k) {
    // through a_{k+1} = U(-dt_k) a_k and b_{k+1} = U(-dt_k) b_k
    if (k + 1 < Nt) {
      std::vector<cplx> c(Np[k]);
      evolve_coefs(h.dE * dt[k], -1, Np[k], c.data());
      // J = Re sum_m c_m <abar|T_m a>  ->  coefficient conj(c_m) on <abar| form:
      // poly_adjoint takes lambda_m = conj(coef_m) * vec, so pass coef = c.
      poly_adjoint(h, c.data(), Np[k], abar.data(), A[k].data(), g, na.data());
      poly_adjoint(h, c.data(), Np[k], bbar.data(), B[k].data(), g, nb.data());
      abar.swap(na);
      bbar.swap(nb);
    } else {
      std::fill(abar.begin(), abar.end(), cplx(0.0));
      std::fill(bbar.begin(), bbar.end(), cplx(0.0));
    }
    // KPM term: J_k = Re sum_n beta_n <l_k|T_n|b_k>
    apply_V(h, A[k].data(), l.data());
    for (int m = 0; m < M; ++m) cb[m] = beta[(int64_t)k * M + m];
    poly_adjoint(h, cb.data(), M, l.data(), B[k].data(), g, nb.data());
    for (int64_t i = 0; i < n; ++i) bbar[i] += nb[i];
    // lbar = sum_n beta_n T_n b_k  (real beta)
    // lbar = sum_n beta_n T_n b_k (forward recursion on b_k)
    {
      std::vector<cplx> t0(B[k]), t1(n), t2(n), ht(n);
      for (int64_t i = 0; i < n; ++i) lbar[i] = cb[0].real() * t0[i];
      if (M > 1) {
        apply_Ht(h, t0.data(), t1.data());
        for (int64_t i = 0; i < n; ++i) lbar[i] += cb[1].real() * t1[i];
      }
      for (int m = 2; m < M; ++m) {
        apply_Ht(h, t1.data(), ht.data());
        for (int64_t i = 0; i < n; ++i) t2[i] = 2.0 * ht[i] - t0[i];
        for (int64_t i = 0; i < n; ++i) lbar[i] += cb[m].real() * t2[i];
        t0.swap(t1);
        t1.swap(t2);
      }
    }
    // l_k = V a_k
    velocity_adjoint(h, lbar.data(), A[k].data(), g);
    apply_V(h, lbar.data(), tmp.data());
    for (int64_t i = 0; i < n; ++i) abar[i] += tmp[i];
  }
  // b_0 = V phi
  velocity_adjoint(h, bbar.data(), phi, g);
  std::memcpy(g_eps, g.eps.data(), n * sizeof(double));
  std::memcpy(g_slot, g.slot.data(), n * h.K * sizeof(cplx));
  return loss;
}

}  // extern "C"

// ---------------------------------------------------------------- Hall conductivity
// Beyond the paper's diagonal conductivity: the paper names the Hall
// conductivity of the Kubo-Bastin formula (Garcia, Covaci, Rappoport 2015) as
// computable in the same Chebyshev framework (Sec. 6).  Definitions used here:
//  * velocity along a direction with bond displacements d (d_ik = Y_idx - Y_i,
//    minimum image), in units of dE/hbar: v~ = i d o H~, i.e.
//    (v~ x)_i = i sum_k d_ik H~_{i,idx} x_idx  (the v = i[H, X]/hbar of Eq. 34
//    divided by dE, along that direction);
//  * Lambda_mn = Tr[v~_a T_m(H~) v~_b T_n(H~)] (Kubo-Bastin moments);
//  * sigma_ab(mu)/(e^2/h) = (2/Omega) int_{-1}^{mu/dE} dx F(x),
//    F(x) = (1 - x^2)^{-2} Re sum_mn c_m c_n g_m g_n Gamma_mn(x) Lambda_mn,
//    Gamma_mn(x) = T_m(x) e^{-i n th} (x + i n sin th) + T_n(x) e^{i m th} (x - i m sin th),
//    x = cos th, c_0 = 1, c_n = 2 (n > 0), g_n the Jackson factors (Eq. 31):
//    the Kubo-Bastin formula at zero temperature with the Chebyshev series of
//    delta(x - H~) and of the derivative of (x - H~ +- i0)^{-1} inserted.
namespace {

void apply_vd(const Ham& h, const double* d, const cplx* x, cplx* y) {
  const cplx I(0.0, 1.0);
  for (int64_t i = 0; i < h.n; ++i) {
    cplx s = 0.0;
    for (int k = 0; k < h.cnt[i]; ++k) {
      int64_t j = h.idx[i * h.K + k];
      s += I * d[i * h.K + k] * (h.hop[i * h.K + k] / h.dE) * x[j];
    }
    y[i] = s;
  }
}

// F(x_j) = (1 - x^2)^{-2} Re sum_mn c_m c_n g_m g_n Gamma_mn(x) Lambda_mn at x_j = E_j/dE.
std::vector<double> kb_integrand(const double* lam, int M, const double* E, int NE, double dE, int kernel) {
  const cplx I(0.0, 1.0);
  std::vector<double> w(M);
  for (int n = 0; n < M; ++n) w[n] = (n == 0 ? 1.0 : 2.0) * (kernel == 0 ? jackson(n, M) : 1.0);
  std::vector<double> F(NE);
  for (int j = 0; j < NE; ++j) {
    const double x = E[j] / dE;
    const double th = std::acos(x);
    const double s = std::sin(th);
    cplx acc = 0.0;
    for (int m = 0; m < M; ++m)
      for (int n = 0; n < M; ++n) {
        const cplx g = std::cos(m * th) * std::exp(-I * (double)n * th) * (x + I * (double)n * s) +
                       std::cos(n * th) * std::exp(I * (double)m * th) * (x - I * (double)m * s);
        const cplx l(lam[2 * ((size_t)m * M + n)], lam[2 * ((size_t)m * M + n) + 1]);
        acc += w[m] * w[n] * g * l;
      }
    F[j] = acc.real() / ((1.0 - x * x) * (1.0 - x * x));
  }
  return F;
}

// T_0 x .. T_{M-1} x by the three-term recursion (Eq. 21).
std::vector<std::vector<cplx>> cheb_vectors(const Ham& h, const cplx* x, int M) {
  std::vector<std::vector<cplx>> T(M, std::vector<cplx>(h.n));
  if (M > 0) T[0].assign(x, x + h.n);
  if (M > 1) apply_Ht(h, T[0].data(), T[1].data());
  std::vector<cplx> hx(h.n);
  for (int m = 2; m < M; ++m) {
    apply_Ht(h, T[m - 1].data(), hx.data());
    for (int64_t i = 0; i < h.n; ++i) T[m][i] = 2.0 * hx[i] - T[m - 2][i];
  }
  return T;
}

}  // namespace

extern "C" {

// Lambda_mn estimated as (N/R) sum_r <r| v~_a T_m v~_b T_n |r> over unit-norm
// vectors r (R vectors, r[q*n + i]); with v~_a and T_m Hermitian,
// <r| v~_a T_m = (T_m v~_a r)^dagger, so Lambda_mn = (N/R) sum_r <P_m | B_n>,
// P_m = T_m (v~_a r), B_n = v~_b T_n r.  lam: [M][M] complex (row m).
void orc_kb_moments(const orc_ham* hp, const double* d_a, const double* d_b, const double* r, int R, int M,
                    double* lam) {
  const Ham& h = H(hp);
  std::vector<cplx> L((size_t)M * M, cplx(0.0, 0.0));
  std::vector<cplx> u(h.n);
  for (int q = 0; q < R; ++q) {
    const cplx* rq = reinterpret_cast<const cplx*>(r) + (size_t)q * h.n;
    apply_vd(h, d_a, rq, u.data());
    std::vector<std::vector<cplx>> P = cheb_vectors(h, u.data(), M);
    std::vector<std::vector<cplx>> Tn = cheb_vectors(h, rq, M);
    std::vector<std::vector<cplx>> B(M, std::vector<cplx>(h.n));
    for (int n = 0; n < M; ++n) apply_vd(h, d_b, Tn[n].data(), B[n].data());
    for (int m = 0; m < M; ++m)
      for (int n = 0; n < M; ++n) {
        cplx s = 0.0;
        for (int64_t i = 0; i < h.n; ++i) s += std::conj(P[m][i]) * B[n][i];
        L[(size_t)m * M + n] += s;
      }
  }
  const double scale = (double)h.n / R;
  for (size_t t = 0; t < L.size(); ++t) {
    lam[2 * t] = scale * L[t].real();
    lam[2 * t + 1] = scale * L[t].imag();
  }
}

// sigma_ab(E_j)/(e^2/h) for ascending energies E_0 < .. < E_{NE-1} inside
// (-dE, dE): F(x) at x_j = E_j/dE, then the trapezoid rule from x_0 (the lower
// integration limit, below the spectrum) to x_j; sigma_0 = 0.  kernel 0 =
// Jackson, 1 = none.  area = Omega.
void orc_kubo_bastin(const double* lam, int M, const double* E, int NE, double dE, double area, int kernel,
                     double* sigma) {
  const std::vector<double> F = kb_integrand(lam, M, E, NE, dE, kernel);
  double run = 0.0;
  for (int j = 0; j < NE; ++j) {
    if (j > 0) run += 0.5 * (E[j] - E[j - 1]) / dE * (F[j] + F[j - 1]);
    sigma[j] = 2.0 / area * run;
  }
}

}  // extern "C"

extern "C" {

// Finite-temperature Hall conductivity: sigma_ab(mu_j, T)/(e^2/h) =
// (2/Omega) int dx f((E - mu_j)/kT) F(x), f(u) = 1/(1 + e^u) the Fermi function,
// with F(x) as in orc_kubo_bastin on the ascending energy grid E (the trapezoid
// rule over the grid; kT in the units of E, kT = 0 the step function with
// f(0) = 1/2).
void orc_kubo_bastin_fermi(const double* lam, int M, const double* E, int NE, double dE, double area, int kernel,
                           const double* mu, int Nmu, double kT, double* sigma) {
  const std::vector<double> F = kb_integrand(lam, M, E, NE, dE, kernel);
  for (int q = 0; q < Nmu; ++q) {
    auto fermi = [&](double e) {
      if (kT <= 0.0) return e < mu[q] ? 1.0 : (e > mu[q] ? 0.0 : 0.5);
      return 1.0 / (1.0 + std::exp((e - mu[q]) / kT));
    };
    double run = 0.0;
    for (int j = 1; j < NE; ++j)
      run += 0.5 * (E[j] - E[j - 1]) / dE * (fermi(E[j]) * F[j] + fermi(E[j - 1]) * F[j - 1]);
    sigma[q] = 2.0 / area * run;
  }
}

}  // extern "C"
