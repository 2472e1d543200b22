/*
 * gqt.h -- C ABI of the GB300 library for linear-scaling Kubo transport.
 *
 * The method is that of Fan, Vierimaa and Harju, "GPUQT: An efficient
 * linear-scaling quantum transport code fully implemented on graphics
 * processing units" (arXiv:1705.01387): Chebyshev moments of a sparse
 * tight-binding Hamiltonian applied to random-phase vectors (Sec. 3.1, 3.3),
 * Chebyshev-Bessel time evolution (Sec. 3.2) and the kernel polynomial method
 * (Eqs. 25-31), giving the DOS, the velocity autocorrelation (VAC) and the mean
 * square displacement (MSD), and from them the running conductivity.
 *
 * Conventions for every entry point
 * ---------------------------------
 *  * Units: hbar = e = 1.  H~ = H / dE and dt~ = dE * dt (Eqs. 19-20); dE is
 *    the handle's energy scale.
 *  * Device vectors are caller-owned, contiguous, site-major: element (i, r)
 *    of R vectors sits at index i*R + r.  A vector element is complex:
 *    two doubles (re, im) for a GQT_FP64 handle, two floats for a
 *    GQT_FP32_ACC64 handle.  R must be 1, 2, 4, 8, 16 or 32.
 *  * Random vectors are normalised to 1 per segment (the paper normalises
 *    <phi|phi> = N, Eq. 13; every moment here is the paper's C_n divided by the
 *    segment's site count, and gqt_kpm_reconstruct restores the factor).
 *  * Moment outputs are FP64 and may be host or device memory: a host pointer
 *    makes the call copy the result back and synchronise the stream before it
 *    returns; a device pointer leaves the call asynchronous on the stream.
 *  * "stream" is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  All device work of a call is ordered on that stream.  Calls on
 *    one handle must not run concurrently (the handle owns its workspace).
 *  * No entry point aborts, traps or prints.  Errors return a non-zero
 *    gqt_status and leave a message for gqt_last_error() (thread-local).
 *    Device-side checks (moment bound, norm, NaN) are read back at the end of
 *    the call that made them.
 */
#ifndef GQT_H
#define GQT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GQT_OK = 0,
  GQT_EINVAL = 1,   /* bad argument: size, pointer, non-Hermitian input, index out of range */
  GQT_ENOMEM = 2,   /* device or host allocation failed */
  GQT_ECUDA = 3,    /* a CUDA runtime call failed (message holds the CUDA error string) */
  GQT_ERANGE = 4,   /* |mu_m| > |l||r|(1+1e-6): spectrum of H/dE outside [-1,1], dE too small (Sec. 4.2 para.in) */
  GQT_ENORM = 5,    /* | |U psi| - |psi| | above tolerance after an evolution step */
  GQT_ENAN = 6,     /* NaN or Inf met in an input or a result */
  GQT_ETIMEOUT = 7  /* a bounded device wait gave up */
} gqt_status;

typedef enum { GQT_FP64 = 0, GQT_FP32_ACC64 = 1 } gqt_precision;

typedef enum {
  GQT_LATTICE_CUSTOM = 0,    /* the paper's input form (neighbour list etc., Sec. 4.2) */
  GQT_LATTICE_CHAIN = 1,     /* periodic chain, L1 sites, slots +x, -x */
  GQT_LATTICE_SQUARE = 2,    /* periodic L1 x L2 square lattice, slots +x, -x, +y, -y */
  GQT_LATTICE_HONEYCOMB = 3, /* periodic L1 x L2 honeycomb cells (2 sites), C-C distance 1 */
  GQT_LATTICE_CUBIC = 4      /* periodic L1^3 simple cubic, slots +x, -x, +y, -y, +z, -z */
} gqt_lattice_kind;

/* A tight-binding model (Eq. 32) with positions along the transport direction (Eq. 33).
 * For the built-in kinds the library generates the lattice itself: hopping t on
 * every bond, on-site energies W*(u - 1/2) with u from the SplitMix64 stream 1 of
 * seed, and round(vacancy_frac*N) vacancies (all bonds of the site with the
 * smallest draws of stream 2 zeroed).  For GQT_LATTICE_CUSTOM, the host arrays
 * below are read (row-major [n][max_nb]); hop_im may be NULL (real hoppings),
 * onsite may be NULL (zero), hop_re may be NULL (every listed bond -1, as the
 * paper's default when hopping.in is absent).  bond_dx[i][k] = X_j - X_i for
 * the bond to j = nb_idx[i][k], taken as the minimum image under periodic
 * boundaries (Eq. 34).  Slots k >= nb_count[i] are ignored. */
typedef struct {
  int kind;
  int64_t L1, L2, L3;
  double t;
  double W;
  double vacancy_frac;
  uint64_t seed;
  int64_t n;
  int max_nb;
  const int32_t* nb_count;
  const int32_t* nb_idx;
  const double* hop_re;
  const double* hop_im;
  const double* onsite;
  const double* bond_dx;
  double length_x;
  double volume;
  const double* bond_dy; /* optional (may be NULL): y displacements [n][max_nb], same
                            rules as bond_dx; needed only by the Hall moments */
} gqt_lattice;

typedef struct gqt_ham gqt_ham;

/* Build H~ = H/dE on the current CUDA device in ELL form (slot-major arrays,
 * Sec. 4.2 neighbour list; Eqs. 19, 32-34).  energy_scale <= 0 selects
 * dE = 1.05 * max_i (|U_i| + sum_k |H_ik|) (Gershgorin bound with 5% margin).
 * seg_offsets (host, nseg+1 ascending entries from 0 to n) declares a block-
 * diagonal batch of independent realisations; NULL / nseg <= 1 means one.
 * Moments are then reduced per segment.  The input must be Hermitian:
 * H_ji = conj(H_ij) and dx_ji = -dx_ij for every listed bond (EINVAL
 * otherwise), bonds may not cross segments, and indices must lie in [0, n).
 * On success *out owns the device arrays until gqt_free_hamiltonian. */
gqt_status gqt_build_hamiltonian(const gqt_lattice* lattice, double energy_scale, gqt_precision precision,
                                 const int64_t* seg_offsets, int nseg, gqt_ham** out);
void gqt_free_hamiltonian(gqt_ham* ham);

/* The model a built-in lattice kind generates, in the input form (row-major
 * [n][K] host arrays, caller-allocated; any output may be NULL).  Lets a
 * caller see exactly which H, positions and disorder gqt_build_hamiltonian
 * uploads for that kind. */
gqt_status gqt_generate_lattice(const gqt_lattice* lattice, int64_t* n, int* K, int32_t* nb_count, int32_t* nb_idx,
                                double* hop_re, double* hop_im, double* onsite, double* bond_dx, double* length_x,
                                double* volume);

/* n = sites, energy_scale = dE, volume = Omega, nseg = segments, hop_real = 1
 * when every hopping is real (the library then stores real hoppings). Any output
 * pointer may be NULL. */
gqt_status gqt_ham_info(const gqt_ham* ham, int64_t* n, double* energy_scale, double* volume, int* nseg,
                        int* precision, int* hop_real);

/* Storage forms the handle's rows can take, recognised when it is built (and
 * after gqt_update_hamiltonian), as bits of *flags:
 *   GQT_FORM_HONEYCOMB (1): the neighbour lists follow the built-in honeycomb
 *     cell layout (the temporally blocked rows, gqt_set_temporal_blocking);
 *   GQT_FORM_UNIFORM_HOP (2): FP64 handle whose slots all hold one real hopping
 *     (the Anderson form, disorder on the sites only): its blocked rows read no
 *     hop array and sum each row's neighbour values before one product;
 *   GQT_FORM_CUBIC_SWEEP (4): built-in simple-cubic lattice with the blocked
 *     sweep order (gqt_set_sweep_order).
 * The forms change the arithmetic order only; results agree with the general
 * kernels to rounding.  EINVAL on a null handle or flags. */
#define GQT_FORM_HONEYCOMB 1
#define GQT_FORM_UNIFORM_HOP 2
#define GQT_FORM_CUBIC_SWEEP 4
gqt_status gqt_ham_forms(const gqt_ham* ham, int* flags);

/* Random-phase vectors (Sec. 3.1, Eq. 13): phi[i*R + r] = exp(i 2 pi u)/sqrt(n_s),
 * u = top 53 bits of draw i of SplitMix64 stream (2^20 + first_vector + r) of
 * seed / 2^53, n_s = sites of i's segment.  d_phi: device, [n][R], the
 * handle's element type. */
gqt_status gqt_random_phase(const gqt_ham* ham, uint64_t seed, int first_vector, int R, void* d_phi, void* stream);

/* mu[s][r][m] = <l_r| T_m(H~) |r_r> restricted to segment s, m < M (Eqs. 21, 23;
 * Eq. 28 with l = r).  mu is complex: 2*nseg*R*M doubles, host or device.
 * d_l, d_r: device [n][R].  Fails with ERANGE if some |mu_m| exceeds
 * |l||r|(1 + 1e-6) (values are still written). */
gqt_status gqt_cheb_moments(gqt_ham* ham, const void* d_l, const void* d_r, int R, int M, double* mu, void* stream);

/* DOS moments C_n^DOS (Eq. 28): mu[s][r][m] = Re <phi|T_m(H~)|phi>, nseg*R*M doubles. */
gqt_status gqt_dos_moments(gqt_ham* ham, const void* d_phi, int R, int M, double* mu, void* stream);

/* In place psi <- U(sign*dt) psi (Eq. 17): sum over m < Np of
 * (2 - delta_m0) (-sign i)^m J_m(dE dt) T_m(H~) psi.  Np <= 0 selects
 * Np = 1 + max{m : |J_m(dE dt)| >= 1e-15} (machine precision, Sec. 3.2),
 * capped at 4096.  The Bessel sum accumulates in FP64.  norm (host, [nseg*R]
 * or NULL) receives |U psi| per segment and vector; the call fails with ENORM
 * if it differs from |psi| by more than 1e-10 (FP64) / 1e-5 (FP32). */
gqt_status gqt_evolve(gqt_ham* ham, void* d_psi, int R, double dt, int sign, int Np, double* norm, void* stream);

/* d_out = [X, U(dt)] d_psi (Eqs. 18, 22, 24), [X,H~]_ij = -dx_ij H~_ij; Np as in gqt_evolve. */
gqt_status gqt_commutator_evolve(gqt_ham* ham, const void* d_psi, void* d_out, int R, double dt, int Np,
                                 void* stream);

/* d_y = V d_x with V = i sum (X_n - X_m) H_mn |m><n| (Eq. 34).  d_x != d_y. */
gqt_status gqt_apply_velocity(gqt_ham* ham, const void* d_x, void* d_y, int R, void* stream);

/* VAC state set-up: d_a = phi, d_b = V phi. */
gqt_status gqt_vac_init(gqt_ham* ham, const void* d_phi, void* d_a, void* d_b, int R, void* stream);

/* VAC moments (Eq. 29).  On entry (d_a, d_b) = (U(-t) phi, U(-t) V phi) at some t;
 * for k < Nt: row k = Re <V a| T_n(H~) |b>, then a, b <- U(-dt[k]) (a, b).  So rows
 * are at t, t+dt_0, ..., and on return the state is at t + sum dt (resumable).
 * dt: host [Nt]; Np: host [Nt] or NULL (rule of gqt_evolve).
 * mu: [Nt][nseg][R][M] doubles, host or device.
 * d_a, d_b: both device or both host memory (pinned or pageable) [n][R]; host
 * state is copied to the device before the rows and back after them, inside the
 * call (two n R vectors of handle workspace). */
gqt_status gqt_vac_moments(gqt_ham* ham, void* d_a, void* d_b, int R, const double* dt, const int* Np, int Nt,
                           int M, double* mu, void* stream);

/* MSD state set-up: d_p = phi, d_px = 0. */
gqt_status gqt_msd_init(gqt_ham* ham, const void* d_phi, void* d_p, void* d_px, int R, void* stream);

/* MSD moments (Eq. 30).  On entry (d_p, d_px) = (U(t) phi, [X, U(t)] phi); for k < Nt:
 * px <- [X, U(dt_k)] p + U(dt_k) px, p <- U(dt_k) p (Eqs. 17-18), then row k =
 * Re <px| T_n(H~) |px>.  Rows are at t + dt_0, ..., t + sum dt.  Layout and host
 * state as VAC. */
gqt_status gqt_msd_moments(gqt_ham* ham, void* d_p, void* d_px, int R, const double* dt, const int* Np, int Nt,
                           int M, double* mu, void* stream);

/* Kernel-polynomial reconstruction (Eqs. 25-27, Jackson damping Eq. 31):
 * out[row][e] = 2 n_over_omega / (pi dE sqrt(1 - x^2)) * sum_{n<M} g_n (2 - delta_n0) T_n(x) mu[row][n],
 * x = E[e]/dE, g_n = (1 - n a) cos(pi n a) + a sin(pi n a) cot(pi a), a = 1/(M+1).
 * n_over_omega = N/Omega (sites per volume).  |x| >= 1 gives NaN.  kernel: 0 =
 * Jackson, 1 = none (g_n = 1).  d_mu [rows][M], d_E [NE], d_out [rows][NE]:
 * device FP64. */
gqt_status gqt_kpm_reconstruct(const double* d_mu, int rows, int M, const double* d_E, int NE, double energy_scale,
                               double n_over_omega, int kernel, double* d_out, void* stream);

/* Transpose of gqt_kpm_reconstruct: d_beta[n] = sum_e w[e] * (the coefficient of mu[n]
 * in out[e]), so that sum_e w[e] out[row][e] = sum_n d_beta[n] mu[row][n].  Turns an
 * energy-weighted loss on reconstructed DOS/VAC/MSD values into moment weights
 * (the beta of gqt_vac_loss_grad).  Energies with |E| >= dE must have w = 0.
 * d_E, d_w [NE], d_beta [M]: device FP64. */
gqt_status gqt_kpm_weights(int M, const double* d_E, int NE, const double* d_w, double energy_scale,
                           double n_over_omega, int kernel, double* d_beta, void* stream);

/* Moment weights of the loss L = sum_e w[e] sigma_VAC(E_e, t_K) over K+1 VAC rows at
 * t_0 = 0 .. t_K (dt: host [K]): sigma_VAC(t_K) is the trapezoid sum
 * sum_k c_k rho C_vv(t_k) (Eq. 2) with c_0 = dt_0/2, c_k = (dt_{k-1} + dt_k)/2,
 * c_K = dt_{K-1}/2, and rho C_vv is linear in the moments (gqt_kpm_weights), so
 * d_beta[k][n] = c_k * kw[n] (device FP64 [K+1][M]); feed it to gqt_vac_loss_grad. */
gqt_status gqt_sigma_vac_loss_weights(int M, const double* d_E, int NE, const double* d_w, double energy_scale,
                                      double n_over_omega, int kernel, const double* dt, int K, double* d_beta,
                                      void* stream);

/* Gradients of real (and imaginary) bond hoppings from the slot gradients of
 * gqt_vac_loss_grad (d_g_slot: device FP64 [n_slots][2], n_slots = n * max_nb):
 * bond b is the Hermitian pair of slots d_slot_a[b] and d_slot_b[b] (flat indices
 * i*max_nb + k, device int64); d_g_re[b] = Re(G_a + G_b), d_g_im[b] (may be NULL)
 * = Im(G_a) - Im(G_b).  A slot index outside [0, n_slots) is not read: that bond's
 * outputs are NaN.  Stream-ordered, asynchronous. */
gqt_status gqt_bond_gradients(const double* d_g_slot, long long n_slots, const long long* d_slot_a,
                              const long long* d_slot_b, int nbonds, double* d_g_re, double* d_g_im, void* stream);

/* Hall conductivity (Kubo-Bastin formula in the Chebyshev framework; the paper
 * names it as computable "within the same framework", Sec. 6, after Garcia,
 * Covaci and Rappoport 2015).  Kubo-Bastin moments
 *   Lambda_mn = Tr[v~_a T_m(H~) v~_b T_n(H~)],  m, n < M,
 * with v~ = i d o H~ the velocity along direction a (b) in units of dE/hbar
 * (d = bond_dx for 0, bond_dy for 1: (v~ x)_i = i sum_k d_ik H~_ik x_j),
 * estimated from R unit-norm vectors d_r [n][R] (FP64 complex, site-major) as
 * (N/R) sum_r <T_m v~_a r | v~_b T_n r>.  d_lambda: device FP64 complex
 * [M][M] (row m, interleaved re, im).  One segment only; direction 1 needs a
 * lattice with bond_dy.  FP64 handles take d_r complex128; FP32 handles
 * (GQT_FP32_ACC64) take complex64, run the chains in FP32 and need the
 * tensor-core contraction (gqt_set_kb_contraction(ham, 1)), else GQT_EINVAL.  Workspace of the handle:
 * 2 M N R + 3 N R complex vectors (the stacks T_m v~_a r and v~_b T_n r) plus
 * the split partial sums.  Synchronises the stream before returning. */
gqt_status gqt_kb_moments(gqt_ham* ham, const void* d_r, int R, int M, int alpha, int beta, double* d_lambda,
                          void* stream);

/* How gqt_kb_moments contracts the two stacks (default 0):
 * 0 = FP64 (complex FP64 GEMM on the FP64 pipe; Lambda to FP64 rounding);
 * 1 = split TF32 on the tcgen05 tensor cores: both stacks are rounded to pairs of
 *     TF32 numbers (hi + lo, about 22 bits), each product is hi*hi + hi*lo + lo*hi,
 *     accumulated in FP32 over splits of at most 8192 sites and summed in FP64
 *     (Lambda to about 1e-5 of its largest entries).  The chains run in the
 *     handle's precision (FP64, or FP32 for GQT_FP32_ACC64 handles, which
 *     require this mode).
 * Other values: GQT_EINVAL. */
gqt_status gqt_set_kb_contraction(gqt_ham* ham, int mode);

/* Polls of each bounded device wait of the handle's kernels (default 2^24, a
 * few tenths of a second to seconds; 0 = give up at once).  The only kernel
 * that waits is the tensor-core Hall contraction (gqt_set_kb_contraction mode
 * 1): its single issuing thread waits on mbarriers for the bulk tensor copies of
 * each stage and for the commit of the products that read a buffer.  A wait that
 * runs out stops the pipeline; the thread then drains what is in flight (the
 * last committed products and the issued copies, 2^24 polls each, independent of
 * this setting), frees its tensor memory and the call returns GQT_ETIMEOUT; the
 * moments it wrote are not valid.  The handle stays usable.  If the drain
 * itself gives up (the error message then says so), products or copies may still
 * be in flight when the CTA frees its tensor memory and exits: treat the CUDA
 * context as suspect and restart the process.  This is the library's failure
 * detection for a device wait that never completes (Sec. 4.2 names a too-small
 * energy scale as the method's failure mode; a stalled copy engine is the
 * hardware's).  polls < 0: GQT_EINVAL. */
gqt_status gqt_set_wait_limit(gqt_ham* ham, int polls);

/* sigma_ab(E_j) in units of e^2/h at zero temperature from Kubo-Bastin moments:
 *   sigma(E_j) = (2/area) int_{x_0}^{x_j} dx F(x),  x = E/dE = cos th,
 *   F(x) = (1 - x^2)^-2 Re sum_mn c_m c_n g_m g_n Gamma_mn(x) Lambda_mn,
 *   Gamma_mn(x) = T_m(x) e^{-i n th}(x + i n sin th) + T_n(x) e^{i m th}(x - i m sin th),
 * c_0 = 1, c_n = 2, g_n the Jackson factors (kernel 0; kernel 1: g_n = 1), the
 * integral by the trapezoid rule over the given energies (so E_0, the lower
 * limit, belongs below the spectrum and sigma(E_0) = 0).  d_E [NE] ascending
 * with |E| < dE, d_sigma [NE], d_lambda [M][M] complex: device FP64.  area =
 * Omega of the 2D sample (hbar = e = 1, lengths of bond_dx/bond_dy).  M <= 8192.
 * Synchronises the stream before returning. */
gqt_status gqt_kubo_bastin(const double* d_lambda, int M, const double* d_E, int NE, double energy_scale, double area,
                           int kernel, double* d_sigma, void* stream);

/* sigma_ab(mu_q, T) in units of e^2/h at temperature kT (same units as E):
 * (2/area) int dx f((E - mu_q)/kT) F(x) with F as in gqt_kubo_bastin and the
 * Fermi function f(u) = 1/(1 + e^u) (kT = 0: the step, 1/2 at E = mu), by the
 * trapezoid rule over the ascending grid d_E [NE] (NE >= 2, |E| < dE; it should
 * cover the spectrum and a few kT above the largest mu).  d_mu [Nmu], d_sigma
 * [Nmu], d_lambda [M][M] complex: device FP64.  Synchronises the stream. */
gqt_status gqt_kubo_bastin_fermi(const double* d_lambda, int M, const double* d_E, int NE, double energy_scale,
                                 double area, int kernel, const double* d_mu, int Nmu, double kT, double* d_sigma,
                                 void* stream);

/* Running conductivity from the VAC (Eq. 2): sigma[k][e] = sum_{j<k} dt[j] (v[j][e] + v[j+1][e]) / 2
 * over rows at t_0 = 0 .. t_{Nt-1} of rho*C_vv (device [Nt][NE]); dt host [Nt]. */
gqt_status gqt_sigma_vac(const double* d_vac, const double* dt, int Nt, int NE, double* d_sigma, void* stream);

/* Running conductivity from the MSD (Eq. 5): sigma[k][e] = (m[k][e] - m[k-1][e]) / (2 dt[k]),
 * m[-1] = 0, over rows at t_1 .. t_Nt of rho*dX^2 (device [Nt][NE]). */
gqt_status gqt_sigma_msd(const double* d_msd, const double* dt, int Nt, int NE, double* d_sigma, void* stream);

/* Reverse-mode gradient of J = sum_k sum_n beta[k][n] C_n^VAC(t_k) (Eq. 29 moments with
 * rows at t_0 = 0 .. t_{Nt-1}, one vector, one segment).  The paper has no
 * derivatives; this differentiates its VAC moments, including the dependence of
 * V on H (Eq. 34), with dE held fixed.  beta: host [Nt][M].  Outputs (device
 * FP64): d_g_onsite [n] = dJ/dU_i; d_g_slot [n][max_nb] complex G_ik with
 * dJ = Re sum conj(G_ik) dH_{i,idx(i,k)} over slots, every slot independent
 * (a real bond's hopping t_ij has dJ/dt = Re(G_ij + G_ji)).  *loss receives J.
 * Intermediate Chebyshev vectors are recomputed from checkpoints taken every
 * `stride` orders (stride <= 0: ceil(sqrt(M))).  beta may be host or device memory. */
gqt_status gqt_vac_loss_grad(gqt_ham* ham, const void* d_phi, const double* dt, const int* Np, int Nt, int M,
                             const double* beta, int stride, double* loss, double* d_g_onsite, double* d_g_slot,
                             void* stream);

/* New on-site energies (NULL: zero) and hoppings (hop_im NULL: real) for an
 * existing handle, row-major [n][max_nb] in the handle's neighbour order, with the
 * same neighbour list, positions, energy scale and precision.  Validated as in a
 * build (Hermitian, finite; EINVAL / ENAN) and uploaded into the same device
 * arrays, so workspace and captured graphs stay valid: repeated evaluations of
 * a loss at nearby parameters (finite differences, optimisation loops) reuse
 * them.  A handle built with real hoppings accepts only real ones. */
gqt_status gqt_update_hamiltonian(gqt_ham* ham, const double* onsite, const double* hop_re, const double* hop_im);

/* Host-side Bessel coefficients J_m(x), m < count (Miller backward recurrence
 * normalised by J_0 + 2 sum J_2k = 1), and the expansion-length rule used when
 * Np <= 0.  x >= 0. */
gqt_status gqt_bessel(double x, int count, double* J);
int gqt_np_rule(double x, int cap);

/* Kernel launch shape for a handle: threads per block and blocks per SM of the
 * Chebyshev kernels (0 = library default).  gqt_autotune times every variant x
 * threads x blocks-per-SM candidate (0, the per-kernel default, among them) on
 * zero-filled scratch vectors (a few Re <l|T_m|r> orders for the given R) and
 * keeps the fastest. */
gqt_status gqt_set_launch(gqt_ham* ham, int threads, int blocks_per_sm);
/* Moment-kernel variant: 0 = each CTA walks one contiguous chunk of sites; 1 =
 * wavefront order (the CTAs of a segment stride through it together, so
 * neighbour gathers hit in L2); 2 = wavefront with more work in flight per
 * thread: two sites per thread for R = 1; for R >= 2 (at most 128 threads per
 * CTA) consecutive vectors of one site per thread, sharing one load of its H~
 * row: 4 vectors (R >= 4) in l = r orders, 2 in l != r orders; 3 = as 2 with 2
 * vectors per thread everywhere.  Unless blocks_per_sm is set, each moment
 * launch uses exactly as many CTAs as fit on the GPU at once for its kernel.  Variants 1-2 cover 2, 3, 4 or 6 neighbour slots and up to 256
 * threads per CTA; otherwise variant 0 runs.  Default 2.  gqt_autotune also
 * chooses the variant. */
gqt_status gqt_set_variant(gqt_ham* ham, int variant);
gqt_status gqt_autotune(gqt_ham* ham, int R, int* threads, int* blocks_per_sm, int* variant, void* stream);

/* Cluster-resident moment rows (default 1): for R = 1 on a single segment, when
 * a row's two Chebyshev vectors, l and the H~ rows fit in the shared memory of
 * one thread-block cluster (16 CTAs where the GPU allows, else 8), the whole row
 * runs as one launch; vectors are exchanged through distributed shared memory
 * and orders are separated by hardware cluster barriers.  0 keeps the
 * one-launch-per-order path. */
gqt_status gqt_set_cluster(gqt_ham* ham, int enable);

/* Moment rows Re <l|T_m|r> with l != r (VAC rows, gqt_vac_moments) by two
 * recurrences at once (default 1): A_k = T_k l and B_k = T_k r give
 * mu_2k = 2 Re <A_k|B_k> - mu_0 and mu_2k+1 = 2 Re <A_k|B_k+1> - mu_1
 * (Chebyshev product identities, H~ Hermitian), so each step streams H~ once for
 * two moments.  Applies to the wavefront kernels, one element per thread or
 * the multi-vector form (not the chunk-ordered variant 0 or cluster rows).  0
 * runs one recurrence on r with a dot against l per order. */
gqt_status gqt_set_vac_pair(gqt_ham* ham, int enable);

/* Arithmetic of the moment rows of FP64 handles (GQT_FP64) with R = 1 (default 1):
 * 0 = FP64 fused multiply-adds;
 * 1 = pairs of FP32 numbers (hi + lo, about 48 significant bits; Dekker's and
 *     Knuth's error-free sums and products on the FP32 pipes): the two-recurrence
 *     VAC rows (gqt_vac_moments) and the l = r rows
 *     (gqt_dos_moments, gqt_msd_moments) of lattices with 2, 3, 4 or 6 neighbour
 *     slots.  Storage stays FP64-sized (16 bytes per complex element, the
 *     handle's vectors complex128); moments agree with the FP64 mode to about
 *     1e-12 of mu_0 at M = 3000.  GB300 issues 64 FP32 fused multiply-adds for
 *     each FP64 one, so mode 1 is bound by HBM instead of the FP64 pipe.  The
 *     first call in mode 1 splits 2H~ into pairs (K n (8 or 16) + 8 n bytes of
 *     device memory held by the handle).
 * Other values: GQT_EINVAL.  Evolution, velocity, adjoint and Hall kernels, and
 * R > 1 rows, always use the FP64 pipe. */
gqt_status gqt_set_fp64_arith(gqt_ham* ham, int mode);

/* Temporal blocking of the moment rows (Eq. 21 advanced two orders per
 * launch; default 1).  Applies to handles whose neighbour lists follow the
 * honeycomb cell layout of the built-in lattice (site 2(c1 + L1 c2) + s,
 * A(c1,c2) bonded to B(c1,c2), B(c1+1,c2-1), B(c1,c2-1), one slot order per
 * sublattice, every row with three neighbours; recognised when the handle is
 * built, vacancies included) with one segment: FP64 handles in paired-FP32 mode
 * with R = 1 and L1 a multiple of 32 cells, and FP32-storage handles with R = 2,
 * 4, 8 or 16 vectors (one band per 128/(R/2), 64/(R/2) or 32/(R/2) cells, the
 * largest dividing L1), run by the default multi-vector kernels.  Each CTA
 * walks a band of cells (128, 64 or 32 for the FP64 handles) down the rows: per
 * row it computes T_{m+1} from T_m and T_{m-1}, and T_{m+2} two rows behind from
 * the T_{m+1} rows it wrote just before (still in L2), so per two orders each
 * orbital's vectors and hoppings come from DRAM once and the index array is not
 * read (FP64 VAC rows 160 bytes per orbital instead of 280, l = r rows 96
 * instead of 184; FP32 VAC rows 64 + 16/R instead of 96 + 56/R).  Each CTA
 * recomputes the T_{m+1} values at its band's edges itself.  Results agree with
 * the single-order kernels to rounding (the chains are the same; the moment sums
 * are split over CTAs differently).  The handle holds two more vectors per
 * chain.  0 = one order per launch; other handles always run one order per
 * launch. */
gqt_status gqt_set_temporal_blocking(gqt_ham* ham, int enable);

/* Blocked sweep order of the multi-vector kernels (default 1; built-in simple-
 * cubic lattices whose side is a power of two >= 64): the CTAs walk the x-rows in
 * strips of 32 y-rows through all z before the next strip, so the +-z neighbour
 * tiles are re-read from L2 rather than DRAM once an xy-plane of the vectors no
 * longer fits there.  Results equal the natural order up to the summation order
 * of the moment dots.  0 walks the sites in index order. */
gqt_status gqt_set_sweep_order(gqt_ham* ham, int enable);

/* Use CUDA graphs for repeated loops (default 1). */
gqt_status gqt_set_graphs(gqt_ham* ham, int enable);

/* Per-kernel timing with CUDA events on the launch stream.  After
 * gqt_profile_start every launch of the Chebyshev kernels is bracketed by two
 * events; gqt_profile_stop waits for them and returns, per family, the summed
 * milliseconds and the launch count: 0 = first moment order, 1 = moment orders
 * m >= 2 with l != r (the fused SpMV + recurrence + dot kernel), 2 = one-set
 * evolution order, 3 = two-set evolution order, 4 = coupled commutator order,
 * 5 = moment steps m >= 2 with l = r (two moments per step), 6 = moment steps
 * m >= 2 of the two-recurrence l != r rows (two moments per step), 7 = Hall
 * chain orders (gqt_kb_moments), 8 = Hall moment contraction (the M x M
 * complex GEMM), 9 = Kubo-Bastin energy sums (gqt_kubo_bastin), 10 =
 * temporally blocked passes of the two-recurrence rows (two steps, four moments
 * per launch), 11 = temporally blocked passes of the l = r rows, 12 and 13 =
 * the same for FP32-storage handles with several vectors.  Graph
 * capture is bypassed while profiling. */
gqt_status gqt_profile_start(void);
gqt_status gqt_profile_stop(double* ms, uint64_t* launches, int ncat);

/* DOS moments (same result as gqt_dos_moments) for callers that cannot allocate
 * device memory: callers whose device memory belongs to another allocator (a
 * framework's caching pool, a fixed budget) that must not be bypassed, and
 * callers on latency-critical paths where cudaMalloc/cudaFree would synchronise
 * the device.  The paper has no counterpart; this is a deployment variant of the
 * fused moment kernel.  The call allocates nothing: its scratch (two Chebyshev
 * vectors, per-CTA partial sums, CTA table, status word) lives in one fixed
 * file-scope device array of GQT_NOALLOC_SCRATCH_BYTES bytes, which every GPU
 * that loads the library holds until the process exits.
 *  - Limit: 2*n*R*e + (max(M,2)+1)*nb*R*16 + a few KB must fit in the array
 *    (e = 16 bytes FP64 / 8 bytes FP32 per element, nb = min(2*SMs,
 *    ceil(n*R/1024)) CTAs); larger requests return GQT_EINVAL naming the size.
 *  - Single-segment handles only.  d_phi: device [n][R] of the handle's device;
 *    d_mu: DEVICE memory of the same device, nseg*R*M doubles
 *    (Re <phi|T_m|phi>); the handle must have been built earlier.  A host
 *    pointer or another device's pointer returns GQT_EINVAL.
 *  - The first call on a device (and the first after that device's context was
 *    destroyed and created again) looks up the array's device address on that
 *    device (cudaGetSymbolAddress); make that first call before any stream
 *    capture.
 *  - Every call shares the one array and it keeps the previous call's contents
 *    (the call re-initialises what must start at zero); calls whose GPU work
 *    overlaps (other streams, other threads) race on it and must be serialised.
 *  - The call waits for its stream before returning (status check). */
#define GQT_NOALLOC_SCRATCH_BYTES (4u << 20)
gqt_status gqt_dos_moments_noalloc(const gqt_ham* ham, const void* d_phi, int R, int M, double* d_mu, void* stream);

/* Measured FP64 fused-multiply-add throughput of the current GPU in GFLOP/s
 * (an FMA counts 2 flops): best of five timed launches of a kernel running 8
 * independent FMA chains per thread on every SM.  The peak of the FP64
 * arithmetic roofline. */
gqt_status gqt_probe_fp64(double* gflops, void* stream);

/* Number of kernel launches the library has enqueued since load (for accounting). */
uint64_t gqt_launch_count(void);

const char* gqt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GQT_H */
