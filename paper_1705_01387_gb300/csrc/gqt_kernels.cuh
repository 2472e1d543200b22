// gqt_kernels.cuh -- device kernels of the GB300 Kubo-transport library.
//
// Every kernel streams the Hamiltonian H~ (ELL, slot-major) and the vectors
// once per Chebyshev order; the grid is a fixed set of CTAs, each owning one
// contiguous range of sites that never crosses a segment boundary, so moment
// partial sums are per CTA and per segment and their final reduction is a
// fixed-order (deterministic) sum.
//
// Storage of the scaled Hamiltonian (Eqs. 19, 32):
//   idx  [K][n] int32      neighbour j of slot k of row i (padding: i itself)
//   hop2 [K][n] HT         2 * H~_{i,j}  (complex V, or real S when all hoppings are real)
//   diag2[n]    S          2 * U_i / dE
//   dx   [K][n] S          X_j - X_i (minimum image; 0 on padding)
// Storing 2H~ turns the Chebyshev step T_m = 2H~T_{m-1} - T_{m-2} (Eq. 21)
// into one fused multiply-add chain; T_1 = H~T_0 uses the exact factor 1/2.
//
// Vectors: [n][R], element (i, r) at i*R + r, complex V = double2 or float2.
#pragma once

// A translation unit that includes this file inside a namespace of its own
// includes these headers first, at file scope, and defines
// GQT_KERNELS_NO_SYSTEM_INCLUDES, so that no system declaration lands in its
// namespace.
#ifndef GQT_KERNELS_NO_SYSTEM_INCLUDES
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>
#endif

namespace gqt {

template <bool FP64>
struct Prec;
template <>
struct Prec<true> {
  using S = double;
  using V = double2;
};
template <>
struct Prec<false> {
  using S = float;
  using V = float2;
};

template <class S, bool CH>
struct HopT;
template <class S>
struct HopT<S, true> {
  using T = typename Prec<sizeof(S) == 8>::V;
};
template <class S>
struct HopT<S, false> {
  using T = S;
};

template <bool FP64, bool CH>
struct Ell {
  using S = typename Prec<FP64>::S;
  using HT = typename HopT<S, CH>::T;
  int n;
  int K;
  const int* __restrict__ idx;
  const HT* __restrict__ hop2;
  const S* __restrict__ diag2;
  const S* __restrict__ dx;
  // optional blocked sweep order of the multi-vector kernels for a simple-cubic
  // lattice of side L = 2^row_shift (0: sites in index order), see site_of
  int row_shift;
};

// Site visited at wave position w.  Blocked order (row_shift = log2 L > 0): the
// x-rows are walked in strips of 32 y-rows through all z, i.e. w = x + L (yy +
// 32 (z + L yb)) visits site x + L (32 yb + yy) + L^2 z.  Shifts and masks only.
template <class E>
__device__ __forceinline__ int site_of(const E& H, int w) {
  const int lx = H.row_shift;
  if (lx == 0) return w;
  const int m = (1 << lx) - 1;
  const int r = w >> lx, t = r >> 5;
  return (w & m) | ((((t >> lx) << 5) | (r & 31)) << lx) | ((t & m) << (2 * lx));
}

// ---------------------------------------------------------------- arithmetic

__device__ __forceinline__ double2 cmul_acc(double2 acc, double2 h, double2 t) {
  acc.x = fma(h.x, t.x, acc.x);
  acc.x = fma(-h.y, t.y, acc.x);
  acc.y = fma(h.x, t.y, acc.y);
  acc.y = fma(h.y, t.x, acc.y);
  return acc;
}
__device__ __forceinline__ double2 cmul_acc(double2 acc, double h, double2 t) {
  acc.x = fma(h, t.x, acc.x);
  acc.y = fma(h, t.y, acc.y);
  return acc;
}
__device__ __forceinline__ float2 cmul_acc(float2 acc, float2 h, float2 t) {
  acc.x = fmaf(h.x, t.x, acc.x);
  acc.x = fmaf(-h.y, t.y, acc.x);
  acc.y = fmaf(h.x, t.y, acc.y);
  acc.y = fmaf(h.y, t.x, acc.y);
  return acc;
}
__device__ __forceinline__ float2 cmul_acc(float2 acc, float h, float2 t) {
  acc.x = fmaf(h, t.x, acc.x);
  acc.y = fmaf(h, t.y, acc.y);
  return acc;
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cneg(double2 a) { return make_double2(-a.x, -a.y); }
__device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ double2 to_d2(double2 a) { return a; }
__device__ __forceinline__ double2 to_d2(float2 a) { return make_double2((double)a.x, (double)a.y); }
template <class V>
__device__ __forceinline__ V from_d2(double2 a);
template <>
__device__ __forceinline__ double2 from_d2<double2>(double2 a) {
  return a;
}
template <>
__device__ __forceinline__ float2 from_d2<float2>(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}

// acc += c * t with c complex double, t storage precision, acc double2.
template <class V>
__device__ __forceinline__ double2 cfma_d(double2 acc, double2 c, V t) {
  double2 td = to_d2(t);
  acc.x = fma(c.x, td.x, acc.x);
  acc.x = fma(-c.y, td.y, acc.x);
  acc.y = fma(c.x, td.y, acc.y);
  acc.y = fma(c.y, td.x, acc.y);
  return acc;
}

// Dot-product accumulators: conj(l) * t summed over a thread's elements.
// FP64: plain FMA chains.  FP32: the products and sums run in FP32 with the
// error-free transformations of Ogita, Rump and Oishi ("Accurate sum and dot
// product", SIAM J. Sci. Comput. 26, 2005: TwoProduct by fmaf, TwoSum); the
// compensated (hi, lo) pair becomes FP64 once per thread and the CTA and
// segment sums run in FP64.
template <class V>
struct DotAcc;

template <>
struct DotAcc<double2> {
  double2 s = make_double2(0.0, 0.0);
  __device__ __forceinline__ void add(double2 l, double2 t) {
    s.x = fma(l.x, t.x, s.x);
    s.x = fma(l.y, t.y, s.x);
    s.y = fma(l.x, t.y, s.y);
    s.y = fma(-l.y, t.x, s.y);
  }
  __device__ __forceinline__ void add_norm(double2 t) {  // |t|^2 into .x
    s.x = fma(t.x, t.x, s.x);
    s.x = fma(t.y, t.y, s.x);
  }
  __device__ __forceinline__ void add_re(double2 l, double2 t) {  // Re conj(l) t into .x
    s.x = fma(l.x, t.x, s.x);
    s.x = fma(l.y, t.y, s.x);
  }
  __device__ __forceinline__ double2 get() { return s; }
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

struct CompF {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_prod(float a, float b) {
    float p = a * b;
    float pe = fmaf(a, b, -p);
    float s, e;
    two_sum(hi, p, s, e);
    hi = s;
    lo += e + pe;
  }
  __device__ __forceinline__ void add_val(float v) {
    float s, e;
    two_sum(hi, v, s, e);
    hi = s;
    lo += e;
  }
};

// The (hi, lo) pair is converted to FP64 once per thread, in get(): the
// compensated sum of n products is accurate to about n * 2^-48 of the sum of
// their magnitudes (Dot2 bound), far below the FP32 rounding of the vectors,
// and FP32->FP64 conversions run on the narrow FP64 pipe, so converting per
// element would make the kernel FP64-bound.
template <>
struct DotAcc<float2> {
  CompF re, im;
  __device__ __forceinline__ void add(float2 l, float2 t) {
    re.add_prod(l.x, t.x);
    re.add_prod(l.y, t.y);
    im.add_prod(l.x, t.y);
    im.add_prod(-l.y, t.x);
  }
  // Real-valued terms (norms, Re conj(l) t): the element's value is formed with one
  // rounding (fmaf) and then added with TwoSum, so only the sum is compensated.
  __device__ __forceinline__ void add_norm(float2 t) { re.add_val(fmaf(t.x, t.x, t.y * t.y)); }
  __device__ __forceinline__ void add_re(float2 l, float2 t) { re.add_val(fmaf(l.x, t.x, l.y * t.y)); }
  __device__ __forceinline__ double2 get() {
    return make_double2((double)re.hi + (double)re.lo, (double)im.hi + (double)im.lo);
  }
};

// Dynamic shared memory for the CTA reductions: NV * (blockDim/32) * R double2.
__device__ __forceinline__ double2* dyn_smem() {
  extern __shared__ __align__(16) unsigned char gqt_smem_raw[];
  return reinterpret_cast<double2*>(gqt_smem_raw);
}

// Sum a per-thread double2 over the threads of a CTA that share the same
// vector index r (= threadIdx.x & (R-1)); thread r < R of the CTA then holds
// the CTA total for vector r.  blockDim.x is a multiple of 32, R divides 32.
template <int NV>
__device__ __forceinline__ void block_reduce_r(double2 (&v)[NV], int R, double2* smem /*[NV][warps][R]*/) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    for (int off = 16; off >= R; off >>= 1) {
      v[q].x += __shfl_xor_sync(0xffffffffu, v[q].x, off);
      v[q].y += __shfl_xor_sync(0xffffffffu, v[q].y, off);
    }
  }
  if (lane < R) {
#pragma unroll
    for (int q = 0; q < NV; ++q) smem[(q * nw + warp) * R + lane] = v[q];
  }
  __syncthreads();
  if ((int)threadIdx.x < R) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double2 s = make_double2(0.0, 0.0);
      for (int w = 0; w < nw; ++w) {
        double2 t = smem[(q * nw + w) * R + threadIdx.x];
        s.x += t.x;
        s.y += t.y;
      }
      v[q] = s;
    }
  }
}

// block_reduce_r for real values (Re dots and norms have no imaginary part): half
// the FP64 adds, which matters where the FP64 pipe bounds the kernel.
template <int NV>
__device__ __forceinline__ void block_reduce_rx(double (&v)[NV], int R, double* smem /*[NV][warps][R]*/) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q)
    for (int off = 16; off >= R; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
  if (lane < R) {
#pragma unroll
    for (int q = 0; q < NV; ++q) smem[(q * nw + warp) * R + lane] = v[q];
  }
  __syncthreads();
  if ((int)threadIdx.x < R) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += smem[(q * nw + w) * R + threadIdx.x];
      v[q] = t;
    }
  }
}

// y = sum_k hop2[k][i] * x[idx[k][i]*R + r] + diag2[i] * x[i*R + r]  (= 2 H~ x, element (i, r)).
template <bool FP64, bool CH>
__device__ __forceinline__ typename Prec<FP64>::V apply2h(const Ell<FP64, CH>& H, const typename Prec<FP64>::V* __restrict__ x,
                                                         int i, int r, int rs, typename Prec<FP64>::V acc) {
  using V = typename Prec<FP64>::V;
  acc = cmul_acc(acc, __ldg(H.diag2 + i), __ldg(x + (((size_t)i << rs) + r)));
  for (int k = 0; k < H.K; ++k) {
    const size_t s = (size_t)k * H.n + i;
    const int j = __ldg(H.idx + s);
    acc = cmul_acc(acc, __ldg(H.hop2 + s), __ldg(x + (((size_t)j << rs) + r)));
  }
  return acc;
}

// y = 2 [X, H~] x  (element (i, r)): [X,H~]_ij = -dx_ij H~_ij.
template <bool FP64, bool CH>
__device__ __forceinline__ typename Prec<FP64>::V apply2xh(const Ell<FP64, CH>& H, const typename Prec<FP64>::V* __restrict__ x,
                                                          int i, int r, int rs, typename Prec<FP64>::V acc) {
  for (int k = 0; k < H.K; ++k) {
    const size_t s = (size_t)k * H.n + i;
    const int j = __ldg(H.idx + s);
    const auto h = __ldg(H.hop2 + s);
    const auto d = -__ldg(H.dx + s);
    acc = cmul_acc(acc, h, cscale(__ldg(x + (((size_t)j << rs) + r)), d));
  }
  return acc;
}

// ------------------------------------------------------------ K2: moments

// One Chebyshev order fused with the moment dot product (Eqs. 21, 28).
// first != 0: tout = H~ tm1 (T_1 from T_0 = tm1) and partials for m = 0, 1 and
// the norms (|l|^2, |r|^2) into slots slot0, slot0+1, slot_norm.
// first == 0: tout = 2 H~ tm1 - tm2 (tout may alias tm2) and the partial of
// <l|tout> into slot slot0.
template <bool FP64, bool CH>
__global__ void k_cheb(Ell<FP64, CH> H, const int* __restrict__ blk, int R, int rs,
                       const typename Prec<FP64>::V* __restrict__ tm1, const typename Prec<FP64>::V* tm2,
                       typename Prec<FP64>::V* tout, const typename Prec<FP64>::V* __restrict__ l,
                       double2* __restrict__ partial, int nblocks, int slot0, int slot_norm, int first) {
  using V = typename Prec<FP64>::V;
  using S = typename Prec<FP64>::S;
  double2* smem = dyn_smem();
  const int b = blockIdx.x;
  const size_t beg = (size_t)blk[b] << rs, end = (size_t)blk[b + 1] << rs;
  const int r = threadIdx.x & (R - 1);
  DotAcc<V> d1, d0, nl, nr;
  for (size_t e = beg + threadIdx.x; e < end; e += blockDim.x) {
    const int i = (int)(e >> rs);
    const V lv = __ldg(l + e);
    if (first) {
      V zero;
      zero.x = 0;
      zero.y = 0;
      V y = apply2h<FP64, CH>(H, tm1, i, r, rs, zero);
      y = cscale(y, (S)0.5);
      tout[e] = y;
      const V t0 = __ldg(tm1 + e);
      d0.add(lv, t0);
      d1.add(lv, y);
      nl.add_norm(lv);
      nr.add_norm(t0);
    } else {
      V y = apply2h<FP64, CH>(H, tm1, i, r, rs, cneg(tm2[e]));
      tout[e] = y;
      d1.add(lv, y);
    }
  }
  if (first) {
    double2 v[3] = {d0.get(), d1.get(), make_double2(nl.get().x, nr.get().x)};
    block_reduce_r<3>(v, R, smem);
    if ((int)threadIdx.x < R) {
      partial[((size_t)slot0 * nblocks + b) * R + threadIdx.x] = v[0];
      partial[((size_t)(slot0 + 1) * nblocks + b) * R + threadIdx.x] = v[1];
      partial[((size_t)slot_norm * nblocks + b) * R + threadIdx.x] = v[2];
    }
  } else {
    double2 v[1] = {d1.get()};
    block_reduce_r<1>(v, R, smem);
    if ((int)threadIdx.x < R) partial[((size_t)slot0 * nblocks + b) * R + threadIdx.x] = v[0];
  }
}

// Deterministic second pass: out[s][r][m] = sum over the segment's CTAs, in
// CTA order, of partial[m][b][r].  mode 0: complex out (double2), mode 1: real
// part (double).  Bound check: |mu_m|^2 <= bound_factor |l|^2 |r|^2 (norms
// from slot slot_norm), failure sets bit 1 of *flag; NaN/Inf sets bit 2.
static __global__ void k_reduce(const double2* __restrict__ partial, int nslots_m, int nblocks, int R,
                         const int* __restrict__ seg_blk, int nseg, int slot_norm, double bound_factor, void* out,
                         int mode, int* __restrict__ flag) {
  const size_t total = (size_t)nseg * R * nslots_m;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % R);
    const int m = (int)((t / R) % nslots_m);
    const int s = (int)(t / ((size_t)R * nslots_m));
    double2 acc = make_double2(0.0, 0.0);
    double2 nrm = make_double2(0.0, 0.0);
    for (int b = seg_blk[s]; b < seg_blk[s + 1]; ++b) {
      const double2 p = partial[((size_t)m * nblocks + b) * R + r];
      acc.x += p.x;
      acc.y += p.y;
      if (slot_norm >= 0) {
        const double2 q = partial[((size_t)slot_norm * nblocks + b) * R + r];
        nrm.x += q.x;
        nrm.y += q.y;
      }
    }
    const size_t o = ((size_t)s * R + r) * nslots_m + m;
    if (mode == 0)
      reinterpret_cast<double2*>(out)[o] = acc;
    else
      reinterpret_cast<double*>(out)[o] = acc.x;
    if (!isfinite(acc.x) || !isfinite(acc.y)) atomicOr(flag, 4);
    if (slot_norm >= 0) {
      const double bound = nrm.x * nrm.y * bound_factor + 1e-300;
      if (acc.x * acc.x + acc.y * acc.y > bound) atomicOr(flag, 2);
    }
  }
}

// ------------------------------------------------------------ K3: evolution

// Chebyshev-Bessel evolution (Eq. 17) of NSET independent vector sets that
// share H~.  Order m of the recursion on set q: t1[q] holds T_{m-1} psi, t2[q]
// T_{m-2} psi (tm2 may be the input psi itself for m = 2), out[q] receives T_m
// psi.  acc[q] (FP64) accumulates c_m T_m psi.
//   phase 0 (m = 0, 1): out = H~ psi; acc = c0 psi + c1 out; norm partials of psi.
//   phase 1 (2 <= m < Np-1): out = 2H~t1 - t2; acc += c_m out.
//   phase 2 (m = Np-1): psi_final = acc + c_m (2H~t1 - t2) written to fin[q]
//            (storage precision) and its norm partials.
//   phase 3 (finish, Np <= 2): fin = acc, norm partials.
template <int NSET, bool FP64>
struct EvoSets {
  const typename Prec<FP64>::V* t1[NSET];
  const typename Prec<FP64>::V* t2[NSET];
  typename Prec<FP64>::V* out[NSET];
  double2* acc[NSET];
  typename Prec<FP64>::V* fin[NSET];
};

template <int NSET, bool FP64, bool CH>
__global__ void k_evolve(Ell<FP64, CH> H, const int* __restrict__ blk, int R, int rs, EvoSets<NSET, FP64> A,
                         double2 c0, double2 c1, int phase, double2* __restrict__ partial, int nblocks, int slot) {
  using V = typename Prec<FP64>::V;
  using S = typename Prec<FP64>::S;
  double2* smem = dyn_smem();
  const int b = blockIdx.x;
  const size_t beg = (size_t)blk[b] << rs, end = (size_t)blk[b + 1] << rs;
  const int r = threadIdx.x & (R - 1);
  DotAcc<V> nrm[NSET];
  for (size_t e = beg + threadIdx.x; e < end; e += blockDim.x) {
    const int i = (int)(e >> rs);
#pragma unroll
    for (int q = 0; q < NSET; ++q) {
      if (phase == 0) {
        V zero;
        zero.x = 0;
        zero.y = 0;
        V y = cscale(apply2h<FP64, CH>(H, A.t1[q], i, r, rs, zero), (S)0.5);
        A.out[q][e] = y;
        const V p = __ldg(A.t1[q] + e);
        double2 a = cfma_d(make_double2(0.0, 0.0), c0, p);
        A.acc[q][e] = cfma_d(a, c1, y);
        nrm[q].add_norm(p);
      } else if (phase == 1) {
        V y = apply2h<FP64, CH>(H, A.t1[q], i, r, rs, cneg(A.t2[q][e]));
        A.out[q][e] = y;
        A.acc[q][e] = cfma_d(A.acc[q][e], c0, y);
      } else if (phase == 2) {
        V y = apply2h<FP64, CH>(H, A.t1[q], i, r, rs, cneg(A.t2[q][e]));
        V f = from_d2<V>(cfma_d(A.acc[q][e], c0, y));
        A.fin[q][e] = f;
        nrm[q].add_norm(f);
      } else {
        V f = from_d2<V>(A.acc[q][e]);
        A.fin[q][e] = f;
        nrm[q].add_norm(f);
      }
    }
  }
  if (phase != 1) {
    double2 v[NSET];
#pragma unroll
    for (int q = 0; q < NSET; ++q) v[q] = nrm[q].get();
    block_reduce_r<NSET>(v, R, smem);
    if ((int)threadIdx.x < R) {
#pragma unroll
      for (int q = 0; q < NSET; ++q) partial[((size_t)(slot + q) * nblocks + b) * R + threadIdx.x] = v[q];
    }
  }
}

// ------------------------------------------------ K4: commutator evolution

// One order of the coupled recursions behind one MSD time step (Eqs. 17, 18,
// 22, 24): with p = T_0 input and px the current [X,U(t)]phi,
//   u_m = T_m(H~) p            (u_0 = p, u_1 = H~ p)
//   z_m = [X, T_m] p + T_m px  (z_0 = px, z_1 = [X,H~] p + H~ px)
//   z_m = 2[X,H~] u_{m-1} + 2H~ z_{m-1} - z_{m-2}  (sum of Eq. 22 and Eq. 21)
// and accp += c_m u_m (-> U(dt) p), accx += c_m z_m (-> [X,U(dt)]p + U(dt)px).
// phase 0: m = 0, 1; phase 1: middle orders; phase 2: last order, writes
// p <- U p, px <- [X,U]p + U px (storage precision); phase 3: finish from acc.
template <bool FP64>
struct MsdBufs {
  const typename Prec<FP64>::V* u1;
  const typename Prec<FP64>::V* u2;
  typename Prec<FP64>::V* uo;
  const typename Prec<FP64>::V* z1;
  const typename Prec<FP64>::V* z2;
  typename Prec<FP64>::V* zo;
  double2* accp;
  double2* accx;
  typename Prec<FP64>::V* p;
  typename Prec<FP64>::V* px;
};

template <bool FP64, bool CH>
__global__ void k_msd_evolve(Ell<FP64, CH> H, const int* __restrict__ blk, int R, int rs, MsdBufs<FP64> B, double2 c0,
                             double2 c1, int phase, double2* __restrict__ partial, int nblocks, int slot) {
  using V = typename Prec<FP64>::V;
  using S = typename Prec<FP64>::S;
  double2* smem = dyn_smem();
  const int b = blockIdx.x;
  const size_t beg = (size_t)blk[b] << rs, end = (size_t)blk[b + 1] << rs;
  const int r = threadIdx.x & (R - 1);
  DotAcc<V> n0, n1;
  V zero;
  zero.x = 0;
  zero.y = 0;
  for (size_t e = beg + threadIdx.x; e < end; e += blockDim.x) {
    const int i = (int)(e >> rs);
    if (phase == 0) {
      // u1 = H~ p ; z1 = [X,H~] p + H~ px ; inputs: B.u1 = p, B.z1 = px
      V u = cscale(apply2h<FP64, CH>(H, B.u1, i, r, rs, zero), (S)0.5);
      V z = apply2xh<FP64, CH>(H, B.u1, i, r, rs, zero);
      z = cscale(apply2h<FP64, CH>(H, B.z1, i, r, rs, z), (S)0.5);
      B.uo[e] = u;
      B.zo[e] = z;
      const V p0 = __ldg(B.u1 + e), x0 = __ldg(B.z1 + e);
      B.accp[e] = cfma_d(cfma_d(make_double2(0.0, 0.0), c0, p0), c1, u);
      B.accx[e] = cfma_d(cfma_d(make_double2(0.0, 0.0), c0, x0), c1, z);
      n0.add_norm(p0);
    } else if (phase == 3) {
      V p = from_d2<V>(B.accp[e]);
      V x = from_d2<V>(B.accx[e]);
      B.p[e] = p;
      B.px[e] = x;
      n0.add_norm(p);
      n1.add_norm(x);
    } else {
      V u = apply2h<FP64, CH>(H, B.u1, i, r, rs, cneg(B.u2[e]));
      V z = apply2xh<FP64, CH>(H, B.u1, i, r, rs, cneg(B.z2[e]));
      z = apply2h<FP64, CH>(H, B.z1, i, r, rs, z);
      if (phase == 1) {
        B.uo[e] = u;
        B.zo[e] = z;
        B.accp[e] = cfma_d(B.accp[e], c0, u);
        B.accx[e] = cfma_d(B.accx[e], c0, z);
      } else {
        V p = from_d2<V>(cfma_d(B.accp[e], c0, u));
        V x = from_d2<V>(cfma_d(B.accx[e], c0, z));
        B.p[e] = p;
        B.px[e] = x;
        n0.add_norm(p);
        n1.add_norm(x);
      }
    }
  }
  if (phase != 1) {
    double2 v[2] = {n0.get(), n1.get()};
    block_reduce_r<2>(v, R, smem);
    if ((int)threadIdx.x < R) {
      partial[((size_t)slot * nblocks + b) * R + threadIdx.x] = v[0];
      partial[((size_t)(slot + 1) * nblocks + b) * R + threadIdx.x] = v[1];
    }
  }
}

// Real-part moments Re <l|T_m|r> (the VAC row of Eq. 29 keeps only the real
// part): same recursion as k_cheb with half the dot-product work.  Slots as k_cheb.
template <bool FP64, bool CH>
__global__ void k_cheb_re(Ell<FP64, CH> H, const int* __restrict__ blk, int R, int rs,
                          const typename Prec<FP64>::V* __restrict__ tm1, const typename Prec<FP64>::V* tm2,
                          typename Prec<FP64>::V* tout, const typename Prec<FP64>::V* __restrict__ l,
                          double2* __restrict__ partial, int nblocks, int slot0, int slot_norm, int first) {
  using V = typename Prec<FP64>::V;
  using S = typename Prec<FP64>::S;
  double2* smem = dyn_smem();
  const int b = blockIdx.x;
  const size_t beg = (size_t)blk[b] << rs, end = (size_t)blk[b + 1] << rs;
  const int r = threadIdx.x & (R - 1);
  if (first) {
    DotAcc<V> d0, d1, nl, nr;
    for (size_t e = beg + threadIdx.x; e < end; e += blockDim.x) {
      const int i = (int)(e >> rs);
      const V lv = __ldg(l + e);
      V zero;
      zero.x = 0;
      zero.y = 0;
      V y = cscale(apply2h<FP64, CH>(H, tm1, i, r, rs, zero), (S)0.5);
      tout[e] = y;
      const V t0 = __ldg(tm1 + e);
      d0.add_re(lv, t0);
      d1.add_re(lv, y);
      nl.add_norm(lv);
      nr.add_norm(t0);
    }
    double2 v[3] = {d0.get(), d1.get(), make_double2(nl.get().x, nr.get().x)};
    block_reduce_r<3>(v, R, smem);
    if ((int)threadIdx.x < R) {
      partial[((size_t)slot0 * nblocks + b) * R + threadIdx.x] = v[0];
      partial[((size_t)(slot0 + 1) * nblocks + b) * R + threadIdx.x] = v[1];
      partial[((size_t)slot_norm * nblocks + b) * R + threadIdx.x] = v[2];
    }
  } else {
    DotAcc<V> d1;
    for (size_t e = beg + threadIdx.x; e < end; e += blockDim.x) {
      const int i = (int)(e >> rs);
      V y = apply2h<FP64, CH>(H, tm1, i, r, rs, cneg(tm2[e]));
      tout[e] = y;
      d1.add_re(__ldg(l + e), y);
    }
    double2 v[1] = {d1.get()};
    block_reduce_r<1>(v, R, smem);
    if ((int)threadIdx.x < R) partial[((size_t)slot0 * nblocks + b) * R + threadIdx.x] = v[0];
  }
}

// Moments of l = r = phi by the product identities of Chebyshev polynomials,
// T_{2n} = 2 T_n T_n - T_0 and T_{2n+1} = 2 T_{n+1} T_n - T_1, so that
// mu_{2n} = 2 <u_n|u_n> - mu_0 and mu_{2n+1} = 2 <u_{n+1}|u_n> - mu_1 with
// u_n = T_n(H~) phi: M moments from ceil(M/2) recursion steps (kernel polynomial
// method, Weisse et al., Rev. Mod. Phys. 78, 275 (2006), Sec. II.C).  Both inner
// products are real for Hermitian H~.
// first != 0: tout = u_1 = H~ u_0 (tm1 = u_0); raw sums s_0 = <u_0|u_0>, s_1 = <u_1|u_0>
// into slots 0, 1.  Otherwise (step m >= 2, tm1 = u_{m-1}, tm2 = u_{m-2}): tout = u_m,
// s_{2m-2} = <u_{m-1}|u_{m-1}> and s_{2m-1} = <u_m|u_{m-1}> into slots 2m-2, 2m-1.
template <bool FP64, bool CH>
__global__ void k_cheb_dbl(Ell<FP64, CH> H, const int* __restrict__ blk, int R, int rs,
                           const typename Prec<FP64>::V* __restrict__ tm1, const typename Prec<FP64>::V* tm2,
                           typename Prec<FP64>::V* tout, double2* __restrict__ partial, int nblocks, int m) {
  using V = typename Prec<FP64>::V;
  using S = typename Prec<FP64>::S;
  double2* smem = dyn_smem();
  const int b = blockIdx.x;
  const size_t beg = (size_t)blk[b] << rs, end = (size_t)blk[b + 1] << rs;
  const int r = threadIdx.x & (R - 1);
  DotAcc<V> a0, a1;
  for (size_t e = beg + threadIdx.x; e < end; e += blockDim.x) {
    const int i = (int)(e >> rs);
    const V own = __ldg(tm1 + e);
    V acc;
    if (m == 1) {
      acc.x = 0;
      acc.y = 0;
    } else {
      acc = cneg(tm2[e]);
    }
    acc = cmul_acc(acc, __ldg(H.diag2 + i), own);
    for (int k = 0; k < H.K; ++k) {
      const size_t s = (size_t)k * H.n + i;
      const int j = __ldg(H.idx + s);
      acc = cmul_acc(acc, __ldg(H.hop2 + s), __ldg(tm1 + (((size_t)j << rs) + r)));
    }
    if (m == 1) acc = cscale(acc, (S)0.5);
    tout[e] = acc;
    a0.add_norm(own);
    a1.add_re(acc, own);
  }
  double v[2] = {a0.get().x, a1.get().x};
  block_reduce_rx<2>(v, R, (double*)smem);
  if ((int)threadIdx.x < R) {
    const int k0 = 2 * m - 2;
    partial[((size_t)k0 * nblocks + b) * R + threadIdx.x] = make_double2(v[0], 0.0);
    partial[((size_t)(k0 + 1) * nblocks + b) * R + threadIdx.x] = make_double2(v[1], 0.0);
  }
}

// Second pass of k_cheb_dbl: mu[s][r][k] = s_k for k < 2, 2 s_k - s_{k mod 2} otherwise,
// each s summed over the segment's CTAs in CTA order.  Bound |mu_k| <= (1+tol) mu_0.
static __global__ void k_reduce_dbl(const double2* __restrict__ partial, int M, int nblocks, int R,
                             const int* __restrict__ seg_blk, int nseg, double bound_factor, double* __restrict__ out,
                             int* __restrict__ flag, int slot_norm = -1) {
  // slot_norm < 0: l = r, |mu_k| <= mu_0 (1 + tol); otherwise slot_norm holds
  // (|l|^2, |r|^2) and |mu_k| <= |l| |r| (1 + tol).
  const size_t total = (size_t)nseg * R * M;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % R);
    const int k = (int)((t / R) % M);
    const int s = (int)(t / ((size_t)R * M));
    double sk = 0.0, s0 = 0.0, sp = 0.0, nl = 0.0, nr = 0.0;
    const int kp = k & 1;
    for (int b = seg_blk[s]; b < seg_blk[s + 1]; ++b) {
      sk += partial[((size_t)k * nblocks + b) * R + r].x;
      s0 += partial[((size_t)0 * nblocks + b) * R + r].x;
      sp += partial[((size_t)kp * nblocks + b) * R + r].x;
      if (slot_norm >= 0) {
        const double2 q = partial[((size_t)slot_norm * nblocks + b) * R + r];
        nl += q.x;
        nr += q.y;
      }
    }
    const double mu = (k < 2) ? sk : 2.0 * sk - sp;
    out[((size_t)s * R + r) * M + k] = mu;
    if (!isfinite(mu)) atomicOr(flag, 4);
    const double bound = (slot_norm >= 0 ? sqrt(nl * nr) : s0) * bound_factor + 1e-300;
    if (fabs(mu) > bound) atomicOr(flag, 2);
  }
}

// Norm check of an evolution: slots q (before) and NSET + q (after) hold the
// partial squared norms of set q.  | |after| - |before| | > tol |before| sets
// bit 3 of *flag.  norms (optional) receives [nseg][R][NSET][2] squared norms.
static __global__ void k_norm_check(const double2* __restrict__ partial, int nset, int nblocks, int R,
                             const int* __restrict__ seg_blk, int nseg, double tol, double* __restrict__ norms,
                             int* __restrict__ flag) {
  const int total = nseg * R * nset;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int q = t % nset, r = (t / nset) % R, s = t / (nset * R);
    double a = 0.0, z = 0.0;
    for (int b = seg_blk[s]; b < seg_blk[s + 1]; ++b) {
      a += partial[((size_t)q * nblocks + b) * R + r].x;
      z += partial[((size_t)(nset + q) * nblocks + b) * R + r].x;
    }
    if (norms) {
      norms[(size_t)t * 2] = a;
      norms[(size_t)t * 2 + 1] = z;
    }
    if (!isfinite(z)) atomicOr(flag, 4);
    if (fabs(sqrt(z) - sqrt(a)) > tol * sqrt(a) + 1e-300) atomicOr(flag, 8);
  }
}

// MSD step: slot 0 = |p|^2 before, slot 2 = |U p|^2 after (slot 3 = |px|^2, unchecked).
static __global__ void k_norm_check_msd(const double2* __restrict__ partial, int nblocks, int R,
                                 const int* __restrict__ seg_blk, int nseg, double tol, int* __restrict__ flag) {
  const int total = nseg * R;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int r = t % R, s = t / R;
    double a = 0.0, z = 0.0, x = 0.0;
    for (int b = seg_blk[s]; b < seg_blk[s + 1]; ++b) {
      a += partial[((size_t)0 * nblocks + b) * R + r].x;
      z += partial[((size_t)2 * nblocks + b) * R + r].x;
      x += partial[((size_t)3 * nblocks + b) * R + r].x;
    }
    if (!isfinite(z) || !isfinite(x)) atomicOr(flag, 4);
    if (fabs(sqrt(z) - sqrt(a)) > tol * sqrt(a) + 1e-300) atomicOr(flag, 8);
  }
}

// --------------------------------------------------------------- K5: velocity

// y = V x = i dE sum_k dx_ik H~_ik x_j (Eq. 34); with hop2 = 2H~ the factor is i dE/2.
template <bool FP64, bool CH>
__global__ void k_velocity(Ell<FP64, CH> H, const int* __restrict__ blk, int R, int rs, double half_dE,
                           const typename Prec<FP64>::V* __restrict__ x, typename Prec<FP64>::V* __restrict__ y,
                           typename Prec<FP64>::V* __restrict__ y2 /* optional copy of x */) {
  using V = typename Prec<FP64>::V;
  using S = typename Prec<FP64>::S;
  const int b = blockIdx.x;
  const size_t beg = (size_t)blk[b] << rs, end = (size_t)blk[b + 1] << rs;
  const int r = threadIdx.x & (R - 1);
  for (size_t e = beg + threadIdx.x; e < end; e += blockDim.x) {
    const int i = (int)(e >> rs);
    V a;
    a.x = 0;
    a.y = 0;
    for (int k = 0; k < H.K; ++k) {
      const size_t s = (size_t)k * H.n + i;
      const int j = __ldg(H.idx + s);
      a = cmul_acc(a, __ldg(H.hop2 + s), cscale(__ldg(x + (((size_t)j << rs) + r)), __ldg(H.dx + s)));
    }
    // multiply by i * dE/2
    V o;
    o.x = -a.y * (S)half_dE;
    o.y = a.x * (S)half_dE;
    y[e] = o;
    if (y2) y2[e] = __ldg(x + e);
  }
}

// --------------------------------------------------------------- K7: KPM

// tab[n][e] = g_n (2 - delta_n0) cos(n arccos x_e) * 2 n_over_omega / (pi dE sqrt(1 - x_e^2))
// (Eqs. 25-27, 31); NaN where |x_e| >= 1.
static __global__ void k_kpm_table(int M, const double* __restrict__ E, int NE, double dE, double n_over_omega, int jackson,
                            double* __restrict__ tab) {
  const size_t total = (size_t)M * NE;
  const double a = 1.0 / (M + 1.0);
  const double cot = cos(M_PI * a) / sin(M_PI * a);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int e = (int)(t % NE);
    const int n = (int)(t / NE);
    const double x = E[e] / dE;
    double v;
    if (!(fabs(x) < 1.0)) {
      v = CUDART_NAN;
    } else {
      const double g = jackson ? (1.0 - n * a) * cos(M_PI * n * a) + a * sin(M_PI * n * a) * cot : 1.0;
      v = g * (n == 0 ? 1.0 : 2.0) * cos(n * acos(x)) * 2.0 * n_over_omega / (M_PI * dE * sqrt(1.0 - x * x));
    }
    tab[t] = v;
  }
}

// out[row][e] = sum_n mu[row][n] tab[n][e]: a small FP64 GEMM, 16x16 tiles.
static __global__ void k_kpm_gemm(const double* __restrict__ mu, int rows, int M, const double* __restrict__ tab, int NE,
                           double* __restrict__ out) {
  __shared__ double As[16][17], Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < M; k0 += 16) {
    As[ty][tx] = (row < rows && k0 + tx < M) ? mu[(size_t)row * M + k0 + tx] : 0.0;
    Bs[ty][tx] = (k0 + ty < M && col < NE) ? tab[(size_t)(k0 + ty) * NE + col] : 0.0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = fma(As[ty][k], Bs[k][tx], acc);
    __syncthreads();
  }
  if (row < rows && col < NE) out[(size_t)row * NE + col] = acc;
}

// --------------------------------------------------------------- sigma

static __global__ void k_sigma_vac(const double* __restrict__ v, const double* __restrict__ dt, int Nt, int NE,
                            double* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < NE; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    out[e] = 0.0;
    for (int k = 1; k < Nt; ++k) {
      s += 0.5 * dt[k - 1] * (v[(size_t)(k - 1) * NE + e] + v[(size_t)k * NE + e]);
      out[(size_t)k * NE + e] = s;
    }
  }
}

static __global__ void k_sigma_msd(const double* __restrict__ m, const double* __restrict__ dt, int Nt, int NE,
                            double* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < NE; e += gridDim.x * blockDim.x) {
    double prev = 0.0;
    for (int k = 0; k < Nt; ++k) {
      const double c = m[(size_t)k * NE + e];
      out[(size_t)k * NE + e] = (c - prev) / (2.0 * dt[k]);
      prev = c;
    }
  }
}

// --------------------------------------------------------------- random phase

// SplitMix64 (Steele, Lea, Flood 2014): draw i of the stream keyed by
// key = mix(seed + (stream+1) G) is mix(key + (i+1) G).
__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <bool FP64>
__global__ void k_random_phase(int n, int R, const uint64_t* __restrict__ keys, const int* __restrict__ site_seg,
                               const double* __restrict__ seg_inv_sqrt, typename Prec<FP64>::V* __restrict__ phi) {
  using V = typename Prec<FP64>::V;
  const size_t total = (size_t)n * R;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / R), r = (int)(t % R);
    const uint64_t z = sm64_mix(keys[r] + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull);
    const double u = (double)(z >> 11) * 0x1.0p-53;
    double s, c;
    sincospi(2.0 * u, &s, &c);
    const double w = seg_inv_sqrt[site_seg ? site_seg[i] : 0];
    V v;
    v.x = c * w;
    v.y = s * w;
    phi[t] = v;
  }
}

}  // namespace gqt

namespace gqt {

// ------------------------------------------------------------ K9: adjoint
//
// Reverse-mode derivative of J = Re sum_{m<P} coef_m <lam| T_m(H~) |r> with
// u_m = T_m r (not in the paper; it differentiates Eqs. 17, 21 and 29).  The
// adjoint vectors obey the transposed recurrence
//   w_m = conj(coef_m) lam + 2 H~ w_{m+1} - w_{m+2},   w_P = w_{P+1} = 0,
// and dJ = Re sum_ij conj(G_ij) dH~_ij with G = w_1 u_0^+ + 2 sum_{m>=2} w_m u_{m-1}^+,
// needed only on the diagonal and the ELL slots.

// Plain recurrence step: out = 2H~ t1 - t2 (first: out = H~ t1); if acc != null,
// first: acc = cA t1 + cB out, else acc += cB out.
template <bool FP64, bool CH>
__global__ void k_recur(Ell<FP64, CH> H, const int* __restrict__ blk, const typename Prec<FP64>::V* __restrict__ t1,
                        const typename Prec<FP64>::V* t2, typename Prec<FP64>::V* out, double2* __restrict__ acc,
                        double2 cA, double2 cB, int first) {
  using V = typename Prec<FP64>::V;
  using S = typename Prec<FP64>::S;
  const int b = blockIdx.x;
  for (int i = blk[b] + threadIdx.x; i < blk[b + 1]; i += blockDim.x) {
    V y;
    if (first) {
      V zero;
      zero.x = 0;
      zero.y = 0;
      y = cscale(apply2h<FP64, CH>(H, t1, i, 0, 0, zero), (S)0.5);
    } else {
      y = apply2h<FP64, CH>(H, t1, i, 0, 0, cneg(t2[i]));
    }
    out[i] = y;
    if (acc) {
      if (first)
        acc[i] = cfma_d(cfma_d(make_double2(0.0, 0.0), cA, __ldg(t1 + i)), cB, y);
      else
        acc[i] = cfma_d(acc[i], cB, y);
    }
  }
}

// One adjoint order m: w_m = lc lam + 2H~ w1 - w2 (w1 = w_{m+1}, w2 = w_{m+2},
// w_m overwrites w2) and G += f w_m conj(u_{m-1}) on the diagonal (gdiag, real
// part) and on the slots (gslot [K][n]).  f = (m == 1 ? 1 : 2) / dE.
template <bool FP64, bool CH>
__global__ void k_adj_step(Ell<FP64, CH> H, const int* __restrict__ blk, const typename Prec<FP64>::V* __restrict__ w1,
                           typename Prec<FP64>::V* w2, const typename Prec<FP64>::V* __restrict__ lam, double2 lc,
                           const typename Prec<FP64>::V* __restrict__ u, double f, double* __restrict__ gdiag,
                           double2* __restrict__ gslot) {
  using V = typename Prec<FP64>::V;
  const int b = blockIdx.x;
  for (int i = blk[b] + threadIdx.x; i < blk[b + 1]; i += blockDim.x) {
    V y = apply2h<FP64, CH>(H, w1, i, 0, 0, cneg(w2[i]));
    double2 wd = cfma_d(to_d2(y), lc, __ldg(lam + i));
    const V w = from_d2<V>(wd);
    w2[i] = w;
    wd = to_d2(w);
    const double2 ui = to_d2(__ldg(u + i));
    gdiag[i] += f * (wd.x * ui.x + wd.y * ui.y);
    for (int k = 0; k < H.K; ++k) {
      const size_t s = (size_t)k * H.n + i;
      const double2 uj = to_d2(__ldg(u + __ldg(H.idx + s)));
      double2 g = gslot[s];
      // w * conj(uj)
      g.x += f * (wd.x * uj.x + wd.y * uj.y);
      g.y += f * (wd.y * uj.x - wd.x * uj.y);
      gslot[s] = g;
    }
  }
}

// rbar = lc0 lam + H~ w1 - w2 (Clenshaw end, = sum_m conj(coef_m) T_m lam); w1 may be null (P = 1).
template <bool FP64, bool CH>
__global__ void k_adj_final(Ell<FP64, CH> H, const int* __restrict__ blk, const typename Prec<FP64>::V* __restrict__ w1,
                            const typename Prec<FP64>::V* __restrict__ w2, const typename Prec<FP64>::V* __restrict__ lam,
                            double2 lc0, typename Prec<FP64>::V* __restrict__ rbar) {
  using V = typename Prec<FP64>::V;
  using S = typename Prec<FP64>::S;
  const int b = blockIdx.x;
  for (int i = blk[b] + threadIdx.x; i < blk[b + 1]; i += blockDim.x) {
    double2 acc = cfma_d(make_double2(0.0, 0.0), lc0, __ldg(lam + i));
    if (w1) {
      V zero;
      zero.x = 0;
      zero.y = 0;
      V y = cscale(apply2h<FP64, CH>(H, w1, i, 0, 0, zero), (S)0.5);
      const double2 yd = to_d2(y), w2d = to_d2(__ldg(w2 + i));
      acc.x += yd.x - w2d.x;
      acc.y += yd.y - w2d.y;
    }
    rbar[i] = from_d2<V>(acc);
  }
}

__device__ __forceinline__ double2 hop_d(double2 h) { return h; }
__device__ __forceinline__ double2 hop_d(float2 h) { return to_d2(h); }
__device__ __forceinline__ double hop_d(double h) { return h; }
__device__ __forceinline__ double hop_d(float h) { return (double)h; }

// Velocity part of the gradient: l = V x with V_ij = i dx_ij H_ij (unscaled H), so
// G_ij += lbar_i (-i dx_ij) conj(x_j) (slots only; V has no diagonal).
template <bool FP64, bool CH, class LB>
__global__ void k_vel_adj(Ell<FP64, CH> H, const int* __restrict__ blk, const LB* __restrict__ lbar,
                          const typename Prec<FP64>::V* __restrict__ x, double2* __restrict__ gslot) {
  const int b = blockIdx.x;
  for (int i = blk[b] + threadIdx.x; i < blk[b + 1]; i += blockDim.x) {
    const double2 lb = to_d2(lbar[i]);
    for (int k = 0; k < H.K; ++k) {
      const size_t s = (size_t)k * H.n + i;
      const double2 xj = to_d2(__ldg(x + __ldg(H.idx + s)));
      const double d = (double)__ldg(H.dx + s);
      // lbar * (-i d) * conj(xj) = -i d (lb.x + i lb.y)(xj.x - i xj.y)
      const double re = lb.x * xj.x + lb.y * xj.y, im = lb.y * xj.x - lb.x * xj.y;
      double2 g = gslot[s];
      g.x += d * im;
      g.y += -d * re;
      gslot[s] = g;
    }
  }
}

// y += V x for a double2 accumulator y (x storage precision), V = i dE sum dx H~.
template <bool FP64, bool CH>
__global__ void k_vel_acc(Ell<FP64, CH> H, const int* __restrict__ blk, double half_dE,
                          const double2* __restrict__ x, typename Prec<FP64>::V* __restrict__ y) {
  using V = typename Prec<FP64>::V;
  const int b = blockIdx.x;
  for (int i = blk[b] + threadIdx.x; i < blk[b + 1]; i += blockDim.x) {
    double2 a = make_double2(0.0, 0.0);
    for (int k = 0; k < H.K; ++k) {
      const size_t s = (size_t)k * H.n + i;
      const int j = __ldg(H.idx + s);
      const double d = (double)__ldg(H.dx + s);
      a = cmul_acc(a, hop_d(__ldg(H.hop2 + s)), cscale(x[j], d));
    }
    double2 yo = to_d2(y[i]);
    yo.x += -a.y * half_dE;
    yo.y += a.x * half_dE;
    y[i] = from_d2<V>(yo);
  }
}

// Re <l|x> partial sums per CTA (x double2).
template <class V>
__global__ void k_dot_re(const int* __restrict__ blk, const V* __restrict__ l, const double2* __restrict__ x,
                         double* __restrict__ partial) {
  __shared__ double sh[32];
  const int b = blockIdx.x;
  double s = 0.0;
  for (int i = blk[b] + threadIdx.x; i < blk[b + 1]; i += blockDim.x) {
    const double2 lv = to_d2(l[i]);
    const double2 xv = x[i];
    s += lv.x * xv.x + lv.y * xv.y;
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    partial[b] = t;
  }
}

// y += x (storage precision).
template <class V>
__global__ void k_axpy(const int* __restrict__ blk, V* __restrict__ y, const V* __restrict__ x) {
  const int b = blockIdx.x;
  for (int i = blk[b] + threadIdx.x; i < blk[b + 1]; i += blockDim.x) {
    V a = y[i];
    const V c = x[i];
    a.x += c.x;
    a.y += c.y;
    y[i] = a;
  }
}

// Slot-major [K][n] double2 -> row-major [n][K] double2; diagonal copied.
static __global__ void k_grad_out(int n, int K, const double2* __restrict__ gslot, const double* __restrict__ gdiag,
                           double2* __restrict__ out_slot, double* __restrict__ out_diag) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)n * K; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / K), k = (int)(t % K);
    out_slot[t] = gslot[(size_t)k * n + i];
    if (k == 0) out_diag[i] = gdiag[i];
  }
}

}  // namespace gqt

namespace gqt {
// beta[n] = sum_e w[e] tab[n][e]: the transpose of the reconstruction (the weight
// each moment carries in a weighted sum of reconstructed values).  NaN entries of
// the table (|E| >= dE) must carry zero weight and are skipped when w[e] == 0.
static __global__ void k_kpm_weights(const double* __restrict__ tab, int M, int NE, const double* __restrict__ w,
                              double* __restrict__ beta) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < M; n += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int e = 0; e < NE; ++e) {
      const double we = w[e];
      if (we != 0.0) s += we * tab[(size_t)n * NE + e];
    }
    beta[n] = s;
  }
}
}  // namespace gqt

namespace gqt {

// ------------------------------------------- wavefront-ordered moment kernels
//
// The CTAs of a segment stride through it together: CTA b with tile entry
// (beg, end, q, G) handles elements beg*R + (q + j*G)*blockDim + tid.  At any
// moment the segment's CTAs work on one window of G*blockDim consecutive
// elements, so neighbour gathers (a few lattice rows away) hit in L2 and
// T_{m-1} is read from DRAM about once per order.  Each thread keeps U
// elements in flight: all independent loads of the U elements are issued
// before the dependent neighbour gathers and the arithmetic.

template <bool FP64, bool CH, int U, bool DBL, int KK, bool first>
__device__ __forceinline__ void cheb_wave_body(const Ell<FP64, CH>& H, int4 tb, int R, int rs,
                                               const typename Prec<FP64>::V* __restrict__ tm1,
                                               const typename Prec<FP64>::V* tm2, typename Prec<FP64>::V* tout,
                                               const typename Prec<FP64>::V* __restrict__ l,
                                               DotAcc<typename Prec<FP64>::V>& d0, DotAcc<typename Prec<FP64>::V>& d1,
                                               DotAcc<typename Prec<FP64>::V>& nl, DotAcc<typename Prec<FP64>::V>& nr) {
  using V = typename Prec<FP64>::V;
  using S = typename Prec<FP64>::S;
  using HT = typename Ell<FP64, CH>::HT;
  constexpr int KMAX = KK;  // neighbour slots, a compile-time constant
  const size_t segb = (size_t)tb.x << rs, sege = (size_t)tb.y << rs;
  const size_t step = (size_t)tb.w * blockDim.x;
  const int r = threadIdx.x & (R - 1);
  constexpr int K = KK;
  for (size_t e0 = segb + (size_t)tb.z * blockDim.x + threadIdx.x; e0 < sege; e0 += (size_t)U * step) {
    V own[U], acc[U], lv[U];
    int idx[U][KMAX];
    HT hv[U][KMAX];
    S dg[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const size_t e = e0 + u * step;
      ok[u] = e < sege;
      const size_t ee = ok[u] ? e : e0;
      const int i = (int)(ee >> rs);
      own[u] = __ldg(tm1 + ee);
      dg[u] = __ldg(H.diag2 + i);
      if (DBL) {
        if (first) {
          acc[u].x = 0;
          acc[u].y = 0;
        } else {
          acc[u] = cneg(tm2[ee]);
        }
      } else {
        lv[u] = __ldg(l + ee);
        if (first) {
          acc[u].x = 0;
          acc[u].y = 0;
        } else {
          acc[u] = cneg(tm2[ee]);
        }
      }
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
        if (k < K) {
          const size_t s = (size_t)k * H.n + i;
          idx[u][k] = __ldg(H.idx + s);
          hv[u][k] = __ldg(H.hop2 + s);
        }
    }
    V nbv[U][KMAX];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
        if (k < K) nbv[u][k] = __ldg(tm1 + (((size_t)idx[u][k] << rs) + r));
#pragma unroll
    for (int u = 0; u < U; ++u) {
      V a = first ? cscale(own[u], dg[u]) : cmul_acc(acc[u], dg[u], own[u]);
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
        if (k < K) a = cmul_acc(a, hv[u][k], nbv[u][k]);
      if (first) a = cscale(a, (S)0.5);
      if (ok[u]) {
        tout[e0 + u * step] = a;
        if (DBL) {
          d0.add_norm(own[u]);
          d1.add_re(a, own[u]);
        } else {
          if (first) {
            d0.add_re(lv[u], own[u]);
            nl.add_norm(lv[u]);
            nr.add_norm(own[u]);
          }
          d1.add_re(lv[u], a);
        }
      }
    }
  }
}

// Re <l|T_m|r> orders (VAC rows) in wavefront order; slots as k_cheb_re.
template <bool FP64, bool CH, int U, int KK>
__global__ void __launch_bounds__(256, (U == 1 ? 4 : 2)) k_cheb_re_w(Ell<FP64, CH> H, const int4* __restrict__ tab, int R, int rs,
                                                   const typename Prec<FP64>::V* __restrict__ tm1,
                                                   const typename Prec<FP64>::V* tm2, typename Prec<FP64>::V* tout,
                                                   const typename Prec<FP64>::V* __restrict__ l,
                                                   double2* __restrict__ partial, int nblocks, int slot0, int slot_norm,
                                                   int first) {
  using V = typename Prec<FP64>::V;
  double2* smem = dyn_smem();
  const int b = blockIdx.x;
  DotAcc<V> d0, d1, nl, nr;
  // the first order (no T_{m-2}) is a separate instantiation of the loop body, so the
  // other orders fold -T_{m-2} into the first fused multiply-add
  if (first)
    cheb_wave_body<FP64, CH, U, false, KK, true>(H, tab[b], R, rs, tm1, tm2, tout, l, d0, d1, nl, nr);
  else
    cheb_wave_body<FP64, CH, U, false, KK, false>(H, tab[b], R, rs, tm1, tm2, tout, l, d0, d1, nl, nr);
  if (first) {
    double2 v[3] = {d0.get(), d1.get(), make_double2(nl.get().x, nr.get().x)};
    block_reduce_r<3>(v, R, smem);
    if ((int)threadIdx.x < R) {
      partial[((size_t)slot0 * nblocks + b) * R + threadIdx.x] = v[0];
      partial[((size_t)(slot0 + 1) * nblocks + b) * R + threadIdx.x] = v[1];
      partial[((size_t)slot_norm * nblocks + b) * R + threadIdx.x] = v[2];
    }
  } else {
    double v[1] = {d1.get().x};
    block_reduce_rx<1>(v, R, (double*)smem);
    if ((int)threadIdx.x < R) partial[((size_t)slot0 * nblocks + b) * R + threadIdx.x] = make_double2(v[0], 0.0);
  }
}

// l = r doubling orders (DOS, MSD rows) in wavefront order; slots as k_cheb_dbl.
template <bool FP64, bool CH, int U, int KK>
__global__ void __launch_bounds__(256, (U == 1 ? 4 : 2)) k_cheb_dbl_w(Ell<FP64, CH> H, const int4* __restrict__ tab, int R, int rs,
                                                    const typename Prec<FP64>::V* __restrict__ tm1,
                                                    const typename Prec<FP64>::V* tm2, typename Prec<FP64>::V* tout,
                                                    double2* __restrict__ partial, int nblocks, int m) {
  using V = typename Prec<FP64>::V;
  double2* smem = dyn_smem();
  const int b = blockIdx.x;
  DotAcc<V> a0, a1, u0, u1;
  if (m == 1)
    cheb_wave_body<FP64, CH, U, true, KK, true>(H, tab[b], R, rs, tm1, tm2, tout, nullptr, a0, a1, u0, u1);
  else
    cheb_wave_body<FP64, CH, U, true, KK, false>(H, tab[b], R, rs, tm1, tm2, tout, nullptr, a0, a1, u0, u1);
  double v[2] = {a0.get().x, a1.get().x};
  block_reduce_rx<2>(v, R, (double*)smem);
  if ((int)threadIdx.x < R) {
    const int k0 = 2 * m - 2;
    partial[((size_t)k0 * nblocks + b) * R + threadIdx.x] = make_double2(v[0], 0.0);
    partial[((size_t)(k0 + 1) * nblocks + b) * R + threadIdx.x] = make_double2(v[1], 0.0);
  }
}


// Re <l|T_m(H~)|r> for l != r by two recurrences at once (Eqs. 21, 29): chain A
// from l and chain B from r, A_k = T_k l, B_k = T_k r.  The product identities
// T_2k = 2 T_k T_k - T_0 and T_2k+1 = 2 T_k T_k+1 - T_1 of Chebyshev polynomials,
// with T_k(H~) Hermitian, give mu_2k = 2 Re <A_k|B_k> - mu_0 and mu_2k+1 =
// 2 Re <A_k|B_k+1> - mu_1, so step m (computing A_m, B_m) yields the dots of
// moments 2m-2 (<A_m-1|B_m-1>) and 2m-1 (<A_m-1|B_m>), combined in k_reduce_dbl.
// Each step streams H~ once for two moments; FP64 work per moment is the same as
// the single recurrence with its Re <l|.> dot.  Step 1 also records |l|^2, |r|^2
// (slot_norm) for the moment bound.  Wavefront order, one element per thread.
template <bool FP64, bool CH, int KK, bool first>
__device__ __forceinline__ void cheb_pair_body(const Ell<FP64, CH>& H, int4 tb, int R, int rs,
                                               const typename Prec<FP64>::V* __restrict__ am1,
                                               const typename Prec<FP64>::V* __restrict__ bm1,
                                               const typename Prec<FP64>::V* am2, const typename Prec<FP64>::V* bm2,
                                               typename Prec<FP64>::V* aout, typename Prec<FP64>::V* bout,
                                               DotAcc<typename Prec<FP64>::V>& d0, DotAcc<typename Prec<FP64>::V>& d1,
                                               DotAcc<typename Prec<FP64>::V>& nl, DotAcc<typename Prec<FP64>::V>& nr) {
  using V = typename Prec<FP64>::V;
  using S = typename Prec<FP64>::S;
  using HT = typename Ell<FP64, CH>::HT;
  const size_t segb = (size_t)tb.x << rs, sege = (size_t)tb.y << rs;
  const size_t step = (size_t)tb.w * blockDim.x;
  const int r = threadIdx.x & (R - 1);
  for (size_t e = segb + (size_t)tb.z * blockDim.x + threadIdx.x; e < sege; e += step) {
    const int i = (int)(e >> rs);
    int idx[KK];
    HT hv[KK];
#pragma unroll
    for (int k = 0; k < KK; ++k) {
      const size_t s = (size_t)k * H.n + i;
      idx[k] = __ldg(H.idx + s);
      hv[k] = __ldg(H.hop2 + s);
    }
    const S dg = __ldg(H.diag2 + i);
    const V ao = __ldg(am1 + e), bo = __ldg(bm1 + e);
    V a, b;
    if (first) {
      a = cscale(ao, dg);
      b = cscale(bo, dg);
    } else {
      a = cmul_acc(cneg(am2[e]), dg, ao);
      b = cmul_acc(cneg(bm2[e]), dg, bo);
    }
    V na[KK], nb[KK];
#pragma unroll
    for (int k = 0; k < KK; ++k) {
      const size_t j = ((size_t)idx[k] << rs) + r;
      na[k] = __ldg(am1 + j);
      nb[k] = __ldg(bm1 + j);
    }
#pragma unroll
    for (int k = 0; k < KK; ++k) {
      a = cmul_acc(a, hv[k], na[k]);
      b = cmul_acc(b, hv[k], nb[k]);
    }
    if (first) {
      a = cscale(a, (S)0.5);
      b = cscale(b, (S)0.5);
    }
    aout[e] = a;
    bout[e] = b;
    d0.add_re(ao, bo);
    d1.add_re(ao, b);
    if (first) {
      nl.add_norm(ao);
      nr.add_norm(bo);
    }
  }
}

template <bool FP64, bool CH, int KK>
__global__ void __launch_bounds__(256, 3) k_cheb_pair_w(Ell<FP64, CH> H, const int4* __restrict__ tab, int R, int rs,
                                                       const typename Prec<FP64>::V* __restrict__ am1,
                                                       const typename Prec<FP64>::V* __restrict__ bm1,
                                                       const typename Prec<FP64>::V* am2,
                                                       const typename Prec<FP64>::V* bm2,
                                                       typename Prec<FP64>::V* aout, typename Prec<FP64>::V* bout,
                                                       double2* __restrict__ partial, int nblocks, int m,
                                                       int slot_norm) {
  using V = typename Prec<FP64>::V;
  double2* smem = dyn_smem();
  const int b = blockIdx.x;
  DotAcc<V> d0, d1, nl, nr;
  if (m == 1)
    cheb_pair_body<FP64, CH, KK, true>(H, tab[b], R, rs, am1, bm1, am2, bm2, aout, bout, d0, d1, nl, nr);
  else
    cheb_pair_body<FP64, CH, KK, false>(H, tab[b], R, rs, am1, bm1, am2, bm2, aout, bout, d0, d1, nl, nr);
  const int k0 = 2 * m - 2;
  if (m == 1) {
    double2 v[3] = {d0.get(), d1.get(), make_double2(nl.get().x, nr.get().x)};
    block_reduce_r<3>(v, R, smem);
    if ((int)threadIdx.x < R) {
      partial[((size_t)k0 * nblocks + b) * R + threadIdx.x] = v[0];
      partial[((size_t)(k0 + 1) * nblocks + b) * R + threadIdx.x] = v[1];
      partial[((size_t)slot_norm * nblocks + b) * R + threadIdx.x] = v[2];
    }
  } else {
    double v[2] = {d0.get().x, d1.get().x};
    block_reduce_rx<2>(v, R, (double*)smem);
    if ((int)threadIdx.x < R) {
      partial[((size_t)k0 * nblocks + b) * R + threadIdx.x] = make_double2(v[0], 0.0);
      partial[((size_t)(k0 + 1) * nblocks + b) * R + threadIdx.x] = make_double2(v[1], 0.0);
    }
  }
}

}  // namespace gqt

namespace gqt {
// FP64 FMA throughput probe: 8 independent FMA chains per thread.
static __global__ void k_probe_dfma(double* __restrict__ sink, int iters, double b, double c) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1e-3 * threadIdx.x + k;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == -1.0) sink[blockIdx.x] = s;  // never true; keeps the chains alive
}
}  // namespace gqt


namespace gqt {

// ------------------------------------- several vectors per thread (SpMM form)
//
// For R >= 2 each thread handles VPT consecutive vectors of one site: the
// site's H~ row (indices, hoppings, diagonal) is loaded once for VPT vectors
// and every vector access is a VPT-wide contiguous load (16-byte loads for
// FP32 pairs), so instruction count per vector element drops by ~VPT.
// Vector tiles of the multi-vector kernels.  Lane lg of a site's G-lane group holds
// VPT of the site's R = G * VPT vectors, interleaved so that each load instruction
// of the group covers whole contiguous runs: FP32 pairs (16 B) at element offsets
// 2 lg + q G (q = 0, 2, ..), FP64 vectors (16 B) at lg + q G.  d[q] is vector
// vec_of<FP64>(lg, q, G) of the site.  ldg_v reads T_m (own and neighbour tiles,
// reused from L2 by later sites); ld_v and st_v move the read-once streams
// (T_{m-1}, the left vector, T_{m+1}) with the streaming (evict-first) hint so that
// they do not push T_m's reuse window out of L2.
template <bool FP64>
__device__ __forceinline__ int lane_offset(int lg) { return FP64 ? lg : 2 * lg; }
template <bool FP64>
__device__ __forceinline__ int vec_of(int lg, int q, int G) {
  return FP64 ? q * G + lg : (q & ~1) * G + 2 * lg + (q & 1);
}
template <int VPT>
__device__ __forceinline__ void ldg_v(float2 (&d)[VPT], const float2* __restrict__ p, int G) {
#pragma unroll
  for (int q = 0; q < VPT; q += 2) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p + (size_t)q * G));
    d[q] = make_float2(t.x, t.y);
    d[q + 1] = make_float2(t.z, t.w);
  }
}
template <int VPT>
__device__ __forceinline__ void ld_v(float2 (&d)[VPT], const float2* p, int G) {
#pragma unroll
  for (int q = 0; q < VPT; q += 2) {
    const float4 t = __ldcs(reinterpret_cast<const float4*>(p + (size_t)q * G));
    d[q] = make_float2(t.x, t.y);
    d[q + 1] = make_float2(t.z, t.w);
  }
}
template <int VPT>
__device__ __forceinline__ void st_v(float2* p, const float2 (&d)[VPT], int G) {
#pragma unroll
  for (int q = 0; q < VPT; q += 2)
    __stcs(reinterpret_cast<float4*>(p + (size_t)q * G), make_float4(d[q].x, d[q].y, d[q + 1].x, d[q + 1].y));
}
template <int VPT>
__device__ __forceinline__ void ldg_v(double2 (&d)[VPT], const double2* __restrict__ p, int G) {
#pragma unroll
  for (int q = 0; q < VPT; ++q) d[q] = __ldg(p + (size_t)q * G);
}
template <int VPT>
__device__ __forceinline__ void ld_v(double2 (&d)[VPT], const double2* p, int G) {
#pragma unroll
  for (int q = 0; q < VPT; ++q) d[q] = __ldcs(p + (size_t)q * G);
}
template <int VPT>
__device__ __forceinline__ void st_v(double2* p, const double2 (&d)[VPT], int G) {
#pragma unroll
  for (int q = 0; q < VPT; ++q) __stcs(p + (size_t)q * G, d[q]);
}

// One recurrence order for VPT vectors of each site, wavefront order over groups
// of VPT vectors (gs = log2(R / VPT)).  DBL: l = r doubling dots; otherwise Re <l|.>.
// Lane shuffles of the hopping types (a 64-bit or two-component value moves in parts).
__device__ __forceinline__ float shfl_g(float v, int src, int w) { return __shfl_sync(0xffffffffu, v, src, w); }
__device__ __forceinline__ double shfl_g(double v, int src, int w) { return __shfl_sync(0xffffffffu, v, src, w); }
__device__ __forceinline__ float2 shfl_g(float2 v, int src, int w) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src, w), __shfl_sync(0xffffffffu, v.y, src, w));
}
__device__ __forceinline__ double2 shfl_g(double2 v, int src, int w) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src, w), __shfl_sync(0xffffffffu, v.y, src, w));
}
template <class S>
__device__ __forceinline__ void put_re(S& h, S v) { h = v; }
__device__ __forceinline__ void put_re(float2& h, float v) { h.x = v; }
__device__ __forceinline__ void put_re(double2& h, double v) { h.x = v; }
template <class S>
__device__ __forceinline__ S get_re(S h) { return h; }
__device__ __forceinline__ float get_re(float2 h) { return h.x; }
__device__ __forceinline__ double get_re(double2 h) { return h.x; }

// One CTA's share of a wavefront segment with VPT vectors per thread: G = R/VPT
// consecutive lanes (gs = log2 G) serve one site, each lane its VPT vectors.  The
// loop runs over block-uniform offsets g0, so every lane of the block takes the same
// trip count (lanes past the segment end skip the work, not the loop).
//
// PF (requires KK + 1 <= G <= 32): the site's K indices, K hoppings and diagonal are
// fetched one iteration ahead, one item per lane of the G-lane group (slot g for
// lane g < K, the diagonal for lane K), while the current iteration's neighbour
// loads are in flight; the group then shares them by shuffles.  This takes the
// dependent index load off the iteration's critical path (index -> neighbour
// vector), which is what bounds the FP32 multi-vector form.
template <bool FP64, bool CH, int VPT, bool DBL, int KK, bool first, bool PF>
__device__ __forceinline__ void cheb_wave_vpt(const Ell<FP64, CH>& H, int4 tb, int R, int gs,
                                              const typename Prec<FP64>::V* __restrict__ tm1,
                                              const typename Prec<FP64>::V* tm2, typename Prec<FP64>::V* tout,
                                              const typename Prec<FP64>::V* __restrict__ l,
                                              DotAcc<typename Prec<FP64>::V> (&d0)[VPT],
                                              DotAcc<typename Prec<FP64>::V> (&d1)[VPT],
                                              DotAcc<typename Prec<FP64>::V> (&nl)[VPT],
                                              DotAcc<typename Prec<FP64>::V> (&nr)[VPT]) {
  using V = typename Prec<FP64>::V;
  using S = typename Prec<FP64>::S;
  using HT = typename Ell<FP64, CH>::HT;
  const size_t gb = (size_t)tb.x << gs, ge = (size_t)tb.y << gs;
  const size_t step = (size_t)tb.w * blockDim.x;
  const int gmask = (1 << gs) - 1;
  const int G = 1 << gs;
  const int lg = (int)threadIdx.x & gmask;
  int pidx = 0;
  HT phop{};
  auto fetch_next = [&](size_t gn) {
    if (gn < ge) {
      const int i = site_of(H, (int)(gn >> gs));
      if (lg < KK) {
        const size_t s = (size_t)lg * H.n + i;
        pidx = __ldg(H.idx + s);
        phop = __ldg(H.hop2 + s);
      } else if (lg == KK) {
        put_re(phop, __ldg(H.diag2 + i));
      }
    }
  };
  const size_t g_first = gb + (size_t)tb.z * blockDim.x;
  if (PF) fetch_next(g_first + threadIdx.x);
  for (size_t g0 = g_first; g0 < ge; g0 += step) {
    const size_t gi = g0 + threadIdx.x;
    int idx[KK];
    HT hv[KK];
    S dg;
    if constexpr (PF) {
      const int cidx = pidx;
      const HT chop = phop;
      fetch_next(gi + step);
#pragma unroll
      for (int k = 0; k < KK; ++k) {
        idx[k] = __shfl_sync(0xffffffffu, cidx, k, G);
        hv[k] = shfl_g(chop, k, G);
      }
      dg = get_re(shfl_g(chop, KK, G));
    }
    if (gi >= ge) continue;
    const int i = site_of(H, (int)(gi >> gs));
    const int r0 = lane_offset<FP64>(lg);
    const size_t base = (size_t)i * R + r0;
    V own[VPT], acc[VPT], lv[VPT];
    if constexpr (!PF) {
#pragma unroll
      for (int k = 0; k < KK; ++k) {
        const size_t s = (size_t)k * H.n + i;
        idx[k] = __ldg(H.idx + s);
        hv[k] = __ldg(H.hop2 + s);
      }
      dg = __ldg(H.diag2 + i);
    }
    ldg_v<VPT>(own, tm1 + base, G);
    if (first) {
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        acc[v].x = 0;
        acc[v].y = 0;
      }
    } else {
      ld_v<VPT>(acc, tm2 + base, G);
#pragma unroll
      for (int v = 0; v < VPT; ++v) acc[v] = cneg(acc[v]);
    }
    if (!DBL) ld_v<VPT>(lv, l + base, G);
#pragma unroll
    for (int k = 0; k < KK; ++k) {
      V nb[VPT];
      ldg_v<VPT>(nb, tm1 + (size_t)idx[k] * R + r0, G);
#pragma unroll
      for (int v = 0; v < VPT; ++v) acc[v] = cmul_acc(acc[v], hv[k], nb[v]);
    }
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      acc[v] = cmul_acc(acc[v], dg, own[v]);
      if (first) acc[v] = cscale(acc[v], (S)0.5);
    }
    st_v<VPT>(tout + base, acc, G);
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      if (DBL) {
        d0[v].add_norm(own[v]);
        d1[v].add_re(acc[v], own[v]);
      } else {
        if (first) {
          d0[v].add_re(lv[v], own[v]);
          nl[v].add_norm(lv[v]);
          nr[v].add_norm(own[v]);
        }
        d1[v].add_re(lv[v], acc[v]);
      }
    }
  }
}

template <bool FP64, int VPT, int NQ>
__device__ __forceinline__ void write_partials_vpt(double2 (&v)[NQ * VPT], int R, int G, double2* smem,
                                                   double2* __restrict__ partial, int nblocks, const int (&slot)[NQ]) {
  block_reduce_r<NQ * VPT>(v, G, smem);
  if ((int)threadIdx.x < G) {
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int w = 0; w < VPT; ++w)
        partial[((size_t)slot[q] * nblocks + blockIdx.x) * R + vec_of<FP64>(threadIdx.x, w, G)] = v[q * VPT + w];
  }
}

template <bool FP64, bool CH, int VPT, int KK, bool PF = false>
__global__ void __launch_bounds__(128, 5) k_cheb_re_wv(Ell<FP64, CH> H, const int4* __restrict__ tab, int R, int gs,
                                                       const typename Prec<FP64>::V* __restrict__ tm1,
                                                       const typename Prec<FP64>::V* tm2, typename Prec<FP64>::V* tout,
                                                       const typename Prec<FP64>::V* __restrict__ l,
                                                       double2* __restrict__ partial, int nblocks, int slot0,
                                                       int slot_norm, int first) {
  using V = typename Prec<FP64>::V;
  DotAcc<V> d0[VPT], d1[VPT], nl[VPT], nr[VPT];
  if (first)
    cheb_wave_vpt<FP64, CH, VPT, false, KK, true, PF>(H, tab[blockIdx.x], R, gs, tm1, tm2, tout, l, d0, d1, nl, nr);
  else
    cheb_wave_vpt<FP64, CH, VPT, false, KK, false, PF>(H, tab[blockIdx.x], R, gs, tm1, tm2, tout, l, d0, d1, nl, nr);
  const int G = 1 << gs;
  if (first) {
    double2 v[3 * VPT];
#pragma unroll
    for (int w = 0; w < VPT; ++w) {
      v[w] = d0[w].get();
      v[VPT + w] = d1[w].get();
      v[2 * VPT + w] = make_double2(nl[w].get().x, nr[w].get().x);
    }
    const int slots[3] = {slot0, slot0 + 1, slot_norm};
    write_partials_vpt<FP64, VPT, 3>(v, R, G, dyn_smem(), partial, nblocks, slots);
  } else {
    double2 v[VPT];
#pragma unroll
    for (int w = 0; w < VPT; ++w) v[w] = d1[w].get();
    const int slots[1] = {slot0};
    write_partials_vpt<FP64, VPT, 1>(v, R, G, dyn_smem(), partial, nblocks, slots);
  }
}

template <bool FP64, bool CH, int VPT, int KK, bool PF = false>
__global__ void __launch_bounds__(128, PF ? 5 : 6) k_cheb_dbl_wv(Ell<FP64, CH> H, const int4* __restrict__ tab, int R, int gs,
                                                        const typename Prec<FP64>::V* __restrict__ tm1,
                                                        const typename Prec<FP64>::V* tm2, typename Prec<FP64>::V* tout,
                                                        double2* __restrict__ partial, int nblocks, int m) {
  using V = typename Prec<FP64>::V;
  DotAcc<V> a0[VPT], a1[VPT], u0[VPT], u1[VPT];
  if (m == 1)
    cheb_wave_vpt<FP64, CH, VPT, true, KK, true, PF>(H, tab[blockIdx.x], R, gs, tm1, tm2, tout, nullptr, a0, a1, u0,
                                                     u1);
  else
    cheb_wave_vpt<FP64, CH, VPT, true, KK, false, PF>(H, tab[blockIdx.x], R, gs, tm1, tm2, tout, nullptr, a0, a1, u0,
                                                      u1);
  double2 v[2 * VPT];
#pragma unroll
  for (int w = 0; w < VPT; ++w) {
    v[w] = a0[w].get();
    v[VPT + w] = a1[w].get();
  }
  const int slots[2] = {2 * m - 2, 2 * m - 1};
  write_partials_vpt<FP64, VPT, 2>(v, R, 1 << gs, dyn_smem(), partial, nblocks, slots);
}


// Two-recurrence (l != r) steps in the multi-vector form: the lane layout, the
// block-uniform loop and the PF prefetch of cheb_wave_vpt, with chain A (from l)
// and chain B (from r) advanced together; dots and slots as k_cheb_pair_w.
template <bool FP64, bool CH, int VPT, int KK, bool first, bool PF>
__device__ __forceinline__ void cheb_pair_vpt(const Ell<FP64, CH>& H, int4 tb, int R, int gs,
                                              const typename Prec<FP64>::V* __restrict__ am1,
                                              const typename Prec<FP64>::V* __restrict__ bm1,
                                              const typename Prec<FP64>::V* am2, const typename Prec<FP64>::V* bm2,
                                              typename Prec<FP64>::V* aout, typename Prec<FP64>::V* bout,
                                              DotAcc<typename Prec<FP64>::V> (&d0)[VPT],
                                              DotAcc<typename Prec<FP64>::V> (&d1)[VPT],
                                              DotAcc<typename Prec<FP64>::V> (&nl)[VPT],
                                              DotAcc<typename Prec<FP64>::V> (&nr)[VPT]) {
  using V = typename Prec<FP64>::V;
  using S = typename Prec<FP64>::S;
  using HT = typename Ell<FP64, CH>::HT;
  const size_t gb = (size_t)tb.x << gs, ge = (size_t)tb.y << gs;
  const size_t step = (size_t)tb.w * blockDim.x;
  const int G = 1 << gs;
  const int lg = (int)threadIdx.x & (G - 1);
  int pidx = 0;
  HT phop{};
  auto fetch_next = [&](size_t gn) {
    if (gn < ge) {
      const int i = site_of(H, (int)(gn >> gs));
      if (lg < KK) {
        const size_t s = (size_t)lg * H.n + i;
        pidx = __ldg(H.idx + s);
        phop = __ldg(H.hop2 + s);
      } else if (lg == KK) {
        put_re(phop, __ldg(H.diag2 + i));
      }
    }
  };
  const size_t g_first = gb + (size_t)tb.z * blockDim.x;
  if (PF) fetch_next(g_first + threadIdx.x);
  for (size_t g0 = g_first; g0 < ge; g0 += step) {
    const size_t gi = g0 + threadIdx.x;
    int idx[KK];
    HT hv[KK];
    S dg;
    if constexpr (PF) {
      const int cidx = pidx;
      const HT chop = phop;
      fetch_next(gi + step);
#pragma unroll
      for (int k = 0; k < KK; ++k) {
        idx[k] = __shfl_sync(0xffffffffu, cidx, k, G);
        hv[k] = shfl_g(chop, k, G);
      }
      dg = get_re(shfl_g(chop, KK, G));
    }
    if (gi >= ge) continue;
    const int i = site_of(H, (int)(gi >> gs));
    const int r0 = lane_offset<FP64>(lg);
    const size_t base = (size_t)i * R + r0;
    if constexpr (!PF) {
#pragma unroll
      for (int k = 0; k < KK; ++k) {
        const size_t s = (size_t)k * H.n + i;
        idx[k] = __ldg(H.idx + s);
        hv[k] = __ldg(H.hop2 + s);
      }
      dg = __ldg(H.diag2 + i);
    }
    V ao[VPT], bo[VPT], a[VPT], b[VPT];
    ldg_v<VPT>(ao, am1 + base, G);
    ldg_v<VPT>(bo, bm1 + base, G);
    if (first) {
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        a[v] = cscale(ao[v], dg);
        b[v] = cscale(bo[v], dg);
      }
    } else {
      ld_v<VPT>(a, am2 + base, G);
      ld_v<VPT>(b, bm2 + base, G);
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        a[v] = cmul_acc(cneg(a[v]), dg, ao[v]);
        b[v] = cmul_acc(cneg(b[v]), dg, bo[v]);
      }
    }
#pragma unroll
    for (int k = 0; k < KK; ++k) {
      V na[VPT], nb[VPT];
      const size_t jb = (size_t)idx[k] * R + r0;
      ldg_v<VPT>(na, am1 + jb, G);
      ldg_v<VPT>(nb, bm1 + jb, G);
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        a[v] = cmul_acc(a[v], hv[k], na[v]);
        b[v] = cmul_acc(b[v], hv[k], nb[v]);
      }
    }
    if (first) {
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        a[v] = cscale(a[v], (S)0.5);
        b[v] = cscale(b[v], (S)0.5);
      }
    }
    st_v<VPT>(aout + base, a, G);
    st_v<VPT>(bout + base, b, G);
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      d0[v].add_re(ao[v], bo[v]);
      d1[v].add_re(ao[v], b[v]);
      if (first) {
        nl[v].add_norm(ao[v]);
        nr[v].add_norm(bo[v]);
      }
    }
  }
}

template <bool FP64, bool CH, int VPT, int KK, bool PF = false>
__global__ void __launch_bounds__(128, 5) k_cheb_pair_wv(Ell<FP64, CH> H, const int4* __restrict__ tab, int R, int gs,
                                                         const typename Prec<FP64>::V* __restrict__ am1,
                                                         const typename Prec<FP64>::V* __restrict__ bm1,
                                                         const typename Prec<FP64>::V* am2,
                                                         const typename Prec<FP64>::V* bm2,
                                                         typename Prec<FP64>::V* aout, typename Prec<FP64>::V* bout,
                                                         double2* __restrict__ partial, int nblocks, int m,
                                                         int slot_norm) {
  using V = typename Prec<FP64>::V;
  DotAcc<V> d0[VPT], d1[VPT], nl[VPT], nr[VPT];
  if (m == 1)
    cheb_pair_vpt<FP64, CH, VPT, KK, true, PF>(H, tab[blockIdx.x], R, gs, am1, bm1, am2, bm2, aout, bout, d0, d1, nl,
                                               nr);
  else
    cheb_pair_vpt<FP64, CH, VPT, KK, false, PF>(H, tab[blockIdx.x], R, gs, am1, bm1, am2, bm2, aout, bout, d0, d1, nl,
                                                nr);
  const int G = 1 << gs;
  if (m == 1) {
    double2 v[3 * VPT];
#pragma unroll
    for (int w = 0; w < VPT; ++w) {
      v[w] = d0[w].get();
      v[VPT + w] = d1[w].get();
      v[2 * VPT + w] = make_double2(nl[w].get().x, nr[w].get().x);
    }
    const int slots[3] = {0, 1, slot_norm};
    write_partials_vpt<FP64, VPT, 3>(v, R, G, dyn_smem(), partial, nblocks, slots);
  } else {
    double2 v[2 * VPT];
#pragma unroll
    for (int w = 0; w < VPT; ++w) {
      v[w] = d0[w].get();
      v[VPT + w] = d1[w].get();
    }
    const int slots[2] = {2 * m - 2, 2 * m - 1};
    write_partials_vpt<FP64, VPT, 2>(v, R, G, dyn_smem(), partial, nblocks, slots);
  }
}

}  // namespace gqt

namespace gqt {
// Bond gradients from slot gradients: bond b joins slots sa[b] and sb[b] (the two
// directions of one Hermitian pair); for the real and imaginary part of its
// hopping, dJ/dRe = Re(G_a + G_b) and dJ/dIm = Im(G_a) - Im(G_b).
static __global__ void k_bond_grad(const double2* __restrict__ gslot, long long n_slots,
                                   const long long* __restrict__ sa, const long long* __restrict__ sb, int nbonds,
                                   double* __restrict__ g_re, double* __restrict__ g_im) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbonds; b += gridDim.x * blockDim.x) {
    const long long ia = sa[b], ib = sb[b];
    if (ia < 0 || ia >= n_slots || ib < 0 || ib >= n_slots) {
      g_re[b] = CUDART_NAN;
      if (g_im) g_im[b] = CUDART_NAN;
      continue;
    }
    const double2 a = gslot[ia], c = gslot[ib];
    g_re[b] = a.x + c.x;
    if (g_im) g_im[b] = a.y - c.y;
  }
}

// beta[k][n] = c_k * kw[n] with trapezoid weights c_k of sigma_VAC at the last row.
static __global__ void k_trapezoid_outer(const double* __restrict__ c, int rows, const double* __restrict__ kw, int M,
                                         double* __restrict__ beta) {
  const size_t total = (size_t)rows * M;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x)
    beta[t] = c[t / M] * kw[t % M];
}
}  // namespace gqt
