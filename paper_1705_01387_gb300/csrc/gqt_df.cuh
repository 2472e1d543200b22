// gqt_df.cuh -- FP64-storage moment rows and evolution orders computed on the FP32 pipes.
//
// GB300 issues about 2 FP64 fused multiply-adds per clock per SM and 128 FP32
// ones, so the FP64 moment kernels (k_cheb_pair_w, k_cheb_dbl_w) are bound by
// the FP64 pipe, well below the HBM roofline.  These kernels keep FP64-sized
// storage (16 bytes per complex element) and FP64-level results, but do the
// arithmetic of the recursion (Eq. 21) and of the moment dots (Eqs. 28-30) on
// unevaluated pairs of FP32 numbers ("double-float": x = hi + lo with
// |lo| <= ulp(hi)/2, about 48 significant bits), using the error-free
// transformations of Dekker (1971) and Knuth (TwoSum), with TwoProduct by the
// fused multiply-add (Ogita, Rump and Oishi 2005):
//   TwoProduct(a, b): p = fl(a b), e = fma(a, b, -p), a b = p + e exactly;
//   TwoSum(a, b):     s = fl(a + b), v = s - a, e = (a - (s - v)) + (b - v),
//                     a + b = s + e exactly.
// A product of two pairs keeps p and e + a_hi b_lo + a_lo b_hi (the a_lo b_lo
// term is below 2^-48 of the product); sums keep the TwoSum error in the low
// word and renormalise once per element.  Every operation is written with the
// _rn intrinsics, which the compiler never contracts into fused multiply-adds
// (a contraction would break the error-free transformations).
//
// Storage: the chain vectors T_k are float4 per complex element
// (re.hi, re.lo, im.hi, im.lo); the caller's input vectors stay complex128 and
// are split on the first order only.  The Hamiltonian's 2H~ (real hoppings:
// float2 (hi, lo) per slot; complex: float4) and 2U/dE (float2) are split once
// per handle from its FP64 arrays.  Moment partial sums leave each thread as
// FP64 (hi + lo) and are reduced in FP64 as in the FP64 kernels, into the same
// partial slots, so k_reduce_dbl combines them unchanged.
#pragma once

namespace gqt {

template <bool CH>
struct DfHop;
template <>
struct DfHop<false> {
  using T = float2;  // (hi, lo) of a real 2H~_ij
};
template <>
struct DfHop<true> {
  using T = float4;  // (re.hi, re.lo, im.hi, im.lo) of a complex 2H~_ij
};

template <bool CH>
struct DfEll {
  int n = 0;
  int K = 0;
  const int* idx = nullptr;                    // [K][n]
  const typename DfHop<CH>::T* hop = nullptr;  // [K][n]
  const float2* diag = nullptr;                // [n]
  const typename DfHop<CH>::T* xhop = nullptr;  // [K][n] 2[X,H~]_ij = -dx_ij 2H~_ij (commutator orders)
  float2 h0 = {0.f, 0.f};  // the common 2H~_ij of handles whose slots all hold one real hopping
};

// ---------------------------------------------------------------- pair arithmetic

// An FP64 value as a pair (the first order reads the caller's FP64 vectors).
__device__ __forceinline__ float2 df_split(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ float4 df_split(double2 z) {
  const float2 a = df_split(z.x), b = df_split(z.y);
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ double df_value(float h, float l) { return (double)h + (double)l; }

// (sh, sl) += (ah, al) * (bh, bl), the sum kept unnormalised (sl collects the
// TwoSum error and the low part of the product).
__device__ __forceinline__ void df_mac(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  const float s = __fadd_rn(sh, p);
  const float v = __fsub_rn(s, sh);
  const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, v)), __fsub_rn(p, v));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(t, e));
}

// (sh, sl) -> normalised pair (TwoSum of the two words).
__device__ __forceinline__ float2 df_norm(float sh, float sl) {
  const float s = __fadd_rn(sh, sl);
  const float v = __fsub_rn(s, sh);
  const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, v)), __fsub_rn(sl, v));
  return make_float2(s, t);
}

// Complex accumulator (re: x, y; im: z, w as hi, lo), unnormalised.
struct DfC {
  float rh, rl, ih, il;
};

__device__ __forceinline__ DfC dfc_zero() { return DfC{0.f, 0.f, 0.f, 0.f}; }
__device__ __forceinline__ DfC dfc_neg(float4 a) { return DfC{-a.x, -a.y, -a.z, -a.w}; }

// acc += c * x, c real pair
__device__ __forceinline__ void dfc_mac(DfC& a, float2 c, float4 x) {
  df_mac(a.rh, a.rl, c.x, c.y, x.x, x.y);
  df_mac(a.ih, a.il, c.x, c.y, x.z, x.w);
}
// acc += c * x, c complex pair (re.hi, re.lo, im.hi, im.lo)
__device__ __forceinline__ void dfc_mac(DfC& a, float4 c, float4 x) {
  df_mac(a.rh, a.rl, c.x, c.y, x.x, x.y);
  df_mac(a.rh, a.rl, -c.z, -c.w, x.z, x.w);
  df_mac(a.ih, a.il, c.x, c.y, x.z, x.w);
  df_mac(a.ih, a.il, c.z, c.w, x.x, x.y);
}

__device__ __forceinline__ float4 dfc_out(const DfC& a, bool half) {
  float2 r = df_norm(a.rh, a.rl), i = df_norm(a.ih, a.il);
  if (half) {  // exact scaling of both words (T_1 = H~ T_0 from 2H~)
    r.x *= 0.5f;
    r.y *= 0.5f;
    i.x *= 0.5f;
    i.y *= 0.5f;
  }
  return make_float4(r.x, r.y, i.x, i.y);
}

// Per-thread real dot accumulator: sum of Re conj(a) b or |a|^2 over the
// thread's elements, as an unnormalised pair; FP64 once per thread.
struct DfDot {
  float h = 0.f, l = 0.f;
  __device__ __forceinline__ void add_re(float4 a, float4 b) {
    df_mac(h, l, a.x, a.y, b.x, b.y);
    df_mac(h, l, a.z, a.w, b.z, b.w);
  }
  __device__ __forceinline__ void add_norm(float4 a) { add_re(a, a); }
  __device__ __forceinline__ double get() const { return df_value(h, l); }
};

// ---------------------------------------------------------------- split of H~

// 2H~ and 2U/dE of an FP64 handle as pairs (once per handle).
template <bool CH>
__global__ void k_split_hamiltonian(long long nslots, const void* __restrict__ hop64, int n,
                                    const double* __restrict__ diag64, void* __restrict__ hop_df,
                                    float2* __restrict__ diag_df) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < nslots; s += stride) {
    if (CH)
      ((float4*)hop_df)[s] = df_split(((const double2*)hop64)[s]);
    else
      ((float2*)hop_df)[s] = df_split(((const double*)hop64)[s]);
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride)
    diag_df[i] = df_split(diag64[i]);
}

// 2[X,H~] slot values -dx_ij 2H~_ij (Eq. 34 with [X,H]_ij = -dx_ij H_ij) as pairs,
// formed in FP64 and split once per handle.
template <bool CH>
__global__ void k_split_xhop(long long nslots, const void* __restrict__ hop64, const double* __restrict__ dx,
                             void* __restrict__ xhop_df) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < nslots; s += stride) {
    const double d = -dx[s];
    if (CH) {
      const double2 h = ((const double2*)hop64)[s];
      ((float4*)xhop_df)[s] = df_split(make_double2(d * h.x, d * h.y));
    } else {
      ((float2*)xhop_df)[s] = df_split(d * ((const double*)hop64)[s]);
    }
  }
}

// ---------------------------------------------------------------- moment rows

// Element e's chain value: a pair vector, or (first order) the caller's FP64
// vector split on the fly.
template <bool IN64>
__device__ __forceinline__ float4 df_load(const void* v, size_t e) {
  if (IN64) return df_split(__ldg((const double2*)v + e));
  return __ldg((const float4*)v + e);
}

// T_m = 2H~ T_{m-1} - T_{m-2} at element i of a pair chain (T_1 = H~ T_0 when
// FIRST); own = T_{m-1}[i], nb[k] = T_{m-1}[idx[k][i]].
template <bool CH, int KK, bool FIRST>
__device__ __forceinline__ float4 df_step(const typename DfHop<CH>::T (&hv)[KK], float2 dg, float4 own,
                                          const float4 (&nb)[KK], float4 tm2) {
  DfC a = FIRST ? dfc_zero() : dfc_neg(tm2);
  dfc_mac(a, dg, own);
#pragma unroll
  for (int k = 0; k < KK; ++k) dfc_mac(a, hv[k], nb[k]);
  return dfc_out(a, FIRST);
}

// (sh, sl) += (bh, bl) for pairs, unnormalised (TwoSum of the high words, the
// low words and the TwoSum error added into sl).
__device__ __forceinline__ void df_add(float& sh, float& sl, float bh, float bl) {
  const float s = __fadd_rn(sh, bh);
  const float v = __fsub_rn(s, sh);
  const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, v)), __fsub_rn(bh, v));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(bl, t));
}

// a += h0 * (sum_k nb[k]) for a real pair h0: the neighbour values are summed as
// pairs first, so one product with h0 replaces KK.
template <int KK>
__device__ __forceinline__ void dfc_mac_sum(DfC& a, float2 h0, const float4 (&nb)[KK]) {
  float rh = nb[0].x, rl = nb[0].y, ih = nb[0].z, il = nb[0].w;
#pragma unroll
  for (int k = 1; k < KK; ++k) {
    df_add(rh, rl, nb[k].x, nb[k].y);
    df_add(ih, il, nb[k].z, nb[k].w);
  }
  df_mac(a.rh, a.rl, h0.x, h0.y, rh, rl);
  df_mac(a.ih, a.il, h0.x, h0.y, ih, il);
}

// T_m at one element when every hopping equals h0 (a real 2H~ value), as
// df_step (T_1 = H~ T_0 when FIRST).
template <int KK, bool FIRST = false>
__device__ __forceinline__ float4 df_step_uh(float2 h0, float2 dg, float4 own, const float4 (&nb)[KK], float4 tm2) {
  DfC a = FIRST ? dfc_zero() : dfc_neg(tm2);
  dfc_mac(a, dg, own);
  dfc_mac_sum<KK>(a, h0, nb);
  return dfc_out(a, FIRST);
}

// T_m with the hoppings of the slots (hv) or, when UH, the common value H.h0.
template <bool CH, int KK, bool FIRST, bool UH>
__device__ __forceinline__ float4 df_step_any(const DfEll<CH>& H, const typename DfHop<CH>::T (&hv)[KK], float2 dg,
                                              float4 own, const float4 (&nb)[KK], float4 tm2) {
  if constexpr (UH)
    return df_step_uh<KK, FIRST>(H.h0, dg, own, nb, tm2);
  else
    return df_step<CH, KK, FIRST>(hv, dg, own, nb, tm2);
}

// VAC rows by two recurrences (the pair form of k_cheb_pair_w): chain A from l,
// chain B from r, A_k = T_k l, B_k = T_k r; step m writes A_m, B_m and adds
// Re <A_{m-1}|B_{m-1}> (moment slot 2m-2) and Re <A_{m-1}|B_m> (slot 2m-1); the
// first step reads l and r as FP64, adds |l|^2 and |r|^2 (slot_norm) and also
// writes l and r as pairs into a0out, b0out (the T_{m-2} of step 2).  R = 1,
// wavefront CTA order, one element per thread.
template <bool CH, int KK, bool FIRST>
__global__ void __launch_bounds__(256, 3) k_cheb_pair_df(DfEll<CH> H, const int4* __restrict__ tab,
                                                         const void* __restrict__ am1, const void* __restrict__ bm1,
                                                         const float4* am2, const float4* bm2, float4* aout,
                                                         float4* bout, float4* __restrict__ a0out,
                                                         float4* __restrict__ b0out, double2* __restrict__ partial,
                                                         int nblocks, int m, int slot_norm) {
  using HT = typename DfHop<CH>::T;
  double2* smem = dyn_smem();
  const int b = blockIdx.x;
  const int4 tb = tab[b];
  const size_t segb = (size_t)tb.x, sege = (size_t)tb.y;
  const size_t step = (size_t)tb.w * blockDim.x;
  DfDot d0, d1, nl, nr;
  for (size_t e = segb + (size_t)tb.z * blockDim.x + threadIdx.x; e < sege; e += step) {
    const int i = (int)e;
    int idx[KK];
    HT hv[KK];
#pragma unroll
    for (int k = 0; k < KK; ++k) {
      const size_t s = (size_t)k * H.n + i;
      idx[k] = __ldg(H.idx + s);
      hv[k] = __ldg(H.hop + s);
    }
    const float2 dg = __ldg(H.diag + i);
    const float4 ao = df_load<FIRST>(am1, e), bo = df_load<FIRST>(bm1, e);
    float4 a2 = make_float4(0.f, 0.f, 0.f, 0.f), b2 = a2;
    if (!FIRST) {
      a2 = am2[e];
      b2 = bm2[e];
    }
    float4 na[KK], nbv[KK];
#pragma unroll
    for (int k = 0; k < KK; ++k) {
      na[k] = df_load<FIRST>(am1, (size_t)idx[k]);
      nbv[k] = df_load<FIRST>(bm1, (size_t)idx[k]);
    }
    const float4 a = df_step<CH, KK, FIRST>(hv, dg, ao, na, a2);
    const float4 bb = df_step<CH, KK, FIRST>(hv, dg, bo, nbv, b2);
    aout[e] = a;
    bout[e] = bb;
    d0.add_re(ao, bo);
    d1.add_re(ao, bb);
    if (FIRST) {
      a0out[e] = ao;
      b0out[e] = bo;
      nl.add_norm(ao);
      nr.add_norm(bo);
    }
  }
  const int k0 = 2 * m - 2;
  if (FIRST) {
    double v[4] = {d0.get(), d1.get(), nl.get(), nr.get()};
    block_reduce_rx<4>(v, 1, (double*)smem);
    if (threadIdx.x == 0) {
      partial[(size_t)k0 * nblocks + b] = make_double2(v[0], 0.0);
      partial[(size_t)(k0 + 1) * nblocks + b] = make_double2(v[1], 0.0);
      partial[(size_t)slot_norm * nblocks + b] = make_double2(v[2], v[3]);
    }
  } else {
    double v[2] = {d0.get(), d1.get()};
    block_reduce_rx<2>(v, 1, (double*)smem);
    if (threadIdx.x == 0) {
      partial[(size_t)k0 * nblocks + b] = make_double2(v[0], 0.0);
      partial[(size_t)(k0 + 1) * nblocks + b] = make_double2(v[1], 0.0);
    }
  }
}

// l = r rows (DOS, MSD) by the doubling identities (the pair form of
// k_cheb_dbl_w): step m writes u_m and adds <u_{m-1}|u_{m-1}> (slot 2m-2) and
// Re <u_m|u_{m-1}> (slot 2m-1); the first step reads u_0 as FP64 and also writes
// it as pairs into t0out (the T_{m-2} of step 2).  R = 1, wavefront CTA order,
// U elements in flight per thread.
template <bool CH, int KK, int U, bool FIRST>
__global__ void __launch_bounds__(256, 3) k_cheb_dbl_df(DfEll<CH> H, const int4* __restrict__ tab,
                                                        const void* __restrict__ tm1, const float4* tm2,
                                                        float4* tout, float4* __restrict__ t0out,
                                                        double2* __restrict__ partial, int nblocks, int m) {
  using HT = typename DfHop<CH>::T;
  double2* smem = dyn_smem();
  const int b = blockIdx.x;
  const int4 tb = tab[b];
  const size_t segb = (size_t)tb.x, sege = (size_t)tb.y;
  const size_t step = (size_t)tb.w * blockDim.x;
  DfDot a0, a1;
  for (size_t e0 = segb + (size_t)tb.z * blockDim.x + threadIdx.x; e0 < sege; e0 += (size_t)U * step) {
    int idx[U][KK];
    HT hv[U][KK];
    float2 dg[U];
    float4 own[U], t2[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const size_t e = e0 + u * step;
      ok[u] = e < sege;
      const size_t ee = ok[u] ? e : e0;
      const int i = (int)ee;
#pragma unroll
      for (int k = 0; k < KK; ++k) {
        const size_t s = (size_t)k * H.n + i;
        idx[u][k] = __ldg(H.idx + s);
        hv[u][k] = __ldg(H.hop + s);
      }
      dg[u] = __ldg(H.diag + i);
      own[u] = df_load<FIRST>(tm1, ee);
      t2[u] = FIRST ? make_float4(0.f, 0.f, 0.f, 0.f) : tm2[ee];
    }
    float4 nb[U][KK];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < KK; ++k) nb[u][k] = df_load<FIRST>(tm1, (size_t)idx[u][k]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float4 a = df_step<CH, KK, FIRST>(hv[u], dg[u], own[u], nb[u], t2[u]);
      if (ok[u]) {
        const size_t e = e0 + u * step;
        tout[e] = a;
        if (FIRST) t0out[e] = own[u];
        a0.add_norm(own[u]);
        a1.add_re(a, own[u]);
      }
    }
  }
  double v[2] = {a0.get(), a1.get()};
  block_reduce_rx<2>(v, 1, (double*)smem);
  if (threadIdx.x == 0) {
    const int k0 = 2 * m - 2;
    partial[(size_t)k0 * nblocks + b] = make_double2(v[0], 0.0);
    partial[(size_t)(k0 + 1) * nblocks + b] = make_double2(v[1], 0.0);
  }
}

// ---------------------------------------------------------------- evolution

// U(dt) psi = sum_m c_m T_m(H~) psi (Eq. 17) for NSET vector sets sharing H~,
// R = 1, on pairs of FP32 numbers: the chains T_m as pairs (16 bytes per complex
// element, the size of the FP64 workspace), the sum of c_m T_m as pairs, the
// caller's FP64 vectors split at the first order and formed again at the last
// (hi + lo of two FP32 numbers is exact in FP64).  Orders by phase:
//   PH 0 (m = 0, 1): out = T_1 = H~ psi, t0 = psi as pairs, acc = c0 psi + c1 T_1;
//                    |psi|^2 partials (slot);
//   PH 1 (2 <= m < Np - 1): out = 2H~ t1 - t2 (over t2, same element and thread),
//                    acc += c0 out;
//   PH 2 (m = Np - 1): psi = acc + c0 (2H~ t1 - t2) in FP64, |psi|^2 partials;
//   PH 3 (Np <= 2): psi = acc in FP64, |psi|^2 partials.
// c0, c1: complex coefficients as pairs (re.hi, re.lo, im.hi, im.lo).  The
// partial slots are those of k_evolve (k_norm_check reads them).
template <int NSET>
struct DfEvo {
  double2* psi[NSET];
  const float4* t1[NSET];
  const float4* t2[NSET];
  float4* out[NSET];
  float4* t0[NSET];
  float4* acc[NSET];
};

__device__ __forceinline__ double2 df_to_d2(float4 f) { return make_double2(df_value(f.x, f.y), df_value(f.z, f.w)); }
__device__ __forceinline__ DfC dfc_of(float4 a) { return DfC{a.x, a.y, a.z, a.w}; }

template <bool CH, int KK, bool UH = false>
__device__ __forceinline__ void df_row_ops(const DfEll<CH>& H, int i, int (&idx)[KK],
                                           typename DfHop<CH>::T (&hv)[KK], float2& dg) {
#pragma unroll
  for (int k = 0; k < KK; ++k) {
    const size_t s = (size_t)k * H.n + i;
    idx[k] = __ldg(H.idx + s);
    if (!UH) hv[k] = __ldg(H.hop + s);
  }
  dg = __ldg(H.diag + i);
}

template <bool CH, int KK, int NSET, int PH, bool UH = false>
__global__ void __launch_bounds__(256) k_evolve_df(DfEll<CH> H, const int4* __restrict__ tab, DfEvo<NSET> A,
                                                   float4 c0, float4 c1, double2* __restrict__ partial, int nblocks,
                                                   int slot) {
  using HT = typename DfHop<CH>::T;
  const int4 tb = tab[blockIdx.x];
  const size_t sege = (size_t)tb.y, step = (size_t)tb.w * blockDim.x;
  DfDot nrm[NSET];
  for (size_t e = (size_t)tb.x + (size_t)tb.z * blockDim.x + threadIdx.x; e < sege; e += step) {
    const int i = (int)e;
    if (PH == 3) {
#pragma unroll
      for (int q = 0; q < NSET; ++q) {
        const float4 f = A.acc[q][e];
        A.psi[q][e] = df_to_d2(f);
        nrm[q].add_norm(f);
      }
      continue;
    }
    int idx[KK];
    HT hv[KK];
    float2 dg;
    df_row_ops<CH, KK, UH>(H, i, idx, hv, dg);
#pragma unroll
    for (int q = 0; q < NSET; ++q) {
      float4 nb[KK];
      if (PH == 0) {
        const float4 own = df_load<true>(A.psi[q], e);
#pragma unroll
        for (int k = 0; k < KK; ++k) nb[k] = df_load<true>(A.psi[q], (size_t)idx[k]);
        const float4 y = df_step_any<CH, KK, true, UH>(H, hv, dg, own, nb, make_float4(0.f, 0.f, 0.f, 0.f));
        A.out[q][e] = y;
        A.t0[q][e] = own;
        DfC a = dfc_zero();
        dfc_mac(a, c0, own);
        dfc_mac(a, c1, y);
        A.acc[q][e] = dfc_out(a, false);
        nrm[q].add_norm(own);
      } else {
        const float4 own = __ldg(A.t1[q] + e);
#pragma unroll
        for (int k = 0; k < KK; ++k) nb[k] = __ldg(A.t1[q] + idx[k]);
        const float4 y = df_step_any<CH, KK, false, UH>(H, hv, dg, own, nb, A.t2[q][e]);
        DfC a = dfc_of(A.acc[q][e]);
        dfc_mac(a, c0, y);
        const float4 f = dfc_out(a, false);
        if (PH == 1) {
          A.out[q][e] = y;
          A.acc[q][e] = f;
        } else {
          A.psi[q][e] = df_to_d2(f);
          nrm[q].add_norm(f);
        }
      }
    }
  }
  if (PH != 1) {
    double v[NSET];
#pragma unroll
    for (int q = 0; q < NSET; ++q) v[q] = nrm[q].get();
    block_reduce_rx<NSET>(v, 1, reinterpret_cast<double*>(dyn_smem()));
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < NSET; ++q) partial[(size_t)(slot + q) * nblocks + blockIdx.x] = make_double2(v[q], 0.0);
    }
  }
}

// One MSD time step's coupled orders (Eqs. 17, 18, 22, 24) on pairs, R = 1:
//   u_m = T_m(H~) p,  z_m = [X, T_m] p + T_m px,
//   z_m = 2[X,H~] u_{m-1} + 2H~ z_{m-1} - z_{m-2}  (z_1 = [X,H~] p + H~ px),
//   accp += c_m u_m (-> U(dt) p), accx += c_m z_m (-> [X,U(dt)]p + U(dt)px).
// Phases as k_evolve_df (PH 0 also writes p and px as pairs into u0, z0); the
// partial slots are those of k_msd_evolve (k_norm_check_msd reads them).
struct DfMsd {
  double2* p;
  double2* px;
  const float4* u1;
  const float4* u2;
  const float4* z1;
  const float4* z2;
  float4* uo;
  float4* zo;
  float4* u0;
  float4* z0;
  float4* accp;
  float4* accx;
};

template <bool CH, int KK, int PH, bool UH = false>
__global__ void __launch_bounds__(256) k_msd_evolve_df(DfEll<CH> H, const int4* __restrict__ tab, DfMsd B, float4 c0,
                                                       float4 c1, double2* __restrict__ partial, int nblocks,
                                                       int slot) {
  using HT = typename DfHop<CH>::T;
  const int4 tb = tab[blockIdx.x];
  const size_t sege = (size_t)tb.y, step = (size_t)tb.w * blockDim.x;
  DfDot n0, n1;
  for (size_t e = (size_t)tb.x + (size_t)tb.z * blockDim.x + threadIdx.x; e < sege; e += step) {
    const int i = (int)e;
    if (PH == 3) {
      const float4 fp = B.accp[e], fx = B.accx[e];
      B.p[e] = df_to_d2(fp);
      B.px[e] = df_to_d2(fx);
      n0.add_norm(fp);
      n1.add_norm(fx);
      continue;
    }
    int idx[KK];
    HT hv[KK];
    float2 dg;
    df_row_ops<CH, KK, UH>(H, i, idx, hv, dg);
    float4 uo, zo;  // u_m and z_m at this element
    float4 u_own, z_own;
    if (PH == 0) {
      u_own = df_load<true>(B.p, e);
      z_own = df_load<true>(B.px, e);
      float4 un[KK];
#pragma unroll
      for (int k = 0; k < KK; ++k) un[k] = df_load<true>(B.p, (size_t)idx[k]);
      uo = df_step_any<CH, KK, true, UH>(H, hv, dg, u_own, un, make_float4(0.f, 0.f, 0.f, 0.f));
      DfC a = dfc_zero();
      dfc_mac(a, dg, z_own);
      float4 zn[KK];
#pragma unroll
      for (int k = 0; k < KK; ++k) zn[k] = df_load<true>(B.px, (size_t)idx[k]);
      if constexpr (UH) {
        dfc_mac_sum<KK>(a, H.h0, zn);
      } else {
#pragma unroll
        for (int k = 0; k < KK; ++k) dfc_mac(a, hv[k], zn[k]);
      }
#pragma unroll
      for (int k = 0; k < KK; ++k) dfc_mac(a, __ldg(H.xhop + (size_t)k * H.n + i), un[k]);
      zo = dfc_out(a, true);
    } else {
      u_own = __ldg(B.u1 + e);
      z_own = __ldg(B.z1 + e);
      float4 un[KK];
#pragma unroll
      for (int k = 0; k < KK; ++k) un[k] = __ldg(B.u1 + idx[k]);
      uo = df_step_any<CH, KK, false, UH>(H, hv, dg, u_own, un, B.u2[e]);
      DfC a = dfc_neg(B.z2[e]);
      dfc_mac(a, dg, z_own);
      float4 zn[KK];
#pragma unroll
      for (int k = 0; k < KK; ++k) zn[k] = __ldg(B.z1 + idx[k]);
      if constexpr (UH) {
        dfc_mac_sum<KK>(a, H.h0, zn);
      } else {
#pragma unroll
        for (int k = 0; k < KK; ++k) dfc_mac(a, hv[k], zn[k]);
      }
#pragma unroll
      for (int k = 0; k < KK; ++k) dfc_mac(a, __ldg(H.xhop + (size_t)k * H.n + i), un[k]);
      zo = dfc_out(a, false);
    }
    if (PH == 0) {
      B.uo[e] = uo;
      B.zo[e] = zo;
      B.u0[e] = u_own;
      B.z0[e] = z_own;
      DfC ap = dfc_zero(), ax = dfc_zero();
      dfc_mac(ap, c0, u_own);
      dfc_mac(ap, c1, uo);
      dfc_mac(ax, c0, z_own);
      dfc_mac(ax, c1, zo);
      B.accp[e] = dfc_out(ap, false);
      B.accx[e] = dfc_out(ax, false);
      n0.add_norm(u_own);
    } else {
      DfC ap = dfc_of(B.accp[e]), ax = dfc_of(B.accx[e]);
      dfc_mac(ap, c0, uo);
      dfc_mac(ax, c0, zo);
      const float4 fp = dfc_out(ap, false), fx = dfc_out(ax, false);
      if (PH == 1) {
        B.uo[e] = uo;
        B.zo[e] = zo;
        B.accp[e] = fp;
        B.accx[e] = fx;
      } else {
        B.p[e] = df_to_d2(fp);
        B.px[e] = df_to_d2(fx);
        n0.add_norm(fp);
        n1.add_norm(fx);
      }
    }
  }
  if (PH != 1) {
    double v[2] = {n0.get(), n1.get()};
    block_reduce_rx<2>(v, 1, reinterpret_cast<double*>(dyn_smem()));
    if (threadIdx.x == 0) {
      partial[(size_t)slot * nblocks + blockIdx.x] = make_double2(v[0], 0.0);
      partial[(size_t)(slot + 1) * nblocks + blockIdx.x] = make_double2(v[1], 0.0);
    }
  }
}

}  // namespace gqt
