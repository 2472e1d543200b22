// gqt_tile.cuh -- two Chebyshev orders per launch on honeycomb lattices
// (temporal blocking of the paired-FP32 rows, Eq. 21, staged through L2).
//
// A single-order launch reads T_m (its gathers hit L2), T_{m-1} and H~, and
// writes T_{m+1}: for the two-recurrence VAC row 140 bytes per orbital, 280 per
// two orders.  Here each CTA walks down a band of BW honeycomb cells (the
// built-in layout: site 2(c1 + L1 c2) + s, periodic), one cell row per
// iteration, and in iteration t
//   - computes T_{m+1} = 2H~T_m - T_{m-1} on row y0 - 1 + t of the band and
//     writes it to its output vector, and
//   - computes T_{m+2} = 2H~T_{m+1} - T_m on row y0 + t - 3, reading T_{m+1}
//     back from rows written one to three iterations before (they are still in
//     L1 or L2) and writes it to the second output vector.
// One barrier per row orders the two (a CTA's global writes before
// __syncthreads are visible to its threads after it).  From DRAM this moves,
// per two orders and orbital, T_m, T_{m-1} and H~ once and the two outputs
// once: 4 x 16 + 32 + 2 x 32 = 160 bytes for the VAC row instead of 280 (l = r
// rows: 2 x 16 + 32 + 2 x 16 = 96 instead of 184); the index array is not read at all, since the
// neighbours follow from the cell layout (one slot order per sublattice,
// checked on the host when the handle is built).
//
// Neighbours in the layout: A(c1,c2) -> B(c1,c2), B(c1+1,c2-1), B(c1,c2-1);
// B(c1,c2) -> A(c1,c2), A(c1-1,c2+1), A(c1,c2+1).  So T_{m+2} on the band needs
// T_{m+1} on the band plus, per row, one A site left of it (cell B1 - 1) and one
// B site right of it (cell B1 + BW), and on one row above and below the CTA's
// rows.  The CTA computes those itself (a prologue for the two halo columns,
// and two extra rows in the walk) from the inputs, which no CTA writes.  The
// neighbouring CTA writes the same T_{m+1} entries from the same inputs by the
// same instructions: both writes carry the same bits, so whichever a read
// observes is the value.  Recomputation: 2 of 2 BW sites per row and 2 rows per
// segment of a CTA (146 rows on the 4096 x 2048 lattice).
//
// Work split: one CTA per band and segment of rows, the segments as many as the
// resident CTAs allow, so that the CTAs of a segment walk its rows across all
// bands at about the same time (contiguous DRAM rows).  With more bands than
// resident CTAs the band rows, band-major, are cut into gridDim.x equal ranges
// instead; a range that crosses a band's end is walked as two pieces.  The
// two-chain kernel also prefetches the rows it will stream two rows ahead into
// L2 (bulk prefetch, one instruction per array and row).
//
// Arithmetic, dots and partial-sum slots are those of k_cheb_pair_df (NC = 2
// chains, A from l and B from r) and k_cheb_dbl_df (NC = 1, l = r): the pass
// over steps m and m + 1 adds the dots of moment slots 2m-2 .. 2m+1.  The
// outputs go to buffers other than the inputs.  When every slot holds the same
// real hopping (the Anderson form), the UH instances read no hop array and sum
// a row's neighbour values before one product with it (136 and 72 bytes per
// orbital instead of 160 and 96).
//
// The same walk serves FP32-storage handles with R = 2..16 vectors per site
// (k_cheb2_honey_wv, below): G = R/2 lanes per site, FP32 arithmetic in the
// single-order kernels' order, FP32 compensated dots per vector.
#pragma once

namespace gqt {


// Honeycomb cell layout of a handle: cell counts and, per sublattice s and ELL
// slot k, the cell offsets (o1, o2) of that slot's neighbour (on sublattice 1 - s).
struct Honey {
  int L1 = 0, L2 = 0;
  int o1[2][3] = {}, o2[2][3] = {};
};

// Band width for L1 cells: the largest of 128, 64, 32 dividing it (0: none).
__host__ __device__ inline int tl_band_width(int L1) {
  return L1 % 128 == 0 ? 128 : L1 % 64 == 0 ? 64 : L1 % 32 == 0 ? 32 : 0;
}

// Loads of a chain vector: inputs of the launch through the read-only path,
// vectors this launch writes (T_{m+1}) through plain coherent loads.
template <bool RO>
__device__ __forceinline__ float4 tl_ld(const float4* p, int i) {
  if (RO) return __ldg(p + i);
  return p[i];
}

// L2 prefetch of a contiguous range (16-byte aligned, a multiple of 16 bytes).
__device__ __forceinline__ void tl_prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The operands of one order at a site: H~ row, own value, the three neighbours
// and the order before, for NC chains.
template <bool CH, int NC>
struct TlSite {
  typename DfHop<CH>::T hv[3];
  float2 dg;
  float4 own[NC], nb[NC][3], prev[NC];
};

// Loads for site i with neighbours j[3]: in = the order the step multiplies,
// pv = the order before.
template <bool CH, int NC, bool IN_RO, bool UH = false>
__device__ __forceinline__ void tl_load(TlSite<CH, NC>& S, const DfEll<CH>& H, int i, const int (&j)[3],
                                        const float4* in0, const float4* in1, const float4* __restrict__ pv0,
                                        const float4* __restrict__ pv1) {
  if (!UH) {
#pragma unroll
    for (int k = 0; k < 3; ++k) S.hv[k] = __ldg(H.hop + (size_t)k * H.n + i);
  }
  S.dg = __ldg(H.diag + i);
#pragma unroll
  for (int ch = 0; ch < NC; ++ch) {
    const float4* in = ch ? in1 : in0;
    S.own[ch] = tl_ld<IN_RO>(in, i);
#pragma unroll
    for (int k = 0; k < 3; ++k) S.nb[ch][k] = tl_ld<IN_RO>(in, j[k]);
    S.prev[ch] = __ldg((ch ? pv1 : pv0) + i);
  }
}

// UH: every hopping is the real value H.h0 (no hop array is read).
template <bool CH, int NC, bool UH = false>
__device__ __forceinline__ void tl_compute(const TlSite<CH, NC>& S, const DfEll<CH>& H, float4 (&v)[NC]) {
#pragma unroll
  for (int ch = 0; ch < NC; ++ch) {
    if (UH)
      v[ch] = df_step_uh<3>(H.h0, S.dg, S.own[ch], S.nb[ch], S.prev[ch]);
    else
      v[ch] = df_step<CH, 3, false>(S.hv, S.dg, S.own[ch], S.nb[ch], S.prev[ch]);
  }
}

// Dots of one order at an owned site: NC = 2, Re <A_k|B_k> and Re <A_k|B_k+1>;
// NC = 1, <u_k|u_k> and Re <u_k+1|u_k>.
template <int NC>
__device__ __forceinline__ void tl_dots(DfDot& p, DfDot& q, const float4 (&own)[NC], const float4 (&v)[NC]) {
  if (NC == 2) {
    p.add_re(own[0], own[NC - 1]);
    q.add_re(own[0], v[NC - 1]);
  } else {
    p.add_norm(own[0]);
    q.add_re(v[0], own[0]);
  }
}

// A thread's site in its band row (cell c1, sublattice s, fixed for the whole
// walk): the column part of its own index and of its neighbours' (periodic in
// c1), and the neighbours' row steps.  Per row only the three row bases change.
struct TlCols {
  int own, col[3], dr[3];
  __device__ __forceinline__ TlCols(const Honey& G, int c1, int s) {
    own = 2 * c1 + s;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int o1 = s ? G.o1[1][k] : G.o1[0][k];
      int e1 = c1 + o1;
      e1 += (e1 < 0) ? G.L1 : 0;
      e1 -= (e1 >= G.L1) ? G.L1 : 0;
      col[k] = 2 * e1 + (1 - s);
      dr[k] = s ? G.o2[1][k] : G.o2[0][k];
    }
  }
  // own index and neighbours on row y (y at most one outside the lattice)
  __device__ __forceinline__ int at(const Honey& G, int y, int (&j)[3]) const {
    const int L2 = G.L2, r2 = 2 * G.L1;
    const int y0 = y + ((y < 0) ? L2 : 0) - ((y >= L2) ? L2 : 0);
    const int ym = y0 == 0 ? L2 - 1 : y0 - 1, yp = y0 == L2 - 1 ? 0 : y0 + 1;
    const int b0 = r2 * y0, bm = r2 * ym, bp = r2 * yp;
#pragma unroll
    for (int k = 0; k < 3; ++k) j[k] = (dr[k] < 0 ? bm : dr[k] > 0 ? bp : b0) + col[k];
    return b0 + own;
  }
};

// Threads per CTA: two per cell of a band (one per site of a band row), at most
// 256; three CTAs per SM (at most 85 registers).
template <bool CH, int NC, bool UH = false>
__global__ void __launch_bounds__(256, 3) k_cheb2_honey_df(
    DfEll<CH> H, Honey G, int bw, int nseg, const float4* __restrict__ xa, const float4* __restrict__ ya,
    const float4* __restrict__ xb, const float4* __restrict__ yb, float4* za, float4* __restrict__ wa, float4* zb,
    float4* __restrict__ wb, double2* __restrict__ pout, int ostride, int nzero) {
  const int nsite = 2 * bw;  // sites of a band row; thread t takes cell B1 + t / 2, sublattice t % 2
  const int s = (int)threadIdx.x & 1, cc = (int)threadIdx.x >> 1;
  const int nbands = G.L1 / bw;
  long long r_beg, r_end;  // band rows, band-major
  if (nseg > 0) {
    // segment blockIdx.x / nbands of band blockIdx.x % nbands: the CTAs of a
    // segment walk its rows across all bands together
    const int band = (int)blockIdx.x % nbands, seg = (int)blockIdx.x / nbands;
    r_beg = (long long)band * G.L2 + (long long)G.L2 * seg / nseg;
    r_end = (long long)band * G.L2 + (long long)G.L2 * (seg + 1) / nseg;
  } else {
    const long long total = (long long)nbands * G.L2;
    r_beg = total * blockIdx.x / gridDim.x;
    r_end = total * (blockIdx.x + 1) / gridDim.x;
  }
  DfDot q0, q1, q2, q3;
  for (long long p = r_beg; p < r_end;) {
    const int band = (int)(p / G.L2), y0 = (int)(p % G.L2);
    const int S = (int)min((long long)(G.L2 - y0), r_end - p);  // rows y0 .. y0 + S - 1 of this piece
    p += S;
    const int B1 = band * bw;
    // T_{m+1} on the halo columns (A at cell B1 - 1, B at cell B1 + bw) of rows y0 - 1 .. y0 + S
    for (int q = threadIdx.x; q < 2 * (S + 2); q += blockDim.x) {
      const int hs = q & 1, c1 = hs ? B1 + bw : B1 - 1;
      const TlCols C(G, c1 + (c1 < 0 ? G.L1 : 0) - (c1 >= G.L1 ? G.L1 : 0), hs);
      int j[3];
      const int i = C.at(G, y0 - 1 + (q >> 1), j);
      TlSite<CH, NC> T;
      tl_load<CH, NC, true, UH>(T, H, i, j, xa, xb, ya, yb);
      float4 v[NC];
      tl_compute<CH, NC, UH>(T, H, v);
      za[i] = v[0];
      if (NC == 2) zb[i] = v[NC - 1];
    }
    __syncthreads();
    const TlCols C(G, B1 + cc, s);
    // T_{m+1} on row y0 - 1 + t (rows y0 - 1 and y0 + S only as halo)
    auto first = [&](int t) {
      int j[3];
      const int i = C.at(G, y0 - 1 + t, j);
      TlSite<CH, NC> T;
      tl_load<CH, NC, true, UH>(T, H, i, j, xa, xb, ya, yb);
      float4 v[NC];
      tl_compute<CH, NC, UH>(T, H, v);
      za[i] = v[0];
      if (NC == 2) zb[i] = v[NC - 1];
      if (t >= 1 && t <= S) tl_dots<NC>(q0, q1, T.own, v);
    };
    // T_{m+2} on row y0 + t - 3: its T_{m+1} rows were written in earlier iterations
    auto second = [&](int t) {
      int j[3];
      const int i = C.at(G, y0 + t - 3, j);
      TlSite<CH, NC> U;
      tl_load<CH, NC, false, UH>(U, H, i, j, za, zb, xa, xb);
      float4 v[NC];
      tl_compute<CH, NC, UH>(U, H, v);
      wa[i] = v[0];
      if (NC == 2) wb[i] = v[NC - 1];
      tl_dots<NC>(q2, q3, U.own, v);
    };
    // With one chain the second order comes first in the iterations that do
    // both, so that the first order's loads (inputs of the launch, never written
    // by it) need not wait for the second order's stores (l = r pass 375 -> 349
    // us at N = 16.8M); the two-chain pass keeps one loop in which the first
    // order comes first.
    if constexpr (NC == 1) {
      int t = 0;
      for (; t <= min(2, S + 1); ++t) {
        first(t);
        __syncthreads();
      }
      for (; t <= S + 1; ++t) {
        second(t);
        first(t);
        __syncthreads();
      }
      for (; t <= S + 2; ++t) {
        second(t);
        __syncthreads();
      }
    } else {
      for (int t = 0; t <= S + 2; ++t) {
        if (threadIdx.x < 8) {
          // the rows that the first order streams, two rows ahead, into L2
          const int yp = y0 + 1 + t;
          if (yp <= y0 + S) {
            const int i0 = 2 * (B1 + G.L1 * (yp - (yp >= G.L2 ? G.L2 : 0)));
            const int lane = threadIdx.x;
            const uint32_t vb = (uint32_t)nsite * 16u;
            if (lane == 0) tl_prefetch_l2(xa + i0, vb);
            if (lane == 1) tl_prefetch_l2(ya + i0, vb);
            if (lane == 2) tl_prefetch_l2(xb + i0, vb);
            if (lane == 3) tl_prefetch_l2(yb + i0, vb);
            if (!UH && lane >= 4 && lane < 7)
              tl_prefetch_l2(H.hop + (size_t)(lane - 4) * H.n + i0,
                             (uint32_t)(nsite * sizeof(typename DfHop<CH>::T)));
            if (lane == 7) tl_prefetch_l2(H.diag + i0, (uint32_t)nsite * 8u);
          }
        }
        if (t <= S + 1) {
          int j[3];
          const int i = C.at(G, y0 - 1 + t, j);
          TlSite<CH, NC> T;
          tl_load<CH, NC, true, UH>(T, H, i, j, xa, xb, ya, yb);
          float4 v[NC];
          tl_compute<CH, NC, UH>(T, H, v);
          za[i] = v[0];
          if (NC == 2) zb[i] = v[NC - 1];
          if (t >= 1 && t <= S) tl_dots<NC>(q0, q1, T.own, v);
        }
        if (t >= 3) {
          int j[3];
          const int i = C.at(G, y0 + t - 3, j);
          TlSite<CH, NC> U;
          tl_load<CH, NC, false, UH>(U, H, i, j, za, zb, xa, xb);
          float4 v[NC];
          tl_compute<CH, NC, UH>(U, H, v);
          wa[i] = v[0];
          if (NC == 2) wb[i] = v[NC - 1];
          tl_dots<NC>(q2, q3, U.own, v);
        }
        __syncthreads();
      }
    }
  }
  double r[4] = {q0.get(), q1.get(), q2.get(), q3.get()};
  block_reduce_rx<4>(r, 1, reinterpret_cast<double*>(dyn_smem()));
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) pout[(size_t)j * ostride + blockIdx.x] = make_double2(r[j], 0.0);
  }
  // entries gridDim.x .. nzero - 1 of each slot hold zero (the moment reduction
  // sums nzero entries per slot)
  for (int b = blockIdx.x + gridDim.x; b < nzero; b += gridDim.x)
    if (threadIdx.x < 4) pout[(size_t)threadIdx.x * ostride + b] = make_double2(0.0, 0.0);
}

// ---------------------------------------------------------------- FP32 storage, R vectors

// Band width (cells) of the FP32 multi-vector walk for G lanes per site: the
// largest of 128/G, 64/G, 32/G dividing L1 (0: none), so that a CTA has at
// most 256 threads (two sites per cell, G lanes per site).
__host__ __device__ inline int tl_band_width_wv(int L1, int G) {
  for (int c = 128; c >= 32; c >>= 1) {
    const int bw = c / G;
    if (bw >= 1 && L1 % bw == 0) return bw;
  }
  return 0;
}

// One chain value of VP = 2 vectors at a site: a 16-byte load of the lane's two
// complex64 elements (vectors 2g and 2g + 1 of the site's row of R).
template <int MODE>  // 0: read-only path, 1: coherent (vectors this launch writes), 2: evict-first stream
__device__ __forceinline__ void tl_ld2(float2 (&d)[2], const float2* p, size_t e) {
  float4 t;
  if (MODE == 0)
    t = __ldg(reinterpret_cast<const float4*>(p + e));
  else if (MODE == 1)
    t = *reinterpret_cast<const float4*>(p + e);
  else
    t = __ldcs(reinterpret_cast<const float4*>(p + e));
  d[0] = make_float2(t.x, t.y);
  d[1] = make_float2(t.z, t.w);
}
__device__ __forceinline__ void tl_st2(float2* p, size_t e, const float2 (&d)[2]) {
  *reinterpret_cast<float4*>(p + e) = make_float4(d[0].x, d[0].y, d[1].x, d[1].y);
}

// The operands of one order at a site for the lane's two vectors, NC chains.
template <bool CH, int NC>
struct TlSiteWv {
  typename Ell<false, CH>::HT hv[3];
  float dg;
  float2 own[NC][2], nb[NC][3][2], prev[NC][2];
};

template <bool CH, int NC, bool IN_RO>
__device__ __forceinline__ void tl_load_wv(TlSiteWv<CH, NC>& S, const Ell<false, CH>& H, int i, const int (&j)[3],
                                           int R, int off, const float2* in0, const float2* in1,
                                           const float2* __restrict__ pv0, const float2* __restrict__ pv1) {
#pragma unroll
  for (int k = 0; k < 3; ++k) S.hv[k] = __ldg(H.hop2 + (size_t)k * H.n + i);
  S.dg = __ldg(H.diag2 + i);
  const size_t e = (size_t)i * R + off;
#pragma unroll
  for (int ch = 0; ch < NC; ++ch) {
    const float2* in = ch ? in1 : in0;
    tl_ld2<IN_RO ? 0 : 1>(S.own[ch], in, e);
#pragma unroll
    for (int k = 0; k < 3; ++k) tl_ld2<IN_RO ? 0 : 1>(S.nb[ch][k], in, (size_t)j[k] * R + off);
    tl_ld2<2>(S.prev[ch], ch ? pv1 : pv0, e);
  }
}

// T = 2H~ T_in - T_prev for the lane's two vectors of each chain, in FP32, with
// the fused multiply-adds in the order of the single-order kernels (two chains:
// diagonal first, as k_cheb_pair_wv; one chain: neighbours first, as
// k_cheb_dbl_wv), so that the chains equal theirs bit for bit.
template <bool CH, int NC>
__device__ __forceinline__ void tl_compute_wv(const TlSiteWv<CH, NC>& S, float2 (&v)[NC][2]) {
#pragma unroll
  for (int ch = 0; ch < NC; ++ch)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float2 a = cneg(S.prev[ch][q]);
      if (NC == 2) a = cmul_acc(a, S.dg, S.own[ch][q]);
#pragma unroll
      for (int k = 0; k < 3; ++k) a = cmul_acc(a, S.hv[k], S.nb[ch][k][q]);
      if (NC == 1) a = cmul_acc(a, S.dg, S.own[ch][q]);
      v[ch][q] = a;
    }
}

// Dots of one order: NC = 2, Re <A_k|B_k> and Re <A_k|B_k+1>; NC = 1, <u_k|u_k>
// and Re <u_k+1|u_k> (per vector, FP32 compensated sums).
template <int NC>
__device__ __forceinline__ void tl_dots_wv(DotAcc<float2> (&p)[2], DotAcc<float2> (&q)[2],
                                           const float2 (&own)[NC][2], const float2 (&v)[NC][2]) {
#pragma unroll
  for (int w = 0; w < 2; ++w) {
    if (NC == 2) {
      p[w].add_re(own[0][w], own[NC - 1][w]);
      q[w].add_re(own[0][w], v[NC - 1][w]);
    } else {
      p[w].add_norm(own[0][w]);
      q[w].add_re(v[0][w], own[0][w]);
    }
  }
}

// Two orders per launch for FP32-storage handles with R = 2G vectors per site
// (G = 1, 2, 4, 8 lanes per site, lane g holding vectors 2g and 2g + 1, the
// vector rows of the multi-vector kernels): the band walk of k_cheb2_honey_df
// with a band of bw cells served by 2 bw G <= 256 threads, FP32 arithmetic (the
// recursion of the FP32 kernels) and FP32 compensated dots per vector,
// converted to FP64 once per thread and reduced per vector into the partial
// slots [slot][CTA][R] of the multi-vector kernels.  Per two orders and
// orbital, DRAM moves T_m, T_{m-1} and the two outputs once, 8 bytes each per
// chain, plus H~ once per site and no index array: for the two-recurrence rows
// 64 + 16/R bytes instead of 2 x (48 + 28/R) for two single-order launches.
template <bool CH, int NC>
__global__ void __launch_bounds__(256, 3) k_cheb2_honey_wv(
    Ell<false, CH> H, Honey G, int bw, int nseg, int R, int gs, const float2* __restrict__ xa,
    const float2* __restrict__ ya, const float2* __restrict__ xb, const float2* __restrict__ yb, float2* za,
    float2* __restrict__ wa, float2* zb, float2* __restrict__ wb, double2* __restrict__ pout, int ostride,
    int nzero) {
  const int Gl = 1 << gs;
  const int lg = (int)threadIdx.x & (Gl - 1);
  const int st = (int)threadIdx.x >> gs;  // site of the band row: cell B1 + st / 2, sublattice st % 2
  const int s = st & 1, cc = st >> 1;
  const int off = 2 * lg;
  const int nbands = G.L1 / bw;
  long long r_beg, r_end;  // band rows, band-major
  if (nseg > 0) {
    const int band = (int)blockIdx.x % nbands, seg = (int)blockIdx.x / nbands;
    r_beg = (long long)band * G.L2 + (long long)G.L2 * seg / nseg;
    r_end = (long long)band * G.L2 + (long long)G.L2 * (seg + 1) / nseg;
  } else {
    const long long total = (long long)nbands * G.L2;
    r_beg = total * blockIdx.x / gridDim.x;
    r_end = total * (blockIdx.x + 1) / gridDim.x;
  }
  DotAcc<float2> q0[2], q1[2], q2[2], q3[2];
  for (long long p = r_beg; p < r_end;) {
    const int band = (int)(p / G.L2), y0 = (int)(p % G.L2);
    const int S = (int)min((long long)(G.L2 - y0), r_end - p);
    p += S;
    const int B1 = band * bw;
    // T_{m+1} on the halo columns (A at cell B1 - 1, B at cell B1 + bw) of rows y0 - 1 .. y0 + S
    for (int q = threadIdx.x; q < 2 * (S + 2) * Gl; q += blockDim.x) {
      const int hl = q & (Gl - 1), hq = q >> gs;
      const int hs = hq & 1, c1 = hs ? B1 + bw : B1 - 1;
      const TlCols C(G, c1 + (c1 < 0 ? G.L1 : 0) - (c1 >= G.L1 ? G.L1 : 0), hs);
      int j[3];
      const int i = C.at(G, y0 - 1 + (hq >> 1), j);
      TlSiteWv<CH, NC> T;
      tl_load_wv<CH, NC, true>(T, H, i, j, R, 2 * hl, xa, xb, ya, yb);
      float2 v[NC][2];
      tl_compute_wv<CH, NC>(T, v);
      const size_t e = (size_t)i * R + 2 * hl;
      tl_st2(za, e, v[0]);
      if (NC == 2) tl_st2(zb, e, v[NC - 1]);
    }
    __syncthreads();
    const TlCols C(G, B1 + cc, s);
    // iteration t: T_{m+1} on row y0 - 1 + t (t <= S + 1; rows y0 - 1 and y0 + S
    // only as halo) and T_{m+2} on row y0 + t - 3 (t >= 3; its T_{m+1} rows were
    // written in earlier iterations).  With one chain the second order comes
    // first, so that in the steady iterations the first order's loads (inputs of
    // the launch, never written by it) need not wait for the second order's
    // stores (measured: l = r pass 590 -> 547 us at the precision workload); the
    // two-chain pass, whose operands take twice the registers, keeps one loop in
    // which the first order comes first (the other order measured 928 -> 992 us).
    auto first = [&](int t) {
      int j[3];
      const int i = C.at(G, y0 - 1 + t, j);
      TlSiteWv<CH, NC> T;
      tl_load_wv<CH, NC, true>(T, H, i, j, R, off, xa, xb, ya, yb);
      float2 v[NC][2];
      tl_compute_wv<CH, NC>(T, v);
      const size_t e = (size_t)i * R + off;
      tl_st2(za, e, v[0]);
      if (NC == 2) tl_st2(zb, e, v[NC - 1]);
      if (t >= 1 && t <= S) tl_dots_wv<NC>(q0, q1, T.own, v);
    };
    auto second = [&](int t) {
      int j[3];
      const int i = C.at(G, y0 + t - 3, j);
      TlSiteWv<CH, NC> U;
      tl_load_wv<CH, NC, false>(U, H, i, j, R, off, za, zb, xa, xb);
      float2 v[NC][2];
      tl_compute_wv<CH, NC>(U, v);
      const size_t e = (size_t)i * R + off;
      __stcs(reinterpret_cast<float4*>(wa + e), make_float4(v[0][0].x, v[0][0].y, v[0][1].x, v[0][1].y));
      if (NC == 2)
        __stcs(reinterpret_cast<float4*>(wb + e),
               make_float4(v[NC - 1][0].x, v[NC - 1][0].y, v[NC - 1][1].x, v[NC - 1][1].y));
      tl_dots_wv<NC>(q2, q3, U.own, v);
    };
    if constexpr (NC == 1) {
      int t = 0;
      for (; t <= min(2, S + 1); ++t) {
        first(t);
        __syncthreads();
      }
      for (; t <= S + 1; ++t) {
        second(t);
        first(t);
        __syncthreads();
      }
      for (; t <= S + 2; ++t) {
        second(t);
        __syncthreads();
      }
    } else {
      for (int t = 0; t <= S + 2; ++t) {
        if (t <= S + 1) first(t);
        if (t >= 3) second(t);
        __syncthreads();
      }
    }
  }
  double2 r[8];
#pragma unroll
  for (int w = 0; w < 2; ++w) {
    r[w] = q0[w].get();
    r[2 + w] = q1[w].get();
    r[4 + w] = q2[w].get();
    r[6 + w] = q3[w].get();
  }
  const int slots[4] = {0, 1, 2, 3};
  write_partials_vpt<false, 2, 4>(r, R, Gl, dyn_smem(), pout, ostride, slots);
  // entries gridDim.x .. nzero - 1 of each slot hold zero
  for (int b = blockIdx.x + gridDim.x; b < nzero; b += gridDim.x)
    for (int t = threadIdx.x; t < 4 * R; t += blockDim.x)
      pout[((size_t)(t / R) * ostride + b) * R + t % R] = make_double2(0.0, 0.0);
}

// Sum of the blocked kernel's per-CTA partials (4 slots of ngrid x R entries, CTA
// order) into entry 0 of the moment slots slot0 .. slot0 + 3 (stride nblocks x R),
// the other entries zero: used when the blocked grid is larger than the
// single-order grid whose size the slots have.
__global__ void k_tl_fold(const double2* __restrict__ scratch, int ngrid, int R, double2* __restrict__ partial,
                          int nblocks, int slot0) {
  const int j = (int)blockIdx.x;  // slot
  for (int t = threadIdx.x; t < nblocks * R; t += blockDim.x) {
    const int b = t / R, r = t % R;
    double v = 0.0;
    if (b == 0)
      for (int c = 0; c < ngrid; ++c) v += scratch[((size_t)j * ngrid + c) * R + r].x;
    partial[((size_t)(slot0 + j) * nblocks + b) * R + r] = make_double2(v, 0.0);
  }
}

}  // namespace gqt
