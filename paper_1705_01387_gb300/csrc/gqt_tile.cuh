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
// outputs go to buffers other than the inputs.
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
template <bool CH, int NC, bool IN_RO>
__device__ __forceinline__ void tl_load(TlSite<CH, NC>& S, const DfEll<CH>& H, int i, const int (&j)[3],
                                        const float4* in0, const float4* in1, const float4* __restrict__ pv0,
                                        const float4* __restrict__ pv1) {
#pragma unroll
  for (int k = 0; k < 3; ++k) S.hv[k] = __ldg(H.hop + (size_t)k * H.n + i);
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

template <bool CH, int NC>
__device__ __forceinline__ void tl_compute(const TlSite<CH, NC>& S, float4 (&v)[NC]) {
#pragma unroll
  for (int ch = 0; ch < NC; ++ch) v[ch] = df_step<CH, 3, false>(S.hv, S.dg, S.own[ch], S.nb[ch], S.prev[ch]);
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
template <bool CH, int NC>
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
      tl_load<CH, NC, true>(T, H, i, j, xa, xb, ya, yb);
      float4 v[NC];
      tl_compute<CH, NC>(T, v);
      za[i] = v[0];
      if (NC == 2) zb[i] = v[NC - 1];
    }
    __syncthreads();
    const TlCols C(G, B1 + cc, s);
    for (int t = 0; t <= S + 2; ++t) {
      if (NC == 2 && threadIdx.x < 8) {
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
          if (lane >= 4 && lane < 7)
            tl_prefetch_l2(H.hop + (size_t)(lane - 4) * H.n + i0, (uint32_t)(nsite * sizeof(typename DfHop<CH>::T)));
          if (lane == 7) tl_prefetch_l2(H.diag + i0, (uint32_t)nsite * 8u);
        }
      }
      if (t <= S + 1) {  // T_{m+1} on row y0 - 1 + t (rows y0 - 1 and y0 + S only as halo)
        int j[3];
        const int i = C.at(G, y0 - 1 + t, j);
        TlSite<CH, NC> T;
        tl_load<CH, NC, true>(T, H, i, j, xa, xb, ya, yb);
        float4 v[NC];
        tl_compute<CH, NC>(T, v);
        za[i] = v[0];
        if (NC == 2) zb[i] = v[NC - 1];
        if (t >= 1 && t <= S) tl_dots<NC>(q0, q1, T.own, v);
      }
      if (t >= 3) {  // T_{m+2} on row y0 + t - 3: its T_{m+1} rows were written in earlier iterations
        int j[3];
        const int i = C.at(G, y0 + t - 3, j);
        TlSite<CH, NC> U;
        tl_load<CH, NC, false>(U, H, i, j, za, zb, xa, xb);
        float4 v[NC];
        tl_compute<CH, NC>(U, v);
        wa[i] = v[0];
        if (NC == 2) wb[i] = v[NC - 1];
        tl_dots<NC>(q2, q3, U.own, v);
      }
      __syncthreads();
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

// Sum of the blocked kernel's per-CTA partials (4 slots of ngrid entries, CTA
// order) into entry 0 of the moment slots slot0 .. slot0 + 3 (stride nblocks),
// the other entries zero: used when the blocked grid is larger than the
// single-order grid whose size the slots have.
__global__ void k_tl_fold(const double2* __restrict__ scratch, int ngrid, double2* __restrict__ partial, int nblocks,
                          int slot0) {
  const int j = (int)blockIdx.x;  // slot
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    double v = 0.0;
    if (b == 0)
      for (int c = 0; c < ngrid; ++c) v += scratch[(size_t)j * ngrid + c].x;
    partial[(size_t)(slot0 + j) * nblocks + b] = make_double2(v, 0.0);
  }
}

}  // namespace gqt
