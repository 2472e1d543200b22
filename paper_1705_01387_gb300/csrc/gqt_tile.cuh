// gqt_tile.cuh -- temporal blocking of the paired-FP32 moment rows on the
// honeycomb lattice: two Chebyshev orders per pass over HBM.
//
// A single-order launch reads T_m (its gathers hit L2), T_{m-1} and H~, and
// writes T_{m+1}: for the two-recurrence VAC row 140 bytes per orbital, twice
// per two orders.  Here one CTA takes a tile of TX x TY honeycomb cells (the
// built-in layout: site 2(c1 + L1 c2) + s, periodic), loads T_m on the tile
// plus a two-cell halo into shared memory, computes T_{m+1} = 2H~T_m - T_{m-1}
// on the tile plus a one-cell halo (the halo ring is recomputed by the
// neighbouring tiles as well), then T_{m+2} = 2H~T_{m+1} - T_m on the tile from
// shared memory, and writes T_{m+1} and T_{m+2} of the tile.  Per two orders and
// orbital that is T_m, T_{m-1} and H~ read once (the halo rings come from L2,
// their tiles being neighbours in the CTAs' tile order) and two vectors written:
// for the VAC row 4 x 16 + 32 + 2 x 32 = 160 bytes instead of 280; the index
// array is not read at all, since the neighbours follow from the cell layout
// (one slot order per sublattice, checked on the host when the handle is built).
//
// Neighbours in the layout: A(c1,c2) -> B(c1,c2), B(c1+1,c2-1), B(c1,c2-1);
// B(c1,c2) -> A(c1,c2), A(c1-1,c2+1), A(c1,c2+1).  One hop changes c1 and c2 by
// at most one, so a one-cell halo holds every neighbour of the tile and a
// two-cell halo every neighbour of the one-cell ring.
//
// Arithmetic, dots and partial-sum slots are those of k_cheb_pair_df (NC = 2
// chains, A from l and B from r) and k_cheb_dbl_df (NC = 1, l = r): the pass
// over steps j and j + 1 adds the dots of moment slots 2j-2 .. 2j+1.  The
// outputs go to buffers other than the inputs (the halo rings of T_m and
// T_{m-1} are read by other CTAs during the pass).
#pragma once

namespace gqt {

constexpr int TL_TX = 16, TL_TY = 16;                     // interior cells of a tile
constexpr int TL_W0 = TL_TX + 4, TL_H0 = TL_TY + 4;       // T_m region: two-cell halo
constexpr int TL_W1 = TL_TX + 2, TL_H1 = TL_TY + 2;       // T_{m+1} region: one-cell halo
constexpr int TL_N0 = 2 * TL_W0 * TL_H0;                  // 800 sites
constexpr int TL_N1 = 2 * TL_W1 * TL_H1;                  // 648 sites
constexpr int TL_NI = 2 * TL_TX * TL_TY;                  // 512 interior sites
// threads of a tile CTA: 21 warps, so that the 648 sites of the one-cell region
// take one round (a barrier separates the two orders of a tile); one CTA per SM
// for the two-chain rows (shared memory), two for the l = r rows
template <int NC>
constexpr int tl_threads() { return 672; }
template <int NC>
constexpr int tl_min_blocks() { return NC == 2 ? 1 : 2; }

// Honeycomb cell layout of a handle: cell counts and, per sublattice s and ELL
// slot k, the cell offset (o1, o2) of that slot's neighbour (on sublattice 1 - s).
struct Honey {
  int L1 = 0, L2 = 0;
  int o1[2][3] = {}, o2[2][3] = {};
};

template <int W>
__device__ __forceinline__ int tl_loc(int e1, int e2, int s) {
  return 2 * (e1 + W * e2) + s;
}

// global site of cell (c1, c2) (one cell or two outside the lattice at most: periodic)
__device__ __forceinline__ int tl_site(const Honey& G, int c1, int c2, int s) {
  c1 += (c1 < 0) ? G.L1 : 0;
  c1 -= (c1 >= G.L1) ? G.L1 : 0;
  c2 += (c2 < 0) ? G.L2 : 0;
  c2 -= (c2 >= G.L2) ? G.L2 : 0;
  return 2 * (c1 + G.L1 * c2) + s;
}

// Site q of the T_{m+1} region in the order interior cells first, then the ring:
// cell (f1, f2) of the region (width TL_W1) and sublattice s.
__device__ __forceinline__ void tl_s1_site(int q, int& f1, int& f2, int& s) {
  s = q & 1;
  const int c = q >> 1;
  if (c < TL_TX * TL_TY) {
    f1 = c % TL_TX + 1;
    f2 = c / TL_TX + 1;
    return;
  }
  const int r = c - TL_TX * TL_TY;  // ring: top row, bottom row, left column, right column
  if (r < TL_W1) {
    f1 = r;
    f2 = 0;
  } else if (r < 2 * TL_W1) {
    f1 = r - TL_W1;
    f2 = TL_H1 - 1;
  } else if (r < 2 * TL_W1 + TL_TY) {
    f1 = 0;
    f2 = r - 2 * TL_W1 + 1;
  } else {
    f1 = TL_W1 - 1;
    f2 = r - 2 * TL_W1 - TL_TY + 1;
  }
}

__device__ __forceinline__ uint32_t tl_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void tl_cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tl_saddr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void tl_cp8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(tl_saddr(dst)), "l"(src) : "memory");
}

// Shared-memory image of the tiles (NC chains).  Two staging buffers, so that the
// next tile's copies are in flight while the current tile computes; each holds
// T_m on the two-cell region, T_{m-1} on the one-cell region and the H~ pairs of
// the one-cell region (slot-major: K hoppings, then the diagonal).  T_{m+1} on
// the one-cell region is computed into one buffer of its own.
template <bool CH, int NC>
struct TileSmem {
  using HT = typename DfHop<CH>::T;
  static constexpr size_t s0 = 0;                                        // float4 [NC][TL_N0]
  static constexpr size_t y = s0 + (size_t)NC * TL_N0 * sizeof(float4);   // float4 [NC][TL_N1]
  static constexpr size_t hop = y + (size_t)NC * TL_N1 * sizeof(float4);  // HT [3][TL_N1]
  static constexpr size_t diag = hop + (size_t)3 * TL_N1 * sizeof(HT);    // float2 [TL_N1]
  static constexpr size_t stage = (diag + (size_t)TL_N1 * sizeof(float2) + 127) / 128 * 128;
  static constexpr size_t s1 = 2 * stage;                                 // float4 [NC][TL_N1]
  static constexpr size_t bytes = s1 + (size_t)NC * TL_N1 * sizeof(float4);
};

// One order at a site of the one-cell region whose neighbours are in src (a
// region of width W, the site at cell (e1, e2)); hoppings and diagonal from the
// staged rows (entry q of the one-cell region); tm2 the order before.
template <bool CH, int W>
__device__ __forceinline__ float4 tl_step(const typename DfHop<CH>::T* hs, const float2* ds, const Honey& G, int q,
                                          const float4* src, int e1, int e2, int s, float4 own, float4 tm2) {
  typename DfHop<CH>::T hv[3];
  float4 nb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    hv[k] = hs[k * TL_N1 + q];
    const int o1 = s ? G.o1[1][k] : G.o1[0][k], o2 = s ? G.o2[1][k] : G.o2[0][k];  // constant indices
    nb[k] = src[tl_loc<W>(e1 + o1, e2 + o2, 1 - s)];
  }
  return df_step<CH, 3, false>(hv, ds[q], own, nb, tm2);
}

// Copies of one tile into staging buffer st (all in flight at once; one commit group).
template <bool CH, int NC, int THR>
__device__ __forceinline__ void tl_stage(unsigned char* st, const DfEll<CH>& H, const Honey& G, int t1, int t2,
                                         const float4* __restrict__ xa, const float4* __restrict__ ya,
                                         const float4* __restrict__ xb, const float4* __restrict__ yb) {
  using L = TileSmem<CH, NC>;
  using HT = typename DfHop<CH>::T;
  float4* S0 = reinterpret_cast<float4*>(st + L::s0);
  float4* Ys = reinterpret_cast<float4*>(st + L::y);
  HT* Hs = reinterpret_cast<HT*>(st + L::hop);
  float2* Ds = reinterpret_cast<float2*>(st + L::diag);
  for (int q = threadIdx.x; q < TL_N0; q += THR) {
    const int s = q & 1, c = q >> 1;
    const int gi = tl_site(G, t1 - 2 + c % TL_W0, t2 - 2 + c / TL_W0, s);
#pragma unroll
    for (int ch = 0; ch < NC; ++ch) tl_cp16(S0 + ch * TL_N0 + q, (ch ? xb : xa) + gi);
  }
  for (int q = threadIdx.x; q < TL_N1; q += THR) {
    int f1, f2, s;
    tl_s1_site(q, f1, f2, s);
    const int gi = tl_site(G, t1 - 1 + f1, t2 - 1 + f2, s);
#pragma unroll
    for (int ch = 0; ch < NC; ++ch) tl_cp16(Ys + ch * TL_N1 + q, (ch ? yb : ya) + gi);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (CH)
        tl_cp16(Hs + k * TL_N1 + q, H.hop + (size_t)k * H.n + gi);
      else
        tl_cp8(Hs + k * TL_N1 + q, H.hop + (size_t)k * H.n + gi);
    }
    tl_cp8(Ds + q, H.diag + gi);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <bool CH, int NC, int THR = tl_threads<NC>()>
__global__ void __launch_bounds__(THR, tl_min_blocks<NC>()) k_cheb2_honey_df(
    DfEll<CH> H, Honey G, const float4* __restrict__ xa, const float4* __restrict__ ya,
    const float4* __restrict__ xb, const float4* __restrict__ yb, float4* __restrict__ za,
    float4* __restrict__ wa, float4* __restrict__ zb, float4* __restrict__ wb, double2* __restrict__ partial,
    int nblocks, int slot0) {
  using L = TileSmem<CH, NC>;
  using HT = typename DfHop<CH>::T;
  unsigned char* sm = reinterpret_cast<unsigned char*>(dyn_smem());
  float4* S1 = reinterpret_cast<float4*>(sm + L::s1);
  const int ntx = G.L1 / TL_TX, ntiles = ntx * (G.L2 / TL_TY);
  DfDot q0, q1, q2, q3;
  auto origin = [&](int tile, int& t1, int& t2) {
    t1 = (tile % ntx) * TL_TX;
    t2 = (tile / ntx) * TL_TY;
  };
  if ((int)blockIdx.x < ntiles) {
    int t1, t2;
    origin(blockIdx.x, t1, t2);
    tl_stage<CH, NC, THR>(sm, H, G, t1, t2, xa, ya, xb, yb);
  }
  int it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    unsigned char* st = sm + (it & 1) * L::stage;
    const float4* S0 = reinterpret_cast<const float4*>(st + L::s0);
    const float4* Ys = reinterpret_cast<const float4*>(st + L::y);
    const HT* Hs = reinterpret_cast<const HT*>(st + L::hop);
    const float2* Ds = reinterpret_cast<const float2*>(st + L::diag);
    int t1, t2;
    origin(tile, t1, t2);
    // the next tile's copies go out now; this tile's must have landed
    if (tile + (int)gridDim.x < ntiles) {
      int n1, n2;
      origin(tile + gridDim.x, n1, n2);
      tl_stage<CH, NC, THR>(sm + ((it + 1) & 1) * L::stage, H, G, n1, n2, xa, ya, xb, yb);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    // T_{m+1} on the tile and its one-cell ring
    for (int q = threadIdx.x; q < TL_N1; q += THR) {
      int f1, f2, s;
      tl_s1_site(q, f1, f2, s);
      const int l0 = tl_loc<TL_W0>(f1 + 1, f2 + 1, s), l1 = tl_loc<TL_W1>(f1, f2, s);
      float4 v[NC], own[NC];
#pragma unroll
      for (int ch = 0; ch < NC; ++ch) {
        own[ch] = S0[ch * TL_N0 + l0];
        v[ch] = tl_step<CH, TL_W0>(Hs, Ds, G, q, S0 + ch * TL_N0, f1 + 1, f2 + 1, s, own[ch], Ys[ch * TL_N1 + q]);
        S1[ch * TL_N1 + l1] = v[ch];
      }
      if (q < TL_NI) {
        const int gi = tl_site(G, t1 - 1 + f1, t2 - 1 + f2, s);
#pragma unroll
        for (int ch = 0; ch < NC; ++ch) (ch ? zb : za)[gi] = v[ch];
        if (NC == 2) {
          q0.add_re(own[0], own[NC - 1]);  // Re <A_m|B_m>
          q1.add_re(own[0], v[NC - 1]);    // Re <A_m|B_m+1>
        } else {
          q0.add_norm(own[0]);             // <u_m|u_m>
          q1.add_re(v[0], own[0]);         // Re <u_m+1|u_m>
        }
      }
    }
    __syncthreads();
    // T_{m+2} on the tile
    for (int q = threadIdx.x; q < TL_NI; q += THR) {
      int f1, f2, s;
      tl_s1_site(q, f1, f2, s);
      const int gi = tl_site(G, t1 - 1 + f1, t2 - 1 + f2, s);
      const int l0 = tl_loc<TL_W0>(f1 + 1, f2 + 1, s), l1 = tl_loc<TL_W1>(f1, f2, s);
      float4 v[NC], own[NC];
#pragma unroll
      for (int ch = 0; ch < NC; ++ch) {
        own[ch] = S1[ch * TL_N1 + l1];
        v[ch] = tl_step<CH, TL_W1>(Hs, Ds, G, q, S1 + ch * TL_N1, f1, f2, s, own[ch], S0[ch * TL_N0 + l0]);
        (ch ? wb : wa)[gi] = v[ch];
      }
      if (NC == 2) {
        q2.add_re(own[0], own[NC - 1]);  // Re <A_m+1|B_m+1>
        q3.add_re(own[0], v[NC - 1]);    // Re <A_m+1|B_m+2>
      } else {
        q2.add_norm(own[0]);
        q3.add_re(v[0], own[0]);
      }
    }
    __syncthreads();  // this staging buffer and S1 are reused two and one tiles on
  }
  double r[4] = {q0.get(), q1.get(), q2.get(), q3.get()};
  block_reduce_rx<4>(r, 1, reinterpret_cast<double*>(dyn_smem()));
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) partial[(size_t)(slot0 + j) * nblocks + blockIdx.x] = make_double2(r[j], 0.0);
  }
  // the slots have nblocks entries (the grid of the single-order kernels); the
  // entries beyond this grid hold zero
  for (int b = blockIdx.x + gridDim.x; b < nblocks; b += gridDim.x)
    if (threadIdx.x < 4) partial[(size_t)(slot0 + threadIdx.x) * nblocks + b] = make_double2(0.0, 0.0);
}

}  // namespace gqt
