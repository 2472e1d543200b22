// gqt_cluster.cuh -- moment rows of small systems in one persistent launch on a
// thread-block cluster.
//
// When the whole problem fits on chip, the per-order kernel launches of the
// large-N path (a few microseconds each) dominate.  Here one cluster of C CTAs
// (C = 16 where the GPU allows, else 8) runs all orders of a row: CTA c keeps
// sites [c*chunk, (c+1)*chunk) of the two Chebyshev vectors (and of l, and its
// rows of H~) in its shared memory; neighbour gathers read other CTAs' shared
// memory through the cluster's distributed shared memory; orders are separated
// by hardware cluster barriers (no software waits).  Per-CTA partial dot
// products go to the same [slot][CTA] layout as the large-N kernels and are
// reduced by the same deterministic pass.
#pragma once

#include <cooperative_groups.h>

#include "gqt_kernels.cuh"

namespace gqt {

namespace cgc = cooperative_groups;

// Shared-memory bytes per site of a cluster-resident row.
// Per-order partial sums kept until the end: (slots) x (warps) double2.
inline size_t cluster_red_bytes(int M, int slot_norm, int warps) {
  const int slots = (M > slot_norm ? M : slot_norm + 1) + 2;
  return (size_t)slots * warps * 16;
}

template <bool FP64, bool CH>
__host__ __device__ constexpr int cluster_site_bytes(int K, bool with_l) {
  return (int)(sizeof(typename Prec<FP64>::V) * (with_l ? 3 : 2) + K * (4 + sizeof(typename Ell<FP64, CH>::HT)) +
               sizeof(typename Prec<FP64>::S));
}

// DBL: l = r doubling (slots 2m-2, 2m-1 for step m = 1 .. steps); else Re <l|T_m|r>
// for m = 0 .. M-1 (slots m, norms in slot_norm).  R = 1, single segment.
template <bool FP64, bool CH, bool DBL>
__global__ void k_cheb_cluster(Ell<FP64, CH> H, int chunk, const typename Prec<FP64>::V* __restrict__ r,
                               const typename Prec<FP64>::V* __restrict__ l, double2* __restrict__ partial, int M,
                               int slot_norm) {
  using V = typename Prec<FP64>::V;
  using S = typename Prec<FP64>::S;
  using HT = typename Ell<FP64, CH>::HT;
  cgc::cluster_group cluster = cgc::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int me = (int)cluster.block_rank();
  const int K = H.K;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  V* TA = reinterpret_cast<V*>(sm_raw);
  V* TB = TA + chunk;
  V* LV = TB + chunk;  // only with !DBL
  HT* hs = reinterpret_cast<HT*>(DBL ? (void*)LV : (void*)(LV + chunk));
  S* ds = reinterpret_cast<S*>(hs + (size_t)K * chunk);
  int* is = reinterpret_cast<int*>(ds + chunk);
  // per-order partial sums: one double2 per (slot, warp), summed over warps at the end
  double2* red = reinterpret_cast<double2*>(is + (size_t)K * chunk + 4);
  red = reinterpret_cast<double2*>((reinterpret_cast<uintptr_t>(red) + 15) & ~(uintptr_t)15);
  const int nw = blockDim.x >> 5, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int beg = me * chunk;
  const int cnt = max(0, min(chunk, H.n - beg));
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
    const int i = beg + q;
    TA[q] = r[i];
    if (!DBL) LV[q] = l[i];
    ds[q] = H.diag2[i];
    for (int k = 0; k < K; ++k) {
      is[k * chunk + q] = H.idx[(size_t)k * H.n + i];
      hs[k * chunk + q] = H.hop2[(size_t)k * H.n + i];
    }
  }
  cluster.sync();
  auto reduce = [&](double2 v, int slot) {  // warp sum into red[slot][warp]; no block barrier
    for (int off = 16; off > 0; off >>= 1) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    if (lane == 0) red[(size_t)slot * nw + warp] = v;
  };
  // order m computes T_m into the buffer of T_{m-2}; T_{m-1} is read across the cluster
  const int last = DBL ? max((M + 1) / 2, 1) : M - 1;
  V* prev = TA;  // T_{m-1}
  V* cur = TB;   // T_{m-2} -> T_m
  for (int m = 1; m <= last; ++m) {
    DotAcc<V> d0, d1, n0, n1;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
      const V own = prev[q];
      V a;
      if (m == 1) {
        a = cscale(own, ds[q]);
      } else {
        a = cmul_acc(cneg(cur[q]), ds[q], own);
      }
      for (int k = 0; k < K; ++k) {
        const int j = is[k * chunk + q];
        const int rk = j / chunk;
        const V* src = cluster.map_shared_rank(prev, rk);
        a = cmul_acc(a, hs[k * chunk + q], src[j - rk * chunk]);
      }
      if (m == 1) a = cscale(a, (S)0.5);
      if (DBL) {
        d0.add_norm(own);
        d1.add_re(a, own);
      } else {
        if (m == 1) {
          d0.add_re(LV[q], own);
          n0.add_norm(LV[q]);
          n1.add_norm(own);
        }
        d1.add_re(LV[q], a);
      }
      cur[q] = a;
    }
    if (DBL) {
      reduce(d0.get(), 2 * m - 2);
      reduce(d1.get(), 2 * m - 1);
    } else {
      if (m == 1) {
        reduce(d0.get(), 0);
        reduce(make_double2(n0.get().x, n1.get().x), slot_norm);
      }
      reduce(d1.get(), m);
    }
    cluster.sync();  // T_m complete everywhere; nobody reads T_{m-1} any more
    V* t = prev;
    prev = cur;
    cur = t;
  }
  if (!DBL && M == 1) {  // only mu_0 and the norms
    DotAcc<V> d0, n0, n1;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
      d0.add_re(LV[q], TA[q]);
      n0.add_norm(LV[q]);
      n1.add_norm(TA[q]);
    }
    reduce(d0.get(), 0);
    reduce(make_double2(n0.get().x, n1.get().x), slot_norm);
  }
  __syncthreads();
  const int nslots = DBL ? 2 * max((M + 1) / 2, 1) : slot_norm + 1;
  for (int sl = threadIdx.x; sl < nslots; sl += blockDim.x) {
    if (!DBL && sl > M - 1 && sl != slot_norm) continue;
    double2 a = make_double2(0.0, 0.0);
    for (int w = 0; w < nw; ++w) {
      a.x += red[(size_t)sl * nw + w].x;
      a.y += red[(size_t)sl * nw + w].y;
    }
    partial[(size_t)sl * C + me] = a;
  }
  cluster.sync();  // no CTA leaves while another may still read its shared memory
}

}  // namespace gqt
