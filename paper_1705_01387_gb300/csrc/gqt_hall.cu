// gqt_hall.cu -- Hall conductivity by the Kubo-Bastin formula in the Chebyshev
// framework of the library (the paper's outlook, Sec. 6, after Garcia, Covaci
// and Rappoport 2015).
//
//   Lambda_mn = Tr[v~_a T_m(H~) v~_b T_n(H~)],  v~ = i d o H~ (velocity along
//   the direction with bond displacements d, in units of dE/hbar), estimated
//   with R unit random vectors r as (N/R) sum_r <P_m|B_n>,
//   P_m = T_m(H~) v~_a r,  B_n = v~_b T_n(H~) r;
//
//   sigma_ab(mu)/(e^2/h) = (2/Omega) int dx (1 - x^2)^-2 Re sum_mn c_m c_n g_m g_n
//   Gamma_mn(x) Lambda_mn,  Gamma_mn(x) = T_m(x) e^{-i n th}(x + i n sin th)
//   + T_n(x) e^{i m th}(x - i m sin th),  x = cos th.
//
// Three kernels carry the work.  k_kb_step advances both Chebyshev chains one
// order and applies v~_b to T_k r from the same neighbour gathers, writing the
// stacks P (M vectors) and B (M vectors).  k_kb_gemm forms all M x M inner
// products <P_m|B_n> -- a dense complex contraction over N*R, the dominant cost
// (4 M^2 N R FP64 FMAs) -- as a register-blocked FP64 GEMM with a deterministic
// split over the contraction; k_kb_gemm_tma does the same contraction in split
// TF32 on the tcgen05 tensor cores, its operands brought in by TMA.
// k_kb_integrand evaluates the double sum on an energy grid (a bilinear form per
// energy), and k_kb_scan integrates it.

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <type_traits>
#include <vector>

#include "gqt_internal.h"

using gqt::check_cuda;
using gqt::check_launch;
using gqt::prof_begin;
using gqt::prof_end;
using gqt::Error;
using gqt::set_error;

namespace {

enum { WS_HALL_P = 40, WS_HALL_B, WS_HALL_Q, WS_HALL_PART, WS_HALL_F, WS_HALL_W };

// H~ of a handle in the chain kernels: FP64 (double, double2 vectors) or FP32
// storage (float, float2 vectors; the tensor-core contraction only).
template <bool F64, bool CH>
struct HallEll {
  using S = typename std::conditional<F64, double, float>::type;
  using V = typename std::conditional<F64, double2, float2>::type;
  using HT = typename std::conditional<CH, V, S>::type;
  int64_t n;
  int K;
  const int* __restrict__ idx;  // slot-major [K][n]
  const HT* __restrict__ hop2;  // 2 H~ per slot
  const S* __restrict__ diag2;
};

__device__ __forceinline__ double2 mla(double2 acc, double h, double2 x) {
  acc.x = fma(h, x.x, acc.x);
  acc.y = fma(h, x.y, acc.y);
  return acc;
}
__device__ __forceinline__ double2 mla(double2 acc, double2 h, double2 x) {
  acc.x = fma(h.x, x.x, acc.x);
  acc.x = fma(-h.y, x.y, acc.x);
  acc.y = fma(h.x, x.y, acc.y);
  acc.y = fma(h.y, x.x, acc.y);
  return acc;
}
__device__ __forceinline__ float2 mla(float2 acc, float h, float2 x) {
  acc.x = fmaf(h, x.x, acc.x);
  acc.y = fmaf(h, x.y, acc.y);
  return acc;
}
__device__ __forceinline__ float2 mla(float2 acc, float2 h, float2 x) {
  acc.x = fmaf(h.x, x.x, acc.x);
  acc.x = fmaf(-h.y, x.y, acc.x);
  acc.y = fmaf(h.x, x.y, acc.y);
  acc.y = fmaf(h.y, x.x, acc.y);
  return acc;
}
__device__ __forceinline__ double2 mk(double2, double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ float2 mk(float2, float x, float y) { return make_float2(x, y); }

// Split of a value into two TF32 numbers (FP32 with the low 13 mantissa bits
// zero, as the tensor cores read them): f = x rounded to FP32, hi = f rounded to
// TF32, lo = f - hi (exact in FP32; the tensor cores keep its top 11 bits).
// hi + lo carries about 22 significant bits; the FP32 rounding of an FP64 x
// (2^-24) is below that, and forming lo from f keeps the split to one FP64-pipe
// conversion.
template <class T>
__device__ __forceinline__ void split_tf32(T x, float& hi, float& lo) {
  const float f = (float)x;
  hi = __uint_as_float((__float_as_uint(f) + 0x1000u) & 0xFFFFE000u);
  lo = f - hi;
}
// TF32-split stack entry (row m of the re_hi, im_hi, re_lo, im_lo planes; null
// re_hi: none).  A plane is blocked by 8 contraction sites, [chunk][row][8], so
// that an operand tile of the tensor-core contraction (8 sites of 128 rows) is
// one contiguous 4 KB block: the pointers address row m of chunk 0, cs is the
// chunk stride (M * 8 floats).
struct TcPlanes {
  float *re_hi, *im_hi, *re_lo, *im_lo;
  size_t cs;
};
template <class V>
__device__ __forceinline__ void store_split(const TcPlanes& t, size_t e, V v) {
  const size_t o = (e >> 3) * t.cs + (e & 7);
  float h, l;
  split_tf32(v.x, h, l);
  t.re_hi[o] = h;
  t.re_lo[o] = l;
  split_tf32(v.y, h, l);
  t.im_hi[o] = h;
  t.im_lo[o] = l;
}

// y = v~ x = i sum_s d_s H~_s x_j (hop2 = 2 H~, so the factor is i/2); with ys
// also its TF32 split (the tensor-core contraction's operands).  D: the type of
// the displacements (FP32 handles keep dx in FP32, dy always in FP64).
template <bool F64, bool CH, class D>
__global__ void k_kb_velocity(HallEll<F64, CH> H, const D* __restrict__ d, int R, size_t total,
                              const typename HallEll<F64, CH>::V* __restrict__ x,
                              typename HallEll<F64, CH>::V* __restrict__ y, TcPlanes ys) {
  using V = typename HallEll<F64, CH>::V;
  using S = typename HallEll<F64, CH>::S;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / R;
    const int r = (int)(e - i * R);
    V s = mk(V(), (S)0, (S)0);
    for (int k = 0; k < H.K; ++k) {
      const size_t sl = (size_t)k * H.n + i;
      const V xj = x[(size_t)H.idx[sl] * R + r];
      const S dd = (S)d[sl];
      s = mla(s, H.hop2[sl], mk(V(), dd * xj.x, dd * xj.y));
    }
    const V v = mk(V(), (S)-0.5 * s.y, (S)0.5 * s.x);
    y[e] = v;
    if (ys.re_hi) store_split(ys, e, v);
  }
}

// Velocity hoppings vh_s = d_s * hop2_s of direction b (slot-major like hop2), so
// that the velocity in k_kb_step costs one multiply-add per slot.
template <bool F64, bool CH, class D>
__global__ void k_kb_vhop(HallEll<F64, CH> H, const D* __restrict__ d, typename HallEll<F64, CH>::HT* __restrict__ vh) {
  using S = typename HallEll<F64, CH>::S;
  using V = typename HallEll<F64, CH>::V;
  const size_t total = (size_t)H.K * H.n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const auto h = H.hop2[t];
    const S dd = (S)d[t];
    if constexpr (CH)
      vh[t] = mk(V(), dd * h.x, dd * h.y);
    else
      vh[t] = dd * h;
  }
}

// Order k of both chains, element e = i*R + r:
//   P_{k+1} = 2H~P_k - P_{k-1}   (P_1 = H~P_0 at k = 0), unless last
//   Q_{k+1} = 2H~Q_k - Q_{k-1}   (Q_1 = H~Q_0),           unless last
//   B_k = v~_b Q_k                (from the same gathers of Q_k; vh = d_b * hop2)
// TC: P_{k+1} and B_k also (or, for B_k, only) go to the planar TF32-split stacks
// (ps: entry k+1, bs: entry k); bout may then be null.
template <bool F64, bool CH>
__global__ void __launch_bounds__(256) k_kb_step(HallEll<F64, CH> H,
                                                 const typename HallEll<F64, CH>::HT* __restrict__ vh, int R,
                                                 size_t total, const typename HallEll<F64, CH>::V* __restrict__ pk,
                                                 const typename HallEll<F64, CH>::V* __restrict__ pkm1,
                                                 typename HallEll<F64, CH>::V* __restrict__ pout,
                                                 const typename HallEll<F64, CH>::V* __restrict__ qk,
                                                 const typename HallEll<F64, CH>::V* __restrict__ qkm1,
                                                 typename HallEll<F64, CH>::V* __restrict__ qout,
                                                 typename HallEll<F64, CH>::V* __restrict__ bout, int first, int last,
                                                 TcPlanes ps, TcPlanes bs) {
  using V = typename HallEll<F64, CH>::V;
  using S = typename HallEll<F64, CH>::S;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / R;
    const int r = (int)(e - i * R);
    const S dg = H.diag2[i];
    V a = mk(V(), (S)0, (S)0), q = a, b = a;
    if constexpr (F64) {
      // bound by the FP64 pipe: one slot at a time
      for (int k = 0; k < H.K; ++k) {
        const size_t sl = (size_t)k * H.n + i;
        const size_t j = (size_t)H.idx[sl] * R + r;
        const auto h2 = H.hop2[sl];
        const V qj = qk[j];
        q = mla(q, h2, qj);
        b = mla(b, vh[sl], qj);
        if (!last) a = mla(a, h2, pk[j]);
      }
    } else {
      // FP32 storage: slots in groups of KG -- the group's indices and hoppings,
      // then its gathers, then the multiply-adds in slot order (the order of the
      // one-slot loop), so that more gathers are in flight
      constexpr int KG = 4;
      using HT = typename HallEll<F64, CH>::HT;
      for (int k0 = 0; k0 < H.K; k0 += KG) {
        size_t jj[KG];
        HT hh[KG], vv[KG];
        V qq[KG], pp[KG];
#pragma unroll
        for (int u = 0; u < KG; ++u)
          if (k0 + u < H.K) {
            const size_t sl = (size_t)(k0 + u) * H.n + i;
            jj[u] = (size_t)H.idx[sl] * R + r;
            hh[u] = H.hop2[sl];
            vv[u] = vh[sl];
          }
#pragma unroll
        for (int u = 0; u < KG; ++u)
          if (k0 + u < H.K) {
            qq[u] = qk[jj[u]];
            if (!last) pp[u] = pk[jj[u]];
          }
#pragma unroll
        for (int u = 0; u < KG; ++u)
          if (k0 + u < H.K) {
            q = mla(q, hh[u], qq[u]);
            b = mla(b, vv[u], qq[u]);
            if (!last) a = mla(a, hh[u], pp[u]);
          }
      }
    }
    const V bv = mk(V(), (S)-0.5 * b.y, (S)0.5 * b.x);
    if (bout) bout[e] = bv;
    if (bs.re_hi) store_split(bs, e, bv);
    if (last) continue;
    a = mla(a, dg, pk[e]);
    q = mla(q, dg, qk[e]);
    V pn;
    if (first) {
      pn = mk(V(), (S)0.5 * a.x, (S)0.5 * a.y);
      qout[e] = mk(V(), (S)0.5 * q.x, (S)0.5 * q.y);
    } else {
      const V p0 = pkm1[e], q0 = qkm1[e];
      pn = mk(V(), a.x - p0.x, a.y - p0.y);
      qout[e] = mk(V(), q.x - q0.x, q.y - q0.y);
    }
    pout[e] = pn;
    if (ps.re_hi) store_split(ps, e, pn);
  }
}

// part[s][m][n] = sum_{k in split s} conj(P[m][k]) B[n][k], P and B row-major
// [M][Kt].  64 x 64 output tile per CTA, 4 x 4 complex outputs per thread
// (rows tm + 16 i, columns tn + 16 j), contraction chunks of 16 staged in
// shared memory (columns padded by one element against bank conflicts).
constexpr int KB_TM = 64, KB_TK = 16;

__global__ void __launch_bounds__(256, 2) k_kb_gemm(const double2* __restrict__ P, const double2* __restrict__ B, int M,
                                                    size_t Kt, size_t kchunk, double2* __restrict__ part) {
  __shared__ double2 Ps[KB_TK][KB_TM + 1];
  __shared__ double2 Bs[KB_TK][KB_TM + 1];
  const int m0 = blockIdx.x * KB_TM, n0 = blockIdx.y * KB_TM;
  const size_t kb = (size_t)blockIdx.z * kchunk;
  const size_t ke = (kb + kchunk < Kt) ? kb + kchunk : Kt;
  const int tid = threadIdx.x, tm = tid & 15, tn = tid >> 4;
  double2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = make_double2(0.0, 0.0);
  for (size_t k0 = kb; k0 < ke; k0 += KB_TK) {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int q = tid + 256 * p;
      const int row = q >> 4, kk = q & 15;
      const size_t k = k0 + kk;
      const bool kin = k < ke;
      Ps[kk][row] = (kin && m0 + row < M) ? P[(size_t)(m0 + row) * Kt + k] : make_double2(0.0, 0.0);
      Bs[kk][row] = (kin && n0 + row < M) ? B[(size_t)(n0 + row) * Kt + k] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KB_TK; ++kk) {
      double2 a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = Ps[kk][tm + 16 * u];
        b[u] = Bs[kk][tn + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          acc[u][v].x = fma(a[u].x, b[v].x, acc[u][v].x);
          acc[u][v].x = fma(a[u].y, b[v].y, acc[u][v].x);
          acc[u][v].y = fma(a[u].x, b[v].y, acc[u][v].y);
          acc[u][v].y = fma(-a[u].y, b[v].x, acc[u][v].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int m = m0 + tm + 16 * u, nn = n0 + tn + 16 * v;
      if (m < M && nn < M) part[((size_t)blockIdx.z * M + m) * M + nn] = acc[u][v];
    }
}

// ------------------------------------------------------------ tensor-core contraction
// The same contraction on the tcgen05 tensor cores in split TF32 (three products
// hi*hi + hi*lo + lo*hi per pair, FP32 accumulation in tensor memory over one
// split of the contraction, splits summed in FP64).  The stacks are planar
// (real and imaginary planes, blocked by 8 sites as described at TcPlanes), so
// with
//   Re Lambda = Pre.Bre + Pim.Bim,  Im Lambda = Pre.Bim - Pim.Bre
// every operand is a plain tile of a plane.
// Polls of the drain after a timeout (copies and products still in flight);
// the pipeline's own waits take the handle's limit (gqt_set_wait_limit, by
// default the same number).
constexpr int TC_WAIT_LIMIT = 1 << 24;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Bounded wait for the completion of phase `parity` of an mbarrier: at most
// `limit` polls (0: give up at once); false on timeout.
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, int limit) {
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; ++it)
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity));
  return done != 0;
}

__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
}

// Wide tiles fed by TMA: one CTA computes a 128 x 256 output tile into two
// accumulators of 256 tensor-memory columns (Re, Im).  The instruction
// descriptor's negate-A bit gives Im = Pre.Bim - Pim.Bre in one accumulator, so
// each 8-site stage is 12 products of 128 x 256 x 8 from 4 A tiles of 128 rows
// and 4 B tiles of 256 rows (48 KB): a third fewer operand bytes per product
// than a 128 x 128 tile.  One thread drives the pipeline: a 4-D tensor map over
// the blocked planes (site within chunk, row, chunk, plane) brings each tile in
// as bulk tensor copies of contiguous 4 KB blocks (32-B rows, 32-B swizzle; rows
// past M read as zeros) that complete on the stage's mbarrier, the products of
// a stage go out as soon as it has landed,
// and a buffer is refilled, NBUF - 1 stages ahead, once the products that read
// it have completed.  Every wait is bounded (wait_limit polls); after a timeout
// the thread drains what is still in flight (the last committed products and
// the copies issued but not waited for, TC_WAIT_LIMIT polls each) and the
// kernel reports it (err bit 16; bit 32 if the drain gave up as well).  The
// tensor memory is freed in every case: a CTA that exited holding it would make
// the next CTA's allocation on that SM wait without end.
constexpr int TM_TM = 128, TM_TN = 256, TM_TK = 8;       // 8 FP32 sites: one 32-B swizzle span per row
constexpr int TM_ATILE = TM_TM * 32, TM_BTILE = TM_TN * 32;  // 4 KB, 8 KB
constexpr int TM_BOX = 128 * 32;                            // one copy: 8 sites x 128 rows
constexpr int TM_STAGE = 4 * TM_ATILE + 4 * TM_BTILE;       // 48 KB
constexpr int TM_NBUF = 4;
constexpr int TM_SMEM = TM_NBUF * TM_STAGE + 1024 + 128;    // + 1 KB alignment slack, barriers
constexpr int TM_THREADS = 256;

// K-major operand, 32-B swizzle: rows of 32 B, 8-row groups 256 B apart.
__device__ __forceinline__ uint64_t tm_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(256 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)6 << 61);
}

// kind::tf32, D f32, A and B K-major, M = 128, N = 256; NEG: negate A (bit 13).
template <bool NEG>
__device__ __forceinline__ void tm_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  constexpr uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (NEG ? (1u << 13) : 0u) |
                             ((uint32_t)(TM_TN >> 3) << 17) | ((uint32_t)(TM_TM >> 4) << 24);
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Box of 8 sites x 128 rows at (row y, chunk c, plane z).
__device__ __forceinline__ void tm_load(uint32_t dst, const CUtensorMap* map, int y, int c, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(y), "r"(c), "r"(z), "r"(bar)
      : "memory");
}

struct TmPlanes {
  int a[4];  // plane (z coordinate) of Pre_hi, Pre_lo, Pim_hi, Pim_lo
  int b[4];  // Bre_hi, Bre_lo, Bim_hi, Bim_lo
};

__global__ void __launch_bounds__(TM_THREADS, 1) k_kb_gemm_tma(const __grid_constant__ CUtensorMap map, TmPlanes pz,
                                                        int M, size_t kt, size_t kchunk, double2* __restrict__ part,
                                                        int* __restrict__ err, int wait_limit) {
  extern __shared__ __align__(1024) unsigned char tm_raw[];
  const uint32_t raw = smem_addr(tm_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // swizzled tiles start on 1 KB
  unsigned char* sm = tm_raw + (base - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + TM_NBUF * TM_STAGE);
  uint64_t* done = full + TM_NBUF;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + TM_NBUF);
  int* okp = reinterpret_cast<int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * TM_TM, n0 = blockIdx.y * TM_TN;
  const size_t kb = (size_t)blockIdx.z * kchunk;
  const size_t ke = (kb + kchunk < kt) ? kb + kchunk : kt;
  const int nst = (int)((ke - kb + TM_TK - 1) / TM_TK);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int b = 0; b < TM_NBUF; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&full[b])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&done[b])), "r"(1));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    *okp = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map)) : "memory");
    auto issue = [&](int s) {
      const int b = s % TM_NBUF;
      const uint32_t st = base + b * TM_STAGE, fb = smem_addr(&full[b]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(TM_STAGE) : "memory");
      const int c = (int)(kb / TM_TK) + s;
#pragma unroll
      for (int t = 0; t < 4; ++t) tm_load(st + t * TM_ATILE, &map, m0, c, pz.a[t], fb);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const uint32_t bt = st + 4 * TM_ATILE + t * TM_BTILE;
        tm_load(bt, &map, n0, c, pz.b[t], fb);
        tm_load(bt + TM_BOX, &map, n0 + 128, c, pz.b[t], fb);
      }
    };
    int issued = 0, landed = 0, committed = 0;
    bool ok = true;
    for (; issued < nst && issued < TM_NBUF; ++issued) issue(issued);
    for (int s = 0; s < nst; ++s) {
      const int b = s % TM_NBUF;
      if (!tc_wait(&full[b], (uint32_t)((s / TM_NBUF) & 1), wait_limit)) {
        ok = false;
        break;
      }
      landed = s + 1;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t st = base + b * TM_STAGE;
      uint64_t a[4], bb[4];  // a: Pre_hi, Pre_lo, Pim_hi, Pim_lo; bb: Bre_hi, Bre_lo, Bim_hi, Bim_lo
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        a[t] = tm_desc(st + t * TM_ATILE);
        bb[t] = tm_desc(st + 4 * TM_ATILE + t * TM_BTILE);
      }
      const uint32_t acc = s > 0 ? 1u : 0u;
      tm_mma<false>(tmem, a[0], bb[0], acc);  // Re = Pre.Bre + Pim.Bim
      tm_mma<false>(tmem, a[0], bb[1], 1u);
      tm_mma<false>(tmem, a[1], bb[0], 1u);
      tm_mma<false>(tmem, a[2], bb[2], 1u);
      tm_mma<false>(tmem, a[2], bb[3], 1u);
      tm_mma<false>(tmem, a[3], bb[2], 1u);
      tm_mma<false>(tmem + TM_TN, a[0], bb[2], acc);  // Im = Pre.Bim - Pim.Bre
      tm_mma<false>(tmem + TM_TN, a[0], bb[3], 1u);
      tm_mma<false>(tmem + TM_TN, a[1], bb[2], 1u);
      tm_mma<true>(tmem + TM_TN, a[2], bb[0], 1u);
      tm_mma<true>(tmem + TM_TN, a[2], bb[1], 1u);
      tm_mma<true>(tmem + TM_TN, a[3], bb[0], 1u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(&done[b])));
      committed = s + 1;
      // the products of stage s - 1 have read their buffer: refill it with stage
      // s - 1 + NBUF while those of stage s run
      if (s >= 1 && issued < nst) {
        const int p = s - 1;
        if (!tc_wait(&done[p % TM_NBUF], (uint32_t)((p / TM_NBUF) & 1), wait_limit)) {
          ok = false;
          break;
        }
        issue(issued++);
      }
    }
    // the last products (their completion implies that of all earlier ones)
    const int lb = (committed - 1) % TM_NBUF;
    const uint32_t lp = (uint32_t)(((committed - 1) / TM_NBUF) & 1);
    if (ok && committed > 0 && !tc_wait(&done[lb], lp, wait_limit)) ok = false;
    if (!ok) {
      // drain: the last committed products, then the copies still in flight
      bool drained = committed == 0 || tc_wait(&done[lb], lp, TC_WAIT_LIMIT);
      for (int s = landed; s < issued; ++s) drained = tc_wait(&full[s % TM_NBUF], (uint32_t)((s / TM_NBUF) & 1),
                                                               TC_WAIT_LIMIT) && drained;
      *okp = 0;
      atomicOr(err, drained ? 16 : (16 | 32));
    }
  }
  __syncthreads();
  const bool ok = *okp != 0;
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    // warp w reads tensor-memory lanes 32 (w % 4) .. +31; warps 0-3 take columns
    // 0..127, warps 4-7 columns 128..255
    const int quarter = warp & 3;
    const int m = m0 + quarter * 32 + (tid & 31);
    const uint32_t lane = (uint32_t)(quarter * 32) << 16;
    const int cbeg = (warp >> 2) * (TM_TN / 2);
    for (int c = cbeg; c < cbeg + TM_TN / 2; c += 32) {
      uint32_t re[32], im[32];
      tc_ld32(tmem + lane + c, re);
      tc_ld32(tmem + lane + TM_TN + c, im);
      if (m < M) {
        double2* dst = part + ((size_t)blockIdx.z * M + m) * M + n0 + c;
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (n0 + c + j < M)
            dst[j] = make_double2((double)__uint_as_float(re[j]), (double)__uint_as_float(im[j]));
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// lam[m][n] = scale * sum_s part[s][m][n], splits summed in order (deterministic).
__global__ void k_kb_reduce(const double2* __restrict__ part, int S, int M, double scale, double2* __restrict__ lam) {
  const size_t total = (size_t)M * M;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int q = 0; q < S; ++q) {
      const double2 v = part[(size_t)q * total + t];
      s.x += v.x;
      s.y += v.y;
    }
    lam[t] = make_double2(scale * s.x, scale * s.y);
  }
}

// F(x_e) = (1 - x^2)^-2 Re sum_mn Gamma_mn(x) W_mn Lambda_mn for EB energies per
// CTA, W_mn = w_m w_n (w = c_n g_n).  Per energy the sum is
//   sum_m Tw_m z1_m + conj(aw_m) z2_m,  z1_m = sum_n Lambda_mn aw_n,  z2_m = sum_n Lambda_mn Tw_n,
// Tw_n = w_n T_n(x), aw_n = w_n e^{-i n th}(x + i n sin th) (and w_m e^{i m th}(x - i m sin th)
// = conj(aw_m)).  Tables in shared memory; one warp per row m, lanes over n.
template <int EB>
__global__ void __launch_bounds__(256) k_kb_integrand(const double2* __restrict__ lam, int M,
                                                      const double* __restrict__ E, int NE, double inv_dE,
                                                      const double* __restrict__ w, double* __restrict__ F) {
  extern __shared__ double kb_sm[];
  double2* aw = reinterpret_cast<double2*>(kb_sm);  // [EB][M], first: 16-byte aligned for any M
  double* Tw = kb_sm + 2 * EB * M;                   // [EB][M]
  __shared__ double2 red[EB][8];
  const int e0 = blockIdx.x * EB;
  for (int t = threadIdx.x; t < EB * M; t += blockDim.x) {
    const int e = t / M, n = t - e * M;
    double x = 0.0;
    if (e0 + e < NE) x = E[e0 + e] * inv_dE;
    const double th = acos(x), s = sin(th);
    double sn, cn;
    sincos((double)n * th, &sn, &cn);
    Tw[t] = w[n] * cn;
    // e^{-i n th}(x + i n s) = (cn - i sn)(x + i n s)
    aw[t] = make_double2(w[n] * (cn * x + sn * n * s), w[n] * (cn * n * s - sn * x));
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double2 acc[EB];
#pragma unroll
  for (int e = 0; e < EB; ++e) acc[e] = make_double2(0.0, 0.0);
  for (int m = warp; m < M; m += nw) {
    double2 z1[EB], z2[EB];
#pragma unroll
    for (int e = 0; e < EB; ++e) z1[e] = z2[e] = make_double2(0.0, 0.0);
    const double2* row = lam + (size_t)m * M;
    for (int nn = lane; nn < M; nn += 32) {
      const double2 l = row[nn];
#pragma unroll
      for (int e = 0; e < EB; ++e) {
        const double2 a = aw[e * M + nn];
        const double t = Tw[e * M + nn];
        z1[e].x = fma(l.x, a.x, fma(-l.y, a.y, z1[e].x));
        z1[e].y = fma(l.x, a.y, fma(l.y, a.x, z1[e].y));
        z2[e].x = fma(l.x, t, z2[e].x);
        z2[e].y = fma(l.y, t, z2[e].y);
      }
    }
#pragma unroll
    for (int e = 0; e < EB; ++e) {
      for (int off = 16; off > 0; off >>= 1) {
        z1[e].x += __shfl_xor_sync(0xffffffffu, z1[e].x, off);
        z1[e].y += __shfl_xor_sync(0xffffffffu, z1[e].y, off);
        z2[e].x += __shfl_xor_sync(0xffffffffu, z2[e].x, off);
        z2[e].y += __shfl_xor_sync(0xffffffffu, z2[e].y, off);
      }
      if (lane == 0) {
        const double tm = Tw[e * M + m];
        const double2 am = aw[e * M + m];  // conj(am) multiplies z2
        acc[e].x += tm * z1[e].x + am.x * z2[e].x + am.y * z2[e].y;
        acc[e].y += tm * z1[e].y + am.x * z2[e].y - am.y * z2[e].x;
      }
    }
  }
  if (lane == 0)
#pragma unroll
    for (int e = 0; e < EB; ++e) red[e][warp] = acc[e];
  __syncthreads();
  if ((int)threadIdx.x < EB && e0 + (int)threadIdx.x < NE) {
    const int e = threadIdx.x;
    double s = 0.0;
    for (int q = 0; q < nw; ++q) s += red[e][q].x;
    const double x = E[e0 + e] * inv_dE;
    F[e0 + e] = s / ((1.0 - x * x) * (1.0 - x * x));
  }
}

// sigma_j = pref * sum_{k<j} (x_{k+1} - x_k)(F_k + F_{k+1})/2 (one thread: a running sum).
__global__ void k_kb_scan(const double* __restrict__ F, const double* __restrict__ E, int NE, double inv_dE,
                          double pref, double* __restrict__ sigma) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double run = 0.0;
  for (int j = 0; j < NE; ++j) {
    if (j > 0) run += 0.5 * (E[j] - E[j - 1]) * inv_dE * (F[j] + F[j - 1]);
    sigma[j] = pref * run;
  }
}

// sigma(mu_q, T) = pref * sum_k (x_{k+1} - x_k)(f_k F_k + f_{k+1} F_{k+1})/2 with the
// Fermi weights f_k = 1/(1 + exp((E_k - mu_q)/kT)) (kT = 0: the step, 1/2 at E = mu);
// one thread per chemical potential.
__global__ void k_kb_fermi(const double* __restrict__ F, const double* __restrict__ E, int NE, double inv_dE,
                           const double* __restrict__ mu, int Nmu, double kT, double pref,
                           double* __restrict__ sigma) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Nmu) return;
  const double m = mu[q];
  auto fermi = [&](double e) {
    if (kT <= 0.0) return e < m ? 1.0 : (e > m ? 0.0 : 0.5);
    return 1.0 / (1.0 + exp((e - m) / kT));
  };
  double run = 0.0, prev = fermi(E[0]) * F[0];
  for (int j = 1; j < NE; ++j) {
    const double cur = fermi(E[j]) * F[j];
    run += 0.5 * (E[j] - E[j - 1]) * inv_dE * (prev + cur);
    prev = cur;
  }
  sigma[q] = pref * run;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    return (e == cudaSuccess && q == cudaDriverEntryPointSuccess) ? (PFN_cuTensorMapEncodeTiled_v12000)p : nullptr;
  }();
  if (!fn) throw Error(GQT_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  return fn;
}

double jackson_g(int n, int M) {
  const double a = 1.0 / (M + 1.0), pi = 3.14159265358979323846;
  return (1.0 - n * a) * std::cos(pi * n * a) + a * std::sin(pi * n * a) / std::tan(pi * a);
}

int grid_for(size_t total) {
  const size_t want = (total + 255) / 256;
  return (int)std::max<size_t>(1, std::min<size_t>(want, (size_t)gqt::sm_count() * 8));
}

// F64: the handle's storage precision (FP32 handles run the chains in FP32 and
// use the tensor-core contraction); DA, DB: the types of the two directions'
// displacements.
template <bool F64, bool CH, class DA, class DB>
void kb_moments_impl(gqt_ham* h, const void* rv, int R, int M, const DA* da, const DB* db, double2* lam,
                     cudaStream_t st) {
  using HE = HallEll<F64, CH>;
  using V = typename HE::V;
  HE H;
  H.n = h->n;
  H.K = h->K;
  H.idx = (const int*)h->d_idx.p;
  H.hop2 = (const typename HE::HT*)h->d_hop.p;
  H.diag2 = (const typename HE::S*)h->d_diag.p;
  const V* r = (const V*)rv;
  const bool tc = h->kb_mode == 1;
  const size_t total = (size_t)h->n * R;
  const size_t vb = total * sizeof(V);
  const int g = grid_for(total);
  // FP32 chain steps: one element per thread (every neighbour gather in flight at once)
  const int gs = F64 ? g : (int)std::min<size_t>((total + 255) / 256, (size_t)INT32_MAX);
  V* Q = (V*)h->ws(WS_HALL_Q, vb * 3).p;
  auto qbuf = [&](int k) -> V* { return Q + (size_t)(k % 3) * total; };
  const size_t mm = (size_t)M * M;
  using HT = typename HE::HT;
  HT* vh = (HT*)h->ws(WS_HALL_W, (size_t)H.K * H.n * sizeof(HT)).p;
  k_kb_vhop<F64, CH, DB><<<grid_for((size_t)H.K * H.n), 256, 0, st>>>(H, db, vh);
  check_launch("k_kb_vhop");
  if constexpr (F64) if (!tc) {
    double2* Pst = (double2*)h->ws(WS_HALL_P, vb * M).p;
    double2* Bst = (double2*)h->ws(WS_HALL_B, vb * M).p;
    const TcPlanes none = {nullptr, nullptr, nullptr, nullptr, 0};
    k_kb_velocity<F64, CH, DA><<<g, 256, 0, st>>>(H, da, R, total, r, Pst, none);
    check_launch("k_kb_velocity");
    for (int k = 0; k < M; ++k) {
      const bool last = k == M - 1;
      const V* qk = k == 0 ? r : qbuf(k);
      const V* qkm1 = k == 0 ? nullptr : (k == 1 ? r : qbuf(k - 1));
      const size_t pe = prof_begin(st);
      k_kb_step<F64, CH><<<g, 256, 0, st>>>(H, vh, R, total, Pst + (size_t)k * total,
                                        k == 0 ? nullptr : Pst + (size_t)(k - 1) * total,
                                        last ? nullptr : Pst + (size_t)(k + 1) * total, qk, qkm1,
                                        last ? nullptr : qbuf(k + 1), Bst + (size_t)k * total, k == 0, last, none,
                                        none);
      check_launch("k_kb_step");
      prof_end(pe, 7, st);
    }
    // split of the contraction: about eight waves of two resident CTAs per SM, at
    // least 512 contraction elements per split
    const int tiles = (M + KB_TM - 1) / KB_TM;
    const long long slots = 2LL * gqt::sm_count();
    long long S = std::max<long long>(1, (8 * slots + (long long)tiles * tiles - 1) / ((long long)tiles * tiles));
    S = std::min<long long>(S, std::max<long long>(1, (long long)(total / 512)));
    const size_t kchunk = ((total + S - 1) / S + KB_TK - 1) / KB_TK * KB_TK;
    S = (long long)((total + kchunk - 1) / kchunk);
    double2* part = (double2*)h->ws(WS_HALL_PART, (size_t)S * mm * sizeof(double2)).p;
    const size_t pg = prof_begin(st);
    k_kb_gemm<<<dim3(tiles, tiles, (unsigned)S), 256, 0, st>>>(Pst, Bst, M, total, kchunk, part);
    check_launch("k_kb_gemm");
    prof_end(pg, 8, st);
    k_kb_reduce<<<(int)std::min<size_t>((mm + 255) / 256, 4096), 256, 0, st>>>(part, (int)S, M,
                                                                                (double)h->n / R, lam);
    check_launch("k_kb_reduce");
    return;
  }
  // tensor-core contraction: chains in the handle's precision (rolling buffers),
  // stacks in planar split TF32 blocked by 8 sites ([chunk][row][8] per plane,
  // planes an odd number of 128-B lines apart)
  V* Pr = (V*)h->ws(WS_HALL_P, vb * 3).p;
  auto pbuf = [&](int k) -> V* { return Pr + (size_t)(k % 3) * total; };
  const size_t nk = (total + TM_TK - 1) / TM_TK;  // chunks; the contraction runs over nk * 8 sites
  if (nk > (size_t)INT32_MAX) throw Error(GQT_EINVAL, "gqt_kb_moments: N R too large");
  const size_t cs = (size_t)M * TM_TK;             // chunk stride in floats
  const size_t plane = [](size_t x) {
    x = (x + 31) / 32 * 32;
    return (x / 32) % 2 ? x : x + 32;
  }(nk * cs);
  float* pl = (float*)h->ws(WS_HALL_B, plane * 8 * sizeof(float)).p;
  if (total % TM_TK)  // sites past N R in the last chunk: zeros
    check_cuda(cudaMemset2DAsync(pl + (nk - 1) * cs, plane * sizeof(float), 0, cs * sizeof(float), 8, st),
               "stack padding");
  // planes: P re_hi, im_hi, re_lo, im_lo (0..3); B the same (4..7)
  auto planes = [&](int first, size_t entry) {
    TcPlanes t;
    t.re_hi = pl + (first + 0) * plane + entry * TM_TK;
    t.im_hi = pl + (first + 1) * plane + entry * TM_TK;
    t.re_lo = pl + (first + 2) * plane + entry * TM_TK;
    t.im_lo = pl + (first + 3) * plane + entry * TM_TK;
    t.cs = cs;
    return t;
  };
  const TcPlanes none = {nullptr, nullptr, nullptr, nullptr, 0};
  k_kb_velocity<F64, CH, DA><<<g, 256, 0, st>>>(H, da, R, total, r, pbuf(0), planes(0, 0));
  check_launch("k_kb_velocity");
  for (int k = 0; k < M; ++k) {
    const bool last = k == M - 1;
    const V* qk = k == 0 ? r : qbuf(k);
    const V* qkm1 = k == 0 ? nullptr : (k == 1 ? r : qbuf(k - 1));
    const size_t pe = prof_begin(st);
    k_kb_step<F64, CH><<<gs, 256, 0, st>>>(H, vh, R, total, pbuf(k), k == 0 ? nullptr : pbuf(k - 1),
                                      last ? nullptr : pbuf(k + 1), qk, qkm1, last ? nullptr : qbuf(k + 1), nullptr,
                                      k == 0, last, last ? none : planes(0, k + 1), planes(4, k));
    check_launch("k_kb_step");
    prof_end(pe, 7, st);
  }
  // splits: contraction chunks of about 8K sites (the FP32 accumulation span) and
  // at least four waves of one CTA per SM; among up to 1.5x that many splits the
  // count whose last wave is fullest
  const size_t kt = nk * TM_TK;
  const int tm = (M + TM_TM - 1) / TM_TM, tn = (M + TM_TN - 1) / TM_TN;
  const long long tiles = (long long)tm * tn, sms = gqt::sm_count();
  long long S = std::max<long long>((long long)((kt + 8191) / 8192), (4 * sms + tiles - 1) / tiles);
  {
    long long best = S;
    double best_cost = 1e300;
    for (long long c = S; c <= S + S / 2; ++c) {
      const double cost = (double)((tiles * c + sms - 1) / sms) / (double)c;
      if (cost < best_cost * (1 - 1e-9)) best_cost = cost, best = c;
    }
    S = best;
  }
  S = std::min<long long>(S, (long long)nk);
  S = std::min<long long>(S, 65535);  // gridDim.z limit (longer splits beyond N R ~ 5e8)
  const size_t kchunk = ((kt + S - 1) / S + TM_TK - 1) / TM_TK * TM_TK;
  S = (long long)((kt + kchunk - 1) / kchunk);
  double2* part = (double2*)h->ws(WS_HALL_PART, (size_t)S * mm * sizeof(double2)).p;
  // one 4-D tensor map over the eight planes: (site within chunk < 8, row < M,
  // chunk < nk, plane < 8); boxes of 8 sites x 128 rows, 32-B swizzle
  CUtensorMap map;
  const cuuint64_t dims[4] = {(cuuint64_t)TM_TK, (cuuint64_t)M, (cuuint64_t)nk, 8};
  const cuuint64_t strides[3] = {(cuuint64_t)(TM_TK * sizeof(float)), (cuuint64_t)(cs * sizeof(float)),
                                 (cuuint64_t)(plane * sizeof(float))};
  const cuuint32_t box[4] = {(cuuint32_t)TM_TK, 128, 1, 1}, estr[4] = {1, 1, 1, 1};
  const CUresult cr = tensor_map_encoder()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, pl, dims, strides, box, estr,
                                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) throw Error(GQT_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)cr));
  // plane of each operand tile: P re_hi 0, im_hi 1, re_lo 2, im_lo 3; B 4..7
  const TmPlanes pz = {{0, 2, 1, 3}, {4, 6, 5, 7}};  // Pre_hi, Pre_lo, Pim_hi, Pim_lo; Bre_hi, Bre_lo, Bim_hi, Bim_lo
  check_cuda(cudaMemsetAsync(h->d_flag.p, 0, sizeof(int), st), "flag reset");
  check_cuda(cudaFuncSetAttribute(k_kb_gemm_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, TM_SMEM),
             "smem attribute");
  const size_t pg = prof_begin(st);
  k_kb_gemm_tma<<<dim3(tm, tn, (unsigned)S), TM_THREADS, TM_SMEM, st>>>(map, pz, M, kt, kchunk, part,
                                                                        (int*)h->d_flag.p, h->wait_limit);
  check_launch("k_kb_gemm_tma");
  prof_end(pg, 8, st);
  k_kb_reduce<<<(int)std::min<size_t>((mm + 255) / 256, 4096), 256, 0, st>>>(part, (int)S, M, (double)h->n / R,
                                                                              lam);
  check_launch("k_kb_reduce");
}

}  // namespace

extern "C" gqt_status gqt_kb_moments(gqt_ham* h, const void* d_r, int R, int M, int alpha, int beta,
                                     double* d_lambda, void* stream) {
  gqt::NvtxRange nvtx_call_(__func__);
  try {
    if (!h || !d_r || !d_lambda || R < 1 || M < 1 || alpha < 0 || alpha > 1 || beta < 0 || beta > 1)
      throw Error(GQT_EINVAL, "gqt_kb_moments: bad argument");
    if (h->prec != GQT_FP64 && h->kb_mode != 1)
      throw Error(GQT_EINVAL, "gqt_kb_moments: an FP32 handle needs the tensor-core contraction "
                              "(gqt_set_kb_contraction(ham, 1))");
    if (h->nseg != 1) throw Error(GQT_EINVAL, "gqt_kb_moments: one segment only");
    if ((alpha == 1 || beta == 1) && !h->has_dy)
      throw Error(GQT_EINVAL, "gqt_kb_moments: the lattice has no y displacements (bond_dy)");
    check_cuda(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    double2* lam = (double2*)d_lambda;
    if (h->prec == GQT_FP64) {
      const double* d[2] = {(const double*)h->d_dx.p, (const double*)h->d_dy.p};
      if (h->hop_real)
        kb_moments_impl<true, false>(h, d_r, R, M, d[alpha], d[beta], lam, st);
      else
        kb_moments_impl<true, true>(h, d_r, R, M, d[alpha], d[beta], lam, st);
    } else {
      // FP32 storage: dx is FP32, dy FP64
      const float* dxf = (const float*)h->d_dx.p;
      const double* dyd = (const double*)h->d_dy.p;
      auto run = [&](auto ch) {
        constexpr bool CH = decltype(ch)::value;
        if (alpha == 0 && beta == 0) kb_moments_impl<false, CH>(h, d_r, R, M, dxf, dxf, lam, st);
        if (alpha == 0 && beta == 1) kb_moments_impl<false, CH>(h, d_r, R, M, dxf, dyd, lam, st);
        if (alpha == 1 && beta == 0) kb_moments_impl<false, CH>(h, d_r, R, M, dyd, dxf, lam, st);
        if (alpha == 1 && beta == 1) kb_moments_impl<false, CH>(h, d_r, R, M, dyd, dyd, lam, st);
      };
      if (h->hop_real)
        run(std::integral_constant<bool, false>());
      else
        run(std::integral_constant<bool, true>());
    }
    int flag = 0;
    if (h->kb_mode != 0)
      check_cuda(cudaMemcpyAsync(&flag, h->d_flag.p, sizeof(int), cudaMemcpyDeviceToHost, st), "flag readback");
    check_cuda(cudaStreamSynchronize(st), "gqt_kb_moments");
    if (flag & 32)
      throw Error(GQT_ETIMEOUT, "gqt_kb_moments: a bounded tensor-core wait gave up and so did the drain of the "
                                "copies and products in flight: later results in this CUDA context are not trusted");
    if (flag & 16) throw Error(GQT_ETIMEOUT, "gqt_kb_moments: a bounded tensor-core wait gave up");
    return GQT_OK;
  } catch (const Error& e) {
    set_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return GQT_ENOMEM;
  } catch (const std::exception& e) {
    set_error(std::string("internal error: ") + e.what());
    return GQT_ECUDA;
  }
}

extern "C" gqt_status gqt_set_wait_limit(gqt_ham* h, int polls) {
  if (!h || polls < 0) {
    set_error("gqt_set_wait_limit: bad argument");
    return GQT_EINVAL;
  }
  h->wait_limit = polls;
  return GQT_OK;
}

extern "C" gqt_status gqt_set_kb_contraction(gqt_ham* h, int mode) {
  if (!h || mode < 0 || mode > 1) {
    set_error("gqt_set_kb_contraction: bad argument");
    return GQT_EINVAL;
  }
  h->kb_mode = mode;
  return GQT_OK;
}

// Device F (the Kubo-Bastin integrand) on the energy grid into buf + M (buf: M
// weights then NE values); returns an error code of the launches.
static cudaError_t kb_integrand_dev(const double* d_lambda, int M, const double* d_E, int NE, double energy_scale,
                                    int kernel, double* buf, cudaStream_t st) {
  std::vector<double> hw(M);
  for (int n = 0; n < M; ++n) hw[n] = (n == 0 ? 1.0 : 2.0) * (kernel == 0 ? jackson_g(n, M) : 1.0);
  // energies per CTA: as many as keep the tables (24 B per energy and moment) within 200 KB
  const int EB = (size_t)4 * M * 24 <= 200 * 1024 ? 4 : ((size_t)2 * M * 24 <= 200 * 1024 ? 2 : 1);
  const size_t smem = (size_t)EB * M * (sizeof(double) + sizeof(double2));
  const void* kern = EB == 4 ? (const void*)k_kb_integrand<4>
                             : (EB == 2 ? (const void*)k_kb_integrand<2> : (const void*)k_kb_integrand<1>);
  cudaError_t err = cudaSuccess;
  if (smem > 48 * 1024) err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  double* w = buf;
  double* F = buf + M;
  const double inv = 1.0 / energy_scale;
  if (err == cudaSuccess) err = cudaMemcpyAsync(w, hw.data(), M * sizeof(double), cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) {
    // the host copy of the weights must outlive the copy: wait for it here
    err = cudaStreamSynchronize(st);
  }
  if (err == cudaSuccess) {
    const dim3 grid((NE + EB - 1) / EB);
    const double2* lam = (const double2*)d_lambda;
    const size_t pi = prof_begin(st);
    if (EB == 4)
      k_kb_integrand<4><<<grid, 256, smem, st>>>(lam, M, d_E, NE, inv, w, F);
    else if (EB == 2)
      k_kb_integrand<2><<<grid, 256, smem, st>>>(lam, M, d_E, NE, inv, w, F);
    else
      k_kb_integrand<1><<<grid, 256, smem, st>>>(lam, M, d_E, NE, inv, w, F);
    err = cudaGetLastError();
    if (err == cudaSuccess) {
      check_launch("k_kb_integrand");
      prof_end(pi, 9, st);
    }
  }
  return err;
}

static std::vector<double> check_energies(const double* d_E, int NE, double energy_scale, cudaStream_t st) {
  std::vector<double> hE(NE);
  check_cuda(cudaMemcpyAsync(hE.data(), d_E, NE * sizeof(double), cudaMemcpyDeviceToHost, st), "energies");
  check_cuda(cudaStreamSynchronize(st), "energies");
  for (int j = 0; j < NE; ++j) {
    if (!(std::fabs(hE[j]) < energy_scale)) throw Error(GQT_EINVAL, "Kubo-Bastin: |E| must be < dE");
    if (j > 0 && !(hE[j] > hE[j - 1])) throw Error(GQT_EINVAL, "Kubo-Bastin: energies must ascend");
  }
  return hE;
}

extern "C" gqt_status gqt_kubo_bastin(const double* d_lambda, int M, const double* d_E, int NE, double energy_scale,
                                      double area, int kernel, double* d_sigma, void* stream) {
  gqt::NvtxRange nvtx_call_(__func__);
  try {
    if (!d_lambda || !d_E || !d_sigma || M < 1 || M > 8192 || NE < 1 || !(energy_scale > 0) || !(area > 0) ||
        kernel < 0 || kernel > 1)
      throw Error(GQT_EINVAL, "gqt_kubo_bastin: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    check_energies(d_E, NE, energy_scale, st);
    // device scratch owned by this call (no handle): weights and F
    double* buf = nullptr;
    check_cuda(cudaMallocAsync((void**)&buf, (size_t)(M + NE) * sizeof(double), st), "cudaMallocAsync");
    cudaError_t err = kb_integrand_dev(d_lambda, M, d_E, NE, energy_scale, kernel, buf, st);
    if (err == cudaSuccess) {
      k_kb_scan<<<1, 32, 0, st>>>(buf + M, d_E, NE, 1.0 / energy_scale, 2.0 / area, d_sigma);
      err = cudaGetLastError();
      if (err == cudaSuccess) check_launch("k_kb_scan");
    }
    cudaFreeAsync(buf, st);
    check_cuda(err, "gqt_kubo_bastin");
    check_cuda(cudaStreamSynchronize(st), "gqt_kubo_bastin");
    return GQT_OK;
  } catch (const Error& e) {
    set_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return GQT_ENOMEM;
  } catch (const std::exception& e) {
    set_error(std::string("internal error: ") + e.what());
    return GQT_ECUDA;
  }
}

extern "C" gqt_status gqt_kubo_bastin_fermi(const double* d_lambda, int M, const double* d_E, int NE,
                                            double energy_scale, double area, int kernel, const double* d_mu, int Nmu,
                                            double kT, double* d_sigma, void* stream) {
  gqt::NvtxRange nvtx_call_(__func__);
  try {
    if (!d_lambda || !d_E || !d_mu || !d_sigma || M < 1 || M > 8192 || NE < 2 || Nmu < 1 || !(energy_scale > 0) ||
        !(area > 0) || kernel < 0 || kernel > 1 || !(kT >= 0) || !std::isfinite(kT))
      throw Error(GQT_EINVAL, "gqt_kubo_bastin_fermi: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    check_energies(d_E, NE, energy_scale, st);
    double* buf = nullptr;
    check_cuda(cudaMallocAsync((void**)&buf, (size_t)(M + NE) * sizeof(double), st), "cudaMallocAsync");
    cudaError_t err = kb_integrand_dev(d_lambda, M, d_E, NE, energy_scale, kernel, buf, st);
    if (err == cudaSuccess) {
      k_kb_fermi<<<(Nmu + 127) / 128, 128, 0, st>>>(buf + M, d_E, NE, 1.0 / energy_scale, d_mu, Nmu, kT, 2.0 / area,
                                                    d_sigma);
      err = cudaGetLastError();
      if (err == cudaSuccess) check_launch("k_kb_fermi");
    }
    cudaFreeAsync(buf, st);
    check_cuda(err, "gqt_kubo_bastin_fermi");
    check_cuda(cudaStreamSynchronize(st), "gqt_kubo_bastin_fermi");
    return GQT_OK;
  } catch (const Error& e) {
    set_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return GQT_ENOMEM;
  } catch (const std::exception& e) {
    set_error(std::string("internal error: ") + e.what());
    return GQT_ECUDA;
  }
}
