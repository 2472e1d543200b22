// gqt_host.cu -- host runtime behind the C ABI of include/gqt.h.
//
// Owns the device copy of H~ (one allocation per array, ELL slot-major),
// per-handle workspace that grows on demand, the CTA-to-sites tables, CUDA
// graphs of repeated loops, and the drivers of the DOS, VAC and MSD loops of
// arXiv:1705.01387 (Sec. 3, Eqs. 17-30).  No entry point aborts: every failure
// becomes a gqt_status plus a thread-local message.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/gqt.h"
#include "gqt_internal.h"
#include "gqt_kernels.cuh"
#include "gqt_cluster.cuh"
#include "gqt_df.cuh"
#include "gqt_tile.cuh"

using namespace gqt;

namespace gqt {

thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};

void set_error(const std::string& s) { g_last_error = s; }

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw Error(GQT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void check_launch(const char* what) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Error(GQT_ECUDA, std::string("launch ") + what + ": " + cudaGetErrorString(e));
}

DevBuf::~DevBuf() {
  if (p) cudaFree(p);
}
void DevBuf::ensure(size_t n) {
  if (n <= bytes) return;
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
  cudaError_t e = cudaMalloc(&p, n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    throw Error(GQT_ENOMEM, "cudaMalloc of " + std::to_string(n) + " bytes failed: " + cudaGetErrorString(e));
  }
  bytes = n;
}

// ------------------------------------------------------------ Bessel (host)

// J_m(x), m < count, by Miller's backward recurrence J_{m-1} = (2m/x) J_m - J_{m+1}
// started far above max(count, x) and normalised with J_0 + 2 sum_k J_2k = 1.
void bessel_miller(double x, int count, double* J) {
  if (count <= 0) return;
  if (x == 0.0) {
    for (int m = 0; m < count; ++m) J[m] = (m == 0) ? 1.0 : 0.0;
    return;
  }
  const int top = std::max(count, (int)x) + 40 + (int)(6.0 * std::cbrt(x));
  const int start = top + (top & 1);  // even
  std::vector<double> j(start + 2, 0.0);
  j[start + 1] = 0.0;
  j[start] = 1e-300;
  double norm = 0.0;
  for (int m = start; m >= 1; --m) {
    j[m - 1] = (2.0 * m / x) * j[m] - j[m + 1];
    if (std::fabs(j[m - 1]) > 1e250) {  // rescale to stay in range
      for (int q = m - 1; q <= start; ++q) j[q] *= 1e-250;
    }
  }
  norm = j[0];
  for (int m = 2; m <= start; m += 2) norm += 2.0 * j[m];
  for (int m = 0; m < count; ++m) J[m] = j[m] / norm;
}

int np_rule_lib(double x, int cap) {
  const int probe = std::max(cap, (int)x + 64) + 64;
  std::vector<double> J(probe);
  bessel_miller(x, probe, J.data());
  int last = 0;
  for (int m = 0; m < probe; ++m)
    if (std::fabs(J[m]) >= 1e-15) last = m;
  return std::min(last + 1, cap);
}

// (2 - delta_m0) (-sign i)^m J_m(x), m < Np  (Eq. 17)
std::vector<double2> evolve_coefs(double x, int sign, int Np) {
  std::vector<double> J(Np);
  bessel_miller(x, Np, J.data());
  std::vector<double2> c(Np);
  for (int m = 0; m < Np; ++m) {
    const double f = (m == 0 ? 1.0 : 2.0) * J[m];
    // (-sign i)^m : m mod 4 cycle of (1, -sign i, -1, sign i)
    double re = 0, im = 0;
    switch (m & 3) {
      case 0: re = 1; break;
      case 1: im = -sign; break;
      case 2: re = -1; break;
      case 3: im = sign; break;
    }
    c[m] = make_double2(f * re, f * im);
  }
  return c;
}

}  // namespace gqt

// ====================================================================== profiler

// Optional per-kernel timing: CUDA events recorded on the launch stream
// around each launch of the profiled kernel families, summed on read.
namespace {
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<std::pair<int, size_t>> pairs;  // (category, index of start event)
  cudaEvent_t get() {
    if (used == pool.size()) {
      cudaEvent_t e;
      check_cuda(cudaEventCreate(&e), "cudaEventCreate");
      pool.push_back(e);
    }
    return pool[used++];
  }
};
Profiler g_prof;
}  // namespace

size_t gqt::prof_begin(cudaStream_t st) {
  if (!g_prof.on) return (size_t)-1;
  size_t i = g_prof.used;
  check_cuda(cudaEventRecord(g_prof.get(), st), "cudaEventRecord");
  return i;
}
void gqt::prof_end(size_t i, int cat, cudaStream_t st) {
  if (i == (size_t)-1) return;
  check_cuda(cudaEventRecord(g_prof.get(), st), "cudaEventRecord");
  g_prof.pairs.push_back({cat, i});
}

// ====================================================================== graphs

// Replays a loop of launches as a CUDA graph keyed by everything the launches
// depend on (kind, sizes, pointers, coefficients).  Capture and replay run on
// the handle's own non-blocking stream, ordered after and before the caller's
// stream by events, so the caller may pass the legacy default stream.
// 64-bit digest of a coefficient array (SplitMix64 finaliser folded over the
// words, so sign patterns cannot cancel); the array itself is stored with the
// graph and compared exactly on reuse.
static uint64_t digest(const std::vector<double>& v) {
  uint64_t x = 0x243F6A8885A308D3ull ^ (uint64_t)v.size();
  for (double d : v) {
    uint64_t u;
    memcpy(&u, &d, 8);
    x = splitmix_mix(x ^ u) + 0x9E3779B97F4A7C15ull;
  }
  return x;
}

template <class F>
static void run_graph(gqt_ham* h, std::string key, cudaStream_t st, F&& launches,
                      const std::vector<double>* data = nullptr) {
  if (!h->use_graphs || g_prof.on) {
    launches(st);
    return;
  }
  if (data) {
    char buf[40];
    snprintf(buf, sizeof buf, "|d%016llx", (unsigned long long)digest(*data));
    key += buf;
    auto d = h->graph_data.find(key);
    if (d != h->graph_data.end() && d->second != *data) {  // digest collision: no graph
      launches(st);
      return;
    }
  }
  if (!h->gstream) {
    check_cuda(cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking), "cudaStreamCreate");
    check_cuda(cudaEventCreateWithFlags(&h->gev[0], cudaEventDisableTiming), "cudaEventCreate");
    check_cuda(cudaEventCreateWithFlags(&h->gev[1], cudaEventDisableTiming), "cudaEventCreate");
  }
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    if (h->graphs.size() >= 512) {
      for (auto& g : h->graphs) cudaGraphExecDestroy(g.second);
      h->graphs.clear();
      h->graph_data.clear();
    }
    cudaGraph_t graph = nullptr;
    check_cuda(cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    try {
      launches(h->gstream);
    } catch (...) {
      cudaStreamEndCapture(h->gstream, &graph);
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      throw;
    }
    check_cuda(cudaStreamEndCapture(h->gstream, &graph), "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    check_cuda(e, "cudaGraphInstantiate");
    it = h->graphs.emplace(key, exec).first;
    if (data) h->graph_data[key] = *data;
  }
  check_cuda(cudaEventRecord(h->gev[0], st), "cudaEventRecord");
  check_cuda(cudaStreamWaitEvent(h->gstream, h->gev[0], 0), "cudaStreamWaitEvent");
  check_cuda(cudaGraphLaunch(it->second, h->gstream), "cudaGraphLaunch");
  g_launches.fetch_add(1, std::memory_order_relaxed);
  check_cuda(cudaEventRecord(h->gev[1], h->gstream), "cudaEventRecord");
  check_cuda(cudaStreamWaitEvent(st, h->gev[1], 0), "cudaStreamWaitEvent");
}

static std::string key_of(const char* op, std::initializer_list<const void*> ptrs, std::initializer_list<double> nums) {
  std::string k(op);
  char buf[64];
  for (auto p : ptrs) {
    snprintf(buf, sizeof buf, "|%p", p);
    k += buf;
  }
  for (auto x : nums) {
    snprintf(buf, sizeof buf, "|%.17g", x);
    k += buf;
  }
  return k;
}

// The exact bits of every expansion coefficient, as part of a graph key (a
// lossy hash can map U(+dt) and U(-dt), whose coefficients differ only in
// signs, to the same key).
static std::string coef_bits(const std::vector<double2>& c) {
  std::string k("|c");
  char buf[40];
  for (const double2& q : c) {
    uint64_t u[2];
    memcpy(u, &q, 16);
    snprintf(buf, sizeof buf, "%016llx%016llx", (unsigned long long)u[0], (unsigned long long)u[1]);
    k += buf;
  }
  return k;
}

// ====================================================================== handle

static bool is_pow2_r(int R) { return R == 1 || R == 2 || R == 4 || R == 8 || R == 16 || R == 32; }

// dynamic shared memory of the CTA reductions (NV values per vector per warp)
static size_t smem_bytes(const gqt_ham* h, int R, int nv) { return (size_t)nv * (h->threads / 32) * R * sizeof(double2); }

static int rshift_of(int R) {
  int s = 0;
  while ((1 << s) < R) ++s;
  return s;
}

// Next-iteration prefetch of the multi-vector kernels (FP32 storage, where the
// dependent index load bounds the iteration): needs a lane group of at least K + 1
// lanes per site within one warp.
template <bool FP64>
static bool vpt_prefetch(int KK, int R, int vpt) {
  const int G = R / vpt;
  return !FP64 && G >= KK + 1 && G <= 32;
}

// Resident CTAs per SM of the handle's main moment kernel for R vectors (the
// kernel the default variant runs), so that the default grid is exactly one
// wave: SMs x resident CTAs.
template <bool FP64, bool CH, int KK>
static int wave_occupancy_k(int R, int variant, int threads, bool dbl) {
  const void* f = nullptr;
  const bool vpt = threads <= 128 && R >= 2 && (variant == 2 || variant == 3);
  if (dbl) {
    if (vpt && variant == 2 && R >= 4)
      f = vpt_prefetch<FP64>(KK, R, 4) ? (const void*)k_cheb_dbl_wv<FP64, CH, 4, KK, !FP64>
                                       : (const void*)k_cheb_dbl_wv<FP64, CH, 4, KK>;
    else if (vpt)
      f = vpt_prefetch<FP64>(KK, R, 2) ? (const void*)k_cheb_dbl_wv<FP64, CH, 2, KK, !FP64>
                                       : (const void*)k_cheb_dbl_wv<FP64, CH, 2, KK>;
    else if (variant == 2)
      f = (const void*)k_cheb_dbl_w<FP64, CH, 2, KK>;
    else
      f = (const void*)k_cheb_dbl_w<FP64, CH, 1, KK>;
  } else {
    if (vpt)
      f = vpt_prefetch<FP64>(KK, R, 2) ? (const void*)k_cheb_re_wv<FP64, CH, 2, KK, !FP64>
                                       : (const void*)k_cheb_re_wv<FP64, CH, 2, KK>;
    else if (variant == 2)
      f = (const void*)k_cheb_re_w<FP64, CH, 2, KK>;
    else
      f = (const void*)k_cheb_re_w<FP64, CH, 1, KK>;
  }
  int n = 0;
  const size_t smem = (size_t)3 * (threads / 32) * R * sizeof(double2);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 4;
  }
  return std::max(1, n);
}

template <bool FP64, bool CH, int KK>
static int pair_occupancy_k(int R, int threads) {
  int n = 0;
  const size_t smem = (size_t)3 * (threads / 32) * R * sizeof(double2);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, (const void*)k_cheb_pair_w<FP64, CH, KK>, threads, smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 3;
  }
  return std::max(1, n);
}

template <bool FP64, bool CH>
static int pair_occupancy(int K, int R, int threads) {
  switch (K) {
    case 2: return pair_occupancy_k<FP64, CH, 2>(R, threads);
    case 3: return pair_occupancy_k<FP64, CH, 3>(R, threads);
    case 4: return pair_occupancy_k<FP64, CH, 4>(R, threads);
    default: return pair_occupancy_k<FP64, CH, 6>(R, threads);
  }
}

// l != r moment rows by two recurrences: the wavefront kernels' neighbour counts,
// one element per thread (k_cheb_pair_w) or, where the multi-vector form applies,
// two vectors per lane (k_cheb_pair_wv).
static bool pair_applies(const gqt_ham* h, int R) {
  if (!h->use_pair || h->variant == 0 || h->threads > 256) return false;
  return h->K == 2 || h->K == 3 || h->K == 4 || h->K == 6;
}
static bool pair_vpt(const gqt_ham* h, int R) {
  return (h->variant == 2 || h->variant == 3) && R >= 2 && h->threads <= 128;
}

template <bool FP64, bool CH, int KK>
static int pair_wv_occupancy_k(int R, int threads) {
  int n = 0;
  const void* f = vpt_prefetch<FP64>(KK, R, 2) ? (const void*)k_cheb_pair_wv<FP64, CH, 2, KK, !FP64>
                                               : (const void*)k_cheb_pair_wv<FP64, CH, 2, KK>;
  const size_t smem = (size_t)3 * (threads / 32) * R * sizeof(double2);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 4;
  }
  return std::max(1, n);
}

template <bool FP64, bool CH>
static int pair_wv_occupancy(int K, int R, int threads) {
  switch (K) {
    case 2: return pair_wv_occupancy_k<FP64, CH, 2>(R, threads);
    case 3: return pair_wv_occupancy_k<FP64, CH, 3>(R, threads);
    case 4: return pair_wv_occupancy_k<FP64, CH, 4>(R, threads);
    default: return pair_wv_occupancy_k<FP64, CH, 6>(R, threads);
  }
}

template <bool FP64, bool CH>
static int wave_occupancy(int K, int R, int variant, int threads, bool dbl) {
  switch (K) {
    case 2: return wave_occupancy_k<FP64, CH, 2>(R, variant, threads, dbl);
    case 3: return wave_occupancy_k<FP64, CH, 3>(R, variant, threads, dbl);
    case 4: return wave_occupancy_k<FP64, CH, 4>(R, variant, threads, dbl);
    case 6: return wave_occupancy_k<FP64, CH, 6>(R, variant, threads, dbl);
    default: return 4;
  }
}

// Resident CTAs per SM of the moment kernel a call of this kind will launch
// (kind 1: Re <l|T|r> orders, kind 2: l = r orders); 0 when the chunk-ordered
// kernels run (they use the default table).
static int moment_grid_per_sm(const gqt_ham* h, int R, int kind) {
  if (h->blocks_per_sm > 0 || h->variant == 0 || h->threads > 256 || kind == 0) return 0;
  if (!(h->K == 2 || h->K == 3 || h->K == 4 || h->K == 6)) return 0;
  const bool dbl = kind == 2;
  int occ;
  if (kind == 1 && pair_applies(h, R) && pair_vpt(h, R))
    occ = h->prec == GQT_FP64 ? (h->hop_real ? pair_wv_occupancy<true, false>(h->K, R, h->threads)
                                             : pair_wv_occupancy<true, true>(h->K, R, h->threads))
                              : (h->hop_real ? pair_wv_occupancy<false, false>(h->K, R, h->threads)
                                             : pair_wv_occupancy<false, true>(h->K, R, h->threads));
  else if (kind == 1 && pair_applies(h, R))
    occ = h->prec == GQT_FP64 ? (h->hop_real ? pair_occupancy<true, false>(h->K, R, h->threads)
                                             : pair_occupancy<true, true>(h->K, R, h->threads))
                              : (h->hop_real ? pair_occupancy<false, false>(h->K, R, h->threads)
                                             : pair_occupancy<false, true>(h->K, R, h->threads));
  else if (h->prec == GQT_FP64)
    occ = h->hop_real ? wave_occupancy<true, false>(h->K, R, h->variant, h->threads, dbl)
                      : wave_occupancy<true, true>(h->K, R, h->variant, h->threads, dbl);
  else
    occ = h->hop_real ? wave_occupancy<false, false>(h->K, R, h->variant, h->threads, dbl)
                      : wave_occupancy<false, true>(h->K, R, h->variant, h->threads, dbl);
  return std::max(1, std::min(occ, 16));
}

const BlockTable& gqt_ham::table(int R, int grid_per_sm) {
  const int tkey = R * 64 + grid_per_sm;
  auto it = tables.find(tkey);
  if (it != tables.end()) return *it->second;
  auto t = std::make_unique<BlockTable>();
  int per_sm = grid_per_sm > 0 ? grid_per_sm : blocks_per_sm;
  if (per_sm <= 0) {
    if (variant == 0 || threads > 256)
      per_sm = 4;
    else if (prec == GQT_FP64)
      per_sm = hop_real ? wave_occupancy<true, false>(K, R, variant, threads, false)
                        : wave_occupancy<true, true>(K, R, variant, threads, false);
    else
      per_sm = hop_real ? wave_occupancy<false, false>(K, R, variant, threads, false)
                        : wave_occupancy<false, true>(K, R, variant, threads, false);
    per_sm = std::max(4, std::min(per_sm, 8));  // the chunk-ordered kernels (evolution, velocity) want >= 4
  }
  const int thr = threads;
  const long long max_blocks = (long long)sm_count() * per_sm;
  // at least ~2 elements per thread per CTA
  const long long want = std::max<long long>(nseg, std::min<long long>(max_blocks, (n * (long long)R + 2LL * thr - 1) / (2LL * thr)));
  std::vector<int> blk{0}, seg_blk{0};
  for (int s = 0; s < nseg; ++s) {
    const int64_t a = seg[s], b = seg[s + 1];
    const int64_t ns = b - a;
    long long nb = std::max<long long>(1, (long long)std::llround((double)want * (double)ns / (double)n));
    nb = std::min<long long>(nb, std::max<int64_t>(1, ns));
    for (long long q = 1; q <= nb; ++q) blk.push_back((int)(a + (ns * q) / nb));
    seg_blk.push_back((int)blk.size() - 1);
  }
  t->nblocks = (int)blk.size() - 1;
  std::vector<int4> tab4(t->nblocks);
  for (int s = 0; s < nseg; ++s) {
    const int G = seg_blk[s + 1] - seg_blk[s];
    for (int q = 0; q < G; ++q) tab4[seg_blk[s] + q] = make_int4((int)seg[s], (int)seg[s + 1], q, G);
  }
  t->d_tab4.ensure(tab4.size() * sizeof(int4));
  check_cuda(cudaMemcpy(t->d_tab4.p, tab4.data(), tab4.size() * sizeof(int4), cudaMemcpyHostToDevice), "table");
  t->d_blk.ensure(blk.size() * sizeof(int));
  t->d_seg_blk.ensure(seg_blk.size() * sizeof(int));
  check_cuda(cudaMemcpy(t->d_blk.p, blk.data(), blk.size() * sizeof(int), cudaMemcpyHostToDevice), "table");
  check_cuda(cudaMemcpy(t->d_seg_blk.p, seg_blk.data(), seg_blk.size() * sizeof(int), cudaMemcpyHostToDevice), "table");
  auto& ref = *t;
  tables[tkey] = std::move(t);
  return ref;
}

DevBuf& gqt_ham::ws(int slot, size_t bytes) {
  if ((int)work.size() <= slot) work.resize(slot + 1);
  if (!work[slot]) work[slot] = std::make_unique<DevBuf>();
  work[slot]->ensure(bytes);
  return *work[slot];
}

// ====================================================================== dispatch helpers

template <bool FP64, bool CH>
static Ell<FP64, CH> ell_of(const gqt_ham* h) {
  Ell<FP64, CH> e;
  e.n = (int)h->n;
  e.K = h->K;
  e.idx = (const int*)h->d_idx.p;
  e.hop2 = (const typename Ell<FP64, CH>::HT*)h->d_hop.p;
  e.diag2 = (const typename Ell<FP64, CH>::S*)h->d_diag.p;
  e.dx = (const typename Ell<FP64, CH>::S*)h->d_dx.p;
  e.row_shift = (h->use_sweep_order && h->row_shift > 0) ? h->row_shift : 0;
  return e;
}

template <class F>
static void dispatch(const gqt_ham* h, F&& f) {
  if (h->prec == GQT_FP64) {
    if (h->hop_real)
      f(ell_of<true, false>(h));
    else
      f(ell_of<true, true>(h));
  } else {
    if (h->hop_real)
      f(ell_of<false, false>(h));
    else
      f(ell_of<false, true>(h));
  }
}

template <class E>
struct EllTraits;
template <bool FP64, bool CH>
struct EllTraits<Ell<FP64, CH>> {
  static constexpr bool fp64 = FP64;
  static constexpr bool ch = CH;
  using V = typename Prec<FP64>::V;
};

size_t gqt_ham::vec_bytes(int R) const { return (size_t)n * R * (prec == GQT_FP64 ? 16 : 8); }

// ====================================================================== status

static gqt_status finish_call(gqt_ham* h, cudaStream_t st, const char* what) {
  int flag = 0;
  check_cuda(cudaMemcpyAsync(h->h_flag, h->d_flag.p, sizeof(int), cudaMemcpyDeviceToHost, st), "flag readback");
  check_cuda(cudaStreamSynchronize(st), what);
  flag = *h->h_flag;
  if (flag & 4) throw Error(GQT_ENAN, std::string(what) + ": NaN or Inf in a result");
  if (flag & 2)
    throw Error(GQT_ERANGE, std::string(what) +
                                ": a Chebyshev moment exceeds |l||r|: the spectrum of H/dE is not inside [-1,1] "
                                "(energy scale too small)");
  if (flag & 8) throw Error(GQT_ENORM, std::string(what) + ": |U psi| differs from |psi| beyond tolerance");
  if (flag & 16) throw Error(GQT_ETIMEOUT, std::string(what) + ": a bounded device wait gave up");
  return GQT_OK;
}

static void reset_flag(gqt_ham* h, cudaStream_t st) {
  check_cuda(cudaMemsetAsync(h->d_flag.p, 0, sizeof(int), st), "flag reset");
}

// ====================================================================== moments core

// Wavefront-ordered moment kernels for the common neighbour counts (2, 3, 4, 6
// slots); other counts return false and use the chunk-ordered kernels.
template <bool FP64, bool CH, class V>
static bool launch_wave_re(gqt_ham* h, const Ell<FP64, CH>& H, const BlockTable& T, int R, int rs, const V* tm1,
                           const V* tm2, V* tout, const V* l, double2* partial, int slot0, int slot_norm, int first,
                           cudaStream_t st) {
  if (h->threads > 256 || h->variant == 0) return false;
  const int4* tab = (const int4*)T.d_tab4.p;
  const size_t sm = smem_bytes(h, R, 3);
#define GQT_WAVE_RE(KK)                                                                                          \
  if ((h->variant == 2 || h->variant == 3) && R >= 2 && h->threads <= 128 && vpt_prefetch<FP64>(KK, R, 2))    \
    k_cheb_re_wv<FP64, CH, 2, KK, !FP64><<<T.nblocks, h->threads, sm, st>>>(                                     \
        H, tab, R, rs - 1, tm1, tm2, tout, l, partial, T.nblocks, slot0, slot_norm, first);                      \
  else if ((h->variant == 2 || h->variant == 3) && R >= 2 && h->threads <= 128)                                  \
    k_cheb_re_wv<FP64, CH, 2, KK><<<T.nblocks, h->threads, sm, st>>>(H, tab, R, rs - 1, tm1, tm2, tout, l,       \
                                                                     partial, T.nblocks, slot0, slot_norm, first); \
  else if (h->variant == 1)                                                                                      \
    k_cheb_re_w<FP64, CH, 1, KK><<<T.nblocks, h->threads, sm, st>>>(H, tab, R, rs, tm1, tm2, tout, l, partial, \
                                                                    T.nblocks, slot0, slot_norm, first);       \
  else                                                                                                           \
    k_cheb_re_w<FP64, CH, 2, KK><<<T.nblocks, h->threads, sm, st>>>(H, tab, R, rs, tm1, tm2, tout, l, partial, \
                                                                    T.nblocks, slot0, slot_norm, first);       \
  return true;
  switch (H.K) {
    case 2: GQT_WAVE_RE(2)
    case 3: GQT_WAVE_RE(3)
    case 4: GQT_WAVE_RE(4)
    case 6: GQT_WAVE_RE(6)
    default: return false;
  }
#undef GQT_WAVE_RE
}

template <bool FP64, bool CH, class V>
static bool launch_wave_dbl(gqt_ham* h, const Ell<FP64, CH>& H, const BlockTable& T, int R, int rs, const V* tm1,
                            const V* tm2, V* tout, double2* partial, int m, cudaStream_t st) {
  if (h->threads > 256 || h->variant == 0) return false;
  const int4* tab = (const int4*)T.d_tab4.p;
  const size_t sm = smem_bytes(h, R, 3);
#define GQT_WAVE_DBL(KK)                                                                                           \
  if (h->variant == 3 && R >= 2 && h->threads <= 128 && vpt_prefetch<FP64>(KK, R, 2))                            \
    k_cheb_dbl_wv<FP64, CH, 2, KK, !FP64><<<T.nblocks, h->threads, sm, st>>>(H, tab, R, rs - 1, tm1, tm2, tout,   \
                                                                             partial, T.nblocks, m);             \
  else if (h->variant == 3 && R >= 2 && h->threads <= 128)                                                         \
    k_cheb_dbl_wv<FP64, CH, 2, KK><<<T.nblocks, h->threads, sm, st>>>(H, tab, R, rs - 1, tm1, tm2, tout, partial, \
                                                                      T.nblocks, m);                              \
  else if (h->variant == 2 && R >= 4 && h->threads <= 128 && vpt_prefetch<FP64>(KK, R, 4))                       \
    k_cheb_dbl_wv<FP64, CH, 4, KK, !FP64><<<T.nblocks, h->threads, sm, st>>>(H, tab, R, rs - 2, tm1, tm2, tout,   \
                                                                             partial, T.nblocks, m);             \
  else if (h->variant == 2 && R >= 4 && h->threads <= 128)                                                         \
    k_cheb_dbl_wv<FP64, CH, 4, KK><<<T.nblocks, h->threads, sm, st>>>(H, tab, R, rs - 2, tm1, tm2, tout, partial, \
                                                                      T.nblocks, m);                              \
  else if (h->variant == 2 && R == 2 && h->threads <= 128)                                                         \
    k_cheb_dbl_wv<FP64, CH, 2, KK><<<T.nblocks, h->threads, sm, st>>>(H, tab, R, rs - 1, tm1, tm2, tout, partial, \
                                                                      T.nblocks, m);                              \
  else if (h->variant == 1)                                                                                        \
    k_cheb_dbl_w<FP64, CH, 1, KK><<<T.nblocks, h->threads, sm, st>>>(H, tab, R, rs, tm1, tm2, tout, partial,     \
                                                                     T.nblocks, m);                               \
  else                                                                                                             \
    k_cheb_dbl_w<FP64, CH, 2, KK><<<T.nblocks, h->threads, sm, st>>>(H, tab, R, rs, tm1, tm2, tout, partial,     \
                                                                     T.nblocks, m);                               \
  return true;
  switch (H.K) {
    case 2: GQT_WAVE_DBL(2)
    case 3: GQT_WAVE_DBL(3)
    case 4: GQT_WAVE_DBL(4)
    case 6: GQT_WAVE_DBL(6)
    default: return false;
  }
#undef GQT_WAVE_DBL
}

// Cluster-resident moment rows (small systems, R = 1, one segment): one launch of
// k_cheb_cluster per row instead of one launch per order.  Returns false when
// the row does not fit on chip or clusters are unavailable.
template <bool FP64, bool CH, bool DBL, class V>
static bool launch_cluster_row(gqt_ham* h, const Ell<FP64, CH>& H, const V* r, const V* l, double2* partial, int M,
                               int slot_norm, cudaStream_t st, int* nblk) {
  if (!h->use_cluster) return false;
  auto kern = k_cheb_cluster<FP64, CH, DBL>;
  const int per_site = cluster_site_bytes<FP64, CH>(h->K, !DBL);
  for (int C : {16, 8}) {
    const int chunk = (int)((h->n + C - 1) / C);
    const int thr = std::min(1024, std::max(32, (chunk + 31) / 32 * 32));
    const size_t smem = (size_t)chunk * per_site + 64 + cluster_red_bytes(M, slot_norm, thr / 32) + 16;
    if (smem > 220 * 1024) continue;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(thr, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      continue;
    }
    check_cuda(cudaLaunchKernelEx(&cfg, kern, H, chunk, r, l, partial, M, slot_norm), "k_cheb_cluster");
    check_launch("k_cheb_cluster");
    *nblk = C;
    return true;
  }
  return false;
}

template <bool FP64, bool CH, class V>
static void launch_wave_pair(gqt_ham* h, const Ell<FP64, CH>& H, const BlockTable& T, int R, int rs, const V* am1,
                             const V* bm1, const V* am2, const V* bm2, V* aout, V* bout, double2* partial, int m,
                             int slot_norm, cudaStream_t st) {
  const int4* tab = (const int4*)T.d_tab4.p;
  const size_t sm = smem_bytes(h, R, 3);
#define GQT_PAIR(KK)                                                                                              \
  if (pair_vpt(h, R) && vpt_prefetch<FP64>(KK, R, 2))                                                            \
    k_cheb_pair_wv<FP64, CH, 2, KK, !FP64><<<T.nblocks, h->threads, sm, st>>>(                                   \
        H, tab, R, rs - 1, am1, bm1, am2, bm2, aout, bout, partial, T.nblocks, m, slot_norm);                    \
  else if (pair_vpt(h, R))                                                                                       \
    k_cheb_pair_wv<FP64, CH, 2, KK><<<T.nblocks, h->threads, sm, st>>>(H, tab, R, rs - 1, am1, bm1, am2, bm2,     \
                                                                       aout, bout, partial, T.nblocks, m,        \
                                                                       slot_norm);                               \
  else                                                                                                           \
    k_cheb_pair_w<FP64, CH, KK><<<T.nblocks, h->threads, sm, st>>>(H, tab, R, rs, am1, bm1, am2, bm2, aout, bout, \
                                                                   partial, T.nblocks, m, slot_norm);            \
  break;
  switch (H.K) {
    case 2: GQT_PAIR(2)
    case 3: GQT_PAIR(3)
    case 4: GQT_PAIR(4)
    default: GQT_PAIR(6)
  }
#undef GQT_PAIR
}

// ------------------------------------------------ FP64 rows on the FP32 pipes

// Moment rows of FP64 handles with R = 1 run on pairs of FP32 numbers when the
// handle's FP64 arithmetic mode is 1 (gqt_set_fp64_arith): the two-recurrence
// VAC rows and the l = r rows, for the neighbour counts of the wavefront kernels.
static bool df_applies(const gqt_ham* h, int R, int kind) {
  if (!(h->prec == GQT_FP64 && h->fp64_arith == 1 && R == 1 && h->variant != 0 && h->threads <= 256)) return false;
  if (!(h->K == 2 || h->K == 3 || h->K == 4 || h->K == 6)) return false;
  return kind == 2 || (kind == 1 && pair_applies(h, R));
}

// 2H~ and 2U/dE as (hi, lo) pairs, split once from the FP64 arrays (again after
// gqt_update_hamiltonian).  Runs on the call's stream before any graph capture.
static void ensure_df(gqt_ham* h, cudaStream_t st) {
  if (h->df_ready) return;
  const size_t nslots = (size_t)h->K * h->n;
  h->d_hop_df.ensure(nslots * (h->hop_real ? sizeof(float2) : sizeof(float4)));
  h->d_diag_df.ensure((size_t)h->n * sizeof(float2));
  const int blocks = sm_count() * 8;
  if (h->hop_real)
    k_split_hamiltonian<false><<<blocks, 256, 0, st>>>((long long)nslots, h->d_hop.p, (int)h->n,
                                                       (const double*)h->d_diag.p, h->d_hop_df.p,
                                                       (float2*)h->d_diag_df.p);
  else
    k_split_hamiltonian<true><<<blocks, 256, 0, st>>>((long long)nslots, h->d_hop.p, (int)h->n,
                                                      (const double*)h->d_diag.p, h->d_hop_df.p,
                                                      (float2*)h->d_diag_df.p);
  check_launch("k_split_hamiltonian");
  h->df_ready = true;
}

template <bool CH>
static DfEll<CH> df_ell_of(const gqt_ham* h) {
  DfEll<CH> e;
  e.n = (int)h->n;
  e.K = h->K;
  e.idx = (const int*)h->d_idx.p;
  e.hop = (const typename DfHop<CH>::T*)h->d_hop_df.p;
  e.diag = (const float2*)h->d_diag_df.p;
  e.xhop = (const typename DfHop<CH>::T*)h->d_xhop_df.p;
  if (h->hop_uniform) {
    const float a = (float)h->hop0;
    e.h0 = make_float2(a, (float)(h->hop0 - (double)a));
  }
  return e;
}

// 2[X,H~] slot values as pairs for the commutator orders (once per handle, again
// after gqt_update_hamiltonian).  Runs on the call's stream before any capture.
static void ensure_df_x(gqt_ham* h, cudaStream_t st) {
  if (h->dfx_ready) return;
  const size_t nslots = (size_t)h->K * h->n;
  h->d_xhop_df.ensure(nslots * (h->hop_real ? sizeof(float2) : sizeof(float4)));
  const int blocks = sm_count() * 8;
  if (h->hop_real)
    k_split_xhop<false><<<blocks, 256, 0, st>>>((long long)nslots, h->d_hop.p, (const double*)h->d_dx.p,
                                                h->d_xhop_df.p);
  else
    k_split_xhop<true><<<blocks, 256, 0, st>>>((long long)nslots, h->d_hop.p, (const double*)h->d_dx.p,
                                               h->d_xhop_df.p);
  check_launch("k_split_xhop");
  h->dfx_ready = true;
}

// elements in flight per thread in the l = r rows (two, within 85 registers, up
// to four neighbour slots)
constexpr int df_u(int KK) { return KK <= 4 ? 2 : 1; }

template <bool CH, int KK>
static int df_occupancy_k(bool pair, int threads) {
  const void* f = pair ? (const void*)k_cheb_pair_df<CH, KK, false> : (const void*)k_cheb_dbl_df<CH, KK, df_u(KK), false>;
  int n = 0;
  const size_t smem = (size_t)3 * (threads / 32) * sizeof(double2);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 3;
  }
  return std::max(1, std::min(n, 16));
}

template <bool CH>
static int df_occupancy(int K, bool pair, int threads) {
  switch (K) {
    case 2: return df_occupancy_k<CH, 2>(pair, threads);
    case 3: return df_occupancy_k<CH, 3>(pair, threads);
    case 4: return df_occupancy_k<CH, 4>(pair, threads);
    default: return df_occupancy_k<CH, 6>(pair, threads);
  }
}

// Temporal blocking of the paired-FP32 rows (two orders per pass, gqt_tile.cuh):
// honeycomb handles whose rows follow the built-in cell layout, one segment,
// L1 a multiple of 32 cells (the band width).
static bool tiled_applies(const gqt_ham* h) {
  return h->use_tiling && h->honey_L1 > 0 && h->nseg == 1 && h->K == 3 && tl_band_width(h->honey_L1) > 0 &&
         h->honey_L2 >= 2;
}

static Honey honey_of(const gqt_ham* h) {
  Honey G;
  G.L1 = h->honey_L1;
  G.L2 = h->honey_L2;
  // cell offsets of the three neighbour types, A (s = 0) and B (s = 1)
  static const int O1[2][3] = {{0, 1, 0}, {0, -1, 0}}, O2[2][3] = {{0, -1, -1}, {0, 1, 1}};
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < 3; ++k) {
      G.o1[s][k] = O1[s][h->honey_type[s][k]];
      G.o2[s][k] = O2[s][h->honey_type[s][k]];
    }
  return G;
}


// CTAs of the blocked kernel: as many as are resident at once (each takes an
// equal share of the band rows), at most the single-order grid nb (the stride of
// the moment partial slots).
constexpr size_t TL_SMEM = 4 * 8 * sizeof(double);  // block_reduce_rx<4> over at most 8 warps

template <bool CH, int NC>
static int tiled_grid(int threads) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cheb2_honey_df<CH, NC>, threads, TL_SMEM) != cudaSuccess) {
    cudaGetLastError();
    n = 1;
  }
  return std::max(1, n) * sm_count();
}

// The rows' chains live in rotating buffers (4 per chain when tiled, else 2):
// after step j, T_j is in buffer cur and T_{j-1} in buffer prv.  A single-order
// step writes T_{j+1} over T_{j-1} (same element, same thread); a tiled pass
// reads T_j and T_{j-1} and writes T_{j+1} and T_{j+2} into the two other buffers.
template <bool CH, int KK>
static void df_rows(gqt_ham* h, const BlockTable& T, bool pair, int steps, const void* l, const void* r,
                    float4* const* A, float4* const* B, int tgrid, int tnseg, double2* partial,
                    double2* tscratch, cudaStream_t s2) {
  const bool tiled = tgrid > 0;
  const DfEll<CH> H = df_ell_of<CH>(h);
  const int4* tab = (const int4*)T.d_tab4.p;
  const int nb = T.nblocks;
  const size_t sm = smem_bytes(h, 1, 3);
  int cur = 0, prv = 1;
  for (int m = 1; m <= std::max(steps, 1);) {
    size_t pe = prof_begin(s2);
    if (m == 1) {
      if (pair)
        k_cheb_pair_df<CH, KK, true><<<nb, h->threads, sm, s2>>>(H, tab, l, r, nullptr, nullptr, A[0], B[0], A[1],
                                                                 B[1], partial, nb, 1, 2 * steps);
      else
        k_cheb_dbl_df<CH, KK, df_u(KK), true><<<nb, h->threads, sm, s2>>>(H, tab, r, nullptr, B[0], B[1], partial, nb,
                                                                          1);
      check_launch(pair ? "k_cheb_pair_df(first)" : "k_cheb_dbl_df(first)");
      prof_end(pe, 0, s2);
      m = 2;
      continue;
    }
    if constexpr (KK == 3) {
      if (tiled && m + 1 <= steps) {
        int f[2], nf = 0;
        for (int b = 0; b < 4 && nf < 2; ++b)
          if (b != cur && b != prv) f[nf++] = b;
        const Honey G = honey_of(h);
        const int bw = tl_band_width(G.L1);
        // partial dots: straight into the moment slots when the grid fits them, else
        // per CTA into scratch and folded
        const bool fold = tgrid > nb;
        double2* pout = fold ? tscratch : partial + (size_t)(2 * m - 2) * nb;
        const int ostride = fold ? tgrid : nb, nzero = fold ? 0 : nb;
        // handles whose slots all hold one real hopping read no hop array (UH)
        auto blocked = [&](auto uh) {
          constexpr bool UH = decltype(uh)::value && !CH;
          if (pair)
            k_cheb2_honey_df<CH, 2, UH><<<tgrid, 2 * bw, TL_SMEM, s2>>>(H, G, bw, tnseg, A[cur], A[prv], B[cur],
                                                                       B[prv], A[f[0]], A[f[1]], B[f[0]], B[f[1]],
                                                                       pout, ostride, nzero);
          else
            k_cheb2_honey_df<CH, 1, UH><<<tgrid, 2 * bw, TL_SMEM, s2>>>(H, G, bw, tnseg, B[cur], B[prv], nullptr,
                                                                       nullptr, B[f[0]], B[f[1]], nullptr, nullptr,
                                                                       pout, ostride, nzero);
        };
        if (h->hop_uniform)
          blocked(std::true_type());
        else
          blocked(std::false_type());
        check_launch("k_cheb2_honey_df");
        if (fold) {
          k_tl_fold<<<4, 128, 0, s2>>>(tscratch, tgrid, 1, partial, nb, 2 * m - 2);
          check_launch("k_tl_fold");
        }
        prof_end(pe, pair ? 10 : 11, s2);
        prv = f[0];
        cur = f[1];
        m += 2;
        continue;
      }
    }
    if (pair)
      k_cheb_pair_df<CH, KK, false><<<nb, h->threads, sm, s2>>>(H, tab, A[cur], B[cur], A[prv], B[prv], A[prv],
                                                                B[prv], nullptr, nullptr, partial, nb, m, 2 * steps);
    else
      k_cheb_dbl_df<CH, KK, df_u(KK), false><<<nb, h->threads, sm, s2>>>(H, tab, B[cur], B[prv], B[prv], nullptr,
                                                                         partial, nb, m);
    check_launch(pair ? "k_cheb_pair_df" : "k_cheb_dbl_df");
    prof_end(pe, pair ? 6 : 5, s2);
    std::swap(cur, prv);
    ++m;
  }
}

// kind 1 (two-recurrence VAC rows) or 2 (l = r rows) of an FP64 handle, R = 1,
// on the FP32 pipes; same partial slots and reduction as the FP64 kernels.
static void launch_moments_df(gqt_ham* h, const void* l, const void* r, int M, void* out, int kind,
                              cudaStream_t st) {
  ensure_df(h, st);
  const bool pair = kind == 1;
  const int occ = h->blocks_per_sm > 0 ? h->blocks_per_sm
                                       : (h->hop_real ? df_occupancy<false>(h->K, pair, h->threads)
                                                      : df_occupancy<true>(h->K, pair, h->threads));
  const BlockTable& T = h->table(1, occ);
  const int nb = T.nblocks;
  const size_t vb = h->vec_bytes(1);
  const bool tiled = tiled_applies(h);
  float4* A[4] = {nullptr, nullptr, nullptr, nullptr};
  float4* B[4] = {(float4*)h->ws(WS_T1, vb).p, (float4*)h->ws(WS_T2, vb).p, nullptr, nullptr};
  if (pair) {
    A[0] = (float4*)h->ws(WS_PA1, vb).p;
    A[1] = (float4*)h->ws(WS_PA2, vb).p;
  }
  if (tiled) {
    B[2] = (float4*)h->ws(WS_TILE0, vb).p;
    B[3] = (float4*)h->ws(WS_TILE0 + 1, vb).p;
    if (pair) {
      A[2] = (float4*)h->ws(WS_TILE0 + 2, vb).p;
      A[3] = (float4*)h->ws(WS_TILE0 + 3, vb).p;
    }
  }
  const int slots = std::max(M, 2) + 4;
  double2* partial = (double2*)h->ws(WS_PARTIAL, (size_t)slots * std::max(nb, 16) * sizeof(double2)).p;
  const int steps = (M + 1) / 2;
  const double tol = 1e-6;
  const size_t total = (size_t)h->nseg * M;
  const int rb = (int)std::min<size_t>((total + 255) / 256, 4096);
  // grid of the tiled passes: their resident CTAs (set before any capture)
  int tgrid = 0, tnseg = 0;
  double2* tscratch = nullptr;
  if (tiled) {
    // one CTA per band and segment, the segments as many as the resident CTAs allow
    // (the CTAs of a segment then walk its rows across all bands together)
    const int bw = tl_band_width(h->honey_L1), thr = 2 * bw, nbands = h->honey_L1 / bw;
    const int res = pair ? (h->hop_real ? tiled_grid<false, 2>(thr) : tiled_grid<true, 2>(thr))
                         : (h->hop_real ? tiled_grid<false, 1>(thr) : tiled_grid<true, 1>(thr));
    if (nbands <= res) {
      tnseg = res / nbands;
      tgrid = nbands * tnseg;
    } else {
      tgrid = res;  // more bands than resident CTAs: equal ranges of band rows
    }
    if (tgrid > nb) tscratch = (double2*)h->ws(WS_TILE_SCRATCH, (size_t)4 * tgrid * sizeof(double2)).p;
  }
  const std::string key = key_of("momdf", {l, r, out, A[0], A[1], A[2], A[3], B[0], B[1], B[2], B[3], partial,
                                           T.d_blk.p, tscratch},
                                 {(double)kind, (double)M, (double)h->threads, (double)nb, (double)tgrid, (double)tnseg});
  run_graph(h, key, st, [&](cudaStream_t s2) {
    auto rows = [&](auto ch) {
      constexpr bool CH = decltype(ch)::value;
      switch (h->K) {
        case 2: df_rows<CH, 2>(h, T, pair, steps, l, r, A, B, 0, 0, partial, nullptr, s2); break;
        case 3: df_rows<CH, 3>(h, T, pair, steps, l, r, A, B, tgrid, tnseg, partial, tscratch, s2); break;
        case 4: df_rows<CH, 4>(h, T, pair, steps, l, r, A, B, 0, 0, partial, nullptr, s2); break;
        default: df_rows<CH, 6>(h, T, pair, steps, l, r, A, B, 0, 0, partial, nullptr, s2); break;
      }
    };
    if (h->hop_real)
      rows(std::integral_constant<bool, false>());
    else
      rows(std::integral_constant<bool, true>());
    k_reduce_dbl<<<rb, 256, 0, s2>>>(partial, M, nb, 1, (const int*)T.d_seg_blk.p, h->nseg, 1.0 + tol, (double*)out,
                                     (int*)h->d_flag.p, pair ? 2 * steps : -1);
    check_launch("k_reduce_dbl");
  });
}

// Temporal blocking of the FP32 multi-vector rows (k_cheb2_honey_wv): FP32
// handles whose rows follow the honeycomb cell layout, one segment, R = 2, 4, 8
// or 16 vectors (G = R/2 lanes per site) and a band width dividing L1, when the
// default multi-vector kernels run.  Returns log2 G, or -1 where it does not apply.
static int tiled_wv_gs(const gqt_ham* h, int R) {
  if (!h->use_tiling || h->prec != GQT_FP32_ACC64 || h->honey_L1 <= 0 || h->nseg != 1 || h->K != 3 ||
      h->honey_L2 < 2 || !(h->variant == 2 || h->variant == 3) || h->threads > 128)
    return -1;
  const int gs = R == 2 ? 0 : R == 4 ? 1 : R == 8 ? 2 : R == 16 ? 3 : -1;
  if (gs < 0 || tl_band_width_wv(h->honey_L1, 1 << gs) == 0) return -1;
  return gs;
}

static size_t tl_wv_smem(int threads, int G) { return (size_t)8 * (threads / 32) * G * sizeof(double2); }

template <bool CH, int NC>
static int tiled_wv_grid(int threads, int G) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cheb2_honey_wv<CH, NC>, threads, tl_wv_smem(threads, G)) !=
      cudaSuccess) {
    cudaGetLastError();
    n = 1;
  }
  return std::max(1, n) * sm_count();
}

// Rows of an FP32 multi-vector handle with temporal blocking: the first order and
// a last odd order by the single-order kernels, the orders between them two per
// launch.  A chain's four buffers rotate: after step j, T_j is at cur and T_{j-1}
// at prv (the caller's vector after step 1); a blocked pass writes T_{j+1} and
// T_{j+2} into two buffers that hold neither, a single order writes T_{j+1} over
// T_{j-1} when that is a buffer of the chain (same element, same thread).
template <bool CH>
static void wv_rows_tiled(gqt_ham* h, const Ell<false, CH>& H, const BlockTable& T, int R, int rs, bool pair,
                          int steps, const float2* l, const float2* r, float2* const* A, float2* const* B, int gs,
                          int tgrid, int tnseg, double2* partial, double2* tscratch, int slot_norm, cudaStream_t s2) {
  const int nb = T.nblocks;
  const Honey G = honey_of(h);
  const int Gl = 1 << gs, bw = tl_band_width_wv(G.L1, Gl), thr = 2 * bw * Gl;
  auto internal = [](float2* const* X, const float2* p) {
    for (int b = 0; b < 4; ++b)
      if (X[b] == p) return true;
    return false;
  };
  auto free_of = [](float2* const* X, const float2* c, const float2* p, float2** f, int want) {
    int n = 0;
    for (int b = 0; b < 4 && n < want; ++b)
      if (X[b] != c && X[b] != p) f[n++] = X[b];
  };
  size_t pe = prof_begin(s2);
  if (pair)
    launch_wave_pair<false, CH>(h, H, T, R, rs, l, r, (const float2*)nullptr, (const float2*)nullptr, A[0], B[0],
                                partial, 1, slot_norm, s2);
  else
    launch_wave_dbl<false, CH>(h, H, T, R, rs, r, (const float2*)nullptr, B[0], partial, 1, s2);
  check_launch(pair ? "k_cheb_pair_wv(first)" : "k_cheb_dbl_wv(first)");
  prof_end(pe, 0, s2);
  const float2 *ac = A[0], *ap = l, *bc = B[0], *bp = r;
  for (int m = 2; m <= steps;) {
    if (m + 1 <= steps) {
      float2 *fa[2] = {nullptr, nullptr}, *fb[2] = {nullptr, nullptr};
      free_of(B, bc, bp, fb, 2);
      if (pair) free_of(A, ac, ap, fa, 2);
      const bool fold = tgrid > nb;
      double2* pout = fold ? tscratch : partial + (size_t)(2 * m - 2) * nb * R;
      const int ostride = fold ? tgrid : nb, nzero = fold ? 0 : nb;
      pe = prof_begin(s2);
      if (pair)
        k_cheb2_honey_wv<CH, 2><<<tgrid, thr, tl_wv_smem(thr, Gl), s2>>>(H, G, bw, tnseg, R, gs, ac, ap, bc, bp,
                                                                        fa[0], fa[1], fb[0], fb[1], pout, ostride,
                                                                        nzero);
      else
        k_cheb2_honey_wv<CH, 1><<<tgrid, thr, tl_wv_smem(thr, Gl), s2>>>(H, G, bw, tnseg, R, gs, bc, bp, nullptr,
                                                                        nullptr, fb[0], fb[1], nullptr, nullptr,
                                                                        pout, ostride, nzero);
      check_launch("k_cheb2_honey_wv");
      if (fold) {
        k_tl_fold<<<4, 128, 0, s2>>>(tscratch, tgrid, R, partial, nb, 2 * m - 2);
        check_launch("k_tl_fold");
      }
      prof_end(pe, pair ? 12 : 13, s2);
      ap = fa[0];
      ac = fa[1];
      bp = fb[0];
      bc = fb[1];
      m += 2;
    } else {
      float2* bo = nullptr;
      float2* ao = nullptr;
      if (internal(B, bp))
        bo = const_cast<float2*>(bp);
      else
        free_of(B, bc, bp, &bo, 1);
      if (pair) {
        if (internal(A, ap))
          ao = const_cast<float2*>(ap);
        else
          free_of(A, ac, ap, &ao, 1);
      }
      pe = prof_begin(s2);
      if (pair)
        launch_wave_pair<false, CH>(h, H, T, R, rs, ac, bc, ap, bp, ao, bo, partial, m, slot_norm, s2);
      else
        launch_wave_dbl<false, CH>(h, H, T, R, rs, bc, bp, bo, partial, m, s2);
      check_launch(pair ? "k_cheb_pair_wv" : "k_cheb_dbl_wv");
      prof_end(pe, pair ? 6 : 5, s2);
      ap = ac;
      ac = ao;
      bp = bc;
      bc = bo;
      m += 1;
    }
  }
}

// Launch the moment recursion of r against l and reduce into out, layout
// [nseg][R][M].  kind 0: complex <l|T_m|r> (double2 out); kind 1: Re <l|T_m|r>
// (double out); kind 2: l = r, Re <r|T_m|r> by the doubling identities
// (ceil(M/2) recursion steps, double out).
void gqt::launch_moments(gqt_ham* h, const void* l, const void* r, int R, int M, void* out, int kind,
                         cudaStream_t st) {
  const BlockTable& T = h->table(R, moment_grid_per_sm(h, R, kind));
  const int nb = T.nblocks, rs = rshift_of(R);
  const size_t vb = h->vec_bytes(R);
  void* w1 = h->ws(WS_T1, vb).p;
  void* w2 = h->ws(WS_T2, vb).p;
  const int slots = std::max(M, 2) + 2;
  // room for the chunk/wavefront grid and for a 16-CTA cluster row
  double2* partial = (double2*)h->ws(WS_PARTIAL, (size_t)slots * std::max(nb, 16) * R * sizeof(double2)).p;
  const int slot_norm = std::max(M, 2);
  // |mu_m| <= |l||r| (1 + tol): tol 1e-6 for FP64; FP32 storage rounds the vectors, so 1e-3.
  const double tol = (h->prec == GQT_FP64) ? 1e-6 : 1e-3;
  const size_t total = (size_t)h->nseg * R * M;
  const int rb = (int)std::min<size_t>((total + 255) / 256, 4096);
  if (R == 1 && h->nseg == 1 && kind != 0 && h->use_cluster) {
    int C = 0;
    bool done = false;
    DevBuf& cseg = h->ws(WS_CLUSTER_SEG, 4 * sizeof(int));
    dispatch(h, [&](auto H) {
      using Tr = EllTraits<decltype(H)>;
      using V = typename Tr::V;
      if (kind == 2)
        done = launch_cluster_row<Tr::fp64, Tr::ch, true>(h, H, (const V*)r, (const V*)nullptr, partial, M, slot_norm,
                                                          st, &C);
      else
        done = launch_cluster_row<Tr::fp64, Tr::ch, false>(h, H, (const V*)r, (const V*)l, partial, M, slot_norm, st,
                                                           &C);
    });
    if (done) {
      const int segs[2] = {0, C};
      check_cuda(cudaMemcpyAsync(cseg.p, segs, sizeof segs, cudaMemcpyHostToDevice, st), "cluster table");
      if (kind == 2)
        k_reduce_dbl<<<rb, 256, 0, st>>>(partial, M, C, 1, (const int*)cseg.p, 1, 1.0 + tol, (double*)out,
                                         (int*)h->d_flag.p);
      else
        k_reduce<<<rb, 256, 0, st>>>(partial, M, C, 1, (const int*)cseg.p, 1, slot_norm, (1.0 + tol) * (1.0 + tol),
                                     out, 1, (int*)h->d_flag.p);
      check_launch("k_reduce(cluster)");
      return;
    }
  }
  if (df_applies(h, R, kind)) {
    launch_moments_df(h, l, r, M, out, kind, st);
    return;
  }
  const bool pair = kind == 1 && pair_applies(h, R);
  void* wa1 = pair ? h->ws(WS_PA1, vb).p : nullptr;
  void* wa2 = pair ? h->ws(WS_PA2, vb).p : nullptr;
  // temporally blocked FP32 rows: two more buffers per chain, the blocked grid
  const int tgs = (pair || kind == 2) ? tiled_wv_gs(h, R) : -1;
  void* tb[4] = {nullptr, nullptr, nullptr, nullptr};
  int tgrid = 0, tnseg = 0;
  double2* tscratch = nullptr;
  if (tgs >= 0) {
    tb[0] = h->ws(WS_TILE0, vb).p;
    tb[1] = h->ws(WS_TILE0 + 1, vb).p;
    if (pair) {
      tb[2] = h->ws(WS_TILE0 + 2, vb).p;
      tb[3] = h->ws(WS_TILE0 + 3, vb).p;
    }
    const int Gl = 1 << tgs, bw = tl_band_width_wv(h->honey_L1, Gl), thr = 2 * bw * Gl, nbands = h->honey_L1 / bw;
    const int res = pair ? (h->hop_real ? tiled_wv_grid<false, 2>(thr, Gl) : tiled_wv_grid<true, 2>(thr, Gl))
                         : (h->hop_real ? tiled_wv_grid<false, 1>(thr, Gl) : tiled_wv_grid<true, 1>(thr, Gl));
    if (nbands <= res) {
      tnseg = res / nbands;
      tgrid = nbands * tnseg;
    } else {
      tgrid = res;
    }
    if (tgrid > nb)
      tscratch = (double2*)h->ws(WS_TILE_SCRATCH, (size_t)4 * tgrid * R * sizeof(double2)).p;
  }
  const std::string key = key_of("mom", {l, r, out, w1, w2, partial, T.d_blk.p, wa1, wa2, tb[0], tb[1], tb[2], tb[3],
                                         tscratch},
                                 {(double)kind, (double)R, (double)M, (double)h->threads, (double)nb,
                                  (double)h->variant, (double)pair, (double)tgs, (double)tgrid, (double)tnseg});
  run_graph(h, key, st, [&](cudaStream_t s2) {
    dispatch(h, [&](auto H) {
      using Tr = EllTraits<decltype(H)>;
      using V = typename Tr::V;
      const V* lv = (const V*)l;
      const V* rv = (const V*)r;
      V* W1 = (V*)w1;
      V* W2 = (V*)w2;
      const int* blk = (const int*)T.d_blk.p;
      if constexpr (!Tr::fp64) {
        if (tgs >= 0) {
          float2* const A4[4] = {(float2*)wa1, (float2*)wa2, (float2*)tb[2], (float2*)tb[3]};
          float2* const B4[4] = {(float2*)w1, (float2*)w2, (float2*)tb[0], (float2*)tb[1]};
          const int steps = (M + 1) / 2;
          wv_rows_tiled<Tr::ch>(h, H, T, R, rs, pair, std::max(steps, 1), (const float2*)l, (const float2*)r, A4, B4,
                                tgs, tgrid, tnseg, partial, tscratch, 2 * steps, s2);
          return;
        }
      }
      if (pair) {
        // chain A from l in wa1/wa2, chain B from r in W1/W2; step m yields the dots of
        // moments 2m-2 and 2m-1, and step 1 the norms (slot 2 * steps)
        const int steps = (M + 1) / 2;
        V* A1 = (V*)wa1;
        V* A2 = (V*)wa2;
        for (int m = 1; m <= steps; ++m) {
          const V* am1 = (m == 1) ? lv : ((m - 1) % 2 == 1 ? A1 : A2);
          const V* bm1 = (m == 1) ? rv : ((m - 1) % 2 == 1 ? W1 : W2);
          V* aout = (m % 2 == 1) ? A1 : A2;
          V* bout = (m % 2 == 1) ? W1 : W2;
          const V* am2 = (m == 1) ? nullptr : ((m == 2) ? lv : aout);
          const V* bm2 = (m == 1) ? nullptr : ((m == 2) ? rv : bout);
          size_t pe = prof_begin(s2);
          launch_wave_pair<Tr::fp64, Tr::ch>(h, H, T, R, rs, am1, bm1, am2, bm2, aout, bout, partial, m, 2 * steps,
                                             s2);
          check_launch("k_cheb_pair");
          prof_end(pe, m == 1 ? 0 : 6, s2);
        }
        return;
      }
      if (kind == 2) {
        const int steps = (M + 1) / 2;  // step m yields moments 2m-2 and 2m-1
        for (int m = 1; m <= std::max(steps, 1); ++m) {
          const V* tm1 = (m == 1) ? rv : ((m - 1) % 2 == 1 ? W1 : W2);
          V* tout = (m % 2 == 1) ? W1 : W2;
          const V* tm2 = (m == 1) ? nullptr : ((m == 2) ? rv : tout);
          size_t pe = prof_begin(s2);
          if (!launch_wave_dbl<Tr::fp64, Tr::ch>(h, H, T, R, rs, tm1, tm2, tout, partial, m, s2))
            k_cheb_dbl<Tr::fp64, Tr::ch><<<nb, h->threads, smem_bytes(h, R, 3), s2>>>(H, blk, R, rs, tm1, tm2, tout,
                                                                                      partial, nb, m);
          check_launch("k_cheb_dbl");
          prof_end(pe, m == 1 ? 0 : 5, s2);
        }
        return;
      }
      size_t pe = prof_begin(s2);
      if (kind == 0)
        k_cheb<Tr::fp64, Tr::ch><<<nb, h->threads, smem_bytes(h, R, 3), s2>>>(H, blk, R, rs, rv, nullptr, W1, lv,
                                                                              partial, nb, 0, slot_norm, 1);
      else if (!launch_wave_re<Tr::fp64, Tr::ch>(h, H, T, R, rs, rv, (const V*)nullptr, W1, lv, partial, 0, slot_norm, 1, s2))
        k_cheb_re<Tr::fp64, Tr::ch><<<nb, h->threads, smem_bytes(h, R, 3), s2>>>(H, blk, R, rs, rv, nullptr, W1, lv,
                                                                                 partial, nb, 0, slot_norm, 1);
      check_launch("k_cheb(first)");
      prof_end(pe, 0, s2);
      for (int m = 2; m < M; ++m) {
        const V* tm1 = (m - 1) % 2 == 1 ? W1 : W2;
        V* tout = (m % 2 == 1) ? W1 : W2;
        const V* tm2 = (m == 2) ? rv : tout;
        pe = prof_begin(s2);
        if (kind == 0)
          k_cheb<Tr::fp64, Tr::ch><<<nb, h->threads, smem_bytes(h, R, 3), s2>>>(H, blk, R, rs, tm1, tm2, tout, lv,
                                                                                partial, nb, m, slot_norm, 0);
        else if (!launch_wave_re<Tr::fp64, Tr::ch>(h, H, T, R, rs, tm1, tm2, tout, lv, partial, m, slot_norm, 0, s2))
          k_cheb_re<Tr::fp64, Tr::ch><<<nb, h->threads, smem_bytes(h, R, 3), s2>>>(H, blk, R, rs, tm1, tm2, tout, lv,
                                                                                   partial, nb, m, slot_norm, 0);
        check_launch("k_cheb");
        prof_end(pe, 1, s2);
      }
    });
    if (kind == 2 || pair) {
      k_reduce_dbl<<<rb, 256, 0, s2>>>(partial, M, nb, R, (const int*)T.d_seg_blk.p, h->nseg, 1.0 + tol, (double*)out,
                                       (int*)h->d_flag.p, pair ? 2 * ((M + 1) / 2) : -1);
      check_launch("k_reduce_dbl");
    } else {
      k_reduce<<<rb, 256, 0, s2>>>(partial, M, nb, R, (const int*)T.d_seg_blk.p, h->nseg, slot_norm,
                                   (1.0 + tol) * (1.0 + tol), out, kind == 0 ? 0 : 1, (int*)h->d_flag.p);
      check_launch("k_reduce");
    }
  });
}

// ====================================================================== evolution core

// Evolution orders of FP64 handles with one vector on the FP32 pipes (pairs of
// FP32 numbers, gqt_df.cuh), when their moment rows run there too (FP64
// arithmetic mode 1): the wavefront table and neighbour counts of the pair rows.
static bool df_evo_applies(const gqt_ham* h, int R) {
  return h->prec == GQT_FP64 && h->fp64_arith == 1 && R == 1 && h->variant != 0 && h->threads <= 256 &&
         (h->K == 2 || h->K == 3 || h->K == 4 || h->K == 6) && h->d_dx.p != nullptr;
}

// An expansion coefficient as pairs (re.hi, re.lo, im.hi, im.lo).
static float4 coef_df(double2 c) {
  const float a = (float)c.x, b = (float)c.y;
  return make_float4(a, (float)(c.x - (double)a), b, (float)(c.y - (double)b));
}

template <class F>
static void df_dispatch(const gqt_ham* h, F&& f) {
  auto kk = [&](auto ch) {
    switch (h->K) {
      case 2: f(ch, std::integral_constant<int, 2>()); break;
      case 3: f(ch, std::integral_constant<int, 3>()); break;
      case 4: f(ch, std::integral_constant<int, 4>()); break;
      default: f(ch, std::integral_constant<int, 6>()); break;
    }
  };
  if (h->hop_real)
    kk(std::integral_constant<bool, false>());
  else
    kk(std::integral_constant<bool, true>());
}

static int occupancy_of(const void* f, int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 4;
  }
  return std::max(1, n);
}

template <int NSET>
static void launch_evolve_df(gqt_ham* h, void* const* psi, const std::vector<double2>& c, cudaStream_t st,
                             double* d_norms) {
  ensure_df(h, st);
  const int Np = (int)c.size();
  const size_t smem = (size_t)NSET * (h->threads / 32) * sizeof(double) + 16;
  int occ = h->blocks_per_sm;
  if (occ <= 0)
    df_dispatch(h, [&](auto ch, auto kk) {
      occ = occupancy_of((const void*)k_evolve_df<decltype(ch)::value, decltype(kk)::value, NSET, 1>, h->threads,
                         smem);
    });
  const BlockTable& T = h->table(1, occ);
  const int nb = T.nblocks;
  const size_t vb = h->vec_bytes(1);
  float4* W1[NSET];
  float4* W2[NSET];
  float4* ACC[NSET];
  for (int q = 0; q < NSET; ++q) {
    W1[q] = (float4*)h->ws(WS_E1 + 2 * q, vb).p;
    W2[q] = (float4*)h->ws(WS_E1 + 2 * q + 1, vb).p;
    ACC[q] = (float4*)h->ws(WS_ACC0 + q, vb).p;
  }
  double2* partial = (double2*)h->ws(WS_PARTIAL_EVO, (size_t)(2 * NSET) * nb * sizeof(double2)).p;
  const std::string key = key_of("evodf", {psi[0], psi[NSET - 1], W1[0], W2[0], ACC[0], partial, d_norms, T.d_blk.p},
                                 {(double)NSET, (double)Np, (double)h->threads, (double)nb}) + coef_bits(c);
  run_graph(h, key, st, [&](cudaStream_t s2) {
    df_dispatch(h, [&](auto ch, auto kk) {
      constexpr bool CH = decltype(ch)::value;
      constexpr int KK = decltype(kk)::value;
      const DfEll<CH> H = df_ell_of<CH>(h);
      const int4* tab = (const int4*)T.d_tab4.p;
      DfEvo<NSET> A;
      for (int q = 0; q < NSET; ++q) {
        A.psi[q] = (double2*)psi[q];
        A.t1[q] = nullptr;
        A.t2[q] = nullptr;
        A.out[q] = W1[q];
        A.t0[q] = W2[q];
        A.acc[q] = ACC[q];
      }
      const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
      auto orders = [&](auto uh) {
        constexpr bool UH = decltype(uh)::value && !CH;  // one common hopping: no hop array read
        k_evolve_df<CH, KK, NSET, 0, UH><<<nb, h->threads, smem, s2>>>(H, tab, A, coef_df(c[0]),
                                                                       Np > 1 ? coef_df(c[1]) : zero, partial, nb, 0);
        check_launch("k_evolve_df(0)");
        if (Np <= 2) {
          k_evolve_df<CH, KK, NSET, 3, UH><<<nb, h->threads, smem, s2>>>(H, tab, A, zero, zero, partial, nb, NSET);
          check_launch("k_evolve_df(3)");
          return;
        }
        for (int m = 2; m < Np; ++m) {
          for (int q = 0; q < NSET; ++q) {
            A.t1[q] = (m - 1) % 2 == 1 ? W1[q] : W2[q];
            A.out[q] = (m % 2 == 1) ? W1[q] : W2[q];
            A.t2[q] = A.out[q];
          }
          size_t pe = prof_begin(s2);
          if (m == Np - 1)
            k_evolve_df<CH, KK, NSET, 2, UH><<<nb, h->threads, smem, s2>>>(H, tab, A, coef_df(c[m]), zero, partial, nb,
                                                                           NSET);
          else
            k_evolve_df<CH, KK, NSET, 1, UH><<<nb, h->threads, smem, s2>>>(H, tab, A, coef_df(c[m]), zero, partial, nb,
                                                                           NSET);
          check_launch("k_evolve_df");
          prof_end(pe, 1 + NSET, s2);
        }
      };
      if (h->hop_uniform)
        orders(std::true_type());
      else
        orders(std::false_type());
    });
    k_norm_check<<<1, 256, 0, s2>>>(partial, NSET, nb, 1, (const int*)T.d_seg_blk.p, h->nseg, 1e-10, d_norms,
                                    (int*)h->d_flag.p);
    check_launch("k_norm_check");
  });
}

static void launch_msd_df(gqt_ham* h, void* p, void* px, const std::vector<double2>& c, cudaStream_t st) {
  ensure_df(h, st);
  ensure_df_x(h, st);
  const int Np = (int)c.size();
  const size_t smem = (size_t)2 * (h->threads / 32) * sizeof(double) + 16;
  int occ = h->blocks_per_sm;
  if (occ <= 0)
    df_dispatch(h, [&](auto ch, auto kk) {
      occ = occupancy_of((const void*)k_msd_evolve_df<decltype(ch)::value, decltype(kk)::value, 1>, h->threads,
                         smem);
    });
  const BlockTable& T = h->table(1, occ);
  const int nb = T.nblocks;
  const size_t vb = h->vec_bytes(1);
  float4* U1 = (float4*)h->ws(WS_E1, vb).p;
  float4* U2 = (float4*)h->ws(WS_E1 + 1, vb).p;
  float4* Z1 = (float4*)h->ws(WS_E1 + 2, vb).p;
  float4* Z2 = (float4*)h->ws(WS_E1 + 3, vb).p;
  float4* AP = (float4*)h->ws(WS_ACC0, vb).p;
  float4* AX = (float4*)h->ws(WS_ACC0 + 1, vb).p;
  double2* partial = (double2*)h->ws(WS_PARTIAL_EVO, (size_t)4 * nb * sizeof(double2)).p;
  const std::string key = key_of("msddf", {p, px, U1, Z1, AP, AX, partial, T.d_blk.p},
                                 {(double)Np, (double)h->threads, (double)nb}) + coef_bits(c);
  run_graph(h, key, st, [&](cudaStream_t s2) {
    df_dispatch(h, [&](auto ch, auto kk) {
      constexpr bool CH = decltype(ch)::value;
      constexpr int KK = decltype(kk)::value;
      const DfEll<CH> H = df_ell_of<CH>(h);
      const int4* tab = (const int4*)T.d_tab4.p;
      DfMsd B;
      B.p = (double2*)p;
      B.px = (double2*)px;
      B.u1 = B.u2 = B.z1 = B.z2 = nullptr;
      B.uo = U1;
      B.zo = Z1;
      B.u0 = U2;
      B.z0 = Z2;
      B.accp = AP;
      B.accx = AX;
      const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
      auto orders = [&](auto uh) {
        constexpr bool UH = decltype(uh)::value && !CH;  // one common hopping: no hop array read
        k_msd_evolve_df<CH, KK, 0, UH><<<nb, h->threads, smem, s2>>>(H, tab, B, coef_df(c[0]),
                                                                     Np > 1 ? coef_df(c[1]) : zero, partial, nb, 0);
        check_launch("k_msd_evolve_df(0)");
        if (Np <= 2) {
          k_msd_evolve_df<CH, KK, 3, UH><<<nb, h->threads, smem, s2>>>(H, tab, B, zero, zero, partial, nb, 2);
          check_launch("k_msd_evolve_df(3)");
          return;
        }
        for (int m = 2; m < Np; ++m) {
          B.u1 = (m - 1) % 2 == 1 ? U1 : U2;
          B.z1 = (m - 1) % 2 == 1 ? Z1 : Z2;
          B.uo = (m % 2 == 1) ? U1 : U2;
          B.zo = (m % 2 == 1) ? Z1 : Z2;
          B.u2 = B.uo;
          B.z2 = B.zo;
          size_t pe = prof_begin(s2);
          if (m == Np - 1)
            k_msd_evolve_df<CH, KK, 2, UH><<<nb, h->threads, smem, s2>>>(H, tab, B, coef_df(c[m]), zero, partial, nb,
                                                                         2);
          else
            k_msd_evolve_df<CH, KK, 1, UH><<<nb, h->threads, smem, s2>>>(H, tab, B, coef_df(c[m]), zero, partial, nb,
                                                                         2);
          check_launch("k_msd_evolve_df");
          prof_end(pe, 4, s2);
        }
      };
      if (h->hop_uniform)
        orders(std::true_type());
      else
        orders(std::false_type());
    });
    k_norm_check_msd<<<1, 256, 0, s2>>>(partial, nb, 1, (const int*)T.d_seg_blk.p, h->nseg, 1e-10,
                                        (int*)h->d_flag.p);
    check_launch("k_norm_check_msd");
  });
}

// In-place evolution of NSET vector sets (each [n][R]) by U(sign*dt) with Np
// orders.  Norms before/after are checked on the device against tol.
template <int NSET>
static void launch_evolve_sets(gqt_ham* h, void* const* psi, int R, const std::vector<double2>& c, cudaStream_t st,
                               double* d_norms /* [nseg][R][2*NSET] or null */) {
  if (df_evo_applies(h, R)) {
    launch_evolve_df<NSET>(h, psi, c, st, d_norms);
    return;
  }
  const int Np = (int)c.size();
  const BlockTable& T = h->table(R);
  const int nb = T.nblocks, rs = rshift_of(R);
  const size_t vb = h->vec_bytes(R);
  void* W1[NSET];
  void* W2[NSET];
  double2* ACC[NSET];
  for (int q = 0; q < NSET; ++q) {
    W1[q] = h->ws(WS_E1 + 2 * q, vb).p;
    W2[q] = h->ws(WS_E1 + 2 * q + 1, vb).p;
    ACC[q] = (double2*)h->ws(WS_ACC0 + q, (size_t)h->n * R * sizeof(double2)).p;
  }
  double2* partial = (double2*)h->ws(WS_PARTIAL_EVO, (size_t)(2 * NSET) * nb * R * sizeof(double2)).p;
  const std::string cbits = coef_bits(c);
  const std::string key = key_of("evo", {psi[0], psi[NSET - 1], W1[0], W2[0], ACC[0], partial, d_norms, T.d_blk.p},
                                 {(double)NSET, (double)R, (double)Np, (double)h->threads}) + cbits;
  run_graph(h, key, st, [&](cudaStream_t s2) {
    dispatch(h, [&](auto H) {
      using Tr = EllTraits<decltype(H)>;
      using V = typename Tr::V;
      EvoSets<NSET, Tr::fp64> A;
      // phase 0: m = 0, 1
      for (int q = 0; q < NSET; ++q) {
        A.t1[q] = (const V*)psi[q];
        A.t2[q] = nullptr;
        A.out[q] = (V*)W1[q];
        A.acc[q] = ACC[q];
        A.fin[q] = (V*)psi[q];
      }
      const double2 zero = make_double2(0.0, 0.0);
      k_evolve<NSET, Tr::fp64, Tr::ch><<<nb, h->threads, smem_bytes(h, R, 3), s2>>>(H, (const int*)T.d_blk.p, R, rs, A, c[0],
                                                                   Np > 1 ? c[1] : zero, 0, partial, nb, 0);
      check_launch("k_evolve(0)");
      if (Np <= 2) {
        k_evolve<NSET, Tr::fp64, Tr::ch><<<nb, h->threads, smem_bytes(h, R, 3), s2>>>(H, (const int*)T.d_blk.p, R, rs, A, zero, zero, 3,
                                                                     partial, nb, NSET);
        check_launch("k_evolve(3)");
      } else {
        for (int m = 2; m < Np; ++m) {
          for (int q = 0; q < NSET; ++q) {
            V* w1 = (V*)W1[q];
            V* w2 = (V*)W2[q];
            A.t1[q] = (m - 1) % 2 == 1 ? w1 : w2;
            V* o = (m % 2 == 1) ? w1 : w2;
            A.t2[q] = (m == 2) ? (const V*)psi[q] : o;
            A.out[q] = o;
          }
          const int phase = (m == Np - 1) ? 2 : 1;
          size_t pe = prof_begin(s2);
          k_evolve<NSET, Tr::fp64, Tr::ch><<<nb, h->threads, smem_bytes(h, R, 3), s2>>>(H, (const int*)T.d_blk.p, R, rs, A, c[m], zero,
                                                                       phase, partial, nb, NSET);
          check_launch("k_evolve");
          prof_end(pe, 1 + NSET, s2);
        }
      }
    });
    const double tol = h->prec == GQT_FP64 ? 1e-10 : 1e-5;
    k_norm_check<<<1, 256, 0, s2>>>(partial, NSET, nb, R, (const int*)T.d_seg_blk.p, h->nseg, tol, d_norms,
                                    (int*)h->d_flag.p);
    check_launch("k_norm_check");
  });
}

static void launch_msd_step(gqt_ham* h, void* p, void* px, int R, const std::vector<double2>& c, cudaStream_t st) {
  if (df_evo_applies(h, R)) {
    launch_msd_df(h, p, px, c, st);
    return;
  }
  const int Np = (int)c.size();
  const BlockTable& T = h->table(R);
  const int nb = T.nblocks, rs = rshift_of(R);
  const size_t vb = h->vec_bytes(R);
  void* U1 = h->ws(WS_E1, vb).p;
  void* U2 = h->ws(WS_E1 + 1, vb).p;
  void* Z1 = h->ws(WS_E1 + 2, vb).p;
  void* Z2 = h->ws(WS_E1 + 3, vb).p;
  double2* AP = (double2*)h->ws(WS_ACC0, (size_t)h->n * R * sizeof(double2)).p;
  double2* AX = (double2*)h->ws(WS_ACC0 + 1, (size_t)h->n * R * sizeof(double2)).p;
  double2* partial = (double2*)h->ws(WS_PARTIAL_EVO, (size_t)4 * nb * R * sizeof(double2)).p;
  const std::string cbits = coef_bits(c);
  const std::string key = key_of("msd", {p, px, U1, Z1, AP, AX, partial, T.d_blk.p},
                                 {(double)R, (double)Np, (double)h->threads}) + cbits;
  run_graph(h, key, st, [&](cudaStream_t s2) {
    dispatch(h, [&](auto H) {
      using Tr = EllTraits<decltype(H)>;
      using V = typename Tr::V;
      MsdBufs<Tr::fp64> B;
      B.u1 = (const V*)p;
      B.z1 = (const V*)px;
      B.u2 = nullptr;
      B.z2 = nullptr;
      B.uo = (V*)U1;
      B.zo = (V*)Z1;
      B.accp = AP;
      B.accx = AX;
      B.p = (V*)p;
      B.px = (V*)px;
      const double2 zero = make_double2(0.0, 0.0);
      k_msd_evolve<Tr::fp64, Tr::ch><<<nb, h->threads, smem_bytes(h, R, 3), s2>>>(H, (const int*)T.d_blk.p, R, rs, B, c[0],
                                                                 Np > 1 ? c[1] : zero, 0, partial, nb, 0);
      check_launch("k_msd_evolve(0)");
      if (Np <= 2) {
        k_msd_evolve<Tr::fp64, Tr::ch><<<nb, h->threads, smem_bytes(h, R, 3), s2>>>(H, (const int*)T.d_blk.p, R, rs, B, zero, zero, 3,
                                                                   partial, nb, 2);
        check_launch("k_msd_evolve(3)");
      } else {
        for (int m = 2; m < Np; ++m) {
          B.u1 = (m - 1) % 2 == 1 ? (const V*)U1 : (const V*)U2;
          B.z1 = (m - 1) % 2 == 1 ? (const V*)Z1 : (const V*)Z2;
          V* uo = (m % 2 == 1) ? (V*)U1 : (V*)U2;
          V* zo = (m % 2 == 1) ? (V*)Z1 : (V*)Z2;
          B.u2 = (m == 2) ? (const V*)p : uo;
          B.z2 = (m == 2) ? (const V*)px : zo;
          B.uo = uo;
          B.zo = zo;
          const int phase = (m == Np - 1) ? 2 : 1;
          size_t pe = prof_begin(s2);
          k_msd_evolve<Tr::fp64, Tr::ch><<<nb, h->threads, smem_bytes(h, R, 3), s2>>>(H, (const int*)T.d_blk.p, R, rs, B, c[m], zero,
                                                                     phase, partial, nb, 2);
          check_launch("k_msd_evolve");
          prof_end(pe, 4, s2);
        }
      }
    });
    // only |U p| vs |p| is a unitarity check; the px norm changes by construction.
    const double tol = h->prec == GQT_FP64 ? 1e-10 : 1e-5;
    k_norm_check_msd<<<1, 256, 0, s2>>>(partial, nb, R, (const int*)T.d_seg_blk.p, h->nseg, tol, (int*)h->d_flag.p);
    check_launch("k_norm_check_msd");
  });
}

void gqt::launch_velocity(gqt_ham* h, const void* x, void* y, void* ycopy, int R, cudaStream_t st) {
  const BlockTable& T = h->table(R);
  const int nb = T.nblocks, rs = rshift_of(R);
  dispatch(h, [&](auto H) {
    using Tr = EllTraits<decltype(H)>;
    using V = typename Tr::V;
    k_velocity<Tr::fp64, Tr::ch><<<nb, h->threads, smem_bytes(h, R, 3), st>>>(H, (const int*)T.d_blk.p, R, rs, 0.5 * h->dE, (const V*)x,
                                                             (V*)y, (V*)ycopy);
    check_launch("k_velocity");
  });
}

// ====================================================================== API helpers

#define API_BEGIN \
  gqt::NvtxRange nvtx_call_(__func__); \
  try {
#define API_END                                        \
  }                                                    \
  catch (const Error& e) {                             \
    set_error(e.what());                               \
    return e.code;                                     \
  }                                                    \
  catch (const std::bad_alloc&) {                      \
    set_error("host allocation failed");               \
    return GQT_ENOMEM;                                 \
  }                                                    \
  catch (const std::exception& e) {                    \
    set_error(std::string("internal error: ") + e.what()); \
    return GQT_EINVAL;                                 \
  }                                                    \
  return GQT_OK;

static void require(bool c, const std::string& msg) {
  if (!c) throw Error(GQT_EINVAL, msg);
}

static bool is_host_ptr(const void* p) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeUnregistered || a.type == cudaMemoryTypeHost;
}

static void check_common(gqt_ham* h, int R) {
  require(h != nullptr, "null handle");
  require(is_pow2_r(R), "R must be 1, 2, 4, 8, 16 or 32");
  int dev = -1;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  require(dev == h->device, "the current CUDA device is not the handle's device");
}

// Copy a device result to the caller's pointer (host or device).
static void deliver(const void* dsrc, double* dst, size_t bytes, cudaStream_t st) {
  if (is_host_ptr(dst))
    check_cuda(cudaMemcpyAsync(dst, dsrc, bytes, cudaMemcpyDeviceToHost, st), "result copy");
  else
    check_cuda(cudaMemcpyAsync(dst, dsrc, bytes, cudaMemcpyDeviceToDevice, st), "result copy");
}

// State vectors of the VAC and MSD rows may live in host memory (pinned or
// pageable): they are copied into two workspace slots of the handle before the
// call's kernels and back after them, on the call's stream.
struct StagedPair {
  void* x = nullptr;
  void* y = nullptr;
  void* hx = nullptr;
  void* hy = nullptr;
  size_t bytes = 0;
};

static StagedPair stage_in(gqt_ham* h, void* x, void* y, int R, cudaStream_t st) {
  const bool hx = is_host_ptr(x), hy = is_host_ptr(y);
  require(hx == hy, "the two state vectors must both be device memory or both host memory");
  StagedPair s;
  s.x = x;
  s.y = y;
  if (!hx) return s;
  s.bytes = h->vec_bytes(R);
  s.hx = x;
  s.hy = y;
  s.x = h->ws(WS_STAGE0, s.bytes).p;
  s.y = h->ws(WS_STAGE0 + 1, s.bytes).p;
  check_cuda(cudaMemcpyAsync(s.x, x, s.bytes, cudaMemcpyHostToDevice, st), "state upload");
  check_cuda(cudaMemcpyAsync(s.y, y, s.bytes, cudaMemcpyHostToDevice, st), "state upload");
  return s;
}

static void stage_out(const StagedPair& s, cudaStream_t st) {
  if (!s.hx) return;
  check_cuda(cudaMemcpyAsync(s.hx, s.x, s.bytes, cudaMemcpyDeviceToHost, st), "state download");
  check_cuda(cudaMemcpyAsync(s.hy, s.y, s.bytes, cudaMemcpyDeviceToHost, st), "state download");
}

static int resolve_np(gqt_ham* h, double dt, int Np) {
  require(std::isfinite(dt) && dt >= 0.0, "time step must be finite and >= 0");
  if (Np > 0) return Np;
  return np_rule_lib(h->dE * dt, 4096);
}

// ====================================================================== C ABI

extern "C" {

const char* gqt_last_error(void) { return g_last_error.c_str(); }

gqt_status gqt_profile_start(void) {
  API_BEGIN
  g_prof.on = true;
  g_prof.used = 0;
  g_prof.pairs.clear();
  API_END
}

gqt_status gqt_profile_stop(double* ms, uint64_t* launches, int ncat) {
  API_BEGIN
  require(ncat >= 0 && (ncat == 0 || (ms && launches)), "gqt_profile_stop: bad argument");
  for (int c = 0; c < ncat; ++c) {
    ms[c] = 0.0;
    launches[c] = 0;
  }
  for (auto& pr : g_prof.pairs) {
    check_cuda(cudaEventSynchronize(g_prof.pool[pr.second + 1]), "cudaEventSynchronize");
    float t = 0.f;
    check_cuda(cudaEventElapsedTime(&t, g_prof.pool[pr.second], g_prof.pool[pr.second + 1]), "cudaEventElapsedTime");
    if (pr.first < ncat) {
      ms[pr.first] += t;
      launches[pr.first] += 1;
    }
  }
  g_prof.on = false;
  g_prof.used = 0;
  g_prof.pairs.clear();
  API_END
}
uint64_t gqt_launch_count(void) { return g_launches.load(); }

void gqt_free_hamiltonian(gqt_ham* h) { delete h; }

gqt_status gqt_ham_info(const gqt_ham* h, int64_t* n, double* energy_scale, double* volume, int* nseg, int* precision,
                        int* hop_real) {
  API_BEGIN
  require(h != nullptr, "null handle");
  if (n) *n = h->n;
  if (energy_scale) *energy_scale = h->dE;
  if (volume) *volume = h->volume;
  if (nseg) *nseg = h->nseg;
  if (precision) *precision = h->prec;
  if (hop_real) *hop_real = h->hop_real ? 1 : 0;
  API_END
}

gqt_status gqt_ham_forms(const gqt_ham* h, int* flags) {
  API_BEGIN
  require(h != nullptr && flags != nullptr, "gqt_ham_forms: null argument");
  *flags = (h->honey_L1 > 0 ? GQT_FORM_HONEYCOMB : 0) | (h->hop_uniform ? GQT_FORM_UNIFORM_HOP : 0) |
           (h->row_shift > 0 ? GQT_FORM_CUBIC_SWEEP : 0);
  API_END
}

gqt_status gqt_bessel(double x, int count, double* J) {
  API_BEGIN
  require(J != nullptr && count >= 0 && std::isfinite(x) && x >= 0.0, "gqt_bessel: bad argument");
  bessel_miller(x, count, J);
  API_END
}

int gqt_np_rule(double x, int cap) {
  if (!(std::isfinite(x) && x >= 0.0) || cap <= 0) return 0;
  return np_rule_lib(x, cap);
}

gqt_status gqt_set_graphs(gqt_ham* h, int enable) {
  API_BEGIN
  require(h != nullptr, "null handle");
  h->use_graphs = enable != 0;
  API_END
}

// A setting that changes which kernels run, or their parameters, retires the
// handle's captured graphs (their launches carry the old choice).
static void drop_graphs(gqt_ham* h) {
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.second);
  h->graphs.clear();
  h->graph_data.clear();
}

gqt_status gqt_set_cluster(gqt_ham* h, int enable) {
  API_BEGIN
  require(h != nullptr, "null handle");
  h->use_cluster = enable != 0;
  drop_graphs(h);
  API_END
}

gqt_status gqt_set_vac_pair(gqt_ham* h, int enable) {
  API_BEGIN
  require(h != nullptr, "null handle");
  h->use_pair = enable != 0;
  drop_graphs(h);
  API_END
}

gqt_status gqt_set_temporal_blocking(gqt_ham* h, int enable) {
  API_BEGIN
  require(h != nullptr, "null handle");
  h->use_tiling = enable != 0;
  drop_graphs(h);
  API_END
}

gqt_status gqt_set_fp64_arith(gqt_ham* h, int mode) {
  API_BEGIN
  require(h != nullptr && (mode == 0 || mode == 1), "gqt_set_fp64_arith: mode must be 0 or 1");
  h->fp64_arith = mode;
  drop_graphs(h);
  API_END
}

gqt_status gqt_set_sweep_order(gqt_ham* h, int enable) {
  API_BEGIN
  require(h != nullptr, "null handle");
  h->use_sweep_order = enable != 0;
  drop_graphs(h);
  API_END
}

gqt_status gqt_set_variant(gqt_ham* h, int variant) {
  API_BEGIN
  require(h != nullptr && variant >= 0 && variant <= 3, "gqt_set_variant: variant must be 0, 1, 2 or 3");
  h->variant = variant;
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.second);
  h->graphs.clear();
  API_END
}

gqt_status gqt_set_launch(gqt_ham* h, int threads, int blocks_per_sm) {
  API_BEGIN
  require(h != nullptr, "null handle");
  if (threads <= 0) threads = 256;
  require(threads % 32 == 0 && threads <= 1024, "threads must be a multiple of 32, at most 1024");
  require(blocks_per_sm >= 0 && blocks_per_sm <= 32, "blocks_per_sm out of range");
  h->threads = threads;
  h->blocks_per_sm = blocks_per_sm;
  h->tables.clear();
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.second);
  h->graphs.clear();
  API_END
}

gqt_status gqt_random_phase(const gqt_ham* hc, uint64_t seed, int first_vector, int R, void* d_phi, void* stream) {
  API_BEGIN
  gqt_ham* h = const_cast<gqt_ham*>(hc);
  check_common(h, R);
  require(d_phi != nullptr && first_vector >= 0, "gqt_random_phase: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<uint64_t> keys(R);
  for (int r = 0; r < R; ++r) {
    const uint64_t stream_id = (1ull << 20) + (uint64_t)first_vector + (uint64_t)r;
    keys[r] = splitmix_key(seed, stream_id);
  }
  std::vector<double> inv(h->nseg);
  for (int s = 0; s < h->nseg; ++s) inv[s] = 1.0 / std::sqrt((double)(h->seg[s + 1] - h->seg[s]));
  DevBuf& dk = h->ws(WS_SMALL0, keys.size() * 8 + inv.size() * 8);
  check_cuda(cudaMemcpyAsync(dk.p, keys.data(), keys.size() * 8, cudaMemcpyHostToDevice, st), "keys");
  check_cuda(cudaMemcpyAsync((char*)dk.p + keys.size() * 8, inv.data(), inv.size() * 8, cudaMemcpyHostToDevice, st),
             "norms");
  const size_t total = (size_t)h->n * R;
  const int nbk = (int)std::min<size_t>((total + 255) / 256, (size_t)sm_count() * 8);
  if (h->prec == GQT_FP64)
    k_random_phase<true><<<nbk, 256, 0, st>>>((int)h->n, R, (const uint64_t*)dk.p, (const int*)h->d_site_seg.p,
                                              (const double*)((char*)dk.p + keys.size() * 8), (double2*)d_phi);
  else
    k_random_phase<false><<<nbk, 256, 0, st>>>((int)h->n, R, (const uint64_t*)dk.p, (const int*)h->d_site_seg.p,
                                               (const double*)((char*)dk.p + keys.size() * 8), (float2*)d_phi);
  check_launch("k_random_phase");
  check_cuda(cudaStreamSynchronize(st), "gqt_random_phase");
  API_END
}

gqt_status gqt_cheb_moments(gqt_ham* h, const void* d_l, const void* d_r, int R, int M, double* mu, void* stream) {
  API_BEGIN
  check_common(h, R);
  require(d_l && d_r && mu && M >= 1, "gqt_cheb_moments: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  reset_flag(h, st);
  const size_t bytes = (size_t)h->nseg * R * M * sizeof(double2);
  DevBuf& out = h->ws(WS_MU, bytes);
  launch_moments(h, d_l, d_r, R, M, out.p, 0, st);
  deliver(out.p, mu, bytes, st);
  return finish_call(h, st, "gqt_cheb_moments");
  API_END
}

gqt_status gqt_dos_moments(gqt_ham* h, const void* d_phi, int R, int M, double* mu, void* stream) {
  API_BEGIN
  check_common(h, R);
  require(d_phi && mu && M >= 1, "gqt_dos_moments: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  reset_flag(h, st);
  const size_t bytes = (size_t)h->nseg * R * M * sizeof(double);
  if (is_host_ptr(mu)) {
    DevBuf& out = h->ws(WS_MU, bytes);
    launch_moments(h, d_phi, d_phi, R, M, out.p, 2, st);
    deliver(out.p, mu, bytes, st);
  } else {
    launch_moments(h, d_phi, d_phi, R, M, mu, 2, st);
  }
  return finish_call(h, st, "gqt_dos_moments");
  API_END
}

gqt_status gqt_evolve(gqt_ham* h, void* d_psi, int R, double dt, int sign, int Np, double* norm, void* stream) {
  API_BEGIN
  check_common(h, R);
  require(d_psi && (sign == 1 || sign == -1), "gqt_evolve: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  Np = resolve_np(h, dt, Np);
  reset_flag(h, st);
  const auto c = evolve_coefs(h->dE * dt, sign, Np);
  DevBuf& dn = h->ws(WS_NORMS, (size_t)h->nseg * R * 2 * sizeof(double));
  void* sets[1] = {d_psi};
  launch_evolve_sets<1>(h, sets, R, c, st, (double*)dn.p);
  gqt_status s = GQT_OK;
  std::vector<double> hn((size_t)h->nseg * R * 2);
  check_cuda(cudaMemcpyAsync(hn.data(), dn.p, hn.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "norms");
  s = finish_call(h, st, "gqt_evolve");
  if (norm)
    for (size_t q = 0; q < (size_t)h->nseg * R; ++q) norm[q] = std::sqrt(hn[2 * q + 1]);
  return s;
  API_END
}

gqt_status gqt_commutator_evolve(gqt_ham* h, const void* d_psi, void* d_out, int R, double dt, int Np,
                                 void* stream) {
  API_BEGIN
  check_common(h, R);
  require(d_psi && d_out && d_psi != d_out, "gqt_commutator_evolve: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  Np = resolve_np(h, dt, Np);
  reset_flag(h, st);
  const auto c = evolve_coefs(h->dE * dt, +1, Np);
  // [X,U]psi = the px output of one MSD step started from (p, px) = (psi, 0).
  const size_t vb = h->vec_bytes(R);
  void* p = h->ws(WS_P, vb).p;
  check_cuda(cudaMemcpyAsync(p, d_psi, vb, cudaMemcpyDeviceToDevice, st), "copy");
  check_cuda(cudaMemsetAsync(d_out, 0, vb, st), "memset");
  launch_msd_step(h, p, d_out, R, c, st);
  return finish_call(h, st, "gqt_commutator_evolve");
  API_END
}

gqt_status gqt_apply_velocity(gqt_ham* h, const void* d_x, void* d_y, int R, void* stream) {
  API_BEGIN
  check_common(h, R);
  require(d_x && d_y && d_x != d_y, "gqt_apply_velocity: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  reset_flag(h, st);
  launch_velocity(h, d_x, d_y, nullptr, R, st);
  return finish_call(h, st, "gqt_apply_velocity");
  API_END
}

gqt_status gqt_vac_init(gqt_ham* h, const void* d_phi, void* d_a, void* d_b, int R, void* stream) {
  API_BEGIN
  check_common(h, R);
  require(d_phi && d_a && d_b && d_phi != d_b && d_a != d_b, "gqt_vac_init: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  reset_flag(h, st);
  launch_velocity(h, d_phi, d_b, d_a == d_phi ? nullptr : d_a, R, st);
  return finish_call(h, st, "gqt_vac_init");
  API_END
}

gqt_status gqt_msd_init(gqt_ham* h, const void* d_phi, void* d_p, void* d_px, int R, void* stream) {
  API_BEGIN
  check_common(h, R);
  require(d_phi && d_p && d_px && d_p != d_px, "gqt_msd_init: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t vb = h->vec_bytes(R);
  if (d_p != d_phi) check_cuda(cudaMemcpyAsync(d_p, d_phi, vb, cudaMemcpyDeviceToDevice, st), "copy");
  check_cuda(cudaMemsetAsync(d_px, 0, vb, st), "memset");
  check_cuda(cudaStreamSynchronize(st), "gqt_msd_init");
  API_END
}

gqt_status gqt_vac_moments(gqt_ham* h, void* d_a, void* d_b, int R, const double* dt, const int* Np, int Nt, int M,
                           double* mu, void* stream) {
  API_BEGIN
  check_common(h, R);
  require(d_a && d_b && d_a != d_b && dt && mu && Nt >= 0 && M >= 1, "gqt_vac_moments: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  reset_flag(h, st);
  const size_t row = (size_t)h->nseg * R * M;
  const bool host = is_host_ptr(mu);
  double* dmu = host ? (double*)h->ws(WS_MU, std::max<size_t>(1, Nt * row) * sizeof(double)).p : mu;
  void* l = h->ws(WS_L, h->vec_bytes(R)).p;
  const StagedPair sp = stage_in(h, d_a, d_b, R, st);
  void* a = sp.x;
  void* b = sp.y;
  for (int k = 0; k < Nt; ++k) {
    NvtxRange step("gqt_vac_moments time step");
    const int np = resolve_np(h, dt[k], Np ? Np[k] : 0);
    const auto c = evolve_coefs(h->dE * dt[k], -1, np);
    launch_velocity(h, a, l, nullptr, R, st);
    launch_moments(h, l, b, R, M, dmu + k * row, 1, st);
    void* sets[2] = {a, b};
    launch_evolve_sets<2>(h, sets, R, c, st, nullptr);
  }
  stage_out(sp, st);
  if (host && Nt > 0) deliver(dmu, mu, Nt * row * sizeof(double), st);
  return finish_call(h, st, "gqt_vac_moments");
  API_END
}

gqt_status gqt_msd_moments(gqt_ham* h, void* d_p, void* d_px, int R, const double* dt, const int* Np, int Nt, int M,
                           double* mu, void* stream) {
  API_BEGIN
  check_common(h, R);
  require(d_p && d_px && d_p != d_px && dt && mu && Nt >= 0 && M >= 1, "gqt_msd_moments: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  reset_flag(h, st);
  const size_t row = (size_t)h->nseg * R * M;
  const bool host = is_host_ptr(mu);
  double* dmu = host ? (double*)h->ws(WS_MU, std::max<size_t>(1, Nt * row) * sizeof(double)).p : mu;
  const StagedPair sp = stage_in(h, d_p, d_px, R, st);
  void* p = sp.x;
  void* px = sp.y;
  for (int k = 0; k < Nt; ++k) {
    NvtxRange step("gqt_msd_moments time step");
    const int np = resolve_np(h, dt[k], Np ? Np[k] : 0);
    const auto c = evolve_coefs(h->dE * dt[k], +1, np);
    launch_msd_step(h, p, px, R, c, st);
    launch_moments(h, px, px, R, M, dmu + k * row, 2, st);
  }
  stage_out(sp, st);
  if (host && Nt > 0) deliver(dmu, mu, Nt * row * sizeof(double), st);
  return finish_call(h, st, "gqt_msd_moments");
  API_END
}

gqt_status gqt_kpm_reconstruct(const double* d_mu, int rows, int M, const double* d_E, int NE, double energy_scale,
                               double n_over_omega, int kernel, double* d_out, void* stream) {
  API_BEGIN
  require(d_mu && d_E && d_out && rows >= 0 && M >= 1 && NE >= 0 && energy_scale > 0 && (kernel == 0 || kernel == 1),
          "gqt_kpm_reconstruct: bad argument");
  if (rows == 0 || NE == 0) return GQT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  double* tab = nullptr;
  check_cuda(cudaMallocAsync((void**)&tab, (size_t)M * NE * sizeof(double), st), "cudaMallocAsync");
  const size_t total = (size_t)M * NE;
  k_kpm_table<<<(int)std::min<size_t>((total + 255) / 256, 8192), 256, 0, st>>>(M, d_E, NE, energy_scale, n_over_omega,
                                                                                 kernel == 0, tab);
  check_launch("k_kpm_table");
  dim3 grid((NE + 15) / 16, (rows + 15) / 16);
  k_kpm_gemm<<<grid, 256, 0, st>>>(d_mu, rows, M, tab, NE, d_out);
  check_launch("k_kpm_gemm");
  check_cuda(cudaFreeAsync(tab, st), "cudaFreeAsync");
  check_cuda(cudaStreamSynchronize(st), "gqt_kpm_reconstruct");
  API_END
}

static gqt_status sigma_common(const double* d_in, const double* dt, int Nt, int NE, double* d_out, void* stream,
                               bool vac) {
  require(d_in && dt && d_out && Nt >= 0 && NE >= 0, "gqt_sigma: bad argument");
  if (Nt == 0 || NE == 0) return GQT_OK;
  for (int k = 0; k < Nt; ++k) require(std::isfinite(dt[k]) && dt[k] > 0, "time steps must be positive");
  cudaStream_t st = (cudaStream_t)stream;
  double* ddt = nullptr;
  check_cuda(cudaMallocAsync((void**)&ddt, Nt * sizeof(double), st), "cudaMallocAsync");
  check_cuda(cudaMemcpyAsync(ddt, dt, Nt * sizeof(double), cudaMemcpyHostToDevice, st), "dt copy");
  const int nbk = std::max(1, std::min(1024, (NE + 127) / 128));
  if (vac)
    k_sigma_vac<<<nbk, 128, 0, st>>>(d_in, ddt, Nt, NE, d_out);
  else
    k_sigma_msd<<<nbk, 128, 0, st>>>(d_in, ddt, Nt, NE, d_out);
  check_launch("k_sigma");
  check_cuda(cudaFreeAsync(ddt, st), "cudaFreeAsync");
  check_cuda(cudaStreamSynchronize(st), "gqt_sigma");
  return GQT_OK;
}

gqt_status gqt_sigma_vac(const double* d_vac, const double* dt, int Nt, int NE, double* d_sigma, void* stream) {
  API_BEGIN
  return sigma_common(d_vac, dt, Nt, NE, d_sigma, stream, true);
  API_END
}

gqt_status gqt_sigma_msd(const double* d_msd, const double* dt, int Nt, int NE, double* d_sigma, void* stream) {
  API_BEGIN
  return sigma_common(d_msd, dt, Nt, NE, d_sigma, stream, false);
  API_END
}

}  // extern "C"

// ====================================================================== adjoint (K9)

namespace {

// Adds to (gdiag, gslot) the gradient of J = Re sum_{m<P} coef_m <lam|T_m(H~)|r>
// and writes rbar = sum_m conj(coef_m) T_m lam (dJ = Re <rbar|dr>).  If lbar is
// non-null it receives sum_m coef_m T_m r (FP64).  u_m = T_m r is recomputed
// from checkpoint pairs (u_c, u_{c+1}) taken every `stride` orders.
template <class HT>
void poly_adjoint(gqt_ham* h, const HT& H, const void* r, const void* lam, const std::vector<double2>& coef,
                  int stride, void* rbar, double2* lbar, double* gdiag, double2* gslot, cudaStream_t st) {
  using Tr = EllTraits<HT>;
  using V = typename Tr::V;
  const int P = (int)coef.size();
  const BlockTable& T = h->table(1);
  const int nb = T.nblocks;
  const int* blk = (const int*)T.d_blk.p;
  const size_t vb = h->vec_bytes(1);
  const int s = std::max(2, stride);
  const int nck = (P + s - 1) / s;
  char* ck = (char*)h->ws(WS_ADJ0, (size_t)2 * nck * vb).p;
  char* seg = (char*)h->ws(WS_ADJ0 + 1, (size_t)s * vb).p;
  V* WA = (V*)h->ws(WS_ADJ0 + 2, vb).p;
  V* WB = (V*)h->ws(WS_ADJ0 + 3, vb).p;
  auto ckp = [&](int j, int q) { return (V*)(ck + ((size_t)2 * j + q) * vb); };
  const double2 z = make_double2(0.0, 0.0);
  const int thr = h->threads;
  std::vector<double> cdata(2 * coef.size());
  for (size_t q = 0; q < coef.size(); ++q) {
    cdata[2 * q] = coef[q].x;
    cdata[2 * q + 1] = coef[q].y;
  }
  const std::string key = key_of("padj", {r, lam, rbar, lbar, gdiag, gslot, ck, seg, WA, WB, blk},
                                 {(double)P, (double)s, (double)thr});
  run_graph(h, key, st, [&](cudaStream_t s2) {
    // forward pass: checkpoints (and lbar)
    check_cuda(cudaMemcpyAsync(ckp(0, 0), r, vb, cudaMemcpyDeviceToDevice, s2), "checkpoint");
    if (P > 1) {
      k_recur<Tr::fp64, Tr::ch><<<nb, thr, 0, s2>>>(H, blk, (const V*)r, nullptr, WA, lbar, coef[0], coef[1], 1);
      check_launch("k_recur(first)");
      if (1 % s == 1) check_cuda(cudaMemcpyAsync(ckp(0, 1), WA, vb, cudaMemcpyDeviceToDevice, s2), "checkpoint");
    } else if (lbar) {
      k_recur<Tr::fp64, Tr::ch><<<nb, thr, 0, s2>>>(H, blk, (const V*)r, nullptr, WA, lbar, coef[0], z, 1);
      check_launch("k_recur(first)");
    }
    const V* um2 = (const V*)r;
    V* um1 = WA;
    for (int m = 2; m < P; ++m) {
      V* out = (m == 2) ? WB : const_cast<V*>(um2);
      k_recur<Tr::fp64, Tr::ch><<<nb, thr, 0, s2>>>(H, blk, um1, um2, out, lbar, z, coef[m], 0);
      check_launch("k_recur");
      if (m % s == 0) check_cuda(cudaMemcpyAsync(ckp(m / s, 0), out, vb, cudaMemcpyDeviceToDevice, s2), "checkpoint");
      if (m % s == 1) check_cuda(cudaMemcpyAsync(ckp(m / s, 1), out, vb, cudaMemcpyDeviceToDevice, s2), "checkpoint");
      um2 = um1;
      um1 = out;
    }
    // backward pass
    check_cuda(cudaMemsetAsync(WA, 0, vb, s2), "memset");
    check_cuda(cudaMemsetAsync(WB, 0, vb, s2), "memset");
    V* X = WA;  // w_{m+1}
    V* Y = WB;  // w_{m+2} -> w_m
    for (int j = nck - 1; j >= 0; --j) {
      const int c = j * s;
      const int len = std::min(s, P - c);
      std::vector<const V*> useg(len);
      for (int q = 0; q < len; ++q) {
        if (q < 2) {
          useg[q] = ckp(j, q);
        } else {
          V* o = (V*)(seg + (size_t)q * vb);
          k_recur<Tr::fp64, Tr::ch><<<nb, thr, 0, s2>>>(H, blk, useg[q - 1], useg[q - 2], o, nullptr, z, z, 0);
          check_launch("k_recur(segment)");
          useg[q] = o;
        }
      }
      for (int m = std::min(c + len, P - 1); m >= c + 1; --m) {
        const double2 lc = make_double2(coef[m].x, -coef[m].y);
        const double f = (m == 1 ? 1.0 : 2.0) / h->dE;
        k_adj_step<Tr::fp64, Tr::ch><<<nb, thr, 0, s2>>>(H, blk, X, Y, (const V*)lam, lc, useg[m - 1 - c], f, gdiag,
                                                           gslot);
        check_launch("k_adj_step");
        std::swap(X, Y);
      }
    }
    const double2 lc0 = make_double2(coef[0].x, -coef[0].y);
    k_adj_final<Tr::fp64, Tr::ch><<<nb, thr, 0, s2>>>(H, blk, P > 1 ? X : nullptr, Y, (const V*)lam, lc0, (V*)rbar);
    check_launch("k_adj_final");
  }, &cdata);
}

}  // namespace

extern "C" gqt_status gqt_vac_loss_grad(gqt_ham* h, const void* d_phi, const double* dt, const int* Np, int Nt,
                                        int M, const double* beta, int stride, double* loss, double* d_g_onsite,
                                        double* d_g_slot, void* stream) {
  API_BEGIN
  check_common(h, 1);
  require(d_phi && dt && beta && loss && d_g_onsite && d_g_slot && Nt >= 1 && M >= 1, "gqt_vac_loss_grad: bad argument");
  require(h->nseg == 1, "gqt_vac_loss_grad: single-segment handles only");
  cudaStream_t st = (cudaStream_t)stream;
  reset_flag(h, st);
  const int64_t n = h->n;
  const int K = h->K;
  const size_t vb = h->vec_bytes(1);
  const BlockTable& T = h->table(1);
  const int nb = T.nblocks;
  const int* blk = (const int*)T.d_blk.p;
  const int thr = h->threads;
  if (stride <= 0) stride = (int)std::ceil(std::sqrt((double)M));
  std::vector<double> hbeta;
  if (!is_host_ptr(beta)) {  // device weights: one copy to the host (they become kernel arguments)
    hbeta.resize((size_t)Nt * M);
    check_cuda(cudaMemcpy(hbeta.data(), beta, hbeta.size() * sizeof(double), cudaMemcpyDeviceToHost), "beta");
    beta = hbeta.data();
  }
  char* A = (char*)h->ws(WS_ADJ0 + 4, (size_t)Nt * vb).p;
  char* B = (char*)h->ws(WS_ADJ0 + 5, (size_t)Nt * vb).p;
  double* gdiag = (double*)h->ws(WS_ADJ0 + 6, (size_t)n * sizeof(double)).p;
  double2* gslot = (double2*)h->ws(WS_ADJ0 + 7, (size_t)n * K * sizeof(double2)).p;
  void* abar = h->ws(WS_ADJ0 + 8, vb).p;
  void* bbar = h->ws(WS_ADJ0 + 9, vb).p;
  double2* LB = (double2*)h->ws(WS_ADJ0 + 10, (size_t)n * sizeof(double2)).p;
  void* tmp = h->ws(WS_ADJ0 + 11, vb).p;
  void* l = h->ws(WS_L, vb).p;
  double* dpart = (double*)h->ws(WS_ADJ0 + 12, (size_t)Nt * nb * sizeof(double)).p;  // loss partials per row
  auto Ak = [&](int k) { return (void*)(A + (size_t)k * vb); };
  auto Bk = [&](int k) { return (void*)(B + (size_t)k * vb); };
  // forward states a_k = U(-t_k) phi, b_k = U(-t_k) V phi
  launch_velocity(h, d_phi, Bk(0), Ak(0), 1, st);
  std::vector<int> nps(Nt);
  for (int k = 0; k < Nt; ++k) nps[k] = resolve_np(h, dt[k], Np ? Np[k] : 0);
  for (int k = 0; k + 1 < Nt; ++k) {
    check_cuda(cudaMemcpyAsync(Ak(k + 1), Ak(k), vb, cudaMemcpyDeviceToDevice, st), "copy");
    check_cuda(cudaMemcpyAsync(Bk(k + 1), Bk(k), vb, cudaMemcpyDeviceToDevice, st), "copy");
    void* sets[2] = {Ak(k + 1), Bk(k + 1)};
    launch_evolve_sets<2>(h, sets, 1, evolve_coefs(h->dE * dt[k], -1, nps[k]), st, nullptr);
  }
  check_cuda(cudaMemsetAsync(gdiag, 0, (size_t)n * sizeof(double), st), "memset");
  check_cuda(cudaMemsetAsync(gslot, 0, (size_t)n * K * sizeof(double2), st), "memset");
  check_cuda(cudaMemsetAsync(abar, 0, vb, st), "memset");
  check_cuda(cudaMemsetAsync(bbar, 0, vb, st), "memset");
  std::vector<double> hpart((size_t)Nt * nb);
  double total = 0.0;
  dispatch(h, [&](auto H) {
    using Tr = EllTraits<decltype(H)>;
    using V = typename Tr::V;
    for (int k = Nt - 1; k >= 0; --k) {
      if (k + 1 < Nt) {
        const auto c = evolve_coefs(h->dE * dt[k], -1, nps[k]);
        poly_adjoint(h, H, Ak(k), abar, c, std::max(2, (int)std::ceil(std::sqrt((double)c.size()))), tmp, nullptr,
                     gdiag, gslot, st);
        std::swap(abar, tmp);
        poly_adjoint(h, H, Bk(k), bbar, c, std::max(2, (int)std::ceil(std::sqrt((double)c.size()))), tmp, nullptr,
                     gdiag, gslot, st);
        std::swap(bbar, tmp);
      }
      launch_velocity(h, Ak(k), l, nullptr, 1, st);
      std::vector<double2> bc(M);
      for (int m = 0; m < M; ++m) bc[m] = make_double2(beta[(size_t)k * M + m], 0.0);
      poly_adjoint(h, H, Bk(k), l, bc, stride, tmp, LB, gdiag, gslot, st);
      k_axpy<V><<<nb, thr, 0, st>>>(blk, (V*)bbar, (const V*)tmp);
      check_launch("k_axpy");
      k_dot_re<V><<<nb, thr, 0, st>>>(blk, (const V*)l, LB, dpart + (size_t)k * nb);
      check_launch("k_dot_re");
      k_vel_adj<Tr::fp64, Tr::ch, double2><<<nb, thr, 0, st>>>(H, blk, LB, (const V*)Ak(k), gslot);
      check_launch("k_vel_adj");
      k_vel_acc<Tr::fp64, Tr::ch><<<nb, thr, 0, st>>>(H, blk, 0.5 * h->dE, LB, (V*)abar);
      check_launch("k_vel_acc");
    }
    k_vel_adj<Tr::fp64, Tr::ch, V><<<nb, thr, 0, st>>>(H, blk, (const V*)bbar, (const V*)d_phi, gslot);
    check_launch("k_vel_adj");
  });
  const size_t tot = (size_t)n * K;
  k_grad_out<<<(int)std::min<size_t>((tot + 255) / 256, 8192), 256, 0, st>>>((int)n, K, gslot, gdiag,
                                                                            (double2*)d_g_slot, d_g_onsite);
  check_launch("k_grad_out");
  check_cuda(cudaMemcpyAsync(hpart.data(), dpart, hpart.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "loss");
  check_cuda(cudaStreamSynchronize(st), "loss");
  for (int k = Nt - 1; k >= 0; --k)  // the order the rows were summed before: last row first
    for (int b = 0; b < nb; ++b) total += hpart[(size_t)k * nb + b];
  *loss = total;
  return finish_call(h, st, "gqt_vac_loss_grad");
  API_END
}

extern "C" gqt_status gqt_kpm_weights(int M, const double* d_E, int NE, const double* d_w, double energy_scale,
                                      double n_over_omega, int kernel, double* d_beta, void* stream) {
  API_BEGIN
  require(d_E && d_w && d_beta && M >= 1 && NE >= 0 && energy_scale > 0 && (kernel == 0 || kernel == 1),
          "gqt_kpm_weights: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  double* tab = nullptr;
  check_cuda(cudaMallocAsync((void**)&tab, std::max<size_t>(1, (size_t)M * NE) * sizeof(double), st),
             "cudaMallocAsync");
  const size_t total = (size_t)M * NE;
  if (total) {
    k_kpm_table<<<(int)std::min<size_t>((total + 255) / 256, 8192), 256, 0, st>>>(M, d_E, NE, energy_scale,
                                                                                   n_over_omega, kernel == 0, tab);
    check_launch("k_kpm_table");
  }
  k_kpm_weights<<<(M + 127) / 128, 128, 0, st>>>(tab, M, NE, d_w, d_beta);
  check_launch("k_kpm_weights");
  check_cuda(cudaFreeAsync(tab, st), "cudaFreeAsync");
  check_cuda(cudaStreamSynchronize(st), "gqt_kpm_weights");
  API_END
}

// Autotuner: times the fused moment kernel (Re <l|T_m|r> orders, the VAC inner
// loop) on zero-filled scratch vectors of the handle for each launch shape and
// keeps the fastest.  Candidates: threads per CTA x CTAs per SM.
extern "C" gqt_status gqt_autotune(gqt_ham* h, int R, int* threads, int* blocks_per_sm, int* variant, void* stream) {
  API_BEGIN
  check_common(h, R);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t vb = h->vec_bytes(R);
  void* x = h->ws(WS_P, vb).p;
  void* l = h->ws(WS_L, vb).p;
  check_cuda(cudaMemsetAsync(x, 0, vb, st), "memset");
  check_cuda(cudaMemsetAsync(l, 0, vb, st), "memset");
  const int cand_t[] = {128, 256, 512};
  const int cand_b[] = {0, 2, 4, 8};  // 0: each kernel's own resident-CTA count (the default)
  const int cand_v[] = {0, 1, 2, 3};
  const int M = 12;
  DevBuf scratch_mu;
  scratch_mu.ensure((size_t)h->nseg * R * M * sizeof(double));
  cudaEvent_t e0, e1;
  check_cuda(cudaEventCreate(&e0), "cudaEventCreate");
  check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
  const bool graphs = h->use_graphs;
  h->use_graphs = false;
  float best = 1e30f;
  int bt = h->threads, bb = h->blocks_per_sm, bv = h->variant;
  try {
    for (int v : cand_v)
    for (int t : cand_t)
      for (int b : cand_b) {
        if (v != 0 && t > 256) continue;
        if (v == 3 && R < 2) continue;
        h->variant = v;
        h->threads = t;
        h->blocks_per_sm = b;
        h->tables.clear();
        launch_moments(h, l, x, R, 4, scratch_mu.p, 1, st);  // warm-up (also builds the table)
        check_cuda(cudaEventRecord(e0, st), "cudaEventRecord");
        launch_moments(h, l, x, R, M, scratch_mu.p, 1, st);
        check_cuda(cudaEventRecord(e1, st), "cudaEventRecord");
        check_cuda(cudaEventSynchronize(e1), "cudaEventSynchronize");
        float ms = 0.f;
        check_cuda(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
        if (ms < best) {
          best = ms;
          bt = t;
          bb = b;
          bv = v;
        }
      }
  } catch (...) {
    h->use_graphs = graphs;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->use_graphs = graphs;
  h->threads = bt;
  h->blocks_per_sm = bb;
  h->variant = bv;
  h->tables.clear();
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.second);
  h->graphs.clear();
  reset_flag(h, st);
  check_cuda(cudaStreamSynchronize(st), "gqt_autotune");
  if (threads) *threads = bt;
  if (blocks_per_sm) *blocks_per_sm = bb;
  if (variant) *variant = bv;
  API_END
}

// Measured FP64 FMA throughput of the current GPU (GFLOP/s, an FMA = 2 flops):
// best of five launches of a kernel with 8 independent FMA chains per thread on
// every SM.  Used as the peak of the FP64 arithmetic roofline.
extern "C" gqt_status gqt_probe_fp64(double* gflops, void* stream) {
  API_BEGIN
  require(gflops != nullptr, "gqt_probe_fp64: null output");
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = sm_count() * 8, threads = 256, iters = 4096;
  DevBuf sink;
  sink.ensure((size_t)blocks * sizeof(double));
  cudaEvent_t e0, e1;
  check_cuda(cudaEventCreate(&e0), "cudaEventCreate");
  check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
  float best = 1e30f;
  for (int rep = 0; rep < 6; ++rep) {
    check_cuda(cudaEventRecord(e0, st), "cudaEventRecord");
    k_probe_dfma<<<blocks, threads, 0, st>>>((double*)sink.p, iters, 0.9999999, 1e-7);
    check_launch("k_probe_dfma");
    check_cuda(cudaEventRecord(e1, st), "cudaEventRecord");
    check_cuda(cudaEventSynchronize(e1), "cudaEventSynchronize");
    float ms = 0.f;
    check_cuda(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *gflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e9;
  API_END
}

// Moment weights of the loss L = sum_e w[e] sigma_VAC(E_e, t_K): sigma_VAC at the
// last of the K+1 rows t_0 .. t_K is the trapezoid sum sum_k c_k rho C_vv(t_k)
// (Eq. 2; c_0 = dt_0/2, c_k = (dt_{k-1} + dt_k)/2, c_K = dt_{K-1}/2), and each
// rho C_vv is linear in the moments (gqt_kpm_weights), so beta[k][n] = c_k kw[n].
extern "C" gqt_status gqt_sigma_vac_loss_weights(int M, const double* d_E, int NE, const double* d_w,
                                                 double energy_scale, double n_over_omega, int kernel,
                                                 const double* dt, int K, double* d_beta, void* stream) {
  API_BEGIN
  require(d_beta && dt && K >= 1 && M >= 1, "gqt_sigma_vac_loss_weights: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<double> c(K + 1, 0.0);
  for (int k = 0; k < K; ++k) {
    require(std::isfinite(dt[k]) && dt[k] > 0, "time steps must be positive");
    c[k] += 0.5 * dt[k];
    c[k + 1] += 0.5 * dt[k];
  }
  double* buf = nullptr;
  check_cuda(cudaMallocAsync((void**)&buf, (size_t)(M + K + 1) * sizeof(double), st), "cudaMallocAsync");
  check_cuda(cudaMemcpyAsync(buf + M, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, st), "copy");
  gqt_status s = gqt_kpm_weights(M, d_E, NE, d_w, energy_scale, n_over_omega, kernel, buf, stream);
  if (s != GQT_OK) {
    cudaFreeAsync(buf, st);
    return s;
  }
  const size_t total = (size_t)(K + 1) * M;
  k_trapezoid_outer<<<(int)std::min<size_t>((total + 255) / 256, 4096), 256, 0, st>>>(buf + M, K + 1, buf, M, d_beta);
  check_launch("k_trapezoid_outer");
  check_cuda(cudaFreeAsync(buf, st), "cudaFreeAsync");
  check_cuda(cudaStreamSynchronize(st), "gqt_sigma_vac_loss_weights");
  API_END
}

extern "C" gqt_status gqt_bond_gradients(const double* d_g_slot, long long n_slots, const long long* d_slot_a,
                                         const long long* d_slot_b, int nbonds, double* d_g_re, double* d_g_im,
                                         void* stream) {
  API_BEGIN
  require(d_g_slot && d_slot_a && d_slot_b && d_g_re && nbonds >= 0 && n_slots >= 0,
          "gqt_bond_gradients: bad argument");
  if (nbonds == 0) return GQT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  k_bond_grad<<<(int)std::min(4096, (nbonds + 255) / 256), 256, 0, st>>>((const double2*)d_g_slot, n_slots, d_slot_a,
                                                                          d_slot_b, nbonds, d_g_re, d_g_im);
  check_launch("k_bond_grad");
  API_END
}
