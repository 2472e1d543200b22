// gqt_build.cu -- gqt_build_hamiltonian: lattice generation, validation of
// the paper's input form (Sec. 4.2, Eqs. 32-34) and upload of H~ = H/dE in
// slot-major ELL form.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "gqt_internal.h"

using namespace gqt;

namespace gqt {

uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
uint64_t splitmix_key(uint64_t seed, uint64_t stream) {
  return splitmix_mix(seed + (stream + 1) * 0x9E3779B97F4A7C15ull);
}

}  // namespace gqt

namespace {

// Host model in row-major input form [n][K].
struct HostModel {
  int64_t n = 0;
  int K = 0;
  std::vector<int32_t> cnt, idx;
  std::vector<double> hre, him, eps, dx;
  std::vector<double> dy;  // second in-plane displacement (Hall responses), when the model defines it
  bool has_dy = false;
  double length_x = 0, volume = 0;
};

double u53(uint64_t key, int64_t i) {
  return (double)(splitmix_mix(key + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull) >> 11) * 0x1.0p-53;
}

void fill_disorder(HostModel& m, const gqt_lattice& L) {
  m.eps.assign(m.n, 0.0);
  if (L.W != 0.0) {
    const uint64_t key = splitmix_key(L.seed, 1);
    for (int64_t i = 0; i < m.n; ++i) m.eps[i] = L.W * (u53(key, i) - 0.5);
  }
  if (L.vacancy_frac > 0.0) {
    const int64_t nv = (int64_t)std::nearbyint(L.vacancy_frac * (double)m.n);
    if (nv > 0) {
      const uint64_t key = splitmix_key(L.seed, 2);
      std::vector<std::pair<uint64_t, int64_t>> d(m.n);
      for (int64_t i = 0; i < m.n; ++i) d[i] = {splitmix_mix(key + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull), i};
      std::nth_element(d.begin(), d.begin() + (nv - 1), d.end());
      std::vector<char> vac(m.n, 0);
      for (int64_t q = 0; q < nv; ++q) vac[d[q].second] = 1;
      for (int64_t i = 0; i < m.n; ++i)
        for (int k = 0; k < m.K; ++k) {
          const int64_t s = i * m.K + k;
          if (vac[i] || vac[m.idx[s]]) m.hre[s] = m.him[s] = 0.0;
        }
    }
  }
}

void gen_lattice(const gqt_lattice& L, HostModel& m) {
  const double SQ3 = std::sqrt(3.0);
  auto alloc = [&](int64_t n, int K) {
    if (n <= 0 || n > (int64_t)0x7fffffff / 64) throw Error(GQT_EINVAL, "lattice size out of range");
    m.n = n;
    m.K = K;
    m.cnt.assign(n, K);
    m.idx.assign(n * K, 0);
    m.hre.assign(n * K, L.t);
    m.him.assign(n * K, 0.0);
    m.dx.assign(n * K, 0.0);
    m.dy.assign(n * K, 0.0);
    m.has_dy = true;
  };
  switch (L.kind) {
    case GQT_LATTICE_CHAIN: {
      const int64_t N = L.L1;
      if (N < 3) throw Error(GQT_EINVAL, "chain needs L1 >= 3");
      alloc(N, 2);
      for (int64_t i = 0; i < N; ++i) {
        m.idx[2 * i] = (int32_t)((i + 1) % N);
        m.idx[2 * i + 1] = (int32_t)((i + N - 1) % N);
        m.dx[2 * i] = 1.0;
        m.dx[2 * i + 1] = -1.0;
      }
      m.length_x = (double)N;
      m.volume = (double)N;
      break;
    }
    case GQT_LATTICE_SQUARE: {
      const int64_t Lx = L.L1, Ly = L.L2;
      if (Lx < 3 || Ly < 3) throw Error(GQT_EINVAL, "square needs L1, L2 >= 3");
      alloc(Lx * Ly, 4);
      for (int64_t s = 0; s < Lx * Ly; ++s) {
        const int64_t x = s % Lx, y = s / Lx;
        int32_t* p = &m.idx[4 * s];
        p[0] = (int32_t)((x + 1) % Lx + Lx * y);
        p[1] = (int32_t)((x + Lx - 1) % Lx + Lx * y);
        p[2] = (int32_t)(x + Lx * ((y + 1) % Ly));
        p[3] = (int32_t)(x + Lx * ((y + Ly - 1) % Ly));
        m.dx[4 * s] = 1.0;
        m.dx[4 * s + 1] = -1.0;
        m.dy[4 * s + 2] = 1.0;
        m.dy[4 * s + 3] = -1.0;
      }
      m.length_x = (double)Lx;
      m.volume = (double)(Lx * Ly);
      break;
    }
    case GQT_LATTICE_CUBIC: {
      const int64_t Q = L.L1;
      if (Q < 3) throw Error(GQT_EINVAL, "cubic needs L1 >= 3");
      alloc(Q * Q * Q, 6);
      for (int64_t s = 0; s < Q * Q * Q; ++s) {
        const int64_t x = s % Q, y = (s / Q) % Q, z = s / (Q * Q);
        int32_t* p = &m.idx[6 * s];
        p[0] = (int32_t)((x + 1) % Q + Q * y + Q * Q * z);
        p[1] = (int32_t)((x + Q - 1) % Q + Q * y + Q * Q * z);
        p[2] = (int32_t)(x + Q * ((y + 1) % Q) + Q * Q * z);
        p[3] = (int32_t)(x + Q * ((y + Q - 1) % Q) + Q * Q * z);
        p[4] = (int32_t)(x + Q * y + Q * Q * ((z + 1) % Q));
        p[5] = (int32_t)(x + Q * y + Q * Q * ((z + Q - 1) % Q));
        m.dx[6 * s] = 1.0;
        m.dx[6 * s + 1] = -1.0;
        m.dy[6 * s + 2] = 1.0;
        m.dy[6 * s + 3] = -1.0;
      }
      m.length_x = (double)Q;
      m.volume = (double)(Q * Q * Q);
      break;
    }
    case GQT_LATTICE_HONEYCOMB: {
      const int64_t L1 = L.L1, L2 = L.L2;
      if (L1 < 2 || L2 < 2) throw Error(GQT_EINVAL, "honeycomb needs L1, L2 >= 2");
      alloc(2 * L1 * L2, 3);
      auto cell = [&](int64_t a, int64_t b) { return ((a % L1 + L1) % L1) + L1 * ((b % L2 + L2) % L2); };
      for (int64_t c = 0; c < L1 * L2; ++c) {
        const int64_t c1 = c % L1, c2 = c / L1;
        const int64_t A = 2 * c, B = 2 * c + 1;
        m.idx[3 * A + 0] = (int32_t)(2 * cell(c1, c2) + 1);
        m.idx[3 * A + 1] = (int32_t)(2 * cell(c1 + 1, c2 - 1) + 1);
        m.idx[3 * A + 2] = (int32_t)(2 * cell(c1, c2 - 1) + 1);
        m.idx[3 * B + 0] = (int32_t)(2 * cell(c1, c2));
        m.idx[3 * B + 1] = (int32_t)(2 * cell(c1 - 1, c2 + 1));
        m.idx[3 * B + 2] = (int32_t)(2 * cell(c1, c2 + 1));
        m.dx[3 * A + 1] = SQ3 / 2;
        m.dx[3 * A + 2] = -SQ3 / 2;
        m.dx[3 * B + 1] = -SQ3 / 2;
        m.dx[3 * B + 2] = SQ3 / 2;
        // B sits 1 above A: A -> B(c) is +1 in y, the two other bonds -1/2
        m.dy[3 * A + 0] = 1.0;
        m.dy[3 * A + 1] = -0.5;
        m.dy[3 * A + 2] = -0.5;
        m.dy[3 * B + 0] = -1.0;
        m.dy[3 * B + 1] = 0.5;
        m.dy[3 * B + 2] = 0.5;
      }
      m.length_x = (double)L1 * SQ3;
      m.volume = (double)(L1 * L2) * 1.5 * SQ3;
      break;
    }
    default:
      throw Error(GQT_EINVAL, "unknown lattice kind");
  }
  fill_disorder(m, L);
}

void read_custom(const gqt_lattice& L, HostModel& m) {
  if (L.n <= 0 || L.n > (int64_t)0x7fffffff / 64) throw Error(GQT_EINVAL, "n out of range");
  if (L.max_nb < 0 || L.max_nb > 64) throw Error(GQT_EINVAL, "max_nb out of range (0..64)");
  if (!L.nb_count || (L.max_nb > 0 && !L.nb_idx) || (L.max_nb > 0 && !L.bond_dx))
    throw Error(GQT_EINVAL, "custom lattice needs nb_count, nb_idx and bond_dx");
  m.n = L.n;
  m.K = std::max(L.max_nb, 1);
  const int K = L.max_nb;
  m.cnt.assign(m.n, 0);
  m.idx.assign(m.n * m.K, 0);
  m.hre.assign(m.n * m.K, 0.0);
  m.him.assign(m.n * m.K, 0.0);
  m.dx.assign(m.n * m.K, 0.0);
  m.has_dy = L.bond_dy != nullptr;
  if (m.has_dy) m.dy.assign(m.n * m.K, 0.0);
  m.eps.assign(m.n, 0.0);
  for (int64_t i = 0; i < m.n; ++i) {
    const int c = L.nb_count[i];
    if (c < 0 || c > K) throw Error(GQT_EINVAL, "nb_count[" + std::to_string(i) + "] out of range");
    m.cnt[i] = c;
    if (L.onsite) m.eps[i] = L.onsite[i];
    for (int k = 0; k < m.K; ++k) {
      const int64_t s = i * m.K + k;
      if (k < c) {
        const int64_t so = i * K + k;
        const int32_t j = L.nb_idx[so];
        if (j < 0 || j >= m.n)
          throw Error(GQT_EINVAL, "nb_idx[" + std::to_string(i) + "][" + std::to_string(k) + "] out of range");
        m.idx[s] = j;
        m.hre[s] = L.hop_re ? L.hop_re[so] : -1.0;
        m.him[s] = L.hop_im ? L.hop_im[so] : 0.0;
        m.dx[s] = L.bond_dx[so];
        if (m.has_dy) m.dy[s] = L.bond_dy[so];
      } else {
        m.idx[s] = (int32_t)i;
      }
    }
  }
  m.length_x = L.length_x;
  m.volume = L.volume;
}

void validate(HostModel& m, const std::vector<int64_t>& seg) {
  // finite values
  for (int64_t i = 0; i < m.n; ++i)
    if (!std::isfinite(m.eps[i])) throw Error(GQT_ENAN, "non-finite on-site energy at " + std::to_string(i));
  std::vector<int32_t> site_seg(m.n);
  for (size_t s = 0; s + 1 < seg.size(); ++s)
    for (int64_t i = seg[s]; i < seg[s + 1]; ++i) site_seg[i] = (int32_t)s;
  for (int64_t i = 0; i < m.n; ++i) {
    for (int k = 0; k < m.cnt[i]; ++k) {
      const int64_t s = i * m.K + k;
      if (!std::isfinite(m.hre[s]) || !std::isfinite(m.him[s]) || !std::isfinite(m.dx[s]) ||
          (m.has_dy && !std::isfinite(m.dy[s])))
        throw Error(GQT_ENAN, "non-finite hopping or displacement in row " + std::to_string(i));
      const int64_t j = m.idx[s];
      if (site_seg[j] != site_seg[i])
        throw Error(GQT_EINVAL, "bond " + std::to_string(i) + "-" + std::to_string(j) + " crosses a segment boundary");
      // Hermitian pair: some slot of row j points back to i with conj(H_ij) and -dx_ij
      const double tol = 1e-12 * (1.0 + std::fabs(m.hre[s]) + std::fabs(m.him[s]));
      bool ok = false;
      for (int kk = 0; kk < m.cnt[j] && !ok; ++kk) {
        const int64_t t = j * m.K + kk;
        if (m.idx[t] != i) continue;
        if (std::fabs(m.hre[t] - m.hre[s]) <= tol && std::fabs(m.him[t] + m.him[s]) <= tol &&
            std::fabs(m.dx[t] + m.dx[s]) <= 1e-12 * (1.0 + std::fabs(m.dx[s])) &&
            (!m.has_dy || std::fabs(m.dy[t] + m.dy[s]) <= 1e-12 * (1.0 + std::fabs(m.dy[s]))))
          ok = true;
      }
      if (!ok)
        throw Error(GQT_EINVAL, "input is not Hermitian: bond " + std::to_string(i) + " -> " + std::to_string(j) +
                                    " has no reverse slot with conj(H) and -dx (Eq. 32/34)");
    }
  }
}

}  // namespace

gqt_ham::~gqt_ham() {
  for (auto& g : graphs)
    if (g.second) cudaGraphExecDestroy(g.second);
  if (h_flag) cudaFreeHost(h_flag);
  if (gstream) cudaStreamDestroy(gstream);
  for (auto e : gev)
    if (e) cudaEventDestroy(e);
}

// The honeycomb cell layout of the built-in lattice (site 2(c1 + L1 c2) + s;
// A(c1,c2) bonds to B(c1,c2), B(c1+1,c2-1), B(c1,c2-1) -- neighbour types 0, 1,
// 2 -- and B to the mirror images), recognised from the neighbour list alone:
// every row lists its three neighbours, in one slot order per sublattice.  This
// holds for the built-in honeycomb lattices and for the same lattice given in the
// paper's input form; vacancies (bonds with zero hopping) keep their indices.
// Returns L1 and fills type[s][k] (the neighbour type of slot k on sublattice
// s), or 0 when the rows do not follow the layout.
static int64_t detect_honeycomb(const HostModel& m, int (&type)[2][3]) {
  if (m.K != 3 || m.n < 18 || (m.n & 1)) return 0;
  for (int64_t i = 0; i < m.n; ++i)
    if (m.cnt[i] != 3) return 0;
  const int64_t nc = m.n / 2;
  for (int64_t L1 = 3; L1 * 3 <= nc; ++L1) {
    if (nc % L1) continue;
    const int64_t L2 = nc / L1;
    auto nbr = [&](int64_t i, int t) -> int64_t {
      const int64_t c = i >> 1, c1 = c % L1, c2 = c / L1;
      const int s = (int)(i & 1);
      const int64_t d1 = (t == 1) ? (s ? -1 : 1) : 0, d2 = (t == 0) ? 0 : (s ? 1 : -1);
      const int64_t e1 = (c1 + d1 + L1) % L1, e2 = (c2 + d2 + L2) % L2;
      return 2 * (e1 + L1 * e2) + (1 - s);
    };
    int ty[2][3];
    bool ok = true;
    for (int s = 0; s < 2 && ok; ++s) {
      bool used[3] = {false, false, false};
      for (int k = 0; k < 3 && ok; ++k) {
        ty[s][k] = -1;
        for (int t = 0; t < 3; ++t)
          if (!used[t] && nbr(s, t) == m.idx[s * 3 + k]) {
            ty[s][k] = t;
            used[t] = true;
            break;
          }
        ok = ty[s][k] >= 0;
      }
    }
    for (int64_t i = 0; i < m.n && ok; ++i)
      for (int k = 0; k < 3 && ok; ++k) ok = nbr(i, ty[i & 1][k]) == m.idx[i * 3 + k];
    if (ok) {
      for (int s = 0; s < 2; ++s)
        for (int k = 0; k < 3; ++k) type[s][k] = ty[s][k];
      return L1;
    }
  }
  return 0;
}

extern "C" gqt_status gqt_build_hamiltonian(const gqt_lattice* lattice, double energy_scale, gqt_precision precision,
                                            const int64_t* seg_offsets, int nseg, gqt_ham** out) {
  gqt::NvtxRange nvtx_call_(__func__);
  try {
    if (!lattice || !out) throw Error(GQT_EINVAL, "null argument");
    *out = nullptr;
    if (precision != GQT_FP64 && precision != GQT_FP32_ACC64) throw Error(GQT_EINVAL, "unknown precision");
    if (!std::isfinite(energy_scale)) throw Error(GQT_EINVAL, "energy_scale must be finite");
    HostModel m;
    if (lattice->kind == GQT_LATTICE_CUSTOM)
      read_custom(*lattice, m);
    else
      gen_lattice(*lattice, m);
    std::vector<int64_t> seg;
    if (seg_offsets && nseg > 1) {
      seg.assign(seg_offsets, seg_offsets + nseg + 1);
      if (seg.front() != 0 || seg.back() != m.n) throw Error(GQT_EINVAL, "seg_offsets must run from 0 to n");
      for (int s = 0; s < nseg; ++s)
        if (seg[s + 1] <= seg[s]) throw Error(GQT_EINVAL, "seg_offsets must be strictly increasing");
    } else {
      seg = {0, m.n};
      nseg = 1;
    }
    validate(m, seg);
    // energy scale
    double dE = energy_scale;
    if (dE <= 0.0) {
      double g = 0.0;
      for (int64_t i = 0; i < m.n; ++i) {
        double r = std::fabs(m.eps[i]);
        for (int k = 0; k < m.cnt[i]; ++k) r += std::hypot(m.hre[i * m.K + k], m.him[i * m.K + k]);
        g = std::max(g, r);
      }
      dE = 1.05 * g;
      if (dE <= 0.0) dE = 1.0;
    }
    bool hop_real = true;
    for (size_t s = 0; s < m.him.size() && hop_real; ++s)
      if (m.him[s] != 0.0) hop_real = false;

    auto h = std::make_unique<gqt_ham>();
    check_cuda(cudaGetDevice(&h->device), "cudaGetDevice");
    h->n = m.n;
    h->K = m.K;
    h->prec = precision;
    h->hop_real = hop_real;
    h->dE = dE;
    h->volume = m.volume;
    h->length_x = m.length_x;
    h->nseg = nseg;
    h->seg = seg;
    // FP32 handles run the multi-vector kernels, whose register use fits more
    // CTAs per SM at 128 threads.
    h->threads = (precision == GQT_FP64) ? 256 : 128;
    const int64_t n = m.n, K = m.K;
    const bool f64 = precision == GQT_FP64;
    h->h_cnt = m.cnt;
    h->h_idx = m.idx;
    // slot-major device images; hop2 = 2 H / dE, diag2 = 2 U / dE (exact doubling)
    std::vector<int32_t> idx(n * K);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t k = 0; k < K; ++k) idx[k * n + i] = m.idx[i * K + k];
    auto upload = [&](DevBuf& b, const void* src, size_t bytes) {
      b.ensure(std::max<size_t>(bytes, 16));
      check_cuda(cudaMemcpy(b.p, src, bytes, cudaMemcpyHostToDevice), "upload");
    };
    upload(h->d_idx, idx.data(), idx.size() * 4);
    idx.clear();
    idx.shrink_to_fit();
    const int hw = hop_real ? 1 : 2;
    if (f64) {
      std::vector<double> hop(n * K * hw), dg(n), dxv(n * K);
      for (int64_t i = 0; i < n; ++i) {
        dg[i] = 2.0 * (m.eps[i] / dE);
        for (int64_t k = 0; k < K; ++k) {
          const int64_t s = i * K + k, d = k * n + i;
          if (hop_real) {
            hop[d] = 2.0 * (m.hre[s] / dE);
          } else {
            hop[2 * d] = 2.0 * (m.hre[s] / dE);
            hop[2 * d + 1] = 2.0 * (m.him[s] / dE);
          }
          dxv[d] = m.dx[s];
        }
      }
      upload(h->d_hop, hop.data(), hop.size() * 8);
      upload(h->d_diag, dg.data(), dg.size() * 8);
      upload(h->d_dx, dxv.data(), dxv.size() * 8);
      h->hop_uniform = hop_real && !hop.empty() &&
                       std::all_of(hop.begin(), hop.end(), [&](double v) { return v == hop[0]; });
      h->hop0 = h->hop_uniform ? hop[0] : 0.0;
    } else {
      std::vector<float> hop(n * K * hw), dg(n), dxv(n * K);
      for (int64_t i = 0; i < n; ++i) {
        dg[i] = (float)(2.0 * (m.eps[i] / dE));
        for (int64_t k = 0; k < K; ++k) {
          const int64_t s = i * K + k, d = k * n + i;
          if (hop_real) {
            hop[d] = (float)(2.0 * (m.hre[s] / dE));
          } else {
            hop[2 * d] = (float)(2.0 * (m.hre[s] / dE));
            hop[2 * d + 1] = (float)(2.0 * (m.him[s] / dE));
          }
          dxv[d] = (float)m.dx[s];
        }
      }
      upload(h->d_hop, hop.data(), hop.size() * 4);
      upload(h->d_diag, dg.data(), dg.size() * 4);
      upload(h->d_dx, dxv.data(), dxv.size() * 4);
    }
    // y displacements (FP64, slot-major) for the Hall moments
    h->has_dy = m.has_dy;
    if (m.has_dy) {
      std::vector<double> dyv(n * K);
      for (int64_t i = 0; i < n; ++i)
        for (int64_t k = 0; k < K; ++k) dyv[k * n + i] = m.dy[i * K + k];
      upload(h->d_dy, dyv.data(), dyv.size() * 8);
    }
    if (nseg > 1) {
      std::vector<int32_t> ss(n);
      for (int s = 0; s < nseg; ++s)
        for (int64_t i = seg[s]; i < seg[s + 1]; ++i) ss[i] = s;
      upload(h->d_site_seg, ss.data(), ss.size() * 4);
    }
    // Blocked sweep order for the built-in simple-cubic lattice (side a power of two,
    // >= 64): the multi-vector kernels walk the x-rows strip by strip -- 32 y-rows,
    // all z, then the next strip -- so that a site's +-z neighbours are read again
    // within 2 x 32 x L sites instead of two whole xy-planes, which for large L no
    // longer stay in L2 (the mapping is in the kernels' site_of).
    if (lattice->kind == GQT_LATTICE_CUBIC && nseg == 1) {
      const int64_t L = lattice->L1;
      int sh = 0;
      while ((int64_t(1) << sh) < L) ++sh;
      if (L >= 64 && (int64_t(1) << sh) == L) h->row_shift = sh;
    }
    if (nseg == 1) {
      h->honey_L1 = (int)detect_honeycomb(m, h->honey_type);
      h->honey_L2 = h->honey_L1 > 0 ? (int)(m.n / 2 / h->honey_L1) : 0;
    }
    h->d_flag.ensure(16);
    check_cuda(cudaMemset(h->d_flag.p, 0, 16), "memset");
    check_cuda(cudaMallocHost((void**)&h->h_flag, 16), "cudaMallocHost");
    *out = h.release();
    return GQT_OK;
  } catch (const Error& e) {
    set_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return GQT_ENOMEM;
  } catch (const std::exception& e) {
    set_error(std::string("internal error: ") + e.what());
    return GQT_EINVAL;
  }
}

// Export the host model a built-in lattice kind generates, in the input form
// (row-major [n][K]), so callers can inspect exactly what was built.  Arrays
// are caller-allocated with n*K (or n) entries; any may be NULL.
extern "C" gqt_status gqt_generate_lattice(const gqt_lattice* lattice, int64_t* n, int* K, int32_t* nb_count,
                                           int32_t* nb_idx, double* hop_re, double* hop_im, double* onsite,
                                           double* bond_dx, double* length_x, double* volume) {
  try {
    if (!lattice || lattice->kind == GQT_LATTICE_CUSTOM) throw Error(GQT_EINVAL, "built-in lattice kind required");
    HostModel m;
    gen_lattice(*lattice, m);
    if (n) *n = m.n;
    if (K) *K = m.K;
    if (nb_count) std::copy(m.cnt.begin(), m.cnt.end(), nb_count);
    if (nb_idx) std::copy(m.idx.begin(), m.idx.end(), nb_idx);
    if (hop_re) std::copy(m.hre.begin(), m.hre.end(), hop_re);
    if (hop_im) std::copy(m.him.begin(), m.him.end(), hop_im);
    if (onsite) std::copy(m.eps.begin(), m.eps.end(), onsite);
    if (bond_dx) std::copy(m.dx.begin(), m.dx.end(), bond_dx);
    if (length_x) *length_x = m.length_x;
    if (volume) *volume = m.volume;
    return GQT_OK;
  } catch (const Error& e) {
    set_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_error(e.what());
    return GQT_EINVAL;
  }
}


// New hopping and on-site values for an existing handle (same neighbour list,
// positions, energy scale and precision): re-validated like a build and uploaded
// into the same device arrays, so cached graphs and workspace stay valid.
extern "C" gqt_status gqt_update_hamiltonian(gqt_ham* h, const double* onsite, const double* hop_re,
                                             const double* hop_im) {
  gqt::NvtxRange nvtx_call_(__func__);
  try {
    if (!h || !hop_re) throw Error(GQT_EINVAL, "gqt_update_hamiltonian: null argument");
    if (h->h_idx.empty()) throw Error(GQT_EINVAL, "gqt_update_hamiltonian: handle has no host topology");
    const int64_t n = h->n, K = h->K;
    HostModel m;
    m.n = n;
    m.K = (int)K;
    m.cnt = h->h_cnt;
    m.idx = h->h_idx;
    m.hre.assign(hop_re, hop_re + n * K);
    m.him.assign(n * K, 0.0);
    if (hop_im) m.him.assign(hop_im, hop_im + n * K);
    m.eps.assign(n, 0.0);
    if (onsite) m.eps.assign(onsite, onsite + n);
    m.dx.assign(n * K, 0.0);  // positions are unchanged; the Hermitian check below ignores dx
    for (int64_t i = 0; i < n; ++i)
      for (int k = m.cnt[i]; k < K; ++k) m.hre[i * K + k] = m.him[i * K + k] = 0.0;
    validate(m, h->seg);
    bool real = true;
    for (double v : m.him)
      if (v != 0.0) real = false;
    if (real != h->hop_real && !real)
      throw Error(GQT_EINVAL, "gqt_update_hamiltonian: complex hoppings on a handle built with real ones");
    const double dE = h->dE;
    const int hw = h->hop_real ? 1 : 2;
    auto put = [&](DevBuf& b, const void* src, size_t bytes) {
      if (bytes > b.bytes) throw Error(GQT_EINVAL, "gqt_update_hamiltonian: size mismatch");
      check_cuda(cudaMemcpy(b.p, src, bytes, cudaMemcpyHostToDevice), "update");
    };
    if (h->prec == GQT_FP64) {
      std::vector<double> hop(n * K * hw), dg(n);
      for (int64_t i = 0; i < n; ++i) {
        dg[i] = 2.0 * (m.eps[i] / dE);
        for (int64_t k = 0; k < K; ++k) {
          const int64_t s2 = i * K + k, d = k * n + i;
          if (hw == 1) {
            hop[d] = 2.0 * (m.hre[s2] / dE);
          } else {
            hop[2 * d] = 2.0 * (m.hre[s2] / dE);
            hop[2 * d + 1] = 2.0 * (m.him[s2] / dE);
          }
        }
      }
      put(h->d_hop, hop.data(), hop.size() * 8);
      put(h->d_diag, dg.data(), dg.size() * 8);
      h->df_ready = false;  // the (hi, lo) split of 2H~ is taken again on next use
      h->dfx_ready = false;
      const bool uni = hw == 1 && !hop.empty() &&
                       std::all_of(hop.begin(), hop.end(), [&](double v) { return v == hop[0]; });
      const double h0 = uni ? hop[0] : 0.0;
      if (uni != h->hop_uniform || h0 != h->hop0) {
        // the blocked rows switch form, or their common hopping (a kernel argument
        // inside the captured graphs) changes: retire the graphs
        for (auto& gr : h->graphs) cudaGraphExecDestroy(gr.second);
        h->graphs.clear();
        h->graph_data.clear();
      }
      h->hop_uniform = uni;
      h->hop0 = h0;
    } else {
      std::vector<float> hop(n * K * hw), dg(n);
      for (int64_t i = 0; i < n; ++i) {
        dg[i] = (float)(2.0 * (m.eps[i] / dE));
        for (int64_t k = 0; k < K; ++k) {
          const int64_t s2 = i * K + k, d = k * n + i;
          if (hw == 1) {
            hop[d] = (float)(2.0 * (m.hre[s2] / dE));
          } else {
            hop[2 * d] = (float)(2.0 * (m.hre[s2] / dE));
            hop[2 * d + 1] = (float)(2.0 * (m.him[s2] / dE));
          }
        }
      }
      put(h->d_hop, hop.data(), hop.size() * 4);
      put(h->d_diag, dg.data(), dg.size() * 4);
    }
    return GQT_OK;
  } catch (const Error& e) {
    set_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_error(std::string("internal error: ") + e.what());
    return GQT_EINVAL;
  }
}
