// gqt_internal.h -- shared declarations of the library's host translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gqt.h"

namespace gqt {

// NVTX range for the lifetime of the object: every C-ABI call and every time
// step of the VAC and MSD loops is one named range on the host timeline (seen
// by Nsight Systems and usable as an ncu --nvtx-include filter).  Header-only
// NVTX 3: without a tool attached a push/pop is a null-injection check.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct Error : std::runtime_error {
  gqt_status code;
  Error(gqt_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void set_error(const std::string& s);
// Per-kernel timing (gqt_profile_start/stop): events around a launch of family cat.
size_t prof_begin(cudaStream_t st);
void prof_end(size_t i, int cat, cudaStream_t st);
void check_cuda(cudaError_t e, const char* what);
void check_launch(const char* what);
int sm_count();

// Device allocation owned by its holder, grown on demand (contents not kept).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf();
  void ensure(size_t n);
};

// CTA -> site range table for one vector count R: CTA b owns sites
// [blk[b], blk[b+1]); the CTAs of segment s are seg_blk[s] .. seg_blk[s+1]-1.
struct BlockTable {
  int nblocks = 0;
  DevBuf d_blk, d_seg_blk;
  DevBuf d_tab4;  // int4 per CTA: segment begin, segment end, rank q in the segment's CTAs, their count G
};

enum WorkSlot {
  WS_T1 = 0,
  WS_T2,
  WS_L,
  WS_P,
  WS_PARTIAL,
  WS_PARTIAL_EVO,
  WS_MU,
  WS_NORMS,
  WS_SMALL0,
  WS_ACC0,      // +0, +1
  WS_E1 = 12,   // +0..+3 evolution Chebyshev buffers
  WS_CLUSTER_SEG = 17,
  WS_PA1 = 18,  // chain A buffers of the two-recurrence (pair) moment rows
  WS_PA2 = 19,
  WS_ADJ0 = 20,  // adjoint workspace slots start here
  WS_STAGE0 = 96,  // +0, +1: host-resident VAC/MSD state staged on the device
  WS_TILE0 = 98,   // +0..+3: the third and fourth chain buffers of the tiled rows
  WS_TILE_SCRATCH = 102  // per-CTA partial dots of a tiled grid larger than the single-order grid
};

uint64_t splitmix_mix(uint64_t z);
uint64_t splitmix_key(uint64_t seed, uint64_t stream);
void bessel_miller(double x, int count, double* J);
int np_rule_lib(double x, int cap);

}  // namespace gqt

struct gqt_ham {
  int device = 0;
  int64_t n = 0;
  int K = 0;
  gqt_precision prec = GQT_FP64;
  bool hop_real = true;
  // every ELL slot holds the same real hopping (FP64 handles; the Anderson form:
  // disorder on the sites only): its 2H~ value, used by the blocked rows
  bool hop_uniform = false;
  double hop0 = 0.0;
  double dE = 1.0;
  double volume = 0.0;
  double length_x = 0.0;
  int nseg = 1;
  std::vector<int64_t> seg;  // nseg + 1 offsets
  gqt::DevBuf d_idx, d_hop, d_diag, d_dx, d_site_seg, d_flag;
  gqt::DevBuf d_dy;     // FP64 slot-major y displacements (Hall moments), when the model defines them
  int row_shift = 0;       // blocked sweep order (built-in cubic lattices): log2 of the side, 0 = off
  bool use_sweep_order = true;
  bool has_dy = false;
  int* h_flag = nullptr;  // pinned
  int threads = 256;
  int blocks_per_sm = 0;
  int variant = 2;  // moment kernels: 0 chunk order, 1 wavefront, 2 wavefront with two elements per thread
  bool use_graphs = true;
  bool use_cluster = true;  // cluster-resident moment rows for small systems
  bool use_pair = true;     // l != r moment rows by two recurrences (two moments per step)
  int kb_mode = 0;          // Hall moment contraction: 0 FP64, 1 split TF32 on the tensor cores
  int wait_limit = 1 << 24; // polls of each bounded device wait (gqt_set_wait_limit)
  int fp64_arith = 1;       // FP64 handles' R = 1 moment rows: 0 FP64 pipe, 1 pairs of FP32 (gqt_set_fp64_arith)
  gqt::DevBuf d_hop_df, d_diag_df;  // 2H~ and 2U/dE as (hi, lo) FP32 pairs, split on first use
  bool df_ready = false;
  gqt::DevBuf d_xhop_df;  // -dx 2H~ (2[X,H~] slot values) as pairs, for the commutator orders
  bool dfx_ready = false;
  // honeycomb cell layout recognised at build (site 2(c1 + L1 c2) + s; 0 = not that
  // layout) and, per sublattice and ELL slot, the neighbour type; enables the
  // temporally blocked rows (gqt_set_temporal_blocking)
  int honey_L1 = 0, honey_L2 = 0;
  int honey_type[2][3] = {{0, 1, 2}, {0, 1, 2}};
  bool use_tiling = true;
  std::map<int, std::unique_ptr<gqt::BlockTable>> tables;
  std::vector<std::unique_ptr<gqt::DevBuf>> work;
  std::map<std::string, cudaGraphExec_t> graphs;
  std::map<std::string, std::vector<double>> graph_data;  // exact data behind hashed graph keys
  std::vector<int32_t> h_cnt, h_idx;                      // host topology (row-major), for updates
  cudaStream_t gstream = nullptr;  // capture/replay stream of the graphs
  cudaEvent_t gev[2] = {nullptr, nullptr};

  const gqt::BlockTable& table(int R, int grid_per_sm = 0);
  gqt::DevBuf& ws(int slot, size_t bytes);
  size_t vec_bytes(int R) const;
  ~gqt_ham();
};

namespace gqt {
void launch_moments(gqt_ham* h, const void* l, const void* r, int R, int M, void* out, int kind, cudaStream_t st);
void launch_velocity(gqt_ham* h, const void* x, void* y, void* ycopy, int R, cudaStream_t st);
}  // namespace gqt
