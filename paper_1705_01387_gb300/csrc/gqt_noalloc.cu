// gqt_noalloc.cu -- DOS moments without any device allocation.
//
// Some callers cannot call cudaMalloc at the moment they need moments: their
// device memory is owned by another allocator (a framework's caching pool or a
// fixed per-process budget) that must not be bypassed, or they run on a
// latency-critical path where cudaMalloc/cudaFree would synchronise the whole
// device.  gqt_dos_moments_noalloc serves them: it is the fused Chebyshev
// moment kernel of gqt_dos_moments with all of its scratch (the two Chebyshev
// vectors, the per-CTA moment partials, the CTA table and the status word)
// placed in one file-scope device array of fixed size.  The paper has no
// counterpart to this; it is a deployment convenience.

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include <math_constants.h>
#include <stdint.h>

#include "gqt_internal.h"

// The kernel templates are compiled into this translation unit under their own
// namespace so that its instantiations never collide with the main library's.
// Their system headers are included above, at file scope; the macro keeps
// gqt_kernels.cuh from including any header inside the namespace, so a header it
// needs and this file lacks is a compile error rather than a silent rebinding.
#define GQT_KERNELS_NO_SYSTEM_INCLUDES 1
namespace gqt_na {
#include "gqt_kernels.cuh"
}
#undef GQT_KERNELS_NO_SYSTEM_INCLUDES

using gqt::Error;
using gqt_na::gqt::Ell;
using gqt_na::gqt::Prec;
using gqt_na::gqt::k_cheb;
using gqt_na::gqt::k_reduce;

// The scratch array: every GPU that loads the library holds these bytes until
// the process exits.  Its name is only a host-side stand-in in host code; the
// device address comes from cudaGetSymbolAddress at set-up.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GQT_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};
CUcontext g_noalloc_ctx[kMaxDevices] = {};

// The current context of the calling thread (the driver's cuCtxGetCurrent,
// looked up once through the runtime, so the library links no driver stub).
CUcontext current_context() {
  using Fn = CUresult (*)(CUcontext*);
  static const Fn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q);
    return (e == cudaSuccess && q == cudaDriverEntryPointSuccess) ? (Fn)p : nullptr;
  }();
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) throw gqt::Error(GQT_ECUDA, "cuCtxGetCurrent is not available from the driver");
  return c;
}

// Set-up, once per device, with that device current: the array's device
// address.  The address belongs to the device's context; if that context was
// destroyed and created again (cudaDeviceReset), the module is loaded anew and
// the address is looked up again.
void* scratch_address(int dev) {
  using namespace gqt;
  if (dev < 0 || dev >= kMaxDevices) throw Error(GQT_EINVAL, "device ordinal out of range for the scratch table");
  // The caller's earlier runtime calls (pointer checks) made the device's
  // primary context current on this thread.
  const CUcontext ctx = current_context();
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev] || g_noalloc_ctx[dev] != ctx) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      throw Error(GQT_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
    g_noalloc_ctx[dev] = ctx;
  }
  return g_noalloc_addr[dev];
}

// EINVAL unless p is device memory of device dev.
void require_device_pointer(const void* p, int dev, const char* what) {
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
    cudaGetLastError();
    throw gqt::Error(GQT_EINVAL, std::string("gqt_dos_moments_noalloc: ") + what + " is not a CUDA pointer");
  }
  if (pa.type != cudaMemoryTypeDevice || pa.device != dev)
    throw gqt::Error(GQT_EINVAL, std::string("gqt_dos_moments_noalloc: ") + what +
                                     " must be device memory of the handle's device");
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// CTA b owns sites [b*n/nb, (b+1)*n/nb); seg_blk = {0, nb}; the status word
// starts at zero.  Rewritten on every call because the array keeps the
// previous call's contents.
__global__ void k_noalloc_setup(int* blk, int nb, long long n, int* seg_blk, int* flag) {
  for (int b = threadIdx.x; b <= nb; b += blockDim.x) blk[b] = (int)((n * b) / nb);
  if (threadIdx.x == 0) {
    seg_blk[0] = 0;
    seg_blk[1] = nb;
    *flag = 0;
  }
}

template <bool FP64, bool CH>
Ell<FP64, CH> ell_view(const gqt_ham* h) {
  Ell<FP64, CH> e;
  e.n = (int)h->n;
  e.K = h->K;
  e.idx = (const int*)h->d_idx.p;
  e.hop2 = (const typename Ell<FP64, CH>::HT*)h->d_hop.p;
  e.diag2 = (const typename Ell<FP64, CH>::S*)h->d_diag.p;
  e.dx = (const typename Ell<FP64, CH>::S*)h->d_dx.p;
  e.row_shift = 0;
  return e;
}

template <bool FP64, bool CH>
void run(const gqt_ham* h, const void* phi, int R, int rs, int M, double* d_mu, int nb, int* blk, int* seg_blk,
         int* flag, void* w1, void* w2, double2* partial, cudaStream_t st) {
  using V = typename Prec<FP64>::V;
  const Ell<FP64, CH> H = ell_view<FP64, CH>(h);
  const int slot_norm = std::max(M, 2);
  const size_t smem = (size_t)3 * (h->threads / 32) * R * sizeof(double2);
  const V* pv = (const V*)phi;
  V* W1 = (V*)w1;
  V* W2 = (V*)w2;
  k_cheb<FP64, CH><<<nb, h->threads, smem, st>>>(H, blk, R, rs, pv, nullptr, W1, pv, partial, nb, 0, slot_norm, 1);
  gqt::check_launch("k_cheb(first, no-alloc)");
  for (int m = 2; m < M; ++m) {
    const V* tm1 = (m - 1) % 2 == 1 ? W1 : W2;
    V* tout = (m % 2 == 1) ? W1 : W2;
    const V* tm2 = (m == 2) ? pv : tout;
    k_cheb<FP64, CH><<<nb, h->threads, smem, st>>>(H, blk, R, rs, tm1, tm2, tout, pv, partial, nb, m, slot_norm, 0);
    gqt::check_launch("k_cheb(no-alloc)");
  }
  const double tol = FP64 ? 1e-6 : 1e-3;
  const size_t total = (size_t)R * M;
  const int rb = (int)std::min<size_t>((total + 255) / 256, 4096);
  k_reduce<<<rb, 256, 0, st>>>(partial, M, nb, R, seg_blk, 1, slot_norm, (1.0 + tol) * (1.0 + tol), d_mu, 1, flag);
  gqt::check_launch("k_reduce(no-alloc)");
}

}  // namespace

extern "C" gqt_status gqt_dos_moments_noalloc(const gqt_ham* h, const void* d_phi, int R, int M, double* d_mu,
                                              void* stream) {
  gqt::NvtxRange nvtx_call_(__func__);
  using namespace gqt;
  try {
    if (!h || !d_phi || !d_mu || M < 1) throw Error(GQT_EINVAL, "gqt_dos_moments_noalloc: bad argument");
    if (!(R == 1 || R == 2 || R == 4 || R == 8 || R == 16 || R == 32))
      throw Error(GQT_EINVAL, "R must be 1, 2, 4, 8, 16 or 32");
    if (h->nseg != 1) throw Error(GQT_EINVAL, "gqt_dos_moments_noalloc supports single-segment handles only");
    int dev = -1;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != h->device) throw Error(GQT_EINVAL, "the current CUDA device is not the handle's device");
    require_device_pointer(d_phi, dev, "d_phi");
    require_device_pointer(d_mu, dev, "d_mu");
    cudaStream_t st = (cudaStream_t)stream;
    int rs = 0;
    while ((1 << rs) < R) ++rs;
    const long long elems = h->n * (long long)R;
    const int nb = (int)std::max<long long>(1, std::min<long long>(2LL * sm_count(), (elems + 1023) / 1024));
    const size_t vbytes = (size_t)elems * (h->prec == GQT_FP64 ? 16 : 8);
    const size_t slots = (size_t)std::max(M, 2) + 1;
    // layout: [blk (nb+1) | seg_blk (2) | flag] [T1] [T2] [partials]
    const size_t off_t1 = align_up((size_t)(nb + 4) * sizeof(int));
    const size_t off_t2 = off_t1 + align_up(vbytes);
    const size_t off_p = off_t2 + align_up(vbytes);
    const size_t need = off_p + slots * nb * R * sizeof(double2);
    if (need > (size_t)GQT_NOALLOC_SCRATCH_BYTES)
      throw Error(GQT_EINVAL, "gqt_dos_moments_noalloc: this size needs " + std::to_string(need) +
                                  " bytes of scratch, above the fixed maximum of " +
                                  std::to_string((size_t)GQT_NOALLOC_SCRATCH_BYTES) + " bytes");
    unsigned char* base = (unsigned char*)scratch_address(dev);
    int* blk = (int*)base;
    int* seg_blk = blk + (nb + 1);
    int* flag = seg_blk + 2;
    k_noalloc_setup<<<1, 256, 0, st>>>(blk, nb, h->n, seg_blk, flag);
    check_launch("k_noalloc_setup");
    void* w1 = base + off_t1;
    void* w2 = base + off_t2;
    double2* partial = (double2*)(base + off_p);
    if (h->prec == GQT_FP64) {
      if (h->hop_real)
        run<true, false>(h, d_phi, R, rs, M, d_mu, nb, blk, seg_blk, flag, w1, w2, partial, st);
      else
        run<true, true>(h, d_phi, R, rs, M, d_mu, nb, blk, seg_blk, flag, w1, w2, partial, st);
    } else {
      if (h->hop_real)
        run<false, false>(h, d_phi, R, rs, M, d_mu, nb, blk, seg_blk, flag, w1, w2, partial, st);
      else
        run<false, true>(h, d_phi, R, rs, M, d_mu, nb, blk, seg_blk, flag, w1, w2, partial, st);
    }
    int hflag = 0;  // pageable host word: the copy completes before the call returns
    check_cuda(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st), "status readback");
    check_cuda(cudaStreamSynchronize(st), "gqt_dos_moments_noalloc");
    if (hflag & 4) throw Error(GQT_ENAN, "gqt_dos_moments_noalloc: NaN or Inf in a result");
    if (hflag & 2)
      throw Error(GQT_ERANGE,
                  "gqt_dos_moments_noalloc: a moment exceeds |phi|^2: the spectrum of H/dE is not inside [-1,1]");
    return GQT_OK;
  } catch (const Error& e) {
    set_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_error(std::string("internal error: ") + e.what());
    return GQT_EINVAL;
  }
}
