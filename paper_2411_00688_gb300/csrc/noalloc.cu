// tv_prox_noalloc: the TV prox for callers that may not allocate device memory.
//
// Some applications own every byte of device memory themselves (they reserve the
// GPU with their own pool when they start, or they run next to a thread that is
// capturing a CUDA graph in global capture mode, where cudaMalloc is not
// allowed), so a library call that reaches cudaMalloc breaks them.  This entry
// point runs the same inner iterations as tv_prox but keeps its working dual
// fields in one fixed-size array that lives in the library's device image: no
// context is needed and nothing is allocated or freed, on the device or on the
// host.
//
// The array is a file-scope __device__ variable of TVS_NOALLOC_SCRATCH_BYTES.  A
// device holds it from the moment CUDA loads this file's device image there --
// with the default lazy module loading, at the first call's address lookup on
// that device -- until the process exits.  Host code cannot use the variable's
// name as a device address; the first call on a device (with that device
// current) asks the runtime for the address once and keeps it, so that call
// belongs before the application reserves the device's memory for itself.  All calls on a device share the array and it keeps the previous
// call's contents: the part that must start at zero (the cold-start dual) is
// cleared on every call, and calls whose work overlaps on the GPU race on it.
#include <mutex>

#include "common.cuh"
#include "kernels.hpp"
#include "tvs.h"

using namespace tvs;

namespace {

constexpr size_t kScratchBytes = TVS_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Once per device, with that device current: the device address of the scratch
// array, and the dynamic shared-memory limits the blocked FGP kernel needs.
tvs_status scratch_for_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return TVS_ECUDA;
  if (dev >= kMaxDevices) return TVS_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return TVS_ECUDA;
    if (fgp_prepare_device() != cudaSuccess) return TVS_ECUDA;
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return TVS_OK;
}

// Momentum coefficient of inner iteration i (1-based), advanced one step at a
// time: 0 for i = 1, (t_{i-1} - 1) / t_i afterwards, t_1 = 1.
struct BetaStream {
  double t = 1.0;
  int i = 0;
  float next() {
    ++i;
    if (i == 1) return 0.f;
    const double tn = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
    const float b = (float)((t - 1.0) / tn);
    t = tn;
    return b;
  }
};

}  // namespace

extern "C" tvs_status tv_prox_noalloc(int ndim, const int dims[3], const float* z, float* u,
                                      double lambda, int n_iter, tvs_dual_dtype dual,
                                      void* dual_state, int nonneg, void* cuda_stream) {
  if (!dims || !z || !u || z == u) return TVS_EINVAL;
  if (ndim != 2 && ndim != 3) return TVS_EINVAL;
  if (dims[0] < 1 || dims[1] < 1 || (ndim == 3 && dims[2] < 1)) return TVS_EINVAL;
  if (!(lambda >= 0.0) || !isfinite(lambda) || n_iter < 0) return TVS_EINVAL;
  if (dual != TVS_DUAL_F32 && dual != TVS_DUAL_BF16 && dual != TVS_DUAL_F16 && dual != TVS_DUAL_Q15)
    return TVS_EINVAL;
  Dims d;
  d.nx = dims[0];
  d.ny = dims[1];
  d.nz = ndim == 3 ? dims[2] : 1;
  d.ndim = ndim;
  // Pixels that fit in the static scratch, bounded before any product is formed
  // so that no size wraps around.
  const size_t planes = (size_t)ndim * (dual_state ? 3 : 4);
  const size_t max_px = kScratchBytes / (dual_elem_bytes(dual) * planes);
  size_t n = 0;
  if (!pixels_within(d.nx, d.ny, d.nz, max_px, &n)) return TVS_EUNSUPPORTED;
  const size_t plane_bytes = dual_elem_bytes(dual) * (size_t)ndim * n;

  void* base = nullptr;
  tvs_status st = scratch_for_current_device(&base);
  if (st != TVS_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  char* sc = (char*)base;
  void* buf[4];
  if (dual_state) {
    buf[0] = dual_state;
    for (int i = 1; i < 4; ++i) buf[i] = sc + (size_t)(i - 1) * plane_bytes;
  } else {
    for (int i = 0; i < 4; ++i) buf[i] = sc + (size_t)i * plane_bytes;
    if (cudaMemsetAsync(buf[0], 0, plane_bytes, s) != cudaSuccess) return TVS_ECUDA;
  }

  const bool use = lambda > 0.0;
  const float lam = (float)lambda;
  int fin = 0;
  if (use && n_iter > 0) {
    const float inv_step = (float)(1.0 / (4.0 * ndim * lambda));
    BetaStream beta;
    if (ndim == 2) {
      FgpConfig cfg;  // the default blocked variant of tv_prox: 4 iterations per launch
      cfg.tb = 4;
      cfg.cpl = 1;
      cfg.rpw = 5;
      int q = 0;
      for (int g = 1; g <= n_iter;) {
        const int it = n_iter - g + 1 < cfg.tb ? n_iter - g + 1 : cfg.tb;
        float b[8];
        for (int j = 0; j < it; ++j) b[j] = beta.next();
        void* pc = buf[2 * q];
        void* pp = g == 1 ? pc : buf[2 * q + 1];
        if (launch_fgp_block(cfg, d, z, pc, pp, buf[2 * (1 - q)], buf[2 * (1 - q) + 1], lam, inv_step, b,
                             it, dual, nonneg != 0, s) != cudaSuccess)
          return TVS_ECUDA;
        q = 1 - q;
        g += it;
      }
      fin = 2 * q;
    } else {
      for (int i = 1; i <= n_iter; ++i) {
        void* cur = buf[(i - 1) % 3];
        void* prev = i >= 2 ? buf[(i - 2) % 3] : cur;
        if (launch_fgp_iter(d, z, cur, prev, buf[i % 3], lam, inv_step, beta.next(), dual, nonneg != 0, s) !=
            cudaSuccess)
          return TVS_ECUDA;
      }
      fin = n_iter % 3;
    }
  }
  if (launch_fgp_finalize(d, z, buf[fin], dual, use ? lam : 0.f, nonneg != 0, u, nullptr, 0.f,
                          (fin != 0 && dual_state) ? dual_state : nullptr, nullptr, nullptr, nullptr,
                          nullptr, InnerStamp{}, s) != cudaSuccess)
    return TVS_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TVS_ECUDA;
  return TVS_OK;
}
