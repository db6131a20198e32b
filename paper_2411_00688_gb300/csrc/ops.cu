// Data-term kernels: separable Gaussian blur with fused residual / gradient-step
// / PDHG-dual epilogues, the pointwise identity-operator step, objective partial
// sums, the deterministic objective reduction, and small utilities.
//
// ProxSkip step (Algorithm 4): x^ = x - gamma (grad f(x) - h) with
// grad f = A^T (A x - b).  Every step kernel writes out = x - gamma g + ch h, so
//   skip iteration:  ch = gamma            -> out = x^            (= x_{k+1})
//   prox iteration:  ch = gamma - gamma/p  -> out = x^ - (gamma/p) h (prox input)
//   PGD / FISTA:     ch = 0 (h unused)     -> out = x - gamma grad f(x)
// The objective F(x) = 1/2 ||A x - b||^2 + alpha TV(x) (Eq. 5) is accumulated in
// the same passes: per-pixel FP32 terms, FP64 per-thread and per-block sums,
// block totals summed in a fixed order by one block (bitwise reproducible).
#include <cstdlib>

#include "blur_body.cuh"
#include "common.cuh"
#include "kernels.hpp"

namespace tvs {

namespace {

constexpr int PW_NT = 256;

template <int MODE, int R>
__global__ void __launch_bounds__(BNT)
blur_kernel(const float* __restrict__ src, int H, int W, BlurW w, const float* __restrict__ b,
            float* __restrict__ out, const float* __restrict__ x, const float* __restrict__ h,
            float gamma, float ch, float* __restrict__ axp, float* __restrict__ y, float tau,
            Partial* __restrict__ part_a, Partial* __restrict__ part_b) {
  pdl_enter();
  blur_tile_body<MODE, R>(src, H, W, w, b, out, x, h, gamma, ch, axp, y, tau, part_a, part_b, blockIdx.x,
                          blockIdx.y, blockIdx.y * gridDim.x + blockIdx.x);
}

template <int R>
__global__ void __launch_bounds__(FNT, 4)  // four CTAs per SM: 572 tiles of a 1024^2 image in one wave
blur_fb_step_kernel(const float* __restrict__ x, const float* __restrict__ b, const float* __restrict__ h,
                    float* __restrict__ out, int H, int W, BlurW w, float gamma, float ch,
                    Partial* __restrict__ part_a, Partial* __restrict__ part_b) {
  pdl_enter();
  blur_fb_step_body<R>(x, b, h, out, H, W, w, gamma, ch, part_a, part_b, blockIdx.x, blockIdx.y,
                       blockIdx.y * gridDim.x + blockIdx.x);
}

// Identity data term, 2D or 3D (nz slices of ny x nx).
__global__ void __launch_bounds__(PW_NT)
identity_step_kernel(const float* __restrict__ x, const float* __restrict__ b,
                     const float* __restrict__ h, float* __restrict__ out, int D, int H, int W,
                     int ndim, float gamma, float ch, Partial* __restrict__ part_a,
                     Partial* __restrict__ part_b, IndexMap im) {
  pdl_enter();
  const size_t n = (size_t)D * H * W, HW = (size_t)H * W;
  FAcc acc_a, acc_b;
  for (size_t o = blockIdx.x * (size_t)PW_NT + threadIdx.x; o < n; o += (size_t)gridDim.x * PW_NT) {
    int gk, gi, gj;
    im.coords(o, gk, gi, gj);
    const float xc = __ldg(x + o), bb = __ldg(b + o);
    const float r = xc - bb;
    if (out) {
      float v = xc - gamma * r;
      if (h) v = fmaf(ch, __ldg(h + o), v);
      out[o] = v;
    }
    acc_a.add(0.5f * (r * r));
    const float d0 = (ndim == 3 && gk < D - 1) ? __ldg(x + o + HW) - xc : 0.f;
    const float d1 = gi < H - 1 ? __ldg(x + o + W) - xc : 0.f;
    const float d2 = gj < W - 1 ? __ldg(x + o + 1) - xc : 0.f;
    acc_b.add(tv_term(d0, d1, d2));
  }
  block_sum2_store<PW_NT>(acc_a, acc_b, part_a, part_b, blockIdx.x);
}

__global__ void __launch_bounds__(PW_NT)
axpy_step_kernel(const float* __restrict__ g, const float* __restrict__ x,
                 const float* __restrict__ h, float* __restrict__ out, int D, int H, int W,
                 int ndim, float sigma, float ch, Partial* __restrict__ part_b, IndexMap im) {
  pdl_enter();
  const size_t n = (size_t)D * H * W, HW = (size_t)H * W;
  FAcc acc_b;
  for (size_t o = blockIdx.x * (size_t)PW_NT + threadIdx.x; o < n; o += (size_t)gridDim.x * PW_NT) {
    const float xc = __ldg(x + o);
    float v = xc - sigma * __ldg(g + o);
    if (h) v = fmaf(ch, __ldg(h + o), v);
    out[o] = v;
    if (part_b) {
      int gk, gi, gj;
    im.coords(o, gk, gi, gj);
      const float d0 = (ndim == 3 && gk < D - 1) ? __ldg(x + o + HW) - xc : 0.f;
      const float d1 = gi < H - 1 ? __ldg(x + o + W) - xc : 0.f;
      const float d2 = gj < W - 1 ? __ldg(x + o + 1) - xc : 0.f;
      acc_b.add(tv_term(d0, d1, d2));
    }
  }
  if (part_b) block_sum2_store<PW_NT>(FAcc(), acc_b, nullptr, part_b, blockIdx.x);
}

__global__ void __launch_bounds__(PW_NT)
tv_partials_kernel(const float* __restrict__ x, int D, int H, int W, int ndim,
                   Partial* __restrict__ part_b, IndexMap im) {
  pdl_enter();
  const size_t n = (size_t)D * H * W, HW = (size_t)H * W;
  FAcc acc_b;
  for (size_t o = blockIdx.x * (size_t)PW_NT + threadIdx.x; o < n; o += (size_t)gridDim.x * PW_NT) {
    int gk, gi, gj;
    im.coords(o, gk, gi, gj);
    const float xc = __ldg(x + o);
    const float d0 = (ndim == 3 && gk < D - 1) ? __ldg(x + o + HW) - xc : 0.f;
    const float d1 = gi < H - 1 ? __ldg(x + o + W) - xc : 0.f;
    const float d2 = gj < W - 1 ? __ldg(x + o + 1) - xc : 0.f;
    acc_b.add(tv_term(d0, d1, d2));
  }
  block_sum2_store<PW_NT>(FAcc(), acc_b, nullptr, part_b, blockIdx.x);
}

// PDHGSkip-1 dual step for the identity operator (ax = x^), or, with ax == null,
// the skipped iteration y <- prox(y + tau A x_k) from the stored A x_k.
__global__ void __launch_bounds__(PW_NT)
pd1_dual_pointwise_kernel(size_t m, const float* __restrict__ axh, float* __restrict__ axp,
                          float* __restrict__ y, const float* __restrict__ b, float p, float tau,
                          Partial* __restrict__ part_a) {
  pdl_enter();
  FAcc acc;
  for (size_t o = blockIdx.x * (size_t)PW_NT + threadIdx.x; o < m; o += (size_t)gridDim.x * PW_NT) {
    const float bb = __ldg(b + o);
    if (axh) {
      const float v = __ldg(axh + o);
      const float axn = axp[o] + p * v;
      y[o] = (y[o] + tau * (axn + v) - tau * bb) / (1.f + tau);
      axp[o] = axn;
      const float r = axn - bb;
      acc.add(0.5f * (r * r));
    } else {
      y[o] = (y[o] + tau * axp[o] - tau * bb) / (1.f + tau);
    }
  }
  if (part_a) block_sum2_store<PW_NT>(acc, FAcc(), part_a, nullptr, blockIdx.x);
}

__global__ void __launch_bounds__(PW_NT)
pd_dual_pointwise_kernel(size_t m, const float* __restrict__ ax, float* __restrict__ axp,
                         float* __restrict__ y, const float* __restrict__ b, float tau,
                         Partial* __restrict__ part_a) {
  pdl_enter();
  FAcc acc;
  for (size_t o = blockIdx.x * (size_t)PW_NT + threadIdx.x; o < m; o += (size_t)gridDim.x * PW_NT) {
    const float v = __ldg(ax + o), bb = __ldg(b + o);
    const float prev = axp[o];
    y[o] = (y[o] + tau * (2.f * v - prev) - tau * bb) / (1.f + tau);
    axp[o] = v;
    const float r = v - bb;
    acc.add(0.5f * (r * r));
  }
  block_sum2_store<PW_NT>(acc, FAcc(), part_a, nullptr, blockIdx.x);
}

// block_sum_partials<NT> of two arrays at once: the loads of both are issued in the
// same pass and the two block reductions share their barriers.  Each sum is formed
// in the order block_sum_partials<NT> forms it (per thread, per warp, then over the
// warps), so the results are the same bits.
template <int NT>
__device__ __forceinline__ void block_sum_partials2(const Partial* __restrict__ pa, int na,
                                                    const Partial* __restrict__ pb, int nb, double* sum_a,
                                                    double* sum_b) {
  __shared__ Partial spa[NT / 32], spb[NT / 32];
  __shared__ double ta, tb;
  FAcc a, b;
  const int n = na > nb ? na : nb;
  for (int i = threadIdx.x; i < n; i += NT) {
    if (i < na) a.add(pa[i]);
    if (i < nb) b.add(pb[i]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_sum<32>(a);
  warp_sum<32>(b);
  if (lane == 0) {
    spa[warp] = Partial{a.s, a.c};
    spb[warp] = Partial{b.s, b.c};
  }
  __syncthreads();
  if (warp == 0) {
    a = FAcc();
    b = FAcc();
    if (lane < NT / 32) {
      a.s = spa[lane].s; a.c = spa[lane].c;
      b.s = spb[lane].s; b.c = spb[lane].c;
    }
    warp_sum<32>(a);
    warp_sum<32>(b);
    if (lane == 0) {
      ta = (double)a.s + (double)a.c;
      tb = (double)b.s + (double)b.c;
    }
  }
  __syncthreads();
  *sum_a = ta;
  *sum_b = tb;
}

__global__ void __launch_bounds__(512)
reduce_record_kernel(const Partial* __restrict__ part_a, int n_a, const Partial* __restrict__ part_b,
                     int n_b, double alpha, int every, double* obj, unsigned long long* ts,
                     double f_star, double target, int* flags, int* done_host, double* f_out) {
  pdl_enter();
  double sum_a, sum_b;
  block_sum_partials2<512>(part_a, n_a, part_b, n_b, &sum_a, &sum_b);
  if (threadIdx.x == 0) {
    const double F = sum_a + alpha * sum_b;
    if (f_out) *f_out = F;
    if (!flags) return;
    if (!isfinite(F)) {  // divergence or non-finite data: stop the solve, the host reports it
      flags[4] = 1;
      if (done_host) {
        *(volatile int*)done_host = 1;
        __threadfence_system();
      }
    }
    const int k = flags[2];
    flags[2] = k + 1;
    if (k < 0 || !obj || (every > 1 && k % every != 0)) return;
    obj[k] = F;
    if (ts) ts[k] = globaltimer_ns();
    if (f_star > 0.0 && flags[0] == 0 && (F - f_star) <= target * f_star) {
      flags[0] = 1;
      flags[1] = k;
      if (done_host) {
        *(volatile int*)done_host = 1;
        __threadfence_system();
      }
    }
  }
}

__global__ void __launch_bounds__(PW_NT)
dist_partials_kernel(size_t n, const float* __restrict__ x, const float* __restrict__ u, Partial* __restrict__ part) {
  pdl_enter();
  FAcc acc;
  for (size_t o = blockIdx.x * (size_t)PW_NT + threadIdx.x; o < n; o += (size_t)gridDim.x * PW_NT) {
    const float d = __ldg(x + o) - __ldg(u + o);
    acc.add(d * d);
  }
  block_sum2_store<PW_NT>(acc, FAcc(), part, nullptr, blockIdx.x);
}

__global__ void __launch_bounds__(512)
dist_record_kernel(const Partial* __restrict__ part, int n_part, double ref_norm2, double* dist, double target,
                   int* flags, int* done_host) {
  pdl_enter();
  const double sum = block_sum_partials<512>(part, n_part);
  if (threadIdx.x != 0) return;
  const int k = flags[2] - 1;
  if (k < 0) return;
  const double d = sqrt(sum / ref_norm2);
  dist[k] = d;
  if (target > 0.0 && flags[0] == 0 && d <= target) {
    flags[0] = 1;
    flags[1] = k;
    if (done_host) {
      *(volatile int*)done_host = 1;
      __threadfence_system();
    }
  }
}

__global__ void timestamp_kernel(unsigned long long* ts) {
  pdl_enter(); *ts = globaltimer_ns(); }

// Start stamp of an InnerStamp; the finalisation after the inner iterations
// writes the end stamp.
__global__ void inner_start_stamp_kernel(unsigned long long* arr, const int* ctr) {
  pdl_enter();
  arr[2 * *ctr] = globaltimer_ns();
}

__global__ void count_nonfinite_kernel(const float* __restrict__ x, size_t n, int* count) {
  pdl_enter();
  int c = 0;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n;
       o += (size_t)gridDim.x * blockDim.x)
    c += isfinite(x[o]) ? 0 : 1;
  if (c) atomicAdd(count, c);
}

__global__ void coin_kernel(uint64_t seed, double p, int64_t k0, int K, unsigned char* out) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < K) out[i] = (unsigned char)Philox4x64::coin(seed, p, (uint64_t)(k0 + i));
}

template <int MODE>
cudaError_t blur_launch(int H, int W, const float* src, const BlurW& w, const float* b, float* out,
                        const float* x, const float* h, float gamma, float ch, float* axp, float* y,
                        float tau, Partial* pa, Partial* pb, cudaStream_t s) {
  dim3 grid((W + BX - 1) / BX, (H + BY - 1) / BY);
  switch (w.R) {
#define TVS_BLUR_R(R_) \
  case R_: launch_kernel(blur_kernel<MODE, R_>, dim3(grid), dim3(BNT), 0, s, src, H, W, w, b, out, x, h, gamma, ch, axp, y, tau, pa, pb); break;
    TVS_BLUR_R(1) TVS_BLUR_R(2) TVS_BLUR_R(3) TVS_BLUR_R(4) TVS_BLUR_R(5) TVS_BLUR_R(6) TVS_BLUR_R(7) TVS_BLUR_R(8)
#undef TVS_BLUR_R
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

bool pdl_enabled() {
  static const bool on = [] {
    const char* e = getenv("TVS_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

int tile_blocks_2d(int H, int W) { return ((W + BX - 1) / BX) * ((H + BY - 1) / BY); }
int fb_step_tile_w(int R) { return fb_tile_w(R); }
int fb_step_tile_h(int R) { return fb_tile_h(R); }
int fb_step_blocks_2d(int H, int W, int R) {
  const int fx = fb_tile_w(R), fy = fb_tile_h(R);
  return ((W + fx - 1) / fx) * ((H + fy - 1) / fy);
}

cudaError_t launch_blur_fb_step(int H, int W, const float* x, const float* b, const float* h, float* out,
                                const BlurW& w, float gamma, float ch, Partial* part_data, Partial* part_tv,
                                cudaStream_t s) {
  dim3 grid((W + fb_tile_w(w.R) - 1) / fb_tile_w(w.R), (H + fb_tile_h(w.R) - 1) / fb_tile_h(w.R));
  switch (w.R) {
#define TVS_FB_R(R_) \
  case R_: launch_kernel(blur_fb_step_kernel<R_>, dim3(grid), dim3(FNT), 0, s, x, b, h, out, H, W, w, gamma, ch, part_data, part_tv); break;
    TVS_FB_R(1) TVS_FB_R(2) TVS_FB_R(3) TVS_FB_R(4) TVS_FB_R(5) TVS_FB_R(6) TVS_FB_R(7) TVS_FB_R(8)
#undef TVS_FB_R
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int pointwise_blocks(size_t n) {
  size_t b = (n + PW_NT - 1) / PW_NT;
  const size_t cap = 152 * 8;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_blur_residual(int H, int W, const float* x, const float* b, float* r_out,
                                 const BlurW& w, Partial* part_data, Partial* part_tv, cudaStream_t s) {
  return blur_launch<BM_RESID>(H, W, x, w, b, r_out, nullptr, nullptr, 0.f, 0.f, nullptr, nullptr,
                               0.f, part_data, part_tv, s);
}

cudaError_t launch_blur_step(int H, int W, const float* in, const float* x, const float* h,
                             float* out, const BlurW& w, float gamma, float ch, Partial* part_tv,
                             cudaStream_t s) {
  return blur_launch<BM_STEP>(H, W, in, w, nullptr, out, x, h, gamma, ch, nullptr, nullptr, 0.f,
                              nullptr, part_tv, s);
}

cudaError_t launch_blur_pd_dual(int H, int W, const float* x, float* ax_prev, float* y,
                                const float* b, const BlurW& w, float tau, Partial* part_data,
                                cudaStream_t s) {
  return blur_launch<BM_PD>(H, W, x, w, b, nullptr, nullptr, nullptr, 0.f, 0.f, ax_prev, y, tau,
                            part_data, nullptr, s);
}

cudaError_t launch_blur_pd1_dual(int H, int W, const float* xh, float* ax_prev, float* y, const float* b,
                                 const BlurW& w, float p, float tau, Partial* part_data, cudaStream_t s) {
  return blur_launch<BM_PD1>(H, W, xh, w, b, nullptr, nullptr, nullptr, p, 0.f, ax_prev, y, tau, part_data,
                             nullptr, s);
}

cudaError_t launch_blur(int H, int W, const float* x, float* y, const BlurW& w, cudaStream_t s) {
  return blur_launch<BM_PLAIN>(H, W, x, w, nullptr, y, nullptr, nullptr, 0.f, 0.f, nullptr, nullptr,
                               0.f, nullptr, nullptr, s);
}

cudaError_t launch_identity_step(const Dims& d, const float* x, const float* b, const float* h,
                                 float* out, float gamma, float ch, Partial* part_data,
                                 Partial* part_tv, cudaStream_t s) {
  launch_kernel(identity_step_kernel, dim3(pointwise_blocks(d.n())), dim3(PW_NT), 0, s, x, b, h, out, d.nz, d.ny, d.nx,
                                                                  d.ndim, gamma, ch, part_data, part_tv, IndexMap(d.nz, d.ny, d.nx));
  return cudaGetLastError();
}

cudaError_t launch_axpy_step(const Dims& d, const float* g, const float* x, const float* h,
                             float* out, float sigma, float ch, Partial* part_tv, cudaStream_t s) {
  launch_kernel(axpy_step_kernel, dim3(pointwise_blocks(d.n())), dim3(PW_NT), 0, s, g, x, h, out, d.nz, d.ny, d.nx, d.ndim,
                                                              sigma, ch, part_tv, IndexMap(d.nz, d.ny, d.nx));
  return cudaGetLastError();
}

cudaError_t launch_pd1_dual_pointwise(size_t m, const float* axh, float* ax_prev, float* y, const float* b,
                                      float p, float tau, Partial* part_data, cudaStream_t s) {
  launch_kernel(pd1_dual_pointwise_kernel, dim3(pointwise_blocks(m)), dim3(PW_NT), 0, s, m, axh, ax_prev, y, b, p, tau, part_data);
  return cudaGetLastError();
}

cudaError_t launch_tv_partials(const Dims& d, const float* x, Partial* part_tv, cudaStream_t s) {
  launch_kernel(tv_partials_kernel, dim3(pointwise_blocks(d.n())), dim3(PW_NT), 0, s, x, d.nz, d.ny, d.nx, d.ndim, part_tv,
                IndexMap(d.nz, d.ny, d.nx));
  return cudaGetLastError();
}

cudaError_t launch_pd_dual_pointwise(size_t m, const float* ax, float* ax_prev, float* y,
                                     const float* b, float tau, Partial* part_data, cudaStream_t s) {
  launch_kernel(pd_dual_pointwise_kernel, dim3(pointwise_blocks(m)), dim3(PW_NT), 0, s, m, ax, ax_prev, y, b, tau, part_data);
  return cudaGetLastError();
}

cudaError_t launch_reduce_record(const Partial* part_data, int n_data, const Partial* part_tv,
                                 int n_tv, double alpha, int every, double* obj,
                                 unsigned long long* ts, double f_star, double target, int* flags,
                                 int* done_host, double* f_out, cudaStream_t s) {
  launch_kernel(reduce_record_kernel, dim3(1), dim3(512), 0, s, part_data, n_data, part_tv, n_tv, alpha, every, obj, ts,
                                         f_star, target, flags, done_host, f_out);
  return cudaGetLastError();
}

cudaError_t launch_dist_partials(size_t n, const float* x, const float* u_ref, Partial* part, cudaStream_t s) {
  launch_kernel(dist_partials_kernel, dim3(pointwise_blocks(n)), dim3(PW_NT), 0, s, n, x, u_ref, part);
  return cudaGetLastError();
}

cudaError_t launch_dist_record(const Partial* part, int n_part, double ref_norm2, double* dist, double target,
                               int* flags, int* done_host, cudaStream_t s) {
  launch_kernel(dist_record_kernel, dim3(1), dim3(512), 0, s, part, n_part, ref_norm2, dist, target, flags, done_host);
  return cudaGetLastError();
}

cudaError_t launch_timestamp(unsigned long long* ts, cudaStream_t s) {
  launch_kernel(timestamp_kernel, dim3(1), dim3(1), 0, s, ts);
  return cudaGetLastError();
}

cudaError_t launch_inner_start_stamp(const InnerStamp& st, cudaStream_t s) {
  launch_kernel(inner_start_stamp_kernel, dim3(1), dim3(1), 0, s, st.arr, (const int*)st.ctr);
  return cudaGetLastError();
}

cudaError_t launch_count_nonfinite(const float* x, size_t n, int* count, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  launch_kernel(count_nonfinite_kernel, dim3(pointwise_blocks(n)), dim3(PW_NT), 0, s, x, n, count);
  return cudaGetLastError();
}

cudaError_t launch_coin_schedule(uint64_t seed, double p, int64_t k0, int K, unsigned char* out,
                                 cudaStream_t s) {
  if (K <= 0) return cudaSuccess;
  launch_kernel(coin_kernel, dim3((K + 255) / 256), dim3(256), 0, s, seed, p, k0, K, out);
  return cudaGetLastError();
}

}  // namespace tvs
