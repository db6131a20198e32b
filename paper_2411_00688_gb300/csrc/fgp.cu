// Inner TV-prox kernels: one fused accelerated dual projected-gradient (FGP)
// iteration per launch, and the finalisation u = P_X(z + lam div p).
//
// Sign convention (Section 2.1): div = -D^T, so u = z + lam div p = z - lam D^T p.
// One iteration, for the unit-ball dual p (the paper's q with |q_i| <= alpha is
// lam p), with r the momentum point of the FISTA acceleration (Algorithm 3):
//     r  = p_k + beta_k (p_k - p_{k-1})
//     u  = P_X(z + lam div r)                 (P_X = max(., 0) when nonneg)
//     p_{k+1} = P_B(r + D u / (4 ndim lam))   (P_B: pointwise unit-ball projection, Eq. 7)
// Each CTA stages r over its tile plus a one-pixel halo in shared memory, forms
// u over the tile plus the row/column after it, then writes p_{k+1}: the whole
// iteration is one pass over z, p_k, p_{k-1} and one write of p_{k+1}.
//
// This file holds the one-iteration 2D kernel and the finalisations; the
// temporally blocked 2D kernels are in fgp_tb.cu and the 3D ones in fgp3d.cu.
#include <cstdio>
#include <cstdlib>

#include "common.cuh"
#include "kernels.hpp"

namespace tvs {

namespace {

// End stamp of an InnerStamp, by the first thread of the first block of the kernel
// that follows the inner iterations (after pdl_enter(): they have completed).
__device__ __forceinline__ void stamp_inner_end(const InnerStamp& st) {
  if (st.arr && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
    const int c = *st.ctr;
    st.arr[2 * c + 1] = globaltimer_ns();
    *st.ctr = c + 1;
  }
}


constexpr int TX2 = 32, TY2 = 16, NT2 = 256;

template <typename T, bool NONNEG>
__global__ void __launch_bounds__(NT2)
fgp2d_kernel(const float* __restrict__ z, const T* __restrict__ pc, const T* __restrict__ pp,
             T* __restrict__ pn, int H, int W, float lam, float inv_step, float beta) {
  pdl_enter();
  __shared__ float sry[TY2 + 2][TX2 + 3];
  __shared__ float srx[TY2 + 2][TX2 + 3];
  __shared__ float su[TY2 + 1][TX2 + 2];
  const int j0 = blockIdx.x * TX2, i0 = blockIdx.y * TY2;
  const size_t n = (size_t)H * W;
  // r over rows i0-1 .. i0+TY2, columns j0-1 .. j0+TX2
  for (int e = threadIdx.x; e < (TY2 + 2) * (TX2 + 2); e += NT2) {
    const int a = e / (TX2 + 2), b = e - a * (TX2 + 2);
    const int gi = i0 - 1 + a, gj = j0 - 1 + b;
    float ry = 0.f, rx = 0.f;
    if (gi >= 0 && gi < H && gj >= 0 && gj < W) {
      const size_t o = (size_t)gi * W + gj;
      const float cy = Elem<T>::ld(pc + o), cx = Elem<T>::ld(pc + n + o);
      if (beta != 0.f) {
        const float qy = Elem<T>::ld(pp + o), qx = Elem<T>::ld(pp + n + o);
        ry = cy + beta * (cy - qy);
        rx = cx + beta * (cx - qx);
      } else {
        ry = cy;
        rx = cx;
      }
    }
    sry[a][b] = ry;
    srx[a][b] = rx;
  }
  __syncthreads();
  // u over rows i0 .. i0+TY2, columns j0 .. j0+TX2
  for (int e = threadIdx.x; e < (TY2 + 1) * (TX2 + 1); e += NT2) {
    const int a = e / (TX2 + 1), b = e - a * (TX2 + 1);
    const int gi = i0 + a, gj = j0 + b;
    float u = 0.f;
    if (gi < H && gj < W) {
      float dv = 0.f;
      if (gi < H - 1) dv += sry[a + 1][b + 1];
      if (gi > 0) dv -= sry[a][b + 1];
      if (gj < W - 1) dv += srx[a + 1][b + 1];
      if (gj > 0) dv -= srx[a + 1][b];
      u = __ldg(z + (size_t)gi * W + gj) + lam * dv;
      if (NONNEG) u = fmaxf(u, 0.f);
    }
    su[a][b] = u;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TY2 * TX2; e += NT2) {
    const int a = e / TX2, b = e - a * TX2;
    const int gi = i0 + a, gj = j0 + b;
    if (gi < H && gj < W) {
      const float uc = su[a][b];
      const float gy = gi < H - 1 ? su[a + 1][b] - uc : 0.f;
      const float gx = gj < W - 1 ? su[a][b + 1] - uc : 0.f;
      const float qy = sry[a + 1][b + 1] + inv_step * gy;
      const float qx = srx[a + 1][b + 1] + inv_step * gx;
      const float nrm2 = qy * qy + qx * qx;
      const float sc = nrm2 > 1.f ? rsqrtf(nrm2) : 1.f;
      const size_t o = (size_t)gi * W + gj;
      Elem<T>::st(pn + o, qy * sc);
      Elem<T>::st(pn + n + o, qx * sc);
    }
  }
}

// Pointwise finalisation; div p at a pixel needs p at the pixel and at the
// previous pixel along each axis.
template <typename T, bool NONNEG>
__global__ void fgp_finalize_kernel(const float* __restrict__ z, const T* __restrict__ p, int D,
                                    int H, int W, int ndim, float lam, float* __restrict__ x_out,
                                    float* __restrict__ h_out, float h_coef, T* __restrict__ p_home,
                                    const float* __restrict__ x_prev, float* __restrict__ fista_y,
                                    const float* __restrict__ beta_tab, const int* __restrict__ beta_idx,
                                    IndexMap im, InnerStamp st) {
  pdl_enter();
  stamp_inner_end(st);
  const float beta_x = fista_y ? beta_tab[*beta_idx] : 0.f;
  const size_t n = (size_t)D * H * W;
  const size_t HW = (size_t)H * W;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n;
       o += (size_t)gridDim.x * blockDim.x) {
    int gk, gi, gj;
    im.coords(o, gk, gi, gj);
    float dv = 0.f;
    int c = 0;
    if (ndim == 3) {
      if (gk < D - 1) dv += Elem<T>::ld(p + o);
      if (gk > 0) dv -= Elem<T>::ld(p + o - HW);
      c = 1;
    }
    const T* py = p + (size_t)c * n;
    const T* px = p + (size_t)(c + 1) * n;
    if (gi < H - 1) dv += Elem<T>::ld(py + o);
    if (gi > 0) dv -= Elem<T>::ld(py + o - W);
    if (gj < W - 1) dv += Elem<T>::ld(px + o);
    if (gj > 0) dv -= Elem<T>::ld(px + o - 1);
    const float zz = __ldg(z + o);
    float u = zz + lam * dv;
    if (NONNEG) u = fmaxf(u, 0.f);
    if (fista_y) {
      const float xp = __ldg(x_prev + o);
      fista_y[o] = u + beta_x * (u - xp);
    }
    x_out[o] = u;
    if (h_out) h_out[o] = h_coef * (u - zz);
    if (p_home) {
      for (int a = 0; a < ndim; ++a) p_home[(size_t)a * n + o] = p[(size_t)a * n + o];
    }
  }
}

// 2D finalisation over a (row, column-pair) grid: the arithmetic of
// fgp_finalize_kernel without its index division and grid-stride loop, two
// adjacent pixels of a row per thread (the generic kernel held 124 registers
// and two CTAs per SM; this one needs a few dozen).
template <typename T, bool NONNEG>
__global__ void __launch_bounds__(256)
fgp_finalize2d_kernel(const float* __restrict__ z, const T* __restrict__ p, int H, int W, float lam,
                      float* __restrict__ x_out, float* __restrict__ h_out, float h_coef, T* __restrict__ p_home,
                      const float* __restrict__ x_prev, float* __restrict__ fista_y,
                      const float* __restrict__ beta_tab, const int* __restrict__ beta_idx, InnerStamp st) {
  pdl_enter();
  stamp_inner_end(st);
  const int gi = blockIdx.y * blockDim.y + threadIdx.y;
  const int gj0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (gi >= H) return;
  const float beta_x = fista_y ? beta_tab[*beta_idx] : 0.f;
  const size_t n = (size_t)H * W;
  const T* py = p;
  const T* px = p + n;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int gj = gj0 + q;
    if (gj >= W) break;
    const size_t o = (size_t)gi * W + gj;
    float dv = 0.f;
    if (gi < H - 1) dv += Elem<T>::ld(py + o);
    if (gi > 0) dv -= Elem<T>::ld(py + o - W);
    if (gj < W - 1) dv += Elem<T>::ld(px + o);
    if (gj > 0) dv -= Elem<T>::ld(px + o - 1);
    const float zz = __ldg(z + o);
    float u = zz + lam * dv;
    if (NONNEG) u = fmaxf(u, 0.f);
    if (fista_y) {
      const float xp = __ldg(x_prev + o);
      fista_y[o] = u + beta_x * (u - xp);
    }
    x_out[o] = u;
    if (h_out) h_out[o] = h_coef * (u - zz);
    if (p_home) {
      p_home[o] = py[o];
      p_home[n + o] = px[o];
    }
  }
}

// PDHGSkip-1 finalisation (Algorithm 5 with omega + 1 = 1/p):
// u = P_X(z + lam div p_N); x^ = (u - x) / p; x <- x + p x^ (in place).
template <typename T, bool NONNEG>
__global__ void fgp_finalize_pd1_kernel(const float* __restrict__ z, const T* __restrict__ p, int H, int W,
                                        float lam, float prob_p, float* __restrict__ x,
                                        float* __restrict__ xh, T* __restrict__ p_home, IndexMap im,
                                        InnerStamp st) {
  pdl_enter();
  stamp_inner_end(st);
  const size_t n = (size_t)H * W;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    int gk, gi, gj;
    im.coords(o, gk, gi, gj);
    float dv = 0.f;
    if (gi < H - 1) dv += Elem<T>::ld(p + o);
    if (gi > 0) dv -= Elem<T>::ld(p + o - W);
    if (gj < W - 1) dv += Elem<T>::ld(p + n + o);
    if (gj > 0) dv -= Elem<T>::ld(p + n + o - 1);
    float u = __ldg(z + o) + lam * dv;
    if (NONNEG) u = fmaxf(u, 0.f);
    const float xc = x[o];
    const float h = (u - xc) / prob_p;
    xh[o] = h;
    x[o] = xc + prob_p * h;
    if (p_home) {
      p_home[o] = p[o];
      p_home[n + o] = p[n + o];
    }
  }
}

template <typename T, bool NN>
cudaError_t fgp_iter_t(const Dims& d, const float* z, const void* pc, const void* pp, void* pn,
                       float lam, float inv_step, float beta, cudaStream_t s) {
  dim3 grid((d.nx + TX2 - 1) / TX2, (d.ny + TY2 - 1) / TY2);
  launch_kernel(fgp2d_kernel<T, NN>, dim3(grid), dim3(NT2), 0, s, z, (const T*)pc, (const T*)pp, (T*)pn, d.ny, d.nx, lam,
                inv_step, beta);
  return cudaGetLastError();
}

template <typename T, bool NN>
cudaError_t fgp_finalize_t(const Dims& d, const float* z, const void* p, float lam, float* x_out,
                           float* h_out, float h_coef, void* p_home, const float* x_prev,
                           float* fista_y, const float* beta_tab, const int* beta_idx, InnerStamp st,
                           cudaStream_t s) {
  if (d.ndim == 2 && d.ny <= 65535 * 8) {
    const dim3 grid((d.nx + 63) / 64, (d.ny + 7) / 8);
    launch_kernel(fgp_finalize2d_kernel<T, NN>, grid, dim3(32, 8), 0, s, z, (const T*)p, d.ny, d.nx, lam, x_out,
                  h_out, h_coef, (T*)p_home, x_prev, fista_y, beta_tab, beta_idx, st);
    return cudaGetLastError();
  }
  const size_t n = d.n();
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  launch_kernel(fgp_finalize_kernel<T, NN>, dim3(blocks), dim3(256), 0, s, z, (const T*)p, d.nz, d.ny, d.nx, d.ndim, lam,
                                                    x_out, h_out, h_coef, (T*)p_home, x_prev,
                                                    fista_y, beta_tab, beta_idx, IndexMap(d.nz, d.ny, d.nx), st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fgp_iter(const Dims& d, const float* z, const void* pc, const void* pp, void* pn,
                            float lam, float inv_step, float beta, int dtype, bool nonneg,
                            cudaStream_t s) {
  if (d.n() == 0) return cudaSuccess;
  if (d.ndim == 3) return launch_fgp3d_iter(d, z, pc, pp, pn, lam, inv_step, beta, dtype, nonneg, s);
  return with_dual_type(dtype, [&](auto tag) {
    using T = typename decltype(tag)::type;
    return nonneg ? fgp_iter_t<T, true>(d, z, pc, pp, pn, lam, inv_step, beta, s)
                  : fgp_iter_t<T, false>(d, z, pc, pp, pn, lam, inv_step, beta, s);
  });
}

cudaError_t launch_fgp_finalize_pd1(const Dims& d, const float* z, const void* p, int dtype, float lam,
                                    bool nonneg, float prob_p, float* x, float* xh, void* p_home,
                                    InnerStamp st, cudaStream_t s) {
  const size_t n = d.n();
  if (n == 0) return cudaSuccess;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
#define TVS_PD1(T_)                                                                                   \
  if (nonneg)                                                                                         \
    launch_kernel(fgp_finalize_pd1_kernel<T_, true>, dim3(blocks), dim3(256), 0, s, z, (const T_*)p, d.ny, d.nx, lam, prob_p, x, xh, \
                                                             (T_*)p_home, IndexMap(1, d.ny, d.nx), st); \
  else                                                                                                \
    launch_kernel(fgp_finalize_pd1_kernel<T_, false>, dim3(blocks), dim3(256), 0, s, z, (const T_*)p, d.ny, d.nx, lam, prob_p, x, xh, \
                                                              (T_*)p_home, IndexMap(1, d.ny, d.nx), st);
  if (dtype == DUAL_F32) {
    TVS_PD1(float)
  } else if (dtype == DUAL_BF16) {
    TVS_PD1(__nv_bfloat16)
  } else if (dtype == DUAL_F16) {
    TVS_PD1(__half)
  } else {
    TVS_PD1(q15)
  }
#undef TVS_PD1
  return cudaGetLastError();
}

cudaError_t launch_fgp_finalize(const Dims& d, const float* z, const void* p, int dtype, float lam,
                                bool nonneg, float* x_out, float* h_out, float h_coef,
                                void* p_home, const float* x_prev, float* fista_y,
                                const float* beta_tab, const int* beta_idx, InnerStamp st, cudaStream_t s) {
  if (d.n() == 0) return cudaSuccess;
  return with_dual_type(dtype, [&](auto tag) {
    using T = typename decltype(tag)::type;
    return nonneg ? fgp_finalize_t<T, true>(d, z, p, lam, x_out, h_out, h_coef, p_home, x_prev, fista_y, beta_tab, beta_idx, st, s)
                  : fgp_finalize_t<T, false>(d, z, p, lam, x_out, h_out, h_coef, p_home, x_prev, fista_y, beta_tab, beta_idx, st, s);
  });
}

}  // namespace tvs
