// Temporally blocked 2D TV-prox kernels: up to TB accelerated dual projected-
// gradient (FGP) iterations per launch over a tile with a TB-pixel halo, in
// shared memory (fgp2d_tb_kernel) or in registers (fgp2d_rb_kernel, body in
// fgp_rb.cuh).  Each iteration is the one of fgp.cu:
//     r  = p_k + beta_k (p_k - p_{k-1})
//     u  = P_X(z + lam div r)
//     p_{k+1} = P_B(r + D u / (4 ndim lam))
// and every configuration computes the same iterates as the one-iteration kernel.
#include <cstdio>
#include <cstdlib>

#include "common.cuh"
#include "fgp_rb.cuh"
#include "kernels.hpp"

namespace tvs {

namespace {

// ---------------------------------------------------------------------------
// Temporally blocked 2D variant: `iters` (<= TB) inner iterations per launch.
// The CTA stages z, p_k and r_{k+1} = p_k + beta (p_k - p_{k-1}) over its tile
// plus a TB-pixel halo (RH x RW cells, one warp row = 32 * CPL cells) and then
// iterates entirely in shared memory: iteration t forms u on the region shrunk
// by t-1 (top/left) / t-2 (bottom/right) and p, r on the region shrunk by t, so
// after TB iterations the tile interior holds exact values.  Each iteration is
//   phase 1: U = P_X(Z + lam div R)
//   phase 2: p_new = P_B(R + inv_step D U);  R = p_new + beta' (p_new - P);  P = p_new
// (both pointwise in R and P, so two barriers per iteration).  The last
// iteration keeps p_{k+iters-1} in R instead, and the tile interior of
// P = p_{k+iters} and R = p_{k+iters-1} is written out: one read of z, p_k,
// p_{k-1} and one write of two dual fields per `iters` iterations.

template <typename T, bool NONNEG, int TB, int CPL, int RPW>
__global__ void __launch_bounds__(256)
fgp2d_tb_kernel(const float* __restrict__ z, const T* __restrict__ pc, const T* __restrict__ pp,
                T* __restrict__ pn, T* __restrict__ pnp, int H, int W, float lam, float inv_step,
                TBBetas betas, int iters) {
  pdl_enter();
  constexpr int NW = 8;
  constexpr int RW = 32 * CPL, RH = NW * RPW;
  constexpr int TW = RW - 2 * TB, TH = RH - 2 * TB;
  extern __shared__ float sm[];
  float* Z = sm;
  float* U = Z + RH * RW;
  float* Ry = U + RH * RW;
  float* Rx = Ry + RH * RW;
  float* Py = Rx + RH * RW;
  float* Px = Py + RH * RW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gi0 = blockIdx.y * TH - TB, gj0 = blockIdx.x * TW - TB;
  const size_t n = (size_t)H * W;
  const float b0 = betas.b[0];
#pragma unroll
  for (int rr = 0; rr < RPW; ++rr) {
    const int a = warp + NW * rr;
    const int gi = gi0 + a;
#pragma unroll
    for (int cc = 0; cc < CPL; ++cc) {
      const int c = lane + 32 * cc;
      const int gj = gj0 + c;
      float zz = 0.f, cy = 0.f, cx = 0.f, ry = 0.f, rx = 0.f;
      if (gi >= 0 && gi < H && gj >= 0 && gj < W) {
        const size_t o = (size_t)gi * W + gj;
        zz = __ldg(z + o);
        cy = Elem<T>::ld(pc + o);
        cx = Elem<T>::ld(pc + n + o);
        if (b0 != 0.f) {
          ry = cy + b0 * (cy - Elem<T>::ld(pp + o));
          rx = cx + b0 * (cx - Elem<T>::ld(pp + n + o));
        } else {
          ry = cy;
          rx = cx;
        }
      }
      const int e = a * RW + c;
      Z[e] = zz;
      Py[e] = cy;
      Px[e] = cx;
      Ry[e] = ry;
      Rx[e] = rx;
    }
  }
  __syncthreads();
  for (int t = 1; t <= iters; ++t) {
    // phase 1: u on rows/cols [t, R - t + 1)
#pragma unroll
    for (int rr = 0; rr < RPW; ++rr) {
      const int a = warp + NW * rr;
      const int gi = gi0 + a;
#pragma unroll
      for (int cc = 0; cc < CPL; ++cc) {
        const int c = lane + 32 * cc;
        const int gj = gj0 + c;
        if (a >= t && a < RH - t + 1 && c >= t && c < RW - t + 1) {
          const int e = a * RW + c;
          float u = 0.f;
          if (gi >= 0 && gi < H && gj >= 0 && gj < W) {
            float dv = 0.f;
            if (gi < H - 1) dv += Ry[e];
            if (gi > 0) dv -= Ry[e - RW];
            if (gj < W - 1) dv += Rx[e];
            if (gj > 0) dv -= Rx[e - 1];
            u = Z[e] + lam * dv;
            if (NONNEG) u = fmaxf(u, 0.f);
          }
          U[e] = u;
        }
      }
    }
    __syncthreads();
    const bool last = (t == iters);
    const float bn = last ? 0.f : betas.b[t];
    // phase 2: p, r on rows/cols [t, R - t)
#pragma unroll
    for (int rr = 0; rr < RPW; ++rr) {
      const int a = warp + NW * rr;
      const int gi = gi0 + a;
#pragma unroll
      for (int cc = 0; cc < CPL; ++cc) {
        const int c = lane + 32 * cc;
        const int gj = gj0 + c;
        if (a >= t && a < RH - t && c >= t && c < RW - t) {
          const int e = a * RW + c;
          const float uc = U[e];
          const float gy = gi < H - 1 ? U[e + RW] - uc : 0.f;
          const float gx = gj < W - 1 ? U[e + 1] - uc : 0.f;
          const float qy = Ry[e] + inv_step * gy;
          const float qx = Rx[e] + inv_step * gx;
          const float nrm2 = qy * qy + qx * qx;
          const float sc = nrm2 > 1.f ? rsqrtf(nrm2) : 1.f;
          float ny = qy * sc, nx = qx * sc;
          // stored values go through the dual storage type, as in the one-step kernel
          ny = Elem<T>::round(ny);
          nx = Elem<T>::round(nx);
          const float oy = Py[e], ox = Px[e];
          if (last) {
            Ry[e] = oy;
            Rx[e] = ox;
          } else {
            Ry[e] = ny + bn * (ny - oy);
            Rx[e] = nx + bn * (nx - ox);
          }
          Py[e] = ny;
          Px[e] = nx;
        }
      }
    }
    __syncthreads();
  }
  // write the tile interior: P = p_{k+iters}, R = p_{k+iters-1}
#pragma unroll
  for (int rr = 0; rr < RPW; ++rr) {
    const int a = warp + NW * rr;
    const int gi = gi0 + a;
#pragma unroll
    for (int cc = 0; cc < CPL; ++cc) {
      const int c = lane + 32 * cc;
      const int gj = gj0 + c;
      if (a >= TB && a < TB + TH && c >= TB && c < TB + TW && gi < H && gj < W) {
        const int e = a * RW + c;
        const size_t o = (size_t)gi * W + gj;
        Elem<T>::st(pn + o, Py[e]);
        Elem<T>::st(pn + n + o, Px[e]);
        Elem<T>::st(pnp + o, Ry[e]);
        Elem<T>::st(pnp + n + o, Rx[e]);
      }
    }
  }
}

template <typename T, bool NONNEG, int TB, int CPL, int RPW>
__global__ void __launch_bounds__(256, (RPW * CPL > 10) ? 1 : (CPL == 2 ? 3 : 2))
fgp2d_rb_kernel(const float* __restrict__ z, const T* __restrict__ pc, const T* __restrict__ pp,
                T* __restrict__ pn, T* __restrict__ pnp, int H, int W, float lam, float inv_step,
                TBBetas betas, int iters) {
  pdl_enter();
  T* const dst_p = pn;
  T* const dst_r = pnp;
  const int tx = blockIdx.x, ty = blockIdx.y;
  fgp2d_rb_body<T, NONNEG, TB, CPL, RPW>(z, pc, pp, dst_p, dst_r, H, W, lam, inv_step, betas, iters, tx, ty);
}

template <typename T, bool NN, int TB, int CPL, int RPW>
cudaError_t fgp_tb_t(const Dims& d, const float* z, const void* pc, const void* pp, void* pn, void* pnp,
                     float lam, float inv_step, const float* betas, int iters, cudaStream_t s) {
  constexpr int RW = 32 * CPL, RH = 8 * RPW, TW = RW - 2 * TB, TH = RH - 2 * TB;
  constexpr size_t smem = 6 * (size_t)RH * RW * sizeof(float);
  if (iters < 0) {  // preparation call: allow the dynamic shared memory this tile needs
    return cudaFuncSetAttribute(fgp2d_tb_kernel<T, NN, TB, CPL, RPW>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  TBBetas b{};
  for (int i = 0; i < iters && i < 8; ++i) b.b[i] = betas[i];
  dim3 grid((d.nx + TW - 1) / TW, (d.ny + TH - 1) / TH);
  launch_kernel(fgp2d_tb_kernel<T, NN, TB, CPL, RPW>, dim3(grid), dim3(256), smem, s, 
      z, (const T*)pc, (const T*)pp, (T*)pn, (T*)pnp, d.ny, d.nx, lam, inv_step, b, iters);
  return cudaGetLastError();
}

template <typename T, bool NN, int TB, int CPL, int RPW>
cudaError_t fgp_rb_t(const Dims& d, const float* z, const void* pc, const void* pp, void* pn, void* pnp,
                     float lam, float inv_step, const float* betas, int iters, cudaStream_t s) {
  constexpr int RW = 32 * CPL, RH = 8 * RPW, TW = RW - 2 * TB, TH = RH - 2 * TB;
  if (iters < 0) return cudaSuccess;  // preparation call: static shared memory only
  TBBetas b{};
  for (int i = 0; i < iters && i < 8; ++i) b.b[i] = betas[i];
  dim3 grid((d.nx + TW - 1) / TW, (d.ny + TH - 1) / TH);
  launch_kernel(fgp2d_rb_kernel<T, NN, TB, CPL, RPW>, dim3(grid), dim3(256), 0, s, 
      z, (const T*)pc, (const T*)pp, (T*)pn, (T*)pnp, d.ny, d.nx, lam, inv_step, b, iters);
  return cudaGetLastError();
}

template <typename T, bool NN>
cudaError_t fgp_tb_dispatch(const FgpConfig& c, const Dims& d, const float* z, const void* pc,
                            const void* pp, void* pn, void* pnp, float lam, float inv_step,
                            const float* betas, int iters, cudaStream_t s) {
#define TVS_TB_CASE(TB_, CPL_, RPW_)                                                          \
  if (c.tb == TB_ && c.cpl == CPL_ && c.rpw == RPW_)                                         \
    return fgp_tb_t<T, NN, TB_, CPL_, RPW_>(d, z, pc, pp, pn, pnp, lam, inv_step, betas, iters, s);
  TVS_TB_CASE(2, 2, 4)
  TVS_TB_CASE(3, 2, 4)
  TVS_TB_CASE(4, 2, 4)
  TVS_TB_CASE(4, 2, 5)
  TVS_TB_CASE(4, 1, 5)
  TVS_TB_CASE(6, 2, 6)
  TVS_TB_CASE(8, 2, 6)
#undef TVS_TB_CASE
#define TVS_RB_CASE(TB_, CPL_, RPW_)                                                          \
  if (c.tb == TB_ && c.cpl == CPL_ && c.rpw == RPW_ + 100)                                   \
    return fgp_rb_t<T, NN, TB_, CPL_, RPW_>(d, z, pc, pp, pn, pnp, lam, inv_step, betas, iters, s);
  TVS_RB_CASE(2, 2, 4)
  TVS_RB_CASE(4, 1, 5)
  TVS_RB_CASE(4, 2, 5)
  TVS_RB_CASE(4, 2, 8)
  TVS_RB_CASE(4, 1, 8)
  TVS_RB_CASE(6, 2, 8)
  TVS_RB_CASE(3, 2, 6)
  TVS_RB_CASE(4, 2, 4)
  TVS_RB_CASE(4, 1, 6)
  TVS_RB_CASE(5, 2, 4)
#undef TVS_RB_CASE
  return cudaErrorInvalidValue;
}

}  // namespace

bool fgp_config_valid(const FgpConfig& c) {
  if (c.tb <= 1) return true;
  const int ok[][3] = {{2, 2, 4},   {3, 2, 4},   {4, 2, 4},   {4, 2, 5},   {4, 1, 5},   {6, 2, 6},
                       {8, 2, 6},   {2, 2, 104}, {4, 1, 105}, {4, 2, 105}, {4, 2, 108}, {4, 1, 108},
                       {6, 2, 108}, {3, 2, 106}, {4, 2, 104}, {4, 1, 106}, {5, 2, 104}};
  for (const auto& k : ok)
    if (k[0] == c.tb && k[1] == c.cpl && k[2] == c.rpw) return true;
  return false;
}

cudaError_t fgp_prepare_device() {
  const int cfgs[][3] = {{2, 2, 4}, {3, 2, 4}, {4, 2, 4}, {4, 2, 5}, {4, 1, 5}, {6, 2, 6}, {8, 2, 6}};
  Dims d;
  for (const auto& k : cfgs) {
    FgpConfig c;
    c.tb = k[0];
    c.cpl = k[1];
    c.rpw = k[2];
    for (int dt = 0; dt < 4; ++dt)
      for (int nn = 0; nn < 2; ++nn) {
        const cudaError_t e = with_dual_type(dt, [&](auto tag) {
          using T = typename decltype(tag)::type;
          return nn ? fgp_tb_dispatch<T, true>(c, d, nullptr, nullptr, nullptr, nullptr, nullptr, 0.f, 0.f, nullptr, -1, 0)
                    : fgp_tb_dispatch<T, false>(c, d, nullptr, nullptr, nullptr, nullptr, nullptr, 0.f, 0.f, nullptr, -1, 0);
        });
        if (e != cudaSuccess) return e;
      }
  }
  return cudaSuccess;
}

cudaError_t launch_fgp_block(const FgpConfig& c, const Dims& d, const float* z, const void* pc,
                             const void* pp, void* pn, void* pnp, float lam, float inv_step,
                             const float* betas, int iters, int dtype, bool nonneg, cudaStream_t s) {
  if (d.n() == 0 || iters <= 0) return cudaSuccess;
  if (d.ndim != 2 || iters > c.tb) return cudaErrorInvalidValue;
  return with_dual_type(dtype, [&](auto tag) {
    using T = typename decltype(tag)::type;
    return nonneg ? fgp_tb_dispatch<T, true>(c, d, z, pc, pp, pn, pnp, lam, inv_step, betas, iters, s)
                  : fgp_tb_dispatch<T, false>(c, d, z, pc, pp, pn, pnp, lam, inv_step, betas, iters, s);
  });
}

}  // namespace tvs
