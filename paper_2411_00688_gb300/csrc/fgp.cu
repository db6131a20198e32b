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
#include <cstdio>
#include <cstdlib>

#include "common.cuh"
#include "fgp_rb.cuh"
#include "kernels.hpp"

namespace tvs {

namespace {

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

constexpr int TX3 = 32, TY3 = 8, TZ3 = 4, NT3 = 256;

template <typename T, bool NONNEG>
__global__ void __launch_bounds__(NT3)
fgp3d_kernel(const float* __restrict__ z, const T* __restrict__ pc, const T* __restrict__ pp,
             T* __restrict__ pn, int D, int H, int W, float lam, float inv_step, float beta) {
  pdl_enter();
  __shared__ float sr[3][TZ3 + 2][TY3 + 2][TX3 + 2];
  __shared__ float su[TZ3 + 1][TY3 + 1][TX3 + 1];
  const int j0 = blockIdx.x * TX3, i0 = blockIdx.y * TY3, k0 = blockIdx.z * TZ3;
  const size_t n = (size_t)D * H * W;
  constexpr int RX = TX3 + 2, RY = TY3 + 2, RZ = TZ3 + 2;
  for (int e = threadIdx.x; e < RZ * RY * RX; e += NT3) {
    const int c = e / (RY * RX), rem = e - c * (RY * RX);
    const int a = rem / RX, b = rem - a * RX;
    const int gk = k0 - 1 + c, gi = i0 - 1 + a, gj = j0 - 1 + b;
    float r0 = 0.f, r1 = 0.f, r2 = 0.f;
    if (gk >= 0 && gk < D && gi >= 0 && gi < H && gj >= 0 && gj < W) {
      const size_t o = ((size_t)gk * H + gi) * W + gj;
      const float c0 = Elem<T>::ld(pc + o), c1 = Elem<T>::ld(pc + n + o), c2 = Elem<T>::ld(pc + 2 * n + o);
      if (beta != 0.f) {
        r0 = c0 + beta * (c0 - Elem<T>::ld(pp + o));
        r1 = c1 + beta * (c1 - Elem<T>::ld(pp + n + o));
        r2 = c2 + beta * (c2 - Elem<T>::ld(pp + 2 * n + o));
      } else {
        r0 = c0; r1 = c1; r2 = c2;
      }
    }
    sr[0][c][a][b] = r0;
    sr[1][c][a][b] = r1;
    sr[2][c][a][b] = r2;
  }
  __syncthreads();
  constexpr int UX = TX3 + 1, UY = TY3 + 1, UZ = TZ3 + 1;
  for (int e = threadIdx.x; e < UZ * UY * UX; e += NT3) {
    const int c = e / (UY * UX), rem = e - c * (UY * UX);
    const int a = rem / UX, b = rem - a * UX;
    const int gk = k0 + c, gi = i0 + a, gj = j0 + b;
    float u = 0.f;
    if (gk < D && gi < H && gj < W) {
      float dv = 0.f;
      if (gk < D - 1) dv += sr[0][c + 1][a + 1][b + 1];
      if (gk > 0) dv -= sr[0][c][a + 1][b + 1];
      if (gi < H - 1) dv += sr[1][c + 1][a + 1][b + 1];
      if (gi > 0) dv -= sr[1][c + 1][a][b + 1];
      if (gj < W - 1) dv += sr[2][c + 1][a + 1][b + 1];
      if (gj > 0) dv -= sr[2][c + 1][a + 1][b];
      u = __ldg(z + ((size_t)gk * H + gi) * W + gj) + lam * dv;
      if (NONNEG) u = fmaxf(u, 0.f);
    }
    su[c][a][b] = u;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TZ3 * TY3 * TX3; e += NT3) {
    const int c = e / (TY3 * TX3), rem = e - c * (TY3 * TX3);
    const int a = rem / TX3, b = rem - a * TX3;
    const int gk = k0 + c, gi = i0 + a, gj = j0 + b;
    if (gk < D && gi < H && gj < W) {
      const float uc = su[c][a][b];
      const float g0 = gk < D - 1 ? su[c + 1][a][b] - uc : 0.f;
      const float g1 = gi < H - 1 ? su[c][a + 1][b] - uc : 0.f;
      const float g2 = gj < W - 1 ? su[c][a][b + 1] - uc : 0.f;
      const float q0 = sr[0][c + 1][a + 1][b + 1] + inv_step * g0;
      const float q1 = sr[1][c + 1][a + 1][b + 1] + inv_step * g1;
      const float q2 = sr[2][c + 1][a + 1][b + 1] + inv_step * g2;
      const float nrm2 = q0 * q0 + q1 * q1 + q2 * q2;
      const float sc = nrm2 > 1.f ? rsqrtf(nrm2) : 1.f;
      const size_t o = ((size_t)gk * H + gi) * W + gj;
      Elem<T>::st(pn + o, q0 * sc);
      Elem<T>::st(pn + n + o, q1 * sc);
      Elem<T>::st(pn + 2 * n + o, q2 * sc);
    }
  }
}

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

// ---------------------------------------------------------------------------
// 3D, one inner iteration per launch, marching through z ("2.5D").  A CTA owns an
// x-y region of 32*CPL x 8*RPW cells (warp w: RPW consecutive rows, lane: CPL
// adjacent columns) and a chunk of ZC planes.  Per plane k it loads r(k+1)
// (from z, p_k, p_{k-1}), forms u(k+1), then writes p_{k+1} at plane k from
// r(k), u(k), u(k+1): each voxel is read once (z, p_k, p_{k-1}) and written once,
// plus one warm-up plane per chunk and a one-cell x-y halo.  x neighbours come
// from warp shuffles, y neighbours from registers or, across warps, from a
// double-buffered shared row (one barrier per plane).
template <typename T, bool NONNEG, int CPL, int RPW, int ZC>
__global__ void __launch_bounds__(256)
fgp3d_zm_kernel(const float* __restrict__ z, const T* __restrict__ pc, const T* __restrict__ pp,
                T* __restrict__ pn, int D, int H, int W, float lam, float inv_step, float beta) {
  pdl_enter();
  constexpr int NW = 8;
  constexpr int RW = 32 * CPL, RH = NW * RPW;
  constexpr int TW = RW - 2, TH = RH - 2;
  __shared__ float sh_ry[2][NW][RW];   // bottom row of r_y(k+1) of each warp block
  __shared__ float sh_u[2][NW][RW];    // top row of u(k+1) of each warp block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gi0 = blockIdx.y * TH - 1 + warp * RPW;
  const int gj0 = blockIdx.x * TW - 1 + lane * CPL;
  const int k0 = blockIdx.z * ZC;
  const int k1 = min(k0 + ZC, D);
  const size_t HW = (size_t)H * W, n = (size_t)D * HW;
  bool row_in[RPW], row_dn[RPW], row_up[RPW], col_in[CPL], col_rt[CPL], col_lf[CPL];
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const int gi = gi0 + r;
    row_in[r] = gi >= 0 && gi < H;
    row_dn[r] = gi < H - 1;
    row_up[r] = gi > 0;
  }
#pragma unroll
  for (int q = 0; q < CPL; ++q) {
    const int gj = gj0 + q;
    col_in[q] = gj >= 0 && gj < W;
    col_rt[q] = gj < W - 1;
    col_lf[q] = gj > 0;
  }
  // r(k) (three components), r_z(k-1), u(k) of the thread's cells
  float Rz[RPW][CPL], Ry[RPW][CPL], Rx[RPW][CPL], Rzm[RPW][CPL], Uk[RPW][CPL];

  auto load_r = [&](int k, float (&rz)[RPW][CPL], float (&ry)[RPW][CPL], float (&rx)[RPW][CPL],
                    float (&zz)[RPW][CPL], bool need_all) {
#pragma unroll
    for (int r = 0; r < RPW; ++r)
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, zv = 0.f;
        if (k >= 0 && k < D && row_in[r] && col_in[q]) {
          const size_t o = (size_t)k * HW + (size_t)(gi0 + r) * W + (gj0 + q);
          const float c0 = Elem<T>::ld(pc + o);
          a0 = beta != 0.f ? c0 + beta * (c0 - Elem<T>::ld(pp + o)) : c0;
          if (need_all) {
            const float c1 = Elem<T>::ld(pc + n + o), c2 = Elem<T>::ld(pc + 2 * n + o);
            if (beta != 0.f) {
              a1 = c1 + beta * (c1 - Elem<T>::ld(pp + n + o));
              a2 = c2 + beta * (c2 - Elem<T>::ld(pp + 2 * n + o));
            } else {
              a1 = c1;
              a2 = c2;
            }
            zv = __ldg(z + o);
          }
        }
        rz[r][q] = a0;
        ry[r][q] = a1;
        rx[r][q] = a2;
        zz[r][q] = zv;
      }
  };
  // u at plane k from r(k) (Rz/Ry/Rx), r_z(k-1) and the staged r_y row above.
  auto form_u = [&](int k, const float (&rz)[RPW][CPL], const float (&ry)[RPW][CPL],
                    const float (&rx)[RPW][CPL], const float (&rzm)[RPW][CPL],
                    const float (&zz)[RPW][CPL], const float* ry_above, float (&u)[RPW][CPL]) {
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const float rx_left = __shfl_up_sync(0xffffffffu, rx[r][CPL - 1], 1);
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        const float up = r > 0 ? ry[r - 1][q] : ry_above[q];
        const float lf = q > 0 ? rx[r][q - 1] : rx_left;
        float dv = 0.f;
        if (k < D - 1) dv += rz[r][q];
        if (k > 0) dv -= rzm[r][q];
        if (row_dn[r]) dv += ry[r][q];
        if (row_up[r]) dv -= up;
        if (col_rt[q]) dv += rx[r][q];
        if (col_lf[q]) dv -= lf;
        float v = zz[r][q] + lam * dv;
        if (NONNEG) v = fmaxf(v, 0.f);
        u[r][q] = (k < D && row_in[r] && col_in[q]) ? v : 0.f;
      }
    }
  };

  // FP32 duals: plane k+2's stored values are fetched into registers while plane
  // k is computed, so their loads are in flight for a whole plane before make_r
  // forms r(k+2) from them (measured at 512^3: 1.08 -> 0.98 ms per iteration).
  // With 16-bit duals the extra registers cost more occupancy than the overlap
  // gains, so those load each plane when they need it.
  constexpr bool kPrefetch = sizeof(T) == 4;
  T Pc[RPW][CPL][3], Pp[RPW][CPL][3];
  float Zr[RPW][CPL];
  auto fetch = [&](int k) {
#pragma unroll
    for (int r = 0; r < RPW; ++r)
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        const bool in = k >= 0 && k < D && row_in[r] && col_in[q];
        const size_t o = in ? (size_t)k * HW + (size_t)(gi0 + r) * W + (gj0 + q) : 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          Pc[r][q][c] = in ? Elem<T>::raw(pc + (size_t)c * n + o) : T();
          Pp[r][q][c] = (in && beta != 0.f) ? Elem<T>::raw(pp + (size_t)c * n + o) : T();
        }
        Zr[r][q] = in ? __ldg(z + o) : 0.f;
      }
  };
  // r = p_k + beta (p_k - p_{k-1}) and z from the fetched values (cells outside
  // the volume were fetched as zero, which decodes to 0)
  auto make_r = [&](float (&rz)[RPW][CPL], float (&ry)[RPW][CPL], float (&rx)[RPW][CPL],
                    float (&zz)[RPW][CPL]) {
#pragma unroll
    for (int r = 0; r < RPW; ++r)
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        float a[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float cc = Elem<T>::cvt(Pc[r][q][c]);
          a[c] = beta != 0.f ? cc + beta * (cc - Elem<T>::cvt(Pp[r][q][c])) : cc;
        }
        rz[r][q] = a[0];
        ry[r][q] = a[1];
        rx[r][q] = a[2];
        zz[r][q] = Zr[r][q];
      }
  };

  float Zt[RPW][CPL], Dy[RPW][CPL], Dx[RPW][CPL];
  // warm-up: r_z(k0-1) and r(k0), then u(k0)
  load_r(k0 - 1, Rzm, Dy, Dx, Zt, false);
  load_r(k0, Rz, Ry, Rx, Zt, true);
  if constexpr (kPrefetch) fetch(k0 + 1);
  int buf = 0;
#pragma unroll
  for (int q = 0; q < CPL; ++q) sh_ry[buf][warp][lane * CPL + q] = Ry[RPW - 1][q];
  __syncthreads();
  {
    float above[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) above[q] = warp > 0 ? sh_ry[buf][warp - 1][lane * CPL + q] : 0.f;
    form_u(k0, Rz, Ry, Rx, Rzm, Zt, above, Uk);
#pragma unroll
    for (int q = 0; q < CPL; ++q) sh_u[buf][warp][lane * CPL + q] = Uk[0][q];
  }
  for (int k = k0; k < k1; ++k) {
    // next plane: r(k+1), u(k+1)
    float Rz1[RPW][CPL], Ry1[RPW][CPL], Rx1[RPW][CPL], U1[RPW][CPL];
    if constexpr (kPrefetch) {
      make_r(Rz1, Ry1, Rx1, Zt);
      fetch(k + 2);
    } else {
      load_r(k + 1, Rz1, Ry1, Rx1, Zt, true);
    }
    const int nb = buf ^ 1;
#pragma unroll
    for (int q = 0; q < CPL; ++q) sh_ry[nb][warp][lane * CPL + q] = Ry1[RPW - 1][q];
    __syncthreads();
    float above[CPL], below_u[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      above[q] = warp > 0 ? sh_ry[nb][warp - 1][lane * CPL + q] : 0.f;
      below_u[q] = warp < NW - 1 ? sh_u[buf][warp + 1][lane * CPL + q] : 0.f;
    }
    form_u(k + 1, Rz1, Ry1, Rx1, Rz, Zt, above, U1);
#pragma unroll
    for (int q = 0; q < CPL; ++q) sh_u[nb][warp][lane * CPL + q] = U1[0][q];
    // p_{k+1} at plane k
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const float u_right = __shfl_down_sync(0xffffffffu, Uk[r][0], 1);
      const int a = warp * RPW + r;
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        const float uc = Uk[r][q];
        const float dn = r < RPW - 1 ? Uk[r + 1][q] : below_u[q];
        const float rt = q < CPL - 1 ? Uk[r][q + 1] : u_right;
        const float g0 = k < D - 1 ? U1[r][q] - uc : 0.f;
        const float g1 = row_dn[r] ? dn - uc : 0.f;
        const float g2 = col_rt[q] ? rt - uc : 0.f;
        const float q0 = Rz[r][q] + inv_step * g0;
        const float q1 = Ry[r][q] + inv_step * g1;
        const float q2 = Rx[r][q] + inv_step * g2;
        const float nrm2 = q0 * q0 + q1 * q1 + q2 * q2;
        const float sc = nrm2 > 1.f ? rsqrtf(nrm2) : 1.f;
        const int c = lane * CPL + q;
        if (a >= 1 && a <= TH && c >= 1 && c <= TW && row_in[r] && col_in[q]) {
          const size_t o = (size_t)k * HW + (size_t)(gi0 + r) * W + (gj0 + q);
          Elem<T>::st(pn + o, q0 * sc);
          Elem<T>::st(pn + n + o, q1 * sc);
          Elem<T>::st(pn + 2 * n + o, q2 * sc);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RPW; ++r)
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        Rzm[r][q] = Rz[r][q];
        Rz[r][q] = Rz1[r][q];
        Ry[r][q] = Ry1[r][q];
        Rx[r][q] = Rx1[r][q];
        Uk[r][q] = U1[r][q];
      }
    buf = nb;
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
                                    IndexMap im) {
  pdl_enter();
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

// z-marching variants: (columns per lane, rows per warp, planes per chunk);
// TVS_FGP3D_CFG="cpl,rpw,zc" selects one.
template <typename T, bool NN, int CPL, int RPW, int ZC>
cudaError_t fgp3d_zm_launch(const Dims& d, const float* z, const void* pc, const void* pp, void* pn, float lam,
                            float inv_step, float beta, cudaStream_t s) {
  constexpr int TW = 32 * CPL - 2, TH = 8 * RPW - 2;
  dim3 grid((d.nx + TW - 1) / TW, (d.ny + TH - 1) / TH, (d.nz + ZC - 1) / ZC);
  launch_kernel(fgp3d_zm_kernel<T, NN, CPL, RPW, ZC>, dim3(grid), dim3(256), 0, s, z, (const T*)pc, (const T*)pp, (T*)pn, d.nz, d.ny,
                                                             d.nx, lam, inv_step, beta);
  return cudaGetLastError();
}

struct ZmCfg {
  int cpl = 0, rpw = 0, zc = 0;
};
// Defaults: the fastest variant measured at 512^3 for each dual width (FP32:
// 1,2,64; BF16 and FP16: 2,2,32); TVS_FGP3D_CFG overrides both.
ZmCfg fgp3d_zm_cfg(bool half_dual) {
  static const ZmCfg env = [] {
    ZmCfg r;
    if (const char* e = getenv("TVS_FGP3D_CFG")) {
      ZmCfg t;
      if (sscanf(e, "%d,%d,%d", &t.cpl, &t.rpw, &t.zc) == 3) r = t;
    }
    return r;
  }();
  if (env.cpl > 0) return env;
  ZmCfg c;
  c.cpl = half_dual ? 2 : 1;
  c.rpw = 2;
  c.zc = half_dual ? 32 : 64;
  return c;
}

template <typename T, bool NN>
cudaError_t fgp3d_zm_dispatch(const Dims& d, const float* z, const void* pc, const void* pp, void* pn, float lam,
                              float inv_step, float beta, cudaStream_t s) {
  const ZmCfg c = fgp3d_zm_cfg(sizeof(T) == 2);
#define TVS_ZM(C_, R_, Z_) \
  if (c.cpl == C_ && c.rpw == R_ && c.zc == Z_) return fgp3d_zm_launch<T, NN, C_, R_, Z_>(d, z, pc, pp, pn, lam, inv_step, beta, s);
  TVS_ZM(1, 4, 64)
  TVS_ZM(1, 2, 64)
  TVS_ZM(2, 2, 64)
  TVS_ZM(2, 4, 64)
  TVS_ZM(1, 8, 64)
  TVS_ZM(1, 4, 128)
  TVS_ZM(1, 4, 32)
  TVS_ZM(1, 2, 32)
  TVS_ZM(1, 2, 16)
  TVS_ZM(2, 2, 32)
#undef TVS_ZM
  return fgp3d_zm_launch<T, NN, 1, 2, 64>(d, z, pc, pp, pn, lam, inv_step, beta, s);
}

// The z-marching 3D kernel is the default; TVS_FGP3D=tile selects the tiled one.
bool fgp3d_use_zmarch() {
  static const bool zm = [] {
    const char* e = getenv("TVS_FGP3D");
    return !(e && e[0] == 't');
  }();
  return zm;
}

// PDHGSkip-1 finalisation (Algorithm 5 with omega + 1 = 1/p):
// u = P_X(z + lam div p_N); x^ = (u - x) / p; x <- x + p x^ (in place).
template <typename T, bool NONNEG>
__global__ void fgp_finalize_pd1_kernel(const float* __restrict__ z, const T* __restrict__ p, int H, int W,
                                        float lam, float prob_p, float* __restrict__ x,
                                        float* __restrict__ xh, T* __restrict__ p_home, IndexMap im) {
  pdl_enter();
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
  if (d.ndim == 2) {
    dim3 grid((d.nx + TX2 - 1) / TX2, (d.ny + TY2 - 1) / TY2);
    launch_kernel(fgp2d_kernel<T, NN>, dim3(grid), dim3(NT2), 0, s, z, (const T*)pc, (const T*)pp, (T*)pn, d.ny, d.nx, lam,
                                             inv_step, beta);
  } else if (fgp3d_use_zmarch() &&
             (long long)((d.nx + 29) / 30) * ((d.ny + 13) / 14) * ((d.nz + 63) / 64) >= 4 * 152) {
    // z-marching needs enough (x-y tile, z chunk) pairs to fill the GPU; small
    // volumes use the tiled kernel
    const cudaError_t e = fgp3d_zm_dispatch<T, NN>(d, z, pc, pp, pn, lam, inv_step, beta, s);
    if (e != cudaSuccess) return e;
  } else {
    dim3 grid((d.nx + TX3 - 1) / TX3, (d.ny + TY3 - 1) / TY3, (d.nz + TZ3 - 1) / TZ3);
    launch_kernel(fgp3d_kernel<T, NN>, dim3(grid), dim3(NT3), 0, s, z, (const T*)pc, (const T*)pp, (T*)pn, d.nz, d.ny,
                                             d.nx, lam, inv_step, beta);
  }
  return cudaGetLastError();
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
#undef TVS_RB_CASE
  return cudaErrorInvalidValue;
}

template <typename T, bool NN>
cudaError_t fgp_finalize_t(const Dims& d, const float* z, const void* p, float lam, float* x_out,
                           float* h_out, float h_coef, void* p_home, const float* x_prev,
                           float* fista_y, const float* beta_tab, const int* beta_idx, cudaStream_t s) {
  const size_t n = d.n();
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  launch_kernel(fgp_finalize_kernel<T, NN>, dim3(blocks), dim3(256), 0, s, z, (const T*)p, d.nz, d.ny, d.nx, d.ndim, lam,
                                                    x_out, h_out, h_coef, (T*)p_home, x_prev,
                                                    fista_y, beta_tab, beta_idx, IndexMap(d.nz, d.ny, d.nx));
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fgp_iter(const Dims& d, const float* z, const void* pc, const void* pp, void* pn,
                            float lam, float inv_step, float beta, int dtype, bool nonneg,
                            cudaStream_t s) {
  if (d.n() == 0) return cudaSuccess;
  return with_dual_type(dtype, [&](auto tag) {
    using T = typename decltype(tag)::type;
    return nonneg ? fgp_iter_t<T, true>(d, z, pc, pp, pn, lam, inv_step, beta, s)
                  : fgp_iter_t<T, false>(d, z, pc, pp, pn, lam, inv_step, beta, s);
  });
}

cudaError_t launch_fgp_finalize_pd1(const Dims& d, const float* z, const void* p, int dtype, float lam,
                                    bool nonneg, float prob_p, float* x, float* xh, void* p_home,
                                    cudaStream_t s) {
  const size_t n = d.n();
  if (n == 0) return cudaSuccess;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
#define TVS_PD1(T_)                                                                                   \
  if (nonneg)                                                                                         \
    launch_kernel(fgp_finalize_pd1_kernel<T_, true>, dim3(blocks), dim3(256), 0, s, z, (const T_*)p, d.ny, d.nx, lam, prob_p, x, xh, \
                                                             (T_*)p_home, IndexMap(1, d.ny, d.nx));   \
  else                                                                                                \
    launch_kernel(fgp_finalize_pd1_kernel<T_, false>, dim3(blocks), dim3(256), 0, s, z, (const T_*)p, d.ny, d.nx, lam, prob_p, x, xh, \
                                                              (T_*)p_home, IndexMap(1, d.ny, d.nx));
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

bool fgp_config_valid(const FgpConfig& c) {
  if (c.tb <= 1) return true;
  const int ok[][3] = {{2, 2, 4},   {3, 2, 4},   {4, 2, 4},   {4, 2, 5},   {4, 1, 5},   {6, 2, 6},
                       {8, 2, 6},   {2, 2, 104}, {4, 1, 105}, {4, 2, 105}, {4, 2, 108}, {4, 1, 108},
                       {6, 2, 108}, {3, 2, 106}, {4, 2, 104}, {4, 1, 106}};
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

cudaError_t launch_fgp_finalize(const Dims& d, const float* z, const void* p, int dtype, float lam,
                                bool nonneg, float* x_out, float* h_out, float h_coef,
                                void* p_home, const float* x_prev, float* fista_y,
                                const float* beta_tab, const int* beta_idx, cudaStream_t s) {
  if (d.n() == 0) return cudaSuccess;
  return with_dual_type(dtype, [&](auto tag) {
    using T = typename decltype(tag)::type;
    return nonneg ? fgp_finalize_t<T, true>(d, z, p, lam, x_out, h_out, h_coef, p_home, x_prev, fista_y, beta_tab, beta_idx, s)
                  : fgp_finalize_t<T, false>(d, z, p, lam, x_out, h_out, h_coef, p_home, x_prev, fista_y, beta_tab, beta_idx, s);
  });
}

}  // namespace tvs
