// Separable blur tile body (9x9 Gaussian etc.) with its epilogues, shared by the
// single-problem kernels (ops.cu) and the batched kernels (batch.cu).
#pragma once

#include "common.cuh"
#include "kernels.hpp"

namespace tvs {

constexpr int BX = 32, BY = 16, BNT = 256, RMAX = 8;

enum BlurMode { BM_RESID = 0, BM_STEP = 1, BM_PD = 2, BM_PLAIN = 3, BM_PD1 = 4 };

// TV term |(D x)_(gi,gj)| from global memory (Neumann: zero last differences).
__device__ __forceinline__ float tv_at_2d(const float* __restrict__ x, int gi, int gj, int H, int W) {
  const size_t o = (size_t)gi * W + gj;
  const float c = __ldg(x + o);
  const float dy = gi < H - 1 ? __ldg(x + o + W) - c : 0.f;
  const float dx = gj < W - 1 ? __ldg(x + o + 1) - c : 0.f;
  return tv_term(0.f, dy, dx);
}

// R: blur radius (compile time, so the tap loops unroll and the weights stay in
// registers).
template <int MODE, int R>
__device__ __forceinline__ void blur_tile_body(const float* __restrict__ src, int H, int W, const BlurW& w,
                                               const float* __restrict__ b, float* __restrict__ out,
                                               const float* __restrict__ x, const float* __restrict__ h,
                                               float gamma, float ch, float* __restrict__ axp,
                                               float* __restrict__ y, float tau, Partial* __restrict__ part_a,
                                               Partial* __restrict__ part_b, int tile_x, int tile_y,
                                               int part_index) {
  __shared__ float s_in[BY + 2 * RMAX][BX + 2 * RMAX + 1];
  __shared__ float s_tmp[BY + 2 * RMAX][BX + 1];
  float wk[2 * R + 1];
#pragma unroll
  for (int k = 0; k <= 2 * R; ++k) wk[k] = w.w[k];
  const int j0 = tile_x * BX, i0 = tile_y * BY;
  const int rows = BY + 2 * R, cols = BX + 2 * R;
  for (int e = threadIdx.x; e < rows * cols; e += BNT) {
    const int a = e / cols, c = e - a * cols;
    const int gi = reflect_index(i0 - R + a, H), gj = reflect_index(j0 - R + c, W);
    s_in[a][c] = __ldg(src + (size_t)gi * W + gj);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rows * BX; e += BNT) {
    const int a = e / BX, c = e - a * BX;
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) acc = fmaf(wk[k], s_in[a][c + k], acc);
    s_tmp[a][c] = acc;
  }
  __syncthreads();
  FAcc acc_a, acc_b;
  for (int e = threadIdx.x; e < BY * BX; e += BNT) {
    const int a = e / BX, c = e - a * BX;
    const int gi = i0 + a, gj = j0 + c;
    if (gi >= H || gj >= W) continue;
    float v = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) v = fmaf(wk[k], s_tmp[a + k][c], v);
    const size_t o = (size_t)gi * W + gj;
    if (MODE == BM_RESID) {
      const float r = v - __ldg(b + o);
      if (out) out[o] = r;
      acc_a.add(0.5f * (r * r));
      // TV of the blurred image's source x = src, from the staged tile
      const float xc = s_in[a + R][c + R];
      const float dy = gi < H - 1 ? s_in[a + R + 1][c + R] - xc : 0.f;
      const float dx = gj < W - 1 ? s_in[a + R][c + R + 1] - xc : 0.f;
      acc_b.add(tv_term(0.f, dy, dx));
    } else if (MODE == BM_STEP) {
      float o_v = __ldg(x + o) - gamma * v;
      if (h) o_v = fmaf(ch, __ldg(h + o), o_v);
      out[o] = o_v;
      if (part_b) acc_b.add(tv_at_2d(x, gi, gj, H, W));
    } else if (MODE == BM_PD) {
      const float bb = __ldg(b + o);
      const float prev = axp[o];
      const float yn = (y[o] + tau * (2.f * v - prev) - tau * bb) / (1.f + tau);
      y[o] = yn;
      axp[o] = v;
      const float r = v - bb;
      acc_a.add(0.5f * (r * r));
    } else if (MODE == BM_PD1) {
      // v = A x^; A x_{k+1} = A x_k + p A x^ (A x_k in axp); y <- prox(y + tau A(x_{k+1} + x^))
      const float bb = __ldg(b + o);
      const float axn = axp[o] + gamma * v;  // gamma carries p here
      y[o] = (y[o] + tau * (axn + v) - tau * bb) / (1.f + tau);
      axp[o] = axn;
      const float r = axn - bb;
      acc_a.add(0.5f * (r * r));
    } else {
      out[o] = v;
    }
  }
  if (part_a || part_b)
    block_sum2_store<BNT>(acc_a, acc_b, part_a, part_b, part_index);
}

// Fused forward-backward step for the blur operator (A = A^T) (out may be null:
// partials only):
//   r = A x - b on the FX x FY tile plus an R-cell ring, the ring cells outside the
//   image copied from their mirror cells (the reflective A reads r there), then
//   out = x - gamma A r + ch h on the tile, with the partials of 1/2 ||r||^2 and
//   TV(x) over the tile.  The arithmetic of every output value is the residual
//   kernel's followed by the step kernel's (same taps, same order); only the
//   residual never leaves shared memory.
constexpr int FX = 32, FY = 32, FNT = 256;

template <int R>
__device__ __forceinline__ void blur_fb_step_body(const float* __restrict__ x, const float* __restrict__ b,
                                                  const float* __restrict__ h, float* __restrict__ out, int H,
                                                  int W, const BlurW& w, float gamma, float ch,
                                                  Partial* __restrict__ part_a, Partial* __restrict__ part_b,
                                                  int tile_x, int tile_y, int part_index) {
  constexpr int XR = FY + 4 * R, XC = FX + 4 * R;  // staged x: rows/cols i0-2R .. i0+FY+2R
  constexpr int RR = FY + 2 * R, RC = FX + 2 * R;  // residual region: i0-R .. i0+FY+R
  constexpr int NW = FNT / 32;                     // warps; lane = column, warp = row phase
  constexpr int VR = (RR + NW - 1) / NW;           // residual rows per warp (vertical pass)
  constexpr int VO = FY / NW;                      // output rows per warp (final pass)
  static_assert(FX == 32 && FY % NW == 0, "tile layout");
  __shared__ float sx[XR][XC + 1];
  __shared__ float sh[XR][RC + 1];  // horizontal pass of x, later of r
  __shared__ float sr[RR][RC + 1];
  float wk[2 * R + 1];
#pragma unroll
  for (int k = 0; k <= 2 * R; ++k) wk[k] = w.w[k];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int j0 = tile_x * FX, i0 = tile_y * FY;
  const bool c1x = lane + 32 < XC, c1r = lane + 32 < RC;  // second column of a lane
  {
    const int gj0 = reflect_index(j0 - 2 * R + lane, W);
    const int gj1 = c1x ? reflect_index(j0 - 2 * R + lane + 32, W) : 0;
#pragma unroll
    for (int t = 0; t < (XR + NW - 1) / NW; ++t) {
      const int a = wp + NW * t;
      if (a < XR) {
        const float* row = x + (size_t)reflect_index(i0 - 2 * R + a, H) * W;
        sx[a][lane] = __ldg(row + gj0);
        if (c1x) sx[a][lane + 32] = __ldg(row + gj1);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < (XR + NW - 1) / NW; ++t) {
    const int a = wp + NW * t;
    if (a < XR) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * R; ++k) acc = fmaf(wk[k], sx[a][lane + k], acc);
      sh[a][lane] = acc;
      if (c1r) {
        float acc1 = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * R; ++k) acc1 = fmaf(wk[k], sx[a][lane + 32 + k], acc1);
        sh[a][lane + 32] = acc1;
      }
    }
  }
  __syncthreads();
  // vertical pass -> r = A x - b on the in-image cells of the residual region; each
  // warp owns VR consecutive rows and slides a register window down its columns
  FAcc acc_a, acc_b;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int c = lane + 32 * half;
    if (half == 1 && !c1r) break;
    const int a0 = wp * VR;
    float win[VR + 2 * R];
#pragma unroll
    for (int t = 0; t < VR + 2 * R; ++t) win[t] = a0 + t < XR ? sh[a0 + t][c] : 0.f;
    const int gj = j0 - R + c;
#pragma unroll
    for (int t = 0; t < VR; ++t) {
      const int a = a0 + t;
      const int gi = i0 - R + a;
      if (a >= RR || gi < 0 || gi >= H || gj < 0 || gj >= W) continue;
      float v = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * R; ++k) v = fmaf(wk[k], win[t + k], v);
      const float r = v - __ldg(b + (size_t)gi * W + gj);
      sr[a][c] = r;
      if (a >= R && a < R + FY && c >= R && c < R + FX) acc_a.add(0.5f * (r * r));
    }
  }
  __syncthreads();
  // ring cells outside the image take their mirror cell's residual
  if (i0 < R || j0 < R || i0 + FY + R > H || j0 + FX + R > W) {
    for (int a = wp; a < RR; a += NW) {
      const int gi = i0 - R + a;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int c = lane + 32 * half;
        if (c >= RC) continue;
        const int gj = j0 - R + c;
        if (gi >= 0 && gi < H && gj >= 0 && gj < W) continue;
        sr[a][c] = sr[reflect_index(gi, H) - (i0 - R)][reflect_index(gj, W) - (j0 - R)];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < (RR + NW - 1) / NW; ++t) {
    const int a = wp + NW * t;
    if (a < RR) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * R; ++k) acc = fmaf(wk[k], sr[a][lane + k], acc);
      sh[a][lane] = acc;
    }
  }
  __syncthreads();
  {
    const int a0 = wp * VO;
    float win[VO + 2 * R];
#pragma unroll
    for (int t = 0; t < VO + 2 * R; ++t) win[t] = sh[a0 + t][lane];
    const int gj = j0 + lane;
#pragma unroll
    for (int t = 0; t < VO; ++t) {
      const int a = a0 + t;
      const int gi = i0 + a;
      if (gi >= H || gj >= W) continue;
      float v = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * R; ++k) v = fmaf(wk[k], win[t + k], v);
      const size_t o = (size_t)gi * W + gj;
      const float xc = sx[a + 2 * R][lane + 2 * R];
      if (out) {
        float o_v = xc - gamma * v;
        if (h) o_v = fmaf(ch, __ldg(h + o), o_v);
        out[o] = o_v;
      }
      const float dy = gi < H - 1 ? sx[a + 2 * R + 1][lane + 2 * R] - xc : 0.f;
      const float dx = gj < W - 1 ? sx[a + 2 * R][lane + 2 * R + 1] - xc : 0.f;
      acc_b.add(tv_term(0.f, dy, dx));
    }
  }
  block_sum2_store<FNT>(acc_a, acc_b, part_a, part_b, part_index);
}

}  // namespace tvs
