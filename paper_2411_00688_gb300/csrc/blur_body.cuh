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

// Fused forward-backward step for the blur operator (A = A^T):
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
  __shared__ float sx[XR][XC + 1];
  __shared__ float sh[XR][RC + 1];  // horizontal pass of x, later of r
  __shared__ float sr[RR][RC + 1];
  float wk[2 * R + 1];
#pragma unroll
  for (int k = 0; k <= 2 * R; ++k) wk[k] = w.w[k];
  const int j0 = tile_x * FX, i0 = tile_y * FY;
  for (int e = threadIdx.x; e < XR * XC; e += FNT) {
    const int a = e / XC, c = e - a * XC;
    const int gi = reflect_index(i0 - 2 * R + a, H), gj = reflect_index(j0 - 2 * R + c, W);
    sx[a][c] = __ldg(x + (size_t)gi * W + gj);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < XR * RC; e += FNT) {
    const int a = e / RC, c = e - a * RC;
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) acc = fmaf(wk[k], sx[a][c + k], acc);
    sh[a][c] = acc;
  }
  __syncthreads();
  FAcc acc_a, acc_b;
  for (int e = threadIdx.x; e < RR * RC; e += FNT) {
    const int a = e / RC, c = e - a * RC;
    const int gi = i0 - R + a, gj = j0 - R + c;
    if (gi < 0 || gi >= H || gj < 0 || gj >= W) continue;
    float v = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) v = fmaf(wk[k], sh[a + k][c], v);
    const float r = v - __ldg(b + (size_t)gi * W + gj);
    sr[a][c] = r;
    if (a >= R && a < R + FY && c >= R && c < R + FX) acc_a.add(0.5f * (r * r));
  }
  __syncthreads();
  for (int e = threadIdx.x; e < RR * RC; e += FNT) {
    const int a = e / RC, c = e - a * RC;
    const int gi = i0 - R + a, gj = j0 - R + c;
    if (gi >= 0 && gi < H && gj >= 0 && gj < W) continue;
    sr[a][c] = sr[reflect_index(gi, H) - (i0 - R)][reflect_index(gj, W) - (j0 - R)];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < RR * FX; e += FNT) {
    const int a = e / FX, c = e - a * FX;
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) acc = fmaf(wk[k], sr[a][c + k], acc);
    sh[a][c] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < FY * FX; e += FNT) {
    const int a = e / FX, c = e - a * FX;
    const int gi = i0 + a, gj = j0 + c;
    if (gi >= H || gj >= W) continue;
    float v = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) v = fmaf(wk[k], sh[a + k][c], v);
    const size_t o = (size_t)gi * W + gj;
    const float xc = sx[a + 2 * R][c + 2 * R];
    float o_v = xc - gamma * v;
    if (h) o_v = fmaf(ch, __ldg(h + o), o_v);
    out[o] = o_v;
    const float dy = gi < H - 1 ? sx[a + 2 * R + 1][c + 2 * R] - xc : 0.f;
    const float dx = gj < W - 1 ? sx[a + 2 * R][c + 2 * R + 1] - xc : 0.f;
    acc_b.add(tv_term(0.f, dy, dx));
  }
  block_sum2_store<FNT>(acc_a, acc_b, part_a, part_b, part_index);
}

}  // namespace tvs
