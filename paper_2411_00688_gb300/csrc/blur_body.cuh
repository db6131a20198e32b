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
                                               float* __restrict__ y, float tau, double* __restrict__ part_a,
                                               double* __restrict__ part_b, int tile_x, int tile_y,
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
  double acc_a = 0.0, acc_b = 0.0;
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
      acc_a += 0.5 * (double)(r * r);
      // TV of the blurred image's source x = src, from the staged tile
      const float xc = s_in[a + R][c + R];
      const float dy = gi < H - 1 ? s_in[a + R + 1][c + R] - xc : 0.f;
      const float dx = gj < W - 1 ? s_in[a + R][c + R + 1] - xc : 0.f;
      acc_b += (double)tv_term(0.f, dy, dx);
    } else if (MODE == BM_STEP) {
      float o_v = __ldg(x + o) - gamma * v;
      if (h) o_v = fmaf(ch, __ldg(h + o), o_v);
      out[o] = o_v;
      if (part_b) acc_b += (double)tv_at_2d(x, gi, gj, H, W);
    } else if (MODE == BM_PD) {
      const float bb = __ldg(b + o);
      const float prev = axp[o];
      const float yn = (y[o] + tau * (2.f * v - prev) - tau * bb) / (1.f + tau);
      y[o] = yn;
      axp[o] = v;
      const float r = v - bb;
      acc_a += 0.5 * (double)(r * r);
    } else if (MODE == BM_PD1) {
      // v = A x^; A x_{k+1} = A x_k + p A x^ (A x_k in axp); y <- prox(y + tau A(x_{k+1} + x^))
      const float bb = __ldg(b + o);
      const float axn = axp[o] + gamma * v;  // gamma carries p here
      y[o] = (y[o] + tau * (axn + v) - tau * bb) / (1.f + tau);
      axp[o] = axn;
      const float r = axn - bb;
      acc_a += 0.5 * (double)(r * r);
    } else {
      out[o] = v;
    }
  }
  if (part_a || part_b)
    block_sum2_store<BNT>(acc_a, acc_b, part_a, part_b, part_index);
}

}  // namespace tvs
