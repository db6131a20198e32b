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
//   r = A x - b on the tile plus an R-cell ring, the ring cells outside the image
//   copied from their mirror cells (the reflective A reads r there), then
//   out = x - gamma A r + ch h on the tile, with the partials of 1/2 ||r||^2 and
//   TV(x) over the tile.  The arithmetic of every output value is the residual
//   kernel's followed by the step kernel's (same taps, same order); only the
//   residual never leaves shared memory.
// Layout: every lane owns two adjacent columns (one float2) in every pass, so a
// tap is one packed FP32x2 FMA and a horizontal pass reads R + 1 float2 per two
// outputs; the staged region is 64 columns wide, the tile fb_tile_w(R) =
// 64 - 4R columns by fb_tile_h(R) rows: 40 rows up to radius 6 (a 1024^2 image is
// then 572 tiles of radius 4, one wave of four CTAs per SM, where 32 rows gave
// 704 tiles and a second wave of 96), 32 beyond (the staged rows of 40 would
// pass the 48 KB of static shared memory).
constexpr int FNT = 256;
__host__ __device__ constexpr int fb_tile_w(int R) { return 64 - 4 * R; }
__host__ __device__ constexpr int fb_tile_h(int R) { return R <= 6 ? 40 : 32; }

// Two adjacent taps positions: (v[c], v[c + 1]) for even c is one float2; for odd
// c it straddles two.
template <int K>
__device__ __forceinline__ float2 fb_pair(const float2* v) {
  return (K & 1) ? make_float2(v[K / 2].y, v[K / 2 + 1].x) : v[K / 2];
}
template <int R, int K = 0>
__device__ __forceinline__ float2 fb_taps(const float2* v, const float* wk, float2 acc) {
  if constexpr (K > 2 * R) {
    return acc;
  } else {
    acc = __ffma2_rn(make_float2(wk[K], wk[K]), fb_pair<K>(v), acc);
    return fb_taps<R, K + 1>(v, wk, acc);
  }
}

// IN: the staged region (rows i0 - 2R .. i0 + FY + 2R, columns j0 - 2R ..
// j0 - 2R + 63) lies inside the image, so no index is reflected, every residual
// cell is in the image and no Neumann mask of the TV term applies; the checks are
// dropped and the arithmetic is unchanged.
template <int R, bool IN>
__device__ __forceinline__ void blur_fb_step_body_impl(const float* __restrict__ x, const float* __restrict__ b,
                                                       const float* __restrict__ h, float* __restrict__ out, int H,
                                                       int W, const BlurW& w, float gamma, float ch,
                                                       Partial* __restrict__ part_a, Partial* __restrict__ part_b,
                                                       int tile_x, int tile_y, int part_index,
                                                       float2 (*__restrict__ sx)[32], float2 (*__restrict__ sh)[32],
                                                       float2 (*__restrict__ sr)[32]) {
  constexpr int FX = fb_tile_w(R), FY = fb_tile_h(R);
  constexpr int XR = FY + 4 * R;                   // staged x: rows i0-2R .., columns j0-2R .. j0-2R+63
  constexpr int RR = FY + 2 * R;                   // residual region rows i0-R .., columns j0-R .. j0+FX+R
  constexpr int NW = FNT / 32;                     // warps; lane = column pair, warp = row phase
  constexpr int RP = 32 - R, OP = 32 - 2 * R;      // column pairs of the residual region / of the tile
  constexpr int VR = (RR + NW - 1) / NW;           // residual rows per warp (vertical pass)
  constexpr int VO = FY / NW;                      // output rows per warp (final pass)
  static_assert(FY % NW == 0 && R >= 1 && R <= 8, "tile layout");
  // shared memory (the caller's): sx[XR] staged x, sh[XR] horizontal pass of x and
  // later of r, sr[RR] the residual
  float wk[2 * R + 1];
#pragma unroll
  for (int k = 0; k <= 2 * R; ++k) wk[k] = w.w[k];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int j0 = tile_x * FX, i0 = tile_y * FY;
  {
    const int gj0 = IN ? j0 - 2 * R + 2 * lane : reflect_index(j0 - 2 * R + 2 * lane, W);
    const int gj1 = IN ? gj0 + 1 : reflect_index(j0 - 2 * R + 2 * lane + 1, W);
#pragma unroll
    for (int t = 0; t < (XR + NW - 1) / NW; ++t) {
      const int a = wp + NW * t;
      if (a < XR) {
        const float* row = x + (size_t)(IN ? i0 - 2 * R + a : reflect_index(i0 - 2 * R + a, H)) * W;
        sx[a][lane] = make_float2(__ldg(row + gj0), __ldg(row + gj1));
      }
    }
  }
  // the b values the vertical pass needs, issued now so that they arrive during
  // the horizontal pass
  float2 bv[VR];
  {
    const int a0 = wp * VR, gj = j0 - R + 2 * lane;
    const bool cin0 = IN || (gj >= 0 && gj < W), cin1 = IN || (gj + 1 >= 0 && gj + 1 < W);
#pragma unroll
    for (int t = 0; t < VR; ++t) {
      const int gi = i0 - R + a0 + t;
      const bool rin = lane < RP && a0 + t < RR && (IN || (gi >= 0 && gi < H));
      const float* brow = b + (size_t)(rin ? gi : 0) * W;
      bv[t] = make_float2(rin && cin0 ? __ldg(brow + gj) : 0.f, rin && cin1 ? __ldg(brow + gj + 1) : 0.f);
    }
  }
  __syncthreads();
  // horizontal pass of x over all staged rows, output columns 2m, 2m+1 < 64 - 2R
#pragma unroll
  for (int t = 0; t < (XR + NW - 1) / NW; ++t) {
    const int a = wp + NW * t;
    if (a < XR && lane < RP) {
      float2 v[R + 1];
#pragma unroll
      for (int j = 0; j <= R; ++j) v[j] = sx[a][lane + j];
      sh[a][lane] = fb_taps<R>(v, wk, make_float2(0.f, 0.f));
    }
  }
  __syncthreads();
  // vertical pass -> r = A x - b on the in-image cells of the residual region;
  // each warp owns VR consecutive rows and slides a register window down them
  FAcc acc_a, acc_b;
  if (lane < RP) {
    const int a0 = wp * VR;
    float2 win[VR + 2 * R];
#pragma unroll
    for (int t = 0; t < VR + 2 * R; ++t) win[t] = a0 + t < XR ? sh[a0 + t][lane] : make_float2(0.f, 0.f);
    const int gj = j0 - R + 2 * lane;  // global column of the pair's left cell
    const bool cin0 = IN || (gj >= 0 && gj < W), cin1 = IN || (gj + 1 >= 0 && gj + 1 < W);
    const bool own0 = 2 * lane >= R && 2 * lane < R + FX, own1 = 2 * lane + 1 >= R && 2 * lane + 1 < R + FX;
#pragma unroll
    for (int t = 0; t < VR; ++t) {
      const int a = a0 + t;
      const int gi = i0 - R + a;
      if (a >= RR || (!IN && (gi < 0 || gi >= H))) continue;
      float2 v = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k <= 2 * R; ++k) v = __ffma2_rn(make_float2(wk[k], wk[k]), win[t + k], v);
      float2 r = make_float2(0.f, 0.f);
      if (cin0) r.x = v.x - bv[t].x;
      if (cin1) r.y = v.y - bv[t].y;
      sr[a][lane] = r;
      if (a >= R && a < R + FY) {
        if (cin0 && own0) acc_a.add(0.5f * (r.x * r.x));
        if (cin1 && own1) acc_a.add(0.5f * (r.y * r.y));
      }
    }
  }
  __syncthreads();
  // ring cells outside the image take their mirror cell's residual
  if (!IN && (i0 < R || j0 < R || i0 + FY + R > H || j0 + FX + R > W)) {
    float* srf = &sr[0][0].x;  // row stride 64 floats
    for (int a = wp; a < RR; a += NW) {
      const int gi = i0 - R + a;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int c = 2 * lane + q;
        if (c >= 2 * RP) continue;
        const int gj = j0 - R + c;
        if (gi >= 0 && gi < H && gj >= 0 && gj < W) continue;
        srf[a * 64 + c] = srf[(reflect_index(gi, H) - (i0 - R)) * 64 + (reflect_index(gj, W) - (j0 - R))];
      }
    }
  }
  __syncthreads();
  // horizontal pass of r, output columns 2m, 2m+1 < FX
#pragma unroll
  for (int t = 0; t < (RR + NW - 1) / NW; ++t) {
    const int a = wp + NW * t;
    if (a < RR && lane < OP) {
      float2 v[R + 1];
#pragma unroll
      for (int j = 0; j <= R; ++j) v[j] = sr[a][lane + j];
      sh[a][lane] = fb_taps<R>(v, wk, make_float2(0.f, 0.f));
    }
  }
  __syncthreads();
  if (lane < OP) {
    const int a0 = wp * VO;
    float2 win[VO + 2 * R];
#pragma unroll
    for (int t = 0; t < VO + 2 * R; ++t) win[t] = sh[a0 + t][lane];
    const int gj = j0 + 2 * lane;
    float2 hv[VO];  // the control variate of the pair's cells, loaded up front
#pragma unroll
    for (int t = 0; t < VO; ++t) {
      const int gi = i0 + a0 + t;
      const size_t o = (size_t)(IN || gi < H ? gi : 0) * W + gj;
      hv[t] = make_float2(h && out && (IN || (gi < H && gj < W)) ? __ldg(h + o) : 0.f,
                          h && out && (IN || (gi < H && gj + 1 < W)) ? __ldg(h + o + 1) : 0.f);
    }
#pragma unroll
    for (int t = 0; t < VO; ++t) {
      const int a = a0 + t;
      const int gi = i0 + a;
      if (!IN && gi >= H) continue;
      float2 v = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k <= 2 * R; ++k) v = __ffma2_rn(make_float2(wk[k], wk[k]), win[t + k], v);
      const float2 xc = sx[a + 2 * R][lane + R];
      const float2 xd = sx[a + 2 * R + 1][lane + R];
      const float xr = sx[a + 2 * R][lane + R + 1].x;  // right neighbour of the pair's right cell
      const size_t o = (size_t)gi * W + gj;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (!IN && gj + q >= W) continue;
        const float xq = q ? xc.y : xc.x, vq = q ? v.y : v.x;
        if (out) {
          float o_v = xq - gamma * vq;
          if (h) o_v = fmaf(ch, q ? hv[t].y : hv[t].x, o_v);
          out[o + q] = o_v;
        }
        const float dy = IN || gi < H - 1 ? (q ? xd.y : xd.x) - xq : 0.f;
        const float dx = IN || gj + q < W - 1 ? (q ? xr : xc.y) - xq : 0.f;
        acc_b.add(tv_term(0.f, dy, dx));
      }
    }
  }
  block_sum2_store<FNT>(acc_a, acc_b, part_a, part_b, part_index);
}

template <int R>
__device__ __forceinline__ void blur_fb_step_body(const float* __restrict__ x, const float* __restrict__ b,
                                                  const float* __restrict__ h, float* __restrict__ out, int H,
                                                  int W, const BlurW& w, float gamma, float ch,
                                                  Partial* __restrict__ part_a, Partial* __restrict__ part_b,
                                                  int tile_x, int tile_y, int part_index) {
  constexpr int FY = fb_tile_h(R), XR = FY + 4 * R, RR = FY + 2 * R;
  __shared__ float2 sx[XR][32];
  __shared__ float2 sh[XR][32];
  __shared__ float2 sr[RR][32];
  const int i0 = tile_y * FY, j0 = tile_x * fb_tile_w(R);
  const bool in = i0 >= 2 * R && i0 + FY + 2 * R <= H && j0 >= 2 * R && j0 - 2 * R + 64 <= W;
  if (in)
    blur_fb_step_body_impl<R, true>(x, b, h, out, H, W, w, gamma, ch, part_a, part_b, tile_x, tile_y, part_index,
                                    sx, sh, sr);
  else
    blur_fb_step_body_impl<R, false>(x, b, h, out, H, W, w, gamma, ch, part_a, part_b, tile_x, tile_y, part_index,
                                     sx, sh, sr);
}

}  // namespace tvs
