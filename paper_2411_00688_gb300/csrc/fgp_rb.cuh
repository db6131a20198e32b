// Register-blocked temporally blocked FGP body for 2D images, shared by the
// single-problem kernel (fgp_tb.cu) and the batched kernel (batch.cu).
#pragma once

#include "common.cuh"

namespace tvs {

// b[0]: momentum coefficient forming r for the first iteration of a launch;
// b[t]: for iteration t+1.
struct TBBetas {
  float b[8];
};

// ---------------------------------------------------------------------------
// Register-blocked temporally blocked 2D variant.  Same staged region and the
// same per-iteration arithmetic as fgp2d_tb_kernel, but every cell lives in the
// registers of one thread for the whole launch: warp w owns RPW consecutive
// region rows, lane l owns CPL adjacent columns.  Horizontal neighbours come
// from warp shuffles, vertical neighbours from the thread's own registers; only
// the row shared by two warps goes through shared memory (one row of r before
// phase 1, one row of u before phase 2).  Cells are updated unconditionally:
// values in the shrinking halo are stale but finite and never reach a cell of
// the valid region (masks keep out-of-image cells out of in-image stencils).
// INTERIOR: the whole staged region lies in rows/columns 1 .. n-2, so every
// Neumann mask is true and the masked terms are dropped (same arithmetic).
template <typename T, bool NONNEG, int TB, int CPL, int RPW, bool INTERIOR>
__device__ __forceinline__ void fgp2d_rb_body_impl(const float* __restrict__ z, const T* __restrict__ pc,
                                                   const T* __restrict__ pp, T* __restrict__ pn,
                                                   T* __restrict__ pnp, int H, int W, float lam,
                                                   float inv_step, const TBBetas& betas, int iters,
                                                   int tile_x, int tile_y) {
  constexpr int NW = 8;
  constexpr int RW = 32 * CPL, RH = NW * RPW;
  constexpr int TW = RW - 2 * TB, TH = RH - 2 * TB;
  __shared__ float edge_ry[NW][RW];  // bottom row of r_y of each warp's block
  __shared__ float edge_u[NW][RW];   // top row of u of each warp's block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gi0 = tile_y * TH - TB + warp * RPW;   // global row of the thread's first cell
  const int gj0 = tile_x * TW - TB + lane * CPL;   // global column of its first cell
  const size_t n = (size_t)H * W;

  float Z[RPW][CPL], Ry[RPW][CPL], Rx[RPW][CPL], Py[RPW][CPL], Px[RPW][CPL], U[RPW][CPL];
  // boundary masks: row masks per row, column masks per column (Neumann)
  bool row_in[RPW], row_dn[RPW], row_up[RPW], col_in[CPL], col_rt[CPL], col_lf[CPL];
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const int gi = gi0 + r;
    row_in[r] = INTERIOR || (gi >= 0 && gi < H);
    row_dn[r] = INTERIOR || gi < H - 1;   // has a row below (D_y defined, div uses p_y here)
    row_up[r] = INTERIOR || gi > 0;       // has a row above (div uses p_y of the row above)
  }
#pragma unroll
  for (int q = 0; q < CPL; ++q) {
    const int gj = gj0 + q;
    col_in[q] = INTERIOR || (gj >= 0 && gj < W);
    col_rt[q] = INTERIOR || gj < W - 1;
    col_lf[q] = INTERIOR || gj > 0;
  }
  const float b0 = betas.b[0];
#pragma unroll
  for (int r = 0; r < RPW; ++r)
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      float zz = 0.f, cy = 0.f, cx = 0.f, ry = 0.f, rx = 0.f;
      if (row_in[r] && col_in[q]) {
        const size_t o = (size_t)(gi0 + r) * W + (gj0 + q);
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
      Z[r][q] = zz;
      Py[r][q] = cy;
      Px[r][q] = cx;
      Ry[r][q] = ry;
      Rx[r][q] = rx;
    }
#pragma unroll
  for (int q = 0; q < CPL; ++q) edge_ry[warp][lane * CPL + q] = Ry[RPW - 1][q];
  __syncthreads();

  for (int t = 1; t <= iters; ++t) {
    // phase 1: U = P_X(Z + lam div R)
    float ry_above[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) ry_above[q] = warp > 0 ? edge_ry[warp - 1][lane * CPL + q] : 0.f;
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const float rx_left = __shfl_up_sync(0xffffffffu, Rx[r][CPL - 1], 1);
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        const float up = r > 0 ? Ry[r - 1][q] : ry_above[q];
        const float lf = q > 0 ? Rx[r][q - 1] : rx_left;
        float dv = 0.f;
        if (row_dn[r]) dv += Ry[r][q];
        if (row_up[r]) dv -= up;
        if (col_rt[q]) dv += Rx[r][q];
        if (col_lf[q]) dv -= lf;
        float u = Z[r][q] + lam * dv;
        if (NONNEG) u = fmaxf(u, 0.f);
        U[r][q] = (row_in[r] && col_in[q]) ? u : 0.f;
      }
    }
#pragma unroll
    for (int q = 0; q < CPL; ++q) edge_u[warp][lane * CPL + q] = U[0][q];
    __syncthreads();
    // phase 2: p_new = P_B(R + inv_step D U); R = next momentum point (or p_prev); P = p_new
    const bool last = (t == iters);
    const float bn = last ? 0.f : betas.b[t];
    float u_below[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) u_below[q] = warp < NW - 1 ? edge_u[warp + 1][lane * CPL + q] : 0.f;
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const float u_right = __shfl_down_sync(0xffffffffu, U[r][0], 1);
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        const float uc = U[r][q];
        const float dn = r < RPW - 1 ? U[r + 1][q] : u_below[q];
        const float rt = q < CPL - 1 ? U[r][q + 1] : u_right;
        const float gy = row_dn[r] ? dn - uc : 0.f;
        const float gx = col_rt[q] ? rt - uc : 0.f;
        const float qy = Ry[r][q] + inv_step * gy;
        const float qx = Rx[r][q] + inv_step * gx;
        const float nrm2 = __fmaf_rn(qy, qy, __fmul_rn(qx, qx));
        const float sc = fminf(1.f, rsqrtf(nrm2));  // 1 / max(1, |q|): rsqrt(n2) < 1 iff n2 > 1
        const float ny = Elem<T>::round(qy * sc), nx = Elem<T>::round(qx * sc);
        const float oy = Py[r][q], ox = Px[r][q];
        if (last) {
          Ry[r][q] = oy;
          Rx[r][q] = ox;
        } else {
          Ry[r][q] = ny + bn * (ny - oy);
          Rx[r][q] = nx + bn * (nx - ox);
        }
        Py[r][q] = ny;
        Px[r][q] = nx;
      }
    }
    if (!last) {
#pragma unroll
      for (int q = 0; q < CPL; ++q) edge_ry[warp][lane * CPL + q] = Ry[RPW - 1][q];
    }
    __syncthreads();
  }
  // tile interior: P = p_{k+iters}, R = p_{k+iters-1}
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const int a = warp * RPW + r;
    if (a < TB || a >= TB + TH || !row_in[r]) continue;
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      const int c = lane * CPL + q;
      if (c < TB || c >= TB + TW || !col_in[q]) continue;
      const size_t o = (size_t)(gi0 + r) * W + (gj0 + q);
      Elem<T>::st(pn + o, Py[r][q]);
      Elem<T>::st(pn + n + o, Px[r][q]);
      Elem<T>::st(pnp + o, Ry[r][q]);
      Elem<T>::st(pnp + n + o, Rx[r][q]);
    }
  }
}

// ---------------------------------------------------------------------------
// The two-columns-per-lane layout with packed FP32x2 arithmetic (Blackwell's
// paired FMA/ADD/MUL): a lane's two cells of a row form one float2 (left column
// in .x), so each step of the iteration above is one paired instruction instead
// of two.  The per-value arithmetic is unchanged (a - b is formed as
// fma(b, -1, a), which rounds exactly like the subtraction; a masked-out term is
// added as zero instead of skipped, which changes no value), so it agrees bitwise
// with the scalar body.  The Neumann masks are split by direction: ROWM keeps the
// row masks (the region meets the first or last image row), COLM the column masks
// (first or last column); a region meeting neither is the interior case.  u is not
// masked outside the image: an in-image cell reads u only of in-image cells (the
// differences toward the last row / column are masked), and outside values never
// reach an in-image cell (the div terms from row -1 / column -1 are masked), so
// they stay finite and unused.
__device__ __forceinline__ float2 p2_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 p2_mask(float2 v, bool mx, bool my) {
  return make_float2(mx ? v.x : 0.f, my ? v.y : 0.f);
}

template <typename T, bool NONNEG, int TB, int RPW, bool ROWM, bool COLM>
__device__ __forceinline__ void fgp2d_rb_body_packed(const float* __restrict__ z, const T* __restrict__ pc,
                                                     const T* __restrict__ pp, T* const& pn, T* const& pnp,
                                                     const int& H, const int& W, float lam, float inv_step,
                                                     const TBBetas& betas, int iters, const int& tile_x,
                                                     const int& tile_y) {
  constexpr int NW = 8, CPL = 2;
  constexpr int RW = 32 * CPL, RH = NW * RPW;
  constexpr int TW = RW - 2 * TB, TH = RH - 2 * TB;
  __shared__ float2 edge_ry2[NW][32];
  __shared__ float2 edge_u2[NW][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gi0 = tile_y * TH - TB + warp * RPW;
  const int gj0 = tile_x * TW - TB + lane * CPL;
  const size_t n = (size_t)H * W;
  float2 Z[RPW], Ry[RPW], Rx[RPW], Py[RPW], Px[RPW], U[RPW];
  bool row_in[RPW], row_dn[RPW], row_up[RPW];
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const int gi = gi0 + r;
    row_in[r] = !ROWM || (gi >= 0 && gi < H);
    row_dn[r] = !ROWM || gi < H - 1;
    row_up[r] = !ROWM || gi > 0;
  }
  // column masks of the lane's left (.x) and right (.y) cell
  const bool in0 = !COLM || (gj0 >= 0 && gj0 < W), in1 = !COLM || (gj0 + 1 >= 0 && gj0 + 1 < W);
  const bool rt0 = !COLM || gj0 < W - 1, rt1 = !COLM || gj0 + 1 < W - 1;
  const bool lf0 = !COLM || gj0 > 0, lf1 = !COLM || gj0 + 1 > 0;
  const float b0 = betas.b[0];
  const float2 bb = make_float2(b0, b0);
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    float2 zz = make_float2(0.f, 0.f), cy = zz, cx = zz, qy = zz, qx = zz;
    const size_t o = (size_t)(gi0 + r) * W + gj0;
    if (row_in[r]) {
      if (in0) {
        zz.x = __ldg(z + o);
        cy.x = Elem<T>::ld(pc + o);
        cx.x = Elem<T>::ld(pc + n + o);
        if (b0 != 0.f) {
          qy.x = Elem<T>::ld(pp + o);
          qx.x = Elem<T>::ld(pp + n + o);
        }
      }
      if (in1) {
        zz.y = __ldg(z + o + 1);
        cy.y = Elem<T>::ld(pc + o + 1);
        cx.y = Elem<T>::ld(pc + n + o + 1);
        if (b0 != 0.f) {
          qy.y = Elem<T>::ld(pp + o + 1);
          qx.y = Elem<T>::ld(pp + n + o + 1);
        }
      }
    }
    Z[r] = zz;
    Py[r] = cy;
    Px[r] = cx;
    if (b0 != 0.f) {
      Ry[r] = __ffma2_rn(bb, p2_sub(cy, qy), cy);
      Rx[r] = __ffma2_rn(bb, p2_sub(cx, qx), cx);
    } else {
      Ry[r] = cy;
      Rx[r] = cx;
    }
  }
  edge_ry2[warp][lane] = Ry[RPW - 1];
  __syncthreads();
  const float2 lam2 = make_float2(lam, lam), inv2 = make_float2(inv_step, inv_step);
  for (int t = 1; t <= iters; ++t) {
    // phase 1: U = P_X(Z + lam div R), div R = Ry - Ry(above) + Rx - Rx(left)
    const float2 ry_above = warp > 0 ? edge_ry2[warp - 1][lane] : make_float2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const float rx_left = __shfl_up_sync(0xffffffffu, Rx[r].y, 1);
      const float2 up = r > 0 ? Ry[r - 1] : ry_above;
      const float2 lf = make_float2(rx_left, Rx[r].x);
      float2 ry = Ry[r], upv = up, rx = Rx[r], lfv = lf;
      if (ROWM) {
        ry = p2_mask(ry, row_dn[r], row_dn[r]);
        upv = p2_mask(upv, row_up[r], row_up[r]);
      }
      if (COLM) {
        rx = p2_mask(rx, rt0, rt1);
        lfv = p2_mask(lfv, lf0, lf1);
      }
      float2 dv = p2_sub(ry, upv);
      dv = __fadd2_rn(dv, rx);
      dv = p2_sub(dv, lfv);
      float2 u = __ffma2_rn(lam2, dv, Z[r]);
      if (NONNEG) u = make_float2(fmaxf(u.x, 0.f), fmaxf(u.y, 0.f));
      U[r] = u;
    }
    edge_u2[warp][lane] = U[0];
    __syncthreads();
    // phase 2: p_new = P_B(R + inv_step D U); R = next momentum point (or p_prev); P = p_new
    const bool last = (t == iters);
    const float bn = last ? 0.f : betas.b[t];
    const float2 bn2 = make_float2(bn, bn);
    const float2 u_below = warp < NW - 1 ? edge_u2[warp + 1][lane] : make_float2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const float u_right = __shfl_down_sync(0xffffffffu, U[r].x, 1);
      const float2 uc = U[r];
      const float2 dn = r < RPW - 1 ? U[r + 1] : u_below;
      const float2 rt = make_float2(uc.y, u_right);
      float2 gy = p2_sub(dn, uc), gx = p2_sub(rt, uc);
      if (ROWM) gy = p2_mask(gy, row_dn[r], row_dn[r]);
      if (COLM) gx = p2_mask(gx, rt0, rt1);
      const float2 qy = __ffma2_rn(inv2, gy, Ry[r]);
      const float2 qx = __ffma2_rn(inv2, gx, Rx[r]);
      const float2 nrm2 = __ffma2_rn(qy, qy, __fmul2_rn(qx, qx));
      const float2 sc = make_float2(fminf(1.f, rsqrtf(nrm2.x)), fminf(1.f, rsqrtf(nrm2.y)));
      float2 ny = __fmul2_rn(qy, sc), nx = __fmul2_rn(qx, sc);
      ny = Elem<T>::round2(ny);
      nx = Elem<T>::round2(nx);
      if (last) {
        Ry[r] = Py[r];
        Rx[r] = Px[r];
      } else {
        Ry[r] = __ffma2_rn(bn2, p2_sub(ny, Py[r]), ny);
        Rx[r] = __ffma2_rn(bn2, p2_sub(nx, Px[r]), nx);
      }
      Py[r] = ny;
      Px[r] = nx;
    }
    if (!last) edge_ry2[warp][lane] = Ry[RPW - 1];
    __syncthreads();
  }
  // The store phase takes the tile's geometry and destinations afresh through the
  // references (kernel parameters, or a shared-memory tile record read after the
  // last barrier), so none of them stays live in registers across the iterations.
  const int Hs = H, Ws = W;
  const size_t ns = (size_t)Hs * Ws;
  const int gi0s = tile_y * TH - TB + warp * RPW, gj0s = tile_x * TW - TB + lane * CPL;
  T* const dst_p = pn;
  T* const dst_r = pnp;
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const int a = warp * RPW + r, gi = gi0s + r;
    if (a < TB || a >= TB + TH || (ROWM && (gi < 0 || gi >= Hs))) continue;
    const size_t o = (size_t)gi * Ws + gj0s;
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      const int c = lane * CPL + q, gj = gj0s + q;
      if (c < TB || c >= TB + TW || (COLM && (gj < 0 || gj >= Ws))) continue;
      Elem<T>::st(dst_p + o + q, q ? Py[r].y : Py[r].x);
      Elem<T>::st(dst_p + ns + o + q, q ? Px[r].y : Px[r].x);
      Elem<T>::st(dst_r + o + q, q ? Ry[r].y : Ry[r].x);
      Elem<T>::st(dst_r + ns + o + q, q ? Rx[r].y : Rx[r].x);
    }
  }
}

// pn, pnp, H, W and the tile coordinates are taken by reference: the two-column
// body reads them again for its store phase (see there).
template <typename T, bool NONNEG, int TB, int CPL, int RPW>
__device__ __forceinline__ void fgp2d_rb_body(const float* __restrict__ z, const T* __restrict__ pc,
                                              const T* __restrict__ pp, T* const& pn, T* const& pnp,
                                              const int& H, const int& W, float lam, float inv_step,
                                              const TBBetas& betas, int iters, const int& tile_x,
                                              const int& tile_y) {
  constexpr int RW = 32 * CPL, RH = 8 * RPW, TW = RW - 2 * TB, TH = RH - 2 * TB;
  const int r0 = tile_y * TH - TB, c0 = tile_x * TW - TB;
  const bool rows_in = r0 >= 1 && r0 + RH <= H - 1, cols_in = c0 >= 1 && c0 + RW <= W - 1;
  const bool interior = rows_in && cols_in;
  if constexpr (CPL == 2) {
    if (interior)
      fgp2d_rb_body_packed<T, NONNEG, TB, RPW, false, false>(z, pc, pp, pn, pnp, H, W, lam, inv_step, betas,
                                                             iters, tile_x, tile_y);
    else if (cols_in)
      fgp2d_rb_body_packed<T, NONNEG, TB, RPW, true, false>(z, pc, pp, pn, pnp, H, W, lam, inv_step, betas,
                                                            iters, tile_x, tile_y);
    else if (rows_in)
      fgp2d_rb_body_packed<T, NONNEG, TB, RPW, false, true>(z, pc, pp, pn, pnp, H, W, lam, inv_step, betas,
                                                            iters, tile_x, tile_y);
    else
      fgp2d_rb_body_packed<T, NONNEG, TB, RPW, true, true>(z, pc, pp, pn, pnp, H, W, lam, inv_step, betas,
                                                           iters, tile_x, tile_y);
  } else {
    if (interior)
      fgp2d_rb_body_impl<T, NONNEG, TB, CPL, RPW, true>(z, pc, pp, pn, pnp, H, W, lam, inv_step, betas, iters,
                                                        tile_x, tile_y);
    else
      fgp2d_rb_body_impl<T, NONNEG, TB, CPL, RPW, false>(z, pc, pp, pn, pnp, H, W, lam, inv_step, betas, iters,
                                                         tile_x, tile_y);
  }
}

}  // namespace tvs
