// Explicit PDHG with diagonal preconditioning (the explicit formulation of
// Section 3.2; the solver behind the reference solutions of Section 4.1, with the
// step sizes of Pock and Chambolle, ICCV 2011, Lemma 2 with exponent 1).
//
// K = [A; D], dual variables y (one per row of A) and q (one 2-vector per pixel),
// f(v, w) = 1/2 ||v - b||^2 + alpha sum_i |w_i|_2, g = 0 or the indicator of x >= 0:
//     x+  = P_X(x - T (A^T y - div q))           T_j = sigma / sum_i |K_ij|
//     x-  = 2 x+ - x
//     y+  = (y + S_i (A x- - b)) / (1 + S_i)     S_i = tau / sum_j |A_ij|
//     q+  = P_alpha(q + (tau/2) D x-)            (every row of D has entries -1, +1)
// Every operator here has non-negative entries, so the column and row sums of |A|
// are A^T 1 and A 1; column j of D holds one entry per difference touching pixel j.
// An empty row or column takes the bare scale (the matching entries of K are zero).
//
// One iteration = A^T y (operator kernel), the fused TV step below (x+, q+, and the
// TV partials of x), A x+ (operator kernel), and the pointwise dual step, where
// A x- = 2 A x+ - A x comes from the stored A x (no extra operator application).
#include "common.cuh"
#include "kernels.hpp"

namespace tvs {

namespace {

constexpr int QX = 32, QY = 16, QNT = 256;
constexpr int PW = 256;

__global__ void __launch_bounds__(PW)
pdx_precond_kernel(const float* __restrict__ colA, const float* __restrict__ rowA, int H, int W, size_t m,
                   float sigma, float tau, float* __restrict__ T, float* __restrict__ S) {
  pdl_enter();
  const size_t n = (size_t)H * W, total = n > m ? n : m;
  for (size_t o = blockIdx.x * (size_t)PW + threadIdx.x; o < total; o += (size_t)gridDim.x * PW) {
    if (o < n) {
      const int gj = (int)(o % W), gi = (int)(o / W);
      const int nb = (gi < H - 1) + (gi > 0) + (gj < W - 1) + (gj > 0);
      const float c = (colA ? colA[o] : 1.f) + (float)nb;
      T[o] = c > 0.f ? sigma / c : sigma;
    }
    if (o < m) {
      const float r = rowA ? rowA[o] : 1.f;
      S[o] = r > 0.f ? tau / r : tau;
    }
  }
}

__global__ void __launch_bounds__(PW) fill_kernel(float* __restrict__ a, size_t n, float v) {
  pdl_enter();
  for (size_t o = blockIdx.x * (size_t)PW + threadIdx.x; o < n; o += (size_t)gridDim.x * PW) a[o] = v;
}

// Fused TV part of one iteration on a QY x QX tile: q staged over the tile plus one
// row/column on each side, x+ and x- over the tile plus the row/column after it,
// then q+ on the tile.  part_tv gets the TV partials of the incoming x.
template <bool NONNEG>
__global__ void __launch_bounds__(QNT)
pdx_tv_step_kernel(const float* __restrict__ x, const float* __restrict__ g, const float* __restrict__ T,
                   const float* __restrict__ q, float* __restrict__ xn, float* __restrict__ qn, int H, int W,
                   float alpha, float s_d, Partial* __restrict__ part_tv) {
  pdl_enter();
  __shared__ float sqy[QY + 2][QX + 3];
  __shared__ float sqx[QY + 2][QX + 3];
  __shared__ float sxb[QY + 1][QX + 2];  // x- = 2 x+ - x
  __shared__ float sxc[QY + 1][QX + 2];  // incoming x
  const int j0 = blockIdx.x * QX, i0 = blockIdx.y * QY;
  const size_t n = (size_t)H * W;
  for (int e = threadIdx.x; e < (QY + 2) * (QX + 2); e += QNT) {
    const int a = e / (QX + 2), c = e - a * (QX + 2);
    const int gi = i0 - 1 + a, gj = j0 - 1 + c;
    float vy = 0.f, vx = 0.f;
    if (gi >= 0 && gi < H && gj >= 0 && gj < W) {
      const size_t o = (size_t)gi * W + gj;
      vy = __ldg(q + o);
      vx = __ldg(q + n + o);
    }
    sqy[a][c] = vy;
    sqx[a][c] = vx;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < (QY + 1) * (QX + 1); e += QNT) {
    const int a = e / (QX + 1), c = e - a * (QX + 1);
    const int gi = i0 + a, gj = j0 + c;
    float xb = 0.f, xc = 0.f;
    if (gi < H && gj < W) {
      const size_t o = (size_t)gi * W + gj;
      // div q = -D^T q (Neumann): q_y(i) [i < H-1] - q_y(i-1) [i > 0] + the same along x
      float dv = 0.f;
      if (gi < H - 1) dv += sqy[a + 1][c + 1];
      if (gi > 0) dv -= sqy[a][c + 1];
      if (gj < W - 1) dv += sqx[a + 1][c + 1];
      if (gj > 0) dv -= sqx[a + 1][c];
      xc = __ldg(x + o);
      float xp = xc - __ldg(T + o) * (__ldg(g + o) - dv);
      if (NONNEG) xp = fmaxf(xp, 0.f);
      xb = 2.f * xp - xc;
      if (a < QY && c < QX) xn[o] = xp;
    }
    sxb[a][c] = xb;
    sxc[a][c] = xc;
  }
  __syncthreads();
  FAcc acc;
  for (int e = threadIdx.x; e < QY * QX; e += QNT) {
    const int a = e / QX, c = e - a * QX;
    const int gi = i0 + a, gj = j0 + c;
    if (gi >= H || gj >= W) continue;
    const size_t o = (size_t)gi * W + gj;
    const float dy = gi < H - 1 ? sxb[a + 1][c] - sxb[a][c] : 0.f;
    const float dx = gj < W - 1 ? sxb[a][c + 1] - sxb[a][c] : 0.f;
    const float vy = sqy[a + 1][c + 1] + s_d * dy, vx = sqx[a + 1][c + 1] + s_d * dx;
    float sc = 0.f;
    if (alpha > 0.f) sc = alpha / fmaxf(alpha, sqrtf(vy * vy + vx * vx));
    qn[o] = vy * sc;
    qn[n + o] = vx * sc;
    const float ty = gi < H - 1 ? sxc[a + 1][c] - sxc[a][c] : 0.f;
    const float tx = gj < W - 1 ? sxc[a][c + 1] - sxc[a][c] : 0.f;
    acc.add(tv_term(0.f, ty, tx));
  }
  block_sum2_store<QNT>(FAcc(), acc, nullptr, part_tv, blockIdx.y * gridDim.x + blockIdx.x);
}

// y+ = (y + S (2 A x+ - A x - b)) / (1 + S); A x <- A x+; data partials of x+.
// INIT: only A x <- A x+ and the partials (the first iterate).
template <bool INIT>
__global__ void __launch_bounds__(PW)
pdx_dual_kernel(size_t m, const float* __restrict__ ax, float* __restrict__ axp, float* __restrict__ y,
                const float* __restrict__ b, const float* __restrict__ S, Partial* __restrict__ part_a) {
  pdl_enter();
  FAcc acc;
  for (size_t o = blockIdx.x * (size_t)PW + threadIdx.x; o < m; o += (size_t)gridDim.x * PW) {
    const float v = __ldg(ax + o), bb = __ldg(b + o);
    if (!INIT) {
      const float s = __ldg(S + o);
      const float xb = 2.f * v - axp[o];
      y[o] = (y[o] + s * (xb - bb)) / (1.f + s);
    }
    axp[o] = v;
    const float r = v - bb;
    acc.add(0.5f * (r * r));
  }
  block_sum2_store<PW>(acc, FAcc(), part_a, nullptr, blockIdx.x);
}

}  // namespace

int pdx_tv_blocks(int H, int W) { return ((W + QX - 1) / QX) * ((H + QY - 1) / QY); }

cudaError_t launch_pdx_precond(const float* colA, const float* rowA, int H, int W, size_t m, float sigma,
                               float tau, float* T, float* S, cudaStream_t s) {
  const size_t n = (size_t)H * W;
  launch_kernel(pdx_precond_kernel, dim3(pointwise_blocks(n > m ? n : m)), dim3(PW), 0, s, colA, rowA, H, W, m, sigma, tau, T, S);
  return cudaGetLastError();
}

cudaError_t launch_fill(float* a, size_t n, float v, cudaStream_t s) {
  launch_kernel(fill_kernel, dim3(pointwise_blocks(n)), dim3(PW), 0, s, a, n, v);
  return cudaGetLastError();
}

cudaError_t launch_pdx_tv_step(int H, int W, const float* x, const float* g, const float* T, const float* q,
                               float* xn, float* qn, float alpha, float s_d, bool nonneg, Partial* part_tv,
                               cudaStream_t s) {
  dim3 grid((W + QX - 1) / QX, (H + QY - 1) / QY);
  if (nonneg) launch_kernel(pdx_tv_step_kernel<true>, dim3(grid), dim3(QNT), 0, s, x, g, T, q, xn, qn, H, W, alpha, s_d, part_tv);
  else launch_kernel(pdx_tv_step_kernel<false>, dim3(grid), dim3(QNT), 0, s, x, g, T, q, xn, qn, H, W, alpha, s_d, part_tv);
  return cudaGetLastError();
}

cudaError_t launch_pdx_dual(size_t m, const float* ax, float* axp, float* y, const float* b, const float* S,
                            bool init, Partial* part_a, cudaStream_t s) {
  if (init) launch_kernel(pdx_dual_kernel<true>, dim3(pointwise_blocks(m)), dim3(PW), 0, s, m, ax, axp, y, b, S, part_a);
  else launch_kernel(pdx_dual_kernel<false>, dim3(pointwise_blocks(m)), dim3(PW), 0, s, m, ax, axp, y, b, S, part_a);
  return cudaGetLastError();
}

}  // namespace tvs
