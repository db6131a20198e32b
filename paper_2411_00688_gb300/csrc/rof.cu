// ProxSkip (Algorithm 4), projected gradient and its accelerated form on the Dual-ROF problem
// (Section 2.1, Eq. 6) and its Huber-smoothed form (Section 2.2, Eq. 8):
//     min_{|q_i| <= alpha}  F(q) = 1/2 ||div q + b||^2 + (eps / (2 alpha)) ||q||^2,
// grad F(q) = -D(div q + b) + (eps / alpha) q, prox of the constraint = P_C, the
// pointwise projection onto the alpha-ball (Eq. 7).  One fused launch per
// iteration: stage q over the tile plus a one-pixel halo, form w = div q + b on
// the tile plus the row/column after it, then per pixel
//     q^ = q - gamma (grad F(q) - h);
//     prox iteration: q+ = P_C(q^ - (gamma/p) h),  h+ = h + (p/gamma)(q+ - q^);
//     skip iteration: q+ = q^ (h unchanged);
// and the partial sums of F(q) (the current iterate) in the same pass.
#include "common.cuh"
#include "kernels.hpp"

namespace tvs {

namespace {

constexpr int RX = 32, RY = 16, RNT = 256;

template <bool PROX, bool HAS_H>
__global__ void __launch_bounds__(RNT)
dual_rof_step_kernel(const float* __restrict__ q, float* __restrict__ qn, float* __restrict__ h,
                     const float* __restrict__ b, int H, int W, float alpha, float eps_over_alpha,
                     float gamma, float p, Partial* __restrict__ part_a, Partial* __restrict__ part_b,
                     const float* __restrict__ uref, Partial* __restrict__ part_c) {
  pdl_enter();
  __shared__ float sqy[RY + 2][RX + 3];
  __shared__ float sqx[RY + 2][RX + 3];
  __shared__ float sw[RY + 1][RX + 2];
  const int j0 = blockIdx.x * RX, i0 = blockIdx.y * RY;
  const size_t n = (size_t)H * W;
  // q over rows i0-1 .. i0+RY, columns j0-1 .. j0+RX
  for (int e = threadIdx.x; e < (RY + 2) * (RX + 2); e += RNT) {
    const int a = e / (RX + 2), c = e - a * (RX + 2);
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
  // w = div q + b over rows i0 .. i0+RY, columns j0 .. j0+RX
  for (int e = threadIdx.x; e < (RY + 1) * (RX + 1); e += RNT) {
    const int a = e / (RX + 1), c = e - a * (RX + 1);
    const int gi = i0 + a, gj = j0 + c;
    float w = 0.f;
    if (gi < H && gj < W) {
      float dv = 0.f;
      if (gi < H - 1) dv += sqy[a + 1][c + 1];
      if (gi > 0) dv -= sqy[a][c + 1];
      if (gj < W - 1) dv += sqx[a + 1][c + 1];
      if (gj > 0) dv -= sqx[a + 1][c];
      w = dv + __ldg(b + (size_t)gi * W + gj);
    }
    sw[a][c] = w;
  }
  __syncthreads();
  FAcc acc_a, acc_b, acc_c;
  const float step_h = gamma / p, inv_step_h = p / gamma;
  for (int e = threadIdx.x; e < RY * RX; e += RNT) {
    const int a = e / RX, c = e - a * RX;
    const int gi = i0 + a, gj = j0 + c;
    if (gi >= H || gj >= W) continue;
    const size_t o = (size_t)gi * W + gj;
    const float wc = sw[a][c];
    const float qy = sqy[a + 1][c + 1], qx = sqx[a + 1][c + 1];
    // grad F = -D w + (eps/alpha) q
    const float gy = -(gi < H - 1 ? sw[a + 1][c] - wc : 0.f) + eps_over_alpha * qy;
    const float gx = -(gj < W - 1 ? sw[a][c + 1] - wc : 0.f) + eps_over_alpha * qx;
    float hy = 0.f, hx = 0.f;
    if (HAS_H) {
      hy = h[o];
      hx = h[n + o];
    }
    const float ty = qy - gamma * (gy - hy), tx = qx - gamma * (gx - hx);  // q^
    float ny = ty, nx = tx;
    if (PROX) {
      const float vy = ty - step_h * hy, vx = tx - step_h * hx;
      const float nrm = sqrtf(vy * vy + vx * vx);
      const float sc = alpha / fmaxf(alpha, nrm);
      ny = vy * sc;
      nx = vx * sc;
      if (HAS_H) {
        h[o] = hy + inv_step_h * (ny - ty);
        h[n + o] = hx + inv_step_h * (nx - tx);
      }
    }
    qn[o] = ny;
    qn[n + o] = nx;
    acc_a.add(0.5f * (wc * wc));
    acc_b.add(0.5f * (qy * qy + qx * qx));
    if (uref) {
      const float d = wc - __ldg(uref + o);  // u_k = b + div q_k against the reference
      acc_c.add(d * d);
    }
  }
  block_sum2_store<RNT>(acc_a, acc_b, part_a, part_b, blockIdx.y * gridDim.x + blockIdx.x);
  if (uref) {
    __syncthreads();  // the reduction's shared staging is reused
    block_sum2_store<RNT>(acc_c, FAcc(), part_c, nullptr, blockIdx.y * gridDim.x + blockIdx.x);
  }
}

// AProjGD (Section 2.2): the projected gradient step of Algorithm 2 from the
// extrapolated point of Algorithm 3,
//     y = q_k + beta_k (q_k - q_{k-1}),   q_{k+1} = P_C(y - gamma grad F(y)),
// with beta_k read from a device table at the iteration counter the objective
// record keeps (so one captured graph serves every iteration); the partial sums
// of F(q_k) of the current iterate come out of the same pass.
__global__ void __launch_bounds__(RNT)
dual_rof_accel_kernel(const float* __restrict__ q, const float* __restrict__ qp, float* __restrict__ qn,
                      const float* __restrict__ b, int H, int W, float alpha, float eps_over_alpha,
                      float gamma, const float* __restrict__ beta_tab, const int* __restrict__ beta_idx,
                      Partial* __restrict__ part_a, Partial* __restrict__ part_b,
                      const float* __restrict__ uref, Partial* __restrict__ part_c) {
  pdl_enter();
  __shared__ float sqy[RY + 2][RX + 3];
  __shared__ float sqx[RY + 2][RX + 3];
  __shared__ float syy[RY + 2][RX + 3];
  __shared__ float syx[RY + 2][RX + 3];
  __shared__ float swq[RY + 1][RX + 2];
  __shared__ float swy[RY + 1][RX + 2];
  const float beta = beta_tab[*beta_idx + 1];
  const int j0 = blockIdx.x * RX, i0 = blockIdx.y * RY;
  const size_t n = (size_t)H * W;
  // q and y over rows i0-1 .. i0+RY, columns j0-1 .. j0+RX
  for (int e = threadIdx.x; e < (RY + 2) * (RX + 2); e += RNT) {
    const int a = e / (RX + 2), c = e - a * (RX + 2);
    const int gi = i0 - 1 + a, gj = j0 - 1 + c;
    float vy = 0.f, vx = 0.f, yy = 0.f, yx = 0.f;
    if (gi >= 0 && gi < H && gj >= 0 && gj < W) {
      const size_t o = (size_t)gi * W + gj;
      vy = __ldg(q + o);
      vx = __ldg(q + n + o);
      yy = vy + beta * (vy - __ldg(qp + o));
      yx = vx + beta * (vx - __ldg(qp + n + o));
    }
    sqy[a][c] = vy;
    sqx[a][c] = vx;
    syy[a][c] = yy;
    syx[a][c] = yx;
  }
  __syncthreads();
  // w = div q + b and w_y = div y + b over rows i0 .. i0+RY, columns j0 .. j0+RX
  for (int e = threadIdx.x; e < (RY + 1) * (RX + 1); e += RNT) {
    const int a = e / (RX + 1), c = e - a * (RX + 1);
    const int gi = i0 + a, gj = j0 + c;
    float w = 0.f, wy = 0.f;
    if (gi < H && gj < W) {
      float dv = 0.f, dy = 0.f;
      if (gi < H - 1) {
        dv += sqy[a + 1][c + 1];
        dy += syy[a + 1][c + 1];
      }
      if (gi > 0) {
        dv -= sqy[a][c + 1];
        dy -= syy[a][c + 1];
      }
      if (gj < W - 1) {
        dv += sqx[a + 1][c + 1];
        dy += syx[a + 1][c + 1];
      }
      if (gj > 0) {
        dv -= sqx[a + 1][c];
        dy -= syx[a + 1][c];
      }
      const float bb = __ldg(b + (size_t)gi * W + gj);
      w = dv + bb;
      wy = dy + bb;
    }
    swq[a][c] = w;
    swy[a][c] = wy;
  }
  __syncthreads();
  FAcc acc_a, acc_b, acc_c;
  for (int e = threadIdx.x; e < RY * RX; e += RNT) {
    const int a = e / RX, c = e - a * RX;
    const int gi = i0 + a, gj = j0 + c;
    if (gi >= H || gj >= W) continue;
    const size_t o = (size_t)gi * W + gj;
    const float wc = swy[a][c];
    const float yy = syy[a + 1][c + 1], yx = syx[a + 1][c + 1];
    // grad F(y) = -D w_y + (eps/alpha) y
    const float gy = -(gi < H - 1 ? swy[a + 1][c] - wc : 0.f) + eps_over_alpha * yy;
    const float gx = -(gj < W - 1 ? swy[a][c + 1] - wc : 0.f) + eps_over_alpha * yx;
    const float vy = yy - gamma * gy, vx = yx - gamma * gx;
    const float nrm = sqrtf(vy * vy + vx * vx);
    const float sc = alpha / fmaxf(alpha, nrm);
    qn[o] = vy * sc;
    qn[n + o] = vx * sc;
    const float wq = swq[a][c], qy = sqy[a + 1][c + 1], qx = sqx[a + 1][c + 1];
    acc_a.add(0.5f * (wq * wq));
    acc_b.add(0.5f * (qy * qy + qx * qx));
    if (uref) {
      const float d = wq - __ldg(uref + o);
      acc_c.add(d * d);
    }
  }
  block_sum2_store<RNT>(acc_a, acc_b, part_a, part_b, blockIdx.y * gridDim.x + blockIdx.x);
  if (uref) {
    __syncthreads();
    block_sum2_store<RNT>(acc_c, FAcc(), part_c, nullptr, blockIdx.y * gridDim.x + blockIdx.x);
  }
}

// u = b + div q and the objective partials of the final iterate.
__global__ void __launch_bounds__(RNT)
dual_rof_primal_kernel(const float* __restrict__ q, const float* __restrict__ b, float* __restrict__ u,
                       int H, int W, Partial* __restrict__ part_a, Partial* __restrict__ part_b,
                       const float* __restrict__ uref, Partial* __restrict__ part_c) {
  pdl_enter();
  const size_t n = (size_t)H * W;
  FAcc acc_a, acc_b, acc_c;
  for (size_t o = blockIdx.x * (size_t)RNT + threadIdx.x; o < n; o += (size_t)gridDim.x * RNT) {
    const int gj = (int)(o % W), gi = (int)(o / W);
    float dv = 0.f;
    if (gi < H - 1) dv += __ldg(q + o);
    if (gi > 0) dv -= __ldg(q + o - W);
    if (gj < W - 1) dv += __ldg(q + n + o);
    if (gj > 0) dv -= __ldg(q + n + o - 1);
    const float w = dv + __ldg(b + o);
    if (u) u[o] = w;
    const float qy = __ldg(q + o), qx = __ldg(q + n + o);
    acc_a.add(0.5f * (w * w));
    acc_b.add(0.5f * (qy * qy + qx * qx));
    if (uref) {
      const float d = w - __ldg(uref + o);
      acc_c.add(d * d);
    }
  }
  block_sum2_store<RNT>(acc_a, acc_b, part_a, part_b, blockIdx.x);
  if (uref) {
    __syncthreads();
    block_sum2_store<RNT>(acc_c, FAcc(), part_c, nullptr, blockIdx.x);
  }
}

}  // namespace

int dual_rof_blocks(int H, int W) { return ((W + RX - 1) / RX) * ((H + RY - 1) / RY); }

cudaError_t launch_dual_rof_step(int H, int W, const float* q, float* qn, float* h, const float* b,
                                 float alpha, float eps, float gamma, float p, bool prox,
                                 Partial* part_a, Partial* part_b, const float* uref, Partial* part_c,
                                 cudaStream_t s) {
  dim3 grid((W + RX - 1) / RX, (H + RY - 1) / RY);
  const float ea = alpha > 0.f ? eps / alpha : 0.f;
  if (prox) {
    if (h) launch_kernel(dual_rof_step_kernel<true, true>, dim3(grid), dim3(RNT), 0, s, q, qn, h, b, H, W, alpha, ea, gamma, p, part_a, part_b, uref, part_c);
    else launch_kernel(dual_rof_step_kernel<true, false>, dim3(grid), dim3(RNT), 0, s, q, qn, h, b, H, W, alpha, ea, gamma, p, part_a, part_b, uref, part_c);
  } else {
    if (h) launch_kernel(dual_rof_step_kernel<false, true>, dim3(grid), dim3(RNT), 0, s, q, qn, h, b, H, W, alpha, ea, gamma, p, part_a, part_b, uref, part_c);
    else launch_kernel(dual_rof_step_kernel<false, false>, dim3(grid), dim3(RNT), 0, s, q, qn, h, b, H, W, alpha, ea, gamma, p, part_a, part_b, uref, part_c);
  }
  return cudaGetLastError();
}

cudaError_t launch_dual_rof_accel_step(int H, int W, const float* q, const float* q_prev, float* qn,
                                       const float* b, float alpha, float eps, float gamma,
                                       const float* beta_tab, const int* beta_idx, Partial* part_a,
                                       Partial* part_b, const float* uref, Partial* part_c, cudaStream_t s) {
  dim3 grid((W + RX - 1) / RX, (H + RY - 1) / RY);
  const float ea = alpha > 0.f ? eps / alpha : 0.f;
  launch_kernel(dual_rof_accel_kernel, dim3(grid), dim3(RNT), 0, s, q, q_prev, qn, b, H, W, alpha, ea, gamma,
                beta_tab, beta_idx, part_a, part_b, uref, part_c);
  return cudaGetLastError();
}

cudaError_t launch_dual_rof_primal(int H, int W, const float* q, const float* b, float* u, Partial* part_a,
                                   Partial* part_b, const float* uref, Partial* part_c, cudaStream_t s) {
  launch_kernel(dual_rof_primal_kernel, dim3(pointwise_blocks((size_t)H * W)), dim3(RNT), 0, s, q, b, u, H, W, part_a,
                part_b, uref, part_c);
  return cudaGetLastError();
}

}  // namespace tvs
