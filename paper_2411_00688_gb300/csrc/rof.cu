// ProxSkip (Algorithm 4) and projected gradient on the Dual-ROF problem
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
                     float gamma, float p, Partial* __restrict__ part_a, Partial* __restrict__ part_b) {
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
  FAcc acc_a, acc_b;
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
  }
  block_sum2_store<RNT>(acc_a, acc_b, part_a, part_b, blockIdx.y * gridDim.x + blockIdx.x);
}

// u = b + div q and the objective partials of the final iterate.
__global__ void __launch_bounds__(RNT)
dual_rof_primal_kernel(const float* __restrict__ q, const float* __restrict__ b, float* __restrict__ u,
                       int H, int W, Partial* __restrict__ part_a, Partial* __restrict__ part_b) {
  pdl_enter();
  const size_t n = (size_t)H * W;
  FAcc acc_a, acc_b;
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
  }
  block_sum2_store<RNT>(acc_a, acc_b, part_a, part_b, blockIdx.x);
}

}  // namespace

int dual_rof_blocks(int H, int W) { return ((W + RX - 1) / RX) * ((H + RY - 1) / RY); }

cudaError_t launch_dual_rof_step(int H, int W, const float* q, float* qn, float* h, const float* b,
                                 float alpha, float eps, float gamma, float p, bool prox,
                                 Partial* part_a, Partial* part_b, cudaStream_t s) {
  dim3 grid((W + RX - 1) / RX, (H + RY - 1) / RY);
  const float ea = alpha > 0.f ? eps / alpha : 0.f;
  if (prox) {
    if (h) launch_kernel(dual_rof_step_kernel<true, true>, dim3(grid), dim3(RNT), 0, s, q, qn, h, b, H, W, alpha, ea, gamma, p, part_a, part_b);
    else launch_kernel(dual_rof_step_kernel<true, false>, dim3(grid), dim3(RNT), 0, s, q, qn, h, b, H, W, alpha, ea, gamma, p, part_a, part_b);
  } else {
    if (h) launch_kernel(dual_rof_step_kernel<false, true>, dim3(grid), dim3(RNT), 0, s, q, qn, h, b, H, W, alpha, ea, gamma, p, part_a, part_b);
    else launch_kernel(dual_rof_step_kernel<false, false>, dim3(grid), dim3(RNT), 0, s, q, qn, h, b, H, W, alpha, ea, gamma, p, part_a, part_b);
  }
  return cudaGetLastError();
}

cudaError_t launch_dual_rof_primal(int H, int W, const float* q, const float* b, float* u, Partial* part_a,
                                   Partial* part_b, cudaStream_t s) {
  launch_kernel(dual_rof_primal_kernel, dim3(pointwise_blocks((size_t)H * W)), dim3(RNT), 0, s, q, b, u, H, W, part_a, part_b);
  return cudaGetLastError();
}

}  // namespace tvs
