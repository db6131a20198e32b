// Parallel-beam projector in Joseph's discretisation (the discrete Radon transform
// of Section 3.3) and its exact transpose, with the PDHGSkip-2 epilogues fused.
//
// Geometry: an N x N image of pixel size s centred at the origin; angle a is
// theta = a pi / n_angles; bin b is the line x cos + y sin = t_b with
// t_b = (b - (n_det-1)/2) d.  A ray with |cos| >= |sin| is walked row by row,
// otherwise column by column ("line" l); on line l it crosses the fractional
// pixel coordinate
//     fr(b, l) = (t_b - c_l m1) inv + (N-1)/2,   c_l = (l - (N-1)/2) s,
// with m1 = sin, inv = 1/(cos s) for row walks and m1 = cos, inv = 1/(sin s) for
// column walks.  The sample is (1-f) u[k0] + f u[k0+1], k0 = floor(fr), f = fr - k0,
// pixels outside the image being zero, and every sample has weight
// s / max(|cos|, |sin|).
//
// Both kernels evaluate fr with the same explicit FMA sequence (joseph_fr), so
// the backprojector applies bit-identical weights: it is the exact transpose of
// the projector up to the order of floating-point summation.  The projector
// reads column-walked angles from a transposed copy of the image so that both
// kinds of walk read image rows.
#include "common.cuh"
#include "kernels.hpp"

namespace tvs {

namespace {

constexpr int CT_NT = 256;

struct GeomConsts {
  int N, n_angles, n_det;
  float s, t0, d, c0, half;  // t_b = b d + t0; c_l = l s + c0; half = (N-1)/2
};

__device__ __forceinline__ float joseph_fr(const GeomConsts& g, float4 ang, int b, int l) {
  const float tb = __fmaf_rn((float)b, g.d, g.t0);
  const float cl = __fmaf_rn((float)l, g.s, g.c0);
  return __fmaf_rn(__fmaf_rn(-cl, ang.x, tb), ang.y, g.half);
}

__global__ void transpose_kernel(const float* __restrict__ x, float* __restrict__ xt, int N) {
  pdl_enter();
  __shared__ float tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = by + r, j = bx + threadIdx.x;
    if (i < N && j < N) tile[r][threadIdx.x] = x[(size_t)i * N + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = bx + r, j = by + threadIdx.x;
    if (i < N && j < N) xt[(size_t)i * N + j] = tile[threadIdx.x][r];
  }
}

// mode 0: sino = A x.  mode 1: PDHG dual epilogue (sino holds A x_prev on entry).
// mode 2: sino = A x, partials of 1/2 (A x - b)^2.  mode 3: sino = A x - b, same partials.
template <int MODE>
__global__ void __launch_bounds__(CT_NT)
joseph_fwd_kernel(GeomConsts g, const float4* __restrict__ angles, const float* __restrict__ x,
                  const float* __restrict__ xt, float* __restrict__ sino, float* __restrict__ y,
                  const float* __restrict__ b, float tau, Partial* __restrict__ part, float tau2 = 0.f) {
  pdl_enter();
  const int ray = blockIdx.x * CT_NT + threadIdx.x;
  const int n_rays = g.n_angles * g.n_det;
  FAcc acc_d;
  if (ray < n_rays) {
    const int a = ray / g.n_det, bin = ray - a * g.n_det;
    const float4 ang = __ldg(angles + a);
    const float* img = ang.w != 0.f ? x : xt;  // row walk reads x[l][k], column walk xt[l][k]
    const int N = g.N;
    // fr is affine in l, fr(l) = fr(0) - l * rate; only lines with -1 <= fr < N can
    // contribute, so walk a superset of them (one line of margin each side)
    int l_lo = 0, l_hi = N - 1;
    {
      const float fr0 = joseph_fr(g, ang, bin, 0);
      const float rate = fr0 - joseph_fr(g, ang, bin, 1);
      if (fabsf(rate) > 1e-6f) {
        const float la = (fr0 + 1.f) / rate, lb = (fr0 - (float)N) / rate;
        const float lmin = fminf(la, lb), lmax = fmaxf(la, lb);
        l_lo = max(0, (int)floorf(lmin) - 1);
        l_hi = min(N - 1, (int)ceilf(lmax) + 1);
      }
    }
    float acc = 0.f;
    for (int l = l_lo; l <= l_hi; ++l) {
      const float fr = joseph_fr(g, ang, bin, l);
      const float k0f = floorf(fr);
      if (k0f < -1.f || k0f > (float)(N - 1)) continue;
      const int k0 = (int)k0f;
      const float f = fr - k0f;
      const float* row = img + (size_t)l * N;
      const float v0 = k0 >= 0 ? __ldg(row + k0) : 0.f;
      const float v1 = k0 + 1 <= N - 1 ? __ldg(row + k0 + 1) : 0.f;
      acc += (1.f - f) * v0 + f * v1;
    }
    const float ax = ang.z * acc;
    if (MODE == 0) {
      sino[ray] = ax;
    } else {
      const float bb = __ldg(b + ray);
      if (MODE == 4) {  // PDHGSkip-1: ax = A x^, sino holds A x_k on entry, tau2 = p
        const float axn = sino[ray] + tau2 * ax;
        y[ray] = (y[ray] + tau * (axn + ax) - tau * bb) / (1.f + tau);
        sino[ray] = axn;
        const float r = axn - bb;
        acc_d.add(0.5f * (r * r));
      } else {
        if (MODE == 1) {
          const float prev = sino[ray];
          y[ray] = (y[ray] + tau * (2.f * ax - prev) - tau * bb) / (1.f + tau);
        }
        const float r = ax - bb;
        sino[ray] = MODE == 3 ? r : ax;
        acc_d.add(0.5f * (r * r));
      }
    }
  }
  if (MODE != 0) block_sum2_store<CT_NT>(acc_d, FAcc(), part, nullptr, blockIdx.x);
}

// g = A^T y at pixel (i, j); epilogue out = x - sigma g + ch h (when x given).
__global__ void __launch_bounds__(CT_NT)
joseph_bwd_kernel(GeomConsts g, const float4* __restrict__ angles, const float4* __restrict__ angles2,
                  const float* __restrict__ ys,
                  const float* __restrict__ x, const float* __restrict__ h, float* __restrict__ out,
                  float sigma, float ch, Partial* __restrict__ part_tv) {
  pdl_enter();
  const int N = g.N;
  const int pix = blockIdx.x * CT_NT + threadIdx.x;
  FAcc acc_tv;
  if (pix < N * N) {
    const int i = pix / N, j = pix - i * N;
    float total = 0.f;
    for (int a = 0; a < g.n_angles; ++a) {
      const float4 ang = __ldg(angles + a);
      const bool rowwalk = ang.w != 0.f;
      const int l = rowwalk ? i : j;   // line the ray walks
      const int k = rowwalk ? j : i;   // this pixel's index along the line
      // fr is affine in b with slope d * inv, so the bins whose floor(fr) is
      // k - 1 or k lie in an interval of length 2 / |slope| around the b where
      // fr = k; the ncand integers from ceil(bc - 1/|slope| - margin) cover it
      // (3 when bins have the pixel width), and each candidate is decided with
      // the projector's own fr.
      const float4 a2 = __ldg(angles2 + a);  // (1 / slope, 1 / |slope| + margin, ncand, -)
      const float fr0 = joseph_fr(g, ang, 0, l);
      const float bc = ((float)k - fr0) * a2.x;
      const int b_first = (int)ceilf(bc - a2.y);
      const int ncand = (int)a2.z;
      const float* yrow = ys + (size_t)a * g.n_det;
      float acc = 0.f;
#pragma unroll 3
      for (int j = 0; j < ncand; ++j) {
        const int b = b_first + j;
        if (b < 0 || b >= g.n_det) continue;
        const float fr = joseph_fr(g, ang, b, l);
        const float k0f = floorf(fr);
        const float f = fr - k0f;
        const int k0 = (int)k0f;
        // the projector's weight of this pixel on ray b (0 when the ray's two
        // interpolation cells miss it), applied without a divergent branch
        const float wgt = k0 == k ? 1.f - f : (k0 + 1 == k ? f : 0.f);
        acc = fmaf(wgt, __ldg(yrow + b), acc);
      }
      total = fmaf(ang.z, acc, total);
    }
    if (x) {
      const size_t o = (size_t)i * N + j;
      const float xc = __ldg(x + o);
      float v = xc - sigma * total;
      if (h) v = fmaf(ch, __ldg(h + o), v);
      out[o] = v;
      if (part_tv) {
        const float dy = i < N - 1 ? __ldg(x + o + N) - xc : 0.f;
        const float dx = j < N - 1 ? __ldg(x + o + 1) - xc : 0.f;
        acc_tv.add(tv_term(0.f, dy, dx));
      }
    } else {
      out[(size_t)i * N + j] = total;
    }
  }
  if (part_tv) block_sum2_store<CT_NT>(FAcc(), acc_tv, nullptr, part_tv, blockIdx.x);
}

GeomConsts consts(const CTGeom& g) {
  GeomConsts c;
  c.N = g.N;
  c.n_angles = g.n_angles;
  c.n_det = g.n_det;
  c.s = g.pixel_size;
  c.d = g.det_spacing;
  c.t0 = (float)(-0.5 * (g.n_det - 1) * (double)g.det_spacing);
  c.c0 = (float)(-0.5 * (g.N - 1) * (double)g.pixel_size);
  c.half = (float)(0.5 * (g.N - 1));
  return c;
}

}  // namespace

cudaError_t ct_build_angle_table(const CTGeom& g, float4* dev_table, cudaStream_t s) {
  float4* host = new float4[g.n_angles];
  float4* host2 = new float4[g.n_angles];
  const double pi = 3.14159265358979323846;
  for (int a = 0; a < g.n_angles; ++a) {
    const double th = a * pi / g.n_angles;
    const double c = cos(th), sn = sin(th);
    const bool rowwalk = fabs(c) >= fabs(sn);
    float4 v;
    v.x = (float)(rowwalk ? sn : c);
    v.y = (float)(1.0 / ((rowwalk ? c : sn) * (double)g.pixel_size));
    v.z = (float)((double)g.pixel_size / (rowwalk ? fabs(c) : fabs(sn)));
    v.w = rowwalk ? 1.f : 0.f;
    host[a] = v;
    // backprojector helpers: slope of fr in b is d * inv (inv as stored, in float)
    const double slope = (double)g.det_spacing * (double)v.y;
    const double half = 1.0 / fabs(slope) + 0.02;
    host2[a] = make_float4((float)(1.0 / slope), (float)half, (float)(floor(2.0 * half) + 1.0), 0.f);
  }
  cudaError_t e = cudaMemcpyAsync(dev_table, host, sizeof(float4) * g.n_angles,
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g.angles2, host2, sizeof(float4) * g.n_angles, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  delete[] host;
  delete[] host2;
  return e;
}

int ct_fwd_blocks(const CTGeom& g) { return (g.n_angles * g.n_det + CT_NT - 1) / CT_NT; }
int ct_bwd_blocks(const CTGeom& g) { return (g.N * g.N + CT_NT - 1) / CT_NT; }

cudaError_t launch_ct_forward(const CTGeom& g, const float* x, float* sino, float* y,
                              const float* b, float tau, Partial* part_data, int mode,
                              cudaStream_t s, float p) {
  if (!g.xt_scratch) return cudaErrorInvalidValue;
  dim3 tg((g.N + 31) / 32, (g.N + 31) / 32), tb(32, 8);
  launch_kernel(transpose_kernel, dim3(tg), dim3(tb), 0, s, x, g.xt_scratch, g.N);
  const GeomConsts c = consts(g);
  const int blocks = ct_fwd_blocks(g);
  switch (mode) {
    case CT_FWD_PD:
      launch_kernel(joseph_fwd_kernel<1>, dim3(blocks), dim3(CT_NT), 0, s, c, g.angles, x, g.xt_scratch, sino, y, b, tau, part_data, 0.f);
      break;
    case CT_FWD_STORE:
      launch_kernel(joseph_fwd_kernel<2>, dim3(blocks), dim3(CT_NT), 0, s, c, g.angles, x, g.xt_scratch, sino, nullptr, b, 0.f, part_data, 0.f);
      break;
    case CT_FWD_RESID:
      launch_kernel(joseph_fwd_kernel<3>, dim3(blocks), dim3(CT_NT), 0, s, c, g.angles, x, g.xt_scratch, sino, nullptr, b, 0.f, part_data, 0.f);
      break;
    case CT_FWD_PD1:
      launch_kernel(joseph_fwd_kernel<4>, dim3(blocks), dim3(CT_NT), 0, s, c, g.angles, x, g.xt_scratch, sino, y, b, tau, part_data, p);
      break;
    default:
      launch_kernel(joseph_fwd_kernel<0>, dim3(blocks), dim3(CT_NT), 0, s, c, g.angles, x, g.xt_scratch, sino, nullptr, nullptr, 0.f, nullptr, 0.f);
  }
  return cudaGetLastError();
}

cudaError_t launch_ct_backward(const CTGeom& g, const float* y, const float* x, const float* h,
                               float* out, float sigma, float ch, Partial* part_tv, cudaStream_t s) {
  const GeomConsts c = consts(g);
  launch_kernel(joseph_bwd_kernel, dim3(ct_bwd_blocks(g)), dim3(CT_NT), 0, s, c, g.angles, g.angles2, y, x, h, out, sigma, ch,
                                                       part_tv);
  return cudaGetLastError();
}

}  // namespace tvs
