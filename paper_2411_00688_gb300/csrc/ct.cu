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

// g = A^T y; epilogue out = x - sigma g + ch h (when x given).
//
// Four threads per 2 x 2 pixel block (rows i0, i0+1, columns j0, j0+1), each
// summing a quarter of the angles (enough threads to keep the SMs' warp slots
// busy); the four partial sums are added in a fixed order, so the result is
// deterministic.  For each angle the block's pixels sit on two lines l (rows for
// row walks, columns otherwise) at two indices k0, k0+1 along them; ray b gives pixel k the
// projector's weight 1 - f when floor(fr(b, l)) = k and f when floor(fr(b, l)) =
// k - 1 (f = fr - floor(fr)).  fr is affine in b with slope d * inv, so the bins
// that reach either index lie in an interval of length 3 / |slope| around the b
// where fr = k0 + 1/2: the ncand integers from ceil(bc - 1.5/|slope| - margin)
// cover it (4 when bins have the pixel width).  Each candidate is decided with the
// projector's own fr and serves both pixels of the line, and candidates that reach
// a pixel with weight 0 add exactly nothing, so within each quarter of the angles
// every pixel receives the same terms in the same order (increasing angle, then
// increasing bin) as a gather over its own bins: the weights are bit-identical to
// the projector's.
constexpr int CT_BWD_NT = 128;  // 32 pixel blocks x 4 angle groups
constexpr int CT_BWD_AG = 4;

__global__ void __launch_bounds__(CT_BWD_NT)
joseph_bwd_kernel(GeomConsts g, const float4* __restrict__ angles, const float4* __restrict__ angles2,
                  const float* __restrict__ ys,
                  const float* __restrict__ x, const float* __restrict__ h, float* __restrict__ out,
                  float sigma, float ch, Partial* __restrict__ part_tv) {
  pdl_enter();
  __shared__ float s_part[CT_BWD_AG][CT_BWD_NT / CT_BWD_AG][4];
  const int N = g.N;
  const int NB = (N + 1) / 2;  // blocks per row
  constexpr int PB = CT_BWD_NT / CT_BWD_AG;  // pixel blocks per CTA
  const int grp = threadIdx.x / PB, slot = threadIdx.x - grp * PB;
  const int blk = blockIdx.x * PB + slot;
  const int a_lo = (g.n_angles * grp) / CT_BWD_AG, a_hi = (g.n_angles * (grp + 1)) / CT_BWD_AG;
  FAcc acc_tv;
  if (blk < NB * NB) {
    const int i0 = 2 * (blk / NB), j0 = 2 * (blk - (blk / NB) * NB);
    // line coordinates c_l of rows i0, i0+1 and columns j0, j0+1 (the projector's fma)
    const float cr0 = __fmaf_rn((float)i0, g.s, g.c0), cr1 = __fmaf_rn((float)(i0 + 1), g.s, g.c0);
    const float cc0 = __fmaf_rn((float)j0, g.s, g.c0), cc1 = __fmaf_rn((float)(j0 + 1), g.s, g.c0);
    float t00 = 0.f, t01 = 0.f, t10 = 0.f, t11 = 0.f;  // totals of (i0 + a, j0 + b)
    for (int a = a_lo; a < a_hi; ++a) {
      const float4 ang = __ldg(angles + a);
      const float4 a2 = __ldg(angles2 + a);  // (1 / slope, 1.5 / |slope| + margin, ncand, -)
      const bool rowwalk = ang.w != 0.f;
      const float kf = rowwalk ? (float)j0 : (float)i0;  // first index along the lines
      const float* yrow = ys + (size_t)a * g.n_det;
      const int ncand = (int)a2.z;
      float acc[2][2];  // [line][index]
#pragma unroll
      for (int li = 0; li < 2; ++li) {
        const float cl = rowwalk ? (li ? cr1 : cr0) : (li ? cc1 : cc0);
        const float fr0 = __fmaf_rn(__fmaf_rn(-cl, ang.x, g.t0), ang.y, g.half);
        const float bfirst = ceilf((kf + 0.5f - fr0) * a2.x - a2.y);
        const int b_first = (int)bfirst;
        float aa = 0.f, ab = 0.f;
        float bf = bfirst;
        for (int b = b_first; b < b_first + ncand; ++b, bf += 1.f) {
          if (b < 0 || b >= g.n_det) continue;
          const float tb = __fmaf_rn(bf, g.d, g.t0);
          const float fr = __fmaf_rn(__fmaf_rn(-cl, ang.x, tb), ang.y, g.half);
          const float k0f = floorf(fr);
          const float f = fr - k0f;
          const float yv = __ldg(yrow + b);
          // pixel kf: 1 - f if floor(fr) = kf, f if floor(fr) = kf - 1; pixel kf + 1 likewise
          const float wa = k0f == kf ? 1.f - f : (k0f == kf - 1.f ? f : 0.f);
          const float wb = k0f == kf + 1.f ? 1.f - f : (k0f == kf ? f : 0.f);
          aa = fmaf(wa, yv, aa);
          ab = fmaf(wb, yv, ab);
        }
        acc[li][0] = aa;
        acc[li][1] = ab;
      }
      // rows: line li is row i0 + li, index c column j0 + c; columns: transposed
      const float a00 = acc[0][0], a11 = acc[1][1];
      const float a01 = rowwalk ? acc[0][1] : acc[1][0];
      const float a10 = rowwalk ? acc[1][0] : acc[0][1];
      t00 = fmaf(ang.z, a00, t00);
      t01 = fmaf(ang.z, a01, t01);
      t10 = fmaf(ang.z, a10, t10);
      t11 = fmaf(ang.z, a11, t11);
    }
    s_part[grp][slot][0] = t00;
    s_part[grp][slot][1] = t01;
    s_part[grp][slot][2] = t10;
    s_part[grp][slot][3] = t11;
  }
  __syncthreads();
  // group 0 adds the four quarters in angle order and writes the block
  if (grp == 0 && blk < NB * NB) {
    const int i0 = 2 * (blk / NB), j0 = 2 * (blk - (blk / NB) * NB);
    float tot[2][2];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float v = s_part[0][slot][e];
#pragma unroll
      for (int q = 1; q < CT_BWD_AG; ++q) v += s_part[q][slot][e];
      tot[e >> 1][e & 1] = v;
    }
#pragma unroll
    for (int di = 0; di < 2; ++di)
#pragma unroll
      for (int dj = 0; dj < 2; ++dj) {
        const int i = i0 + di, j = j0 + dj;
        if (i >= N || j >= N) continue;
        const size_t o = (size_t)i * N + j;
        const float total = tot[di][dj];
        if (x) {
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
          out[o] = total;
        }
      }
  }
  if (part_tv) block_sum2_store<CT_BWD_NT>(FAcc(), acc_tv, nullptr, part_tv, blockIdx.x);
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
    // backprojector helpers: slope of fr in b is d * inv (inv as stored, in float);
    // the bins reaching two adjacent indices span 3 / |slope| (plus a margin)
    const double slope = (double)g.det_spacing * (double)v.y;
    const double half = 1.5 / fabs(slope) + 0.02;
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
int ct_bwd_blocks(const CTGeom& g) {
  const int nb = (g.N + 1) / 2, per = CT_BWD_NT / CT_BWD_AG;
  return (nb * nb + per - 1) / per;
}

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
  launch_kernel(joseph_bwd_kernel, dim3(ct_bwd_blocks(g)), dim3(CT_BWD_NT), 0, s, c, g.angles, g.angles2, y, x, h, out, sigma, ch,
                                                       part_tv);
  return cudaGetLastError();
}

}  // namespace tvs
