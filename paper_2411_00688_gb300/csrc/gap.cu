// ROF duality gap of a TV-prox dual (the certificate behind tv_prox_gap).
#include "common.cuh"
#include "kernels.hpp"

namespace tvs {

namespace {
// ROF duality gap terms of a unit-ball dual p for prox_{lam TV}(z): with
// u = z + lam div p, g_i = |(D u)_i|_2 - <(D u)_i, p_i>, non-negative for |p_i| <= 1
// (Cauchy-Schwarz), so the sum has no cancellation; lam * sum g_i = P(u) - D(p).
template <typename T>
__global__ void __launch_bounds__(256)
rof_gap_partials_kernel(const float* __restrict__ z, const T* __restrict__ p, int D, int H, int W, int ndim,
                        float lam, Partial* __restrict__ part, IndexMap im) {
  pdl_enter();
  const size_t n = (size_t)D * H * W, HW = (size_t)H * W;
  const T* pz = p;                              // 3D only
  const T* py = p + (ndim == 3 ? n : 0);
  const T* px = py + n;
  auto u_at = [&](int k, int i, int j) -> float {
    const size_t o = (size_t)k * HW + (size_t)i * W + j;
    float dv = 0.f;
    if (ndim == 3) {
      if (k < D - 1) dv += Elem<T>::ld(pz + o);
      if (k > 0) dv -= Elem<T>::ld(pz + o - HW);
    }
    if (i < H - 1) dv += Elem<T>::ld(py + o);
    if (i > 0) dv -= Elem<T>::ld(py + o - W);
    if (j < W - 1) dv += Elem<T>::ld(px + o);
    if (j > 0) dv -= Elem<T>::ld(px + o - 1);
    return __ldg(z + o) + lam * dv;
  };
  FAcc acc;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    int k, i, j;
    im.coords(o, k, i, j);
    const float uc = u_at(k, i, j);
    const float d0 = (ndim == 3 && k < D - 1) ? u_at(k + 1, i, j) - uc : 0.f;
    const float d1 = i < H - 1 ? u_at(k, i + 1, j) - uc : 0.f;
    const float d2 = j < W - 1 ? u_at(k, i, j + 1) - uc : 0.f;
    const float q0 = ndim == 3 ? Elem<T>::ld(pz + o) : 0.f;
    const float q1 = Elem<T>::ld(py + o), q2 = Elem<T>::ld(px + o);
    acc.add(tv_term(d0, d1, d2) - (d0 * q0 + d1 * q1 + d2 * q2));
  }
  block_sum2_store<256>(acc, FAcc(), part, nullptr, blockIdx.x);
}
}  // namespace

int rof_gap_blocks(size_t n) {
  size_t b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_rof_gap_partials(const Dims& d, const float* z, const void* p, int dtype, float lam,
                                    Partial* part, cudaStream_t s) {
  const int blocks = rof_gap_blocks(d.n());
  const IndexMap im(d.nz, d.ny, d.nx);
  with_dual_type(dtype, [&](auto tag) {
    using T = typename decltype(tag)::type;
    launch_kernel(rof_gap_partials_kernel<T>, dim3(blocks), dim3(256), 0, s, z, (const T*)p, d.nz, d.ny, d.nx,
                  d.ndim, lam, part, im);
    return 0;
  });
  return cudaGetLastError();
}

}  // namespace tvs
