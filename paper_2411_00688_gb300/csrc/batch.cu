// Batched ProxSkip (Algorithm 4) over many independent 2D problems of uneven
// sizes, each with its own alpha, gamma, p and Philox seed.  Every kernel covers
// all problems at once: a CTA takes one entry of a concatenated work list (a
// problem and a tile or pixel chunk of it), reads that problem's descriptor and
// its coin for the current outer iteration from device memory, and runs the same
// tile bodies as the single-problem kernels.  Problems whose coin is 0 skip the
// inner iterations; problems that reached their objective target skip
// everything.  The outer iteration index lives in a device counter, so one
// captured graph per buffer parity serves every iteration.
#include "blur_body.cuh"
#include "common.cuh"
#include "fgp_rb.cuh"
#include "kernels.hpp"

namespace tvs {

namespace {

constexpr int BT_TB = 4, BT_CPL = 1, BT_RPW = 5;  // blocked inner kernel of the batch
constexpr int BT_TW = 32 * BT_CPL - 2 * BT_TB, BT_TH = 8 * BT_RPW - 2 * BT_TB;
constexpr int CHUNK = 1024;                        // pixels per pointwise work item

__device__ __forceinline__ bool active(const BatchState& st) { return st.done == 0; }

template <int R>
__global__ void __launch_bounds__(BNT)
batch_blur_resid_kernel(const BatchProb* __restrict__ probs, BatchState* __restrict__ state,
                        const int4* __restrict__ tiles, int par, Partial* part_a, Partial* part_b) {
  pdl_enter();
  const int4 e = tiles[blockIdx.x];
  const BatchProb& P = probs[e.x];
  if (!active(state[e.x])) return;
  blur_tile_body<BM_RESID, R>(par ? P.x1 : P.x0, P.H, P.W, P.bw, P.b, P.r, nullptr, nullptr, 0.f, 0.f,
                           nullptr, nullptr, 0.f, part_a, part_b, e.y, e.z, blockIdx.x);
}

template <int R>
__global__ void __launch_bounds__(BNT)
batch_blur_step_kernel(const BatchProb* __restrict__ probs, BatchState* __restrict__ state,
                       const int4* __restrict__ tiles, const unsigned char* __restrict__ coins, int n,
                       const int* __restrict__ kctr, int par) {
  pdl_enter();
  const int4 e = tiles[blockIdx.x];
  const BatchProb& P = probs[e.x];
  if (!active(state[e.x])) return;
  const int k = *kctr;
  const bool coin = coins[(size_t)k * n + e.x] != 0;
  const float* xc = par ? P.x1 : P.x0;
  float* out = coin ? P.z : (par ? P.x0 : P.x1);
  blur_tile_body<BM_STEP, R>(P.r, P.H, P.W, P.bw, nullptr, out, xc, P.h, P.gamma,
                          coin ? P.ch_prox : P.ch_skip, nullptr, nullptr, 0.f, nullptr, nullptr, e.y,
                          e.z, 0);
}

// Identity data term: out = x - gamma (x - b) + ch h; partials of 1/2 (x-b)^2, TV(x).
__global__ void __launch_bounds__(256)
batch_ident_step_kernel(const BatchProb* __restrict__ probs, BatchState* __restrict__ state,
                        const int2* __restrict__ chunks, const unsigned char* __restrict__ coins, int n,
                        const int* __restrict__ kctr, int par, int write_out, Partial* part_a,
                        Partial* part_b, int part_base) {
  pdl_enter();
  const int2 e = chunks[blockIdx.x];
  const BatchProb& P = probs[e.x];
  if (!active(state[e.x])) return;
  const int k = *kctr;
  const bool coin = write_out && coins[(size_t)k * n + e.x] != 0;
  const float* x = par ? P.x1 : P.x0;
  float* out = coin ? P.z : (par ? P.x0 : P.x1);
  const float ch = coin ? P.ch_prox : P.ch_skip;
  const size_t npx = (size_t)P.H * P.W;
  FAcc acc_a, acc_b;
  for (int t = threadIdx.x; t < CHUNK; t += 256) {
    const size_t o = (size_t)e.y * CHUNK + t;
    if (o >= npx) break;
    const int gi = (int)(o / P.W), gj = (int)(o - (size_t)gi * P.W);
    const float xc = __ldg(x + o), bb = __ldg(P.b + o);
    const float r = xc - bb;
    if (write_out) out[o] = fmaf(ch, __ldg(P.h + o), xc - P.gamma * r);
    acc_a.add(0.5f * (r * r));
    const float dy = gi < P.H - 1 ? __ldg(x + o + P.W) - xc : 0.f;
    const float dx = gj < P.W - 1 ? __ldg(x + o + 1) - xc : 0.f;
    acc_b.add(tv_term(0.f, dy, dx));
  }
  block_sum2_store<256>(acc_a, acc_b, part_a, part_b, part_base + blockIdx.x);
}

// One block per problem: F(x_k) from its partials; records F at index k - 1,
// sets done once (F - f*) <= target f*.  final_pass: records F(x_K) at K - 1.
__global__ void __launch_bounds__(256)
batch_reduce_kernel(const BatchProb* __restrict__ probs, BatchState* __restrict__ state,
                    const int* __restrict__ kctr, const Partial* __restrict__ part_a,
                    const Partial* __restrict__ part_b, int final_pass, int* done_host) {
  pdl_enter();
  const BatchProb& P = probs[blockIdx.x];
  BatchState& S = state[blockIdx.x];
  if (!active(S)) return;
  const double sum_a = block_sum_partials<256>(part_a + P.part_off, P.part_n);
  const double sum_b = block_sum_partials<256>(part_b + P.part_off, P.part_n);
  if (threadIdx.x != 0) return;
  const int k = *kctr;  // F of x_k
  const double F = sum_a + P.alpha * sum_b;
  if (k >= 1) {
    P.obj[k - 1] = F;
    P.ts[k - 1] = globaltimer_ns();
  }
  const bool hit = P.f_star > 0.0 && (F - P.f_star) <= P.target * P.f_star;
  if (hit && !S.pad) {  // pad: target met (reached = its trace index, -1 for x_0)
    S.pad = 1;
    S.reached = k - 1;
  }
  if (hit || final_pass) {
    S.done = 1;
    S.iters = k;
    if (done_host) {
      *(volatile int*)(done_host + blockIdx.x) = 1;
      __threadfence_system();
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256, 2)
batch_fgp_kernel(const BatchProb* __restrict__ probs, BatchState* __restrict__ state,
                 const int4* __restrict__ tiles, const unsigned char* __restrict__ coins, int n,
                 const int* __restrict__ kctr, int q_in, TBBetas betas, int iters) {
  pdl_enter();
  const int4 e = tiles[blockIdx.x];
  const BatchProb& P = probs[e.x];
  if (!active(state[e.x])) return;
  if (coins[(size_t)(*kctr) * n + e.x] == 0 || P.lam == 0.f) return;
  const T* pc = (const T*)(q_in ? P.dual2 : P.dual0);
  const T* pp = (const T*)(q_in ? P.dual3 : P.dual1);
  if (betas.b[0] == 0.f) pp = pc;  // first iteration of a prox call: p_{k-1} unused
  T* pn = (T*)(q_in ? P.dual0 : P.dual2);
  T* pnp = (T*)(q_in ? P.dual1 : P.dual3);
  if (P.nonneg)
    fgp2d_rb_body<T, true, BT_TB, BT_CPL, BT_RPW>(P.z, pc, pp, pn, pnp, P.H, P.W, P.lam, P.inv_step, betas,
                                                  iters, e.y, e.z);
  else
    fgp2d_rb_body<T, false, BT_TB, BT_CPL, BT_RPW>(P.z, pc, pp, pn, pnp, P.H, P.W, P.lam, P.inv_step, betas,
                                                   iters, e.y, e.z);
}

// x_{k+1} = P_X(z + lam div p_N); h = (p/gamma)(x_{k+1} - z); p_N copied home if
// it sits in the second pair.
template <typename T>
__global__ void __launch_bounds__(256)
batch_finalize_kernel(const BatchProb* __restrict__ probs, BatchState* __restrict__ state,
                      const int2* __restrict__ chunks, const unsigned char* __restrict__ coins, int n,
                      const int* __restrict__ kctr, int par, int fin_pair) {
  pdl_enter();
  const int2 e = chunks[blockIdx.x];
  const BatchProb& P = probs[e.x];
  if (!active(state[e.x])) return;
  if (coins[(size_t)(*kctr) * n + e.x] == 0) return;
  const T* p = (const T*)(fin_pair ? P.dual2 : P.dual0);
  T* home = (fin_pair && P.lam != 0.f) ? (T*)P.dual0 : nullptr;
  float* xo = par ? P.x0 : P.x1;
  const int H = P.H, W = P.W;
  const size_t npx = (size_t)H * W;
  for (int t = threadIdx.x; t < CHUNK; t += 256) {
    const size_t o = (size_t)e.y * CHUNK + t;
    if (o >= npx) break;
    const int gi = (int)(o / W), gj = (int)(o - (size_t)gi * W);
    float dv = 0.f;
    if (gi < H - 1) dv += Elem<T>::ld(p + o);
    if (gi > 0) dv -= Elem<T>::ld(p + o - W);
    if (gj < W - 1) dv += Elem<T>::ld(p + npx + o);
    if (gj > 0) dv -= Elem<T>::ld(p + npx + o - 1);
    const float zz = __ldg(P.z + o);
    float u = P.lam != 0.f ? zz + P.lam * dv : zz;
    if (P.nonneg) u = fmaxf(u, 0.f);
    xo[o] = u;
    P.h[o] = P.h_coef * (u - zz);
    if (home) {
      home[o] = p[o];
      home[npx + o] = p[npx + o];
    }
  }
}

__global__ void batch_tick_kernel(int* kctr) {
  pdl_enter(); *kctr += 1; }

}  // namespace

int batch_fgp_tile_w() { return BT_TW; }
int batch_fgp_tile_h() { return BT_TH; }
int batch_chunk() { return CHUNK; }
int batch_fgp_iters_per_launch() { return BT_TB; }

namespace {
cudaError_t batch_blur(const BatchLaunch& L, int par, bool step, cudaStream_t s) {
  switch (L.blur_radius) {
#define TVS_BB_R(R_)                                                                                   \
  case R_:                                                                                             \
    launch_kernel(batch_blur_resid_kernel<R_>, dim3(L.n_blur_tiles), dim3(BNT), 0, s, L.probs, L.state, L.blur_tiles, par,   \
                                                              L.part_a, L.part_b);                     \
    if (step)                                                                                          \
      launch_kernel(batch_blur_step_kernel<R_>, dim3(L.n_blur_tiles), dim3(BNT), 0, s, L.probs, L.state, L.blur_tiles,        \
                                                                L.coins, L.n, L.kctr, par);            \
    break;
    TVS_BB_R(1) TVS_BB_R(2) TVS_BB_R(3) TVS_BB_R(4) TVS_BB_R(5) TVS_BB_R(6) TVS_BB_R(7) TVS_BB_R(8)
#undef TVS_BB_R
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_batch_iteration(const BatchLaunch& L, int par, cudaStream_t s) {
  if (L.n_blur_tiles > 0) {
    cudaError_t e = batch_blur(L, par, true, s);
    if (e != cudaSuccess) return e;
  }
  if (L.n_ident_chunks > 0)
    launch_kernel(batch_ident_step_kernel, dim3(L.n_ident_chunks), dim3(256), 0, s, L.probs, L.state, L.ident_chunks, L.coins, L.n,
                                                             L.kctr, par, 1, L.part_a, L.part_b,
                                                             L.n_blur_tiles);
  launch_kernel(batch_reduce_kernel, dim3(L.n), dim3(256), 0, s, L.probs, L.state, L.kctr, L.part_a, L.part_b, 0, L.done_host);
  if (L.n_inner > 0 && L.use_prox) {
    int q = 0;
    for (int g = 1; g <= L.n_inner;) {
      const int it = L.n_inner - g + 1 < BT_TB ? L.n_inner - g + 1 : BT_TB;
      TBBetas b{};
      for (int j = 0; j < it; ++j) b.b[j] = L.betas[g - 1 + j];
      switch (L.dtype) {
        case DUAL_F32:
          launch_kernel(batch_fgp_kernel<float>, dim3(L.n_fgp_tiles), dim3(256), 0, s, L.probs, L.state, L.fgp_tiles, L.coins, L.n,
                                                                L.kctr, q, b, it);
          break;
        case DUAL_BF16:
          launch_kernel(batch_fgp_kernel<__nv_bfloat16>, dim3(L.n_fgp_tiles), dim3(256), 0, s, L.probs, L.state, L.fgp_tiles, L.coins,
                                                                        L.n, L.kctr, q, b, it);
          break;
        default:
          launch_kernel(batch_fgp_kernel<__half>, dim3(L.n_fgp_tiles), dim3(256), 0, s, L.probs, L.state, L.fgp_tiles, L.coins, L.n,
                                                                 L.kctr, q, b, it);
      }
      q = 1 - q;
      g += it;
    }
    const int fin_pair = q;  // pair holding p_N
    switch (L.dtype) {
      case DUAL_F32:
        launch_kernel(batch_finalize_kernel<float>, dim3(L.n_all_chunks), dim3(256), 0, s, L.probs, L.state, L.all_chunks, L.coins,
                                                                    L.n, L.kctr, par, fin_pair);
        break;
      case DUAL_BF16:
        launch_kernel(batch_finalize_kernel<__nv_bfloat16>, dim3(L.n_all_chunks), dim3(256), 0, s, L.probs, L.state, L.all_chunks,
                                                                            L.coins, L.n, L.kctr, par, fin_pair);
        break;
      default:
        launch_kernel(batch_finalize_kernel<__half>, dim3(L.n_all_chunks), dim3(256), 0, s, L.probs, L.state, L.all_chunks, L.coins,
                                                                     L.n, L.kctr, par, fin_pair);
    }
  } else {
    // no prox work: finalisation reduces to x_{k+1} = z and h = (p/gamma)(z - z) = 0
    // when alpha = 0; handled by the same kernel with lam = 0 through the descriptors
    switch (L.dtype) {
      case DUAL_F32:
        launch_kernel(batch_finalize_kernel<float>, dim3(L.n_all_chunks), dim3(256), 0, s, L.probs, L.state, L.all_chunks, L.coins,
                                                                    L.n, L.kctr, par, 0);
        break;
      case DUAL_BF16:
        launch_kernel(batch_finalize_kernel<__nv_bfloat16>, dim3(L.n_all_chunks), dim3(256), 0, s, L.probs, L.state, L.all_chunks,
                                                                            L.coins, L.n, L.kctr, par, 0);
        break;
      default:
        launch_kernel(batch_finalize_kernel<__half>, dim3(L.n_all_chunks), dim3(256), 0, s, L.probs, L.state, L.all_chunks, L.coins,
                                                                     L.n, L.kctr, par, 0);
    }
  }
  launch_kernel(batch_tick_kernel, dim3(1), dim3(1), 0, s, L.kctr);
  return cudaGetLastError();
}

cudaError_t launch_batch_final_objective(const BatchLaunch& L, int par, cudaStream_t s) {
  if (L.n_blur_tiles > 0) {
    cudaError_t e = batch_blur(L, par, false, s);
    if (e != cudaSuccess) return e;
  }
  if (L.n_ident_chunks > 0)
    launch_kernel(batch_ident_step_kernel, dim3(L.n_ident_chunks), dim3(256), 0, s, L.probs, L.state, L.ident_chunks, L.coins, L.n,
                                                             L.kctr, par, 0, L.part_a, L.part_b,
                                                             L.n_blur_tiles);
  launch_kernel(batch_reduce_kernel, dim3(L.n), dim3(256), 0, s, L.probs, L.state, L.kctr, L.part_a, L.part_b, 1, L.done_host);
  return cudaGetLastError();
}

}  // namespace tvs
