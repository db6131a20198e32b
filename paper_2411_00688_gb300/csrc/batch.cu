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

// Blocked inner kernel of the batch: 5 iterations per launch over a 64 x 40
// region (54 x 30 outputs), two columns per lane, three CTAs per SM without
// spilling.  On the 256-problem workload (sides 64..1024), batched solve:
// 4 iterations on 64 x 32 0.308 s, on 64 x 40 0.291 s, 5 on 64 x 32 0.286 s,
// 5 on 64 x 40 0.267 s (10 launches per 50-iteration prox instead of 13);
// 4 on 64 x 64 (one CTA per SM) 0.438 s.
#ifndef TVS_BATCH_RPW
#define TVS_BATCH_RPW 5
#endif
#ifndef TVS_BATCH_TB
#define TVS_BATCH_TB 5
#endif
constexpr int BT_TB = TVS_BATCH_TB, BT_CPL = 2, BT_RPW = TVS_BATCH_RPW;
constexpr int BT_TW = 32 * BT_CPL - 2 * BT_TB, BT_TH = 8 * BT_RPW - 2 * BT_TB;
constexpr int CHUNK = 2048;                        // pixels per pointwise work item

__device__ __forceinline__ bool active(const BatchState& st) { return st.done == 0; }

// Blur data term, one fused forward-backward step per FX x FY tile:
// out = x - gamma A(A x - b) + ch h (out = z on a prox iteration, the next x on a
// skip), partials of 1/2 ||A x - b||^2 and TV(x).  write_out = 0: partials only
// (the final objective; the coin is not read).
template <int R>
__global__ void __launch_bounds__(FNT, 4)
batch_blur_fb_kernel(const BatchProb* __restrict__ probs, BatchState* __restrict__ state,
                     const int4* __restrict__ tiles, const unsigned char* __restrict__ coins, int n,
                     const int* __restrict__ kctr, int par, int write_out, Partial* part_a, Partial* part_b) {
  pdl_enter();
  const int4 e = tiles[blockIdx.x];
  const BatchProb& P = probs[e.x];
  if (!active(state[e.x])) return;
  const float* xc = par ? P.x1 : P.x0;
  float* out = nullptr;
  float ch = 0.f;
  if (write_out) {
    const bool coin = coins[(size_t)(*kctr) * n + e.x] != 0;
    out = coin ? P.z : (par ? P.x0 : P.x1);
    ch = coin ? P.ch_prox : P.ch_skip;
  }
  blur_fb_step_body<R>(xc, P.b, P.h, out, P.H, P.W, P.bw, P.gamma, ch, part_a, part_b, e.y, e.z, blockIdx.x);
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
  const size_t npx = (size_t)P.H * P.W, base = (size_t)e.y * CHUNK;
  FAcc acc_a, acc_b;
  // predicated, fully unrolled: the loads of every pixel of the chunk are issued together
#pragma unroll
  for (int u = 0; u < CHUNK / 256; ++u) {
    const size_t o = base + u * 256 + threadIdx.x;
    if (o < npx) {
      const int gi = (int)P.fw.div((uint32_t)o), gj = (int)o - gi * P.W;
      const float xc = __ldg(x + o), bb = __ldg(P.b + o);
      const float r = xc - bb;
      if (write_out) out[o] = fmaf(ch, __ldg(P.h + o), xc - P.gamma * r);
      acc_a.add(0.5f * (r * r));
      const float dy = gi < P.H - 1 ? __ldg(x + o + P.W) - xc : 0.f;
      const float dx = gj < P.W - 1 ? __ldg(x + o + 1) - xc : 0.f;
      acc_b.add(tv_term(0.f, dy, dx));
    }
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

// Problem owning entry w of this iteration's compacted work list: the largest i
// with scan[i] <= w (problems without work have scan[i] == scan[i + 1]).  The
// persistent kernels search a shared-memory copy of the scan when it fits.
constexpr int SCAN_SMEM = 2048;
__device__ __forceinline__ const int* stage_scan(const int* __restrict__ scan, int n, int* s_scan) {
  if (n + 1 > SCAN_SMEM) return scan;
  for (int i = threadIdx.x; i <= n; i += blockDim.x) s_scan[i] = scan[i];
  __syncthreads();
  return s_scan;
}
__device__ __forceinline__ int owner_of(const int* scan, int n, int w) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (scan[mid] <= w) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Compacts the work of outer iteration k (one block): a problem takes part in the
// prox of iteration k when it is still running and its coin is 1; its inner tiles
// count only when lam > 0.  Writes exclusive scans of the tile and chunk counts,
// zeroes the work counters of the iteration's inner launches and advances the
// outer iteration counter.
__global__ void __launch_bounds__(1024)
batch_active_kernel(const BatchProb* __restrict__ probs, const BatchState* __restrict__ state,
                    const unsigned char* __restrict__ coins, int n, int* __restrict__ kctr,
                    const int2* __restrict__ tile_range, const int2* __restrict__ chunk_range,
                    int* __restrict__ scan_tiles, int* __restrict__ scan_chunks, int* __restrict__ work,
                    int n_work) {
  pdl_enter();
  __shared__ int wt[32], wc[32];
  for (int j = threadIdx.x; j < n_work; j += blockDim.x) work[j] = 0;
  const int k = *kctr, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int carry_t = 0, carry_c = 0;
  for (int base = 0; base < n; base += 1024) {
    const int i = base + threadIdx.x;
    int ct = 0, cc = 0;
    if (i < n && state[i].done == 0 && coins[(size_t)k * n + i] != 0) {
      cc = chunk_range[i].y;
      if (probs[i].lam != 0.f) ct = tile_range[i].y;
    }
    // inclusive warp scans, then the warp totals
    int st = ct, sc = cc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int vt = __shfl_up_sync(0xffffffffu, st, o), vc = __shfl_up_sync(0xffffffffu, sc, o);
      if (lane >= o) {
        st += vt;
        sc += vc;
      }
    }
    if (lane == 31) {
      wt[warp] = st;
      wc[warp] = sc;
    }
    __syncthreads();
    if (warp == 0) {
      int a = wt[lane], b = wc[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int va = __shfl_up_sync(0xffffffffu, a, o), vb = __shfl_up_sync(0xffffffffu, b, o);
        if (lane >= o) {
          a += va;
          b += vb;
        }
      }
      wt[lane] = a;  // inclusive over warps
      wc[lane] = b;
    }
    __syncthreads();
    const int off_t = carry_t + (warp > 0 ? wt[warp - 1] : 0) + st - ct;
    const int off_c = carry_c + (warp > 0 ? wc[warp - 1] : 0) + sc - cc;
    if (i < n) {
      scan_tiles[i] = off_t;
      scan_chunks[i] = off_c;
    }
    carry_t += wt[31];
    carry_c += wc[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scan_tiles[n] = carry_t;
    scan_chunks[n] = carry_c;
    *kctr = k + 1;  // nothing later in the iteration reads k; every thread read it above
  }
}

// The tile being processed, as thread 0 prepared it (problem lookup and
// descriptor loads done once per tile): the body reads it at the start and again
// in its store phase, so its pointers and sizes need no registers in between.
template <typename T>
struct TileRec {
  const float* z;
  const T *pc, *pp;
  T *pn, *pnp;
  int H, W, tx, ty, nonneg, valid;
  float lam, inv_step;
};

// Persistent inner kernel over the compacted tiles of the problems whose coin is 1
// (no CTA is spent on skipping problems).  Each CTA starts on tile blockIdx.x and
// then takes the next unclaimed tile from the launch's work counter (zeroed by
// batch_active_kernel), so tiles of uneven cost (image borders, partial tiles)
// balance over the grid instead of piling up on CTAs that a fixed stride keeps
// handing the same tile column (the other resident CTAs of the SM cover the
// counter's round trip after each tile).  NN: 0 when no problem of the batch has
// the non-negativity constraint, 1 when all have it, 2 for a mix (both bodies
// compiled in).
#ifndef TVS_BATCH_FGP_MIN_CTAS
#define TVS_BATCH_FGP_MIN_CTAS 3
#endif
template <typename T, int NN>
__global__ void __launch_bounds__(256, TVS_BATCH_FGP_MIN_CTAS)
batch_fgp_kernel(const BatchProb* __restrict__ probs, const int* __restrict__ scan, int n, int q_in, TBBetas betas,
                 int iters, int* __restrict__ work) {
  pdl_enter();
  __shared__ int s_scan[SCAN_SMEM];
  __shared__ int s_w;
  __shared__ TileRec<T> rec;
  if (threadIdx.x == 0) s_w = blockIdx.x;
  const int* sc = stage_scan(scan, n, s_scan);
  __syncthreads();
  for (;;) {
    if (threadIdx.x == 0) {
      const int w = s_w, total = sc[n];
      rec.valid = w < total;
      if (w < total) {
        const int i = owner_of(sc, n, w);
        const BatchProb& P = probs[i];
        const int t = w - sc[i], fx = (P.W + BT_TW - 1) / BT_TW;
        rec.ty = t / fx;
        rec.tx = t - rec.ty * fx;
        rec.z = P.z;
        rec.pc = (const T*)(q_in ? P.dual2 : P.dual0);
        // first iteration of a prox call: p_{k-1} unused
        rec.pp = betas.b[0] == 0.f ? rec.pc : (const T*)(q_in ? P.dual3 : P.dual1);
        rec.pn = (T*)(q_in ? P.dual0 : P.dual2);
        rec.pnp = (T*)(q_in ? P.dual1 : P.dual3);
        rec.H = P.H;
        rec.W = P.W;
        rec.nonneg = P.nonneg;
        rec.lam = P.lam;
        rec.inv_step = P.inv_step;
      }
    }
    __syncthreads();
    if (!rec.valid) break;
    if (NN == 1 || (NN == 2 && rec.nonneg))
      fgp2d_rb_body<T, true, BT_TB, BT_CPL, BT_RPW>(rec.z, rec.pc, rec.pp, rec.pn, rec.pnp, rec.H, rec.W, rec.lam,
                                                    rec.inv_step, betas, iters, rec.tx, rec.ty);
    else
      fgp2d_rb_body<T, false, BT_TB, BT_CPL, BT_RPW>(rec.z, rec.pc, rec.pp, rec.pn, rec.pnp, rec.H, rec.W, rec.lam,
                                                     rec.inv_step, betas, iters, rec.tx, rec.ty);
    if (threadIdx.x == 0) s_w = (int)gridDim.x + atomicAdd(work, 1);
    __syncthreads();  // every thread is done with rec before thread 0 rewrites it
  }
}

// x_{k+1} = P_X(z + lam div p_N); h = (p/gamma)(x_{k+1} - z); p_N copied home if
// it sits in the second pair.
template <typename T>
__global__ void __launch_bounds__(256)
batch_finalize_kernel(const BatchProb* __restrict__ probs, const int2* __restrict__ chunk_range, const int* __restrict__ scan, int n, int par,
                      int fin_pair) {
  pdl_enter();
  __shared__ int s_scan[SCAN_SMEM];
  const int* sc = stage_scan(scan, n, s_scan);
  const int total = sc[n];
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const int i = owner_of(sc, n, w);
    const int2 e = make_int2(i, w - sc[i]);
    const BatchProb& P = probs[i];
    const T* p = (const T*)(fin_pair ? P.dual2 : P.dual0);
    T* home = (fin_pair && P.lam != 0.f) ? (T*)P.dual0 : nullptr;
    float* xo = par ? P.x0 : P.x1;
    const int H = P.H, W = P.W;
    const size_t npx = (size_t)H * W, base = (size_t)e.y * CHUNK;
    // all loads of the chunk first (predicated, unrolled), then the stores, so the
    // loads are not held behind stores the compiler cannot prove disjoint
    constexpr int U = CHUNK / 256;
    float dv[U], zz[U];
    T c0[U], c1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const size_t o = base + u * 256 + threadIdx.x;
      dv[u] = 0.f;
      zz[u] = 0.f;
      if (o < npx) {
        const int gi = (int)P.fw.div((uint32_t)o), gj = (int)o - gi * W;
        float d = 0.f;
        if (gi < H - 1) d += Elem<T>::ld(p + o);
        if (gi > 0) d -= Elem<T>::ld(p + o - W);
        if (gj < W - 1) d += Elem<T>::ld(p + npx + o);
        if (gj > 0) d -= Elem<T>::ld(p + npx + o - 1);
        dv[u] = d;
        zz[u] = __ldg(P.z + o);
        if (home) {
          c0[u] = p[o];
          c1[u] = p[npx + o];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const size_t o = base + u * 256 + threadIdx.x;
      if (o < npx) {
        float v = P.lam != 0.f ? zz[u] + P.lam * dv[u] : zz[u];
        if (P.nonneg) v = fmaxf(v, 0.f);
        xo[o] = v;
        P.h[o] = P.h_coef * (v - zz[u]);
        if (home) {
          home[o] = c0[u];
          home[npx + o] = c1[u];
        }
      }
    }
  }
}

// Per-solve set-up of every problem, one block per pixel chunk: x_0 copied in (when
// the caller's iterates live in device memory; x_src[i] is problem i's), the first
// dual pair and h zeroed, the objective record (K + 1 entries) set to NaN.
__global__ void __launch_bounds__(256)
batch_init_kernel(const BatchProb* __restrict__ probs, const int2* __restrict__ chunk_range, int n,
                  const float* const* __restrict__ x_src, int dual_bytes, int K) {
  pdl_enter();
  int lo = 0, hi = n;  // problem owning chunk blockIdx.x: largest i with first(i) <= blockIdx.x
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (chunk_range[mid].x <= (int)blockIdx.x) lo = mid;
    else hi = mid;
  }
  const BatchProb& P = probs[lo];
  const int c = (int)blockIdx.x - chunk_range[lo].x;
  const size_t npx = (size_t)P.H * P.W, base = (size_t)c * CHUNK;
  const float* src = x_src ? x_src[lo] : nullptr;
#pragma unroll
  for (int u = 0; u < CHUNK / 256; ++u) {
    const size_t o = base + u * 256 + threadIdx.x;
    if (o < npx) {
      if (src) P.x0[o] = src[o];
      P.h[o] = 0.f;
      if (dual_bytes == 4) {
        ((float*)P.dual0)[o] = 0.f;
        ((float*)P.dual0)[npx + o] = 0.f;
      } else {
        ((unsigned short*)P.dual0)[o] = 0;
        ((unsigned short*)P.dual0)[npx + o] = 0;
      }
    }
  }
  if (c == 0)
    for (int k = threadIdx.x; k <= K; k += 256) P.obj[k] = __longlong_as_double(-1ll);
}

// theta_k of every problem for k = 0 .. K-1, as coins[k][i] (Algorithm 4's coin,
// from problem i's seed and p).
__global__ void __launch_bounds__(256)
batch_coins_kernel(const unsigned long long* __restrict__ seeds, const double* __restrict__ ps, int n, int K,
                   unsigned char* __restrict__ coins) {
  pdl_enter();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)K * n) return;
  const int i = (int)(t % n);
  coins[t] = (unsigned char)Philox4x64::coin(seeds[i], ps[i], (uint64_t)(t / n));
}

// After the solve, one block per problem: its objective and timestamp records
// packed as rows of K entries, and (for device-memory iterates) its result copied
// to x_dst[i].
__global__ void __launch_bounds__(256)
batch_trace_kernel(const BatchProb* __restrict__ probs, const BatchState* __restrict__ state, int K,
                   double* __restrict__ obj_out, unsigned long long* __restrict__ ts_out,
                   float* const* __restrict__ x_dst) {
  pdl_enter();
  const BatchProb& P = probs[blockIdx.x];
  const int iters = state[blockIdx.x].iters;
  const size_t row = (size_t)blockIdx.x * K;
  for (int k = threadIdx.x; k < iters; k += blockDim.x) {
    obj_out[row + k] = P.obj[k];
    ts_out[row + k] = P.ts[k];
  }
  if (x_dst) {
    const float* x = (iters & 1) ? P.x1 : P.x0;
    float* dst = x_dst[blockIdx.x];
    const size_t npx = (size_t)P.H * P.W;
    for (size_t o = threadIdx.x; o < npx; o += blockDim.x) dst[o] = x[o];
  }
}

}  // namespace

int batch_fgp_tile_w() { return BT_TW; }
int batch_fgp_tile_h() { return BT_TH; }
int batch_chunk() { return CHUNK; }
int batch_fgp_iters_per_launch() { return BT_TB; }
int batch_fgp_resident_ctas() {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_fgp_kernel<float, 2>, 256, 0) != cudaSuccess)
    return 0;
  return sms * (per_sm > 0 ? per_sm : 1);
}

namespace {
cudaError_t batch_blur(const BatchLaunch& L, int par, bool step, cudaStream_t s) {
  switch (L.blur_radius) {
#define TVS_BB_R(R_)                                                                                   \
  case R_:                                                                                             \
    launch_kernel(batch_blur_fb_kernel<R_>, dim3(L.n_blur_tiles), dim3(FNT), 0, s, L.probs, L.state,   \
                  L.blur_tiles, L.coins, L.n, (const int*)L.kctr, par, step ? 1 : 0, L.part_a, L.part_b); \
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
  launch_kernel(batch_active_kernel, dim3(1), dim3(1024), 0, s, L.probs, (const BatchState*)L.state, L.coins, L.n,
                L.kctr, L.tile_range, L.chunk_range, L.scan_tiles, L.scan_chunks, L.work,
                L.n_work);
  int fin_pair = 0;  // pair holding p_N
  if (L.n_inner > 0 && L.use_prox) {
    int q = 0, j = 0;
    for (int g = 1; g <= L.n_inner; ++j) {
      const int it = L.n_inner - g + 1 < BT_TB ? L.n_inner - g + 1 : BT_TB;
      TBBetas b{};
      for (int m = 0; m < it; ++m) b.b[m] = L.betas[g - 1 + m];
      switch (L.dtype * 3 + L.nonneg_mode) {
#define TVS_BF(IDX, T_, NN_)                                                                              \
  case IDX:                                                                                           \
    launch_kernel(batch_fgp_kernel<T_, NN_>, dim3(L.fgp_grid), dim3(256), 0, s, L.probs,                \
                  (const int*)L.scan_tiles, L.n, q, b, it, L.work + j);                              \
    break;
        TVS_BF(0, float, 0) TVS_BF(1, float, 1) TVS_BF(2, float, 2)
        TVS_BF(3, __nv_bfloat16, 0) TVS_BF(4, __nv_bfloat16, 1) TVS_BF(5, __nv_bfloat16, 2)
        TVS_BF(6, __half, 0) TVS_BF(7, __half, 1) TVS_BF(8, __half, 2)
        TVS_BF(9, q15, 0) TVS_BF(10, q15, 1) default: TVS_BF(11, q15, 2)
#undef TVS_BF
      }
      q = 1 - q;
      g += it;
    }
    fin_pair = q;
  }
  // with no inner iterations the finalisation gives x_{k+1} = z and h = 0 (lam = 0
  // in every descriptor)
  switch (L.dtype) {
    case DUAL_F32:
      launch_kernel(batch_finalize_kernel<float>, dim3(L.fin_grid), dim3(256), 0, s, L.probs,
                    L.chunk_range, (const int*)L.scan_chunks, L.n, par, fin_pair);
      break;
    case DUAL_BF16:
      launch_kernel(batch_finalize_kernel<__nv_bfloat16>, dim3(L.fin_grid), dim3(256), 0, s, L.probs,
                    L.chunk_range, (const int*)L.scan_chunks, L.n, par, fin_pair);
      break;
    case DUAL_F16:
      launch_kernel(batch_finalize_kernel<__half>, dim3(L.fin_grid), dim3(256), 0, s, L.probs,
                    L.chunk_range, (const int*)L.scan_chunks, L.n, par, fin_pair);
      break;
    default:
      launch_kernel(batch_finalize_kernel<q15>, dim3(L.fin_grid), dim3(256), 0, s, L.probs,
                    L.chunk_range, (const int*)L.scan_chunks, L.n, par, fin_pair);
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_init(const BatchLaunch& L, const float* const* x_src, int K, cudaStream_t s) {
  launch_kernel(batch_init_kernel, dim3(L.n_all_chunks), dim3(256), 0, s, L.probs, L.chunk_range, L.n, x_src,
                L.dtype == DUAL_F32 ? 4 : 2, K);
  return cudaGetLastError();
}

cudaError_t launch_batch_coins(const unsigned long long* seeds, const double* ps, int n, int K,
                               unsigned char* coins, cudaStream_t s) {
  const long long total = (long long)K * n;
  if (total == 0) return cudaSuccess;
  launch_kernel(batch_coins_kernel, dim3((unsigned)((total + 255) / 256)), dim3(256), 0, s, seeds, ps, n, K, coins);
  return cudaGetLastError();
}

cudaError_t launch_batch_trace(const BatchLaunch& L, int K, double* obj_out, unsigned long long* ts_out,
                               float* const* x_dst, cudaStream_t s) {
  launch_kernel(batch_trace_kernel, dim3(L.n), dim3(256), 0, s, L.probs, (const BatchState*)L.state, K, obj_out,
                ts_out, x_dst);
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
