// C ABI (include/tvs.h): contexts, problems and the outer-loop drivers.
//
// Every outer iteration of a solver is one CUDA-graph launch.  A solver captures
// one graph per (coin value, buffer parity): the iterate ping-pongs between
// x[0] and x[1], so iteration k reads x[k % 2] and writes x[(k+1) % 2], and the
// Philox coin schedule, a pure function of (seed, p, k), is drawn on the host
// before the loop.  Graphs are iteration-independent: the objective reduction
// takes its trace index from a device counter it increments itself.
//
// ProxSkip (Algorithm 4), iteration k, parity c = k % 2, A the forward operator:
//   step kernels : out = x[c] - gamma A^T(A x[c] - b) + ch h     (+ partials of F(x[c]))
//                  skip: out = x[c+1], ch = gamma          (x_{k+1} = x^)
//                  prox: out = z,      ch = gamma - gamma/p (z = x^ - (gamma/p) h)
//   reduce       : F(x_k) -> trace (index k - 1)
//   prox only    : N x FGP on z with lam = (gamma/p) alpha, warm-started dual;
//                  finalize x[c+1] = P_X(z + lam div p_N), h = (p/gamma)(x[c+1] - z)
// The last line is Algorithm 4's h + (p/gamma)(x_{k+1} - x^_{k+1}) with
// x^ = z + (gamma/p) h substituted; on skip iterations h is left untouched.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.hpp"
#include "tvs.h"

using namespace tvs;

namespace {

thread_local std::string g_err;

tvs_status fail(tvs_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CUDA_TRY(call)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(e_ == cudaErrorMemoryAllocation ? TVS_ENOMEM : TVS_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                         \
  } while (0)

#define TVS_TRY(call)                  \
  do {                                 \
    tvs_status s_ = (call);            \
    if (s_ != TVS_OK) return s_;       \
  } while (0)

constexpr int LAG = 8;  // outer iterations the host may run ahead of the device
// Outer iterations per chunk graph: CHUNK iterations from a multiple of CHUNK run
// as one graph launch, captured for their coin pattern the first time it occurs,
// so the programmatic launch chain continues across those iterations instead of
// ending at a graph boundary (which drains the device and costs a full launch).
// CHUNK_DEPTH chunk launches may be queued ahead of the device.
constexpr int CHUNK = 4;
constexpr int CHUNK_DEPTH = 2;

bool is_fin(double v) { return std::isfinite(v); }

}  // namespace

// The CUDA graphs of one solve: one outer iteration each, by coin and by the
// parity of the iterate buffers, and runs of CHUNK iterations from an even
// iteration, by their coins (bit i: the coin of the run's i-th iteration).
struct GraphSet {
  cudaGraphExec_t exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [coin][parity]
  cudaGraphExec_t chunk[1 << CHUNK] = {};                                 // [coin pattern]
  GraphSet() = default;
  GraphSet(const GraphSet&) = delete;
  GraphSet& operator=(const GraphSet&) = delete;
  ~GraphSet() {
    for (auto& row : exec)
      for (auto& e : row)
        if (e) cudaGraphExecDestroy(e);
    for (auto& e : chunk)
      if (e) cudaGraphExecDestroy(e);
  }
};

// Graphs of one solver family kept in a problem between solves: `key` lists
// every value the captured launches bake in (scalars, kernel configuration, and
// the problem's buffer generation), so a later solve with the same key replays
// them instead of capturing and instantiating them again.
struct GraphCache {
  std::vector<double> key;
  std::unique_ptr<GraphSet> G;
};
enum GraphSlot { GS_FB = 0, GS_PD = 1, GS_PD1 = 2, GS_PDX = 3, GS_COUNT = 4 };

struct tvs_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* prox_scratch = nullptr;
  size_t prox_scratch_bytes = 0;
  double* red_out = nullptr;  // one double for tvs_objective
  int* flags = nullptr;       // scratch flags for tvs_objective
  Partial* parts = nullptr;    // partials for tvs_objective
  size_t parts_cap = 0;
  cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
  cudaEvent_t ring[LAG] = {};
  cudaStream_t side = nullptr;                       // captured side branch (objective records)
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;  // fork / join of that branch
  size_t bytes = 0;
  FgpConfig fgp;          // forced configuration (TVS_FGP_CONFIG), or tb == 0 to autotune
  struct Tuned {
    int nx, ny, dtype;
    FgpConfig cfg;
  };
  std::vector<Tuned> tuned;  // autotuner cache, one entry per 2D shape and dual type
  std::vector<tvs_problem*> problems;  // live problems, destroyed with the context
  struct BatchCache* batch = nullptr;  // set-up and graphs of the last batched solve
};

struct tvs_problem {
  tvs_ctx* ctx = nullptr;
  tvs_problem_desc desc{};
  Dims dims;
  size_t n = 0, m = 0;
  BlurW bw{};
  CTGeom geom{};
  float4* angle_tab = nullptr;
  float4* angle_tab2 = nullptr;
  float* xt = nullptr;
  float* b = nullptr;
  float* x[2] = {nullptr, nullptr};
  float* z = nullptr;
  float* h = nullptr;
  float* r = nullptr;
  float* y = nullptr;
  float* axp = nullptr;
  void* dual[4] = {nullptr, nullptr, nullptr, nullptr};
  Partial* part_a = nullptr;
  Partial* part_b = nullptr;
  int max_parts = 0;
  double* obj_dev = nullptr;
  unsigned long long* ts_dev = nullptr;   // [cap] objective timestamps, [cap] = solve start
  unsigned long long* fgp_ts = nullptr;   // 2 per prox call
  float* beta_dev = nullptr;              // FISTA outer extrapolation table
  int trace_cap = 0;
  int* flags = nullptr;  // [0] done [1] reached k [2] trace counter [3] prox counter [4] non-finite F seen
  int* done_host = nullptr;               // pinned, mapped
  int* done_host_dev = nullptr;
  int* count = nullptr;
  float* uref = nullptr;        // reference solution (tvs_problem_set_reference)
  double uref_norm2 = 0.0;
  Partial* part_c = nullptr;     // partials of ||x - uref||^2
  double* dist_dev = nullptr;   // relative distance per trace entry
  float* aux = nullptr;         // m floats, allocated by the first explicit PDHG solve
  size_t bytes = 0;
  // bumped whenever a buffer that captured graphs name is allocated anew
  unsigned long long gen = 0;
  GraphCache graphs[GS_COUNT];
};

namespace {

// Host-side fault injection for tests, off unless asked for: with
// TVS_FAULT_INJECT=alloc:N in the environment, the N-th device allocation after
// the variable took that value fails as if the device had run out of memory (no
// CUDA call is made for it), so the cleanup of every TVS_ENOMEM path can be
// exercised without touching the GPU's real state.
bool inject_alloc_failure() {
  static std::mutex mu;
  static std::string last;
  static long count = 0;
  const char* e = getenv("TVS_FAULT_INJECT");
  std::lock_guard<std::mutex> lock(mu);
  if (!e || strncmp(e, "alloc:", 6) != 0) {
    last.clear();
    count = 0;
    return false;
  }
  if (last != e) {
    last = e;
    count = 0;
  }
  return ++count == atol(e + 6);
}

tvs_status dalloc(tvs_ctx* ctx, size_t* owner_bytes, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return TVS_OK;
  if (inject_alloc_failure()) return fail(TVS_ENOMEM, "cudaMalloc(%zu bytes) failed: injected", bytes);
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(TVS_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  ctx->bytes += bytes;
  if (owner_bytes) *owner_bytes += bytes;
  return TVS_OK;
}

template <typename T>
tvs_status palloc(tvs_problem* P, T** p, size_t count) {
  return dalloc(P->ctx, &P->bytes, (void**)p, count * sizeof(T));
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

bool valid_dual(int d) {
  return d == TVS_DUAL_F32 || d == TVS_DUAL_BF16 || d == TVS_DUAL_F16 || d == TVS_DUAL_Q15;
}

std::vector<float> fgp_betas(int n_iter) {
  // beta of inner iteration i (1-based): 0 for i = 1, (t_{i-1} - 1) / t_i after,
  // with t_1 = 1 and t_{i} = (1 + sqrt(1 + 4 t_{i-1}^2)) / 2.
  std::vector<float> b(n_iter > 0 ? n_iter : 0, 0.f);
  double t = 1.0;
  for (int i = 2; i <= n_iter; ++i) {
    const double tn = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
    b[i - 1] = (float)((t - 1.0) / tn);
    t = tn;
  }
  return b;
}

// N inner iterations on z starting from the dual in buf[0]; returns the index
// of the buffer that holds p_N.  2D problems use the temporally blocked kernel
// (pairs (buf[0], buf[1]) and (buf[2], buf[3]) alternate as input and output);
// otherwise the one-iteration kernel rotates through buf[0..2].
tvs_status launch_fgp_sequence(const FgpConfig& cfg, const Dims& d, const float* z,
                               void* const buf[4], int n_iter, const std::vector<float>& betas,
                               float lam, int dtype, bool nonneg, cudaStream_t s, int* final_idx) {
  const float inv_step = (float)(1.0 / (4.0 * d.ndim * (double)lam));
  if (d.ndim == 2 && cfg.tb > 1) {
    int q = 0;
    for (int g = 1; g <= n_iter;) {
      const int it = std::min(cfg.tb, n_iter - g + 1);
      void* pc = buf[2 * q];
      void* pp = g == 1 ? pc : buf[2 * q + 1];
      CUDA_TRY(launch_fgp_block(cfg, d, z, pc, pp, buf[2 * (1 - q)], buf[2 * (1 - q) + 1], lam, inv_step,
                                &betas[g - 1], it, dtype, nonneg, s));
      q = 1 - q;
      g += it;
    }
    *final_idx = 2 * q;
    return TVS_OK;
  }
  for (int i = 1; i <= n_iter; ++i) {
    void* cur = buf[(i - 1) % 3];
    void* prev = i >= 2 ? buf[(i - 2) % 3] : cur;
    void* out = buf[i % 3];
    CUDA_TRY(launch_fgp_iter(d, z, cur, prev, out, lam, inv_step, betas[i - 1], dtype, nonneg, s));
  }
  *final_idx = n_iter % 3;
  return TVS_OK;
}

// Configuration forced through TVS_FGP_CONFIG ("tb,cpl,rpw"), else tb = 0
// (autotune per shape).
FgpConfig default_fgp_config() {
  FgpConfig c;
  c.tb = 0;
  if (const char* e = getenv("TVS_FGP_CONFIG")) {
    FgpConfig t;
    if (sscanf(e, "%d,%d,%d", &t.tb, &t.cpl, &t.rpw) >= 1 && fgp_config_valid(t)) c = t;
  }
  return c;
}

// Autotuner for the blocked 2D inner kernel: the first use of a (shape, dual
// type) in a context times each candidate tile shape / depth on the caller's z
// (two launches of 4 iterations after one warm-up, CUDA events on the context's
// stream), reading the dual in `home` and writing only `scratch0/1`, and keeps
// the fastest.  Candidates: register-blocked 32x40, 64x32 and 64x40 regions, the
// shared-memory 32x40 region.
tvs_status fgp_config_for(tvs_ctx* C, const Dims& d, int dtype, const float* z, void* home,
                          void* scratch0, void* scratch1, FgpConfig* out) {
  if (d.ndim != 2) {
    *out = FgpConfig();
    out->tb = 1;
    return TVS_OK;
  }
  if (C->fgp.tb != 0) {
    *out = C->fgp;
    return TVS_OK;
  }
  for (const auto& t : C->tuned)
    if (t.nx == d.nx && t.ny == d.ny && t.dtype == dtype) {
      *out = t.cfg;
      return TVS_OK;
    }
  // optional on-disk cache (TVS_TUNE_CACHE=path): lines "nx ny dtype tb cpl rpw"
  const char* cache = getenv("TVS_TUNE_CACHE");
  if (cache && cache[0]) {
    if (FILE* f = fopen(cache, "r")) {
      int a, b, c, t0, t1, t2;
      bool found = false;
      while (fscanf(f, "%d %d %d %d %d %d", &a, &b, &c, &t0, &t1, &t2) == 6) {
        FgpConfig k;
        k.tb = t0;
        k.cpl = t1;
        k.rpw = t2;
        if (a == d.nx && b == d.ny && c == dtype && fgp_config_valid(k)) {
          *out = k;
          found = true;
        }
      }
      fclose(f);
      if (found) {
        C->tuned.push_back({d.nx, d.ny, dtype, *out});
        return TVS_OK;
      }
    }
  }
  const int cands[][3] = {{4, 1, 105}, {4, 2, 104}, {4, 2, 105}, {4, 1, 5}, {5, 2, 104}};
  const float betas[8] = {0.f, 0.f, 0.2f, 0.4f, 0.5f, 0.55f, 0.6f, 0.65f};
  cudaStream_t s = C->stream;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  FgpConfig best;
  float best_ms = 1e30f;
  // three rounds over the candidates, each timing 6 launches of as many
  // iterations as the candidate blocks after a warm-up; a candidate's score is
  // its best round's time per inner iteration (robust against clock ramps and
  // noise, and comparable across depths)
  const int ncand = (int)(sizeof(cands) / sizeof(cands[0]));
  std::vector<float> score(ncand, 1e30f);
  for (int round = 0; round < 3; ++round) {
    for (int ci = 0; ci < ncand; ++ci) {
      FgpConfig c;
      c.tb = cands[ci][0];
      c.cpl = cands[ci][1];
      c.rpw = cands[ci][2];
      float ms = 0.f;
      cudaError_t e = launch_fgp_block(c, d, z, home, home, scratch0, scratch1, 0.1f, 1.25f, betas, c.tb, dtype,
                                       false, s);
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      for (int r = 0; r < 6 && e == cudaSuccess; ++r)
        e = launch_fgp_block(c, d, z, home, home, scratch0, scratch1, 0.1f, 1.25f, betas, c.tb, dtype, false, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return fail(TVS_ECUDA, "fgp autotune: %s", cudaGetErrorString(e));
      }
      score[ci] = std::min(score[ci], ms / c.tb);
    }
  }
  for (int ci = 0; ci < ncand; ++ci)
    if (score[ci] < best_ms) {
      best_ms = score[ci];
      best.tb = cands[ci][0];
      best.cpl = cands[ci][1];
      best.rpw = cands[ci][2];
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  C->tuned.push_back({d.nx, d.ny, dtype, best});
  if (cache && cache[0]) {
    if (FILE* f = fopen(cache, "a")) {
      fprintf(f, "%d %d %d %d %d %d\n", d.nx, d.ny, dtype, best.tb, best.cpl, best.rpw);
      fclose(f);
    }
  }
  *out = best;
  return TVS_OK;
}

tvs_status copy_in(float* dst, const float* src, size_t n, tvs_mem mem, cudaStream_t s) {
  CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(float),
                           mem == TVS_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  return TVS_OK;
}

tvs_status copy_out(float* dst, const float* src, size_t n, tvs_mem mem, cudaStream_t s) {
  CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(float),
                           mem == TVS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  return TVS_OK;
}

tvs_status ensure_trace(tvs_problem* P, int K) {
  if (K + 1 <= P->trace_cap) return TVS_OK;
  if (P->trace_cap > 0) {
    const size_t old = (size_t)P->trace_cap * (2 * sizeof(double) + 2 * sizeof(unsigned long long) + sizeof(float)) +
                       sizeof(unsigned long long);
    P->bytes -= old;
    P->ctx->bytes -= old;
  }
  dfree(P->obj_dev);
  dfree(P->ts_dev);
  dfree(P->fgp_ts);
  dfree(P->beta_dev);
  dfree(P->dist_dev);
  P->dist_dev = nullptr;
  P->obj_dev = nullptr;
  P->ts_dev = nullptr;
  P->fgp_ts = nullptr;
  P->beta_dev = nullptr;
  const int cap = K + 1;
  ++P->gen;
  TVS_TRY(palloc(P, &P->obj_dev, cap));
  TVS_TRY(palloc(P, &P->ts_dev, cap + 1));
  TVS_TRY(palloc(P, &P->fgp_ts, 2 * (size_t)cap));
  TVS_TRY(palloc(P, &P->beta_dev, cap));
  TVS_TRY(palloc(P, &P->dist_dev, cap));
  P->trace_cap = cap;
  return TVS_OK;
}

// ---------------------------------------------------------------- per-operator pieces
// Partials of the data term / TV term written by the step kernels.
int step_parts_a(const tvs_problem* P) {
  switch (P->desc.op.kind) {
    case TVS_OP_GAUSS_BLUR: return fb_step_blocks_2d(P->dims.ny, P->dims.nx, P->bw.R);
    case TVS_OP_PARALLEL_BEAM: return ct_fwd_blocks(P->geom);
    default: return pointwise_blocks(P->n);
  }
}
int step_parts_b(const tvs_problem* P) {
  switch (P->desc.op.kind) {
    case TVS_OP_GAUSS_BLUR: return fb_step_blocks_2d(P->dims.ny, P->dims.nx, P->bw.R);
    case TVS_OP_PARALLEL_BEAM: return ct_bwd_blocks(P->geom);
    default: return pointwise_blocks(P->n);
  }
}

// out = src - gamma A^T(A src - b) + ch h; partials of F(src) into part_a/part_b.
tvs_status fb_step(tvs_problem* P, const float* src, float* out, const float* h, float gamma,
                   float ch, cudaStream_t s) {
  const Dims& d = P->dims;
  switch (P->desc.op.kind) {
    case TVS_OP_GAUSS_BLUR:
      CUDA_TRY(launch_blur_fb_step(d.ny, d.nx, src, P->b, h, out, P->bw, gamma, ch, P->part_a, P->part_b, s));
      break;
    case TVS_OP_PARALLEL_BEAM:
      CUDA_TRY(launch_ct_forward(P->geom, src, P->r, nullptr, P->b, 0.f, P->part_a, CT_FWD_RESID, s));
      CUDA_TRY(launch_ct_backward(P->geom, P->r, src, h, out, gamma, ch, P->part_b, s));
      break;
    default:
      CUDA_TRY(launch_identity_step(d, src, P->b, h, out, gamma, ch, P->part_a, P->part_b, s));
  }
  return TVS_OK;
}

InnerStamp inner_stamp(tvs_problem* P) { return InnerStamp{P->fgp_ts, P->flags + 3}; }

// Partials of F(x) only; returns their counts.
tvs_status objective_parts(tvs_problem* P, const float* x, Partial* pa, Partial* pb, int* na, int* nb,
                           cudaStream_t s) {
  const Dims& d = P->dims;
  switch (P->desc.op.kind) {
    case TVS_OP_GAUSS_BLUR:
      CUDA_TRY(launch_blur_residual(d.ny, d.nx, x, P->b, nullptr, P->bw, pa, pb, s));
      *na = *nb = tile_blocks_2d(d.ny, d.nx);
      break;
    case TVS_OP_PARALLEL_BEAM:
      CUDA_TRY(launch_ct_forward(P->geom, x, P->r, nullptr, P->b, 0.f, pa, CT_FWD_STORE, s));
      CUDA_TRY(launch_tv_partials(d, x, pb, s));
      *na = ct_fwd_blocks(P->geom);
      *nb = pointwise_blocks(P->n);
      break;
    default:
      CUDA_TRY(launch_identity_step(d, x, P->b, nullptr, nullptr, 0.f, 0.f, pa, pb, s));
      *na = *nb = pointwise_blocks(P->n);
  }
  return TVS_OK;
}

// PDHG pieces.  Backward step: out = x - sigma A^T y + ch h, TV(x) partials -> part_b.
tvs_status pd_backward(tvs_problem* P, const float* x, float* out, const float* h, float sigma,
                       float ch, cudaStream_t s, bool tv_partials = true) {
  const Dims& d = P->dims;
  Partial* pb = tv_partials ? P->part_b : nullptr;
  switch (P->desc.op.kind) {
    case TVS_OP_GAUSS_BLUR:
      CUDA_TRY(launch_blur_step(d.ny, d.nx, P->y, x, h, out, P->bw, sigma, ch, pb, s));
      break;
    case TVS_OP_PARALLEL_BEAM:
      CUDA_TRY(launch_ct_backward(P->geom, P->y, x, h, out, sigma, ch, pb, s));
      break;
    default:
      CUDA_TRY(launch_axpy_step(d, P->y, x, h, out, sigma, ch, pb, s));
  }
  return TVS_OK;
}

// PDHGSkip-1 dual step from x^ (xh): A x_{k+1} = A x_k + p A x^ kept in axp,
// y <- prox(y + tau A(x_{k+1} + x^)), data partials of F(x_{k+1}).
tvs_status pd1_forward(tvs_problem* P, const float* xh, float prob_p, float tau, cudaStream_t s) {
  const Dims& d = P->dims;
  switch (P->desc.op.kind) {
    case TVS_OP_GAUSS_BLUR:
      CUDA_TRY(launch_blur_pd1_dual(d.ny, d.nx, xh, P->axp, P->y, P->b, P->bw, prob_p, tau, P->part_a, s));
      break;
    case TVS_OP_PARALLEL_BEAM:
      CUDA_TRY(launch_ct_forward(P->geom, xh, P->axp, P->y, P->b, tau, P->part_a, CT_FWD_PD1, s, prob_p));
      break;
    default:
      CUDA_TRY(launch_pd1_dual_pointwise(P->m, xh, P->axp, P->y, P->b, prob_p, tau, P->part_a, s));
  }
  return TVS_OK;
}
int pd_parts_a(const tvs_problem* P) {
  switch (P->desc.op.kind) {
    case TVS_OP_GAUSS_BLUR: return tile_blocks_2d(P->dims.ny, P->dims.nx);
    case TVS_OP_PARALLEL_BEAM: return ct_fwd_blocks(P->geom);
    default: return pointwise_blocks(P->m);
  }
}
int pd_parts_b(const tvs_problem* P) {
  switch (P->desc.op.kind) {
    case TVS_OP_GAUSS_BLUR: return tile_blocks_2d(P->dims.ny, P->dims.nx);
    case TVS_OP_PARALLEL_BEAM: return ct_bwd_blocks(P->geom);
    default: return pointwise_blocks(P->n);
  }
}
// Forward dual step: y = prox_{tau f*}(y + tau A(2 x - x_prev)) using axp = A x_prev;
// axp <- A x; data partials of F(x) -> part_a.  init: only axp <- A x and partials.
tvs_status pd_forward(tvs_problem* P, const float* x, float tau, bool init, cudaStream_t s) {
  const Dims& d = P->dims;
  switch (P->desc.op.kind) {
    case TVS_OP_GAUSS_BLUR:
      if (init) {
        CUDA_TRY(launch_blur_residual(d.ny, d.nx, x, P->b, nullptr, P->bw, P->part_a, nullptr, s));
        CUDA_TRY(launch_blur(d.ny, d.nx, x, P->axp, P->bw, s));
      } else {
        CUDA_TRY(launch_blur_pd_dual(d.ny, d.nx, x, P->axp, P->y, P->b, P->bw, tau, P->part_a, s));
      }
      break;
    case TVS_OP_PARALLEL_BEAM:
      CUDA_TRY(launch_ct_forward(P->geom, x, P->axp, init ? nullptr : P->y, P->b, tau, P->part_a,
                                 init ? CT_FWD_STORE : CT_FWD_PD, s));
      break;
    default:
      if (init) {
        CUDA_TRY(launch_identity_step(d, x, P->b, nullptr, nullptr, 0.f, 0.f, P->part_a, nullptr, s));
        CUDA_TRY(cudaMemcpyAsync(P->axp, x, P->n * sizeof(float), cudaMemcpyDeviceToDevice, s));
      } else {
        CUDA_TRY(launch_pd_dual_pointwise(P->m, x, P->axp, P->y, P->b, tau, P->part_a, s));
      }
  }
  return TVS_OK;
}

template <typename F>
tvs_status capture(cudaStream_t s, cudaGraphExec_t* exec, F&& body) {
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  tvs_status st = body();
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (st != TVS_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(TVS_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(TVS_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  return TVS_OK;
}

// The problem's cached graphs of `slot` when they were captured under `key`
// (*fresh = false); otherwise an empty set, now cached under `key`, to capture
// into (*fresh = true).  The key is completed with the problem's buffer
// generation and the presence of a reference solution.
GraphSet& cached_graphs(tvs_problem* P, GraphSlot slot, std::vector<double> key, bool* fresh) {
  key.push_back((double)P->gen);
  key.push_back(P->uref ? 1.0 : 0.0);
  GraphCache& c = P->graphs[slot];
  if (c.G && c.key == key) {
    *fresh = false;
    return *c.G;
  }
  c.G.reset(new GraphSet());
  c.key = std::move(key);
  *fresh = true;
  return *c.G;
}

// Shared outer-loop machinery: pacing, trace readback.
struct LoopState {
  int iters = 0;
  int prox = 0;
  bool timed_out = false;
};

// Wall-clock limit of a solve's host loop (TVS_SOLVE_TIMEOUT_MS, none by
// default): once it has passed, no further iteration is launched and the solve
// returns TVS_ETIMEDOUT after its usual clean-up, with the trace of the
// iterations that ran.
double solve_timeout_ms() {
  const char* e = getenv("TVS_SOLVE_TIMEOUT_MS");
  const double v = e ? atof(e) : 0.0;
  return v > 0.0 ? v : 0.0;
}

// Captures the stream work of one outer iteration with the given coin, reading
// the iterate buffer of the given parity.
using IterBody = std::function<tvs_status(int coin, int parity)>;

// Launches the outer iterations: with `body`, runs of CHUNK iterations from a
// multiple of CHUNK as one chunk graph each (captured on first use of its coin
// pattern) and the remaining iterations one graph each, at most CHUNK_DEPTH
// launches ahead of the device; without it, one graph per iteration, LAG ahead.
// The host stops launching once the device has raised done_host.
tvs_status run_loop(tvs_problem* P, int K, const std::vector<unsigned char>& coins, GraphSet& G,
                    LoopState* ls, const IterBody* body = nullptr) {
  tvs_ctx* C = P->ctx;
  cudaStream_t s = C->stream;
  const double limit = solve_timeout_ms();
  const auto t0 = std::chrono::steady_clock::now();
  const int depth = body ? CHUNK_DEPTH : LAG;
  int k = 0;
  for (int j = 0; k < K; ++j) {
    if (j >= depth) {
      CUDA_TRY(cudaEventSynchronize(C->ring[(j - depth) % LAG]));
      if (*(volatile int*)P->done_host) break;
    }
    if (limit > 0.0 &&
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() > limit) {
      ls->timed_out = true;
      break;
    }
    if (body && k % CHUNK == 0 && K - k >= CHUNK) {
      int pat = 0, np = 0;
      for (int i = 0; i < CHUNK; ++i) {
        const int c = coins[k + i] ? 1 : 0;
        pat |= c << i;
        np += c;
      }
      if (!G.chunk[pat]) {
        const tvs_status st = capture(s, &G.chunk[pat], [&]() -> tvs_status {
          for (int i = 0; i < CHUNK; ++i) TVS_TRY((*body)((pat >> i) & 1, i & 1));
          return TVS_OK;
        });
        if (st != TVS_OK) {
          G.chunk[pat] = nullptr;
          return st;
        }
      }
      CUDA_TRY(cudaGraphLaunch(G.chunk[pat], s));
      k += CHUNK;
      ls->prox += np;
    } else {
      const int c = coins[k] ? 1 : 0;
      CUDA_TRY(cudaGraphLaunch(G.exec[c][k & 1], s));
      k += 1;
      ls->prox += c;
    }
    CUDA_TRY(cudaEventRecord(C->ring[j % LAG], s));
    ls->iters = k;
  }
  return TVS_OK;
}

tvs_status begin_solve(tvs_problem* P, int K, int flags_counter_start) {
  cudaStream_t s = P->ctx->stream;
  TVS_TRY(ensure_trace(P, K));
  *(volatile int*)P->done_host = 0;
  int f[5] = {0, -1, flags_counter_start, 0, 0};
  CUDA_TRY(cudaMemcpyAsync(P->flags, f, sizeof(f), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemsetAsync(P->obj_dev, 0xff, sizeof(double) * (K + 1), s));  // NaN pattern
  CUDA_TRY(cudaMemsetAsync(P->dist_dev, 0xff, sizeof(double) * (K + 1), s));
  CUDA_TRY(cudaEventRecord(P->ctx->ev_start, s));
  CUDA_TRY(launch_timestamp(P->ts_dev + P->trace_cap, s));
  return TVS_OK;
}

// Distance of x to the problem's reference, recorded at the trace index the
// preceding objective reduction used (no-op without a reference).
tvs_status track_distance(tvs_problem* P, const float* x, double target, cudaStream_t s) {
  if (!P->uref) return TVS_OK;
  CUDA_TRY(launch_dist_partials(P->n, x, P->uref, P->part_c, s));
  CUDA_TRY(launch_dist_record(P->part_c, pointwise_blocks(P->n), P->uref_norm2, P->dist_dev, target, P->flags,
                              P->done_host_dev, s));
  return TVS_OK;
}

tvs_status zero_dual(tvs_problem* P, int dtype) {
  CUDA_TRY(cudaMemsetAsync(P->dual[0], 0, dual_elem_bytes(dtype) * P->dims.ndim * P->n, P->ctx->stream));
  return TVS_OK;
}

tvs_status finish_solve(tvs_problem* P, int K, const LoopState& ls,
                        const std::vector<unsigned char>& coins, int n_inner, const FgpConfig& fc,
                        tvs_trace* tr) {
  tvs_ctx* C = P->ctx;
  cudaStream_t s = C->stream;
  CUDA_TRY(cudaEventRecord(C->ev_stop, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  const int iters = ls.iters;
  std::vector<double> obj(iters > 0 ? iters : 1);
  std::vector<unsigned long long> ts(iters + 1);
  int flags[5];
  if (iters > 0) {
    CUDA_TRY(cudaMemcpy(obj.data(), P->obj_dev, sizeof(double) * iters, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(ts.data(), P->ts_dev, sizeof(unsigned long long) * iters, cudaMemcpyDeviceToHost));
  }
  CUDA_TRY(cudaMemcpy(&ts[iters], P->ts_dev + P->trace_cap, sizeof(unsigned long long),
                      cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(flags, P->flags, sizeof(flags), cudaMemcpyDeviceToHost));
  const unsigned long long t0 = ts[iters];
  float solve_ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&solve_ms, C->ev_start, C->ev_stop));
  double fgp_ms = 0.0;
  const int nprox = flags[3];
  if (nprox > 0) {
    std::vector<unsigned long long> f(2 * (size_t)nprox);
    CUDA_TRY(cudaMemcpy(f.data(), P->fgp_ts, sizeof(unsigned long long) * f.size(), cudaMemcpyDeviceToHost));
    for (int i = 0; i < nprox; ++i) fgp_ms += (double)(f[2 * i + 1] - f[2 * i]) * 1e-6;
  }
  std::vector<double> dist;
  if (P->uref && iters > 0 && tr && tr->rel_dist) {
    dist.resize(iters);
    CUDA_TRY(cudaMemcpy(dist.data(), P->dist_dev, sizeof(double) * iters, cudaMemcpyDeviceToHost));
  }
  // the reduction raises flags[4] (and stops the solve) when an evaluated
  // objective is not finite: divergence or non-finite data
  const bool bad = flags[4] != 0;
  if (tr) {
    tr->iters_run = iters;
    tr->prox_calls = ls.prox;
    tr->reached = flags[0];
    tr->reached_iter = flags[0] ? flags[1] : -1;
    tr->time_to_target_s = -1.0;
    if (flags[0] && flags[1] >= 0 && flags[1] < iters)
      tr->time_to_target_s = (double)(ts[flags[1]] - t0) * 1e-9;
    tr->solve_ms = solve_ms;
    tr->fgp_ms = fgp_ms;
    const long long per_prox = (P->dims.ndim == 2 && fc.tb > 1) ? (n_inner + fc.tb - 1) / fc.tb : n_inner;
    tr->fgp_launches = (long long)nprox * per_prox;
    tr->fgp_pixel_iters = (long long)nprox * n_inner * (long long)P->n;
    const int lim = tr->cap < iters ? tr->cap : iters;
    for (int k = 0; k < lim; ++k) {
      if (tr->objective) tr->objective[k] = obj[k];
      if (tr->coins) tr->coins[k] = coins[k];
      if (tr->t_s) tr->t_s[k] = std::isnan(obj[k]) ? NAN : (double)(ts[k] - t0) * 1e-9;
      if (tr->rel_dist) tr->rel_dist[k] = dist.empty() ? NAN : dist[k];
    }
  }
  if (bad) return fail(TVS_ENUMERIC, "non-finite objective during the solve");
  if (ls.timed_out) return fail(TVS_ETIMEDOUT, "solve stopped at its time limit after %d iterations", iters);
  if (P->dims.ndim == 3 && fgp3d_take_wait_timeouts())
    return fail(TVS_ETIMEDOUT, "a 3D inner kernel gave up waiting for a TMA tile load; the result is incomplete");
  return TVS_OK;
}

tvs_status check_common(tvs_problem* P, int max_iter, int n_inner, int dual, double f_star,
                        double target, int every, const float* x) {
  if (!P) return fail(TVS_EINVAL, "null problem");
  if (!x) return fail(TVS_EINVAL, "null x_inout");
  if (max_iter < 0 || n_inner < 0) return fail(TVS_EINVAL, "max_iter and n_inner must be >= 0");
  if (!valid_dual(dual)) return fail(TVS_EINVAL, "invalid dual dtype %d", dual);
  if (!is_fin(f_star) || !is_fin(target) || target < 0) return fail(TVS_EINVAL, "invalid f_star/target");
  if (every < 0) return fail(TVS_EINVAL, "objective_every must be >= 1");
  return TVS_OK;
}

enum FBKind { FB_PGD, FB_FISTA, FB_PROXSKIP };

tvs_status fb_solve(tvs_problem* P, const tvs_fb_params* prm, float* x_io, tvs_mem mem,
                    tvs_trace* tr, FBKind kind) {
  if (!prm) return fail(TVS_EINVAL, "null params");
  TVS_TRY(check_common(P, prm->max_iter, prm->n_inner, prm->dual, prm->f_star, prm->target_rel_gap,
                       prm->objective_every, x_io));
  if (!(prm->gamma > 0) || !is_fin(prm->gamma)) return fail(TVS_EINVAL, "gamma must be > 0");
  if (!(prm->target_rel_dist >= 0) || !is_fin(prm->target_rel_dist)) return fail(TVS_EINVAL, "invalid target_rel_dist");
  const double p = kind == FB_PROXSKIP ? prm->p : 1.0;
  if (!(p > 0.0 && p <= 1.0)) return fail(TVS_EINVAL, "p must lie in (0, 1]");
  if (mem != TVS_MEM_DEVICE && mem != TVS_MEM_HOST) return fail(TVS_EINVAL, "invalid mem kind");
  const int K = prm->max_iter, N = prm->n_inner, every = prm->objective_every < 1 ? 1 : prm->objective_every;
  const int dtype = prm->dual;
  const bool nonneg = P->desc.nonneg != 0;
  const double gamma = prm->gamma, alpha = P->desc.alpha;
  const double lam_d = (kind == FB_PROXSKIP ? gamma / p : gamma) * alpha;
  const float lam = (float)lam_d;
  const bool use_prox = lam_d > 0.0;
  tvs_ctx* C = P->ctx;
  cudaStream_t s = C->stream;
  const Dims& d = P->dims;
  const std::vector<float> betas = fgp_betas(N);

  if (prm->resume && kind == FB_FISTA) return fail(TVS_EUNSUPPORTED, "FISTA cannot resume");
  if (prm->resume && prm->k0 < 0) return fail(TVS_EINVAL, "k0 must be >= 0");
  const long long k0 = prm->resume ? prm->k0 : 0;
  std::vector<unsigned char> coins(K, 1);
  if (kind == FB_PROXSKIP)
    for (int k = 0; k < K; ++k) coins[k] = (unsigned char)tvs_coin(prm->seed, p, k0 + k);

  TVS_TRY(begin_solve(P, K, kind == FB_FISTA ? 0 : -1));
  TVS_TRY(copy_in(P->x[0], x_io, P->n, mem, s));
  if (!prm->resume) TVS_TRY(zero_dual(P, dtype));
  float* aux = P->h;  // control variate h (ProxSkip) or extrapolated point y (FISTA)
  if (kind == FB_PROXSKIP && !prm->resume) CUDA_TRY(cudaMemsetAsync(P->h, 0, P->n * sizeof(float), s));
  if (kind == FB_FISTA) {
    CUDA_TRY(cudaMemcpyAsync(aux, P->x[0], P->n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    std::vector<float> bx(K > 0 ? K : 1, 0.f);
    double t = 1.0;
    for (int k = 0; k < K; ++k) {
      const double tn = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
      bx[k] = (float)((t - 1.0) / tn);
      t = tn;
    }
    CUDA_TRY(cudaMemcpyAsync(P->beta_dev, bx.data(), sizeof(float) * bx.size(), cudaMemcpyHostToDevice, s));
  }
  FgpConfig fcfg;
  TVS_TRY(fgp_config_for(C, d, dtype, P->x[0], P->dual[0], P->dual[2], P->dual[3], &fcfg));
  const int na = step_parts_a(P), nb = step_parts_b(P);
  const float fgamma = (float)gamma;
  const float h_coef = (float)(p / gamma);

  bool fresh = false;
  GraphSet& G = cached_graphs(P, GS_FB,
                              {(double)kind, gamma, p, alpha, nonneg ? 1.0 : 0.0, (double)dtype, (double)N,
                               (double)every, prm->f_star, prm->target_rel_gap, prm->target_rel_dist,
                               (double)fcfg.tb, (double)fcfg.cpl, (double)fcfg.rpw},
                              &fresh);
  // one outer iteration from x[par] to x[par ^ 1]
  const IterBody body = [&](int c, int par) -> tvs_status {
    float* xc = P->x[par];
    float* xn = P->x[par ^ 1];
    if (kind == FB_PROXSKIP) {
      if (c == 0) {
        TVS_TRY(fb_step(P, xc, xn, P->h, fgamma, fgamma, s));
      } else {
        TVS_TRY(fb_step(P, xc, P->z, P->h, fgamma, (float)(gamma - gamma / p), s));
      }
    } else {
      TVS_TRY(fb_step(P, kind == FB_FISTA ? aux : xc, P->z, nullptr, fgamma, 0.f, s));
    }
    const bool branch = kind != FB_FISTA && c == 1;  // overlap the record with the prox
    if (kind != FB_FISTA) {
      cudaStream_t rs = s;
      if (branch) {
        CUDA_TRY(cudaEventRecord(C->fork_ev, s));
        CUDA_TRY(cudaStreamWaitEvent(C->side, C->fork_ev, 0));
        rs = C->side;
      }
      CUDA_TRY(launch_reduce_record(P->part_a, na, P->part_b, nb, alpha, every, P->obj_dev,
                                    P->ts_dev, prm->f_star, prm->target_rel_gap, P->flags,
                                    P->done_host_dev, nullptr, rs));
      TVS_TRY(track_distance(P, xc, prm->target_rel_dist, rs));
      if (branch) CUDA_TRY(cudaEventRecord(C->join_ev, C->side));
    }
    if (c == 1) {
      int fin = 0;
      CUDA_TRY(launch_inner_start_stamp(inner_stamp(P), s));
      if (use_prox) TVS_TRY(launch_fgp_sequence(fcfg, d, P->z, P->dual, N, betas, lam, dtype, nonneg, s, &fin));
      CUDA_TRY(launch_fgp_finalize(d, P->z, P->dual[fin], dtype, use_prox ? lam : 0.f, nonneg, xn,
                                   kind == FB_PROXSKIP ? P->h : nullptr, h_coef,
                                   fin != 0 ? P->dual[0] : nullptr, xc,
                                   kind == FB_FISTA ? aux : nullptr, P->beta_dev, P->flags + 2,
                                   inner_stamp(P), s));
    }
    if (branch) CUDA_TRY(cudaStreamWaitEvent(s, C->join_ev, 0));
    if (kind == FB_FISTA) {
      int a = 0, b = 0;
      TVS_TRY(objective_parts(P, xn, P->part_a, P->part_b, &a, &b, s));
      CUDA_TRY(launch_reduce_record(P->part_a, a, P->part_b, b, alpha, every, P->obj_dev,
                                    P->ts_dev, prm->f_star, prm->target_rel_gap, P->flags,
                                    P->done_host_dev, nullptr, s));
      TVS_TRY(track_distance(P, xn, prm->target_rel_dist, s));
    }
    return TVS_OK;
  };
  if (fresh) {
    const tvs_status cst = [&]() -> tvs_status {
      for (int c = 0; c < 2; ++c) {
        if (c == 0 && kind != FB_PROXSKIP) continue;
        for (int par = 0; par < 2; ++par)
          TVS_TRY(capture(s, &G.exec[c][par], [&]() -> tvs_status { return body(c, par); }));
      }
      return TVS_OK;
    }();
    if (cst != TVS_OK) {
      P->graphs[GS_FB].G.reset();
      return cst;
    }
  }
  LoopState ls;
  TVS_TRY(run_loop(P, K, coins, G, &ls, &body));
  float* xfin = P->x[ls.iters & 1];
  if (kind != FB_FISTA && ls.iters > 0) {
    int a = 0, b = 0;
    TVS_TRY(objective_parts(P, xfin, P->part_a, P->part_b, &a, &b, s));
    CUDA_TRY(launch_reduce_record(P->part_a, a, P->part_b, b, alpha, 1, P->obj_dev, P->ts_dev,
                                  prm->f_star, prm->target_rel_gap, P->flags, P->done_host_dev,
                                  nullptr, s));
    TVS_TRY(track_distance(P, xfin, prm->target_rel_dist, s));
  }
  TVS_TRY(copy_out(x_io, xfin, P->n, mem, s));
  return finish_solve(P, K, ls, coins, use_prox ? N : 0, fcfg, tr);
}

tvs_status pd_solve(tvs_problem* P, const tvs_pd_params* prm, float* x_io, float* y_io, tvs_mem mem,
                    tvs_trace* tr, bool skip) {
  if (!prm) return fail(TVS_EINVAL, "null params");
  TVS_TRY(check_common(P, prm->max_iter, prm->n_inner, prm->dual, prm->f_star, prm->target_rel_gap,
                       prm->objective_every, x_io));
  if (!y_io) return fail(TVS_EINVAL, "null y_inout");
  if (!(prm->sigma > 0) || !(prm->tau > 0) || !is_fin(prm->sigma) || !is_fin(prm->tau))
    return fail(TVS_EINVAL, "sigma and tau must be > 0");
  if (!(prm->target_rel_dist >= 0) || !is_fin(prm->target_rel_dist)) return fail(TVS_EINVAL, "invalid target_rel_dist");
  const double p = skip ? prm->p : 1.0;
  if (!(p > 0.0 && p <= 1.0)) return fail(TVS_EINVAL, "p must lie in (0, 1]");
  if (mem != TVS_MEM_DEVICE && mem != TVS_MEM_HOST) return fail(TVS_EINVAL, "invalid mem kind");
  if (P->dims.ndim != 2) return fail(TVS_EUNSUPPORTED, "primal-dual solvers are 2D");
  const int K = prm->max_iter, N = prm->n_inner, every = prm->objective_every < 1 ? 1 : prm->objective_every;
  const int dtype = prm->dual;
  const bool nonneg = P->desc.nonneg != 0;
  const double sigma = prm->sigma, tau = prm->tau, alpha = P->desc.alpha;
  const double lam_d = (skip ? sigma / p : sigma) * alpha;
  const float lam = (float)lam_d;
  const bool use_prox = lam_d > 0.0;
  tvs_ctx* C = P->ctx;
  cudaStream_t s = C->stream;
  const Dims& d = P->dims;
  const std::vector<float> betas = fgp_betas(N);
  if (prm->resume && prm->k0 < 0) return fail(TVS_EINVAL, "k0 must be >= 0");
  const long long k0 = prm->resume ? prm->k0 : 0;
  std::vector<unsigned char> coins(K, 1);
  if (skip)
    for (int k = 0; k < K; ++k) coins[k] = (unsigned char)tvs_coin(prm->seed, p, k0 + k);

  TVS_TRY(begin_solve(P, K, -1));
  TVS_TRY(copy_in(P->x[0], x_io, P->n, mem, s));
  TVS_TRY(copy_in(P->y, y_io, P->m, mem, s));
  if (!prm->resume) TVS_TRY(zero_dual(P, dtype));
  if (skip && !prm->resume) CUDA_TRY(cudaMemsetAsync(P->h, 0, P->n * sizeof(float), s));
  TVS_TRY(pd_forward(P, P->x[0], (float)tau, true, s));
  FgpConfig fcfg;
  TVS_TRY(fgp_config_for(C, d, dtype, P->x[0], P->dual[0], P->dual[2], P->dual[3], &fcfg));
  const int na = pd_parts_a(P), nb = pd_parts_b(P);
  const float fs = (float)sigma, ft = (float)tau;
  bool fresh = false;
  GraphSet& G = cached_graphs(P, GS_PD,
                              {skip ? 1.0 : 0.0, sigma, tau, p, alpha, nonneg ? 1.0 : 0.0, (double)dtype,
                               (double)N, (double)every, prm->f_star, prm->target_rel_gap, prm->target_rel_dist,
                               (double)fcfg.tb, (double)fcfg.cpl, (double)fcfg.rpw},
                              &fresh);
  // one outer iteration from x[par] to x[par ^ 1]
  const IterBody body = [&](int c, int par) -> tvs_status {
    float* xc = P->x[par];
    float* xn = P->x[par ^ 1];
    if (skip) {
      if (c == 0) TVS_TRY(pd_backward(P, xc, xn, P->h, fs, fs, s));
      else TVS_TRY(pd_backward(P, xc, P->z, P->h, fs, (float)(sigma - sigma / p), s));
    } else {
      TVS_TRY(pd_backward(P, xc, P->z, nullptr, fs, 0.f, s));
    }
    // on prox iterations the objective record runs beside the inner iterations
    cudaStream_t rs = s;
    if (c == 1) {
      CUDA_TRY(cudaEventRecord(C->fork_ev, s));
      CUDA_TRY(cudaStreamWaitEvent(C->side, C->fork_ev, 0));
      rs = C->side;
    }
    CUDA_TRY(launch_reduce_record(P->part_a, na, P->part_b, nb, alpha, every, P->obj_dev,
                                  P->ts_dev, prm->f_star, prm->target_rel_gap, P->flags,
                                  P->done_host_dev, nullptr, rs));
    TVS_TRY(track_distance(P, xc, prm->target_rel_dist, rs));
    if (c == 1) CUDA_TRY(cudaEventRecord(C->join_ev, C->side));
    if (c == 1) {
      int fin = 0;
      CUDA_TRY(launch_inner_start_stamp(inner_stamp(P), s));
      if (use_prox) TVS_TRY(launch_fgp_sequence(fcfg, d, P->z, P->dual, N, betas, lam, dtype, nonneg, s, &fin));
      CUDA_TRY(launch_fgp_finalize(d, P->z, P->dual[fin], dtype, use_prox ? lam : 0.f, nonneg, xn,
                                   skip ? P->h : nullptr, (float)(p / sigma),
                                   fin != 0 ? P->dual[0] : nullptr, nullptr, nullptr, nullptr,
                                   nullptr, inner_stamp(P), s));
      CUDA_TRY(cudaStreamWaitEvent(s, C->join_ev, 0));  // the record read part_a
    }
    TVS_TRY(pd_forward(P, xn, ft, false, s));
    return TVS_OK;
  };
  if (fresh) {
    const tvs_status cst = [&]() -> tvs_status {
      for (int c = 0; c < 2; ++c) {
        if (c == 0 && !skip) continue;
        for (int par = 0; par < 2; ++par)
          TVS_TRY(capture(s, &G.exec[c][par], [&]() -> tvs_status { return body(c, par); }));
      }
      return TVS_OK;
    }();
    if (cst != TVS_OK) {
      P->graphs[GS_PD].G.reset();
      return cst;
    }
  }
  LoopState ls;
  TVS_TRY(run_loop(P, K, coins, G, &ls, &body));
  float* xfin = P->x[ls.iters & 1];
  if (ls.iters > 0) {
    CUDA_TRY(launch_tv_partials(d, xfin, P->part_b, s));
    CUDA_TRY(launch_reduce_record(P->part_a, na, P->part_b, pointwise_blocks(P->n), alpha, 1,
                                  P->obj_dev, P->ts_dev, prm->f_star, prm->target_rel_gap, P->flags,
                                  P->done_host_dev, nullptr, s));
    TVS_TRY(track_distance(P, xfin, prm->target_rel_dist, s));
  }
  TVS_TRY(copy_out(x_io, xfin, P->n, mem, s));
  TVS_TRY(copy_out(y_io, P->y, P->m, mem, s));
  return finish_solve(P, K, ls, coins, use_prox ? N : 0, fcfg, tr);
}

// PDHGSkip-1 (Algorithm 5, omega + 1 = 1/p).  Iteration k with theta_k = 1:
//   z = x - sigma A^T y; u = prox_{sigma g}(z) (N FGP iterations, warm dual);
//   x^ = (u - x)/p; x <- x + p x^ (in place); A x <- A x + p A x^;
//   y <- prox_{tau f*}(y + tau A(x + x^)); TV partials of the new x.
// With theta_k = 0, x^ = 0: x and A x are unchanged and y <- prox(y + tau A x) is a
// pointwise update from the stored A x (no prox, no projector application).
tvs_status pd1_solve(tvs_problem* P, const tvs_pd_params* prm, float* x_io, float* y_io, tvs_mem mem,
                     tvs_trace* tr) {
  if (!prm) return fail(TVS_EINVAL, "null params");
  TVS_TRY(check_common(P, prm->max_iter, prm->n_inner, prm->dual, prm->f_star, prm->target_rel_gap,
                       prm->objective_every, x_io));
  if (!y_io) return fail(TVS_EINVAL, "null y_inout");
  if (!(prm->sigma > 0) || !(prm->tau > 0) || !is_fin(prm->sigma) || !is_fin(prm->tau))
    return fail(TVS_EINVAL, "sigma and tau must be > 0");
  const double p = prm->p;
  if (!(p > 0.0 && p <= 1.0)) return fail(TVS_EINVAL, "p must lie in (0, 1]");
  if (mem != TVS_MEM_DEVICE && mem != TVS_MEM_HOST) return fail(TVS_EINVAL, "invalid mem kind");
  if (P->dims.ndim != 2) return fail(TVS_EUNSUPPORTED, "primal-dual solvers are 2D");
  const int K = prm->max_iter, N = prm->n_inner, every = prm->objective_every < 1 ? 1 : prm->objective_every;
  const int dtype = prm->dual;
  const bool nonneg = P->desc.nonneg != 0;
  const double sigma = prm->sigma, tau = prm->tau, alpha = P->desc.alpha;
  const double lam_d = sigma * alpha;
  const float lam = (float)lam_d;
  const bool use_prox = lam_d > 0.0;
  tvs_ctx* C = P->ctx;
  cudaStream_t s = C->stream;
  const Dims& d = P->dims;
  const std::vector<float> betas = fgp_betas(N);
  if (prm->resume && prm->k0 < 0) return fail(TVS_EINVAL, "k0 must be >= 0");
  const long long k0 = prm->resume ? prm->k0 : 0;
  std::vector<unsigned char> coins(K);
  for (int k = 0; k < K; ++k) coins[k] = (unsigned char)tvs_coin(prm->seed, p, k0 + k);

  TVS_TRY(begin_solve(P, K, -1));
  TVS_TRY(copy_in(P->x[0], x_io, P->n, mem, s));
  TVS_TRY(copy_in(P->y, y_io, P->m, mem, s));
  if (!prm->resume) {
    TVS_TRY(zero_dual(P, dtype));
    TVS_TRY(pd_forward(P, P->x[0], (float)tau, true, s));
    CUDA_TRY(launch_tv_partials(d, P->x[0], P->part_b, s));
  }
  // on resume, A x_k (kept up to date incrementally, A x += p A x^) and the
  // objective partials of x_k are the ones the previous solve left in the problem
  FgpConfig fcfg;
  TVS_TRY(fgp_config_for(C, d, dtype, P->x[0], P->dual[0], P->dual[2], P->dual[3], &fcfg));
  const int na = pd_parts_a(P), nb = pointwise_blocks(P->n);
  float* x = P->x[0];
  bool fresh = false;
  GraphSet& G = cached_graphs(P, GS_PD1,
                              {sigma, tau, p, alpha, nonneg ? 1.0 : 0.0, (double)dtype, (double)N, (double)every,
                               prm->f_star, prm->target_rel_gap, prm->target_rel_dist, (double)fcfg.tb,
                               (double)fcfg.cpl, (double)fcfg.rpw},
                              &fresh);
  // one outer iteration (x is updated in place: both parities are the same work)
  const IterBody body = [&](int c, int) -> tvs_status {
    CUDA_TRY(launch_reduce_record(P->part_a, na, P->part_b, nb, alpha, every, P->obj_dev, P->ts_dev,
                                  prm->f_star, prm->target_rel_gap, P->flags, P->done_host_dev, nullptr, s));
    TVS_TRY(track_distance(P, x, prm->target_rel_dist, s));
    if (c == 0) {
      CUDA_TRY(launch_pd1_dual_pointwise(P->m, nullptr, P->axp, P->y, P->b, (float)p, (float)tau, nullptr, s));
      return TVS_OK;
    }
    TVS_TRY(pd_backward(P, x, P->z, nullptr, (float)sigma, 0.f, s, false));
    int fin = 0;
    CUDA_TRY(launch_inner_start_stamp(inner_stamp(P), s));
    if (use_prox) TVS_TRY(launch_fgp_sequence(fcfg, d, P->z, P->dual, N, betas, lam, dtype, nonneg, s, &fin));
    CUDA_TRY(launch_fgp_finalize_pd1(d, P->z, P->dual[fin], dtype, use_prox ? lam : 0.f, nonneg, (float)p, x,
                                     P->h, fin != 0 ? P->dual[0] : nullptr, inner_stamp(P), s));
    TVS_TRY(pd1_forward(P, P->h, (float)p, (float)tau, s));
    CUDA_TRY(launch_tv_partials(d, x, P->part_b, s));
    return TVS_OK;
  };
  if (fresh) {
    const tvs_status cst = [&]() -> tvs_status {
      for (int c = 0; c < 2; ++c)
        for (int par = 0; par < 2; ++par)
          TVS_TRY(capture(s, &G.exec[c][par], [&]() -> tvs_status { return body(c, par); }));
      return TVS_OK;
    }();
    if (cst != TVS_OK) {
      P->graphs[GS_PD1].G.reset();
      return cst;
    }
  }
  LoopState ls;
  TVS_TRY(run_loop(P, K, coins, G, &ls, &body));
  if (ls.iters > 0) {
    CUDA_TRY(launch_reduce_record(P->part_a, na, P->part_b, nb, alpha, 1, P->obj_dev, P->ts_dev, prm->f_star,
                                  prm->target_rel_gap, P->flags, P->done_host_dev, nullptr, s));
    TVS_TRY(track_distance(P, x, prm->target_rel_dist, s));
  }
  TVS_TRY(copy_out(x_io, x, P->n, mem, s));
  TVS_TRY(copy_out(y_io, P->y, P->m, mem, s));
  return finish_solve(P, K, ls, coins, use_prox ? N : 0, fcfg, tr);
}

// Explicit PDHG with diagonal preconditioning (kernels and formulas in pdx.cu).
// Buffers: x[2] primal parity, dual[0..1] q parity (FP32, 2 n), z = A^T y,
// h = T (pixel steps), r = S (row steps), aux = A x+, axp = A x.
tvs_status apply_A(tvs_problem* P, const float* x, float* out, cudaStream_t s) {
  const Dims& d = P->dims;
  switch (P->desc.op.kind) {
    case TVS_OP_GAUSS_BLUR: CUDA_TRY(launch_blur(d.ny, d.nx, x, out, P->bw, s)); break;
    case TVS_OP_PARALLEL_BEAM:
      CUDA_TRY(launch_ct_forward(P->geom, x, out, nullptr, nullptr, 0.f, nullptr, CT_FWD_PLAIN, s));
      break;
    default: CUDA_TRY(cudaMemcpyAsync(out, x, P->n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  }
  return TVS_OK;
}
tvs_status apply_At(tvs_problem* P, const float* y, float* out, cudaStream_t s) {
  const Dims& d = P->dims;
  switch (P->desc.op.kind) {
    case TVS_OP_GAUSS_BLUR: CUDA_TRY(launch_blur(d.ny, d.nx, y, out, P->bw, s)); break;  // A = A^T
    case TVS_OP_PARALLEL_BEAM:
      CUDA_TRY(launch_ct_backward(P->geom, y, nullptr, nullptr, out, 0.f, 0.f, nullptr, s));
      break;
    default: CUDA_TRY(cudaMemcpyAsync(out, y, P->n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  }
  return TVS_OK;
}

tvs_status pdx_solve(tvs_problem* P, const tvs_pdx_params* prm, float* x_io, float* y_io, float* q_io,
                     tvs_mem mem, tvs_trace* tr) {
  if (!prm) return fail(TVS_EINVAL, "null params");
  TVS_TRY(check_common(P, prm->max_iter, 0, TVS_DUAL_F32, prm->f_star, prm->target_rel_gap,
                       prm->objective_every, x_io));
  if (!y_io) return fail(TVS_EINVAL, "null y_inout");
  if (!(prm->sigma > 0) || !(prm->tau > 0) || !is_fin(prm->sigma) || !is_fin(prm->tau))
    return fail(TVS_EINVAL, "sigma and tau must be > 0");
  if (prm->sigma * prm->tau > 1.0 + 1e-12) return fail(TVS_EINVAL, "sigma * tau must be <= 1");
  if (!(prm->target_rel_dist >= 0) || !is_fin(prm->target_rel_dist)) return fail(TVS_EINVAL, "invalid target_rel_dist");
  if (mem != TVS_MEM_DEVICE && mem != TVS_MEM_HOST) return fail(TVS_EINVAL, "invalid mem kind");
  if (P->dims.ndim != 2) return fail(TVS_EUNSUPPORTED, "primal-dual solvers are 2D");
  const int K = prm->max_iter, every = prm->objective_every < 1 ? 1 : prm->objective_every;
  const bool nonneg = P->desc.nonneg != 0;
  const double alpha = P->desc.alpha;
  const bool ident = P->desc.op.kind == TVS_OP_IDENTITY;
  tvs_ctx* C = P->ctx;
  cudaStream_t s = C->stream;
  const Dims& d = P->dims;
  if (!P->aux) TVS_TRY(palloc(P, &P->aux, P->m));
  float* T = P->h;
  float* S = P->r;

  TVS_TRY(begin_solve(P, K, -1));
  // step sizes from the row sums A 1 (into aux) and column sums A^T 1 (into z)
  if (ident) {
    CUDA_TRY(launch_pdx_precond(nullptr, nullptr, d.ny, d.nx, P->m, (float)prm->sigma, (float)prm->tau, T, S, s));
  } else {
    CUDA_TRY(launch_fill(P->x[1], P->n, 1.f, s));
    TVS_TRY(apply_A(P, P->x[1], P->aux, s));
    CUDA_TRY(launch_fill(P->axp, P->m, 1.f, s));
    TVS_TRY(apply_At(P, P->axp, P->z, s));
    CUDA_TRY(launch_pdx_precond(P->z, P->aux, d.ny, d.nx, P->m, (float)prm->sigma, (float)prm->tau, T, S, s));
  }
  TVS_TRY(copy_in(P->x[0], x_io, P->n, mem, s));
  TVS_TRY(copy_in(P->y, y_io, P->m, mem, s));
  float* q0 = (float*)P->dual[0];
  if (q_io) TVS_TRY(copy_in(q0, q_io, 2 * P->n, mem, s));
  else CUDA_TRY(cudaMemsetAsync(q0, 0, 2 * P->n * sizeof(float), s));
  // A x_0 and the data partials of x_0
  const float* ax0 = P->x[0];
  if (!ident) {
    TVS_TRY(apply_A(P, P->x[0], P->aux, s));
    ax0 = P->aux;
  }
  CUDA_TRY(launch_pdx_dual(P->m, ax0, P->axp, P->y, P->b, S, true, P->part_a, s));
  const int na = pointwise_blocks(P->m), nb = pdx_tv_blocks(d.ny, d.nx);
  const float s_d = (float)(0.5 * prm->tau);
  GraphSet G;
  // one iteration from (x, q)[par] to (x, q)[par ^ 1]
  const IterBody body = [&](int, int par) -> tvs_status {
    float* xc = P->x[par];
    float* xn = P->x[par ^ 1];
    const float* qc = (const float*)P->dual[par];
    float* qn = (float*)P->dual[par ^ 1];
    const float* g = P->y;
    if (!ident) {
      TVS_TRY(apply_At(P, P->y, P->z, s));
      g = P->z;
    }
    CUDA_TRY(launch_pdx_tv_step(d.ny, d.nx, xc, g, T, qc, xn, qn, (float)alpha, s_d, nonneg, P->part_b, s));
    CUDA_TRY(launch_reduce_record(P->part_a, na, P->part_b, nb, alpha, every, P->obj_dev, P->ts_dev,
                                  prm->f_star, prm->target_rel_gap, P->flags, P->done_host_dev, nullptr, s));
    TVS_TRY(track_distance(P, xc, prm->target_rel_dist, s));
    const float* ax = xn;
    if (!ident) {
      TVS_TRY(apply_A(P, xn, P->aux, s));
      ax = P->aux;
    }
    CUDA_TRY(launch_pdx_dual(P->m, ax, P->axp, P->y, P->b, S, false, P->part_a, s));
    return TVS_OK;
  };
  for (int par = 0; par < 2; ++par)
    TVS_TRY(capture(s, &G.exec[1][par], [&]() -> tvs_status { return body(1, par); }));
  std::vector<unsigned char> coins(K, 1);
  LoopState ls;
  TVS_TRY(run_loop(P, K, coins, G, &ls, &body));
  float* xfin = P->x[ls.iters & 1];
  const float* qfin = (const float*)P->dual[ls.iters & 1];
  if (ls.iters > 0) {
    CUDA_TRY(launch_tv_partials(d, xfin, P->part_b, s));
    CUDA_TRY(launch_reduce_record(P->part_a, na, P->part_b, pointwise_blocks(P->n), alpha, 1, P->obj_dev,
                                  P->ts_dev, prm->f_star, prm->target_rel_gap, P->flags, P->done_host_dev,
                                  nullptr, s));
    TVS_TRY(track_distance(P, xfin, prm->target_rel_dist, s));
  }
  TVS_TRY(copy_out(x_io, xfin, P->n, mem, s));
  TVS_TRY(copy_out(y_io, P->y, P->m, mem, s));
  if (q_io) TVS_TRY(copy_out(q_io, qfin, 2 * P->n, mem, s));
  return finish_solve(P, K, ls, coins, 0, FgpConfig{}, tr);
}

}  // namespace


// ---------------------------------------------------------------- batched ProxSkip
namespace {

struct BatchScratch {
  std::vector<void*> bufs;
  int* done_host = nullptr;
  ~BatchScratch() {
    for (void* b : bufs) cudaFree(b);
    if (done_host) cudaFreeHost(done_host);
  }
  template <typename T>
  tvs_status upload(const std::vector<T>& v, T** out, cudaStream_t s) {
    *out = nullptr;
    if (v.empty()) return TVS_OK;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, v.size() * sizeof(T));
    if (e != cudaSuccess) return fail(TVS_ENOMEM, "batch scratch: %s", cudaGetErrorString(e));
    bufs.push_back(p);
    e = cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(TVS_ECUDA, "batch upload: %s", cudaGetErrorString(e));
    *out = (T*)p;
    return TVS_OK;
  }
  template <typename T>
  tvs_status zeros(size_t count, T** out, cudaStream_t s) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T) + 8);
    if (e != cudaSuccess) return fail(TVS_ENOMEM, "batch scratch: %s", cudaGetErrorString(e));
    bufs.push_back(p);
    e = cudaMemsetAsync(p, 0, count * sizeof(T) + 8, s);
    if (e != cudaSuccess) return fail(TVS_ECUDA, "batch memset: %s", cudaGetErrorString(e));
    *out = (T*)p;
    return TVS_OK;
  }
};


bool same_fb_params(const tvs_fb_params& a, const tvs_fb_params& b) {
  return a.gamma == b.gamma && a.p == b.p && a.seed == b.seed && a.max_iter == b.max_iter &&
         a.n_inner == b.n_inner && a.dual == b.dual && a.f_star == b.f_star &&
         a.target_rel_gap == b.target_rel_gap && a.objective_every == b.objective_every && a.resume == b.resume &&
         a.k0 == b.k0 && a.target_rel_dist == b.target_rel_dist;
}

}  // namespace

// The set-up of a batched solve -- descriptors, work lists, coins, scratch and
// the two captured iteration graphs -- kept in the context for the next batched
// solve of the same problems (same buffer generations), parameters and memory
// kind, which then only resets the per-solve state.  Destroying any of its
// problems, or the context, drops it.
struct BatchCache {
  std::vector<tvs_problem*> probs;
  std::vector<unsigned long long> gens;
  std::vector<tvs_fb_params> prm;
  tvs_mem mem = TVS_MEM_DEVICE;
  BatchScratch S;
  BatchLaunch L{};
  GraphSet G;
  std::vector<BatchState> st0;
  std::vector<float> betas;  // L.betas points here
  unsigned long long* t0_dev = nullptr;
  double* obj_pack = nullptr;
  unsigned long long* ts_pack = nullptr;
  float** x_dev_list = nullptr;  // the caller's device iterates (set-up and trace kernels)
  size_t rows = 0;
  bool matches(int n, tvs_problem* const* P, const tvs_fb_params* p, tvs_mem m) const {
    if ((int)probs.size() != n || m != mem) return false;
    for (int i = 0; i < n; ++i)
      if (probs[i] != P[i] || gens[i] != P[i]->gen || !same_fb_params(prm[i], p[i])) return false;
    return true;
  }
  bool uses(const tvs_problem* P) const { return std::find(probs.begin(), probs.end(), P) != probs.end(); }
};

void drop_batch_cache(tvs_ctx* C) {
  if (!C->batch) return;
  cudaStreamSynchronize(C->stream);
  delete C->batch;
  C->batch = nullptr;
}

namespace {

tvs_status build_batch(tvs_ctx* C, int n, tvs_problem* const* probs, const tvs_fb_params* prm, tvs_mem mem,
                       int blur_radius, BatchCache* B) {
  const int K = prm[0].max_iter, N = prm[0].n_inner, dtype = prm[0].dual;
  cudaStream_t s = C->stream;
  B->probs.assign(probs, probs + n);
  B->gens.resize(n);
  for (int i = 0; i < n; ++i) B->gens[i] = probs[i]->gen;
  B->prm.assign(prm, prm + n);
  B->mem = mem;
  BatchScratch& S = B->S;
  BatchLaunch& L = B->L;
  // per-problem descriptors and work lists
  std::vector<BatchProb> desc(n);
  std::vector<int4> blur_tiles;
  std::vector<int2> ident_chunks, tile_range(n), chunk_range(n);
  int n_fgp_tiles = 0, n_all_chunks = 0;  // inner tiles / pixel chunks of all problems
  const int chunk = batch_chunk(), ftw = batch_fgp_tile_w(), fth = batch_fgp_tile_h();
  for (int i = 0; i < n; ++i) {
    tvs_problem* P = probs[i];
    const int H = P->dims.ny, W = P->dims.nx;
    const double gamma = prm[i].gamma, p = prm[i].p, alpha = P->desc.alpha;
    BatchProb& D = desc[i];
    memset(&D, 0, sizeof(D));
    D.H = H;
    D.W = W;
    D.fw = FastDiv((uint32_t)W);
    D.nonneg = P->desc.nonneg != 0;
    D.b = P->b;
    D.x0 = P->x[0];
    D.x1 = P->x[1];
    D.z = P->z;
    D.h = P->h;
    D.r = P->r;
    D.dual0 = P->dual[0];
    D.dual1 = P->dual[1];
    D.dual2 = P->dual[2];
    D.dual3 = P->dual[3];
    const double lam = gamma / p * alpha;
    D.lam = (float)lam;
    D.inv_step = lam > 0 ? (float)(1.0 / (8.0 * lam)) : 0.f;
    D.gamma = (float)gamma;
    D.ch_skip = (float)gamma;
    D.ch_prox = (float)(gamma - gamma / p);
    D.h_coef = (float)(p / gamma);
    D.alpha = alpha;
    D.f_star = prm[i].f_star;
    D.target = prm[i].target_rel_gap;
    D.bw = P->bw;
    D.obj = P->obj_dev;
    D.ts = P->ts_dev;
    const size_t npx = P->n;
    const int nchunks = (int)((npx + chunk - 1) / chunk);
    if (P->desc.op.kind == TVS_OP_GAUSS_BLUR) {
      D.part_off = (int)blur_tiles.size();
      const int fx = fb_step_tile_w(P->bw.R);  // tiles of the fused blur step
      const int tx = (W + fx - 1) / fx, ty = (H + fb_step_tile_h(P->bw.R) - 1) / fb_step_tile_h(P->bw.R);
      for (int y = 0; y < ty; ++y)
        for (int x = 0; x < tx; ++x) blur_tiles.push_back(make_int4(i, x, y, 0));
      D.part_n = tx * ty;
    } else {
      D.part_off = -1 - (int)ident_chunks.size();  // fixed up below (after the blur tiles)
      for (int c = 0; c < nchunks; ++c) ident_chunks.push_back(make_int2(i, c));
      D.part_n = nchunks;
    }
    chunk_range[i] = make_int2(n_all_chunks, nchunks);
    n_all_chunks += nchunks;
    const int fx = (W + ftw - 1) / ftw, fy = (H + fth - 1) / fth;
    tile_range[i] = make_int2(n_fgp_tiles, fx * fy);  // row-major tiles, decoded in the kernel
    n_fgp_tiles += fx * fy;
  }
  const int n_blur = (int)blur_tiles.size();
  for (auto& D : desc)
    if (D.part_off < 0) D.part_off = n_blur + (-1 - D.part_off);
  B->st0.assign(n, BatchState{0, -1, 0, 0});
  std::vector<unsigned long long> seeds(n);
  std::vector<double> pvals(n);
  for (int i = 0; i < n; ++i) {
    seeds[i] = prm[i].seed;
    pvals[i] = prm[i].p;
  }
  L.n = n;
  TVS_TRY(S.upload(desc, (BatchProb**)&L.probs, s));
  TVS_TRY(S.upload(B->st0, &L.state, s));
  TVS_TRY(S.upload(blur_tiles, (int4**)&L.blur_tiles, s));
  TVS_TRY(S.upload(ident_chunks, (int2**)&L.ident_chunks, s));
  {
    // the coins of every problem and outer iteration, drawn on the device
    unsigned long long* seeds_dev = nullptr;
    double* p_dev = nullptr;
    unsigned char* coins_dev = nullptr;
    TVS_TRY(S.upload(seeds, &seeds_dev, s));
    TVS_TRY(S.upload(pvals, &p_dev, s));
    TVS_TRY(S.zeros<unsigned char>((size_t)K * n, &coins_dev, s));
    CUDA_TRY(launch_batch_coins(seeds_dev, p_dev, n, K, coins_dev, s));
    L.coins = coins_dev;
  }
  TVS_TRY(S.upload(tile_range, (int2**)&L.tile_range, s));
  TVS_TRY(S.upload(chunk_range, (int2**)&L.chunk_range, s));
  TVS_TRY(S.zeros<int>((size_t)n + 1, &L.scan_tiles, s));
  TVS_TRY(S.zeros<int>((size_t)n + 1, &L.scan_chunks, s));
  L.n_blur_tiles = n_blur;
  L.n_ident_chunks = (int)ident_chunks.size();
  L.n_fgp_tiles = n_fgp_tiles;
  L.n_all_chunks = n_all_chunks;
  {
    int nn = 0;
    for (int i = 0; i < n; ++i) nn += probs[i]->desc.nonneg != 0;
    L.nonneg_mode = nn == 0 ? 0 : (nn == n ? 1 : 2);
  }
  {
    // persistent grids: every resident CTA slot of the inner kernel, and eight
    // 256-thread CTAs per SM for the finalisation (never more than the work)
    const int resident = batch_fgp_resident_ctas();
    if (resident <= 0) return fail(TVS_ECUDA, "cannot size the batched inner kernel");
    L.fgp_grid = std::max(1, std::min(resident, L.n_fgp_tiles));
    L.fin_grid = std::max(1, std::min(pointwise_blocks((size_t)L.n_all_chunks * 256), L.n_all_chunks));
  }
  TVS_TRY(S.zeros<int>(1, &L.kctr, s));
  L.n_work = std::max(1, (N + batch_fgp_iters_per_launch() - 1) / batch_fgp_iters_per_launch());
  TVS_TRY(S.zeros<int>((size_t)L.n_work, &L.work, s));
  TVS_TRY(S.zeros<Partial>((size_t)n_blur + ident_chunks.size(), &L.part_a, s));
  TVS_TRY(S.zeros<Partial>((size_t)n_blur + ident_chunks.size(), &L.part_b, s));
  TVS_TRY(S.zeros<unsigned long long>(1, &B->t0_dev, s));
  {
    cudaError_t e = cudaHostAlloc((void**)&S.done_host, sizeof(int) * n, cudaHostAllocMapped);
    if (e != cudaSuccess) {
      S.done_host = nullptr;
      return fail(TVS_ENOMEM, "cudaHostAlloc: %s", cudaGetErrorString(e));
    }
    memset(S.done_host, 0, sizeof(int) * n);
    CUDA_TRY(cudaHostGetDevicePointer((void**)&L.done_host, S.done_host, 0));
  }
  B->betas = fgp_betas(N);
  L.betas = B->betas.data();
  L.n_inner = N;
  L.dtype = dtype;
  L.blur_radius = blur_radius;
  L.use_prox = N > 0;
  if (mem == TVS_MEM_DEVICE) TVS_TRY(S.zeros<float*>((size_t)n, &B->x_dev_list, s));
  B->rows = (size_t)n * (K > 0 ? K : 1);
  TVS_TRY(S.zeros<double>(B->rows, &B->obj_pack, s));
  TVS_TRY(S.zeros<unsigned long long>(B->rows, &B->ts_pack, s));
  for (int par = 0; par < 2; ++par) {
    TVS_TRY(capture(s, &B->G.exec[1][par], [&]() -> tvs_status {
      CUDA_TRY(launch_batch_iteration(L, par, s));
      return TVS_OK;
    }));
  }
  return TVS_OK;
}

}  // namespace

namespace {
tvs_status validate_batch(tvs_ctx* C, int n, tvs_problem* const* probs, const tvs_fb_params* prm,
                          float* const* x_io, tvs_mem mem);
tvs_status batch_solve_in_order(tvs_ctx* C, int n, tvs_problem* const* probs, const tvs_fb_params* prm,
                                float* const* x_io, tvs_mem mem, tvs_trace* traces);
}  // namespace

// The batch is solved with its problems ordered by pixel count, smallest first:
// each inner launch hands out the tiles of the active problems in that order, so
// its last tiles are interior tiles of large images, the cheapest per tile (no
// edge masks), and the launch's tail is shorter.  Results and traces are
// returned in the caller's order.
extern "C" tvs_status proxskip_solve_batch(tvs_ctx* C, int n, tvs_problem* const* probs,
                                           const tvs_fb_params* prm, float* const* x_io, tvs_mem mem,
                                           tvs_trace* traces) {
  if (!C || n < 1 || !probs || !prm || !x_io) return fail(TVS_EINVAL, "null argument or n < 1");
  TVS_TRY(validate_batch(C, n, probs, prm, x_io, mem));
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return probs[a]->n < probs[b]->n; });
  std::vector<tvs_problem*> pp(n);
  std::vector<tvs_fb_params> pm(n);
  std::vector<float*> px(n);
  std::vector<tvs_trace> pt(traces ? n : 0);
  for (int j = 0; j < n; ++j) {
    pp[j] = probs[ord[j]];
    pm[j] = prm[ord[j]];
    px[j] = x_io[ord[j]];
    if (traces) pt[j] = traces[ord[j]];
  }
  const tvs_status st = batch_solve_in_order(C, n, pp.data(), pm.data(), px.data(), mem, traces ? pt.data() : nullptr);
  if (traces)
    for (int j = 0; j < n; ++j) traces[ord[j]] = pt[j];
  return st;
}

namespace {
// Arguments as for proxskip_solve_batch, checked (messages give the caller's
// problem indices).
tvs_status validate_batch(tvs_ctx* C, int n, tvs_problem* const* probs, const tvs_fb_params* prm,
                          float* const* x_io, tvs_mem mem) {
  if (mem != TVS_MEM_DEVICE && mem != TVS_MEM_HOST) return fail(TVS_EINVAL, "invalid mem kind");
  const int K = prm[0].max_iter, N = prm[0].n_inner, dtype = prm[0].dual;
  for (int i = 0; i < n; ++i) {
    tvs_problem* P = probs[i];
    if (!P || P->ctx != C) return fail(TVS_EINVAL, "problem %d is null or from another context", i);
    if (!x_io[i]) return fail(TVS_EINVAL, "x_inout[%d] is null", i);
    if (P->dims.ndim != 2 || P->desc.op.kind == TVS_OP_PARALLEL_BEAM)
      return fail(TVS_EUNSUPPORTED, "batched solves take 2D identity or blur problems (problem %d)", i);
    if (P->n >= ((size_t)1 << 31)) return fail(TVS_EUNSUPPORTED, "batched problems have fewer than 2^31 pixels");
    TVS_TRY(check_common(P, prm[i].max_iter, prm[i].n_inner, prm[i].dual, prm[i].f_star,
                         prm[i].target_rel_gap, prm[i].objective_every, x_io[i]));
    if (prm[i].max_iter != K || prm[i].n_inner != N || prm[i].dual != dtype)
      return fail(TVS_EINVAL, "max_iter, n_inner and dual must agree across the batch");
    if (!(prm[i].gamma > 0) || !is_fin(prm[i].gamma)) return fail(TVS_EINVAL, "gamma must be > 0");
    if (!(prm[i].p > 0.0 && prm[i].p <= 1.0)) return fail(TVS_EINVAL, "p must lie in (0, 1]");
    if (prm[i].resume) return fail(TVS_EUNSUPPORTED, "batched solves do not resume");
    for (int j = 0; j < i; ++j)
      if (probs[j] == P) return fail(TVS_EINVAL, "problem %d appears twice", i);
  }
  for (int i = 1; i < n; ++i)
    if (probs[i]->desc.op.kind == TVS_OP_GAUSS_BLUR)
      for (int j = 0; j < i; ++j)
        if (probs[j]->desc.op.kind == TVS_OP_GAUSS_BLUR && probs[j]->bw.R != probs[i]->bw.R)
          return fail(TVS_EUNSUPPORTED, "blur problems of a batch must share the blur radius");
  return TVS_OK;
}

tvs_status batch_solve_in_order(tvs_ctx* C, int n, tvs_problem* const* probs, const tvs_fb_params* prm,
                                float* const* x_io, tvs_mem mem, tvs_trace* traces) {
  const int K = prm[0].max_iter, N = prm[0].n_inner;
  int blur_radius = 0;
  for (int i = 0; i < n; ++i)
    if (probs[i]->desc.op.kind == TVS_OP_GAUSS_BLUR) {
      if (blur_radius && probs[i]->bw.R != blur_radius)
        return fail(TVS_EUNSUPPORTED, "blur problems of a batch must share the blur radius");
      blur_radius = probs[i]->bw.R;
    }
  cudaStream_t s = C->stream;
  for (int i = 0; i < n; ++i) TVS_TRY(ensure_trace(probs[i], K));
  // A batch solved again with the same problems (same buffers), parameters and
  // memory kind reuses the work lists, scratch and captured graphs of the last
  // one: only the per-solve state is reset.
  BatchCache* B = C->batch;
  if (!B || !B->matches(n, probs, prm, mem)) {
    drop_batch_cache(C);
    std::unique_ptr<BatchCache> nb(new BatchCache);
    TVS_TRY(build_batch(C, n, probs, prm, mem, blur_radius, nb.get()));
    C->batch = nb.release();
    B = C->batch;
  }
  BatchLaunch& L = B->L;
  BatchScratch& S = B->S;
  // per-solve state: iterates, counters, work lists of the iteration, records
  for (int i = 0; i < n; ++i)
    if (mem == TVS_MEM_HOST) TVS_TRY(copy_in(probs[i]->x[0], x_io[i], probs[i]->n, mem, s));
  CUDA_TRY(cudaMemcpyAsync(L.state, B->st0.data(), sizeof(BatchState) * n, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemsetAsync(L.scan_tiles, 0, sizeof(int) * (n + 1), s));
  CUDA_TRY(cudaMemsetAsync(L.scan_chunks, 0, sizeof(int) * (n + 1), s));
  CUDA_TRY(cudaMemsetAsync(L.kctr, 0, sizeof(int), s));
  CUDA_TRY(cudaMemsetAsync(L.work, 0, sizeof(int) * L.n_work, s));
  const size_t nparts = (size_t)L.n_blur_tiles + L.n_ident_chunks;
  if (nparts) {
    CUDA_TRY(cudaMemsetAsync(L.part_a, 0, sizeof(Partial) * nparts, s));
    CUDA_TRY(cudaMemsetAsync(L.part_b, 0, sizeof(Partial) * nparts, s));
  }
  CUDA_TRY(cudaMemsetAsync(B->t0_dev, 0, sizeof(unsigned long long), s));
  CUDA_TRY(cudaMemsetAsync(B->obj_pack, 0, sizeof(double) * B->rows, s));
  CUDA_TRY(cudaMemsetAsync(B->ts_pack, 0, sizeof(unsigned long long) * B->rows, s));
  memset(S.done_host, 0, sizeof(int) * n);
  if (mem == TVS_MEM_DEVICE) {
    std::vector<float*> xs(x_io, x_io + n);
    CUDA_TRY(cudaMemcpyAsync(B->x_dev_list, xs.data(), sizeof(float*) * n, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));  // xs is a local vector
  }
  CUDA_TRY(launch_batch_init(L, mem == TVS_MEM_DEVICE ? (const float* const*)B->x_dev_list : nullptr, K, s));
  CUDA_TRY(cudaEventRecord(C->ev_start, s));
  CUDA_TRY(launch_timestamp(B->t0_dev, s));
  // iterations in runs of CHUNK per graph launch (one chunk graph: the batch's
  // coins are drawn on the device), CHUNK_DEPTH launches ahead of the device
  int launched = 0;
  for (int j = 0; launched < K; ++j) {
    if (j >= CHUNK_DEPTH) {
      CUDA_TRY(cudaEventSynchronize(C->ring[(j - CHUNK_DEPTH) % LAG]));
      int ndone = 0;
      for (int i = 0; i < n; ++i) ndone += ((volatile int*)S.done_host)[i];
      if (ndone == n) break;
    }
    if (launched % CHUNK == 0 && K - launched >= CHUNK) {
      if (!B->G.chunk[0]) {
        const tvs_status st = capture(s, &B->G.chunk[0], [&]() -> tvs_status {
          for (int i = 0; i < CHUNK; ++i) CUDA_TRY(launch_batch_iteration(L, i & 1, s));
          return TVS_OK;
        });
        if (st != TVS_OK) {
          B->G.chunk[0] = nullptr;
          return st;
        }
      }
      CUDA_TRY(cudaGraphLaunch(B->G.chunk[0], s));
      launched += CHUNK;
    } else {
      CUDA_TRY(cudaGraphLaunch(B->G.exec[1][launched & 1], s));
      launched += 1;
    }
    CUDA_TRY(cudaEventRecord(C->ring[j % LAG], s));
  }
  CUDA_TRY(launch_batch_final_objective(L, launched & 1, s));
  CUDA_TRY(cudaEventRecord(C->ev_stop, s));
  // records of every problem packed on the device (and device results copied
  // out), then brought back in four copies
  const size_t rows = B->rows;
  CUDA_TRY(launch_batch_trace(L, K, B->obj_pack, B->ts_pack, mem == TVS_MEM_DEVICE ? B->x_dev_list : nullptr, s));
  std::vector<BatchState> st(n);
  std::vector<double> obj_all(rows);
  std::vector<unsigned long long> ts_all(rows);
  std::vector<unsigned char> coins((size_t)K * n);
  unsigned long long t0 = 0;
  CUDA_TRY(cudaMemcpyAsync(st.data(), L.state, sizeof(BatchState) * n, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(obj_all.data(), B->obj_pack, sizeof(double) * rows, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(ts_all.data(), B->ts_pack, sizeof(unsigned long long) * rows, cudaMemcpyDeviceToHost, s));
  if (!coins.empty())
    CUDA_TRY(cudaMemcpyAsync(coins.data(), L.coins, coins.size(), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(&t0, B->t0_dev, sizeof(t0), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  float solve_ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&solve_ms, C->ev_start, C->ev_stop));
  bool bad = false;
  for (int i = 0; i < n; ++i) {
    tvs_problem* P = probs[i];
    const int iters = st[i].iters;
    if (mem == TVS_MEM_HOST) TVS_TRY(copy_out(x_io[i], P->x[iters & 1], P->n, mem, s));
    const double* obj = obj_all.data() + (size_t)i * K;
    const unsigned long long* ts = ts_all.data() + (size_t)i * K;
    if (iters > 0 && !is_fin(obj[iters - 1])) bad = true;
    if (traces) {
      tvs_trace* tr = &traces[i];
      int prox = 0;
      for (int k = 0; k < iters; ++k) prox += coins[(size_t)k * n + i];
      tr->iters_run = iters;
      tr->prox_calls = prox;
      tr->reached = st[i].pad;
      tr->reached_iter = st[i].reached;
      tr->time_to_target_s = -1.0;
      if (st[i].reached >= 0 && st[i].reached < iters) tr->time_to_target_s = (double)(ts[st[i].reached] - t0) * 1e-9;
      tr->solve_ms = solve_ms;
      tr->fgp_ms = 0.0;
      tr->fgp_launches = (long long)prox * ((N + batch_fgp_iters_per_launch() - 1) / batch_fgp_iters_per_launch());
      tr->fgp_pixel_iters = (long long)prox * N * (long long)P->n;
      const int lim = tr->cap < iters ? tr->cap : iters;
      for (int k = 0; k < lim; ++k) {
        if (tr->objective) tr->objective[k] = obj[k];
        if (tr->coins) tr->coins[k] = coins[(size_t)k * n + i];
        if (tr->t_s) tr->t_s[k] = (double)(ts[k] - t0) * 1e-9;
      }
    }
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  if (bad) return fail(TVS_ENUMERIC, "non-finite objective in the batch");
  return TVS_OK;
}

}  // namespace

// ---------------------------------------------------------------- Dual-ROF (light prox)
extern "C" tvs_status dual_rof_solve(tvs_ctx* C, const int dims[2], const float* b,
                                     const tvs_rof_params* prm, float* q_io, float* u_out, tvs_mem mem,
                                     tvs_trace* tr) {
  if (!C || !dims || !b || !prm || !q_io) return fail(TVS_EINVAL, "null argument");
  if (mem != TVS_MEM_DEVICE && mem != TVS_MEM_HOST) return fail(TVS_EINVAL, "invalid mem kind");
  const int W = dims[0], H = dims[1];
  if (W < 1 || H < 1) return fail(TVS_EINVAL, "dims must be >= 1");
  if (!(prm->alpha > 0) || !is_fin(prm->alpha)) return fail(TVS_EINVAL, "alpha must be > 0");
  if (!(prm->eps >= 0) || !is_fin(prm->eps)) return fail(TVS_EINVAL, "eps must be >= 0");
  if (!(prm->gamma > 0) || !is_fin(prm->gamma)) return fail(TVS_EINVAL, "gamma must be > 0");
  if (!(prm->p > 0.0 && prm->p <= 1.0)) return fail(TVS_EINVAL, "p must lie in (0, 1]");
  if (prm->max_iter < 0) return fail(TVS_EINVAL, "max_iter must be >= 0");
  if (!is_fin(prm->f_star) || !(prm->target_rel_gap >= 0)) return fail(TVS_EINVAL, "invalid f_star/target");
  if (prm->accelerated != 0 && prm->accelerated != 1) return fail(TVS_EINVAL, "accelerated must be 0 or 1");
  if (prm->accelerated && prm->p < 1.0) return fail(TVS_EINVAL, "the accelerated solver takes p = 1");
  if (!(prm->target_rel_dist >= 0) || !is_fin(prm->target_rel_dist)) return fail(TVS_EINVAL, "invalid target_rel_dist");
  const int K = prm->max_iter;
  const size_t n = (size_t)H * W;
  const bool skip = prm->p < 1.0;
  const bool accel = prm->accelerated != 0;
  cudaStream_t s = C->stream;
  BatchScratch S;
  float *q0, *q1, *q2 = nullptr, *h = nullptr, *bd, *beta_tab = nullptr, *uref = nullptr;
  Partial *pa, *pb, *pc = nullptr;
  double* dist = nullptr;
  double uref_norm2 = 0.0;
  double* obj;
  unsigned long long* ts;
  int* flags;
  const int nparts = std::max(dual_rof_blocks(H, W), pointwise_blocks(n));
  TVS_TRY(S.zeros<float>(2 * n, &q0, s));
  TVS_TRY(S.zeros<float>(2 * n, &q1, s));
  if (accel) {
    TVS_TRY(S.zeros<float>(2 * n, &q2, s));
    TVS_TRY(S.zeros<float>((size_t)K + 1, &beta_tab, s));
  }
  if (skip) TVS_TRY(S.zeros<float>(2 * n, &h, s));
  TVS_TRY(S.zeros<float>(n, &bd, s));
  TVS_TRY(S.zeros<Partial>(nparts, &pa, s));
  TVS_TRY(S.zeros<Partial>(nparts, &pb, s));
  TVS_TRY(S.zeros<double>((size_t)K + 1, &obj, s));
  TVS_TRY(S.zeros<unsigned long long>((size_t)K + 2, &ts, s));
  TVS_TRY(S.zeros<int>(5, &flags, s));
  int* done_host = nullptr;
  int* done_dev = nullptr;
  {
    cudaError_t e = cudaHostAlloc((void**)&S.done_host, sizeof(int), cudaHostAllocMapped);
    if (e != cudaSuccess) {
      S.done_host = nullptr;
      return fail(TVS_ENOMEM, "cudaHostAlloc: %s", cudaGetErrorString(e));
    }
    done_host = S.done_host;
    *done_host = 0;
    CUDA_TRY(cudaHostGetDevicePointer((void**)&done_dev, done_host, 0));
  }
  TVS_TRY(copy_in(bd, b, n, mem, s));
  TVS_TRY(copy_in(q0, q_io, 2 * n, mem, s));
  if (prm->u_ref) {
    // the reference: a device copy, and its squared norm (FP64, on the host)
    std::vector<float> host(n);
    if (mem == TVS_MEM_HOST)
      memcpy(host.data(), prm->u_ref, n * sizeof(float));
    else
      CUDA_TRY(cudaMemcpy(host.data(), prm->u_ref, n * sizeof(float), cudaMemcpyDeviceToHost));
    for (float v : host) {
      if (!std::isfinite(v)) return fail(TVS_ENUMERIC, "u_ref holds a non-finite value");
      uref_norm2 += (double)v * (double)v;
    }
    if (!(uref_norm2 > 0.0)) return fail(TVS_EINVAL, "u_ref must be nonzero");
    TVS_TRY(S.zeros<float>(n, &uref, s));
    TVS_TRY(S.zeros<Partial>(nparts, &pc, s));
    TVS_TRY(S.zeros<double>((size_t)K + 1, &dist, s));
    CUDA_TRY(cudaMemcpyAsync(uref, host.data(), n * sizeof(float), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemsetAsync(dist, 0xff, sizeof(double) * (K + 1), s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  int f0[4] = {0, -1, -1, 0};
  CUDA_TRY(cudaMemcpyAsync(flags, f0, sizeof(f0), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemsetAsync(obj, 0xff, sizeof(double) * (K + 1), s));
  std::vector<unsigned char> coins(K, 1);
  if (skip)
    for (int k = 0; k < K; ++k) coins[k] = (unsigned char)tvs_coin(prm->seed, prm->p, k);
  const float alpha = (float)prm->alpha, eps = (float)prm->eps, gamma = (float)prm->gamma, p = (float)prm->p;
  const double ea = prm->eps / prm->alpha;
  const int nb = dual_rof_blocks(H, W);
  float* q[3] = {q0, q1, q2};
  std::vector<float> bt;
  if (accel) {
    // beta_tab[k]: the extrapolation coefficient of iteration k, (t_{k-1} - 1) / t_k
    // with t_0 = 1 (0 for k = 0); the step kernel of iteration k finds the record
    // counter at k - 1
    bt.assign((size_t)K + 1, 0.f);
    double t = 1.0;
    for (int k = 1; k <= K; ++k) {
      const double tn = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
      bt[k] = (float)((t - 1.0) / tn);
      t = tn;
    }
    CUDA_TRY(cudaMemcpyAsync(beta_tab, bt.data(), sizeof(float) * bt.size(), cudaMemcpyHostToDevice, s));
  }
  CUDA_TRY(cudaEventRecord(C->ev_start, s));
  CUDA_TRY(launch_timestamp(ts + K + 1, s));
  // plain / ProxSkip iterations: graph [coin][k mod 2]; accelerated: [k mod 3]
  GraphSet G, G3;
  if (accel) {
    for (int r = 0; r < 3; ++r) {
      cudaGraphExec_t* slot = r < 2 ? &G.exec[1][r] : &G3.exec[1][0];
      TVS_TRY(capture(s, slot, [&]() -> tvs_status {
        CUDA_TRY(launch_dual_rof_accel_step(H, W, q[r], q[(r + 2) % 3], q[(r + 1) % 3], bd, alpha, eps, gamma,
                                            beta_tab, flags + 2, pa, pb, uref, pc, s));
        CUDA_TRY(launch_reduce_record(pa, nb, pb, nb, ea, 1, obj, ts, prm->f_star, prm->target_rel_gap, flags,
                                      done_dev, nullptr, s));
        if (uref)
          CUDA_TRY(launch_dist_record(pc, nb, uref_norm2, dist, prm->target_rel_dist, flags, done_dev, s));
        return TVS_OK;
      }));
    }
  } else {
    for (int c = 0; c < 2; ++c) {
      if (c == 0 && !skip) continue;
      for (int par = 0; par < 2; ++par) {
        TVS_TRY(capture(s, &G.exec[c][par], [&]() -> tvs_status {
          CUDA_TRY(launch_dual_rof_step(H, W, q[par], q[par ^ 1], h, bd, alpha, eps, gamma, p, c == 1, pa, pb,
                                        uref, pc, s));
          CUDA_TRY(launch_reduce_record(pa, nb, pb, nb, ea, 1, obj, ts, prm->f_star, prm->target_rel_gap, flags,
                                        done_dev, nullptr, s));
          if (uref)
            CUDA_TRY(launch_dist_record(pc, nb, uref_norm2, dist, prm->target_rel_dist, flags, done_dev, s));
          return TVS_OK;
        }));
      }
    }
  }
  int iters = 0, prox = 0;
  for (int k = 0; k < K; ++k) {
    if (k >= LAG) {
      CUDA_TRY(cudaEventSynchronize(C->ring[k % LAG]));
      if (*(volatile int*)done_host) break;
    }
    const int c = coins[k] ? 1 : 0;
    cudaGraphExec_t ex = G.exec[c][k & 1];
    if (accel) ex = k % 3 < 2 ? G.exec[1][k % 3] : G3.exec[1][0];
    CUDA_TRY(cudaGraphLaunch(ex, s));
    CUDA_TRY(cudaEventRecord(C->ring[k % LAG], s));
    iters = k + 1;
    prox += c;
  }
  float* qf = accel ? q[iters % 3] : q[iters & 1];
  float* u_dev = nullptr;
  if (u_out) TVS_TRY(S.zeros<float>(n, &u_dev, s));
  CUDA_TRY(launch_dual_rof_primal(H, W, qf, bd, u_dev, pa, pb, uref, pc, s));
  if (iters > 0) {
    CUDA_TRY(launch_reduce_record(pa, pointwise_blocks(n), pb, pointwise_blocks(n), ea, 1, obj, ts, prm->f_star,
                                  prm->target_rel_gap, flags, done_dev, nullptr, s));
    if (uref)
      CUDA_TRY(launch_dist_record(pc, pointwise_blocks(n), uref_norm2, dist, prm->target_rel_dist, flags, done_dev,
                                  s));
  }
  TVS_TRY(copy_out(q_io, qf, 2 * n, mem, s));
  if (u_out) TVS_TRY(copy_out(u_out, u_dev, n, mem, s));
  CUDA_TRY(cudaEventRecord(C->ev_stop, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  int fl[5];
  CUDA_TRY(cudaMemcpy(fl, flags, sizeof(fl), cudaMemcpyDeviceToHost));
  if (tr) {
    std::vector<double> o(iters > 0 ? iters : 1);
    std::vector<unsigned long long> t(iters + 1);
    if (iters > 0) {
      CUDA_TRY(cudaMemcpy(o.data(), obj, sizeof(double) * iters, cudaMemcpyDeviceToHost));
      CUDA_TRY(cudaMemcpy(t.data(), ts, sizeof(unsigned long long) * iters, cudaMemcpyDeviceToHost));
    }
    CUDA_TRY(cudaMemcpy(&t[iters], ts + K + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, C->ev_start, C->ev_stop));
    tr->iters_run = iters;
    tr->prox_calls = prox;
    tr->reached = fl[0];
    tr->reached_iter = fl[0] ? fl[1] : -1;
    tr->time_to_target_s = (fl[0] && fl[1] >= 0 && fl[1] < iters) ? (double)(t[fl[1]] - t[iters]) * 1e-9 : -1.0;
    tr->solve_ms = ms;
    tr->fgp_ms = 0.0;
    tr->fgp_launches = 0;
    tr->fgp_pixel_iters = 0;
    const int lim = tr->cap < iters ? tr->cap : iters;
    std::vector<double> dv;
    if (dist && iters > 0 && tr->rel_dist) {
      dv.resize(iters);
      CUDA_TRY(cudaMemcpy(dv.data(), dist, sizeof(double) * iters, cudaMemcpyDeviceToHost));
    }
    for (int k = 0; k < lim; ++k) {
      if (tr->objective) tr->objective[k] = o[k];
      if (tr->coins) tr->coins[k] = coins[k];
      if (tr->t_s) tr->t_s[k] = (double)(t[k] - t[iters]) * 1e-9;
      if (tr->rel_dist) tr->rel_dist[k] = dv.empty() ? NAN : dv[k];
    }
  }
  if (fl[4]) return fail(TVS_ENUMERIC, "non-finite objective during the solve");
  return TVS_OK;
}

// =====================================================================================
extern "C" {

const char* tvs_last_error(void) { return g_err.c_str(); }

tvs_status tvs_create(tvs_ctx** out, int device, void* cuda_stream) {
  if (!out) return fail(TVS_EINVAL, "null output pointer");
  *out = nullptr;
  int ndev = 0;
  CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(TVS_EINVAL, "device %d out of range (%d devices)", device, ndev);
  CUDA_TRY(cudaSetDevice(device));
  tvs_ctx* C = new tvs_ctx();
  C->device = device;
  C->fgp = default_fgp_config();
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread) {
    cudaError_t e = cudaStreamCreateWithFlags(&C->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete C;
      return fail(TVS_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
    C->own_stream = true;
  } else {
    C->stream = s;
  }
  cudaError_t e = cudaEventCreate(&C->ev_start);
  if (e == cudaSuccess) e = cudaEventCreate(&C->ev_stop);
  for (int i = 0; i < LAG && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&C->ring[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&C->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&C->fork_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&C->join_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&C->red_out, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&C->flags, 5 * sizeof(int));
  if (e == cudaSuccess) e = fgp_prepare_device();
  if (e != cudaSuccess) {
    tvs_destroy(C);
    return fail(TVS_ECUDA, "context setup: %s", cudaGetErrorString(e));
  }
  *out = C;
  return TVS_OK;
}

tvs_status tvs_destroy(tvs_ctx* C) {
  if (!C) return TVS_OK;
  cudaSetDevice(C->device);
  if (C->stream) cudaStreamSynchronize(C->stream);
  drop_batch_cache(C);
  while (!C->problems.empty()) tvs_problem_destroy(C->problems.back());
  dfree(C->prox_scratch);
  dfree(C->red_out);
  dfree(C->flags);
  dfree(C->parts);
  if (C->ev_start) cudaEventDestroy(C->ev_start);
  if (C->ev_stop) cudaEventDestroy(C->ev_stop);
  for (auto& ev : C->ring)
    if (ev) cudaEventDestroy(ev);
  if (C->fork_ev) cudaEventDestroy(C->fork_ev);
  if (C->join_ev) cudaEventDestroy(C->join_ev);
  if (C->side) cudaStreamDestroy(C->side);
  if (C->own_stream && C->stream) cudaStreamDestroy(C->stream);
  delete C;
  return TVS_OK;
}

size_t tvs_device_bytes(const tvs_ctx* C) { return C ? C->bytes : 0; }

tvs_status tvs_problem_create(tvs_ctx* C, const tvs_problem_desc* desc, const float* b,
                              tvs_mem b_mem, tvs_problem** out) {
  if (!C || !desc || !b || !out) return fail(TVS_EINVAL, "null argument");
  *out = nullptr;
  const tvs_problem_desc& D = *desc;
  if (D.ndim != 2 && D.ndim != 3) return fail(TVS_EINVAL, "ndim must be 2 or 3");
  if (D.nx < 1 || D.ny < 1 || D.nz < 1) return fail(TVS_EINVAL, "dims must be >= 1");
  if (D.ndim == 2 && D.nz != 1) return fail(TVS_EINVAL, "2D problems need nz = 1");
  if (!(D.alpha >= 0) || !is_fin(D.alpha)) return fail(TVS_EINVAL, "alpha must be finite and >= 0");
  if (b_mem != TVS_MEM_DEVICE && b_mem != TVS_MEM_HOST) return fail(TVS_EINVAL, "invalid mem kind");
  const tvs_op_desc& op = D.op;
  if (op.kind != TVS_OP_IDENTITY && op.kind != TVS_OP_GAUSS_BLUR && op.kind != TVS_OP_PARALLEL_BEAM)
    return fail(TVS_EINVAL, "invalid operator kind");
  if (op.kind != TVS_OP_IDENTITY && D.ndim != 2) return fail(TVS_EUNSUPPORTED, "3D supports the identity operator only");
  if (op.kind == TVS_OP_GAUSS_BLUR &&
      (op.blur_radius < 1 || op.blur_radius > 8 || !(op.blur_sigma > 0) || !is_fin(op.blur_sigma)))
    return fail(TVS_EINVAL, "blur needs 1 <= radius <= 8 and sigma > 0");
  if (op.kind == TVS_OP_PARALLEL_BEAM &&
      (D.nx != D.ny || op.n_angles < 1 || op.n_det < 1 || !(op.pixel_size > 0) || !(op.det_spacing > 0)))
    return fail(TVS_EINVAL, "parallel beam needs a square image, n_angles, n_det >= 1 and positive spacings");
  size_t n = 0;
  if (!pixels_within(D.nx, D.ny, D.nz, kMaxPixels, &n)) return fail(TVS_EINVAL, "image too large");
  CUDA_TRY(cudaSetDevice(C->device));
  tvs_problem* P = new tvs_problem();
  P->ctx = C;
  P->desc = D;
  P->dims.nx = D.nx;
  P->dims.ny = D.ny;
  P->dims.nz = D.nz;
  P->dims.ndim = D.ndim;
  P->n = n;
  P->m = op.kind == TVS_OP_PARALLEL_BEAM ? (size_t)op.n_angles * op.n_det : n;
  auto bail = [&](tvs_status st) {
    tvs_problem_destroy(P);
    return st;
  };
  if (op.kind == TVS_OP_GAUSS_BLUR) {
    const int R = op.blur_radius;
    double w[17], sum = 0.0;
    for (int i = -R; i <= R; ++i) sum += (w[i + R] = std::exp(-(double)(i * i) / (2.0 * op.blur_sigma * op.blur_sigma)));
    P->bw.R = R;
    for (int i = 0; i < 17; ++i) P->bw.w[i] = i <= 2 * R ? (float)(w[i] / sum) : 0.f;
  }
  tvs_status st;
  const size_t n_img = n, m = P->m;
  if ((st = palloc(P, &P->b, m)) || (st = palloc(P, &P->x[0], n_img)) || (st = palloc(P, &P->x[1], n_img)) ||
      (st = palloc(P, &P->z, n_img)) || (st = palloc(P, &P->h, n_img)) || (st = palloc(P, &P->r, m)) ||
      (st = palloc(P, &P->y, m)) || (st = palloc(P, &P->axp, m)))
    return bail(st);
  for (int i = 0; i < 4; ++i)
    if ((st = dalloc(C, &P->bytes, &P->dual[i], 4 * (size_t)D.ndim * n_img))) return bail(st);
  if (op.kind == TVS_OP_PARALLEL_BEAM) {
    if ((st = palloc(P, &P->angle_tab, (size_t)op.n_angles)) || (st = palloc(P, &P->angle_tab2, (size_t)op.n_angles)) ||
        (st = palloc(P, &P->xt, n_img)))
      return bail(st);
    P->geom.N = D.nx;
    P->geom.n_angles = op.n_angles;
    P->geom.n_det = op.n_det;
    P->geom.pixel_size = (float)op.pixel_size;
    P->geom.det_spacing = (float)op.det_spacing;
    P->geom.angles = P->angle_tab;
    P->geom.angles2 = P->angle_tab2;
    P->geom.xt_scratch = P->xt;
    cudaError_t e = ct_build_angle_table(P->geom, P->angle_tab, C->stream);
    if (e != cudaSuccess) return bail(fail(TVS_ECUDA, "angle table: %s", cudaGetErrorString(e)));
  }
  int parts = tile_blocks_2d(D.ny * D.nz, D.nx);
  parts = std::max(parts, pointwise_blocks(n_img));
  parts = std::max(parts, pointwise_blocks(m));
  if (op.kind == TVS_OP_PARALLEL_BEAM) {
    parts = std::max(parts, ct_fwd_blocks(P->geom));
    parts = std::max(parts, ct_bwd_blocks(P->geom));
  }
  P->max_parts = parts;
  if ((st = palloc(P, &P->part_a, (size_t)parts)) || (st = palloc(P, &P->part_b, (size_t)parts)) ||
      (st = palloc(P, &P->flags, 5)) || (st = palloc(P, &P->count, 1)))
    return bail(st);
  {
    cudaError_t e = cudaHostAlloc((void**)&P->done_host, sizeof(int), cudaHostAllocMapped);
    if (e != cudaSuccess) {
      P->done_host = nullptr;
      return bail(fail(TVS_ENOMEM, "cudaHostAlloc: %s", cudaGetErrorString(e)));
    }
    *P->done_host = 0;
    e = cudaHostGetDevicePointer((void**)&P->done_host_dev, P->done_host, 0);
    if (e != cudaSuccess) return bail(fail(TVS_ECUDA, "cudaHostGetDevicePointer: %s", cudaGetErrorString(e)));
  }
  if ((st = tvs_problem_set_data(P, b, b_mem))) return bail(st);
  C->problems.push_back(P);
  *out = P;
  return TVS_OK;
}

tvs_status tvs_problem_set_reference(tvs_problem* P, const float* u_ref, tvs_mem mem) {
  if (!P) return fail(TVS_EINVAL, "null problem");
  if (mem != TVS_MEM_DEVICE && mem != TVS_MEM_HOST) return fail(TVS_EINVAL, "invalid mem kind");
  cudaStream_t s = P->ctx->stream;
  if (!u_ref) {
    dfree(P->uref);
    dfree(P->part_c);
    P->uref = nullptr;
    P->part_c = nullptr;
    ++P->gen;
    return TVS_OK;
  }
  std::vector<float> host(P->n);
  if (mem == TVS_MEM_HOST) {
    memcpy(host.data(), u_ref, P->n * sizeof(float));
  } else {
    CUDA_TRY(cudaMemcpy(host.data(), u_ref, P->n * sizeof(float), cudaMemcpyDeviceToHost));
  }
  double nrm = 0.0;
  for (float v : host) {
    if (!std::isfinite(v)) return fail(TVS_ENUMERIC, "reference holds a non-finite value");
    nrm += (double)v * (double)v;
  }
  if (!(nrm > 0.0)) return fail(TVS_EINVAL, "reference must be nonzero");
  if (!P->uref) {
    ++P->gen;
    TVS_TRY(palloc(P, &P->uref, P->n));
    TVS_TRY(palloc(P, &P->part_c, (size_t)pointwise_blocks(P->n)));
  }
  CUDA_TRY(cudaMemcpyAsync(P->uref, host.data(), P->n * sizeof(float), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  P->uref_norm2 = nrm;
  return TVS_OK;
}

tvs_status tvs_problem_set_data(tvs_problem* P, const float* b, tvs_mem b_mem) {
  if (!P || !b) return fail(TVS_EINVAL, "null argument");
  if (b_mem != TVS_MEM_DEVICE && b_mem != TVS_MEM_HOST) return fail(TVS_EINVAL, "invalid mem kind");
  cudaStream_t s = P->ctx->stream;
  TVS_TRY(copy_in(P->b, b, P->m, b_mem, s));
  CUDA_TRY(cudaMemsetAsync(P->count, 0, sizeof(int), s));
  CUDA_TRY(launch_count_nonfinite(P->b, P->m, P->count, s));
  int cnt = 0;
  CUDA_TRY(cudaMemcpyAsync(&cnt, P->count, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (cnt) return fail(TVS_ENUMERIC, "b holds %d non-finite values", cnt);
  return TVS_OK;
}

tvs_status tvs_problem_destroy(tvs_problem* P) {
  if (!P) return TVS_OK;
  tvs_ctx* C = P->ctx;
  cudaSetDevice(C->device);
  cudaStreamSynchronize(C->stream);
  if (C->batch && C->batch->uses(P)) drop_batch_cache(C);
  void* bufs[] = {P->b, P->x[0], P->x[1], P->z, P->h, P->r, P->y, P->axp, P->dual[0], P->dual[1],
                  P->dual[2], P->dual[3], P->part_a, P->part_b, P->obj_dev, P->ts_dev, P->fgp_ts, P->beta_dev,
                  P->flags, P->count, P->angle_tab, P->angle_tab2, P->xt, P->uref, P->part_c, P->dist_dev,
                  P->aux};
  for (void* b : bufs) dfree(b);
  if (P->done_host) cudaFreeHost(P->done_host);
  C->bytes -= P->bytes;
  auto& v = C->problems;
  v.erase(std::remove(v.begin(), v.end(), P), v.end());
  delete P;
  return TVS_OK;
}

tvs_status tvs_op_apply(tvs_problem* P, const float* x, float* y, int adjoint) {
  if (!P || !x || !y) return fail(TVS_EINVAL, "null argument");
  cudaStream_t s = P->ctx->stream;
  const Dims& d = P->dims;
  switch (P->desc.op.kind) {
    case TVS_OP_GAUSS_BLUR:
      CUDA_TRY(launch_blur(d.ny, d.nx, x, y, P->bw, s));
      break;
    case TVS_OP_PARALLEL_BEAM:
      if (adjoint) CUDA_TRY(launch_ct_backward(P->geom, x, nullptr, nullptr, y, 0.f, 0.f, nullptr, s));
      else CUDA_TRY(launch_ct_forward(P->geom, x, y, nullptr, nullptr, 0.f, nullptr, CT_FWD_PLAIN, s));
      break;
    default:
      CUDA_TRY(cudaMemcpyAsync(y, x, P->n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  return TVS_OK;
}

tvs_status tvs_objective(tvs_problem* P, const float* x, double* out) {
  if (!P || !x || !out) return fail(TVS_EINVAL, "null argument");
  cudaStream_t s = P->ctx->stream;
  int na = 0, nb = 0;
  TVS_TRY(objective_parts(P, x, P->part_a, P->part_b, &na, &nb, s));
  CUDA_TRY(launch_reduce_record(P->part_a, na, P->part_b, nb, P->desc.alpha, 1, nullptr, nullptr, 0.0,
                                0.0, nullptr, nullptr, P->ctx->red_out, s));
  CUDA_TRY(cudaMemcpyAsync(out, P->ctx->red_out, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return TVS_OK;
}

tvs_status tv_prox(tvs_ctx* C, int ndim, const int dims[3], const float* z, float* u, double lambda,
                   int n_iter, tvs_dual_dtype dual, void* dual_state, int nonneg) {
  if (!C || !dims || !z || !u) return fail(TVS_EINVAL, "null argument");
  if (ndim != 2 && ndim != 3) return fail(TVS_EINVAL, "ndim must be 2 or 3");
  if (dims[0] < 1 || dims[1] < 1 || (ndim == 3 && dims[2] < 1)) return fail(TVS_EINVAL, "dims must be >= 1");
  if (!(lambda >= 0) || !is_fin(lambda)) return fail(TVS_EINVAL, "lambda must be finite and >= 0");
  if (n_iter < 0) return fail(TVS_EINVAL, "n_iter must be >= 0");
  if (!valid_dual(dual)) return fail(TVS_EINVAL, "invalid dual dtype");
  if (z == u) return fail(TVS_EINVAL, "z and u may not alias");
  Dims d;
  d.nx = dims[0];
  d.ny = dims[1];
  d.nz = ndim == 3 ? dims[2] : 1;
  d.ndim = ndim;
  size_t n = 0;
  if (!pixels_within(d.nx, d.ny, d.nz, kMaxPixels, &n)) return fail(TVS_EINVAL, "image too large");
  const size_t plane_bytes = dual_elem_bytes(dual) * ndim * n;
  const size_t need = plane_bytes * (dual_state ? 3 : 4);
  cudaStream_t s = C->stream;
  if (need > C->prox_scratch_bytes) {
    dfree(C->prox_scratch);
    C->bytes -= C->prox_scratch_bytes;
    C->prox_scratch = nullptr;
    C->prox_scratch_bytes = 0;
    TVS_TRY(dalloc(C, nullptr, &C->prox_scratch, need));
    C->prox_scratch_bytes = need;
  }
  char* sc = (char*)C->prox_scratch;
  void* buf[4];
  if (dual_state) {
    buf[0] = dual_state;
    for (int i = 1; i < 4; ++i) buf[i] = sc + (i - 1) * plane_bytes;
  } else {
    for (int i = 0; i < 4; ++i) buf[i] = sc + i * plane_bytes;
    CUDA_TRY(cudaMemsetAsync(buf[0], 0, plane_bytes, s));
  }
  const bool use = lambda > 0.0;
  int fin = 0;
  FgpConfig fcfg;
  if (use && n_iter > 0) TVS_TRY(fgp_config_for(C, d, dual, z, buf[0], buf[2], buf[3], &fcfg));
  if (use) TVS_TRY(launch_fgp_sequence(fcfg, d, z, buf, n_iter, fgp_betas(n_iter), (float)lambda,
                                       dual, nonneg != 0, s, &fin));
  CUDA_TRY(launch_fgp_finalize(d, z, buf[fin], dual, use ? (float)lambda : 0.f, nonneg != 0, u,
                               nullptr, 0.f, (fin != 0 && dual_state) ? dual_state : nullptr,
                               nullptr, nullptr, nullptr, nullptr, InnerStamp{}, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (ndim == 3 && use && n_iter > 0 && fgp3d_take_wait_timeouts())
    return fail(TVS_ETIMEDOUT, "a 3D inner kernel gave up waiting for a TMA tile load; the result is incomplete");
  return TVS_OK;
}

tvs_status tv_prox_gap(tvs_ctx* C, int ndim, const int dims[3], const float* z, double lambda,
                       tvs_dual_dtype dual, const void* dual_state, double* gap) {
  if (!C || !dims || !z || !dual_state || !gap) return fail(TVS_EINVAL, "null argument");
  if (ndim != 2 && ndim != 3) return fail(TVS_EINVAL, "ndim must be 2 or 3");
  if (dims[0] < 1 || dims[1] < 1 || (ndim == 3 && dims[2] < 1)) return fail(TVS_EINVAL, "dims must be >= 1");
  if (!(lambda >= 0) || !is_fin(lambda)) return fail(TVS_EINVAL, "lambda must be finite and >= 0");
  if (!valid_dual(dual)) return fail(TVS_EINVAL, "invalid dual dtype");
  Dims d;
  d.nx = dims[0];
  d.ny = dims[1];
  d.nz = ndim == 3 ? dims[2] : 1;
  d.ndim = ndim;
  size_t n = 0;
  if (!pixels_within(d.nx, d.ny, d.nz, kMaxPixels, &n)) return fail(TVS_EINVAL, "image too large");
  cudaStream_t s = C->stream;
  const size_t nb = (size_t)rof_gap_blocks(n);
  if (nb > C->parts_cap) {
    dfree(C->parts);
    C->bytes -= C->parts_cap * sizeof(Partial);
    C->parts = nullptr;
    C->parts_cap = 0;
    TVS_TRY(dalloc(C, nullptr, (void**)&C->parts, nb * sizeof(Partial)));
    C->parts_cap = nb;
  }
  CUDA_TRY(launch_rof_gap_partials(d, z, dual_state, dual, (float)lambda, C->parts, s));
  CUDA_TRY(launch_reduce_record(C->parts, (int)nb, nullptr, 0, 0.0, 1, nullptr, nullptr, 0.0, 0.0, nullptr,
                                nullptr, C->red_out, s));
  double sum = 0.0;
  CUDA_TRY(cudaMemcpyAsync(&sum, C->red_out, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  *gap = lambda * sum;
  return TVS_OK;
}

tvs_status tvs_fgp_config(tvs_ctx* C, int ndim, const int dims[3], tvs_dual_dtype dual, int out[3]) {
  if (!C || !dims || !out) return fail(TVS_EINVAL, "null argument");
  if (ndim != 2 && ndim != 3) return fail(TVS_EINVAL, "ndim must be 2 or 3");
  if (dims[0] < 1 || dims[1] < 1 || (ndim == 3 && dims[2] < 1)) return fail(TVS_EINVAL, "dims must be >= 1");
  if (!valid_dual(dual)) return fail(TVS_EINVAL, "invalid dual dtype");
  Dims d;
  d.nx = dims[0];
  d.ny = dims[1];
  d.nz = ndim == 3 ? dims[2] : 1;
  d.ndim = ndim;
  size_t n = 0;
  if (!pixels_within(d.nx, d.ny, d.nz, kMaxPixels, &n)) return fail(TVS_EINVAL, "image too large");
  FgpConfig c;
  if (ndim == 2) {
    // tune on a scratch image and scratch dual fields of this shape
    const size_t plane_bytes = dual_elem_bytes(dual) * 2 * n;
    const size_t need = plane_bytes * 4 + n * sizeof(float);
    cudaStream_t s = C->stream;
    if (need > C->prox_scratch_bytes) {
      dfree(C->prox_scratch);
      C->bytes -= C->prox_scratch_bytes;
      C->prox_scratch = nullptr;
      C->prox_scratch_bytes = 0;
      TVS_TRY(dalloc(C, nullptr, &C->prox_scratch, need));
      C->prox_scratch_bytes = need;
    }
    char* sc = (char*)C->prox_scratch;
    CUDA_TRY(cudaMemsetAsync(sc, 0, need, s));
    TVS_TRY(fgp_config_for(C, d, dual, (const float*)(sc + 4 * plane_bytes), sc, sc + plane_bytes,
                           sc + 2 * plane_bytes, &c));
  } else {
    c.tb = 1;
  }
  out[0] = c.tb;
  out[1] = c.cpl;
  out[2] = c.rpw;
  return TVS_OK;
}

tvs_status pgd_solve(tvs_problem* P, const tvs_fb_params* prm, float* x, tvs_mem mem, tvs_trace* tr) {
  return fb_solve(P, prm, x, mem, tr, FB_PGD);
}
tvs_status fista_solve(tvs_problem* P, const tvs_fb_params* prm, float* x, tvs_mem mem, tvs_trace* tr) {
  return fb_solve(P, prm, x, mem, tr, FB_FISTA);
}
tvs_status proxskip_solve(tvs_problem* P, const tvs_fb_params* prm, float* x, tvs_mem mem, tvs_trace* tr) {
  return fb_solve(P, prm, x, mem, tr, FB_PROXSKIP);
}
tvs_status pdhg_solve(tvs_problem* P, const tvs_pd_params* prm, float* x, float* y, tvs_mem mem,
                      tvs_trace* tr) {
  return pd_solve(P, prm, x, y, mem, tr, false);
}
tvs_status pdhgskip_solve(tvs_problem* P, const tvs_pd_params* prm, float* x, float* y, tvs_mem mem,
                          tvs_trace* tr) {
  return pd_solve(P, prm, x, y, mem, tr, true);
}

tvs_status pdhg_explicit_solve(tvs_problem* P, const tvs_pdx_params* prm, float* x, float* y, float* q,
                               tvs_mem mem, tvs_trace* tr) {
  return pdx_solve(P, prm, x, y, q, mem, tr);
}
tvs_status pdhgskip1_solve(tvs_problem* P, const tvs_pd_params* prm, float* x, float* y, tvs_mem mem,
                           tvs_trace* tr) {
  return pd1_solve(P, prm, x, y, mem, tr);
}

int tvs_coin(uint64_t seed, double p, int64_t k) {
  if (!(p > 0.0 && p <= 1.0)) return -1;
  return Philox4x64::coin(seed, p, (uint64_t)k);
}

tvs_status tvs_coin_schedule_device(tvs_ctx* C, uint64_t seed, double p, int64_t k0, int K,
                                    unsigned char* out) {
  if (!C || (!out && K > 0) || K < 0) return fail(TVS_EINVAL, "invalid argument");
  if (!(p > 0.0 && p <= 1.0)) return fail(TVS_EINVAL, "p must lie in (0, 1]");
  if (K == 0) return TVS_OK;
  unsigned char* dev = nullptr;
  TVS_TRY(dalloc(C, nullptr, (void**)&dev, (size_t)K));
  cudaStream_t s = C->stream;
  cudaError_t e = launch_coin_schedule(seed, p, k0, K, dev, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dev, (size_t)K, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dev);
  C->bytes -= (size_t)K;
  if (e != cudaSuccess) return fail(TVS_ECUDA, "coin schedule: %s", cudaGetErrorString(e));
  return TVS_OK;
}

}  // extern "C"
