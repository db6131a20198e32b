// Host-side launchers of the device kernels (internal C++ interface).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace tvs {

struct Dims {
  int nx = 1, ny = 1, nz = 1, ndim = 2;
  size_t n() const { return (size_t)nx * ny * nz; }
};

// Largest pixel count any entry point accepts.
constexpr size_t kMaxPixels = (size_t)1 << 34;

// nx * ny * nz without wrap-around: false when the product of the (positive)
// sides exceeds cap, true with *n set otherwise.
inline bool pixels_within(int nx, int ny, int nz, size_t cap, size_t* n) {
  if (nx < 1 || ny < 1 || nz < 1) return false;
  const size_t a = (size_t)nx * (size_t)ny;  // < 2^62
  if (a > cap || (size_t)nz > cap / a) return false;
  *n = a * (size_t)nz;
  return true;
}

enum DualType { DUAL_F32 = 0, DUAL_BF16 = 1, DUAL_F16 = 2, DUAL_Q15 = 3 };

// floor(n / d) for 0 <= n < 2^31 by one multiply and shift (division by an
// invariant integer, Granlund and Montgomery, PLDI 1994, Theorem 4.2 with N = 31):
// L = 31 + ceil(log2 d) and m = ceil(2^L / d), which is below 2^32.
struct FastDiv {
  uint32_t m = 1u << 31, L = 31;
  FastDiv() = default;
  explicit FastDiv(uint32_t d) {
    uint32_t s = 0;
    while ((1ull << s) < d) ++s;
    L = 31 + s;
    m = (uint32_t)(((1ull << L) + d - 1) / d);
  }
#ifdef __CUDACC__
  __device__ __forceinline__ uint32_t div(uint32_t n) const { return (uint32_t)(((uint64_t)n * m) >> L); }
#endif
};

// Row-major coordinates (k, i, j) of a linear index over a D x H x W grid, by
// FastDiv when the grid has fewer than 2^31 cells, else by 64-bit division.
struct IndexMap {
  FastDiv fW, fH;
  int W = 1, H = 1, small = 1;
  IndexMap() = default;
  IndexMap(int D, int H_, int W_)
      : fW((uint32_t)W_), fH((uint32_t)H_), W(W_), H(H_), small((size_t)D * H_ * W_ < ((size_t)1 << 31)) {}
#ifdef __CUDACC__
  __device__ __forceinline__ void coords(size_t o, int& k, int& i, int& j) const {
    if (small) {
      const uint32_t u = (uint32_t)o, r = fW.div(u), kk = fH.div(r);
      j = (int)(u - r * (uint32_t)W);
      i = (int)(r - kk * (uint32_t)H);
      k = (int)kk;
    } else {
      const size_t r = o / (size_t)W;
      j = (int)(o - r * W);
      k = (int)(r / (size_t)H);
      i = (int)(r - (size_t)k * H);
    }
  }
#endif
};

// One block's partial sum of an objective term: a compensated FP32 pair whose
// value is s + c (see FAcc in common.cuh).
struct Partial {
  float s, c;
};
// Timing of the inner iterations of a solve's prox calls: a pair of device times
// per call, arr[2c] at the start of the inner iterations and arr[2c + 1] at their
// end, c = *ctr, which the end stamp advances.  arr == null: no stamp.
struct InnerStamp {
  unsigned long long* arr;
  int* ctr;
};

inline size_t dual_elem_bytes(int t) { return t == DUAL_F32 ? 4 : 2; }

// ---- TV prox (fgp.cu, fgp_tb.cu, fgp3d.cu) ----
// One inner iteration: r = pc + beta (pc - pp); u = P_X(z + lam div r);
// pn = P_B(r + inv_step * D u).  pp may equal pc when beta == 0.
cudaError_t launch_fgp_iter(const Dims& d, const float* z, const void* pc, const void* pp, void* pn,
                            float lam, float inv_step, float beta, int dtype, bool nonneg,
                            cudaStream_t s);
// One 3D iteration (fgp3d.cu); launch_fgp_iter forwards 3D volumes here.
cudaError_t launch_fgp3d_iter(const Dims& d, const float* z, const void* pc, const void* pp, void* pn,
                              float lam, float inv_step, float beta, int dtype, bool nonneg, cudaStream_t s);
// True (and the count cleared) when a bounded wait of a TMA-staged 3D kernel
// gave up since the last call; call only after the stream has been synchronised.
bool fgp3d_take_wait_timeouts();
// PDHGSkip-1 finalisation: u = P_X(z + lam div p); xh = (u - x)/prob_p; x += prob_p xh.
cudaError_t launch_fgp_finalize_pd1(const Dims& d, const float* z, const void* p, int dtype, float lam,
                                    bool nonneg, float prob_p, float* x, float* xh, void* p_home,
                                    InnerStamp st, cudaStream_t s);
// Temporally blocked inner iterations (2D): tile-shape / depth configuration.
// tb <= 1 selects the one-iteration kernel.  A launch of the blocked kernel runs
// `iters` <= tb iterations from (pc = p_k, pp = p_{k-1}) and writes
// pn = p_{k+iters}, pnp = p_{k+iters-1}; betas[i] is the momentum coefficient of
// its i-th iteration.  pn/pnp may not alias pc/pp.
// rpw >= 100 selects the register-blocked variant with rpw - 100 rows per warp.
struct FgpConfig {
  int tb = 1, cpl = 2, rpw = 5;
};
bool fgp_config_valid(const FgpConfig& c);
// Raises the dynamic shared-memory limit of every blocked-kernel variant on the
// current device (called once per context, outside any stream capture).
cudaError_t fgp_prepare_device();
cudaError_t launch_fgp_block(const FgpConfig& c, const Dims& d, const float* z, const void* pc,
                             const void* pp, void* pn, void* pnp, float lam, float inv_step,
                             const float* betas, int iters, int dtype, bool nonneg, cudaStream_t s);
// ROF duality-gap partials of a unit-ball dual p (rof_gap_blocks(n) of them):
// lam * their sum = P(u) - D(p) at u = z + lam div p.
int rof_gap_blocks(size_t n);
cudaError_t launch_rof_gap_partials(const Dims& d, const float* z, const void* p, int dtype, float lam,
                                    Partial* part, cudaStream_t s);
// x_out = P_X(z + lam div p); if h_out: h_out = h_coef (x_out - z);
// if p_home: p_home = p.  When fista_y is set: fista_y = x_out + beta (x_out - x_prev) with
// beta = beta_tab[*beta_idx] (FISTA extrapolation, read on the device).
// st: the end stamp of the inner iterations before it (InnerStamp).
cudaError_t launch_fgp_finalize(const Dims& d, const float* z, const void* p, int dtype, float lam,
                                bool nonneg, float* x_out, float* h_out, float h_coef,
                                void* p_home, const float* x_prev, float* fista_y,
                                const float* beta_tab, const int* beta_idx, InnerStamp st, cudaStream_t s);

// ---- objective pieces and pointwise steps (ops.cu) ----
struct BlurW {
  float w[17];
  int R;
};
int tile_blocks_2d(int H, int W);        // blocks of the 2D tile kernels
int fb_step_blocks_2d(int H, int W, int R);  // blocks of launch_blur_fb_step (blur radius R)
int fb_step_tile_w(int R);                   // its tile: fb_step_tile_w(R) x fb_step_tile_h(R)
int fb_step_tile_h(int R);
// Fused forward-backward step: out = x - gamma A (A x - b) + ch h (h may be null),
// partials of 1/2 ||A x - b||^2 and TV(x) (fb_step_blocks_2d of each).
cudaError_t launch_blur_fb_step(int H, int W, const float* x, const float* b, const float* h, float* out,
                                const BlurW& w, float gamma, float ch, Partial* part_data, Partial* part_tv,
                                cudaStream_t s);
int pointwise_blocks(size_t n);          // blocks of the grid-stride kernels

// r_out = A x - b (r_out may be null); partials of 1/2 r^2 and of TV(x).
cudaError_t launch_blur_residual(int H, int W, const float* x, const float* b, float* r_out,
                                 const BlurW& w, Partial* part_data, Partial* part_tv, cudaStream_t s);
// out = x - gamma A(in) + ch h   (h may be null); optional TV(x) partials.
cudaError_t launch_blur_step(int H, int W, const float* in, const float* x, const float* h,
                             float* out, const BlurW& w, float gamma, float ch, Partial* part_tv,
                             cudaStream_t s);
// y_out = (y + tau (2 A x - ax_prev) - tau b) / (1 + tau); ax_prev <- A x; partial 1/2 (A x - b)^2.
cudaError_t launch_blur_pd_dual(int H, int W, const float* x, float* ax_prev, float* y,
                                const float* b, const BlurW& w, float tau, Partial* part_data,
                                cudaStream_t s);
cudaError_t launch_blur(int H, int W, const float* x, float* y, const BlurW& w, cudaStream_t s);
// PDHGSkip-1 dual step: v = A x^; A x_new = ax_prev + p v (stored back);
// y = (y + tau (A x_new + v) - tau b)/(1+tau); partial 1/2 (A x_new - b)^2.
cudaError_t launch_blur_pd1_dual(int H, int W, const float* xh, float* ax_prev, float* y, const float* b,
                                 const BlurW& w, float p, float tau, Partial* part_data, cudaStream_t s);
// Identity-operator form of the same (axh = x^), or with axh == null the skipped
// iteration y = (y + tau ax_prev - tau b)/(1+tau) (part_data unused then).
cudaError_t launch_pd1_dual_pointwise(size_t m, const float* axh, float* ax_prev, float* y, const float* b,
                                      float p, float tau, Partial* part_data, cudaStream_t s);

// Identity data term (2D or 3D): out = x - gamma (x - b) + ch h; partials of
// 1/2 (x - b)^2 and TV(x).  out may be null (objective only).
cudaError_t launch_identity_step(const Dims& d, const float* x, const float* b, const float* h,
                                 float* out, float gamma, float ch, Partial* part_data,
                                 Partial* part_tv, cudaStream_t s);
// Generic pointwise step used by PDHG with identity/CT adjoint already formed:
// out = x - sigma g + ch h; optional TV(x) partials.
cudaError_t launch_axpy_step(const Dims& d, const float* g, const float* x, const float* h,
                             float* out, float sigma, float ch, Partial* part_tv, cudaStream_t s);
// y = (y + tau (2 ax - ax_prev) - tau b)/(1+tau); ax_prev <- ax; partial 1/2 (ax - b)^2.
cudaError_t launch_pd_dual_pointwise(size_t m, const float* ax, float* ax_prev, float* y,
                                     const float* b, float tau, Partial* part_data, cudaStream_t s);
// Partials of TV(x) only (grid-stride, pointwise_blocks(n) blocks).
cudaError_t launch_tv_partials(const Dims& d, const float* x, Partial* part_tv, cudaStream_t s);

// Sum partials (fixed order), F = data + alpha tv.  k = flags[2] (then flags[2]++);
// when k >= 0 and k % every == 0: obj[k] = F, ts[k] = now, and once
// (F - f*) <= target f*: flags[0] = 1 (done), flags[1] = k, *done_host = 1.
// obj == null: write F to *f_out only.
cudaError_t launch_reduce_record(const Partial* part_data, int n_data, const Partial* part_tv,
                                 int n_tv, double alpha, int every, double* obj,
                                 unsigned long long* ts, double f_star, double target, int* flags,
                                 int* done_host, double* f_out, cudaStream_t s);
// Distance to a reference: partials of (x - u_ref)^2 (pointwise_blocks(n) blocks),
// then one block records dist[k] = sqrt(sum / ref_norm2) at k = flags[2] - 1 (the
// index the preceding reduce_record used) and, when target > 0 and dist <= target,
// raises the same done flags.
cudaError_t launch_dist_partials(size_t n, const float* x, const float* u_ref, Partial* part, cudaStream_t s);
cudaError_t launch_dist_record(const Partial* part, int n_part, double ref_norm2, double* dist, double target,
                               int* flags, int* done_host, cudaStream_t s);
cudaError_t launch_timestamp(unsigned long long* ts, cudaStream_t s);
// The start stamp of an InnerStamp as a launch of its own (st.arr[2 * *st.ctr] = now).
cudaError_t launch_inner_start_stamp(const InnerStamp& st, cudaStream_t s);
cudaError_t launch_count_nonfinite(const float* x, size_t n, int* count, cudaStream_t s);
cudaError_t launch_coin_schedule(uint64_t seed, double p, int64_t k0, int K, unsigned char* out,
                                 cudaStream_t s);

// ---- Dual-ROF / Dual-Huber-ROF (rof.cu) ----
// Explicit, diagonally preconditioned PDHG (pdx.cu).
int pdx_tv_blocks(int H, int W);
cudaError_t launch_pdx_precond(const float* colA, const float* rowA, int H, int W, size_t m, float sigma,
                               float tau, float* T, float* S, cudaStream_t s);
cudaError_t launch_fill(float* a, size_t n, float v, cudaStream_t s);
cudaError_t launch_pdx_tv_step(int H, int W, const float* x, const float* g, const float* T, const float* q,
                               float* xn, float* qn, float alpha, float s_d, bool nonneg, Partial* part_tv,
                               cudaStream_t s);
cudaError_t launch_pdx_dual(size_t m, const float* ax, float* axp, float* y, const float* b, const float* S,
                            bool init, Partial* part_a, cudaStream_t s);

int dual_rof_blocks(int H, int W);
// One ProxSkip / projected-gradient step on q (2 planes) -> qn; h updated in place
// on prox iterations (h == null: projected gradient).  Partials: 1/2 (div q + b)^2
// and 1/2 |q|^2 of the current q; with uref, partials of |b + div q - uref|^2 into
// part_c as well.
cudaError_t launch_dual_rof_step(int H, int W, const float* q, float* qn, float* h, const float* b,
                                 float alpha, float eps, float gamma, float p, bool prox,
                                 Partial* part_a, Partial* part_b, const float* uref, Partial* part_c,
                                 cudaStream_t s);
// AProjGD step: y = q + beta (q - q_prev) with beta = beta_tab[*beta_idx + 1];
// qn = P_C(y - gamma grad F(y)); partials of F(q) (the current iterate), and of
// the distance to uref as above.
cudaError_t launch_dual_rof_accel_step(int H, int W, const float* q, const float* q_prev, float* qn,
                                       const float* b, float alpha, float eps, float gamma,
                                       const float* beta_tab, const int* beta_idx, Partial* part_a,
                                       Partial* part_b, const float* uref, Partial* part_c, cudaStream_t s);
// u = b + div q (u may be null) and the same partials (pointwise_blocks(H W) blocks).
cudaError_t launch_dual_rof_primal(int H, int W, const float* q, const float* b, float* u, Partial* part_a,
                                   Partial* part_b, const float* uref, Partial* part_c, cudaStream_t s);

// ---- batched ProxSkip (batch.cu) ----
// Descriptor of one problem of a batch (device memory).  Partials of its
// objective occupy part_a/part_b[part_off, part_off + part_n).
struct BatchProb {
  int H, W, nonneg, pad;
  FastDiv fw;  // division by W (every batched problem has fewer than 2^31 pixels)
  const float* b;
  float *x0, *x1, *z, *h, *r;
  void *dual0, *dual1, *dual2, *dual3;
  float lam, inv_step, gamma, ch_skip, ch_prox, h_coef;
  double alpha, f_star, target;
  BlurW bw;
  int part_off, part_n;
  double* obj;
  unsigned long long* ts;
};
struct BatchState {
  int done, reached, iters, pad;  // reached: trace index of the first iterate on target; pad: hit
};
struct BatchLaunch {
  const BatchProb* probs;
  BatchState* state;
  int n;
  const int4* blur_tiles;   // (problem, tile x, tile y) of the blur problems (fused-step tiles)
  int n_blur_tiles;
  const int2* ident_chunks; // (problem, chunk) of the identity problems
  int n_ident_chunks;
  int n_fgp_tiles;          // blocked inner tiles of all problems
  int n_all_chunks;         // pixel chunks of all problems
  const unsigned char* coins;  // [K][n]
  int* kctr;                   // outer iteration counter (device; advanced by the compaction kernel)
  Partial *part_a, *part_b;
  int* done_host;              // n flags in mapped host memory
  int n_inner, dtype;
  int blur_radius;             // shared by every blur problem of the batch
  bool use_prox;
  const float* betas;          // host: momentum coefficient of each inner iteration
  // per-problem ranges of fgp_tiles / all_chunks (each problem's entries are contiguous)
  const int2* tile_range;      // (first, count)
  const int2* chunk_range;     // (first, count)
  int* scan_tiles;             // [n + 1]: exclusive scan of the tiles of this iteration's active problems
  int* scan_chunks;            // [n + 1]: the same for their chunks
  int fgp_grid, fin_grid;      // persistent grid sizes of the inner and finalisation kernels
  int nonneg_mode;             // 0: no problem constrained, 1: all, 2: mixed
  int* work;                   // [n_work]: tile counter of each inner launch of an iteration
  int n_work;
};
int batch_fgp_tile_w();
int batch_fgp_tile_h();
int batch_chunk();
int batch_fgp_iters_per_launch();
int batch_fgp_resident_ctas();  // SMs x resident CTAs of the batched inner kernel (0 on error)
// One outer iteration of every problem (graph-capturable; reads k from kctr).
cudaError_t launch_batch_iteration(const BatchLaunch& L, int par, cudaStream_t s);
// F(x_k) of the problems still running, recorded as their final trace entry.
cudaError_t launch_batch_final_objective(const BatchLaunch& L, int par, cudaStream_t s);
// Per-solve set-up of every problem (x_0 from x_src[i] when x_src is not null,
// first dual pair and h zeroed, objective record set to NaN).
cudaError_t launch_batch_init(const BatchLaunch& L, const float* const* x_src, int K, cudaStream_t s);
// coins[k * n + i] = theta_k of problem i for k < K.
cudaError_t launch_batch_coins(const unsigned long long* seeds, const double* ps, int n, int K,
                               unsigned char* coins, cudaStream_t s);
// Objective / timestamp records packed as [n][K] rows; results copied to x_dst[i]
// when x_dst is not null.
cudaError_t launch_batch_trace(const BatchLaunch& L, int K, double* obj_out, unsigned long long* ts_out,
                               float* const* x_dst, cudaStream_t s);

// ---- parallel-beam projector (ct.cu) ----
struct CTGeom {
  int N, n_angles, n_det;
  float pixel_size, det_spacing;
  const float4* angles;  // device table: (m1, inv, weight, row_walk) per angle
  float4* angles2;       // device table: (1 / slope of fr in b, 1 / |slope| + margin, candidates, -)
  float* xt_scratch;     // N*N floats: transposed image used by the projector
};
cudaError_t ct_build_angle_table(const CTGeom& g, float4* dev_table, cudaStream_t s);
int ct_fwd_blocks(const CTGeom& g);
int ct_bwd_blocks(const CTGeom& g);
enum CTFwdMode { CT_FWD_PLAIN = 0, CT_FWD_PD = 1, CT_FWD_STORE = 2, CT_FWD_RESID = 3, CT_FWD_PD1 = 4 };
// PLAIN: sino = A x.  PD: y = (y + tau (2 Ax - sino) - tau b)/(1+tau), then sino = Ax.
// STORE: sino = A x; RESID: sino = A x - b.  PD1 (x = x^ of PDHGSkip-1): sino <- sino + p A x^,
// y = (y + tau (sino + A x^) - tau b)/(1+tau).  PD/STORE/RESID/PD1 write partials of
// 1/2 (A x_new - b)^2.
cudaError_t launch_ct_forward(const CTGeom& g, const float* x, float* sino, float* y,
                              const float* b, float tau, Partial* part_data, int mode,
                              cudaStream_t s, float p = 0.f);
// g = A^T y; when x != null: out = x - sigma g + ch h (+ TV(x) partials); else out = g.
cudaError_t launch_ct_backward(const CTGeom& g, const float* y, const float* x, const float* h,
                               float* out, float sigma, float ch, Partial* part_tv, cudaStream_t s);

}  // namespace tvs
