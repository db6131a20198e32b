/*
 * tvs.h -- C ABI of the GB300 ProxSkip / PDHGSkip path for
 *
 *     min_u  1/2 || A u - b ||_2^2 + alpha TV(u)      (Eq. 5; Eq. 1 with D = 1/2||.||^2, R = TV)
 *
 * with isotropic TV and forward differences under Neumann boundary conditions
 * (Eq. 5), A the identity, a separable Gaussian blur (Section 3.1) or a 2D
 * parallel-beam projector (Section 3.3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Arrays are dense, row-major float32.  A 2D image has dims {nx, ny, 1} and is
 * stored as ny rows of nx values; a 3D volume has dims {nx, ny, nz} (nz slices).
 * A sinogram is n_angles rows of n_det values.  A dual TV field holds `ndim`
 * planes of the image size, plane a differentiating along the a-th slowest
 * array axis (2D: plane 0 = vertical, plane 1 = horizontal; 3D: z, y, x).
 *
 * Pointers are device pointers on the context's stream unless a `tvs_mem`
 * argument says TVS_MEM_HOST; the caller owns every pointer it passes.  Calls
 * that return results synchronise the context's stream before returning.
 * Every call validates its arguments first: on TVS_EINVAL nothing has been
 * launched and no state has changed.  The message of the last failure on the
 * calling thread is returned by tvs_last_error().  A context must be used by
 * one host thread at a time.
 *
 * The dual step of the TV prox uses the bound ||D||^2 <= 4 * ndim (8 in 2D, 12
 * in 3D), so one inner iteration is p <- P_B(r + D u / (4 ndim lambda)).
 */
#ifndef TVS_H
#define TVS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TVS_OK = 0,
  TVS_EINVAL = 1,        /* invalid argument; nothing was launched           */
  TVS_ENOMEM = 2,        /* a device or pinned-host allocation failed        */
  TVS_ECUDA = 3,         /* a CUDA runtime call failed (message has details) */
  TVS_ENUMERIC = 4,      /* non-finite value in an input or in the objective */
  TVS_ETIMEDOUT = 5,     /* a solve passed its wall-clock limit (the
                            TVS_SOLVE_TIMEOUT_MS environment variable, in ms;
                            PGD, FISTA, ProxSkip, PDHG, PDHGSkip-2,
                            PDHGSkip-1, explicit PDHG): it stopped
                            launching iterations and cleaned up; or a 3D inner
                            kernel gave up (after 2 s) waiting for a tile load
                            and left part of its output unwritten              */
  TVS_EUNSUPPORTED = 6   /* valid request this build does not implement       */
} tvs_status;

typedef enum { TVS_OP_IDENTITY = 0, TVS_OP_GAUSS_BLUR = 1, TVS_OP_PARALLEL_BEAM = 2 } tvs_op_kind;
/* Storage type of the TV dual field (the inner iterations always compute in
 * float32; stores round to nearest).  TVS_DUAL_Q15 is signed 16-bit fixed point
 * for values in [-1, 1] -- the range of every stored dual component, each being a
 * component of a vector projected onto the unit ball: integer i stands for
 * i / 32767, stores clamp to [-1, 1].  Not in the paper: at the two bytes of
 * bfloat16 and half it resolves 2^-15 over the whole range (64x bfloat16's and 8x
 * half's step near 1), which keeps the prox result within 2e-3 of an FP64 dual
 * at prox steps lambda where bfloat16 does not. */
typedef enum { TVS_DUAL_F32 = 0, TVS_DUAL_BF16 = 1, TVS_DUAL_F16 = 2, TVS_DUAL_Q15 = 3 } tvs_dual_dtype;
typedef enum { TVS_MEM_DEVICE = 0, TVS_MEM_HOST = 1 } tvs_mem;

typedef struct tvs_ctx tvs_ctx;
typedef struct tvs_problem tvs_problem;

/* Forward operator A.
 * TVS_OP_GAUSS_BLUR: 2*blur_radius+1 taps w_i = exp(-i^2/(2 sigma^2)), normalised
 *   to sum 1, applied along x then y with half-sample symmetric extension
 *   ("... b a | a b ..."); this A is symmetric, so A^T = A.  1 <= radius <= 8.
 * TVS_OP_PARALLEL_BEAM (2D, nx == ny == N): Joseph's ray-driven projector.  The
 *   image spans [-N s/2, N s/2]^2 (s = pixel_size); angle a is a*pi/n_angles;
 *   bin b is the line x cos + y sin = (b - (n_det-1)/2) * det_spacing.  Rays with
 *   |cos| >= |sin| are walked over rows, others over columns, interpolating
 *   linearly between the two nearest pixels with weight s / max(|cos|,|sin|);
 *   pixels outside the image count as zero.  The backprojector is the exact
 *   transpose of the same weights. */
typedef struct {
  tvs_op_kind kind;
  int blur_radius;
  double blur_sigma;
  int n_angles;
  int n_det;
  double pixel_size;
  double det_spacing;
} tvs_op_desc;

typedef struct {
  int ndim;            /* 2 or 3 (3 only with TVS_OP_IDENTITY)              */
  int nx, ny, nz;      /* nz = 1 for 2D                                      */
  double alpha;        /* TV weight, >= 0                                    */
  int nonneg;          /* 1: add the constraint u >= 0 (Section 3.3)         */
  tvs_op_desc op;
} tvs_problem_desc;

/* Forward-backward solvers (PGD = Algorithm 2, FISTA = Algorithm 3, ProxSkip =
 * Algorithm 4).  gamma > 0; p in (0, 1] (ProxSkip only); n_inner >= 0 inner FGP
 * iterations per prox, warm-started from the dual of the previous prox call;
 * max_iter >= 0 outer iterations.  When f_star > 0 the solve stops (within a
 * few iterations) once (F(x_k) - f_star) / f_star <= target_rel_gap.
 * objective_every >= 1: F is evaluated every that many iterations (NaN between).
 * Checkpoint / resume: with resume = 1 the solve continues the previous solve of
 * the same problem instead of starting afresh -- the control variate h and the
 * warm-start TV dual kept in the problem are not reset, x_inout (and y_inout)
 * hold the iterate it returned, and iteration numbering (hence the coins)
 * starts at k0, the number of iterations already done.  A run of K iterations
 * followed by a resumed run of K' iterations with k0 = K computes the same
 * iterates as one run of K + K' iterations.  Not available for FISTA (its
 * extrapolation state is not kept). */
typedef struct {
  double gamma;
  double p;
  uint64_t seed;
  int max_iter;
  int n_inner;
  tvs_dual_dtype dual;
  double f_star;
  double target_rel_gap;
  int objective_every;
  int resume;
  long long k0;
  double target_rel_dist;  /* > 0: also stop once ||x_k - u*|| / ||u*|| <= this
                              (needs a reference set with tvs_problem_set_reference) */
} tvs_fb_params;

/* Primal-dual solvers (PDHG, PDHGSkip-2 = Algorithm 6) with the naming of
 * Algorithm 6: sigma is the primal and tau the dual step, sigma tau ||A||^2 <= 1.
 * resume / k0 as for tvs_fb_params. */
typedef struct {
  double sigma;
  double tau;
  double p;
  uint64_t seed;
  int max_iter;
  int n_inner;
  tvs_dual_dtype dual;
  double f_star;
  double target_rel_gap;
  int objective_every;
  int resume;
  long long k0;
  double target_rel_dist;  /* as in tvs_fb_params */
} tvs_pd_params;

/* Solve record.  The caller owns the three host arrays (any may be NULL) and
 * sets cap to their length; entry k describes outer iteration k: objective[k]
 * = F(x_{k+1}), coins[k] = theta_k, t_s[k] = device time in seconds from the
 * start of the solve until F(x_{k+1}) was known.  The scalars are outputs. */
typedef struct {
  int cap;
  double* objective;
  unsigned char* coins;
  double* t_s;
  int iters_run;          /* outer iterations executed                          */
  int prox_calls;         /* prox evaluations among them                        */
  int reached;            /* 1 if the relative-gap target was met               */
  int reached_iter;       /* first k with (F(x_{k+1}) - f*)/f* <= target, else -1 */
  double time_to_target_s;/* t_s[reached_iter], or -1                           */
  double solve_ms;        /* device time of the whole solve (CUDA events)       */
  double fgp_ms;          /* device time inside inner-iteration launches        */
  long long fgp_launches; /* inner-iteration kernel launches (a 2D launch runs up
                             to 4 inner iterations)                              */
  long long fgp_pixel_iters; /* pixels x inner iterations processed by them    */
  double* rel_dist;       /* host, may be NULL: ||x_{k+1} - u*|| / ||u*|| per iteration
                             when the problem has a reference (NaN otherwise)   */
} tvs_trace;

/* ---- context ----------------------------------------------------------- */
/* Creates a context on `device`.  `cuda_stream` is a cudaStream_t to launch on;
 * NULL creates a private non-blocking stream owned by the context. */
tvs_status tvs_create(tvs_ctx** ctx, int device, void* cuda_stream);
/* Destroys the context and every problem still attached to it. */
tvs_status tvs_destroy(tvs_ctx* ctx);
const char* tvs_last_error(void);
/* Bytes of device memory currently held by the context and its problems. */
size_t tvs_device_bytes(const tvs_ctx* ctx);

/* ---- problems ------------------------------------------------------------ */
/* Copies b (measurement: image-sized, or n_angles x n_det for CT) into memory
 * the problem owns, together with all its workspace.  Returns TVS_ENUMERIC if b
 * holds a non-finite value. */
tvs_status tvs_problem_create(tvs_ctx* ctx, const tvs_problem_desc* desc, const float* b,
                              tvs_mem b_mem, tvs_problem** out);
/* Reference solution u* (image size; NULL removes it).  While set, every solve
 * of the problem records the relative distance ||x_k - u*|| / ||u*|| -- the
 * error measure of Sections 2 and 3 -- next to the objective, and can stop on it
 * (target_rel_dist). */
tvs_status tvs_problem_set_reference(tvs_problem* prob, const float* u_ref, tvs_mem mem);
/* Replaces the problem's copy of b (same size). */
tvs_status tvs_problem_set_data(tvs_problem* prob, const float* b, tvs_mem b_mem);
tvs_status tvs_problem_destroy(tvs_problem* prob);
/* y = A x (adjoint = 0) or y = A^T x (adjoint = 1); device pointers. */
tvs_status tvs_op_apply(tvs_problem* prob, const float* x, float* y, int adjoint);
/* F(x) = 1/2 ||A x - b||^2 + alpha TV(x) for a device image x (FP32 terms,
 * FP64 accumulation). */
tvs_status tvs_objective(tvs_problem* prob, const float* x, double* out);

/* ---- TV prox (Eq. 3 with R = TV; inner solver of Sections 2.2, 3.1) ------ */
/* u = prox_{lambda TV}(z) (with u >= 0 if nonneg) by n_iter iterations of the
 * accelerated dual projected gradient.  dual_state: NULL for a cold start (p =
 * 0), else a device buffer of ndim planes of `dual` elements holding the warm
 * start; it receives the final dual p_N.  lambda = 0 or n_iter = 0 returns
 * u = P(z + lambda div p0).  z and u may not alias. */
tvs_status tv_prox(tvs_ctx* ctx, int ndim, const int dims[3], const float* z, float* u,
                   double lambda, int n_iter, tvs_dual_dtype dual, void* dual_state, int nonneg);

/* Kernel configuration the context uses for the inner iterations of an image of
 * this shape and dual type: out = {iterations per launch, columns per lane,
 * rows per warp (+100 for the register-blocked kernel)}; {1, ., .} means one
 * iteration per launch (3D).  The first query (or the first prox / solve) of a
 * 2D shape times the candidates on the device and caches the fastest;
 * TVS_FGP_CONFIG="tb,cpl,rpw" in the environment forces one, and
 * TVS_TUNE_CACHE=path keeps the choices in a text file across processes.  3D volumes
 * large enough to fill the GPU with (x-y tile, z chunk) pairs take the z-marching
 * kernel whose planes arrive by TMA tile loads (register loads where a buffer or
 * the row pitch is not 16-byte aligned), smaller ones the tiled kernel;
 * TVS_FGP3D=tma, zm or tile forces one (tma falls back to zm where the row pitch or
 * a buffer is not 16-byte aligned), TVS_FGP3D_CFG="cpl,rpw,zc" picks a z-marching
 * variant and TVS_FGP3D_STAGES=3 a three-stage TMA ring (all read at each launch).
 * Not in the paper: a performance knob only (with an FP32, BF16 or FP16 dual every
 * configuration computes identical iterates; with the 16-bit fixed point the
 * stored codes may differ by a few units, see TVS_DUAL_Q15). */
tvs_status tvs_fgp_config(tvs_ctx* ctx, int ndim, const int dims[3], tvs_dual_dtype dual, int out[3]);

/* ---- allocation-free TV prox -------------------------------------------------- */
/* The paper has no counterpart to this entry point.  It serves callers that may
 * not allocate device memory: applications that reserve all of the GPU's memory
 * for their own pool, or that run beside a thread capturing a CUDA graph in
 * global mode (where cudaMalloc is refused).  It computes exactly what tv_prox
 * computes, without a context and without allocating or freeing anything: the
 * working dual fields live in one array of TVS_NOALLOC_SCRATCH_BYTES inside the
 * library's device image.  CUDA loads that image onto a device lazily (by
 * default), so the array takes its device memory when the first call on that
 * device looks up its address, and keeps it until the process exits.
 *
 * Arguments are those of tv_prox, on the current device, plus the cudaStream_t
 * to launch on (NULL = the default stream); the call synchronises that stream
 * before returning.  The scratch needed is (dual_state ? 3 : 4) * ndim * n
 * elements of the dual type (n = pixels): a 1024 x 1024 FP32 image fits, and a
 * larger request returns TVS_EUNSUPPORTED without launching anything.  Invalid
 * arguments give TVS_EINVAL, CUDA failures TVS_ECUDA; no message is recorded
 * for tvs_last_error().  The first call on a device looks up the array's device
 * address (and sets kernel attributes) with that device current; make it -- a
 * call with n_iter = 0 on a 1 x 1 image will do -- before the application
 * reserves the device's memory for its own pool and before any stream capture
 * begins.  All calls on a device share the array, which keeps
 * the last call's contents (the cold-start dual is cleared on every call): calls
 * whose GPU work overlaps -- from several host threads or several streams --
 * race on it and must be serialised by the caller. */
#define TVS_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
tvs_status tv_prox_noalloc(int ndim, const int dims[3], const float* z, float* u, double lambda,
                           int n_iter, tvs_dual_dtype dual, void* dual_state, int nonneg,
                           void* cuda_stream);

/* ROF duality gap of a TV-prox dual, the certificate of the prox's accuracy
 * (Section 2.1: prox_{lambda TV}(z) and its dual, the Dual-ROF problem Eq. 6,
 * written for the unit-ball dual p = q / lambda).  With u = z + lambda div p,
 *   G = P(u) - D(p) = lambda * sum_i ( |(D u)_i|_2 - <(D u)_i, p_i> ),
 * which is >= 0 whenever every |p_i| <= 1 and 0 exactly at the optimum.
 * dual_state: p as tv_prox leaves it (ndim planes of the dual dtype, device
 * memory); z as passed to tv_prox (device).  For the unconstrained prox
 * (nonneg = 0).  Synchronous: *gap (host) receives G, accumulated in compensated
 * FP32 and combined in FP64. */
tvs_status tv_prox_gap(tvs_ctx* ctx, int ndim, const int dims[3], const float* z, double lambda,
                       tvs_dual_dtype dual, const void* dual_state, double* gap);

/* ---- outer solvers --------------------------------------------------------- */
/* x_inout: initial iterate in, final iterate out (image size, TVS_MEM_* says
 * where it lives).  The control variate starts at h_0 = 0, the TV dual at 0. */
tvs_status pgd_solve(tvs_problem* prob, const tvs_fb_params* prm, float* x_inout, tvs_mem mem,
                     tvs_trace* trace);
tvs_status fista_solve(tvs_problem* prob, const tvs_fb_params* prm, float* x_inout, tvs_mem mem,
                       tvs_trace* trace);
tvs_status proxskip_solve(tvs_problem* prob, const tvs_fb_params* prm, float* x_inout,
                          tvs_mem mem, tvs_trace* trace);
/* y_inout: dual iterate (measurement size) in and out; h_0 = 0. */
tvs_status pdhg_solve(tvs_problem* prob, const tvs_pd_params* prm, float* x_inout,
                      float* y_inout, tvs_mem mem, tvs_trace* trace);
tvs_status pdhgskip_solve(tvs_problem* prob, const tvs_pd_params* prm, float* x_inout,
                          float* y_inout, tvs_mem mem, tvs_trace* trace);

/* PDHGSkip-1 (Algorithm 5, Condat's skipping PDHG) with omega + 1 = 1/p: when
 * theta_k = 0 the iteration skips the prox and both applications of A (only
 * y <- prox_{tau f*}(y + tau A x_k) runs, from the stored A x_k).  Same arguments
 * and trace as pdhgskip_solve. */
tvs_status pdhgskip1_solve(tvs_problem* prob, const tvs_pd_params* prm, float* x_inout,
                           float* y_inout, tvs_mem mem, tvs_trace* trace);

/* Explicit PDHG with diagonal preconditioning: the explicit formulation of
 * Section 3.2 (K = [A; D], f = 1/2 ||. - b||^2 + alpha ||.||_{2,1}, g = 0 or the
 * non-negativity indicator when the problem has nonneg set, every prox closed
 * form), the solver the paper uses for its reference solutions (Section 4.1),
 * with the step sizes of Pock and Chambolle (ICCV 2011, Lemma 2, exponent 1):
 * pixel j steps T_j = sigma / sum_i |K_ij| = sigma / ((A^T 1)_j + n_j), where n_j
 * counts the differences touching pixel j; row i of A steps S_i = tau / (A 1)_i;
 * the rows of D step tau / 2.  An empty row or column steps by the bare scale.
 * Per iteration:
 *   x+ = P_X(x - T (A^T y - div q));  x- = 2 x+ - x;
 *   y+ = (y + S (A x- - b)) / (1 + S);  q+ = P_alpha(q + (tau/2) D x-).
 * sigma, tau > 0 with sigma * tau <= 1 (1, 1 is the lemma's choice).  2D only. */
typedef struct {
  double sigma;            /* primal step scale                                  */
  double tau;              /* dual step scale                                    */
  int max_iter;
  double f_star;           /* > 0: stop at the relative-gap target               */
  double target_rel_gap;
  int objective_every;     /* record F(x_{k+1}) every this many iterations (>= 1) */
  double target_rel_dist;  /* as in tvs_fb_params                                */
} tvs_pdx_params;
/* x_inout (image), y_inout (measurement size) and q_inout (two planes of the
 * image size, vertical then horizontal differences; may be NULL for q_0 = 0 and
 * no output) carry the iterates in and out, so a long solve can run in pieces.
 * The trace as for the other solvers (every iteration counts as a prox call; the
 * inner-iteration fields are 0).  The first call on a problem allocates one
 * measurement-sized work buffer that the problem keeps. */
tvs_status pdhg_explicit_solve(tvs_problem* prob, const tvs_pdx_params* prm, float* x_inout,
                               float* y_inout, float* q_inout, tvs_mem mem, tvs_trace* trace);

/* ---- many independent problems at once -------------------------------------- */
/* ProxSkip on n independent 2D problems (identity or blur operators; any sizes),
 * each with its own alpha (from its problem), gamma, p, seed, f_star and target
 * (prm[i]); max_iter, n_inner and the dual type must agree.  All problems advance
 * in lockstep through shared launches (one CUDA graph per outer iteration covers
 * every problem); problem i follows exactly the iteration proxskip_solve would
 * run on it (same coins, same arithmetic) and stops at the first x_k whose
 * objective meets its target, or after max_iter iterations.  x_inout[i] and
 * traces[i] (may be NULL) as for proxskip_solve; problems must belong to ctx and
 * be distinct, and blur problems must share one blur radius.  Not in the paper:
 * a batching mode for many small solves. */
tvs_status proxskip_solve_batch(tvs_ctx* ctx, int n, tvs_problem* const* probs,
                                const tvs_fb_params* prm, float* const* x_inout, tvs_mem mem,
                                tvs_trace* traces);

/* ---- the light-prox case: Dual-ROF (Section 2.1, Eq. 6) and Dual-Huber-ROF
 * (Section 2.2, Eq. 8) -------------------------------------------------------- */
/* min over |q_i| <= alpha of F(q) = 1/2 ||div q + b||^2 + (eps/(2 alpha)) ||q||^2
 * (eps = 0: Dual-ROF), by projected gradient (p = 1), its accelerated form
 * AProjGD (p = 1, accelerated = 1) or ProxSkip with the pointwise alpha-ball
 * projection (Eq. 7) as the prox (p < 1), step gamma (Section 2.1 uses 1/8).  dims = {nx, ny}; b is a 2D image; q_inout holds the
 * two dual planes (vertical, horizontal), initial value in, final out; u_out
 * (may be NULL) receives u = b + div q.  The trace's objective[k] = F(q_{k+1});
 * f_star > 0 stops at the relative-gap target as for the other solvers. */
typedef struct {
  double alpha;
  double eps;
  double gamma;
  double p;
  uint64_t seed;
  int max_iter;
  double f_star;
  double target_rel_gap;
  int accelerated;  /* 1 (with p = 1): AProjGD -- each projected gradient step is
                       taken from the extrapolated point y_k = q_k + ((t_{k-1} - 1)/t_k)
                       (q_k - q_{k-1}) of Algorithm 3 (t_0 = 1), Section 2.2 */
  const float* u_ref;      /* NULL, or a reference solution u* (image size, in the
                              memory `mem` names): the trace's rel_dist[k] then holds
                              ||u_{k+1} - u*|| / ||u*|| with u = b + div q, the
                              error measure of Sections 2.1 and 2.2             */
  double target_rel_dist;  /* > 0 (with u_ref): also stop once rel_dist <= this   */
} tvs_rof_params;
tvs_status dual_rof_solve(tvs_ctx* ctx, const int dims[2], const float* b, const tvs_rof_params* prm,
                          float* q_inout, float* u_out, tvs_mem mem, tvs_trace* trace);

/* ---- the coin (Algorithms 4 and 6) ----------------------------------------- */
/* theta_k = [(w >> 11) < p 2^53], w the first word of Philox4x64-10 with counter
 * (k, 0, 0, 0) and key (seed, 0).  Returns 0/1, or -1 if p is not in (0, 1]. */
int tvs_coin(uint64_t seed, double p, int64_t k);
/* theta_{k0}, ..., theta_{k0+K-1} computed by a device kernel, written to the
 * host array out (K bytes). */
tvs_status tvs_coin_schedule_device(tvs_ctx* ctx, uint64_t seed, double p, int64_t k0, int K,
                                    unsigned char* out);

#ifdef __cplusplus
}
#endif
#endif /* TVS_H */
