/*
 * tvo.c -- the oracle's 2D/3D TV prox, Gaussian blur, objective and
 * forward-backward solvers (PGD, FISTA, ProxSkip) written out in plain FP64 C.
 *
 * Test and measurement infrastructure only: it restates, loop for loop, what
 * oracle/tv.py, oracle/operators.py and oracle/solvers.py compute (and is
 * checked against them to 1e-12 by tests/test_oracle_c.py), so that full-size
 * oracle runs -- the reference optimum of a 1024 x 1024 deblurring problem, the
 * CPU baseline timed on every host core -- finish in minutes instead of hours.
 * OpenMP spreads each pass over image rows; the arithmetic per pixel is that of
 * the numpy code (sums over the image are reduced in a different order).  It
 * shares nothing with the CUDA library.
 *
 * Conventions (Eq. 5, Section 2.1): component a of D u differentiates along
 * array axis a (slowest first) with a zero last difference (Neumann); div = -D^T;
 * TV(u) = sum_i |(D u)_i|_2.  The TV prox prox_{lam TV}(z) runs the accelerated
 * dual projected gradient (AProjGD of Section 2.2 with the momentum of
 * Algorithm 3) on the unit-ball dual: t_1 = 1, r_1 = p_0 (the warm start),
 *   u = P_X(z + lam div r_k),  p_k = P_B(r_k + D u / (4 ndim lam)),
 *   t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,
 *   r_{k+1} = p_k + ((t_k - 1) / t_{k+1}) (p_k - p_{k-1}),
 * and returns u = P_X(z + lam div p_N) with p_N as the next warm start.
 * The blur is the separable, unit-sum sampled Gaussian with half-sample
 * symmetric extension (Section 3.1); its adjoint is formed by scattering.
 * The CT operator is the parallel-beam projector in Joseph's discretisation of
 * operators.py (Section 3.3), its adjoint the scatter of the same weights.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int ndim;
  long n0, n1, n2; /* slowest .. fastest; n0 = 1 for 2D */
} tvo_shape;

static tvo_shape mk_shape(int ndim, const long* s) {
  tvo_shape sh;
  sh.ndim = ndim;
  if (ndim == 2) {
    sh.n0 = 1;
    sh.n1 = s[0];
    sh.n2 = s[1];
  } else {
    sh.n0 = s[0];
    sh.n1 = s[1];
    sh.n2 = s[2];
  }
  return sh;
}

/* D u: ndim planes, plane a differentiating along the a-th slowest axis. */
static void grad_sh(tvo_shape sh, const double* u, double* g) {
  const long n = sh.n0 * sh.n1 * sh.n2, HW = sh.n1 * sh.n2, W = sh.n2;
  double* gz = sh.ndim == 3 ? g : NULL;
  double* gy = sh.ndim == 3 ? g + n : g;
  double* gx = gy + n;
#pragma omp parallel for schedule(static)
  for (long r = 0; r < sh.n0 * sh.n1; ++r) {
    const long k = r / sh.n1, i = r % sh.n1;
    for (long j = 0; j < W; ++j) {
      const long o = r * W + j;
      if (gz) gz[o] = k < sh.n0 - 1 ? u[o + HW] - u[o] : 0.0;
      gy[o] = i < sh.n1 - 1 ? u[o + W] - u[o] : 0.0;
      gx[o] = j < W - 1 ? u[o + 1] - u[o] : 0.0;
    }
  }
}

/* div p = -D^T p: sum_a ( p_a[i] [i_a < n_a - 1] - p_a[i - e_a] [i_a > 0] ). */
static void div_sh(tvo_shape sh, const double* p, double* out) {
  const long n = sh.n0 * sh.n1 * sh.n2, HW = sh.n1 * sh.n2, W = sh.n2;
  const double* pz = sh.ndim == 3 ? p : NULL;
  const double* py = sh.ndim == 3 ? p + n : p;
  const double* px = py + n;
#pragma omp parallel for schedule(static)
  for (long r = 0; r < sh.n0 * sh.n1; ++r) {
    const long k = r / sh.n1, i = r % sh.n1;
    for (long j = 0; j < W; ++j) {
      const long o = r * W + j;
      double d = 0.0;
      if (pz) {
        if (k < sh.n0 - 1) d += pz[o];
        if (k > 0) d -= pz[o - HW];
      }
      if (i < sh.n1 - 1) d += py[o];
      if (i > 0) d -= py[o - W];
      if (j < W - 1) d += px[o];
      if (j > 0) d -= px[o - 1];
      out[o] = d;
    }
  }
}

void tvo_grad(int ndim, const long* shape, const double* u, double* g) {
  grad_sh(mk_shape(ndim, shape), u, g);
}

void tvo_div(int ndim, const long* shape, const double* p, double* out) {
  div_sh(mk_shape(ndim, shape), p, out);
}

static double tv_sh(tvo_shape sh, const double* u, double* g) {
  const long n = sh.n0 * sh.n1 * sh.n2;
  grad_sh(sh, u, g);
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (long o = 0; o < n; ++o) {
    double q = 0.0;
    for (int a = 0; a < sh.ndim; ++a) q += g[a * n + o] * g[a * n + o];
    s += sqrt(q);
  }
  return s;
}

/* Isotropic TV(u); g is scratch of ndim * n doubles. */
double tvo_tv(int ndim, const long* shape, const double* u, double* g) {
  return tv_sh(mk_shape(ndim, shape), u, g);
}

/* prox_{lam TV}(z) by n_iter AProjGD iterations; p: warm start in (zeros for a
 * cold start), p_N out; u: the result.  Returns 0, or -1 if memory ran out. */
int tvo_fgp_prox(int ndim, const long* shape, const double* z, double lam, int n_iter, double* p,
                 int nonneg, double* u) {
  const tvo_shape sh = mk_shape(ndim, shape);
  const long n = sh.n0 * sh.n1 * sh.n2, nd = (long)ndim * n;
  if (lam == 0.0) {
    for (long o = 0; o < n; ++o) u[o] = nonneg ? fmax(z[o], 0.0) : z[o];
    return 0;
  }
  double* r = (double*)malloc(sizeof(double) * nd);
  double* p_prev = (double*)malloc(sizeof(double) * nd);
  double* g = (double*)malloc(sizeof(double) * nd);
  double* dv = (double*)malloc(sizeof(double) * n);
  if (!r || !p_prev || !g || !dv) {
    free(r);
    free(p_prev);
    free(g);
    free(dv);
    return -1;
  }
  const double L = 4.0 * ndim;
  memcpy(r, p, sizeof(double) * nd);       /* r_1 = p_0 */
  memcpy(p_prev, p, sizeof(double) * nd);  /* p_0 */
  double t = 1.0;                          /* t_1 */
  for (int it = 0; it < n_iter; ++it) {
    div_sh(sh, r, dv);
#pragma omp parallel for schedule(static)
    for (long o = 0; o < n; ++o) {
      const double v = z[o] + lam * dv[o];
      u[o] = nonneg ? fmax(v, 0.0) : v;
    }
    grad_sh(sh, u, g);
    const double t_new = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
    const double beta = (t - 1.0) / t_new;
#pragma omp parallel for schedule(static)
    for (long o = 0; o < n; ++o) {
      double q[3], nrm2 = 0.0;
      for (int a = 0; a < ndim; ++a) {
        q[a] = r[a * n + o] + g[a * n + o] / (L * lam);
        nrm2 += q[a] * q[a];
      }
      const double den = fmax(1.0, sqrt(nrm2));
      for (int a = 0; a < ndim; ++a) {
        const double pn = q[a] / den;
        r[a * n + o] = pn + beta * (pn - p_prev[a * n + o]);
        p_prev[a * n + o] = pn;
      }
    }
    t = t_new;
  }
  memcpy(p, p_prev, sizeof(double) * nd);
  div_sh(sh, p, dv);
  for (long o = 0; o < n; ++o) {
    const double v = z[o] + lam * dv[o];
    u[o] = nonneg ? fmax(v, 0.0) : v;
  }
  free(r);
  free(p_prev);
  free(g);
  free(dv);
  return 0;
}

/* ------------------------------------------------------------------ blur */
static long reflect(long j, long n) {
  j %= 2 * n;
  if (j < 0) j += 2 * n;
  return j >= n ? 2 * n - 1 - j : j;
}

/* out = A u: taps w[0..2R] along x (axis 1), then along y (axis 0). */
static void blur_fwd(long H, long W, const double* w, int R, const double* u, double* tmp, double* out) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < H; ++i)
    for (long j = 0; j < W; ++j) {
      double s = 0.0;
      for (int k = 0; k <= 2 * R; ++k) s += w[k] * u[i * W + reflect(j + k - R, W)];
      tmp[i * W + j] = s;
    }
#pragma omp parallel for schedule(static)
  for (long i = 0; i < H; ++i)
    for (long j = 0; j < W; ++j) {
      double s = 0.0;
      for (int k = 0; k <= 2 * R; ++k) s += w[k] * tmp[reflect(i + k - R, H) * W + j];
      out[i * W + j] = s;
    }
}

/* out = A^T y by scattering: every tap of every output sample is added back to
 * the input it came from, first along y (axis 0), then along x (axis 1). */
static void blur_adj(long H, long W, const double* w, int R, const double* y, double* tmp, double* out) {
  memset(tmp, 0, sizeof(double) * H * W);
  /* columns are independent: blocks of 64 of them per thread, each element still
   * receiving its contributions in the order (tap k, then source row i) */
#pragma omp parallel for schedule(static)
  for (long j0 = 0; j0 < W; j0 += 64) {
    const long j1 = j0 + 64 < W ? j0 + 64 : W;
    for (int k = 0; k <= 2 * R; ++k)
      for (long i = 0; i < H; ++i) {
        double* dst = tmp + reflect(i + k - R, H) * W;
        for (long j = j0; j < j1; ++j) dst[j] += w[k] * y[i * W + j];
      }
  }
  memset(out, 0, sizeof(double) * H * W);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < H; ++i)
    for (int k = 0; k <= 2 * R; ++k)
      for (long j = 0; j < W; ++j) out[i * W + reflect(j + k - R, W)] += w[k] * tmp[i * W + j];
}

void tvo_blur(long H, long W, const double* w, int R, const double* u, double* out, int adjoint) {
  double* tmp = (double*)malloc(sizeof(double) * H * W);
  if (!tmp) return;
  if (adjoint)
    blur_adj(H, W, w, R, u, tmp, out);
  else
    blur_fwd(H, W, w, R, u, tmp, out);
  free(tmp);
}

/* ------------------------------------------------------------------ projector */
/* Parallel-beam geometry (Section 3.3): an N x N image of pixel size s centred at
 * the origin, angle a at theta = a pi / n_angles, bin b on the line
 * x cos + y sin = t_b with t_b = (b - (n_det - 1)/2) d.  Joseph's discretisation,
 * as operators.py states it: a ray with |cos| >= |sin| is walked over the image
 * rows (line l = row l, at y_l = (l - (N-1)/2) s), otherwise over the columns
 * (line l = column l, at x_l); on line l it crosses the position
 * pos = (t_b - y_l sin) / cos (rows) or (t_b - x_l cos) / sin (columns), i.e.
 * the fractional pixel index c = pos / s + (N-1)/2 along the line; the sample is
 * (1 - f) u[k0] + f u[k0 + 1] with k0 = floor(c), f = c - k0, pixels outside the
 * image counting zero, and the ray sum is weighted by s / max(|cos|, |sin|). */
typedef struct {
  long N, na, nd;
  double s, d;
} tvo_geom;

static const double TVO_PI = 3.14159265358979323846;

typedef struct {
  int row;       /* walked over rows */
  double c, sn;  /* cos, sin of the angle */
  double weight; /* s / max(|cos|, |sin|) */
} ray_dir;

static ray_dir ray_direction(const tvo_geom* g, long a) {
  ray_dir r;
  const double th = (double)a * TVO_PI / (double)g->na;
  r.c = cos(th);
  r.sn = sin(th);
  r.row = fabs(r.c) >= fabs(r.sn);
  r.weight = r.row ? g->s / fabs(r.c) : g->s / fabs(r.sn);
  return r;
}

/* k0 and f of the crossing of bin b's ray with line l */
static void crossing(const tvo_geom* g, const ray_dir* r, long b, long l, long* k0, double* f) {
  const double t = ((double)b - (double)(g->nd - 1) / 2.0) * g->d;
  const double coord = ((double)l - (double)(g->N - 1) / 2.0) * g->s;
  const double pos = r->row ? (t - coord * r->sn) / r->c : (t - coord * r->c) / r->sn;
  const double frac = pos / g->s + (double)(g->N - 1) / 2.0;
  const double i0 = floor(frac);
  *k0 = (long)i0;
  *f = frac - i0;
}

/* y = A u: y[a][b] = weight_a sum_l ((1 - f) u_l[k0] + f u_l[k0 + 1]), u_l the
 * image line l (a row or a column). */
static void joseph_fwd(const tvo_geom* g, const double* u, double* y) {
  const long N = g->N;
#pragma omp parallel for schedule(dynamic)
  for (long a = 0; a < g->na; ++a) {
    const ray_dir r = ray_direction(g, a);
    for (long b = 0; b < g->nd; ++b) {
      double acc = 0.0;
      for (long l = 0; l < N; ++l) {
        long k0;
        double f;
        crossing(g, &r, b, l, &k0, &f);
        if (k0 < -1 || k0 > N - 1) continue; /* both terms outside the image */
        double term = 0.0;
        if (k0 >= 0) term += (1.0 - f) * (r.row ? u[l * N + k0] : u[k0 * N + l]);
        if (k0 + 1 <= N - 1) term += f * (r.row ? u[l * N + k0 + 1] : u[(k0 + 1) * N + l]);
        acc += term;
      }
      y[a * g->nd + b] = r.weight * acc;
    }
  }
}

/* out = A^T y: every sample's weights scattered back, angle by angle, each
 * sample adding (1 - f) y to pixel k0 and f y to pixel k0 + 1 of its line.  The
 * lines of one angle touch disjoint pixels, so they are spread over the threads. */
static void joseph_adj(const tvo_geom* g, const double* y, double* out) {
  const long N = g->N;
  memset(out, 0, sizeof(double) * N * N);
  for (long a = 0; a < g->na; ++a) {
    const ray_dir r = ray_direction(g, a);
#pragma omp parallel for schedule(static)
    for (long l = 0; l < N; ++l)
      for (long b = 0; b < g->nd; ++b) {
        long k0;
        double f;
        crossing(g, &r, b, l, &k0, &f);
        if (k0 < -1 || k0 > N - 1) continue;
        const double ya = y[a * g->nd + b];
        double* line = r.row ? out + l * N : out + l;
        const long step = r.row ? 1 : N;
        if (k0 >= 0) line[k0 * step] += r.weight * (1.0 - f) * ya;
        if (k0 + 1 <= N - 1) line[(k0 + 1) * step] += r.weight * f * ya;
      }
  }
}

void tvo_joseph(long N, long n_angles, long n_det, double s, double d, const double* in, double* out,
                int adjoint) {
  tvo_geom g = {N, n_angles, n_det, s, d};
  if (adjoint)
    joseph_adj(&g, in, out);
  else
    joseph_fwd(&g, in, out);
}

/* ------------------------------------------------------------------ solvers */
/* min_x 1/2 ||A x - b||^2 + alpha TV(x) with A the identity (R = 0, geom null),
 * the blur with taps w[0..2R] (2D only; 3D problems take the identity) or the
 * CT projector of geom (2D, b of n_angles x n_det). */
typedef struct {
  tvo_shape sh;
  long n, m; /* image size, data size */
  const double* w;
  int R;
  const tvo_geom* geom;
  const double* b;
  double alpha;
  int nonneg;
  double *t1, *t2, *t3, *g; /* scratch: t1 of the data size, t2 and t3 images, ndim planes */
} prob_t;

static void op_fwd(prob_t* P, const double* x, double* y) {
  if (P->geom)
    joseph_fwd(P->geom, x, y);
  else if (P->R == 0)
    memcpy(y, x, sizeof(double) * P->n);
  else
    blur_fwd(P->sh.n1, P->sh.n2, P->w, P->R, x, P->t3, y);
}

static void op_adj(prob_t* P, const double* x, double* y) {
  if (P->geom)
    joseph_adj(P->geom, x, y);
  else if (P->R == 0)
    memcpy(y, x, sizeof(double) * P->n);
  else
    blur_adj(P->sh.n1, P->sh.n2, P->w, P->R, x, P->t3, y);
}

/* grad f(x) = A^T (A x - b) into out. */
static void grad_f(prob_t* P, const double* x, double* out) {
  op_fwd(P, x, P->t1);
  for (long o = 0; o < P->m; ++o) P->t1[o] -= P->b[o];
  op_adj(P, P->t1, out);
}

static double objective(prob_t* P, const double* x) {
  op_fwd(P, x, P->t1);
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (long o = 0; o < P->m; ++o) {
    const double r = P->t1[o] - P->b[o];
    s += r * r;
  }
  return 0.5 * s + P->alpha * tv_sh(P->sh, x, P->g);
}

double tvo_objective(int ndim, const long* shape, const double* w, int R, const double* b, double alpha,
                     const double* x) {
  prob_t P;
  P.sh = mk_shape(ndim, shape);
  P.n = P.m = P.sh.n0 * P.sh.n1 * P.sh.n2;
  P.w = w;
  P.R = ndim == 2 ? R : 0;
  P.geom = NULL;
  P.b = b;
  P.alpha = alpha;
  P.nonneg = 0;
  P.t1 = (double*)malloc(sizeof(double) * P.n);
  P.t3 = (double*)malloc(sizeof(double) * P.n);
  P.g = (double*)malloc(sizeof(double) * P.n * ndim);
  double v = NAN;
  if (P.t1 && P.t3 && P.g) v = objective(&P, x);
  free(P.t1);
  free(P.t3);
  free(P.g);
  return v;
}

/* kind 0: PGD (Algorithm 2); 1: FISTA (Algorithm 3, Beck-Teboulle form);
 * 2: ProxSkip (Algorithm 4) with the coin of iteration k in coins[k].
 * x: x_0 in, last iterate out.  dual: the warm-start TV dual (ndim planes, zeros
 * for a fresh solve), kept across prox calls and returned.  obj (may be NULL):
 * F(x_{k+1}) per iteration.  With f_star > 0 the solve stops after the first
 * iteration whose (F - f_star)/f_star <= target.  Returns the number of
 * iterations run (>= 0), or -1 if memory ran out; *prox_calls receives the prox
 * evaluations among them. */
static int fb_core(prob_t* P_, int kind, int ndim, const long* shape, int nonneg, double gamma, double p,
                   const unsigned char* coins, int K, int n_inner, double* x, double* dual, double* obj,
                   double f_star, double target, int* prox_calls) {
  prob_t P = *P_;
  const long n = P.n;
  const double alpha = P.alpha;
  P.t1 = (double*)malloc(sizeof(double) * P.m);
  P.t2 = (double*)malloc(sizeof(double) * n);
  P.t3 = (double*)malloc(sizeof(double) * n);
  P.g = (double*)malloc(sizeof(double) * n * ndim);
  double* gf = (double*)malloc(sizeof(double) * n);
  double* v = (double*)malloc(sizeof(double) * n);
  double* xn = (double*)malloc(sizeof(double) * n);
  double* aux = (double*)malloc(sizeof(double) * n); /* FISTA: y;  ProxSkip: h */
  int ran = -1, n_prox = 0;
  if (!P.t1 || !P.t2 || !P.t3 || !P.g || !gf || !v || !xn || !aux) goto done;
  double t = 1.0;
  if (kind == 1) memcpy(aux, x, sizeof(double) * n); /* y_0 = x_0 */
  if (kind == 2) memset(aux, 0, sizeof(double) * n); /* h_0 = 0 */
  ran = 0;
  for (int k = 0; k < K; ++k) {
    if (kind == 0) {
      grad_f(&P, x, gf);
      for (long o = 0; o < n; ++o) v[o] = x[o] - gamma * gf[o];
      if (tvo_fgp_prox(ndim, shape, v, gamma * alpha, n_inner, dual, nonneg, xn)) { ran = -1; goto done; }
      ++n_prox;
    } else if (kind == 1) {
      grad_f(&P, aux, gf);
      for (long o = 0; o < n; ++o) v[o] = aux[o] - gamma * gf[o];
      if (tvo_fgp_prox(ndim, shape, v, gamma * alpha, n_inner, dual, nonneg, xn)) { ran = -1; goto done; }
      ++n_prox;
      const double t_new = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
      const double beta = (t - 1.0) / t_new;
      for (long o = 0; o < n; ++o) aux[o] = xn[o] + beta * (xn[o] - x[o]);
      t = t_new;
    } else {
      /* x^ = x - gamma (grad f(x) - h) */
      grad_f(&P, x, gf);
      for (long o = 0; o < n; ++o) P.t2[o] = x[o] - gamma * (gf[o] - aux[o]);
      if (coins[k]) {
        for (long o = 0; o < n; ++o) v[o] = P.t2[o] - (gamma / p) * aux[o];
        if (tvo_fgp_prox(ndim, shape, v, (gamma / p) * alpha, n_inner, dual, nonneg, xn)) {
          ran = -1;
          goto done;
        }
        ++n_prox;
      } else {
        memcpy(xn, P.t2, sizeof(double) * n);
      }
      for (long o = 0; o < n; ++o) aux[o] = aux[o] + (p / gamma) * (xn[o] - P.t2[o]);
    }
    memcpy(x, xn, sizeof(double) * n);
    ran = k + 1;
    if (obj || f_star > 0.0) {
      const double F = objective(&P, x);
      if (obj) obj[k] = F;
      if (f_star > 0.0 && (F - f_star) / f_star <= target) break;
    }
  }
done:
  if (prox_calls) *prox_calls = n_prox;
  free(P.t1);
  free(P.t2);
  free(P.t3);
  free(P.g);
  free(gf);
  free(v);
  free(xn);
  free(aux);
  return ran;
}

int tvo_fb_solve(int kind, int ndim, const long* shape, const double* w, int R, const double* b,
                 double alpha, int nonneg, double gamma, double p, const unsigned char* coins, int K,
                 int n_inner, double* x, double* dual, double* obj, double f_star, double target,
                 int* prox_calls) {
  prob_t P;
  P.sh = mk_shape(ndim, shape);
  P.n = P.m = P.sh.n0 * P.sh.n1 * P.sh.n2;
  P.w = w;
  P.R = ndim == 2 ? R : 0;
  P.geom = NULL;
  P.b = b;
  P.alpha = alpha;
  P.nonneg = nonneg;
  return fb_core(&P, kind, ndim, shape, nonneg, gamma, p, coins, K, n_inner, x, dual, obj, f_star, target,
                 prox_calls);
}

/* The same solvers with A the CT projector of an N x N image (pixel size s) onto
 * n_angles x n_det bins of spacing d; b is the n_angles x n_det sinogram. */
int tvo_ct_fb_solve(int kind, long N, long n_angles, long n_det, double s, double d, const double* b,
                    double alpha, int nonneg, double gamma, double p, const unsigned char* coins, int K,
                    int n_inner, double* x, double* dual, double* obj, double f_star, double target,
                    int* prox_calls) {
  const long shape[2] = {N, N};
  tvo_geom g = {N, n_angles, n_det, s, d};
  prob_t P;
  P.sh = mk_shape(2, shape);
  P.n = N * N;
  P.m = n_angles * n_det;
  P.w = NULL;
  P.R = 0;
  P.geom = &g;
  P.b = b;
  P.alpha = alpha;
  P.nonneg = nonneg;
  return fb_core(&P, kind, 2, shape, nonneg, gamma, p, coins, K, n_inner, x, dual, obj, f_star, target,
                 prox_calls);
}

/* Implicit PDHG (solvers.pdhg; Algorithm 6 at p = 1) with K = the CT projector,
 * f = 1/2 ||. - b||^2, g = alpha TV (+ the indicator of x >= 0 with nonneg):
 *   x_{k+1} = prox_{sigma g}(x_k - sigma K^T y_k),  x-bar = 2 x_{k+1} - x_k,
 *   y_{k+1} = prox_{tau f*}(y_k + tau K x-bar),
 * prox_{tau f*}(v) = v - tau (tau (v / tau) + b) / (tau + 1) (Moreau).  K x-bar is
 * formed as 2 K x_{k+1} - K x_k from the K x_{k+1} the objective needs anyway.
 * x, y: x_0, y_0 in, last iterates out; dual: the TV prox's warm start;
 * obj (may be NULL): F(x_{k+1}).  Returns K, or -1 if memory ran out. */
int tvo_ct_pdhg(long N, long n_angles, long n_det, double s, double d, const double* b, double alpha,
                int nonneg, double sigma, double tau, int K, int n_inner, double* x, double* y, double* dual,
                double* obj) {
  const long shape[2] = {N, N};
  const long n = N * N, m = n_angles * n_det;
  tvo_geom g = {N, n_angles, n_det, s, d};
  prob_t P;
  P.sh = mk_shape(2, shape);
  P.n = n;
  P.m = m;
  P.w = NULL;
  P.R = 0;
  P.geom = &g;
  P.b = b;
  P.alpha = alpha;
  P.nonneg = nonneg;
  P.g = (double*)malloc(sizeof(double) * n * 2);
  double* aty = (double*)malloc(sizeof(double) * n);
  double* v = (double*)malloc(sizeof(double) * n);
  double* xn = (double*)malloc(sizeof(double) * n);
  double* ax = (double*)malloc(sizeof(double) * m);
  double* axn = (double*)malloc(sizeof(double) * m);
  int ran = -1;
  if (!P.g || !aty || !v || !xn || !ax || !axn) goto done;
  joseph_fwd(&g, x, ax);
  for (int k = 0; k < K; ++k) {
    joseph_adj(&g, y, aty);
    for (long o = 0; o < n; ++o) v[o] = x[o] - sigma * aty[o];
    if (tvo_fgp_prox(2, shape, v, sigma * alpha, n_inner, dual, nonneg, xn)) goto done;
    joseph_fwd(&g, xn, axn);
    for (long o = 0; o < m; ++o) {
      const double vv = y[o] + tau * (2.0 * axn[o] - ax[o]);
      const double w = vv / tau;
      y[o] = vv - tau * (tau * w + b[o]) / (tau + 1.0);
    }
    memcpy(x, xn, sizeof(double) * n);
    memcpy(ax, axn, sizeof(double) * m);
    if (obj) {
      double r2 = 0.0;
#pragma omp parallel for reduction(+ : r2) schedule(static)
      for (long o = 0; o < m; ++o) {
        const double r = ax[o] - b[o];
        r2 += r * r;
      }
      obj[k] = 0.5 * r2 + alpha * tv_sh(P.sh, x, P.g);
    }
    ran = k + 1;
  }
  if (K == 0) ran = 0;
done:
  free(P.g);
  free(aty);
  free(v);
  free(xn);
  free(ax);
  free(axn);
  return ran;
}

/* Threads the OpenMP passes use (1 without OpenMP). */
int tvo_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
