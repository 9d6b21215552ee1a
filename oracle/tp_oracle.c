/*
 * FP64 CPU oracle for the probed (randomized-trace) FWI gradient of
 * Louboutin & Herrmann, "Ultra-low memory seismic inversion with randomized
 * trace estimation" (arXiv 2104.00794).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * Plain loops in double precision, OpenMP over grid points, no blocking or
 * fusion beyond what the equations state.
 *
 * Discrete system (the paper does not give its discretisation; this is the
 * reading used throughout, chosen so that adjoint and gradient are exact):
 *   grid  : nz x ny x nx nodes (ny = 1 in 2-D), spacing h, flat index
 *           (z*ny + y)*nx + x; zero (Dirichlet) values outside the grid.
 *   L     : centred 2k-order Laplacian, weights from Fornberg's algorithm.
 *   time  : levels t = 0..nt-1, u[0] = u[1] = 0 (Algorithm 1 starts its
 *           loop at the third level with two zero levels before it).
 *   F     : for t = 1..nt-2 (Algorithm 1, line 1, operator f)
 *             u[t+1] = 2u[t] - u[t-1] + dt^2 v^2 (L u[t] + S^T q[t]),
 *           data d[t] = R u[t] (Eq. 2, F(m; q)); m = 1/v^2 (squared slowness).
 *   F^T   : lambda[nt] = lambda[nt+1] = 0, for j = nt-1 .. 2
 *             lambda[j] = 2 lambda[j+1] - lambda[j+2]
 *                         + dt^2 v^2 (L lambda[j+1] + R^T s[j])
 *           (Algorithm 1, line 5, operator f^T: the exact transpose of the
 *           block lower-triangular time-stepping system), and
 *           (F^T s)[t] = S lambda[t+1] for t = 1..nt-2, zero otherwise.
 *   J     : 1/2 sum_t ||R u[t] - d_obs[t]||^2                     (Eq. 2)
 *   grad  : dJ/dm = - sum_{k=2}^{nt-1} lambda[k] * udd[k],
 *           udd[k] = (u[k] - 2u[k-1] + u[k-2]) / dt^2             (Eq. 3)
 *           with lambda driven by the residual s = R u - d_obs.  Eq. 3 is
 *           printed without a sign; the exact derivative carries a minus.
 *   sponge: optional absorbing layer (not in the paper): damping m*eta*du/dt
 *           with eta(x) = eta_max ((w - d)/w)^2 at nodes whose distance d (in
 *           cells) to the nearest face is below w; every face but the top
 *           (z = 0), which stays the zero-pressure free surface where sources
 *           and receivers sit.  The step becomes
 *             (1+a) u[t+1] = 2u[t] - (1-a) u[t-1] + dt^2 v^2 (L u[t] + S^T q[t]),
 *           a = eta dt / 2; the time-stepping blocks stay symmetric, so the
 *           adjoint keeps the same form, and udd above becomes
 *           udd[k] + eta (u[k] - u[k-2]) / (2 dt) (the derivative of the
 *           damped system with respect to m).  w = 0 is the undamped scheme.
 *   probed: ubar[x,i] = sum_k Q[k,i] udd[k,x], vbar[x,i] = sum_k Q[k,i]
 *           lambda[k,x], output -scale * sum_i ubar[x,i] vbar[x,i]
 *           (Algorithm 1 lines 2, 6, 8; Eq. 4), scale = 1/r for random
 *           probes (Eq. 1), 1 for orthonormal / identity probes.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int ndim, nx, ny, nz, nt, order;
  double h, dt;
  int sponge;        /* width w of the absorbing layer in cells (0: none) */
  double sponge_eta; /* eta_max [1/s] */
} oracle_grid;

#define MAXR 8

/* ------------------------------------------------------------ FD weights */
/* Fornberg (1988), "Generation of finite difference formulas on arbitrarily
 * spaced grids", Math. Comp. 51: recursive weights for derivatives 0..m at
 * point z from nodes x[0..n].  Returns weights for the second derivative at
 * 0 on the nodes -R..R (R = order/2): w[k] multiplies u(+-k h), k = 0..R. */
int oracle_fd_weights(int order, double* w) {
  if (order < 2 || order % 2 || order / 2 > MAXR) return 1;
  const int R = order / 2, n = 2 * R, m = 2;
  double x[2 * MAXR + 1];
  double c[2 * MAXR + 1][3];
  for (int i = 0; i <= n; ++i) {
    x[i] = (double)(i - R);
    for (int k = 0; k <= m; ++k) c[i][k] = 0.0;
  }
  const double z = 0.0;
  double c1 = 1.0, c4 = x[0] - z;
  c[0][0] = 1.0;
  for (int i = 1; i <= n; ++i) {
    int mn = i < m ? i : m;
    double c2 = 1.0, c5 = c4;
    c4 = x[i] - z;
    for (int j = 0; j < i; ++j) {
      double c3 = x[i] - x[j];
      c2 *= c3;
      if (j == i - 1) {
        for (int k = mn; k >= 1; --k) c[i][k] = c1 * (k * c[i - 1][k - 1] - c5 * c[i - 1][k]) / c2;
        c[i][0] = -c1 * c5 * c[i - 1][0] / c2;
      }
      for (int k = mn; k >= 1; --k) c[j][k] = (c4 * c[j][k] - k * c[j][k - 1]) / c3;
      c[j][0] = c4 * c[j][0] / c3;
    }
    c1 = c2;
  }
  for (int k = 0; k <= R; ++k) w[k] = c[R + k][2];
  return 0;
}

/* ------------------------------------------------------------ Laplacian */
static inline double at(const oracle_grid* g, const double* u, long z, long y, long x) {
  if (z < 0 || z >= g->nz || y < 0 || y >= g->ny || x < 0 || x >= g->nx) return 0.0;
  return u[(z * g->ny + y) * g->nx + x];
}

/* out = L u with zero values outside the grid (1/h^2 included). */
void oracle_laplacian(const oracle_grid* g, const double* u, double* out) {
  double w[MAXR + 1];
  oracle_fd_weights(g->order, w);
  const int R = g->order / 2;
  const double ih2 = 1.0 / (g->h * g->h);
  const long nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for schedule(static)
  for (long z = 0; z < nz; ++z)
    for (long y = 0; y < ny; ++y)
      for (long x = 0; x < nx; ++x) {
        double c = u[(z * ny + y) * nx + x];
        double s = g->ndim * w[0] * c;
        for (int k = 1; k <= R; ++k) {
          s += w[k] * (at(g, u, z, y, x + k) + at(g, u, z, y, x - k));
          s += w[k] * (at(g, u, z + k, y, x) + at(g, u, z - k, y, x));
          if (g->ndim == 3) s += w[k] * (at(g, u, z, y + k, x) + at(g, u, z, y - k, x));
        }
        out[(z * ny + y) * nx + x] = s * ih2;
      }
}

static long npts(const oracle_grid* g) { return (long)g->nx * g->ny * g->nz; }

/* eta at flat node index p (see the header); 0 without a sponge */
static double sponge_eta(const oracle_grid* g, long p) {
  if (g->sponge <= 0) return 0.0;
  const long x = p % g->nx, y = (p / g->nx) % g->ny, z = p / ((long)g->nx * g->ny);
  long d = x < g->nx - 1 - x ? x : g->nx - 1 - x;
  const long dz = g->nz - 1 - z; /* the top face z = 0 stays the free surface */
  if (dz < d) d = dz;
  if (g->ndim == 3) {
    const long dy = y < g->ny - 1 - y ? y : g->ny - 1 - y;
    if (dy < d) d = dy;
  }
  if (d >= g->sponge) return 0.0;
  const double t = (double)(g->sponge - d) / (double)g->sponge;
  return g->sponge_eta * t * t;
}

static double* zalloc(long n) { return (double*)calloc((size_t)n, sizeof(double)); }

/* One time step of operator f (forward) or f^T (adjoint); both have the form
 *   (1+a) out = 2 cur - (1-a) old + dt^2 v^2 (L cur + rhs),
 * where rhs is a sparse set of point values added at idx[k] and a = eta dt/2
 * (zero outside the sponge). */
static void leapfrog(const oracle_grid* g, const double* vel, const double* cur, const double* old,
                     double* out, double* lap, int nrhs, const int64_t* idx, const double* val) {
  const long N = npts(g);
  const double dt2 = g->dt * g->dt;
  oracle_laplacian(g, cur, lap);
  for (int k = 0; k < nrhs; ++k) lap[idx[k]] += val[k];
#pragma omp parallel for schedule(static)
  for (long x = 0; x < N; ++x) {
    const double a = 0.5 * sponge_eta(g, x) * g->dt;
    out[x] = (2.0 * cur[x] - (1.0 - a) * old[x] + dt2 * vel[x] * vel[x] * lap[x]) / (1.0 + a);
  }
}

/* ------------------------------------------------------------ operator F */
/* d[t][j] = u[t][rec[j]], t = 0..nt-1.  q is [nt][nsrc].  If u_hist is not
 * NULL it receives every level u[t] ([nt][N]). */
int oracle_forward(const oracle_grid* g, int nsrc, const int64_t* src, int nrec, const int64_t* rec,
                   const double* vel, const double* q, double* d, double* u_hist) {
  const long N = npts(g);
  const int nt = g->nt;
  double *um = zalloc(N), *u0 = zalloc(N), *up = zalloc(N), *lap = zalloc(N);
  if (!um || !u0 || !up || !lap) return 1;
  memset(d, 0, sizeof(double) * (size_t)nt * nrec);
  if (u_hist) memset(u_hist, 0, sizeof(double) * (size_t)nt * N);
  for (int t = 1; t <= nt - 2; ++t) {
    leapfrog(g, vel, u0, um, up, lap, nsrc, src, q + (long)t * nsrc);
    double* tmp = um; um = u0; u0 = up; up = tmp; /* u0 = u[t+1] */
    for (int j = 0; j < nrec; ++j) d[(long)(t + 1) * nrec + j] = u0[rec[j]];
    if (u_hist) memcpy(u_hist + (long)(t + 1) * N, u0, sizeof(double) * N);
  }
  free(um); free(u0); free(up); free(lap);
  return 0;
}

/* ------------------------------------------------------------ operator F^T */
/* s is [nt][nrec]; q_out is [nt][nsrc] with q_out[t] = lambda[t+1][src].
 * If lam_hist is not NULL it receives lambda[k] for k = 0..nt-1 (levels
 * below 2 are left zero: they are never formed). */
int oracle_adjoint(const oracle_grid* g, int nsrc, const int64_t* src, int nrec, const int64_t* rec,
                   const double* vel, const double* s, double* q_out, double* lam_hist) {
  const long N = npts(g);
  const int nt = g->nt;
  double *l2 = zalloc(N), *l1 = zalloc(N), *l0 = zalloc(N), *lap = zalloc(N);
  if (!l2 || !l1 || !l0 || !lap) return 1;
  memset(q_out, 0, sizeof(double) * (size_t)nt * nsrc);
  if (lam_hist) memset(lam_hist, 0, sizeof(double) * (size_t)nt * N);
  /* l2 = lambda[j+2], l1 = lambda[j+1], l0 = lambda[j] */
  for (int j = nt - 1; j >= 2; --j) {
    leapfrog(g, vel, l1, l2, l0, lap, nrec, rec, s + (long)j * nrec);
    for (int k = 0; k < nsrc; ++k) q_out[(long)(j - 1) * nsrc + k] = l0[src[k]];
    if (lam_hist) memcpy(lam_hist + (long)j * N, l0, sizeof(double) * N);
    double* tmp = l2; l2 = l1; l1 = l0; l0 = tmp;
  }
  free(l2); free(l1); free(l0); free(lap);
  return 0;
}

static double residual(int nt, int nrec, const double* d, const double* dobs, double* res) {
  double J = 0.0;
  for (long i = 0; i < (long)nt * nrec; ++i) {
    res[i] = d[i] - dobs[i];
    J += res[i] * res[i];
  }
  return 0.5 * J;
}

/* ------------------------------------------------------------ full gradient */
/* Conventional adjoint-state gradient (Eq. 3) with the complete forward
 * history stored (N x nt values).  grad is dJ/dm. */
int oracle_gradient_full(const oracle_grid* g, int nsrc, const int64_t* src, int nrec,
                         const int64_t* rec, const double* vel, const double* q, const double* dobs,
                         double* grad, double* misfit) {
  const long N = npts(g);
  const int nt = g->nt;
  const double idt2 = 1.0 / (g->dt * g->dt);
  double* hist = zalloc((long)nt * N);
  double* d = zalloc((long)nt * nrec);
  double* res = zalloc((long)nt * nrec);
  double *l2 = zalloc(N), *l1 = zalloc(N), *l0 = zalloc(N), *lap = zalloc(N);
  if (!hist || !d || !res || !l2 || !l1 || !l0 || !lap) return 1;
  oracle_forward(g, nsrc, src, nrec, rec, vel, q, d, hist);
  *misfit = residual(nt, nrec, d, dobs, res);
  memset(grad, 0, sizeof(double) * N);
  for (int j = nt - 1; j >= 2; --j) {
    leapfrog(g, vel, l1, l2, l0, lap, nrec, rec, res + (long)j * nrec);
    const double *a = hist + (long)j * N, *b = hist + (long)(j - 1) * N, *c = hist + (long)(j - 2) * N;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x)
      grad[x] -= l0[x] * ((a[x] - 2.0 * b[x] + c[x]) * idt2 + sponge_eta(g, x) * (a[x] - c[x]) / (2.0 * g->dt));
    double* tmp = l2; l2 = l1; l1 = l0; l0 = tmp;
  }
  free(hist); free(d); free(res); free(l2); free(l1); free(l0); free(lap);
  return 0;
}

/* ------------------------------------------------------------ probed gradient */
/* Algorithm 1.  Q is [nt][r]; only rows 2..nt-1 enter (the levels at which
 * udd and lambda are formed).  form = 0 accumulates Q^T udd with udd formed
 * from three wavefield levels, exactly as line 2 prints it; form = 1 folds the
 * second time difference into the probes, ubar += Qt[j] u[j] with
 * Qt[j] = (Q'[j] - 2 Q'[j+1] + Q'[j+2]) / dt^2 and Q'[k] = Q[k] for
 * 2 <= k <= nt-1, zero otherwise.  The two are algebraically identical.
 * ubar_out / vbar_out ([N][r]) are optional copies of the accumulators. */
int oracle_gradient_probed(const oracle_grid* g, int nsrc, const int64_t* src, int nrec,
                           const int64_t* rec, const double* vel, const double* q,
                           const double* dobs, int r, const double* Q, double scale, int form,
                           double* grad, double* misfit, double* ubar_out, double* vbar_out) {
  const long N = npts(g);
  const int nt = g->nt;
  const double idt2 = 1.0 / (g->dt * g->dt);
  double* ubar = zalloc(N * r);
  double* vbar = zalloc(N * r);
  double* d = zalloc((long)nt * nrec);
  double* res = zalloc((long)nt * nrec);
  double *um = zalloc(N), *u0 = zalloc(N), *up = zalloc(N), *lap = zalloc(N);
  double* Qt = zalloc((long)(nt + 2) * r);
  double* Qd = zalloc((long)(nt + 2) * r);
  if (!ubar || !vbar || !d || !res || !um || !u0 || !up || !lap || !Qt || !Qd) return 1;
  if (form == 1) {
    /* u[j] enters udd[k] for k = j, j+1, j+2 with weights 1, -2, 1 (/dt^2)
     * and the sponge's first difference for k = j, j+2 with +1, -1 (/2dt) */
    for (int j = 0; j < nt; ++j)
      for (int i = 0; i < r; ++i) {
        double s = 0.0, sd = 0.0;
        for (int o = 0; o <= 2; ++o) {
          int k = j + o;
          double wk = (o == 1) ? -2.0 : 1.0;
          double wd = o == 0 ? 1.0 : (o == 2 ? -1.0 : 0.0);
          if (k >= 2 && k <= nt - 1) {
            s += wk * Q[(long)k * r + i];
            sd += wd * Q[(long)k * r + i];
          }
        }
        Qt[(long)j * r + i] = s * idt2;
        Qd[(long)j * r + i] = sd / (2.0 * g->dt);
      }
  }
  /* forward propagation, lines 0-3 */
  for (int t = 1; t <= nt - 2; ++t) {
    leapfrog(g, vel, u0, um, up, lap, nsrc, src, q + (long)t * nsrc);
    const int k = t + 1; /* level just formed: u[k] = up, u[k-1] = u0, u[k-2] = um */
    for (int j = 0; j < nrec; ++j) d[(long)k * nrec + j] = up[rec[j]];
    if (form == 0) {
      const double* Qk = Q + (long)k * r;
#pragma omp parallel for schedule(static)
      for (long x = 0; x < N; ++x) {
        double udd = (up[x] - 2.0 * u0[x] + um[x]) * idt2 + sponge_eta(g, x) * (up[x] - um[x]) / (2.0 * g->dt);
        for (int i = 0; i < r; ++i) ubar[x * r + i] += Qk[i] * udd;
      }
    } else {
      const double* Qk = Qt + (long)k * r;
      const double* Qdk = Qd + (long)k * r;
#pragma omp parallel for schedule(static)
      for (long x = 0; x < N; ++x) {
        const double eta = sponge_eta(g, x);
        for (int i = 0; i < r; ++i) ubar[x * r + i] += (Qk[i] + eta * Qdk[i]) * up[x];
      }
    }
    double* tmp = um; um = u0; u0 = up; up = tmp;
  }
  *misfit = residual(nt, nrec, d, dobs, res);
  /* back propagation, lines 4-7 (um/u0/up reused as lambda levels) */
  memset(um, 0, sizeof(double) * N);
  memset(u0, 0, sizeof(double) * N);
  double *l2 = um, *l1 = u0, *l0 = up;
  for (int j = nt - 1; j >= 2; --j) {
    leapfrog(g, vel, l1, l2, l0, lap, nrec, rec, res + (long)j * nrec);
    const double* Qj = Q + (long)j * r;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x)
      for (int i = 0; i < r; ++i) vbar[x * r + i] += Qj[i] * l0[x];
    double* tmp = l2; l2 = l1; l1 = l0; l0 = tmp;
  }
  /* line 8: trace of the outer product as a pointwise sum over probes */
#pragma omp parallel for schedule(static)
  for (long x = 0; x < N; ++x) {
    double s = 0.0;
    for (int i = 0; i < r; ++i) s += ubar[x * r + i] * vbar[x * r + i];
    grad[x] = -scale * s;
  }
  if (ubar_out) memcpy(ubar_out, ubar, sizeof(double) * N * r);
  if (vbar_out) memcpy(vbar_out, vbar, sizeof(double) * N * r);
  free(ubar); free(vbar); free(d); free(res); free(um); free(u0); free(up); free(lap); free(Qt); free(Qd);
  return 0;
}

/* ------------------------------------------------------------ probes */
/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the generator adds the odd constant
 * GAMMA = 0x9E3779B97F4A7C15 to its state and returns a mix of the new state.
 * The n-th output (n >= 1) of a generator whose state starts at s is
 * therefore mix(s + n*GAMMA) (mod 2^64). */
static uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t oracle_splitmix64(uint64_t state, uint64_t n) {
  return sm64_mix(state + n * 0x9E3779B97F4A7C15ULL);
}

/* Probe matrix Z [nt][r] for one shot (Eq. 1: columns with E[z z^T] = I).
 *   key_shot = sm64(seed, shot + 1), key_col = sm64(key_shot, i + 1),
 *   draw (t, d) = sm64(key_col, D*t + d + 1), D draws per entry.
 * kind 0, Rademacher: z = +1 if the top bit of the draw is 0, else -1 (D=1).
 * kind 1, Gaussian (Irwin-Hall of 12 uniforms, D=12):
 *   S = sum_d (draw >> 32) - 6*2^32 (exact in int64),
 *   z = (2*floor(S / 2^12) + 1) * 2^-21  (exactly representable in float32).
 * kind 2, identity: r must equal nt, Z = I. */
int oracle_probes(int kind, int nt, int r, uint64_t seed, int shot, double* Z) {
  if (kind == 2) {
    if (r != nt) return 1;
    memset(Z, 0, sizeof(double) * (size_t)nt * r);
    for (int t = 0; t < nt; ++t) Z[(long)t * r + t] = 1.0;
    return 0;
  }
  if (kind != 0 && kind != 1) return 1;
  const uint64_t ks = oracle_splitmix64(seed, (uint64_t)shot + 1);
  for (int i = 0; i < r; ++i) {
    const uint64_t kc = oracle_splitmix64(ks, (uint64_t)i + 1);
    for (int t = 0; t < nt; ++t) {
      double z;
      if (kind == 0) {
        uint64_t x = oracle_splitmix64(kc, (uint64_t)t + 1);
        z = (x >> 63) ? -1.0 : 1.0;
      } else {
        int64_t S = 0;
        for (int d = 0; d < 12; ++d) S += (int64_t)(oracle_splitmix64(kc, (uint64_t)12 * t + d + 1) >> 32);
        S -= (int64_t)6 << 32;
        int64_t fl = (S >= 0) ? (S >> 12) : -((-S + 4095) >> 12); /* floor(S / 4096) */
        z = (double)(2 * fl + 1) * ldexp(1.0, -21);
      }
      Z[(long)t * r + i] = z;
    }
  }
  return 0;
}
