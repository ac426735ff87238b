/*
 * FP64 CPU oracle for the KDE-on-grid hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the CUDA library computes.  It shares no code, header,
 * table or constant generator with the library under paper_2004_13653_gb300/,
 * and only the tests, __graft_entry__.smoke() and the CPU-baseline leg of
 * bench.py may load it.  Nothing here is tuned: every function is the
 * definition written out, summed in the order the definition states.
 *
 * Passages followed (arXiv 2004.13653):
 *   - Mercator projection .................. Sec. III-A, Eq. 1-4
 *   - the eight 2-D product kernels ........ Sec. III-C, Table 1, and their
 *     radial variants K(|u|) on the unit disk (kernel ids 8..15)
 *   - indicator I(.) (inclusive |s| <= 1) .. Sec. III-C, Eq. 8
 *   - density as a kernel sum over points .. Sec. III-C, Eq. 7, read as the
 *     direct sum F[i,j] = 1/(N h^2) sum_p w_p k((gx_i-x_p)/h) k((gy_j-y_p)/h)
 *     at cell centres gx_i = ox + (i+1/2) cell, gy_j = oy + (j+1/2) cell
 *   - Douglas-Peucker with the vertical Euclidean distance of Eq. 9 and the
 *     "larger than epsilon" split rule ..... Sec. III-B, Sec. IV-A
 *   - the paper's binned estimator: count matrix M_D of the projected fixes
 *     with linear interpolation of skipped cells (Sec. IV-B, Eq. InterX/
 *     InterY, Algorithm 3) and its discrete convolution (Eq. 7)
 *
 * Readings where the paper is silent:
 *   - s and t in Table 1 are offsets divided by the bandwidth h, with support
 *     |s|,|t| <= 1 (every Table 1 factor then integrates to one);
 *   - Mercator uses the WGS84 ellipsoid, longitude in radians of the absolute
 *     longitude, and the caller's standard latitude phi0;
 *   - the normaliser uses N = number of points, not the weight sum;
 *   - the LSCV loss is the grid form described at oracle_lscv_loss().
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum {
  OR_UNIFORM = 0,
  OR_TRIANGULAR = 1,
  OR_EPANECHNIKOV = 2,
  OR_QUARTIC = 3,
  OR_TRIWEIGHT = 4,
  OR_TRICUBE = 5,
  OR_GAUSSIAN = 6,
  OR_COSINE = 7
};

/* One factor k(s) of the product kernel f(s,t) = k(s) k(t) of Table 1.  The
 * 2-D constant of each row of Table 1 is the square of the 1-D constant used
 * here.  I(s) = 1 when |s| <= 1 (Eq. 8 with s measured in bandwidths). */
double oracle_kernel_1d(int kid, double s) {
  const double a = fabs(s);
  const int inside = a <= 1.0;
  switch (kid) {
    case OR_UNIFORM:
      return inside ? 0.5 : 0.0;
    case OR_TRIANGULAR:
      return inside ? (1.0 - a) : 0.0;
    case OR_EPANECHNIKOV:
      return inside ? 0.75 * (1.0 - s * s) : 0.0;
    case OR_QUARTIC: {
      const double u = 1.0 - s * s;
      return inside ? (15.0 / 16.0) * u * u : 0.0;
    }
    case OR_TRIWEIGHT: {
      const double u = 1.0 - s * s;
      return inside ? (35.0 / 32.0) * u * u * u : 0.0;
    }
    case OR_TRICUBE: {
      const double u = 1.0 - a * a * a;
      return inside ? (70.0 / 81.0) * u * u * u : 0.0;
    }
    case OR_GAUSSIAN:
      return exp(-0.5 * s * s) / sqrt(2.0 * M_PI);
    case OR_COSINE:
      return inside ? (M_PI / 4.0) * cos(0.5 * M_PI * s) : 0.0;
    default:
      return NAN;
  }
}

/* Radial variants of the Table 1 kernels (kernel ids 8..15 = 8 + the Table 1
 * id): K(u) = c k~(|u|) on the unit disk, k~ the Table 1 profile without its
 * 1-D constant, c = 1 / (2 pi int_0^1 r k~(r) dr) so that K integrates to one
 * over the plane.  The integrals, by hand:
 *   uniform 1            -> 1/2      c = 1/pi
 *   triangular 1-r       -> 1/6      c = 3/pi
 *   epanechnikov 1-r^2   -> 1/4      c = 2/pi
 *   quartic (1-r^2)^2    -> 1/6      c = 3/pi
 *   triweight (1-r^2)^3  -> 1/8      c = 4/pi
 *   tricube (1-r^3)^3    -> 81/440   c = 220/(81 pi)
 *   cosine cos(pi r/2)   -> 2/pi - 4/pi^2   c = pi/(4 pi - 8)
 *   gaussian exp(-r^2/2) -> 1 (whole plane)  c = 1/(2 pi): the product kernel.
 * kid here is the Table 1 id (0..7). */
double oracle_kernel_radial(int kid, double r) {
  const int inside = r <= 1.0;
  switch (kid) {
    case OR_UNIFORM:
      return inside ? 1.0 / M_PI : 0.0;
    case OR_TRIANGULAR:
      return inside ? (3.0 / M_PI) * (1.0 - r) : 0.0;
    case OR_EPANECHNIKOV:
      return inside ? (2.0 / M_PI) * (1.0 - r * r) : 0.0;
    case OR_QUARTIC: {
      const double u = 1.0 - r * r;
      return inside ? (3.0 / M_PI) * u * u : 0.0;
    }
    case OR_TRIWEIGHT: {
      const double u = 1.0 - r * r;
      return inside ? (4.0 / M_PI) * u * u * u : 0.0;
    }
    case OR_TRICUBE: {
      const double u = 1.0 - r * r * r;
      return inside ? (220.0 / (81.0 * M_PI)) * u * u * u : 0.0;
    }
    case OR_GAUSSIAN:
      return exp(-0.5 * r * r) / (2.0 * M_PI);
    case OR_COSINE:
      return inside ? (M_PI / (4.0 * M_PI - 8.0)) * cos(0.5 * M_PI * r) : 0.0;
    default:
      return NAN;
  }
}

/* ---------------------------------------------------------------- Mercator */

/* Eq. 1-4: r0 = a cos(phi0) / sqrt(1 - e^2 sin^2 phi0);
 * q = ln tan(pi/4 + phi/2) + (e/2) ln((1 - e sin phi)/(1 + e sin phi));
 * x = lambda r0;  y = q r0.   lonlat is interleaved (lon, lat) in degrees. */
void oracle_mercator(const double* lonlat, int64_t n, double lat0_deg,
                     double semi_major, double ecc2, double* xy) {
  const double e = sqrt(ecc2);
  const double phi0 = lat0_deg * M_PI / 180.0;
  const double r0 =
      semi_major * cos(phi0) / sqrt(1.0 - ecc2 * sin(phi0) * sin(phi0));
  for (int64_t p = 0; p < n; ++p) {
    const double lam = lonlat[2 * p] * M_PI / 180.0;
    const double phi = lonlat[2 * p + 1] * M_PI / 180.0;
    const double sp = sin(phi);
    const double q = log(tan(M_PI / 4.0 + phi / 2.0)) +
                     0.5 * e * log((1.0 - e * sp) / (1.0 + e * sp));
    xy[2 * p] = lam * r0;
    xy[2 * p + 1] = q * r0;
  }
}

/* ------------------------------------------------------- parallel for-loop */

typedef struct {
  void (*body)(void* ctx, int64_t lo, int64_t hi);
  void* ctx;
  int64_t n, chunk;
  int64_t next; /* protected by mu */
  pthread_mutex_t mu;
} pfor_t;

static void* pfor_worker(void* arg) {
  pfor_t* pf = (pfor_t*)arg;
  for (;;) {
    pthread_mutex_lock(&pf->mu);
    const int64_t lo = pf->next;
    pf->next += pf->chunk;
    pthread_mutex_unlock(&pf->mu);
    if (lo >= pf->n) break;
    const int64_t hi = lo + pf->chunk < pf->n ? lo + pf->chunk : pf->n;
    pf->body(pf->ctx, lo, hi);
  }
  return NULL;
}

static int oracle_threads(int requested) {
  if (requested > 0) return requested;
  const char* env = getenv("ORACLE_THREADS");
  if (env && atoi(env) > 0) return atoi(env);
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}

static void parallel_for(int64_t n, int64_t chunk, int nthreads,
                         void (*body)(void*, int64_t, int64_t), void* ctx) {
  pfor_t pf;
  pf.body = body;
  pf.ctx = ctx;
  pf.n = n;
  pf.chunk = chunk > 0 ? chunk : 1;
  pf.next = 0;
  pthread_mutex_init(&pf.mu, NULL);
  nthreads = oracle_threads(nthreads);
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  int started = 0;
  for (int t = 1; t < nthreads; ++t)
    if (pthread_create(&th[started], NULL, pfor_worker, &pf) == 0) ++started;
  pfor_worker(&pf);
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&pf.mu);
}

/* ----------------------------------------------------------- KDE on a grid */

typedef struct {
  const double* xy;
  const double* w;
  int64_t n;
  double ox, oy, cell, h;
  int nx, ny, kid;
  const int64_t* cells;
  double* out;
} kde_ctx_t;

static void kde_body(void* vctx, int64_t lo, int64_t hi) {
  const kde_ctx_t* c = (const kde_ctx_t*)vctx;
  const double norm = 1.0 / ((double)c->n * c->h * c->h);
  for (int64_t q = lo; q < hi; ++q) {
    const int64_t flat = c->cells ? c->cells[q] : q;
    const int64_t i = flat % c->nx; /* column index along x */
    const int64_t j = flat / c->nx; /* row index along y    */
    const double gx = c->ox + ((double)i + 0.5) * c->cell;
    const double gy = c->oy + ((double)j + 0.5) * c->cell;
    double acc = 0.0;
    for (int64_t p = 0; p < c->n; ++p) {
      const double s = (gx - c->xy[2 * p]) / c->h;
      const double t = (gy - c->xy[2 * p + 1]) / c->h;
      const double wp = c->w ? c->w[p] : 1.0;
      if (c->kid >= 8)
        acc += wp * oracle_kernel_radial(c->kid - 8, sqrt(s * s + t * t));
      else
        acc += wp * oracle_kernel_1d(c->kid, s) * oracle_kernel_1d(c->kid, t);
    }
    c->out[q] = norm * acc;
  }
}

/* F at the listed cells (flat index j*nx + i), or at every cell when cells is
 * NULL (then ncells must be nx*ny).  xy is interleaved absolute metres, w may
 * be NULL (unit weights). */
int oracle_kde_cells(const double* xy, const double* w, int64_t n, double ox,
                     double oy, double cell, int nx, int ny, double h, int kid,
                     const int64_t* cells, int64_t ncells, double* out,
                     int nthreads) {
  if (n <= 0) {
    for (int64_t q = 0; q < ncells; ++q) out[q] = 0.0;
    return 0;
  }
  if (kid < 0 || kid > 15 || nx <= 0 || ny <= 0 || !(h > 0)) return -1;
  kde_ctx_t c = {xy, w, n, ox, oy, cell, h, nx, ny, kid, cells, out};
  parallel_for(ncells, 1, nthreads, kde_body, &c);
  return 0;
}

/* --------------------------------------- Gaussian vector-Jacobian product */

/* With F as above (Gaussian kernel) and a cotangent G on the grid,
 * L = sum_ij G_ij F_ij.  For each point p:
 *   dL/dw_p = c sum_ij G_ij k(s_ip) k(t_jp)
 *   dL/dx_p = c w_p / h sum_ij G_ij s_ip k(s_ip) k(t_jp)     (k'(s) = -s k(s))
 *   dL/dy_p = c w_p / h sum_ij G_ij t_jp k(s_ip) k(t_jp)
 *   dL/dh   = -(2/h) L + c/h sum_p w_p sum_ij G_ij (s^2 + t^2) k k
 * with c = 1/(N h^2), s_ip = (gx_i - x_p)/h, t_jp = (gy_j - y_p)/h. */
typedef struct {
  const double* xy;
  const double* w;
  int64_t n;
  double ox, oy, cell, h;
  int nx, ny;
  const double* G;
  const int64_t* pts;
  double *gw, *gxy, *hterm, *lterm;
} vjp_ctx_t;

static void vjp_body(void* vctx, int64_t lo, int64_t hi) {
  const vjp_ctx_t* c = (const vjp_ctx_t*)vctx;
  const double norm = 1.0 / ((double)c->n * c->h * c->h);
  for (int64_t q = lo; q < hi; ++q) {
    const int64_t p = c->pts ? c->pts[q] : q;
    const double xp = c->xy[2 * p], yp = c->xy[2 * p + 1];
    const double wp = c->w ? c->w[p] : 1.0;
    double sw = 0.0, sx = 0.0, sy = 0.0, s2 = 0.0;
    for (int j = 0; j < c->ny; ++j) {
      const double t = (c->oy + (j + 0.5) * c->cell - yp) / c->h;
      const double kt = oracle_kernel_1d(OR_GAUSSIAN, t);
      for (int i = 0; i < c->nx; ++i) {
        const double s = (c->ox + (i + 0.5) * c->cell - xp) / c->h;
        const double ks = oracle_kernel_1d(OR_GAUSSIAN, s);
        const double g = c->G[(int64_t)j * c->nx + i] * ks * kt;
        sw += g;
        sx += g * s;
        sy += g * t;
        s2 += g * (s * s + t * t);
      }
    }
    c->gw[q] = norm * sw;
    c->gxy[2 * q] = norm * wp * sx / c->h;
    c->gxy[2 * q + 1] = norm * wp * sy / c->h;
    c->hterm[q] = norm * wp * s2 / c->h;
    c->lterm[q] = norm * wp * sw;
  }
}

/* Gradients for the listed points (all when pts is NULL, then npts = n).
 * grad_h (may be NULL) is written only when every point is listed. */
int oracle_kde_vjp_gauss(const double* xy, const double* w, int64_t n,
                         double ox, double oy, double cell, int nx, int ny,
                         double h, const double* G, const int64_t* pts,
                         int64_t npts, double* gw, double* gxy, double* grad_h,
                         int nthreads) {
  if (n <= 0 || nx <= 0 || ny <= 0 || !(h > 0)) return -1;
  double* hterm = (double*)calloc((size_t)npts, sizeof(double));
  double* lterm = (double*)calloc((size_t)npts, sizeof(double));
  if (!hterm || !lterm) {
    free(hterm);
    free(lterm);
    return -2;
  }
  vjp_ctx_t c = {xy, w,  n,   ox,  oy, cell,  h,    nx,
                 ny, G,  pts, gw,  gxy, hterm, lterm};
  parallel_for(npts, 1, nthreads, vjp_body, &c);
  if (grad_h && !pts) {
    double L = 0.0, hs = 0.0;
    for (int64_t q = 0; q < npts; ++q) {
      L += lterm[q];
      hs += hterm[q];
    }
    *grad_h = -2.0 / h * L + hs;
  }
  free(hterm);
  free(lterm);
  return 0;
}

/* ------------------------------------------------------------ LSCV (grid) */

/* Bilinear interpolation of a grid sampled at cell centres, zero outside the
 * grid.  Writes the four (flat index, weight) pairs; returns their count. */
static int bilerp_taps(double x, double y, double ox, double oy, double cell,
                       int nx, int ny, int64_t* idx, double* wt) {
  const double fx = (x - ox) / cell - 0.5;
  const double fy = (y - oy) / cell - 0.5;
  const double i0 = floor(fx), j0 = floor(fy);
  const double ax = fx - i0, ay = fy - j0;
  int m = 0;
  for (int b = 0; b < 2; ++b)
    for (int a = 0; a < 2; ++a) {
      const double ii = i0 + a, jj = j0 + b;
      if (ii < 0 || jj < 0 || ii >= nx || jj >= ny) continue;
      idx[m] = (int64_t)jj * nx + (int64_t)ii;
      wt[m] = (a ? ax : 1.0 - ax) * (b ? ay : 1.0 - ay);
      ++m;
    }
  return m;
}

/* Least-squares cross-validation on the grid (Gaussian kernel):
 *   L = cell^2 sum_ij F_ij^2 - (2/N) sum_p w_p bilerp(F - F_p, x_p)
 * where F is the density above on the grid, F_p = w_p K(|g - x_p|/h)/(N h^2)
 * is point p's own term at each cell centre g (K(u) = exp(-u^2/2)/(2 pi)), and
 * bilerp samples a grid at x_p.  bilerp(F - F_p, x_p) is the interpolated
 * density of the other points, the leave-one-out density at x_p; the first
 * term approximates the integral of the squared density.  F is passed in
 * (computed by oracle_kde_grid). */
double oracle_lscv_loss(const double* F, const double* xy, const double* w,
                        int64_t n, double ox, double oy, double cell, int nx,
                        int ny, double h) {
  double sq = 0.0;
  for (int64_t q = 0; q < (int64_t)nx * ny; ++q) sq += F[q] * F[q];
  const double k0 = 1.0 / (2.0 * M_PI);
  double loo = 0.0;
  for (int64_t p = 0; p < n; ++p) {
    int64_t idx[4];
    double wt[4];
    const double x = xy[2 * p], y = xy[2 * p + 1];
    const int m = bilerp_taps(x, y, ox, oy, cell, nx, ny, idx, wt);
    const double wp = w ? w[p] : 1.0;
    double v = 0.0;
    for (int t = 0; t < m; ++t) {
      const double gx = ox + ((double)(idx[t] % nx) + 0.5) * cell;
      const double gy = oy + ((double)(idx[t] / nx) + 0.5) * cell;
      const double dx = (gx - x) / h, dy = (gy - y) / h;
      const double own = wp * k0 * exp(-0.5 * (dx * dx + dy * dy)) / ((double)n * h * h);
      v += wt[t] * (F[idx[t]] - own);
    }
    loo += wp * v;
  }
  return cell * cell * sq - 2.0 / (double)n * loo;
}

/* Cotangent of the LSCV loss with respect to the grid:
 *   G_ij = 2 cell^2 F_ij - (2/N) sum_p w_p beta_p,ij
 * where beta_p,ij are the bilinear weights of point p. */
void oracle_lscv_cotangent(const double* F, const double* xy, const double* w,
                           int64_t n, double ox, double oy, double cell,
                           int nx, int ny, double* G) {
  for (int64_t q = 0; q < (int64_t)nx * ny; ++q) G[q] = 2.0 * cell * cell * F[q];
  for (int64_t p = 0; p < n; ++p) {
    int64_t idx[4];
    double wt[4];
    const int m = bilerp_taps(xy[2 * p], xy[2 * p + 1], ox, oy, cell, nx, ny,
                              idx, wt);
    const double wp = w ? w[p] : 1.0;
    for (int t = 0; t < m; ++t) G[idx[t]] -= 2.0 / (double)n * wp * wt[t];
  }
}

/* ---------------------------------------------------------- Douglas-Peucker */

/* Vertical Euclidean distance of Eq. 9: distance from p to the line through
 * s and e; when s and e coincide, the distance to that point. */
double oracle_ved(double px, double py, double sx, double sy, double ex,
                  double ey) {
  const double dx = ex - sx, dy = ey - sy;
  const double len = sqrt(dx * dx + dy * dy);
  const double vx = px - sx, vy = py - sy;
  if (len == 0.0) return sqrt(vx * vx + vy * vy);
  return fabs(vx * dy - vy * dx) / len;
}

/* Sec. III-B: keep both ends; split at the point of largest VED (the first
 * one on ties) while that distance is larger than eps.  Trajectories are the
 * index ranges [off[k], off[k+1]).  keep[] receives 1 for kept points. */
int oracle_dp(const double* xy, const int64_t* off, int64_t ntraj, double eps,
              uint8_t* keep) {
  for (int64_t k = 0; k < ntraj; ++k) {
    const int64_t a = off[k], b = off[k + 1];
    if (b <= a) continue;
    for (int64_t p = a; p < b; ++p) keep[p] = 0;
    keep[a] = 1;
    keep[b - 1] = 1;
    if (b - a < 3) continue;
    /* explicit stack of (start, end) index pairs */
    int64_t cap = 64, top = 0;
    int64_t* st = (int64_t*)malloc((size_t)cap * 2 * sizeof(int64_t));
    if (!st) return -2;
    st[0] = a;
    st[1] = b - 1;
    top = 1;
    while (top > 0) {
      --top;
      const int64_t s = st[2 * top], e = st[2 * top + 1];
      if (e - s < 2) continue;
      double dmax = -1.0;
      int64_t kmax = -1;
      for (int64_t p = s + 1; p < e; ++p) {
        const double d = oracle_ved(xy[2 * p], xy[2 * p + 1], xy[2 * s],
                                    xy[2 * s + 1], xy[2 * e], xy[2 * e + 1]);
        if (d > dmax) {
          dmax = d;
          kmax = p;
        }
      }
      if (dmax > eps) {
        keep[kmax] = 1;
        if (top + 2 > cap) {
          cap *= 2;
          int64_t* ns = (int64_t*)realloc(st, (size_t)cap * 2 * sizeof(int64_t));
          if (!ns) {
            free(st);
            return -2;
          }
          st = ns;
        }
        st[2 * top] = s;
        st[2 * top + 1] = kmax;
        ++top;
        st[2 * top] = kmax;
        st[2 * top + 1] = e;
        ++top;
      }
    }
    free(st);
  }
  return 0;
}

/* ------------------------------------------- binned estimator (Eq. 7) */

/* Cell of coordinate v on an axis with origin o, cell side d, n cells; -1 when
 * outside [o, o + n d). */
static int64_t cell_of(double v, double o, double d, int n) {
  const double f = floor((v - o) / d);
  if (!(f >= 0.0) || f >= (double)n) return -1;
  return (int64_t)f;
}

/* Count matrix M_D (Sec. IV-B, Algorithm 3): every fix adds one to its cell;
 * when `interpolate` is set, between consecutive fixes of one trajectory
 * (both inside the grid) whose cells differ by c_max = max(|di|, |dj|) > 1
 * the cells round(i0 + c/c_max di), round(j0 + c/c_max dj), c = 1..c_max-1,
 * are added too (Eq. InterX / InterY; rounding = floor(v + 1/2)).
 * off: trajectory boundaries [off[k], off[k+1]) (ntraj of them).  Returns the
 * number of interpolated cells added. */
int64_t oracle_count_matrix(const double* xy, const int64_t* off, int64_t ntraj, double ox,
                            double oy, double cell, int nx, int ny, int interpolate,
                            int32_t* counts) {
  int64_t added = 0;
  for (int64_t q = 0; q < (int64_t)nx * ny; ++q) counts[q] = 0;
  for (int64_t k = 0; k < ntraj; ++k) {
    for (int64_t p = off[k]; p < off[k + 1]; ++p) {
      const int64_t i = cell_of(xy[2 * p], ox, cell, nx);
      const int64_t j = cell_of(xy[2 * p + 1], oy, cell, ny);
      if (i < 0 || j < 0) continue;
      counts[j * nx + i] += 1;
      if (!interpolate || p + 1 >= off[k + 1]) continue;
      const int64_t i1 = cell_of(xy[2 * p + 2], ox, cell, nx);
      const int64_t j1 = cell_of(xy[2 * p + 3], oy, cell, ny);
      if (i1 < 0 || j1 < 0) continue;
      const int64_t di = i1 - i, dj = j1 - j;
      const int64_t cmax = llabs(di) > llabs(dj) ? llabs(di) : llabs(dj);
      for (int64_t c = 1; c < cmax; ++c) {
        const double t = (double)c / (double)cmax;
        const int64_t ic = (int64_t)floor((double)i + t * (double)di + 0.5);
        const int64_t jc = (int64_t)floor((double)j + t * (double)dj + 0.5);
        counts[jc * nx + ic] += 1;
        ++added;
      }
    }
  }
  return added;
}

/* Eq. 7: out(i,j) = sum_{s,t=-a..a} f(s,t) M_D(i-s, j-t) with the Table 1
 * stencil f(s,t) = k(s cell/h) k(t cell/h) / (N h^2) (cells outside the grid
 * count zero), a = (window-1)/2. */
void oracle_convolve(const int32_t* counts, int nx, int ny, double cell, double h, int kid,
                     int window, int64_t n_points, double* out) {
  const int a = (window - 1) / 2;
  const double norm = 1.0 / ((double)n_points * h * h);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double acc = 0.0;
      for (int t = -a; t <= a; ++t)
        for (int s = -a; s <= a; ++s) {
          const int ii = i - s, jj = j - t;
          if (ii < 0 || jj < 0 || ii >= nx || jj >= ny) continue;
          acc += oracle_kernel_1d(kid, s * cell / h) * oracle_kernel_1d(kid, t * cell / h) *
                 (double)counts[(int64_t)jj * nx + ii];
        }
      out[(int64_t)j * nx + i] = norm * acc;
    }
}
