/*
 * sea_oracle.c -- plain, slow, FP64 CPU oracle for the exact-exchange
 * (exx) application of SCDM+exx+ACE (arXiv 2208.06097, Sec. II B, II C).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the timed CPU baseline
 * of the benchmark use it.  It shares no code with the CUDA library.
 *
 * Every function follows the paper's definitions step by step, in plain
 * loops, in double precision, compiled with -ffp-contract=off so that no
 * multiply-add is fused behind the reader's back.  Where the paper is silent
 * the reading taken is stated next to the code.
 *
 * Grid conventions: orthorhombic periodic cell with edge lengths cell[a]
 * (bohr) sampled by N[a] points, h[a] = cell[a]/N[a], dV = h0 h1 h2.
 * Orbital i lives at phi[((i*nz + z)*ny + y)*nx + x], x fastest.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_LMAX_MAX 8
#define ORA_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Finite-difference second derivative of order 2p (App. C: O(h^12)).  */
/* ------------------------------------------------------------------ */

static double fact(int n) {
  double f = 1.0;
  for (int k = 2; k <= n; ++k) f *= (double)k;
  return f;
}

/* Central second-derivative weights c[0..p] for a symmetric (2p+1)-point
 * stencil of accuracy order 2p:  f''(x) ~ (1/h^2) sum_{k=-p..p} c_|k| f(x+kh)
 * with c_k = 2 (-1)^{k+1} (p!)^2 / (k^2 (p-k)! (p+k)!) and c_0 = -2 sum c_k.
 * App. C fixes the order (h^12, p = 6). */
void ora_fd_coeffs(int p, double* c) {
  double s = 0.0;
  for (int k = 1; k <= p; ++k) {
    double sign = (k % 2 == 1) ? 1.0 : -1.0;
    c[k] = 2.0 * sign * fact(p) * fact(p) / ((double)k * k * fact(p - k) * fact(p + k));
    s += c[k];
  }
  c[0] = -2.0 * s;
}

/* out = -Lap_h v on an ex*ey*ez box, v taken as zero outside the box
 * (homogeneous Dirichlet).  Layout [z][y][x]. */
void ora_apply_neg_lap(const double* v, double* out, int ex, int ey, int ez,
                       const double h[3], int p) {
  double c[16];
  ora_fd_coeffs(p, c);
  const int e[3] = {ex, ey, ez};
  for (int z = 0; z < ez; ++z)
    for (int y = 0; y < ey; ++y)
      for (int x = 0; x < ex; ++x) {
        const int t[3] = {x, y, z};
        double lap = 0.0;
        for (int a = 0; a < 3; ++a) {
          double s = c[0] * v[((size_t)z * ey + y) * ex + x];
          for (int k = 1; k <= p; ++k) {
            for (int sgn = -1; sgn <= 1; sgn += 2) {
              int u[3] = {t[0], t[1], t[2]};
              u[a] += sgn * k;
              if (u[a] < 0 || u[a] >= e[a]) continue;
              s += c[k] * v[((size_t)u[2] * ey + u[1]) * ex + u[0]];
            }
          }
          lap += s / (h[a] * h[a]);
        }
        out[((size_t)z * ey + y) * ex + x] = -lap;
      }
}

/* ------------------------------------------------------------------ */
/* Real spherical harmonics (Eqs. me, mepole).                          */
/* ------------------------------------------------------------------ */

/* Associated Legendre P_l^m(x), m >= 0, Condon-Shortley phase included,
 * by the textbook three-term recurrence in l. */
static double assoc_legendre(int l, int m, double x) {
  double pmm = 1.0;
  if (m > 0) {
    double s = sqrt((1.0 - x) * (1.0 + x));
    double f = 1.0;
    for (int k = 1; k <= m; ++k) {
      pmm *= -f * s;
      f += 2.0;
    }
  }
  if (l == m) return pmm;
  double pm1 = x * (2 * m + 1) * pmm;
  if (l == m + 1) return pm1;
  double pll = 0.0;
  for (int ll = m + 2; ll <= l; ++ll) {
    pll = (x * (2 * ll - 1) * pm1 - (ll + m - 1) * pmm) / (ll - m);
    pmm = pm1;
    pm1 = pll;
  }
  return pll;
}

/* Regular real solid harmonic S_lm(r) = r^l Y_lm(theta, phi), with the
 * real orthonormal Y_lm:  Y_l0 = N_l0 P_l^0,  Y_lm = sqrt2 N_lm P_l^m cos(m phi),
 * Y_l,-m = sqrt2 N_lm P_l^m sin(m phi),
 * N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).
 * For real densities the real basis gives the same potential as the
 * complex Y*_lm of Eq. mepole (addition theorem). */
double ora_solid_harmonic(int l, int m, double x, double y, double z) {
  double r = sqrt(x * x + y * y + z * z);
  int am = m < 0 ? -m : m;
  double nlm = sqrt((2.0 * l + 1.0) / (4.0 * ORA_PI) * fact(l - am) / fact(l + am));
  if (r == 0.0) return (l == 0) ? nlm : 0.0;
  double ct = z / r;
  if (ct > 1.0) ct = 1.0;
  if (ct < -1.0) ct = -1.0;
  double ph = atan2(y, x);
  double plm = assoc_legendre(l, am, ct);
  double ang;
  if (m == 0)
    ang = nlm * plm;
  else if (m > 0)
    ang = sqrt(2.0) * nlm * plm * cos(am * ph);
  else
    ang = sqrt(2.0) * nlm * plm * sin(am * ph);
  return pow(r, l) * ang;
}

/* Index of (l, m) in a packed moment array: l*l + l + m. */
static int lm_index(int l, int m) { return l * l + l + m; }

/* All S_lm(r), l <= lmax, packed by lm_index (same definitions as above,
 * angles evaluated once per point). */
void ora_solid_harmonics_all(int lmax, double x, double y, double z, double* out) {
  double r = sqrt(x * x + y * y + z * z);
  if (r == 0.0) {
    for (int l = 0; l <= lmax; ++l)
      for (int m = -l; m <= l; ++m) out[lm_index(l, m)] = 0.0;
    out[0] = sqrt(1.0 / (4.0 * ORA_PI));
    return;
  }
  double ct = z / r;
  if (ct > 1.0) ct = 1.0;
  if (ct < -1.0) ct = -1.0;
  double ph = atan2(y, x);
  for (int l = 0; l <= lmax; ++l) {
    double rl = pow(r, l);
    for (int m = -l; m <= l; ++m) {
      int am = m < 0 ? -m : m;
      double nlm = sqrt((2.0 * l + 1.0) / (4.0 * ORA_PI) * fact(l - am) / fact(l + am));
      double plm = assoc_legendre(l, am, ct);
      double ang;
      if (m == 0)
        ang = nlm * plm;
      else if (m > 0)
        ang = sqrt(2.0) * nlm * plm * cos(am * ph);
      else
        ang = sqrt(2.0) * nlm * plm * sin(am * ph);
      out[lm_index(l, m)] = rl * ang;
    }
  }
}

/* Multipole moments, Eq. mepole: Q_lm = sum_box rho S_lm(r - c) dV, about the
 * box's geometric centre (reading: the paper does not fix the centre).
 * rho is [ez][ey][ex]; point t sits at (t - (e-1)/2) h relative to the centre. */
void ora_moments(const double* rho, int ex, int ey, int ez, const double h[3],
                 double dV, int lmax, double* Q) {
  int nq = (lmax + 1) * (lmax + 1);
  double S[(ORA_LMAX_MAX + 1) * (ORA_LMAX_MAX + 1)];
  for (int q = 0; q < nq; ++q) Q[q] = 0.0;
  for (int z = 0; z < ez; ++z)
    for (int y = 0; y < ey; ++y)
      for (int x = 0; x < ex; ++x) {
        double rv = rho[((size_t)z * ey + y) * ex + x];
        double px = (x - 0.5 * (ex - 1)) * h[0];
        double py = (y - 0.5 * (ey - 1)) * h[1];
        double pz = (z - 0.5 * (ez - 1)) * h[2];
        ora_solid_harmonics_all(lmax, px, py, pz, S);
        for (int q = 0; q < nq; ++q) Q[q] += rv * S[q] * dV;
      }
}

/* Multipole expansion of the potential, Eq. me:
 *   v(r) = 4 pi sum_lm Q_lm Y_lm(r^) / ((2l+1) r^(l+1))
 *        = 4 pi sum_lm Q_lm S_lm(r) / ((2l+1) r^(2l+1)),
 * r relative to the expansion centre (must be non-zero). */
double ora_me_eval(const double* Q, int lmax, double x, double y, double z) {
  double S[(ORA_LMAX_MAX + 1) * (ORA_LMAX_MAX + 1)];
  ora_solid_harmonics_all(lmax, x, y, z, S);
  double r = sqrt(x * x + y * y + z * z);
  double v = 0.0;
  for (int l = 0; l <= lmax; ++l) {
    double rl = pow(r, 2 * l + 1);
    for (int m = -l; m <= l; ++m)
      v += Q[lm_index(l, m)] * S[lm_index(l, m)] / ((2.0 * l + 1.0) * rl);
  }
  return 4.0 * ORA_PI * v;
}

/* ------------------------------------------------------------------ */
/* Conjugate gradient for A v = b, A = -Lap_h with zero Dirichlet data */
/* (Eq. pe; the known boundary values are moved into b by the caller). */
/* ------------------------------------------------------------------ */

static double dot(const double* a, const double* b, size_t n) {
  double s = 0.0;
  for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Textbook (Hestenes-Stiefel) CG from x0 = 0.
 * tol_mode 0: stop when ||r||_2 <= tol ||b||_2.
 * tol_mode 1: stop when rms(r)/(4 pi) <= tol (residual as a density, bohr^-3).
 * Returns the iteration count, or -(count) if max_iter was reached. */
int ora_cg(const double* b, double* x, int ex, int ey, int ez, const double h[3],
           int p, double tol, int tol_mode, int max_iter, double* res_out) {
  size_t n = (size_t)ex * ey * ez;
  double* r = (double*)malloc(n * sizeof(double));
  double* pv = (double*)malloc(n * sizeof(double));
  double* q = (double*)malloc(n * sizeof(double));
  for (size_t i = 0; i < n; ++i) {
    x[i] = 0.0;
    r[i] = b[i];
    pv[i] = b[i];
  }
  double rr = dot(r, r, n);
  double bnorm = sqrt(rr);
  double target = (tol_mode == 0) ? tol * bnorm : tol * 4.0 * ORA_PI * sqrt((double)n);
  int it = 0;
  int converged = (sqrt(rr) <= target);
  while (!converged && it < max_iter) {
    ora_apply_neg_lap(pv, q, ex, ey, ez, h, p);
    double alpha = rr / dot(pv, q, n);
    for (size_t i = 0; i < n; ++i) x[i] += alpha * pv[i];
    for (size_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
    double rr_new = dot(r, r, n);
    ++it;
    if (sqrt(rr_new) <= target) {
      rr = rr_new;
      converged = 1;
      break;
    }
    double beta = rr_new / rr;
    for (size_t i = 0; i < n; ++i) pv[i] = r[i] + beta * pv[i];
    rr = rr_new;
  }
  if (res_out) *res_out = (bnorm > 0.0) ? sqrt(rr) / bnorm : 0.0;
  free(r);
  free(pv);
  free(q);
  return converged ? it : -it;
}

/* ------------------------------------------------------------------ */
/* Domain truncation, Eq. oii: one tight periodic AABB per orbital.     */
/* ------------------------------------------------------------------ */

/* Per-axis marginals of |phi|^2 dV, with exact sums.  Each square is
 * taken on the fixed-point grid 2^-64:
 *   F(v) = min(floor(v^2 2^64), 2^96)      (v^2 >= 2^32 saturates),
 * computed exactly from v's integer significand; the marginal sums of F
 * are exact integers (so their order is immaterial) and
 *   m_a(x) = fl(fl(2^-64 sum F) dV)
 * with one rounding to nearest for the sum and one for the product.  The
 * paper fixes no rounding for the marginals of Eq. oii; this reading makes
 * them independent of any summation order.  Squares below 2^-64 (|v| below
 * about 2.3e-10) count as zero, which moves a marginal by at most
 * (points in a plane) 2^-64 dV. */
typedef unsigned __int128 u128;

static u128 sq_fixed(double v) {
  if (v == 0.0 || !isfinite(v)) return 0;
  int e;
  double fr = frexp(fabs(v), &e); /* |v| = fr 2^e, fr in [0.5, 1) */
  if (e > 16) return (u128)1 << 96; /* |v| >= 2^16: v^2 >= 2^32 */
  /* |v| = m 2^(e - 53) with the integer m = fr 2^53 < 2^53 */
  unsigned long long m = (unsigned long long)ldexp(fr, 53);
  u128 mm = (u128)m * m; /* v^2 = mm 2^(2e - 106) */
  int sh = 2 * e - 106 + 64; /* F = floor(mm 2^sh) */
  if (sh >= 0) return mm << sh; /* sh <= -10 for e <= 16; kept for clarity */
  if (-sh >= 128) return 0;
  return mm >> (-sh);
}

void ora_marginals(const double* f, const int N[3], double dV, double* mx,
                   double* my, double* mz) {
  int nx = N[0], ny = N[1], nz = N[2];
  u128* sx = (u128*)calloc((size_t)nx, sizeof(u128));
  u128* sy = (u128*)calloc((size_t)ny, sizeof(u128));
  u128* sz = (u128*)calloc((size_t)nz, sizeof(u128));
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        u128 F = sq_fixed(f[((size_t)z * ny + y) * nx + x]);
        sx[x] += F;
        sy[y] += F;
        sz[z] += F;
      }
  /* (double) of an unsigned 128-bit integer rounds to nearest, ties even */
  for (int x = 0; x < nx; ++x) mx[x] = ldexp((double)sx[x], -64) * dV;
  for (int y = 0; y < ny; ++y) my[y] = ldexp((double)sy[y], -64) * dV;
  for (int z = 0; z < nz; ++z) mz[z] = ldexp((double)sz[z], -64) * dV;
  free(sx);
  free(sy);
  free(sz);
}

/* Shortest cyclic interval [s, s+len) whose complement holds at most tail
 * of the marginal's mass (ties: smaller start).  Reading of Eq. oii: the
 * paper asks for a tight AABB with in-box mass >= 1 - eps; with tail =
 * eps/3 per axis, the union bound guarantees that.  The in-interval mass is
 * accumulated from s upward; T is the ascending sum of the marginal. */
void ora_fit_interval(const double* m, int n, double tail, int* start, int* len) {
  double T = 0.0;
  for (int x = 0; x < n; ++x) T = T + m[x];
  for (int L = 1; L <= n; ++L) {
    for (int s = 0; s < n; ++s) {
      double inside = 0.0;
      for (int k = 0; k < L; ++k) inside = inside + m[(s + k) % n];
      if (T - inside <= tail) {
        *start = s;
        *len = L;
        return;
      }
    }
  }
  *start = 0;
  *len = n;
}

/* box[i*6 + 0..2] = start (x, y, z), box[i*6 + 3..5] = extent. */
void ora_boxes(const double* phi, int n_orb, const int N[3], double dV, double eps,
               int* box) {
  size_t ng = (size_t)N[0] * N[1] * N[2];
#pragma omp parallel for schedule(dynamic)
  for (int i = 0; i < n_orb; ++i) {
    double* mx = (double*)malloc(N[0] * sizeof(double));
    double* my = (double*)malloc(N[1] * sizeof(double));
    double* mz = (double*)malloc(N[2] * sizeof(double));
    ora_marginals(phi + (size_t)i * ng, N, dV, mx, my, mz);
    ora_fit_interval(mx, N[0], eps / 3.0, &box[i * 6 + 0], &box[i * 6 + 3]);
    ora_fit_interval(my, N[1], eps / 3.0, &box[i * 6 + 1], &box[i * 6 + 4]);
    ora_fit_interval(mz, N[2], eps / 3.0, &box[i * 6 + 2], &box[i * 6 + 5]);
    free(mx);
    free(my);
    free(mz);
  }
}

/* ------------------------------------------------------------------ */
/* Pair domains and pair selection (Sec. II B, Eq. sij).               */
/* ------------------------------------------------------------------ */

/* Intersection of the cyclic intervals [s1, s1+L1) (orbital i) and
 * [s2, s2+L2) (orbital j) on a ring of n points, in i's unwrapped frame.
 * Reading (the paper is silent on wrap-around): minimum image, i.e. j's
 * interval is shifted by k n, k in {-1, 0, 1}, and the shift with the
 * largest overlap is kept (first k on ties); an interval spanning the whole
 * axis leaves the other interval unchanged.  Returns 0 when empty. */
int ora_intersect(int s1, int L1, int s2, int L2, int n, int* lo, int* ext, int* kshift) {
  if (L1 >= n && L2 >= n) { *lo = s1; *ext = n; *kshift = 0; return 1; }
  if (L1 >= n) { *lo = s2; *ext = L2; *kshift = 0; return 1; }
  if (L2 >= n) { *lo = s1; *ext = L1; *kshift = 0; return 1; }
  int best = 0, bk = 0, blo = 0;
  for (int k = -1; k <= 1; ++k) {
    int a0 = s1 > s2 + k * n ? s1 : s2 + k * n;
    int a1 = (s1 + L1) < (s2 + k * n + L2) ? (s1 + L1) : (s2 + k * n + L2);
    if (a1 - a0 > best) { best = a1 - a0; bk = k; blo = a0; }
  }
  if (best <= 0) return 0;
  *lo = blo; *ext = best; *kshift = bk;
  return 1;
}

static int wrap(int x, int n) {
  int r = x % n;
  return r < 0 ? r + n : r;
}

/* S_|ij| = sum over Omega_ij of |phi_i phi_j| dV (Eq. sij).  Order: each
 * (z, y) row of the box is summed over x ascending; rows are added in
 * (z, y) ascending order; the total is multiplied by dV once. */
double ora_overlap_abs(const double* fi, const double* fj, const int N[3],
                       const int lo[3], const int ext[3], double dV) {
  double tot = 0.0;
  for (int z = 0; z < ext[2]; ++z)
    for (int y = 0; y < ext[1]; ++y) {
      double row = 0.0;
      int gz = wrap(lo[2] + z, N[2]), gy = wrap(lo[1] + y, N[1]);
      for (int x = 0; x < ext[0]; ++x) {
        int gx = wrap(lo[0] + x, N[0]);
        size_t g = ((size_t)gz * N[1] + gy) * N[0] + gx;
        row = row + fabs(fi[g] * fj[g]);
      }
      tot = tot + row;
    }
  return tot * dV;
}

/* Pair list: all i <= j with Omega_ij = Omega_ii cap Omega_jj non-empty
 * (proto-pairs) and S_|ij| >= delta; i == j is always kept.  Sorted by
 * (i, j).  Per pair: pair[2], lo[3], ext[3] (Omega_ij, i's unwrapped frame),
 * kshift[3] (shift of j's interval, in units of N), S.
 * Returns the pair count (or -count_needed if max_pairs is too small). */
int ora_pairs(const double* phi, int n_orb, const int N[3], double dV,
              const int* box, double delta, int max_pairs, int* pair, int* plo,
              int* pext, int* pk, double* S) {
  size_t ng = (size_t)N[0] * N[1] * N[2];
  int np = 0;
  for (int i = 0; i < n_orb; ++i)
    for (int j = i; j < n_orb; ++j) {
      int lo[3], ext[3], k[3], ok = 1;
      for (int a = 0; a < 3 && ok; ++a)
        ok = ora_intersect(box[i * 6 + a], box[i * 6 + 3 + a], box[j * 6 + a],
                           box[j * 6 + 3 + a], N[a], &lo[a], &ext[a], &k[a]);
      if (!ok) continue;
      double s = ora_overlap_abs(phi + (size_t)i * ng, phi + (size_t)j * ng, N, lo, ext, dV);
      if (!(i == j || s >= delta)) continue;
      if (np < max_pairs) {
        pair[np * 2] = i;
        pair[np * 2 + 1] = j;
        for (int a = 0; a < 3; ++a) {
          plo[np * 3 + a] = lo[a];
          pext[np * 3 + a] = ext[a];
          pk[np * 3 + a] = k[a];
        }
        S[np] = s;
      }
      ++np;
    }
  return np <= max_pairs ? np : -np;
}

/* ------------------------------------------------------------------ */
/* Accumulation domains (Sec. II B, text after Eq. sij).               */
/* ------------------------------------------------------------------ */

/* A window is an unwrapped interval [start, start + len) on one axis. */

/* Window of orbital o's box for a pair whose domain is [lo, lo+ext):
 * the box itself, shifted by kshift*n; a box spanning the whole axis is
 * placed as the n-point window centred on the pair domain (reading). */
static void box_window(int s, int L, int kshift, int n, int lo, int ext, int* ws,
                       int* wl) {
  if (L >= n) {
    *ws = lo - (n - ext) / 2;
    *wl = n;
  } else {
    *ws = s + kshift * n;
    *wl = L;
  }
}

/* scale_2x of an interval (reading; the paper does not define it): double
 * the extent about the interval's centre c = s + (L-1)/2, keeping the grid
 * points whose cells meet [c - L, c + L] (rounded outward): for even L this
 * is [s - L/2, s + 3L/2), for odd L [c - L, c + L]; capped at n points by the
 * n-point window centred as nearly as possible on the interval (ties low). */
void ora_scale2x(int s, int L, int n, int* ws, int* wl) {
  int lo2, len2;
  if (L % 2 == 0) {
    lo2 = s - L / 2;
    len2 = 2 * L;
  } else {
    int c = s + (L - 1) / 2;
    lo2 = c - L;
    len2 = 2 * L + 1;
  }
  if (len2 >= n) {
    lo2 = lo2 + (len2 - n) / 2;
    len2 = n;
  }
  *ws = lo2;
  *wl = len2;
}

/* ------------------------------------------------------------------ */
/* Per-pair Poisson problem (Eqs. pe, me, mepole).                      */
/* ------------------------------------------------------------------ */

typedef struct {
  double eps;      /* orbital coverage threshold, Eq. oii        */
  double delta;    /* pair screening threshold, Eq. sij          */
  double cg_tol;   /* CG stopping tolerance                      */
  int cg_tol_mode; /* 0: relative L2, 1: absolute rms / (4 pi)   */
  int cg_max_iter;
  int lmax;        /* multipole order, App. C: 6                 */
  int fd_half;     /* stencil half width p, App. C: 6 (O(h^12))  */
} ora_params;

/* Solve the pair problem on Omega_ij = [lo, lo+ext):
 *   rho = phi_i phi_j on the box (zero outside, Eq. exxGen_mlwf),
 *   Q_lm of rho about the box centre (Eq. mepole),
 *   boundary values from the ME (Eq. me) at every point outside the box
 *   that the stencil reaches (exactly one coordinate outside, by <= p),
 *   then CG for -Lap_h v = 4 pi rho with those values moved to the RHS.
 * v is [ez][ey][ex].  Returns the CG iteration count (negative: capped). */
int ora_pair_solve(const double* fi, const double* fj, const int N[3],
                   const double cell[3], const int lo[3], const int ext[3],
                   const ora_params* prm, double* v, double* Q, double* rho_v) {
  const double h[3] = {cell[0] / N[0], cell[1] / N[1], cell[2] / N[2]};
  const double dV = h[0] * h[1] * h[2];
  const int ex = ext[0], ey = ext[1], ez = ext[2];
  const size_t n = (size_t)ex * ey * ez;
  const int p = prm->fd_half;
  double c[16];
  ora_fd_coeffs(p, c);
  double* rho = (double*)malloc(n * sizeof(double));
  double* b = (double*)malloc(n * sizeof(double));
  for (int z = 0; z < ez; ++z)
    for (int y = 0; y < ey; ++y)
      for (int x = 0; x < ex; ++x) {
        size_t g = ((size_t)wrap(lo[2] + z, N[2]) * N[1] + wrap(lo[1] + y, N[1])) * N[0] +
                   wrap(lo[0] + x, N[0]);
        rho[((size_t)z * ey + y) * ex + x] = fi[g] * fj[g];
      }
  ora_moments(rho, ex, ey, ez, h, dV, prm->lmax, Q);
  /* Boundary values: the ME (Eq. me) at every point outside the box that
   * the stencil reaches (exactly one coordinate outside, by 1..p), stored
   * in a zero-padded copy of the box; then the right-hand side is 4 pi rho
   * plus the stencil's weights on those known values. */
  const int px_ = ex + 2 * p, py_ = ey + 2 * p, pz_ = ez + 2 * p;
  double* G = (double*)calloc((size_t)px_ * py_ * pz_, sizeof(double));
  for (int z = -p; z < ez + p; ++z)
    for (int y = -p; y < ey + p; ++y)
      for (int x = -p; x < ex + p; ++x) {
        int out = (x < 0 || x >= ex) + (y < 0 || y >= ey) + (z < 0 || z >= ez);
        if (out != 1) continue;
        double gx = (x - 0.5 * (ex - 1)) * h[0];
        double gy = (y - 0.5 * (ey - 1)) * h[1];
        double gz = (z - 0.5 * (ez - 1)) * h[2];
        G[((size_t)(z + p) * py_ + (y + p)) * px_ + (x + p)] = ora_me_eval(Q, prm->lmax, gx, gy, gz);
      }
  const int e[3] = {ex, ey, ez};
  for (int z = 0; z < ez; ++z)
    for (int y = 0; y < ey; ++y)
      for (int x = 0; x < ex; ++x) {
        const int t[3] = {x, y, z};
        double rhs = 4.0 * ORA_PI * rho[((size_t)z * ey + y) * ex + x];
        for (int a = 0; a < 3; ++a)
          for (int k = 1; k <= p; ++k)
            for (int sgn = -1; sgn <= 1; sgn += 2) {
              int u[3] = {t[0], t[1], t[2]};
              u[a] += sgn * k;
              if (u[a] >= 0 && u[a] < e[a]) continue;
              double g = G[((size_t)(u[2] + p) * py_ + (u[1] + p)) * px_ + (u[0] + p)];
              rhs += c[k] / (h[a] * h[a]) * g;
            }
        b[((size_t)z * ey + y) * ex + x] = rhs;
      }
  free(G);
  double res = 0.0;
  int it = ora_cg(b, v, ex, ey, ez, h, p, prm->cg_tol, prm->cg_tol_mode, prm->cg_max_iter, &res);
  /* Pair energy integral of Eq. exxGen_mlwf: sum rho v dV over Omega_ij. */
  double e_pair = 0.0;
  for (size_t q = 0; q < n; ++q) e_pair += rho[q] * v[q];
  *rho_v = e_pair * dV;
  free(rho);
  free(b);
  return it;
}

/* v_ij at an unwrapped grid point u (grid units): the CG solution inside
 * Omega_ij, the multipole expansion (Eq. me) outside it (Eq. tDxx). */
static double pair_potential(const double* v, const double* Q, int lmax, const int lo[3],
                             const int ext[3], const double h[3], const int u[3]) {
  int t0 = u[0] - lo[0], t1 = u[1] - lo[1], t2 = u[2] - lo[2];
  if (t0 >= 0 && t0 < ext[0] && t1 >= 0 && t1 < ext[1] && t2 >= 0 && t2 < ext[2])
    return v[((size_t)t2 * ext[1] + t1) * ext[0] + t0];
  double px = (t0 - 0.5 * (ext[0] - 1)) * h[0];
  double py = (t1 - 0.5 * (ext[1] - 1)) * h[1];
  double pz = (t2 - 0.5 * (ext[2] - 1)) * h[2];
  return ora_me_eval(Q, lmax, px, py, pz);
}

/* ------------------------------------------------------------------ */
/* Whole application: boxes, pairs, per-pair PE, D_xx and E_xx.        */
/* ------------------------------------------------------------------ */

/* V_xx phi_i = -D^i (Eq. DxxVxx) with D^i from Eq. tDxx:
 *   D^i += v_ij phi_j on Omega^D_ij, Omega^D_ij = Omega_jj (j != i),
 *   Omega^D_ii = scale_2x Omega_ii; for j != i also D^j += v_ij phi_i on
 *   Omega_ii (v_ji = v_ij).  phi is the full orbital (reading).
 *   E_xx = -sum_{i<=j} (2 - delta_ij) sum_{Omega_ij} rho v dV (Eq. exxGen_mlwf
 *   over ordered pairs, each unordered pair counted twice).
 * Outputs: vxx[n][nz][ny][nx], *exx.  Optional diagnostics (may be NULL):
 * box[n*6], and, sized by max_pairs, pair[2P], plo[3P], pext[3P], pk[3P],
 * S[P], iters[P], epair[P], Q[P*(lmax+1)^2].  *n_pairs receives the count.
 * Returns 0 on success, 1 if max_pairs is too small, 2 if a CG hit its cap. */
int ora_apply_vxx(const double* phi, int n_orb, const int N[3], const double cell[3],
                  const ora_params* prm, double* vxx, double* exx, int* box_out,
                  int max_pairs, int* n_pairs, int* pair_out, int* plo_out,
                  int* pext_out, int* pk_out, double* S_out, int* iters_out,
                  double* epair_out, double* Q_out) {
  const size_t ng = (size_t)N[0] * N[1] * N[2];
  const double h[3] = {cell[0] / N[0], cell[1] / N[1], cell[2] / N[2]};
  const double dV = h[0] * h[1] * h[2];
  const int nq = (prm->lmax + 1) * (prm->lmax + 1);
  int* box = (int*)malloc((size_t)n_orb * 6 * sizeof(int));
  ora_boxes(phi, n_orb, N, dV, prm->eps, box);
  if (box_out) memcpy(box_out, box, (size_t)n_orb * 6 * sizeof(int));

  int cap = n_orb * n_orb;
  int* pair = (int*)malloc((size_t)cap * 2 * sizeof(int));
  int* plo = (int*)malloc((size_t)cap * 3 * sizeof(int));
  int* pext = (int*)malloc((size_t)cap * 3 * sizeof(int));
  int* pk = (int*)malloc((size_t)cap * 3 * sizeof(int));
  double* S = (double*)malloc((size_t)cap * sizeof(double));
  int np = ora_pairs(phi, n_orb, N, dV, box, prm->delta, cap, pair, plo, pext, pk, S);
  if (n_pairs) *n_pairs = np;

  double** vp = (double**)calloc((size_t)np, sizeof(double*));
  double* Q = (double*)malloc((size_t)np * nq * sizeof(double));
  double* ep = (double*)malloc((size_t)np * sizeof(double));
  int* its = (int*)malloc((size_t)np * sizeof(int));
  int capped = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : capped)
  for (int q = 0; q < np; ++q) {
    const int* lo = plo + q * 3;
    const int* ext = pext + q * 3;
    vp[q] = (double*)malloc((size_t)ext[0] * ext[1] * ext[2] * sizeof(double));
    its[q] = ora_pair_solve(phi + (size_t)pair[q * 2] * ng, phi + (size_t)pair[q * 2 + 1] * ng,
                            N, cell, lo, ext, prm, vp[q], Q + (size_t)q * nq, &ep[q]);
    if (its[q] < 0) capped = 1;
  }

  /* E_xx: fixed pair order. */
  double e = 0.0;
  for (int q = 0; q < np; ++q)
    e += (pair[q * 2] == pair[q * 2 + 1] ? 1.0 : 2.0) * ep[q];
  *exx = -e;

  /* D^o for every orbital o: its pairs in pair order, D^i before D^j. */
  double* D = vxx; /* accumulate D, negate at the end */
#pragma omp parallel for schedule(dynamic)
  for (int o = 0; o < n_orb; ++o) {
    double* Do = D + (size_t)o * ng;
    for (size_t g = 0; g < ng; ++g) Do[g] = 0.0;
    for (int q = 0; q < np; ++q) {
      int i = pair[q * 2], j = pair[q * 2 + 1];
      if (i != o && j != o) continue;
      const int* lo = plo + q * 3;
      const int* ext = pext + q * 3;
      const int* k = pk + q * 3;
      for (int role = 0; role < 2; ++role) {
        /* role 0: D^i += v phi_j ; role 1: D^j += v phi_i (j != i). */
        if (role == 0 && i != o) continue;
        if (role == 1 && (j != o || i == j)) continue;
        int ws[3], wl[3];
        const double* partner;
        for (int a = 0; a < 3; ++a) {
          if (role == 0 && i == j) {
            int s0, l0;
            box_window(box[i * 6 + a], box[i * 6 + 3 + a], 0, N[a], lo[a], ext[a], &s0, &l0);
            ora_scale2x(s0, l0, N[a], &ws[a], &wl[a]);
          } else if (role == 0) {
            box_window(box[j * 6 + a], box[j * 6 + 3 + a], k[a], N[a], lo[a], ext[a], &ws[a], &wl[a]);
          } else {
            box_window(box[i * 6 + a], box[i * 6 + 3 + a], 0, N[a], lo[a], ext[a], &ws[a], &wl[a]);
          }
        }
        partner = phi + (size_t)(role == 0 ? j : i) * ng;
        for (int z = 0; z < wl[2]; ++z)
          for (int y = 0; y < wl[1]; ++y)
            for (int x = 0; x < wl[0]; ++x) {
              int u[3] = {ws[0] + x, ws[1] + y, ws[2] + z};
              size_t g = ((size_t)wrap(u[2], N[2]) * N[1] + wrap(u[1], N[1])) * N[0] +
                         wrap(u[0], N[0]);
              double vv = pair_potential(vp[q], Q + (size_t)q * nq, prm->lmax, lo, ext, h, u);
              Do[g] += vv * partner[g];
            }
      }
    }
    for (size_t g = 0; g < ng; ++g) Do[g] = -Do[g];
  }

  if (pair_out) {
    int m = np < max_pairs ? np : max_pairs;
    memcpy(pair_out, pair, (size_t)m * 2 * sizeof(int));
    if (plo_out) memcpy(plo_out, plo, (size_t)m * 3 * sizeof(int));
    if (pext_out) memcpy(pext_out, pext, (size_t)m * 3 * sizeof(int));
    if (pk_out) memcpy(pk_out, pk, (size_t)m * 3 * sizeof(int));
    if (S_out) memcpy(S_out, S, (size_t)m * sizeof(double));
    if (iters_out) memcpy(iters_out, its, (size_t)m * sizeof(int));
    if (epair_out) memcpy(epair_out, ep, (size_t)m * sizeof(double));
    if (Q_out) memcpy(Q_out, Q, (size_t)m * nq * sizeof(double));
  }
  for (int q = 0; q < np; ++q) free(vp[q]);
  free(vp);
  free(Q);
  free(ep);
  free(its);
  free(pair);
  free(plo);
  free(pext);
  free(pk);
  free(S);
  free(box);
  if (max_pairs < np) return 1;
  return capped ? 2 : 0;
}

/* Per-pair potential on an arbitrary list of unwrapped points (for tests
 * that sample v_ij at full size): CG solution inside, ME outside. */
void ora_pair_potential_at(const double* v, const double* Q, int lmax, const int lo[3],
                           const int ext[3], const double h[3], int npts, const int* u,
                           double* out) {
  for (int t = 0; t < npts; ++t) out[t] = pair_potential(v, Q, lmax, lo, ext, h, u + 3 * t);
}

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
