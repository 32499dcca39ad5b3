/*
 * ader_oracle.c -- plain FP64 CPU oracle of the 1D ADER-DG and ADER-WENO
 * finite-volume schemes of Popov, arXiv 2409.12483 (Euler equations, S = B = 0).
 *
 * TEST INFRASTRUCTURE ONLY (see ader_oracle.h): used by the tests, the smoke
 * check and the CPU-baseline leg of the benchmark, never by the product path.
 *
 * Construction choices that keep it independent of the CUDA library:
 *  - nodes by Newton on the Legendre polynomial P_{N+1} (Bonnet recurrence)
 *    in long double;
 *  - every integral of basis functions is done exactly on monomial
 *    expansions of the Lagrange polynomials (long double), not by quadrature;
 *  - operators are the definitions written out (Gauss-Jordan inverses);
 *  - the Picard loop, the traces, the Riemann solver and the updates follow
 *    the sums of the paper in their stated order, one cell at a time.
 */
#include "ader_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef long double ld;

#define NMAX OB_MAXN
#define PMAX (2 * OB_MAXN + 2)

/* ------------------------------------------------------------------------ */
/* monomial polynomial helpers, coefficient c[j] of x^j                      */
/* ------------------------------------------------------------------------ */

static ld poly_eval(const ld* c, int len, ld x) {
  ld s = 0;
  for (int j = len - 1; j >= 0; --j) s = s * x + c[j];
  return s;
}

/* derivative: out has len-1 coefficients (len >= 1; len == 1 gives zero poly of len 1) */
static int poly_deriv(const ld* c, int len, ld* out) {
  if (len <= 1) {
    out[0] = 0;
    return 1;
  }
  for (int j = 1; j < len; ++j) out[j - 1] = (ld)j * c[j];
  return len - 1;
}

/* integral over [lo, hi] of a polynomial */
static ld poly_integral(const ld* c, int len, ld lo, ld hi) {
  ld s_hi = 0, s_lo = 0;
  for (int j = len - 1; j >= 0; --j) {
    s_hi = s_hi * hi + c[j] / (ld)(j + 1);
    s_lo = s_lo * lo + c[j] / (ld)(j + 1);
  }
  return s_hi * hi - s_lo * lo;
}

/* integral over [lo, hi] of the product a*b */
static ld poly_integral_prod(const ld* a, int la, const ld* b, int lb, ld lo, ld hi) {
  ld prod[2 * PMAX];
  int lp = la + lb - 1;
  for (int j = 0; j < lp; ++j) prod[j] = 0;
  for (int i = 0; i < la; ++i)
    for (int j = 0; j < lb; ++j) prod[i + j] += a[i] * b[j];
  return poly_integral(prod, lp, lo, hi);
}

/* Lagrange polynomial phi_k on the nodes x[0..n-1], as monomial coefficients (n of them) */
static void lagrange_coeffs(const ld* x, int n, int k, ld* c) {
  for (int j = 0; j < n; ++j) c[j] = 0;
  c[0] = 1;
  int len = 1;
  for (int m = 0; m < n; ++m) {
    if (m == k) continue;
    ld inv = 1.0L / (x[k] - x[m]);
    /* multiply by (X - x[m]) * inv */
    ld next[NMAX + 1];
    for (int j = 0; j <= len; ++j) next[j] = 0;
    for (int j = 0; j < len; ++j) {
      next[j + 1] += c[j] * inv;
      next[j] -= c[j] * x[m] * inv;
    }
    len += 1;
    for (int j = 0; j < len; ++j) c[j] = next[j];
  }
}

/* Gauss-Jordan inverse with partial pivoting; returns 0 on success */
static int gj_inverse(int n, ld A[NMAX][NMAX], ld Ainv[NMAX][NMAX]) {
  ld M[NMAX][2 * NMAX];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) M[i][j] = (j < n) ? A[i][j] : (ld)((j - n) == i);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int i = col + 1; i < n; ++i)
      if (fabsl(M[i][col]) > fabsl(M[piv][col])) piv = i;
    if (M[piv][col] == 0) return -1;
    if (piv != col)
      for (int j = 0; j < 2 * n; ++j) {
        ld t = M[col][j];
        M[col][j] = M[piv][j];
        M[piv][j] = t;
      }
    ld d = M[col][col];
    for (int j = 0; j < 2 * n; ++j) M[col][j] /= d;
    for (int i = 0; i < n; ++i) {
      if (i == col) continue;
      ld f = M[i][col];
      if (f == 0) continue;
      for (int j = 0; j < 2 * n; ++j) M[i][j] -= f * M[col][j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i][j] = M[i][n + j];
  return 0;
}

/* Legendre P_n(x) and P_n'(x), Bonnet recurrence */
static void legendre(int n, ld x, ld* p, ld* dp) {
  ld p0 = 1, p1 = x;
  if (n == 0) {
    *p = 1;
    *dp = 0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    ld p2 = ((ld)(2 * k - 1) * x * p1 - (ld)(k - 1) * p0) / (ld)k;
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = (ld)n * (x * p1 - p0) / (x * x - 1);
}

/* Gauss-Legendre nodes/weights mapped to [0,1], ascending */
static void gauss_legendre01(int n, ld* xi, ld* w) {
  const ld pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < n; ++k) {
    ld x = cosl(pi * ((ld)k + 0.75L) / ((ld)n + 0.5L));
    ld p, dp;
    for (int it = 0; it < 200; ++it) {
      legendre(n, x, &p, &dp);
      ld dx = p / dp;
      x -= dx;
      if (fabsl(dx) <= 4 * LDBL_EPSILON) break;
    }
    legendre(n, x, &p, &dp);
    ld W = 2.0L / ((1 - x * x) * dp * dp);
    /* x descends with k: store ascending in xi */
    xi[n - 1 - k] = (1 + x) / 2;
    w[n - 1 - k] = W / 2;
  }
}

/* ------------------------------------------------------------------------ */
/* basis and operators (Sec. 1.1: eq. gl_rule, eq. m_and_kappa_matrices,     */
/* the Kronecker forms, Dphi; Sec. 1.4: subcell projection P)                 */
/* ------------------------------------------------------------------------ */

int ob_basis_build(int N, ob_basis* b) {
  if (!b || N < 0 || N > OB_MAXDEG) return OB_ERR_ARG;
  memset(b, 0, sizeof(*b));
  const int n = N + 1;
  b->N = N;
  b->n = n;
  b->Ns = 2 * N + 1;

  ld xi[NMAX], wq[NMAX], tn[NMAX];
  gauss_legendre01(n, xi, wq);
  /* Polynomials are expanded in the centred variable t = 2 xi - 1 (monomials on
   * [-1, 1] are far better conditioned than on [0, 1]); d/dxi = 2 d/dt and
   * int_a^b d xi = (1/2) int_{2a-1}^{2b-1} dt. */
  for (int k = 0; k < n; ++k) tn[k] = 2 * xi[k] - 1;

  ld c[NMAX][NMAX + 1];  /* phi_k coefficients in t */
  ld dc[NMAX][NMAX + 1]; /* d phi_k / d xi coefficients in t */
  int dlen[NMAX];
  for (int k = 0; k < n; ++k) {
    lagrange_coeffs(tn, n, k, c[k]);
    dlen[k] = poly_deriv(c[k], n, dc[k]);
    for (int j = 0; j < dlen[k]; ++j) dc[k][j] *= 2;
  }

  ld lam[NMAX][NMAX], xim[NMAX][NMAX], ups[NMAX][NMAX], tmp[NMAX][NMAX];
  for (int k = 0; k < n; ++k) {
    b->xi[k] = (double)xi[k];
    b->w[k] = (double)wq[k];
    b->psi0[k] = (double)poly_eval(c[k], n, -1.0L);
    b->psi1[k] = (double)poly_eval(c[k], n, 1.0L);
    for (int l = 0; l < n; ++l) {
      b->dphi[k][l] = (double)poly_eval(dc[k], dlen[k], tn[l]);
      lam[k][l] = 0.5L * poly_integral_prod(c[k], n, c[l], n, -1.0L, 1.0L);
      xim[k][l] = 0.5L * poly_integral_prod(c[k], n, dc[l], dlen[l], -1.0L, 1.0L);
    }
  }
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l)
      ups[k][l] = poly_eval(c[k], n, 1.0L) * poly_eval(c[l], n, 1.0L) - xim[l][k];

  /* kappa~ = Upsilon^-1 Lambda */
  ld inv[NMAX][NMAX];
  if (gj_inverse(n, ups, inv)) return OB_ERR_ARG;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      ld s = 0;
      for (int m = 0; m < n; ++m) s += inv[i][m] * lam[m][j];
      b->kap[i][j] = (double)s;
    }
  /* k~ = Lambda^-1 Xi */
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) tmp[i][j] = lam[i][j];
  if (gj_inverse(n, tmp, inv)) return OB_ERR_ARG;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      ld s = 0;
      for (int m = 0; m < n; ++m) s += inv[i][m] * xim[m][j];
      b->kt[i][j] = (double)s;
    }
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) {
      b->lam[k][l] = (double)lam[k][l];
      b->xi_m[k][l] = (double)xim[k][l];
      b->ups[k][l] = (double)ups[k][l];
      /* D~_kl = w_l Dphi_kl */
      b->dt_m[k][l] = (double)(wq[l] * poly_eval(dc[k], dlen[k], tn[l]));
    }
  /* P_jk = Ns * int_{j/Ns}^{(j+1)/Ns} phi_k d xi */
  for (int j = 0; j < b->Ns; ++j)
    for (int k = 0; k < n; ++k) {
      const ld a = 2.0L * (ld)j / (ld)b->Ns - 1, e = 2.0L * (ld)(j + 1) / (ld)b->Ns - 1;
      b->P[j][k] = (double)((ld)b->Ns * 0.5L * poly_integral(c[k], n, a, e));
    }
  return OB_OK;
}

void ob_basis_eval(const ob_basis* b, double x, double* phi_out) {
  /* direct product form of the Lagrange polynomials */
  for (int k = 0; k < b->n; ++k) {
    double v = 1.0;
    for (int m = 0; m < b->n; ++m)
      if (m != k) v *= (x - b->xi[m]) / (b->xi[k] - b->xi[m]);
    phi_out[k] = v;
  }
}

/* ------------------------------------------------------------------------ */
/* Euler equations (Sec. 2, eq. system_of_equations) in 1D, and the Riemann  */
/* solver (Rusanov / local Lax-Friedrichs; the paper leaves it unnamed)      */
/* ------------------------------------------------------------------------ */

void ob_euler_flux(double gamma, const double* U, double* F) {
  const double rho = U[0], m = U[1], E = U[2];
  const double u = m / rho;
  const double p = (gamma - 1.0) * (E - 0.5 * m * u);
  F[0] = m;
  F[1] = m * u + p;
  F[2] = (E + p) * u;
}

double ob_wave_speed(double gamma, const double* U) {
  const double rho = U[0], m = U[1], E = U[2];
  const double u = m / rho;
  const double p = (gamma - 1.0) * (E - 0.5 * m * u);
  if (!(rho > 0.0) || !(p > 0.0)) return NAN;
  return fabs(u) + sqrt(gamma * p / rho);
}

void ob_rusanov(double gamma, const double* a, const double* b, double* G) {
  double Fa[OB_M], Fb[OB_M];
  ob_euler_flux(gamma, a, Fa);
  ob_euler_flux(gamma, b, Fb);
  const double sa = ob_wave_speed(gamma, a), sb = ob_wave_speed(gamma, b);
  /* a non-physical state on either side (NaN speed) makes the flux NaN, so the
   * candidate fails the admissibility check instead of taking one side's speed */
  const double s = (isnan(sa) || isnan(sb)) ? NAN : (sa > sb ? sa : sb);
  for (int r = 0; r < OB_M; ++r) G[r] = 0.5 * (Fa[r] + Fb[r]) - 0.5 * s * (b[r] - a[r]);
}

/* ------------------------------------------------------------------------ */
/* LST-DG predictor (eq. lst_dg_predictor_picard with S = B = 0; eq. ind_prop) */
/* ------------------------------------------------------------------------ */

#define QIDX(p0, p1, r) ((((p0) * n) + (p1)) * OB_M + (r))

int ob_predict_cell(const ob_basis* b, const ob_params* p, double lam, const double* u, double* q,
                    int* iters) {
  const int n = b->n;
  double f[NMAX * NMAX * OB_M], s[NMAX * NMAX * OB_M], qn[NMAX * NMAX * OB_M];
  /* initial iterate: q_{p0,p1} = u_{p1} for every time node (L0 = delta) */
  for (int p0 = 0; p0 < n; ++p0)
    for (int p1 = 0; p1 < n; ++p1)
      for (int r = 0; r < OB_M; ++r) q[QIDX(p0, p1, r)] = u[p1 * OB_M + r];
  const int cap = p->fixed_iter > 0 ? p->fixed_iter : p->max_iter;
  int it = 0, converged = 0;
  while (it < cap) {
    ++it;
    /* rescaled point-wise flux f = (dt/dx) F(q) at every space-time node */
    for (int p0 = 0; p0 < n; ++p0)
      for (int p1 = 0; p1 < n; ++p1) {
        double F[OB_M];
        ob_euler_flux(p->gamma, &q[QIDX(p0, p1, 0)], F);
        for (int r = 0; r < OB_M; ++r) f[QIDX(p0, p1, r)] = lam * F[r];
      }
    /* k~ along xi:  s_{p0,p1} = sum_q1 k~_{p1 q1} f_{p0,q1} */
    for (int p0 = 0; p0 < n; ++p0)
      for (int p1 = 0; p1 < n; ++p1)
        for (int r = 0; r < OB_M; ++r) {
          double acc = 0.0;
          for (int q1 = 0; q1 < n; ++q1) acc += b->kt[p1][q1] * f[QIDX(p0, q1, r)];
          s[QIDX(p0, p1, r)] = acc;
        }
    /* kappa~ along tau:  q'_{p0,p1} = u_{p1} - sum_q0 kappa~_{p0 q0} s_{q0,p1} */
    for (int p0 = 0; p0 < n; ++p0)
      for (int p1 = 0; p1 < n; ++p1)
        for (int r = 0; r < OB_M; ++r) {
          double acc = 0.0;
          for (int q0 = 0; q0 < n; ++q0) acc += b->kap[p0][q0] * s[QIDX(q0, p1, r)];
          qn[QIDX(p0, p1, r)] = u[p1 * OB_M + r] - acc;
        }
    double delta = 0.0, qmax = 0.0;
    for (int i = 0; i < n * n * OB_M; ++i) {
      const double d = fabs(qn[i] - q[i]);
      if (d > delta) delta = d;
      if (fabs(qn[i]) > qmax) qmax = fabs(qn[i]);
      q[i] = qn[i];
    }
    if (p->fixed_iter <= 0 && delta <= p->tol * (qmax > 1.0 ? qmax : 1.0)) {
      converged = 1;
      break;
    }
  }
  if (p->fixed_iter > 0) converged = 1;
  if (iters) *iters = it;
  return converged ? OB_OK : OB_ERR_NOT_CONVERGED;
}

/* The nested outer/inner form of Algorithm lst_dg_predictor, written with its
 * own arrays (q_init, q_prev, q_next, kf_sum, q_int_prev, q_int_next, s, b).
 * With s = b = 0 the inner loop reaches its fixed point after one pass and
 * confirms it on the second. */
int ob_predict_cell_nested(const ob_basis* b, const ob_params* p, double lam, const double* u,
                           double* q, int* iters) {
  const int n = b->n, sz = n * n * OB_M;
  double q_init[NMAX * NMAX * OB_M], q_prev[NMAX * NMAX * OB_M], q_next[NMAX * NMAX * OB_M];
  double kf_sum[NMAX * NMAX * OB_M], q_int_prev[NMAX * NMAX * OB_M], q_int_next[NMAX * NMAX * OB_M];
  double s_arr[NMAX * NMAX * OB_M], b_arr[NMAX * NMAX * OB_M], f_ksi[NMAX * NMAX * OB_M];
  for (int p0 = 0; p0 < n; ++p0)
    for (int i = 0; i < n * OB_M; ++i) q_init[p0 * n * OB_M + i] = u[i];
  memcpy(q_prev, q_init, sizeof(double) * sz);
  int outer = 0;
  const int cap = p->fixed_iter > 0 ? p->fixed_iter : p->max_iter;
  int converged = 0;
  while (outer < cap) {
    ++outer;
    memcpy(q_next, q_init, sizeof(double) * sz);
    /* set_flux_terms_sum: flux at nodes, then k~ along xi */
    for (int p0 = 0; p0 < n; ++p0)
      for (int p1 = 0; p1 < n; ++p1) {
        double F[OB_M];
        ob_euler_flux(p->gamma, &q_prev[QIDX(p0, p1, 0)], F);
        for (int r = 0; r < OB_M; ++r) f_ksi[QIDX(p0, p1, r)] = lam * F[r];
      }
    for (int p0 = 0; p0 < n; ++p0)
      for (int p1 = 0; p1 < n; ++p1)
        for (int r = 0; r < OB_M; ++r) {
          double acc = 0.0;
          for (int q1 = 0; q1 < n; ++q1) acc += b->kt[p1][q1] * f_ksi[QIDX(p0, q1, r)];
          kf_sum[QIDX(p0, p1, r)] = acc;
        }
    memcpy(q_int_prev, q_prev, sizeof(double) * sz);
    for (int inner = 0; inner < cap; ++inner) {
      memcpy(q_int_next, q_init, sizeof(double) * sz);
      for (int i = 0; i < sz; ++i) {
        s_arr[i] = 0.0; /* rescaled source: zero for the Euler equations */
        b_arr[i] = 0.0; /* non-conservative products: zero */
      }
      for (int i = 0; i < sz; ++i) s_arr[i] = s_arr[i] - b_arr[i] - kf_sum[i];
      /* kappa_kernel: q_int_next += kappa~ s along tau */
      for (int p1 = 0; p1 < n; ++p1)
        for (int p0 = 0; p0 < n; ++p0)
          for (int r = 0; r < OB_M; ++r) {
            double acc = 0.0;
            for (int q0 = 0; q0 < n; ++q0) acc += b->kap[p0][q0] * s_arr[QIDX(q0, p1, r)];
            q_int_next[QIDX(p0, p1, r)] += acc;
          }
      double e_in = 0.0;
      for (int i = 0; i < sz; ++i) {
        const double d = fabs(q_int_next[i] - q_int_prev[i]);
        if (d > e_in) e_in = d;
      }
      memcpy(q_int_prev, q_int_next, sizeof(double) * sz);
      if (e_in <= p->tol) break;
    }
    memcpy(q_next, q_int_next, sizeof(double) * sz);
    double e_out = 0.0, qmax = 0.0;
    for (int i = 0; i < sz; ++i) {
      const double d = fabs(q_next[i] - q_prev[i]);
      if (d > e_out) e_out = d;
      if (fabs(q_next[i]) > qmax) qmax = fabs(q_next[i]);
    }
    memcpy(q_prev, q_next, sizeof(double) * sz);
    if (p->fixed_iter <= 0 && e_out <= p->tol * (qmax > 1.0 ? qmax : 1.0)) {
      converged = 1;
      break;
    }
  }
  if (p->fixed_iter > 0) converged = 1;
  memcpy(q, q_next, sizeof(double) * sz);
  if (iters) *iters = outer;
  return converged ? OB_OK : OB_ERR_NOT_CONVERGED;
}

/* ------------------------------------------------------------------------ */
/* time step constraint (Sec. 1.5); lambda over the subcell averages of     */
/* Sec. 1.4 for DG and over the cell averages for FV                        */
/* ------------------------------------------------------------------------ */

double ob_dg_lambda_max(const ob_basis* b, double gamma, int64_t ncells, const double* u) {
  const int n = b->n;
  double lmax = 0.0;
  for (int64_t i = 0; i < ncells; ++i) {
    const double* ui = u + i * n * OB_M;
    for (int j = 0; j < b->Ns; ++j) {
      double v[OB_M];
      for (int r = 0; r < OB_M; ++r) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc += b->P[j][k] * ui[k * OB_M + r];
        v[r] = acc;
      }
      const double s = ob_wave_speed(gamma, v);
      if (isnan(s)) return NAN;
      if (s > lmax) lmax = s;
    }
  }
  return lmax;
}

/* The paper gives the subcell averages as one way to obtain lambda (Sec. 1.5);
   the nodal values of the DG polynomial are the other representation at hand. */
double ob_dg_lambda_max_nodal(const ob_basis* b, double gamma, int64_t ncells, const double* u) {
  double lmax = 0.0;
  for (int64_t i = 0; i < ncells * b->n; ++i) {
    const double s = ob_wave_speed(gamma, u + i * OB_M);
    if (isnan(s)) return NAN;
    if (s > lmax) lmax = s;
  }
  return lmax;
}

double ob_fv_lambda_max(double gamma, int64_t ncells, const double* v) {
  double lmax = 0.0;
  for (int64_t i = 0; i < ncells; ++i) {
    const double s = ob_wave_speed(gamma, v + i * OB_M);
    if (isnan(s)) return NAN;
    if (s > lmax) lmax = s;
  }
  return lmax;
}

double ob_dg_dt(const ob_basis* b, const ob_params* p, double dx, int64_t ncells, const double* u) {
  const double lmax = p->cfl_mode == 1 ? ob_dg_lambda_max_nodal(b, p->gamma, ncells, u)
                                       : ob_dg_lambda_max(b, p->gamma, ncells, u);
  /* d = 1 spatial dimension */
  return p->cfl / (double)(2 * b->N + 1) * dx / lmax;
}

double ob_fv_dt(const ob_params* p, double dx, int64_t ncells, const double* v) {
  const double lmax = ob_fv_lambda_max(p->gamma, ncells, v);
  return p->cfl * dx / lmax;
}

/* ------------------------------------------------------------------------ */
/* corrector pieces (eq. ader_dg_method_full and eq. ader_weno_fv_method_full */
/* reduced to 1D)                                                             */
/* ------------------------------------------------------------------------ */

static int64_t wrap(int64_t i, int64_t n) {
  i %= n;
  return i < 0 ? i + n : i;
}

/* traces at xi = 1 (qR) and xi = 0 (qL) for every time node */
static void cell_traces(const ob_basis* b, const double* q, double* qR, double* qL) {
  const int n = b->n;
  for (int l0 = 0; l0 < n; ++l0)
    for (int r = 0; r < OB_M; ++r) {
      double aR = 0.0, aL = 0.0;
      for (int p1 = 0; p1 < n; ++p1) {
        aR += b->psi1[p1] * q[QIDX(l0, p1, r)];
        aL += b->psi0[p1] * q[QIDX(l0, p1, r)];
      }
      qR[l0 * OB_M + r] = aR;
      qL[l0 * OB_M + r] = aL;
    }
}

/* time-integrated rescaled Riemann flux through one face:
 * G = sum_l0 w_l0 (dt/dx) Rusanov(qR of the left cell, qL of the right cell) at tau_l0 */
static void face_flux(const ob_basis* b, const ob_params* p, double lam, const double* qR_left,
                      const double* qL_right, double* G) {
  for (int r = 0; r < OB_M; ++r) G[r] = 0.0;
  for (int l0 = 0; l0 < b->n; ++l0) {
    double g[OB_M];
    ob_rusanov(p->gamma, qR_left + l0 * OB_M, qL_right + l0 * OB_M, g);
    for (int r = 0; r < OB_M; ++r) G[r] += b->w[l0] * (lam * g[r]);
  }
}

/* get_dg_solution for one cell: u_next = u_prev + volume terms + interface terms */
static void dg_cell_update(const ob_basis* b, const ob_params* p, double lam, const double* u,
                           const double* q, const double* G_left, const double* G_right,
                           double* u_next) {
  const int n = b->n;
  for (int i = 0; i < n * OB_M; ++i) u_next[i] = u[i];
  /* volume terms: time average of the rescaled flux (w-conv), then D~, then / w_k */
  double fbar[NMAX * OB_M];
  for (int l = 0; l < n; ++l)
    for (int r = 0; r < OB_M; ++r) fbar[l * OB_M + r] = 0.0;
  for (int l0 = 0; l0 < n; ++l0)
    for (int l = 0; l < n; ++l) {
      double F[OB_M];
      ob_euler_flux(p->gamma, &q[QIDX(l0, l, 0)], F);
      for (int r = 0; r < OB_M; ++r) fbar[l * OB_M + r] += b->w[l0] * (lam * F[r]);
    }
  for (int k = 0; k < n; ++k)
    for (int r = 0; r < OB_M; ++r) {
      double acc = 0.0;
      for (int l = 0; l < n; ++l) acc += b->dt_m[k][l] * fbar[l * OB_M + r];
      u_next[k * OB_M + r] += acc / b->w[k];
    }
  /* interface terms: -(psi~_k G_{i+1/2} - psi_k G_{i-1/2}) / w_k */
  for (int k = 0; k < n; ++k)
    for (int r = 0; r < OB_M; ++r)
      u_next[k * OB_M + r] += -(b->psi1[k] * G_right[r] - b->psi0[k] * G_left[r]) / b->w[k];
}

int ob_dg_correct(const ob_basis* b, const ob_params* p, int64_t ncells, double dx, double dt,
                  const double* u, const double* q, double* u_new) {
  if (ncells <= 0) return OB_ERR_ARG;
  const int n = b->n;
  const double lam = dt / dx;
  const int64_t qs = (int64_t)n * n * OB_M, us = (int64_t)n * OB_M;
  double* qR = malloc(sizeof(double) * ncells * n * OB_M);
  double* qL = malloc(sizeof(double) * ncells * n * OB_M);
  double* G = malloc(sizeof(double) * ncells * OB_M); /* G[i] = face i+1/2 */
  if (!qR || !qL || !G) {
    free(qR);
    free(qL);
    free(G);
    return OB_ERR_ARG;
  }
  for (int64_t i = 0; i < ncells; ++i) cell_traces(b, q + i * qs, qR + i * us, qL + i * us);
  for (int64_t i = 0; i < ncells; ++i)
    face_flux(b, p, lam, qR + i * us, qL + wrap(i + 1, ncells) * us, G + i * OB_M);
  for (int64_t i = 0; i < ncells; ++i)
    dg_cell_update(b, p, lam, u + i * us, q + i * qs, G + wrap(i - 1, ncells) * OB_M,
                   G + i * OB_M, u_new + i * us);
  free(qR);
  free(qL);
  free(G);
  return OB_OK;
}

static void stats_add(ob_stats* st, int it) {
  if (!st) return;
  if (st->cells == 0 || it > st->max_iters) st->max_iters = it;
  if (st->cells == 0 || it < st->min_iters) st->min_iters = it;
  st->mean_iters = (st->mean_iters * (double)st->cells + it) / (double)(st->cells + 1);
  st->cells += 1;
}

int ob_dg_step(const ob_basis* b, const ob_params* p, int64_t ncells, double dx, double dt,
               const double* u, double* u_new, double* q_out, ob_stats* st) {
  if (ncells <= 0) return OB_ERR_ARG;
  const int n = b->n;
  const double lam = dt / dx;
  const int64_t qs = (int64_t)n * n * OB_M, us = (int64_t)n * OB_M;
  double* q = q_out ? q_out : malloc(sizeof(double) * ncells * qs);
  if (!q) return OB_ERR_ARG;
  if (st) memset(st, 0, sizeof(*st));
  int status = OB_OK;
  for (int64_t i = 0; i < ncells; ++i) {
    int it = 0;
    if (ob_predict_cell(b, p, lam, u + i * us, q + i * qs, &it) != OB_OK)
      status = OB_ERR_NOT_CONVERGED;
    stats_add(st, it);
  }
  int rc = ob_dg_correct(b, p, ncells, dx, dt, u, q, u_new);
  if (!q_out) free(q);
  if (st) st->status = rc ? rc : status;
  return rc ? rc : status;
}

int ob_dg_step_cells(const ob_basis* b, const ob_params* p, int64_t ncells, double dx, double dt,
                     const double* u, const int64_t* cells, int64_t count, double* u_new_sel) {
  const int n = b->n;
  const double lam = dt / dx;
  const int64_t us = (int64_t)n * OB_M;
  double q[3][NMAX * NMAX * OB_M], qR[3][NMAX * OB_M], qL[3][NMAX * OB_M];
  int status = OB_OK;
  for (int64_t s = 0; s < count; ++s) {
    const int64_t i = cells[s];
    if (i < 0 || i >= ncells) return OB_ERR_ARG;
    for (int d = 0; d < 3; ++d) {
      const int64_t c = wrap(i + d - 1, ncells);
      int it;
      if (ob_predict_cell(b, p, lam, u + c * us, q[d], &it) != OB_OK) status = OB_ERR_NOT_CONVERGED;
      cell_traces(b, q[d], qR[d], qL[d]);
    }
    double Gl[OB_M], Gr[OB_M];
    face_flux(b, p, lam, qR[0], qL[1], Gl);
    face_flux(b, p, lam, qR[1], qL[2], Gr);
    dg_cell_update(b, p, lam, u + i * us, q[1], Gl, Gr, u_new_sel + s * us);
  }
  return status;
}

/* ------------------------------------------------------------------------ */
/* WENO reconstruction (eq. weno_reconstr): polynomial WENO from three       */
/* stencils of N+1 cells; constants are this oracle's reading of the paper,  */
/* which leaves stencils and weights unspecified                             */
/* ------------------------------------------------------------------------ */

int ob_weno_build(int N, const ob_basis* b, ob_weno* wt) {
  if (!wt || !b || N != b->N || N < 2 || (N % 2) != 0) return OB_ERR_ARG;
  memset(wt, 0, sizeof(*wt));
  const int n = N + 1;
  wt->N = N;
  wt->n = n;
  wt->shift[0] = -N / 2; /* central */
  wt->shift[1] = -N;     /* left-biased */
  wt->shift[2] = 0;      /* right-biased */
  wt->lin[0] = 1.0e5;
  wt->lin[1] = 1.0;
  wt->lin[2] = 1.0;
  wt->eps = 1.0e-14;
  wt->r = 8;
  /* re-derive the Lagrange coefficients (centred variable t = 2 xi - 1) from the stored nodes */
  ld x[NMAX], c[NMAX][NMAX + 1];
  for (int k = 0; k < n; ++k) x[k] = 2.0L * (ld)b->xi[k] - 1;
  for (int k = 0; k < n; ++k) lagrange_coeffs(x, n, k, c[k]);
  for (int S = 0; S < 3; ++S) {
    ld A[NMAX][NMAX], Ai[NMAX][NMAX];
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        /* average of phi_k over cell i+shift+j, i.e. xi in [shift+j, shift+j+1] */
        const ld lo = 2.0L * (ld)(wt->shift[S] + j) - 1, hi = lo + 2;
        A[j][k] = 0.5L * poly_integral(c[k], n, lo, hi);
      }
    if (gj_inverse(n, A, Ai)) return OB_ERR_ARG;
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) wt->ainv[S][j][k] = (double)Ai[j][k];
  }
  /* Sigma_kl = sum_{alpha=1..N} int_0^1 phi_k^(alpha) phi_l^(alpha) d xi (xi-derivatives) */
  ld d[NMAX][NMAX + 1];
  int len[NMAX];
  for (int k = 0; k < n; ++k) {
    for (int j = 0; j < n; ++j) d[k][j] = c[k][j];
    len[k] = n;
  }
  ld sig[NMAX][NMAX];
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) sig[k][l] = 0;
  for (int alpha = 1; alpha <= N; ++alpha) {
    for (int k = 0; k < n; ++k) {
      ld tmp[NMAX + 1];
      len[k] = poly_deriv(d[k], len[k], tmp);
      for (int j = 0; j < len[k]; ++j) d[k][j] = 2 * tmp[j];
    }
    for (int k = 0; k < n; ++k)
      for (int l = 0; l < n; ++l)
        sig[k][l] += 0.5L * poly_integral_prod(d[k], len[k], d[l], len[l], -1.0L, 1.0L);
  }
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) wt->sig[k][l] = (double)sig[k][l];
  /* derivative tables for the stable form of sigma */
  for (int k = 0; k < n; ++k) {
    for (int j = 0; j < n; ++j) d[k][j] = c[k][j];
    len[k] = n;
  }
  for (int alpha = 1; alpha <= N; ++alpha)
    for (int k = 0; k < n; ++k) {
      ld tmp[NMAX + 1];
      len[k] = poly_deriv(d[k], len[k], tmp);
      for (int j = 0; j < len[k]; ++j) d[k][j] = 2 * tmp[j];
      for (int q = 0; q < n; ++q) wt->dal[alpha - 1][q][k] = (double)poly_eval(d[k], len[k], x[q]);
    }
  for (int q = 0; q < n; ++q) wt->wq[q] = b->w[q];
  return OB_OK;
}

double ob_weno_sigma(const ob_weno* wt, const double* c) {
  const int n = wt->n;
  double sigma = 0.0;
  for (int a = 0; a < wt->N; ++a)
    for (int q = 0; q < n; ++q) {
      double d = 0.0;
      for (int k = 0; k < n; ++k) d += wt->dal[a][q][k] * c[k];
      sigma += wt->wq[q] * d * d;
    }
  return sigma;
}

int ob_weno_cell(const ob_weno* wt, int64_t ncells, const double* v, int64_t i, double* w_i,
                 double* omega) {
  const int n = wt->n;
  for (int r = 0; r < OB_M; ++r) {
    double cS[3][NMAX], wtil[3], wsum = 0.0;
    for (int S = 0; S < 3; ++S) {
      for (int k = 0; k < n; ++k) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j)
          acc += wt->ainv[S][k][j] * v[wrap(i + wt->shift[S] + j, ncells) * OB_M + r];
        cS[S][k] = acc;
      }
      const double sigma = ob_weno_sigma(wt, cS[S]);
      wtil[S] = wt->lin[S] / pow(sigma + wt->eps, (double)wt->r);
      wsum += wtil[S];
    }
    for (int k = 0; k < n; ++k) w_i[k * OB_M + r] = 0.0;
    for (int S = 0; S < 3; ++S) {
      const double om = wtil[S] / wsum;
      if (omega) omega[S * OB_M + r] = om;
      for (int k = 0; k < n; ++k) w_i[k * OB_M + r] += om * cS[S][k];
    }
  }
  return OB_OK;
}

int ob_weno_reconstruct(const ob_weno* wt, int64_t ncells, const double* v, double* w) {
  for (int64_t i = 0; i < ncells; ++i) ob_weno_cell(wt, ncells, v, i, w + i * wt->n * OB_M, NULL);
  return OB_OK;
}

int ob_fv_step(const ob_basis* b, const ob_weno* wt, const ob_params* p, int64_t ncells, double dx,
               double dt, const double* v, double* v_new, ob_stats* st) {
  if (ncells <= 0 || wt->N != b->N) return OB_ERR_ARG;
  const int n = b->n;
  const double lam = dt / dx;
  const int64_t us = (int64_t)n * OB_M;
  double* wrec = malloc(sizeof(double) * ncells * us);
  double* qR = malloc(sizeof(double) * ncells * us);
  double* qL = malloc(sizeof(double) * ncells * us);
  double* G = malloc(sizeof(double) * ncells * OB_M);
  if (!wrec || !qR || !qL || !G) {
    free(wrec);
    free(qR);
    free(qL);
    free(G);
    return OB_ERR_ARG;
  }
  if (st) memset(st, 0, sizeof(*st));
  int status = OB_OK;
  ob_weno_reconstruct(wt, ncells, v, wrec);
  for (int64_t i = 0; i < ncells; ++i) {
    double q[NMAX * NMAX * OB_M];
    int it = 0;
    if (ob_predict_cell(b, p, lam, wrec + i * us, q, &it) != OB_OK) status = OB_ERR_NOT_CONVERGED;
    stats_add(st, it);
    cell_traces(b, q, qR + i * us, qL + i * us);
  }
  for (int64_t i = 0; i < ncells; ++i)
    face_flux(b, p, lam, qR + i * us, qL + wrap(i + 1, ncells) * us, G + i * OB_M);
  /* get_fv_solution: v_next = v_prev - (G_{i+1/2} - G_{i-1/2}) (volume terms vanish for S = B = 0) */
  for (int64_t i = 0; i < ncells; ++i)
    for (int r = 0; r < OB_M; ++r)
      v_new[i * OB_M + r] =
          v[i * OB_M + r] - (G[i * OB_M + r] - G[wrap(i - 1, ncells) * OB_M + r]);
  free(wrec);
  free(qR);
  free(qL);
  free(G);
  if (st) st->status = status;
  return status;
}

int ob_fv_step_cells(const ob_basis* b, const ob_weno* wt, const ob_params* p, int64_t ncells,
                     double dx, double dt, const double* v, const int64_t* cells, int64_t count,
                     double* v_new_sel) {
  const int n = b->n;
  const double lam = dt / dx;
  int status = OB_OK;
  for (int64_t s = 0; s < count; ++s) {
    const int64_t i = cells[s];
    if (i < 0 || i >= ncells) return OB_ERR_ARG;
    double qR[3][NMAX * OB_M], qL[3][NMAX * OB_M];
    for (int d = 0; d < 3; ++d) {
      const int64_t c = wrap(i + d - 1, ncells);
      double wc[NMAX * OB_M], q[NMAX * NMAX * OB_M];
      int it;
      ob_weno_cell(wt, ncells, v, c, wc, NULL);
      if (ob_predict_cell(b, p, lam, wc, q, &it) != OB_OK) status = OB_ERR_NOT_CONVERGED;
      cell_traces(b, q, qR[d], qL[d]);
    }
    double Gl[OB_M], Gr[OB_M];
    face_flux(b, p, lam, qR[0], qL[1], Gl);
    face_flux(b, p, lam, qR[1], qL[2], Gr);
    for (int r = 0; r < OB_M; ++r) v_new_sel[s * OB_M + r] = v[i * OB_M + r] - (Gr[r] - Gl[r]);
  }
  (void)n;
  return status;
}

/* ------------------------------------------------------------------------ */
/* time loop                                                                */
/* ------------------------------------------------------------------------ */

int ob_solve(int scheme, const ob_basis* b, const ob_weno* wt, const ob_params* p, int64_t ncells,
             double dx, double* u, double t_end, int64_t max_steps, int64_t* steps_out,
             double* t_out) {
  if (ncells <= 0 || (scheme == 1 && !wt)) return OB_ERR_ARG;
  const int64_t cnt = scheme == 0 ? ncells * b->n * OB_M : ncells * OB_M;
  double* tmp = malloc(sizeof(double) * cnt);
  if (!tmp) return OB_ERR_ARG;
  double t = 0.0;
  int64_t steps = 0;
  int status = OB_OK;
  for (;;) {
    if (t_end > 0.0 && t >= t_end) break;
    if (max_steps > 0 && steps >= max_steps) break;
    double dt = scheme == 0 ? ob_dg_dt(b, p, dx, ncells, u) : ob_fv_dt(p, dx, ncells, u);
    if (!(dt > 0.0) || !isfinite(dt)) {
      status = OB_ERR_NONPHYSICAL;
      break;
    }
    int last = 0;
    if (t_end > 0.0 && t + dt >= t_end) {
      dt = t_end - t;
      last = 1;
    }
    int rc = scheme == 0 ? ob_dg_step(b, p, ncells, dx, dt, u, tmp, NULL, NULL)
                         : ob_fv_step(b, wt, p, ncells, dx, dt, u, tmp, NULL);
    if (rc != OB_OK && rc != OB_ERR_NOT_CONVERGED) {
      status = rc;
      break;
    }
    if (rc == OB_ERR_NOT_CONVERGED) status = rc;
    memcpy(u, tmp, sizeof(double) * cnt);
    ++steps;
    t = last ? t_end : t + dt;
  }
  free(tmp);
  if (steps_out) *steps_out = steps;
  if (t_out) *t_out = t;
  return status;
}
