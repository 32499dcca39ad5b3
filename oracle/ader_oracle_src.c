/*
 * ader_oracle_src.c -- the oracle's ADER-DG for a system with algebraic source
 * terms: the 1D two-component reacting flow (Sec. 2, eq. pdes_2_comps reduced
 * to one space dimension), predictor by the nested Picard iteration of
 * eq. lst_dg_predictor_nested_picards, corrector eq. ader_dg_method_full with
 * its source term.  Plain C, FP64, one cell at a time, sums in the order of the
 * paper's formulas.
 *
 * TEST INFRASTRUCTURE ONLY (see ader_oracle.h).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ader_oracle.h"

#define NMAXS OB_MAXN
#define MS OB_MRS
#define QI(p0, p1, r) ((((p0) * n) + (p1)) * MS + (r))

/* F = (m, m u + p, (E + p) u, rho c1 u, rho c2 u), p = (gamma - 1)(E - m u / 2) */
void ob_rs_flux(double gamma, const double* U, double* F) {
  const double u = U[1] / U[0];
  const double p = (gamma - 1.0) * (U[2] - 0.5 * U[1] * u);
  F[0] = U[1];
  F[1] = U[1] * u + p;
  F[2] = (U[2] + p) * u;
  F[3] = U[3] * u;
  F[4] = U[4] * u;
}

/* S = (0, 0, 0, rho c2, -omega^2 rho c1) */
void ob_rs_source(double omega, const double* U, double* S) {
  S[0] = 0.0;
  S[1] = 0.0;
  S[2] = 0.0;
  S[3] = U[4];
  S[4] = -omega * omega * U[3];
}

/* Rusanov with the Euler wave speed |u| + c (the species do not change it) */
void ob_rs_rusanov(double gamma, const double* a, const double* b, double* G) {
  double Fa[MS], Fb[MS];
  ob_rs_flux(gamma, a, Fa);
  ob_rs_flux(gamma, b, Fb);
  const double sa = ob_wave_speed(gamma, a), sb = ob_wave_speed(gamma, b);
  /* a non-physical state on either side (NaN speed) makes the flux NaN, so the
   * candidate fails the admissibility check instead of taking one side's speed */
  const double s = (isnan(sa) || isnan(sb)) ? NAN : (sa > sb ? sa : sb);
  for (int r = 0; r < MS; ++r) G[r] = 0.5 * (Fa[r] + Fb[r]) - 0.5 * s * (b[r] - a[r]);
}

static double max_abs_diff(const double* a, const double* b, int len, double* amax) {
  double d = 0.0, m = 0.0;
  for (int i = 0; i < len; ++i) {
    const double e = fabs(a[i] - b[i]);
    if (e > d) d = e;
    if (fabs(a[i]) > m) m = fabs(a[i]);
  }
  if (amax) *amax = m;
  return d;
}

/* Nested Picard (eq. lst_dg_predictor_nested_picards, B = 0):
 *   outer l:  f^(l) = (dt/dx) F(q^(l)),  g = (I (x) k~) f^(l)   (along xi)
 *   inner m:  s^(m) = dt S(q^(l+1,m)),   q^(l+1,m+1) = u (x) 1 - (kappa~ (x) I)(g - s^(m))
 *             from q^(l+1,0) = q^(l) until max|q^(m+1) - q^(m)| <= tol max(1, max|q|)
 *   until max|q^(l+1) - q^(l)| <= tol max(1, max|q|).                                   */
int ob_rs_predict_cell(const ob_basis* b, const ob_rs_params* p, double lam, double dt,
                       const double* u, double* q, int* iters, int* inner_total) {
  const int n = b->n, sz = n * n * MS;
  double g[NMAXS * NMAXS * MS], qo[NMAXS * NMAXS * MS], qi[NMAXS * NMAXS * MS],
      qn[NMAXS * NMAXS * MS], d[NMAXS * NMAXS * MS];
  for (int p0 = 0; p0 < n; ++p0)
    for (int p1 = 0; p1 < n; ++p1)
      for (int r = 0; r < MS; ++r) q[QI(p0, p1, r)] = u[p1 * MS + r];
  const int cap = p->fixed_iter > 0 ? p->fixed_iter : p->max_iter;
  int it = 0, inner_sum = 0, converged = 0, inner_ok = 1;
  while (it < cap) {
    ++it;
    memcpy(qo, q, sizeof(double) * sz);
    /* outer: rescaled flux and k~ along xi */
    for (int p0 = 0; p0 < n; ++p0) {
      double f[NMAXS][MS];
      for (int p1 = 0; p1 < n; ++p1) {
        ob_rs_flux(p->gamma, &qo[QI(p0, p1, 0)], f[p1]);
        for (int r = 0; r < MS; ++r) f[p1][r] *= lam;
      }
      for (int p1 = 0; p1 < n; ++p1)
        for (int r = 0; r < MS; ++r) {
          double acc = 0.0;
          for (int q1 = 0; q1 < n; ++q1) acc += b->kt[p1][q1] * f[q1][r];
          g[QI(p0, p1, r)] = acc;
        }
    }
    /* inner: sources with the latest iterate, kappa~ along tau */
    memcpy(qi, qo, sizeof(double) * sz);
    int m = 0, ok = 0;
    while (m < p->max_iter) {
      ++m;
      for (int p0 = 0; p0 < n; ++p0)
        for (int p1 = 0; p1 < n; ++p1) {
          double S[MS];
          ob_rs_source(p->omega, &qi[QI(p0, p1, 0)], S);
          for (int r = 0; r < MS; ++r) d[QI(p0, p1, r)] = g[QI(p0, p1, r)] - dt * S[r];
        }
      for (int p0 = 0; p0 < n; ++p0)
        for (int p1 = 0; p1 < n; ++p1)
          for (int r = 0; r < MS; ++r) {
            double acc = 0.0;
            for (int q0 = 0; q0 < n; ++q0) acc += b->kap[p0][q0] * d[QI(q0, p1, r)];
            qn[QI(p0, p1, r)] = u[p1 * MS + r] - acc;
          }
      double qmax;
      const double e_in = max_abs_diff(qn, qi, sz, &qmax);
      memcpy(qi, qn, sizeof(double) * sz);
      if (e_in <= p->tol * (qmax > 1.0 ? qmax : 1.0)) {
        ok = 1;
        break;
      }
    }
    inner_sum += m;
    if (!ok) inner_ok = 0;
    memcpy(q, qi, sizeof(double) * sz);
    double qmax;
    const double e_out = max_abs_diff(q, qo, sz, &qmax);
    if (p->fixed_iter <= 0 && e_out <= p->tol * (qmax > 1.0 ? qmax : 1.0)) {
      converged = 1;
      break;
    }
  }
  if (p->fixed_iter > 0) converged = 1;
  if (iters) *iters = it;
  if (inner_total) *inner_total = inner_sum;
  return (converged && inner_ok) ? OB_OK : OB_ERR_NOT_CONVERGED;
}

/* Single Picard loop: q' = u (x) 1 - (kappa~ (x) I)((I (x) k~) f(q) - s(q)), flux
 * and source from the same iterate (eq. lst_dg_predictor_picard with S != 0). */
int ob_rs_predict_cell_direct(const ob_basis* b, const ob_rs_params* p, double lam, double dt,
                              const double* u, double* q, int* iters) {
  const int n = b->n, sz = n * n * MS;
  double d[NMAXS * NMAXS * MS], qn[NMAXS * NMAXS * MS];
  for (int p0 = 0; p0 < n; ++p0)
    for (int p1 = 0; p1 < n; ++p1)
      for (int r = 0; r < MS; ++r) q[QI(p0, p1, r)] = u[p1 * MS + r];
  const int cap = p->fixed_iter > 0 ? p->fixed_iter : p->max_iter;
  int it = 0, converged = 0;
  while (it < cap) {
    ++it;
    for (int p0 = 0; p0 < n; ++p0) {
      double f[NMAXS][MS];
      for (int p1 = 0; p1 < n; ++p1) {
        ob_rs_flux(p->gamma, &q[QI(p0, p1, 0)], f[p1]);
        for (int r = 0; r < MS; ++r) f[p1][r] *= lam;
      }
      for (int p1 = 0; p1 < n; ++p1) {
        double S[MS];
        ob_rs_source(p->omega, &q[QI(p0, p1, 0)], S);
        for (int r = 0; r < MS; ++r) {
          double acc = 0.0;
          for (int q1 = 0; q1 < n; ++q1) acc += b->kt[p1][q1] * f[q1][r];
          d[QI(p0, p1, r)] = acc - dt * S[r];
        }
      }
    }
    for (int p0 = 0; p0 < n; ++p0)
      for (int p1 = 0; p1 < n; ++p1)
        for (int r = 0; r < MS; ++r) {
          double acc = 0.0;
          for (int q0 = 0; q0 < n; ++q0) acc += b->kap[p0][q0] * d[QI(q0, p1, r)];
          qn[QI(p0, p1, r)] = u[p1 * MS + r] - acc;
        }
    double qmax;
    const double e = max_abs_diff(qn, q, sz, &qmax);
    memcpy(q, qn, sizeof(double) * sz);
    if (p->fixed_iter <= 0 && e <= p->tol * (qmax > 1.0 ? qmax : 1.0)) {
      converged = 1;
      break;
    }
  }
  if (p->fixed_iter > 0) converged = 1;
  if (iters) *iters = it;
  return converged ? OB_OK : OB_ERR_NOT_CONVERGED;
}

/* CFL rule of Sec. 1.5 on the Euler part: lambda over the 2N+1 subcell averages */
double ob_rs_dg_dt(const ob_basis* b, const ob_rs_params* p, double dx, int64_t ncells,
                   const double* u) {
  const int n = b->n;
  double lmax = 0.0;
  for (int64_t i = 0; i < ncells; ++i)
    for (int j = 0; j < b->Ns; ++j) {
      double v[3] = {0.0, 0.0, 0.0};
      for (int k = 0; k < n; ++k)
        for (int r = 0; r < 3; ++r) v[r] += b->P[j][k] * u[(i * n + k) * MS + r];
      const double s = ob_wave_speed(p->gamma, v);
      if (!(s == s)) return NAN;
      if (s > lmax) lmax = s;
    }
  return p->cfl / (2.0 * b->N + 1.0) * dx / lmax;
}

static int64_t wrap_rs(int64_t i, int64_t n) {
  i %= n;
  return i < 0 ? i + n : i;
}

static void traces_rs(const ob_basis* b, const double* q, double* qR, double* qL) {
  const int n = b->n;
  for (int l0 = 0; l0 < n; ++l0)
    for (int r = 0; r < MS; ++r) {
      double aR = 0.0, aL = 0.0;
      for (int p1 = 0; p1 < n; ++p1) {
        aR += b->psi1[p1] * q[QI(l0, p1, r)];
        aL += b->psi0[p1] * q[QI(l0, p1, r)];
      }
      qR[l0 * MS + r] = aR;
      qL[l0 * MS + r] = aL;
    }
}

static void face_rs(const ob_basis* b, const ob_rs_params* p, double lam, const double* qR_left,
                    const double* qL_right, double* G) {
  for (int r = 0; r < MS; ++r) G[r] = 0.0;
  for (int l0 = 0; l0 < b->n; ++l0) {
    double g[MS];
    ob_rs_rusanov(p->gamma, qR_left + l0 * MS, qL_right + l0 * MS, g);
    for (int r = 0; r < MS; ++r) G[r] += b->w[l0] * (lam * g[r]);
  }
}

/* eq. ader_dg_method_full in 1D with the source term:
 * u_k' = u_k + (sum_l D~_kl fbar_l - psi~_k G_{i+1/2} + psi_k G_{i-1/2}) / w_k
 *            + sum_l0 w_l0 dt S(q_{l0,k})                                     */
static void update_rs(const ob_basis* b, const ob_rs_params* p, double lam, double dt,
                      const double* u, const double* q, const double* Gl, const double* Gr,
                      double* un) {
  const int n = b->n;
  double fbar[NMAXS * MS], sbar[NMAXS * MS];
  for (int i = 0; i < n * MS; ++i) fbar[i] = sbar[i] = 0.0;
  for (int l0 = 0; l0 < n; ++l0)
    for (int l = 0; l < n; ++l) {
      double F[MS], S[MS];
      ob_rs_flux(p->gamma, &q[QI(l0, l, 0)], F);
      ob_rs_source(p->omega, &q[QI(l0, l, 0)], S);
      for (int r = 0; r < MS; ++r) {
        fbar[l * MS + r] += b->w[l0] * (lam * F[r]);
        sbar[l * MS + r] += b->w[l0] * (dt * S[r]);
      }
    }
  for (int k = 0; k < n; ++k)
    for (int r = 0; r < MS; ++r) {
      double acc = 0.0;
      for (int l = 0; l < n; ++l) acc += b->dt_m[k][l] * fbar[l * MS + r];
      un[k * MS + r] = u[k * MS + r] + acc / b->w[k] -
                       (b->psi1[k] * Gr[r] - b->psi0[k] * Gl[r]) / b->w[k] + sbar[k * MS + r];
    }
}

int ob_rs_dg_step(const ob_basis* b, const ob_rs_params* p, int64_t ncells, double dx, double dt,
                  const double* u, double* u_new, double* q_out, ob_stats* st) {
  if (ncells <= 0) return OB_ERR_ARG;
  const int n = b->n;
  const double lam = dt / dx;
  const int64_t qs = (int64_t)n * n * MS, us = (int64_t)n * MS;
  double* q = q_out ? q_out : malloc(sizeof(double) * ncells * qs);
  double* qR = malloc(sizeof(double) * ncells * us);
  double* qL = malloc(sizeof(double) * ncells * us);
  double* G = malloc(sizeof(double) * ncells * MS);
  if (!q || !qR || !qL || !G) {
    if (!q_out) free(q);
    free(qR);
    free(qL);
    free(G);
    return OB_ERR_ARG;
  }
  if (st) memset(st, 0, sizeof(*st));
  int status = OB_OK;
  for (int64_t i = 0; i < ncells; ++i) {
    int it = 0;
    if (ob_rs_predict_cell(b, p, lam, dt, u + i * us, q + i * qs, &it, NULL) != OB_OK)
      status = OB_ERR_NOT_CONVERGED;
    if (st) {
      if (st->cells == 0 || it > st->max_iters) st->max_iters = it;
      if (st->cells == 0 || it < st->min_iters) st->min_iters = it;
      st->mean_iters = (st->mean_iters * (double)st->cells + it) / (double)(st->cells + 1);
      st->cells += 1;
    }
  }
  for (int64_t i = 0; i < ncells; ++i) traces_rs(b, q + i * qs, qR + i * us, qL + i * us);
  for (int64_t i = 0; i < ncells; ++i)
    face_rs(b, p, lam, qR + i * us, qL + wrap_rs(i + 1, ncells) * us, G + i * MS);
  for (int64_t i = 0; i < ncells; ++i)
    update_rs(b, p, lam, dt, u + i * us, q + i * qs, G + wrap_rs(i - 1, ncells) * MS, G + i * MS,
              u_new + i * us);
  if (!q_out) free(q);
  free(qR);
  free(qL);
  free(G);
  if (st) st->status = status;
  return status;
}

int ob_rs_dg_step_cells(const ob_basis* b, const ob_rs_params* p, int64_t ncells, double dx,
                        double dt, const double* u, const int64_t* cells, int64_t count,
                        double* u_new_sel) {
  const int n = b->n;
  const double lam = dt / dx;
  const int64_t us = (int64_t)n * MS;
  double q[3][NMAXS * NMAXS * MS], qR[3][NMAXS * MS], qL[3][NMAXS * MS];
  int status = OB_OK;
  for (int64_t s = 0; s < count; ++s) {
    const int64_t i = cells[s];
    if (i < 0 || i >= ncells) return OB_ERR_ARG;
    for (int d = 0; d < 3; ++d) {
      const int64_t c = wrap_rs(i + d - 1, ncells);
      if (ob_rs_predict_cell(b, p, lam, dt, u + c * us, q[d], NULL, NULL) != OB_OK)
        status = OB_ERR_NOT_CONVERGED;
      traces_rs(b, q[d], qR[d], qL[d]);
    }
    double Gl[MS], Gr[MS];
    face_rs(b, p, lam, qR[0], qL[1], Gl);
    face_rs(b, p, lam, qR[1], qL[2], Gr);
    update_rs(b, p, lam, dt, u + i * us, q[1], Gl, Gr, u_new_sel + s * us);
  }
  return status;
}

int ob_rs_solve(const ob_basis* b, const ob_rs_params* p, int64_t ncells, double dx, double* u,
                double t_end, int64_t max_steps, double dt_fixed, int64_t* steps_out,
                double* t_out) {
  if (ncells <= 0) return OB_ERR_ARG;
  const int64_t cnt = ncells * b->n * MS;
  double* tmp = malloc(sizeof(double) * cnt);
  if (!tmp) return OB_ERR_ARG;
  double t = 0.0;
  int64_t steps = 0;
  int status = OB_OK;
  for (;;) {
    if (t_end > 0.0 && t >= t_end) break;
    if (max_steps > 0 && steps >= max_steps) break;
    double dt = dt_fixed > 0.0 ? dt_fixed : ob_rs_dg_dt(b, p, dx, ncells, u);
    if (!(dt > 0.0) || !isfinite(dt)) {
      status = OB_ERR_NONPHYSICAL;
      break;
    }
    int last = 0;
    if (t_end > 0.0 && t + dt >= t_end) {
      dt = t_end - t;
      last = 1;
    }
    const int rc = ob_rs_dg_step(b, p, ncells, dx, dt, u, tmp, NULL, NULL);
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
