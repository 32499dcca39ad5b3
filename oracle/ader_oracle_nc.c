/*
 * ader_oracle_nc.c -- the oracle's ADER-DG scheme with a non-conservative product
 * (eq. pde_src with B != 0) for the 1D Euler equations carrying a passive tracer
 * in non-conservative form:
 *     U = (rho, m, E, phi),  F = (m, m u + p, (E + p) u, 0),
 *     B(U) dU/dx = (0, 0, 0, u dphi/dx)          (u = m / rho).
 * Predictor: the nested Picard iteration of eq. lst_dg_predictor_nested_picards
 * with s = 0: the outer loop freezes the rescaled fluxes, the inner loop updates
 * the rescaled non-conservative term b = (dt/dx) B(q) (D^xi q) with the latest
 * iterate (D^xi = k~ along xi, Algorithm lst_dg_predictor:supp_2).  Corrector:
 * eq. ader_dg_method_full in 1D with the volume term of B and a path-
 * conservative Rusanov face flux: G +- (1/2) Bt, Bt = (int_0^1 B(psi(s)) ds)
 * (q+ - q-) along the straight segment psi(s) = q- + s (q+ - q-), the integral
 * by the 3-point Gauss-Legendre rule; the cell on the minus side takes G + Bt/2,
 * the cell on the plus side G - Bt/2 (the paper names no Riemann solver).
 * Plain C, FP64, one cell at a time.
 *
 * TEST INFRASTRUCTURE ONLY: tests, the package's smoke check and the CPU
 * baseline of the benchmark use this file; the library never does.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ader_oracle.h"

#define NM OB_MAXN
#define MN OB_NC_M

#define QN(p0, p1, r) ((((p0) * n) + (p1)) * MN + (r))

void ob_nc_flux(double gamma, const double* U, double* F) {
  const double rho = U[0], m = U[1], E = U[2];
  const double u = m / rho;
  const double p = (gamma - 1.0) * (E - 0.5 * m * u);
  F[0] = m;
  F[1] = m * u + p;
  F[2] = (E + p) * u;
  F[3] = 0.0;
}

/* the non-conservative product B(U) dU for an increment dU: (0, 0, 0, u dphi) */
static double nc_b(const double* U, double dphi) { return U[1] / U[0] * dphi; }

/* Rusanov part (Euler wave speed) and the path integral of B between a (minus
 * side) and b (plus side): G[4] and Bt (the phi component; the others vanish) */
void ob_nc_face(double gamma, const double* a, const double* b, double* G, double* Bt) {
  double Fa[MN], Fb[MN];
  ob_nc_flux(gamma, a, Fa);
  ob_nc_flux(gamma, b, Fb);
  const double sa = ob_wave_speed(gamma, a), sb = ob_wave_speed(gamma, b);
  const double s = (isnan(sa) || isnan(sb)) ? NAN : (sa > sb ? sa : sb);
  for (int r = 0; r < MN; ++r) G[r] = 0.5 * (Fa[r] + Fb[r]) - 0.5 * s * (b[r] - a[r]);
  /* 3-point Gauss-Legendre nodes and weights on [0, 1] */
  const double g = sqrt(0.6);
  const double sn[3] = {0.5 * (1.0 - g), 0.5, 0.5 * (1.0 + g)};
  const double sw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  double ubar = 0.0;
  for (int j = 0; j < 3; ++j) {
    double psi[MN];
    for (int r = 0; r < MN; ++r) psi[r] = a[r] + sn[j] * (b[r] - a[r]);
    ubar += sw[j] * (psi[1] / psi[0]);
  }
  *Bt = ubar * (b[3] - a[3]);
}

int ob_nc_predict_cell(const ob_basis* b, const ob_params* p, double lam, const double* u,
                       double* q, int* iters) {
  const int n = b->n;
  double g[NM * NM * MN], qo[NM * NM * MN], bb[NM * NM * MN], qn[NM * NM * MN];
  for (int p0 = 0; p0 < n; ++p0)
    for (int p1 = 0; p1 < n; ++p1)
      for (int r = 0; r < MN; ++r) q[QN(p0, p1, r)] = u[p1 * MN + r];
  const int cap = p->fixed_iter > 0 ? p->fixed_iter : p->max_iter;
  int it = 0, ok = 1, done = 0;
  while (it < cap && !done) {
    ++it;
    /* outer: rescaled fluxes of the current iterate and k~ along xi, frozen below */
    for (int p0 = 0; p0 < n; ++p0)
      for (int p1 = 0; p1 < n; ++p1)
        for (int r = 0; r < MN; ++r) {
          double acc = 0.0;
          for (int q1 = 0; q1 < n; ++q1) {
            double F[MN];
            ob_nc_flux(p->gamma, &q[QN(p0, q1, 0)], F);
            acc += b->kt[p1][q1] * (lam * F[r]);
          }
          g[QN(p0, p1, r)] = acc;
        }
    memcpy(qo, q, sizeof(double) * n * n * MN);
    /* inner: b with the latest iterate, kappa~ along tau, to tolerance */
    int m = 0, inner_done = 0;
    while (m < p->max_iter && !inner_done) {
      ++m;
      for (int p0 = 0; p0 < n; ++p0)
        for (int p1 = 0; p1 < n; ++p1) {
          double dphi = 0.0; /* (D^xi phi) at node p1 of row p0 */
          for (int q1 = 0; q1 < n; ++q1) dphi += b->kt[p1][q1] * q[QN(p0, q1, 3)];
          for (int r = 0; r < MN; ++r) bb[QN(p0, p1, r)] = 0.0;
          bb[QN(p0, p1, 3)] = lam * nc_b(&q[QN(p0, p1, 0)], dphi);
        }
      double delta = 0.0, qmax = 0.0;
      for (int p0 = 0; p0 < n; ++p0)
        for (int p1 = 0; p1 < n; ++p1)
          for (int r = 0; r < MN; ++r) {
            double acc = 0.0;
            for (int q0 = 0; q0 < n; ++q0) acc += b->kap[p0][q0] * (g[QN(q0, p1, r)] + bb[QN(q0, p1, r)]);
            const double v = u[p1 * MN + r] - acc;
            const double d = fabs(v - q[QN(p0, p1, r)]);
            if (d > delta) delta = d;
            if (fabs(v) > qmax) qmax = fabs(v);
            qn[QN(p0, p1, r)] = v;
          }
      memcpy(q, qn, sizeof(double) * n * n * MN);
      if (delta <= p->tol * (qmax > 1.0 ? qmax : 1.0)) inner_done = 1;
    }
    if (!inner_done) ok = 0;
    if (p->fixed_iter > 0) continue;
    double delta = 0.0, qmax = 0.0;
    for (int i = 0; i < n * n * MN; ++i) {
      const double d = fabs(q[i] - qo[i]);
      if (d > delta) delta = d;
      if (fabs(q[i]) > qmax) qmax = fabs(q[i]);
    }
    if (delta <= p->tol * (qmax > 1.0 ? qmax : 1.0)) done = 1;
  }
  if (p->fixed_iter > 0) done = 1;
  if (iters) *iters = it;
  return (ok && done) ? OB_OK : OB_ERR_NOT_CONVERGED;
}

static int64_t wrapn(int64_t i, int64_t n) { return ((i % n) + n) % n; }

int ob_nc_step(const ob_basis* b, const ob_params* p, int64_t ncells, double dx, double dt,
               const double* u, double* u_new, ob_stats* st) {
  if (ncells <= 0) return OB_ERR_ARG;
  const int n = b->n;
  const double lam = dt / dx;
  const int64_t us = (int64_t)n * MN, qs = (int64_t)n * n * MN;
  double* q = malloc(sizeof(double) * ncells * qs);
  double* G = malloc(sizeof(double) * ncells * MN);  /* face i - 1/2 */
  double* Bt = malloc(sizeof(double) * ncells);
  if (!q || !G || !Bt) {
    free(q), free(G), free(Bt);
    return OB_ERR_ARG;
  }
  if (st) memset(st, 0, sizeof(*st));
  int status = OB_OK;
  for (int64_t i = 0; i < ncells; ++i) {
    int it = 0;
    if (ob_nc_predict_cell(b, p, lam, u + i * us, q + i * qs, &it) != OB_OK)
      status = OB_ERR_NOT_CONVERGED;
    if (st) {
      if (st->cells == 0 || it > st->max_iters) st->max_iters = it;
      if (st->cells == 0 || it < st->min_iters) st->min_iters = it;
      st->mean_iters = (st->mean_iters * (double)st->cells + it) / (double)(st->cells + 1);
      st->cells += 1;
    }
  }
  /* faces: time-integrated rescaled Rusanov part and path term of face i - 1/2 */
  for (int64_t i = 0; i < ncells; ++i) {
    const double* ql = q + wrapn(i - 1, ncells) * qs;
    const double* qr = q + i * qs;
    double gs[MN] = {0}, bs = 0.0;
    for (int l0 = 0; l0 < n; ++l0) {
      double a[MN], c[MN];
      for (int r = 0; r < MN; ++r) {
        double aR = 0.0, aL = 0.0;
        for (int m = 0; m < n; ++m) {
          aR += b->psi1[m] * ql[QN(l0, m, r)];
          aL += b->psi0[m] * qr[QN(l0, m, r)];
        }
        a[r] = aR;
        c[r] = aL;
      }
      double g[MN], bt;
      ob_nc_face(p->gamma, a, c, g, &bt);
      for (int r = 0; r < MN; ++r) gs[r] += b->w[l0] * (lam * g[r]);
      bs += b->w[l0] * (lam * bt);
    }
    for (int r = 0; r < MN; ++r) G[i * MN + r] = gs[r];
    Bt[i] = bs;
  }
  for (int64_t i = 0; i < ncells; ++i) {
    const double* qi = q + i * qs;
    const int64_t ir = wrapn(i + 1, ncells);
    double fbar[NM * MN];
    for (int k = 0; k < n * MN; ++k) fbar[k] = 0.0;
    for (int l0 = 0; l0 < n; ++l0)
      for (int l = 0; l < n; ++l) {
        double F[MN];
        ob_nc_flux(p->gamma, &qi[QN(l0, l, 0)], F);
        for (int r = 0; r < MN; ++r) fbar[l * MN + r] += b->w[l0] * (lam * F[r]);
      }
    for (int k = 0; k < n; ++k) {
      /* volume term of B: sum_l0 w_l0 (dt/dx) B(q_l0k) (D^xi q)_l0k */
      double vb = 0.0;
      for (int l0 = 0; l0 < n; ++l0) {
        double dphi = 0.0;
        for (int r1 = 0; r1 < n; ++r1) dphi += b->kt[k][r1] * qi[QN(l0, r1, 3)];
        vb += b->w[l0] * (lam * nc_b(&qi[QN(l0, k, 0)], dphi));
      }
      for (int r = 0; r < MN; ++r) {
        double acc = 0.0;
        for (int l = 0; l < n; ++l) acc += b->dt_m[k][l] * fbar[l * MN + r];
        const double gr = G[ir * MN + r] + (r == 3 ? 0.5 * Bt[ir] : 0.0); /* minus side of i+1/2 */
        const double gl = G[i * MN + r] - (r == 3 ? 0.5 * Bt[i] : 0.0);   /* plus side of i-1/2 */
        u_new[i * us + k * MN + r] = u[i * us + k * MN + r] + acc / b->w[k] -
                                     (b->psi1[k] * gr - b->psi0[k] * gl) / b->w[k] -
                                     (r == 3 ? vb : 0.0);
      }
    }
  }
  free(q), free(G), free(Bt);
  if (st) st->status = status;
  return status;
}

int ob_nc_solve(const ob_basis* b, const ob_params* p, int64_t ncells, double dx, double* u,
                double t_end, int64_t max_steps, int64_t* steps_out, double* t_out) {
  if (ncells <= 0) return OB_ERR_ARG;
  const int n = b->n;
  const int64_t cnt = ncells * n * MN;
  double* tmp = malloc(sizeof(double) * cnt);
  double* e3 = malloc(sizeof(double) * ncells * n * 3);
  if (!tmp || !e3) {
    free(tmp), free(e3);
    return OB_ERR_ARG;
  }
  double t = 0.0;
  int64_t steps = 0;
  int status = OB_OK;
  for (;;) {
    if (t_end > 0.0 && t >= t_end) break;
    if (max_steps > 0 && steps >= max_steps) break;
    /* the time step of the Euler part (the tracer moves with u <= |u| + c) */
    for (int64_t i = 0; i < ncells * n; ++i)
      for (int r = 0; r < 3; ++r) e3[i * 3 + r] = u[i * MN + r];
    double dt = ob_dg_dt(b, p, dx, ncells, e3);
    if (!(dt > 0.0) || !isfinite(dt)) {
      status = OB_ERR_NONPHYSICAL;
      break;
    }
    int last = 0;
    if (t_end > 0.0 && t + dt >= t_end) {
      dt = t_end - t;
      last = 1;
    }
    const int rc = ob_nc_step(b, p, ncells, dx, dt, u, tmp, NULL);
    if (rc != OB_OK && rc != OB_ERR_NOT_CONVERGED) {
      status = rc;
      break;
    }
    if (rc == OB_ERR_NOT_CONVERGED) status = rc;
    memcpy(u, tmp, sizeof(double) * cnt);
    t = last ? t_end : t + dt;
    ++steps;
  }
  free(tmp), free(e3);
  if (steps_out) *steps_out = steps;
  if (t_out) *t_out = t;
  return status;
}
