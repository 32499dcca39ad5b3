/*
 * ader_oracle_lim.c -- the oracle's outflow boundaries and a posteriori subcell
 * limiter for the 1D Euler ADER-DG scheme (Sec. 1.4 eq. p_operator /
 * eq. r_operator, Sec. 1.6 PAD and NAD eq. nad_ineq).  Plain C, FP64 (R in long
 * double), one cell at a time.  See ader_oracle.h for the readings.
 *
 * TEST INFRASTRUCTURE ONLY (see ader_oracle.h).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ader_oracle.h"

#define NM OB_MAXN
#define NSM OB_MAXNS
#define MM OB_M
typedef long double ld;

int ob_r_matrix(const ob_basis* b, double* R) {
  const int n = b->n, Ns = b->Ns;
  ld A[NM][NM], I[NM][NM];
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) {
      ld s = 0;
      for (int j = 0; j < Ns; ++j) s += (ld)b->P[j][k] * (ld)b->P[j][l];
      A[k][l] = s;
      I[k][l] = (k == l);
    }
  /* Gauss-Jordan with partial pivoting: I <- (P^T P)^-1 */
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(A[r][c]) > fabsl(A[piv][c])) piv = r;
    if (A[piv][c] == 0) return OB_ERR_ARG;
    for (int j = 0; j < n; ++j) {
      ld t = A[c][j];
      A[c][j] = A[piv][j];
      A[piv][j] = t;
      t = I[c][j];
      I[c][j] = I[piv][j];
      I[piv][j] = t;
    }
    const ld d = A[c][c];
    for (int j = 0; j < n; ++j) {
      A[c][j] /= d;
      I[c][j] /= d;
    }
    for (int r = 0; r < n; ++r)
      if (r != c) {
        const ld f = A[r][c];
        for (int j = 0; j < n; ++j) {
          A[r][j] -= f * A[c][j];
          I[r][j] -= f * I[c][j];
        }
      }
  }
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < Ns; ++j) {
      ld s = 0;
      for (int l = 0; l < n; ++l) s += I[k][l] * (ld)b->P[j][l];
      R[k * Ns + j] = (double)s;
    }
  return OB_OK;
}

#define QX(p0, p1, r) ((((p0) * n) + (p1)) * MM + (r))

static void traces(const ob_basis* b, const double* q, double* qR, double* qL) {
  const int n = b->n;
  for (int l0 = 0; l0 < n; ++l0)
    for (int r = 0; r < MM; ++r) {
      double aR = 0.0, aL = 0.0;
      for (int p1 = 0; p1 < n; ++p1) {
        aR += b->psi1[p1] * q[QX(l0, p1, r)];
        aL += b->psi0[p1] * q[QX(l0, p1, r)];
      }
      qR[l0 * MM + r] = aR;
      qL[l0 * MM + r] = aL;
    }
}

/* time-integrated rescaled Rusanov flux from tau-node traces */
static void dg_face(const ob_basis* b, const ob_params* p, double lam, const double* left,
                    const double* right, double* G) {
  for (int r = 0; r < MM; ++r) G[r] = 0.0;
  for (int l0 = 0; l0 < b->n; ++l0) {
    double g[MM];
    ob_rusanov(p->gamma, left + l0 * MM, right + l0 * MM, g);
    for (int r = 0; r < MM; ++r) G[r] += b->w[l0] * (lam * g[r]);
  }
}

/* subcell averages v[j][r] = sum_k P_jk u_k */
static void project(const ob_basis* b, const double* u, double* v) {
  const int n = b->n;
  for (int j = 0; j < b->Ns; ++j)
    for (int r = 0; r < MM; ++r) {
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc += b->P[j][k] * u[k * MM + r];
      v[j * MM + r] = acc;
    }
}

/* WENO reconstruction of degree 1 on one subcell (the reconstruction of the
 * ADER-WENO2 subcell scheme): the two candidate linear polynomials with the
 * subcell's average v0 and the average of one neighbour (stencils {j-1, j} and
 * {j, j+1}); smoothness sigma_S = int_0^1 (dw_S/dxi)^2 dxi = slope_S^2; weights
 * omega_S = w~_S / sum w~, w~_S = lambda_S / (sigma_S + eps)^r with lambda_S = 1,
 * eps = 1e-14, r = 8 (the constants of the WENO reading of eq. weno_reconstr);
 * nodal values at the two Gauss nodes xi_k of the subcell. */
void ob_lim_weno2(const double* vm, const double* v0, const double* vp, const double* xi,
                  double* w) {
  for (int r = 0; r < MM; ++r) {
    const double sl = v0[r] - vm[r], sr = vp[r] - v0[r];
    const double al = 1.0 / pow(sl * sl + 1.0e-14, 8.0);
    const double ar = 1.0 / pow(sr * sr + 1.0e-14, 8.0);
    const double slope = (al * sl + ar * sr) / (al + ar);
    for (int k = 0; k < 2; ++k) w[k * MM + r] = v0[r] + slope * (xi[k] - 0.5);
  }
}

/* subcell g of the global subcell grid (cell i, subcell j: g = i Ns + j) with
 * the boundary condition: periodic wrap, or (outflow) the boundary subcell */
static const double* sub_v(const double* V, int64_t g, int64_t nsub, int outflow) {
  if (outflow) {
    if (g < 0) g = 0;
    if (g >= nsub) g = nsub - 1;
  } else {
    while (g < 0) g += nsub;
    while (g >= nsub) g -= nsub;
  }
  return V + g * MM;
}

/* ADER-WENO2 flux through the face between subcells g-1 and g: WENO
 * reconstruction of degree 1 on both subcells, the LST-DG predictor of degree 1
 * on each (subcell width dx / Ns, so dt / (dx / Ns) = Ns lam), and the
 * time-integrated Rusanov flux of their traces, rescaled by lam = dt / dx like
 * the DG face fluxes. */
static int sub_face(const ob_basis* b1, const ob_params* p, double lam, int Ns, const double* V,
                    int64_t nsub, int outflow, int64_t g, double* G) {
  double wl[2 * MM], wr[2 * MM], q[4 * MM], qRl[2 * MM], qLl[2 * MM], qRr[2 * MM], qLr[2 * MM];
  ob_lim_weno2(sub_v(V, g - 2, nsub, outflow), sub_v(V, g - 1, nsub, outflow),
               sub_v(V, g, nsub, outflow), b1->xi, wl);
  ob_lim_weno2(sub_v(V, g - 1, nsub, outflow), sub_v(V, g, nsub, outflow),
               sub_v(V, g + 1, nsub, outflow), b1->xi, wr);
  int it = 0, status = OB_OK;
  if (ob_predict_cell(b1, p, (double)Ns * lam, wl, q, &it) != OB_OK) status = OB_ERR_NOT_CONVERGED;
  traces(b1, q, qRl, qLl);
  if (ob_predict_cell(b1, p, (double)Ns * lam, wr, q, &it) != OB_OK) status = OB_ERR_NOT_CONVERGED;
  traces(b1, q, qRr, qLr);
  dg_face(b1, p, lam, qRl, qLr, G);
  return status;
}

static int admissible(double gamma, const double* U) {
  const double rho = U[0];
  const double e = U[2] - 0.5 * U[1] * U[1] / rho;  /* internal energy density */
  (void)gamma;
  return rho > 0.0 && e > 0.0 && isfinite(rho) && isfinite(e);
}

int ob_dgl_step(const ob_basis* b, const ob_params* p, const ob_lim_params* lp, int64_t ncells,
                double dx, double dt, const double* u, double* u_new, int* troubled_out,
                ob_stats* st) {
  if (ncells <= 0 || !lp || lp->limiter < 0 || lp->limiter > 2) return OB_ERR_ARG;
  if (lp->limiter && b->N < 1) return OB_ERR_ARG;  /* P0: the subcell grid is the mesh */
  const int n = b->n, Ns = b->Ns;
  const double lam = dt / dx;
  const int64_t qs = (int64_t)n * n * MM, us = (int64_t)n * MM, vs = (int64_t)Ns * MM;
  const int outflow = lp->bc == 1;
  double* q = malloc(sizeof(double) * ncells * qs);
  double* qR = malloc(sizeof(double) * ncells * us);
  double* qL = malloc(sizeof(double) * ncells * us);
  double* G = malloc(sizeof(double) * (ncells + 1) * MM);   /* face f: between cells f-1 and f */
  double* G2 = malloc(sizeof(double) * (ncells + 1) * MM);
  double* vn = malloc(sizeof(double) * ncells * vs);
  int* tr = calloc((size_t)ncells, sizeof(int));
  if (!q || !qR || !qL || !G || !G2 || !vn || !tr) {
    free(q), free(qR), free(qL), free(G), free(G2), free(vn), free(tr);
    return OB_ERR_ARG;
  }
  if (st) memset(st, 0, sizeof(*st));
  int status = OB_OK;
  for (int64_t i = 0; i < ncells; ++i) {
    int it = 0;
    if (ob_predict_cell(b, p, lam, u + i * us, q + i * qs, &it) != OB_OK) status = OB_ERR_NOT_CONVERGED;
    if (st) {
      if (st->cells == 0 || it > st->max_iters) st->max_iters = it;
      if (st->cells == 0 || it < st->min_iters) st->min_iters = it;
      st->mean_iters = (st->mean_iters * (double)st->cells + it) / (double)(st->cells + 1);
      st->cells += 1;
    }
    traces(b, q + i * qs, qR + i * us, qL + i * us);
  }
  /* outflow ghosts: the boundary cell's mean state of u^n at every tau node */
  double ghost_l[NM * MM], ghost_r[NM * MM];
  for (int r = 0; r < MM; ++r) {
    double ml = 0.0, mr = 0.0;
    for (int k = 0; k < n; ++k) {
      ml += b->w[k] * u[k * MM + r];
      mr += b->w[k] * u[(ncells - 1) * us + k * MM + r];
    }
    for (int l0 = 0; l0 < n; ++l0) {
      ghost_l[l0 * MM + r] = ml;
      ghost_r[l0 * MM + r] = mr;
    }
  }
  /* face fluxes with the boundary condition */
  for (int64_t f = 0; f <= ncells; ++f) {
    const double *left, *right;
    if (f == 0)
      left = outflow ? ghost_l : qR + (ncells - 1) * us;
    else
      left = qR + (f - 1) * us;
    if (f == ncells)
      right = outflow ? ghost_r : qL;
    else
      right = qL + f * us;
    dg_face(b, p, lam, left, right, G + f * MM);
  }
  /* candidate: eq. ader_dg_method_full in 1D */
  for (int64_t i = 0; i < ncells; ++i) {
    const double* qi = q + i * qs;
    double fbar[NM * MM];
    for (int k = 0; k < n * MM; ++k) fbar[k] = 0.0;
    for (int l0 = 0; l0 < n; ++l0)
      for (int l = 0; l < n; ++l) {
        double F[MM];
        ob_euler_flux(p->gamma, &qi[QX(l0, l, 0)], F);
        for (int r = 0; r < MM; ++r) fbar[l * MM + r] += b->w[l0] * (lam * F[r]);
      }
    for (int k = 0; k < n; ++k)
      for (int r = 0; r < MM; ++r) {
        double acc = 0.0;
        for (int l = 0; l < n; ++l) acc += b->dt_m[k][l] * fbar[l * MM + r];
        u_new[i * us + k * MM + r] =
            u[i * us + k * MM + r] + acc / b->w[k] -
            (b->psi1[k] * G[(i + 1) * MM + r] - b->psi0[k] * G[i * MM + r]) / b->w[k];
      }
  }
  int64_t ntroubled = 0;
  if (lp->limiter) {
    for (int64_t i = 0; i < ncells; ++i) project(b, u + i * us, vn + i * vs);
    /* detection on the subcell averages of the candidate (limiter 2: every cell) */
    for (int64_t i = 0; i < ncells && lp->limiter == 2; ++i) tr[i] = 1;
    ntroubled = lp->limiter == 2 ? ncells : 0;
    for (int64_t i = 0; i < ncells && lp->limiter == 1; ++i) {
      double vs_[NSM * MM];
      project(b, u_new + i * us, vs_);
      int bad = 0;
      for (int j = 0; j < Ns && !bad; ++j)
        if (!admissible(p->gamma, vs_ + j * MM)) bad = 1;  /* PAD */
      for (int r = 0; r < MM && !bad; ++r) {                  /* NAD */
        double lo = INFINITY, hi = -INFINITY;
        for (int d = -1; d <= 1; ++d) {
          int64_t c = i + d;
          if (c < 0 || c >= ncells) {
            if (outflow) continue;
            c = (c + ncells) % ncells;
          }
          for (int j = 0; j < Ns; ++j) {
            const double x = vn[c * vs + j * MM + r];
            if (x < lo) lo = x;
            if (x > hi) hi = x;
          }
        }
        double delta = lp->eps * (hi - lo);
        if (delta < lp->delta0) delta = lp->delta0;
        for (int j = 0; j < Ns; ++j) {
          const double x = vs_[j * MM + r];
          if (x < lo - delta || x > hi + delta) bad = 1;
        }
      }
      tr[i] = bad;
      ntroubled += bad;
    }
    /* faces next to a troubled cell carry the ADER-WENO2 subcell flux */
    ob_basis b1;
    if (ob_basis_build(1, &b1) != OB_OK) status = OB_ERR_ARG;
    const int64_t nsub = ncells * Ns;
    memcpy(G2, G, sizeof(double) * (ncells + 1) * MM);
    for (int64_t f = 0; f <= ncells; ++f) {
      const int64_t cl = f - 1, cr = f;
      const int tl = cl >= 0 ? tr[cl] : (outflow ? 0 : tr[ncells - 1]);
      const int tr_ = cr < ncells ? tr[cr] : (outflow ? 0 : tr[0]);
      if (!tl && !tr_) continue;
      if (sub_face(&b1, p, lam, Ns, vn, nsub, outflow, f * Ns, G2 + f * MM) != OB_OK)
        status = OB_ERR_NOT_CONVERGED;
    }
    double R[NM * NSM];
    if (ob_r_matrix(b, R) != OB_OK) status = OB_ERR_ARG;
    for (int64_t i = 0; i < ncells; ++i) {
      double* un = u_new + i * us;
      if (!tr[i]) {
        /* DG neighbour of a limited face: the face term with the subcell flux */
        for (int k = 0; k < n; ++k)
          for (int r = 0; r < MM; ++r)
            un[k * MM + r] += -(b->psi1[k] * (G2[(i + 1) * MM + r] - G[(i + 1) * MM + r]) -
                                b->psi0[k] * (G2[i * MM + r] - G[i * MM + r])) / b->w[k];
        continue;
      }
      /* ADER-WENO2 finite volumes on the 2N+1 subcells (eq.
       * ader_weno_fv_method_full on the subgrid, with the cell's own faces) */
      const double* v = vn + i * vs;
      double F[(NSM + 1) * MM], vnew[NSM * MM];
      for (int r = 0; r < MM; ++r) {
        F[r] = G2[i * MM + r];
        F[Ns * MM + r] = G2[(i + 1) * MM + r];
      }
      for (int j = 1; j < Ns; ++j)
        if (sub_face(&b1, p, lam, Ns, vn, nsub, outflow, i * Ns + j, F + j * MM) != OB_OK)
          status = OB_ERR_NOT_CONVERGED;
      for (int j = 0; j < Ns; ++j)
        for (int r = 0; r < MM; ++r)
          vnew[j * MM + r] = v[j * MM + r] - (double)Ns * (F[(j + 1) * MM + r] - F[j * MM + r]);
      /* reconstruction u = R v, with the cell mean as fallback */
      for (int k = 0; k < n; ++k)
        for (int r = 0; r < MM; ++r) {
          double acc = 0.0;
          for (int j = 0; j < Ns; ++j) acc += R[k * Ns + j] * vnew[j * MM + r];
          un[k * MM + r] = acc;
        }
      double chk[NSM * MM];
      project(b, un, chk);
      int ok = 1;
      for (int j = 0; j < Ns; ++j)
        if (!admissible(p->gamma, chk + j * MM)) ok = 0;
      if (!ok) {
        for (int r = 0; r < MM; ++r) {
          double mean = 0.0;
          for (int j = 0; j < Ns; ++j) mean += vnew[j * MM + r];
          mean /= (double)Ns;
          for (int k = 0; k < n; ++k) un[k * MM + r] = mean;
        }
      }
    }
  }
  if (troubled_out) memcpy(troubled_out, tr, sizeof(int) * (size_t)ncells);
  free(q), free(qR), free(qL), free(G), free(G2), free(vn), free(tr);
  if (st) st->status = status;
  return status;
}

int ob_dgl_solve(const ob_basis* b, const ob_params* p, const ob_lim_params* lp, int64_t ncells,
                 double dx, double* u, double t_end, int64_t max_steps, int64_t* steps_out,
                 double* t_out, int64_t* troubled_total) {
  if (ncells <= 0) return OB_ERR_ARG;
  const int64_t cnt = ncells * b->n * MM;
  double* tmp = malloc(sizeof(double) * cnt);
  int* tr = malloc(sizeof(int) * (size_t)ncells);
  if (!tmp || !tr) {
    free(tmp), free(tr);
    return OB_ERR_ARG;
  }
  double t = 0.0;
  int64_t steps = 0, ttot = 0;
  int status = OB_OK;
  for (;;) {
    if (t_end > 0.0 && t >= t_end) break;
    if (max_steps > 0 && steps >= max_steps) break;
    double dt = ob_dg_dt(b, p, dx, ncells, u);
    if (!(dt > 0.0) || !isfinite(dt)) {
      status = OB_ERR_NONPHYSICAL;
      break;
    }
    int last = 0;
    if (t_end > 0.0 && t + dt >= t_end) {
      dt = t_end - t;
      last = 1;
    }
    const int rc = ob_dgl_step(b, p, lp, ncells, dx, dt, u, tmp, tr, NULL);
    if (rc != OB_OK && rc != OB_ERR_NOT_CONVERGED) {
      status = rc;
      break;
    }
    if (rc == OB_ERR_NOT_CONVERGED) status = rc;
    for (int64_t i = 0; i < ncells; ++i) ttot += tr[i];
    memcpy(u, tmp, sizeof(double) * cnt);
    ++steps;
    t = last ? t_end : t + dt;
  }
  free(tmp), free(tr);
  if (steps_out) *steps_out = steps;
  if (t_out) *t_out = t;
  if (troubled_total) *troubled_total = ttot;
  return status;
}
