/*
 * ader_oracle_2d.c -- the oracle's ADER-DG scheme for the 2D Euler equations on
 * a periodic Cartesian mesh: the tensor-product LST-DG predictor of Sec. 1.1
 * (eq. lst_dg_predictor_picard with L^xi = kappa~ (x) k~ (x) I and
 * L^eta = kappa~ (x) I (x) k~, L^0 = delta by eq. ind_prop), the one-step
 * corrector of Sec. 1.2 (eq. ader_dg_method_full with x- and y-faces) and the
 * time step of Sec. 1.5 with d = 2.  Plain C, FP64, one cell at a time, in the
 * order of the paper's sums.
 *
 * Layout: state u[cell][k1][k2][r] with cell = iy nx + ix, k1 the xi node, k2
 * the eta node, r = (rho, m_x, m_y, E); predictor q[p0][p1][p2][r] with p0 the
 * tau node.
 *
 * TEST INFRASTRUCTURE ONLY: tests, the package's smoke check and the CPU
 * baseline of the benchmark use this file; the library never does.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ader_oracle.h"

#define NM OB_MAXN
#define M2 OB2_M

#define Q2(p0, p1, p2, r) (((((p0) * n + (p1)) * n + (p2)) * M2) + (r))
#define U2(k1, k2, r) ((((k1) * n + (k2)) * M2) + (r))

/* Euler fluxes in x and y (Sec. 2, eq. system_of_equations in 2D) */
void ob2_flux(double gamma, const double* U, double* F, double* G) {
  const double rho = U[0], mx = U[1], my = U[2], E = U[3];
  const double u = mx / rho, v = my / rho;
  const double p = (gamma - 1.0) * (E - 0.5 * (mx * u + my * v));
  F[0] = mx;
  F[1] = mx * u + p;
  F[2] = my * u;
  F[3] = (E + p) * u;
  G[0] = my;
  G[1] = mx * v;
  G[2] = my * v + p;
  G[3] = (E + p) * v;
}

/* |u_dir| + c; NaN for a non-physical state */
double ob2_speed(double gamma, const double* U, int dir) {
  const double rho = U[0], mx = U[1], my = U[2], E = U[3];
  const double u = mx / rho, v = my / rho;
  const double p = (gamma - 1.0) * (E - 0.5 * (mx * u + my * v));
  if (!(rho > 0.0) || !(p > 0.0)) return NAN;
  return fabs(dir == 0 ? u : v) + sqrt(gamma * p / rho);
}

/* Rusanov flux in direction dir between a (low side) and b (high side) */
void ob2_rusanov(double gamma, int dir, const double* a, const double* b, double* H) {
  double Fa[M2], Ga[M2], Fb[M2], Gb[M2];
  ob2_flux(gamma, a, Fa, Ga);
  ob2_flux(gamma, b, Fb, Gb);
  const double* fa = dir == 0 ? Fa : Ga;
  const double* fb = dir == 0 ? Fb : Gb;
  const double sa = ob2_speed(gamma, a, dir), sb = ob2_speed(gamma, b, dir);
  const double s = (isnan(sa) || isnan(sb)) ? NAN : (sa > sb ? sa : sb);
  for (int r = 0; r < M2; ++r) H[r] = 0.5 * (fa[r] + fb[r]) - 0.5 * s * (b[r] - a[r]);
}

int ob2_predict_cell(const ob_basis* b, const ob_params* p, double lx, double ly, const double* u,
                     double* q, int* iters) {
  const int n = b->n;
  const int cnt = n * n * n * M2;
  double* f = malloc(sizeof(double) * cnt);
  double* g = malloc(sizeof(double) * cnt);
  double* s = malloc(sizeof(double) * cnt);
  double* qn = malloc(sizeof(double) * cnt);
  if (!f || !g || !s || !qn) {
    free(f), free(g), free(s), free(qn);
    return OB_ERR_ARG;
  }
  /* initial iterate: q_{p0 p1 p2} = u_{p1 p2} (L^0 = delta) */
  for (int p0 = 0; p0 < n; ++p0)
    for (int p1 = 0; p1 < n; ++p1)
      for (int p2 = 0; p2 < n; ++p2)
        for (int r = 0; r < M2; ++r) q[Q2(p0, p1, p2, r)] = u[U2(p1, p2, r)];
  const int cap = p->fixed_iter > 0 ? p->fixed_iter : p->max_iter;
  int it = 0, converged = 0;
  while (it < cap) {
    ++it;
    /* rescaled fluxes (dt/dx) F(q), (dt/dy) G(q) at every space-time node */
    for (int p0 = 0; p0 < n; ++p0)
      for (int p1 = 0; p1 < n; ++p1)
        for (int p2 = 0; p2 < n; ++p2) {
          double F[M2], G[M2];
          ob2_flux(p->gamma, &q[Q2(p0, p1, p2, 0)], F, G);
          for (int r = 0; r < M2; ++r) {
            f[Q2(p0, p1, p2, r)] = lx * F[r];
            g[Q2(p0, p1, p2, r)] = ly * G[r];
          }
        }
    /* k~ along xi on f plus k~ along eta on g */
    for (int p0 = 0; p0 < n; ++p0)
      for (int p1 = 0; p1 < n; ++p1)
        for (int p2 = 0; p2 < n; ++p2)
          for (int r = 0; r < M2; ++r) {
            double acc = 0.0;
            for (int q1 = 0; q1 < n; ++q1) acc += b->kt[p1][q1] * f[Q2(p0, q1, p2, r)];
            for (int q2 = 0; q2 < n; ++q2) acc += b->kt[p2][q2] * g[Q2(p0, p1, q2, r)];
            s[Q2(p0, p1, p2, r)] = acc;
          }
    /* kappa~ along tau */
    for (int p0 = 0; p0 < n; ++p0)
      for (int p1 = 0; p1 < n; ++p1)
        for (int p2 = 0; p2 < n; ++p2)
          for (int r = 0; r < M2; ++r) {
            double acc = 0.0;
            for (int q0 = 0; q0 < n; ++q0) acc += b->kap[p0][q0] * s[Q2(q0, p1, p2, r)];
            qn[Q2(p0, p1, p2, r)] = u[U2(p1, p2, r)] - acc;
          }
    double delta = 0.0, qmax = 0.0;
    for (int i = 0; i < cnt; ++i) {
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
  free(f), free(g), free(s), free(qn);
  return converged ? OB_OK : OB_ERR_NOT_CONVERGED;
}

static int64_t wrap2(int64_t i, int64_t n) { return ((i % n) + n) % n; }

/* predictor, face traces [l0][k][r] (xR, xL, yR, yL) and volume term of one cell */
static int cell_record(const ob_basis* b, const ob_params* p, double lx, double ly,
                       const double* uc, double* q, double* xR, double* xL, double* yR,
                       double* yL, double* vol, int* iters) {
  const int n = b->n;
  const int64_t us = (int64_t)n * n * M2;
  const int status = ob2_predict_cell(b, p, lx, ly, uc, q, iters);
  for (int l0 = 0; l0 < n; ++l0)
    for (int k = 0; k < n; ++k)
      for (int r = 0; r < M2; ++r) {
        double aR = 0.0, aL = 0.0, bR = 0.0, bL = 0.0;
        for (int m = 0; m < n; ++m) {
          aR += b->psi1[m] * q[Q2(l0, m, k, r)];
          aL += b->psi0[m] * q[Q2(l0, m, k, r)];
          bR += b->psi1[m] * q[Q2(l0, k, m, r)];
          bL += b->psi0[m] * q[Q2(l0, k, m, r)];
        }
        const int64_t o = ((int64_t)l0 * n + k) * M2 + r;
        xR[o] = aR;
        xL[o] = aL;
        yR[o] = bR;
        yL[o] = bL;
      }
  /* volume terms: time-averaged rescaled fluxes, D~ along xi and eta */
  double* fbar = malloc(sizeof(double) * us);
  double* gbar = malloc(sizeof(double) * us);
  if (!fbar || !gbar) {
    free(fbar), free(gbar);
    return OB_ERR_ARG;
  }
  for (int i = 0; i < us; ++i) fbar[i] = gbar[i] = 0.0;
  for (int l0 = 0; l0 < n; ++l0)
    for (int l1 = 0; l1 < n; ++l1)
      for (int l2 = 0; l2 < n; ++l2) {
        double F[M2], G[M2];
        ob2_flux(p->gamma, &q[Q2(l0, l1, l2, 0)], F, G);
        for (int r = 0; r < M2; ++r) {
          fbar[U2(l1, l2, r)] += b->w[l0] * (lx * F[r]);
          gbar[U2(l1, l2, r)] += b->w[l0] * (ly * G[r]);
        }
      }
  for (int k1 = 0; k1 < n; ++k1)
    for (int k2 = 0; k2 < n; ++k2)
      for (int r = 0; r < M2; ++r) {
        double ax = 0.0, ay = 0.0;
        for (int l = 0; l < n; ++l) {
          ax += b->dt_m[k1][l] * fbar[U2(l, k2, r)];
          ay += b->dt_m[k2][l] * gbar[U2(k1, l, r)];
        }
        vol[U2(k1, k2, r)] = uc[U2(k1, k2, r)] + ax / b->w[k1] + ay / b->w[k2];
      }
  free(fbar), free(gbar);
  return status;
}

int ob2_dg_step(const ob_basis* b, const ob_params* p, int64_t nx, int64_t ny, double dx,
                double dy, double dt, const double* u, double* u_new, ob_stats* st) {
  if (nx <= 0 || ny <= 0) return OB_ERR_ARG;
  const int n = b->n;
  const int64_t nc = nx * ny;
  const double lx = dt / dx, ly = dt / dy;
  const int64_t us = (int64_t)n * n * M2, ts = (int64_t)n * n * M2;
  double* q = malloc(sizeof(double) * n * us);
  /* traces: [cell][l0][k][r] at the x = 1 (xR), x = 0 (xL), y = 1 (yR), y = 0 (yL) sides */
  double* xR = malloc(sizeof(double) * nc * ts);
  double* xL = malloc(sizeof(double) * nc * ts);
  double* yR = malloc(sizeof(double) * nc * ts);
  double* yL = malloc(sizeof(double) * nc * ts);
  double* vol = malloc(sizeof(double) * nc * us);
  double* Gx = malloc(sizeof(double) * nc * n * M2); /* left x-face of each cell, [cell][k2][r] */
  double* Gy = malloc(sizeof(double) * nc * n * M2); /* bottom y-face of each cell, [cell][k1][r] */
  if (!q || !xR || !xL || !yR || !yL || !vol || !Gx || !Gy) {
    free(q), free(xR), free(xL), free(yR), free(yL), free(vol), free(Gx), free(Gy);
    return OB_ERR_ARG;
  }
  if (st) memset(st, 0, sizeof(*st));
  int status = OB_OK;
  for (int64_t c = 0; c < nc; ++c) {
    int it = 0;
    if (cell_record(b, p, lx, ly, u + c * us, q, xR + c * ts, xL + c * ts, yR + c * ts, yL + c * ts,
                    vol + c * us, &it) != OB_OK)
      status = OB_ERR_NOT_CONVERGED;
    if (st) {
      if (st->cells == 0 || it > st->max_iters) st->max_iters = it;
      if (st->cells == 0 || it < st->min_iters) st->min_iters = it;
      st->mean_iters = (st->mean_iters * (double)st->cells + it) / (double)(st->cells + 1);
      st->cells += 1;
    }
  }
  /* time-integrated Rusanov fluxes through the left x-face and the bottom y-face of each cell */
  for (int64_t iy = 0; iy < ny; ++iy)
    for (int64_t ix = 0; ix < nx; ++ix) {
      const int64_t c = iy * nx + ix;
      const int64_t cl = iy * nx + wrap2(ix - 1, nx), cb = wrap2(iy - 1, ny) * nx + ix;
      for (int k = 0; k < n; ++k) {
        double hx[M2] = {0}, hy[M2] = {0};
        for (int l0 = 0; l0 < n; ++l0) {
          double H[M2];
          ob2_rusanov(p->gamma, 0, &xR[cl * ts + ((int64_t)l0 * n + k) * M2],
                      &xL[c * ts + ((int64_t)l0 * n + k) * M2], H);
          for (int r = 0; r < M2; ++r) hx[r] += b->w[l0] * (lx * H[r]);
          ob2_rusanov(p->gamma, 1, &yR[cb * ts + ((int64_t)l0 * n + k) * M2],
                      &yL[c * ts + ((int64_t)l0 * n + k) * M2], H);
          for (int r = 0; r < M2; ++r) hy[r] += b->w[l0] * (ly * H[r]);
        }
        for (int r = 0; r < M2; ++r) {
          Gx[(c * n + k) * M2 + r] = hx[r];
          Gy[(c * n + k) * M2 + r] = hy[r];
        }
      }
    }
  /* u^{n+1} = volume terms - face terms (eq. ader_dg_method_full) */
  for (int64_t iy = 0; iy < ny; ++iy)
    for (int64_t ix = 0; ix < nx; ++ix) {
      const int64_t c = iy * nx + ix;
      const int64_t cr = iy * nx + wrap2(ix + 1, nx), ct = wrap2(iy + 1, ny) * nx + ix;
      for (int k1 = 0; k1 < n; ++k1)
        for (int k2 = 0; k2 < n; ++k2)
          for (int r = 0; r < M2; ++r) {
            const double fx = b->psi1[k1] * Gx[(cr * n + k2) * M2 + r] - b->psi0[k1] * Gx[(c * n + k2) * M2 + r];
            const double fy = b->psi1[k2] * Gy[(ct * n + k1) * M2 + r] - b->psi0[k2] * Gy[(c * n + k1) * M2 + r];
            u_new[c * us + U2(k1, k2, r)] = vol[c * us + U2(k1, k2, r)] - fx / b->w[k1] - fy / b->w[k2];
          }
    }
  free(q), free(xR), free(xL), free(yR), free(yL), free(vol), free(Gx), free(Gy);
  if (st) st->status = status;
  return status;
}

/* u^{n+1} of the listed cells only (each from its own and its four face
 * neighbours' predictors, the same arithmetic as ob2_dg_step): out[count][n][n][4] */
int ob2_dg_step_cells(const ob_basis* b, const ob_params* p, int64_t nx, int64_t ny, double dx,
                      double dy, double dt, const double* u, const int64_t* cells, int64_t count,
                      double* out) {
  const int n = b->n;
  const double lx = dt / dx, ly = dt / dy;
  const int64_t us = (int64_t)n * n * M2, ts = (int64_t)n * n * M2;
  double* q = malloc(sizeof(double) * n * us);
  double* rec = malloc(sizeof(double) * 5 * 5 * ts);  /* 5 cells x (xR, xL, yR, yL, vol) */
  if (!q || !rec) {
    free(q), free(rec);
    return OB_ERR_ARG;
  }
  int status = OB_OK;
  for (int64_t s = 0; s < count; ++s) {
    const int64_t c = cells[s];
    if (c < 0 || c >= nx * ny) {
      status = OB_ERR_ARG;
      break;
    }
    const int64_t iy = c / nx, ix = c - iy * nx;
    /* this cell, left, right, bottom, top */
    const int64_t nb[5] = {c, iy * nx + wrap2(ix - 1, nx), iy * nx + wrap2(ix + 1, nx),
                           wrap2(iy - 1, ny) * nx + ix, wrap2(iy + 1, ny) * nx + ix};
    for (int j = 0; j < 5; ++j) {
      double* R = rec + j * 5 * ts;
      int it = 0;
      if (cell_record(b, p, lx, ly, u + nb[j] * us, q, R, R + ts, R + 2 * ts, R + 3 * ts, R + 4 * ts,
                      &it) != OB_OK)
        status = OB_ERR_NOT_CONVERGED;
    }
#define REC(j, part) (rec + ((j) * 5 + (part)) * ts)
    double Gx[2][NM * M2], Gy[2][NM * M2]; /* [0]: low face, [1]: high face */
    for (int k = 0; k < n; ++k) {
      double h[4][M2] = {{0}};
      for (int l0 = 0; l0 < n; ++l0) {
        const int64_t o = ((int64_t)l0 * n + k) * M2;
        double H[M2];
        ob2_rusanov(p->gamma, 0, REC(1, 0) + o, REC(0, 1) + o, H);  /* left x-face */
        for (int r = 0; r < M2; ++r) h[0][r] += b->w[l0] * (lx * H[r]);
        ob2_rusanov(p->gamma, 0, REC(0, 0) + o, REC(2, 1) + o, H);  /* right x-face */
        for (int r = 0; r < M2; ++r) h[1][r] += b->w[l0] * (lx * H[r]);
        ob2_rusanov(p->gamma, 1, REC(3, 2) + o, REC(0, 3) + o, H);  /* bottom y-face */
        for (int r = 0; r < M2; ++r) h[2][r] += b->w[l0] * (ly * H[r]);
        ob2_rusanov(p->gamma, 1, REC(0, 2) + o, REC(4, 3) + o, H);  /* top y-face */
        for (int r = 0; r < M2; ++r) h[3][r] += b->w[l0] * (ly * H[r]);
      }
      for (int r = 0; r < M2; ++r) {
        Gx[0][k * M2 + r] = h[0][r];
        Gx[1][k * M2 + r] = h[1][r];
        Gy[0][k * M2 + r] = h[2][r];
        Gy[1][k * M2 + r] = h[3][r];
      }
    }
    for (int k1 = 0; k1 < n; ++k1)
      for (int k2 = 0; k2 < n; ++k2)
        for (int r = 0; r < M2; ++r) {
          const double fx = b->psi1[k1] * Gx[1][k2 * M2 + r] - b->psi0[k1] * Gx[0][k2 * M2 + r];
          const double fy = b->psi1[k2] * Gy[1][k1 * M2 + r] - b->psi0[k2] * Gy[0][k1 * M2 + r];
          out[s * us + U2(k1, k2, r)] = REC(0, 4)[U2(k1, k2, r)] - fx / b->w[k1] - fy / b->w[k2];
        }
#undef REC
  }
  free(q), free(rec);
  return status;
}

/* dt = CFL / (d (2N+1)) min_k (h_k / lambda_k^max), d = 2 (Sec. 1.5), lambda over
 * the Ns x Ns subcell averages (P (x) P) u of every cell; NaN on a non-physical state */
double ob2_dt(const ob_basis* b, const ob_params* p, int64_t nx, int64_t ny, double dx, double dy,
              const double* u) {
  const int n = b->n, Ns = b->Ns;
  const int64_t us = (int64_t)n * n * M2;
  double lam = 0.0;
  for (int64_t c = 0; c < nx * ny; ++c)
    for (int j1 = 0; j1 < Ns; ++j1)
      for (int j2 = 0; j2 < Ns; ++j2) {
        double v[M2];
        for (int r = 0; r < M2; ++r) {
          double acc = 0.0;
          for (int k1 = 0; k1 < n; ++k1)
            for (int k2 = 0; k2 < n; ++k2)
              acc += b->P[j1][k1] * b->P[j2][k2] * u[c * us + U2(k1, k2, r)];
          v[r] = acc;
        }
        const double sx = ob2_speed(p->gamma, v, 0), sy = ob2_speed(p->gamma, v, 1);
        if (isnan(sx) || isnan(sy)) return NAN;
        if (sx / dx > lam) lam = sx / dx;
        if (sy / dy > lam) lam = sy / dy;
      }
  return p->cfl / (2.0 * (2.0 * b->N + 1.0)) / lam;
}

int ob2_solve(const ob_basis* b, const ob_params* p, int64_t nx, int64_t ny, double dx, double dy,
              double* u, double t_end, int64_t max_steps, int64_t* steps_out, double* t_out) {
  if (nx <= 0 || ny <= 0) return OB_ERR_ARG;
  const int64_t cnt = nx * ny * b->n * b->n * M2;
  double* tmp = malloc(sizeof(double) * cnt);
  if (!tmp) return OB_ERR_ARG;
  double t = 0.0;
  int64_t steps = 0;
  int status = OB_OK;
  for (;;) {
    if (t_end > 0.0 && t >= t_end) break;
    if (max_steps > 0 && steps >= max_steps) break;
    double dt = ob2_dt(b, p, nx, ny, dx, dy, u);
    if (!(dt > 0.0) || !isfinite(dt)) {
      status = OB_ERR_NONPHYSICAL;
      break;
    }
    int last = 0;
    if (t_end > 0.0 && t + dt >= t_end) {
      dt = t_end - t;
      last = 1;
    }
    const int rc = ob2_dg_step(b, p, nx, ny, dx, dy, dt, u, tmp, NULL);
    if (rc != OB_OK && rc != OB_ERR_NOT_CONVERGED) {
      status = rc;
      break;
    }
    if (rc == OB_ERR_NOT_CONVERGED) status = rc;
    memcpy(u, tmp, sizeof(double) * cnt);
    t = last ? t_end : t + dt;
    ++steps;
  }
  free(tmp);
  if (steps_out) *steps_out = steps;
  if (t_out) *t_out = t;
  return status;
}
