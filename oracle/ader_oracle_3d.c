/*
 * ader_oracle_3d.c -- the oracle's ADER-DG scheme for the 3D Euler equations on
 * a periodic Cartesian mesh: the tensor-product LST-DG predictor of Sec. 1.1
 * (eq. lst_dg_predictor_picard with L^xi = kappa~ (x) k~ (x) I (x) I,
 * L^eta = kappa~ (x) I (x) k~ (x) I, L^zeta = kappa~ (x) I (x) I (x) k~,
 * L^0 = delta by eq. ind_prop), the one-step corrector of Sec. 1.2 with x-, y-
 * and z-faces, and the time step of Sec. 1.5 with d = 3.  Plain C, FP64, one
 * cell at a time, in the order of the paper's sums.
 *
 * Layout: state u[cell][k1][k2][k3][r] with cell = (iz ny + iy) nx + ix, k1 the
 * xi node, k2 the eta node, k3 the zeta node, r = (rho, m_x, m_y, m_z, E);
 * predictor q[p0][p1][p2][p3][r] with p0 the tau node (the pass-through index
 * of the paper).
 *
 * TEST INFRASTRUCTURE ONLY: tests, the package's smoke check and the CPU
 * baseline of the benchmark use this file; the library never does.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ader_oracle.h"

#define M3 OB3_M

#define Q3(p0, p1, p2, p3, r) ((((((p0) * n + (p1)) * n + (p2)) * n + (p3)) * M3) + (r))
#define U3(k1, k2, k3, r) (((((k1) * n + (k2)) * n + (k3)) * M3) + (r))

/* fluxes in x, y, z (Sec. 2, eq. system_of_equations in 3D): F[d][r] */
void ob3_flux(double gamma, const double* U, double* F) {
  const double rho = U[0], E = U[4];
  const double v[3] = {U[1] / rho, U[2] / rho, U[3] / rho};
  const double p = (gamma - 1.0) * (E - 0.5 * (U[1] * v[0] + U[2] * v[1] + U[3] * v[2]));
  for (int d = 0; d < 3; ++d) {
    double* f = F + d * M3;
    f[0] = U[1 + d];
    for (int c = 0; c < 3; ++c) f[1 + c] = U[1 + c] * v[d] + (c == d ? p : 0.0);
    f[4] = (E + p) * v[d];
  }
}

/* |u_dir| + c; NaN for a non-physical state */
double ob3_speed(double gamma, const double* U, int dir) {
  const double rho = U[0];
  const double v[3] = {U[1] / rho, U[2] / rho, U[3] / rho};
  const double p = (gamma - 1.0) * (U[4] - 0.5 * (U[1] * v[0] + U[2] * v[1] + U[3] * v[2]));
  if (!(rho > 0.0) || !(p > 0.0)) return NAN;
  return fabs(v[dir]) + sqrt(gamma * p / rho);
}

void ob3_rusanov(double gamma, int dir, const double* a, const double* b, double* H) {
  double Fa[3 * M3], Fb[3 * M3];
  ob3_flux(gamma, a, Fa);
  ob3_flux(gamma, b, Fb);
  const double sa = ob3_speed(gamma, a, dir), sb = ob3_speed(gamma, b, dir);
  const double s = (isnan(sa) || isnan(sb)) ? NAN : (sa > sb ? sa : sb);
  for (int r = 0; r < M3; ++r)
    H[r] = 0.5 * (Fa[dir * M3 + r] + Fb[dir * M3 + r]) - 0.5 * s * (b[r] - a[r]);
}

int ob3_predict_cell(const ob_basis* b, const ob_params* p, double lx, double ly, double lz,
                     const double* u, double* q, int* iters) {
  const int n = b->n;
  const int cnt = n * n * n * n * M3;
  const double lam[3] = {lx, ly, lz};
  double* f = malloc(sizeof(double) * 3 * cnt); /* f[d][node][r] */
  double* s = malloc(sizeof(double) * cnt);
  double* qn = malloc(sizeof(double) * cnt);
  if (!f || !s || !qn) {
    free(f), free(s), free(qn);
    return OB_ERR_ARG;
  }
  for (int p0 = 0; p0 < n; ++p0)
    for (int p1 = 0; p1 < n; ++p1)
      for (int p2 = 0; p2 < n; ++p2)
        for (int p3 = 0; p3 < n; ++p3)
          for (int r = 0; r < M3; ++r) q[Q3(p0, p1, p2, p3, r)] = u[U3(p1, p2, p3, r)];
  const int cap = p->fixed_iter > 0 ? p->fixed_iter : p->max_iter;
  int it = 0, converged = 0;
  while (it < cap) {
    ++it;
    /* rescaled fluxes (dt/dx_d) F_d(q) at every space-time node */
    for (int p0 = 0; p0 < n; ++p0)
      for (int p1 = 0; p1 < n; ++p1)
        for (int p2 = 0; p2 < n; ++p2)
          for (int p3 = 0; p3 < n; ++p3) {
            double F[3 * M3];
            ob3_flux(p->gamma, &q[Q3(p0, p1, p2, p3, 0)], F);
            for (int d = 0; d < 3; ++d)
              for (int r = 0; r < M3; ++r) f[d * cnt + Q3(p0, p1, p2, p3, r)] = lam[d] * F[d * M3 + r];
          }
    /* k~ along xi, eta and zeta on the x-, y- and z-fluxes */
    for (int p0 = 0; p0 < n; ++p0)
      for (int p1 = 0; p1 < n; ++p1)
        for (int p2 = 0; p2 < n; ++p2)
          for (int p3 = 0; p3 < n; ++p3)
            for (int r = 0; r < M3; ++r) {
              double acc = 0.0;
              for (int m = 0; m < n; ++m) acc += b->kt[p1][m] * f[0 * cnt + Q3(p0, m, p2, p3, r)];
              for (int m = 0; m < n; ++m) acc += b->kt[p2][m] * f[1 * cnt + Q3(p0, p1, m, p3, r)];
              for (int m = 0; m < n; ++m) acc += b->kt[p3][m] * f[2 * cnt + Q3(p0, p1, p2, m, r)];
              s[Q3(p0, p1, p2, p3, r)] = acc;
            }
    /* kappa~ along tau */
    for (int p0 = 0; p0 < n; ++p0)
      for (int p1 = 0; p1 < n; ++p1)
        for (int p2 = 0; p2 < n; ++p2)
          for (int p3 = 0; p3 < n; ++p3)
            for (int r = 0; r < M3; ++r) {
              double acc = 0.0;
              for (int m = 0; m < n; ++m) acc += b->kap[p0][m] * s[Q3(m, p1, p2, p3, r)];
              qn[Q3(p0, p1, p2, p3, r)] = u[U3(p1, p2, p3, r)] - acc;
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
  free(f), free(s), free(qn);
  return converged ? OB_OK : OB_ERR_NOT_CONVERGED;
}

static int64_t wrap3(int64_t i, int64_t n) { return ((i % n) + n) % n; }

/* the predictor at the face of direction d (side 1: coordinate 1, side 0:
 * coordinate 0) for tau node l0 and transverse nodes (a, b) in the order of
 * the remaining two directions: tr[l0][a][b][r] */
static void face_trace(const ob_basis* b, const double* q, int d, int side, double* tr) {
  const int n = b->n;
  const double* psi = side ? b->psi1 : b->psi0;
  for (int l0 = 0; l0 < n; ++l0)
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c)
        for (int r = 0; r < M3; ++r) {
          double acc = 0.0;
          for (int m = 0; m < n; ++m) {
            int i1 = m, i2 = a, i3 = c;       /* d = 0: (m, a, c) */
            if (d == 1) i1 = a, i2 = m, i3 = c; /* d = 1: (a, m, c) */
            if (d == 2) i1 = a, i2 = c, i3 = m; /* d = 2: (a, c, m) */
            acc += psi[m] * q[Q3(l0, i1, i2, i3, r)];
          }
          tr[((l0 * n + a) * n + c) * M3 + r] = acc;
        }
}

/* predictor, six face traces [d][side][l0][a][c][r] and volume term of one cell
 * (fbar: scratch of 3 n^3 M3 doubles) */
static int cell_record3(const ob_basis* b, const ob_params* p, const double* lam, const double* uc,
                        double* q, double* fbar, double* trc, double* vol, int* iters) {
  const int n = b->n;
  const int64_t us = (int64_t)n * n * n * M3, ts = us;
  const int status = ob3_predict_cell(b, p, lam[0], lam[1], lam[2], uc, q, iters);
  for (int d = 0; d < 3; ++d)
    for (int side = 0; side < 2; ++side) face_trace(b, q, d, side, trc + (d * 2 + side) * ts);
  /* volume terms: time-averaged rescaled fluxes, D~ along each direction */
  for (int i = 0; i < 3 * us; ++i) fbar[i] = 0.0;
  for (int l0 = 0; l0 < n; ++l0)
    for (int l1 = 0; l1 < n; ++l1)
      for (int l2 = 0; l2 < n; ++l2)
        for (int l3 = 0; l3 < n; ++l3) {
          double F[3 * M3];
          ob3_flux(p->gamma, &q[Q3(l0, l1, l2, l3, 0)], F);
          for (int d = 0; d < 3; ++d)
            for (int r = 0; r < M3; ++r)
              fbar[d * us + U3(l1, l2, l3, r)] += b->w[l0] * (lam[d] * F[d * M3 + r]);
        }
  for (int k1 = 0; k1 < n; ++k1)
    for (int k2 = 0; k2 < n; ++k2)
      for (int k3 = 0; k3 < n; ++k3)
        for (int r = 0; r < M3; ++r) {
          double ax = 0.0, ay = 0.0, az = 0.0;
          for (int l = 0; l < n; ++l) {
            ax += b->dt_m[k1][l] * fbar[0 * us + U3(l, k2, k3, r)];
            ay += b->dt_m[k2][l] * fbar[1 * us + U3(k1, l, k3, r)];
            az += b->dt_m[k3][l] * fbar[2 * us + U3(k1, k2, l, r)];
          }
          vol[U3(k1, k2, k3, r)] =
              uc[U3(k1, k2, k3, r)] + ax / b->w[k1] + ay / b->w[k2] + az / b->w[k3];
        }
  return status;
}

int ob3_dg_step(const ob_basis* b, const ob_params* p, int64_t nx, int64_t ny, int64_t nz,
                double dx, double dy, double dz, double dt, const double* u, double* u_new,
                ob_stats* st) {
  if (nx <= 0 || ny <= 0 || nz <= 0) return OB_ERR_ARG;
  const int n = b->n;
  const int64_t nc = nx * ny * nz;
  const double lam[3] = {dt / dx, dt / dy, dt / dz};
  const int64_t us = (int64_t)n * n * n * M3, ts = (int64_t)n * n * n * M3;
  double* q = malloc(sizeof(double) * n * us);
  double* trc = malloc(sizeof(double) * nc * 6 * ts); /* [cell][d][side][l0][a][c][r] */
  double* vol = malloc(sizeof(double) * nc * us);
  double* G = malloc(sizeof(double) * nc * 3 * n * n * M3); /* low face of each cell per d */
  double* fbar = malloc(sizeof(double) * 3 * us);
  if (!q || !trc || !vol || !G || !fbar) {
    free(q), free(trc), free(vol), free(G), free(fbar);
    return OB_ERR_ARG;
  }
  if (st) memset(st, 0, sizeof(*st));
  int status = OB_OK;
  for (int64_t c = 0; c < nc; ++c) {
    int it = 0;
    if (cell_record3(b, p, lam, u + c * us, q, fbar, trc + c * 6 * ts, vol + c * us, &it) != OB_OK)
      status = OB_ERR_NOT_CONVERGED;
    if (st) {
      if (st->cells == 0 || it > st->max_iters) st->max_iters = it;
      if (st->cells == 0 || it < st->min_iters) st->min_iters = it;
      st->mean_iters = (st->mean_iters * (double)st->cells + it) / (double)(st->cells + 1);
      st->cells += 1;
    }
  }
  /* time-integrated Rusanov fluxes through the low face of each cell per direction */
  for (int64_t iz = 0; iz < nz; ++iz)
    for (int64_t iy = 0; iy < ny; ++iy)
      for (int64_t ix = 0; ix < nx; ++ix) {
        const int64_t c = (iz * ny + iy) * nx + ix;
        const int64_t lo[3] = {(iz * ny + iy) * nx + wrap3(ix - 1, nx),
                               (iz * ny + wrap3(iy - 1, ny)) * nx + ix,
                               (wrap3(iz - 1, nz) * ny + iy) * nx + ix};
        for (int d = 0; d < 3; ++d)
          for (int a = 0; a < n; ++a)
            for (int e = 0; e < n; ++e) {
              double h[M3] = {0};
              for (int l0 = 0; l0 < n; ++l0) {
                double H[M3];
                const int64_t o = ((int64_t)(l0 * n + a) * n + e) * M3;
                ob3_rusanov(p->gamma, d, trc + (lo[d] * 6 + d * 2 + 1) * ts + o,
                            trc + (c * 6 + d * 2 + 0) * ts + o, H);
                for (int r = 0; r < M3; ++r) h[r] += b->w[l0] * (lam[d] * H[r]);
              }
              for (int r = 0; r < M3; ++r) G[(((c * 3 + d) * n + a) * n + e) * M3 + r] = h[r];
            }
      }
  /* u^{n+1} = volume terms - face terms (eq. ader_dg_method_full) */
  for (int64_t iz = 0; iz < nz; ++iz)
    for (int64_t iy = 0; iy < ny; ++iy)
      for (int64_t ix = 0; ix < nx; ++ix) {
        const int64_t c = (iz * ny + iy) * nx + ix;
        const int64_t hi[3] = {(iz * ny + iy) * nx + wrap3(ix + 1, nx),
                               (iz * ny + wrap3(iy + 1, ny)) * nx + ix,
                               (wrap3(iz + 1, nz) * ny + iy) * nx + ix};
        for (int k1 = 0; k1 < n; ++k1)
          for (int k2 = 0; k2 < n; ++k2)
            for (int k3 = 0; k3 < n; ++k3)
              for (int r = 0; r < M3; ++r) {
                /* direction d: own node k_d, transverse nodes in order */
                const int kk[3] = {k1, k2, k3};
                const int ta[3] = {k2, k1, k1}, tb[3] = {k3, k3, k2};
                double val = vol[c * us + U3(k1, k2, k3, r)];
                for (int d = 0; d < 3; ++d) {
                  const double gh = G[(((hi[d] * 3 + d) * n + ta[d]) * n + tb[d]) * M3 + r];
                  const double gl = G[(((c * 3 + d) * n + ta[d]) * n + tb[d]) * M3 + r];
                  val -= (b->psi1[kk[d]] * gh - b->psi0[kk[d]] * gl) / b->w[kk[d]];
                }
                u_new[c * us + U3(k1, k2, k3, r)] = val;
              }
      }
  free(q), free(trc), free(vol), free(G), free(fbar);
  if (st) st->status = status;
  return status;
}

/* u^{n+1} of the listed cells only (each from its own and its six face
 * neighbours' predictors, the same arithmetic as ob3_dg_step): out[count][n^3][5] */
int ob3_dg_step_cells(const ob_basis* b, const ob_params* p, int64_t nx, int64_t ny, int64_t nz,
                      double dx, double dy, double dz, double dt, const double* u,
                      const int64_t* cells, int64_t count, double* out) {
  const int n = b->n;
  const double lam[3] = {dt / dx, dt / dy, dt / dz};
  const int64_t us = (int64_t)n * n * n * M3, ts = us;
  double* q = malloc(sizeof(double) * n * us);
  double* fbar = malloc(sizeof(double) * 3 * us);
  double* trc = malloc(sizeof(double) * 7 * 6 * ts);
  double* vol = malloc(sizeof(double) * us);
  double* tmpv = malloc(sizeof(double) * us);
  if (!q || !fbar || !trc || !vol || !tmpv) {
    free(q), free(fbar), free(trc), free(vol), free(tmpv);
    return OB_ERR_ARG;
  }
  int status = OB_OK;
  for (int64_t s = 0; s < count; ++s) {
    const int64_t c = cells[s];
    if (c < 0 || c >= nx * ny * nz) {
      status = OB_ERR_ARG;
      break;
    }
    const int64_t plane = nx * ny, iz = c / plane, iy = (c - iz * plane) / nx,
                  ix = c - iz * plane - iy * nx;
    /* this cell, then low / high neighbour per direction */
    const int64_t nb[7] = {c,
                           (iz * ny + iy) * nx + wrap3(ix - 1, nx), (iz * ny + iy) * nx + wrap3(ix + 1, nx),
                           (iz * ny + wrap3(iy - 1, ny)) * nx + ix, (iz * ny + wrap3(iy + 1, ny)) * nx + ix,
                           (wrap3(iz - 1, nz) * ny + iy) * nx + ix, (wrap3(iz + 1, nz) * ny + iy) * nx + ix};
    for (int j = 0; j < 7; ++j) {
      int it = 0;
      if (cell_record3(b, p, lam, u + nb[j] * us, q, fbar, trc + j * 6 * ts, j == 0 ? vol : tmpv,
                       &it) != OB_OK)
        status = OB_ERR_NOT_CONVERGED;
    }
    for (int k1 = 0; k1 < n; ++k1)
      for (int k2 = 0; k2 < n; ++k2)
        for (int k3 = 0; k3 < n; ++k3)
          for (int r = 0; r < M3; ++r) {
            const int kk[3] = {k1, k2, k3};
            const int ta[3] = {k2, k1, k1}, tb[3] = {k3, k3, k2};
            double val = vol[U3(k1, k2, k3, r)];
            for (int d = 0; d < 3; ++d) {
              double gl = 0.0, gh = 0.0;
              for (int l0 = 0; l0 < n; ++l0) {
                double H[M3];
                const int64_t o = ((int64_t)(l0 * n + ta[d]) * n + tb[d]) * M3;
                /* low face: high side of the low neighbour against this cell's low side */
                ob3_rusanov(p->gamma, d, trc + ((1 + 2 * d) * 6 + d * 2 + 1) * ts + o,
                            trc + (0 * 6 + d * 2 + 0) * ts + o, H);
                gl += b->w[l0] * (lam[d] * H[r]);
                ob3_rusanov(p->gamma, d, trc + (0 * 6 + d * 2 + 1) * ts + o,
                            trc + ((2 + 2 * d) * 6 + d * 2 + 0) * ts + o, H);
                gh += b->w[l0] * (lam[d] * H[r]);
              }
              val -= (b->psi1[kk[d]] * gh - b->psi0[kk[d]] * gl) / b->w[kk[d]];
            }
            out[s * us + U3(k1, k2, k3, r)] = val;
          }
  }
  free(q), free(fbar), free(trc), free(vol), free(tmpv);
  return status;
}

/* dt = CFL / (3 (2N+1)) min_d (h_d / lambda_d) over the Ns^3 subcell averages */
double ob3_dt(const ob_basis* b, const ob_params* p, int64_t nx, int64_t ny, int64_t nz, double dx,
              double dy, double dz, const double* u) {
  const int n = b->n, Ns = b->Ns;
  const int64_t us = (int64_t)n * n * n * M3;
  const double h[3] = {dx, dy, dz};
  double lam = 0.0;
  for (int64_t c = 0; c < nx * ny * nz; ++c)
    for (int j1 = 0; j1 < Ns; ++j1)
      for (int j2 = 0; j2 < Ns; ++j2)
        for (int j3 = 0; j3 < Ns; ++j3) {
          double v[M3];
          for (int r = 0; r < M3; ++r) {
            double acc = 0.0;
            for (int k1 = 0; k1 < n; ++k1)
              for (int k2 = 0; k2 < n; ++k2)
                for (int k3 = 0; k3 < n; ++k3)
                  acc += b->P[j1][k1] * b->P[j2][k2] * b->P[j3][k3] * u[c * us + U3(k1, k2, k3, r)];
            v[r] = acc;
          }
          for (int d = 0; d < 3; ++d) {
            const double s = ob3_speed(p->gamma, v, d);
            if (isnan(s)) return NAN;
            if (s / h[d] > lam) lam = s / h[d];
          }
        }
  return p->cfl / (3.0 * (2.0 * b->N + 1.0)) / lam;
}

int ob3_solve(const ob_basis* b, const ob_params* p, int64_t nx, int64_t ny, int64_t nz, double dx,
              double dy, double dz, double* u, double t_end, int64_t max_steps, int64_t* steps_out,
              double* t_out) {
  if (nx <= 0 || ny <= 0 || nz <= 0) return OB_ERR_ARG;
  const int64_t cnt = nx * ny * nz * b->n * b->n * b->n * M3;
  double* tmp = malloc(sizeof(double) * cnt);
  if (!tmp) return OB_ERR_ARG;
  double t = 0.0;
  int64_t steps = 0;
  int status = OB_OK;
  for (;;) {
    if (t_end > 0.0 && t >= t_end) break;
    if (max_steps > 0 && steps >= max_steps) break;
    double dt = ob3_dt(b, p, nx, ny, nz, dx, dy, dz, u);
    if (!(dt > 0.0) || !isfinite(dt)) {
      status = OB_ERR_NONPHYSICAL;
      break;
    }
    int last = 0;
    if (t_end > 0.0 && t + dt >= t_end) {
      dt = t_end - t;
      last = 1;
    }
    const int rc = ob3_dg_step(b, p, nx, ny, nz, dx, dy, dz, dt, u, tmp, NULL);
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
