// ader_ops.cpp -- host construction of the operator tables (see ader_ops.h).
#include "ader_ops.h"

#include <cmath>
#include <cstring>

namespace ader {
namespace {

using ld = long double;

// Golub-Welsch: eigenvalues of the symmetric Jacobi matrix of the Legendre
// recurrence are the GL nodes on [-1,1]; the squared first components of the
// normalised eigenvectors times mu0 = 2 are the weights.  Eigen-decomposition by
// cyclic Jacobi rotations.
void golub_welsch(int n, ld* x, ld* wts) {
  ld A[kMaxN][kMaxN] = {}, V[kMaxN][kMaxN] = {};
  for (int k = 1; k < n; ++k) {
    const ld beta = (ld)k / sqrtl(4.0L * k * k - 1.0L);
    A[k - 1][k] = A[k][k - 1] = beta;
  }
  for (int i = 0; i < n; ++i) V[i][i] = 1;
  for (int sweep = 0; sweep < 100; ++sweep) {
    ld off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[p][q] * A[p][q];
    if (off < 1e-70L) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const ld apq = A[p][q];
        if (fabsl(apq) < 1e-40L) continue;
        const ld theta = (A[q][q] - A[p][p]) / (2 * apq);
        const ld t = (theta >= 0 ? 1 : -1) / (fabsl(theta) + sqrtl(theta * theta + 1));
        const ld c = 1 / sqrtl(t * t + 1), s = t * c;
        for (int k = 0; k < n; ++k) {
          if (k == p || k == q) continue;
          const ld akp = A[k][p], akq = A[k][q];
          A[k][p] = A[p][k] = c * akp - s * akq;
          A[k][q] = A[q][k] = s * akp + c * akq;
        }
        A[p][p] -= t * apq;
        A[q][q] += t * apq;
        A[p][q] = A[q][p] = 0;
        for (int k = 0; k < n; ++k) {
          const ld vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  int idx[kMaxN];
  for (int i = 0; i < n; ++i) idx[i] = i;
  for (int i = 0; i < n; ++i)  // sort ascending by eigenvalue
    for (int j = i + 1; j < n; ++j)
      if (A[idx[j]][idx[j]] < A[idx[i]][idx[i]]) {
        int tmp = idx[i];
        idx[i] = idx[j];
        idx[j] = tmp;
      }
  for (int i = 0; i < n; ++i) {
    x[i] = A[idx[i]][idx[i]];
    wts[i] = 2 * V[0][idx[i]] * V[0][idx[i]];
  }
}

// LU with partial pivoting: solves A X = B (n x n, m right-hand sides) in place in B.
int lu_solve(int n, ld A[kMaxN][kMaxN], ld B[kMaxN][kMaxN], int m) {
  int perm[kMaxN];
  for (int i = 0; i < n; ++i) perm[i] = i;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (fabsl(A[i][k]) > fabsl(A[piv][k])) piv = i;
    if (A[piv][k] == 0) return -1;
    if (piv != k) {
      for (int j = 0; j < n; ++j) {
        ld t = A[k][j];
        A[k][j] = A[piv][j];
        A[piv][j] = t;
      }
      for (int j = 0; j < m; ++j) {
        ld t = B[k][j];
        B[k][j] = B[piv][j];
        B[piv][j] = t;
      }
    }
    for (int i = k + 1; i < n; ++i) {
      const ld l = A[i][k] / A[k][k];
      A[i][k] = l;
      for (int j = k + 1; j < n; ++j) A[i][j] -= l * A[k][j];
      for (int j = 0; j < m; ++j) B[i][j] -= l * B[k][j];
    }
  }
  for (int j = 0; j < m; ++j)
    for (int i = n - 1; i >= 0; --i) {
      ld s = B[i][j];
      for (int k = i + 1; k < n; ++k) s -= A[i][k] * B[k][j];
      B[i][j] = s / A[i][i];
    }
  return 0;
}

// barycentric Lagrange basis on nodes xi (n of them)
struct Bary {
  int n;
  ld xi[kMaxN], b[kMaxN];
  void init(int nn, const ld* x) {
    n = nn;
    for (int j = 0; j < n; ++j) {
      xi[j] = x[j];
      ld p = 1;
      for (int m = 0; m < n; ++m)
        if (m != j) p *= (x[j] - x[m]);
      b[j] = 1 / p;
    }
  }
  void eval(ld x, ld* phi) const {
    for (int k = 0; k < n; ++k)
      if (x == xi[k]) {
        for (int j = 0; j < n; ++j) phi[j] = (j == k);
        return;
      }
    ld ell = 1;
    for (int m = 0; m < n; ++m) ell *= (x - xi[m]);
    for (int k = 0; k < n; ++k) phi[k] = ell * b[k] / (x - xi[k]);
  }
  // D[k][l] = phi_k'(xi_l)
  void deriv_at_nodes(ld D[kMaxN][kMaxN]) const {
    for (int k = 0; k < n; ++k)
      for (int l = 0; l < n; ++l) {
        if (l != k) {
          D[k][l] = (b[k] / b[l]) / (xi[l] - xi[k]);
        } else {
          ld s = 0;
          for (int m = 0; m < n; ++m)
            if (m != k) s += 1 / (xi[k] - xi[m]);
          D[k][l] = s;
        }
      }
  }
};

// v = hi + lo: hi = v rounded to float, lo = the remainder rounded to float
void split_ff(ld v, float* hi, float* lo) {
  *hi = (float)v;
  *lo = (float)(v - (ld)*hi);
}

ld factorial_ratio(int j, int a) {  // j! / (j-a)!
  ld r = 1;
  for (int i = 0; i < a; ++i) r *= (ld)(j - i);
  return r;
}

}  // namespace

int build_basis(int N, bool weno, Basis* out) {
  if (!out || N < 0 || N > kMaxDeg) return -1;
  std::memset(out, 0, sizeof(*out));
  const int n = N + 1;
  out->N = N;
  out->n = n;
  out->Ns = 2 * N + 1;

  ld x[kMaxN], W[kMaxN], xi[kMaxN], w[kMaxN];
  golub_welsch(n, x, W);
  for (int k = 0; k < n; ++k) {
    xi[k] = (1 + x[k]) / 2;
    w[k] = W[k] / 2;
  }
  Bary B;
  B.init(n, xi);
  ld D[kMaxN][kMaxN];
  B.deriv_at_nodes(D);
  ld ph0[kMaxN], ph1[kMaxN];
  B.eval(0.0L, ph0);
  B.eval(1.0L, ph1);

  // Lambda = diag(w) (GL exact for degree 2N); Xi_kl = int phi_k phi_l' = w_k phi_l'(xi_k)
  ld Xi[kMaxN][kMaxN], Ups[kMaxN][kMaxN], kap[kMaxN][kMaxN];
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) Xi[k][l] = w[k] * D[l][k];
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) Ups[k][l] = ph1[k] * ph1[l] - Xi[l][k];
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) kap[k][l] = (k == l) ? w[k] : 0;
  if (lu_solve(n, Ups, kap, n)) return -2;  // kappa~ = Upsilon^-1 Lambda

  OpsD& d = out->d;
  for (int k = 0; k < n; ++k) {
    ld rs = 0;
    for (int l = 0; l < n; ++l) rs += kap[k][l];
    OpsF& f = out->f;
    d.kaprow[k] = (double)rs;
    split_ff(rs, &f.kaprow[k], &f.kaprowlo[k]);
    d.xi[k] = (double)xi[k];
    d.w[k] = (double)w[k];
    d.rw[k] = (double)(1 / w[k]);
    d.psi0[k] = (double)ph0[k];
    d.psi1[k] = (double)ph1[k];
    split_ff(w[k], &f.w[k], &f.wlo[k]);
    split_ff(ph0[k], &f.psi0[k], &f.psi0lo[k]);
    split_ff(ph1[k], &f.psi1[k], &f.psi1lo[k]);
    for (int l = 0; l < n; ++l) {
      const ld vt = w[l] * D[k][l] / w[k];
      d.kt[k][l] = (double)D[l][k];  // k~ = Lambda^-1 Xi = Dphi^T
      d.kap[k][l] = (double)kap[k][l];
      d.vt[k][l] = (double)vt;
      out->dphi[k][l] = (double)D[k][l];
      out->dtil[k][l] = (double)(w[l] * D[k][l]);
      split_ff(D[l][k], &f.kt[k][l], &f.ktlo[k][l]);
      split_ff(kap[k][l], &f.kap[k][l], &f.kaplo[k][l]);
      split_ff(vt, &f.vt[k][l], &f.vtlo[k][l]);
    }
  }
  // k~ (= Dphi^T) in even/odd form
  {
    const int h = n / 2, H = (n + 1) / 2;
    for (int p = 0; p < H; ++p)
      for (int q = 0; q < H; ++q) {
        ld a = 0, b = 0;
        if (p < h && q < h) a = (D[q][p] + D[n - 1 - q][p]) / 2;
        if (p < h && q == h && H > h) a = D[h][p];
        if (q < h) b = (D[q][p] - D[n - 1 - q][p]) / 2;
        d.ksa[p][q] = (double)a;
        d.ksb[p][q] = (double)b;
        out->f.ksa[p][q] = (float)a;
        out->f.ksb[p][q] = (float)b;
      }
  }
  // subcell projection (Sec. 1.4): P_jk = Ns int_{j/Ns}^{(j+1)/Ns} phi_k = sum_q w_q phi_k((j+xi_q)/Ns)
  for (int j = 0; j < out->Ns; ++j)
    for (int k = 0; k < n; ++k) {
      ld s = 0;
      for (int q = 0; q < n; ++q) {
        ld phi[kMaxN];
        B.eval(((ld)j + xi[q]) / (ld)out->Ns, phi);
        s += w[q] * phi[k];
      }
      d.P[j][k] = (double)s;
    }

  // pseudo-inverse of the subcell projection: R = (P^T P)^-1 P^T (eq. r_operator)
  {
    ld PtP[kMaxN][kMaxN], Pt[kMaxN][kMaxN];
    for (int k = 0; k < n; ++k)
      for (int l = 0; l < n; ++l) {
        ld s = 0;
        for (int j = 0; j < out->Ns; ++j) s += (ld)d.P[j][k] * (ld)d.P[j][l];
        PtP[k][l] = s;
      }
    // solve PtP X = P^T column block by block (n x Ns right-hand sides, in chunks of n)
    for (int j0 = 0; j0 < out->Ns; j0 += n) {
      const int m = (out->Ns - j0) < n ? (out->Ns - j0) : n;
      ld A[kMaxN][kMaxN];
      for (int k = 0; k < n; ++k)
        for (int l = 0; l < n; ++l) A[k][l] = PtP[k][l];
      for (int k = 0; k < n; ++k)
        for (int c = 0; c < m; ++c) Pt[k][c] = (ld)d.P[j0 + c][k];
      if (lu_solve(n, A, Pt, m)) return -6;
      for (int k = 0; k < n; ++k)
        for (int c = 0; c < m; ++c) out->R[k][j0 + c] = (double)Pt[k][c];
    }
  }
  if (weno) {
    if (N < 2 || (N % 2) != 0) return -3;
    WenoOps& wo = out->weno;
    wo.shift[0] = -N / 2;  // central
    wo.shift[1] = -N;      // left-biased
    wo.shift[2] = 0;       // right-biased
    wo.lin[0] = 1.0e5;
    wo.lin[1] = 1.0;
    wo.lin[2] = 1.0;
    wo.eps = 1.0e-14;
    // monomial coefficients in t = 2 xi - 1: solve Vandermonde V a = c, V_qj = t_q^j
    ld Mono[kMaxN][kMaxN];
    {
      ld V[kMaxN][kMaxN];
      for (int q = 0; q < n; ++q) {
        ld tq = 2 * xi[q] - 1, p = 1;
        for (int j = 0; j < n; ++j) {
          V[q][j] = p;
          wo.vnod[q][j] = (double)p;
          p *= tq;
          Mono[q][j] = (q == j);
        }
      }
      if (lu_solve(n, V, Mono, n)) return -5;
      for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) wo.mono[j][k] = (double)Mono[j][k];
    }
    for (int S = 0; S < 3; ++S) {
      ld A[kMaxN][kMaxN], I[kMaxN][kMaxN];
      for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) {
          ld s = 0;  // average of phi_k over the cell [shift+j, shift+j+1]
          for (int q = 0; q < n; ++q) {
            ld phi[kMaxN];
            B.eval((ld)(wo.shift[S] + j) + xi[q], phi);
            s += w[q] * phi[k];
          }
          A[j][k] = s;
          I[j][k] = (j == k);
        }
      if (lu_solve(n, A, I, n)) return -4;
      for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) {
          wo.ainv[S][j][k] = (double)I[j][k];
          ld a = 0;  // mono * ainv[S] in long double
          for (int m = 0; m < n; ++m) a += Mono[j][m] * I[m][k];
          wo.amono[S][j][k] = (double)a;
        }
    }
    // sigma = sum_{a=1..N} int_0^1 (d^a p / d xi^a)^2 d xi, p = sum_j a_j t^j:
    // d^a t^j / d xi^a = 2^a j!/(j-a)! t^(j-a);  int_0^1 d xi = 1/2 int_{-1}^{1} dt
    for (int j = 1; j < n; ++j)
      for (int l = 1; l < n; ++l) {
        ld s = 0;
        for (int a = 1; a <= N; ++a) {
          if (a > j || a > l) continue;
          const int m = j + l - 2 * a;
          if (m % 2) continue;
          s += powl(4.0L, (ld)a) * factorial_ratio(j, a) * factorial_ratio(l, a) / (ld)(m + 1);
        }
        wo.smono[j][l] = (double)s;
        wo.smonof[j][l] = (float)wo.smono[j][l];
      }
    wo.epsf = (float)wo.eps;
    for (int S = 0; S < 3; ++S) wo.linf[S] = (float)wo.lin[S];
  }
  return 0;
}

}  // namespace ader
