// ader_ops.h -- operator tables of the LST-DG predictor, the DG corrector, the
// subcell projection and the WENO reconstruction (Popov, arXiv 2409.12483,
// Sec. 1.1 eq. gl_rule / eq. m_and_kappa_matrices / Kronecker forms, Sec. 1.2
// D~, psi, psi~, Sec. 1.4 P, eq. weno_reconstr), built on the host in long double.
//
// Construction (deliberately unlike a textbook monomial route):
//   nodes/weights by Golub-Welsch (Jacobi rotations on the Legendre Jacobi matrix),
//   Lagrange basis in barycentric form, integrals by Gauss-Legendre quadrature,
//   inverses by LU with partial pivoting.
#pragma once

#include <cstdint>

namespace ader {

constexpr int kMaxDeg = 7;
constexpr int kMax3DDegree = 7;           // 3D: N = 7 splits each tau column over a 2-CTA cluster
constexpr int kMaxN = kMaxDeg + 1;        // GL nodes per direction
constexpr int kMaxNs = 2 * kMaxDeg + 1;   // subcells of Sec. 1.4
constexpr int kMaxH = (kMaxN + 1) / 2;    // half rows of the symmetric k~ form
constexpr int kM = 3;                     // conserved variables of 1D Euler
constexpr int kMR = 5;                    // variables of the 1D two-component reacting flow
constexpr int kMN = 4;                    // 1D Euler + non-conservative tracer (rho, m, E, phi)
constexpr int kM2 = 4;                    // conserved variables of 2D Euler (rho, m_x, m_y, E)
constexpr int kM3 = 5;                    // conserved variables of 3D Euler (rho, m_x, m_y, m_z, E)

// Tables in the layout the kernels read (row-major, unused entries zero).
struct OpsD {
  double xi[kMaxN], w[kMaxN], rw[kMaxN];  // GL nodes on [0,1], weights, 1/w
  double psi0[kMaxN], psi1[kMaxN];        // phi_k(0), phi_k(1)
  double kt[kMaxN][kMaxN];                // k~[p][q] = Lambda^-1 Xi = phi_q'(xi_p)
  double kap[kMaxN][kMaxN];               // kappa~ = Upsilon^-1 Lambda
  double kaprow[kMaxN];                   // row sums of kappa~ (= tau nodes: kappa~ 1 = tau)
  double vt[kMaxN][kMaxN];                // D~[k][l] / w_k, D~[k][l] = w_l phi_k'(xi_l)
  double P[kMaxNs][kMaxN];                // P[j][k] = Ns int_{j/Ns}^{(j+1)/Ns} phi_k
  // k~ in even/odd form (the GL nodes are symmetric about 1/2, so
  // k~[n-1-p][n-1-q] = -k~[p][q]); h = n / 2, H = (n + 1) / 2, m = h the middle
  // node of odd n:
  //   ksa[p][q] = (k~[p][q] + k~[p][n-1-q]) / 2, p < h, q < h;  ksa[p][m] = k~[p][m]
  //   ksb[p][q] = (k~[p][q] - k~[p][n-1-q]) / 2, p < H, q < h
  double ksa[kMaxH][kMaxH];
  double ksb[kMaxH][kMaxH];
};

// Float tables; the *lo members hold x - (float)x rounded to float, so that
// hi + lo carries a table entry to ~48 bits (the float-float form).
struct OpsF {
  float kt[kMaxN][kMaxN];
  float kap[kMaxN][kMaxN];
  float kaprow[kMaxN];
  float ktlo[kMaxN][kMaxN];
  float kaplo[kMaxN][kMaxN];
  float kaprowlo[kMaxN];
  float psi0[kMaxN], psi0lo[kMaxN], psi1[kMaxN], psi1lo[kMaxN];
  float w[kMaxN], wlo[kMaxN];
  float vt[kMaxN][kMaxN], vtlo[kMaxN][kMaxN];
  float ksa[kMaxH][kMaxH], ksb[kMaxH][kMaxH];
};

// WENO tables for even N (order N+1), three stencils of N+1 cells.
struct WenoOps {
  int shift[3];                   // first cell of each stencil relative to i
  double lin[3];                  // linear weights lambda_S
  double eps;                     // epsilon of (sigma + eps)^r, r = 8
  double ainv[3][kMaxN][kMaxN];   // nodal values in cell i = ainv[S] * stencil averages
  double mono[kMaxN][kMaxN];      // monomial coefficients in t = 2 xi - 1: a_j = sum_k mono[j][k] c_k
  double smono[kMaxN][kMaxN];     // sigma = sum_{j,l >= 1} a_j smono[j][l] a_l (0 when j + l is odd)
  double amono[3][kMaxN][kMaxN];  // a_j of stencil S from its averages: sum_k amono[S][j][k] v_{S,k} (= mono ainv[S])
  double vnod[kMaxN][kMaxN];      // nodal values from monomial coefficients: c_q = sum_j vnod[q][j] a_j, t_q^j
  float smonof[kMaxN][kMaxN];     // smono, eps and lin rounded to FP32 (the screened weights)
  float epsf, linf[3];
};

struct Basis {
  int N = 0, n = 1, Ns = 1;
  OpsD d{};
  OpsF f{};
  WenoOps weno{};
  // extra host-only tables for inspection
  double dphi[kMaxN][kMaxN]{};    // dphi[k][l] = phi_k'(xi_l)
  double dtil[kMaxN][kMaxN]{};    // D~[k][l]
  double R[kMaxN][kMaxNs]{};      // (P^T P)^-1 P^T: DG coefficients from subcell averages (eq. r_operator)
};

// Returns 0 on success.  weno != 0 also builds the WENO tables (N even, 2 <= N).
int build_basis(int N, bool weno, Basis* out);

}  // namespace ader
