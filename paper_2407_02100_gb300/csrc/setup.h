// Host-side set-up math of the smoother library (FP64, runs once per
// problem): Gauss-Lobatto support points, Gauss quadrature, the 1D reference
// mass/stiffness matrices of a unit cell, the two-cell patch matrices and
// their generalised eigendecomposition (fast diagonalisation, App. A.3), and
// the 1D embedding prolongation of one coarse cell (Sec. 2).
#pragma once
#include <vector>

namespace gmg {

constexpr int kMaxDegree = 8;

// k+1 Gauss-Lobatto points on [0, 1], ascending.
std::vector<double> gauss_lobatto(int k);
// n-point Gauss-Legendre rule on [0, 1].
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
// Lagrange basis on `nodes`, value (deriv = 0) or derivative (deriv = 1) of
// basis function p at t.
double lagrange(const std::vector<double>& nodes, int p, double t, int deriv);

// Unit-cell 1D matrices ((k+1) x (k+1), row-major): M[i][j] = int phi_i phi_j,
// K[i][j] = int phi_i' phi_j' on [0, 1].
void cell_matrices_1d(int k, std::vector<double>& M, std::vector<double>& K);

// 1D mesh of `ncells` unit cells: matrices restricted to rows `r0..r0+nr-1`
// and columns `c0..c0+nc-1` of the assembled (ncells k + 1)^2 matrix.
void assembled_1d(int k, int ncells, int r0, int nr, int c0, int nc,
                  std::vector<double>& M, std::vector<double>& K);

// Generalised symmetric eigenproblem K t = lambda M t, M SPD, n x n
// row-major: T (row-major, column j = eigenvector j) with T^T M T = I and
// T^T K T = diag(lambda).  Cholesky of M, then cyclic Jacobi on
// L^{-1} K L^{-T}.  Returns false if M is not positive definite.
bool generalized_eigen(int n, const std::vector<double>& M, const std::vector<double>& K,
                       std::vector<double>& T, std::vector<double>& lambda);

// Same eigenproblem for matrices that commute with the reflection
// i -> n-1-i (n odd), solved separately on the even and the odd subspace so
// that the eigenvectors are exactly mirror-symmetric: columns 0..(n-1)/2 of
// T are even (T[n-1-j][i] = T[j][i]), the remaining (n-1)/2 columns are odd
// (T[n-1-j][i] = -T[j][i], zero at the centre row).  Lambda follows the same
// order.
bool generalized_eigen_mirror(int n, const std::vector<double>& M, const std::vector<double>& K,
                              std::vector<double>& T, std::vector<double>& lambda);

// Interior stiffness matrix (dense, row-major, interior nodes x fastest) of
// -div(a grad u) on a uniform mesh of n cells of width h = 1/n with one
// coefficient per cell (coef: n^dim values, c_0 fastest).
void assemble_dense_var(int dim, int k, int n, const double* coef, std::vector<double>& A);

// Inverse of a symmetric positive definite matrix (Cholesky); false if not SPD.
bool spd_inverse(int n, const std::vector<double>& A, std::vector<double>& Ainv);

// Embedding prolongation of one coarse unit cell split in two fine cells:
// P[r][p] = phi^coarse_p(x_r) for the 2k+1 fine nodes r of the coarse cell
// ((2k+1) x (k+1), row-major).
void prolongation_cell_1d(int k, std::vector<double>& P);

}  // namespace gmg
