// Host FP64 set-up of the 1D tables of the condensed HDG operator.
//
// arXiv:2007.11891, Sec. 2.2-2.3: the standard matrices of Eq. (element_matrices)
// on the GLL Lagrange basis, L = E + D M^-1 D^T, the generalised eigenpairs
// S^T M S = I, S^T L S = Lambda (Eq. (generalized_eigenvalue_decomposition)),
// the row matrix B_S = S^T B - S^T D M^-1 C (Eq. (hdg_bs)) and the 2x2 face
// matrix H = G + C^T M^-1 C used in Alg. (hdg_op_3d_transformed).
//
// Mirror symmetry: the GLL points are symmetric about 0, so M and L commute
// with the reversal J (J_ij = delta_{i, n-1-j}) and the eigenproblem splits
// into an even and an odd block.  The eigenvectors are computed per block and
// ordered [even modes | odd modes]; then B_S[m][1] = sigma_m B_S[m][0] with
// sigma_m = +1 for even and -1 for odd modes, which the kernels exploit.
#pragma once

namespace hdg {

constexpr int kMaxN = 33;  // degree p <= 32

struct Setup1D {
  int n = 0;                       // p + 1
  int n_even = 0;                  // number of even modes (ceil(n/2))
  double tau_hat = 0.0;
  int mass_lumped = 0;
  double nodes[kMaxN];             // GLL points on [-1, 1]
  double weights[kMaxN];           // GLL weights
  double M[kMaxN * kMaxN];         // row-major n x n
  double D[kMaxN * kMaxN];
  double L[kMaxN * kMaxN];
  double S[kMaxN * kMaxN];         // S[i * n + m]: node i, mode m
  double Lambda[kMaxN];            // eigenvalues, mode order
  double bs[kMaxN];                // c_m = B_S[m][0]
  double h0 = 0.0, h1 = 0.0;       // H = [[h0, h1], [h1, h0]]
  double StM[kMaxN * kMaxN];       // (S^T M)[m * n + i]
  double MS[kMaxN * kMaxN];        // (M S)[i * n + m]
  double St[kMaxN * kMaxN];        // (S^T)[m * n + i]
  double Mdiag_face[kMaxN * kMaxN];// M (for face-mass of Neumann data), row-major
  // residuals of the identities, checked at set-up
  double err_orth = 0.0;           // max |S^T M S - I|
  double err_diag = 0.0;           // max |S^T L S - Lambda|, relative to max Lambda
  double err_parity = 0.0;         // max |B_S[m][1] - sigma_m B_S[m][0]|
};

// Returns 0 on success, nonzero (and a message) on failure.
int build_setup1d(int p, double tau_hat, int mass_lumped, Setup1D* out, const char** msg);

}  // namespace hdg
