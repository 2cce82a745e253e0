// Host FP64 set-up of the 1D tables (see setup1d.h for what and why).
#include "setup1d.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace hdg {
namespace {

using Mat = std::vector<double>;  // row-major

// Legendre P_k, P_k' at x by the three-term recurrence
// (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1},  P_{k+1}' = P_{k-1}' + (2k+1) P_k.
void legendre(int k, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (k == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int m = 1; m < k; ++m) {
    double p2 = ((2.0 * m + 1.0) * x * p1 - m * p0) / (m + 1.0);
    double d2 = d0 + (2.0 * m + 1.0) * p1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *P = p1; *dP = d1;
}

// GLL points: +-1 and the roots of P_p' (Newton with P_p'' from the Legendre
// equation (1 - x^2) P'' = 2 x P' - p (p+1) P); weights 2 / (p (p+1) P_p^2).
void gll(int n, double* x, double* w) {
  const int p = n - 1;
  x[0] = -1.0; x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double t = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, t, &P, &dP);
      double ddP = (2.0 * t * dP - p * (p + 1.0) * P) / (1.0 - t * t);
      double dt = dP / ddP;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = t;
  }
  for (int i = 0; i < n; ++i) {
    double P, dP;
    legendre(p, x[i], &P, &dP);
    w[i] = 2.0 / (p * (p + 1.0) * P * P);
  }
  // exact mirror symmetry of the point set
  for (int i = 0; i < n / 2; ++i) {
    double a = 0.5 * (x[n - 1 - i] - x[i]);
    x[i] = -a; x[n - 1 - i] = a;
    double b = 0.5 * (w[i] + w[n - 1 - i]);
    w[i] = b; w[n - 1 - i] = b;
  }
  if (n % 2) x[n / 2] = 0.0;
}

// Gauss-Legendre rule: roots of P_q by Newton, weights 2 / ((1 - x^2) P_q'^2).
void gauss(int q, double* x, double* w) {
  for (int i = 0; i < q; ++i) {
    double t = -std::cos(M_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(q, t, &P, &dP);
      double dt = P / dP;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double P, dP;
    legendre(q, t, &P, &dP);
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dP * dP);
  }
}

// Lagrange basis on `nodes` at t: values v[i] and derivatives dv[i].
void lagrange(int n, const double* nodes, double t, double* v, double* dv) {
  for (int i = 0; i < n; ++i) {
    double val = 1.0, der = 0.0;
    for (int m = 0; m < n; ++m) {
      if (m == i) continue;
      double fac = 1.0 / (nodes[i] - nodes[m]);
      der = der * (t - nodes[m]) * fac + val * fac;
      val *= (t - nodes[m]) * fac;
    }
    v[i] = val; dv[i] = der;
  }
}

// Cholesky A = R R^T (R lower), in place in R.  Returns false if not SPD.
bool cholesky(int n, const Mat& A, Mat& R) {
  R.assign(n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= R[j * n + k] * R[j * n + k];
    if (!(s > 0.0)) return false;
    R[j * n + j] = std::sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= R[i * n + k] * R[j * n + k];
      R[i * n + j] = t / R[j * n + j];
    }
  }
  return true;
}

// Solve A X = B (A SPD, n x n; B n x m) via Cholesky.
bool spd_solve(int n, const Mat& A, int m, const Mat& B, Mat& X) {
  Mat R;
  if (!cholesky(n, A, R)) return false;
  X = B;
  for (int c = 0; c < m; ++c) {
    for (int i = 0; i < n; ++i) {            // R y = b
      double t = X[i * m + c];
      for (int k = 0; k < i; ++k) t -= R[i * n + k] * X[k * m + c];
      X[i * m + c] = t / R[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {       // R^T x = y
      double t = X[i * m + c];
      for (int k = i + 1; k < n; ++k) t -= R[k * n + i] * X[k * m + c];
      X[i * m + c] = t / R[i * n + i];
    }
  }
  return true;
}

// Cyclic Jacobi eigen-decomposition of a symmetric matrix (Golub & Van Loan,
// "Matrix Computations", Sec. 8.5): A = V diag(ev) V^T.
void jacobi_eigen(int n, Mat A, Mat& V, std::vector<double>& ev) {
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += A[i * n + j] * A[i * n + j];
        if (i != j) off += A[i * n + j] * A[i * n + j];
      }
    if (off <= 1e-32 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (apq == 0.0) continue;
        double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {        // A <- A J (columns p, q)
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {        // A <- J^T A (rows p, q)
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {        // V <- V J
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  ev.resize(n);
  for (int i = 0; i < n; ++i) ev[i] = A[i * n + i];
}

// Generalised eigenpairs of (Lb, Mb) restricted to span(P) (n x k basis):
// returns columns S_blk (n x k) with S^T M S = I, S^T L S = diag(mu), ascending.
bool block_eigen(int n, int k, const Mat& P, const Mat& M, const Mat& L, Mat& Sblk,
                 std::vector<double>& mu) {
  Mat Mk(k * k, 0.0), Lk(k * k, 0.0);
  for (int a = 0; a < k; ++a)
    for (int b = 0; b < k; ++b) {
      double sm = 0.0, sl = 0.0;
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          sm += P[i * k + a] * M[i * n + j] * P[j * k + b];
          sl += P[i * k + a] * L[i * n + j] * P[j * k + b];
        }
      Mk[a * k + b] = sm; Lk[a * k + b] = sl;
    }
  Mat R;
  if (!cholesky(k, Mk, R)) return false;
  // A = R^-1 Lk R^-T
  Mat X(k * k), A(k * k);
  for (int c = 0; c < k; ++c)                 // X = R^-1 Lk  (column c)
    for (int i = 0; i < k; ++i) {
      double t = Lk[i * k + c];
      for (int m = 0; m < i; ++m) t -= R[i * k + m] * X[m * k + c];
      X[i * k + c] = t / R[i * k + i];
    }
  for (int r = 0; r < k; ++r)                 // A = X R^-T  (row r: solve R a = x_r)
    for (int i = 0; i < k; ++i) {
      double t = X[r * k + i];
      for (int m = 0; m < i; ++m) t -= R[i * k + m] * A[r * k + m];
      A[r * k + i] = t / R[i * k + i];
    }
  for (int a = 0; a < k; ++a)                 // symmetrise round-off
    for (int b = a + 1; b < k; ++b) {
      double s = 0.5 * (A[a * k + b] + A[b * k + a]);
      A[a * k + b] = s; A[b * k + a] = s;
    }
  Mat V;
  std::vector<double> ev;
  jacobi_eigen(k, A, V, ev);
  std::vector<int> order(k);
  for (int i = 0; i < k; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return ev[a] < ev[b]; });
  // W = R^-T V  (back substitution with R^T upper)
  Mat W(k * k);
  for (int c = 0; c < k; ++c)
    for (int i = k - 1; i >= 0; --i) {
      double t = V[i * k + c];
      for (int m = i + 1; m < k; ++m) t -= R[m * k + i] * W[m * k + c];
      W[i * k + c] = t / R[i * k + i];
    }
  Sblk.assign(n * k, 0.0);
  mu.resize(k);
  for (int c = 0; c < k; ++c) {
    int src = order[c];
    mu[c] = ev[src];
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int a = 0; a < k; ++a) s += P[i * k + a] * W[a * k + src];
      Sblk[i * k + c] = s;
    }
  }
  return true;
}

}  // namespace

int build_setup1d(int p, double tau_hat, int mass_lumped, Setup1D* out, const char** msg) {
  static const char* kOk = "";
  *msg = kOk;
  if (p < 1 || p + 1 > kMaxN) { *msg = "degree p must be in 1..32"; return 1; }
  if (!(tau_hat > 0.0)) { *msg = "tau_hat must be > 0"; return 1; }
  Setup1D& s = *out;
  s = Setup1D();
  const int n = p + 1;
  s.n = n;
  s.tau_hat = tau_hat;
  s.mass_lumped = mass_lumped;
  gll(n, s.nodes, s.weights);

  // M (exact: Gauss rule with n+1 points, exact for degree 2n+1) and D
  const int q = n + 1;
  double tq[kMaxN + 1], wq[kMaxN + 1];
  gauss(q, tq, wq);
  Mat V(q * n), dV(q * n);
  for (int a = 0; a < q; ++a) lagrange(n, s.nodes, tq[a], &V[a * n], &dV[a * n]);
  Mat M(n * n, 0.0), D(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double sm = 0.0, sd = 0.0;
      for (int a = 0; a < q; ++a) {
        sm += wq[a] * V[a * n + i] * V[a * n + j];
        sd += wq[a] * V[a * n + i] * dV[a * n + j];
      }
      M[i * n + j] = sm;
      D[i * n + j] = sd;
    }
  if (mass_lumped) {
    std::fill(M.begin(), M.end(), 0.0);
    for (int i = 0; i < n; ++i) M[i * n + i] = s.weights[i];
  }
  // mirror-symmetrise M (exact in arithmetic; removes round-off asymmetry)
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double a = 0.5 * (M[i * n + j] + M[(n - 1 - i) * n + (n - 1 - j)]);
      M[i * n + j] = a;
    }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double a = 0.5 * (M[i * n + j] + M[j * n + i]);
      M[i * n + j] = a; M[j * n + i] = a;
    }

  // boundary matrices on the GLL basis: phi_i(-1) = delta_{i0}, phi_i(1) = delta_{i,n-1}
  Mat E(n * n, 0.0), Bm(n * 2, 0.0), Cm(n * 2, 0.0);
  E[0] = tau_hat;
  E[(n - 1) * n + (n - 1)] = tau_hat;
  Bm[0 * 2 + 0] = -tau_hat;
  Bm[(n - 1) * 2 + 1] = -tau_hat;
  Cm[0 * 2 + 0] = -1.0;
  Cm[(n - 1) * 2 + 1] = 1.0;

  // L = E + D M^-1 D^T
  Mat Dt(n * n), MinvDt;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Dt[i * n + j] = D[j * n + i];
  if (!spd_solve(n, M, n, Dt, MinvDt)) { *msg = "mass matrix not SPD"; return 2; }
  Mat L(n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double t = E[i * n + j];
      for (int k = 0; k < n; ++k) t += D[i * n + k] * MinvDt[k * n + j];
      L[i * n + j] = t;
    }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double a = 0.5 * (L[i * n + j] + L[j * n + i]);
      L[i * n + j] = a; L[j * n + i] = a;
    }

  // parity-split generalised eigen-decomposition
  const int ne = (n + 1) / 2, no = n / 2;
  s.n_even = ne;
  const double r2 = 1.0 / std::sqrt(2.0);
  Mat Pe(n * ne, 0.0), Po(n * std::max(no, 1), 0.0);
  for (int i = 0; i < n / 2; ++i) {
    Pe[i * ne + i] = r2; Pe[(n - 1 - i) * ne + i] = r2;
    Po[i * no + i] = r2; Po[(n - 1 - i) * no + i] = -r2;
  }
  if (n % 2) Pe[(n / 2) * ne + (ne - 1)] = 1.0;
  Mat Se, So;
  std::vector<double> mue, muo;
  if (!block_eigen(n, ne, Pe, M, L, Se, mue)) { *msg = "even eigenblock failed"; return 3; }
  if (no > 0 && !block_eigen(n, no, Po, M, L, So, muo)) { *msg = "odd eigenblock failed"; return 3; }
  for (int i = 0; i < n; ++i) {
    for (int m = 0; m < ne; ++m) s.S[i * n + m] = Se[i * ne + m];
    for (int m = 0; m < no; ++m) s.S[i * n + ne + m] = So[i * no + m];
  }
  for (int m = 0; m < ne; ++m) s.Lambda[m] = mue[m];
  for (int m = 0; m < no; ++m) s.Lambda[ne + m] = muo[m];

  // B_S = S^T (B - D M^-1 C); H = G + C^T M^-1 C
  Mat MinvC;
  if (!spd_solve(n, M, 2, Cm, MinvC)) { *msg = "mass solve failed"; return 2; }
  double v0[kMaxN], v1[kMaxN];
  for (int i = 0; i < n; ++i) {
    double t0 = Bm[i * 2 + 0], t1 = Bm[i * 2 + 1];
    for (int k = 0; k < n; ++k) {
      t0 -= D[i * n + k] * MinvC[k * 2 + 0];
      t1 -= D[i * n + k] * MinvC[k * 2 + 1];
    }
    v0[i] = t0; v1[i] = t1;
  }
  double maxc = 0.0;
  for (int m = 0; m < n; ++m) {
    double b0 = 0.0, b1 = 0.0;
    for (int i = 0; i < n; ++i) { b0 += s.S[i * n + m] * v0[i]; b1 += s.S[i * n + m] * v1[i]; }
    // sign convention of the face eigenbasis: every mode couples to the low
    // face with B_S[m][0] > 0 (|B_S[m][0]| stays near pi/2 or above for every
    // degree, so the sign is well defined, unlike an endpoint value of S)
    if (b0 < 0.0) {
      for (int i = 0; i < n; ++i) s.S[i * n + m] = -s.S[i * n + m];
      b0 = -b0;
      b1 = -b1;
    }
    s.bs[m] = b0;
    double sigma = m < ne ? 1.0 : -1.0;
    s.err_parity = std::max(s.err_parity, std::fabs(b1 - sigma * b0));
    maxc = std::max(maxc, std::fabs(b0));
  }
  s.err_parity /= (maxc > 0 ? maxc : 1.0);
  double CtMinvC[4] = {0, 0, 0, 0};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      double t = 0.0;
      for (int k = 0; k < n; ++k) t += Cm[k * 2 + a] * MinvC[k * 2 + b];
      CtMinvC[a * 2 + b] = t;
    }
  s.h0 = tau_hat + 0.5 * (CtMinvC[0] + CtMinvC[3]);
  s.h1 = 0.5 * (CtMinvC[1] + CtMinvC[2]);

  // transforms and identity residuals
  double maxl = 0.0;
  for (int m = 0; m < n; ++m) maxl = std::max(maxl, std::fabs(s.Lambda[m]));
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      double om = 0.0, ol = 0.0;
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          om += s.S[i * n + a] * M[i * n + j] * s.S[j * n + b];
          ol += s.S[i * n + a] * L[i * n + j] * s.S[j * n + b];
        }
      s.err_orth = std::max(s.err_orth, std::fabs(om - (a == b ? 1.0 : 0.0)));
      s.err_diag = std::max(s.err_diag, std::fabs(ol - (a == b ? s.Lambda[a] : 0.0)) / maxl);
    }
  for (int m = 0; m < n; ++m)
    for (int i = 0; i < n; ++i) {
      double stm = 0.0, ms = 0.0;
      for (int k = 0; k < n; ++k) {
        stm += s.S[k * n + m] * M[k * n + i];
        ms += M[i * n + k] * s.S[k * n + m];
      }
      s.StM[m * n + i] = stm;
      s.MS[i * n + m] = ms;
      s.St[m * n + i] = s.S[i * n + m];
    }
  std::memcpy(s.M, M.data(), sizeof(double) * n * n);
  std::memcpy(s.D, D.data(), sizeof(double) * n * n);
  std::memcpy(s.L, L.data(), sizeof(double) * n * n);
  std::memcpy(s.Mdiag_face, M.data(), sizeof(double) * n * n);
  if (s.err_orth > 1e-12 || s.err_diag > 1e-12 || s.err_parity > 1e-10) {
    *msg = "eigen-decomposition identities not met";
    return 4;
  }
  return 0;
}

}  // namespace hdg
