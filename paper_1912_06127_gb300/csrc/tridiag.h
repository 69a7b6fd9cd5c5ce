// Eigen-decomposition T = Q Theta Q^T of a small real symmetric tridiagonal
// matrix, and from it either c = exp(-i t T) e_0 = Q exp(-i t Theta) Q^T e_0
// (the Lanczos exponentiation of Park and Light, which needs only the k x k
// tridiagonal projection of H_eff, Sec. III A, Eq. 18 / Eq. 20) or the
// eigenvector of the lowest eigenvalue (the Lanczos ground state of the
// two-site DMRG update).
//
// The eigen-decomposition is the implicit symmetric QR iteration with
// Wilkinson shifts (Golub and Van Loan, "Matrix Computations", Sec. 8.3):
// each step chases a bulge with Givens rotations from the top of the active
// block; converged eigenvalues are deflated from the bottom. k <= 24, so the
// matrix is held densely and the rotations are applied to whole rows and
// columns, which keeps the bookkeeping plain.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace tdvp {

// work must hold 2*k*k doubles; on return the diagonal of T (first k*k) holds
// the eigenvalues and Q (next k*k, columns) the eigenvectors. Returns the
// number of QR steps, or -1 if the iteration did not converge within its limit.
__host__ __device__ inline int tridiag_eig_impl(int k, const double* alpha, const double* beta, double* work) {
  double* T = work;          // k x k, row-major
  double* Q = work + k * k;  // k x k eigenvectors (columns)
  for (int i = 0; i < k * k; ++i) {
    T[i] = 0.0;
    Q[i] = 0.0;
  }
  for (int i = 0; i < k; ++i) {
    T[i * k + i] = alpha[i];
    Q[i * k + i] = 1.0;
    if (i + 1 < k) {
      T[i * k + i + 1] = beta[i];
      T[(i + 1) * k + i] = beta[i];
    }
  }
  const double eps = 2.220446049250313e-16;
  int hi = k - 1;
  int steps = 0;
  const int max_steps = 60 * k + 60;
  while (hi > 0) {
    double sub = fabs(T[hi * k + hi - 1]);
    if (sub <= eps * (fabs(T[hi * k + hi]) + fabs(T[(hi - 1) * k + hi - 1])) || sub == 0.0) {
      T[hi * k + hi - 1] = 0.0;
      T[(hi - 1) * k + hi] = 0.0;
      --hi;
      continue;
    }
    if (steps >= max_steps) return -1;
    int lo = hi - 1;
    while (lo > 0) {
      double s2 = fabs(T[lo * k + lo - 1]);
      if (s2 <= eps * (fabs(T[lo * k + lo]) + fabs(T[(lo - 1) * k + lo - 1]))) {
        T[lo * k + lo - 1] = 0.0;
        T[(lo - 1) * k + lo] = 0.0;
        break;
      }
      --lo;
    }
    // Wilkinson shift from the trailing 2x2 block of the active part
    double a = T[(hi - 1) * k + hi - 1];
    double b = T[hi * k + hi - 1];
    double cc = T[hi * k + hi];
    double delta = 0.5 * (a - cc);
    double sgn = delta >= 0.0 ? 1.0 : -1.0;
    double mu = cc - b * b / (delta + sgn * sqrt(delta * delta + b * b));
    double x = T[lo * k + lo] - mu;
    double z = T[(lo + 1) * k + lo];
    for (int p = lo; p < hi; ++p) {
      double r = hypot(x, z);
      double cs = 1.0, sn = 0.0;
      if (r != 0.0) {
        cs = x / r;
        sn = z / r;
      }
      // rows p, p+1 of T
      for (int i = lo; i <= hi; ++i) {
        double u = T[p * k + i], v = T[(p + 1) * k + i];
        T[p * k + i] = cs * u + sn * v;
        T[(p + 1) * k + i] = -sn * u + cs * v;
      }
      // columns p, p+1 of T
      for (int i = lo; i <= hi; ++i) {
        double u = T[i * k + p], v = T[i * k + p + 1];
        T[i * k + p] = cs * u + sn * v;
        T[i * k + p + 1] = -sn * u + cs * v;
      }
      // eigenvector accumulation Q <- Q R^T
      for (int i = 0; i < k; ++i) {
        double u = Q[i * k + p], v = Q[i * k + p + 1];
        Q[i * k + p] = cs * u + sn * v;
        Q[i * k + p + 1] = -sn * u + cs * v;
      }
      if (p + 1 < hi) {
        x = T[(p + 1) * k + p];
        z = T[(p + 2) * k + p];
      }
    }
    ++steps;
  }
  return steps;
}

// c = exp(-i t T) e_0; same return value as tridiag_eig_impl.
__host__ __device__ inline int tridiag_expm_e0_impl(int k, const double* alpha, const double* beta,
                                                    double t, double2* c, double* work) {
  const int steps = tridiag_eig_impl(k, alpha, beta, work);
  if (steps < 0) return steps;
  const double* T = work;
  const double* Q = work + k * k;
  for (int i = 0; i < k; ++i) c[i] = make_double2(0.0, 0.0);
  for (int l = 0; l < k; ++l) {
    double th = T[l * k + l];
    double sn, cs;
    sincos(-t * th, &sn, &cs);
    double w = Q[0 * k + l];
    for (int i = 0; i < k; ++i) {
      double q = Q[i * k + l] * w;
      c[i].x += q * cs;
      c[i].y += q * sn;
    }
  }
  return steps;
}

// c = eigenvector of the lowest eigenvalue (real, unit norm, sign fixed by
// c_0 >= 0), *e0 = that eigenvalue; same return value as tridiag_eig_impl.
__host__ __device__ inline int tridiag_ground_impl(int k, const double* alpha, const double* beta, double2* c,
                                                   double* e0, double* work) {
  const int steps = tridiag_eig_impl(k, alpha, beta, work);
  if (steps < 0) return steps;
  const double* T = work;
  const double* Q = work + k * k;
  int lmin = 0;
  for (int l = 1; l < k; ++l)
    if (T[l * k + l] < T[lmin * k + lmin]) lmin = l;
  *e0 = T[lmin * k + lmin];
  const double sg = Q[0 * k + lmin] < 0.0 ? -1.0 : 1.0;
  for (int i = 0; i < k; ++i) c[i] = make_double2(sg * Q[i * k + lmin], 0.0);
  return steps;
}

}  // namespace tdvp
