// Host-side numerics: the power-law fit of Sec. II C and small dense helpers.
//
// The paper approximates f(r) = r^-alpha by a sum of exponentials with the
// method of Pirvu et al. (their MPO paper's appendix). We use that method's
// shift-invariance formulation: the samples f(1..R) fill a Hankel matrix whose
// dominant right singular subspace Q satisfies Q[1:] ~ Q[:-1] S; the
// eigenvalues of S are the decay factors lam_k, and the weights x_k follow by
// linear least squares on f(r) = sum_k x_k lam_k^r.
#include <algorithm>
#include <cmath>
#include <complex>

#include "common.h"
#include "tridiag.h"

namespace tdvp {

using cd = std::complex<double>;

// One-sided Jacobi SVD of a complex m x n matrix A (column-major, m >= 1).
// On return A holds U*S (columns), s the singular values (unsorted), V the
// accumulated right rotations (n x n, column-major), so A_in = (U S) V^H.
static void jacobi_svd_host(std::vector<cd>& A, int m, int n, std::vector<double>& s,
                            std::vector<cd>& V) {
  V.assign((size_t)n * n, cd(0.0, 0.0));
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  const double tol = 1e-15;
  for (int sweep = 0; sweep < 60; ++sweep) {
    int rotated = 0;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        cd* x = &A[(size_t)p * m];
        cd* y = &A[(size_t)q * m];
        double a = 0, b = 0;
        cd k(0.0, 0.0);
        for (int i = 0; i < m; ++i) {
          a += std::norm(x[i]);
          b += std::norm(y[i]);
          k += std::conj(x[i]) * y[i];
        }
        double ak = std::abs(k);
        if (ak <= tol * std::sqrt(a * b) || ak == 0.0) continue;
        ++rotated;
        // columns: [x' y'] = [x y] G with G = [[cs, -sn e^{i phi}], [sn e^{-i phi}, cs]]^H form
        cd ph = k / ak;  // e^{i phi}
        double zeta = (b - a) / (2.0 * ak);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
        for (int i = 0; i < m; ++i) {
          cd xi = x[i], yi = y[i];
          x[i] = cs * xi - sn * std::conj(ph) * yi;
          y[i] = sn * ph * xi + cs * yi;
        }
        cd* vx = &V[(size_t)p * n];
        cd* vy = &V[(size_t)q * n];
        for (int i = 0; i < n; ++i) {
          cd xi = vx[i], yi = vy[i];
          vx[i] = cs * xi - sn * std::conj(ph) * yi;
          vy[i] = sn * ph * xi + cs * yi;
        }
      }
    }
    if (!rotated) break;
  }
  s.resize(n);
  for (int j = 0; j < n; ++j) {
    double a = 0;
    for (int i = 0; i < m; ++i) a += std::norm(A[(size_t)j * m + i]);
    s[j] = std::sqrt(a);
  }
}

// Pseudo-inverse of a complex m x n matrix (column-major) -> n x m (column-major)
static std::vector<cd> pinv_host(const std::vector<cd>& Ain, int m, int n) {
  std::vector<cd> A = Ain, V;
  std::vector<double> s;
  jacobi_svd_host(A, m, n, s, V);
  double smax = 0;
  for (double v : s) smax = std::max(smax, v);
  double cut = smax * 1e-13 * std::max(m, n);
  std::vector<cd> P((size_t)n * m, cd(0.0, 0.0));
  // A = sum_j u_j s_j v_j^H  ->  pinv = sum_j v_j s_j^-1 u_j^H, u_j s_j = A[:, j]
  for (int j = 0; j < n; ++j) {
    if (s[j] <= cut) continue;
    double inv2 = 1.0 / (s[j] * s[j]);
    for (int r = 0; r < n; ++r) {      // row of pinv
      cd vr = V[(size_t)j * n + r];
      for (int c = 0; c < m; ++c) {    // column of pinv
        P[(size_t)c * n + r] += vr * std::conj(A[(size_t)j * m + c]) * inv2;
      }
    }
  }
  return P;
}

// Eigenvalues of a complex n x n matrix (row-major): Householder reduction to
// upper Hessenberg form, then shifted QR steps with Givens rotations and
// deflation from the bottom (textbook complex QR algorithm).
static std::vector<cd> eigvals_host(std::vector<cd> H, int n) {
  auto at = [&](int i, int j) -> cd& { return H[(size_t)i * n + j]; };
  for (int k = 0; k < n - 2; ++k) {
    double alpha = 0;
    for (int i = k + 1; i < n; ++i) alpha += std::norm(at(i, k));
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    std::vector<cd> v(n, cd(0.0, 0.0));
    cd x0 = at(k + 1, k);
    cd ph = std::abs(x0) > 0 ? x0 / std::abs(x0) : cd(1.0, 0.0);
    v[k + 1] = x0 + ph * alpha;
    for (int i = k + 2; i < n; ++i) v[i] = at(i, k);
    double vn = 0;
    for (int i = k + 1; i < n; ++i) vn += std::norm(v[i]);
    if (vn == 0.0) continue;
    // H <- (I - 2 v v^H / vn) H (I - 2 v v^H / vn)
    for (int j = 0; j < n; ++j) {
      cd d(0.0, 0.0);
      for (int i = k + 1; i < n; ++i) d += std::conj(v[i]) * at(i, j);
      d *= 2.0 / vn;
      for (int i = k + 1; i < n; ++i) at(i, j) -= v[i] * d;
    }
    for (int i = 0; i < n; ++i) {
      cd d(0.0, 0.0);
      for (int j = k + 1; j < n; ++j) d += at(i, j) * v[j];
      d *= 2.0 / vn;
      for (int j = k + 1; j < n; ++j) at(i, j) -= d * std::conj(v[j]);
    }
  }
  std::vector<cd> ev(n);
  int hi = n - 1;
  int iter = 0;
  const double eps = 2.220446049250313e-16;
  while (hi >= 0) {
    if (hi == 0) {
      ev[0] = at(0, 0);
      break;
    }
    if (std::abs(at(hi, hi - 1)) <= eps * (std::abs(at(hi, hi)) + std::abs(at(hi - 1, hi - 1)))) {
      ev[hi] = at(hi, hi);
      --hi;
      iter = 0;
      continue;
    }
    if (++iter > 200) fail(TDVP_ENUMERIC, "eigenvalue iteration of the fit did not converge");
    int lo = hi - 1;
    while (lo > 0 && std::abs(at(lo, lo - 1)) >
                         eps * (std::abs(at(lo, lo)) + std::abs(at(lo - 1, lo - 1))))
      --lo;
    // Wilkinson shift: eigenvalue of the trailing 2x2 closer to H[hi][hi]
    cd a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
    cd tr = a + d, det = a * d - b * c;
    cd disc = std::sqrt(tr * tr * 0.25 - det);
    cd mu1 = tr * 0.5 + disc, mu2 = tr * 0.5 - disc;
    cd mu = std::abs(mu1 - d) < std::abs(mu2 - d) ? mu1 : mu2;
    if (iter % 11 == 10) mu += std::abs(at(hi, hi - 1));  // exceptional shift
    for (int i = lo; i <= hi; ++i) at(i, i) -= mu;
    std::vector<double> cs(hi - lo);
    std::vector<cd> sn(hi - lo);
    for (int p = lo; p < hi; ++p) {
      cd x = at(p, p), y = at(p + 1, p);
      double r = std::sqrt(std::norm(x) + std::norm(y));
      double cc = r == 0 ? 1.0 : std::abs(x) / r;
      cd ss = r == 0 ? cd(0.0, 0.0)
                     : (std::abs(x) == 0 ? cd(1.0, 0.0) : (x / std::abs(x))) * std::conj(y) / r;
      cs[p - lo] = cc;
      sn[p - lo] = ss;
      for (int j = lo; j < n; ++j) {
        cd u = at(p, j), v = at(p + 1, j);
        at(p, j) = cc * u + ss * v;
        at(p + 1, j) = -std::conj(ss) * u + cc * v;
      }
    }
    for (int p = lo; p < hi; ++p) {
      double cc = cs[p - lo];
      cd ss = sn[p - lo];
      for (int i = 0; i <= std::min(hi, p + 2); ++i) {
        cd u = at(i, p), v = at(i, p + 1);
        at(i, p) = cc * u + std::conj(ss) * v;
        at(i, p + 1) = -ss * u + cc * v;
      }
    }
    for (int i = lo; i <= hi; ++i) at(i, i) += mu;
  }
  return ev;
}

void host_fit_power_law(double alpha, int n_exp, int r_max, std::vector<double2>& x_out,
                        std::vector<double2>& lam_out) {
  if (n_exp < 1 || n_exp > 64 || r_max < 2 || !(alpha > 0))
    fail(TDVP_EINVAL, "tdvp_fit_power_law: need 1 <= n_exp <= 64, r_max >= 2, alpha > 0");
  std::vector<double> f(r_max);
  for (int r = 1; r <= r_max; ++r) f[r - 1] = std::pow((double)r, -alpha);
  const int K = n_exp;
  const int L = r_max / 2;
  const int rows = r_max - L;
  const int keff = std::min(K, std::min(L, rows));
  // Hankel Y[i][j] = f(1 + i + j), rows x (L+1), column-major
  std::vector<cd> Y((size_t)rows * (L + 1));
  for (int j = 0; j <= L; ++j)
    for (int i = 0; i < rows; ++i) Y[(size_t)j * rows + i] = f[i + j];
  std::vector<double> s;
  std::vector<cd> V;
  jacobi_svd_host(Y, rows, L + 1, s, V);
  std::vector<int> order(L + 1);
  for (int i = 0; i <= L; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return s[a] > s[b]; });
  // Q = dominant right singular vectors, (L+1) x keff column-major
  std::vector<cd> Q1((size_t)L * keff), Q2((size_t)L * keff);
  for (int c = 0; c < keff; ++c) {
    const cd* v = &V[(size_t)order[c] * (L + 1)];
    for (int i = 0; i < L; ++i) {
      Q1[(size_t)c * L + i] = v[i];
      Q2[(size_t)c * L + i] = v[i + 1];
    }
  }
  std::vector<cd> P = pinv_host(Q1, L, keff);  // keff x L column-major
  std::vector<cd> S((size_t)keff * keff, cd(0.0, 0.0));  // row-major
  for (int i = 0; i < keff; ++i)
    for (int j = 0; j < keff; ++j) {
      cd acc(0.0, 0.0);
      for (int l = 0; l < L; ++l) acc += P[(size_t)l * keff + i] * Q2[(size_t)j * L + l];
      S[(size_t)i * keff + j] = acc;
    }
  std::vector<cd> lam = eigvals_host(S, keff);
  // x from least squares: f(r) = sum_k x_k lam_k^r
  std::vector<cd> M((size_t)r_max * keff);
  for (int k = 0; k < keff; ++k)
    for (int r = 1; r <= r_max; ++r) M[(size_t)k * r_max + r - 1] = std::pow(lam[k], r);
  std::vector<cd> Mp = pinv_host(M, r_max, keff);  // keff x r_max
  std::vector<cd> x(keff, cd(0.0, 0.0));
  for (int k = 0; k < keff; ++k)
    for (int r = 0; r < r_max; ++r) x[k] += Mp[(size_t)r * keff + k] * f[r];
  x_out.assign(K, make_double2(0.0, 0.0));
  lam_out.assign(K, make_double2(0.5, 0.0));
  for (int k = 0; k < keff; ++k) {
    x_out[k] = make_double2(x[k].real(), x[k].imag());
    lam_out[k] = make_double2(lam[k].real(), lam[k].imag());
  }
}

// Levenberg-Marquardt refinement of the sum-of-exponentials fit (the alternative
// to the shift-invariance fit that the Supplemental Material compares in its
// power-law section): real x_k, lam_k minimising sum_r (w_r e_r)^2 with
// e_r = sum_k x_k lam_k^r - r^-alpha, w_r = 1 (absolute) or r^alpha (relative),
// r = 1..r_max. Marquardt's damped normal equations (J^T J + mu diag(J^T J)) d =
// -J^T e, mu divided by 10 after an accepted step and multiplied by 10 after a
// rejected one; stops after 1000 iterations or 10000 evaluations, when the
// relative step is below 1e-6 or the relative decrease of the sum of squares
// below 1e-14 (the stopping values of the Supplemental Material's fit). Starts
// from the real parts of the shift-invariance fit; returns the start unchanged
// if the result leaves 0 < |lam| < 1.
void host_fit_power_law_lm(double alpha, int n_exp, int r_max, int relative, std::vector<double2>& x_out,
                           std::vector<double2>& lam_out, double* rms_out) {
  host_fit_power_law(alpha, n_exp, r_max, x_out, lam_out);
  const int K = n_exp, P = 2 * K, R = r_max;
  std::vector<double> p(P), f(R), w(R);
  for (int k = 0; k < K; ++k) {
    p[k] = x_out[k].x;
    p[K + k] = lam_out[k].x;
  }
  for (int r = 1; r <= R; ++r) {
    f[r - 1] = std::pow((double)r, -alpha);
    w[r - 1] = relative ? 1.0 / f[r - 1] : 1.0;
  }
  auto residual = [&](const std::vector<double>& q, std::vector<double>& e) {
    double ss = 0.0;
    for (int r = 1; r <= R; ++r) {
      double v = -f[r - 1];
      for (int k = 0; k < K; ++k) v += q[k] * std::pow(q[K + k], r);
      e[r - 1] = w[r - 1] * v;
      ss += e[r - 1] * e[r - 1];
    }
    return ss;
  };
  std::vector<double> e(R), e2(R), J((size_t)R * P), A((size_t)P * P), g(P), d(P), q(P), Lc((size_t)P * P);
  double S = residual(p, e);
  const std::vector<double> p0 = p;
  const double S0 = S;
  double mu = 1e-3;
  int nfev = 1;
  for (int it = 0; it < 1000 && nfev < 10000; ++it) {
    for (int r = 1; r <= R; ++r)
      for (int k = 0; k < K; ++k) {
        const double lk = p[K + k];
        J[(size_t)(r - 1) * P + k] = w[r - 1] * std::pow(lk, r);
        J[(size_t)(r - 1) * P + K + k] = w[r - 1] * p[k] * r * std::pow(lk, r - 1);
      }
    for (int i = 0; i < P; ++i) {
      double gi = 0.0;
      for (int r = 0; r < R; ++r) gi += J[(size_t)r * P + i] * e[r];
      g[i] = gi;
      for (int j = 0; j <= i; ++j) {
        double a = 0.0;
        for (int r = 0; r < R; ++r) a += J[(size_t)r * P + i] * J[(size_t)r * P + j];
        A[(size_t)i * P + j] = A[(size_t)j * P + i] = a;
      }
    }
    bool accepted = false, done = false;
    while (!accepted && nfev < 10000 && mu < 1e20) {
      // Cholesky of A + mu diag(A)
      bool pd = true;
      for (int i = 0; i < P && pd; ++i)
        for (int j = 0; j <= i; ++j) {
          double v = A[(size_t)i * P + j] + (i == j ? mu * std::max(A[(size_t)i * P + i], 1e-300) : 0.0);
          for (int k = 0; k < j; ++k) v -= Lc[(size_t)i * P + k] * Lc[(size_t)j * P + k];
          if (i == j) {
            if (!(v > 0.0)) { pd = false; break; }
            Lc[(size_t)i * P + i] = std::sqrt(v);
          } else {
            Lc[(size_t)i * P + j] = v / Lc[(size_t)j * P + j];
          }
        }
      if (!pd) { mu *= 10.0; continue; }
      for (int i = 0; i < P; ++i) {  // L y = -g
        double v = -g[i];
        for (int k = 0; k < i; ++k) v -= Lc[(size_t)i * P + k] * d[k];
        d[i] = v / Lc[(size_t)i * P + i];
      }
      for (int i = P - 1; i >= 0; --i) {  // L^T d = y
        double v = d[i];
        for (int k = i + 1; k < P; ++k) v -= Lc[(size_t)k * P + i] * d[k];
        d[i] = v / Lc[(size_t)i * P + i];
      }
      double dn = 0.0, pn = 0.0;
      for (int i = 0; i < P; ++i) {
        q[i] = p[i] + d[i];
        dn += d[i] * d[i];
        pn += p[i] * p[i];
      }
      const double S2 = residual(q, e2);
      ++nfev;
      if (S2 < S) {
        const double rel = (S - S2) / S;
        p = q;
        e = e2;
        S = S2;
        mu = std::max(mu / 10.0, 1e-15);
        accepted = true;
        if (std::sqrt(dn) < 1e-6 * (std::sqrt(pn) + 1e-6) || rel < 1e-14) done = true;
      } else {
        mu *= 10.0;
      }
    }
    if (!accepted || done) break;
  }
  bool ok = S <= S0;
  for (int k = 0; k < K; ++k) ok = ok && std::fabs(p[K + k]) < 1.0 && p[K + k] != 0.0;
  if (!ok) {
    p = p0;
    S = S0;
  }
  for (int k = 0; k < K; ++k) {
    x_out[k] = make_double2(p[k], 0.0);
    lam_out[k] = make_double2(p[K + k], 0.0);
  }
  if (rms_out) *rms_out = std::sqrt(S / R);
}

__host__ __device__ int tridiag_expm_e0(int k, const double* alpha, const double* beta, double t,
                                        double2* c, double* work) {
  return tridiag_expm_e0_impl(k, alpha, beta, t, c, work);
}

}  // namespace tdvp
