// Kernels of the forward-mode derivative (tangent) of the sweep with respect
// to model parameters: the full SVD of a split exported as explicit factors,
// the tangent of the truncated split, and complex linear combinations (the
// quadrature of the Frechet derivative of exp(-i t H_eff)).
#include "engine.h"

namespace tdvp {

// U [rows][n_vec], Vh [n_vec][cols] and s [n_vec], descending, from the
// converged one-sided Jacobi state of one split (the layout that svd_write
// reads). Vectors on the X side of a zero singular value are set to zero.
__global__ void svd_export_full_kernel(const __grid_constant__ SvdFullDesc P) {
  const int64_t nu = (int64_t)P.rows * P.n_vec, nv = (int64_t)P.n_vec * P.cols;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nu + nv + P.n_vec;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (idx < nu) {
      const int r = (int)(idx / P.n_vec), i = (int)(idx % P.n_vec);
      const int p = P.perm[i];
      const double sp = P.sig[p];
      double2 v;
      if (P.trans) v = sp > 0.0 ? zscale(P.X[(int64_t)p * P.len + r], 1.0 / sp) : make_double2(0, 0);
      else v = zconj(P.Acc[(int64_t)p * P.n_vec + r]);
      P.U[idx] = v;
    } else if (idx < nu + nv) {
      const int64_t q = idx - nu;
      const int i = (int)(q / P.cols), c = (int)(q % P.cols);
      const int p = P.perm[i];
      const double sp = P.sig[p];
      double2 v;
      if (P.trans) v = zconj(P.Acc[(int64_t)p * P.n_vec + c]);
      else v = sp > 0.0 ? zscale(P.X[(int64_t)p * P.len + c], 1.0 / sp) : make_double2(0, 0);
      P.Vh[q] = v;
    } else {
      const int i = (int)(idx - nu - nv);
      P.s[i] = P.sig[P.perm[i]];
    }
  }
}

void launch_svd_export_full(const SvdFullDesc& d, cudaStream_t s) {
  const int64_t total = (int64_t)d.rows * d.n_vec + (int64_t)d.n_vec * d.cols + d.n_vec;
  const int grid = (int)std::min<int64_t>(cdiv64(total, 256), 152 * 8);
  svd_export_full_kernel<<<grid, 256, 0, s>>>(d);
  LAUNCH_CHECK();
  ++g_launches;
}

// Tangent of the truncated split Theta = U S V^H -> (Psi_L = U_k S_k,
// V = 1/S_k, Psi_R = S_k V_k^H) for dP = U^H dTheta V (all r singular
// triplets). With the phase gauge Im(U^H dU)_jj = s_j^-1 Im dP_jj, (V^H dV)_jj = 0:
//   dPsi_L = U CL + dTheta V_k,   dPsi_R = CR^H V^H + U_k^H dTheta,
//   dV_j = -Re(dP_jj) / s_j^2,
// CL[i][j] = s_i (s_i dP_ij + s_j conj(dP_ji)) / (s_j^2 - s_i^2),
// CR[i][j] = s_i (s_j dP_ij + s_i conj(dP_ji)) / (s_j^2 - s_i^2)  (i != j),
// CL[j][j] = 0, CR[j][j] = i Im dP_jj. These follow from differentiating
// Theta = U S V^H with U^H dU and V^H dV anti-Hermitian; the kept-discarded
// couplings use the discarded values, so the result is the derivative at
// fixed kept rank k. Equal nonzero values (a singular derivative) give 0.
__global__ void svd_tangent_coef_kernel(const __grid_constant__ SvdTanBatch B) {
  const SvdTanDesc& P = B.d[blockIdx.y];
  const int r = P.r, k = P.k;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)r * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / k), j = (int)(idx % k);
    double2 cl = make_double2(0, 0), cr = make_double2(0, 0);
    const double2 pij = P.dP[(int64_t)i * r + j];
    if (i == j) {
      cr = make_double2(0.0, pij.y);
      P.dV[j] = -pij.x / (P.s[j] * P.s[j]);
    } else {
      const double si = P.s[i], sj = P.s[j];
      const double den = sj * sj - si * si;
      if (den != 0.0 && si != 0.0) {
        const double2 pji = zconj(P.dP[(int64_t)j * r + i]);
        const double f = si / den;
        cl = make_double2(f * (si * pij.x + sj * pji.x), f * (si * pij.y + sj * pji.y));
        cr = make_double2(f * (sj * pij.x + si * pji.x), f * (sj * pij.y + si * pji.y));
      }
    }
    P.CL[idx] = cl;
    P.CR[idx] = cr;
  }
}

void launch_svd_tangent_coef(const SvdTanBatch& b, cudaStream_t s) {
  if (b.n <= 0) return;
  int64_t mx = 1;
  for (int i = 0; i < b.n; ++i) mx = std::max<int64_t>(mx, (int64_t)b.d[i].r * b.d[i].k);
  dim3 grid((unsigned)std::min<int64_t>(cdiv64(mx, 256), 152 * 4), b.n);
  svd_tangent_coef_kernel<<<grid, 256, 0, s>>>(b);
  LAUNCH_CHECK();
  ++g_launches;
}

// y = (accumulate ? y : 0) + sum_t c_t x_t
__global__ void zcombine_kernel(const __grid_constant__ ZCombBatch B) {
  const ZCombDesc& P = B.d[blockIdx.y];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 acc = P.accumulate ? P.y[i] : make_double2(0, 0);
    for (int t = 0; t < P.n_terms; ++t) {
      const double2 x = P.x[t][i];
      const double2 c = P.c[t];
      acc.x = fma(c.x, x.x, fma(-c.y, x.y, acc.x));
      acc.y = fma(c.x, x.y, fma(c.y, x.x, acc.y));
    }
    P.y[i] = acc;
  }
}

void launch_zcombine(const ZCombBatch& b, cudaStream_t s) {
  if (b.n <= 0) return;
  int64_t mx = 1;
  for (int i = 0; i < b.n; ++i) mx = std::max<int64_t>(mx, b.d[i].n);
  dim3 grid((unsigned)std::min<int64_t>(cdiv64(mx, 256), 152 * 4), b.n);
  zcombine_kernel<<<grid, 256, 0, s>>>(b);
  LAUNCH_CHECK();
  ++g_launches;
}

// Gauss-Legendre nodes and weights on [0, 1] (Newton iteration on the
// three-term recurrence of the Legendre polynomials).
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      // P_n = p1, P_{n-1} = p0
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

}  // namespace tdvp
