// Truncated SVD split of the evolved two-site state (Fig. 5), FP64.
//
// Theta' is reshaped to a (chi_l d) x (d chi_r) matrix and decomposed with the
// one-sided (Hestenes) Jacobi method: the smaller of its row set and column
// set is orthogonalised by plane rotations, each rotation chosen to make one
// pair of vectors orthogonal (a 2x2 Hermitian eigenproblem), until a full
// sweep over all pairs applies none. The rotations are accumulated, which
// gives the other set of singular vectors. Pairs are visited in round-robin
// order, so that each round holds n/2 disjoint pairs, one warp per pair and
// all problems of a stage in the same launch. The final vector norms are the
// singular values.
//
// Truncation (Sec. III C, Eq. 22 and Sec. III D): the smallest rank chi_w
// whose discarded weight sum_{j >= chi_w} lambda_j^2 is <= w_max, capped at
// chi_max and at the values above eps * lambda_1, at least 1. Then
// Psi_L = A' Lambda', Psi_R = Lambda' B', V' = Lambda'^{-1} (Sec. II B).
#include "common.h"
#include "svd.h"

namespace tdvp {

constexpr double JACOBI_TOL = 1e-14;
constexpr int SVD_WARPS = 8;
constexpr int SVD_MAX_SWEEPS = 40;

__global__ void svd_setup(const __grid_constant__ SvdBatch B) {
  const SvdDesc& P = B.d[blockIdx.y];
  const int64_t nx = (int64_t)P.n_vec * P.len;
  const int64_t na = (int64_t)P.n_vec * P.n_vec;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nx + na;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nx) {
      int v = (int)(i / P.len), e = (int)(i % P.len);
      // trans 0: vector v = row v of theta; trans 1: vector v = column v
      P.X[i] = P.trans ? P.theta[(int64_t)e * P.cols + v] : P.theta[(int64_t)v * P.cols + e];
    } else {
      int64_t q = i - nx;
      int r = (int)(q / P.n_vec), c = (int)(q % P.n_vec);
      P.Acc[q] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *P.rotated = 0;
    *P.conv = 0;
  }
}

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(SVD_WARPS * 32) svd_round(const __grid_constant__ SvdBatch B, int r) {
  const SvdDesc& P = B.d[blockIdx.y];
  if (*P.conv) return;
  const int npad = P.n_vec + (P.n_vec & 1);
  if (npad < 2 || r >= npad - 1) return;
  const int pair = blockIdx.x * SVD_WARPS + (threadIdx.x >> 5);
  if (pair >= npad / 2) return;
  const int lane = threadIdx.x & 31;
  int p, q;
  if (pair == 0) {
    p = npad - 1;
    q = r;
  } else {
    p = (r + pair) % (npad - 1);
    q = (r - pair + (npad - 1)) % (npad - 1);
  }
  if (p > q) {
    int t = p;
    p = q;
    q = t;
  }
  if (q >= P.n_vec) return;
  double2* x = P.X + (int64_t)p * P.len;
  double2* y = P.X + (int64_t)q * P.len;
  double a = 0, b = 0, kr = 0, ki = 0;
  for (int i = lane; i < P.len; i += 32) {
    double2 u = x[i], v = y[i];
    a += u.x * u.x + u.y * u.y;
    b += v.x * v.x + v.y * v.y;
    kr += u.x * v.x + u.y * v.y;  // conj(u) v
    ki += u.x * v.y - u.y * v.x;
  }
  a = warp_sum(a);
  b = warp_sum(b);
  kr = warp_sum(kr);
  ki = warp_sum(ki);
  const double ak = sqrt(kr * kr + ki * ki);
  if (!(ak > JACOBI_TOL * sqrt(a * b))) return;
  if (lane == 0) atomicAdd(P.rotated, 1);
  const double phr = kr / ak, phi = ki / ak;  // e^{i phi}
  const double zeta = (b - a) / (2.0 * ak);
  const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
  // x' = cs x - sn e^{-i phi} y ; y' = sn e^{i phi} x + cs y
  const double2 m1 = make_double2(-sn * phr, sn * phi);   // -sn e^{-i phi}
  const double2 m2 = make_double2(sn * phr, sn * phi);    //  sn e^{+i phi}
  for (int i = lane; i < P.len; i += 32) {
    double2 u = x[i], v = y[i];
    double2 nu = zscale(u, cs), nv = zscale(v, cs);
    zfma(nu, m1, v);
    zfma(nv, m2, u);
    x[i] = nu;
    y[i] = nv;
  }
  double2* ax = P.Acc + (int64_t)p * P.n_vec;
  double2* ay = P.Acc + (int64_t)q * P.n_vec;
  for (int i = lane; i < P.n_vec; i += 32) {
    double2 u = ax[i], v = ay[i];
    double2 nu = zscale(u, cs), nv = zscale(v, cs);
    zfma(nu, m1, v);
    zfma(nv, m2, u);
    ax[i] = nu;
    ay[i] = nv;
  }
}

// After a sweep: problems with no rotation are converged; count the others.
__global__ void svd_sweep_end(const __grid_constant__ SvdBatch B, int* unconv) {
  if (threadIdx.x != 0) return;
  int cnt = 0;
  for (int i = 0; i < B.n; ++i) {
    const SvdDesc& P = B.d[i];
    if (!*P.conv) {
      if (*P.rotated == 0) *P.conv = 1;
      else ++cnt;
    }
    *P.rotated = 0;
  }
  *unconv = cnt;
}

__global__ void svd_norms(const __grid_constant__ SvdBatch B) {
  const SvdDesc& P = B.d[blockIdx.y];
  const int v = blockIdx.x * SVD_WARPS + (threadIdx.x >> 5);
  if (v >= P.n_vec) return;
  const int lane = threadIdx.x & 31;
  const double2* x = P.X + (int64_t)v * P.len;
  double s = 0;
  for (int i = lane; i < P.len; i += 32) s += x[i].x * x[i].x + x[i].y * x[i].y;
  s = warp_sum(s);
  if (lane == 0) P.sig[v] = sqrt(s);
}

__global__ void svd_truncate(const __grid_constant__ SvdBatch B) {
  const SvdDesc& P = B.d[blockIdx.x];
  const int n = P.n_vec;
  __shared__ int has_nan;
  if (threadIdx.x == 0) {
    has_nan = 0;
    for (int i = 0; i < n; ++i)
      if (!(P.sig[i] == P.sig[i])) has_nan = 1;
  }
  __syncthreads();
  if (!has_nan) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double si = P.sig[i];
      int rank = 0;
      for (int j = 0; j < n; ++j) {
        const double sj = P.sig[j];
        rank += (sj > si) || (sj == si && j < i);
      }
      P.perm[rank] = i;
    }
  } else {
    for (int i = threadIdx.x; i < n; i += blockDim.x) P.perm[i] = i;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double s0 = P.sig[P.perm[0]];
  if (has_nan || !(s0 > 0.0)) {
    atomicOr(B.status, 8);
    *P.chi = 1;
    *P.w = 0.0;
    return;
  }
  // smallest chi_w with tail weight <= w_max (Eq. 22), tail[n] = 0
  double tail = 0.0;
  int chi_w = n;
  // walk from the end; tail(k) = sum_{j >= k} s_j^2
  // chi_w = min k >= 1 with tail(k) <= w_max
  {
    double acc = 0.0;
    int best = n;
    for (int k = n - 1; k >= 1; --k) {
      const double sk = P.sig[P.perm[k]];
      acc += sk * sk;
      if (acc <= P.w_max) best = k;
      else break;
    }
    chi_w = best;
  }
  int n_eps = 0;
  for (int k = 0; k < n; ++k)
    if (P.sig[P.perm[k]] > P.eps * s0) ++n_eps;
  int chi = chi_w < P.chi_max ? chi_w : P.chi_max;
  if (n_eps < chi) chi = n_eps;
  if (chi < 1) chi = 1;
  for (int k = n - 1; k >= chi; --k) {
    const double sk = P.sig[P.perm[k]];
    tail += sk * sk;
  }
  *P.chi = chi;
  *P.w = tail;
}

__global__ void svd_write(const __grid_constant__ SvdBatch B) {
  const SvdDesc& P = B.d[blockIdx.y];
  const int chi = *P.chi;
  const int64_t nl = (int64_t)P.rows * chi;
  const int64_t nr = (int64_t)chi * P.cols;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nl + nr + P.n_vec;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (idx < nl) {
      const int r = (int)(idx / chi), c = (int)(idx % chi);
      const int i = P.perm[c];
      double2 v;
      if (!P.trans) v = zscale(zconj(P.Acc[(int64_t)i * P.n_vec + r]), P.sig[i]);
      else v = P.X[(int64_t)i * P.len + r];
      P.PsiL[idx] = v;
    } else if (idx < nl + nr) {
      const int64_t q = idx - nl;
      const int c = (int)(q / P.cols), col = (int)(q % P.cols);
      const int i = P.perm[c];
      double2 v;
      if (!P.trans) v = P.X[(int64_t)i * P.len + col];
      else v = zscale(zconj(P.Acc[(int64_t)i * P.n_vec + col]), P.sig[i]);
      P.PsiR[q] = v;
    } else {
      const int c = (int)(idx - nl - nr);
      const double sc = P.sig[P.perm[c]];
      if (c < chi) P.V[c] = 1.0 / sc;
      if (P.s_sorted) P.s_sorted[c] = sc;
    }
  }
}

void svd_split(SvdBatch& b, int* d_flag, int* h_flag, cudaStream_t s) {
  if (b.n <= 0) return;
  int64_t max_elems = 1;
  int npad_max = 2, nvec_max = 1;
  for (int i = 0; i < b.n; ++i) {
    auto& P = b.d[i];
    P.trans = P.rows > P.cols ? 1 : 0;
    P.n_vec = P.trans ? P.cols : P.rows;
    P.len = P.trans ? P.rows : P.cols;
    max_elems = std::max<int64_t>(max_elems, (int64_t)P.n_vec * (P.len + P.n_vec));
    npad_max = std::max(npad_max, P.n_vec + (P.n_vec & 1));
    nvec_max = std::max(nvec_max, P.n_vec);
  }
  dim3 g1((unsigned)std::min<int64_t>(cdiv64(max_elems, 256), 152 * 8), b.n);
  svd_setup<<<g1, 256, 0, s>>>(b);
  LAUNCH_CHECK();
  ++g_launches;
  dim3 gr(cdiv(npad_max / 2, SVD_WARPS), b.n);
  bool converged = false;
  for (int sweep = 0; sweep < SVD_MAX_SWEEPS && !converged; ++sweep) {
    double fl = 0;
    for (int i = 0; i < b.n; ++i)
      fl += 16.0 * (double)b.d[i].len * (b.d[i].n_vec / 2) * (b.d[i].n_vec - 1);
    ProfScope ps("svd_jacobi_sweep", s, fl, 0.0);
    for (int r = 0; r < npad_max - 1; ++r) {
      svd_round<<<gr, SVD_WARPS * 32, 0, s>>>(b, r);
    }
    LAUNCH_CHECK();
    g_launches += npad_max - 1;
    svd_sweep_end<<<1, 32, 0, s>>>(b, d_flag);
    LAUNCH_CHECK();
    ++g_launches;
    CUDA_TRY(cudaMemcpyAsync(h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    converged = (*h_flag == 0);
  }
  if (!converged) fail(TDVP_ENUMERIC, "Jacobi SVD did not converge");
  dim3 gn(cdiv(nvec_max, SVD_WARPS), b.n);
  svd_norms<<<gn, SVD_WARPS * 32, 0, s>>>(b);
  LAUNCH_CHECK();
  svd_truncate<<<b.n, 256, 0, s>>>(b);
  LAUNCH_CHECK();
  dim3 gw((unsigned)std::min<int64_t>(cdiv64(max_elems, 256), 152 * 8), b.n);
  svd_write<<<gw, 256, 0, s>>>(b);
  LAUNCH_CHECK();
  g_launches += 3;
}

}  // namespace tdvp
