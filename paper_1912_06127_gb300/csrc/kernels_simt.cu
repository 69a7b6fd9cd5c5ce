// SIMT kernels: batched complex FP64 GEMM, the sparse MPO ("W") stage of the
// effective-Hamiltonian and environment contractions, bond scaling and the
// operand preparation for the tensor-core path.
//
// The contraction order follows the cost bound of Eq. 21: the environment
// legs (chi^3 m d^2 work) are dense GEMMs, the MPO legs (chi^2 m^2 d^3 work,
// sparse in the MPO's finite-state structure) are applied block by block.
#include "common.h"

namespace tdvp {

// ---------------------------------------------------------------------------
// Complex FP64 GEMM. 64x64 output tile per 256-thread block, 8-deep K steps,
// 4x4 outputs per thread. FP64 throughput, not memory, bounds this kernel.
// ---------------------------------------------------------------------------
constexpr int ZG_BK = 8;

// TT outputs per thread along each side: a (16 TT) x (16 TT) tile per CTA of
// 256 threads. Every tile size sums each output over k in the same order, so
// the results are bitwise the same; the autotuner picks one per shape.
template <int TT>
__global__ void __launch_bounds__(256) zgemm_kernel(const __grid_constant__ ZGemmBatch batch) {
  constexpr int BM = 16 * TT, BN = 16 * TT;
  const int pid = blockIdx.y;
  if (pid >= batch.n) return;
  const ZGemmDesc& P = batch.d[pid];
  if (P.skip && *P.skip) return;
  const int tiles_m = (P.M + BM - 1) / BM;
  const int tiles_n = (P.N + BN - 1) / BN;
  if ((int)blockIdx.x >= tiles_m * tiles_n) return;
  const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
  const int m0 = tm * BM, n0 = tn * BN;
  // Hermitian results: the blocks of 64 on or above the diagonal (any tile size)
  if (P.upper_only && m0 / 64 > n0 / 64) return;
  __shared__ double2 As[ZG_BK][BM];
  __shared__ double2 Bs[ZG_BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  double2 acc[TT][TT];
#pragma unroll
  for (int i = 0; i < TT; ++i)
#pragma unroll
    for (int j = 0; j < TT; ++j) acc[i][j] = make_double2(0.0, 0.0);
  const bool a_k_fast = (P.a_cs == 1);
  const bool b_n_fast = (P.b_cs == 1);
  for (int k0 = 0; k0 < P.K; k0 += ZG_BK) {
#pragma unroll
    for (int r = 0; r < ZG_BK * BM / 256; ++r) {
      int e = tid + r * 256;
      int i, k;
      if (a_k_fast) {
        k = e % ZG_BK;
        i = e / ZG_BK;
      } else {
        i = e % BM;
        k = e / BM;
      }
      double2 v = make_double2(0.0, 0.0);
      int gi = m0 + i, gk = k0 + k;
      if (gi < P.M && gk < P.K) {
        v = P.A[(int64_t)gi * P.a_rs + (int64_t)gk * P.a_cs];
        if (P.conj_a) v.y = -v.y;
        if (P.kscale) {
          double sc = P.kscale[gk];
          v.x *= sc;
          v.y *= sc;
        }
      }
      As[k][i] = v;
      int j, kb;
      if (b_n_fast) {
        j = e % BN;
        kb = e / BN;
      } else {
        kb = e % ZG_BK;
        j = e / ZG_BK;
      }
      double2 w = make_double2(0.0, 0.0);
      int gj = n0 + j, gkb = k0 + kb;
      if (gj < P.N && gkb < P.K) {
        w = P.B[(int64_t)gkb * P.b_rs + (int64_t)gj * P.b_cs];
        if (P.conj_b) w.y = -w.y;
      }
      Bs[kb][j] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < ZG_BK; ++kk) {
      double2 a[TT], b[TT];
#pragma unroll
      for (int i = 0; i < TT; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TT; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TT; ++i)
#pragma unroll
        for (int j = 0; j < TT; ++j) zfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TT; ++i) {
    int gi = m0 + ty + 16 * i;
    if (gi >= P.M) continue;
#pragma unroll
    for (int j = 0; j < TT; ++j) {
      int gj = n0 + tx + 16 * j;
      if (gj >= P.N) continue;
      double2* c = P.C + (int64_t)gi * P.c_rs + (int64_t)gj * P.c_cs;
      double2 v = acc[i][j];
      if (P.accumulate) v = zadd(v, *c);
      *c = v;
    }
  }
}

// the largest M, N, K of a batch and whether any problem accumulates into C
static void batch_shape(const ZGemmBatch& b, int64_t& M, int64_t& N, int64_t& K, bool& acc) {
  M = N = K = 0;
  acc = false;
  for (int i = 0; i < b.n; ++i) {
    M = std::max<int64_t>(M, b.d[i].M);
    N = std::max<int64_t>(N, b.d[i].N);
    K = std::max<int64_t>(K, b.d[i].K);
    acc = acc || b.d[i].accumulate;
  }
}

void launch_zgemm(const ZGemmBatch& b, cudaStream_t s, const char* prof_name) {
  if (b.n <= 0) return;
  int64_t M, N, K;
  bool acc;
  batch_shape(b, M, N, K, acc);
  if (M <= 0 || N <= 0) return;
  double fl = 0, by = 0;
  for (int i = 0; i < b.n; ++i) {
    const auto& d = b.d[i];
    fl += (d.upper_only ? 4.0 : 8.0) * d.M * d.N * d.K;
    by += 16.0 * ((double)d.M * d.K + (double)d.K * d.N + (double)d.M * d.N);
  }
  auto run = [&](int c) {
    const int bm = c == 0 ? 64 : 32;
    int maxt = 0;
    for (int i = 0; i < b.n; ++i) {
      const auto& d = b.d[i];
      if (d.M <= 0 || d.N <= 0) continue;
      maxt = std::max(maxt, cdiv(d.M, bm) * cdiv(d.N, bm));
    }
    ProfScope ps(prof_name, s, fl, by);
    dim3 grid(maxt, b.n);
    if (c == 0) zgemm_kernel<4><<<grid, 256, 0, s>>>(b);
    else zgemm_kernel<2><<<grid, 256, 0, s>>>(b);
    LAUNCH_CHECK();
    ++g_launches;
  };
  if (!tune_enabled()) run(0);
  else tune_pick(TUNE_ZGEMM, M, N, K, b.n, 2, !acc, run, s);
}

// ---------------------------------------------------------------------------
// Complex GEMM in double-float: the zgemm_kernel tiling, operands converted to
// (hi, lo) pairs when staged in shared memory, each product's leading term
// exact through FMA and accumulated with two_sum, the small terms in FP32.
// ---------------------------------------------------------------------------
template <int TT>  // outputs per thread along each side: tile (16 TT) x (16 TT)
__global__ void __launch_bounds__(256) zgemm_dd_kernel(const __grid_constant__ ZGemmBatch batch) {
  constexpr int BM = 16 * TT, BN = 16 * TT;
  const int pid = blockIdx.y;
  if (pid >= batch.n) return;
  const ZGemmDesc& P = batch.d[pid];
  if (P.skip && *P.skip) return;
  const int tiles_m = (P.M + BM - 1) / BM;
  const int tiles_n = (P.N + BN - 1) / BN;
  if ((int)blockIdx.x >= tiles_m * tiles_n) return;
  const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
  const int m0 = tm * BM, n0 = tn * BN;
  // Hermitian results: the blocks of 64 on or above the diagonal (any tile size)
  if (P.upper_only && m0 / 64 > n0 / 64) return;
  __shared__ float4 As[ZG_BK][BM];  // (re_hi, im_hi, re_lo, im_lo)
  __shared__ float4 Bs[ZG_BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  // accumulators as packed pairs: S = (sr, si), C = (cr, ci)
  f32x2 S2[TT][TT], C2[TT][TT];
#pragma unroll
  for (int i = 0; i < TT; ++i)
#pragma unroll
    for (int j = 0; j < TT; ++j) S2[i][j] = C2[i][j] = 0ull;
  const bool a_k_fast = (P.a_cs == 1);
  const bool b_n_fast = (P.b_cs == 1);
  for (int k0 = 0; k0 < P.K; k0 += ZG_BK) {
#pragma unroll
    for (int r = 0; r < (ZG_BK * BM) / 256; ++r) {
      int e = tid + r * 256;
      int i, k;
      if (a_k_fast) {
        k = e % ZG_BK;
        i = e / ZG_BK;
      } else {
        i = e % BM;
        k = e / BM;
      }
      double2 v = make_double2(0.0, 0.0);
      int gi = m0 + i, gk = k0 + k;
      if (gi < P.M && gk < P.K) {
        v = P.A[(int64_t)gi * P.a_rs + (int64_t)gk * P.a_cs];
        if (P.conj_a) v.y = -v.y;
        if (P.kscale) {
          double sc = P.kscale[gk];
          v.x *= sc;
          v.y *= sc;
        }
      }
      {
        const float2 re = dd_split(v.x), im = dd_split(v.y);
        As[k][i] = make_float4(re.x, im.x, re.y, im.y);
      }
      int j, kb;
      if (b_n_fast) {
        j = e % BN;
        kb = e / BN;
      } else {
        kb = e % ZG_BK;
        j = e / ZG_BK;
      }
      double2 w = make_double2(0.0, 0.0);
      int gj = n0 + j, gkb = k0 + kb;
      if (gj < P.N && gkb < P.K) {
        w = P.B[(int64_t)gkb * P.b_rs + (int64_t)gj * P.b_cs];
        if (P.conj_b) w.y = -w.y;
      }
      {
        const float2 re = dd_split(w.x), im = dd_split(w.y);
        Bs[kb][j] = make_float4(re.x, im.x, re.y, im.y);
      }
    }
    __syncthreads();
#pragma unroll 2
    for (int kk = 0; kk < ZG_BK; ++kk) {
      // re += a.re b.re - a.im b.im ; im += a.re b.im + a.im b.re, as two packed
      // compensated accumulations per product (the scalar form's four, in the
      // same order per lane): (sr, si) += (a.re, a.re) (b.re, b.im), then
      // (sr, si) += (-a.im, a.im) (b.im, b.re)
      f32x2 bh[TT], bl[TT], bsh[TT], bsl[TT];
#pragma unroll
      for (int j = 0; j < TT; ++j) {
        const float4 b = Bs[kk][tx + 16 * j];
        bh[j] = pk2(b.x, b.y);
        bl[j] = pk2(b.z, b.w);
        bsh[j] = pk2(b.y, b.x);
        bsl[j] = pk2(b.w, b.z);
      }
#pragma unroll
      for (int i = 0; i < TT; ++i) {
        const float4 a = As[kk][ty + 16 * i];
        const f32x2 rh = pk2(a.x, a.x), nrh = pk2(-a.x, -a.x), rl = pk2(a.z, a.z);
        const f32x2 ih = pk2(-a.y, a.y), nih = pk2(a.y, -a.y), il = pk2(-a.w, a.w);
#pragma unroll
        for (int j = 0; j < TT; ++j) {
          dd_acc2(S2[i][j], C2[i][j], rh, nrh, rl, bh[j], bl[j]);
          dd_acc2(S2[i][j], C2[i][j], ih, nih, il, bsh[j], bsl[j]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TT; ++i) {
    int gi = m0 + ty + 16 * i;
    if (gi >= P.M) continue;
#pragma unroll
    for (int j = 0; j < TT; ++j) {
      int gj = n0 + tx + 16 * j;
      if (gj >= P.N) continue;
      double2* c = P.C + (int64_t)gi * P.c_rs + (int64_t)gj * P.c_cs;
      const float2 sv = upk2(S2[i][j]), cv = upk2(C2[i][j]);
      double2 v = make_double2((double)sv.x + (double)cv.x, (double)sv.y + (double)cv.y);
      if (P.accumulate) v = zadd(v, *c);
      *c = v;
    }
  }
}

void launch_zgemm_dd(const ZGemmBatch& b, cudaStream_t s, const char* prof_name) {
  if (b.n <= 0) return;
  int64_t M, N, K;
  bool acc;
  batch_shape(b, M, N, K, acc);
  if (M <= 0 || N <= 0) return;
  double fl = 0, by = 0;
  for (int i = 0; i < b.n; ++i) {
    const auto& d = b.d[i];
    fl += (d.upper_only ? 4.0 : 8.0) * d.M * d.N * d.K;
    by += 16.0 * ((double)d.M * d.K + (double)d.K * d.N + (double)d.M * d.N);
  }
  auto run = [&](int c) {
    const int tt = c == 0 ? 4 : 2;
    const int bm = 16 * tt;
    int maxt = 0;
    for (int i = 0; i < b.n; ++i) {
      const auto& d = b.d[i];
      if (d.M <= 0 || d.N <= 0) continue;
      maxt = std::max(maxt, cdiv(d.M, bm) * cdiv(d.N, bm));
    }
    ProfScope ps(prof_name, s, fl, by);
    dim3 grid(maxt, b.n);
    if (tt == 4) zgemm_dd_kernel<4><<<grid, 256, 0, s>>>(b);
    else zgemm_dd_kernel<2><<<grid, 256, 0, s>>>(b);
    LAUNCH_CHECK();
    ++g_launches;
  };
  if (!tune_enabled()) {
    // fixed rule: 64 x 64 tiles when the batch fills the GPU, else 32 x 32 (4x the CTAs)
    int64_t tiles64 = 0;
    for (int i = 0; i < b.n; ++i) tiles64 += (int64_t)cdiv(b.d[i].M, 64) * cdiv(b.d[i].N, 64);
    run(tiles64 >= 2 * 152 ? 0 : 1);
  } else {
    tune_pick(TUNE_ZGEMM_DD, M, N, K, b.n, 2, !acc, run, s);
  }
}

// ---------------------------------------------------------------------------
// W stage: Y[a, w', S, b] = sum_{w, S'} Wop[w, w', S, S'] X[a, w, S', b].
// One thread per output element, b fastest; the block list of each w' is
// read from global memory (a few KB, cached).
// ---------------------------------------------------------------------------
__device__ inline float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <typename T>
struct Acc;
template <>
struct Acc<double2> {
  using blk_t = double2;
  __device__ static const double2* blk(const WOp& W) { return W.blk64; }
  __device__ static void fma(double2& a, double2 w, double2 x) { zfma(a, w, x); }
};
template <>
struct Acc<float2> {
  using blk_t = float2;
  __device__ static const float2* blk(const WOp& W) { return W.blk32; }
  __device__ static void fma(float2& a, float2 w, float2 x) { cfma(a, w, x); }
};

template <typename T>
__global__ void __launch_bounds__(256) wstage_kernel(const __grid_constant__ WStageBatch<T> batch) {
  const int pid = blockIdx.y;
  if (pid >= batch.n) return;
  const WStageDesc<T>& P = batch.d[pid];
  if (P.skip && *P.skip) return;
  const int D = P.W.D, m = P.W.m;
  const int64_t total = (int64_t)P.A * m * D * P.B;
  const auto* blk = Acc<T>::blk(P.W);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = idx;
    const int b = (int)(r % P.B);
    r /= P.B;
    const int S = (int)(r % D);
    r /= D;
    const int wo = (int)(r % m);
    const int a = (int)(r / m);
    T acc;
    acc.x = 0;
    acc.y = 0;
    const T* xa = P.X + (int64_t)a * P.x_a + (int64_t)b * P.x_b;
    for (int q = P.W.col_ptr[wo]; q < P.W.col_ptr[wo + 1]; ++q) {
      const int wi = P.W.row_idx[q];
      const auto* bq = blk + (int64_t)q * D * D + (int64_t)S * D;
      const T* xw = xa + (int64_t)wi * P.x_w;
      for (int s2 = 0; s2 < D; ++s2) Acc<T>::fma(acc, bq[s2], xw[(int64_t)s2 * P.x_s]);
    }
    const int64_t o = (int64_t)a * P.y_a + (int64_t)wo * P.y_w + (int64_t)S * P.y_s + (int64_t)b * P.y_b;
    if constexpr (sizeof(T) == sizeof(float2)) {
      if (batch.round_tf32) {
        float2 hi = make_float2(tf32_round(acc.x), tf32_round(acc.y));
        P.Y[o] = hi;
        if (P.Ylo) P.Ylo[o] = make_float2(tf32_round(acc.x - hi.x), tf32_round(acc.y - hi.y));
      } else {
        P.Y[o] = acc;
      }
    } else {
      P.Y[o] = acc;
    }
  }
}

template <typename T>
static void launch_wstage_t(const WStageBatch<T>& b, cudaStream_t s) {
  if (b.n <= 0) return;
  int64_t maxt = 0;
  for (int i = 0; i < b.n; ++i)
    maxt = std::max(maxt, (int64_t)b.d[i].A * b.d[i].W.m * b.d[i].W.D * b.d[i].B);
  if (maxt == 0) return;
  int blocks = (int)std::min<int64_t>(cdiv64(maxt, 256), 152 * 16);
  double fl = 0, by = 0;
  for (int i = 0; i < b.n; ++i) {
    const auto& d = b.d[i];
    const double outs = (double)d.A * d.W.m * d.W.D * d.B;
    fl += 8.0 * d.A * d.B * (double)d.W.D * d.W.D * d.W.nnz;
    by += 2.0 * outs * sizeof(T) * ((d.Ylo ? 1.5 : 1.0));
  }
  ProfScope ps(sizeof(T) == 16 ? "wstage_fp64" : "wstage_fp32", s, fl, by);
  dim3 grid(blocks, b.n);
  wstage_kernel<T><<<grid, 256, 0, s>>>(b);
  LAUNCH_CHECK();
  ++g_launches;
}
void launch_wstage(const WStageBatch<double2>& b, cudaStream_t s) { launch_wstage_t(b, s); }
void launch_wstage(const WStageBatch<float2>& b, cudaStream_t s) { launch_wstage_t(b, s); }

// ---------------------------------------------------------------------------
// dst = src scaled along its first (left) or last (right) bond index.
// ---------------------------------------------------------------------------
__global__ void scale_bond_kernel(const __grid_constant__ ScaleBatch batch) {
  const int pid = blockIdx.y;
  if (pid >= batch.n) return;
  const ScaleDesc& P = batch.d[pid];
  const int64_t total = (int64_t)P.rows * P.d * P.cols;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int c = (int)(i % P.cols);
    int r = (int)(i / ((int64_t)P.d * P.cols));
    double sc = P.left ? P.v[r] : P.v[c];
    double2 x = P.src[i];
    double2 o = make_double2(x.x * sc, x.y * sc);
    if (P.src2) {
      const double s2 = P.left ? P.v2[r] : P.v2[c];
      const double2 x2 = P.src2[i];
      o.x = fma(x2.x, s2, o.x);
      o.y = fma(x2.y, s2, o.y);
    }
    P.dst[i] = o;
  }
}

void launch_scale_bond(const ScaleBatch& b, cudaStream_t s) {
  if (b.n <= 0) return;
  int64_t maxt = 0;
  for (int i = 0; i < b.n; ++i) maxt = std::max(maxt, (int64_t)b.d[i].rows * b.d[i].d * b.d[i].cols);
  if (maxt == 0) return;
  double by = 0;
  for (int i = 0; i < b.n; ++i) by += 32.0 * b.d[i].rows * b.d[i].d * b.d[i].cols;
  ProfScope ps("scale_bond", s, 0.0, by);
  dim3 grid((unsigned)std::min<int64_t>(cdiv64(maxt, 256), 152 * 8), b.n);
  scale_bond_kernel<<<grid, 256, 0, s>>>(b);
  LAUNCH_CHECK();
  ++g_launches;
}

// ---------------------------------------------------------------------------
// Operand preparation for the tensor-core GEMM (see PrepDesc). Threads run
// along the source's contiguous index.
// ---------------------------------------------------------------------------
__global__ void prep_kernel(const __grid_constant__ PrepBatch batch) {
  const int pid = blockIdx.y;
  if (pid >= batch.n) return;
  const PrepDesc& P = batch.d[pid];
  if (P.skip && *P.skip) return;
  const int64_t total = (int64_t)P.rows * P.cols;
  const bool row_fast = (P.rs == 1 && P.cs != 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int r, k;
    if (row_fast) {
      r = (int)(i % P.rows);
      k = (int)(i / P.rows);
    } else {
      k = (int)(i % P.cols);
      r = (int)(i / P.cols);
    }
    double2 v;
    if (P.src) {
      v = P.src[(int64_t)r * P.rs + (int64_t)k * P.cs];
    } else {
      float2 f = P.src32[(int64_t)r * P.rs + (int64_t)k * P.cs];
      v = make_double2((double)f.x, (double)f.y);
    }
    if (P.conj) v.y = -v.y;
    float re = (float)v.x, im = (float)v.y;
    float hre = tf32_round(re), him = tf32_round(im);
    float lre = tf32_round((float)(v.x - (double)hre)), lim = tf32_round((float)(v.y - (double)him));
    if (!P.embed) {
      int64_t o = (int64_t)r * P.ld + 2 * (int64_t)k;
      *reinterpret_cast<float2*>(P.hi + o) = make_float2(hre, him);
      if (P.lo) *reinterpret_cast<float2*>(P.lo + o) = make_float2(lre, lim);
    } else {
      int64_t o0 = (int64_t)(2 * r) * P.ld + 2 * (int64_t)k;
      int64_t o1 = o0 + P.ld;
      *reinterpret_cast<float2*>(P.hi + o0) = make_float2(hre, -him);
      *reinterpret_cast<float2*>(P.hi + o1) = make_float2(him, hre);
      if (P.lo) {
        *reinterpret_cast<float2*>(P.lo + o0) = make_float2(lre, -lim);
        *reinterpret_cast<float2*>(P.lo + o1) = make_float2(lim, lre);
      }
    }
  }
}

void launch_prep(const PrepBatch& b, cudaStream_t s) {
  if (b.n <= 0) return;
  int64_t maxt = 0;
  for (int i = 0; i < b.n; ++i) maxt = std::max(maxt, (int64_t)b.d[i].rows * b.d[i].cols);
  if (maxt == 0) return;
  double by = 0;
  for (int i = 0; i < b.n; ++i)
    by += (double)b.d[i].rows * b.d[i].cols * (16.0 + (b.d[i].embed ? 16.0 : 8.0) * (b.d[i].lo ? 2 : 1));
  ProfScope ps("prep_operands", s, 0.0, by);
  dim3 grid((unsigned)std::min<int64_t>(cdiv64(maxt, 256), 152 * 16), b.n);
  prep_kernel<<<grid, 256, 0, s>>>(b);
  LAUNCH_CHECK();
  ++g_launches;
}

}  // namespace tdvp
