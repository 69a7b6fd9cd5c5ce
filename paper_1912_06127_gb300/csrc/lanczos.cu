// Lanczos exponentiation exp(-i t H) x (Park and Light), batched over the
// local problems of a stage; in ground mode the lowest Ritz vector instead
// (the two-site DMRG update). Only products H v are needed (Sec. III A), which
// the caller provides as batched launches between the steps below.
//
// Per Krylov vector j (all problems of the batch at once, each with its own
// length, time and stopping state held in device memory):
//   w = H v_j                      (caller's matvec, writes v_{j+1} slot)
//   h_i = <v_i, w>, w -= sum h_i v_i        (classical Gram-Schmidt, pass 1)
//   g_i = <v_i, w>, w -= sum g_i v_i        (pass 2: full re-orthogonalisation)
//   alpha_j = Re(h_j + g_j), beta_{j+1} = ||w||
//   c = exp(-i t T_{j+1}) e_0, error estimate beta_{j+1} |c_j|
//   stop on breakdown (beta_{j+1} <= 1e-12 (|alpha_j| + beta_j)), on the
//   estimate falling below tol, or at kmax vectors; else v_{j+1} = w / beta_{j+1}
// Finally y = ||x|| sum_i c_i v_i.
// All reductions are two-level (per-block partials, then a fixed-order sum
// in the last block to arrive), so results do not depend on scheduling.
#include "common.h"
#include "lanczos.h"
#include "tridiag.h"

namespace tdvp {

constexpr int LZ_THREADS = 256;
constexpr int LZ_ELEMS = 8;  // elements per thread per block-chunk

__device__ inline double2 warp_sum2(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Reduce `cnt` complex values per thread over the block; result valid in
// thread 0 in out[]. scratch: [LZ_THREADS/32][cnt]
__device__ inline void block_sum(const double2* vals, int cnt, double2* scratch, double2* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < KRYLOV_MAX; ++i) {
    if (i >= cnt) break;
    double2 v = warp_sum2(vals[i]);
    if (lane == 0) scratch[warp * KRYLOV_MAX + i] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < cnt; ++i) {
      double2 acc = make_double2(0, 0);
      for (int w = 0; w < LZ_THREADS / 32; ++w) acc = zadd(acc, scratch[w * KRYLOV_MAX + i]);
      out[i] = acc;
    }
  }
  __syncthreads();
}

// Returns true in thread 0 of the last block of problem `p` to finish.
__device__ inline bool last_block(int* counter, int nblk) {
  __shared__ int is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    int prev = atomicAdd(counter, 1);
    is_last = (prev == nblk - 1);
    if (is_last) *counter = 0;
  }
  __syncthreads();
  return is_last != 0;
}

__device__ inline int lz_nblk(int64_t n) {
  int64_t per = (int64_t)LZ_THREADS * LZ_ELEMS;
  int64_t b = (n + per - 1) / per;
  return (int)(b < 1 ? 1 : b);
}

// ---- start: beta0 = ||x||, v_0 = x / beta0 --------------------------------
__global__ void __launch_bounds__(LZ_THREADS) lz_start_norm(const __grid_constant__ LzBatch B) {
  const LzDesc& P = B.d[blockIdx.y];
  const int nblk = lz_nblk(P.n);
  if ((int)blockIdx.x >= nblk) return;
  __shared__ double2 scratch[(LZ_THREADS / 32) * KRYLOV_MAX];
  __shared__ double2 tot[1];
  double2 s = make_double2(0, 0);
  const int64_t base = (int64_t)blockIdx.x * LZ_THREADS * LZ_ELEMS;
  for (int e = 0; e < LZ_ELEMS; ++e) {
    int64_t i = base + (int64_t)e * LZ_THREADS + threadIdx.x;
    if (i < P.n) {
      double2 v = P.x[i];
      s.x += v.x * v.x + v.y * v.y;
    }
  }
  block_sum(&s, 1, scratch, tot);
  double2* part = P.part + (int64_t)blockIdx.x * KRYLOV_MAX;
  if (threadIdx.x == 0) part[0] = tot[0];
  if (last_block(P.counter, nblk) && threadIdx.x == 0) {
    double acc = 0;
    for (int b = 0; b < nblk; ++b) acc += P.part[(int64_t)b * KRYLOV_MAX].x;
    LzState* st = P.st;
    st->beta0 = sqrt(acc);
    st->t = P.t;
    st->tol = P.tol;
    st->kmax = P.kmax;
    st->ground = P.ground;
    st->energy = 0.0;
    st->k = 0;
    st->err = 0;
    st->nvec_used = 0;
    st->done = (acc == 0.0) ? 1 : 0;
    if (!(acc == acc)) {
      st->done = 1;
      atomicOr(B.status, 2);
    }
  }
}

__global__ void __launch_bounds__(LZ_THREADS) lz_start_scale(const __grid_constant__ LzBatch B) {
  const LzDesc& P = B.d[blockIdx.y];
  const LzState* st = P.st;
  if (st->done) return;
  const double inv = 1.0 / st->beta0;
  for (int64_t i = (int64_t)blockIdx.x * LZ_THREADS + threadIdx.x; i < P.n;
       i += (int64_t)gridDim.x * LZ_THREADS) {
    double2 v = P.x[i];
    P.V[i] = make_double2(v.x * inv, v.y * inv);
  }
}

// ---- pass: coefficients <v_i, w> for i <= j --------------------------------
template <int NMAX>
__global__ void __launch_bounds__(LZ_THREADS) lz_dots(const __grid_constant__ LzBatch B, int j,
                                                      int pass) {
  const LzDesc& P = B.d[blockIdx.y];
  if (P.st->done) return;
  const int nblk = lz_nblk(P.n);
  if ((int)blockIdx.x >= nblk) return;
  __shared__ double2 scratch[(LZ_THREADS / 32) * KRYLOV_MAX];
  __shared__ double2 tot[KRYLOV_MAX];
  // accumulators indexed by compile-time constants only (registers, no local
  // memory); NMAX >= j + 1 is chosen at launch
  double2 acc[NMAX];
  const int cnt = j + 1;
#pragma unroll
  for (int i = 0; i < NMAX; ++i) acc[i] = make_double2(0, 0);
  const double2* w = P.V + (int64_t)(j + 1) * P.vs;
  const int64_t base = (int64_t)blockIdx.x * LZ_THREADS * LZ_ELEMS;
  for (int e = 0; e < LZ_ELEMS; ++e) {
    int64_t idx = base + (int64_t)e * LZ_THREADS + threadIdx.x;
    if (idx >= P.n) break;
    double2 wv = w[idx];
#pragma unroll
    for (int i = 0; i < NMAX; ++i)
      if (i < cnt) zfma_cj(acc[i], P.V[(int64_t)i * P.vs + idx], wv);
  }
  block_sum(acc, cnt, scratch, tot);
  double2* part = P.part + (int64_t)blockIdx.x * KRYLOV_MAX;
  if (threadIdx.x == 0)
    for (int i = 0; i < cnt; ++i) part[i] = tot[i];
  if (last_block(P.counter, nblk) && threadIdx.x == 0) {
    double2* dst = pass == 0 ? P.st->h : P.st->g;
    for (int i = 0; i < cnt; ++i) {
      double2 s = make_double2(0, 0);
      for (int b = 0; b < nblk; ++b) s = zadd(s, P.part[(int64_t)b * KRYLOV_MAX + i]);
      dst[i] = s;
    }
  }
}

// ---- pass: w -= sum_i coef_i v_i; pass 1 also finishes the Krylov step ------
__global__ void __launch_bounds__(LZ_THREADS) lz_update(const __grid_constant__ LzBatch B, int j,
                                                        int pass) {
  const LzDesc& P = B.d[blockIdx.y];
  LzState* st = P.st;
  if (st->done) return;
  const int nblk = lz_nblk(P.n);
  if ((int)blockIdx.x >= nblk) return;
  __shared__ double2 scratch[(LZ_THREADS / 32) * KRYLOV_MAX];
  __shared__ double2 tot[1];
  __shared__ double2 coef[KRYLOV_MAX];
  __shared__ double work[2 * KRYLOV_MAX * KRYLOV_MAX];  // tridiagonal solver, last block only
  const int cnt = j + 1;
  if (threadIdx.x < cnt) coef[threadIdx.x] = pass == 0 ? st->h[threadIdx.x] : st->g[threadIdx.x];
  __syncthreads();
  double2* w = P.V + (int64_t)(j + 1) * P.vs;
  double2 nrm = make_double2(0, 0);
  const int64_t base = (int64_t)blockIdx.x * LZ_THREADS * LZ_ELEMS;
  for (int e = 0; e < LZ_ELEMS; ++e) {
    int64_t idx = base + (int64_t)e * LZ_THREADS + threadIdx.x;
    if (idx >= P.n) break;
    double2 wv = w[idx];
    for (int i = 0; i < cnt; ++i) {
      double2 v = P.V[(int64_t)i * P.vs + idx];
      double2 c = coef[i];
      wv.x -= c.x * v.x - c.y * v.y;
      wv.y -= c.x * v.y + c.y * v.x;
    }
    w[idx] = wv;
    nrm.x += wv.x * wv.x + wv.y * wv.y;
  }
  if (pass == 0) return;
  block_sum(&nrm, 1, scratch, tot);
  double2* part = P.part + (int64_t)blockIdx.x * KRYLOV_MAX;
  if (threadIdx.x == 0) part[0] = tot[0];
  if (last_block(P.counter, nblk) && threadIdx.x == 0) {
    double s = 0;
    for (int b = 0; b < nblk; ++b) s += P.part[(int64_t)b * KRYLOV_MAX].x;
    const double bnorm = sqrt(s);
    st->alpha[j] = st->h[j].x + st->g[j].x;
    const int k = j + 1;
    int rc;
    if (st->ground) {
      // lowest Ritz pair; the estimate below is then the residual beta_{j+1} |z_j|
      double e0 = 0.0;
      rc = tridiag_ground_impl(k, st->alpha, st->beta, st->c, &e0, work);
      st->energy = e0;
    } else {
      rc = tridiag_expm_e0_impl(k, st->alpha, st->beta, st->t, st->c, work);
    }
    if (rc < 0) atomicOr(B.status, 4);
    const double2 ck = st->c[j];
    st->err = bnorm * sqrt(ck.x * ck.x + ck.y * ck.y);
    st->nvec_used = k;
    st->k = k;
    const double scale = fabs(st->alpha[j]) + (j > 0 ? st->beta[j - 1] : 0.0);
    if (!(bnorm == bnorm)) {
      st->done = 1;
      atomicOr(B.status, 2);
    } else if (bnorm <= 1e-12 * scale) {
      st->done = 1;
    } else if (st->tol > 0.0 && st->err < st->tol) {
      st->done = 1;
    } else if (k >= st->kmax) {
      st->done = 1;
    } else {
      st->beta[j] = bnorm;
    }
  }
}

__global__ void __launch_bounds__(LZ_THREADS) lz_normalize(const __grid_constant__ LzBatch B, int j) {
  const LzDesc& P = B.d[blockIdx.y];
  const LzState* st = P.st;
  if (st->done) return;
  const double inv = 1.0 / st->beta[j];
  double2* w = P.V + (int64_t)(j + 1) * P.vs;
  for (int64_t i = (int64_t)blockIdx.x * LZ_THREADS + threadIdx.x; i < P.n;
       i += (int64_t)gridDim.x * LZ_THREADS) {
    double2 v = w[i];
    w[i] = make_double2(v.x * inv, v.y * inv);
  }
}

__global__ void __launch_bounds__(LZ_THREADS) lz_combine(const __grid_constant__ LzBatch B) {
  const LzDesc& P = B.d[blockIdx.y];
  const LzState* st = P.st;
  __shared__ double2 coef[KRYLOV_MAX];
  const int cnt = st->nvec_used;
  const double b0 = st->beta0;
  if (threadIdx.x < cnt) coef[threadIdx.x] = zscale(st->c[threadIdx.x], b0);
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * LZ_THREADS + threadIdx.x; i < P.n;
       i += (int64_t)gridDim.x * LZ_THREADS) {
    double2 acc = make_double2(0, 0);
    for (int q = 0; q < cnt; ++q) zfma(acc, coef[q], P.V[(int64_t)q * P.vs + i]);
    if (b0 == 0.0) acc = make_double2(0, 0);
    P.y[i] = acc;
  }
}

// ---------------------------------------------------------------------------
static dim3 lz_grid(const LzBatch& b, bool chunked) {
  int64_t nmax = 1;
  for (int i = 0; i < b.n; ++i) nmax = std::max<int64_t>(nmax, b.d[i].n);
  int blocks;
  if (chunked) {
    int64_t per = (int64_t)LZ_THREADS * LZ_ELEMS;
    blocks = (int)((nmax + per - 1) / per);
  } else {
    blocks = (int)std::min<int64_t>(cdiv64(nmax, LZ_THREADS), 152 * 4);
  }
  return dim3(std::max(blocks, 1), b.n);
}

int lz_max_blocks(int64_t n) {
  int64_t per = (int64_t)LZ_THREADS * LZ_ELEMS;
  return (int)std::max<int64_t>(1, (n + per - 1) / per);
}

void lz_start(const LzBatch& b, cudaStream_t s) {
  if (b.n <= 0) return;
  lz_start_norm<<<lz_grid(b, true), LZ_THREADS, 0, s>>>(b);
  LAUNCH_CHECK();
  lz_start_scale<<<lz_grid(b, false), LZ_THREADS, 0, s>>>(b);
  LAUNCH_CHECK();
  g_launches += 2;
}

void lz_orthogonalize(const LzBatch& b, int j, cudaStream_t s) {
  if (b.n <= 0) return;
  double n_all = 0;
  for (int i = 0; i < b.n; ++i) n_all += (double)b.d[i].n;
  // bytes: 2 passes x (dots: j+2 vectors read; update: j+2 read + 1 write) + normalize
  ProfScope ps("lanczos_orth", s, 2.0 * 2 * 8.0 * (j + 1) * n_all,
               16.0 * n_all * (2.0 * ((j + 2) + (j + 3)) + 2.0));
  for (int pass = 0; pass < 2; ++pass) {
    if (j + 1 <= 8) lz_dots<8><<<lz_grid(b, true), LZ_THREADS, 0, s>>>(b, j, pass);
    else if (j + 1 <= 16) lz_dots<16><<<lz_grid(b, true), LZ_THREADS, 0, s>>>(b, j, pass);
    else lz_dots<KRYLOV_MAX><<<lz_grid(b, true), LZ_THREADS, 0, s>>>(b, j, pass);
    LAUNCH_CHECK();
    lz_update<<<lz_grid(b, true), LZ_THREADS, 0, s>>>(b, j, pass);
    LAUNCH_CHECK();
  }
  lz_normalize<<<lz_grid(b, false), LZ_THREADS, 0, s>>>(b, j);
  LAUNCH_CHECK();
  g_launches += 5;
}

// count of problems still iterating, written to host-mapped memory
__global__ void lz_count_open(const __grid_constant__ LzBatch B, int* out) {
  __shared__ int open;
  if (threadIdx.x == 0) open = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < B.n; i += blockDim.x)
    if (!B.d[i].st->done) atomicAdd(&open, 1);
  __syncthreads();
  if (threadIdx.x == 0) *(volatile int*)out = open;
}

bool lz_all_done(const LzBatch& b, cudaStream_t s) {
  thread_local int* h_open = nullptr;
  thread_local int* d_open = nullptr;
  thread_local int dev_of = -1;
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (!h_open || dev_of != dev) {
    CUDA_TRY(cudaHostAlloc((void**)&h_open, sizeof(int), cudaHostAllocMapped));
    CUDA_TRY(cudaHostGetDevicePointer((void**)&d_open, h_open, 0));
    dev_of = dev;
  }
  *h_open = 1;
  lz_count_open<<<1, 64, 0, s>>>(b, d_open);
  LAUNCH_CHECK();
  ++g_launches;
  CUDA_TRY(cudaStreamSynchronize(s));
  return *(volatile int*)h_open == 0;
}

void lz_finish(const LzBatch& b, cudaStream_t s) {
  if (b.n <= 0) return;
  lz_combine<<<lz_grid(b, false), LZ_THREADS, 0, s>>>(b);
  LAUNCH_CHECK();
  g_launches += 1;
}

}  // namespace tdvp
