// Internal declarations shared by the translation units of libtdvp.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <functional>
#include <string>
#include <vector>

#include "tdvp.h"

namespace tdvp {

// ---------------------------------------------------------------------------
// Errors: internal code throws TdvpError; the C ABI converts it to a code.
// ---------------------------------------------------------------------------
struct TdvpError {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string& msg);
void cuda_check(cudaError_t e, const char* what, const char* file, int line);
#define CUDA_TRY(x) ::tdvp::cuda_check((x), #x, __FILE__, __LINE__)
#define LAUNCH_CHECK() ::tdvp::cuda_check(cudaGetLastError(), "kernel launch", __FILE__, __LINE__)

// Global counter of kernels launched (for the statistics only).
extern int64_t g_launches;

// GEMM tile autotuner (tune.cu): run(c) launches candidate c of a family
// (candidate 0 is the default); the first launch with a new shape key times
// every candidate and keeps the fastest. may_repeat = false (the launch
// accumulates into its output) always runs candidate 0 untuned.
enum { TUNE_TC_TF32 = 0, TUNE_TC_TF32X3 = 1, TUNE_ZGEMM = 2, TUNE_ZGEMM_DD = 3 };
int tune_pick(int family, int64_t M, int64_t N, int64_t K, int n, int n_cand, bool may_repeat,
              const std::function<void(int)>& run, cudaStream_t s);
void tune_enable(bool on);  // clears the decisions
bool tune_enabled();
std::string tune_report();  // the decisions as a JSON list

// Optional per-kernel timing with CUDA events recorded on the launching
// stream around each launch (enabled by tdvp_profile). `flops` and `bytes`
// are the algorithmic work of the launch.
extern bool g_prof_on;
struct ProfScope {
  int slot = -1;
  cudaStream_t s = 0;
  ProfScope(const char* name, cudaStream_t s, double flops, double bytes, const double* dev_flops_host = nullptr);
  ~ProfScope();
};
void prof_enable(bool on);
// two doubles: [0] work (flops) and [1] an auxiliary count, written by the kernel
double* prof_work_slot(double** dev);
void op_heff_noalloc(int nsite, int chi_l, int chi_r, int m, int d, const double* W, const double* L,
                     const double* R, const double* x, double* y, cudaStream_t s);
int prof_read(int idx, std::string& name, double& ms, int64_t& launches, double& flops, double& bytes,
              double& aux);

// ---------------------------------------------------------------------------
// Complex helpers (double2 / float2 hold re, im)
// ---------------------------------------------------------------------------
__host__ __device__ inline double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ inline double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 zscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// a += b * c
__host__ __device__ inline void zfma(double2& a, double2 b, double2 c) {
  a.x = fma(b.x, c.x, a.x);
  a.x = fma(-b.y, c.y, a.x);
  a.y = fma(b.x, c.y, a.y);
  a.y = fma(b.y, c.x, a.y);
}
// a += conj(b) * c
__host__ __device__ inline void zfma_cj(double2& a, double2 b, double2 c) {
  a.x = fma(b.x, c.x, a.x);
  a.x = fma(b.y, c.y, a.x);
  a.y = fma(b.x, c.y, a.y);
  a.y = fma(-b.y, c.x, a.y);
}
__host__ __device__ inline void cfma(float2& a, float2 b, float2 c) {
  a.x = fmaf(b.x, c.x, a.x);
  a.x = fmaf(-b.y, c.y, a.x);
  a.y = fmaf(b.x, c.y, a.y);
  a.y = fmaf(b.y, c.x, a.y);
}

// ---- double-float arithmetic (error-free transformations with FMA) ----
// A double-float value is hi + lo with two FP32 numbers (~48 significant
// bits); on GB300 it is computed on the FP32 pipe, 64x wider than FP64.
// two_sum: s + e = a + b exactly; fast_two_sum needs |a| >= |b|.
__device__ inline void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ inline void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
// compensated accumulation of (ah + al)(bh + bl) into the pair (s, c): the
// leading product exactly (FMA), the cross terms in plain FP32
__device__ inline void dd_acc(float& s, float& c, float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  const float e = fmaf(ah, bh, -p);
  float t;
  two_sum(s, p, s, t);
  c += t + fmaf(ah, bl, fmaf(al, bh, e));
}
// ---- packed FP32 pairs (sm_100 and later: the .f32x2 forms of add, sub, mul
// and fma, two lanes per instruction, each lane rounded as its scalar form) ----
// A pair is a 64-bit register with its first element in the low half, as a
// float2 in memory.
typedef unsigned long long f32x2;
__device__ inline f32x2 pk2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ inline float2 upk2(f32x2 v) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
  return make_float2(lo, hi);
}
__device__ inline f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ inline f32x2 sub2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ inline f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ inline f32x2 fma2r(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ inline void fma2(f32x2& acc, f32x2 a, f32x2 b) { acc = fma2r(a, b, acc); }
// dd_acc on both lanes of the pairs (s, c) with the same operations in the
// same order as the scalar form, so each lane's result is bitwise the scalar
// one: nah = -ah (exact), so np = (-ah) bh = -p exactly, e = fma(ah, bh, np),
// s + p = s - np and p - bb = -(np + bb).
__device__ inline void dd_acc2(f32x2& s, f32x2& c, f32x2 ah, f32x2 nah, f32x2 al, f32x2 bh, f32x2 bl) {
  const f32x2 np = mul2(nah, bh);
  const f32x2 e = fma2r(ah, bh, np);
  const f32x2 s1 = sub2(s, np);
  const f32x2 bb = sub2(s1, s);
  const f32x2 t = sub2(sub2(s, sub2(s1, bb)), add2(np, bb));
  s = s1;
  c = add2(c, add2(t, fma2r(ah, bl, fma2r(al, bh, e))));
}
// double -> (hi, lo) floats
__device__ inline float2 dd_split(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

inline int cdiv(int a, int b) { return (a + b - 1) / b; }
inline int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

constexpr int MAXB = 32;        // largest batch of local problems in one launch
constexpr int KRYLOV_MAX = 24;  // largest Krylov dimension

// ---------------------------------------------------------------------------
// FP64 complex GEMM (SIMT), batched. op(A)(i,k) = A[i*a_rs + k*a_cs] (conj if
// conj_a, times kscale[k] if given); B(k,j) = B[k*b_rs + j*b_cs]; C(i,j) at
// C[i*c_rs + j*c_cs]; C = op(A) op(B) (+ C if accumulate).
// ---------------------------------------------------------------------------
struct ZGemmDesc {
  int M, N, K;
  int conj_a, conj_b, accumulate;
  int upper_only;         // only output blocks of 64 x 64 on or above the diagonal (Hermitian results)
  const int* skip;        // optional: nonzero -> problem skipped
  const double2* A;
  const double2* B;
  double2* C;
  const double* kscale;
  int64_t a_rs, a_cs, b_rs, b_cs, c_rs, c_cs;
};
struct ZGemmBatch {
  int n;
  ZGemmDesc d[MAXB];
};
void launch_zgemm(const ZGemmBatch& b, cudaStream_t s, const char* prof_name = "zgemm_fp64");
// The same product with double-float arithmetic on the FP32 pipe (inputs
// rounded to ~48 bits, compensated accumulation): for the mixed-precision
// path, where ~1e-14 relative accuracy is ample.
void launch_zgemm_dd(const ZGemmBatch& b, cudaStream_t s, const char* prof_name = "zgemm_dd");

// ---------------------------------------------------------------------------
// Sparse MPO operator applied in the "W stage" of a contraction:
// Y[a, w', S, b] = sum_{w, S'} Wop[w, w', S, S'] X[a, w, S', b]
// Blocks are grouped by w' (CSR over w'): blocks col_ptr[w']..col_ptr[w'+1]-1
// have w_left = row_idx[blk] and values blk64/blk32 [D][D] (S_out, S_in).
// ---------------------------------------------------------------------------
struct WOp {
  int m, D, nnz;
  const int* col_ptr;
  const int* row_idx;
  const double2* blk64;
  const float2* blk32;
};
template <typename T>
struct WStageDesc {
  int A, B;
  const int* skip;
  const T* X;
  int64_t x_a, x_w, x_s, x_b;
  T* Y;         // output (fp64 complex or fp32 complex)
  T* Ylo;       // fp32 only: optional second output holding x - tf32(x) (3xTF32 operands)
  int64_t y_a, y_w, y_s, y_b;
  WOp W;
};
template <typename T>
struct WStageBatch {
  int n;
  int round_tf32;  // fp32 only: round outputs to tf32 (and write Ylo residuals)
  WStageDesc<T> d[MAXB];
};
void launch_wstage(const WStageBatch<double2>& b, cudaStream_t s);
void launch_wstage(const WStageBatch<float2>& b, cudaStream_t s);

// ---------------------------------------------------------------------------
// Small elementwise kernels
// ---------------------------------------------------------------------------
// dst[i, s, j] = src[i, s, j] * (left ? v[i] : v[j]) for a [rows][d][cols] tensor
struct ScaleDesc {
  const double2* src;
  double2* dst;
  const double* v;
  int rows, d, cols, left;
  const double2* src2;  // optional: dst = src v + src2 v2 (tangent of a bond scaling)
  const double* v2;
};
struct ScaleBatch {
  int n;
  ScaleDesc d[MAXB];
};
void launch_scale_bond(const ScaleBatch& b, cudaStream_t s);

// ---------------------------------------------------------------------------
// Operand preparation for the tensor-core path.
//  A form: fp32 complex [M][K] row-major, row pitch lda (floats), from an
//          FP64 complex source with element (i,k) at src[i*rs + k*cs].
//  B form: the real embedding of a complex B (N x K, element (n,k) at
//          src[n*rs + k*cs]) as fp32 [2N][2K] rows, pitch ldb (floats):
//          row 2n = (Re b, -Im b) pairs, row 2n+1 = (Im b, Re b) pairs, so that
//          [A_re A_im ...] . row gives Re / Im of sum_k a_k b_k.
//  hi = tf32(x), lo = tf32(x - hi) when lo != nullptr; conj applies to src.
// ---------------------------------------------------------------------------
struct PrepDesc {
  const int* skip;
  const double2* src;
  const float2* src32;  // alternative fp32 complex source (src == nullptr)
  int64_t rs, cs;
  int rows, cols;     // complex rows (M or N) and complex K
  int conj;
  float* hi;
  float* lo;
  int64_t ld;         // row pitch of the destination in floats
  int embed;          // 0: A form, 1: B form
};
struct PrepBatch {
  int n;
  PrepDesc d[MAXB];
};
void launch_prep(const PrepBatch& b, cudaStream_t s);

// ---------------------------------------------------------------------------
// Tensor-core (tcgen05, kind::tf32) real GEMM, batched:
// C[M][N] = sum_pass A_pass[M][K] B_pass[N][K]^T, operands K-major fp32 in
// global memory, staged by TMA (128B swizzle) into shared memory,
// accumulated in TMEM (FP32). passes = 1 (A_hi B_hi) or 3 (+ A_hi B_lo + A_lo B_hi).
// Output: fp32 (c_fp64 = 0) or fp64 (c_fp64 = 1), row pitch ldc elements.
// ---------------------------------------------------------------------------
struct TcOperand {
  const float* hi;
  const float* lo;
  int rows, k;        // logical rows and K (floats)
  int64_t ld;         // row pitch in floats (multiple of 4)
};
struct TcProblem {
  const int* skip;
  TcOperand A, B;
  int M, N, K;
  void* C;
  int64_t ldc;
  int c_fp64;
  // K-split: the K range is cut into chunks of kchunk elements (a multiple of
  // 32; 0 = no split), each chunk's product is accumulated in FP32 into its own
  // partial tile part[chunk][M][N], and the partials are summed in FP64 into C.
  // FP32 accumulation error grows with the number of terms; the split bounds
  // it by the chunk length.
  float* part = nullptr;
  int kchunk = 0;
};
// Chooses the K-split of q for a partial buffer of cap floats: chunks of at
// least TC_KCHUNK_MIN elements, as few as fit; no split for short K.
constexpr int TC_KCHUNK_MIN = 512;
void tc_set_ksplit(TcProblem& q, float* part, int64_t cap);
void launch_tc_gemm(const std::vector<TcProblem>& probs, int passes, int* d_status, cudaStream_t s);
bool tc_available();

// ---------------------------------------------------------------------------
// Lanczos exponentiation, batched. Each problem evolves x (length n) by
// exp(-i t H) with H applied by a callback that runs one batched matvec.
// ---------------------------------------------------------------------------
struct LzState {
  double alpha[KRYLOV_MAX];
  double beta[KRYLOV_MAX];
  double2 h[KRYLOV_MAX];
  double2 g[KRYLOV_MAX];
  double2 c[KRYLOV_MAX];
  double beta0;
  double t;
  double tol;
  double err;
  int k;         // vectors in the basis so far
  int done;      // 1 = converged / breakdown / zero vector
  int kmax;
  int nvec_used;
  int ground;    // 1: lowest eigenvector instead of the exponential
  double energy; // ground mode: the Ritz value
};

// ---------------------------------------------------------------------------
// Host numerics (host_numerics.cpp)
// ---------------------------------------------------------------------------
void host_fit_power_law(double alpha, int n_exp, int r_max, std::vector<double2>& x,
                        std::vector<double2>& lam);
void host_fit_power_law_lm(double alpha, int n_exp, int r_max, int relative, std::vector<double2>& x,
                           std::vector<double2>& lam, double* rms);
// c = exp(-i t T) e_0 for symmetric tridiagonal T (alpha diag, beta off-diag)
__host__ __device__ int tridiag_expm_e0(int k, const double* alpha, const double* beta, double t,
                                        double2* c, double* work);

// Sweep schedule (schedule.cpp)
struct SchedOp {
  int seg, kind;      // kind 0 = fwd2 (pair j, j+1), 1 = back1 (site j)
  int j, tfac, env;   // env bit 1 = build beta_{j+1}, bit 2 = build gamma_j
  int boundary, stage;
};
void build_half(int N, const std::vector<int>& seg_len, int half, int merge, std::vector<SchedOp>& ops);
// segmented one-site step: kind 0 = site forward, 1 / 2 = bond backward with the
// centre moving right / left, 3 = boundary pair (boundary = 1)
void build_half1(int N, const std::vector<int>& seg_len, int half, int merge, std::vector<SchedOp>& ops);
// point-to-point messages of a half step with the segments spread over ranks
enum { XCH_PSI = 0, XCH_V = 1, XCH_BETA = 2, XCH_GAMMA = 3 };
struct ExchangeMsg {
  int stage, after;   // the boundary update's stage; 0 = before it, 1 = after it
  int src, dst, kind, j;
};
void exchange_plan(int N, const std::vector<int>& seg_len, const std::vector<int>& seg_rank, int scheme,
                   int merge, int half, std::vector<ExchangeMsg>& out);

}  // namespace tdvp
