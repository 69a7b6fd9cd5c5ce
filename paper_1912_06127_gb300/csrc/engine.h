// Engine state: MPO and MPS handles, per-problem workspaces, batched local
// operations of the two-site TDVP sweep.
#pragma once

#include <memory>
#include <vector>

#include "common.h"
#include "lanczos.h"
#include "svd.h"

namespace tdvp {

template <class T>
T* dalloc(size_t n);
void dfree(void* p);
void set_allocator(tdvp_alloc_fn a, tdvp_free_fn f, void* ctx);

// Sparse MPO operator on the device (CSR over the output bond index).
struct DeviceWOp {
  int m = 0, D = 0, nnz = 0;
  int* col_ptr = nullptr;
  int* row_idx = nullptr;
  double2* blk64 = nullptr;
  float2* blk32 = nullptr;
  // dense: [m][m][D][D] host tensor W[w_left][w_right][s_out][s_in];
  // out_left = false: output index w_right (sum over w_left), else the reverse
  void build(const std::vector<double2>& dense, int m, int D, bool out_left);
  void release();
  WOp op() const { return WOp{m, D, nnz, col_ptr, row_idx, blk64, blk32}; }
  ~DeviceWOp() { release(); }
};

// Workspace of one local problem of a batch.
struct Slot {
  int64_t cap_vec = 0, cap_T = 0, cap_f = 0, cap_svd = 0;
  int kmax = 0;
  double2* theta = nullptr;   // two-site state Theta
  double2* theta2 = nullptr;  // evolved state
  double2* V = nullptr;       // Krylov vectors
  double2* T1 = nullptr;      // FP64 intermediates
  double2* T2 = nullptr;
  double2* Amat = nullptr;    // Psi V / V Psi for environment updates
  double2* Bmat = nullptr;
  float* f[9] = {};           // fp32 operand / intermediate buffers (cap_f floats each)
  LzState* st = nullptr;
  double2* part = nullptr;
  int* counter = nullptr;
  double2* svdX = nullptr;
  double2* svdAcc = nullptr;
  double2* svdP = nullptr;
  double2* svdT = nullptr;
  float2* svdX32 = nullptr;
  float2* svdAcc32 = nullptr;
  unsigned* maxr = nullptr;
  unsigned* sync = nullptr;
  double* sig = nullptr;
  int* perm = nullptr;
  int* rot = nullptr;
  int* conv = nullptr;
  double* bv = nullptr;       // two bond vectors of cap_svd values (one-site bond steps)
  void ensure(int64_t vec, int64_t T, int64_t fsz, int64_t svd_n, int kmax_);
  void release();
  ~Slot() { release(); }
};

// One H_eff application (two-site when D = d^2, one-site when D = d).
struct MvProb {
  int A, B, D, m;
  const double2* L;           // [A][m][A]
  const double2* R;           // [B][m][B]
  const float* L32[2];        // mixed: L as A operand [(a w)][ldL]
  const float* R32[2];        // mixed: R as embedded B operand [2B][ldR]
  int64_t ldL, ldR;
  WOp W;
  Slot* slot;
  const int* skip;
};

struct Ctx {
  cudaStream_t s;
  int* d_status;
  int prec;
};

// y = H_eff x; accumulate (FP64 only): y += H_eff x
void matvec_batch(const std::vector<MvProb>& P, const std::vector<const double2*>& x,
                  const std::vector<double2*>& y, const Ctx& c, bool accumulate = false);
void expm_batch(const std::vector<MvProb>& P, const std::vector<const double2*>& x,
                const std::vector<double2*>& y, const std::vector<double>& t, int kmax, double tol,
                const Ctx& c, bool ground = false);
// Environment updates. Left: out [B][m][B] from env [A][m][A], Amat [A][d][B] (= Psi V).
// Right: out [A][m][A] from env [B][m][B], Bmat [A][d][B] (= V Psi).
struct EnvProb {
  int A, B, d, m;
  const double2* env;
  const double2* mat;
  double2* out;
  WOp W;      // left: out index w_right; right: out index w_left
  Slot* slot;
  const double2* bra = nullptr;  // conjugated tensor when it differs from mat (FP64 only)
  int accumulate = 0;            // out += ... (FP64 only)
};
void env_batch(int side, const std::vector<EnvProb>& P, const Ctx& c);
// Mixed operand forms of environments: L as A operand [(a w)][pad4(2a)],
// R as embedded B operand [2b][pad4(2 m b)] (hi, and lo when passes == 3).
int64_t pad4(int64_t x);
int64_t mixed_cap_floats(int chi, int m, int d);
// environment updates of the mixed modes: double-float (default) or the
// mode's tensor-core products
void set_env_on_tensor_cores(bool on);
bool env_on_tensor_cores();
struct EnvFormJob {
  const double2* env;
  int chi, m;
  float* hi;
  float* lo;
};
void prep_L_forms(const std::vector<EnvFormJob>& jobs, cudaStream_t s);
void prep_R_forms(const std::vector<EnvFormJob>& jobs, cudaStream_t s);

// ---- forward-mode derivative of the sweep (tangent.cu) ----
struct SvdFullDesc {
  const double2* X;
  const double2* Acc;
  const double* sig;
  const int* perm;
  int rows, cols, n_vec, len, trans;
  double2* U;   // [rows][n_vec]
  double2* Vh;  // [n_vec][cols]
  double* s;    // [n_vec], descending
};
void launch_svd_export_full(const SvdFullDesc& d, cudaStream_t s);
struct SvdTanDesc {
  const double2* dP;  // [r][r] = U^H dTheta V
  const double* s;    // [r] descending
  int r, k;
  double2* CL;        // [r][k]
  double2* CR;        // [r][k]
  double* dV;         // [k]
};
struct SvdTanBatch {
  int n;
  SvdTanDesc d[MAXB];
};
void launch_svd_tangent_coef(const SvdTanBatch& b, cudaStream_t s);
constexpr int ZCOMB_MAX = 17;
struct ZCombDesc {
  double2* y;
  int64_t n;
  int n_terms, accumulate;
  const double2* x[ZCOMB_MAX];
  double2 c[ZCOMB_MAX];
};
struct ZCombBatch {
  int n;
  ZCombDesc d[8];
};
void launch_zcombine(const ZCombBatch& b, cudaStream_t s);
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w);

}  // namespace tdvp
