// Batched FP64 SVD of two-site states and the truncated re-split (Fig. 5).
#pragma once

#include "common.h"

namespace tdvp {

struct SvdDesc {
  const double2* theta;  // [rows][cols] row-major input
  int rows, cols;
  int n_vec, len, trans; // vectors = rows of theta (trans 0) or its columns (trans 1)
  double2* X;            // [n_vec][len] working vectors
  double2* Acc;          // [n_vec][n_vec] accumulated rotations
  float2* X32;           // FP32 preconditioning phase: vectors and rotations
  float2* Acc32;
  double2* P;            // [n_vec][n_vec] Newton-Schulz temporaries
  double2* T;
  unsigned* maxr;        // largest |<x,y>| / (|x| |y|) met in the current sweep (float bits)
  double* sig;           // [n_vec + 3] vector norms, then scale, ||theta||_F^2 and the tail threshold
  int* perm;             // [n_vec] descending order
  int* rotated;          // [2]: rotations applied and pairs checked in the current sweep
  int* conv;             // 1 once a sweep applied no rotation
  int chi_max;
  double w_max, eps;
  int* chi;              // device outputs of the truncation
  double* w;
  double2* PsiL;         // [rows][chi]
  double* V;             // [chi]
  double2* PsiR;         // [chi][cols]
  double* s_sorted;      // [n_vec] all singular values, descending (may be null)
  double zero_rel;       // FP64 sweeps leave vectors with |x|^2 < zero_rel ||theta||_F^2 alone
                         // (0: 1e-28, the rounding-noise level; the derivative of a split
                         // needs every nonzero vector orthogonalised and passes ~1e-250)
};
struct SvdBatch {
  int n;
  int mode;              // 0: FP64 to ~1e-14 orthogonality; 1: to ~1e-10, with the rotations of the
                         // FP64 sweeps applied to Acc through an FP32-accumulated block rotation
  int* status;           // bit 8: NaN / zero state, 16: no convergence, 32: barrier timeout, 64: tail rule
  unsigned* sync;        // 8 words of device scratch: grid barrier, sweep loop, visit counters
  long long spin_limit;  // polls of a grid-barrier wait before it gives up (set by svd_split)
  SvdDesc d[MAXB];
};

// Full pipeline: FP32 Jacobi sweeps (preconditioner), Newton-Schulz
// re-orthonormalisation of the accumulated rotation and recomputation of the
// vectors in FP64, FP64 Jacobi sweeps until converged (pairs of vectors that
// the truncation certainly discards are skipped), then sort, truncate and
// write Psi_L, V, Psi_R.
// h_flag: pinned host int.
void svd_split(SvdBatch& b, int* d_flag, int* h_flag, cudaStream_t s);

// Polls a grid-barrier wait of the Jacobi sweeps makes before it gives up
// (status bit 32); spins < 0 restores the default. Process-wide; read by
// every later svd_split.
constexpr long long SVD_SPIN_LIMIT_DEFAULT = 1ll << 24;
void svd_set_spin_limit(long long spins);

}  // namespace tdvp
