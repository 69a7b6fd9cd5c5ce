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
  double* sig;           // [n_vec] norms of the final vectors
  int* perm;             // [n_vec] descending order
  int* rotated;          // rotations applied in the current sweep
  int* conv;             // 1 once a sweep applied no rotation
  int chi_max;
  double w_max, eps;
  int* chi;              // device outputs of the truncation
  double* w;
  double2* PsiL;         // [rows][chi]
  double* V;             // [chi]
  double2* PsiR;         // [chi][cols]
  double* s_sorted;      // [n_vec] all singular values, descending (may be null)
};
struct SvdBatch {
  int n;
  int* status;           // bit 8: NaN / zero state, bit 16: no convergence
  SvdDesc d[MAXB];
};

// Full pipeline: Jacobi sweeps until converged (one host synchronisation per
// sweep), then sort, truncate and write Psi_L, V, Psi_R. h_flag: pinned host int.
void svd_split(SvdBatch& b, int* d_flag, int* h_flag, cudaStream_t s);

}  // namespace tdvp
