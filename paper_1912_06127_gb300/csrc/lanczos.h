// Batched Lanczos exponentiation: descriptors and host launchers.
#pragma once

#include "common.h"

namespace tdvp {

struct LzDesc {
  const double2* x;   // input vector (n)
  double2* y;         // output exp(-i t H) x (n); may alias x
  double2* V;         // Krylov storage: kmax+1 vectors of n, vector stride vs
  int64_t n, vs;
  LzState* st;        // device state of this problem
  double2* part;      // partial sums: [blocks][KRYLOV_MAX]
  int* counter;       // arrival counter (zero between launches)
  double t, tol;
  int kmax;
  int ground;         // 1: y = ||x|| times the lowest Ritz vector (t unused)
};
struct LzBatch {
  int n;
  int* status;        // device status word (bit 2: NaN, bit 4: tridiagonal solver failed)
  LzDesc d[MAXB];
};

int lz_max_blocks(int64_t n);
void lz_start(const LzBatch& b, cudaStream_t s);
// call after the matvec that wrote H v_j into slot j+1
void lz_orthogonalize(const LzBatch& b, int j, cudaStream_t s);
void lz_finish(const LzBatch& b, cudaStream_t s);
// whether every problem of the batch has converged or broken down (one small
// launch and a synchronisation of s)
bool lz_all_done(const LzBatch& b, cudaStream_t s);

}  // namespace tdvp
