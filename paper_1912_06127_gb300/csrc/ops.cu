// Batched local operations of the sweep: H_eff application (Fig. 4), Lanczos
// exponentiation (Eq. 18 / Eq. 20) and environment updates (Fig. 3, Eq. 19),
// each for all problems of a stage at once, in FP64 or on the tensor cores.
//
// Contraction order (Eq. 21 cost): y = R . (W . (L . theta)):
//   GEMM1  T1[(a w)][(S' b')] = sum_a' L[(a w)][a'] theta[a'][(S' b')]   chi^3 m D
//   W      T2[(a S)][(w' b')] = sum_{w,S'} W[w,w',S,S'] T1[a,w,S',b']     chi^2 m^2 D^2 (sparse)
//   GEMM2  y[(a S)][b]        = sum_(w' b') T2[(a S)][(w' b')] R[b][(w' b')]  chi^3 m D
// with D = d^2 and W = W_j W_{j+1} (merged on the host) for two sites, D = d for one.
#include <atomic>
#include <algorithm>

#include <mutex>
#include <unordered_map>

#include "engine.h"

namespace tdvp {

// Optional caller-supplied allocator (tdvp_set_allocator). Blocks it hands out
// are remembered with the function that returns them, so changing or removing
// the allocator later still frees each block through its own allocator.
namespace {
std::mutex g_alloc_mutex;
tdvp_alloc_fn g_user_alloc = nullptr;
tdvp_free_fn g_user_free = nullptr;
void* g_user_ctx = nullptr;
struct UserBlock {
  tdvp_free_fn free;
  void* ctx;
};
std::unordered_map<void*, UserBlock> g_user_blocks;
}  // namespace

void set_allocator(tdvp_alloc_fn a, tdvp_free_fn f, void* ctx) {
  std::lock_guard<std::mutex> g(g_alloc_mutex);
  g_user_alloc = a;
  g_user_free = f;
  g_user_ctx = ctx;
}

template <class T>
T* dalloc(size_t n) {
  void* p = nullptr;
  if (n == 0) n = 1;
  {
    std::unique_lock<std::mutex> g(g_alloc_mutex);
    if (g_user_alloc) {
      const tdvp_alloc_fn a = g_user_alloc;
      const UserBlock blk{g_user_free, g_user_ctx};
      g.unlock();
      p = a(n * sizeof(T), blk.ctx);
      if (!p) fail(TDVP_ENOMEM, "the caller's allocator returned NULL for " + std::to_string(n * sizeof(T)) + " bytes");
      g.lock();
      g_user_blocks[p] = blk;
      return (T*)p;
    }
  }
  cudaError_t e = cudaMalloc(&p, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(TDVP_ENOMEM, "cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed");
  }
  return (T*)p;
}
template double2* dalloc<double2>(size_t);
template double* dalloc<double>(size_t);
template float* dalloc<float>(size_t);
template float2* dalloc<float2>(size_t);
template int* dalloc<int>(size_t);
template LzState* dalloc<LzState>(size_t);
void dfree(void* p) {
  if (!p) return;
  UserBlock blk{nullptr, nullptr};
  {
    std::lock_guard<std::mutex> g(g_alloc_mutex);
    auto it = g_user_blocks.find(p);
    if (it != g_user_blocks.end()) {
      blk = it->second;
      g_user_blocks.erase(it);
    }
  }
  if (blk.free) {
    // the library's kernels may still use the block on any stream; a caching
    // allocator may hand it out again at once
    cudaDeviceSynchronize();
    blk.free(p, blk.ctx);
    return;
  }
  cudaFree(p);
}

int64_t pad4(int64_t x) { return (x + 3) & ~(int64_t)3; }

// ---------------------------------------------------------------------------
void DeviceWOp::build(const std::vector<double2>& dense, int m_, int D_, bool out_left) {
  release();
  m = m_;
  D = D_;
  std::vector<int> cp(m + 1, 0), ri;
  std::vector<double2> b64;
  std::vector<float2> b32;
  for (int o = 0; o < m; ++o) {
    cp[o] = (int)ri.size();
    for (int i = 0; i < m; ++i) {
      const int wl = out_left ? o : i, wr = out_left ? i : o;
      const double2* blk = &dense[((size_t)wl * m + wr) * D * D];
      bool nz = false;
      for (int q = 0; q < D * D; ++q) nz |= (blk[q].x != 0.0 || blk[q].y != 0.0);
      if (!nz) continue;
      ri.push_back(i);
      for (int q = 0; q < D * D; ++q) {
        b64.push_back(blk[q]);
        b32.push_back(make_float2((float)blk[q].x, (float)blk[q].y));
      }
    }
  }
  cp[m] = (int)ri.size();
  nnz = (int)ri.size();
  col_ptr = dalloc<int>(m + 1);
  row_idx = dalloc<int>(std::max(nnz, 1));
  blk64 = dalloc<double2>(std::max<size_t>(b64.size(), 1));
  blk32 = dalloc<float2>(std::max<size_t>(b32.size(), 1));
  CUDA_TRY(cudaMemcpy(col_ptr, cp.data(), sizeof(int) * (m + 1), cudaMemcpyHostToDevice));
  if (nnz) {
    CUDA_TRY(cudaMemcpy(row_idx, ri.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(blk64, b64.data(), sizeof(double2) * b64.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(blk32, b32.data(), sizeof(float2) * b32.size(), cudaMemcpyHostToDevice));
  }
}

void DeviceWOp::release() {
  dfree(col_ptr);
  dfree(row_idx);
  dfree(blk64);
  dfree(blk32);
  col_ptr = row_idx = nullptr;
  blk64 = nullptr;
  blk32 = nullptr;
}

// ---------------------------------------------------------------------------
int64_t mixed_cap_floats(int chi, int m, int d) {
  const int64_t c = chi, D = (int64_t)d * d;
  int64_t v = 0;
  auto mx = [&](int64_t x) { v = std::max(v, x); };
  mx(2 * D * c * pad4(2 * c));          // theta embedded
  mx(c * m * 2 * D * c);                  // T1
  mx(c * D * pad4(2 * m * c));            // T2
  mx(c * m * pad4(2 * c));                // env as A operand
  mx(2 * d * c * pad4(2 * c));            // site tensor embedded
  mx(c * m * 2 * d * c);                  // X1 / Y1
  mx(c * d * 2 * m * c);                  // X2 / Y2
  mx(c * pad4(2 * c * d));                // conj site tensor as A operand
  mx(2 * m * c * pad4(2 * c * d));        // X2 / Y2 embedded
  mx(2 * m * c * pad4(2 * c));            // right env embedded along (b w)
  mx(c * d * pad4(2 * c));                // site tensor as A operand
  mx(2 * c * pad4(2 * m * c));            // R as embedded B operand
  return v + 64;
}

void Slot::ensure(int64_t vec, int64_t T, int64_t fsz, int64_t svd_n, int kmax_) {
  if (vec <= cap_vec && T <= cap_T && fsz <= cap_f && kmax_ <= kmax && svd_n <= cap_svd &&
      svd_n * svd_n <= (svdX ? cap_vec : 0))
    return;
  const int64_t nsvd = std::max(svd_n, cap_svd);
  release();
  cap_svd = nsvd;
  cap_vec = std::max(vec, nsvd * nsvd);
  cap_T = T;
  cap_f = fsz;
  kmax = kmax_;
  theta = dalloc<double2>(cap_vec);
  theta2 = dalloc<double2>(cap_vec);
  V = dalloc<double2>((size_t)cap_vec * (kmax + 1));
  T1 = dalloc<double2>(cap_T);
  T2 = dalloc<double2>(cap_T);
  Amat = dalloc<double2>(cap_vec);
  Bmat = dalloc<double2>(cap_vec);
  if (fsz > 0)
    for (auto& p : f) p = dalloc<float>(cap_f);
  st = dalloc<LzState>(1);
  part = dalloc<double2>((size_t)lz_max_blocks(cap_vec) * KRYLOV_MAX);
  counter = dalloc<int>(1);
  CUDA_TRY(cudaMemset(counter, 0, sizeof(int)));
  svdX = dalloc<double2>(cap_vec);
  svdAcc = dalloc<double2>(cap_vec);
  svdP = dalloc<double2>(cap_vec);
  svdT = dalloc<double2>(cap_vec);
  svdX32 = dalloc<float2>(cap_vec);
  svdAcc32 = dalloc<float2>(cap_vec);
  maxr = reinterpret_cast<unsigned*>(dalloc<int>(1));
  sync = reinterpret_cast<unsigned*>(dalloc<int>(8));
  sig = dalloc<double>(nsvd + 3);
  perm = dalloc<int>(nsvd + 1);
  rot = dalloc<int>(2);  // rotations, pairs checked
  conv = dalloc<int>(1);
  bv = dalloc<double>(2 * (nsvd + 1));
}

void Slot::release() {
  for (void* p : {(void*)theta, (void*)theta2, (void*)V, (void*)T1, (void*)T2, (void*)Amat, (void*)Bmat,
                  (void*)st, (void*)part, (void*)counter, (void*)svdX, (void*)svdAcc, (void*)sig,
                  (void*)perm, (void*)rot, (void*)conv, (void*)svdP, (void*)svdT, (void*)svdX32,
                  (void*)svdAcc32, (void*)maxr, (void*)sync, (void*)bv})
    dfree(p);
  bv = nullptr;
  for (auto& p : f) {
    dfree(p);
    p = nullptr;
  }
  theta = theta2 = V = T1 = T2 = Amat = Bmat = part = svdX = svdAcc = svdP = svdT = nullptr;
  svdX32 = svdAcc32 = nullptr;
  maxr = nullptr;
  sync = nullptr;
  st = nullptr;
  counter = perm = rot = conv = nullptr;
  sig = nullptr;
  cap_vec = cap_T = cap_f = cap_svd = 0;
  kmax = 0;
}

// ---------------------------------------------------------------------------
// Operand forms of environments for the tensor-core path
// ---------------------------------------------------------------------------
void prep_L_forms(const std::vector<EnvFormJob>& jobs, cudaStream_t s) {
  for (size_t b0 = 0; b0 < jobs.size(); b0 += MAXB) {
    PrepBatch pb{};
    for (size_t i = b0; i < jobs.size() && pb.n < MAXB; ++i) {
      const auto& J = jobs[i];
      PrepDesc& d = pb.d[pb.n++];
      d = PrepDesc{};
      d.src = J.env;
      d.rs = J.chi;  // element ((a w), a') at env[(a m + w) chi + a']
      d.cs = 1;
      d.rows = J.chi * J.m;
      d.cols = J.chi;
      d.hi = J.hi;
      d.lo = J.lo;
      d.ld = pad4(2 * (int64_t)J.chi);
      d.embed = 0;
    }
    launch_prep(pb, s);
  }
}

void prep_R_forms(const std::vector<EnvFormJob>& jobs, cudaStream_t s) {
  for (size_t b0 = 0; b0 < jobs.size(); b0 += MAXB) {
    PrepBatch pb{};
    for (size_t i = b0; i < jobs.size() && pb.n < MAXB; ++i) {
      const auto& J = jobs[i];
      PrepDesc& d = pb.d[pb.n++];
      d = PrepDesc{};
      d.src = J.env;
      d.rs = (int64_t)J.m * J.chi;  // element (b, (w b')) at env[b m chi + w chi + b']
      d.cs = 1;
      d.rows = J.chi;
      d.cols = J.m * J.chi;
      d.hi = J.hi;
      d.lo = J.lo;
      d.ld = pad4(2 * (int64_t)J.m * J.chi);
      d.embed = 1;
    }
    launch_prep(pb, s);
  }
}

// ---------------------------------------------------------------------------
// H_eff . x for a batch
// ---------------------------------------------------------------------------
void matvec_batch(const std::vector<MvProb>& P, const std::vector<const double2*>& x,
                  const std::vector<double2*>& y, const Ctx& c, bool accumulate) {
  const int n = (int)P.size();
  if (n == 0) return;
  if (n > MAXB) fail(TDVP_EINVAL, "batch too large");
  if (accumulate && c.prec != TDVP_FP64) fail(TDVP_EINVAL, "accumulating H_eff products are FP64 only");
  if (c.prec == TDVP_FP64) {
    ZGemmBatch g1{};
    WStageBatch<double2> ws{};
    ZGemmBatch g2{};
    g1.n = ws.n = g2.n = n;
    for (int i = 0; i < n; ++i) {
      const MvProb& q = P[i];
      const int A = q.A, B = q.B, D = q.D, m = q.m;
      ZGemmDesc& a = g1.d[i];
      a = ZGemmDesc{};
      a.M = A * m;
      a.N = D * B;
      a.K = A;
      a.skip = q.skip;
      a.A = q.L;
      a.a_rs = A;
      a.a_cs = 1;
      a.B = x[i];
      a.b_rs = (int64_t)D * B;
      a.b_cs = 1;
      a.C = q.slot->T1;
      a.c_rs = (int64_t)D * B;
      a.c_cs = 1;
      WStageDesc<double2>& w = ws.d[i];
      w = WStageDesc<double2>{};
      w.A = A;
      w.B = B;
      w.skip = q.skip;
      w.X = q.slot->T1;
      w.x_a = (int64_t)m * D * B;
      w.x_w = (int64_t)D * B;
      w.x_s = B;
      w.x_b = 1;
      w.Y = q.slot->T2;
      w.y_a = (int64_t)D * m * B;
      w.y_w = B;
      w.y_s = (int64_t)m * B;
      w.y_b = 1;
      w.W = q.W;
      ZGemmDesc& b = g2.d[i];
      b = ZGemmDesc{};
      b.M = A * D;
      b.N = B;
      b.K = m * B;
      b.skip = q.skip;
      b.A = q.slot->T2;
      b.a_rs = (int64_t)m * B;
      b.a_cs = 1;
      b.B = q.R;
      b.b_rs = 1;
      b.b_cs = (int64_t)m * B;
      b.C = y[i];
      b.c_rs = B;
      b.c_cs = 1;
      b.accumulate = accumulate ? 1 : 0;
    }
    launch_zgemm(g1, c.s);
    launch_wstage(ws, c.s);
    launch_zgemm(g2, c.s);
    return;
  }
  // ---- tensor-core path ----
  const int passes = c.prec == TDVP_TF32X3 ? 3 : 1;
  PrepBatch pb{};
  pb.n = n;
  WStageBatch<float2> ws{};
  ws.n = n;
  ws.round_tf32 = 1;
  std::vector<TcProblem> t1(n), t2(n);
  for (int i = 0; i < n; ++i) {
    const MvProb& q = P[i];
    const int A = q.A, B = q.B, D = q.D, m = q.m;
    Slot* sl = q.slot;
    // theta as embedded B operand: element (n = (S' b'), k = a') at x[k D B + n]
    PrepDesc& pd = pb.d[i];
    pd = PrepDesc{};
    pd.skip = q.skip;
    pd.src = x[i];
    pd.rs = 1;
    pd.cs = (int64_t)D * B;
    pd.rows = D * B;
    pd.cols = A;
    pd.hi = sl->f[0];
    pd.lo = passes == 3 ? sl->f[1] : nullptr;
    pd.ld = pad4(2 * (int64_t)A);
    pd.embed = 1;
    TcProblem& g = t1[i];
    g.skip = q.skip;
    g.A = TcOperand{q.L32[0], q.L32[1], A * m, 2 * A, q.ldL};
    g.B = TcOperand{sl->f[0], sl->f[1], 2 * D * B, 2 * A, pd.ld};
    g.M = A * m;
    g.N = 2 * D * B;
    g.K = 2 * A;
    g.C = sl->f[2];
    g.ldc = 2 * (int64_t)D * B;
    g.c_fp64 = 0;
    const int64_t ld2 = pad4(2 * (int64_t)m * B);  // floats per T2 row
    WStageDesc<float2>& w = ws.d[i];
    w = WStageDesc<float2>{};
    w.A = A;
    w.B = B;
    w.skip = q.skip;
    w.X = reinterpret_cast<const float2*>(sl->f[2]);
    w.x_a = (int64_t)m * D * B;
    w.x_w = (int64_t)D * B;
    w.x_s = B;
    w.x_b = 1;
    w.Y = reinterpret_cast<float2*>(sl->f[3]);
    w.Ylo = passes == 3 ? reinterpret_cast<float2*>(sl->f[4]) : nullptr;
    w.y_a = (int64_t)D * (ld2 / 2);
    w.y_w = B;
    w.y_s = ld2 / 2;
    w.y_b = 1;
    w.W = q.W;
    TcProblem& h = t2[i];
    h.skip = q.skip;
    h.A = TcOperand{sl->f[3], sl->f[4], A * D, 2 * m * B, ld2};
    h.B = TcOperand{q.R32[0], q.R32[1], 2 * B, 2 * m * B, q.ldR};
    h.M = A * D;
    h.N = 2 * B;
    h.K = 2 * m * B;
    h.C = y[i];
    h.ldc = 2 * (int64_t)B;
    h.c_fp64 = 1;
    // K = 2 m B terms: split, partial tiles in the T1 buffer (consumed by the W stage)
    tc_set_ksplit(h, sl->f[2], sl->cap_f);
  }
  launch_prep(pb, c.s);
  launch_tc_gemm(t1, passes, c.d_status, c.s);
  launch_wstage(ws, c.s);
  launch_tc_gemm(t2, passes, c.d_status, c.s);
}

// ---------------------------------------------------------------------------
// exp(-i t H_eff) x for a batch (Lanczos)
// ---------------------------------------------------------------------------
void expm_batch(const std::vector<MvProb>& P0, const std::vector<const double2*>& x,
                const std::vector<double2*>& y, const std::vector<double>& t, int kmax, double tol,
                const Ctx& c, bool ground) {
  const int n = (int)P0.size();
  if (n == 0) return;
  std::vector<MvProb> P = P0;
  LzBatch lb{};
  lb.n = n;
  lb.status = c.d_status;
  for (int i = 0; i < n; ++i) {
    Slot* sl = P[i].slot;
    LzDesc& d = lb.d[i];
    d.x = x[i];
    d.y = y[i];
    d.V = sl->V;
    d.n = (int64_t)P[i].A * P[i].D * P[i].B;
    d.vs = sl->cap_vec;
    d.st = sl->st;
    d.part = sl->part;
    d.counter = sl->counter;
    d.t = t[i];
    d.tol = tol;
    d.kmax = kmax;
    d.ground = ground ? 1 : 0;
    P[i].skip = &sl->st->done;
  }
  lz_start(lb, c.s);
  std::vector<const double2*> xin(n);
  std::vector<double2*> yout(n);
  // small batches are launch-bound: once every problem has converged (or its
  // Krylov space is exhausted) the remaining iterations would only launch
  // kernels that return at once, so the loop stops (a host check per
  // iteration, from the third on; large batches keep launching instead)
  int64_t n_all = 0;
  for (int i = 0; i < n; ++i) n_all += lb.d[i].n;
  const bool check = n_all <= (int64_t(1) << 20);
  for (int j = 0; j < kmax; ++j) {
    for (int i = 0; i < n; ++i) {
      xin[i] = lb.d[i].V + (int64_t)j * lb.d[i].vs;
      yout[i] = lb.d[i].V + (int64_t)(j + 1) * lb.d[i].vs;
    }
    matvec_batch(P, xin, yout, c);
    lz_orthogonalize(lb, j, c.s);
    if (check && j >= 2 && j + 1 < kmax && lz_all_done(lb, c.s)) break;
  }
  lz_finish(lb, c.s);
}

// ---------------------------------------------------------------------------
// Environment updates (Fig. 3, Eq. 19 and its mirror image)
// ---------------------------------------------------------------------------
// dd: the two GEMMs in double-float on the FP32 pipe (~48 significant bits)
// instead of FP64, the W stage in FP64 as on the FP64 path
static void env_fp64(int side, const std::vector<EnvProb>& P, const Ctx& c, bool dd = false) {
  const int n = (int)P.size();
  ZGemmBatch g1{}, g3{};
  WStageBatch<double2> ws{};
  g1.n = g3.n = ws.n = n;
  for (int i = 0; i < n; ++i) {
    const EnvProb& q = P[i];
    const int A = q.A, B = q.B, d = q.d, m = q.m;
    ZGemmDesc& a = g1.d[i];
    ZGemmDesc& b = g3.d[i];
    WStageDesc<double2>& w = ws.d[i];
    a = ZGemmDesc{};
    b = ZGemmDesc{};
    w = WStageDesc<double2>{};
    w.W = q.W;
    if (side == 0) {
      // X1[(a w)][(s' b')] = sum_a' env[(a w)][a'] mat[a'][(s' b')]
      a.M = A * m;
      a.N = d * B;
      a.K = A;
      a.A = q.env;
      a.a_rs = A;
      a.a_cs = 1;
      a.B = q.mat;
      a.b_rs = (int64_t)d * B;
      a.b_cs = 1;
      a.C = q.slot->T1;
      a.c_rs = (int64_t)d * B;
      a.c_cs = 1;
      // X2[(a s)][(w' b')] = sum_{w, s'} W[w,w',s,s'] X1[a,w,s',b']
      w.A = A;
      w.B = B;
      w.X = q.slot->T1;
      w.x_a = (int64_t)m * d * B;
      w.x_w = (int64_t)d * B;
      w.x_s = B;
      w.x_b = 1;
      w.Y = q.slot->T2;
      w.y_a = (int64_t)d * m * B;
      w.y_w = B;
      w.y_s = (int64_t)m * B;
      w.y_b = 1;
      // out[b][(w' b')] = sum_(a s) conj(mat[(a s)][b]) X2[(a s)][(w' b')]
      b.M = B;
      b.N = m * B;
      b.K = A * d;
      b.A = q.bra ? q.bra : q.mat;
      b.a_rs = 1;
      b.a_cs = B;
      b.conj_a = 1;
      b.B = q.slot->T2;
      b.b_rs = (int64_t)m * B;
      b.b_cs = 1;
      b.C = q.out;
      b.c_rs = (int64_t)m * B;
      b.c_cs = 1;
    } else {
      // Y1[(a' s')][(b w')] = sum_b' mat[(a' s')][b'] env[(b w')][b']
      a.M = A * d;
      a.N = B * m;
      a.K = B;
      a.A = q.mat;
      a.a_rs = B;
      a.a_cs = 1;
      a.B = q.env;
      a.b_rs = 1;
      a.b_cs = B;
      a.C = q.slot->T1;
      a.c_rs = (int64_t)B * m;
      a.c_cs = 1;
      // Y2[(w a')][(s b)] = sum_{w', s'} W[w,w',s,s'] Y1[a',s',b,w']
      w.A = A;
      w.B = B;
      w.X = q.slot->T1;
      w.x_a = (int64_t)d * B * m;
      w.x_s = (int64_t)B * m;
      w.x_b = m;
      w.x_w = 1;
      w.Y = q.slot->T2;
      w.y_a = (int64_t)d * B;
      w.y_w = (int64_t)A * d * B;
      w.y_s = B;
      w.y_b = 1;
      // out[a][(w a')] = sum_(s b) conj(mat[a][(s b)]) Y2[(w a')][(s b)]
      b.M = A;
      b.N = m * A;
      b.K = d * B;
      b.A = q.bra ? q.bra : q.mat;
      b.a_rs = (int64_t)d * B;
      b.a_cs = 1;
      b.conj_a = 1;
      b.B = q.slot->T2;
      b.b_rs = 1;
      b.b_cs = (int64_t)d * B;
      b.C = q.out;
      b.c_rs = (int64_t)m * A;
      b.c_cs = 1;
    }
    b.accumulate = q.accumulate;
  }
  if (dd) {
    launch_zgemm_dd(g1, c.s, "env_zgemm_dd");
    launch_wstage(ws, c.s);
    launch_zgemm_dd(g3, c.s, "env_zgemm_dd");
  } else {
    launch_zgemm(g1, c.s);
    launch_wstage(ws, c.s);
    launch_zgemm(g3, c.s);
  }
}

static void env_tc(int side, const std::vector<EnvProb>& P, const Ctx& c) {
  const int n = (int)P.size();
  const int passes = c.prec == TDVP_TF32X3 ? 3 : 1;
  PrepBatch pa{}, pb{};
  pa.n = pb.n = n;
  std::vector<TcProblem> t1(n), t3(n);
  WStageBatch<float2> ws{};
  ws.n = n;
  ws.round_tf32 = 0;
  PrepBatch pc{}, pdd{};
  pc.n = pdd.n = n;
  for (int i = 0; i < n; ++i) {
    const EnvProb& q = P[i];
    const int A = q.A, B = q.B, d = q.d, m = q.m;
    Slot* sl = q.slot;
    float* lo0 = passes == 3 ? sl->f[1] : nullptr;
    float* lo2 = passes == 3 ? sl->f[3] : nullptr;
    PrepDesc& x0 = pa.d[i];
    PrepDesc& x1 = pb.d[i];
    PrepDesc& x2 = pc.d[i];
    PrepDesc& x3 = pdd.d[i];
    x0 = x1 = x2 = x3 = PrepDesc{};
    WStageDesc<float2>& w = ws.d[i];
    w = WStageDesc<float2>{};
    w.W = q.W;
    w.A = A;
    w.B = B;
    w.X = reinterpret_cast<const float2*>(sl->f[4]);
    w.Y = reinterpret_cast<float2*>(sl->f[5]);
    if (side == 0) {
      // GEMM1: A op = env [(a w)][a'], B op = mat embedded, element (n=(s' b'), k=a')
      x0.src = q.env;
      x0.rs = A;
      x0.cs = 1;
      x0.rows = A * m;
      x0.cols = A;
      x0.hi = sl->f[0];
      x0.lo = lo0;
      x0.ld = pad4(2 * (int64_t)A);
      x1.src = q.mat;
      x1.rs = 1;
      x1.cs = (int64_t)d * B;
      x1.rows = d * B;
      x1.cols = A;
      x1.hi = sl->f[2];
      x1.lo = lo2;
      x1.ld = pad4(2 * (int64_t)A);
      x1.embed = 1;
      t1[i] = TcProblem{nullptr, TcOperand{x0.hi, x0.lo, A * m, 2 * A, x0.ld},
                        TcOperand{x1.hi, x1.lo, 2 * d * B, 2 * A, x1.ld}, A * m, 2 * d * B, 2 * A,
                        sl->f[4], 2 * (int64_t)d * B, 0};
      w.x_a = (int64_t)m * d * B;
      w.x_w = (int64_t)d * B;
      w.x_s = B;
      w.x_b = 1;
      w.y_a = (int64_t)d * m * B;
      w.y_w = B;
      w.y_s = (int64_t)m * B;
      w.y_b = 1;
      // GEMM3: A op = conj(mat)^T: element (i=b, k=(a s)) at mat[k B + i]
      x2.src = q.mat;
      x2.rs = 1;
      x2.cs = B;
      x2.conj = 1;
      x2.rows = B;
      x2.cols = A * d;
      x2.hi = sl->f[0];
      x2.lo = lo0;
      x2.ld = pad4(2 * (int64_t)A * d);
      // B op = X2 embedded: element (n=(w' b'), k=(a s)) at X2[k m B + n]
      x3.src32 = reinterpret_cast<const float2*>(sl->f[5]);
      x3.rs = 1;
      x3.cs = (int64_t)m * B;
      x3.rows = m * B;
      x3.cols = A * d;
      x3.hi = sl->f[2];
      x3.lo = lo2;
      x3.ld = pad4(2 * (int64_t)A * d);
      x3.embed = 1;
      t3[i] = TcProblem{nullptr, TcOperand{x2.hi, x2.lo, B, 2 * A * d, x2.ld},
                        TcOperand{x3.hi, x3.lo, 2 * m * B, 2 * A * d, x3.ld}, B, 2 * m * B, 2 * A * d,
                        q.out, 2 * (int64_t)m * B, 1};
      tc_set_ksplit(t3[i], sl->f[4], sl->cap_f);  // X1 buffer, consumed by the W stage
    } else {
      // GEMM1: A op = mat [(a' s')][b'], B op = env embedded: element (n=(b w'), k=b') at env[n B + k]
      x0.src = q.mat;
      x0.rs = B;
      x0.cs = 1;
      x0.rows = A * d;
      x0.cols = B;
      x0.hi = sl->f[0];
      x0.lo = lo0;
      x0.ld = pad4(2 * (int64_t)B);
      x1.src = q.env;
      x1.rs = B;
      x1.cs = 1;
      x1.rows = B * m;
      x1.cols = B;
      x1.hi = sl->f[2];
      x1.lo = lo2;
      x1.ld = pad4(2 * (int64_t)B);
      x1.embed = 1;
      t1[i] = TcProblem{nullptr, TcOperand{x0.hi, x0.lo, A * d, 2 * B, x0.ld},
                        TcOperand{x1.hi, x1.lo, 2 * B * m, 2 * B, x1.ld}, A * d, 2 * B * m, 2 * B,
                        sl->f[4], 2 * (int64_t)B * m, 0};
      w.x_a = (int64_t)d * B * m;
      w.x_s = (int64_t)B * m;
      w.x_b = m;
      w.x_w = 1;
      w.y_a = (int64_t)d * B;
      w.y_w = (int64_t)A * d * B;
      w.y_s = B;
      w.y_b = 1;
      // GEMM3: A op = conj(mat) [a][(s b)], B op = Y2 embedded: (n=(w a'), k=(s b)) at Y2[n d B + k]
      x2.src = q.mat;
      x2.rs = (int64_t)d * B;
      x2.cs = 1;
      x2.conj = 1;
      x2.rows = A;
      x2.cols = d * B;
      x2.hi = sl->f[0];
      x2.lo = lo0;
      x2.ld = pad4(2 * (int64_t)d * B);
      x3.src32 = reinterpret_cast<const float2*>(sl->f[5]);
      x3.rs = (int64_t)d * B;
      x3.cs = 1;
      x3.rows = m * A;
      x3.cols = d * B;
      x3.hi = sl->f[2];
      x3.lo = lo2;
      x3.ld = pad4(2 * (int64_t)d * B);
      x3.embed = 1;
      t3[i] = TcProblem{nullptr, TcOperand{x2.hi, x2.lo, A, 2 * d * B, x2.ld},
                        TcOperand{x3.hi, x3.lo, 2 * m * A, 2 * d * B, x3.ld}, A, 2 * m * A, 2 * d * B,
                        q.out, 2 * (int64_t)m * A, 1};
      tc_set_ksplit(t3[i], sl->f[4], sl->cap_f);  // Y1 buffer, consumed by the W stage
    }
  }
  launch_prep(pa, c.s);
  launch_prep(pb, c.s);
  launch_tc_gemm(t1, passes, c.d_status, c.s);
  launch_wstage(ws, c.s);
  launch_prep(pc, c.s);
  launch_prep(pdd, c.s);
  launch_tc_gemm(t3, passes, c.d_status, c.s);
}

namespace {
std::atomic<int> g_env_tc{0};
}

void set_env_on_tensor_cores(bool on) { g_env_tc = on ? 1 : 0; }
bool env_on_tensor_cores() { return g_env_tc.load() != 0; }

// Mixed modes update the environments in double-float by default: they are
// reused by every later H_eff of the half sweep, so their error acts like a
// fixed perturbation of H and moves observables linearly in time; on the
// tensor cores (FP32 accumulation) that drift was ~30x that of the
// double-float environments at chi = 64.
void env_batch(int side, const std::vector<EnvProb>& P, const Ctx& c) {
  if (P.empty()) return;
  if ((int)P.size() > MAXB) fail(TDVP_EINVAL, "batch too large");
  if (c.prec == TDVP_FP64) {
    env_fp64(side, P, c);
    return;
  }
  for (const auto& q : P)
    if (q.bra || q.accumulate) fail(TDVP_EINVAL, "mixed bra/ket and accumulating environments are FP64 only");
  if (env_on_tensor_cores()) env_tc(side, P, c);
  else env_fp64(side, P, c, true);
}

}  // namespace tdvp
