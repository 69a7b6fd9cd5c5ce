// C ABI of libtdvp and the sweep executor.
//
// tdvp_step runs each half of a time step as a list of stages (schedule.cu).
// All two-site updates of a stage run together -- Theta = Psi_j V_j Psi_{j+1}
// (Fig. 5 input), exp(-i H2_eff tau) Theta by Lanczos (Eq. 18), the truncated
// SVD re-split (Fig. 5) and the environment updates (Eq. 19) -- as one set of
// batched launches, followed by all one-site backward updates of the stage
// (Eq. 20). One synchronisation per stage reads the new bond dimensions.
//
// Also here: two-site DMRG (dmrg_impl), measurements by transfer matrices,
// the forward-mode derivative of the sweep with respect to h and J
// (step_tangent_impl, measure_tangent_impl; kernels in tangent.cu), one-site
// operators and mixed expectations for dynamical correlations, and the one-site
// TDVP step with the hybrid two-site -> one-site scheme (step1_impl).
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "engine.h"

using namespace tdvp;

namespace tdvp {

int64_t g_launches = 0;
static thread_local std::string g_last_error;

[[noreturn]] void fail(int code, const std::string& msg) { throw TdvpError{code, msg}; }

void cuda_check(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return;
  cudaGetLastError();
  fail(TDVP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" + std::to_string(line) + ")");
}

}  // namespace tdvp

// ---------------------------------------------------------------------------
// Handles
// ---------------------------------------------------------------------------
struct tdvp_mpo_s {
  int kind = 0, N = 0, m = 0, d = 2, n_exp = 0;
  double alpha = 0, J = 0, h = 0;
  std::vector<double2> x, lam;
  std::vector<double2> W;    // [m][m][d][d]
  std::vector<double2> W12;  // [m][m][d^2][d^2]
  DeviceWOp w1, w1t, w2;     // one-site (out right), one-site (out left), two-site
  DeviceWOp w0;              // the bond (zero-site) term: identity over w, physical dimension 1
  uint64_t id = 0;
  uint64_t base_id = 0;      // derivative MPOs: id of the MPO they differentiate
  int param = -1;            // derivative MPOs: TDVP_PARAM_H or TDVP_PARAM_J
};

struct tdvp_mps_s {
  int N = 0, d = 2, chi_cap = 1;
  std::vector<int> dims;  // N-1 bond dimensions
  std::vector<int> cap;   // N-1 bond capacities
  std::vector<double2*> Psi;
  std::vector<double*> V;
  // environments for the attached MPO
  uint64_t env_id = 0;
  int env_m = 0;
  std::vector<double2*> beta, gamma;
  // tensor-core operand forms of the environments
  int form_passes = 0;
  std::vector<float*> beta32[2], gamma32[2];
  std::vector<char> beta32_ok, gamma32_ok;
  // per-problem workspaces
  std::vector<std::unique_ptr<Slot>> slots;
  int* d_status = nullptr;
  int* d_chi = nullptr;
  double* d_w = nullptr;
  int* d_flag = nullptr;
  int* h_pinned = nullptr;  // [0] = flag, [1] = status, [2..2+MAXB) chi
  double* h_w = nullptr;
  // one-site sweeps: split factors and a staging buffer (chi_cap^2 d^2 each), two bond vectors
  double2* w1s[4] = {};
  double* w1v[2] = {};

  int chiL(int j) const { return j == 0 ? 1 : dims[j - 1]; }
  int chiR(int j) const { return j == N - 1 ? 1 : dims[j]; }
  int capL(int j) const { return j == 0 ? 1 : cap[j - 1]; }
  int capR(int j) const { return j == N - 1 ? 1 : cap[j]; }
};

static uint64_t g_next_id = 1;
static std::mutex g_id_mutex;

namespace {

int ok_or_code(const std::function<void()>& f) {
  try {
    f();
    return TDVP_OK;
  } catch (const TdvpError& e) {
    g_last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return TDVP_ENOMEM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return TDVP_EINVAL;
  }
}

void require_device() {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    fail(TDVP_ECUDA, "no usable CUDA device");
  }
}

// W12[a][c] = sum_b W1[a][b] (x) W2[b][c] (two-site MPO tensor over pairs of sites)
std::vector<double2> two_site_mpo(const std::vector<double2>& W1, const std::vector<double2>& W2, int m, int d) {
  const int D = d * d;
  std::vector<double2> W12((size_t)m * m * D * D, make_double2(0, 0));
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b)
      for (int c = 0; c < m; ++c) {
        const double2* w1 = &W1[((size_t)a * m + b) * d * d];
        const double2* w2 = &W2[((size_t)b * m + c) * d * d];
        bool nz1 = false, nz2 = false;
        for (int q = 0; q < d * d; ++q) {
          nz1 |= w1[q].x != 0 || w1[q].y != 0;
          nz2 |= w2[q].x != 0 || w2[q].y != 0;
        }
        if (!nz1 || !nz2) continue;
        double2* o = &W12[((size_t)a * m + c) * D * D];
        for (int s1 = 0; s1 < d; ++s1)
          for (int s2 = 0; s2 < d; ++s2)
            for (int t1 = 0; t1 < d; ++t1)
              for (int t2 = 0; t2 < d; ++t2) {
                double2& r = o[(s1 * d + s2) * D + (t1 * d + t2)];
                r = zadd(r, zmul(w1[s1 * d + t1], w2[s2 * d + t2]));
              }
      }
  return W12;
}

void build_site_W(tdvp_mpo_s* M) {
  const int d = 2, m = M->m, K = M->n_exp;
  const double2 Z = make_double2(0, 0), One = make_double2(1, 0);
  // Pauli matrices [s_out][s_in]
  const double2 SX[4] = {Z, One, One, Z};
  const double2 SY[4] = {Z, make_double2(0, -1), make_double2(0, 1), Z};
  const double2 SZ[4] = {One, Z, Z, make_double2(-1, 0)};
  const double2 I2[4] = {One, Z, Z, One};
  std::vector<std::pair<const double2*, double>> terms;
  if (M->kind == TDVP_ISING) terms = {{SZ, 1.0}};
  else if (M->kind == TDVP_XY) terms = {{SX, 1.0}, {SY, 1.0}};
  else terms = {{SX, 0.5}, {SY, 0.5}, {SZ, 0.5}};
  M->W.assign((size_t)m * m * d * d, Z);
  auto put = [&](int a, int b, const double2* op, double2 coef) {
    double2* o = &M->W[((size_t)a * m + b) * d * d];
    for (int q = 0; q < 4; ++q) o[q] = zmul(op[q], coef);
  };
  // finite-state layout: m-1 = nothing placed yet, 0 = all placed (Sec. II C)
  put(0, 0, I2, One);
  put(m - 1, m - 1, I2, One);
  put(m - 1, 0, SX, make_double2(M->h, 0));
  for (size_t t = 0; t < terms.size(); ++t) {
    const double sc = terms[t].second;
    for (int k = 0; k < K; ++k) {
      const int c = 1 + (int)t * K + k;
      put(m - 1, c, terms[t].first, make_double2(sc, 0));
      put(c, c, I2, M->lam[k]);
      put(c, 0, terms[t].first, zscale(zmul(M->x[k], M->lam[k]), M->J * sc));
    }
  }
}

Slot* slot_for(tdvp_mps_s* S, size_t i, int m, int kmax) {
  while (S->slots.size() <= i) S->slots.emplace_back(new Slot());
  const int64_t c = S->chi_cap, d = S->d;
  const int64_t vec = c * c * d * d;
  const int64_t T = c * c * m * d * d;
  const int64_t f = mixed_cap_floats((int)c, m, (int)d);
  S->slots[i]->ensure(vec, T, f, c * d, kmax);
  return S->slots[i].get();
}

void ensure_small_buffers(tdvp_mps_s* S) {
  if (S->d_status) return;
  S->d_status = dalloc<int>(1);
  S->d_chi = dalloc<int>(MAXB);
  S->d_w = dalloc<double>(MAXB);
  S->d_flag = dalloc<int>(1);
  CUDA_TRY(cudaMemset(S->d_status, 0, sizeof(int)));
  CUDA_TRY(cudaMallocHost((void**)&S->h_pinned, sizeof(int) * (2 + MAXB)));
  CUDA_TRY(cudaMallocHost((void**)&S->h_w, sizeof(double) * MAXB));
}

void free_envs(tdvp_mps_s* S) {
  for (auto p : S->beta) dfree(p);
  for (auto p : S->gamma) dfree(p);
  for (int h = 0; h < 2; ++h) {
    for (auto p : S->beta32[h]) dfree(p);
    for (auto p : S->gamma32[h]) dfree(p);
    S->beta32[h].clear();
    S->gamma32[h].clear();
  }
  S->beta.clear();
  S->gamma.clear();
  S->env_id = 0;
  S->env_m = 0;
  S->form_passes = 0;
}

// Left/right environment of every site from scratch (Sec. III A: all gamma
// built right to left at the start; Sec. III B: each partition needs the
// environments of its own sites, so both sides are built once).
void build_all_envs(tdvp_mps_s* S, tdvp_mpo_s* M, cudaStream_t s) {
  const int N = S->N, m = M->m, d = S->d;
  if (S->env_id != M->id) {
    free_envs(S);
    S->beta.resize(N);
    S->gamma.resize(N);
    for (int j = 0; j < N; ++j) {
      S->beta[j] = dalloc<double2>((size_t)S->capL(j) * S->capL(j) * m);
      S->gamma[j] = dalloc<double2>((size_t)S->capR(j) * S->capR(j) * m);
    }
    S->env_m = m;
    S->beta32_ok.assign(N, 0);
    S->gamma32_ok.assign(N, 0);
  }
  std::vector<double2> bl(m, make_double2(0, 0)), br(m, make_double2(0, 0));
  bl[m - 1] = make_double2(1, 0);
  br[0] = make_double2(1, 0);
  CUDA_TRY(cudaMemcpyAsync(S->beta[0], bl.data(), sizeof(double2) * m, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(S->gamma[N - 1], br.data(), sizeof(double2) * m, cudaMemcpyHostToDevice, s));
  Slot* sl = slot_for(S, 0, m, 1);
  Ctx c{s, S->d_status, TDVP_FP64};
  for (int j = 0; j + 1 < N; ++j) {
    ScaleBatch sb{};
    sb.n = 1;
    sb.d[0] = ScaleDesc{S->Psi[j], sl->Amat, S->V[j], S->chiL(j), d, S->chiR(j), 0};
    launch_scale_bond(sb, s);
    env_batch(0, {EnvProb{S->chiL(j), S->chiR(j), d, m, S->beta[j], sl->Amat, S->beta[j + 1], M->w1.op(), sl}}, c);
  }
  for (int j = N - 2; j >= 0; --j) {
    ScaleBatch sb{};
    sb.n = 1;
    sb.d[0] = ScaleDesc{S->Psi[j + 1], sl->Bmat, S->V[j], S->chiL(j + 1), d, S->chiR(j + 1), 1};
    launch_scale_bond(sb, s);
    env_batch(1, {EnvProb{S->chiL(j + 1), S->chiR(j + 1), d, m, S->gamma[j + 1], sl->Bmat, S->gamma[j], M->w1t.op(), sl}}, c);
  }
  S->env_id = M->id;
  S->beta32_ok.assign(N, 0);
  S->gamma32_ok.assign(N, 0);
}

// tensor-core operand forms of beta_j (as L) / gamma_j (as R), built on demand
void ensure_forms(tdvp_mps_s* S, const std::vector<int>& Lsites, const std::vector<int>& Rsites, int passes,
                  cudaStream_t s) {
  const int N = S->N, m = S->env_m;
  if (S->form_passes != passes || S->beta32[0].empty()) {
    for (int h = 0; h < 2; ++h) {
      for (auto p : S->beta32[h]) dfree(p);
      for (auto p : S->gamma32[h]) dfree(p);
      S->beta32[h].assign(N, nullptr);
      S->gamma32[h].assign(N, nullptr);
    }
    for (int j = 0; j < N; ++j) {
      const int64_t cl = S->capL(j), cr = S->capR(j);
      for (int h = 0; h < passes && h < 2; ++h) {
        S->beta32[h][j] = dalloc<float>(cl * m * pad4(2 * cl));
        S->gamma32[h][j] = dalloc<float>(2 * cr * pad4(2 * m * cr));
      }
    }
    S->form_passes = passes;
    S->beta32_ok.assign(N, 0);
    S->gamma32_ok.assign(N, 0);
  }
  std::vector<EnvFormJob> jl, jr;
  for (int j : Lsites)
    if (!S->beta32_ok[j]) {
      jl.push_back(EnvFormJob{S->beta[j], S->chiL(j), m, S->beta32[0][j], passes == 3 ? S->beta32[1][j] : nullptr});
      S->beta32_ok[j] = 1;
    }
  for (int j : Rsites)
    if (!S->gamma32_ok[j]) {
      jr.push_back(EnvFormJob{S->gamma[j], S->chiR(j), m, S->gamma32[0][j], passes == 3 ? S->gamma32[1][j] : nullptr});
      S->gamma32_ok[j] = 1;
    }
  prep_L_forms(jl, s);
  prep_R_forms(jr, s);
}

MvProb make_mv(tdvp_mps_s* S, tdvp_mpo_s* M, int A, int B, int D, int Lsite, int Rsite, bool two, Slot* sl,
               int prec) {
  MvProb p{};
  p.A = A;
  p.B = B;
  p.D = D;
  p.m = M->m;
  p.L = S->beta[Lsite];
  p.R = S->gamma[Rsite];
  p.W = two ? M->w2.op() : M->w1.op();
  p.slot = sl;
  if (prec != TDVP_FP64) {
    p.L32[0] = S->beta32[0][Lsite];
    p.L32[1] = prec == TDVP_TF32X3 ? S->beta32[1][Lsite] : nullptr;
    p.R32[0] = S->gamma32[0][Rsite];
    p.R32[1] = prec == TDVP_TF32X3 ? S->gamma32[1][Rsite] : nullptr;
    p.ldL = pad4(2 * (int64_t)A);
    p.ldR = pad4(2 * (int64_t)M->m * B);
  }
  return p;
}

double heff_flops(int A, int B, int D, int m, int nnz) {
  // complex multiply-add = 8 real flops
  return 8.0 * ((double)A * A * B * m * D + (double)A * B * B * m * D + (double)A * B * D * D * nnz);
}

void read_stage_results(tdvp_mps_s* S, int n, cudaStream_t s) {
  CUDA_TRY(cudaMemcpyAsync(S->h_pinned + 1, S->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (n > 0) {
    CUDA_TRY(cudaMemcpyAsync(S->h_pinned + 2, S->d_chi, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(S->h_w, S->d_w, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  const int st = S->h_pinned[1];
  // a wait that gave up comes first: what the later kernels of the stage
  // computed from the abandoned work may have set the numeric bits too
  if (st & 1) fail(TDVP_ETIMEOUT, "a bounded device wait gave up (tensor-core pipeline)");
  if (st & 32) fail(TDVP_ETIMEOUT, "a bounded grid barrier gave up (SVD sweeps)");
  if (st & (2 | 8)) fail(TDVP_ENUMERIC, "NaN or zero norm in a local update");
  if (st & 4) fail(TDVP_ENUMERIC, "tridiagonal eigen-solver did not converge");
  if (st & 16) fail(TDVP_ENUMERIC, "Jacobi SVD did not converge");
  if (st & 64) fail(TDVP_ENUMERIC, "SVD tail rule violated: a kept singular value lies below the tail threshold");
}

struct StageOp {
  int j, tfac, env;
  int chi_max = 0;  // > 0: this update's bond dimension cap instead of the step's chi_max
};

// Two-site updates of one stage. ground = false: Theta' = exp(-i H2_eff t) Theta
// (Eq. 18); ground = true: Theta' = the lowest Ritz vector of H2_eff in the
// Krylov space of Theta (two-site DMRG), its Ritz value written to *energy
// (one problem).
// s_full (one problem only): all singular values written there and every pair
// of vectors converged (no tail rule), as the derivative of the split needs.
void run_fwd2(tdvp_mps_s* S, tdvp_mpo_s* M, const std::vector<StageOp>& ops, const tdvp_step_params* p,
              tdvp_step_stats* st, cudaStream_t s, bool ground = false, double* energy = nullptr,
              double* s_full = nullptr) {
  const int n = (int)ops.size();
  const int d = S->d, m = M->m, prec = p->precision;
  const double tau = 0.5 * p->dt;
  Ctx c{s, S->d_status, prec};
  std::vector<Slot*> sl(n);
  for (int i = 0; i < n; ++i) sl[i] = slot_for(S, i, m, p->krylov_max);
  // Theta = Psi_j V_j Psi_{j+1}
  ZGemmBatch g{};
  g.n = n;
  for (int i = 0; i < n; ++i) {
    const int j = ops[i].j, A = S->chiL(j), cb = S->dims[j], B = S->chiR(j + 1);
    ZGemmDesc& q = g.d[i];
    q = ZGemmDesc{};
    q.M = A * d;
    q.N = d * B;
    q.K = cb;
    q.A = S->Psi[j];
    q.a_rs = cb;
    q.a_cs = 1;
    q.kscale = S->V[j];
    q.B = S->Psi[j + 1];
    q.b_rs = (int64_t)d * B;
    q.b_cs = 1;
    q.C = sl[i]->theta;
    q.c_rs = (int64_t)d * B;
    q.c_cs = 1;
  }
  // the mixed path forms Theta in double-float (~48 bits, on the FP32 pipe)
  if (prec == TDVP_FP64) launch_zgemm(g, s, "theta_form_zgemm");
  else launch_zgemm_dd(g, s, "theta_form_dd");
  // exp(-i H2_eff t) Theta
  std::vector<MvProb> P(n);
  std::vector<const double2*> x(n);
  std::vector<double2*> y(n);
  std::vector<double> t(n);
  std::vector<int> Ls, Rs;
  for (int i = 0; i < n; ++i) {
    const int j = ops[i].j;
    Ls.push_back(j);
    Rs.push_back(j + 1);
  }
  if (prec != TDVP_FP64) ensure_forms(S, Ls, Rs, prec == TDVP_TF32X3 ? 3 : 1, s);
  for (int i = 0; i < n; ++i) {
    const int j = ops[i].j, A = S->chiL(j), B = S->chiR(j + 1);
    P[i] = make_mv(S, M, A, B, d * d, j, j + 1, true, sl[i], prec);
    x[i] = sl[i]->theta;
    y[i] = sl[i]->theta2;
    t[i] = ops[i].tfac * tau;
    if (st) st->heff_flops += p->krylov_max * heff_flops(A, B, d * d, m, M->w2.nnz);
  }
  expm_batch(P, x, y, t, p->krylov_max, p->krylov_tol, c, ground);
  if (ground && energy) {
    LzState h{};
    CUDA_TRY(cudaMemcpyAsync(&h, sl[0]->st, sizeof(LzState), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    *energy = h.energy;
    if (st) st->krylov_vectors += h.nvec_used;
  }
  // truncated SVD re-split (Fig. 5)
  SvdBatch sb{};
  sb.n = n;
  sb.mode = prec == TDVP_FP64 ? 0 : 1;
  sb.status = S->d_status;
  sb.sync = sl[0]->sync;
  for (int i = 0; i < n; ++i) {
    const int j = ops[i].j, A = S->chiL(j), B = S->chiR(j + 1);
    SvdDesc& q = sb.d[i];
    q = SvdDesc{};
    q.theta = sl[i]->theta2;
    q.rows = A * d;
    q.cols = d * B;
    q.X = sl[i]->svdX;
    q.Acc = sl[i]->svdAcc;
    q.X32 = sl[i]->svdX32;
    q.Acc32 = sl[i]->svdAcc32;
    q.P = sl[i]->svdP;
    q.T = sl[i]->svdT;
    q.maxr = sl[i]->maxr;
    q.sig = sl[i]->sig;
    q.perm = sl[i]->perm;
    q.rotated = sl[i]->rot;
    q.conv = sl[i]->conv;
    q.chi_max = std::min(ops[i].chi_max > 0 ? ops[i].chi_max : p->chi_max, S->cap[j]);
    q.w_max = p->w_max;
    q.eps = p->eps;
    q.chi = S->d_chi + i;
    q.w = S->d_w + i;
    q.PsiL = S->Psi[j];
    q.V = S->V[j];
    q.PsiR = S->Psi[j + 1];
    q.s_sorted = n == 1 ? s_full : nullptr;
    q.zero_rel = n == 1 && s_full ? 1e-250 : 0.0;
  }
  svd_split(sb, S->d_flag, S->h_pinned, s);
  read_stage_results(S, n, s);
  for (int i = 0; i < n; ++i) {
    const int chi = S->h_pinned[2 + i];
    S->dims[ops[i].j] = chi;
    if (st) {
      st->w_total += S->h_w[i];
      st->chi_max_seen = std::max(st->chi_max_seen, chi);
    }
  }
  // environment updates (Eq. 19 and mirror)
  std::vector<EnvProb> le, re;
  ScaleBatch scl{}, scr{};
  for (int i = 0; i < n; ++i) {
    const int j = ops[i].j;
    if (ops[i].env & 1) {
      scl.d[scl.n++] = ScaleDesc{S->Psi[j], sl[i]->Amat, S->V[j], S->chiL(j), d, S->chiR(j), 0};
      le.push_back(EnvProb{S->chiL(j), S->chiR(j), d, m, S->beta[j], sl[i]->Amat, S->beta[j + 1], M->w1.op(), sl[i]});
      S->beta32_ok[j + 1] = 0;
    }
    if (ops[i].env & 2) {
      scr.d[scr.n++] = ScaleDesc{S->Psi[j + 1], sl[i]->Bmat, S->V[j], S->chiL(j + 1), d, S->chiR(j + 1), 1};
      re.push_back(EnvProb{S->chiL(j + 1), S->chiR(j + 1), d, m, S->gamma[j + 1], sl[i]->Bmat, S->gamma[j], M->w1t.op(), sl[i]});
      S->gamma32_ok[j] = 0;
    }
  }
  launch_scale_bond(scl, s);
  launch_scale_bond(scr, s);
  // env_batch uses slot temporaries; the left batch must finish its use of a
  // slot before the right batch of the same slot starts (same stream: ordered)
  env_batch(0, le, c);
  env_batch(1, re, c);
  if (st) st->n_fwd2 += n;
}

void run_back1(tdvp_mps_s* S, tdvp_mpo_s* M, const std::vector<StageOp>& ops, const tdvp_step_params* p,
               tdvp_step_stats* st, cudaStream_t s) {
  const int n = (int)ops.size();
  const int d = S->d, m = M->m, prec = p->precision;
  const double tau = 0.5 * p->dt;
  Ctx c{s, S->d_status, prec};
  std::vector<MvProb> P(n);
  std::vector<const double2*> x(n);
  std::vector<double2*> y(n);
  std::vector<double> t(n);
  std::vector<int> sites;
  for (auto& o : ops) sites.push_back(o.j);
  if (prec != TDVP_FP64) ensure_forms(S, sites, sites, prec == TDVP_TF32X3 ? 3 : 1, s);
  for (int i = 0; i < n; ++i) {
    // the two-site ops of the stage are complete (same stream): reuse their slots
    Slot* sl = slot_for(S, i, m, p->krylov_max);
    const int j = ops[i].j, A = S->chiL(j), B = S->chiR(j);
    P[i] = make_mv(S, M, A, B, d, j, j, false, sl, prec);
    x[i] = S->Psi[j];
    y[i] = S->Psi[j];
    t[i] = -tau * ops[i].tfac;
    if (st) st->heff_flops += p->krylov_max * heff_flops(A, B, d, m, M->w1.nnz);
  }
  expm_batch(P, x, y, t, p->krylov_max, p->krylov_tol, c);
  if (st) st->n_back1 += n;
}

void check_params(const tdvp_mps_s* S, const tdvp_mpo_s* M, const tdvp_step_params* p) {
  if (!p) fail(TDVP_EINVAL, "params is NULL");
  if (M->N != S->N) fail(TDVP_EINVAL, "MPO and MPS have different N");
  if (!(p->dt > 0) || p->chi_max < 1 || p->krylov_max < 1 || p->krylov_max > KRYLOV_MAX || p->w_max < 0 ||
      p->eps < 0)
    fail(TDVP_EINVAL, "invalid step parameters");
  if (p->precision < TDVP_FP64 || p->precision > TDVP_TF32X3) fail(TDVP_EINVAL, "invalid precision");
  if (p->precision != TDVP_FP64 && !tc_available()) fail(TDVP_ECUDA, "tensor-core path unavailable");
  if (S->N < 2) fail(TDVP_EINVAL, "need N >= 2");
}

void step_impl(tdvp_mps_s* S, tdvp_mpo_s* M, const tdvp_step_params* p, int n_steps, tdvp_step_stats* st,
               cudaStream_t s) {
  check_params(S, M, p);
  ensure_small_buffers(S);
  std::vector<int> seg;
  if (p->n_seg <= 1 || !p->seg_len) seg = {S->N};
  else seg.assign(p->seg_len, p->seg_len + p->n_seg);
  if ((int)seg.size() > MAXB) fail(TDVP_EINVAL, "too many segments");
  std::vector<SchedOp> halves[2];
  build_half(S->N, seg, 1, p->merge_turning, halves[0]);
  build_half(S->N, seg, 2, p->merge_turning, halves[1]);
  const int64_t l0 = g_launches;
  if (S->env_id != M->id) build_all_envs(S, M, s);
  // NVTX ranges (no cost without a tool attached): step > half > stage > fwd2 / back1
  for (int step = 0; step < n_steps; ++step) {
    nvtxRangePushA("tdvp_step");
    for (int h = 0; h < 2; ++h) {
      nvtxRangePushA(h == 0 ? "half_1" : "half_2");
      const auto& ops = halves[h];
      size_t i = 0;
      while (i < ops.size()) {
        const int stage = ops[i].stage;
        std::vector<StageOp> f, b;
        while (i < ops.size() && ops[i].stage == stage) {
          if (ops[i].kind == 0) f.push_back(StageOp{ops[i].j, ops[i].tfac, ops[i].env});
          else b.push_back(StageOp{ops[i].j, ops[i].tfac, 0});
          ++i;
        }
        nvtxRangePushA("stage");
        if (!f.empty()) {
          nvtxRangePushA("fwd2");
          run_fwd2(S, M, f, p, st, s);
          nvtxRangePop();
        }
        if (!b.empty()) {
          nvtxRangePushA("back1");
          run_back1(S, M, b, p, st, s);
          nvtxRangePop();
        }
        nvtxRangePop();
        if (st) st->n_stages += 1;
      }
      nvtxRangePop();
    }
    read_stage_results(S, 0, s);
    nvtxRangePop();
  }
  if (st) {
    st->kernel_launches += g_launches - l0;
  }
}

// Two-site DMRG sweeps: left to right over the pairs (rebuilding left
// environments), then right to left (rebuilding right environments), each
// update replacing Theta by the lowest eigenvector of H2_eff.
void dmrg_impl(tdvp_mps_s* S, tdvp_mpo_s* M, const tdvp_dmrg_params* dp, int n_sweeps, tdvp_dmrg_stats* ds,
               cudaStream_t s) {
  if (!dp) fail(TDVP_EINVAL, "params is NULL");
  tdvp_step_params p{};
  p.dt = 1.0;  // unused in ground mode
  p.chi_max = dp->chi_max;
  p.w_max = dp->w_max;
  p.eps = dp->eps;
  p.krylov_max = dp->krylov_max;
  p.krylov_tol = dp->krylov_tol;
  p.precision = dp->precision;
  check_params(S, M, &p);
  ensure_small_buffers(S);
  const int64_t l0 = g_launches;
  if (S->env_id != M->id) build_all_envs(S, M, s);
  tdvp_step_stats st{};
  double e = 0.0;
  for (int sw = 0; sw < n_sweeps; ++sw) {
    for (int j = 0; j < S->N - 1; ++j) run_fwd2(S, M, {StageOp{j, 0, 1}}, &p, &st, s, true, &e);
    for (int j = S->N - 2; j >= 0; --j) run_fwd2(S, M, {StageOp{j, 0, 2}}, &p, &st, s, true, &e);
  }
  read_stage_results(S, 0, s);
  if (ds) {
    ds->energy = e;
    ds->w_total = st.w_total;
    ds->chi_max_seen = st.chi_max_seen;
    ds->krylov_vectors = st.krylov_vectors;
    ds->n_updates = st.n_fwd2;
    ds->kernel_launches = g_launches - l0;
  }
}

// ---------------------------------------------------------------------------
// MPS creation
// ---------------------------------------------------------------------------
tdvp_mps_s* new_mps(int N, int d, int chi_cap) {
  if (N < 2 || d < 2 || d > 4 || chi_cap < 1) fail(TDVP_EINVAL, "need N >= 2, 2 <= d <= 4, chi_cap >= 1");
  require_device();
  auto* S = new tdvp_mps_s();
  S->N = N;
  S->d = d;
  S->chi_cap = chi_cap;
  S->dims.assign(N - 1, 1);
  S->cap.resize(N - 1);
  for (int j = 0; j < N - 1; ++j) {
    int64_t c = chi_cap;
    int64_t l = 1, r = 1;
    for (int e = 0; e < j + 1 && l < c; ++e) l *= d;
    for (int e = 0; e < N - 1 - j && r < c; ++e) r *= d;
    S->cap[j] = (int)std::min(c, std::min(l, r));
  }
  S->Psi.resize(N);
  S->V.resize(N - 1);
  for (int j = 0; j < N; ++j) S->Psi[j] = dalloc<double2>((size_t)S->capL(j) * d * S->capR(j));
  for (int j = 0; j < N - 1; ++j) S->V[j] = dalloc<double>(S->cap[j]);
  ensure_small_buffers(S);
  return S;
}

void free_mps(tdvp_mps_s* S) {
  if (!S) return;
  cudaDeviceSynchronize();
  for (auto p : S->Psi) dfree(p);
  for (auto p : S->V) dfree(p);
  free_envs(S);
  S->slots.clear();
  dfree(S->d_status);
  dfree(S->d_chi);
  dfree(S->d_w);
  dfree(S->d_flag);
  if (S->h_pinned) cudaFreeHost(S->h_pinned);
  if (S->h_w) cudaFreeHost(S->h_w);
  for (auto p : S->w1s) dfree(p);
  for (auto p : S->w1v) dfree(p);
  delete S;
}

// split of a (rows x cols) matrix on the device with the engine's SVD
int device_split(tdvp_mps_s* S, Slot* sl, const double2* theta, int rows, int cols, int chi_max, double w_max,
                 double eps, double2* PsiL, double* V, double2* PsiR, double* s_sorted, double* w_out,
                 cudaStream_t s) {
  SvdBatch sb{};
  sb.n = 1;
  sb.status = S->d_status;
  sb.sync = sl->sync;
  SvdDesc& q = sb.d[0];
  q = SvdDesc{};
  q.theta = theta;
  q.rows = rows;
  q.cols = cols;
  q.X = sl->svdX;
  q.Acc = sl->svdAcc;
  q.X32 = sl->svdX32;
  q.Acc32 = sl->svdAcc32;
  q.P = sl->svdP;
  q.T = sl->svdT;
  q.maxr = sl->maxr;
  q.sig = sl->sig;
  q.perm = sl->perm;
  q.rotated = sl->rot;
  q.conv = sl->conv;
  q.chi_max = chi_max;
  q.w_max = w_max;
  q.eps = eps;
  q.chi = S->d_chi;
  q.w = S->d_w;
  q.PsiL = PsiL;
  q.V = V;
  q.PsiR = PsiR;
  q.s_sorted = s_sorted;
  svd_split(sb, S->d_flag, S->h_pinned, s);
  read_stage_results(S, 1, s);
  if (w_out) *w_out = S->h_w[0];
  return S->h_pinned[2];
}

}  // namespace

// Brings the MPS with raw site tensors raw[j] ([rd[j]][d][rd[j+1]], device,
// each with room for d * chi_cap * max(rd[j+1], chi_cap) elements) to the
// inverse canonical gauge of Sec. II B in S: a left-to-right SVD sweep (A_j = U,
// Lambda V^dagger carried right), normalisation, then a right-to-left sweep
// (Psi_j = Lambda V^dagger, V_{j-1} = 1 / Lambda), truncating at chi_cap and
// the relative cutoff eps. Consumes raw. Synchronises s.
void canonicalize_device(tdvp_mps_s* S, std::vector<double2*>& raw, std::vector<int> rd, int chi_cap, double eps,
                         cudaStream_t s) {
  const int N = S->N, d = S->d;
  int64_t big = 1;
  for (int j = 0; j < N; ++j) big = std::max<int64_t>(big, (int64_t)std::max(rd[j], chi_cap) * d);
  for (int j = 0; j <= N; ++j) big = std::max<int64_t>(big, rd[j]);
  auto* sl = new Slot();
  std::unique_ptr<Slot> guard(sl);
  sl->ensure(big * big, 1, 0, big, 1);
  double2* L = dalloc<double2>(big * big);
  double2* R = dalloc<double2>(big * big);
  double* Vt = dalloc<double>(big);
  // left-to-right: A_j = U, carry Lambda V^dagger into site j+1
  for (int j = 0; j + 1 < N; ++j) {
    const int a = rd[j], b = rd[j + 1];
    const int chi = device_split(S, sl, raw[j], a * d, b, chi_cap, 0.0, eps, L, Vt, R, nullptr, nullptr, s);
    // A_j = Psi_L V  (= U), stored back in raw[j] as [a][d][chi]
    ScaleBatch sb{};
    sb.n = 1;
    sb.d[0] = ScaleDesc{L, raw[j], Vt, a * d, 1, chi, 0};
    launch_scale_bond(sb, s);
    // site j+1 <- (Lambda V^dagger) site j+1
    const int c = rd[j + 2];
    ZGemmBatch g{};
    g.n = 1;
    g.d[0] = ZGemmDesc{};
    auto& q = g.d[0];
    q.M = chi;
    q.N = d * c;
    q.K = b;
    q.A = R;
    q.a_rs = b;
    q.a_cs = 1;
    q.B = raw[j + 1];
    q.b_rs = (int64_t)d * c;
    q.b_cs = 1;
    q.C = sl->theta;
    q.c_rs = (int64_t)d * c;
    q.c_cs = 1;
    launch_zgemm(g, s);
    CUDA_TRY(cudaMemcpyAsync(raw[j + 1], sl->theta, sizeof(double2) * chi * d * c, cudaMemcpyDeviceToDevice, s));
    rd[j + 1] = chi;
  }
  // normalise: the norm is carried by the last tensor
  {
    const int64_t n = (int64_t)rd[N - 1] * d;
    std::vector<double2> h(n);
    CUDA_TRY(cudaMemcpy(h.data(), raw[N - 1], sizeof(double2) * n, cudaMemcpyDeviceToHost));
    double nrm = 0;
    for (auto& v : h) nrm += v.x * v.x + v.y * v.y;
    nrm = std::sqrt(nrm);
    if (!(nrm > 0)) fail(TDVP_ENUMERIC, "initial state has zero norm");
    for (auto& v : h) v = zscale(v, 1.0 / nrm);
    CUDA_TRY(cudaMemcpy(raw[N - 1], h.data(), sizeof(double2) * n, cudaMemcpyHostToDevice));
  }
  // right-to-left: C = U Lambda V^dagger; Psi_j = Lambda V^dagger, V_{j-1} = 1/Lambda
  for (int j = N - 1; j >= 1; --j) {
    const int a = rd[j], c = rd[j + 1];
    const int chi = device_split(S, sl, raw[j], a, d * c, chi_cap, 0.0, eps, L, S->V[j - 1], S->Psi[j],
                                 nullptr, nullptr, s);
    S->dims[j - 1] = chi;
    // site j-1 <- A_{j-1} (U Lambda)
    const int p = rd[j - 1];
    ZGemmBatch g{};
    g.n = 1;
    g.d[0] = ZGemmDesc{};
    auto& q = g.d[0];
    q.M = p * d;
    q.N = chi;
    q.K = a;
    q.A = raw[j - 1];
    q.a_rs = a;
    q.a_cs = 1;
    q.B = L;
    q.b_rs = chi;
    q.b_cs = 1;
    q.C = sl->theta;
    q.c_rs = chi;
    q.c_cs = 1;
    launch_zgemm(g, s);
    CUDA_TRY(cudaMemcpyAsync(raw[j - 1], sl->theta, sizeof(double2) * p * d * chi, cudaMemcpyDeviceToDevice, s));
    rd[j] = chi;
  }
  CUDA_TRY(cudaMemcpyAsync(S->Psi[0], raw[0], sizeof(double2) * d * rd[1], cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  dfree(L);
  dfree(R);
  dfree(Vt);
}

namespace {
void site_matrix(tdvp_mps_s* S, int j, double2* dst, cudaStream_t s);
}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* tdvp_last_error(void) { return g_last_error.c_str(); }

int tdvp_set_allocator(tdvp_alloc_fn alloc, tdvp_free_fn free_fn, void* ctx) {
  return ok_or_code([&] {
    if ((alloc == nullptr) != (free_fn == nullptr)) fail(TDVP_EINVAL, "alloc and free must both be set or both NULL");
    set_allocator(alloc, free_fn, ctx);
  });
}
const char* tdvp_version(void) { return "libtdvp 0.1 (sm_103a)"; }

int tdvp_device_ok(void) {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
    cudaGetLastError();
    return 0;
  }
  int dev = 0, major = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return 0;
  return major >= 10 ? 1 : 0;
}

int tdvp_fit_power_law(double alpha, int n_exp, int r_max, double* x_out, double* lam_out) {
  return ok_or_code([&] {
    if (!x_out || !lam_out) fail(TDVP_EINVAL, "NULL output");
    std::vector<double2> x, lam;
    host_fit_power_law(alpha, n_exp, r_max, x, lam);
    std::memcpy(x_out, x.data(), sizeof(double2) * n_exp);
    std::memcpy(lam_out, lam.data(), sizeof(double2) * n_exp);
  });
}

int tdvp_couplings(int n_exp, const double* x, const double* lam, int r_max, double* V_out) {
  return ok_or_code([&] {
    if (n_exp < 1 || r_max < 1 || !x || !lam || !V_out) fail(TDVP_EINVAL, "need n_exp >= 1, r_max >= 1, arrays");
    const double2* xx = reinterpret_cast<const double2*>(x);
    const double2* ll = reinterpret_cast<const double2*>(lam);
    for (int r = 1; r <= r_max; ++r) {
      double2 v = make_double2(0, 0);
      for (int k = 0; k < n_exp; ++k) {
        double2 p = make_double2(1, 0);  // lam_k^r by repeated multiplication
        for (int e = 0; e < r; ++e) p = zmul(p, ll[k]);
        v = zadd(v, zmul(xx[k], p));
      }
      V_out[2 * (r - 1)] = v.x;
      V_out[2 * (r - 1) + 1] = v.y;
    }
  });
}

int tdvp_mpo_couplings(tdvp_mpo mpo, int r_max, double* V_out) {
  if (!mpo) return ok_or_code([] { fail(TDVP_EINVAL, "NULL mpo"); });
  return tdvp_couplings(mpo->n_exp, reinterpret_cast<const double*>(mpo->x.data()),
                        reinterpret_cast<const double*>(mpo->lam.data()), r_max, V_out);
}

int tdvp_fit_power_law_lm(double alpha, int n_exp, int r_max, int relative, double* x_out, double* lam_out,
                          double* rms_out) {
  return ok_or_code([&] {
    if (!x_out || !lam_out) fail(TDVP_EINVAL, "NULL output");
    std::vector<double2> x, lam;
    host_fit_power_law_lm(alpha, n_exp, r_max, relative, x, lam, rms_out);
    std::memcpy(x_out, x.data(), sizeof(double2) * n_exp);
    std::memcpy(lam_out, lam.data(), sizeof(double2) * n_exp);
  });
}

int tdvp_build_mpo(const tdvp_model* model, tdvp_mpo* out) {
  return ok_or_code([&] {
    if (!model || !out) fail(TDVP_EINVAL, "NULL argument");
    if (model->kind < TDVP_ISING || model->kind > TDVP_XXX || model->N < 2 || model->n_exp < 1 ||
        model->n_exp > 64)
      fail(TDVP_EINVAL, "invalid model");
    require_device();
    auto M = std::make_unique<tdvp_mpo_s>();
    M->kind = model->kind;
    M->N = model->N;
    M->alpha = model->alpha;
    M->J = model->J;
    M->h = model->h;
    M->n_exp = model->n_exp;
    const int nt = model->kind == TDVP_ISING ? 1 : (model->kind == TDVP_XY ? 2 : 3);
    M->m = nt * model->n_exp + 2;
    if (model->x && model->lam) {
      M->x.assign((const double2*)model->x, (const double2*)model->x + model->n_exp);
      M->lam.assign((const double2*)model->lam, (const double2*)model->lam + model->n_exp);
    } else {
      host_fit_power_law(model->alpha, model->n_exp, model->N - 1, M->x, M->lam);
    }
    build_site_W(M.get());
    M->W12 = two_site_mpo(M->W, M->W, M->m, M->d);
    M->w1.build(M->W, M->m, M->d, false);
    M->w1t.build(M->W, M->m, M->d, true);
    M->w2.build(M->W12, M->m, M->d * M->d, false);
    {
      std::lock_guard<std::mutex> g(g_id_mutex);
      M->id = g_next_id++;
    }
    *out = M.release();
  });
}

int tdvp_mpo_dims(tdvp_mpo mpo, int* m, int* d) {
  return ok_or_code([&] {
    if (!mpo) fail(TDVP_EINVAL, "NULL mpo");
    if (m) *m = mpo->m;
    if (d) *d = mpo->d;
  });
}

int tdvp_mpo_tensor(tdvp_mpo mpo, double* W_out, double* x_out, double* lam_out) {
  return ok_or_code([&] {
    if (!mpo) fail(TDVP_EINVAL, "NULL mpo");
    if (W_out) std::memcpy(W_out, mpo->W.data(), sizeof(double2) * mpo->W.size());
    if (x_out) std::memcpy(x_out, mpo->x.data(), sizeof(double2) * mpo->n_exp);
    if (lam_out) std::memcpy(lam_out, mpo->lam.data(), sizeof(double2) * mpo->n_exp);
  });
}

void tdvp_free_mpo(tdvp_mpo mpo) { delete mpo; }

int tdvp_init_mps(int N, int d, const int* basis_state, int chi_cap, tdvp_mps* out) {
  return ok_or_code([&] {
    if (!basis_state || !out) fail(TDVP_EINVAL, "NULL argument");
    tdvp_mps_s* S = new_mps(N, d, chi_cap);
    try {
      for (int j = 0; j < N; ++j) {
        if (basis_state[j] < 0 || basis_state[j] >= d) fail(TDVP_EINVAL, "basis state out of range");
        std::vector<double2> t(d, make_double2(0, 0));
        t[basis_state[j]] = make_double2(1, 0);
        CUDA_TRY(cudaMemcpy(S->Psi[j], t.data(), sizeof(double2) * d, cudaMemcpyHostToDevice));
      }
      const double one = 1.0;
      for (int j = 0; j < N - 1; ++j) CUDA_TRY(cudaMemcpy(S->V[j], &one, sizeof(double), cudaMemcpyHostToDevice));
    } catch (...) {
      free_mps(S);
      throw;
    }
    *out = S;
  });
}

int tdvp_init_mps_tensors(int N, int d, const int* dims, const double* const* tensors, int chi_cap, double eps,
                          tdvp_mps* out) {
  return ok_or_code([&] {
    if (!dims || !tensors || !out) fail(TDVP_EINVAL, "NULL argument");
    if (dims[0] != 1 || dims[N] != 1) fail(TDVP_EINVAL, "boundary bond dimensions must be 1");
    tdvp_mps_s* S = new_mps(N, d, chi_cap);
    try {
      cudaStream_t s = 0;
      // raw tensors in scratch buffers large enough for the raw bond dimensions
      int64_t maxraw = 1;
      for (int j = 0; j < N; ++j) maxraw = std::max<int64_t>(maxraw, (int64_t)dims[j] * d * dims[j + 1]);
      for (int j = 0; j <= N; ++j)
        if (dims[j] < 1) fail(TDVP_EINVAL, "bond dimensions must be >= 1");
      std::vector<double2*> raw(N);
      for (int j = 0; j < N; ++j) {
        const int64_t n = (int64_t)dims[j] * d * dims[j + 1];
        raw[j] = dalloc<double2>(std::max<int64_t>(n, (int64_t)d * chi_cap * std::max(dims[j + 1], chi_cap)));
        CUDA_TRY(cudaMemcpy(raw[j], tensors[j], sizeof(double2) * n, cudaMemcpyHostToDevice));
      }
      try {
        canonicalize_device(S, raw, std::vector<int>(dims, dims + N + 1), chi_cap, eps, s);
      } catch (...) {
        for (auto p : raw) dfree(p);
        throw;
      }
      for (auto p : raw) dfree(p);
    } catch (...) {
      free_mps(S);
      throw;
    }
    *out = S;
  });
}

int tdvp_reorthonormalize(tdvp_mps mps, double eps) {
  return ok_or_code([&] {
    if (!mps) fail(TDVP_EINVAL, "NULL handle");
    if (eps < 0) fail(TDVP_EINVAL, "eps < 0");
    require_device();
    tdvp_mps_s* S = mps;
    cudaStream_t s = 0;
    CUDA_TRY(cudaDeviceSynchronize());
    const int N = S->N, d = S->d, chi_cap = S->chi_cap;
    std::vector<int> rd(N + 1, 1);
    for (int j = 0; j + 1 < N; ++j) rd[j + 1] = S->dims[j];
    std::vector<double2*> raw(N);
    for (int j = 0; j < N; ++j) {
      raw[j] = dalloc<double2>((size_t)d * chi_cap * std::max(rd[j + 1], chi_cap) +
                               (size_t)rd[j] * d * rd[j + 1]);
      site_matrix(S, j, raw[j], s);  // Psi_j V_j (the last site as it is)
    }
    try {
      canonicalize_device(S, raw, rd, chi_cap, eps, s);
    } catch (...) {
      for (auto p : raw) dfree(p);
      throw;
    }
    for (auto p : raw) dfree(p);
    S->env_id = 0;  // environments are rebuilt by the next tdvp_step / tdvp_dmrg
  });
}

int tdvp_mps_bond_dims(tdvp_mps mps, int* out) {
  return ok_or_code([&] {
    if (!mps || !out) fail(TDVP_EINVAL, "NULL argument");
    std::memcpy(out, mps->dims.data(), sizeof(int) * (mps->N - 1));
  });
}

int tdvp_mps_size(tdvp_mps mps, int* N, int* d) {
  return ok_or_code([&] {
    if (!mps) fail(TDVP_EINVAL, "NULL mps");
    if (N) *N = mps->N;
    if (d) *d = mps->d;
  });
}

int tdvp_mps_get_site(tdvp_mps mps, int j, double* out) {
  return ok_or_code([&] {
    if (!mps || !out || j < 0 || j >= mps->N) fail(TDVP_EINVAL, "bad argument");
    const size_t n = (size_t)mps->chiL(j) * mps->d * mps->chiR(j);
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(out, mps->Psi[j], sizeof(double2) * n, cudaMemcpyDeviceToHost));
  });
}

int tdvp_mps_get_bond(tdvp_mps mps, int j, double* out) {
  return ok_or_code([&] {
    if (!mps || !out || j < 0 || j >= mps->N - 1) fail(TDVP_EINVAL, "bad argument");
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(out, mps->V[j], sizeof(double) * mps->dims[j], cudaMemcpyDeviceToHost));
  });
}

void tdvp_free_mps(tdvp_mps mps) { free_mps(mps); }

int tdvp_step(tdvp_mps mps, tdvp_mpo mpo, const tdvp_step_params* params, int n_steps, tdvp_step_stats* stats,
              void* stream) {
  return ok_or_code([&] {
    if (!mps || !mpo) fail(TDVP_EINVAL, "NULL handle");
    if (n_steps < 0) fail(TDVP_EINVAL, "n_steps < 0");
    step_impl(mps, mpo, params, n_steps, stats, (cudaStream_t)stream);
  });
}

int tdvp_dmrg(tdvp_mps mps, tdvp_mpo mpo, const tdvp_dmrg_params* params, int n_sweeps, tdvp_dmrg_stats* stats,
              void* stream) {
  return ok_or_code([&] {
    if (!mps || !mpo) fail(TDVP_EINVAL, "NULL handle");
    if (n_sweeps < 0) fail(TDVP_EINVAL, "n_sweeps < 0");
    dmrg_impl(mps, mpo, params, n_sweeps, stats, (cudaStream_t)stream);
  });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Measurement (transfer matrices, FP64)
// ---------------------------------------------------------------------------
namespace {

// rho[s][s'] = sum_{a,b} conj(M[a,s,b]) Y[a,s',b]  (one block per (s, s'))
__global__ void rho_kernel(const double2* M, const double2* Y, int A, int d, int B, double2* rho) {
  const int s = blockIdx.x / d, sp = blockIdx.x % d;
  __shared__ double2 red[256];
  double2 acc = make_double2(0, 0);
  for (int64_t i = threadIdx.x; i < (int64_t)A * B; i += blockDim.x) {
    const int a = (int)(i / B), b = (int)(i % B);
    zfma_cj(acc, M[((int64_t)a * d + s) * B + b], Y[((int64_t)a * d + sp) * B + b]);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = zadd(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) rho[blockIdx.x] = red[0];
}

ZGemmDesc gemm(int M, int N, int K, const double2* A, int64_t ars, int64_t acs, int ca, const double2* B,
               int64_t brs, int64_t bcs, double2* C, int64_t crs) {
  ZGemmDesc q{};
  q.M = M;
  q.N = N;
  q.K = K;
  q.A = A;
  q.a_rs = ars;
  q.a_cs = acs;
  q.conj_a = ca;
  q.B = B;
  q.b_rs = brs;
  q.b_cs = bcs;
  q.C = C;
  q.c_rs = crs;
  q.c_cs = 1;
  return q;
}

// measurement products in double-float (~1e-14 relative, on the FP32 pipe)
void run1(const ZGemmDesc& q, cudaStream_t s) {
  ZGemmBatch g{};
  g.n = 1;
  g.d[0] = q;
  launch_zgemm_dd(g, s, "measure_dd");
}

struct MeasureBufs {
  std::vector<double2*> EL, ER;
  double2* Mj = nullptr;
  double2* X = nullptr;
  double2* Y = nullptr;
  double2* rho = nullptr;
  ~MeasureBufs() {
    for (auto p : EL) dfree(p);
    for (auto p : ER) dfree(p);
    dfree(Mj);
    dfree(X);
    dfree(Y);
    dfree(rho);
  }
};

// M_j = Psi_j V_j (V_j omitted on the last site) into dst
void site_matrix(tdvp_mps_s* S, int j, double2* dst, cudaStream_t s) {
  const int A = S->chiL(j), B = S->chiR(j), d = S->d;
  if (j == S->N - 1) {
    CUDA_TRY(cudaMemcpyAsync(dst, S->Psi[j], sizeof(double2) * A * d * B, cudaMemcpyDeviceToDevice, s));
    return;
  }
  ScaleBatch sb{};
  sb.n = 1;
  sb.d[0] = ScaleDesc{S->Psi[j], dst, S->V[j], A, d, B, 0};
  launch_scale_bond(sb, s);
}

// left transfer: E'[b][b'] = sum conj(Ma[a,s,b]) E[a,a'] Mb[a',s,b']
void transfer_left(const double2* E, const double2* Ma, const double2* Mb, int Aa, int Ab, int d, int Ba, int Bb,
                   double2* X, double2* out, cudaStream_t s) {
  run1(gemm(Aa, d * Bb, Ab, E, Ab, 1, 0, Mb, (int64_t)d * Bb, 1, X, (int64_t)d * Bb), s);
  run1(gemm(Ba, Bb, Aa * d, Ma, 1, Ba, 1, X, Bb, 1, out, Bb), s);
}

void measure_impl(tdvp_mps_s* S, const double2 op[4], double* out, bool want_local, double* norm_out) {
  cudaStream_t s = 0;
  const int N = S->N, d = S->d;
  MeasureBufs mb;
  const int64_t big = (int64_t)S->chi_cap * d * S->chi_cap;
  mb.Mj = dalloc<double2>(big);
  mb.X = dalloc<double2>(big);
  mb.Y = dalloc<double2>(big);
  mb.rho = dalloc<double2>((size_t)16 * N);
  mb.EL.resize(N + 1);
  for (int j = 0; j <= N; ++j) {
    const int c = j == 0 ? 1 : S->chiR(j - 1);
    mb.EL[j] = dalloc<double2>((size_t)c * c);
  }
  const double2 one = make_double2(1, 0);
  CUDA_TRY(cudaMemcpy(mb.EL[0], &one, sizeof(double2), cudaMemcpyHostToDevice));
  for (int j = 0; j < N; ++j) {
    site_matrix(S, j, mb.Mj, s);
    const int A = S->chiL(j), B = S->chiR(j);
    transfer_left(mb.EL[j], mb.Mj, mb.Mj, A, A, d, B, B, mb.X, mb.EL[j + 1], s);
  }
  double2 nrm;
  CUDA_TRY(cudaMemcpy(&nrm, mb.EL[N], sizeof(double2), cudaMemcpyDeviceToHost));
  if (norm_out) *norm_out = nrm.x;
  if (!want_local) return;
  if (!(nrm.x > 0)) fail(TDVP_ENUMERIC, "state has zero norm");
  mb.ER.resize(N);
  for (int j = 0; j < N; ++j) {
    const int c = S->chiR(j);
    mb.ER[j] = dalloc<double2>((size_t)c * c);
  }
  CUDA_TRY(cudaMemcpy(mb.ER[N - 1], &one, sizeof(double2), cudaMemcpyHostToDevice));
  for (int j = N - 1; j >= 1; --j) {
    site_matrix(S, j, mb.Mj, s);
    const int A = S->chiL(j), B = S->chiR(j);
    // Y[(a' s)][b] = sum_b' M[(a' s)][b'] E_R[b][b']
    run1(gemm(A * d, B, B, mb.Mj, B, 1, 0, mb.ER[j], 1, B, mb.Y, B), s);
    // E'[a][a'] = sum_(s b) conj(M[a][(s b)]) Y[a'][(s b)]
    run1(gemm(A, A, d * B, mb.Mj, (int64_t)d * B, 1, 1, mb.Y, 1, (int64_t)d * B, mb.ER[j - 1], A), s);
  }
  for (int j = 0; j < N; ++j) {
    site_matrix(S, j, mb.Mj, s);
    const int A = S->chiL(j), B = S->chiR(j);
    run1(gemm(A, d * B, A, mb.EL[j], A, 1, 0, mb.Mj, (int64_t)d * B, 1, mb.X, (int64_t)d * B), s);
    run1(gemm(A * d, B, B, mb.X, B, 1, 0, mb.ER[j], 1, B, mb.Y, B), s);
    rho_kernel<<<d * d, 256, 0, s>>>(mb.Mj, mb.Y, A, d, B, mb.rho + (size_t)16 * j);
    LAUNCH_CHECK();
  }
  std::vector<double2> rho((size_t)16 * N);
  CUDA_TRY(cudaMemcpy(rho.data(), mb.rho, sizeof(double2) * 16 * N, cudaMemcpyDeviceToHost));
  for (int j = 0; j < N; ++j) {
    double v = 0;
    for (int q = 0; q < d * d; ++q) v += rho[16 * j + q].x * op[q].x - rho[16 * j + q].y * op[q].y;
    out[j] = v / nrm.x;
  }
}

// temporary workspace for the kernel-level entry points
struct OpCtx {
  Slot slot;
  int* d_status = nullptr;
  int* d_flag = nullptr;
  int* d_chi = nullptr;
  double* d_w = nullptr;
  int* h_flag = nullptr;
  OpCtx() {
    d_status = dalloc<int>(1);
    d_flag = dalloc<int>(1);
    d_chi = dalloc<int>(1);
    d_w = dalloc<double>(1);
    CUDA_TRY(cudaMemset(d_status, 0, sizeof(int)));
    CUDA_TRY(cudaMallocHost((void**)&h_flag, sizeof(int)));
  }
  ~OpCtx() {
    dfree(d_status);
    dfree(d_flag);
    dfree(d_chi);
    dfree(d_w);
    if (h_flag) cudaFreeHost(h_flag);
  }
  void check(cudaStream_t s) {
    int st = 0;
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaMemcpy(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & 1) fail(TDVP_ETIMEOUT, "a bounded device wait gave up (tensor-core pipeline)");
    if (st & 32) fail(TDVP_ETIMEOUT, "a bounded grid barrier gave up (SVD sweeps)");
    if (st & (2 | 8)) fail(TDVP_ENUMERIC, "NaN or zero norm");
    if (st & 4) fail(TDVP_ENUMERIC, "tridiagonal eigen-solver did not converge");
    if (st & 16) fail(TDVP_ENUMERIC, "Jacobi SVD did not converge");
    if (st & 64) fail(TDVP_ENUMERIC, "SVD tail rule violated: a kept singular value lies below the tail threshold");
  }
};

void check_op_dims(int precision, int nsite, int chi_l, int chi_r, int m, int d) {
  if (precision < TDVP_FP64 || precision > TDVP_TF32X3) fail(TDVP_EINVAL, "invalid precision");
  if ((nsite != 1 && nsite != 2) || chi_l < 1 || chi_r < 1 || m < 1 || d < 2 || d > 4 || chi_l > 4096 ||
      chi_r > 4096)
    fail(TDVP_EINVAL, "invalid dimensions");
  if (precision != TDVP_FP64 && !tc_available()) fail(TDVP_ECUDA, "tensor-core path unavailable");
  require_device();
}

// H_eff problem on caller buffers; the sparse MPO is built from host W
struct OpHeff {
  DeviceWOp wop;
  MvProb prob{};
  void setup(OpCtx& C, int precision, int nsite, int chi_l, int chi_r, int m, int d, const double* W,
             const double* L, const double* R, int kmax, cudaStream_t s) {
    std::vector<double2> Wd((const double2*)W, (const double2*)W + (size_t)m * m * d * d);
    const int D = nsite == 2 ? d * d : d;
    if (nsite == 2) wop.build(two_site_mpo(Wd, Wd, m, d), m, D, false);
    else wop.build(Wd, m, D, false);
    const int c = std::max(chi_l, chi_r);
    C.slot.ensure((int64_t)chi_l * D * chi_r, (int64_t)chi_l * m * D * chi_r,
                  precision == TDVP_FP64 ? 0 : mixed_cap_floats(c, m, d), std::max<int64_t>(1, (int64_t)c * d),
                  kmax);
    prob.A = chi_l;
    prob.B = chi_r;
    prob.D = D;
    prob.m = m;
    prob.L = (const double2*)L;
    prob.R = (const double2*)R;
    prob.W = wop.op();
    prob.slot = &C.slot;
    if (precision != TDVP_FP64) {
      const bool x3 = precision == TDVP_TF32X3;
      prep_L_forms({EnvFormJob{prob.L, chi_l, m, C.slot.f[5], x3 ? C.slot.f[6] : nullptr}}, s);
      prep_R_forms({EnvFormJob{prob.R, chi_r, m, C.slot.f[7], x3 ? C.slot.f[8] : nullptr}}, s);
      prob.L32[0] = C.slot.f[5];
      prob.L32[1] = x3 ? C.slot.f[6] : nullptr;
      prob.R32[0] = C.slot.f[7];
      prob.R32[1] = x3 ? C.slot.f[8] : nullptr;
      prob.ldL = pad4(2 * (int64_t)chi_l);
      prob.ldR = pad4(2 * (int64_t)m * chi_r);
    }
  }
};

}  // namespace

extern "C" {

int tdvp_norm(tdvp_mps mps, double* out) {
  return ok_or_code([&] {
    if (!mps || !out) fail(TDVP_EINVAL, "NULL argument");
    CUDA_TRY(cudaDeviceSynchronize());
    const double2 I2[4] = {make_double2(1, 0), make_double2(0, 0), make_double2(0, 0), make_double2(1, 0)};
    measure_impl(mps, I2, nullptr, false, out);
  });
}

int tdvp_measure(tdvp_mps mps, int obs, double* out) {
  return ok_or_code([&] {
    if (!mps || !out) fail(TDVP_EINVAL, "NULL argument");
    if (mps->d != 2) fail(TDVP_EINVAL, "Pauli observables need d = 2");
    double2 op[4];
    const double2 Z = make_double2(0, 0), One = make_double2(1, 0);
    if (obs == TDVP_OBS_SZ) {
      op[0] = One; op[1] = Z; op[2] = Z; op[3] = make_double2(-1, 0);
    } else if (obs == TDVP_OBS_SX) {
      op[0] = Z; op[1] = One; op[2] = One; op[3] = Z;
    } else if (obs == TDVP_OBS_SY) {
      op[0] = Z; op[1] = make_double2(0, -1); op[2] = make_double2(0, 1); op[3] = Z;
    } else {
      fail(TDVP_EINVAL, "unknown observable");
    }
    // the reduced density matrix is rho[s][s'] ~ <s'|rho_j|s>^*: <O> = sum rho[s][s'] O[s][s']
    CUDA_TRY(cudaDeviceSynchronize());
    measure_impl(mps, op, out, true, nullptr);
  });
}

int tdvp_energy(tdvp_mps mps, tdvp_mpo mpo, double* out) {
  return ok_or_code([&] {
    if (!mps || !mpo || !out) fail(TDVP_EINVAL, "NULL argument");
    if (mpo->N != mps->N) fail(TDVP_EINVAL, "MPO and MPS have different N");
    CUDA_TRY(cudaDeviceSynchronize());
    cudaStream_t s = 0;
    ensure_small_buffers(mps);
    const int N = mps->N, m = mpo->m, d = mps->d;
    Slot* sl = slot_for(mps, 0, m, 1);
    const int64_t big = (int64_t)mps->chi_cap * mps->chi_cap * m;
    double2* E0 = dalloc<double2>(big);
    double2* E1 = dalloc<double2>(big);
    std::unique_ptr<double2, void (*)(double2*)> g0(E0, [](double2* p) { dfree(p); });
    std::unique_ptr<double2, void (*)(double2*)> g1(E1, [](double2* p) { dfree(p); });
    std::vector<double2> bl(m, make_double2(0, 0));
    bl[m - 1] = make_double2(1, 0);
    CUDA_TRY(cudaMemcpy(E0, bl.data(), sizeof(double2) * m, cudaMemcpyHostToDevice));
    Ctx c{s, mps->d_status, TDVP_FP64};
    for (int j = 0; j < N; ++j) {
      site_matrix(mps, j, sl->Amat, s);
      env_batch(0, {EnvProb{mps->chiL(j), mps->chiR(j), d, m, E0, sl->Amat, E1, mpo->w1.op(), sl}}, c);
      std::swap(E0, E1);
    }
    std::vector<double2> fin(m);
    CUDA_TRY(cudaMemcpy(fin.data(), E0, sizeof(double2) * m, cudaMemcpyDeviceToHost));
    double nrm = 0;
    const double2 I2[4] = {make_double2(1, 0), make_double2(0, 0), make_double2(0, 0), make_double2(1, 0)};
    measure_impl(mps, I2, nullptr, false, &nrm);
    if (!(nrm > 0)) fail(TDVP_ENUMERIC, "state has zero norm");
    g0.release();
    g1.release();
    dfree(E0);
    dfree(E1);
    *out = fin[0].x / nrm;
  });
}

int tdvp_overlap(tdvp_mps a, tdvp_mps b, double* out) {
  return ok_or_code([&] {
    if (!a || !b || !out) fail(TDVP_EINVAL, "NULL argument");
    if (a->N != b->N || a->d != b->d) fail(TDVP_EINVAL, "states of different shape");
    CUDA_TRY(cudaDeviceSynchronize());
    cudaStream_t s = 0;
    const int N = a->N, d = a->d;
    const int64_t big = (int64_t)std::max(a->chi_cap, b->chi_cap) * d * std::max(a->chi_cap, b->chi_cap);
    MeasureBufs mb;
    mb.Mj = dalloc<double2>(big);
    mb.Y = dalloc<double2>(big);
    mb.X = dalloc<double2>(big);
    double2* E0 = dalloc<double2>(big);
    double2* E1 = dalloc<double2>(big);
    mb.EL = {E0, E1};
    const double2 one = make_double2(1, 0);
    CUDA_TRY(cudaMemcpy(E0, &one, sizeof(double2), cudaMemcpyHostToDevice));
    for (int j = 0; j < N; ++j) {
      site_matrix(a, j, mb.Mj, s);
      site_matrix(b, j, mb.Y, s);
      transfer_left(E0, mb.Mj, mb.Y, a->chiL(j), b->chiL(j), d, a->chiR(j), b->chiR(j), mb.X, E1, s);
      std::swap(E0, E1);
    }
    double2 r;
    CUDA_TRY(cudaMemcpy(&r, E0, sizeof(double2), cudaMemcpyDeviceToHost));
    out[0] = r.x;
    out[1] = r.y;
  });
}

int tdvp_op_heff(int precision, int nsite, int chi_l, int chi_r, int m, int d, const double* W, const double* L,
                 const double* R, const double* x, double* y, void* stream) {
  return ok_or_code([&] {
    if (!W || !L || !R || !x || !y) fail(TDVP_EINVAL, "NULL argument");
    check_op_dims(precision, nsite, chi_l, chi_r, m, d);
    cudaStream_t s = (cudaStream_t)stream;
    OpCtx C;
    OpHeff H;
    H.setup(C, precision, nsite, chi_l, chi_r, m, d, W, L, R, 1, s);
    Ctx c{s, C.d_status, precision};
    matvec_batch({H.prob}, {(const double2*)x}, {(double2*)y}, c);
    C.check(s);
  });
}

int tdvp_op_expm(int precision, int nsite, int chi_l, int chi_r, int m, int d, const double* W, const double* L,
                 const double* R, const double* x, double* y, double t, int kmax, double tol, int* n_vectors,
                 void* stream) {
  return ok_or_code([&] {
    if (!W || !L || !R || !x || !y) fail(TDVP_EINVAL, "NULL argument");
    if (kmax < 1 || kmax > KRYLOV_MAX || tol < 0) fail(TDVP_EINVAL, "invalid Krylov settings");
    check_op_dims(precision, nsite, chi_l, chi_r, m, d);
    cudaStream_t s = (cudaStream_t)stream;
    OpCtx C;
    OpHeff H;
    H.setup(C, precision, nsite, chi_l, chi_r, m, d, W, L, R, kmax, s);
    Ctx c{s, C.d_status, precision};
    expm_batch({H.prob}, {(const double2*)x}, {(double2*)y}, {t}, kmax, tol, c);
    C.check(s);
    if (n_vectors) {
      LzState st;
      CUDA_TRY(cudaMemcpy(&st, C.slot.st, sizeof(LzState), cudaMemcpyDeviceToHost));
      *n_vectors = st.nvec_used;
    }
  });
}

int tdvp_op_env(int precision, int side, int chi_l, int chi_r, int m, int d, const double* W, const double* env,
                const double* A, double* out, void* stream) {
  return ok_or_code([&] {
    if (!W || !env || !A || !out) fail(TDVP_EINVAL, "NULL argument");
    if (side != 0 && side != 1) fail(TDVP_EINVAL, "side must be 0 or 1");
    check_op_dims(precision, 1, chi_l, chi_r, m, d);
    cudaStream_t s = (cudaStream_t)stream;
    OpCtx C;
    DeviceWOp wop;
    std::vector<double2> Wd((const double2*)W, (const double2*)W + (size_t)m * m * d * d);
    wop.build(Wd, m, d, side == 1);
    const int c = std::max(chi_l, chi_r);
    C.slot.ensure((int64_t)chi_l * d * chi_r, (int64_t)c * m * d * c,
                  precision == TDVP_FP64 ? 0 : mixed_cap_floats(c, m, d), (int64_t)c * d, 1);
    Ctx cx{s, C.d_status, precision};
    env_batch(side, {EnvProb{chi_l, chi_r, d, m, (const double2*)env, (const double2*)A, (double2*)out, wop.op(),
                             &C.slot}},
              cx);
    C.check(s);
  });
}

int tdvp_op_split(int rows, int cols, const double* theta, int chi_max, double w_max, double eps, double* Psi_L,
                  double* V, double* Psi_R, double* s_out, int* chi, double* w, void* stream) {
  return tdvp_op_split_prec(TDVP_FP64, rows, cols, theta, chi_max, w_max, eps, Psi_L, V, Psi_R, s_out, chi, w,
                            stream);
}

int tdvp_op_split_prec(int precision, int rows, int cols, const double* theta, int chi_max, double w_max, double eps,
                       double* Psi_L, double* V, double* Psi_R, double* s_out, int* chi, double* w, void* stream) {
  return ok_or_code([&] {
    if (precision < TDVP_FP64 || precision > TDVP_TF32X3) fail(TDVP_EINVAL, "invalid precision");
    if (!theta || !Psi_L || !V || !Psi_R || !chi || !w) fail(TDVP_EINVAL, "NULL argument");
    if (rows < 1 || cols < 1 || rows > 4096 || cols > 4096 || chi_max < 1 || w_max < 0 || eps < 0)
      fail(TDVP_EINVAL, "invalid arguments");
    require_device();
    cudaStream_t s = (cudaStream_t)stream;
    OpCtx C;
    const int64_t nv = std::min(rows, cols), len = std::max(rows, cols);
    C.slot.ensure(nv * len, 1, 0, nv, 1);
    // the Acc buffer must hold nv*nv and X nv*len: both <= cap_vec = max(nv*len, nv*nv)
    SvdBatch sb{};
    sb.n = 1;
    sb.mode = precision == TDVP_FP64 ? 0 : 1;
    sb.status = C.d_status;
    sb.sync = C.slot.sync;
    SvdDesc& q = sb.d[0];
    q = SvdDesc{};
    q.theta = (const double2*)theta;
    q.rows = rows;
    q.cols = cols;
    q.X = C.slot.svdX;
    q.Acc = C.slot.svdAcc;
    q.X32 = C.slot.svdX32;
    q.Acc32 = C.slot.svdAcc32;
    q.P = C.slot.svdP;
    q.T = C.slot.svdT;
    q.maxr = C.slot.maxr;
    q.sig = C.slot.sig;
    q.perm = C.slot.perm;
    q.rotated = C.slot.rot;
    q.conv = C.slot.conv;
    q.chi_max = chi_max;
    q.w_max = w_max;
    q.eps = eps;
    q.chi = C.d_chi;
    q.w = C.d_w;
    q.PsiL = (double2*)Psi_L;
    q.V = V;
    q.PsiR = (double2*)Psi_R;
    q.s_sorted = s_out;
    svd_split(sb, C.d_flag, C.h_flag, s);
    C.check(s);
    CUDA_TRY(cudaMemcpy(chi, C.d_chi, sizeof(int), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(w, C.d_w, sizeof(double), cudaMemcpyDeviceToHost));
  });
}

int tdvp_exchange_plan(int N, int n_seg, const int* seg_len, const int* seg_rank, int scheme, int merge_turning,
                       int half, int* out, int max_msgs) {
  int count = 0;
  int rc = ok_or_code([&] {
    if (half != 1 && half != 2) fail(TDVP_EINVAL, "half must be 1 or 2");
    if (N < 2 || n_seg < 1 || !seg_len || !seg_rank) fail(TDVP_EINVAL, "invalid arguments");
    std::vector<int> seg(seg_len, seg_len + n_seg), rk(seg_rank, seg_rank + n_seg);
    for (int k = 0; k < n_seg; ++k)
      if (rk[k] < 0 || (k > 0 && rk[k] < rk[k - 1])) fail(TDVP_EINVAL, "ranks must hold contiguous groups of segments");
    std::vector<ExchangeMsg> msgs;
    exchange_plan(N, seg, rk, scheme, merge_turning, half, msgs);
    count = (int)msgs.size();
    if (out) {
      if (max_msgs < count) fail(TDVP_EINVAL, "output too small");
      for (int i = 0; i < count; ++i) {
        const ExchangeMsg& m = msgs[i];
        int* r = out + 6 * i;
        r[0] = m.stage;
        r[1] = m.after;
        r[2] = m.src;
        r[3] = m.dst;
        r[4] = m.kind;
        r[5] = m.j;
      }
    }
  });
  return rc == TDVP_OK ? count : rc;
}

int tdvp_schedule1(int N, int n_seg, const int* seg_len, int merge_turning, int half, int* out, int max_ops) {
  int count = 0;
  int rc = ok_or_code([&] {
    if (half != 1 && half != 2) fail(TDVP_EINVAL, "half must be 1 or 2");
    if (N < 2) fail(TDVP_EINVAL, "need N >= 2");
    std::vector<int> seg;
    if (n_seg <= 1 || !seg_len) seg = {N};
    else seg.assign(seg_len, seg_len + n_seg);
    std::vector<SchedOp> ops;
    build_half1(N, seg, half, merge_turning, ops);
    count = (int)ops.size();
    if (out) {
      if (max_ops < count) fail(TDVP_EINVAL, "output too small");
      for (int i = 0; i < count; ++i) {
        const SchedOp& o = ops[i];
        int* r = out + 7 * i;
        r[0] = o.seg;
        r[1] = o.kind;
        r[2] = o.j;
        r[3] = o.tfac;
        r[4] = o.env;
        r[5] = o.boundary;
        r[6] = o.stage;
      }
    }
  });
  return rc == TDVP_OK ? count : rc;
}

int tdvp_schedule(int N, int n_seg, const int* seg_len, int merge_turning, int half, int* out, int max_ops) {
  int count = 0;
  int rc = ok_or_code([&] {
    if (half != 1 && half != 2) fail(TDVP_EINVAL, "half must be 1 or 2");
    std::vector<int> seg;
    if (n_seg <= 1 || !seg_len) seg = {N};
    else seg.assign(seg_len, seg_len + n_seg);
    if (N < 2) fail(TDVP_EINVAL, "need N >= 2");
    std::vector<SchedOp> ops;
    build_half(N, seg, half, merge_turning, ops);
    count = (int)ops.size();
    if (out) {
      if (max_ops < count) fail(TDVP_EINVAL, "output too small");
      for (int i = 0; i < count; ++i) {
        const SchedOp& o = ops[i];
        int* r = out + 7 * i;
        r[0] = o.seg;
        r[1] = o.kind;
        r[2] = o.j;
        r[3] = o.tfac;
        r[4] = o.env;
        r[5] = o.boundary;
        r[6] = o.stage;
      }
    }
  });
  return rc == TDVP_OK ? count : rc;
}

int tdvp_tridiag_expm(int k, const double* alpha, const double* beta, double t, double* c_out) {
  return ok_or_code([&] {
    if (k < 1 || k > KRYLOV_MAX || !alpha || !c_out || (k > 1 && !beta)) fail(TDVP_EINVAL, "bad argument");
    std::vector<double> work(2 * k * k);
    std::vector<double2> c(k);
    if (tridiag_expm_e0(k, alpha, beta, t, c.data(), work.data()) < 0)
      fail(TDVP_ENUMERIC, "tridiagonal eigen-solver did not converge");
    std::memcpy(c_out, c.data(), sizeof(double2) * k);
  });
}

int tdvp_profile(int enable) {
  return ok_or_code([&] {
    CUDA_TRY(cudaDeviceSynchronize());
    prof_enable(enable != 0);
  });
}

static int profile_read_impl(int idx, char* name, int name_len, double* ms, int64_t* launches, double* flops,
                             double* bytes, double* aux) {
  int n = 0;
  int rc = ok_or_code([&] {
    std::string nm;
    double t = 0, f = 0, b = 0, a = 0;
    int64_t l = 0;
    if (idx < 0) {
      n = prof_read(-1, nm, t, l, f, b, a);
      return;
    }
    if (!prof_read(idx, nm, t, l, f, b, a)) fail(TDVP_EINVAL, "profile index out of range");
    if (name && name_len > 0) {
      std::strncpy(name, nm.c_str(), name_len - 1);
      name[name_len - 1] = 0;
    }
    if (ms) *ms = t;
    if (launches) *launches = l;
    if (flops) *flops = f;
    if (bytes) *bytes = b;
    if (aux) *aux = a;
    n = 1;
  });
  return rc == TDVP_OK ? n : rc;
}

int tdvp_profile_read(int idx, char* name, int name_len, double* ms, int64_t* launches, double* flops,
                      double* bytes) {
  return profile_read_impl(idx, name, name_len, ms, launches, flops, bytes, nullptr);
}

int tdvp_profile_read_aux(int idx, double* aux) {
  return profile_read_impl(idx, nullptr, 0, nullptr, nullptr, nullptr, nullptr, aux);
}

int tdvp_set_env_tensor_cores(int enable) {
  set_env_on_tensor_cores(enable != 0);
  return TDVP_OK;
}

int tdvp_set_autotune(int enable) {
  tune_enable(enable != 0);
  return TDVP_OK;
}

int tdvp_autotune_report(char* out, int len) {
  const std::string r = tune_report();
  if (out && len > 0) {
    const size_t n = std::min<size_t>(r.size(), (size_t)len - 1);
    std::memcpy(out, r.data(), n);
    out[n] = 0;
  }
  return (int)r.size();
}

int tdvp_set_wait_limit(long long spins) {
  svd_set_spin_limit(spins);
  return TDVP_OK;
}

int tdvp_op_heff_noalloc(int nsite, int chi_l, int chi_r, int m, int d, const double* W, const double* L,
                         const double* R, const double* x, double* y, void* stream) {
  return ok_or_code([&] {
    if (!W || !L || !R || !x || !y) fail(TDVP_EINVAL, "NULL argument");
    require_device();
    op_heff_noalloc(nsite, chi_l, chi_r, m, d, W, L, R, x, y, (cudaStream_t)stream);
  });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Forward-mode derivative of the sweep with respect to model parameters
// ---------------------------------------------------------------------------
constexpr int TAN_MAX_QUAD = 8;

struct tdvp_tangent_s {
  tdvp_mps_s* S = nullptr;
  int nd = 0;
  int N = 0, d = 2, chi_cap = 1;
  std::vector<double2*> dPsi[TDVP_MAX_DIR];
  std::vector<double*> dV[TDVP_MAX_DIR];
  std::vector<double2*> dbeta[TDVP_MAX_DIR], dgamma[TDVP_MAX_DIR];
  int env_m = 0;
  uint64_t env_id = 0;                 // MPO whose tangent environments are held
  std::vector<uint64_t> env_dids;      // and its derivative MPOs, per direction
  int64_t vec = 0;                     // chi_cap^2 d^2
  double2 *U = nullptr, *Vh = nullptr, *Am = nullptr;
  double* s_full = nullptr;
  double2 *dTh[TDVP_MAX_DIR] = {}, *dTh2[TDVP_MAX_DIR] = {}, *Tm[TDVP_MAX_DIR] = {}, *dP[TDVP_MAX_DIR] = {};
  double2 *CL[TDVP_MAX_DIR] = {}, *CR[TDVP_MAX_DIR] = {}, *dAm[TDVP_MAX_DIR] = {};
  double2* qb[TAN_MAX_QUAD] = {};
  double2* qc[TAN_MAX_QUAD * TDVP_MAX_DIR] = {};

  void free_envs() {
    for (int q = 0; q < TDVP_MAX_DIR; ++q) {
      for (auto p : dbeta[q]) dfree(p);
      for (auto p : dgamma[q]) dfree(p);
      dbeta[q].clear();
      dgamma[q].clear();
    }
    env_id = 0;
    env_m = 0;
    env_dids.clear();
  }
  ~tdvp_tangent_s() {
    cudaDeviceSynchronize();
    for (int q = 0; q < TDVP_MAX_DIR; ++q) {
      for (auto p : dPsi[q]) dfree(p);
      for (auto p : dV[q]) dfree(p);
      for (double2* p : {dTh[q], dTh2[q], Tm[q], dP[q], CL[q], CR[q], dAm[q]}) dfree(p);
    }
    free_envs();
    for (auto p : qb) dfree(p);
    for (auto p : qc) dfree(p);
    dfree(U);
    dfree(Vh);
    dfree(Am);
    dfree(s_full);
  }
};

namespace {

using Tan = tdvp_tangent_s;

double2* dzeros(int64_t n) {
  double2* p = dalloc<double2>((size_t)std::max<int64_t>(n, 1));
  CUDA_TRY(cudaMemset(p, 0, sizeof(double2) * std::max<int64_t>(n, 1)));
  return p;
}

// A_j = Psi_j V_j into T->Am and dA_j = dPsi_j V_j + Psi_j dV_j into T->dAm[q]
// (side 0); B = V_j Psi_{j+1}, dB = dV_j Psi_{j+1} + V_j dPsi_{j+1} (side 1).
void bond_mats(Tan* T, tdvp_mps_s* S, int side, int j, cudaStream_t s) {
  const int d = S->d;
  ScaleBatch sb{};
  const int site = side == 0 ? j : j + 1;
  const int A = S->chiL(site), B = S->chiR(site);
  sb.d[sb.n++] = ScaleDesc{S->Psi[site], T->Am, S->V[j], A, d, B, side, nullptr, nullptr};
  for (int q = 0; q < T->nd; ++q)
    sb.d[sb.n++] = ScaleDesc{T->dPsi[q][site], T->dAm[q], S->V[j], A, d, B, side, S->Psi[site], T->dV[q][j]};
  launch_scale_bond(sb, s);
}

// tangent of beta_{j+1} (side 0) or gamma_j (side 1) by the product rule on Eq. 19:
// dE' = E(dE; M, M; W) + E(E; bra M, ket dM; W) + E(E; bra dM, ket M; W) + E(E; M, M; dW)
void tangent_env(Tan* T, tdvp_mps_s* S, tdvp_mpo_s* M, const std::vector<tdvp_mpo_s*>& dM, int side, int j,
                 cudaStream_t s) {
  const int d = S->d, m = M->m, nd = T->nd;
  bond_mats(T, S, side, j, s);
  Ctx c{s, S->d_status, TDVP_FP64};
  const int site = side == 0 ? j : j + 1;
  const int A = S->chiL(site), B = S->chiR(site);
  for (int term = 0; term < 4; ++term) {
    std::vector<EnvProb> P;
    for (int q = 0; q < nd; ++q) {
      Slot* sl = slot_for(S, 1 + q, m, 1);
      EnvProb e{};
      e.A = A;
      e.B = B;
      e.d = d;
      e.m = m;
      e.slot = sl;
      e.env = side == 0 ? (term == 0 ? T->dbeta[q][j] : S->beta[j]) : (term == 0 ? T->dgamma[q][j + 1] : S->gamma[j + 1]);
      e.mat = term == 1 ? T->dAm[q] : T->Am;                                  // ket
      e.bra = term == 1 ? T->Am : (term == 2 ? T->dAm[q] : nullptr);         // bra (null: = ket)
      if (term == 3) e.W = side == 0 ? dM[q]->w1.op() : dM[q]->w1t.op();
      else e.W = side == 0 ? M->w1.op() : M->w1t.op();
      e.out = side == 0 ? T->dbeta[q][j + 1] : T->dgamma[q][j];
      e.accumulate = term > 0;
      P.push_back(e);
    }
    env_batch(side, P, c);
  }
}

void tangent_alloc(Tan* T, int m) {
  tdvp_mps_s* S = T->S;
  if (T->env_m != m) {
    T->free_envs();
    for (int q = 0; q < T->nd; ++q) {
      T->dbeta[q].resize(S->N);
      T->dgamma[q].resize(S->N);
      for (int j = 0; j < S->N; ++j) {
        T->dbeta[q][j] = dzeros((int64_t)S->capL(j) * S->capL(j) * m);
        T->dgamma[q][j] = dzeros((int64_t)S->capR(j) * S->capR(j) * m);
      }
    }
    T->env_m = m;
  }
}

// all tangent environments from scratch, with the primal ones rebuilt alongside
void build_tangent_envs(Tan* T, tdvp_mps_s* S, tdvp_mpo_s* M, const std::vector<tdvp_mpo_s*>& dM,
                        cudaStream_t s) {
  build_all_envs(S, M, s);
  tangent_alloc(T, M->m);
  const int N = S->N, m = M->m;
  for (int q = 0; q < T->nd; ++q) {
    CUDA_TRY(cudaMemsetAsync(T->dbeta[q][0], 0, sizeof(double2) * m, s));
    CUDA_TRY(cudaMemsetAsync(T->dgamma[q][N - 1], 0, sizeof(double2) * m, s));
  }
  for (int j = 0; j + 1 < N; ++j) tangent_env(T, S, M, dM, 0, j, s);
  for (int j = N - 2; j >= 0; --j) tangent_env(T, S, M, dM, 1, j, s);
  T->env_id = M->id;
  T->env_dids.clear();
  for (auto* p : dM) T->env_dids.push_back(p->id);
}

// d(exp(-i t H) x) for H = H_eff(L, W, R) of one local problem and every
// direction q: dy_q = exp(-i t H) dx_q + sum_n w_n (-i t) exp(-i s_n t H) dH_q exp(-i (1 - s_n) t H) x.
// x: primal input (unchanged); dx[q] -> dy[q] (may alias). base: the primal
// MvProb; dL/dR/dWop: tangent environments and derivative MPO operators.
void tangent_expm(Tan* T, tdvp_mps_s* S, const MvProb& base, const double2* x, const std::vector<double2*>& dx,
                  const std::vector<double2*>& dy, const std::vector<const double2*>& dL,
                  const std::vector<const double2*>& dR, const std::vector<WOp>& dWop, double t,
                  const std::vector<double>& xq, const std::vector<double>& wq, const tdvp_step_params* p,
                  int m, cudaStream_t s) {
  const int nd = T->nd, nq = (int)xq.size();
  Ctx c{s, S->d_status, TDVP_FP64};
  // exp(-i (1 - s_n) t H) x and exp(-i t H) dx_q
  {
    std::vector<MvProb> P;
    std::vector<const double2*> xi;
    std::vector<double2*> yo;
    std::vector<double> tt;
    for (int n = 0; n < nq; ++n) {
      MvProb q = base;
      q.slot = slot_for(S, 1 + P.size(), m, p->krylov_max);
      P.push_back(q);
      xi.push_back(x);
      yo.push_back(T->qb[n]);
      tt.push_back((1.0 - xq[n]) * t);
    }
    for (int k = 0; k < nd; ++k) {
      MvProb q = base;
      q.slot = slot_for(S, 1 + P.size(), m, p->krylov_max);
      P.push_back(q);
      xi.push_back(dx[k]);
      yo.push_back(dy[k]);
      tt.push_back(t);
    }
    expm_batch(P, xi, yo, tt, p->krylov_max, p->krylov_tol, c);
  }
  // c_{n,q} = dH_q b_n (three H_eff products, summed)
  for (int term = 0; term < 3; ++term) {
    std::vector<MvProb> P;
    std::vector<const double2*> xi;
    std::vector<double2*> yo;
    for (int n = 0; n < nq; ++n)
      for (int k = 0; k < nd; ++k) {
        MvProb q = base;
        q.slot = slot_for(S, 1 + P.size(), m, p->krylov_max);
        if (term == 0) q.L = dL[k];
        if (term == 1) q.W = dWop[k];
        if (term == 2) q.R = dR[k];
        P.push_back(q);
        xi.push_back(T->qb[n]);
        yo.push_back(T->qc[n * nd + k]);
      }
    matvec_batch(P, xi, yo, c, term > 0);
  }
  // exp(-i s_n t H) c_{n,q}, in place
  {
    std::vector<MvProb> P;
    std::vector<const double2*> xi;
    std::vector<double2*> yo;
    std::vector<double> tt;
    for (int n = 0; n < nq; ++n)
      for (int k = 0; k < nd; ++k) {
        MvProb q = base;
        q.slot = slot_for(S, 1 + P.size(), m, p->krylov_max);
        P.push_back(q);
        xi.push_back(T->qc[n * nd + k]);
        yo.push_back(T->qc[n * nd + k]);
        tt.push_back(xq[n] * t);
      }
    expm_batch(P, xi, yo, tt, p->krylov_max, p->krylov_tol, c);
  }
  ZCombBatch zb{};
  const int64_t len = (int64_t)base.A * base.D * base.B;
  for (int k = 0; k < nd; ++k) {
    ZCombDesc& z = zb.d[zb.n++];
    z = ZCombDesc{};
    z.y = dy[k];
    z.n = len;
    z.accumulate = 1;
    z.n_terms = nq;
    for (int n = 0; n < nq; ++n) {
      z.x[n] = T->qc[n * nd + k];
      z.c[n] = make_double2(0.0, -t * wq[n]);
    }
  }
  launch_zcombine(zb, s);
}

void tangent_fwd2(Tan* T, tdvp_mps_s* S, tdvp_mpo_s* M, const std::vector<tdvp_mpo_s*>& dM, const StageOp& op,
                  const tdvp_step_params* p, const std::vector<double>& xq, const std::vector<double>& wq,
                  tdvp_step_stats* st, cudaStream_t s) {
  const int j = op.j, d = S->d, m = M->m, nd = T->nd;
  const double t = op.tfac * 0.5 * p->dt;
  {
    // dTheta = dPsi_j V_j Psi_{j+1} + Psi_j dV_j Psi_{j+1} + Psi_j V_j dPsi_{j+1}
    const int A = S->chiL(j), cb = S->dims[j], B = S->chiR(j + 1);
    for (int term = 0; term < 3; ++term) {
      ZGemmBatch g{};
      g.n = nd;
      for (int q = 0; q < nd; ++q) {
        ZGemmDesc& z = g.d[q];
        z = ZGemmDesc{};
        z.M = A * d;
        z.N = d * B;
        z.K = cb;
        z.A = term == 0 ? T->dPsi[q][j] : S->Psi[j];
        z.a_rs = cb;
        z.a_cs = 1;
        z.kscale = term == 1 ? T->dV[q][j] : S->V[j];
        z.B = term == 2 ? T->dPsi[q][j + 1] : S->Psi[j + 1];
        z.b_rs = (int64_t)d * B;
        z.b_cs = 1;
        z.C = T->dTh[q];
        z.c_rs = (int64_t)d * B;
        z.c_cs = 1;
        z.accumulate = term > 0;
      }
      launch_zgemm(g, s, "tangent_zgemm");
    }
  }
  // the primal update, with the full SVD kept converged
  run_fwd2(S, M, {op}, p, st, s, false, nullptr, T->s_full);
  Slot* s0 = S->slots[0].get();
  const int A = S->chiL(j), B = S->chiR(j + 1), k = S->dims[j];
  // d(exp(-i t H2_eff) Theta)
  {
    MvProb base = make_mv(S, M, A, B, d * d, j, j + 1, true, s0, TDVP_FP64);
    std::vector<double2*> dx, dy;
    std::vector<const double2*> dL, dR;
    std::vector<WOp> dW;
    for (int q = 0; q < nd; ++q) {
      dx.push_back(T->dTh[q]);
      dy.push_back(T->dTh2[q]);
      dL.push_back(T->dbeta[q][j]);
      dR.push_back(T->dgamma[q][j + 1]);
      dW.push_back(dM[q]->w2.op());
    }
    tangent_expm(T, S, base, s0->theta, dx, dy, dL, dR, dW, t, xq, wq, p, m, s);
  }
  // derivative of the truncated split
  const int rows = A * d, cols = d * B;
  const int trans = rows > cols ? 1 : 0;
  const int r = trans ? cols : rows, len = trans ? rows : cols;
  launch_svd_export_full(SvdFullDesc{s0->svdX, s0->svdAcc, s0->sig, s0->perm, rows, cols, r, len, trans, T->U, T->Vh,
                                     T->s_full},
                         s);
  auto gemm_batch = [&](auto fill, const char* name) {
    ZGemmBatch g{};
    g.n = nd;
    for (int q = 0; q < nd; ++q) {
      g.d[q] = ZGemmDesc{};
      fill(g.d[q], q);
      g.d[q].c_cs = 1;
    }
    launch_zgemm(g, s, name);
  };
  // Tm = dTheta' V (rows x r), dP = U^H Tm (r x r)
  gemm_batch([&](ZGemmDesc& z, int q) {
    z.M = rows; z.N = r; z.K = cols;
    z.A = T->dTh2[q]; z.a_rs = cols; z.a_cs = 1;
    z.B = T->Vh; z.b_rs = 1; z.b_cs = cols; z.conj_b = 1;
    z.C = T->Tm[q]; z.c_rs = r;
  }, "tangent_zgemm");
  gemm_batch([&](ZGemmDesc& z, int q) {
    z.M = r; z.N = r; z.K = rows;
    z.A = T->U; z.a_rs = 1; z.a_cs = r; z.conj_a = 1;
    z.B = T->Tm[q]; z.b_rs = r; z.b_cs = 1;
    z.C = T->dP[q]; z.c_rs = r;
  }, "tangent_zgemm");
  {
    SvdTanBatch tb{};
    tb.n = nd;
    for (int q = 0; q < nd; ++q) tb.d[q] = SvdTanDesc{T->dP[q], T->s_full, r, k, T->CL[q], T->CR[q], T->dV[q][j]};
    launch_svd_tangent_coef(tb, s);
  }
  // dPsi_L = dTheta' V_k + U CL   (rows x k)
  gemm_batch([&](ZGemmDesc& z, int q) {
    z.M = rows; z.N = k; z.K = cols;
    z.A = T->dTh2[q]; z.a_rs = cols; z.a_cs = 1;
    z.B = T->Vh; z.b_rs = 1; z.b_cs = cols; z.conj_b = 1;
    z.C = T->dPsi[q][j]; z.c_rs = k;
  }, "tangent_zgemm");
  gemm_batch([&](ZGemmDesc& z, int q) {
    z.M = rows; z.N = k; z.K = r;
    z.A = T->U; z.a_rs = r; z.a_cs = 1;
    z.B = T->CL[q]; z.b_rs = k; z.b_cs = 1;
    z.C = T->dPsi[q][j]; z.c_rs = k; z.accumulate = 1;
  }, "tangent_zgemm");
  // dPsi_R = CR^H V^H + U_k^H dTheta'   (k x cols)
  gemm_batch([&](ZGemmDesc& z, int q) {
    z.M = k; z.N = cols; z.K = r;
    z.A = T->CR[q]; z.a_rs = 1; z.a_cs = k; z.conj_a = 1;
    z.B = T->Vh; z.b_rs = cols; z.b_cs = 1;
    z.C = T->dPsi[q][j + 1]; z.c_rs = cols;
  }, "tangent_zgemm");
  gemm_batch([&](ZGemmDesc& z, int q) {
    z.M = k; z.N = cols; z.K = rows;
    z.A = T->U; z.a_rs = 1; z.a_cs = r; z.conj_a = 1;
    z.B = T->dTh2[q]; z.b_rs = cols; z.b_cs = 1;
    z.C = T->dPsi[q][j + 1]; z.c_rs = cols; z.accumulate = 1;
  }, "tangent_zgemm");
  if (op.env & 1) tangent_env(T, S, M, dM, 0, j, s);
  if (op.env & 2) tangent_env(T, S, M, dM, 1, j, s);
}

void tangent_back1(Tan* T, tdvp_mps_s* S, tdvp_mpo_s* M, const std::vector<tdvp_mpo_s*>& dM, const StageOp& op,
                   const tdvp_step_params* p, const std::vector<double>& xq, const std::vector<double>& wq,
                   tdvp_step_stats* st, cudaStream_t s) {
  const int j = op.j, d = S->d, m = M->m, nd = T->nd;
  const double t = -op.tfac * 0.5 * p->dt;
  const int A = S->chiL(j), B = S->chiR(j);
  Slot* s0 = slot_for(S, 0, m, p->krylov_max);
  MvProb base = make_mv(S, M, A, B, d, j, j, false, s0, TDVP_FP64);
  std::vector<double2*> dx;
  std::vector<const double2*> dL, dR;
  std::vector<WOp> dW;
  for (int q = 0; q < nd; ++q) {
    dx.push_back(T->dPsi[q][j]);
    dL.push_back(T->dbeta[q][j]);
    dR.push_back(T->dgamma[q][j]);
    dW.push_back(dM[q]->w1.op());
  }
  tangent_expm(T, S, base, S->Psi[j], dx, dx, dL, dR, dW, t, xq, wq, p, m, s);
  run_back1(S, M, {op}, p, st, s);
}

void tangent_workspace(Tan* T) {
  if (T->U) return;
  const int64_t v = T->vec;
  T->U = dzeros(v);
  T->Vh = dzeros(v);
  T->Am = dzeros(v);
  T->s_full = dalloc<double>((size_t)T->chi_cap * T->d);
  for (int q = 0; q < T->nd; ++q) {
    T->dTh[q] = dzeros(v);
    T->dTh2[q] = dzeros(v);
    T->Tm[q] = dzeros(v);
    T->dP[q] = dzeros(v);
    T->CL[q] = dzeros(v);
    T->CR[q] = dzeros(v);
    T->dAm[q] = dzeros(v);
  }
  for (int n = 0; n < TAN_MAX_QUAD; ++n) T->qb[n] = dzeros(v);
  for (int n = 0; n < TAN_MAX_QUAD * T->nd; ++n) T->qc[n] = dzeros(v);
}

void step_tangent_impl(tdvp_mps_s* S, tdvp_mpo_s* M, Tan* T, const tdvp_mpo* dmpo, const tdvp_step_params* p,
                       int nq, int n_steps, tdvp_step_stats* st, cudaStream_t s) {
  check_params(S, M, p);
  if (T->S != S) fail(TDVP_EINVAL, "tangent belongs to another MPS");
  if (p->precision != TDVP_FP64) fail(TDVP_EINVAL, "derivatives are computed in FP64 only");
  if (nq < 1 || nq > TAN_MAX_QUAD || nq * T->nd > MAXB - 1 || nq + T->nd > MAXB - 1)
    fail(TDVP_EINVAL, "n_quad must be in [1, 8] with n_quad * n_dir <= 31");
  if (!dmpo) fail(TDVP_EINVAL, "NULL derivative MPO list");
  std::vector<tdvp_mpo_s*> dM(T->nd);
  for (int q = 0; q < T->nd; ++q) {
    dM[q] = dmpo[q];
    if (!dM[q] || dM[q]->base_id != M->id || dM[q]->m != M->m)
      fail(TDVP_EINVAL, "derivative MPO does not belong to this MPO");
  }
  ensure_small_buffers(S);
  tangent_workspace(T);
  std::vector<double> xq, wq;
  gauss_legendre01(nq, xq, wq);
  std::vector<int> seg;
  if (p->n_seg <= 1 || !p->seg_len) seg = {S->N};
  else seg.assign(p->seg_len, p->seg_len + p->n_seg);
  if ((int)seg.size() > MAXB) fail(TDVP_EINVAL, "too many segments");
  std::vector<SchedOp> halves[2];
  build_half(S->N, seg, 1, p->merge_turning, halves[0]);
  build_half(S->N, seg, 2, p->merge_turning, halves[1]);
  const int64_t l0 = g_launches;
  bool fresh = T->env_id != M->id || S->env_id != M->id || (int)T->env_dids.size() != T->nd;
  for (int q = 0; q < T->nd && !fresh; ++q) fresh = T->env_dids[q] != dM[q]->id;
  if (fresh) build_tangent_envs(T, S, M, dM, s);
  for (int step = 0; step < n_steps; ++step) {
    for (int h = 0; h < 2; ++h) {
      const auto& ops = halves[h];
      size_t i = 0;
      while (i < ops.size()) {
        const int stage = ops[i].stage;
        std::vector<StageOp> f, b;
        while (i < ops.size() && ops[i].stage == stage) {
          if (ops[i].kind == 0) f.push_back(StageOp{ops[i].j, ops[i].tfac, ops[i].env});
          else b.push_back(StageOp{ops[i].j, ops[i].tfac, 0});
          ++i;
        }
        for (auto& o : f) tangent_fwd2(T, S, M, dM, o, p, xq, wq, st, s);
        for (auto& o : b) tangent_back1(T, S, M, dM, o, p, xq, wq, st, s);
        if (st) st->n_stages += 1;
      }
    }
    read_stage_results(S, 0, s);
  }
  if (st) st->kernel_launches += g_launches - l0;
}

// left transfer with accumulation: out (+)= sum conj(Ma[a,s,b]) E[a,a'] Mb[a',s,b']
void transfer_left_acc(const double2* E, const double2* Ma, const double2* Mb, int Aa, int Ab, int d, int Ba, int Bb,
                       double2* X, double2* out, bool acc, cudaStream_t s) {
  run1(gemm(Aa, d * Bb, Ab, E, Ab, 1, 0, Mb, (int64_t)d * Bb, 1, X, (int64_t)d * Bb), s);
  ZGemmDesc g = gemm(Ba, Bb, Aa * d, Ma, 1, Ba, 1, X, Bb, 1, out, Bb);
  g.accumulate = acc;
  run1(g, s);
}

// right transfer with accumulation: out[a][a'] (+)= sum conj(Ma[a,s,b]) Mb[a',s,b'] E[b][b']
void transfer_right_acc(const double2* E, const double2* Ma, const double2* Mb, int A, int d, int B, double2* Y,
                        double2* out, bool acc, cudaStream_t s) {
  run1(gemm(A * d, B, B, Mb, B, 1, 0, E, 1, B, Y, B), s);
  ZGemmDesc g = gemm(A, A, d * B, Ma, (int64_t)d * B, 1, 1, Y, 1, (int64_t)d * B, out, A);
  g.accumulate = acc;
  run1(g, s);
}

void measure_tangent_impl(tdvp_mps_s* S, Tan* T, const double2 op[4], double* val_out, double* d_out) {
  cudaStream_t s = 0;
  const int N = S->N, d = S->d, nd = T->nd;
  const int64_t big = (int64_t)S->chi_cap * d * S->chi_cap;
  MeasureBufs mb;
  mb.Mj = dalloc<double2>(big);
  mb.X = dalloc<double2>(big);
  mb.Y = dalloc<double2>(big);
  mb.rho = dalloc<double2>((size_t)16 * N * (1 + nd));
  std::vector<double2*> own;
  auto take = [&](int64_t n) {
    own.push_back(dalloc<double2>((size_t)std::max<int64_t>(n, 1)));
    return own.back();
  };
  struct Guard {
    std::vector<double2*>& v;
    ~Guard() {
      for (auto p : v) dfree(p);
    }
  } guard{own};
  std::vector<double2*> dMj(nd), dEL[TDVP_MAX_DIR], dER[TDVP_MAX_DIR];
  for (int q = 0; q < nd; ++q) dMj[q] = take(big);
  double2* X2 = take(big);
  mb.EL.resize(N + 1);
  mb.ER.resize(N);
  for (int j = 0; j <= N; ++j) {
    const int c = j == 0 ? 1 : S->chiR(j - 1);
    mb.EL[j] = dalloc<double2>((size_t)c * c);
    for (int q = 0; q < nd; ++q) dEL[q].push_back(take((int64_t)c * c));
  }
  for (int j = 0; j < N; ++j) {
    const int c = S->chiR(j);
    mb.ER[j] = dalloc<double2>((size_t)c * c);
    for (int q = 0; q < nd; ++q) dER[q].push_back(take((int64_t)c * c));
  }
  const double2 one = make_double2(1, 0);
  CUDA_TRY(cudaMemcpy(mb.EL[0], &one, sizeof(double2), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(mb.ER[N - 1], &one, sizeof(double2), cudaMemcpyHostToDevice));
  for (int q = 0; q < nd; ++q) {
    CUDA_TRY(cudaMemset(dEL[q][0], 0, sizeof(double2)));
    CUDA_TRY(cudaMemset(dER[q][N - 1], 0, sizeof(double2)));
  }
  // M_j = Psi_j V_j and dM_j = dPsi_j V_j + Psi_j dV_j (the last site: Psi_N, dPsi_N)
  auto site_mats = [&](int j) {
    site_matrix(S, j, mb.Mj, s);
    const int A = S->chiL(j), B = S->chiR(j);
    for (int q = 0; q < nd; ++q) {
      if (j == N - 1) {
        CUDA_TRY(cudaMemcpyAsync(dMj[q], T->dPsi[q][j], sizeof(double2) * A * d * B, cudaMemcpyDeviceToDevice, s));
      } else {
        ScaleBatch sb{};
        sb.n = 1;
        sb.d[0] = ScaleDesc{T->dPsi[q][j], dMj[q], S->V[j], A, d, B, 0, S->Psi[j], T->dV[q][j]};
        launch_scale_bond(sb, s);
      }
    }
  };
  for (int j = 0; j < N; ++j) {
    site_mats(j);
    const int A = S->chiL(j), B = S->chiR(j);
    transfer_left_acc(mb.EL[j], mb.Mj, mb.Mj, A, A, d, B, B, mb.X, mb.EL[j + 1], false, s);
    for (int q = 0; q < nd; ++q) {
      transfer_left_acc(dEL[q][j], mb.Mj, mb.Mj, A, A, d, B, B, mb.X, dEL[q][j + 1], false, s);
      transfer_left_acc(mb.EL[j], mb.Mj, dMj[q], A, A, d, B, B, mb.X, dEL[q][j + 1], true, s);
    }
  }
  for (int j = N - 1; j >= 1; --j) {
    site_mats(j);
    const int A = S->chiL(j), B = S->chiR(j);
    transfer_right_acc(mb.ER[j], mb.Mj, mb.Mj, A, d, B, mb.Y, mb.ER[j - 1], false, s);
    for (int q = 0; q < nd; ++q) {
      transfer_right_acc(dER[q][j], mb.Mj, mb.Mj, A, d, B, mb.Y, dER[q][j - 1], false, s);
      transfer_right_acc(mb.ER[j], mb.Mj, dMj[q], A, d, B, mb.Y, dER[q][j - 1], true, s);
    }
  }
  for (int j = 0; j < N; ++j) {
    site_mats(j);
    const int A = S->chiL(j), B = S->chiR(j);
    // X2 = EL M, Y = X2 ER: <psi| (|s><s'| at j) |psi>
    run1(gemm(A, d * B, A, mb.EL[j], A, 1, 0, mb.Mj, (int64_t)d * B, 1, X2, (int64_t)d * B), s);
    run1(gemm(A * d, B, B, X2, B, 1, 0, mb.ER[j], 1, B, mb.Y, B), s);
    rho_kernel<<<d * d, 256, 0, s>>>(mb.Mj, mb.Y, A, d, B, mb.rho + (size_t)16 * j);
    LAUNCH_CHECK();
    for (int q = 0; q < nd; ++q) {
      // X = dEL M + EL dM; Y = X ER + X2 dER: <psi| (|s><s'| at j) |dpsi>
      run1(gemm(A, d * B, A, dEL[q][j], A, 1, 0, mb.Mj, (int64_t)d * B, 1, mb.X, (int64_t)d * B), s);
      ZGemmDesc g = gemm(A, d * B, A, mb.EL[j], A, 1, 0, dMj[q], (int64_t)d * B, 1, mb.X, (int64_t)d * B);
      g.accumulate = 1;
      run1(g, s);
      run1(gemm(A * d, B, B, mb.X, B, 1, 0, mb.ER[j], 1, B, mb.Y, B), s);
      g = gemm(A * d, B, B, X2, B, 1, 0, dER[q][j], 1, B, mb.Y, B);
      g.accumulate = 1;
      run1(g, s);
      rho_kernel<<<d * d, 256, 0, s>>>(mb.Mj, mb.Y, A, d, B, mb.rho + (size_t)16 * (N * (1 + q) + j));
      LAUNCH_CHECK();
    }
  }
  std::vector<double2> rho((size_t)16 * N * (1 + nd));
  CUDA_TRY(cudaMemcpy(rho.data(), mb.rho, sizeof(double2) * rho.size(), cudaMemcpyDeviceToHost));
  double2 nrm;
  CUDA_TRY(cudaMemcpy(&nrm, mb.EL[N], sizeof(double2), cudaMemcpyDeviceToHost));
  if (!(nrm.x > 0)) fail(TDVP_ENUMERIC, "state has zero norm");
  std::vector<double2> dn(nd);
  for (int q = 0; q < nd; ++q) CUDA_TRY(cudaMemcpy(&dn[q], dEL[q][N], sizeof(double2), cudaMemcpyDeviceToHost));
  auto contract = [&](size_t base) {
    double2 v = make_double2(0, 0);
    for (int k = 0; k < d * d; ++k) v = zadd(v, zmul(rho[base + k], op[k]));
    return v;
  };
  for (int j = 0; j < N; ++j) {
    const double val = contract((size_t)16 * j).x / nrm.x;
    if (val_out) val_out[j] = val;
    for (int q = 0; q < nd; ++q) {
      const double2 od = contract((size_t)16 * (N * (1 + q) + j));
      d_out[(size_t)q * N + j] = 2.0 * od.x / nrm.x - val * 2.0 * dn[q].x / nrm.x;
    }
  }
}

void pauli(int obs, double2 op[4]) {
  const double2 Z = make_double2(0, 0), One = make_double2(1, 0);
  if (obs == TDVP_OBS_SZ) {
    op[0] = One; op[1] = Z; op[2] = Z; op[3] = make_double2(-1, 0);
  } else if (obs == TDVP_OBS_SX) {
    op[0] = Z; op[1] = One; op[2] = One; op[3] = Z;
  } else if (obs == TDVP_OBS_SY) {
    op[0] = Z; op[1] = make_double2(0, -1); op[2] = make_double2(0, 1); op[3] = Z;
  } else {
    fail(TDVP_EINVAL, "unknown observable");
  }
}

}  // namespace

extern "C" {

int tdvp_build_mpo_derivative(tdvp_mpo mpo, int param, tdvp_mpo* out) {
  return ok_or_code([&] {
    if (!mpo || !out) fail(TDVP_EINVAL, "NULL argument");
    if (mpo->base_id) fail(TDVP_EINVAL, "already a derivative MPO");
    if (param != TDVP_PARAM_H && param != TDVP_PARAM_J) fail(TDVP_EINVAL, "unknown parameter");
    require_device();
    auto D = std::make_unique<tdvp_mpo_s>();
    D->kind = mpo->kind;
    D->N = mpo->N;
    D->m = mpo->m;
    D->d = mpo->d;
    D->n_exp = mpo->n_exp;
    D->alpha = mpo->alpha;
    D->x = mpo->x;
    D->lam = mpo->lam;
    // W is affine in (J, h): its derivative is W at (J, h) = (1, 0) or (0, 1)
    // minus W at (0, 0) -- the coupling blocks W[c][0] or the field block W[m-1][0]
    tdvp_mpo_s a, b;
    a.kind = b.kind = mpo->kind;
    a.m = b.m = mpo->m;
    a.d = b.d = mpo->d;
    a.n_exp = b.n_exp = mpo->n_exp;
    a.x = b.x = mpo->x;
    a.lam = b.lam = mpo->lam;
    a.J = param == TDVP_PARAM_J ? 1.0 : 0.0;
    a.h = param == TDVP_PARAM_H ? 1.0 : 0.0;
    b.J = b.h = 0.0;
    build_site_W(&a);
    build_site_W(&b);
    D->W.resize(a.W.size());
    for (size_t i = 0; i < a.W.size(); ++i) D->W[i] = make_double2(a.W[i].x - b.W[i].x, a.W[i].y - b.W[i].y);
    D->J = a.J;
    D->h = a.h;
    // d(W W) = dW W + W dW
    auto t1 = two_site_mpo(D->W, mpo->W, D->m, D->d);
    auto t2 = two_site_mpo(mpo->W, D->W, D->m, D->d);
    D->W12.resize(t1.size());
    for (size_t i = 0; i < t1.size(); ++i) D->W12[i] = zadd(t1[i], t2[i]);
    D->w1.build(D->W, D->m, D->d, false);
    D->w1t.build(D->W, D->m, D->d, true);
    D->w2.build(D->W12, D->m, D->d * D->d, false);
    D->base_id = mpo->id;
    D->param = param;
    {
      std::lock_guard<std::mutex> g(g_id_mutex);
      D->id = g_next_id++;
    }
    *out = D.release();
  });
}

int tdvp_tangent_create(tdvp_mps mps, int n_dir, tdvp_tangent* out) {
  return ok_or_code([&] {
    if (!mps || !out) fail(TDVP_EINVAL, "NULL argument");
    if (n_dir < 1 || n_dir > TDVP_MAX_DIR) fail(TDVP_EINVAL, "n_dir must be in [1, TDVP_MAX_DIR]");
    require_device();
    auto T = std::make_unique<tdvp_tangent_s>();
    T->S = mps;
    T->nd = n_dir;
    T->N = mps->N;
    T->d = mps->d;
    T->chi_cap = mps->chi_cap;
    T->vec = (int64_t)mps->chi_cap * mps->chi_cap * mps->d * mps->d;
    for (int q = 0; q < n_dir; ++q) {
      for (int j = 0; j < mps->N; ++j) T->dPsi[q].push_back(dzeros((int64_t)mps->capL(j) * mps->d * mps->capR(j)));
      for (int j = 0; j + 1 < mps->N; ++j) {
        double* v = dalloc<double>((size_t)mps->cap[j]);
        CUDA_TRY(cudaMemset(v, 0, sizeof(double) * mps->cap[j]));
        T->dV[q].push_back(v);
      }
    }
    *out = T.release();
  });
}

void tdvp_free_tangent(tdvp_tangent tan) { delete tan; }

int tdvp_step_tangent(tdvp_mps mps, tdvp_mpo mpo, tdvp_tangent tan, const tdvp_mpo* dmpo,
                      const tdvp_step_params* params, int n_quad, int n_steps, tdvp_step_stats* stats,
                      void* stream) {
  return ok_or_code([&] {
    if (!mps || !mpo || !tan) fail(TDVP_EINVAL, "NULL handle");
    if (n_steps < 0) fail(TDVP_EINVAL, "n_steps < 0");
    step_tangent_impl(mps, mpo, tan, dmpo, params, n_quad, n_steps, stats, (cudaStream_t)stream);
  });
}

int tdvp_measure_tangent(tdvp_mps mps, tdvp_tangent tan, int obs, double* value_out, double* d_out) {
  return ok_or_code([&] {
    if (!mps || !tan || !d_out) fail(TDVP_EINVAL, "NULL argument");
    if (tan->S != mps) fail(TDVP_EINVAL, "tangent belongs to another MPS");
    if (mps->d != 2) fail(TDVP_EINVAL, "Pauli observables need d = 2");
    double2 op[4];
    pauli(obs, op);
    CUDA_TRY(cudaDeviceSynchronize());
    measure_tangent_impl(mps, tan, op, value_out, d_out);
  });
}

int tdvp_gauss_legendre(int n, double* x_out, double* w_out) {
  return ok_or_code([&] {
    if (n < 1 || n > 64 || !x_out || !w_out) fail(TDVP_EINVAL, "need 1 <= n <= 64 and outputs");
    std::vector<double> x, w;
    gauss_legendre01(n, x, w);
    std::copy(x.begin(), x.end(), x_out);
    std::copy(w.begin(), w.end(), w_out);
  });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// One-site operators and mixed expectations (the dynamical correlation
// function of Sec. IV: C(r - k, t) = e^{-i E0 t} <psi0| sz_r |psi(t)>,
// |psi(0)> = sz_k |psi0>)
// ---------------------------------------------------------------------------
namespace {

struct SiteOp {
  double2 o[16];  // [s_out][s_in], d <= 4
};

// Psi[a, s, b] <- sum_t op[s][t] Psi[a, t, b], in place (one thread per (a, b))
__global__ void site_op_kernel(double2* Psi, int A, int d, int B, const SiteOp op) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)A * B;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(i / B), b = (int)(i % B);
    double2 in[4], out[4];
    for (int t = 0; t < d; ++t) in[t] = Psi[((int64_t)a * d + t) * B + b];
    for (int s = 0; s < d; ++s) {
      double2 acc = make_double2(0, 0);
      for (int t = 0; t < d; ++t) acc = zadd(acc, zmul(op.o[s * d + t], in[t]));
      out[s] = acc;
    }
    for (int s = 0; s < d; ++s) Psi[((int64_t)a * d + s) * B + b] = out[s];
  }
}

// right transfer with bra a and ket b: out[x][y] = sum conj(Ma[x,s,p]) Mb[y,s,q] E[p][q]
void transfer_right_mixed(const double2* E, const double2* Ma, const double2* Mb, int Aa, int Ab, int d, int Ba,
                          int Bb, double2* Y, double2* out, cudaStream_t s) {
  run1(gemm(Ab * d, Ba, Bb, Mb, Bb, 1, 0, E, 1, Bb, Y, Ba), s);
  run1(gemm(Aa, Ab, d * Ba, Ma, (int64_t)d * Ba, 1, 1, Y, 1, (int64_t)d * Ba, out, Ab), s);
}

}  // namespace

extern "C" {

int tdvp_mps_copy(tdvp_mps src, tdvp_mps* out) {
  return ok_or_code([&] {
    if (!src || !out) fail(TDVP_EINVAL, "NULL argument");
    CUDA_TRY(cudaDeviceSynchronize());
    tdvp_mps_s* S = new_mps(src->N, src->d, src->chi_cap);
    std::unique_ptr<tdvp_mps_s, void (*)(tdvp_mps_s*)> guard(S, free_mps);
    S->dims = src->dims;
    for (int j = 0; j < S->N; ++j)
      CUDA_TRY(cudaMemcpy(S->Psi[j], src->Psi[j], sizeof(double2) * src->chiL(j) * src->d * src->chiR(j),
                          cudaMemcpyDeviceToDevice));
    for (int j = 0; j + 1 < S->N; ++j)
      CUDA_TRY(cudaMemcpy(S->V[j], src->V[j], sizeof(double) * src->dims[j], cudaMemcpyDeviceToDevice));
    *out = guard.release();
  });
}

int tdvp_apply_site_op(tdvp_mps mps, int j, const double* op) {
  return ok_or_code([&] {
    if (!mps || !op) fail(TDVP_EINVAL, "NULL argument");
    if (j < 0 || j >= mps->N) fail(TDVP_EINVAL, "site out of range");
    SiteOp o{};
    std::memcpy(o.o, op, sizeof(double2) * mps->d * mps->d);
    CUDA_TRY(cudaDeviceSynchronize());
    const int A = mps->chiL(j), B = mps->chiR(j);
    const int grid = (int)std::min<int64_t>(cdiv64((int64_t)A * B, 256), 152 * 8);
    site_op_kernel<<<std::max(grid, 1), 256>>>(mps->Psi[j], A, mps->d, B, o);
    LAUNCH_CHECK();
    ++g_launches;
    CUDA_TRY(cudaDeviceSynchronize());
    mps->env_id = 0;  // cached environments belong to the old state
  });
}

int tdvp_expect_mixed(tdvp_mps a, tdvp_mps b, int obs, double* out) {
  return ok_or_code([&] {
    if (!a || !b || !out) fail(TDVP_EINVAL, "NULL argument");
    if (a->N != b->N || a->d != b->d) fail(TDVP_EINVAL, "states of different shape");
    if (a->d != 2) fail(TDVP_EINVAL, "Pauli observables need d = 2");
    double2 op[4];
    pauli(obs, op);
    CUDA_TRY(cudaDeviceSynchronize());
    cudaStream_t s = 0;
    const int N = a->N, d = a->d;
    const int64_t cc = std::max(a->chi_cap, b->chi_cap);
    const int64_t big = cc * d * cc;
    MeasureBufs mb;
    mb.Mj = dalloc<double2>(big);
    mb.X = dalloc<double2>(big);
    mb.Y = dalloc<double2>(big);
    mb.rho = dalloc<double2>((size_t)16 * N);
    double2* Mb = dalloc<double2>(big);
    std::unique_ptr<double2, void (*)(double2*)> gM(Mb, [](double2* p) { dfree(p); });
    mb.EL.resize(N + 1);
    mb.ER.resize(N);
    for (int j = 0; j <= N; ++j) {
      const int64_t ca = j == 0 ? 1 : a->chiR(j - 1), cb = j == 0 ? 1 : b->chiR(j - 1);
      mb.EL[j] = dalloc<double2>((size_t)ca * cb);
    }
    for (int j = 0; j < N; ++j) mb.ER[j] = dalloc<double2>((size_t)a->chiR(j) * b->chiR(j));
    const double2 one = make_double2(1, 0);
    CUDA_TRY(cudaMemcpy(mb.EL[0], &one, sizeof(double2), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(mb.ER[N - 1], &one, sizeof(double2), cudaMemcpyHostToDevice));
    for (int j = 0; j < N; ++j) {
      site_matrix(a, j, mb.Mj, s);
      site_matrix(b, j, Mb, s);
      transfer_left(mb.EL[j], mb.Mj, Mb, a->chiL(j), b->chiL(j), d, a->chiR(j), b->chiR(j), mb.X, mb.EL[j + 1], s);
    }
    for (int j = N - 1; j >= 1; --j) {
      site_matrix(a, j, mb.Mj, s);
      site_matrix(b, j, Mb, s);
      transfer_right_mixed(mb.ER[j], mb.Mj, Mb, a->chiL(j), b->chiL(j), d, a->chiR(j), b->chiR(j), mb.Y,
                           mb.ER[j - 1], s);
    }
    for (int j = 0; j < N; ++j) {
      site_matrix(a, j, mb.Mj, s);
      site_matrix(b, j, Mb, s);
      const int Aa = a->chiL(j), Ab = b->chiL(j), Ba = a->chiR(j), Bb = b->chiR(j);
      // X = EL Mb (Aa x d Bb), Y[(x s)][p] = sum_q X[(x s)][q] ER[p][q]
      run1(gemm(Aa, d * Bb, Ab, mb.EL[j], Ab, 1, 0, Mb, (int64_t)d * Bb, 1, mb.X, (int64_t)d * Bb), s);
      run1(gemm(Aa * d, Ba, Bb, mb.X, Bb, 1, 0, mb.ER[j], 1, Bb, mb.Y, Ba), s);
      rho_kernel<<<d * d, 256, 0, s>>>(mb.Mj, mb.Y, Aa, d, Ba, mb.rho + (size_t)16 * j);
      LAUNCH_CHECK();
    }
    std::vector<double2> rho((size_t)16 * N);
    CUDA_TRY(cudaMemcpy(rho.data(), mb.rho, sizeof(double2) * rho.size(), cudaMemcpyDeviceToHost));
    for (int j = 0; j < N; ++j) {
      double2 v = make_double2(0, 0);
      for (int k = 0; k < d * d; ++k) v = zadd(v, zmul(rho[(size_t)16 * j + k], op[k]));
      out[2 * j] = v.x;
      out[2 * j + 1] = v.y;
    }
  });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// One-site TDVP (Eq. proj1site: site terms forward, bond terms backward, fixed
// bond dimension) and the hybrid two-site -> one-site scheme of the paper's
// discussion, serial sweep, FP64
// ---------------------------------------------------------------------------
namespace {

void ensure_w0(tdvp_mpo_s* M) {
  if (M->w0.m == M->m && M->w0.col_ptr) return;
  std::vector<double2> I((size_t)M->m * M->m, make_double2(0, 0));
  for (int w = 0; w < M->m; ++w) I[(size_t)w * M->m + w] = make_double2(1, 0);
  M->w0.build(I, M->m, 1, false);
}

void ensure_w1s(tdvp_mps_s* S) {
  if (S->w1s[0]) return;
  const int64_t v = (int64_t)S->chi_cap * S->chi_cap * S->d * S->d;
  for (auto& p : S->w1s) p = dalloc<double2>((size_t)v);
  for (auto& p : S->w1v) p = dalloc<double>((size_t)S->chi_cap * S->d);
}

void zgemm1(int Mm, int Nn, int Kk, const double2* A, int64_t lda, const double* kscale, const double2* B,
            int64_t ldb, double2* C, int64_t ldc, cudaStream_t s) {
  ZGemmBatch g{};
  g.n = 1;
  ZGemmDesc& z = g.d[0];
  z = ZGemmDesc{};
  z.M = Mm;
  z.N = Nn;
  z.K = Kk;
  z.A = A;
  z.a_rs = lda;
  z.a_cs = 1;
  z.kscale = kscale;
  z.B = B;
  z.b_rs = ldb;
  z.b_cs = 1;
  z.C = C;
  z.c_rs = ldc;
  z.c_cs = 1;
  launch_zgemm(g, s, "one_site_zgemm");
}

void site_forward(tdvp_mps_s* S, tdvp_mpo_s* M, int j, double t, const tdvp_step_params* p, tdvp_step_stats* st,
                  cudaStream_t s) {
  Slot* sl = slot_for(S, 0, M->m, p->krylov_max);
  const int A = S->chiL(j), B = S->chiR(j);
  MvProb P = make_mv(S, M, A, B, S->d, j, j, false, sl, TDVP_FP64);
  expm_batch({P}, {S->Psi[j]}, {S->Psi[j]}, {t}, p->krylov_max, p->krylov_tol, Ctx{s, S->d_status, TDVP_FP64});
  if (st) {
    st->heff_flops += p->krylov_max * heff_flops(A, B, S->d, M->m, M->w1.nnz);
    st->n_back1 += 1;
  }
}

// zero-site effective Hamiltonian on the bond matrix C [A][B]: L = env [A][m][A], R = env [B][m][B]
void bond_expm(tdvp_mps_s* S, tdvp_mpo_s* M, const double2* L, const double2* R, int A, int B, double2* C,
               double t, const tdvp_step_params* p, cudaStream_t s) {
  Slot* sl = slot_for(S, 0, M->m, p->krylov_max);
  MvProb P{};
  P.A = A;
  P.B = B;
  P.D = 1;
  P.m = M->m;
  P.L = L;
  P.R = R;
  P.W = M->w0.op();
  P.slot = sl;
  expm_batch({P}, {C}, {C}, {t}, p->krylov_max, p->krylov_tol, Ctx{s, S->d_status, TDVP_FP64});
}

void left_env(tdvp_mps_s* S, tdvp_mpo_s* M, int j, cudaStream_t s) {  // beta_{j+1} from Psi_j V_j
  Slot* sl = slot_for(S, 0, M->m, 1);
  ScaleBatch sb{};
  sb.n = 1;
  sb.d[0] = ScaleDesc{S->Psi[j], sl->Amat, S->V[j], S->chiL(j), S->d, S->chiR(j), 0, nullptr, nullptr};
  launch_scale_bond(sb, s);
  env_batch(0, {EnvProb{S->chiL(j), S->chiR(j), S->d, M->m, S->beta[j], sl->Amat, S->beta[j + 1], M->w1.op(), sl}},
            Ctx{s, S->d_status, TDVP_FP64});
}

void right_env(tdvp_mps_s* S, tdvp_mpo_s* M, int j, cudaStream_t s) {  // gamma_j from V_j Psi_{j+1}
  Slot* sl = slot_for(S, 0, M->m, 1);
  ScaleBatch sb{};
  sb.n = 1;
  sb.d[0] = ScaleDesc{S->Psi[j + 1], sl->Bmat, S->V[j], S->chiL(j + 1), S->d, S->chiR(j + 1), 1, nullptr, nullptr};
  launch_scale_bond(sb, s);
  env_batch(1, {EnvProb{S->chiL(j + 1), S->chiR(j + 1), S->d, M->m, S->gamma[j + 1], sl->Bmat, S->gamma[j],
                        M->w1t.op(), sl}},
            Ctx{s, S->d_status, TDVP_FP64});
}

// split site j as (chi_{j-1} d) x chi_j, evolve the bond matrix of bond j backward
// by tau, move it into site j + 1 (the inverse canonical gauge restored on bond j)
void bond_backward_right(tdvp_mps_s* S, tdvp_mpo_s* M, int j, double tau, const tdvp_step_params* p,
                         cudaStream_t s) {
  const int A = S->chiL(j), d = S->d, b = S->dims[j], Bn = S->chiR(j + 1);
  Slot* sl = slot_for(S, 0, M->m, p->krylov_max);
  double2 *P1 = S->w1s[0], *R1 = S->w1s[1], *P2 = S->w1s[2], *Tm = S->w1s[3];
  double *V1 = S->w1v[0], *V2 = S->w1v[1];
  const int k = device_split(S, sl, S->Psi[j], A * d, b, std::min(A * d, b), 0.0, 0.0, P1, V1, R1, nullptr,
                             nullptr, s);
  // beta_{j+1} from A_j = U = P1 V1
  ScaleBatch sb{};
  sb.n = 1;
  sb.d[0] = ScaleDesc{P1, sl->Amat, V1, A, d, k, 0, nullptr, nullptr};
  launch_scale_bond(sb, s);
  env_batch(0, {EnvProb{A, k, d, M->m, S->beta[j], sl->Amat, S->beta[j + 1], M->w1.op(), sl}},
            Ctx{s, S->d_status, TDVP_FP64});
  bond_expm(S, M, S->beta[j + 1], S->gamma[j], k, b, R1, -tau, p, s);
  // R1 (k x b) -> P2 = u s, V2 = 1/s, R2 = s v^H (into P1's successor buffer Tm)
  double2* R2 = Tm;
  const int k2 = device_split(S, sl, R1, k, b, std::min(k, b), 0.0, 0.0, P2, V2, R2, nullptr, nullptr, s);
  // Psi_{j+1} <- R2 V_j(old) Psi_{j+1}: staged through R1 (free now)
  zgemm1(k2, d * Bn, b, R2, b, S->V[j], S->Psi[j + 1], (int64_t)d * Bn, R1, (int64_t)d * Bn, s);
  CUDA_TRY(cudaMemcpyAsync(S->Psi[j + 1], R1, sizeof(double2) * k2 * d * Bn, cudaMemcpyDeviceToDevice, s));
  // Psi_j <- U u s = P1 V1 P2
  zgemm1(A * d, k2, k, P1, k, V1, P2, k2, S->Psi[j], k2, s);
  CUDA_TRY(cudaMemcpyAsync(S->V[j], V2, sizeof(double) * k2, cudaMemcpyDeviceToDevice, s));
  S->dims[j] = k2;
  left_env(S, M, j, s);
}

// split site j as chi_{j-1} x (d chi_j), evolve the bond matrix of bond j - 1
// backward by tau, move it into site j - 1
void bond_backward_left(tdvp_mps_s* S, tdvp_mpo_s* M, int j, double tau, const tdvp_step_params* p,
                        cudaStream_t s) {
  const int a = S->dims[j - 1], d = S->d, Bn = S->chiR(j), Al = S->chiL(j - 1);
  Slot* sl = slot_for(S, 0, M->m, p->krylov_max);
  double2 *P1 = S->w1s[0], *R1 = S->w1s[1], *P2 = S->w1s[2], *R2 = S->w1s[3];
  double *V1 = S->w1v[0], *V2 = S->w1v[1];
  const int k = device_split(S, sl, S->Psi[j], a, d * Bn, std::min(a, d * Bn), 0.0, 0.0, P1, V1, R1, nullptr,
                             nullptr, s);
  // gamma_{j-1} from B_j = V1 R1
  ScaleBatch sb{};
  sb.n = 1;
  sb.d[0] = ScaleDesc{R1, sl->Bmat, V1, k, d, Bn, 1, nullptr, nullptr};
  launch_scale_bond(sb, s);
  env_batch(1, {EnvProb{k, Bn, d, M->m, S->gamma[j], sl->Bmat, S->gamma[j - 1], M->w1t.op(), sl}},
            Ctx{s, S->d_status, TDVP_FP64});
  bond_expm(S, M, S->beta[j], S->gamma[j - 1], a, k, P1, -tau, p, s);
  // P1 (a x k) -> P2 = u s, V2 = 1/s, R2 = s v^H
  const int k2 = device_split(S, sl, P1, a, k, std::min(a, k), 0.0, 0.0, P2, V2, R2, nullptr, nullptr, s);
  // Psi_j <- R2 V1 R1 (k2 x d Bn)
  zgemm1(k2, d * Bn, k, R2, k, V1, R1, (int64_t)d * Bn, S->Psi[j], (int64_t)d * Bn, s);
  // Psi_{j-1} <- Psi_{j-1} V_{j-1}(old) P2, staged through R1 (free now)
  zgemm1(Al * d, k2, a, S->Psi[j - 1], a, S->V[j - 1], P2, k2, R1, k2, s);
  CUDA_TRY(cudaMemcpyAsync(S->Psi[j - 1], R1, sizeof(double2) * Al * d * k2, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(S->V[j - 1], V2, sizeof(double) * k2, cudaMemcpyDeviceToDevice, s));
  S->dims[j - 1] = k2;
  right_env(S, M, j - 1, s);
}

void step1_seg_impl(tdvp_mps_s* S, tdvp_mpo_s* M, const tdvp_step_params* p, int n_steps, tdvp_step_stats* st,
                    cudaStream_t s);

void step1_impl(tdvp_mps_s* S, tdvp_mpo_s* M, const tdvp_step_params* p, int n_steps, tdvp_step_stats* st,
                cudaStream_t s) {
  check_params(S, M, p);
  if (p->precision != TDVP_FP64) fail(TDVP_EINVAL, "one-site sweeps are FP64 only");
  ensure_small_buffers(S);
  ensure_w0(M);
  ensure_w1s(S);
  const int64_t l0 = g_launches;
  if (S->env_id != M->id) build_all_envs(S, M, s);
  const int N = S->N;
  if (p->n_seg > 1 && p->seg_len) {
    step1_seg_impl(S, M, p, n_steps, st, s);
    S->beta32_ok.assign(N, 0);
    S->gamma32_ok.assign(N, 0);
    if (st) st->kernel_launches += g_launches - l0;
    return;
  }
  const double tau = 0.5 * p->dt;
  for (int step = 0; step < n_steps; ++step) {
    right_env(S, M, 0, s);  // gamma_0 of the current state (a two-site half leaves it behind)
    for (int j = 0; j + 1 < N; ++j) {
      site_forward(S, M, j, tau, p, st, s);
      bond_backward_right(S, M, j, tau, p, s);
    }
    site_forward(S, M, N - 1, 2 * tau, p, st, s);
    for (int j = N - 1; j >= 1; --j) {
      bond_backward_left(S, M, j, tau, p, s);
      site_forward(S, M, j - 1, tau, p, st, s);
    }
    read_stage_results(S, 0, s);
    if (st) st->n_stages += 4 * N - 2;
  }
  // tensor-core operand forms of the environments are stale now
  S->beta32_ok.assign(N, 0);
  S->gamma32_ok.assign(N, 0);
  if (st) st->kernel_launches += g_launches - l0;
}

// one-site forward steps of several sites at once (one batched Lanczos)
void site_forward_batch(tdvp_mps_s* S, tdvp_mpo_s* M, const std::vector<std::pair<int, double>>& js,
                        const tdvp_step_params* p, tdvp_step_stats* st, cudaStream_t s) {
  if (js.empty()) return;
  std::vector<MvProb> P;
  std::vector<const double2*> x;
  std::vector<double2*> y;
  std::vector<double> t;
  for (size_t i = 0; i < js.size(); ++i) {
    const int j = js[i].first, A = S->chiL(j), B = S->chiR(j);
    Slot* sl = slot_for(S, (int)i, M->m, p->krylov_max);
    P.push_back(make_mv(S, M, A, B, S->d, j, j, false, sl, TDVP_FP64));
    x.push_back(S->Psi[j]);
    y.push_back(S->Psi[j]);
    t.push_back(js[i].second);
    if (st) {
      st->heff_flops += p->krylov_max * heff_flops(A, B, S->d, M->m, M->w1.nnz);
      st->n_back1 += 1;
    }
  }
  expm_batch(P, x, y, t, p->krylov_max, p->krylov_tol, Ctx{s, S->d_status, TDVP_FP64});
}

// Segmented one-site steps (build_half1): per stage the site steps run as one
// batch, the boundary pairs as one batched two-site update at each bond's
// current dimension, the bond steps one after another. Stages run in order;
// the ops of a stage touch disjoint tensors, so their order does not matter.
// One SVD split per item (rows[i] x cols[i] of theta[i], every value kept but
// the numerical zeros), all problems in one batched launch sequence, each in
// its own slot; returns the kept ranks.
std::vector<int> device_split_batch(tdvp_mps_s* S, const std::vector<Slot*>& sl,
                                    const std::vector<const double2*>& theta, const std::vector<int>& rows,
                                    const std::vector<int>& cols, const std::vector<double2*>& PsiL,
                                    const std::vector<double*>& V, const std::vector<double2*>& PsiR,
                                    cudaStream_t s) {
  const int n = (int)theta.size();
  SvdBatch sb{};
  sb.n = n;
  sb.status = S->d_status;
  sb.sync = sl[0]->sync;
  for (int i = 0; i < n; ++i) {
    SvdDesc& q = sb.d[i];
    q = SvdDesc{};
    q.theta = theta[i];
    q.rows = rows[i];
    q.cols = cols[i];
    q.X = sl[i]->svdX;
    q.Acc = sl[i]->svdAcc;
    q.X32 = sl[i]->svdX32;
    q.Acc32 = sl[i]->svdAcc32;
    q.P = sl[i]->svdP;
    q.T = sl[i]->svdT;
    q.maxr = sl[i]->maxr;
    q.sig = sl[i]->sig;
    q.perm = sl[i]->perm;
    q.rotated = sl[i]->rot;
    q.conv = sl[i]->conv;
    q.chi_max = std::min(rows[i], cols[i]);
    q.w_max = 0.0;
    q.eps = 0.0;
    q.chi = S->d_chi + i;
    q.w = S->d_w + i;
    q.PsiL = PsiL[i];
    q.V = V[i];
    q.PsiR = PsiR[i];
  }
  svd_split(sb, S->d_flag, S->h_pinned, s);
  read_stage_results(S, n, s);
  std::vector<int> k(n);
  for (int i = 0; i < n; ++i) k[i] = S->h_pinned[2 + i];
  return k;
}

struct BondOp {
  int kind;  // 1: bond j, the centre moving right (site j split, carried into j + 1);
             // 2: bond j - 1, the centre moving left (site j split, carried into j - 1)
  int j;
  double t;  // evolution time of the bond matrix (negative: backward)
};

// The bond steps of one stage (bond_backward_right / _left), every phase
// batched over the ops: split the site, build the environment of its
// isometry, evolve the bond matrices with the zero-site term, split them,
// carry them into the neighbour sites, rebuild the environments. The ops of a
// stage belong to different segments and touch disjoint tensors.
void bond_steps_batch(tdvp_mps_s* S, tdvp_mpo_s* M, const std::vector<BondOp>& ops, const tdvp_step_params* p,
                      cudaStream_t s) {
  const int n = (int)ops.size();
  if (n == 0) return;
  if (n > MAXB) fail(TDVP_EINVAL, "too many bond steps in a stage");
  const int d = S->d, m = M->m;
  const Ctx c64{s, S->d_status, TDVP_FP64};
  std::vector<Slot*> sl(n);
  for (int i = 0; i < n; ++i) sl[i] = slot_for(S, i, m, p->krylov_max);
  std::vector<const double2*> th(n);
  std::vector<int> rows(n), cols(n), A(n), B(n), a(n);
  std::vector<double2*> P1(n), R1(n), P2(n), R2(n);
  std::vector<double*> V1(n), V2(n);
  for (int i = 0; i < n; ++i) {
    const int j = ops[i].j;
    P1[i] = sl[i]->theta;
    R1[i] = sl[i]->theta2;
    P2[i] = sl[i]->T1;
    R2[i] = sl[i]->T2;
    V1[i] = sl[i]->bv;
    V2[i] = sl[i]->bv + sl[i]->cap_svd + 1;
    th[i] = S->Psi[j];
    if (ops[i].kind == 1) {
      A[i] = S->chiL(j);
      a[i] = S->dims[j];          // bond j
      B[i] = S->chiR(j + 1);
      rows[i] = A[i] * d;
      cols[i] = a[i];
    } else {
      A[i] = S->chiL(j - 1);
      a[i] = S->dims[j - 1];      // bond j - 1
      B[i] = S->chiR(j);
      rows[i] = a[i];
      cols[i] = d * B[i];
    }
  }
  // 1. split the site: P1 = U Lambda, V1 = 1 / Lambda, R1 = Lambda V^H
  const std::vector<int> k = device_split_batch(S, sl, th, rows, cols, P1, V1, R1, s);
  // 2. environment of the isometry: beta_{j+1} from U = P1 V1, or gamma_{j-1} from V1 R1
  {
    ScaleBatch scl{}, scr{};
    std::vector<EnvProb> le, re;
    for (int i = 0; i < n; ++i) {
      const int j = ops[i].j;
      if (ops[i].kind == 1) {
        scl.d[scl.n++] = ScaleDesc{P1[i], sl[i]->Amat, V1[i], A[i], d, k[i], 0, nullptr, nullptr};
        le.push_back(EnvProb{A[i], k[i], d, m, S->beta[j], sl[i]->Amat, S->beta[j + 1], M->w1.op(), sl[i]});
      } else {
        scr.d[scr.n++] = ScaleDesc{R1[i], sl[i]->Bmat, V1[i], k[i], d, B[i], 1, nullptr, nullptr};
        re.push_back(EnvProb{k[i], B[i], d, m, S->gamma[j], sl[i]->Bmat, S->gamma[j - 1], M->w1t.op(), sl[i]});
      }
    }
    launch_scale_bond(scl, s);
    launch_scale_bond(scr, s);
    env_batch(0, le, c64);
    env_batch(1, re, c64);
  }
  // 3. the bond matrices (R1: k x a, or P1: a x k) evolved by the zero-site term
  {
    std::vector<MvProb> P(n);
    std::vector<const double2*> x(n);
    std::vector<double2*> y(n);
    std::vector<double> t(n);
    for (int i = 0; i < n; ++i) {
      const int j = ops[i].j;
      MvProb& q = P[i];
      q = MvProb{};
      q.D = 1;
      q.m = m;
      q.W = M->w0.op();
      q.slot = sl[i];
      if (ops[i].kind == 1) {
        q.A = k[i];
        q.B = a[i];
        q.L = S->beta[j + 1];
        q.R = S->gamma[j];
        x[i] = y[i] = R1[i];
      } else {
        q.A = a[i];
        q.B = k[i];
        q.L = S->beta[j];
        q.R = S->gamma[j - 1];
        x[i] = y[i] = P1[i];
      }
      t[i] = ops[i].t;
    }
    expm_batch(P, x, y, t, p->krylov_max, p->krylov_tol, c64);
  }
  // 4. split them: P2 = u s, V2 = 1 / s, R2 = s v^H
  std::vector<const double2*> cm(n);
  std::vector<int> r2(n), c2(n);
  for (int i = 0; i < n; ++i) {
    cm[i] = ops[i].kind == 1 ? R1[i] : P1[i];
    r2[i] = ops[i].kind == 1 ? k[i] : a[i];
    c2[i] = ops[i].kind == 1 ? a[i] : k[i];
  }
  const std::vector<int> k2 = device_split_batch(S, sl, cm, r2, c2, P2, V2, R2, s);
  // 5. carry the bond into the neighbour site and rebuild the split site
  //    kind 1: Psi_{j+1} <- R2 V_j(old) Psi_{j+1} (via R1), Psi_j <- P1 V1 P2
  //    kind 2: Psi_j <- R2 V1 R1, Psi_{j-1} <- Psi_{j-1} V_{j-1}(old) P2 (via P1)
  std::vector<ZGemmDesc> gs;
  auto gemm = [](int Mm, int Nn, int Kk, const double2* Am, int64_t lda, const double* ks, const double2* Bm,
                 int64_t ldb, double2* Cm, int64_t ldc) {
    ZGemmDesc z{};
    z.M = Mm;
    z.N = Nn;
    z.K = Kk;
    z.A = Am;
    z.a_rs = lda;
    z.a_cs = 1;
    z.kscale = ks;
    z.B = Bm;
    z.b_rs = ldb;
    z.b_cs = 1;
    z.C = Cm;
    z.c_rs = ldc;
    z.c_cs = 1;
    return z;
  };
  for (int i = 0; i < n; ++i) {
    const int j = ops[i].j;
    if (ops[i].kind == 1) {
      gs.push_back(gemm(k2[i], d * B[i], a[i], R2[i], a[i], S->V[j], S->Psi[j + 1], (int64_t)d * B[i], R1[i],
                        (int64_t)d * B[i]));
      gs.push_back(gemm(A[i] * d, k2[i], k[i], P1[i], k[i], V1[i], P2[i], k2[i], S->Psi[j], k2[i]));
    } else {
      gs.push_back(gemm(k2[i], d * B[i], k[i], R2[i], k[i], V1[i], R1[i], (int64_t)d * B[i], S->Psi[j],
                        (int64_t)d * B[i]));
      gs.push_back(gemm(A[i] * d, k2[i], a[i], S->Psi[j - 1], a[i], S->V[j - 1], P2[i], k2[i], P1[i], k2[i]));
    }
  }
  for (size_t b0 = 0; b0 < gs.size(); b0 += MAXB) {
    ZGemmBatch g{};
    for (size_t q = b0; q < gs.size() && g.n < MAXB; ++q) g.d[g.n++] = gs[q];
    launch_zgemm(g, s, "one_site_zgemm");
  }
  for (int i = 0; i < n; ++i) {
    const int j = ops[i].j;
    if (ops[i].kind == 1) {
      CUDA_TRY(cudaMemcpyAsync(S->Psi[j + 1], R1[i], sizeof(double2) * k2[i] * d * B[i], cudaMemcpyDeviceToDevice, s));
      CUDA_TRY(cudaMemcpyAsync(S->V[j], V2[i], sizeof(double) * k2[i], cudaMemcpyDeviceToDevice, s));
      S->dims[j] = k2[i];
    } else {
      CUDA_TRY(cudaMemcpyAsync(S->Psi[j - 1], P1[i], sizeof(double2) * A[i] * d * k2[i], cudaMemcpyDeviceToDevice,
                               s));
      CUDA_TRY(cudaMemcpyAsync(S->V[j - 1], V2[i], sizeof(double) * k2[i], cudaMemcpyDeviceToDevice, s));
      S->dims[j - 1] = k2[i];
    }
  }
  // 6. environments of the new gauge: beta_{j+1} from Psi_j V_j, or gamma_{j-1} from V_{j-1} Psi_j
  {
    ScaleBatch scl{}, scr{};
    std::vector<EnvProb> le, re;
    for (int i = 0; i < n; ++i) {
      const int j = ops[i].j;
      if (ops[i].kind == 1) {
        scl.d[scl.n++] = ScaleDesc{S->Psi[j], sl[i]->Amat, S->V[j], S->chiL(j), d, S->chiR(j), 0, nullptr, nullptr};
        le.push_back(EnvProb{S->chiL(j), S->chiR(j), d, m, S->beta[j], sl[i]->Amat, S->beta[j + 1], M->w1.op(),
                             sl[i]});
      } else {
        scr.d[scr.n++] = ScaleDesc{S->Psi[j], sl[i]->Bmat, S->V[j - 1], S->chiL(j), d, S->chiR(j), 1, nullptr,
                                   nullptr};
        re.push_back(EnvProb{S->chiL(j), S->chiR(j), d, m, S->gamma[j], sl[i]->Bmat, S->gamma[j - 1], M->w1t.op(),
                             sl[i]});
      }
    }
    launch_scale_bond(scl, s);
    launch_scale_bond(scr, s);
    env_batch(0, le, c64);
    env_batch(1, re, c64);
  }
}

void step1_seg_impl(tdvp_mps_s* S, tdvp_mpo_s* M, const tdvp_step_params* p, int n_steps, tdvp_step_stats* st,
                    cudaStream_t s) {
  const int N = S->N;
  std::vector<int> seg(p->seg_len, p->seg_len + p->n_seg);
  if ((int)seg.size() > MAXB) fail(TDVP_EINVAL, "too many segments");
  std::vector<SchedOp> halves[2];
  build_half1(N, seg, 1, p->merge_turning, halves[0]);
  build_half1(N, seg, 2, p->merge_turning, halves[1]);
  const double tau = 0.5 * p->dt;
  tdvp_step_params pp = *p;  // boundary pairs: no weight cut beyond the relative cutoff
  pp.w_max = 0.0;
  // the chain-end environment the first half reads first, rebuilt at the start
  // of every step (a two-site half that ends moving away from that end leaves
  // it behind): gamma_0 when segment 0 starts at site 0, beta_{N-1} when the
  // last segment starts at site N-1 (segment k sweeps right first iff k and
  // n_seg / 2 have the same parity)
  const int ns = (int)seg.size();
  const bool first_right = (0 % 2) == ((ns / 2) % 2);
  const bool last_right = ((ns - 1) % 2) == ((ns / 2) % 2);
  for (int step = 0; step < n_steps; ++step) {
    if (first_right) right_env(S, M, 0, s);
    if (!last_right) left_env(S, M, N - 2, s);
    for (int h = 0; h < 2; ++h) {
      const auto& ops = halves[h];
      size_t i = 0;
      while (i < ops.size()) {
        const int stage = ops[i].stage;
        std::vector<std::pair<int, double>> sites;
        std::vector<StageOp> pairs;
        std::vector<const SchedOp*> bonds;
        for (; i < ops.size() && ops[i].stage == stage; ++i) {
          const SchedOp& o = ops[i];
          if (o.kind == 0) sites.push_back({o.j, o.tfac * tau});
          else if (o.kind == 3) pairs.push_back(StageOp{o.j, o.tfac, 3, S->dims[o.j]});
          else bonds.push_back(&o);
        }
        site_forward_batch(S, M, sites, p, st, s);
        {
          std::vector<BondOp> bops;
          for (const SchedOp* o : bonds) bops.push_back(BondOp{o->kind, o->j, -o->tfac * tau});
          bond_steps_batch(S, M, bops, p, s);
        }
        if (!pairs.empty()) run_fwd2(S, M, pairs, &pp, st, s);
        if (st) st->n_stages += 1;
      }
    }
    read_stage_results(S, 0, s);
  }
}

bool bonds_saturated(const tdvp_mps_s* S, int chi_max) {
  for (int j = 0; j + 1 < S->N; ++j)
    if (S->dims[j] < std::min(chi_max, S->cap[j])) return false;
  return true;
}

}  // namespace

extern "C" {

int tdvp_step1(tdvp_mps mps, tdvp_mpo mpo, const tdvp_step_params* params, int n_steps, tdvp_step_stats* stats,
               void* stream) {
  return ok_or_code([&] {
    if (!mps || !mpo) fail(TDVP_EINVAL, "NULL handle");
    if (n_steps < 0) fail(TDVP_EINVAL, "n_steps < 0");
    step1_impl(mps, mpo, params, n_steps, stats, (cudaStream_t)stream);
  });
}

int tdvp_step_hybrid(tdvp_mps mps, tdvp_mpo mpo, const tdvp_step_params* params, int n_steps,
                     tdvp_step_stats* stats, void* stream) {
  int n1 = 0;
  const int rc = ok_or_code([&] {
    if (!mps || !mpo || !params) fail(TDVP_EINVAL, "NULL argument");
    if (n_steps < 0) fail(TDVP_EINVAL, "n_steps < 0");
    if (params->precision != TDVP_FP64) fail(TDVP_EINVAL, "the hybrid scheme is FP64 only");
    for (int i = 0; i < n_steps; ++i) {
      if (bonds_saturated(mps, params->chi_max)) {
        step1_impl(mps, mpo, params, 1, stats, (cudaStream_t)stream);
        ++n1;
      } else {
        step_impl(mps, mpo, params, 1, stats, (cudaStream_t)stream);
      }
    }
  });
  return rc == TDVP_OK ? n1 : rc;
}

}  // extern "C"
