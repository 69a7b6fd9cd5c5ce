/*
 * tdvp.h -- C ABI of libtdvp: parallel two-site TDVP for matrix product states
 * with long-range MPOs on one GB300 GPU (sm_103a).
 *
 * Method: P. Secular et al., "Parallel time-dependent variational principle
 * algorithm for matrix product states" (arXiv:1912.06127). Citations below
 * name the paper's sections, equations and figures.
 *
 * Conventions shared by every entry point
 *   - Complex numbers are interleaved (re, im) doubles ("complex128").
 *   - Indices are 0-based: sites 0..N-1, bonds 0..N-2 (bond j joins sites j, j+1).
 *   - Site tensors Psi_j are row-major [chi_{j-1}][d][chi_j] (chi_{-1} = chi_{N-1} = 1).
 *   - Environments are row-major [bra][mpo][ket]; MPO tensors are row-major
 *     W[w_left][w_right][s_out][s_in].
 *   - Every function returns TDVP_OK (0) or a negative TDVP_E* code and never
 *     aborts; tdvp_last_error() returns a thread-local text for the last failure.
 *   - Handles are owned by the library and released with tdvp_free_*().
 *     Host arrays passed in or out are owned by the caller. Device memory of
 *     handles is allocated by the library (cudaMalloc) at creation time and
 *     held until the handle is freed; tdvp_step allocates nothing further
 *     once the handle has stepped once with a given MPO and batch shape.
 *   - `stream` is a cudaStream_t (NULL = default stream). Calls are ordered on
 *     that stream; functions returning host results synchronise it.
 *   - There is no CPU fallback: without a usable CUDA device every compute
 *     entry point returns TDVP_ECUDA.
 */
#ifndef TDVP_H
#define TDVP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define TDVP_OK 0
#define TDVP_EINVAL (-1)   /* bad argument or size                                  */
#define TDVP_ENOMEM (-2)   /* device or host allocation failed                      */
#define TDVP_ECUDA (-3)    /* CUDA runtime error, or no usable device              */
#define TDVP_ENUMERIC (-4) /* NaN/Inf, zero norm, or a failed decomposition        */
#define TDVP_ETIMEOUT (-5) /* a bounded device wait gave up (status word set)      */
#define TDVP_ESTATE (-6)   /* handle in the wrong state for this call               */

/* ---- model kinds (Sec. IV: Eq. 25 Ising, Eq. 27 XY, Eq. 31 XXX) ---- */
#define TDVP_ISING 0 /* sum_{i<j} J f(r) sz_i sz_j + h sum_i sx_i               */
#define TDVP_XY 1    /* sum_{i<j} J f(r) (sx_i sx_j + sy_i sy_j) + h sum_i sx_i  */
#define TDVP_XXX 2   /* sum_{i<j} J f(r) S_i.S_j (S = sigma/2) + h sum_i sx_i     */

/* ---- contraction precision of H_eff and the environment updates ---- */
#define TDVP_FP64 0   /* complex FP64 throughout                                  */
#define TDVP_TF32 1   /* tensor-core TF32 complex GEMMs, FP32 accumulate          */
#define TDVP_TF32X3 2 /* 3xTF32 split-precision products, FP32 accumulate         */
/* Precision of every step, per mode:
 *   - Lanczos recurrences and re-orthogonalisation, the tridiagonal
 *     exponential and V = Lambda^-1: FP64 in every mode.
 *   - H_eff applications: the mode's GEMMs (FP64 SIMT, or tcgen05 TF32 /
 *     3xTF32 with FP32 accumulation). The tensor cores' FP32 accumulation
 *     loses accuracy with every MMA step, so long sums are cut into chunks
 *     summed in FP64; an H_eff application is then accurate to ~6e-6 to 1e-5
 *     relative to its largest element in 3xTF32, ~4e-4 in TF32.
 *   - Environment updates: FP64 (TDVP_FP64); in the mixed modes double-float
 *     GEMMs on the FP32 pipe (~48 significant bits) unless
 *     tdvp_set_env_tensor_cores moves them to the tensor cores.
 *   - Theta = Psi V Psi and the measurements: FP64 (TDVP_FP64) or
 *     double-float (mixed modes).
 *   - Bond SVD: one-sided Jacobi. TDVP_FP64: an FP32 phase, then FP64 sweeps
 *     to ~1e-14 relative orthogonality; isometries to ~1e-14. Mixed modes: the
 *     FP32 phase, then double-float sweeps that stop at a relative
 *     off-diagonal of 1e-4 (~1e-8 left), the unitary factor updated through
 *     FP32-accumulated block rotations; isometries to ~1e-10 when the kept
 *     singular values lie above ~1e-5 of the largest (the FP32 phase resolves
 *     them), ~3e-7 when they reach down to its noise level (~1e-6).
 * Measured on a 41-site Ising chain with every bond at chi = 64 (8 segments,
 * dt = 0.01), <sigma^z_j> of TDVP_TF32X3 against TDVP_FP64 after 20 steps:
 * 3.6e-7 (default); 1.1e-5 with tensor-core environments; ~2e-12 when only
 * the SVD is the mixed one. */

/* ---- observables for tdvp_measure ---- */
#define TDVP_OBS_SZ 0
#define TDVP_OBS_SX 1
#define TDVP_OBS_SY 2

typedef struct tdvp_mpo_s* tdvp_mpo;
typedef struct tdvp_mps_s* tdvp_mps;

/* Long-range spin chain (Sec. II C). f(r) = 1/r^alpha is represented by
 * n_exp exponentials, f(r) ~ sum_k x_k lam_k^r, giving an MPO of bond
 * dimension m = n_terms * n_exp + 2 (n_terms = 1, 2, 3 for Ising, XY, XXX).
 * x and lam: NULL to fit them inside tdvp_build_mpo (tdvp_fit_power_law on
 * r = 1..N-1), or 2*n_exp doubles each (complex) supplied by the caller. */
typedef struct {
  int kind;
  int N;
  double alpha;
  double J;
  double h;
  int n_exp;
  const double* x;
  const double* lam;
} tdvp_model;

/* Time-step settings.
 * dt: time step; every half sweep evolves by dt/2 (Sec. III A).
 * chi_max, w_max, eps: truncation of every SVD -- keep the smallest rank whose
 *   discarded weight is <= w_max (Eq. 22), at most chi_max (Sec. III C), and
 *   only singular values > eps * lambda_1 (Sec. III D). At least one is kept.
 * krylov_max, krylov_tol: Lanczos exponentiation with at most krylov_max
 *   vectors, stopping when the a-posteriori estimate falls below krylov_tol
 *   (krylov_tol = 0: always krylov_max vectors unless the space is exhausted).
 *   krylov_max <= 24.
 * precision: TDVP_FP64 / TDVP_TF32 / TDVP_TF32X3.
 * n_seg, seg_len: Stoudenmire-White partition into n_seg segments of
 *   seg_len[k] >= 2 sites (Sec. III B, Fig. 6); n_seg <= 1 or seg_len NULL
 *   runs the serial sweep. All segments of a stage run in the same launches.
 * merge_turning: 1 evolves turning pairs once by dt instead of twice by dt/2
 *   (App. A). */
typedef struct {
  double dt;
  int chi_max;
  double w_max;
  double eps;
  int krylov_max;
  double krylov_tol;
  int precision;
  int n_seg;
  const int* seg_len;
  int merge_turning;
} tdvp_step_params;

/* Statistics accumulated by tdvp_step (added to what the struct holds). */
typedef struct {
  double w_total;            /* sum of discarded weights w over all SVDs (Sec. III C) */
  int chi_max_seen;          /* largest bond dimension produced                       */
  int n_stages;              /* batched stages executed                               */
  int64_t krylov_vectors;    /* Krylov vectors used over all local exponentials       */
  int64_t n_fwd2;            /* two-site forward updates                              */
  int64_t n_back1;           /* one-site backward updates                             */
  double heff_flops;         /* algorithmic flops of all H_eff applications           */
  int64_t kernel_launches;   /* kernels launched                                      */
} tdvp_step_stats;

/* ---- library / device ---- */

/* Device memory through the caller's allocator: every buffer the library
 * allocates afterwards (states, environments, MPO blocks, workspaces) comes from
 * alloc(bytes, ctx) -- which returns device memory or NULL (then TDVP_ENOMEM) --
 * and goes back through the free function registered with it, free(ptr, ctx),
 * after the library has synchronised the device (a caching allocator may reuse
 * the block at once). alloc = free = NULL restores cudaMalloc / cudaFree; blocks
 * already handed out keep their own free function. The Python binding offers
 * torch's caching allocator (use_torch_allocator). TDVP_EINVAL if exactly one of
 * alloc and free is NULL. */
typedef void* (*tdvp_alloc_fn)(size_t bytes, void* ctx);
typedef void (*tdvp_free_fn)(void* ptr, void* ctx);
int tdvp_set_allocator(tdvp_alloc_fn alloc, tdvp_free_fn free_fn, void* ctx);

/* Thread-local message of the last failure ("" if none). */
const char* tdvp_last_error(void);
/* Library version string. */
const char* tdvp_version(void);
/* 1 if a CUDA device of compute capability >= 10.0 is usable, else 0. */
int tdvp_device_ok(void);

/* ---- model and MPO (Sec. II C) ---- */

/* Fit r^-alpha on r = 1..r_max by n_exp exponentials (Pirvu et al.'s
 * shift-invariance method, as used by the paper; Sec. II C). Writes 2*n_exp
 * doubles (complex) to x_out and lam_out. Host only, no GPU needed.
 * TDVP_EINVAL for n_exp < 1, n_exp > 64, r_max < 2 or alpha <= 0. */
int tdvp_fit_power_law(double alpha, int n_exp, int r_max, double* x_out, double* lam_out);

/* Host only. The Levenberg-Marquardt alternative to tdvp_fit_power_law that
 * the Supplemental Material compares for 1/r^2: real x_k, lam_k minimising the
 * sum over r = 1..r_max of (w_r e_r)^2, e_r = sum_k x_k lam_k^r - r^-alpha,
 * w_r = 1 (relative = 0) or r^alpha (relative = 1, the relative error), started
 * from tdvp_fit_power_law (real parts), stopped as the paper's lsqnonlin options
 * (1000 iterations, 10000 evaluations, step 1e-6, function 1e-14). If the result
 * has some |lam_k| >= 1 the start is returned. rms_out (may be NULL): the root
 * mean square of w_r e_r. Outputs as tdvp_fit_power_law (complex, imaginary 0);
 * pass them to tdvp_build_mpo through tdvp_model.x / .lam. */
int tdvp_fit_power_law_lm(double alpha, int n_exp, int r_max, int relative, double* x_out, double* lam_out,
                          double* rms_out);
/* Build the MPO of a model on the current device. Host arrays are copied. */
int tdvp_build_mpo(const tdvp_model* model, tdvp_mpo* out);
/* Host only: the couplings V(r) = sum_k x_k lam_k^r, r = 1..r_max, that an MPO
 * with these exponentials realises (Sec. II C): 2*r_max doubles (complex). */
int tdvp_couplings(int n_exp, const double* x, const double* lam, int r_max, double* V_out);
/* The same for the exponentials held by `mpo`. */
int tdvp_mpo_couplings(tdvp_mpo mpo, int r_max, double* V_out);
/* MPO bond dimension m and physical dimension d. */
int tdvp_mpo_dims(tdvp_mpo mpo, int* m, int* d);
/* Copy the bulk tensor W (2*m*m*d*d doubles) and the couplings x, lam
 * (2*n_exp doubles each; any pointer may be NULL). Host only. */
int tdvp_mpo_tensor(tdvp_mpo mpo, double* W_out, double* x_out, double* lam_out);
/* Release an MPO handle (NULL is ignored). */
void tdvp_free_mpo(tdvp_mpo mpo);

/* ---- state (Sec. II A/B: inverse canonical gauge, Eq. 9) ---- */

/* Product state |s_0 s_1 ...>, s_j in {0 (up, sz=+1), 1 (down)}.
 * chi_cap: largest bond dimension the handle will hold (device memory is
 * sized for it: site j holds up to min(chi_cap, d^(j+1), d^(N-1-j))). */
int tdvp_init_mps(int N, int d, const int* basis_state, int chi_cap, tdvp_mps* out);
/* State from raw site tensors (host, complex128, tensors[j] of shape
 * [dims[j]][d][dims[j+1]], dims[0] = dims[N] = 1). The library brings it to
 * the inverse canonical gauge (Sec. II B) with GPU SVDs -- a left-to-right
 * orthonormalisation and a right-to-left sweep giving Lambda_j at every bond,
 * Psi_j = Lambda_{j-1} B_j, V_j = Lambda_j^-1 -- cutting each bond to
 * chi_cap and to singular values > eps * lambda_1, and normalises it. */
int tdvp_init_mps_tensors(int N, int d, const int* dims, const double* const* tensors,
                          int chi_cap, double eps, tdvp_mps* out);
/* Bring `mps` back to the inverse canonical gauge (Sec. II B) and unit norm:
 * a left-to-right then right-to-left SVD sweep over Psi_1 V_1 Psi_2 ... Psi_N
 * (bond dimensions capped at the handle's chi_cap, singular values below
 * eps * lambda_1 dropped). The segment scheme breaks the gauge conditions at
 * segment boundaries; the paper reorthonormalises (and recomputes the
 * environments) when the error in the norm grows (Sec. III D, Fig. 8). The
 * environments are rebuilt by the next tdvp_step / tdvp_dmrg. Synchronises the
 * device. */
int tdvp_reorthonormalize(tdvp_mps mps, double eps);
/* Current bond dimensions (N-1 ints). */
int tdvp_mps_bond_dims(tdvp_mps mps, int* dims_out);
/* Copy Psi_j (2*chi_l*d*chi_r doubles) or V_j (chi_j doubles) to the host. */
int tdvp_mps_get_site(tdvp_mps mps, int j, double* out);
int tdvp_mps_get_bond(tdvp_mps mps, int j, double* out);
/* Site count N and physical dimension d. */
int tdvp_mps_size(tdvp_mps mps, int* N, int* d);
/* Release a state handle and its device memory (NULL is ignored). */
void tdvp_free_mps(tdvp_mps mps);

/* ---- time evolution (Sec. III) ---- */

/* Advance `mps` by n_steps time steps of the symmetric two-site TDVP sweep
 * (Sec. III A, Fig. 2), in the segment scheme when params->n_seg > 1 (Sec.
 * III B, Figs. 6-7). Environments (Fig. 3) are built on the first call with a
 * given MPO (all left ones left to right, all right ones right to left) and
 * cached in the handle. `stats` may be NULL. Synchronises `stream` once per
 * stage (to read the new bond dimensions). TDVP_ENUMERIC on NaN or a zero
 * norm; TDVP_ETIMEOUT if a bounded device wait gave up. */
int tdvp_step(tdvp_mps mps, tdvp_mpo mpo, const tdvp_step_params* params, int n_steps,
              tdvp_step_stats* stats, void* stream);

/* One-site TDVP (Sec. II, Eq. proj1site; the paper's discussion proposes its
 * parallel form and the hybrid scheme below): n_steps symmetric steps of the
 * serial sweep at fixed bond dimension -- left to right, each site evolved
 * forward by dt/2 with H1_eff, then split ((chi_{j-1} d) x chi_j SVD, no
 * truncation) and its bond matrix evolved backward by dt/2 with the bond term
 * H0_eff C = sum beta_{j+1}[a,w,a'] C[a',b'] gamma_j[b,w,b'], re-diagonalised (the
 * inverse canonical gauge restored) and moved into site j+1; the last site
 * forward by dt; then the mirror sweep, ending with site 0 forward by dt/2.
 * Norm and energy are conserved to the Lanczos accuracy.
 * With n_seg > 1 the parallel form (the paper's outlook, read with the
 * segments of Sec. III B): every segment runs this sweep over its own sites in
 * the direction tdvp_step gives it, and the two sites of a boundary are
 * evolved together as in tdvp_step (Theta = Psi_e V_e Psi_{e+1}, V = Lambda^-1)
 * and split back at the bond's current dimension (cut only by eps), which
 * stands for their site terms and the bond term between them; per stage the
 * site steps, the bond steps and the boundary pairs of all segments each run
 * batched. Bond
 * dimensions are kept; the boundary cuts change norm and energy by their
 * discarded weight. Exact at full bond dimension. The schedule is
 * tdvp_schedule1's. FP64 only. stats->n_back1 counts the site updates,
 * stats->n_fwd2 the boundary pair updates. */
int tdvp_step1(tdvp_mps mps, tdvp_mpo mpo, const tdvp_step_params* params, int n_steps,
               tdvp_step_stats* stats, void* stream);
/* The hybrid scheme: per step, a tdvp_step (two-site) while some bond is below
 * min(chi_max, its largest possible dimension), else a tdvp_step1 (one-site),
 * both with the segments of params (serial without). FP64 only. Returns the
 * number of one-site steps (>= 0) or an error. */
int tdvp_step_hybrid(tdvp_mps mps, tdvp_mpo mpo, const tdvp_step_params* params, int n_steps,
                     tdvp_step_stats* stats, void* stream);

/* ---- ground states: two-site DMRG ----
 * The paper prepares its initial states with two-site DMRG (Sec. IV and the
 * Supplemental Material) and notes that a TDVP time step has the sweep
 * pattern and cost of a two-site DMRG sweep (Sec. III A); it prints no DMRG
 * algorithm, so this is the textbook two-site update built from the same
 * pieces as tdvp_step: Theta = Psi_j V_j Psi_{j+1}, the lowest eigenvector of
 * H2_eff by Lanczos on the tridiagonal projection (at most krylov_max vectors
 * started from Theta, stopped when the residual estimate beta_{k} |z_{k-1}|
 * falls below krylov_tol or on breakdown; the new Theta keeps the norm of the
 * old), the truncated split of Fig. 5 and the environment update of the sweep
 * direction. No backward one-site step. */
typedef struct {
  int chi_max;
  double w_max;
  double eps;
  int krylov_max;      /* <= 24 */
  double krylov_tol;   /* 0: always krylov_max vectors */
  int precision;       /* TDVP_FP64, TDVP_TF32 or TDVP_TF32X3 (as tdvp_step) */
} tdvp_dmrg_params;

typedef struct {
  double energy;             /* Ritz value of the last local update (the state's energy) */
  double w_total;            /* discarded weight summed over all splits             */
  int chi_max_seen;
  int64_t krylov_vectors;
  int64_t n_updates;         /* two-site updates                                    */
  int64_t kernel_launches;
} tdvp_dmrg_stats;

/* n_sweeps serial sweeps (left to right over pairs 0..N-2, then right to left)
 * on `mps` in place. Environments are built as in tdvp_step (and cached in the
 * handle). Synchronises `stream` after every update. Errors as tdvp_step. */
int tdvp_dmrg(tdvp_mps mps, tdvp_mpo mpo, const tdvp_dmrg_params* params, int n_sweeps,
              tdvp_dmrg_stats* stats, void* stream);

/* ---- derivatives with respect to the model parameters ----
 * The paper evolves in time only. These calls give d<O_j(t)>/d(h, J) of the
 * sweep that tdvp_step runs (Sec. III A/B, Eqs. 18-20, Fig. 5) by forward-mode
 * differentiation: every local operation of the sweep also advances a tangent
 * (dPsi_j, dV_j, d beta_j, d gamma_j) per parameter direction, in FP64.
 *   Theta:     dTheta = dPsi_j V Psi_{j+1} + Psi_j dV Psi_{j+1} + Psi_j V dPsi_{j+1}
 *   exp:       d(e^{-itH} x) = e^{-itH} dx + int_0^1 e^{-istH} (-it dH) e^{-i(1-s)tH} x ds,
 *              the integral by n_quad-point Gauss-Legendre quadrature, each exponential by
 *              the same Lanczos settings as the primal step, dH = H_eff(d beta, W, gamma) +
 *              H_eff(beta, dW, gamma) + H_eff(beta, W, d gamma);
 *   split:     the derivative of the truncated SVD at fixed kept rank (all singular triplets
 *              of Theta' enter the kept-discarded couplings);
 *   envs:      the product rule on Eq. 19 (bra, ket and W).
 * The derivative is that of the algorithm with exact local exponentials and a
 * fixed truncation pattern; it agrees with finite differences of tdvp_step as long
 * as the kept ranks do not change and the Lanczos runs are converged. */
#define TDVP_PARAM_H 0   /* transverse field h                                     */
#define TDVP_PARAM_J 1   /* coupling J (multiplies every exponential weight x_k)    */
#define TDVP_MAX_DIR 4

typedef struct tdvp_tangent_s* tdvp_tangent;

/* dW/d(param) of `mpo` as an MPO handle (W is affine in h and J, Sec. II C), for
 * tdvp_step_tangent. The handle may be used with tdvp_energy to get <psi|dH|psi>. */
int tdvp_build_mpo_derivative(tdvp_mpo mpo, int param, tdvp_mpo* out);
/* Tangent of `mps` in n_dir (<= TDVP_MAX_DIR) directions, all zero (the state
 * does not depend on the parameters). The tangent follows the bond dimensions
 * of `mps`; it stays valid only while `mps` is advanced by tdvp_step_tangent. */
int tdvp_tangent_create(tdvp_mps mps, int n_dir, tdvp_tangent* out);
/* Release a tangent handle (NULL is ignored). */
void tdvp_free_tangent(tdvp_tangent tan);
/* n_steps time steps of `mps` exactly as tdvp_step (FP64 only), advancing `tan`
 * along dmpo[0..n_dir) (derivative MPOs of `mpo`). n_quad in [1, 8] and
 * n_quad * n_dir <= 31. The local operations of a stage run one at a time.
 * Errors as tdvp_step; TDVP_EINVAL for a derivative MPO of another MPO. */
int tdvp_step_tangent(tdvp_mps mps, tdvp_mpo mpo, tdvp_tangent tan, const tdvp_mpo* dmpo,
                      const tdvp_step_params* params, int n_quad, int n_steps, tdvp_step_stats* stats,
                      void* stream);
/* <O_j> (N doubles, may be NULL) and d<O_j> per direction (n_dir x N doubles,
 * row q = direction q) for <O_j> = <psi|O_j|psi>/<psi|psi>:
 * d<O_j> = 2 Re<psi|O_j|dpsi>/<psi|psi> - <O_j> 2 Re<psi|dpsi>/<psi|psi>.
 * Synchronises. */
int tdvp_measure_tangent(tdvp_mps mps, tdvp_tangent tan, int obs, double* value_out, double* d_out);
/* Host only: n-point Gauss-Legendre nodes and weights on [0, 1] (the quadrature
 * of tdvp_step_tangent). */
int tdvp_gauss_legendre(int n, double* x_out, double* w_out);

/* ---- measurement (Sec. IV; excluded from timing as in the paper) ---- */

/* A device copy of `src` (tensors and bond dimensions; environments are rebuilt
 * on the copy's first step). */
int tdvp_mps_copy(tdvp_mps src, tdvp_mps* out);
/* Psi_j <- O Psi_j on the physical index: O_j |psi>, op = d x d complex
 * [s_out][s_in] (2 d^2 doubles, host). A unitary O (sigma^z for the excitation
 * sigma^z_k |psi_0> of the dynamical correlation function, Sec. IV) keeps the
 * inverse canonical gauge that tdvp_step needs. Synchronises. */
int tdvp_apply_site_op(tdvp_mps mps, int j, const double* op);
/* <a|O_j|b> for every site j, not normalised: out = 2N doubles (re, im per
 * site), by transfer matrices with a in the bra and b in the ket. With
 * |b> = e^{-iHt} sigma^z_k |a>, e^{-i E0 t} out_r is the dynamical correlation
 * function C(r - k, t) of Sec. IV. Synchronises. */
int tdvp_expect_mixed(tdvp_mps a, tdvp_mps b, int obs, double* out);

/* <psi|O_j|psi>/<psi|psi> for every site j (N doubles) by full transfer-matrix
 * contraction of Psi_1 V_1 ... Psi_N (exact in any gauge). Synchronises. */
int tdvp_measure(tdvp_mps mps, int obs, double* out);
/* <psi|psi> and <psi|H|psi>/<psi|psi>. */
int tdvp_norm(tdvp_mps mps, double* out);
int tdvp_energy(tdvp_mps mps, tdvp_mpo mpo, double* out);
/* <a|b> (2 doubles). Infidelity (Eq. 24) is 1 - |<a|b>|/sqrt(<a|a><b|b>). */
int tdvp_overlap(tdvp_mps a, tdvp_mps b, double* out);

/* ---- kernel-level operations on caller device buffers ----
 * One local operation each, for testing and for callers that drive their own
 * sweep. All tensor pointers are device pointers (complex128, layouts above)
 * except W, which is a host pointer to the bulk MPO tensor W[m][m][d][d]
 * (complex128). Temporaries are allocated and freed inside the call. The
 * call synchronises `stream` before returning. */

/* y = H_eff x (Fig. 4). nsite = 2: x, y are [chi_l][d][d][chi_r], H_eff from
 * L = beta_j [chi_l][m][chi_l], W_j = W_{j+1} = W, R = gamma_{j+1}
 * [chi_r][m][chi_r]; nsite = 1: x, y are [chi_l][d][chi_r], R = gamma_j. */
int tdvp_op_heff(int precision, int nsite, int chi_l, int chi_r, int m, int d, const double* W,
                 const double* L, const double* R, const double* x, double* y, void* stream);

/* Environment update (Fig. 3, Eq. 19). side 0: out = beta_{j+1}
 * [chi_r][m][chi_r] from env = beta_j [chi_l][m][chi_l] and A = Psi_j V_j
 * [chi_l][d][chi_r]. side 1: out = gamma_j [chi_l][m][chi_l] from
 * env = gamma_{j+1} [chi_r][m][chi_r] and B = V_j Psi_{j+1} [chi_l][d][chi_r]. */
int tdvp_op_env(int precision, int side, int chi_l, int chi_r, int m, int d, const double* W,
                const double* env, const double* A, double* out, void* stream);

/* y = exp(-i t H_eff) x by Lanczos (Eq. 18 with t = dt/2, Eq. 20 with
 * t = -dt/2), same operands as tdvp_op_heff. Writes the number of Krylov
 * vectors used to *n_vectors (host, may be NULL). kmax <= 24. */
int tdvp_op_expm(int precision, int nsite, int chi_l, int chi_r, int m, int d, const double* W,
                 const double* L, const double* R, const double* x, double* y, double t,
                 int kmax, double tol, int* n_vectors, void* stream);

/* Truncated SVD split of a two-site state (Fig. 5): theta [rows][cols]
 * (rows = chi_l*d, cols = d*chi_r) -> Psi_L [rows][chi] = U Lambda,
 * Psi_R [chi][cols] = Lambda V^dagger, V [chi] = 1/Lambda, with the rank
 * chosen as in tdvp_step_params. Psi_L / Psi_R must hold min(rows, cols)
 * columns / rows; s_out (device, may be NULL) receives all min(rows, cols)
 * singular values in descending order. When s_out is NULL the SVD skips the
 * rotations between vectors that the truncation certainly discards (the
 * kept triplets, chi and w are unchanged; the discarded directions are not
 * resolved). chi and w (discarded weight) are written to host ints/doubles.
 * rows, cols <= 4096. */
int tdvp_op_split(int rows, int cols, const double* theta, int chi_max, double w_max, double eps,
                  double* Psi_L, double* V, double* Psi_R, double* s_out, int* chi, double* w,
                  void* stream);
/* tdvp_op_split with the SVD of a given path: TDVP_FP64 as tdvp_op_split;
 * TDVP_TF32 / TDVP_TF32X3 the mixed-precision path's SVD (FP32 Jacobi phase,
 * double-float finishing sweeps to ~1e-10 relative orthogonality, FP32
 * block-rotation updates of the unitary factor), as used by tdvp_step. */
int tdvp_op_split_prec(int precision, int rows, int cols, const double* theta, int chi_max, double w_max,
                       double eps, double* Psi_L, double* V, double* Psi_R, double* s_out, int* chi,
                       double* w, void* stream);

/* Same as tdvp_op_heff with precision TDVP_FP64, for callers that cannot
 * allocate device memory: plug-ins whose host application owns every device
 * allocation through its own pool, or real-time loops that must never enter
 * an allocator. The paper has no counterpart: this is a deployment variant of
 * the H_eff application of Fig. 4. It calls no cudaMalloc, cudaFree or
 * allocating library routine: its intermediates and the sparse MPO blocks
 * live in one fixed device array of TDVP_NOALLOC_SCRATCH_BYTES bytes inside
 * the library, present on every GPU that loads it until the process exits.
 * Problems whose scratch, 2 * chi_l * m * D * chi_r * 16 bytes (D = d^2 for
 * nsite = 2, d for nsite = 1) plus the MPO blocks, exceeds that size, or with
 * m > TDVP_NOALLOC_MAX_M, are rejected with TDVP_EINVAL before any work. The
 * first call on a device looks the array's address up (cudaGetSymbolAddress)
 * and should come before any stream capture. All calls share the array:
 * calls whose work overlaps on the GPU race on it and must be serialised by
 * the caller. Every call builds the two-site operator on the host
 * (O(m^3 d^4) operations) and copies it from host memory. W is a host
 * pointer; L, R, x, y are device pointers as in tdvp_op_heff. Synchronises
 * `stream` before returning. */
#define TDVP_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
#define TDVP_NOALLOC_MAX_M 64
int tdvp_op_heff_noalloc(int nsite, int chi_l, int chi_r, int m, int d, const double* W, const double* L,
                         const double* R, const double* x, double* y, void* stream);

/* ---- environment precision of the mixed modes ---- */

/* enable = 0 (the default): in TDVP_TF32 / TDVP_TF32X3 the environment
 * updates (Eq. 19 and its mirror) run as double-float GEMMs on the FP32 pipe
 * (~48 significant bits; the W stage in FP64) while H_eff runs on the tensor
 * cores. An environment is reused by every later H_eff of the half sweep, so
 * its error acts like a fixed perturbation of H and moves observables
 * linearly in time; with tensor-core environments that drift was ~30x larger
 * (41-site Ising chain, chi = 64: <sigma^z_j> 1.1e-5 from the FP64 path after
 * 20 steps, against 3.6e-7). enable = 1: the environment updates use the
 * mode's tensor-core products too (faster, less accurate). Process-wide; takes
 * effect at the next environment update. Returns TDVP_OK. */
int tdvp_set_env_tensor_cores(int enable);

/* ---- GEMM tile autotuning ---- */

/* enable != 0 (the default): the first GEMM launch of each family (tcgen05
 * TF32 / 3xTF32 products, FP64 and double-float SIMT products) with a new
 * shape -- its M, N, K (set by chi, the MPO bond dimension m and d) and batch
 * size, bucketed to powers of two -- times every tile candidate on its own
 * operands (tcgen05: N tile 256 or 128; SIMT: 64 x 64 or 32 x 32 outputs per
 * CTA) with CUDA events on the launching stream and keeps the fastest for that
 * shape. The candidates compute every output with the same operations, so
 * tuning changes no result. A tuning launch synchronises its stream once.
 * enable = 0: fixed tiles (tcgen05 N = 256; FP64 64 x 64; double-float 64 x 64
 * when the batch has at least two tiles per SM, else 32 x 32). Either call
 * forgets the decisions made so far. Process-wide. Returns TDVP_OK. */
int tdvp_set_autotune(int enable);
/* The decisions made so far as a JSON list (family, shape bucket, choice,
 * microseconds per candidate), NUL-terminated in out (at most len bytes; out
 * may be NULL to query). Returns the length of the full text, without NUL. */
int tdvp_autotune_report(char* out, int len);

/* ---- failure detection ---- */

/* Number of polls a grid-barrier wait of the SVD's cooperative Jacobi sweeps
 * makes before it gives up (Sec. III D monitors the norm error of the run;
 * the bounded waits are this library's own safeguard, with no counterpart in
 * the paper). A wait that gives up sets the status word and an abort word
 * that makes every other block of the launch return at its next barrier;
 * the calling entry point then returns TDVP_ETIMEOUT. A state handle whose
 * tdvp_step failed keeps its status (its tensors are no longer a valid
 * step); other handles and later kernel-level calls (tdvp_op_*) start from a
 * cleared status. spins < 0 restores the default (2^24 polls of
 * ~64 ns, about a second). Process-wide; takes effect at the next SVD
 * launch. Returns TDVP_OK. */
int tdvp_set_wait_limit(long long spins);

/* ---- profiling ---- */

/* enable != 0: from now on every kernel launch of the library is bracketed by
 * CUDA events recorded on its launching stream, and its algorithmic work
 * (flops, bytes) is accumulated per kernel kind; 0 stops it. Either call
 * discards what was accumulated. Synchronises the device. */
int tdvp_profile(int enable);
/* idx < 0: returns the number of kernel kinds recorded. Otherwise copies kind
 * idx: name (NUL-terminated, at most name_len bytes), total device time in
 * ms, launches, algorithmic flops and bytes; returns 1. Synchronises. */
int tdvp_profile_read(int idx, char* name, int name_len, double* ms, int64_t* launches, double* flops,
                      double* bytes);
/* Auxiliary count accumulated for kind idx (the Jacobi SVD phases: sweeps
 * summed over the problems of each batch). Returns 1 or an error code. */
int tdvp_profile_read_aux(int idx, double* aux);

/* ---- host-only utilities (no GPU needed) ---- */

/* The stage schedule of one half (1 or 2) of a time step (Sec. III A/B, App.
 * A/B): 7 ints per op -- segment, kind (0 = two-site forward step on the pair
 * (j, j+1), 1 = one-site backward step on site j), j, time in units of dt/2,
 * environments rebuilt after a two-site step (bit 0: beta_{j+1}, bit 1:
 * gamma_j), boundary flag, stage index. Returns the number of ops (out may be
 * NULL to query it) or a negative error code. */
int tdvp_schedule(int N, int n_seg, const int* seg_len, int merge_turning, int half, int* out, int max_ops);

/* The stage schedule of one half of a segmented one-site step (tdvp_step1
 * with n_seg > 1), in tdvp_schedule's 7-int layout with kind 0 = one-site
 * forward step on site j, 1 = bond j evolved backward with the centre moving
 * right, 2 = bond j - 1 evolved backward with the centre moving left (site j
 * split), 3 = boundary pair (j, j + 1) (boundary flag 1); the environment
 * field is 0. Returns the number of ops (out may be NULL to query it) or a
 * negative error code. */
int tdvp_schedule1(int N, int n_seg, const int* seg_len, int merge_turning, int half, int* out, int max_ops);

/* Point-to-point messages of one half step (1 or 2) when the segments are
 * spread over ranks, one GPU each (Sec. III B: the segments were MPI
 * processes exchanging O(chi^2 (m + d)) numbers at their boundaries).
 * seg_rank[k]: rank of segment k, non-decreasing (contiguous groups). scheme:
 * 2 = tdvp_step's schedule, 1 = tdvp_step1's. For every boundary update whose
 * two segments live on different ranks: before it the right rank sends
 * Psi_{e+1} and gamma_{e+1} to the left rank, after it the left rank sends
 * Psi_{e+1}, V_e and beta_{e+1} back. 6 ints per message: stage of the
 * boundary update, 0 = before / 1 = after it, source rank, destination rank,
 * tensor (0 = Psi_j, 1 = V_j, 2 = beta_j, 3 = gamma_j), j. Ranks that run the
 * stages in lockstep and exchange these messages reproduce the one-rank
 * sweep. Returns the number of messages (out may be NULL to query it) or a
 * negative error code. Host only. */
int tdvp_exchange_plan(int N, int n_seg, const int* seg_len, const int* seg_rank, int scheme, int merge_turning,
                       int half, int* out, int max_msgs);

/* c = exp(-i t T) e_0 (2*k doubles) for the real symmetric tridiagonal T with
 * diagonal alpha[k] and off-diagonal beta[k-1] -- the small exponential of the
 * Lanczos method; the same routine runs inside the device kernels. k <= 24. */
int tdvp_tridiag_expm(int k, const double* alpha, const double* beta, double t, double* c_out);

#ifdef __cplusplus
}
#endif
#endif /* TDVP_H */
