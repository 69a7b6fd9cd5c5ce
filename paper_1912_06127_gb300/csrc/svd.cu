// Truncated SVD split of the evolved two-site state (Fig. 5), FP64.
//
// Theta' is reshaped to a (chi_l d) x (d chi_r) matrix and decomposed with the
// one-sided (Hestenes) Jacobi method: the smaller of its row set and column
// set is orthogonalised by plane rotations, each rotation chosen to make one
// pair of vectors orthogonal (a 2x2 Hermitian eigenproblem), until a full
// sweep over all pairs applies none. The rotations are accumulated, which
// gives the other set of singular vectors. Pairs are visited in round-robin
// order, so that each round holds n/2 disjoint pairs, one warp per pair and
// all problems of a stage in the same launch. The final vector norms are the
// singular values.
//
// FP64 arithmetic is scarce on this GPU (about 1/64 of the FP32 issue rate), so
// the sweeps run in two phases. First the rotations are found and applied in
// FP32 until the vectors are orthogonal to about 1e-6 (relative). The
// accumulated FP32 rotation is then made unitary to FP64 rounding by two
// Newton-Schulz steps (Acc <- (3 Acc - Acc Acc^H Acc) / 2), the vectors are
// recomputed in FP64 from the input (X = Acc Theta'), and FP64 sweeps finish
// the job. Cyclic Jacobi converges quadratically, so a sweep whose largest
// relative off-diagonal |<x,y>|/(|x||y|) stayed below 1e-7 leaves less than
// ~1e-14 and ends the iteration. The result has FP64 accuracy; the FP32
// phase only shortens the FP64 phase. The FP64 phase skips pairs of vectors
// that both lie below a threshold under which the truncation discards
// everything (svd_tail_threshold): such rotations change neither the kept
// vectors nor the discarded weight, and without them the FP64 phase needs no
// more sweeps for the tail than for the kept part.
//
// Truncation (Sec. III C, Eq. 22 and Sec. III D): the smallest rank chi_w
// whose discarded weight sum_{j >= chi_w} lambda_j^2 is <= w_max, capped at
// chi_max and at the values above eps * lambda_1, at least 1. Then
// Psi_L = A' Lambda', Psi_R = Lambda' B', V' = Lambda'^{-1} (Sec. II B).
#include <atomic>
#include "common.h"
#include "svd.h"

namespace tdvp {

constexpr double JACOBI_TOL = 1e-14;
constexpr int SVD_WARPS = 8;
constexpr int SVD_MAX_SWEEPS = 40;

// Power-of-two scale bringing the largest entry of theta into [0.5, 1), so
// that the FP32 phase cannot overflow or underflow whatever the input's
// magnitude (rotations do not depend on the scale), stored in sig[n_vec];
// and ||theta||_F^2, stored in sig[n_vec + 1], which sets the level below
// which vectors are rounding noise.
__global__ void svd_scale(const __grid_constant__ SvdBatch B) {
  const SvdDesc& P = B.d[blockIdx.x];
  __shared__ double red[512];
  __shared__ double red2[512];
  double mx = 0.0, fr = 0.0;
  const int64_t n = (int64_t)P.rows * P.cols;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 v = P.theta[i];
    mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
    fr += v.x * v.x + v.y * v.y;
  }
  red[threadIdx.x] = mx;
  red2[threadIdx.x] = fr;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
      red2[threadIdx.x] += red2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    P.sig[P.n_vec + 1] = red2[0];
    double sc = 1.0;
    if (red[0] > 0.0 && red[0] < 1e300) {
      int e = 0;
      frexp(red[0], &e);
      sc = ldexp(1.0, -e);
    }
    P.sig[P.n_vec] = sc;
  }
}

__global__ void svd_setup32(const __grid_constant__ SvdBatch B) {
  const SvdDesc& P = B.d[blockIdx.y];
  const double sc = P.sig[P.n_vec];
  const int64_t nx = (int64_t)P.n_vec * P.len;
  const int64_t na = (int64_t)P.n_vec * P.n_vec;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nx + na;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nx) {
      int v = (int)(i / P.len), e = (int)(i % P.len);
      // trans 0: vector v = row v of theta; trans 1: vector v = column v
      double2 t = P.trans ? P.theta[(int64_t)e * P.cols + v] : P.theta[(int64_t)v * P.cols + e];
      P.X32[i] = make_float2((float)(t.x * sc), (float)(t.y * sc));
    } else {
      int64_t q = i - nx;
      int r = (int)(q / P.n_vec), c = (int)(q % P.n_vec);
      P.Acc32[q] = make_float2(r == c ? 1.0f : 0.0f, 0.0f);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    P.rotated[0] = P.rotated[1] = 0;
    *P.conv = 0;
    *P.maxr = 0u;
  }
}

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int GV = 32;  // vectors of a visit in the Gram form of the FP32 phase (below)

// Element types of the Jacobi sweeps: double2 (complex FP64), float2 (complex
// FP32) and float4 (complex double-float: re_hi, im_hi, re_lo, im_lo; value =
// hi + lo, ~48 significant bits, computed on the FP32 pipe). R: Gram entries,
// norms and rotation parameters; CT: complex rotation parameters; AT: the
// element type of Acc.
template <typename T>
struct Prec;
template <>
struct Prec<double2> {
  using R = double;
  using CT = double2;
  using AT = double2;
  static constexpr double tol = JACOBI_TOL;
  static constexpr bool dd = false;
  // vectors below 1e-14 ||theta||_F are rounding noise (unless zero_rel says otherwise)
  __device__ static R zero_level(const SvdDesc& P) {
    const double zr = P.zero_rel > 0.0 ? P.zero_rel : 1e-28;
    return fmax(zr * P.sig[P.n_vec + 1], 1e-290);
  }
  // the FP64 phase tracks the vector norms in sig[0, n_vec) for the tail rule
  static constexpr bool tracks_norms = true;
  __device__ static R wsum(R v) { return warp_sum(v); }
  __device__ static double2* X(const SvdDesc& P) { return P.X; }
  __device__ static double2* Acc(const SvdDesc& P) { return P.Acc; }
  __device__ static double2 mk(R a, R b) { return make_double2(a, b); }
  __device__ static CT mkc(R a, R b) { return make_double2(a, b); }
};
template <>
struct Prec<float4> {
  using R = double;
  using CT = double2;
  using AT = double2;
  static constexpr double tol = JACOBI_TOL;
  static constexpr bool dd = true;
  __device__ static R zero_level(const SvdDesc& P) { return 1e-28 * P.sig[P.n_vec + 1]; }
  static constexpr bool tracks_norms = true;
  __device__ static float4* X(const SvdDesc& P) { return reinterpret_cast<float4*>(P.X); }
  __device__ static double2* Acc(const SvdDesc& P) { return P.Acc; }
  __device__ static float4 mk(R, R) { return make_float4(0.f, 0.f, 0.f, 0.f); }  // zero only
  __device__ static CT mkc(R a, R b) { return make_double2(a, b); }
};
template <>
struct Prec<float2> {
  using R = float;
  using CT = float2;
  using AT = float2;
  static constexpr bool dd = false;
  static constexpr float tol = 2e-6f;  // above the FP32 rounding of the dot products
  // FP32 noise level: 1e-6 ||theta||_F (theta scaled by sig[n_vec] in this phase)
  __device__ static R zero_level(const SvdDesc& P) {
    const double sc = P.sig[P.n_vec];
    return (R)(1e-12 * P.sig[P.n_vec + 1] * sc * sc);
  }
  static constexpr bool tracks_norms = false;
  __device__ static R wsum(R v) { return warp_sumf(v); }
  __device__ static float2* X(const SvdDesc& P) { return P.X32; }
  __device__ static float2* Acc(const SvdDesc& P) { return P.Acc32; }
  __device__ static float2 mk(R a, R b) { return make_float2(a, b); }
  __device__ static CT mkc(R a, R b) { return make_float2(a, b); }
};



template <typename T>
__device__ inline void rot2(T* x, T* y, int n, int lane, typename Prec<T>::R cs, T m1, T m2) {
  // x' = cs x + m1 y ; y' = cs y + m2 x
  for (int i = lane; i < n; i += 32) {
    T u = x[i], v = y[i];
    T nu = Prec<T>::mk(cs * u.x + m1.x * v.x - m1.y * v.y, cs * u.y + m1.x * v.y + m1.y * v.x);
    T nv = Prec<T>::mk(cs * v.x + m2.x * u.x - m2.y * u.y, cs * v.y + m2.x * u.y + m2.y * u.x);
    x[i] = nu;
    y[i] = nv;
  }
}

// Rotation of two rows held in registers: each lane owns elements lane, lane+32, ...
template <typename T, int NR>
__device__ inline void rot_regs(T (&u)[NR], T (&v)[NR], typename Prec<T>::R cs, T m1, T m2) {
#pragma unroll
  for (int e = 0; e < NR; ++e) {
    const T a = u[e], b = v[e];
    u[e] = Prec<T>::mk(cs * a.x + m1.x * b.x - m1.y * b.y, cs * a.y + m1.x * b.y + m1.y * b.x);
    v[e] = Prec<T>::mk(cs * b.x + m2.x * a.x - m2.y * a.y, cs * b.y + m2.x * a.y + m2.y * a.x);
  }
}

// Loads, rotates and stores a pair of rows of length n <= 32 * NR in registers.
template <typename T, int NR>
__device__ inline void rot_rows_regs(T* x, T* y, int n, int lane, typename Prec<T>::R cs, T m1, T m2) {
  T u[NR], v[NR];
#pragma unroll
  for (int e = 0; e < NR; ++e) {
    const int i = lane + 32 * e;
    u[e] = i < n ? x[i] : Prec<T>::mk(0, 0);
    v[e] = i < n ? y[i] : Prec<T>::mk(0, 0);
  }
  rot_regs<T, NR>(u, v, cs, m1, m2);
#pragma unroll
  for (int e = 0; e < NR; ++e) {
    const int i = lane + 32 * e;
    if (i < n) {
      x[i] = u[e];
      y[i] = v[e];
    }
  }
}

// Rotation parameters of a pair from its Gram entries a = |x|^2, b = |y|^2,
// k = kr + i ki = <x, y>; false if the pair needs no rotation. `ratio`
// receives |k| / (|x| |y|), `tk` the norm change (|x|^2 -> a - tk, |y|^2 -> b + tk).
template <typename T>
__device__ inline bool jacobi_rotation(const SvdDesc& P, typename Prec<T>::R a, typename Prec<T>::R b,
                                       typename Prec<T>::R kr, typename Prec<T>::R ki, typename Prec<T>::R& cs,
                                       T& m1, T& m2, typename Prec<T>::R& tk, float& ratio) {
  using R = typename Prec<T>::R;
  const R ak = sqrt(kr * kr + ki * ki);
  const R ab = sqrt(a) * sqrt(b);  // not sqrt(a b): a b can underflow in FP32
  if (!(ak > Prec<T>::tol * ab)) return false;
  // a vector at rounding-noise level has a noise direction: leave it alone
  // (such values are dropped by the truncation's noise floor)
  if (a < Prec<T>::zero_level(P) || b < Prec<T>::zero_level(P)) return false;
  ratio = (float)(ak / ab);
  const R phr = kr / ak, phi = ki / ak;  // e^{i phi}
  const R zeta = (b - a) / (R(2) * ak);
  const R t = (zeta >= 0 ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
  cs = R(1) / sqrt(R(1) + t * t);
  const R sn = cs * t;
  tk = t * ak;
  // x' = cs x - sn e^{-i phi} y ; y' = sn e^{i phi} x + cs y
  m1 = Prec<T>::mk(-sn * phr, sn * phi);
  m2 = Prec<T>::mk(sn * phr, sn * phi);
  return true;
}

// jacobi_rotation plus the convergence bookkeeping of the sweep (lane 0)
template <typename T>
__device__ inline bool jacobi_params(const SvdDesc& P, typename Prec<T>::R a, typename Prec<T>::R b,
                                     typename Prec<T>::R kr, typename Prec<T>::R ki, int lane,
                                     typename Prec<T>::R& cs, T& m1, T& m2, typename Prec<T>::R& tk) {
  float ratio = 0.f;
  if (lane == 0) atomicAdd(P.rotated + 1, 1);  // pairs checked
  if (!jacobi_rotation<T>(P, a, b, kr, ki, cs, m1, m2, tk, ratio)) return false;
  if (lane == 0) {
    atomicAdd(P.rotated, 1);
    atomicMax(P.maxr, __float_as_uint(ratio));
  }
  return true;
}

// One Jacobi rotation: the lanes of a warp handle pair `pair` of round r of
// problem P. Rows of up to 512 elements stay in registers between the dot
// products and the rotation (one load, one store); longer rows stream.
template <typename T>
__device__ inline void jacobi_pair(const SvdDesc& P, int r, int pair, int lane) {
  using R = typename Prec<T>::R;
  constexpr int NR = 16;
  const int npad = P.n_vec + (P.n_vec & 1);
  if (npad < 2 || r >= npad - 1 || pair >= npad / 2) return;
  int p, q;
  if (pair == 0) {
    p = npad - 1;
    q = r;
  } else {
    p = (r + pair) % (npad - 1);
    q = (r - pair + (npad - 1)) % (npad - 1);
  }
  if (p > q) {
    int t = p;
    p = q;
    q = t;
  }
  if (q >= P.n_vec) return;
  if constexpr (Prec<T>::tracks_norms) {
    // tail rule: two vectors that both stay below the truncation threshold
    // need not be orthogonalised against each other (see svd_tail_threshold)
    const double tau = P.sig[P.n_vec + 2];
    if (tau > 0.0 && P.sig[p] < tau && P.sig[q] < tau) return;
  }
  T* X = Prec<T>::X(P);
  T* x = X + (int64_t)p * P.len;
  T* y = X + (int64_t)q * P.len;
  T* A = Prec<T>::Acc(P);
  T* ax = A + (int64_t)p * P.n_vec;
  T* ay = A + (int64_t)q * P.n_vec;
  R cs, tk;
  T m1, m2;
  R a = 0, b = 0, kr = 0, ki = 0;
  if (P.len <= 32 * NR) {
    T u[NR], v[NR];
#pragma unroll
    for (int e = 0; e < NR; ++e) {
      const int i = lane + 32 * e;
      u[e] = i < P.len ? x[i] : Prec<T>::mk(0, 0);
      v[e] = i < P.len ? y[i] : Prec<T>::mk(0, 0);
    }
#pragma unroll
    for (int e = 0; e < NR; ++e) {
      a += u[e].x * u[e].x + u[e].y * u[e].y;
      b += v[e].x * v[e].x + v[e].y * v[e].y;
      kr += u[e].x * v[e].x + u[e].y * v[e].y;  // conj(u) v
      ki += u[e].x * v[e].y - u[e].y * v[e].x;
    }
    a = Prec<T>::wsum(a);
    b = Prec<T>::wsum(b);
    kr = Prec<T>::wsum(kr);
    ki = Prec<T>::wsum(ki);
    if (!jacobi_params<T>(P, a, b, kr, ki, lane, cs, m1, m2, tk)) return;
    rot_regs<T, NR>(u, v, cs, m1, m2);
#pragma unroll
    for (int e = 0; e < NR; ++e) {
      const int i = lane + 32 * e;
      if (i < P.len) {
        x[i] = u[e];
        y[i] = v[e];
      }
    }
  } else {
    for (int i = lane; i < P.len; i += 32) {
      T u = x[i], v = y[i];
      a += u.x * u.x + u.y * u.y;
      b += v.x * v.x + v.y * v.y;
      kr += u.x * v.x + u.y * v.y;
      ki += u.x * v.y - u.y * v.x;
    }
    a = Prec<T>::wsum(a);
    b = Prec<T>::wsum(b);
    kr = Prec<T>::wsum(kr);
    ki = Prec<T>::wsum(ki);
    if (!jacobi_params<T>(P, a, b, kr, ki, lane, cs, m1, m2, tk)) return;
    rot2<T>(x, y, P.len, lane, cs, m1, m2);
  }
  if constexpr (Prec<T>::tracks_norms) {
    // no other warp touches p or q in this round
    if (lane == 0) {
      P.sig[p] = sqrt(fmax((double)(a - tk), 0.0));
      P.sig[q] = sqrt((double)(b + tk));
    }
  }
  if (P.n_vec <= 32 * NR) rot_rows_regs<T, NR>(ax, ay, P.n_vec, lane, cs, m1, m2);
  else rot2<T>(ax, ay, P.n_vec, lane, cs, m1, m2);
}

// Grid-wide barrier for a cooperative launch, with a bounded wait: returns
// false (and sets the status bit and the abort word, which makes every later
// barrier return at once) if the other blocks did not arrive in time.
// sync[0] = arrivals, sync[1] = generation, sync[3] = abort (sync[2]: unconverged
// problems, sync[4..5]: visit counters of the block sweeps).
__device__ inline bool grid_barrier(unsigned* sync, unsigned nblocks, int* status, long long spin_limit) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok_sh = 1;
    volatile unsigned* gen = sync + 1;
    volatile unsigned* abort_w = sync + 3;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(sync, 1u);
    if (arrived == nblocks - 1) {
      sync[0] = 0u;
      __threadfence();
      atomicAdd(sync + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == g) {
        if (*abort_w) {
          ok_sh = 0;
          break;
        }
        if (++spins > spin_limit) {
          ok_sh = 0;
          atomicOr(status, 32);
          atomicExch(sync + 3, 1u);
          break;
        }
        __nanosleep(64);
      }
    }
    if (*abort_w) ok_sh = 0;
    __threadfence();
  }
  __syncthreads();
  return ok_sh != 0;
}

// Tail rule of the FP64 phase. After the FP32 phase the vectors are mutually
// orthogonal to FP32 accuracy and their norms nu_i approximate the singular
// values. The truncation keeps at most k* of them (k* computed below from the
// nu with safety margins), so every vector whose norm stays below
// tau = nu_(k*) / 2 is discarded. A rotation between two such vectors changes
// neither the kept vectors nor the discarded weight (it conserves the sum of
// their squared norms), so the FP64 phase skips those pairs and orthogonalises
// every other pair to FP64 accuracy: all vectors above tau end as singular
// vectors of the FP64 iterate. A vector below tau only shrinks in a rotation
// with a larger partner, so it stays below. k* over-estimates the final rank:
// tail sums of the nu^2 (the diagonal of a unitary transform of Theta Theta^H,
// majorised by the sigma^2) over-estimate the true ones, the weight test uses
// w_max / 4 and the eps and noise tests half their thresholds. svd_truncate
// flags (status bit 64) a kept value below tau; the sweeps check the rule at
// convergence and drop it (tau = 0) if it failed.
// tau = 0 (no skipping) when the whole spectrum is returned. Also writes the
// order of decreasing norm to perm (the FP64 block sweeps group the vectors
// in that order, so that the tail forms whole blocks).
constexpr int SVD_TAIL_MAX = 6144;  // vectors; the sorted norms live in shared memory
__global__ void svd_tail_threshold(const __grid_constant__ SvdBatch B) {
  extern __shared__ double srt[];
  __shared__ int has_nan;
  const SvdDesc& P = B.d[blockIdx.x];
  const int n = P.n_vec;
  if (n > SVD_TAIL_MAX) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) P.perm[i] = i;
    if (threadIdx.x == 0) P.sig[n + 2] = 0.0;
    return;
  }
  if (threadIdx.x == 0) has_nan = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    P.perm[i] = i;
    if (!(P.sig[i] == P.sig[i])) has_nan = 1;
  }
  __syncthreads();
  if (has_nan) {
    if (threadIdx.x == 0) P.sig[n + 2] = 0.0;
    return;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double si = P.sig[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double sj = P.sig[j];
      rank += (sj > si) || (sj == si && j < i);
    }
    srt[rank] = si;
    P.perm[rank] = i;  // the block sweeps visit the vectors in this order
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double tau = 0.0;
  if (srt[0] > 0.0 && P.s_sorted == nullptr) {
    const double s0 = srt[0];
    int kw = n;  // smallest k >= 1 with sum_{j >= k} nu_j^2 <= w_max / 4
    double acc = 0.0;
    for (int k = n - 1; k >= 1; --k) {
      acc += srt[k] * srt[k];
      if (acc <= 0.25 * P.w_max) kw = k;
      else break;
    }
    const double thr = 0.5 * fmax(P.eps * s0, 1e-14 * sqrt(P.sig[n + 1]));
    int ne = 0;
    for (int k = 0; k < n; ++k) ne += srt[k] > thr;
    int ks = kw < P.chi_max ? kw : P.chi_max;
    if (ne < ks) ks = ne;
    if (ks < 1) ks = 1;
    // only where the FP32 phase resolved the norms: well above its noise
    // level (vectors below 1e-6 ||theta||_F are not rotated there)
    if (ks < n && 0.5 * srt[ks] >= 1e-5 * sqrt(P.sig[n + 1])) tau = 0.5 * srt[ks];
  }
  P.sig[n + 2] = tau;
}

// Whether the tail rule held at convergence: the truncation keeps only vectors
// above tau (at least chi_max of them lie above it, or every vector below it
// fails the eps / noise test, or their squared norms sum to at most w_max --
// the three ways svd_truncate can stop before reaching them). Uses the norms
// tracked by the sweeps. One thread.
__device__ inline bool svd_tail_rule_holds(const SvdDesc& P) {
  const int n = P.n_vec;
  const double tau = P.sig[n + 2];
  if (!(tau > 0.0)) return true;
  int cnt = 0;
  double s0 = 0.0, below_max = 0.0, below_w = 0.0;
  for (int i = 0; i < n; ++i) {
    const double si = P.sig[i];
    s0 = fmax(s0, si);
    if (si >= tau) {
      ++cnt;
    } else {
      below_max = fmax(below_max, si);
      below_w += si * si;
    }
  }
  if (cnt >= P.chi_max) return true;
  const double thr = fmax(P.eps * s0, 1e-14 * sqrt(P.sig[n + 1]));
  return below_max <= thr || below_w <= P.w_max;
}

// End of a sweep (one thread): marks the problems whose sweep applied no
// rotation or whose largest relative off-diagonal stayed below `stop` as
// converged, resets the per-sweep counters and stores the number of
// unconverged problems in sync[2].
template <typename T>
__device__ inline void sweep_end(const SvdBatch& B, float stop, double* work_flops, int acc_in_phase) {
  unsigned cnt = 0;
  for (int i = 0; i < B.n; ++i) {
    const SvdDesc& P = B.d[i];
    if (!*P.conv) {
      // arithmetic of this sweep in the phase's precision, counted as in the
      // rotation form: the cross product <x, y> of every pair checked (8 flops
      // per element), the rotation of the vectors (20 per element) and, when it
      // runs in this precision, of the rows of Acc (the Gram form of the FP32
      // phase does the same work as dense block products)
      if (work_flops) {
        const double per_rot = 20.0 * P.len + (acc_in_phase ? 20.0 * P.n_vec : 0.0);
        work_flops[0] += 8.0 * P.len * (double)P.rotated[1] + per_rot * (double)P.rotated[0];
        work_flops[1] += 1.0;  // sweeps, summed over the problems of the batch
      }
      bool done = P.rotated[0] == 0 || __uint_as_float(*P.maxr) < stop;
      if constexpr (Prec<T>::tracks_norms) {
        // the estimate behind the tail rule failed: drop the rule and
        // sweep on until every pair is orthogonal
        if (done && !svd_tail_rule_holds(P)) {
          P.sig[P.n_vec + 2] = 0.0;
          done = false;
        }
      }
      if (done) *P.conv = 1;
      else ++cnt;
    }
    P.rotated[0] = P.rotated[1] = 0;
    *P.maxr = 0u;
  }
  *(volatile unsigned*)(B.sync + 2) = cnt;
  __threadfence_system();
}

// All sweeps of one phase in one cooperative launch: rounds separated by grid
// barriers, warps striding over the pairs of all problems; after each sweep
// block 0 marks converged problems (no rotation, or the largest relative
// off-diagonal below `stop`) and the loop ends when all are converged.
// sync[2] = unconverged count of the last sweep.
template <typename T>
__global__ void __launch_bounds__(SVD_WARPS * 32) svd_sweeps(const __grid_constant__ SvdBatch B, int npad_max,
                                                            float stop, int max_sweeps, int fatal,
                                                            double* work_flops) {
  __shared__ int off[MAXB + 1];
  if (threadIdx.x == 0) {
    off[0] = 0;
    for (int i = 0; i < B.n; ++i) {
      const int n = B.d[i].n_vec;
      off[i + 1] = off[i] + (n + (n & 1)) / 2;
    }
  }
  __syncthreads();
  const int total = off[B.n];
  const int wpb = blockDim.x / 32;
  const int gw = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int nw = gridDim.x * wpb;
  const int lane = threadIdx.x & 31;
  volatile unsigned* unconv = B.sync + 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int r = 0; r < npad_max - 1; ++r) {
      for (int w = gw; w < total; w += nw) {
        int pid = 0;
        while (w >= off[pid + 1]) ++pid;
        const SvdDesc& P = B.d[pid];
        if (*(volatile int*)P.conv) continue;
        jacobi_pair<T>(P, r, w - off[pid], lane);
      }
      if (!grid_barrier(B.sync, gridDim.x, B.status, B.spin_limit)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) sweep_end<T>(B, stop, work_flops, 1);
    if (!grid_barrier(B.sync, gridDim.x, B.status, B.spin_limit)) return;
    if (*unconv == 0) return;
  }
  if (fatal && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(B.status, 16);
}


// ---------------------------------------------------------------------------
// Block Jacobi. The vectors are grouped into blocks of W and the blocks are
// paired round-robin (nb - 1 block rounds per sweep, a grid barrier between
// rounds). A CTA of W warps takes one pair of blocks at a time: it loads the
// 2W vectors into shared memory and rotates them there -- in the first block
// round of a sweep the pairs inside each block, then in every block round the
// W^2 pairs across the two blocks, in local rounds of W disjoint pairs, a warp
// per pair -- so each pair of vectors is visited once per sweep, as in the
// scalar order, while each vector crosses global memory once per W of its
// pairs. The squared norms are computed once per visit and then updated from
// the rotations, so a pair only needs its cross product. The rotations are
// recorded and replayed on the 2W rows of Acc afterwards, a thread per column
// with the column in registers. Vectors of at most 512 elements.
// ---------------------------------------------------------------------------
template <typename T, int W>
struct BlockCfg {
  static constexpr int THREADS = 32 * W;  // a warp per pair of a local round
  static constexpr int LMAX = 512;        // longest vector held in shared memory
  static constexpr int EPT = LMAX / 32;   // elements of each vector per lane
  static constexpr int MAX_STEPS = (W - 1) + W;
  static_assert(W % 2 == 0 && W >= 2, "block shape");
};

template <typename T>
struct RotRec {
  typename Prec<T>::R cs;
  typename Prec<T>::CT m1, m2;  // identity rotation: cs = 1, m1 = m2 = 0
  // FP32 copies for the accumulation of the block rotation in FP32 (cm1 = cs - 1),
  // and the low parts that make (cm1, m1, m2) double-float
  float cm1;
  float2 m1f, m2f;
  float cm1l;
  float2 m1l, m2l;
};


// Round-robin pairing of n_even items: pair `k` of round `r` (0 <= r < n_even - 1).
__host__ __device__ constexpr void rr_pair(int n_even, int r, int k, int& p, int& q) {
  p = k == 0 ? n_even - 1 : (r + k) % (n_even - 1);
  q = k == 0 ? r : (r - k + (n_even - 1)) % (n_even - 1);
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

// Rotation parameters with few FP64 operations: the angle's tangent is found
// in FP32 from the FP64 Gram entries, the rotation built from it is unitary
// to FP64 rounding (cs = 1/sqrt(1 + t^2), |e^{i phi}| = 1 in FP64). A tangent
// off by the FP32 rounding leaves a relative off-diagonal of ~1e-7 of the one
// removed, which the quadratic convergence of the sweeps absorbs. Returns
// false when the pair needs no rotation; a2, b2 receive the new squared norms.
template <typename T>
__device__ inline bool jacobi_rotation_fast(typename Prec<T>::R tol2, typename Prec<T>::R zl, typename Prec<T>::R a,
                                            typename Prec<T>::R b,
                                            typename Prec<T>::R kr, typename Prec<T>::R ki, RotRec<T>& rec,
                                            typename Prec<T>::R& a2, typename Prec<T>::R& b2, float& ratio) {
  using R = typename Prec<T>::R;
  const R k2 = kr * kr + ki * ki;
  if (!(k2 > tol2 * a * b)) return false;  // tol2: squared relative tolerance
  if (a < zl || b < zl) return false;      // zl: Prec<T>::zero_level
  const R rk = rsqrt(k2);
  const R ak = k2 * rk;
  ratio = (float)ak * rsqrtf((float)a) * rsqrtf((float)b);
  const float zf = (float)((b - a) * (R(0.5) * rk));
  // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)); 1 / (2 |zeta|) where zeta^2
  // would overflow (strongly graded pairs: tiny but necessary rotations)
  const float az = fabsf(zf);
  const float tf = copysignf(az > 1e18f ? 0.5f / az : 1.0f / (az + sqrtf(1.0f + az * az)), zf);
  const R t = (R)tf;
  const R cs = rsqrt(R(1) + t * t);
  const R sn = cs * t;
  const R phr = kr * rk, phi = ki * rk;
  // x' = cs x - sn e^{-i phi} y ; y' = sn e^{i phi} x + cs y
  rec.cs = cs;
  rec.m1 = Prec<T>::mkc(-sn * phr, sn * phi);
  rec.m2 = Prec<T>::mkc(sn * phr, sn * phi);
  // |x'|^2 = cs^2 (a + t^2 b - 2 t |k|), |y'|^2 = cs^2 (b + t^2 a + 2 t |k|)
  const R c2 = cs * cs;
  a2 = c2 * (a + t * t * b - R(2) * t * ak);
  b2 = c2 * (b + t * t * a + R(2) * t * ak);
  return true;
}

// x' = cs x + m1 y, y' = cs y + m2 x with m2 = (-re m1, im m1) (the rotation
// is unitary: m2 = -conj(m1)), so only cs and m1 are read
template <typename T>
__device__ inline void apply_rot(T& u, T& v, const RotRec<T>& r) {
  const T x = u, y = v;
  const auto m1x = r.m1.x, m1y = r.m1.y, m2x = -r.m1.x;
  u = Prec<T>::mk(r.cs * x.x + m1x * y.x - m1y * y.y, r.cs * x.y + m1x * y.y + m1y * y.x);
  v = Prec<T>::mk(r.cs * y.x + m2x * x.x - m1y * x.y, r.cs * y.y + m2x * x.y + m1y * x.x);
}

// Cross product <x, y> of two vectors in shared memory, summed over the warp.
template <typename T, int W>
__device__ inline void block_cross(const T* x, const T* y, int lane, typename Prec<T>::R& kr,
                                   typename Prec<T>::R& ki) {
  using C = BlockCfg<T, W>;
  using R = typename Prec<T>::R;
  if constexpr (Prec<T>::dd) {
    // compensated sums (the leading products exact, the rest in FP32): the
    // result carries ~48 bits, as if summed in double-float. Packed (re, im)
    // lanes: (sr, si) += (re u, re u) (re v, im v), then (sr, si) +=
    // (im u, -im u) (im v, re v) -- per lane the operations and the order of
    // four scalar accumulations
    f32x2 acc_s = 0ull, acc_c = 0ull;
#pragma unroll 4
    for (int i = 0; i < C::EPT; ++i) {
      const float4 u = x[lane + 32 * i], v = y[lane + 32 * i];
      dd_acc2(acc_s, acc_c, pk2(u.x, u.x), pk2(-u.x, -u.x), pk2(u.z, u.z), pk2(v.x, v.y), pk2(v.z, v.w));
      dd_acc2(acc_s, acc_c, pk2(u.y, -u.y), pk2(-u.y, u.y), pk2(u.w, -u.w), pk2(v.y, v.x), pk2(v.w, v.z));
    }
    float sr, si, cr, ci;
    {
      const float2 sv = upk2(acc_s), cv = upk2(acc_c);
      sr = sv.x;
      si = sv.y;
      cr = cv.x;
      ci = cv.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float s2 = __shfl_xor_sync(0xffffffffu, sr, o), c2 = __shfl_xor_sync(0xffffffffu, cr, o);
      const float s3 = __shfl_xor_sync(0xffffffffu, si, o), c3 = __shfl_xor_sync(0xffffffffu, ci, o);
      float t;
      two_sum(sr, s2, sr, t);
      cr += c2 + t;
      two_sum(si, s3, si, t);
      ci += c3 + t;
    }
    kr = (R)sr + (R)cr;
    ki = (R)si + (R)ci;
  } else {
    R a = 0, b = 0;
#pragma unroll
    for (int i = 0; i < C::EPT; ++i) {
      const T u = x[lane + 32 * i], v = y[lane + 32 * i];
      a += u.x * v.x + u.y * v.y;  // conj(u) v
      b += u.x * v.y - u.y * v.x;
    }
    kr = Prec<T>::wsum(a);
    ki = Prec<T>::wsum(b);
  }
}

// dd_axpy3 on packed (re, im) lanes: s, c = hi, lo of x; term k is
// (ph_k, pl_k) (qh_k, ql_k) with nph_k = -ph_k
__device__ inline void dd_axpy3_2(f32x2 s, f32x2 c, f32x2 p1h, f32x2 n1h, f32x2 p1l, f32x2 q1h, f32x2 q1l,
                                  f32x2 p2h, f32x2 n2h, f32x2 p2l, f32x2 q2h, f32x2 q2l, f32x2 p3h, f32x2 n3h,
                                  f32x2 p3l, f32x2 q3h, f32x2 q3l, float4& o) {
  dd_acc2(s, c, p1h, n1h, p1l, q1h, q1l);
  dd_acc2(s, c, p2h, n2h, p2l, q2h, q2l);
  dd_acc2(s, c, p3h, n3h, p3l, q3h, q3l);
  // fast_two_sum(s, c) per lane
  const f32x2 oh = add2(s, c);
  const f32x2 ol = sub2(c, sub2(oh, s));
  const float2 h = upk2(oh), l = upk2(ol);
  o = make_float4(h.x, h.y, l.x, l.y);
}

// o = x + sum_k p_k q_k in double-float (x, p_k, q_k given as hi/lo pairs)
__device__ inline void dd_axpy3(float xh, float xl, float p1h, float p1l, float q1h, float q1l, float p2h,
                                float p2l, float q2h, float q2l, float p3h, float p3l, float q3h, float q3l,
                                float& oh, float& ol) {
  float s = xh, c = xl;
  dd_acc(s, c, p1h, p1l, q1h, q1l);
  dd_acc(s, c, p2h, p2l, q2h, q2l);
  dd_acc(s, c, p3h, p3l, q3h, q3l);
  fast_two_sum(s, c, oh, ol);
}

template <typename T>
struct RotOut {
  RotRec<T> rec;
  int rot;
};

// One local round: warp w rotates local vectors (lp, lq); every thread of the
// CTA calls it (it ends with a barrier).
template <typename T, int W>
__device__ inline void block_local_round(typename Prec<T>::R tol2, typename Prec<T>::R zl, T* xs,
                                         typename Prec<T>::R* nrm, RotRec<T>* seq, int slot, const int* vrows,
                                         int lp, int lq, double tau, int* n_rot, unsigned* maxr_bits) {
  using C = BlockCfg<T, W>;
  using R = typename Prec<T>::R;
  const int lane = threadIdx.x & 31;
  bool active = vrows[lp] >= 0 && vrows[lq] >= 0;
  if constexpr (Prec<T>::tracks_norms) {
    // tail rule: both vectors below the threshold -- not even the product is needed
    if (active && tau > 0.0 && (double)nrm[lp] < tau * tau && (double)nrm[lq] < tau * tau) active = false;
  }
  T* x = xs + lp * C::LMAX;
  T* y = xs + lq * C::LMAX;
  R kr = 0, ki = 0;
  if (active) block_cross<T, W>(x, y, lane, kr, ki);
  RotRec<T> rec;
  int rot = 0;
  // the parameters of one pair: lane `who` of the calling warp, with (lp, lq), kr, ki
  auto params = [&](int plp, int plq, R pkr, R pki, bool pact) {
    RotRec<T> r;
    r.cs = 1;
    r.m1 = r.m2 = Prec<T>::mkc(0, 0);
    r.cm1 = r.cm1l = 0.f;
    r.m1f = r.m2f = r.m1l = r.m2l = make_float2(0.f, 0.f);
    int did = 0;
    if (pact) {
      const R a = nrm[plp], b = nrm[plq];
      R a2, b2;
      float ratio = 0.f;
      atomicAdd(n_rot + 1, 1);  // pairs checked
      if (jacobi_rotation_fast<T>(tol2, zl, a, b, pkr, pki, r, a2, b2, ratio)) {
        did = 1;
        r.cm1 = (float)(r.cs - R(1));
        r.m1f = make_float2((float)r.m1.x, (float)r.m1.y);
        r.m2f = make_float2((float)r.m2.x, (float)r.m2.y);
        if constexpr (Prec<T>::dd) {
          r.cm1l = (float)((double)(r.cs - R(1)) - (double)r.cm1);
          r.m1l = make_float2((float)((double)r.m1.x - (double)r.m1f.x), (float)((double)r.m1.y - (double)r.m1f.y));
          r.m2l = make_float2((float)((double)r.m2.x - (double)r.m2f.x), (float)((double)r.m2.y - (double)r.m2f.y));
        }
        nrm[plp] = a2;
        nrm[plq] = b2;
        atomicAdd(n_rot, 1);
        atomicMax(maxr_bits, __float_as_uint(ratio));
      }
    }
    return RotOut<T>{r, did};
  };
  if constexpr (std::is_same<R, double>::value) {
    // FP64 parameters (a few dozen FP64 instructions, each occupying the FP64
    // pipe for a whole warp): one warp computes those of all W pairs of the
    // round, its lanes in parallel, instead of one lane in every warp
    __shared__ double2 pk[W];
    __shared__ int ppq[W], prot[W];
    const int warp = threadIdx.x >> 5;
    if (lane == 0) {
      pk[warp] = make_double2((double)kr, (double)ki);
      ppq[warp] = active ? (lp | (lq << 8)) : -1;
    }
    __syncthreads();
    if (warp == 0 && lane < W) {
      const int pq = ppq[lane];
      const auto res = params(pq & 255, (pq >> 8) & 255, (R)pk[lane].x, (R)pk[lane].y, pq >= 0);
      seq[slot - warp + lane] = res.rec;
      prot[lane] = res.rot;
    }
    __syncthreads();
    rot = prot[warp];
    if (rot) rec = seq[slot];
  } else {
    if (lane == 0) {
      const auto res = params(lp, lq, kr, ki, active);
      rec = res.rec;
      rot = res.rot;
      seq[slot] = rec;
    }
  }
  rot = __shfl_sync(0xffffffffu, rot, 0);
  if (rot) {
    if constexpr (Prec<T>::dd) {
      // x' = x + [(cs - 1) x + m1 y], y' = y + [(cs - 1) y + m2 x] in double-float;
      // every lane holds the record (read from shared memory)
      const float2 c1 = make_float2(rec.cm1, rec.cm1l);
      const float2 a1 = make_float2(rec.m1f.x, rec.m1l.x), b1 = make_float2(rec.m1f.y, rec.m1l.y);
      const float2 a2 = make_float2(rec.m2f.x, rec.m2l.x), b2 = make_float2(rec.m2f.y, rec.m2l.y);
      // the (re, im) lanes packed: term 1 (cs - 1) x, term 2 m re-part times y,
      // term 3 (-im m, im m) times (im y, re y)
      const f32x2 c1h = pk2(c1.x, c1.x), c1n = pk2(-c1.x, -c1.x), c1l = pk2(c1.y, c1.y);
      const f32x2 a1h = pk2(a1.x, a1.x), a1n = pk2(-a1.x, -a1.x), a1l = pk2(a1.y, a1.y);
      const f32x2 b1h = pk2(-b1.x, b1.x), b1n = pk2(b1.x, -b1.x), b1l = pk2(-b1.y, b1.y);
      const f32x2 a2h = pk2(a2.x, a2.x), a2n = pk2(-a2.x, -a2.x), a2l = pk2(a2.y, a2.y);
      const f32x2 b2h = pk2(-b2.x, b2.x), b2n = pk2(b2.x, -b2.x), b2l = pk2(-b2.y, b2.y);
#pragma unroll 2
      for (int i = 0; i < C::EPT; ++i) {
        const float4 u = x[lane + 32 * i], v = y[lane + 32 * i];
        const f32x2 uh = pk2(u.x, u.y), ul = pk2(u.z, u.w), vh = pk2(v.x, v.y), vl = pk2(v.z, v.w);
        const f32x2 uhs = pk2(u.y, u.x), uls = pk2(u.w, u.z), vhs = pk2(v.y, v.x), vls = pk2(v.w, v.z);
        float4 nu, nv;
        // re x' = re u + c1 re u + a1 re v - b1 im v ; im x' = im u + c1 im u + a1 im v + b1 re v
        dd_axpy3_2(uh, ul, c1h, c1n, c1l, uh, ul, a1h, a1n, a1l, vh, vl, b1h, b1n, b1l, vhs, vls, nu);
        // re y' = re v + c1 re v + a2 re u - b2 im u ; im y' = im v + c1 im v + a2 im u + b2 re u
        dd_axpy3_2(vh, vl, c1h, c1n, c1l, vh, vl, a2h, a2n, a2l, uh, ul, b2h, b2n, b2l, uhs, uls, nv);
        x[lane + 32 * i] = nu;
        y[lane + 32 * i] = nv;
      }
    } else {
      rec.cs = __shfl_sync(0xffffffffu, rec.cs, 0);
      rec.m1.x = __shfl_sync(0xffffffffu, rec.m1.x, 0);
      rec.m1.y = __shfl_sync(0xffffffffu, rec.m1.y, 0);
#pragma unroll
      for (int i = 0; i < C::EPT; ++i) {
        T u = x[lane + 32 * i], v = y[lane + 32 * i];
        apply_rot<T>(u, v, rec);
        x[lane + 32 * i] = u;
        y[lane + 32 * i] = v;
      }
    }
  }
  __syncthreads();
}

// Replays the recorded rotations on the 2W rows of Acc (a thread per column).
template <typename T, int W>
__device__ inline void block_replay_acc(const SvdDesc& P, const int* vrows, const RotRec<T>* seq, bool intra,
                                        bool cross) {
  using C = BlockCfg<T, W>;
  T* A = Prec<T>::Acc(P);
  const int n = P.n_vec;
  for (int c = threadIdx.x; c < n; c += C::THREADS) {
    T acc[2 * W];
#pragma unroll
    for (int k = 0; k < 2 * W; ++k) {
      const int r = vrows[k];
      acc[k] = r >= 0 ? A[(int64_t)r * n + c] : Prec<T>::mk(0, 0);
    }
    int base = 0;
    if (intra) {
#pragma unroll
      for (int rr = 0; rr < W - 1; ++rr) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
          int p = 0, q = 0;
          rr_pair(W, rr, w % (W / 2), p, q);
          const int o = w < W / 2 ? 0 : W;
          const RotRec<T>& rec = seq[rr * W + w];
          apply_rot<T>(acc[p + o], acc[q + o], rec);
        }
      }
      base = (W - 1) * W;
    }
    if (cross) {
#pragma unroll
      for (int rr = 0; rr < W; ++rr) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
          const RotRec<T>& rec = seq[base + rr * W + w];
          apply_rot<T>(acc[w], acc[W + (w + rr) % W], rec);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 2 * W; ++k) {
      const int r = vrows[k];
      if (r >= 0) A[(int64_t)r * n + c] = acc[k];
    }
  }
}

// The visit's rotations as one 2W x 2W matrix G = I + D, D accumulated in FP32
// (a thread per column of D, lanes 0 .. 2W-1 of warp 0), then
// Acc rows <- Acc rows + D Acc rows with D Acc in FP32. The rotations of the
// FP64 sweeps are small (the FP32 phase has done the large ones), so D's
// FP32 rounding stays ~1e-9 and Acc keeps the accuracy of the mixed mode at a
// small fraction of the FP64 work of replaying every rotation.
template <typename T, int W>
__device__ inline void block_correct_acc(const SvdDesc& P, const int* vrows, const RotRec<T>* seq, bool intra,
                                         bool cross, float2* D) {
  using C = BlockCfg<T, W>;
  constexpr int N2 = 2 * W;
  const int tid = threadIdx.x;
  if (tid < N2) {
    const int j = tid;
    float2 col[N2];
#pragma unroll
    for (int k = 0; k < N2; ++k) col[k] = make_float2(0.f, 0.f);
    auto rot = [&](float2& u, float2& v, int p, int q, const RotRec<T>& r) {
      // rows p, q of I + D: (e_p + D_p, e_q + D_q) -> rotated, identity parts kept exact
      const float cs = 1.0f + r.cm1;
      const float2 a = u, b = v;
      float2 nu = make_float2(cs * a.x + r.m1f.x * b.x - r.m1f.y * b.y, cs * a.y + r.m1f.x * b.y + r.m1f.y * b.x);
      float2 nv = make_float2(cs * b.x + r.m2f.x * a.x - r.m2f.y * a.y, cs * b.y + r.m2f.x * a.y + r.m2f.y * a.x);
      if (j == p) {
        nu.x += r.cm1;
        nv.x += r.m2f.x;
        nv.y += r.m2f.y;
      }
      if (j == q) {
        nv.x += r.cm1;
        nu.x += r.m1f.x;
        nu.y += r.m1f.y;
      }
      u = nu;
      v = nv;
    };
    int base = 0;
    if (intra) {
#pragma unroll
      for (int rr = 0; rr < W - 1; ++rr) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
          int p = 0, q = 0;
          rr_pair(W, rr, w % (W / 2), p, q);
          const int o = w < W / 2 ? 0 : W;
          rot(col[p + o], col[q + o], p + o, q + o, seq[rr * W + w]);
        }
      }
      base = (W - 1) * W;
    }
    if (cross) {
#pragma unroll
      for (int rr = 0; rr < W; ++rr) {
#pragma unroll
        for (int w = 0; w < W; ++w) rot(col[w], col[W + (w + rr) % W], w, W + (w + rr) % W, seq[base + rr * W + w]);
      }
    }
#pragma unroll
    for (int k = 0; k < N2; ++k) D[k * N2 + j] = col[k];
  }
  __syncthreads();
  using AT = typename Prec<T>::AT;
  AT* A = Prec<T>::Acc(P);
  const int n = P.n_vec;
  for (int c = tid; c < n; c += C::THREADS) {
    float2 af[N2];
#pragma unroll
    for (int k = 0; k < N2; ++k) {
      const int r = vrows[k];
      const AT a = r >= 0 ? A[(int64_t)r * n + c] : AT{};
      af[k] = make_float2((float)a.x, (float)a.y);
    }
#pragma unroll
    for (int k = 0; k < N2; ++k) {
      const int r = vrows[k];
      if (r < 0) continue;
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int jj = 0; jj < N2; ++jj) {
        const float2 d = D[k * N2 + jj];
        s.x = fmaf(d.x, af[jj].x, fmaf(-d.y, af[jj].y, s.x));
        s.y = fmaf(d.x, af[jj].y, fmaf(d.y, af[jj].x, s.y));
      }
      AT a = A[(int64_t)r * n + c];
      a.x += s.x;
      a.y += s.y;
      A[(int64_t)r * n + c] = a;
    }
  }
}

// ---------------------------------------------------------------------------
// Gram form of a visit (the FP32 phase). The rotations of a visit need only
// the norms and cross products of its 2W vectors, i.e. the Hermitian Gram
// matrix G = X^H X of the block pair (G[a][b] = <x_a, x_b>). It is formed once
// per visit, in one pass over the vectors; the rotations -- the same pairs in
// the same order as in the rotation form above -- are found from G and applied
// to G (G <- J^H G J, a 2 x 2 block of pairs per thread) and to the visit's
// rotation Q (Q <- Q J, from the identity); the vectors and the rows of Acc
// are then updated once, x_j <- sum_k Q[k][j] x_k, by register-tiled products.
// The work per pair that grows with the vector length (a cross product and a
// rotation of two vectors, a rotation of two rows of Acc) becomes three dense
// products per visit, and only O(W) work per pair stays in the chain of
// dependent rotations. In exact arithmetic this is the rotation form's visit;
// in FP32, G is updated rather than recomputed between the rotations, which
// changes them at the level of FP32 rounding -- the phase is a preconditioner
// whose rotation is made unitary and whose vectors are recomputed in FP64
// afterwards. W = 16: 32 vectors, 512 threads.
// ---------------------------------------------------------------------------

struct GramRot {
  float cs;
  float2 m1, m2;
  int rot;
};

constexpr int GSTEPS = GV - 1;  // local rounds: W - 1 inside the blocks, W across them

struct __align__(16) GramShared {
  float2 G[GV][GV];
  float2 Q[GV][GV];
  float2 QS[GV][GV];                     // i Q = (-im Q, re Q), for the packed products
  GramRot rr[GV / 2];                    // the rotations of the current local round
  unsigned char pq[GSTEPS][GV / 2][2];   // the pairs (p < q) of each local round
  unsigned char tile[36][2];  // the 4 x 4 tiles (ti <= tj) of G formed by the warps
  unsigned char blk[120][2];  // the pairs of pairs (u < v) whose 2 x 2 blocks the rotations update
  int vrows[GV];
  int n_rot;
};

// Pair w of local round rr: the pairs inside each of the two blocks (intra) or
// across them, as in the rotation form.
template <int W>
__device__ inline void gram_pair(bool intra, int rr, int w, int& p, int& q) {
  if (intra) {
    rr_pair(W, rr, w % (W / 2), p, q);
    if (w >= W / 2) {
      p += W;
      q += W;
    }
  } else {
    p = w;
    q = W + (w + rr) % W;
  }
}

// Sums v[0 .. 31] over the lanes of a warp by recursive halving; lane l returns
// the total of v[l].
__device__ inline float warp_reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = up ? v[i] : v[i + h];
      const float keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  return v[0];
}

__device__ inline float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ inline float2 cmulc(float2 a, float2 b) {  // conj(a) b
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ inline float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ inline float2 cscale(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__device__ inline float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }


// out_j = sum_k Q[k][j] in_k for the GV rows of `rows` (ncols <= 512 columns,
// row stride 512), written to dst[vrows[j] * stride + c] for the present rows.
// A thread holds 4 rows x 4 columns of the result (columns c, c + 64, c + 128,
// c + 192 of a half of 256 columns); the halves are done one after the other.
// `between` runs after the last read of `rows` (all threads have passed a
// barrier), before the second half's results are stored.
// out_j = sum_k Q[k][j] in_k for the GV rows of `rows` (ncols <= 512 columns,
// row stride 512), written to dst[vrows[j] * stride + c] for the present rows.
// A thread holds 4 rows x 4 columns of the result (columns c, c + 64, c + 128,
// c + 192 of a half of 256 columns); the halves are done one after the other.
// A complex multiply-add is two packed FMAs: out += (re x, re x) (re q, im q)
// + (im x, im x) (-im q, re q), the second factors read from Q and QS.
// `between` runs after the last read of `rows` (all threads have passed a
// barrier), before the second half's results are stored.
template <typename F>
__device__ inline void gram_apply_q(const float2* rows, const GramShared& S, int ncols, float2* dst, int stride,
                                    F&& between) {
  constexpr int LMAX = 512;
  const int tid = threadIdx.x;
  const int cg = tid & 63, rg = tid >> 6;
  for (int half = 0; half < 2; ++half) {
    const int c0 = 256 * half + cg;
    const int nu = ncols > c0 ? min(4, (ncols - c0 + 63) >> 6) : 0;
    f32x2 acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[j][u] = 0ull;
    if (256 * half < ncols) {
#pragma unroll 4
      for (int k = 0; k < GV; ++k) {
        float2 x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = rows[k * LMAX + c0 + 64 * u];
        const ulonglong2* qk = reinterpret_cast<const ulonglong2*>(&S.Q[k][4 * rg]);
        const ulonglong2* sk = reinterpret_cast<const ulonglong2*>(&S.QS[k][4 * rg]);
        const ulonglong2 q01 = qk[0], q23 = qk[1], s01 = sk[0], s23 = sk[1];
        const f32x2 q[4] = {q01.x, q01.y, q23.x, q23.y}, qs[4] = {s01.x, s01.y, s23.x, s23.y};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const f32x2 xr = pk2(x[u].x, x[u].x), xi = pk2(x[u].y, x[u].y);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            fma2(acc[j][u], xr, q[j]);
            fma2(acc[j][u], xi, qs[j]);
          }
        }
      }
    }
    if (half == 1) {
      __syncthreads();  // every thread is done reading `rows`
      between();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = S.vrows[4 * rg + j];
      if (r < 0) continue;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (u < nu) dst[(int64_t)r * stride + c0 + 64 * u] = upk2(acc[j][u]);
    }
  }
}

// Loads the GV rows `vrows` of src (row stride `stride`, `ncols` columns) into
// `rows` (row stride 512), zero for columns in [ncols, ncols_pad) and for
// absent rows; 16-byte asynchronous copies (cp.async, zero-filled where there
// is no source) when ncols and stride are even, else plain loads. Ends with
// the copies complete and a barrier.
__device__ inline void gram_load_rows(float2* rows, const float2* src, const int* vrows, int ncols, int ncols_pad,
                                      int stride) {
  constexpr int LMAX = 512;
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (((ncols | stride) & 1) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    const int nch = (ncols_pad + 1) >> 1;  // 16-byte chunks per row
    for (int i = tid; i < GV * nch; i += nthr) {
      const int k = i / nch, ch = i - k * nch;
      const int r = vrows[k];
      const bool have = r >= 0 && 2 * ch < ncols;
      const float2* g = have ? src + (int64_t)r * stride + 2 * ch : src;
      const uint32_t d = (uint32_t)__cvta_generic_to_shared(rows + k * LMAX + 2 * ch);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(g), "r"(have ? 16 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  } else {
    for (int i = tid; i < GV * ncols_pad; i += nthr) {
      const int k = i / ncols_pad, e = i - k * ncols_pad;
      const int r = vrows[k];
      rows[k * LMAX + e] = (r >= 0 && e < ncols) ? src[(int64_t)r * stride + e] : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
}

// The tables of the Gram form (once per kernel).
template <int W>
__device__ inline void gram_tables(GramShared& S) {
  const int tid = threadIdx.x;
  if (tid < GSTEPS * (GV / 2)) {
    const int st = tid / (GV / 2), w = tid % (GV / 2);
    int p, q;
    gram_pair<W>(st < W - 1, st < W - 1 ? st : st - (W - 1), w, p, q);
    S.pq[st][w][0] = (unsigned char)p;
    S.pq[st][w][1] = (unsigned char)q;
  }
  if (tid < 36) {
    int t = tid, ti = 0;
    while (t >= 8 - ti) t -= 8 - ti++;
    S.tile[tid][0] = (unsigned char)ti;
    S.tile[tid][1] = (unsigned char)(ti + t);
  }
  if (tid < 120) {
    int t = tid, u = 0;
    while (t >= 15 - u) t -= 15 - u++;
    S.blk[tid][0] = (unsigned char)u;
    S.blk[tid][1] = (unsigned char)(u + 1 + t);
  }
}

// One visit in the Gram form: blocks bi and bj (bj may be the padding block).
template <int W>
__device__ void block_visit_gram(const SvdDesc& P, int bi, int bj, bool first_round, float tol, float2* xs,
                                 GramShared& S) {
  static_assert(2 * W == GV, "Gram form: blocks of 16");
  constexpr int THREADS = 32 * W;
  constexpr int LMAX = 512;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = P.n_vec, len = P.len;
  const int nb = (n + W - 1) / W;
  __syncthreads();  // the previous visit is done with S and xs
  if (tid < GV) {
    const int blk = tid < W ? bi : bj;
    const int g = blk * W + (tid % W);
    S.vrows[tid] = (blk < nb && g < n) ? g : -1;
  }
  __syncthreads();
  const bool j_real = bj < nb;
  if (!first_round && !j_real) return;
  // Q = I; the vectors (zero up to a multiple of 32 elements and for absent vectors)
  float2* X = P.X32;
  const int nst = (len + 31) >> 5;
  for (int i = tid; i < GV * GV; i += THREADS) (&S.Q[0][0])[i] = make_float2(i / GV == i % GV ? 1.f : 0.f, 0.f);
  gram_load_rows(xs, X, S.vrows, len, 32 * nst, len);
  // G: the upper 4 x 4 tiles, a warp per tile, the lanes splitting the elements
  for (int t = warp; t < 36; t += W) {
    const int ti = S.tile[t][0], tj = S.tile[t][1];
    // conj(a) b = (re a, re a) (re b, im b) + (im a, im a) (im b, -re b), packed
    f32x2 acc2[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc2[i] = 0ull;
    const float2* xa = xs + 4 * ti * LMAX + lane;
    const float2* xb = xs + 4 * tj * LMAX + lane;
    for (int s = 0; s < nst; ++s) {
      float2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = xa[i * LMAX + 32 * s];
        b[i] = xb[i * LMAX + 32 * s];
      }
      f32x2 bv[4], bs[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        bv[j] = pk2(b[j].x, b[j].y);
        bs[j] = pk2(b[j].y, -b[j].x);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const f32x2 ar = pk2(a[i].x, a[i].x), ai = pk2(a[i].y, a[i].y);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          fma2(acc2[4 * i + j], ar, bv[j]);
          fma2(acc2[4 * i + j], ai, bs[j]);
        }
      }
    }
    float acc[32];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float2 v2 = upk2(acc2[i]);
      acc[2 * i] = v2.x;
      acc[2 * i + 1] = v2.y;
    }
    const float v = warp_reduce_scatter32(acc, lane);
    const int e = lane >> 1, i = e >> 2, j = e & 3, c = lane & 1;
    float* Gf = reinterpret_cast<float*>(&S.G[0][0]);
    Gf[((4 * ti + i) * GV + 4 * tj + j) * 2 + c] = v;
    if (ti != tj) Gf[((4 * tj + j) * GV + 4 * ti + i) * 2 + c] = c ? -v : v;
  }
  __syncthreads();
  // the rotations, in local rounds of W disjoint pairs: steps 0 .. W - 2 pair
  // the vectors inside each block, steps W - 1 .. 2W - 2 across the blocks
  const float zl = Prec<float2>::zero_level(P);
  const float tol2 = tol * tol;
  int lrot = 0, lchk = 0;
  float lmax = 0.f;
  const int st0 = first_round ? 0 : W - 1;
  const int st1 = j_real ? 2 * W - 2 : W - 2;  // last step
  for (int st = st0; st <= st1; ++st) {
    if (tid < W) {
      // the parameters of pair tid (one lane per pair), from G
      const int p = S.pq[st][tid][0], q = S.pq[st][tid][1];
      GramRot g{1.f, make_float2(0.f, 0.f), make_float2(0.f, 0.f), 0};
      if (S.vrows[p] >= 0 && S.vrows[q] >= 0) {
        ++lchk;
        const float a = S.G[p][p].x, b = S.G[q][q].x;
        const float2 k = S.G[p][q];
        RotRec<float2> rec;
        float a2, b2, ratio = 0.f;
        if (jacobi_rotation_fast<float2>(tol2, zl, a, b, k.x, k.y, rec, a2, b2, ratio)) {
          g = GramRot{rec.cs, rec.m1, rec.m2, 1};
          ++lrot;
          lmax = fmaxf(lmax, ratio);
          S.G[p][p] = make_float2(a2, 0.f);
          S.G[q][q] = make_float2(b2, 0.f);
          S.G[p][q] = S.G[q][p] = make_float2(0.f, 0.f);
        }
      }
      S.rr[tid] = g;
    }
    __syncthreads();
    {
      // Q <- Q J: row k, pair w (x_p' = cs x_p + m1 x_q, x_q' = m2 x_p + cs x_q)
      const int k = tid >> 4, w = tid & 15;
      const GramRot& g = S.rr[w];
      if (g.rot) {
        const int p = S.pq[st][w][0], q = S.pq[st][w][1];
        const float2 a = S.Q[k][p], b = S.Q[k][q];
        S.Q[k][p] = cadd(cscale(g.cs, a), cmul(g.m1, b));
        S.Q[k][q] = cadd(cmul(g.m2, a), cscale(g.cs, b));
      }
    }
    if (tid >= THREADS - 120) {
      // G <- J^H G J on the 2 x 2 block (pair u) x (pair v), u < v, and its mirror
      const int t = tid - (THREADS - 120);
      const int u = S.blk[t][0], v = S.blk[t][1];
      const GramRot gu = S.rr[u], gv = S.rr[v];
      if (gu.rot | gv.rot) {
        const int p = S.pq[st][u][0], q = S.pq[st][u][1];
        const int r = S.pq[st][v][0], s = S.pq[st][v][1];
        const float2 g_pr = S.G[p][r], g_ps = S.G[p][s], g_qr = S.G[q][r], g_qs = S.G[q][s];
        // columns: (G J_v)[., r] = G[., r] cs + G[., s] m1; (G J_v)[., s] = G[., r] m2 + G[., s] cs
        const float2 t_pr = cadd(cscale(gv.cs, g_pr), cmul(g_ps, gv.m1));
        const float2 t_ps = cadd(cmul(g_pr, gv.m2), cscale(gv.cs, g_ps));
        const float2 t_qr = cadd(cscale(gv.cs, g_qr), cmul(g_qs, gv.m1));
        const float2 t_qs = cadd(cmul(g_qr, gv.m2), cscale(gv.cs, g_qs));
        // rows: (J_u^H T)[p, .] = cs T[p, .] + conj(m1) T[q, .]; [q, .] = conj(m2) T[p, .] + cs T[q, .]
        const float2 n_pr = cadd(cscale(gu.cs, t_pr), cmulc(gu.m1, t_qr));
        const float2 n_ps = cadd(cscale(gu.cs, t_ps), cmulc(gu.m1, t_qs));
        const float2 n_qr = cadd(cmulc(gu.m2, t_pr), cscale(gu.cs, t_qr));
        const float2 n_qs = cadd(cmulc(gu.m2, t_ps), cscale(gu.cs, t_qs));
        S.G[p][r] = n_pr;
        S.G[p][s] = n_ps;
        S.G[q][r] = n_qr;
        S.G[q][s] = n_qs;
        S.G[r][p] = conjf2(n_pr);
        S.G[s][p] = conjf2(n_ps);
        S.G[r][q] = conjf2(n_qr);
        S.G[s][q] = conjf2(n_qs);
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < GV * GV; i += THREADS) {
    const float2 q = (&S.Q[0][0])[i];
    (&S.QS[0][0])[i] = make_float2(-q.y, q.x);
  }
  if (warp == 0) {
    int nr = lrot, nc = lchk;
    float m = lmax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nr += __shfl_xor_sync(0xffffffffu, nr, o);
      nc += __shfl_xor_sync(0xffffffffu, nc, o);
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if (lane == 0) {
      S.n_rot = nr;
      if (nc > 0) atomicAdd(P.rotated + 1, nc);
      if (nr > 0) {
        atomicAdd(P.rotated, nr);
        atomicMax(P.maxr, __float_as_uint(m));
      }
    }
  }
  __syncthreads();
  if (S.n_rot == 0) return;  // the vectors are unchanged
  // X <- X Q; once xs has been read, the rows of Acc are copied into it while
  // the last results of X Q are stored
  float2* A = P.Acc32;
  gram_apply_q(xs, S, len, X, len, [&] { gram_load_rows(xs, A, S.vrows, n, n, n); });
  gram_apply_q(xs, S, n, A, n, [] {});
}

// One visit: blocks bi and bj (bj may be the padding block) of problem P.
// acc_mode 0: replay every rotation on Acc; 1: block_correct_acc (FP64 sweeps
// of the mixed mode).

template <typename T, int W>
__device__ void block_visit(const SvdDesc& P, int bi, int bj, bool first_round, bool use_order, int acc_mode,
                            typename Prec<T>::R tol, T* xs, RotRec<T>* seq, typename Prec<T>::R* nrm) {
  using C = BlockCfg<T, W>;
  using R = typename Prec<T>::R;
  __shared__ int vrows[2 * W];
  __shared__ int n_rot[2];  // rotations, pairs checked
  __shared__ unsigned maxr_bits;
  __shared__ int skip;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = P.n_vec, len = P.len;
  const int nb = (n + W - 1) / W;
  __syncthreads();  // the previous visit's readers of the shared state are done
  if (tid < 2 * W) {
    const int blk = tid < W ? bi : bj;
    const int g = blk * W + (tid % W);
    vrows[tid] = (blk < nb && g < n) ? (use_order ? P.perm[g] : g) : -1;
  }
  if (tid == 0) {
    n_rot[0] = n_rot[1] = 0;
    maxr_bits = 0u;
    skip = 0;
  }
  __syncthreads();
  const bool j_real = bj < nb;
  if (!first_round && !j_real) return;
  double tau = 0.0;
  if constexpr (Prec<T>::tracks_norms) {
    tau = P.sig[n + 2];
    if (tid == 0 && tau > 0.0) {
      int below = 1;
      for (int k = 0; k < 2 * W; ++k)
        if (vrows[k] >= 0 && P.sig[vrows[k]] >= tau) below = 0;
      skip = below;
    }
    __syncthreads();
    if (skip) return;
  }
  T* X = Prec<T>::X(P);
  // load the 2W vectors (zero past len and for absent vectors)
  for (int k = 0; k < 2 * W; ++k) {
    const int r = vrows[k];
    for (int e = tid; e < C::LMAX; e += C::THREADS)
      xs[k * C::LMAX + e] = (r >= 0 && e < len) ? X[(int64_t)r * len + e] : Prec<T>::mk(0, 0);
  }
  __syncthreads();
  // squared norms, a warp per vector
  for (int k = warp; k < 2 * W; k += W) {
    R kr, ki;
    block_cross<T, W>(xs + k * C::LMAX, xs + k * C::LMAX, lane, kr, ki);
    if (lane == 0) nrm[k] = kr;
  }
  __syncthreads();
  const R zl = Prec<T>::zero_level(P);
  const R tol2 = tol * tol;
  int step = 0;
  if (first_round) {
    // pairs inside each block: W - 1 rounds of W/2 pairs per block
    for (int rr = 0; rr < W - 1; ++rr, ++step) {
      int p, q;
      rr_pair(W, rr, warp % (W / 2), p, q);
      const int o = warp < W / 2 ? 0 : W;
      block_local_round<T, W>(tol2, zl, xs, nrm, seq, step * W + warp, vrows, p + o, q + o, tau, n_rot,
                              &maxr_bits);
    }
  }
  if (j_real) {
    for (int rr = 0; rr < W; ++rr, ++step)
      block_local_round<T, W>(tol2, zl, xs, nrm, seq, step * W + warp, vrows, warp, W + (warp + rr) % W, tau,
                              n_rot, &maxr_bits);
  }
  // vectors back to global memory; norms for the tail rule
  for (int k = 0; k < 2 * W; ++k) {
    const int r = vrows[k];
    if (r < 0) continue;
    for (int e = tid; e < len; e += C::THREADS) X[(int64_t)r * len + e] = xs[k * C::LMAX + e];
  }
  if constexpr (Prec<T>::tracks_norms) {
    if (tid < 2 * W && vrows[tid] >= 0) P.sig[vrows[tid]] = sqrt(fmax((double)nrm[tid], 0.0));
  }
  if (tid == 0) {
    if (n_rot[1] > 0) atomicAdd(P.rotated + 1, n_rot[1]);
    if (n_rot[0] > 0) {
      atomicAdd(P.rotated, n_rot[0]);
      atomicMax(P.maxr, maxr_bits);
    }
  }
  if (n_rot[0] > 0) {
    if (acc_mode == 1 || Prec<T>::dd) {
      __syncthreads();  // xs is free: it holds D
      block_correct_acc<T, W>(P, vrows, seq, first_round, j_real, reinterpret_cast<float2*>(xs));
    } else if constexpr (!Prec<T>::dd) {
      block_replay_acc<T, W>(P, vrows, seq, first_round, j_real);
    }
  }
}

template <typename T, int W>
constexpr size_t block_smem_bytes() {
  using C = BlockCfg<T, W>;
  using R = typename Prec<T>::R;
  size_t b = (size_t)2 * W * C::LMAX * sizeof(T);       // the vectors
  if (std::is_same<T, float2>::value) return b + sizeof(GramShared);  // the Gram form's state
  b += (size_t)C::MAX_STEPS * W * sizeof(RotRec<T>);    // rotation record
  b += (size_t)2 * W * sizeof(R);                       // squared norms
  return b;
}

// All sweeps of one phase with the block order (see above); one CTA per SM.
// The FP32 phase (T = float2) runs its visits in the Gram form.
template <typename T, int W, int MINB>
__global__ void __launch_bounds__(32 * W, MINB) svd_block_sweeps(const __grid_constant__ SvdBatch B, int nbpad_max,
                                                                float stop, double tol, int max_sweeps, int fatal,
                                                                int use_order, int acc_mode, double* work_flops) {
  using C = BlockCfg<T, W>;
  using R = typename Prec<T>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);
  RotRec<T>* seq = reinterpret_cast<RotRec<T>*>(smem_raw + (size_t)2 * W * C::LMAX * sizeof(T));
  R* nrm = reinterpret_cast<R*>(seq + C::MAX_STEPS * W);
  GramShared* gs = reinterpret_cast<GramShared*>(smem_raw + (size_t)2 * W * C::LMAX * sizeof(T));
  if constexpr (std::is_same<T, float2>::value) gram_tables<W>(*gs);
  __shared__ int off[MAXB + 1];
  if (threadIdx.x == 0) {
    off[0] = 0;
    for (int i = 0; i < B.n; ++i) {
      const int nb = (B.d[i].n_vec + W - 1) / W;
      off[i + 1] = off[i] + (nb + (nb & 1)) / 2;
    }
  }
  __shared__ int u_sh;
  __syncthreads();
  const int total = off[B.n];
  volatile unsigned* unconv = B.sync + 2;
  // visits are handed out dynamically (their cost varies: the tail rule skips
  // some, the first block round of a sweep adds the intra-block pairs) from
  // two counters used in alternate block rounds: block 0 clears the other one
  // while the current one is in use, and the grid barrier between rounds
  // publishes the clearing.
  unsigned* ctr = B.sync + 4;
  int rnd = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int br = 0; br < nbpad_max - 1; ++br, ++rnd) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(ctr + ((rnd + 1) & 1), 0u);
      for (;;) {
        __syncthreads();  // u_sh of the previous visit has been read
        if (threadIdx.x == 0) u_sh = (int)atomicAdd(ctr + (rnd & 1), 1u);
        __syncthreads();
        const int u = u_sh;
        if (u >= total) break;
        int pid = 0;
        while (u >= off[pid + 1]) ++pid;
        const SvdDesc& P = B.d[pid];
        if (*(volatile int*)P.conv) continue;
        const int nb = (P.n_vec + W - 1) / W;
        const int nbp = nb + (nb & 1);
        if (br >= nbp - 1) continue;
        int bi, bj;
        rr_pair(nbp, br, u - off[pid], bi, bj);
        if constexpr (std::is_same<T, float2>::value)
          block_visit_gram<W>(P, bi, bj, br == 0, (float)tol, xs, *gs);
        else
          block_visit<T, W>(P, bi, bj, br == 0, use_order != 0, acc_mode, (R)tol, xs, seq, nrm);
      }
      if (!grid_barrier(B.sync, gridDim.x, B.status, B.spin_limit)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) sweep_end<T>(B, stop, work_flops, acc_mode == 0);
    if (!grid_barrier(B.sync, gridDim.x, B.status, B.spin_limit)) return;
    if (*unconv == 0) return;
  }
  if (fatal && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(B.status, 16);
}

// The FP64 vectors to double-float and back, in place (16 bytes either way).
__global__ void svd_x_to_dd(const __grid_constant__ SvdBatch B) {
  const SvdDesc& P = B.d[blockIdx.y];
  const int64_t n = (int64_t)P.n_vec * P.len;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = P.X[i];
    const float2 re = dd_split(v.x), im = dd_split(v.y);
    reinterpret_cast<float4*>(P.X)[i] = make_float4(re.x, im.x, re.y, im.y);
  }
}
__global__ void svd_dd_to_x(const __grid_constant__ SvdBatch B) {
  const SvdDesc& P = B.d[blockIdx.y];
  const int64_t n = (int64_t)P.n_vec * P.len;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = reinterpret_cast<const float4*>(P.X)[i];
    P.X[i] = make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
  }
}

// FP32 rotation -> FP64; reset the convergence state for the FP64 phase
__global__ void svd_acc_to64(const __grid_constant__ SvdBatch B) {
  const SvdDesc& P = B.d[blockIdx.y];
  const int64_t na = (int64_t)P.n_vec * P.n_vec;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na; i += (int64_t)gridDim.x * blockDim.x) {
    float2 a = P.Acc32[i];
    P.Acc[i] = make_double2((double)a.x, (double)a.y);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    P.rotated[0] = P.rotated[1] = 0;
    *P.conv = 0;
    *P.maxr = 0u;
  }
}

// Newton-Schulz step for the unitary polar factor, Acc <- 1.5 Acc - 0.5 Acc Acc^H Acc,
// written as Acc <- Acc + 0.5 E Acc with E = I - Acc Acc^H. E is small (the
// unitarity defect), so E Acc only needs FP32: its rounding, ~6e-8 |E|, stays
// below the FP64 rounding of Acc once |E| < 1e-8. P = Acc Acc^H (FP64, upper
// tiles only: Hermitian) comes from the FP64 GEMM; this kernel forms E from it
// and writes T = E Acc (64 x 64 output tiles, 4 x 4 per thread).
constexpr int NS_T = 64, NS_BK = 8;
__global__ void __launch_bounds__(256) svd_ns_correction(const __grid_constant__ SvdBatch B) {
  const SvdDesc& P = B.d[blockIdx.y];
  const int n = P.n_vec;
  const int tiles = (n + NS_T - 1) / NS_T;
  if ((int)blockIdx.x >= tiles * tiles) return;
  const int m0 = (blockIdx.x % tiles) * NS_T, n0 = (blockIdx.x / tiles) * NS_T;
  __shared__ float2 As[NS_BK][NS_T];
  __shared__ float2 Bs[NS_BK][NS_T];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < n; k0 += NS_BK) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int e = tid + r * 256;
      {  // E(i, k) = delta_ik - P(i, k); P(i, k) = conj(P(k, i)) below the diagonal tiles
        const int k = e % NS_BK, i = e / NS_BK;
        const int gi = m0 + i, gk = k0 + k;
        float2 v = make_float2(0.f, 0.f);
        if (gi < n && gk < n) {
          double2 p;
          if (gi / NS_T <= gk / NS_T) {
            p = P.P[(int64_t)gi * n + gk];
          } else {
            p = P.P[(int64_t)gk * n + gi];
            p.y = -p.y;
          }
          v = make_float2((float)((gi == gk ? 1.0 : 0.0) - p.x), (float)(-p.y));
        }
        As[k][i] = v;
      }
      {
        const int j = e % NS_T, k = e / NS_T;
        const int gj = n0 + j, gk = k0 + k;
        float2 w = make_float2(0.f, 0.f);
        if (gj < n && gk < n) {
          const double2 a = P.Acc[(int64_t)gk * n + gj];
          w = make_float2((float)a.x, (float)a.y);
        }
        Bs[k][j] = w;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < NS_BK; ++kk) {
      float2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fmaf(a[i].x, b[j].x, fmaf(-a[i].y, b[j].y, acc[i][j].x));
          acc[i][j].y = fmaf(a[i].x, b[j].y, fmaf(a[i].y, b[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = m0 + ty + 16 * i;
    if (gi >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = n0 + tx + 16 * j;
      if (gj < n) P.T[(int64_t)gi * n + gj] = make_double2(acc[i][j].x, acc[i][j].y);
    }
  }
}

__global__ void svd_ns_combine(const __grid_constant__ SvdBatch B) {
  const SvdDesc& P = B.d[blockIdx.y];
  const int64_t na = (int64_t)P.n_vec * P.n_vec;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = P.Acc[i], t = P.T[i];
    P.Acc[i] = make_double2(a.x + 0.5 * t.x, a.y + 0.5 * t.y);
  }
}

__global__ void svd_norms(const __grid_constant__ SvdBatch B) {
  const SvdDesc& P = B.d[blockIdx.y];
  const int v = blockIdx.x * SVD_WARPS + (threadIdx.x >> 5);
  if (v >= P.n_vec) return;
  const int lane = threadIdx.x & 31;
  const double2* x = P.X + (int64_t)v * P.len;
  double s = 0;
  for (int i = lane; i < P.len; i += 32) s += x[i].x * x[i].x + x[i].y * x[i].y;
  s = warp_sum(s);
  if (lane == 0) P.sig[v] = sqrt(s);
}

__global__ void svd_truncate(const __grid_constant__ SvdBatch B) {
  const SvdDesc& P = B.d[blockIdx.x];
  const int n = P.n_vec;
  __shared__ int has_nan;
  if (threadIdx.x == 0) {
    has_nan = 0;
    for (int i = 0; i < n; ++i)
      if (!(P.sig[i] == P.sig[i])) has_nan = 1;
  }
  __syncthreads();
  if (!has_nan) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double si = P.sig[i];
      int rank = 0;
      for (int j = 0; j < n; ++j) {
        const double sj = P.sig[j];
        rank += (sj > si) || (sj == si && j < i);
      }
      P.perm[rank] = i;
    }
  } else {
    for (int i = threadIdx.x; i < n; i += blockDim.x) P.perm[i] = i;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double s0 = P.sig[P.perm[0]];
  if (has_nan || !(s0 > 0.0)) {
    atomicOr(B.status, 8);
    *P.chi = 1;
    *P.w = 0.0;
    return;
  }
  // smallest chi_w with tail weight <= w_max (Eq. 22), tail[n] = 0
  double tail = 0.0;
  int chi_w = n;
  // walk from the end; tail(k) = sum_{j >= k} s_j^2
  // chi_w = min k >= 1 with tail(k) <= w_max
  {
    double acc = 0.0;
    int best = n;
    for (int k = n - 1; k >= 1; --k) {
      const double sk = P.sig[P.perm[k]];
      acc += sk * sk;
      if (acc <= P.w_max) best = k;
      else break;
    }
    chi_w = best;
  }
  // values above eps * lambda_1 (Sec. III D) and above the FP64 noise floor
  // 1e-14 ||theta||_F (below it a value and its vectors are rounding noise)
  const double noise = 1e-14 * sqrt(P.sig[n + 1]);
  int n_eps = 0;
  for (int k = 0; k < n; ++k) {
    const double sk = P.sig[P.perm[k]];
    if (sk > P.eps * s0 && sk > noise) ++n_eps;
  }
  int chi = chi_w < P.chi_max ? chi_w : P.chi_max;
  if (n_eps < chi) chi = n_eps;
  if (chi < 1) chi = 1;
  for (int k = n - 1; k >= chi; --k) {
    const double sk = P.sig[P.perm[k]];
    tail += sk * sk;
  }
  // the tail rule left the vectors below tau unconverged among themselves
  const double tau = P.sig[n + 2];
  if (tau > 0.0 && P.sig[P.perm[chi - 1]] < tau) atomicOr(B.status, 64);
  *P.chi = chi;
  *P.w = tail;
}

__global__ void svd_write(const __grid_constant__ SvdBatch B) {
  const SvdDesc& P = B.d[blockIdx.y];
  const int chi = *P.chi;
  const int64_t nl = (int64_t)P.rows * chi;
  const int64_t nr = (int64_t)chi * P.cols;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nl + nr + P.n_vec;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (idx < nl) {
      const int r = (int)(idx / chi), c = (int)(idx % chi);
      const int i = P.perm[c];
      double2 v;
      if (P.trans) v = P.X[(int64_t)i * P.len + r];
      else v = zscale(zconj(P.Acc[(int64_t)i * P.n_vec + r]), P.sig[i]);
      P.PsiL[idx] = v;
    } else if (idx < nl + nr) {
      const int64_t q = idx - nl;
      const int c = (int)(q / P.cols), col = (int)(q % P.cols);
      const int i = P.perm[c];
      double2 v;
      if (!P.trans) v = P.X[(int64_t)i * P.len + col];
      else v = zscale(zconj(P.Acc[(int64_t)i * P.n_vec + col]), P.sig[i]);
      P.PsiR[q] = v;
    } else {
      const int c = (int)(idx - nl - nr);
      const double sc = P.sig[P.perm[c]];
      if (c < chi) P.V[c] = 1.0 / sc;
      if (P.s_sorted) P.s_sorted[c] = sc;
    }
  }
}

// all sweeps of one phase as one cooperative launch (no host round trips);
// `fatal`: running out of sweeps is an error (FP64 phase) or not (FP32 phase)
template <typename T>
static void jacobi_sweeps(SvdBatch& b, int npad_max, float stop, int fatal, cudaStream_t s, const char* name) {
  static int max_blocks = -1;
  if (max_blocks < 0) {
    int dev = 0, sms = 0, per_sm = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, svd_sweeps<T>, SVD_WARPS * 32, 0));
    max_blocks = std::max(1, sms * std::min(per_sm, 4));
  }
  int total = 0;
  for (int i = 0; i < b.n; ++i) total += (b.d[i].n_vec + (b.d[i].n_vec & 1)) / 2;
  const int blocks = std::max(1, std::min(max_blocks, cdiv(total, SVD_WARPS)));
  CUDA_TRY(cudaMemsetAsync(b.sync, 0, 8 * sizeof(unsigned), s));
  int max_sweeps = SVD_MAX_SWEEPS;
  double* work_dev = nullptr;
  const double* work_host = prof_work_slot(&work_dev);
  void* args[] = {(void*)&b, (void*)&npad_max, (void*)&stop, (void*)&max_sweeps, (void*)&fatal, (void*)&work_dev};
  ProfScope ps(name, s, 0.0, 0.0, work_host);
  CUDA_TRY(cudaLaunchCooperativeKernel((const void*)svd_sweeps<T>, dim3(blocks), dim3(SVD_WARPS * 32), args, 0, s));
  ++g_launches;
}

// block sweeps (vectors of at most 512 elements) with up to MINB CTAs per SM;
// false if they cannot run. tol: relative off-diagonal below which a pair is
// left alone.
template <typename T, int W, int MINB>
static bool block_sweeps(SvdBatch& b, float stop, double tol, int fatal, int use_order, int acc_mode,
                         cudaStream_t s, const char* name) {
  using C = BlockCfg<T, W>;
  static int max_blocks = -1;
  const size_t smem = block_smem_bytes<T, W>();
  auto kern = svd_block_sweeps<T, W, MINB>;
  if (max_blocks < 0) {
    int dev = 0, sms = 0, per_sm = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::THREADS, smem));
    max_blocks = sms * std::min(per_sm, MINB);
  }
  if (max_blocks <= 0) return false;
  int total = 0, nbpad_max = 2;
  for (int i = 0; i < b.n; ++i) {
    if (b.d[i].len > C::LMAX) return false;
    const int nb = cdiv(b.d[i].n_vec, W);
    total += (nb + (nb & 1)) / 2;
    nbpad_max = std::max(nbpad_max, nb + (nb & 1));
  }
  const int blocks = std::max(1, std::min(max_blocks, total));
  CUDA_TRY(cudaMemsetAsync(b.sync, 0, 8 * sizeof(unsigned), s));
  int max_sweeps = SVD_MAX_SWEEPS;
  double* work_dev = nullptr;
  const double* work_host = prof_work_slot(&work_dev);
  void* args[] = {(void*)&b,     (void*)&nbpad_max, (void*)&stop,     (void*)&tol,     (void*)&max_sweeps,
                  (void*)&fatal, (void*)&use_order, (void*)&acc_mode, (void*)&work_dev};
  ProfScope ps(name, s, 0.0, 0.0, work_host);
  CUDA_TRY(cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(C::THREADS), args, smem, s));
  ++g_launches;
  return true;
}

namespace {
std::atomic<long long> g_spin_limit{SVD_SPIN_LIMIT_DEFAULT};
}

void svd_set_spin_limit(long long spins) { g_spin_limit = spins < 0 ? SVD_SPIN_LIMIT_DEFAULT : spins; }

void svd_split(SvdBatch& b, int* d_flag, int* h_flag, cudaStream_t s) {
  if (b.n <= 0) return;
  b.spin_limit = g_spin_limit.load();
  int64_t max_elems = 1;
  int npad_max = 2, nvec_max = 1;
  for (int i = 0; i < b.n; ++i) {
    auto& P = b.d[i];
    P.trans = P.rows > P.cols ? 1 : 0;
    P.n_vec = P.trans ? P.cols : P.rows;
    P.len = P.trans ? P.rows : P.cols;
    max_elems = std::max<int64_t>(max_elems, (int64_t)P.n_vec * (P.len + P.n_vec));
    npad_max = std::max(npad_max, P.n_vec + (P.n_vec & 1));
    nvec_max = std::max(nvec_max, P.n_vec);
  }
  dim3 g1((unsigned)std::min<int64_t>(cdiv64(max_elems, 256), 152 * 8), b.n);
  // ---- phase 1: FP32 sweeps ----
  svd_scale<<<b.n, 512, 0, s>>>(b);
  LAUNCH_CHECK();
  svd_setup32<<<g1, 256, 0, s>>>(b);
  LAUNCH_CHECK();
  ++g_launches;
  // FP32 phase: until the largest relative off-diagonal of a sweep is < 1e-4
  // (just above the FP32 rounding of the dot products); not converging here
  // only means a weaker preconditioner
  if (!block_sweeps<float2, 16, 1>(b, 1e-4f, Prec<float2>::tol, 0, 0, 0, s, "svd_jacobi_fp32"))
    jacobi_sweeps<float2>(b, npad_max, 1e-4f, 0, s, "svd_jacobi_fp32");
  // ---- phase 2: unitary FP64 rotation and FP64 vectors ----
  svd_acc_to64<<<g1, 256, 0, s>>>(b);
  LAUNCH_CHECK();
  ZGemmBatch gp{}, gx{};
  gp.n = gx.n = b.n;
  for (int i = 0; i < b.n; ++i) {
    const SvdDesc& P = b.d[i];
    const int n = P.n_vec;
    ZGemmDesc& a = gp.d[i];   // P = Acc Acc^H (Hermitian: upper tiles)
    a = ZGemmDesc{};
    a.M = a.N = a.K = n;
    a.A = P.Acc; a.a_rs = n; a.a_cs = 1;
    a.B = P.Acc; a.b_rs = 1; a.b_cs = n; a.conj_b = 1;
    a.C = P.P; a.c_rs = n; a.c_cs = 1;
    a.upper_only = 1;
    ZGemmDesc& x = gx.d[i];   // X = Acc . vectors(theta)
    x = ZGemmDesc{};
    x.M = n; x.N = P.len; x.K = n;
    x.A = P.Acc; x.a_rs = n; x.a_cs = 1;
    x.B = P.theta;
    if (!P.trans) { x.b_rs = P.cols; x.b_cs = 1; }
    else { x.b_rs = 1; x.b_cs = P.cols; }
    x.C = P.X; x.c_rs = P.len; x.c_cs = 1;
  }
  // Newton-Schulz steps: the FP32 rotation's unitarity defect (up to ~1e-4
  // after many sweeps) -> ~1e-8 -> rounding, on both paths
  const int ns_steps = 2;
  for (int it = 0; it < ns_steps; ++it) {
    if (b.mode == 1) launch_zgemm_dd(gp, s, "svd_newton_schulz_dd");
    else launch_zgemm(gp, s, "svd_newton_schulz");
    const int nt = cdiv(nvec_max, NS_T);
    {
      double fl = 0.0;
      for (int i = 0; i < b.n; ++i) fl += 8.0 * (double)b.d[i].n_vec * b.d[i].n_vec * b.d[i].n_vec;
      ProfScope ps("svd_ns_correction_fp32", s, fl, 0.0);
      svd_ns_correction<<<dim3(nt * nt, b.n), 256, 0, s>>>(b);
      LAUNCH_CHECK();
    }
    dim3 gn((unsigned)std::min<int64_t>(cdiv64((int64_t)nvec_max * nvec_max, 256), 152 * 8), b.n);
    svd_ns_combine<<<gn, 256, 0, s>>>(b);
    LAUNCH_CHECK();
    g_launches += 2;
  }
  if (b.mode == 1) launch_zgemm_dd(gx, s, "svd_newton_schulz_dd");
  else launch_zgemm(gx, s, "svd_newton_schulz");
  g_launches += 2;
  // ---- phase 3: FP64 sweeps ----
  dim3 gn(cdiv(nvec_max, SVD_WARPS), b.n);
  svd_norms<<<gn, SVD_WARPS * 32, 0, s>>>(b);
  LAUNCH_CHECK();
  const size_t tail_smem = (size_t)std::min(nvec_max, SVD_TAIL_MAX) * sizeof(double);
  svd_tail_threshold<<<b.n, 256, tail_smem, s>>>(b);
  LAUNCH_CHECK();
  g_launches += 2;
  // stop after a sweep whose largest relative off-diagonal was below 1e-7 (full:
  // ~1e-14 left) or 1e-4 (mixed-precision sweeps: ~1e-8 or less left)
  const float stop64 = b.mode == 0 ? 1e-7f : 1e-4f;
  // mode 1 leaves pairs below 1e-10 alone (its target is ~1e-8)
  const double tol64 = b.mode == 0 ? JACOBI_TOL : 1e-10;
  bool short_rows = true;
  for (int i = 0; i < b.n; ++i) short_rows = short_rows && b.d[i].len <= BlockCfg<float4, 8>::LMAX;
  if (b.mode == 1 && short_rows) {
    // mixed mode: the final sweeps in double-float on the FP32 pipe (~48 bits,
    // ample for its 1e-10 tolerance), Acc updated through FP32 block rotations
    svd_x_to_dd<<<g1, 256, 0, s>>>(b);
    LAUNCH_CHECK();
    if (!block_sweeps<float4, 8, 1>(b, stop64, tol64, 1, 1, 1, s, "svd_jacobi_dd")) fail(TDVP_ECUDA, "block sweeps");
    svd_dd_to_x<<<g1, 256, 0, s>>>(b);
    LAUNCH_CHECK();
    g_launches += 2;
  } else if (!block_sweeps<double2, 8, 1>(b, stop64, tol64, 1, 1, b.mode == 1 ? 1 : 0, s, "svd_jacobi_fp64")) {
    jacobi_sweeps<double2>(b, npad_max, stop64, 1, s, "svd_jacobi_fp64");
  }
  svd_norms<<<gn, SVD_WARPS * 32, 0, s>>>(b);
  LAUNCH_CHECK();
  svd_truncate<<<b.n, 256, 0, s>>>(b);
  LAUNCH_CHECK();
  dim3 gw((unsigned)std::min<int64_t>(cdiv64(max_elems, 256), 152 * 8), b.n);
  svd_write<<<gw, 256, 0, s>>>(b);
  LAUNCH_CHECK();
  g_launches += 3;
}

}  // namespace tdvp
