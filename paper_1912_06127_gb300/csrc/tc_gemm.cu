// Tensor-core GEMM for the mixed-precision contractions (sm_103a).
//
// C[M][N] = sum_pass A_pass[M][K] . B_pass[N][K]^T with fp32 operands read as
// TF32 by tcgen05.mma (kind::tf32) and FP32 accumulation in tensor memory.
// Complex products use the real embedding prepared by the operand kernels
// (A interleaved re/im along K; B expanded to [2N][2K]), so one real GEMM
// computes Re and Im of every complex output. The 3xTF32 mode runs three
// passes (A_hi B_hi + A_hi B_lo + A_lo B_hi) into the same accumulator.
//
// Per CTA: one 128 x 256 output tile. Warp 0 issues TMA loads (128B-swizzled
// 32-float K slices) into a 4-stage shared-memory ring, warp 1 issues the
// MMAs (one elected thread), all four warps drain TMEM (tcgen05.ld) and write
// C. mbarrier waits are bounded: on timeout the CTA records an error in the
// status word, stops issuing, waits (bounded) for its own copies in flight,
// frees its tensor memory and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <memory>
#include <mutex>

#include "common.h"

namespace tdvp {

constexpr int TC_BM = 128;
// N tile: 256 (default) or 128 (twice the CTAs for small batches); chosen per
// shape by the autotuner (tune.cu). Every column of a tile sums over K in the
// same MMA order whatever the tile width, so both give the same result.
template <int BN>
struct TcTile {
  static constexpr int B_BYTES = BN * 32 * 4;
  static constexpr int STAGE_BYTES = 128 * 32 * 4 + B_BYTES;
  static constexpr int SMEM = 4 * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
  static constexpr int TMEM_COLS = BN;
};
constexpr int TC_BK = 32;  // fp32 elements = 128 bytes (one swizzle row)
constexpr int TC_STAGES = 4;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 4;  // 16 KB
constexpr int TC_MAXP = 16;
constexpr long long TC_SPIN_LIMIT = 1ll << 22;

struct TcParams {
  CUtensorMap mapA[TC_MAXP][2];
  CUtensorMap mapB[TC_MAXP][2];
  int M[TC_MAXP], N[TC_MAXP], K[TC_MAXP];
  void* C[TC_MAXP];
  const int* skip[TC_MAXP];
  long long ldc[TC_MAXP];
  int c_fp64[TC_MAXP];
  float* part[TC_MAXP];  // K-split partial tiles [chunk][M][N] (nch > 1)
  int kcb[TC_MAXP];      // K blocks (of TC_BK) per chunk
  int nch[TC_MAXP];      // chunks (1: no split)
  int n, passes;
  int* status;
};

// ---- PTX wrappers ---------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// bounded wait on phase parity; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t addr = smem_u32(bar);
  for (long long it = 0; it < TC_SPIN_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}
// shared-memory matrix descriptor: K-major, 128B swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // 128B swizzle
  return d;
}
// instruction descriptor: D f32, A/B tf32, both K-major, N, M
__host__ __device__ constexpr uint32_t tc_idesc(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

template <int TC_BN>
__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(const __grid_constant__ TcParams P) {
  constexpr int TC_STAGE_BYTES = TcTile<TC_BN>::STAGE_BYTES;
  constexpr int TC_TMEM_COLS = TcTile<TC_BN>::TMEM_COLS;
  static_assert(TC_STAGES == 4 && TC_A_BYTES + TcTile<TC_BN>::B_BYTES == TC_STAGE_BYTES, "stage layout");
  const int pid = blockIdx.y;
  if (pid >= P.n) return;
  if (P.skip[pid] && *P.skip[pid]) return;
  const int M = P.M[pid], N = P.N[pid], K = P.K[pid];
  const int tiles_m = (M + TC_BM - 1) / TC_BM;
  const int tiles_n = (N + TC_BN - 1) / TC_BN;
  const int tiles = tiles_m * tiles_n, nch = P.nch[pid];
  if ((int)blockIdx.x >= tiles * nch) return;
  const int tile = blockIdx.x % tiles, chunk = blockIdx.x / tiles;
  const int tm = tile % tiles_m, tn = tile / tiles_m;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + TC_STAGES * TC_STAGE_BYTES);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* mma_done = empty + TC_STAGES;
  uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
  int* abort_flag = (int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // this CTA's K blocks: [kb_lo, kb_lo + kb_per_pass) of every pass
  const int kb_total = (K + TC_BK - 1) / TC_BK;
  const int kb_lo = nch > 1 ? chunk * P.kcb[pid] : 0;
  const int kb_per_pass = nch > 1 ? min(kb_total, kb_lo + P.kcb[pid]) - kb_lo : kb_total;
  const int num_kb = kb_per_pass * P.passes;
  const CUtensorMap* mA[3];
  const CUtensorMap* mB[3];
  mA[0] = &P.mapA[pid][0];
  mB[0] = &P.mapB[pid][0];
  mA[1] = &P.mapA[pid][0];
  mB[1] = &P.mapB[pid][1];
  mA[2] = &P.mapA[pid][1];
  mB[2] = &P.mapB[pid][0];

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    for (int p = 0; p < P.passes; ++p) {
      prefetch_map(mA[p]);
      prefetch_map(mB[p]);
    }
    int issued = 0;
    for (int kb = 0; kb < num_kb; ++kb) {
      const int s = kb % TC_STAGES;
      const int round = kb / TC_STAGES;
      if (round > 0) {
        if (!mbar_wait(&empty[s], (round - 1) & 1) || *(volatile int*)abort_flag) {
          atomicExch(abort_flag, 1);
          break;
        }
      }
      const int pass = kb / kb_per_pass;
      const int k0 = (kb_lo + kb % kb_per_pass) * TC_BK;
      uint8_t* sa = smem + s * TC_STAGE_BYTES;
      uint8_t* sb = sa + TC_A_BYTES;
      mbar_expect_tx(&full[s], TC_STAGE_BYTES);
      tma_load_2d(sa, mA[pass], &full[s], k0, tm * TC_BM);
      tma_load_2d(sb, mB[pass], &full[s], k0, tn * TC_BN);
      ++issued;
    }
    // on abort: let every issued copy land before the shared memory is released
    if (*(volatile int*)abort_flag) {
      for (int kb = 0; kb < issued; ++kb) mbar_wait(&full[kb % TC_STAGES], (kb / TC_STAGES) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    const uint32_t idesc = tc_idesc(TC_BM, TC_BN);
    for (int kb = 0; kb < num_kb; ++kb) {
      const int s = kb % TC_STAGES;
      if (!mbar_wait(&full[s], (kb / TC_STAGES) & 1) || *(volatile int*)abort_flag) {
        atomicExch(abort_flag, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(smem + s * TC_STAGE_BYTES);
      const uint32_t sb = sa + TC_A_BYTES;
#pragma unroll
      for (int kk = 0; kk < TC_BK / 8; ++kk) {
        const uint64_t da = umma_desc(sa + kk * 32);
        const uint64_t db = umma_desc(sb + kk * 32);
        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty[s]))
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mma_done))
                 : "memory");
  }
  __syncwarp();
  // ---- epilogue: TMEM -> registers -> global ----
  bool ok = mbar_wait(mma_done, 0);
  if (!ok) atomicExch(abort_flag, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (*(volatile int*)abort_flag) {
    if (threadIdx.x == 0) atomicOr(P.status, 1);
  } else {
    const int row = tm * TC_BM + warp * 32 + lane;
    const bool row_ok = row < M;
    for (int c0 = 0; c0 < TC_BN; c0 += 32) {
      if (tn * TC_BN + c0 >= N) break;  // uniform across the CTA
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
            "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
            "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
            "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (!row_ok) continue;
      const int col0 = tn * TC_BN + c0;
      // K-split: this chunk's FP32 partial tile, summed in FP64 by tc_reduce_kernel
      const bool split = nch > 1;
      if (!split && P.c_fp64[pid]) {
        double* crow = (double*)P.C[pid] + (long long)row * P.ldc[pid];
        if (col0 + 32 <= N) {
#pragma unroll
          for (int i = 0; i < 32; i += 2)
            *reinterpret_cast<double2*>(crow + col0 + i) =
                make_double2((double)__uint_as_float(r[i]), (double)__uint_as_float(r[i + 1]));
        } else {
          for (int i = 0; i < 32 && col0 + i < N; ++i) crow[col0 + i] = (double)__uint_as_float(r[i]);
        }
      } else {
        float* crow = split ? P.part[pid] + ((long long)chunk * M + row) * N
                            : (float*)P.C[pid] + (long long)row * P.ldc[pid];
        if (col0 + 32 <= N) {
#pragma unroll
          for (int i = 0; i < 32; i += 2)
            *reinterpret_cast<float2*>(crow + col0 + i) = make_float2(__uint_as_float(r[i]), __uint_as_float(r[i + 1]));
        } else {
          for (int i = 0; i < 32 && col0 + i < N; ++i) crow[col0 + i] = __uint_as_float(r[i]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
  }
}

// FP64 sum of the K-split partial tiles: C[row][col] = sum_chunk part[chunk][row][col].
struct TcReduce {
  const float* part[TC_MAXP];
  void* C[TC_MAXP];
  const int* skip[TC_MAXP];
  long long ldc[TC_MAXP];
  int M[TC_MAXP], N[TC_MAXP], nch[TC_MAXP], c_fp64[TC_MAXP];
  int n;
};

__global__ void __launch_bounds__(256) tc_reduce_kernel(const __grid_constant__ TcReduce R) {
  const int pid = blockIdx.y;
  if (pid >= R.n) return;
  if (R.skip[pid] && *R.skip[pid]) return;
  const int N = R.N[pid], nch = R.nch[pid];
  const long long MN = (long long)R.M[pid] * N;
  const float* part = R.part[pid];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < MN; e += (long long)gridDim.x * blockDim.x) {
    double sum = 0.0;
    for (int c = 0; c < nch; ++c) sum += (double)part[c * MN + e];
    const long long row = e / N, col = e - row * N;
    if (R.c_fp64[pid]) ((double*)R.C[pid])[row * R.ldc[pid] + col] = sum;
    else ((float*)R.C[pid])[row * R.ldc[pid] + col] = (float)sum;
  }
}

void tc_set_ksplit(TcProblem& q, float* part, int64_t cap) {
  q.part = nullptr;
  q.kchunk = 0;
  if (!part || q.K <= TC_KCHUNK_MIN || (q.N & 1)) return;
  const int64_t tile = (int64_t)q.M * q.N;
  const int64_t fit = tile > 0 ? cap / tile : 0;
  if (fit < 2) return;
  // chunks of at least TC_KCHUNK_MIN, as many as the buffer holds
  int nch = (q.K + TC_KCHUNK_MIN - 1) / TC_KCHUNK_MIN;
  if (nch > fit) nch = (int)fit;
  int kc = (q.K + nch - 1) / nch;
  kc = (kc + TC_BK - 1) / TC_BK * TC_BK;
  if (kc >= q.K) return;
  q.part = part;
  q.kchunk = kc;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

static void load_encode() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
}

bool tc_available() {
  load_encode();
  return g_encode != nullptr;
}

static void encode_map(CUtensorMap* map, const float* base, int rows, int k, int64_t ld, int box_rows) {
  if (((uintptr_t)base & 15) != 0 || (ld * 4) % 16 != 0)
    fail(TDVP_EINVAL, "tensor-core operand not 16-byte aligned");
  cuuint64_t gdim[2] = {(cuuint64_t)k, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {TC_BK, (cuuint32_t)box_rows};
  cuuint32_t estride[2] = {1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, gdim, gstride, box, estride,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(TDVP_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
}

// One launch of the problems [base, end) (at most TC_MAXP) with N tile BN, then
// the FP64 sum of their K-split partial tiles.
template <int BN>
static void tc_launch_range(const std::vector<TcProblem>& probs, size_t base, size_t end, int passes,
                            int* d_status, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  TcTile<BN>::SMEM));
    attr_set = true;
  }
  {
    TcParams* P = new TcParams();
    std::unique_ptr<TcParams> guard(P);
    P->n = 0;
    P->passes = passes;
    P->status = d_status;
    int max_tiles = 0;
    for (size_t i = base; i < end; ++i) {
      const TcProblem& q = probs[i];
      if (q.M <= 0 || q.N <= 0 || q.K <= 0) continue;
      const int n = P->n;
      encode_map(&P->mapA[n][0], q.A.hi, q.A.rows, q.A.k, q.A.ld, TC_BM);
      encode_map(&P->mapB[n][0], q.B.hi, q.B.rows, q.B.k, q.B.ld, BN);
      if (passes == 3) {
        encode_map(&P->mapA[n][1], q.A.lo, q.A.rows, q.A.k, q.A.ld, TC_BM);
        encode_map(&P->mapB[n][1], q.B.lo, q.B.rows, q.B.k, q.B.ld, BN);
      } else {
        P->mapA[n][1] = P->mapA[n][0];
        P->mapB[n][1] = P->mapB[n][0];
      }
      P->M[n] = q.M;
      P->N[n] = q.N;
      P->K[n] = q.K;
      P->C[n] = q.C;
      P->skip[n] = q.skip;
      P->ldc[n] = q.ldc;
      P->c_fp64[n] = q.c_fp64;
      const bool split = q.part && q.kchunk > 0 && q.kchunk < q.K && q.kchunk % TC_BK == 0;
      P->part[n] = split ? q.part : nullptr;
      P->kcb[n] = split ? q.kchunk / TC_BK : 0;
      P->nch[n] = split ? cdiv(q.K, q.kchunk) : 1;
      max_tiles = std::max(max_tiles, cdiv(q.M, TC_BM) * cdiv(q.N, BN) * P->nch[n]);
      ++P->n;
    }
    if (P->n == 0) return;
    double fl = 0, by = 0, by_red = 0;
    bool any_split = false;
    for (int i = 0; i < P->n; ++i) {
      const double mn = (double)P->M[i] * P->N[i];
      fl += 2.0 * mn * P->K[i];
      by += 4.0 * ((double)P->M[i] + P->N[i]) * P->K[i] * passes;
      if (P->nch[i] > 1) {
        any_split = true;
        by += 4.0 * mn * P->nch[i];
        by_red += (4.0 * P->nch[i] + (P->c_fp64[i] ? 8.0 : 4.0)) * mn;
      } else {
        by += (P->c_fp64[i] ? 8.0 : 4.0) * mn;
      }
    }
    {
      ProfScope ps(passes == 3 ? "tc_gemm_tf32x3" : "tc_gemm_tf32", s, fl, by);
      dim3 grid(max_tiles, P->n);
      tc_gemm_kernel<BN><<<grid, 128, TcTile<BN>::SMEM, s>>>(*P);
      LAUNCH_CHECK();
      ++g_launches;
    }
    if (any_split) {
      TcReduce R{};
      R.n = P->n;
      int64_t max_mn = 0;
      for (int i = 0; i < P->n; ++i) {
        R.part[i] = P->part[i];
        R.C[i] = P->C[i];
        R.skip[i] = P->skip[i];
        R.ldc[i] = P->ldc[i];
        R.M[i] = P->M[i];
        R.N[i] = P->N[i];
        R.c_fp64[i] = P->c_fp64[i];
        // problems without a split were written by the GEMM itself
        R.nch[i] = P->nch[i];
        if (P->nch[i] <= 1) R.M[i] = 0;
        max_mn = std::max<int64_t>(max_mn, (int64_t)R.M[i] * R.N[i]);
      }
      ProfScope ps("tc_reduce", s, 0.0, by_red);
      dim3 grid((unsigned)std::min<int64_t>(cdiv64(max_mn, 256), 152 * 4), R.n);
      tc_reduce_kernel<<<grid, 256, 0, s>>>(R);
      LAUNCH_CHECK();
      ++g_launches;
    }
  }
}


void launch_tc_gemm(const std::vector<TcProblem>& probs, int passes, int* d_status, cudaStream_t s) {
  if (probs.empty()) return;
  load_encode();
  if (!g_encode) fail(TDVP_ECUDA, "cuTensorMapEncodeTiled unavailable");
  for (size_t base = 0; base < probs.size(); base += TC_MAXP) {
    const size_t end = std::min(probs.size(), base + (size_t)TC_MAXP);
    int64_t M = 0, N = 0, K = 0;
    for (size_t i = base; i < end; ++i) {
      M = std::max<int64_t>(M, probs[i].M);
      N = std::max<int64_t>(N, probs[i].N);
      K = std::max<int64_t>(K, probs[i].K);
    }
    auto run = [&](int c) {
      if (c == 0) tc_launch_range<256>(probs, base, end, passes, d_status, s);
      else tc_launch_range<128>(probs, base, end, passes, d_status, s);
    };
    if (!tune_enabled()) run(0);
    else tune_pick(passes == 3 ? TUNE_TC_TF32X3 : TUNE_TC_TF32, M, N, K, (int)(end - base), 2, true, run, s);
  }
}

}  // namespace tdvp
