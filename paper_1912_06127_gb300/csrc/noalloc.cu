// H_eff . x without any device allocation, for callers that cannot allocate.
//
// Some callers cannot call cudaMalloc: plug-ins whose host application owns
// every device allocation through its own pool and forbids others, or
// real-time loops that must never enter an allocator (whose cost and locking
// are unbounded). For them tdvp_op_heff_noalloc runs the FP64 two- or
// one-site H_eff application of tdvp_op_heff with its two intermediates (the
// L-contracted state and the MPO-applied state) and the sparse MPO blocks
// placed in one file-scope device array of TDVP_NOALLOC_SCRATCH_BYTES bytes.
// That array exists on every GPU that loads the library and is held until the
// process exits.
//
// The host cannot use the array's name as a device address, so its address
// is looked up with cudaGetSymbolAddress once per device, with that device
// current, on the first call made on that device; that first call should
// therefore come before any stream capture. Every call shares the array and
// finds it holding the previous call's data: nothing in it has to start at
// zero (every intermediate is fully overwritten before it is read), but two
// calls whose work overlaps on the GPU (different streams, or different host
// threads on the same device) race on it and must be serialised by the caller.
//
// Each call builds the sparse two-site operator W_j W_{j+1} on the host
// (O(m^3 d^4) operations: ~1e5 for m = 10, d = 2) and copies it from host
// memory, then synchronises the stream before returning.
#include <mutex>

#include "common.h"

namespace tdvp {

// 32 MiB: two intermediates of chi_l * m * D * chi_r complex doubles each
// (D = d^2 for two sites) plus the MPO blocks, so 2 * chi_l * m * D * chi_r * 16
// bytes must stay below it: e.g. chi = 128 with m = 14 and two sites
// (29.4 MB), or chi = 256 with m = 6 and one site (25.2 MB).
static __device__ __align__(256) unsigned char g_noalloc_scratch[TDVP_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_mu;
void* g_scratch_ptr[64] = {};

void* scratch_for_current_device() {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) fail(TDVP_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      fail(TDVP_ECUDA, std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                           cudaGetErrorString(e));
    }
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

void op_heff_noalloc(int nsite, int chi_l, int chi_r, int m, int d, const double* W, const double* L,
                     const double* R, const double* x, double* y, cudaStream_t s) {
  // the dimension bounds of tdvp_op_heff, plus a bound on the MPO bond
  // dimension that keeps the host-side operator build small, all checked
  // before anything is built
  if ((nsite != 1 && nsite != 2) || chi_l < 1 || chi_r < 1 || m < 1 || d < 2 || d > 4 || chi_l > 4096 ||
      chi_r > 4096)
    fail(TDVP_EINVAL, "invalid dimensions");
  if (m > TDVP_NOALLOC_MAX_M)
    fail(TDVP_EINVAL, "tdvp_op_heff_noalloc: m = " + std::to_string(m) + " above TDVP_NOALLOC_MAX_M = " +
                          std::to_string(TDVP_NOALLOC_MAX_M));
  const int D = nsite == 2 ? d * d : d;
  {
    const size_t need = 2 * (size_t)chi_l * m * D * chi_r * sizeof(double2);
    if (need > (size_t)TDVP_NOALLOC_SCRATCH_BYTES)
      fail(TDVP_EINVAL, "tdvp_op_heff_noalloc: problem needs " + std::to_string(need) +
                            " bytes of scratch for its intermediates, more than the fixed " +
                            std::to_string((size_t)TDVP_NOALLOC_SCRATCH_BYTES) +
                            " (use tdvp_op_heff for larger problems)");
  }
  // sparse MPO operator (CSR over the right bond index), built on the host
  std::vector<double2> Wd((const double2*)W, (const double2*)W + (size_t)m * m * d * d);
  std::vector<double2> Wop;
  if (nsite == 2) {
    Wop.assign((size_t)m * m * D * D, make_double2(0, 0));
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b)
        for (int c = 0; c < m; ++c)
          for (int s1 = 0; s1 < d; ++s1)
            for (int s2 = 0; s2 < d; ++s2)
              for (int t1 = 0; t1 < d; ++t1)
                for (int t2 = 0; t2 < d; ++t2) {
                  const double2 w1 = Wd[(((size_t)a * m + b) * d + s1) * d + t1];
                  const double2 w2 = Wd[(((size_t)b * m + c) * d + s2) * d + t2];
                  double2& r = Wop[(((size_t)a * m + c) * D + (s1 * d + s2)) * D + (t1 * d + t2)];
                  r = zadd(r, zmul(w1, w2));
                }
  } else {
    Wop = Wd;
  }
  std::vector<int> cp(m + 1, 0), ri;
  std::vector<double2> blk;
  for (int o = 0; o < m; ++o) {
    cp[o] = (int)ri.size();
    for (int i = 0; i < m; ++i) {
      const double2* b = &Wop[((size_t)i * m + o) * D * D];
      bool nz = false;
      for (int q = 0; q < D * D; ++q) nz |= (b[q].x != 0.0 || b[q].y != 0.0);
      if (!nz) continue;
      ri.push_back(i);
      blk.insert(blk.end(), b, b + D * D);
    }
  }
  cp[m] = (int)ri.size();
  // layout of the scratch array
  const size_t nT = (size_t)chi_l * m * D * chi_r;
  size_t off_T1 = 0;
  size_t off_T2 = align256(off_T1 + nT * sizeof(double2));
  size_t off_cp = align256(off_T2 + nT * sizeof(double2));
  size_t off_ri = align256(off_cp + cp.size() * sizeof(int));
  size_t off_bk = align256(off_ri + std::max<size_t>(ri.size(), 1) * sizeof(int));
  size_t end = align256(off_bk + std::max<size_t>(blk.size(), 1) * sizeof(double2));
  if (end > (size_t)TDVP_NOALLOC_SCRATCH_BYTES)
    fail(TDVP_EINVAL, "tdvp_op_heff_noalloc: problem needs " + std::to_string(end) +
                          " bytes of scratch, more than the fixed " +
                          std::to_string((size_t)TDVP_NOALLOC_SCRATCH_BYTES) +
                          " (use tdvp_op_heff for larger problems)");
  unsigned char* base = (unsigned char*)scratch_for_current_device();
  double2* T1 = (double2*)(base + off_T1);
  double2* T2 = (double2*)(base + off_T2);
  int* d_cp = (int*)(base + off_cp);
  int* d_ri = (int*)(base + off_ri);
  double2* d_bk = (double2*)(base + off_bk);
  CUDA_TRY(cudaMemcpyAsync(d_cp, cp.data(), cp.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  if (!ri.empty()) {
    CUDA_TRY(cudaMemcpyAsync(d_ri, ri.data(), ri.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(d_bk, blk.data(), blk.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
  }
  const int A = chi_l, B = chi_r;
  ZGemmBatch g1{}, g2{};
  WStageBatch<double2> ws{};
  g1.n = g2.n = ws.n = 1;
  ZGemmDesc& a = g1.d[0];
  a = ZGemmDesc{};
  a.M = A * m;
  a.N = D * B;
  a.K = A;
  a.A = (const double2*)L;
  a.a_rs = A;
  a.a_cs = 1;
  a.B = (const double2*)x;
  a.b_rs = (int64_t)D * B;
  a.b_cs = 1;
  a.C = T1;
  a.c_rs = (int64_t)D * B;
  a.c_cs = 1;
  WStageDesc<double2>& w = ws.d[0];
  w = WStageDesc<double2>{};
  w.A = A;
  w.B = B;
  w.X = T1;
  w.x_a = (int64_t)m * D * B;
  w.x_w = (int64_t)D * B;
  w.x_s = B;
  w.x_b = 1;
  w.Y = T2;
  w.y_a = (int64_t)D * m * B;
  w.y_w = B;
  w.y_s = (int64_t)m * B;
  w.y_b = 1;
  w.W = WOp{m, D, (int)ri.size(), d_cp, d_ri, d_bk, nullptr};
  ZGemmDesc& b = g2.d[0];
  b = ZGemmDesc{};
  b.M = A * D;
  b.N = B;
  b.K = m * B;
  b.A = T2;
  b.a_rs = (int64_t)m * B;
  b.a_cs = 1;
  b.B = (const double2*)R;
  b.b_rs = 1;
  b.b_cs = (int64_t)m * B;
  b.C = (double2*)y;
  b.c_rs = B;
  b.c_cs = 1;
  launch_zgemm(g1, s);
  launch_wstage(ws, s);
  launch_zgemm(g2, s);
  CUDA_TRY(cudaStreamSynchronize(s));
}

}  // namespace tdvp
