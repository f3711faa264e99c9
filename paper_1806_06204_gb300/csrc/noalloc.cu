// Allocation-free entry point: the split-precision FP64 GEMM of zolo_dgemm with
// its scratch (the BF16 slice planes, the per-row/column exponents and the
// kernel's error flag) in one file-scope device array instead of memory from
// cudaMalloc.  It exists for callers that cannot allocate device memory at the
// point of the call: code whose device memory is owned by an external
// allocator or reserved up front, and code that must not call cudaMalloc or
// cudaFree while it runs.
//
// The array is 16 MiB and every GPU that loads this library holds it until the
// process exits.  Its device address is looked up once per device, on the
// first call made with that device current (cudaGetSymbolAddress).  Every call
// shares the array and it
// keeps the previous call's contents: the error flag is cleared at the start
// of each call, the slices and exponents are rewritten before they are read.
// Calls whose work overlaps on the GPU (other streams, other host threads)
// race on the array and must be serialised by the caller.
#include <mutex>

#include "../../include/zolo.h"
#include "zolo_internal.h"

namespace zolo {
namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;   // 16 MiB
constexpr size_t kErrBytes = 256;                    // the error flag, padded
constexpr size_t kExpBytes = size_t(64) << 10;       // 16384 exponents
constexpr size_t kSliceBytes = kScratchBytes - kErrBytes - kExpBytes;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ZOLO_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return ZOLO_ECUDA;
    }
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return 0;
}

}  // namespace
}  // namespace zolo

using namespace zolo;

extern "C" int zolo_dgemm_noalloc(int transA, int transB, int64_t m, int64_t n, int64_t k,
                                  double alpha, const double* A, int64_t lda, const double* B,
                                  int64_t ldb, double beta, double* C, int64_t ldc, int slices,
                                  void* stream) {
  if (transA != 0 && transA != 1) return -1;
  if (transB != 0 && transB != 1) return -2;
  if (m < 0 || m > INT32_MAX) return -3;
  if (n < 0 || n > INT32_MAX) return -4;
  if (k < 0 || k > INT32_MAX) return -5;
  if (!(alpha == alpha) || alpha - alpha != 0.0) return -6;
  if (k > 0 && m > 0 && !A) return -7;
  if (lda < (transA ? (k > 1 ? k : 1) : (m > 1 ? m : 1))) return -8;
  if (k > 0 && n > 0 && !B) return -9;
  if (ldb < (transB ? (n > 1 ? n : 1) : (k > 1 ? k : 1))) return -10;
  if (!(beta == beta) || beta - beta != 0.0) return -11;
  if (m > 0 && n > 0 && !C) return -12;
  if (ldc < (m > 1 ? m : 1)) return -13;
  if (slices != 0 && slices != 8 && slices != 9) return -14;
  const int S = slices ? slices : 8;
  // sizes beyond what the fixed scratch holds are refused before any device work
  // (the same counts gemm_split checks against, so a size accepted here runs)
  const size_t need = split_slice_elems(m, n, k, 1, S) * 2;
  const size_t exps = split_exp_elems(m, n, k, 1, 0);
  if (need > kSliceBytes || exps * sizeof(int) > kExpBytes) return ZOLO_ENOMEM;
  void* base = nullptr;
  if (int e = scratch_address(&base)) return e;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* b = static_cast<unsigned char*>(base);
  SplitWork w;
  w.err = reinterpret_cast<int*>(b);
  w.exps = reinterpret_cast<int*>(b + kErrBytes);
  w.exp_elems = kExpBytes / sizeof(int);
  w.slices = b + kErrBytes + kExpBytes;
  w.slice_elems = kSliceBytes / 2;
  w.slices_s = S;
  if (cudaMemsetAsync(w.err, 0, sizeof(int), st) != cudaSuccess) return ZOLO_ECUDA;
  GemmArgs g;
  g.M = (int)m; g.N = (int)n; g.K = (int)k; g.transA = transA; g.transB = transB;
  g.A = A; g.lda = lda; g.B = B; g.ldb = ldb;
  g.Cin = beta != 0.0 ? C : nullptr; g.ldcin = ldc; g.beta = beta;
  g.Cout = C; g.ldcout = ldc;
  g.alpha[0] = alpha;
  if (gemm_split(g, w, st) != cudaSuccess) return ZOLO_ECUDA;
  int herr = 0;
  if (cudaMemcpyAsync(&herr, w.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ZOLO_ECUDA;
  return herr ? ZOLO_ETIMEOUT : 0;
}
