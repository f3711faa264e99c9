// Launch counting and opt-in per-kernel-class timing with CUDA events.
//
// Every launch site constructs a ProfScope around its <<<>>>: the process-wide
// counter always advances; while profiling is on, an event pair is recorded on
// the launching stream and the pair is resolved (one synchronisation) when the
// statistics are read.  Flops/bytes are the algorithmic counts the call site
// states for that launch.
#include <atomic>
#include <cstring>
#include <mutex>
#include <set>
#include <utility>
#include <map>
#include <tuple>
#include <vector>

#include "../../include/zolo.h"
#include "zolo_internal.h"

namespace zolo {
namespace {

const char* kClassNames[kProfClasses] = {"gemm_f64", "qr_panel", "chol_diag", "jacobi_round",
                                         "combine", "other", "gemm_split", "slice", "jacobi32_sweep"};

struct Pending {
  int cls;
  cudaEvent_t a, b;
  double flops, bytes, share;
};

std::atomic<uint64_t> g_launches{0};
std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
zolo_kstat_t g_acc[kProfClasses];

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void resolve_locked() {
  for (Pending& p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      zolo_kstat_t& s = g_acc[p.cls];
      s.launches += 1;
      s.ms += ms;
      s.flops += p.flops;
      s.bytes += p.bytes;
      s.sm_ms += ms * p.share;
    }
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pending.clear();
}

void reset_locked() {
  resolve_locked();
  for (int c = 0; c < kProfClasses; ++c) {
    std::memset(&g_acc[c], 0, sizeof(g_acc[c]));
    std::strncpy(g_acc[c].name, kClassNames[c], sizeof(g_acc[c].name) - 1);
  }
}

}  // namespace

ProfScope::ProfScope(int cls, cudaStream_t st, double flops, double bytes)
    : cls_(cls), st_(st), flops_(flops), bytes_(bytes) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (g_on.load(std::memory_order_relaxed) && cudaStreamIsCapturing(st, &cs) == cudaSuccess &&
      cs == cudaStreamCaptureStatusNone) {
    std::lock_guard<std::mutex> lk(g_mu);
    a_ = take_event();
    cudaEventRecord(static_cast<cudaEvent_t>(a_), st_);
  }
}

ProfScope::~ProfScope() {
  if (!a_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take_event();
  cudaEventRecord(b, st_);
  g_pending.push_back({cls_, static_cast<cudaEvent_t>(a_), b, flops_, bytes_, share_});
  if (g_pending.size() > 100000) resolve_locked();
}

void ProfScope::blocks(const void* kernel, dim3 block, size_t smem, dim3 grid) {
  if (!a_) return;
  const int threads = (int)(block.x * block.y * block.z);
  const double count = (double)grid.x * grid.y * grid.z;
  // (kernel, threads, smem) -> resident blocks per SM; SM count per device
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t, int>, int> occ;
  int dev = 0, per_sm = 1, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(kernel, threads, smem, dev);
    auto it = occ.find(key);
    if (it == occ.end()) {
      int o = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel, threads, smem) != cudaSuccess)
        o = 1;
      it = occ.emplace(key, o < 1 ? 1 : o).first;
    }
    per_sm = it->second;
  }
  const double f = count / ((double)sms * per_sm);
  share_ = f < 1.0 ? f : 1.0;
}

void add_launches(int64_t n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

bool profiling_enabled() { return g_on.load(std::memory_order_relaxed); }

cudaError_t smem_attr_once(const void* func, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;   // (kernel, device)
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({func, dev})) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.insert({func, dev});
  return e;
}

}  // namespace zolo

using namespace zolo;

extern "C" {

uint64_t zolo_kernel_launches(void) { return g_launches.load(); }

int zolo_profile(int enable) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (enable) reset_locked();
  g_on.store(enable != 0);
  return 0;
}

int zolo_profile_read(zolo_kstat_t* out, int max_entries) {
  std::lock_guard<std::mutex> lk(g_mu);
  resolve_locked();
  const int n = max_entries < kProfClasses ? max_entries : kProfClasses;
  for (int c = 0; c < n && out; ++c) out[c] = g_acc[c];
  return kProfClasses;
}

}  // extern "C"
