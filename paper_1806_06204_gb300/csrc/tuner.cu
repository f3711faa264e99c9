// Kernel choice per contraction shape: built-in rules, or a measured choice.
//
// Every contraction of the iteration (QR trailing updates, the r-way sums, the
// Gram matrices, the triangular-solve updates, the eigensolver's products) goes
// through gemm_any (FP64 or split tensor-core path) or gemm_f64 (FP64 only).
// Without a tuner both follow fixed rules: the split path where its cost model
// says it is faster, else the 64 x 64 FP64 tile (32 x 128 for M <= 32).  With
// a handle's tuner current and tuning on, the first call of a shape runs every
// candidate (three FP64 tile shapes, split-K in 2 / 4 / 8 slices when K holds
// at least two 16-deep steps per slice, and the split path when it is on) into
// a scratch output, times each with CUDA events on the call's stream, keeps
// the fastest in the handle's cache, and then runs it for real.  The real
// output is written once, by the chosen variant.
#include <algorithm>
#include <cfloat>
#include <vector>

#include "zolo_internal.h"

namespace zolo {
namespace {

thread_local GemmTuner* t_tuner = nullptr;

bool stream_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return true;   // unknown: do not synchronise or allocate
  }
  return cs != cudaStreamCaptureStatusNone;
}

// [lo, hi) of the elements a strided batch of column-major matrices touches
struct Extent {
  const double* lo;
  const double* hi;
};
Extent extent(const double* p, int64_t ld, int64_t rows, int64_t cols, int64_t stride, int count) {
  return {p, p + (int64_t)(count - 1) * stride + (cols - 1) * ld + rows};
}
bool overlap(Extent a, Extent b) { return a.lo < b.hi && b.lo < a.hi; }

int ksplit_of(int v) {
  return v == kGemmVSplitK2 ? 2 : v == kGemmVSplitK4 ? 4 : v == kGemmVSplitK8 ? 8 : 1;
}

cudaError_t run_variant(const GemmArgs& g, int v, SplitWork* split, double* scratch,
                        size_t scratch_elems, cudaStream_t st) {
  if (v == kGemmVSplit) {
    if (split) return gemm_split(g, *split, st);
    v = gemm_f64_default_variant(g);
  }
  return gemm_f64_variant(g, v, scratch, scratch_elems, st);
}

bool ensure_scratch(GemmTuner& t, size_t elems, cudaStream_t st) {
  if (t.scratch_elems >= elems) return true;
  if (cudaStreamSynchronize(st) != cudaSuccess) return false;
  if (t.scratch) cudaFree(t.scratch);
  t.scratch = nullptr;
  t.scratch_elems = 0;
  if (cudaMalloc(&t.scratch, elems * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  t.scratch_elems = elems;
  return true;
}

// Time every candidate of g's shape; returns the fastest (or -1 when tuning
// could not run: no scratch, a failed launch).  With the split path on, a shape
// whose estimated split time is under a quarter of the FP64 time is given to
// the split path untimed, and one estimated 4x slower on it is not timed
// there; a shape whose built-in kernel takes over 50 ms keeps it.  When the
// output overlaps A or B (a product computed in place, as the Cholesky panel
// update is) the only candidates are the built-in tile, which the call site is
// written for, and the variants that read all of A and B before writing C
// (split-K, split).
int tune(GemmTuner& t, const GemmArgs& g, SplitWork* split, cudaStream_t st) {
  const size_t out = (size_t)(g.reduce ? 1 : g.batch) * (size_t)g.M * (size_t)g.N;
  std::vector<int> cand = {kGemmV64x64, kGemmV32x128, kGemmV32x64};
  if (gemm_output_aliases_input(g)) cand = {gemm_f64_default_variant(g)};
  for (int v : {kGemmVSplitK2, kGemmVSplitK4, kGemmVSplitK8})
    if (g.K >= 2 * 16 * ksplit_of(v)) cand.push_back(v);
  if (split) {
    // where the estimate puts one path 4x ahead of the other, the slower one is
    // not timed (a large FP64 product takes seconds per candidate)
    const double ratio = split_time_ratio(g, *split);
    if (ratio < 0.25) return kGemmVSplit;
    if (ratio <= 4.0) cand.push_back(kGemmVSplit);
  }
  size_t part = 0;
  for (int v : cand) part = std::max(part, gemm_f64_scratch_elems(g, v));
  if (!ensure_scratch(t, out + part, st)) {
    // without split-K partials, if at least the output fits
    cand.erase(std::remove_if(cand.begin(), cand.end(),
                              [&](int v) { return gemm_f64_scratch_elems(g, v) > 0; }),
               cand.end());
    part = 0;
    if (!ensure_scratch(t, out, st)) return -1;
  }
  if (!t.t0 && (cudaEventCreate(&t.t0) != cudaSuccess || cudaEventCreate(&t.t1) != cudaSuccess))
    return -1;
  GemmArgs h = g;   // same inputs (Cin is only read), output to the scratch
  h.Cout = t.scratch;
  h.ldcout = g.M;
  h.strideCout = (int64_t)g.M * g.N;
  double* partials = t.scratch + out;
  // the built-in choice first: a shape that takes it over 50 ms keeps it (large
  // products already fill the GPU, and timing every candidate there would cost
  // seconds per shape)
  const int builtin = split && split_preferred(g, *split) ? (int)kGemmVSplit
                                                          : gemm_f64_default_variant(g);
  std::stable_partition(cand.begin(), cand.end(), [&](int v) { return v == builtin; });
  int best = -1;
  float best_ms = FLT_MAX;
  for (int v : cand) {
    float ms = FLT_MAX;
    for (int rep = 0; rep < 3; ++rep) {
      if (cudaEventRecord(t.t0, st) != cudaSuccess) return -1;
      if (run_variant(h, v, split, partials, part, st) != cudaSuccess) return -1;
      float x = 0.f;
      if (cudaEventRecord(t.t1, st) != cudaSuccess || cudaEventSynchronize(t.t1) != cudaSuccess ||
          cudaEventElapsedTime(&x, t.t0, t.t1) != cudaSuccess)
        return -1;
      ms = std::min(ms, x);
      if (ms > 5.f) break;   // long runs: one timing is enough
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = v;
    }
    if (v == builtin && ms > 50.f) return builtin;
  }
  return best;
}

// The tuned or built-in choice for g (split = the split engine, if allowed).
// In zolo_pd_batched's lanes (split->throughput) the GPU-throughput router alone
// decides the split path; a tuner there only picks among the FP64 kernels of the
// products the router leaves on the FP64 pipe (under the FP64-only key).
int choose(const GemmArgs& g, SplitWork* split_engine, cudaStream_t st) {
  const bool thr = split_engine && split_engine->throughput;
  if (thr && split_preferred(g, *split_engine)) return kGemmVSplit;
  SplitWork* split = thr ? nullptr : split_engine;
  GemmTuner* t = t_tuner;
  if (t && !t->busy) {
    // the split path's slice format in the key: S, plus 100 per form (FP16 108,
    // FP8 211)
    const auto key = gemm_key(g, split ? split->slices_s + 100 * split->form : 0);
    const auto hit = t->choice.find(key);
    if (hit != t->choice.end() && gemm_variant_allowed(key, hit->second)) {
      // a split-K choice (e.g. loaded from a file) needs its partial sums' scratch
      const size_t need = gemm_f64_scratch_elems(g, hit->second);
      if (need <= t->scratch_elems || (!stream_capturing(st) && ensure_scratch(*t, need, st)))
        return hit->second;
      return gemm_f64_default_variant(g);
    }
    if (t->tuning && !stream_capturing(st)) {
      t->busy = true;
      const int v = tune(*t, g, split, st);
      t->busy = false;
      cudaGetLastError();
      if (v >= 0) {
        t->choice[key] = v;
        ++t->gen;
        return v;
      }
    }
  }
  if (split && split_preferred(g, *split)) return kGemmVSplit;
  return gemm_f64_default_variant(g);
}

}  // namespace

GemmTuner::~GemmTuner() {
  if (scratch) cudaFree(scratch);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
}

bool gemm_output_aliases_input(const GemmArgs& g) {
  const Extent c = extent(g.Cout, g.ldcout, g.M, g.N, g.strideCout, g.reduce ? 1 : g.batch);
  const Extent a = extent(g.A, g.lda, g.transA ? g.K : g.M, g.transA ? g.M : g.K, g.strideA,
                          g.batch);
  const Extent b = extent(g.B, g.ldb, g.transB ? g.N : g.K, g.transB ? g.K : g.N, g.strideB,
                          g.batch);
  return overlap(c, a) || overlap(c, b);
}

std::array<int, 7> gemm_key(const GemmArgs& g, int split_slices) {
  const int flags = (g.transA ? 1 : 0) | (g.transB ? 2 : 0) | (g.reduce ? 4 : 0) |
                    (g.b_lower ? 8 : 0) | (g.c_upper ? 16 : 0) |
                    (g.Cin && g.beta != 0.0 ? 32 : 0) | (g.k_equilibrate ? 64 : 0) |
                    (gemm_output_aliases_input(g) ? 128 : 0);
  return {g.M, g.N, g.K, g.batch, flags, split_slices, 0};
}

bool gemm_variant_allowed(const std::array<int, 7>& key, int v) {
  const bool split_k = v == kGemmVSplitK2 || v == kGemmVSplitK4 || v == kGemmVSplitK8;
  const bool tiles = v == kGemmV64x64 || v == kGemmV32x128 || v == kGemmV32x64;
  if (v == kGemmVSplit) return key[5] != 0;
  if (!split_k && !tiles) return false;
  if (!(key[4] & 128) || split_k) return true;
  // in place: only the built-in tile for this M
  return v == (key[0] <= 32 ? kGemmV32x128 : kGemmV64x64);
}

void set_gemm_tuner(GemmTuner* t) { t_tuner = t; }
GemmTuner* get_gemm_tuner() { return t_tuner; }

cudaError_t gemm_f64(const GemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.batch <= 0 || g.batch > kGemmMaxBatch)
    return gemm_f64_variant(g, kGemmV64x64, nullptr, 0, st);
  const int v = choose(g, nullptr, st);
  GemmTuner* t = t_tuner;
  return gemm_f64_variant(g, v, t ? t->scratch : nullptr, t ? t->scratch_elems : 0, st);
}

cudaError_t gemm_any(const GemmArgs& g, cudaStream_t st) {
  SplitWork* split = get_split_engine();
  if (!split || g.M <= 0 || g.N <= 0 || g.K <= 0 || g.batch > kGemmMaxBatch)
    return gemm_f64(g, st);
  const int v = choose(g, split, st);
  GemmTuner* t = t_tuner;
  return run_variant(g, v, split, t ? t->scratch : nullptr, t ? t->scratch_elems : 0, st);
}

}  // namespace zolo
