// Launch profiling: CUDA event pairs recorded on the launching stream around
// instrumented launches, bucketed by kernel category (see Cat).  Off by
// default; gbf_profile(1) clears and enables, gbf_profile_read sums.
#include <mutex>
#include <vector>

#include "gbf_common.cuh"
#include "gbfeast.h"

namespace gbf {
thread_local int g_cat = CAT_OTHER;

namespace {
struct Rec {
  cudaEvent_t a, b;
  int cat;
  double flops;
  int tc;          // 1: a sliced tensor-core GEMM kernel
  double tflops;   // bf16 tensor flops it issues
};
std::mutex mu;
bool enabled = false;
std::vector<Rec> recs;     // in use
std::vector<cudaEvent_t> pool;

cudaEvent_t get_event() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
const char *names[CAT_COUNT] = {"lu_update_gemm", "lu_panel", "lu_swap_trsm", "solve_gemm", "project_gemm_fp64", "reduced_eig",
                                "other"};
}  // namespace

bool prof_on() { return enabled; }

int prof_begin(cudaStream_t st) {
  if (!enabled) return -1;
  std::lock_guard<std::mutex> lk(mu);
  Rec r{get_event(), get_event(), g_cat, 0.0, 0, 0.0};
  if (!r.a || !r.b) return -1;
  cudaEventRecord(r.a, st);
  recs.push_back(r);
  return (int)recs.size() - 1;
}

void prof_end(cudaStream_t st, int slot, double flops) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(mu);
  if (slot >= (int)recs.size()) return;
  recs[slot].flops = flops;
  cudaEventRecord(recs[slot].b, st);
}

void prof_set_flops(int slot, double flops) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(mu);
  if (slot < (int)recs.size()) recs[slot].flops = flops;
}

void prof_end_tc(cudaStream_t st, int slot, double flops, double tensor_flops) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(mu);
  if (slot >= (int)recs.size()) return;
  recs[slot].flops = flops;
  recs[slot].tc = 1;
  recs[slot].tflops = tensor_flops;
  cudaEventRecord(recs[slot].b, st);
}
}  // namespace gbf

using namespace gbf;

extern "C" int gbf_profile(int enable) {
  std::lock_guard<std::mutex> lk(mu);
  for (auto &r : recs) {
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  recs.clear();
  enabled = enable != 0;
  return 0;
}

extern "C" int gbf_profile_categories(void) { return CAT_COUNT; }

extern "C" const char *gbf_profile_name(int cat) { return (cat >= 0 && cat < CAT_COUNT) ? names[cat] : ""; }

extern "C" int gbf_profile_read(int cat, long long *launches, double *ms, double *flops) {
  std::lock_guard<std::mutex> lk(mu);
  long long n = 0;
  double t = 0.0, f = 0.0;
  for (auto &r : recs) {
    if (r.cat != cat) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return -4;
    float x = 0.f;
    if (cudaEventElapsedTime(&x, r.a, r.b) != cudaSuccess) return -4;
    ++n;
    t += x;
    f += r.flops;
  }
  if (launches) *launches = n;
  if (ms) *ms = t;
  if (flops) *flops = f;
  return 0;
}

extern "C" int gbf_profile_tc(long long *launches, double *ms, double *flops, double *tensor_flops) {
  std::lock_guard<std::mutex> lk(mu);
  long long n = 0;
  double t = 0.0, f = 0.0, tf = 0.0;
  for (auto &r : recs) {
    if (!r.tc) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return -4;
    float x = 0.f;
    if (cudaEventElapsedTime(&x, r.a, r.b) != cudaSuccess) return -4;
    ++n;
    t += x;
    f += r.flops;
    tf += r.tflops;
  }
  if (launches) *launches = n;
  if (ms) *ms = t;
  if (flops) *flops = f;
  if (tensor_flops) *tensor_flops = tf;
  return 0;
}
