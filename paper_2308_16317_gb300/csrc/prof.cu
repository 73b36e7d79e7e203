// Per-phase instrumentation of the library's launches (not part of the
// paper's method): when enabled, CUDA events are recorded on the launching
// stream around every phase, so a caller can time individual kernels inside
// a larger timed region; a launch counter is always kept.
#include <atomic>
#include <mutex>
#include <vector>

#include "prof.h"

namespace {

struct Rec {
  int phase;
  cudaEvent_t a, b;
};

std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
std::atomic<int> g_enabled{0};
std::atomic<long long> g_launches{0};
long long g_phase_launches[PH_COUNT] = {0};
long long g_phase_items[PH_COUNT] = {0};
unsigned long long* g_dwork = nullptr;   // device counters of items processed (data-dependent phases)

const char* kNames[PH_COUNT] = {"assemble", "panel", "row_swap", "trsm", "pack", "trailing_update",
                                "schur_inverse", "residual", "correction", "other", "kkr_real_terms",
                                "kkr_recip", "kkr_realsum", "kkr_invert"};

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

}  // namespace

ProfScope::ProfScope(int phase, cudaStream_t st) : phase_(phase), st_(st), a_(nullptr) {
  if (!g_enabled.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  a_ = take_event();
  cudaEventRecord(static_cast<cudaEvent_t>(a_), st_);
}

ProfScope::~ProfScope() {
  if (!a_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take_event();
  cudaEventRecord(b, st_);
  g_recs.push_back(Rec{phase_, static_cast<cudaEvent_t>(a_), b});
}

void prof_launched(int phase, int n, long long items) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  if (g_enabled.load(std::memory_order_relaxed)) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_phase_launches[phase] += n;
    if (items > 0) g_phase_items[phase] += items;
  }
}

unsigned long long* prof_work_counter(int phase) {
  if (!g_enabled.load(std::memory_order_relaxed)) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dwork) {
    if (cudaMalloc(&g_dwork, sizeof(unsigned long long) * PH_COUNT) != cudaSuccess) {
      g_dwork = nullptr;
      return nullptr;
    }
    cudaMemset(g_dwork, 0, sizeof(unsigned long long) * PH_COUNT);
    cudaDeviceSynchronize();
  }
  return g_dwork + phase;
}

int prof_suspend() {
  std::lock_guard<std::mutex> lk(g_mu);
  const int was = g_enabled.load();
  g_enabled.store(0);
  return was;
}

void prof_resume(int state) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_enabled.store(state);
}

void prof_add_launches(long long n) { g_launches.fetch_add(n); }

extern "C" {

void must_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_enabled.store(on ? 1 : 0);
}

int must_profile_read(double* ms, long long* launches, long long* items, int n_phases) {
  std::lock_guard<std::mutex> lk(g_mu);
  const int n = n_phases < PH_COUNT ? n_phases : PH_COUNT;
  unsigned long long dw[PH_COUNT] = {0};
  if (g_dwork) {
    cudaDeviceSynchronize();
    cudaMemcpy(dw, g_dwork, sizeof(dw), cudaMemcpyDeviceToHost);
    cudaMemset(g_dwork, 0, sizeof(dw));
  }
  for (int p = 0; p < n; ++p) {
    if (ms) ms[p] = 0.0;
    if (launches) launches[p] = g_phase_launches[p];
    if (items) items[p] = g_phase_items[p] + (long long)dw[p];
  }
  for (const Rec& r : g_recs) {
    cudaEventSynchronize(r.b);
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess && r.phase < n && ms) ms[r.phase] += t;
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  for (int p = 0; p < PH_COUNT; ++p) g_phase_launches[p] = g_phase_items[p] = 0;
  return PH_COUNT;
}

long long must_launch_count(void) { return g_launches.load(); }

const char* must_phase_name(int phase) { return (phase >= 0 && phase < PH_COUNT) ? kNames[phase] : "?"; }

}  // extern "C"
