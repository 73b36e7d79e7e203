// Phase timers and launch counting (see prof.cu).
#pragma once
#include <cuda_runtime.h>

enum MustPhase {
  PH_ASSEMBLE = 0,
  PH_PANEL,
  PH_SWAP,
  PH_TRSM,
  PH_PACK,
  PH_UPDATE,
  PH_SCHUR,
  PH_RESIDUAL,
  PH_CORRECT,
  PH_OTHER,
  PH_KKR_TERMS,    // full KKR: k-independent real-space Ewald terms
  PH_KKR_RECIP,    // full KKR: reciprocal-space Ewald sums
  PH_KKR_REALSUM,  // full KKR: real-space Ewald sums
  PH_KKR_INVERT,   // full KKR: M(k) assembly, inversion, Brillouin-zone sum
  PH_COUNT
};

// Records CUDA events around the enclosed launches when profiling is on.
class ProfScope {
 public:
  ProfScope(int phase, cudaStream_t st);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  int phase_;
  cudaStream_t st_;
  void* a_;
};

// Count n kernel launches of a phase that together process `items` matrices
// (0 when the kernels count their own items through prof_work_counter).
void prof_launched(int phase, int n, long long items = 0);

// Device counter (items processed) for phases whose work depends on data
// (refinement kernels skip converged items), or NULL when profiling is off.
unsigned long long* prof_work_counter(int phase);

// Suspend event recording (returns the previous state) during graph capture.
int prof_suspend();
void prof_resume(int state);
// Adjust the global launch counter (graph replays add their kernel count).
void prof_add_launches(long long n);
extern "C" long long must_launch_count(void);
