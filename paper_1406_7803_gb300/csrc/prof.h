// prof.h -- optional per-kernel CUDA-event timing of the library's own launches.
//
// When a context enables profiling, each launch wrapped in a ProfScope records a pair of
// events on the launch stream; fde_profile_get sums their elapsed times per kernel name.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

namespace fde {

struct Profiler {
  bool on = false;
  int level = 1;  // record scopes of this level or below: 1 the H psi passes, 2 every kernel
  long long launches = 0;  // kernel launches made by the context's calls (always counted)
  struct Rec {
    std::vector<cudaEvent_t> a, b;
  };
  std::map<std::string, Rec> recs;
  void mark(const char* name, cudaStream_t st, bool begin) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, st);
    Rec& r = recs[name];
    (begin ? r.a : r.b).push_back(e);
  }
  void reset() {
    for (auto& kv : recs) {
      for (auto e : kv.second.a) cudaEventDestroy(e);
      for (auto e : kv.second.b) cudaEventDestroy(e);
    }
    recs.clear();
  }
  bool get(const std::string& name, int* n, double* ms) {
    auto it = recs.find(name);
    *n = 0;
    *ms = 0;
    if (it == recs.end()) return false;
    const size_t m = std::min(it->second.a.size(), it->second.b.size());
    for (size_t i = 0; i < m; ++i) {
      float t = 0;
      cudaEventSynchronize(it->second.b[i]);
      if (cudaEventElapsedTime(&t, it->second.a[i], it->second.b[i]) == cudaSuccess) *ms += t;
    }
    *n = (int)m;
    return true;
  }
  ~Profiler() { reset(); }
};

// Profiler of the context whose ABI call is running on this thread (or null).
extern thread_local Profiler* tl_prof;

inline void count_launches(int n) {
  if (tl_prof) tl_prof->launches += n;
}

struct ProfScope {
  const char* n;
  cudaStream_t st;
  bool rec;
  ProfScope(const char* name, cudaStream_t s, int lvl = 2)
      : n(name), st(s), rec(tl_prof && tl_prof->on && lvl <= tl_prof->level) {
    if (rec) tl_prof->mark(n, st, true);
  }
  ~ProfScope() {
    if (rec) tl_prof->mark(n, st, false);
  }
};

}  // namespace fde
