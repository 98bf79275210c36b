// Per-kernel launch statistics of a context: a launch counter that is always on, and, while
// profiling is enabled, CUDA events around every launch on the launching stream together
// with the launch's algorithmic bytes (operands read once, results written once) and flops.
#ifndef PV_PROF_CUH
#define PV_PROF_CUH
#include <cuda_runtime.h>
#include <cstring>
#include <string>
#include <vector>

namespace pv {

struct KProf {
  struct Rec {
    const char* name;
    double bytes, flops;
  };
  struct Acc {
    std::string name;
    long long launches = 0;
    double ms = 0, bytes = 0, flops = 0;
  };
  bool on = false;
  bool gemm_only = false;   // time only the batched GEMM kernels (names kb_gemm*)
  long long launches = 0;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<Rec> recs;
  std::vector<Acc> acc;

  ~KProf() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
  bool wanted(const char* name) const {
    return on && (!gemm_only || strncmp(name, "kb_gemm", 7) == 0);
  }
  void begin(cudaStream_t st, const char* name) {
    ++launches;
    if (!wanted(name)) return;
    if (used + 2 > pool.size()) {
      for (int i = 0; i < 4096; ++i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
          cudaGetLastError();
          on = false;
          return;
        }
        pool.push_back(e);
      }
    }
    cudaEventRecord(pool[used], st);
  }
  void end(cudaStream_t st, const char* name, double bytes, double flops) {
    if (!wanted(name) || used + 2 > pool.size()) return;
    cudaEventRecord(pool[used + 1], st);
    used += 2;
    recs.push_back(Rec{name, bytes, flops});
  }
  // Folds the recorded launches into the per-kernel sums; the caller has synchronised.
  void fold() {
    for (size_t i = 0; i < recs.size(); ++i) {
      float ms = 0;
      cudaEventElapsedTime(&ms, pool[2 * i], pool[2 * i + 1]);
      Acc* a = nullptr;
      for (Acc& x : acc)
        if (x.name == recs[i].name) a = &x;
      if (!a) {
        acc.push_back(Acc());
        a = &acc.back();
        a->name = recs[i].name;
      }
      a->launches += 1;
      a->ms += ms;
      a->bytes += recs[i].bytes;
      a->flops += recs[i].flops;
    }
    recs.clear();
    used = 0;
  }
  void reset() {
    recs.clear();
    used = 0;
    acc.clear();
  }
};

// Brackets one launch statement: counts it and, when profiling, times it.
#define PV_KLAUNCH(prof, st, name, bytes, flops, ...) \
  do {                                                \
    if (prof) (prof)->begin(st, name);                \
    __VA_ARGS__;                                      \
    if (prof) (prof)->end(st, name, bytes, flops);    \
  } while (0)

}  // namespace pv
#endif
