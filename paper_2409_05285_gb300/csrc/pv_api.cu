// C ABI of the PEPS-VMC cooling step (declarations and contracts: include/peps_vmc.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/peps_vmc.h"
#include "pv_philox.cuh"
#include "pv_sample.cuh"
#include "pv_sr.cuh"
#include "pv_batch.cuh"
#include "pv_su.cuh"
#include "pv_su_dev.cuh"
#include "pv_direct.cuh"
#include "pv_fermion.cuh"
#include "pv_fvmc.cuh"

#include <memory>
#include <map>
#include <mutex>
#include <tuple>
#include <array>

using namespace pv;

namespace {

constexpr int SAMPLE_THREADS = 256;   // narrow blocks
constexpr int WIDE_THREADS = 1024;    // wide blocks (temporaries in shared memory)
constexpr int WIDE_SMEM_MAX = 220 * 1024;
constexpr double JTOL_F64 = 1e-15;
constexpr float JTOL_F32 = 2e-7f;
// TF32 mode: the Jacobi truncation stops once every column pair is orthogonal to the
// operands' own rounding (TF32 unit roundoff 2^-11 = 4.9e-4): the truncated subspace is
// then as accurate as the contractions that produced the matrix
constexpr float JTOL_TF32 = 4.8e-4f;
constexpr int JAC_MAX_SWEEPS = 60;

// ------------------------------------------------------------------ sample kernels

// The Metropolis sweep number the batched engine's accept kernels read (set before every
// sweep, outside any captured graph).
__global__ void k_set_sweep(uint32_t* d, uint32_t v) { *d = v; }

// Initial parameters: the beta = 0 state with its zero entries perturbed (App. A):
// entry t = noise (2u - 1), u = Philox(seed; t lo, t hi, 0, TAG_INIT); the [0,0,0,0]
// entries of the S = 0 and S = 3 slices of every site are 1.
__global__ void k_init_theta(long long Np, int N, const long long* __restrict__ toff,
                             double noise, uint64_t seed, double* __restrict__ theta,
                             float* __restrict__ theta_f) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < Np;
       t += (long long)gridDim.x * blockDim.x) {
    double u = philox_uniform(seed, (uint32_t)t, (uint32_t)(t >> 32), 0u, TAG_INIT);
    double v = noise * (2.0 * u - 1.0);
    int lo = 0, hi = N;   // site of t: toff[j] <= t < toff[j+1]
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (toff[mid] <= t) lo = mid; else hi = mid;
    }
    long long sz = (toff[lo + 1] - toff[lo]) / 4;
    long long rel = t - toff[lo];
    if (rel == 0 || rel == 3 * sz) v = 1.0;
    theta[t] = v;
    if (theta_f) theta_f[t] = (float)v;
  }
}

// Initial chains: diagonal configurations, s_i = low bit of Philox(seed; chain, site, 0, TAG_CFG).
__global__ void k_init_configs(int n, int N, uint64_t seed, uint8_t* __restrict__ S) {
  long long tot = (long long)n * N;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    int ch = (int)(t / N), j = (int)(t % N);
    uint32_t b = philox_bits(seed, (uint32_t)ch, (uint32_t)j, 0u, TAG_CFG) & 1u;
    S[t] = (uint8_t)(3u * b);
  }
}

// Flags a configuration batch holding an entry outside 0..3 (S = 2 s + s').
__global__ void k_check_configs(long long tot, const uint8_t* __restrict__ S, int* __restrict__ bad) {
  int b = 0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x)
    b |= S[t] > 3;
  if (__syncthreads_or(b) && threadIdx.x == 0) *bad = 1;
}

template <typename T>
__device__ void init_shared(Shared<T>& sh) {
  if (threadIdx.x == 0) {
    sh.flops = 0;
    sh.jac_sweeps = 0;
    sh.flag = 0;
  }
  __syncthreads();
}

template <typename T>
__device__ void flush_counters(Shared<T>& sh, double* flops, unsigned long long* jsw) {
  if (threadIdx.x == 0) {
    atomicAdd(flops, sh.flops);
    atomicAdd(jsw, (unsigned long long)sh.jac_sweeps);
  }
}

// Persistent evaluation kernel: block b handles samples b, b + grid, ...  WIDE blocks
// (1024 threads, one per SM) keep every short-lived buffer in shared memory; narrow
// blocks (256 threads, four per SM) keep only the Jacobi matrices there.
template <typename T, typename OT, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)
    k_eval(Geom g, const T* __restrict__ theta, const uint8_t* __restrict__ S, int n,
           T* scratch, int* iscratch, long long sreal, long long sint,
           double* __restrict__ log_abs, int8_t* __restrict__ sign, double* __restrict__ es,
           double* __restrict__ ea, OT* __restrict__ O, long long No, T jtol, int max_sweeps,
           double* flops, unsigned long long* jsw, int smem_bytes, T* ucache, int* ubond,
           long long ustride, long long ubstride) {
  __shared__ Shared<T> sh;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  Scratch<T> sc;
  sc.bind(scratch + (long long)blockIdx.x * sreal, iscratch + (long long)blockIdx.x * sint,
          g.L1, g.L2, g.D, g.chi);
  if (THREADS == WIDE_THREADS) {
    sc.bind_shared((T*)dyn_smem, g.D, g.chi);
  } else {
    sc.alias_global();
    sc.smem = smem_bytes > 0 ? (T*)dyn_smem : nullptr;
    sc.smem_cap = smem_bytes / (int)sizeof(T);
  }
  init_shared(sh);
  const int N = g.N();
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    int bad = 0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      const uint8_t v = S[(long long)s * N + j];
      bad |= v > 3;
      sh.S[j] = v;
    }
    // a configuration entry outside 0..3 would index past the site's parameter slices:
    // such a sample is not evaluated, its scalar outputs are NaN (sign 0), its O row is
    // left as it was
    if (__syncthreads_or(bad)) {
      if (threadIdx.x == 0) {
        if (log_abs) log_abs[s] = NAN;
        if (sign) sign[s] = 0;
        if (es) es[s] = NAN;
        if (ea) ea[s] = NAN;
      }
      continue;
    }
    UCache<T> uc{ucache ? ucache + (long long)s * ustride : nullptr,
                 ucache ? ubond + (long long)s * ubstride : nullptr};
    SampleOut r = eval_sample<T, T, OT>(g, sc, sh, theta, O ? O + (long long)s * No : nullptr,
                                        jtol, max_sweeps, uc);
    if (threadIdx.x == 0) {
      if (log_abs) log_abs[s] = r.log_abs;
      if (sign) sign[s] = (int8_t)r.sign;
      if (es) es[s] = r.e_sys;
      if (ea) ea[s] = r.e_anc;
    }
    __syncthreads();
  }
  flush_counters(sh, flops, jsw);
}

// One problem of a group evaluation: a context's geometry, parameters, chains and outputs.
struct GroupItem {
  Geom g;
  const void* theta;   // T
  const uint8_t* S;
  long long first;     // index of its first chain in the group's chain order
  int n;
  double *log_abs, *es, *ea;
  int8_t* sign;
  void* O;             // T
  long long No;
};

// Evaluation of the chains of several problems of different lattice sizes in one launch:
// chain q of the group (problems in order, each problem's chains in order) is evaluated by
// block q mod grid exactly as k_eval evaluates it (the same per-sample routine, block size
// and reduction order), its scratch laid out for its own geometry.
template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)
    k_eval_group(const GroupItem* __restrict__ items, int n_items, long long total, T* scratch,
                 int* iscratch, long long sreal, long long sint, T jtol, int max_sweeps,
                 double* flops, unsigned long long* jsw, int smem_bytes) {
  __shared__ Shared<T> sh;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  init_shared(sh);
  for (long long q = blockIdx.x; q < total; q += gridDim.x) {
    int k = 0;
    while (k + 1 < n_items && items[k + 1].first <= q) ++k;
    const GroupItem& it = items[k];
    const Geom g = it.g;
    const long long s = q - it.first;
    Scratch<T> sc;
    sc.bind(scratch + (long long)blockIdx.x * sreal, iscratch + (long long)blockIdx.x * sint,
            g.L1, g.L2, g.D, g.chi);
    sc.alias_global();
    sc.smem = smem_bytes > 0 ? (T*)dyn_smem : nullptr;
    sc.smem_cap = smem_bytes / (int)sizeof(T);
    const int N = g.N();
    for (int j = threadIdx.x; j < N; j += blockDim.x) sh.S[j] = it.S[s * N + j];
    __syncthreads();
    UCache<T> uc{nullptr, nullptr};
    T* O = (T*)it.O;
    SampleOut r = eval_sample<T, T, T>(g, sc, sh, (const T*)it.theta, O ? O + s * it.No : nullptr,
                                       jtol, max_sweeps, uc);
    if (threadIdx.x == 0) {
      it.log_abs[s] = r.log_abs;
      it.sign[s] = (int8_t)r.sign;
      it.es[s] = r.e_sys;
      it.ea[s] = r.e_anc;
    }
    __syncthreads();
  }
  flush_counters(sh, flops, jsw);
}

template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)
    k_mc(Geom g, const T* __restrict__ theta, uint8_t* __restrict__ S, int n, T* scratch,
         int* iscratch, long long sreal, long long sint, int p, uint64_t seed, long long sweep0,
         int n_sweeps, int* __restrict__ acc, int* __restrict__ prop, T jtol, int max_sweeps,
         double* flops, unsigned long long* jsw, int smem_bytes, T* ucache, int* ubond,
         long long ustride, long long ubstride) {
  __shared__ Shared<T> sh;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  Scratch<T> sc;
  sc.bind(scratch + (long long)blockIdx.x * sreal, iscratch + (long long)blockIdx.x * sint,
          g.L1, g.L2, g.D, g.chi);
  if (THREADS == WIDE_THREADS) {
    sc.bind_shared((T*)dyn_smem, g.D, g.chi);
  } else {
    sc.alias_global();
    sc.smem = smem_bytes > 0 ? (T*)dyn_smem : nullptr;
    sc.smem_cap = smem_bytes / (int)sizeof(T);
  }
  init_shared(sh);
  const int N = g.N();
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    for (int j = threadIdx.x; j < N; j += blockDim.x) sh.S[j] = S[(long long)s * N + j];
    __syncthreads();
    int a_tot = 0, p_tot = 0;
    for (int k = 0; k < n_sweeps; ++k) {
      int a = 0, pr = 0;
      UCache<T> uc{nullptr, nullptr};
      if (ucache && k == n_sweeps - 1) {   // keep the environments of the final configuration
        uc.env = ucache + (long long)s * ustride;
        uc.bond = ubond + (long long)s * ubstride;
      }
      mc_sweep<T, T>(g, sc, sh, theta, p, seed, (uint32_t)s, (uint32_t)(sweep0 + k), jtol,
                     max_sweeps, &a, &pr, uc);
      a_tot += a;
      p_tot += pr;
    }
    for (int j = threadIdx.x; j < N; j += blockDim.x) S[(long long)s * N + j] = sh.S[j];
    if (threadIdx.x == 0) {
      acc[s] = a_tot;
      prop[s] = p_tot;
    }
    __syncthreads();
  }
  flush_counters(sh, flops, jsw);
}

template <typename T>
__global__ void k_to_real(long long n, const double* __restrict__ a, T* __restrict__ b) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    b[t] = (T)a[t];
}

int grid_for(long long n, int threads, int cap = 152 * 16) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)std::min<long long>(b, cap);
}

}  // namespace

// ------------------------------------------------------------------ batched engine

namespace {

// Type-erased batched engine of a context (float64 or float32 arithmetic).
struct BatchIface {
  virtual ~BatchIface() {}
  virtual int* err_flag() = 0;
  virtual BatchTune& tuning() = 0;
  virtual bool uses_tensor_cores() const = 0;
  virtual void set_graphs(bool on) = 0;   // capture and replay the launch sequences
  virtual bool graphs_on() const = 0;
  virtual int graphs_captured() const = 0;
  virtual void drop_graphs() = 0;         // launch shapes changed: recapture on next use
  // float engines: truncate with a float64 working copy (g64: its global work area, or null)
  virtual bool set_trunc64(bool on, double* g64) = 0;
  virtual long long trunc_cap() const = 0;
  virtual bool trunc_global() const = 0;
  virtual void eval(const uint8_t* S, int nb, double* la, int8_t* sg, double* es, double* ea,
                    void* O, bool cached) = 0;
  virtual void mc(uint8_t* S, int n, int p, uint64_t seed, long long sweep0, int n_sweeps,
                  int* acc, int* prop) = 0;
  // direct draw of every chain (a runner built over double-layer tensors, pv_direct.cuh)
  virtual void draw(uint8_t* S, int n, const double* u, double b_d, double expo,
                    double* logq) = 0;
  double flops = 0;
  int chunk = 0;
};

template <typename T>
struct BatchImpl : BatchIface {
  CudaBE<T, T> be;
  BatchRunner<T, CudaBE<T, T>, T> run;
  int N = 0;
  long long No = 0;
  double *es_tmp = nullptr, *ea_tmp = nullptr;
  uint32_t* d_sweep = nullptr;   // the sweep number the accept kernels read
  double* jflops_dev = nullptr;  // Jacobi flop counter, fed while per-launch profiling is on
  // CUDA graphs: one captured launch sequence per (operation, exponent or cache use, chunk,
  // buffers), replayed on later calls; its flops and launch count are those of the capture
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    double flops = 0;
    long long launches = 0;
  };
  bool graphs = false;
  std::map<std::tuple<int, int, long long, const void*, const void*>, Graph> gcache;
  BatchImpl() : run(be) {}
  ~BatchImpl() override { drop_graphs(); }
  int* err_flag() override { return be.tc_err; }
  BatchTune& tuning() override { return be.tune; }
  bool uses_tensor_cores() const override { return be.tc; }
  void set_graphs(bool on) override {
    if (!on) drop_graphs();
    graphs = on;
  }
  bool graphs_on() const override { return graphs; }
  int graphs_captured() const override { return (int)gcache.size(); }
  bool set_trunc64(bool on, double* g64) override {
    if constexpr (std::is_same<T, float>::value) {
      be.trunc64 = on;
      if (g64) be.trunc_g64 = g64;
      drop_graphs();
      return true;
    }
    (void)on;
    (void)g64;
    return false;
  }
  long long trunc_cap() const override { return be.trunc_cap; }
  bool trunc_global() const override { return be.trunc_g != nullptr; }
  void drop_graphs() override {
    for (auto& kv : gcache)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    gcache.clear();
  }

  // Runs fn's launch sequence on the engine's stream: directly, or (graphs on, no per-launch
  // profiling) from a graph captured on first use.  A capture that fails leaves graphs off.
  template <typename F>
  void launch(const std::tuple<int, int, long long, const void*, const void*>& key, F&& fn) {
    if (!graphs || (be.prof && be.prof->on)) {
      fn();
      return;
    }
    auto it = gcache.find(key);
    if (it == gcache.end()) {
      const double f0 = run.flops;
      const long long l0 = be.prof ? be.prof->launches : 0;
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(be.st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        graphs = false;
        fn();
        return;
      }
      fn();
      Graph rec;
      cudaError_t e = cudaStreamEndCapture(be.st, &g);
      if (e == cudaSuccess) e = cudaGraphInstantiate(&rec.exec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        // nothing ran: run the sequence directly and stay without graphs
        cudaGetLastError();
        graphs = false;
        run.flops = f0;
        if (be.prof) be.prof->launches = l0;
        fn();
        return;
      }
      rec.flops = run.flops - f0;
      rec.launches = be.prof ? be.prof->launches - l0 : 0;
      it = gcache.emplace(key, rec).first;
      run.flops = f0;
      if (be.prof) be.prof->launches = l0;
    }
    cudaGraphLaunch(it->second.exec, be.st);
    run.flops += it->second.flops;
    if (be.prof) be.prof->launches += it->second.launches;
  }

  void count_jacobi() { run.jflops = be.prof && be.prof->on ? jflops_dev : nullptr; }
  void eval(const uint8_t* S, int nb, double* la, int8_t* sg, double* es, double* ea, void* O,
            bool cached) override {
    run.flops = 0;
    count_jacobi();
    for (int off = 0; off < nb; off += chunk) {
      int n = std::min(chunk, nb - off);
      const bool cu = cached && nb <= chunk;
      launch(std::make_tuple(0, cu ? 1 : 0, (long long)off, (const void*)S, (const void*)O),
             [&]() {
               run.eval(S + (long long)off * N, n, la ? la + off : nullptr, sg ? sg + off : nullptr,
                        es ? es + off : es_tmp, ea ? ea + off : ea_tmp,
                        O ? (T*)O + (long long)off * No : nullptr, No, cu);
             });
    }
    flops = run.flops;
  }
  void mc(uint8_t* S, int n_all, int p, uint64_t seed, long long sweep0, int n_sweeps, int* acc,
          int* prop) override {
    run.flops = 0;
    count_jacobi();
    run.sweep_dev = d_sweep;
    for (int off = 0; off < n_all; off += chunk) {
      int n = std::min(chunk, n_all - off);
      for (int k = 0; k < n_sweeps; ++k) {
        k_set_sweep<<<1, 1, 0, be.st>>>(d_sweep, (uint32_t)(sweep0 + k));
        if (be.prof) be.prof->launches += 1;
        launch(std::make_tuple(1, p, (long long)off, (const void*)S, (const void*)acc), [&]() {
          run.mc(S + (long long)off * N, n, p, seed, off, (uint32_t)(sweep0 + k), acc + off,
                 prop + off);
        });
      }
    }
    flops = run.flops;
  }
  void draw(uint8_t* S, int n_all, const double* u, double b_d, double expo,
            double* logq) override {
    run.flops = 0;
    count_jacobi();
    for (int off = 0; off < n_all; off += chunk) {
      const int n = std::min(chunk, n_all - off);
      direct_draw(run, S + (long long)off * N, n, u + (long long)off * N, b_d, expo, logq + off);
    }
    flops = run.flops;
  }
};

// Double-layer site tensors of direct sampling (the layout of double_layer_theta in
// pv_direct.cuh): block y = site, threads over the fused element index of one slice.
template <typename T>
__global__ void k_double_layer(int L1, int L2, int D, const T* __restrict__ theta,
                               const long long* __restrict__ toff, T* __restrict__ out,
                               const long long* __restrict__ toff2) {
  const int i = blockIdx.y, r = i / L2, c = i % L2;
  const int d0 = c == 0 ? 1 : D, d1 = c == L2 - 1 ? 1 : D, d2 = r == 0 ? 1 : D, d3 = r == L1 - 1 ? 1 : D;
  const long long sz = (long long)d0 * d1 * d2 * d3, sz2 = sz * sz;
  const T* th = theta + toff[i];
  T* o = out + toff2[i];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < sz2;
       e += (long long)gridDim.x * blockDim.x) {
    long long t = e;
    const int Dd = (int)(t % d3); t /= d3;
    const int dd = (int)(t % d3); t /= d3;
    const int U = (int)(t % d2); t /= d2;
    const int u = (int)(t % d2); t /= d2;
    const int R = (int)(t % d1); t /= d1;
    const int rr = (int)(t % d1); t /= d1;
    const int L = (int)(t % d0); t /= d0;
    const int l = (int)t;
    const long long ia = (((long long)l * d1 + rr) * d2 + u) * d3 + dd;
    const long long ib = (((long long)L * d1 + R) * d2 + U) * d3 + Dd;
    T acc = 0;
    for (int s = 0; s < 4; ++s) {
      const T x = th[s * sz + ia] * th[s * sz + ib];
      o[s * sz2 + e] = x;
      acc += x;
    }
    o[4 * sz2 + e] = acc;
  }
}

// Uniforms of a direct draw: u[chain][site] = Philox(seed; chain, draw, site, TAG_DIRECT).
__global__ void k_direct_uniforms(double* u, int n, int N, uint64_t seed, uint32_t draw) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < (long long)n * N;
       k += (long long)gridDim.x * blockDim.x)
    u[k] = philox_uniform(seed, (uint32_t)(k / N), draw, (uint32_t)(k % N), TAG_DIRECT);
}

}  // namespace

// ------------------------------------------------------------------ context

struct peps_ctx {
  peps_params P{};
  cudaStream_t stream = nullptr;
  int N = 0;
  long long Np = 0, No = 0;
  std::vector<long long> toff, ooff;
  long long* d_toff = nullptr;
  long long* d_ooff = nullptr;
  int* d_o2site = nullptr;
  double* d_theta = nullptr;
  float* d_theta_f = nullptr;
  uint8_t* d_S = nullptr;   // chains
  // evaluation of the chains
  double *d_log_abs = nullptr, *d_es = nullptr, *d_ea = nullptr;
  int8_t* d_sign = nullptr;
  void* d_O = nullptr;
  bool have_eval = false;
  // external batches
  uint8_t* d_xS = nullptr;
  double *d_xla = nullptr, *d_xes = nullptr, *d_xea = nullptr;
  int8_t* d_xsg = nullptr;
  void* d_xO = nullptr;
  int x_cap = 0;
  // sample scratch
  void* d_scr = nullptr;
  int* d_iscr = nullptr;
  int nblk = 0;
  long long sreal = 0, sint = 0;
  int smem_bytes = 0;   // dynamic shared memory of the sample kernels
  bool wide = false;    // 1024-thread blocks with every short-lived buffer in shared memory
  // up environments of the chains' final configurations, written by the sweep
  void* d_ucache = nullptr;
  int* d_ubond = nullptr;
  long long ustride = 0, ubstride = 0;
  bool ucache_valid = false;
  double* d_flops = nullptr;
  unsigned long long* d_jsw = nullptr;
  int* d_cfgbad = nullptr;   // set by k_check_configs when a configuration entry exceeds 3
  int *d_acc = nullptr, *d_prop = nullptr;
  // SR
  double *d_w = nullptr, *d_E = nullptr, *d_obar = nullptr, *d_g = nullptr, *d_x = nullptr;
  double *d_r = nullptr, *d_p = nullptr, *d_q = nullptr, *d_y = nullptr, *d_part = nullptr;
  double *d_part2 = nullptr, *d_bp1 = nullptr, *d_bp2 = nullptr, *d_ypart = nullptr;
  double* d_pqpart = nullptr;   // per-block partials of p.q of the fused CG product
  unsigned* d_gvbar = nullptr;  // grid-barrier counter and generation of the fused product
  int* d_gverr = nullptr;       // raised when a grid-barrier wait ran out
  int gv_grid = 0, gv_rpb = 1;   // fused product: resident blocks, rows per block per chunk
  int cg_mode = 0;               // CG product: 0 automatic, 1 fused single read, 2 two passes,
                                 // 3 two passes over a float64 copy of float32 O rows
  double* d_O64 = nullptr;       // that copy (allocated on first use)
  bool o64_failed = false;       // ... or its allocation failed once
  SRScalars* d_sc = nullptr;
  int nch = 0, nvb = 0, nyb = 0;
  double t = 0;
  int64_t sweeps = 0;
  double last_accept = 0;
  std::string err;
  std::vector<void*> allocs;
  std::unique_ptr<BatchIface> batch;   // batched engine (block_mode PEPS_BLOCKS_BATCHED)
  // direct sampling: a batched runner at bond D^2 over the double-layer tensors, built on
  // the first draw
  std::unique_ptr<BatchIface> dbatch;
  void* d_theta2 = nullptr;             // double-layer tensors, element type of the engine
  long long* d_toff2 = nullptr;
  std::vector<long long> toff2;
  double *d_logq = nullptr, *d_u = nullptr;
  bool direct_valid = false;            // the chains are the last direct draw, unchanged
  uint32_t n_draws = 0;
  pv::KProf kprof;                      // launch counter, optional per-kernel timing
  double* d_jflops = nullptr;           // Jacobi flops of the truncations while profiling
  double* d_trunc_g64 = nullptr;        // float64 Jacobi work area (peps_set_trunc_fp64)
  bool o_vec4 = false;                  // every site slice of O holds a multiple of 4 entries
};

namespace {

int fail(peps_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define PV_CUDA(ctx, call)                                                               \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(ctx, PEPS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename P>
int dalloc(peps_ctx* c, P** ptr, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, PEPS_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  c->allocs.push_back(p);
  *ptr = (P*)p;
  return PEPS_OK;
}

#define PV_TRY(x)                \
  do {                           \
    int rc_ = (x);               \
    if (rc_ != PEPS_OK) return rc_; \
  } while (0)

Geom make_geom(const peps_ctx* c) {
  Geom g;
  g.L1 = c->P.L1;
  g.L2 = c->P.L2;
  g.D = c->P.D;
  g.chi = c->P.chi;
  g.J1 = c->P.J1;
  g.J2 = c->P.J2;
  g.theta_off = c->d_toff;
  g.o_off = c->d_ooff;
  return g;
}

bool fp64(const peps_ctx* c) { return c->P.precision == PEPS_FP64; }

int ensure_batch(peps_ctx* c, int nb) {
  if (nb <= c->x_cap) return PEPS_OK;
  size_t osz = fp64(c) ? sizeof(double) : sizeof(float);
  PV_TRY(dalloc(c, &c->d_xS, (size_t)nb * c->N));
  PV_TRY(dalloc(c, &c->d_xla, (size_t)nb * sizeof(double)));
  PV_TRY(dalloc(c, &c->d_xes, (size_t)nb * sizeof(double)));
  PV_TRY(dalloc(c, &c->d_xea, (size_t)nb * sizeof(double)));
  PV_TRY(dalloc(c, &c->d_xsg, (size_t)nb));
  PV_TRY(dalloc(c, &c->d_xO, (size_t)nb * c->No * osz));
  c->x_cap = nb;
  return PEPS_OK;
}

// Reads (and clears) the batched engine's device error flag after a synchronised call
// (the context's own engine, or the one given).
int batch_status(peps_ctx* c, BatchIface* eng = nullptr) {
  if (!eng) eng = c->batch.get();
  int* d = eng ? eng->err_flag() : nullptr;
  if (!d) return PEPS_OK;
  int h = 0;
  PV_CUDA(c, cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost));
  if (!h) return PEPS_OK;
  PV_CUDA(c, cudaMemset(d, 0, sizeof(int)));
  if (h & 2)
    return fail(c, PEPS_ETIMEOUT,
                "tensor-core contraction: completion wait and its grace wait ran out; an MMA may "
                "have been in flight when tensor memory was released, so every later result of "
                "this context is undefined: free the context");
  return fail(c, PEPS_ETIMEOUT, "tensor-core contraction: completion wait ran out");
}

// Launches the evaluation kernel on device buffers.
int launch_eval(peps_ctx* c, const uint8_t* dS, int nb, double* la, int8_t* sg, double* es,
                double* ea, void* O, bool use_cache = false) {
  void* ucache = use_cache ? c->d_ucache : nullptr;
  Geom g = make_geom(c);
  PV_CUDA(c, cudaMemsetAsync(c->d_flops, 0, sizeof(double), c->stream));
  PV_CUDA(c, cudaMemsetAsync(c->d_jsw, 0, sizeof(unsigned long long), c->stream));
  if (c->batch) {
    c->batch->eval(dS, nb, la, sg, es, ea, O, use_cache);
    double f = c->batch->flops;
    PV_CUDA(c, cudaMemcpyAsync(c->d_flops, &f, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    PV_CUDA(c, cudaStreamSynchronize(c->stream));   // f lives on this stack frame
    PV_CUDA(c, cudaGetLastError());
    return batch_status(c);
  }
  int grid = std::min(c->nblk, nb);
#define PV_EVAL_LAUNCH(T, TH, THETA)                                                         \
  PV_KLAUNCH(&c->kprof, c->stream, "k_eval", 0.0, 0.0,                                      \
  k_eval<T, T, TH><<<grid, TH, c->smem_bytes, c->stream>>>(                                  \
      g, THETA, dS, nb, (T*)c->d_scr, c->d_iscr, c->sreal, c->sint, la, sg, es, ea, (T*)O, \
      c->No, fp64(c) ? (T)JTOL_F64 : (T)JTOL_F32, JAC_MAX_SWEEPS, c->d_flops, c->d_jsw,   \
      c->smem_bytes, (T*)ucache, c->d_ubond, c->ustride, c->ubstride))
  if (fp64(c)) {
    if (c->wide) PV_EVAL_LAUNCH(double, WIDE_THREADS, c->d_theta);
    else PV_EVAL_LAUNCH(double, SAMPLE_THREADS, c->d_theta);
  } else {
    if (c->wide) PV_EVAL_LAUNCH(float, WIDE_THREADS, c->d_theta_f);
    else PV_EVAL_LAUNCH(float, SAMPLE_THREADS, c->d_theta_f);
  }
#undef PV_EVAL_LAUNCH
  PV_CUDA(c, cudaGetLastError());
  return PEPS_OK;
}

}  // namespace

namespace {

// Builds a batched runner at bond dimension Dn over the site tensors theta (offsets toff):
// the context's own engine (Dn = D) or the direct sampler's double-layer one (Dn = D^2).
// Work buffers for as many chains as half the free device memory holds, at most n_chains.
template <typename T>
int init_runner_t(peps_ctx* c, int sms, BatchImpl<T>* b, int Dn, const T* theta,
                  const std::vector<long long>& toff) {
  const peps_params* P = &c->P;
  const int n = P->n_chains;
  const long long cD = (long long)P->chi * Dn;
  const long long cap = 2 * cD * (cD + 1);
  const size_t trunc_bytes = (size_t)cap * sizeof(T) + (size_t)(cD + 4) * (sizeof(T) + 4) + 16;
  const bool trunc_global = trunc_bytes > 200 * 1024;   // Jacobi matrices in global memory
  if (!trunc_global && trunc_bytes > 48 * 1024) {
    // one cap for every context of the process, so that none lowers it under another
    cudaError_t e = cudaFuncSetAttribute(kb_trunc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return fail(c, PEPS_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
  }
  std::vector<long long> sz;
  long long n8, nd;
  BatchBufs<T>::sizes(P->L1, P->L2, Dn, P->chi, sz, n8, nd);
  long long per = 0;
  for (long long x : sz) per += x;
  size_t per_bytes = (size_t)per * sizeof(T) + (size_t)n8 + (size_t)nd * 8 + 16;
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  long long chunk = std::min<long long>({(long long)n, (long long)(fr / 2 / per_bytes), 65535LL});
  if (chunk < 1) return fail(c, PEPS_ENOMEM, "batched blocks: no room for one chain's buffers");
  b->chunk = (int)chunk;
  T* real = nullptr;
  int8_t* i8 = nullptr;
  double* dbl = nullptr;
  int rc;
  if ((rc = dalloc(c, &real, (size_t)per * chunk * sizeof(T)))) return rc;
  if ((rc = dalloc(c, &i8, (size_t)n8 * chunk))) return rc;
  if ((rc = dalloc(c, &dbl, (size_t)nd * chunk * sizeof(double)))) return rc;
  if ((rc = dalloc(c, &b->es_tmp, (size_t)chunk * sizeof(double)))) return rc;
  if ((rc = dalloc(c, &b->d_sweep, sizeof(uint32_t)))) return rc;
  if (!c->d_jflops) {
    if ((rc = dalloc(c, &c->d_jflops, sizeof(double)))) return rc;
    PV_CUDA(c, cudaMemset(c->d_jflops, 0, sizeof(double)));
  }
  b->jflops_dev = c->d_jflops;
  if ((rc = dalloc(c, &b->ea_tmp, (size_t)chunk * sizeof(double)))) return rc;
  std::vector<int> bi, bj;
  std::vector<double> bJ;
  bond_lists(P->L1, P->L2, P->J1, P->J2, bi, bj, bJ);
  int *dbi = nullptr, *dbj = nullptr;
  double* dbJ = nullptr;
  size_t nb = bi.size() ? bi.size() : 1;
  if ((rc = dalloc(c, &dbi, nb * sizeof(int)))) return rc;
  if ((rc = dalloc(c, &dbj, nb * sizeof(int)))) return rc;
  if ((rc = dalloc(c, &dbJ, nb * sizeof(double)))) return rc;
  if (!bi.empty()) {
    cudaMemcpy(dbi, bi.data(), bi.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(dbj, bj.data(), bj.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(dbJ, bJ.data(), bJ.size() * sizeof(double), cudaMemcpyHostToDevice);
  }
  b->be.st = c->stream;
  b->be.prof = &c->kprof;
  b->be.bi = dbi;
  b->be.bj = dbj;
  b->be.bJ = dbJ;
  b->be.nb = (int)bi.size();
  b->be.N = c->N;
  b->be.trunc_cap = cap;
  if (trunc_global && (rc = dalloc(c, &b->be.trunc_g, (size_t)8 * sms * cap * sizeof(T)))) return rc;
  b->be.sms = sms;
  {
    int lq_max = 96 * 1024;
    cudaError_t e = cudaFuncSetAttribute(kb_lq<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lq_max);
    b->be.lq_smem_max = e == cudaSuccess ? lq_max : 48 * 1024;
    if (e != cudaSuccess) cudaGetLastError();
    if constexpr (std::is_same<T, float>::value) {
      const int tw_max = 220 * 1024;
      e = cudaFuncSetAttribute(kb_trunc_wide<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, tw_max);
      b->be.trunc_wide_max = e == cudaSuccess ? tw_max : 0;
      if (e != cudaSuccess) cudaGetLastError();
      e = cudaFuncSetAttribute(kb_chol<T, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, tw_max);
      b->be.chol_wide_max = e == cudaSuccess ? tw_max : 0;
      if (e != cudaSuccess) cudaGetLastError();
    }
    e = cudaFuncSetAttribute(kb_gemm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    if (e != cudaSuccess) return fail(c, PEPS_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    const int lq2_max = 200 * 1024;
    e = cudaFuncSetAttribute(kb_lq2<T, LQ_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, lq2_max);
    b->be.lq2_smem_max = e == cudaSuccess ? lq2_max : 0;
    if (e != cudaSuccess) cudaGetLastError();
  }
  if constexpr (std::is_same<T, float>::value) {
    // float32 storage: GEMM-shaped contractions on the tensor cores, with split (3xTF32)
    // operands in PEPS_FP32 (float32-accurate products) and plain TF32 in PEPS_TF32, which
    // also takes the right factors from the Gram matrix
    if ((rc = dalloc(c, &b->be.tc_err, sizeof(int)))) return rc;
    cudaError_t e = cudaMemsetAsync(b->be.tc_err, 0, sizeof(int), c->stream);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kb_gemm_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kb_gemm_tc2, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kb_gemm_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kb_chol<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kb_trunc64<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return fail(c, PEPS_ECUDA, std::string("tensor-core setup: ") + cudaGetErrorString(e));
    b->be.tc = true;
    b->be.tc_split = P->precision == PEPS_FP32;
    b->run.gram_lq = P->precision == PEPS_TF32;
  }
  b->N = c->N;
  b->No = c->No;
  auto& r = b->run;
  r.shp.build(P->L1, P->L2, Dn, P->chi);
  r.L1 = P->L1;
  r.L2 = P->L2;
  r.D = Dn;
  r.chi = P->chi;
  r.N = c->N;
  r.J1 = P->J1;
  r.J2 = P->J2;
  r.theta = theta;
  r.toff = toff;
  r.ooff = c->ooff;
  r.jtol = sizeof(T) == 8 ? (T)JTOL_F64 : (P->precision == PEPS_TF32 ? (T)JTOL_TF32 : (T)JTOL_F32);
  r.max_sweeps = JAC_MAX_SWEEPS;
  r.sweeps = c->d_jsw;
  r.b.bind(real, chunk, i8, dbl, P->L1, P->L2, Dn, P->chi);
  return PEPS_OK;
}

template <typename T>
int make_batch_t(peps_ctx* c, int sms) {
  auto* b = new BatchImpl<T>();
  c->batch.reset(b);
  const T* theta = fp64(c) ? (const T*)(const void*)c->d_theta : (const T*)(const void*)c->d_theta_f;
  return init_runner_t<T>(c, sms, b, c->P.D, theta, c->toff);
}

// The direct sampler's runner and buffers: double-layer tensors (five slices per site at
// bond D^2), uniforms and log q of every chain.
template <typename T>
int make_direct_t(peps_ctx* c, int sms) {
  const peps_params* P = &c->P;
  const int N = c->N, D2 = P->D * P->D;
  c->toff2.assign(N + 1, 0);
  for (int i = 0; i < N; ++i) {
    const int r = i / P->L2, q = i % P->L2;
    const long long sz = (long long)(q == 0 ? 1 : D2) * (q == P->L2 - 1 ? 1 : D2) *
                         (r == 0 ? 1 : D2) * (r == P->L1 - 1 ? 1 : D2);
    c->toff2[i + 1] = c->toff2[i] + 5 * sz;
  }
  PV_TRY(dalloc(c, (T**)&c->d_theta2, (size_t)c->toff2[N] * sizeof(T)));
  PV_TRY(dalloc(c, &c->d_toff2, (size_t)(N + 1) * sizeof(long long)));
  PV_CUDA(c, cudaMemcpy(c->d_toff2, c->toff2.data(), (N + 1) * sizeof(long long), cudaMemcpyHostToDevice));
  PV_TRY(dalloc(c, &c->d_logq, (size_t)P->n_chains * sizeof(double)));
  PV_TRY(dalloc(c, &c->d_u, (size_t)P->n_chains * N * sizeof(double)));
  auto* b = new BatchImpl<T>();
  c->dbatch.reset(b);
  const int rc = init_runner_t<T>(c, sms, b, D2, (const T*)c->d_theta2, c->toff2);
  if (rc != PEPS_OK) c->dbatch.reset();
  return rc;
}

// Block layout peps_init takes for automatic mode: the batched engine (measured faster on
// GB300 in every precision at 8x8, D=4, chi=16).  TF32 exists only in the batched engine.
int resolve_block_mode(const peps_params* P) {
  if (P->block_mode != PEPS_BLOCKS_AUTO) return P->block_mode;
  return PEPS_BLOCKS_BATCHED;
}

// Device bytes of one chain's batched-engine buffers.
size_t batched_chain_bytes(const peps_params* P) {
  std::vector<long long> sz;
  long long n8 = 0, nd = 0, per = 0;
  BatchBufs<double>::sizes(P->L1, P->L2, P->D, P->chi, sz, n8, nd);
  for (long long x : sz) per += x;
  const size_t real = P->precision == PEPS_FP64 ? 8 : 4;
  return (size_t)per * real + (size_t)n8 + (size_t)nd * 8 + 16 + 2 * 8;
}

// Autotuned launch shapes per problem geometry (d^2, D, chi, L1, L2, precision), shared by
// every context of the process.
std::mutex g_tune_mu;
std::map<std::array<int, 6>, BatchTune> g_tune;

std::array<int, 6> tune_key(const peps_params* P) {
  return {4, P->D, P->chi, P->L1, P->L2, P->precision};
}

int make_batch(peps_ctx* c, int sms) {
  return fp64(c) ? make_batch_t<double>(c, sms) : make_batch_t<float>(c, sms);
}

}  // namespace

extern "C" {

const char* peps_version(void) { return "peps_vmc 0.1 (sm_103a)"; }

static thread_local std::string g_noalloc_err;

const char* peps_last_error(const peps_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_noalloc_err.c_str();
}

void peps_free(peps_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (void* p : ctx->allocs) cudaFree(p);
  delete ctx;
}

int peps_init(const peps_params* Pin, void* stream, peps_ctx** out) {
  if (!Pin || !out) return PEPS_EINVAL;
  *out = nullptr;
  peps_params Pl = *Pin;
  Pl.block_mode = resolve_block_mode(&Pl);
  const peps_params* P = &Pl;
  if (P->precision == PEPS_TF32 && P->block_mode != PEPS_BLOCKS_BATCHED) return PEPS_EINVAL;
  if (P->L1 < 2 || P->L2 < 2 || P->L1 > MAX_L || P->L2 > MAX_L || P->D < 1 || P->D > 8 ||
      P->chi < 1 || P->chi > 64 || P->n_chains < 1 || P->model != PEPS_MODEL_J1J2 ||
      (P->precision != PEPS_FP64 && P->precision != PEPS_FP32 && P->precision != PEPS_TF32) ||
      P->n_blocks < 0 || !(P->init_noise >= 0) || P->block_mode < PEPS_BLOCKS_AUTO || P->block_mode > PEPS_BLOCKS_BATCHED)
    return PEPS_EINVAL;
  peps_ctx* c = new peps_ctx();
  c->P = *P;
  c->stream = (cudaStream_t)stream;
  c->N = P->L1 * P->L2;
  const int L2 = P->L2;
  c->toff.assign(c->N + 1, 0);
  c->ooff.assign(c->N + 1, 0);
  for (int i = 0; i < c->N; ++i) {
    int r = i / L2, cc = i % L2;
    long long sz = (long long)(cc == 0 ? 1 : P->D) * (cc == L2 - 1 ? 1 : P->D) *
                   (r == 0 ? 1 : P->D) * (r == P->L1 - 1 ? 1 : P->D);
    c->toff[i + 1] = c->toff[i] + 4 * sz;
    c->ooff[i + 1] = c->ooff[i] + sz;
  }
  c->Np = c->toff[c->N];
  c->No = c->ooff[c->N];
  c->o_vec4 = true;
  for (int i = 0; i < c->N; ++i) c->o_vec4 = c->o_vec4 && (c->ooff[i + 1] - c->ooff[i]) % 4 == 0;
  std::vector<int> o2site(c->No);
  for (int i = 0; i < c->N; ++i)
    for (long long o = c->ooff[i]; o < c->ooff[i + 1]; ++o) o2site[o] = i;
  int rc = PEPS_OK;
  auto bail = [&](int code) {
    std::string m = c->err;
    peps_free(c);
    (void)m;
    return code;
  };
  const int n = P->n_chains;
  size_t real = fp64(c) ? sizeof(double) : sizeof(float);
  if ((rc = dalloc(c, &c->d_toff, (c->N + 1) * sizeof(long long)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_ooff, (c->N + 1) * sizeof(long long)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_o2site, c->No * sizeof(int)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_theta, c->Np * sizeof(double)))) return bail(rc);
  if (!fp64(c) && (rc = dalloc(c, &c->d_theta_f, c->Np * sizeof(float)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_S, (size_t)n * c->N))) return bail(rc);
  if ((rc = dalloc(c, &c->d_log_abs, n * sizeof(double)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_es, n * sizeof(double)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_ea, n * sizeof(double)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_sign, n))) return bail(rc);
  if ((rc = dalloc(c, &c->d_O, (size_t)n * c->No * real))) return bail(rc);
  if ((rc = dalloc(c, &c->d_acc, n * sizeof(int)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_prop, n * sizeof(int)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_flops, sizeof(double)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_jsw, sizeof(unsigned long long)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_cfgbad, sizeof(int)))) return bail(rc);
  // persistent sample blocks and their scratch
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  ScratchDims sd = scratch_dims(P->L1, P->L2, P->D, P->chi);
  c->sreal = (sd.n_real + 31) & ~31LL;
  c->sint = (sd.n_int + 31) & ~31LL;
  {
    long long cD = (long long)P->chi * P->D;
    long long wide_bytes = Scratch<double>::shared_elems(P->D, P->chi) * (long long)real;
    long long jac_bytes = cD * (cD + 1) * 2 * (long long)real;
    ScratchDims sd0 = scratch_dims(1, 1, P->D, P->chi);
    bool fits = wide_bytes <= WIDE_SMEM_MAX;
    if (P->block_mode == PEPS_BLOCKS_WIDE && !fits) return bail(fail(c, PEPS_EINVAL, "wide blocks: buffers exceed shared memory"));
    // Measured on GB300 (8x8, D=4, chi=16, float32): four narrow blocks per SM keep four
    // samples in flight and beat one wide block by 2x, so automatic picks narrow blocks.
    (void)sd0;
    c->wide = P->block_mode == PEPS_BLOCKS_WIDE;
    c->smem_bytes = c->wide ? (int)wide_bytes : (jac_bytes <= 96 * 1024 ? (int)jac_bytes : 0);
    cudaError_t ea = cudaSuccess;
    if (c->smem_bytes > 48 * 1024) {
      if (c->wide) {
        ea = fp64(c) ? cudaFuncSetAttribute(k_eval<double, double, WIDE_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, WIDE_SMEM_MAX)
                     : cudaFuncSetAttribute(k_eval<float, float, WIDE_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, WIDE_SMEM_MAX);
        if (ea == cudaSuccess)
          ea = fp64(c) ? cudaFuncSetAttribute(k_mc<double, WIDE_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, WIDE_SMEM_MAX)
                       : cudaFuncSetAttribute(k_mc<float, WIDE_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, WIDE_SMEM_MAX);
      } else {
        ea = fp64(c) ? cudaFuncSetAttribute(k_eval<double, double, SAMPLE_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024)
                     : cudaFuncSetAttribute(k_eval<float, float, SAMPLE_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        if (ea == cudaSuccess)
          ea = fp64(c) ? cudaFuncSetAttribute(k_mc<double, SAMPLE_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024)
                       : cudaFuncSetAttribute(k_mc<float, SAMPLE_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
      }
    }
    if (ea != cudaSuccess) return bail(fail(c, PEPS_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ea)));
  }
  int want = P->n_blocks > 0 ? P->n_blocks : (c->wide ? sms : sms * 4);
  if (P->block_mode == PEPS_BLOCKS_BATCHED) want = 1;   // the batched engine has its own buffers
  c->nblk = std::max(1, std::min(want, n));
  if ((rc = dalloc(c, &c->d_scr, (size_t)c->nblk * c->sreal * real))) return bail(rc);
  if ((rc = dalloc(c, &c->d_iscr, (size_t)c->nblk * c->sint * sizeof(int)))) return bail(rc);
  {
    // up-environment cache: used when it takes at most a quarter of the free memory
    c->ustride = (long long)P->L1 * P->L2 * sd.ENV;
    c->ubstride = (long long)P->L1 * (P->L2 + 1);
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    size_t need = (size_t)n * (c->ustride * real + c->ubstride * sizeof(int));
    if (P->block_mode != PEPS_BLOCKS_BATCHED && need <= fr / 4) {
      if ((rc = dalloc(c, &c->d_ucache, (size_t)n * c->ustride * real))) return bail(rc);
      if ((rc = dalloc(c, &c->d_ubond, (size_t)n * c->ubstride * sizeof(int)))) return bail(rc);
    }
  }
  // SR buffers
  c->nch = (n + OTV_CHUNK - 1) / OTV_CHUNK;
  c->nvb = grid_for(c->Np, SR_THREADS, 1024);
  c->nyb = (n + (SR_THREADS / 32) - 1) / (SR_THREADS / 32);
  if ((rc = dalloc(c, &c->d_w, n * sizeof(double)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_E, n * sizeof(double)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_y, n * sizeof(double)))) return bail(rc);
  for (double** v : {&c->d_obar, &c->d_g, &c->d_x, &c->d_r, &c->d_p, &c->d_q})
    if ((rc = dalloc(c, v, c->Np * sizeof(double)))) return bail(rc);
  {
    // fused CG product: one resident block of GV_THREADS per SM (cooperative launch), chunks
    // of at most 48 MB of O rows so that phase B finds them in L2
    int dev = 0, sms = 152, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t gsm = 4 * GV_THREADS * sizeof(double);
    cudaError_t e1 = cudaFuncSetAttribute(k_gv<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
    if (e1 == cudaSuccess) e1 = cudaFuncSetAttribute(k_gv<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
    if (e1 == cudaSuccess) e1 = cudaFuncSetAttribute(k_gv<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
    if (e1 == cudaSuccess) e1 = cudaFuncSetAttribute(k_gv<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
    if (e1 == cudaSuccess)
      e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gv<double, false>, GV_THREADS, gsm);
    if (e1 != cudaSuccess || occ < 1) return bail(fail(c, PEPS_ECUDA, "fused CG product: no resident block"));
    if (cudaFuncSetAttribute(k_colsum1_f32v<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(32 * SR_THREADS * sizeof(double))) != cudaSuccess ||
        cudaFuncSetAttribute(k_colsum1_f32v<true, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(32 * SR_THREADS * sizeof(double))) != cudaSuccess)
      return bail(fail(c, PEPS_ECUDA, "column-sum kernel: shared-memory attribute"));
    c->gv_grid = sms;
    const double elt = fp64(c) ? 8.0 : 4.0;
    const double rows = 48e6 / ((double)c->gv_grid * (double)c->No * elt);
    c->gv_rpb = std::max(1, std::min(64, (int)rows));
  }
  if ((rc = dalloc(c, &c->d_pqpart, (size_t)std::max(c->gv_grid, c->nvb) * sizeof(double)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_gvbar, 2 * sizeof(unsigned)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_gverr, sizeof(int)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_part, (size_t)c->nch * c->Np * sizeof(double)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_part2, (size_t)c->nch * c->Np * sizeof(double)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_bp1, c->nvb * sizeof(double)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_bp2, c->nvb * sizeof(double)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_ypart, c->nyb * sizeof(double)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_sc, sizeof(SRScalars)))) return bail(rc);
  if (P->block_mode == PEPS_BLOCKS_BATCHED) {
    if ((rc = make_batch(c, sms))) return bail(rc);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(P));
    if (it != g_tune.end()) c->batch->tuning() = it->second;
  }
  cudaError_t e;
  e = cudaMemcpyAsync(c->d_toff, c->toff.data(), (c->N + 1) * sizeof(long long),
                      cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_ooff, c->ooff.data(), (c->N + 1) * sizeof(long long),
                        cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_o2site, o2site.data(), c->No * sizeof(int), cudaMemcpyHostToDevice,
                        c->stream);
  if (e != cudaSuccess) return bail(fail(c, PEPS_ECUDA, cudaGetErrorString(e)));
  PV_KLAUNCH(&c->kprof, c->stream, "k_init_theta", 0.0, 0.0, k_init_theta<<<grid_for(c->Np, 256), 256, 0, c->stream>>>(c->Np, c->N, c->d_toff,
                                                             P->init_noise, P->seed, c->d_theta,
                                                             c->d_theta_f));
  PV_KLAUNCH(&c->kprof, c->stream, "k_init_configs", 0.0, 0.0, k_init_configs<<<grid_for((long long)n * c->N, 256), 256, 0, c->stream>>>(n, c->N, P->seed,
                                                                            c->d_S));
  e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return bail(fail(c, PEPS_ECUDA, cudaGetErrorString(e)));
  *out = c;
  return PEPS_OK;
}

size_t peps_footprint(const peps_params* P) {
  if (!P || P->L1 < 2 || P->L2 < 2 || P->L1 > MAX_L || P->L2 > MAX_L || P->D < 1 || P->D > 8 ||
      P->chi < 1 || P->chi > 64 || P->n_chains < 1)
    return 0;
  const size_t real = P->precision == PEPS_FP64 ? 8 : 4;
  const long long N = (long long)P->L1 * P->L2, n = P->n_chains;
  long long Np = 0, No = 0;
  for (long long i = 0; i < N; ++i) {
    int r = (int)(i / P->L2), c = (int)(i % P->L2);
    long long sz = (long long)(c == 0 ? 1 : P->D) * (c == P->L2 - 1 ? 1 : P->D) *
                   (r == 0 ? 1 : P->D) * (r == P->L1 - 1 ? 1 : P->D);
    Np += 4 * sz;
    No += sz;
  }
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  ScratchDims sd = scratch_dims(P->L1, P->L2, P->D, P->chi);
  long long sreal = (sd.n_real + 31) & ~31LL, sint = (sd.n_int + 31) & ~31LL;
  const int mode = resolve_block_mode(P);
  const bool batched = mode == PEPS_BLOCKS_BATCHED;
  long long nblk = P->n_blocks > 0 ? P->n_blocks : (mode == PEPS_BLOCKS_WIDE ? sms : 4LL * sms);
  nblk = batched ? 1 : std::max(1LL, std::min(nblk, n));
  long long nch = (n + OTV_CHUNK - 1) / OTV_CHUNK;
  size_t b = 0;
  b += 2 * (N + 1) * 8 + No * 4 + Np * 8 + (real == 4 ? Np * 4 : 0);   // tables, theta
  b += n * N + n * (8 * 3 + 1 + 4 * 2) + (size_t)n * No * real;       // chains, outputs, O
  b += (size_t)nblk * (sreal * real + sint * 4);                       // sample scratch
  if (batched) {                                                        // batched buffers
    b += (size_t)n * batched_chain_bytes(P);
    const long long cD = (long long)P->chi * P->D, cap = 2 * cD * (cD + 1);
    if ((size_t)cap * real + (size_t)(cD + 4) * (real + 4) + 16 > 200 * 1024)
      b += (size_t)8 * sms * cap * real;                                 // global Jacobi area
  }
  else b += (size_t)n * ((long long)P->L1 * P->L2 * sd.ENV * real + (long long)P->L1 * (P->L2 + 1) * 4);
  b += n * 8 * 3 + 6 * Np * 8 + (real == 4 ? Np * 4 : 0) + 2 * (size_t)nch * Np * 8;   // SR
  return b + (1 << 20);
}

size_t peps_num_params(const peps_ctx* c) { return c ? (size_t)c->Np : 0; }
size_t peps_o_row_len(const peps_ctx* c) { return c ? (size_t)c->No : 0; }
int64_t peps_sweeps_done(const peps_ctx* c) { return c ? c->sweeps : 0; }
int peps_set_sweeps_done(peps_ctx* c, int64_t s) {
  if (!c || s < 0) return PEPS_EINVAL;
  c->sweeps = s;
  return PEPS_OK;
}

int peps_get_theta(peps_ctx* c, double* host, size_t n) {
  if (!c || !host || n != (size_t)c->Np) return fail(c, PEPS_EINVAL, "get_theta: size");
  PV_CUDA(c, cudaMemcpyAsync(host, c->d_theta, n * sizeof(double), cudaMemcpyDeviceToHost,
                             c->stream));
  PV_CUDA(c, cudaStreamSynchronize(c->stream));
  return PEPS_OK;
}

int peps_set_theta(peps_ctx* c, const double* host, size_t n) {
  if (!c || !host || n != (size_t)c->Np) return fail(c, PEPS_EINVAL, "set_theta: size");
  PV_CUDA(c, cudaMemcpyAsync(c->d_theta, host, n * sizeof(double), cudaMemcpyHostToDevice,
                             c->stream));
  if (c->d_theta_f)
    PV_KLAUNCH(&c->kprof, c->stream, "k_to_real", 0.0, 0.0, k_to_real<float><<<grid_for(c->Np, 256), 256, 0, c->stream>>>(c->Np, c->d_theta,
                                                                   c->d_theta_f));
  PV_CUDA(c, cudaGetLastError());
  PV_CUDA(c, cudaStreamSynchronize(c->stream));
  c->have_eval = false;
  c->direct_valid = false;
  c->ucache_valid = false;
  return PEPS_OK;
}

int peps_get_configs(peps_ctx* c, uint8_t* host, size_t n) {
  if (!c || !host || n != (size_t)c->P.n_chains * c->N) return fail(c, PEPS_EINVAL, "get_configs: size");
  PV_CUDA(c, cudaMemcpyAsync(host, c->d_S, n, cudaMemcpyDeviceToHost, c->stream));
  PV_CUDA(c, cudaStreamSynchronize(c->stream));
  return PEPS_OK;
}

int peps_set_configs(peps_ctx* c, const uint8_t* host, size_t n) {
  if (!c || !host || n != (size_t)c->P.n_chains * c->N) return fail(c, PEPS_EINVAL, "set_configs: size");
  for (size_t i = 0; i < n; ++i)
    if (host[i] > 3) return fail(c, PEPS_EINVAL, "set_configs: entry > 3");
  PV_CUDA(c, cudaMemcpyAsync(c->d_S, host, n, cudaMemcpyHostToDevice, c->stream));
  PV_CUDA(c, cudaStreamSynchronize(c->stream));
  c->have_eval = false;
  c->direct_valid = false;
  c->ucache_valid = false;
  return PEPS_OK;
}

int peps_mc_sweep(peps_ctx* c, int n_sweeps, int p) {
  if (!c || n_sweeps < 0 || (p != 1 && p != 2)) return fail(c, PEPS_EINVAL, "mc_sweep: args");
  if (n_sweeps == 0) return PEPS_OK;
  Geom g = make_geom(c);
  const int n = c->P.n_chains;
  PV_CUDA(c, cudaMemsetAsync(c->d_flops, 0, sizeof(double), c->stream));
  PV_CUDA(c, cudaMemsetAsync(c->d_jsw, 0, sizeof(unsigned long long), c->stream));
  int grid = std::min(c->nblk, n);
  if (c->batch) {
    PV_CUDA(c, cudaMemsetAsync(c->d_acc, 0, n * sizeof(int), c->stream));
    PV_CUDA(c, cudaMemsetAsync(c->d_prop, 0, n * sizeof(int), c->stream));
    c->batch->mc(c->d_S, n, p, c->P.seed, c->sweeps, n_sweeps, c->d_acc, c->d_prop);
    double f = c->batch->flops;
    PV_CUDA(c, cudaMemcpyAsync(c->d_flops, &f, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    PV_CUDA(c, cudaStreamSynchronize(c->stream));
    PV_TRY(batch_status(c));
  } else {
#define PV_MC_LAUNCH(T, TH, THETA)                                                            \
  PV_KLAUNCH(&c->kprof, c->stream, "k_mc", 0.0, 0.0,                                          \
  k_mc<T, TH><<<grid, TH, c->smem_bytes, c->stream>>>(                                        \
      g, THETA, c->d_S, n, (T*)c->d_scr, c->d_iscr, c->sreal, c->sint, p, c->P.seed,          \
      c->sweeps, n_sweeps, c->d_acc, c->d_prop, fp64(c) ? (T)JTOL_F64 : (T)JTOL_F32,          \
      JAC_MAX_SWEEPS, c->d_flops, c->d_jsw, c->smem_bytes, (T*)c->d_ucache, c->d_ubond,       \
      c->ustride, c->ubstride))
  if (fp64(c)) {
    if (c->wide) PV_MC_LAUNCH(double, WIDE_THREADS, c->d_theta);
    else PV_MC_LAUNCH(double, SAMPLE_THREADS, c->d_theta);
  } else {
    if (c->wide) PV_MC_LAUNCH(float, WIDE_THREADS, c->d_theta_f);
    else PV_MC_LAUNCH(float, SAMPLE_THREADS, c->d_theta_f);
  }
#undef PV_MC_LAUNCH
  }
  PV_CUDA(c, cudaGetLastError());
  c->sweeps += n_sweeps;
  c->have_eval = false;
  c->direct_valid = false;
  c->ucache_valid = c->batch ? (n <= c->batch->chunk) : (c->d_ucache != nullptr);
  std::vector<int> a(n), b(n);
  PV_CUDA(c, cudaMemcpyAsync(a.data(), c->d_acc, n * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PV_CUDA(c, cudaMemcpyAsync(b.data(), c->d_prop, n * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PV_CUDA(c, cudaStreamSynchronize(c->stream));
  long long sa = 0, sb = 0;
  for (int i = 0; i < n; ++i) {
    sa += a[i];
    sb += b[i];
  }
  c->last_accept = sb > 0 ? (double)sa / (double)sb : 0.0;
  return PEPS_OK;
}

int peps_direct_draw(peps_ctx* c, const double* u, int on_device, double b_d, double exponent,
                     double* log_q) {
  if (!c || !(b_d > 0.0) || !(b_d <= 1.0) || !(exponent > 0.0) || !std::isfinite(exponent))
    return fail(c, PEPS_EINVAL, "direct_draw: args");
  if (!c->batch)
    return fail(c, PEPS_ESTATE, "direct_draw: direct sampling runs on the batched engine");
  const peps_params* P = &c->P;
  const int n = P->n_chains, N = c->N;
  cudaStream_t st = c->stream;
  if (!c->dbatch) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    PV_TRY(fp64(c) ? make_direct_t<double>(c, sms) : make_direct_t<float>(c, sms));
  }
  c->have_eval = false;
  c->ucache_valid = false;
  c->direct_valid = false;
  long long big = 0;
  for (int i = 0; i < N; ++i) big = std::max(big, (c->toff2[i + 1] - c->toff2[i]) / 5);
  dim3 g((unsigned)std::min<long long>((big + 255) / 256, 1024), (unsigned)N);
  if (fp64(c))
    PV_KLAUNCH(&c->kprof, st, "k_double_layer", 0.0, 0.0,
               k_double_layer<double><<<g, 256, 0, st>>>(P->L1, P->L2, P->D, c->d_theta, c->d_toff,
                                                         (double*)c->d_theta2, c->d_toff2));
  else
    PV_KLAUNCH(&c->kprof, st, "k_double_layer", 0.0, 0.0,
               k_double_layer<float><<<g, 256, 0, st>>>(P->L1, P->L2, P->D, c->d_theta_f, c->d_toff,
                                                        (float*)c->d_theta2, c->d_toff2));
  const double* du = c->d_u;
  if (u && on_device) {
    du = u;
  } else if (u) {
    PV_CUDA(c, cudaMemcpyAsync(c->d_u, u, (size_t)n * N * sizeof(double), cudaMemcpyHostToDevice, st));
  } else {
    PV_KLAUNCH(&c->kprof, st, "k_direct_uniforms", 0.0, 0.0,
               k_direct_uniforms<<<grid_for((long long)n * N, 256), 256, 0, st>>>(c->d_u, n, N, P->seed,
                                                                                 c->n_draws));
  }
  c->dbatch->draw(c->d_S, n, du, b_d, exponent, c->d_logq);
  PV_CUDA(c, cudaGetLastError());
  if (log_q)
    PV_CUDA(c, cudaMemcpyAsync(log_q, c->d_logq, (size_t)n * sizeof(double),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  PV_CUDA(c, cudaStreamSynchronize(st));
  PV_TRY(batch_status(c, c->dbatch.get()));
  c->n_draws += 1;
  c->direct_valid = true;
  return PEPS_OK;
}

double peps_direct_next_bd(double b_d, double diag_frac, int N) {
  if (!(b_d > 0.0) || !(diag_frac >= 0.0) || N < 1) return b_d;
  if (diag_frac > 0.5) b_d *= std::pow(0.5 / diag_frac, 1.0 / N);
  return std::min(b_d, 1.0);
}

int peps_direct_step(peps_ctx* c, double* b_d, double exponent, double tau, double eps,
                     int max_cg, double cg_tol, peps_stats* st) {
  if (!c || !b_d) return fail(c, PEPS_EINVAL, "direct_step: args");
  PV_TRY(peps_direct_draw(c, nullptr, 0, *b_d, exponent, nullptr));
  PV_TRY(peps_eval_batch(c, nullptr, c->P.n_chains, 1, nullptr, nullptr, nullptr, nullptr, nullptr));
  peps_stats tmp;
  peps_stats* sp = st ? st : &tmp;
  const int rc = peps_sr_step(c, tau, eps, max_cg, cg_tol, 0, sp);
  if (rc < 0) return rc;
  *b_d = peps_direct_next_bd(*b_d, sp->diag_frac, c->N);
  return rc;
}

int peps_eval_batch(peps_ctx* c, const uint8_t* S, int nb, int on_device, double* log_abs,
                    int8_t* sign, double* e_sys, double* e_anc, void* O) {
  if (!c || nb < 0) return fail(c, PEPS_EINVAL, "eval_batch: args");
  size_t osz = fp64(c) ? sizeof(double) : sizeof(float);
  if (S == nullptr) {
    if (nb != c->P.n_chains) return fail(c, PEPS_EINVAL, "eval_batch: nb != n_chains");
    PV_TRY(launch_eval(c, c->d_S, nb, c->d_log_abs, c->d_sign, c->d_es, c->d_ea, c->d_O,
                       c->ucache_valid));
    c->have_eval = true;
    if (on_device) {
      if (log_abs) PV_CUDA(c, cudaMemcpyAsync(log_abs, c->d_log_abs, nb * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      if (sign) PV_CUDA(c, cudaMemcpyAsync(sign, c->d_sign, nb, cudaMemcpyDeviceToDevice, c->stream));
      if (e_sys) PV_CUDA(c, cudaMemcpyAsync(e_sys, c->d_es, nb * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      if (e_anc) PV_CUDA(c, cudaMemcpyAsync(e_anc, c->d_ea, nb * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      if (O) PV_CUDA(c, cudaMemcpyAsync(O, c->d_O, (size_t)nb * c->No * osz, cudaMemcpyDeviceToDevice, c->stream));
    } else {
      if (log_abs) PV_CUDA(c, cudaMemcpyAsync(log_abs, c->d_log_abs, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      if (sign) PV_CUDA(c, cudaMemcpyAsync(sign, c->d_sign, nb, cudaMemcpyDeviceToHost, c->stream));
      if (e_sys) PV_CUDA(c, cudaMemcpyAsync(e_sys, c->d_es, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      if (e_anc) PV_CUDA(c, cudaMemcpyAsync(e_anc, c->d_ea, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      if (O) PV_CUDA(c, cudaMemcpyAsync(O, c->d_O, (size_t)nb * c->No * osz, cudaMemcpyDeviceToHost, c->stream));
    }
    PV_CUDA(c, cudaStreamSynchronize(c->stream));
    return PEPS_OK;
  }
  if (nb == 0) return PEPS_OK;
  if (on_device) {
    // device configurations are checked on the device before any evaluation reads them
    int bad = 0;
    PV_CUDA(c, cudaMemsetAsync(c->d_cfgbad, 0, sizeof(int), c->stream));
    const long long tot = (long long)nb * c->N;
    k_check_configs<<<(int)std::min<long long>((tot + 255) / 256, 1024), 256, 0, c->stream>>>(
        tot, S, c->d_cfgbad);
    PV_CUDA(c, cudaGetLastError());
    c->kprof.launches += 1;
    PV_CUDA(c, cudaMemcpyAsync(&bad, c->d_cfgbad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PV_CUDA(c, cudaStreamSynchronize(c->stream));
    if (bad) return fail(c, PEPS_EINVAL, "eval_batch: configuration entry > 3");
    PV_TRY(launch_eval(c, S, nb, log_abs, sign, e_sys, e_anc, O));
    if (c->batch) c->ucache_valid = false;   // the batched engine's environments were reused
    PV_CUDA(c, cudaStreamSynchronize(c->stream));
    return PEPS_OK;
  }
  for (long long i = 0; i < (long long)nb * c->N; ++i)
    if (S[i] > 3) return fail(c, PEPS_EINVAL, "eval_batch: configuration entry > 3");
  PV_TRY(ensure_batch(c, nb));
  PV_CUDA(c, cudaMemcpyAsync(c->d_xS, S, (size_t)nb * c->N, cudaMemcpyHostToDevice, c->stream));
  PV_TRY(launch_eval(c, c->d_xS, nb, c->d_xla, c->d_xsg, c->d_xes, c->d_xea, O ? c->d_xO : nullptr));
  if (c->batch) c->ucache_valid = false;
  if (log_abs) PV_CUDA(c, cudaMemcpyAsync(log_abs, c->d_xla, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (sign) PV_CUDA(c, cudaMemcpyAsync(sign, c->d_xsg, nb, cudaMemcpyDeviceToHost, c->stream));
  if (e_sys) PV_CUDA(c, cudaMemcpyAsync(e_sys, c->d_xes, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (e_anc) PV_CUDA(c, cudaMemcpyAsync(e_anc, c->d_xea, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (O) PV_CUDA(c, cudaMemcpyAsync(O, c->d_xO, (size_t)nb * c->No * osz, cudaMemcpyDeviceToHost, c->stream));
  PV_CUDA(c, cudaStreamSynchronize(c->stream));
  return PEPS_OK;
}

int peps_last_counters(peps_ctx* c, double* flops, int64_t* jsw) {
  if (!c) return PEPS_EINVAL;
  double f = 0;
  unsigned long long j = 0;
  PV_CUDA(c, cudaMemcpyAsync(&f, c->d_flops, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PV_CUDA(c, cudaMemcpyAsync(&j, c->d_jsw, sizeof(j), cudaMemcpyDeviceToHost, c->stream));
  PV_CUDA(c, cudaStreamSynchronize(c->stream));
  if (flops) *flops = f;
  if (jsw) *jsw = (int64_t)j;
  return PEPS_OK;
}

static int fill_stats(peps_ctx* c, int p, peps_stats* st, bool with_cg) {
  SRScalars h;
  PV_CUDA(c, cudaMemcpyAsync(&h, c->d_sc, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  PV_CUDA(c, cudaStreamSynchronize(c->stream));
  if (!st) return PEPS_OK;
  const double N = (double)c->N;
  st->t = c->t;
  st->beta_obs = 4.0 * c->t;
  st->E_site = h.H1 / N;
  st->E_err = h.Eerr / N;
  st->C_site = st->beta_obs * st->beta_obs * (h.H2 - h.H1 * h.H1) / N;
  st->chi_sus = st->beta_obs * h.M2 / N;
  st->accept = c->last_accept;
  st->diag_frac = h.diag;
  st->p = p;
  if (with_cg) {
    st->cg_iters = h.iters;
    st->cg_resid = h.gnorm > 0 ? std::sqrt(h.rr) / h.gnorm : 0.0;
  } else {
    st->cg_iters = 0;
    st->cg_resid = 0;
  }
  return PEPS_OK;
}

static int launch_weights(peps_ctx* c, int p) {
  PV_KLAUNCH(&c->kprof, c->stream, "k_sr_weights", 0.0, 0.0, k_sr_weights<<<1, SR_WEIGHT_THREADS, 0, c->stream>>>(c->P.n_chains, c->N, p, c->d_log_abs,
                                                       c->d_logq, c->d_es, c->d_ea, c->d_S, c->d_w, c->d_E,
                                                       c->d_sc));
  PV_CUDA(c, cudaGetLastError());
  return PEPS_OK;
}

// p = 0 (direct draws) needs the chains to be the last peps_direct_draw, unchanged since.
static int check_weights(peps_ctx* c, int p, const char* who) {
  if (!c->have_eval) return fail(c, PEPS_ESTATE, std::string(who) + ": no evaluation of the chains");
  if (p == 0 && !c->direct_valid)
    return fail(c, PEPS_ESTATE, std::string(who) + ": p = 0 needs the chains of the last direct draw, "
                "unchanged (no sweep, configuration or theta change since)");
  return PEPS_OK;
}

int peps_observables(peps_ctx* c, int p, peps_stats* st) {
  if (!c || p < 0 || p > 2) return fail(c, PEPS_EINVAL, "observables: args");
  PV_TRY(check_weights(c, p, "observables"));
  PV_TRY(launch_weights(c, p));
  return fill_stats(c, p, st, false);
}

int peps_sr_step(peps_ctx* c, double tau, double eps, int max_cg, double cg_tol, int p,
                 peps_stats* st) {
  if (!c || p < 0 || p > 2 || max_cg < 0 || !(eps >= 0) || !(cg_tol >= 0) ||
      !std::isfinite(tau))
    return fail(c, PEPS_EINVAL, "sr_step: args");
  PV_TRY(check_weights(c, p, "sr_step"));
  const int n = c->P.n_chains;
  const long long Np = c->Np, No = c->No;
  cudaStream_t s = c->stream;
  PV_TRY(launch_weights(c, p));
  // float32 rows with 16-byte site slices: the passes read a float64 copy of the rows made
  // once per step (automatic and mode 3), so that no pass spends float64 issue on widening
  bool o64 = !fp64(c) && c->o_vec4 && (c->cg_mode == 0 || c->cg_mode == 3);
  if (o64 && !c->d_O64 && !c->o64_failed) {
    if (cudaMalloc((void**)&c->d_O64, (size_t)n * No * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      c->d_O64 = nullptr;
      c->o64_failed = true;
    } else {
      c->allocs.push_back(c->d_O64);
    }
  }
  if (o64 && !c->d_O64) {
    if (c->cg_mode == 3) return fail(c, PEPS_ENOMEM, "sr_step: no room for the float64 copy of O");
    o64 = false;
  }
  if (o64) {
    const long long n4 = (long long)n * No / 4;
    PV_KLAUNCH(&c->kprof, s, "k_widen_o", (double)n * No * 12.0, 0.0,
               k_widen_o<<<grid_for(n4, 256), 256, 0, s>>>(n4, (const float*)c->d_O, c->d_O64));
  }
  // mean and gradient (one pass over O)
  dim3 cgrid((unsigned)((No + SR_THREADS - 1) / SR_THREADS), (unsigned)c->nch);
  dim3 cgrid4((unsigned)((No / 4 + SR_THREADS - 1) / SR_THREADS), (unsigned)c->nch);   // 4 columns a thread
  if (o64)
    PV_KLAUNCH(&c->kprof, s, "k_colsum1_f32", ((double)n * No * 8.0 + (double)c->nch * Np * 8.0), 0.0, k_colsum1_f32v<true, double><<<cgrid4, SR_THREADS, 32 * SR_THREADS * sizeof(double), s>>>(
        n, c->N, No, c->d_O64, c->d_S, c->d_o2site, c->d_toff, c->d_ooff, c->d_w,
        c->d_E, &c->d_sc->Ebar, c->d_part, c->d_part2, Np, nullptr));
  else if (fp64(c))
    PV_KLAUNCH(&c->kprof, s, "k_colsum1", ((double)n * No * 8.0 + (double)c->nch * Np * 8.0), 0.0, k_colsum1<double, true><<<cgrid, SR_THREADS, 0, s>>>(
        n, c->N, No, (const double*)c->d_O, c->d_S, c->d_o2site, c->d_toff, c->d_ooff, c->d_w,
        c->d_E, &c->d_sc->Ebar, c->d_part, c->d_part2, Np, nullptr));
  else if (c->o_vec4)
    PV_KLAUNCH(&c->kprof, s, "k_colsum1_f32", ((double)n * No * 4.0 + (double)c->nch * Np * 8.0), 0.0, k_colsum1_f32v<true><<<cgrid4, SR_THREADS, 32 * SR_THREADS * sizeof(double), s>>>(
        n, c->N, No, (const float*)c->d_O, c->d_S, c->d_o2site, c->d_toff, c->d_ooff, c->d_w,
        c->d_E, &c->d_sc->Ebar, c->d_part, c->d_part2, Np, nullptr));
  else
    PV_KLAUNCH(&c->kprof, s, "k_colsum1_f32", ((double)n * No * 4.0 + (double)c->nch * Np * 8.0), 0.0, k_colsum1_f32<true><<<cgrid, SR_THREADS, 0, s>>>(
        n, c->N, No, (const float*)c->d_O, c->d_S, c->d_o2site, c->d_toff, c->d_ooff, c->d_w,
        c->d_E, &c->d_sc->Ebar, c->d_part, c->d_part2, Np, nullptr));
  PV_KLAUNCH(&c->kprof, s, "k_colsum2_grad", (2.0 * c->nch * Np * 8.0 + 2.0 * Np * 8.0), 0.0, k_colsum2_grad<<<grid_for(Np, SR_THREADS, 1 << 20), SR_THREADS, 0, s>>>(
      Np, c->nch, c->d_part, c->d_part2, c->d_obar, c->d_g));
  PV_CUDA(c, cudaGetLastError());
  // CG
  const int nvb = c->nvb;
  PV_KLAUNCH(&c->kprof, s, "k_dot_part", (2.0 * Np * 8.0), 0.0, k_dot_part<<<nvb, SR_THREADS, 0, s>>>(Np, c->d_g, c->d_g, c->d_bp1, nullptr));
  PV_KLAUNCH(&c->kprof, s, "k_cg_init", (5.0 * Np * 8.0), 0.0, k_cg_init<<<nvb, SR_THREADS, 0, s>>>(Np, c->d_g, c->d_x, c->d_r, c->d_p, nvb,
                                       c->d_bp1, c->d_sc, max_cg, cg_tol, eps));
  PV_KLAUNCH(&c->kprof, s, "k_dot_part", (2.0 * Np * 8.0), 0.0, k_dot_part<<<nvb, SR_THREADS, 0, s>>>(Np, c->d_obar, c->d_p, c->d_bp2, nullptr));   // obar.p
  PV_CUDA(c, cudaGetLastError());
  PV_CUDA(c, cudaMemsetAsync(c->d_gverr, 0, sizeof(int), s));
  // the fused product reads O once but synchronises the grid once per L2-sized chunk of
  // samples
  const long long gv_rows = (long long)c->gv_grid * c->gv_rpb;
  // automatic: the two passes (measured faster at 8x8 and 10x10: float64 issue bounds both
  // forms, and the fused one adds a grid barrier per chunk), over the float64 copy when made
  const bool fused = c->cg_mode == 1;
  (void)gv_rows;
  const int ov_blocks = c->nyb;
  dim3 cgrid_y((unsigned)((No + SR_THREADS - 1) / SR_THREADS), (unsigned)c->nch);
  dim3 cgrid4_y((unsigned)((No / 4 + SR_THREADS - 1) / SR_THREADS), (unsigned)c->nch);
  for (int it = 0; it < max_cg; ++it) {
    if (!fused) {
      // y_i = w_i (O_i.p - obar.p), then the column sums part = sum_i y_i O_i, then q
      const double ob = (double)n * No * (fp64(c) || o64 ? 8.0 : 4.0);
      if (o64)
        PV_KLAUNCH(&c->kprof, s, "k_ov", ob + (double)Np * 8.0, 2.0 * n * No, k_ov_f32v<double><<<ov_blocks, SR_THREADS, 0, s>>>(n, c->N, No, c->d_O64, c->d_S,
            c->d_o2site, c->d_toff, c->d_ooff, c->d_p, c->d_w, c->d_y, c->d_ypart, nvb, c->d_bp2, c->d_sc));
      else if (fp64(c))
        PV_KLAUNCH(&c->kprof, s, "k_ov", ob + (double)Np * 8.0, 2.0 * n * No, k_ov<double><<<ov_blocks, SR_THREADS, 0, s>>>(n, c->N, No, (const double*)c->d_O, c->d_S,
            c->d_toff, c->d_ooff, c->d_p, c->d_w, c->d_y, c->d_ypart, nvb, c->d_bp2, c->d_sc));
      else if (c->o_vec4)
        PV_KLAUNCH(&c->kprof, s, "k_ov", ob + (double)Np * 8.0, 2.0 * n * No, k_ov_f32v<<<ov_blocks, SR_THREADS, 0, s>>>(n, c->N, No, (const float*)c->d_O, c->d_S,
            c->d_o2site, c->d_toff, c->d_ooff, c->d_p, c->d_w, c->d_y, c->d_ypart, nvb, c->d_bp2, c->d_sc));
      else
        PV_KLAUNCH(&c->kprof, s, "k_ov", ob + (double)Np * 8.0, 2.0 * n * No, k_ov<float><<<ov_blocks, SR_THREADS, 0, s>>>(n, c->N, No, (const float*)c->d_O, c->d_S,
            c->d_toff, c->d_ooff, c->d_p, c->d_w, c->d_y, c->d_ypart, nvb, c->d_bp2, c->d_sc));
      if (o64)
        PV_KLAUNCH(&c->kprof, s, "k_colsum1_f32", ob + (double)c->nch * Np * 8.0, 2.0 * n * No, k_colsum1_f32v<false, double><<<cgrid4_y, SR_THREADS, 16 * SR_THREADS * sizeof(double), s>>>(
            n, c->N, No, c->d_O64, c->d_S, c->d_o2site, c->d_toff, c->d_ooff, c->d_y,
            nullptr, nullptr, c->d_part, nullptr, Np, &c->d_sc->done));
      else if (fp64(c))
        PV_KLAUNCH(&c->kprof, s, "k_colsum1", ob + (double)c->nch * Np * 8.0, 2.0 * n * No, k_colsum1<double, false><<<cgrid_y, SR_THREADS, 0, s>>>(
            n, c->N, No, (const double*)c->d_O, c->d_S, c->d_o2site, c->d_toff, c->d_ooff, c->d_y,
            nullptr, nullptr, c->d_part, nullptr, Np, &c->d_sc->done));
      else if (c->o_vec4)
        PV_KLAUNCH(&c->kprof, s, "k_colsum1_f32", ob + (double)c->nch * Np * 8.0, 2.0 * n * No, k_colsum1_f32v<false><<<cgrid4_y, SR_THREADS, 16 * SR_THREADS * sizeof(double), s>>>(
            n, c->N, No, (const float*)c->d_O, c->d_S, c->d_o2site, c->d_toff, c->d_ooff, c->d_y,
            nullptr, nullptr, c->d_part, nullptr, Np, &c->d_sc->done));
      else
        PV_KLAUNCH(&c->kprof, s, "k_colsum1_f32", ob + (double)c->nch * Np * 8.0, 2.0 * n * No, k_colsum1_f32<false><<<cgrid_y, SR_THREADS, 0, s>>>(
            n, c->N, No, (const float*)c->d_O, c->d_S, c->d_o2site, c->d_toff, c->d_ooff, c->d_y,
            nullptr, nullptr, c->d_part, nullptr, Np, &c->d_sc->done));
      PV_KLAUNCH(&c->kprof, s, "k_otv2", ((double)c->nch * Np * 8.0 + 3.0 * Np * 8.0), 0.0, k_otv2<<<nvb, SR_THREADS, 0, s>>>(Np, c->nch, c->d_part, c->d_obar, c->d_p, c->d_q,
          ov_blocks, c->d_ypart, c->d_pqpart, c->d_sc));
    } else {
      // q = (G + eps) p in one cooperative launch (one read of O)
      PV_CUDA(c, cudaMemsetAsync(c->d_gvbar, 0, 2 * sizeof(unsigned), s));
      {
        int n_ = n, N_ = c->N, ndp = nvb, rpb = c->gv_rpb;
        long long No_ = No;
        const void* Op = c->d_O;
        const uint8_t* Sp = c->d_S;
        const int* o2s = c->d_o2site;
        const long long *tof = c->d_toff, *oof = c->d_ooff;
        const double *pp = c->d_p, *obp = c->d_obar, *wp = c->d_w, *dp = c->d_bp2;
        double *yp = c->d_y, *qp = c->d_q, *pqp = c->d_pqpart;
        unsigned* barp = c->d_gvbar;
        int* errp = c->d_gverr;
        const SRScalars* scp = c->d_sc;
        void* args[] = {&n_, &N_, &No_, &Op, &Sp, &o2s, &tof, &oof, &pp, &obp, &wp, &ndp, &dp,
                        &yp, &qp, &pqp, &rpb, &barp, &errp, &scp};
        const void* fn = fp64(c) ? (c->o_vec4 ? (const void*)k_gv<double, true> : (const void*)k_gv<double, false>)
                                 : (c->o_vec4 ? (const void*)k_gv<float, true> : (const void*)k_gv<float, false>);
        const double obytes = (double)n * No * (fp64(c) ? 8.0 : 4.0);
        PV_KLAUNCH(&c->kprof, s, "k_gv", obytes + (double)n * c->N + 4.0 * Np * 8.0, 4.0 * (double)n * No,
                   PV_CUDA(c, cudaLaunchCooperativeKernel(fn, dim3(c->gv_grid), dim3(GV_THREADS), args,
                                                          4 * GV_THREADS * sizeof(double), s)));
      }
    }
    PV_KLAUNCH(&c->kprof, s, "k_cg_a", (5.0 * Np * 8.0), 0.0, k_cg_a<<<nvb, SR_THREADS, 0, s>>>(Np, c->d_x, c->d_r, c->d_p, c->d_q, fused ? c->gv_grid : nvb, c->d_pqpart,
                                      c->d_bp1, c->d_sc));
    PV_KLAUNCH(&c->kprof, s, "k_cg_b", (5.0 * Np * 8.0), 0.0, k_cg_b<<<nvb, SR_THREADS, 0, s>>>(Np, c->d_r, c->d_p, c->d_obar, nvb, c->d_bp1,
                                      c->d_bp2, c->d_sc));
    PV_KLAUNCH(&c->kprof, s, "k_cg_scalars", 0.0, 0.0, k_cg_scalars<<<1, 1, 0, s>>>(nvb, c->d_bp1, c->d_sc));
    PV_CUDA(c, cudaGetLastError());
    if ((it & 7) == 7) {
      int done = 0;
      PV_CUDA(c, cudaMemcpyAsync(&done, &c->d_sc->done, sizeof(int), cudaMemcpyDeviceToHost, s));
      PV_CUDA(c, cudaStreamSynchronize(s));
      if (done) break;
    }
  }
  {
    int gerr = 0;
    PV_CUDA(c, cudaMemcpyAsync(&gerr, c->d_gverr, sizeof(int), cudaMemcpyDeviceToHost, s));
    PV_CUDA(c, cudaStreamSynchronize(s));
    if (gerr) return fail(c, PEPS_ETIMEOUT, "sr_step: a grid-barrier wait of the CG product ran out");
  }
  PV_KLAUNCH(&c->kprof, s, "k_update", (3.0 * Np * 8.0), 0.0, k_update<<<grid_for(Np, 256), 256, 0, s>>>(Np, tau, c->d_x, c->d_theta, c->d_theta_f));
  PV_CUDA(c, cudaGetLastError());
  int rc = fill_stats(c, p, st, true);
  if (rc != PEPS_OK) return rc;
  SRScalars h;
  PV_CUDA(c, cudaMemcpy(&h, c->d_sc, sizeof(h), cudaMemcpyDeviceToHost));
  c->t += tau;
  c->have_eval = false;
  c->direct_valid = false;
  c->ucache_valid = false;
  if (!std::isfinite(h.rr) || !std::isfinite(h.H1))
    return fail(c, PEPS_ENOTFINITE, "sr_step: non-finite energy or residual");
  return (h.iters >= max_cg && max_cg > 0 && h.gnorm > 0 &&
          std::sqrt(h.rr) > cg_tol * h.gnorm)
             ? PEPS_WARN_CG_MAXIT
             : PEPS_OK;
}

double peps_time(const peps_ctx* c) { return c ? c->t : 0.0; }

long long peps_launches(const peps_ctx* c) { return c ? c->kprof.launches : 0; }

int peps_autotune(peps_ctx* c, int reps, peps_tune* out) {
  if (!c || reps < 0) return fail(c, PEPS_EINVAL, "autotune: args");
  if (!c->batch) return fail(c, PEPS_ESTATE, "autotune: only the batched engine has launch shapes to tune");
  BatchTune& tu = c->batch->tuning();
  // every candidate is timed with direct launches (a graph would replay the shapes it was
  // captured with)
  const bool had_graphs = c->batch->graphs_on();
  c->batch->set_graphs(false);
  struct Restore {
    peps_ctx* c;
    bool on;
    ~Restore() { c->batch->set_graphs(on); }
  } restore{c, had_graphs};
  // time on at most 8192 chains: the best shapes depend on the chain count (a 2048-chain
  // subset picked one chain per FFMA block, which is slower at 8192 chains)
  const int n = c->P.n_chains < 8192 ? c->P.n_chains : 8192;
  auto timed = [&](double* ms) -> int {
    double best = 1e300;
    for (int r = 0; r < (reps > 0 ? reps : 1); ++r) {
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, c->stream);
      int rc = launch_eval(c, c->d_S, n, c->d_log_abs, c->d_sign, c->d_es, c->d_ea, c->d_O, false);
      cudaEventRecord(e1, c->stream);
      cudaEventSynchronize(e1);
      float t = 0;
      cudaEventElapsedTime(&t, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (rc != PEPS_OK) return rc;
      best = t < best ? t : best;
    }
    *ms = best;
    return PEPS_OK;
  };
  double before = 0, cur = 0;
  if (reps > 0) {
    PV_TRY(timed(&before));
    cur = before;
    // coordinate descent over the launch-shape parameters (results are the same for all)
    const int grid_c[] = {50, 100, 200}, db_c[] = {0, 12 * 1024, 48 * 1024}, kc_c[] = {16, 32, 64},
              p_c[] = {0, 1, 2}, sb_c[] = {64 * 1024, 96 * 1024, 192 * 1024}, g_c[] = {1, 16, 256},
              tt_c[] = {32, 64, 256};
    int* fields[] = {&tu.grid_pct, &tu.db_bytes, &tu.kc_max, &tu.pipelined, &tu.stage_budget, &tu.ffma_g,
                     &tu.trunc_threads};
    const int* cands[] = {grid_c, db_c, kc_c, p_c, sb_c, g_c, tt_c};
    for (int knob = c->batch->uses_tensor_cores() ? 0 : 5; knob < 7; ++knob) {
      int* field = fields[knob];
      const int* cand = cands[knob];
      int best_v = *field;
      for (int i = 0; i < 3; ++i) {
        if (cand[i] == best_v) continue;
        const int keep = *field;
        *field = cand[i];
        double ms = 0;
        PV_TRY(timed(&ms));
        if (ms < cur * 0.99) {
          cur = ms;
          best_v = cand[i];
        } else {
          *field = keep;
        }
        *field = best_v;
      }
    }
    c->batch->drop_graphs();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(&c->P)] = tu;
    c->have_eval = n == c->P.n_chains;   // all chains evaluated for the current state
    c->ucache_valid = false;
  }
  if (out) {
    out->grid_pct = tu.grid_pct;
    out->db_bytes = tu.db_bytes;
    out->ffma_g = tu.ffma_g;
    out->kc_max = tu.kc_max;
    out->pipelined = tu.pipelined;
    out->stage_kb = tu.stage_budget / 1024;
    out->trunc_threads = tu.trunc_threads;
    out->ms_before = before;
    out->ms_after = cur;
  }
  return PEPS_OK;
}

int peps_su_theta(int L1, int L2, int D, double J1, double tau, int n_steps, double* theta,
                  size_t n) {
  if (L1 < 2 || L2 < 2 || L1 > MAX_L || L2 > MAX_L || D < 1 || D > 8 || n_steps < 0 ||
      !(tau >= 0.0) || !std::isfinite(J1) || !theta)
    return PEPS_EINVAL;
  size_t Np = 0;
  for (int r = 0; r < L1; ++r)
    for (int c = 0; c < L2; ++c)
      Np += (size_t)4 * (c == 0 ? 1 : D) * (c == L2 - 1 ? 1 : D) * (r == 0 ? 1 : D) * (r == L1 - 1 ? 1 : D);
  if (n != Np) return PEPS_EINVAL;
  pv::SimpleUpdate su(L1, L2, D, J1);
  for (int k = 0; k < n_steps; ++k) su.step(tau);
  su.theta(theta);
  return PEPS_OK;
}

int peps_set_graphs(peps_ctx* c, int enable) {
  if (!c || enable < 0 || enable > 1) return fail(c, PEPS_EINVAL, "set_graphs: args");
  if (!c->batch) return fail(c, PEPS_ESTATE, "set_graphs: only the batched engine captures graphs");
  c->batch->set_graphs(enable != 0);
  return PEPS_OK;
}

int peps_graphs_captured(const peps_ctx* c) {
  return (c && c->batch) ? c->batch->graphs_captured() : 0;
}

int peps_set_trunc_fp64(peps_ctx* c, int enable) {
  if (!c || enable < 0 || enable > 1) return fail(c, PEPS_EINVAL, "set_trunc_fp64: args");
  if (!c->batch || fp64(c))
    return fail(c, PEPS_ESTATE, "set_trunc_fp64: only the batched engine's float32 modes truncate in float32");
  double* g64 = nullptr;
  const long long cap = c->batch->trunc_cap();
  if (enable && (size_t)cap * 8 + 16 > 200 * 1024 && !c->d_trunc_g64) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    PV_TRY(dalloc(c, &c->d_trunc_g64, (size_t)8 * sms * cap * sizeof(double)));
  }
  g64 = c->d_trunc_g64;
  c->batch->set_trunc64(enable == 1, g64);
  return PEPS_OK;
}

int peps_set_cg_product(peps_ctx* c, int mode) {
  if (!c || mode < 0 || mode > 3) return fail(c, PEPS_EINVAL, "set_cg_product: mode");
  c->cg_mode = mode;
  return PEPS_OK;
}

int peps_su_warm_start(peps_ctx* c, double tau, int n_steps) {
  if (!c || n_steps < 0 || !(tau >= 0.0) || !std::isfinite(tau))
    return fail(c, PEPS_EINVAL, "su_warm_start: args");
  if (c->P.J2 != 0.0)
    return fail(c, PEPS_EINVAL, "su_warm_start: the simple update covers nearest-neighbour (J1) bonds only");
  const int L1 = c->P.L1, L2 = c->P.L2, D = c->P.D, N = L1 * L2;
  const long long D4 = (long long)D * D * D * D;
  const int nblk = std::max(L1, L2);
  const long long wds = SuScratch::doubles(D), wis = SuScratch::ints(D);
  SuDev sd;
  sd.L1 = L1;
  sd.L2 = L2;
  sd.D = D;
  double* wd = nullptr;
  int* wi = nullptr;
  std::vector<void*> mine;
  auto cleanup = [&]() {
    cudaStreamSynchronize(c->stream);
    for (void* q : mine) cudaFree(q);
  };
  auto get = [&](void** q, size_t bytes) {
    if (cudaMalloc(q, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    mine.push_back(*q);
    return true;
  };
  if (!get((void**)&sd.T, (size_t)N * 4 * D4 * sizeof(double)) || !get((void**)&sd.dims, (size_t)N * 4 * sizeof(int)) ||
      !get((void**)&sd.lh, (size_t)N * D * sizeof(double)) || !get((void**)&sd.nlh, (size_t)N * sizeof(int)) ||
      !get((void**)&sd.lv, (size_t)N * D * sizeof(double)) || !get((void**)&sd.nlv, (size_t)N * sizeof(int)) ||
      !get((void**)&sd.gate, 256 * sizeof(double)) || !get((void**)&wd, (size_t)nblk * wds * sizeof(double)) ||
      !get((void**)&wi, (size_t)nblk * wis * sizeof(int))) {
    cleanup();
    return fail(c, PEPS_ENOMEM, "su_warm_start: device allocation failed");
  }
  double gate[256];
  pv::SimpleUpdate::bond_gate(c->P.J1, tau, gate);
  cudaError_t e = cudaMemcpyAsync(sd.gate, gate, sizeof(gate), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) {
    k_su_init<<<grid_for(N, 128), 128, 0, c->stream>>>(sd);
    c->kprof.launches += 1;
    for (int k = 0; k < n_steps; ++k) {
      k_su_half<<<L1, SU_THREADS, 0, c->stream>>>(sd, wd, wi, wds, wis, 1);
      k_su_half<<<L2, SU_THREADS, 0, c->stream>>>(sd, wd, wi, wds, wis, 0);
      c->kprof.launches += 2;
    }
    k_su_theta<<<N, 128, 0, c->stream>>>(sd, c->d_toff, c->d_theta);
    c->kprof.launches += 1;
    if (c->d_theta_f) {
      k_to_real<float><<<grid_for(c->Np, 256), 256, 0, c->stream>>>(c->Np, c->d_theta, c->d_theta_f);
      c->kprof.launches += 1;
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cleanup();
  if (e != cudaSuccess) return fail(c, PEPS_ECUDA, std::string("su_warm_start: ") + cudaGetErrorString(e));
  c->t = n_steps * tau;
  c->have_eval = false;
  c->direct_valid = false;
  c->ucache_valid = false;
  return PEPS_OK;
}

int peps_set_tune(peps_ctx* c, const peps_tune* t) {
  if (!c || !t || t->grid_pct < 1 || t->grid_pct > 400 || t->db_bytes < 0 ||
      t->db_bytes > 200 * 1024 || t->ffma_g < 1 || t->ffma_g > 256 || t->kc_max < 8 ||
      t->kc_max > 64 || t->kc_max % 8 || t->pipelined < 0 || t->pipelined > 2 ||
      (t->stage_kb != 0 && (t->stage_kb < 32 || t->stage_kb > 200)) ||
      (t->trunc_threads != 0 && t->trunc_threads != 32 && t->trunc_threads != 64 &&
       t->trunc_threads != 128 && t->trunc_threads != 256))
    return fail(c, PEPS_EINVAL, "set_tune: args");
  if (!c->batch) return fail(c, PEPS_ESTATE, "set_tune: only the batched engine has launch shapes");
  BatchTune& tu = c->batch->tuning();
  tu.grid_pct = t->grid_pct;
  tu.db_bytes = t->db_bytes;
  tu.ffma_g = t->ffma_g;
  tu.kc_max = t->kc_max;
  tu.pipelined = t->pipelined;
  if (t->stage_kb) tu.stage_budget = t->stage_kb * 1024;
  if (t->trunc_threads) tu.trunc_threads = t->trunc_threads;
  c->batch->drop_graphs();   // the captured sequences used the old shapes
  return PEPS_OK;
}

int peps_profile(peps_ctx* c, int enable) {
  if (!c || enable < 0 || enable > 2) return fail(c, PEPS_EINVAL, "profile: args");
  PV_CUDA(c, cudaStreamSynchronize(c->stream));
  if (enable) {
    c->kprof.reset();
    c->kprof.on = true;
    c->kprof.gemm_only = enable == 2;
    if (c->d_jflops) PV_CUDA(c, cudaMemset(c->d_jflops, 0, sizeof(double)));
  } else {
    c->kprof.fold();
    c->kprof.on = false;
  }
  return PEPS_OK;
}

int peps_profile_read(peps_ctx* c, peps_kernel_stat* out, int cap, int* n_out) {
  if (!c || cap < 0 || (cap > 0 && !out) || !n_out) return fail(c, PEPS_EINVAL, "profile_read: args");
  PV_CUDA(c, cudaStreamSynchronize(c->stream));
  c->kprof.fold();
  // the truncations' flops depend on their Jacobi sweeps: counted on the device
  double jf = 0;
  if (c->d_jflops) PV_CUDA(c, cudaMemcpy(&jf, c->d_jflops, sizeof(double), cudaMemcpyDeviceToHost));
  const auto& acc = c->kprof.acc;
  *n_out = (int)acc.size();
  for (int i = 0; i < cap && i < (int)acc.size(); ++i) {
    memset(&out[i], 0, sizeof(out[i]));
    strncpy(out[i].name, acc[i].name.c_str(), sizeof(out[i].name) - 1);
    out[i].launches = acc[i].launches;
    out[i].ms = acc[i].ms;
    out[i].bytes = acc[i].bytes;
    out[i].flops = acc[i].flops + (acc[i].name == "kb_trunc" ? jf : 0.0);
  }
  return PEPS_OK;
}

int peps_profile_launch_bytes(peps_ctx* c, const char* name, double* bytes, int cap, int* n_out) {
  if (!c || !name || cap < 0 || (cap > 0 && !bytes) || !n_out)
    return fail(c, PEPS_EINVAL, "profile_launch_bytes: args");
  int k = 0;
  for (const pv::KProf::Rec& r : c->kprof.recs) {
    if (strcmp(r.name, name) != 0) continue;
    if (k < cap) bytes[k] = r.bytes;
    ++k;
  }
  *n_out = k;
  return PEPS_OK;
}

namespace {
struct CkptHeader {
  char magic[8];
  uint32_t version, pad;
  int L1, L2, model, D, chi, n_chains, precision, pad2;
  double J1, J2, t;
  int64_t sweeps, Np, nS;
};

uint64_t fnv1a(const void* p, size_t n, uint64_t h) {
  const unsigned char* b = (const unsigned char*)p;
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ULL;
  }
  return h;
}
}  // namespace

int peps_checkpoint(peps_ctx* c, const char* path) {
  if (!c || !path) return fail(c, PEPS_EINVAL, "checkpoint: args");
  std::vector<double> th(c->Np);
  std::vector<uint8_t> S((size_t)c->P.n_chains * c->N);
  PV_TRY(peps_get_theta(c, th.data(), th.size()));
  PV_TRY(peps_get_configs(c, S.data(), S.size()));
  CkptHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, "PEPSCKP1", 8);
  h.version = 1;
  h.L1 = c->P.L1;
  h.L2 = c->P.L2;
  h.model = c->P.model;
  h.D = c->P.D;
  h.chi = c->P.chi;
  h.n_chains = c->P.n_chains;
  h.precision = c->P.precision;
  h.J1 = c->P.J1;
  h.J2 = c->P.J2;
  h.t = c->t;
  h.sweeps = c->sweeps;
  h.Np = c->Np;
  h.nS = (int64_t)S.size();
  uint64_t sum = 1469598103934665603ULL;
  sum = fnv1a(&h, sizeof(h), sum);
  sum = fnv1a(th.data(), th.size() * sizeof(double), sum);
  sum = fnv1a(S.data(), S.size(), sum);
  FILE* f = fopen(path, "wb");
  if (!f) return fail(c, PEPS_EIO, std::string("checkpoint: cannot open ") + path);
  bool ok = fwrite(&h, sizeof(h), 1, f) == 1 &&
            fwrite(th.data(), sizeof(double), th.size(), f) == th.size() &&
            fwrite(S.data(), 1, S.size(), f) == S.size() && fwrite(&sum, sizeof(sum), 1, f) == 1;
  ok = (fclose(f) == 0) && ok;
  return ok ? PEPS_OK : fail(c, PEPS_EIO, "checkpoint: write failed");
}

int peps_restore(peps_ctx* c, const char* path) {
  if (!c || !path) return fail(c, PEPS_EINVAL, "restore: args");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(c, PEPS_ECORRUPT, std::string("restore: cannot open ") + path);
  CkptHeader h;
  bool ok = fread(&h, sizeof(h), 1, f) == 1 && memcmp(h.magic, "PEPSCKP1", 8) == 0 &&
            h.version == 1 && h.L1 == c->P.L1 && h.L2 == c->P.L2 && h.model == c->P.model &&
            h.D == c->P.D && h.chi == c->P.chi && h.n_chains == c->P.n_chains &&
            h.J1 == c->P.J1 && h.J2 == c->P.J2 && h.Np == c->Np &&
            h.nS == (int64_t)c->P.n_chains * c->N && h.sweeps >= 0;
  std::vector<double> th;
  std::vector<uint8_t> S;
  uint64_t sum = 0;
  if (ok) {
    th.resize(c->Np);
    S.resize((size_t)h.nS);
    ok = fread(th.data(), sizeof(double), th.size(), f) == th.size() &&
         fread(S.data(), 1, S.size(), f) == S.size() && fread(&sum, sizeof(sum), 1, f) == 1;
  }
  if (ok) {
    char extra;
    ok = fread(&extra, 1, 1, f) == 0;   // no trailing bytes
  }
  fclose(f);
  if (ok) {
    uint64_t chk = 1469598103934665603ULL;
    chk = fnv1a(&h, sizeof(h), chk);
    chk = fnv1a(th.data(), th.size() * sizeof(double), chk);
    chk = fnv1a(S.data(), S.size(), chk);
    ok = chk == sum;
    for (size_t i = 0; ok && i < S.size(); ++i) ok = S[i] <= 3;
  }
  if (!ok) return fail(c, PEPS_ECORRUPT, std::string("restore: corrupt or mismatched checkpoint ") + path);
  PV_TRY(peps_set_theta(c, th.data(), th.size()));
  PV_TRY(peps_set_configs(c, S.data(), S.size()));
  c->t = h.t;
  c->sweeps = h.sweeps;
  return PEPS_OK;
}

int peps_step(peps_ctx* c, int n_sweeps, int p, double tau, double eps, int max_cg,
              double cg_tol, peps_stats* st) {
  PV_TRY(peps_mc_sweep(c, n_sweeps, p));
  if (!c) return PEPS_EINVAL;
  PV_TRY(peps_eval_batch(c, nullptr, c->P.n_chains, 1, nullptr, nullptr, nullptr, nullptr,
                         nullptr));
  return peps_sr_step(c, tau, eps, max_cg, cg_tol, p, st);
}

}  // extern "C"

// ------------------------------------------------------------------ fermionic amplitudes

struct peps_famp {
  peps_ctx* c = nullptr;   // internal context: stream, allocations, the batched runner
  std::vector<long long> toff16, toff32;
  long long n16 = 0;
  int n_max = 0;
  long long *d_toff16 = nullptr, *d_toff32 = nullptr;
  double* d_th16 = nullptr;
  void* d_th32 = nullptr;
  uint8_t *d_S16 = nullptr, *d_S32 = nullptr;
  int8_t *d_csign = nullptr, *d_sg = nullptr;
  double* d_la = nullptr;
  int* d_bad = nullptr;
  BatchImpl<double>* b64 = nullptr;
  BatchImpl<float>* b32 = nullptr;
  // local energies: nearest-neighbour bonds, and the configurations one allowed hop away
  // (at most four per bond and chain, packed per chain at d_off) with their coefficients,
  // slots and amplitudes
  int* d_bi = nullptr;
  int* d_bj = nullptr;
  int nbonds = 0;
  long long x_cap = 0;
  uint8_t* d_Sx = nullptr;
  double *d_coef = nullptr, *d_lax = nullptr, *d_es = nullptr, *d_ea = nullptr;
  int8_t* d_sgx = nullptr;
  int *d_cnt = nullptr, *d_off = nullptr, *d_slot = nullptr;
  void* d_O = nullptr;             // O rows of up to n_max configurations
  long long* d_ooff = nullptr;
  // sampling: the moves of one sweep, the proposed configurations and their amplitudes
  std::vector<FMove> moves;
  uint8_t *d_Sp = nullptr, *d_Sc = nullptr;
  int *d_act = nullptr, *d_pos = nullptr;
  double *d_la2 = nullptr, *d_u = nullptr;
  int8_t* d_sg2 = nullptr;
  int* d_acc = nullptr;
  size_t u_cap = 0;
  // SR over the sixteen-slice parameters: weights, chunk partials, CG vectors
  int nvb = 0;
  int* d_o2site = nullptr;
  double *d_w = nullptr, *d_E = nullptr, *d_y = nullptr, *d_ypart = nullptr;
  double *d_obar = nullptr, *d_g = nullptr, *d_x = nullptr, *d_r = nullptr, *d_p = nullptr,
         *d_q = nullptr;
  double *d_part = nullptr, *d_part2 = nullptr, *d_bp1 = nullptr, *d_bp2 = nullptr,
         *d_pqpart = nullptr;
  SRScalars* d_sc = nullptr;
  FObs* d_fo = nullptr;
  // strip forms (peps_famp_set_strips): the 64 slices per site and their offsets
  bool strips = false;
  std::vector<long long> toff64;
  long long* d_toff64 = nullptr;
  void* d_th64 = nullptr;
};

namespace {

// log|psi| and sign of `count` configurations already on the device (entries checked unless
// `check` is off: the caller knows them valid): in pieces of n_max through the extended
// indices and the engine.
int famp_amplitudes(peps_famp* f, const uint8_t* dS, long long count, double* la, int8_t* sg,
                    bool check = true) {
  peps_ctx* c = f->c;
  const int N = c->N;
  cudaStream_t st = c->stream;
  if (check) PV_CUDA(c, cudaMemsetAsync(f->d_bad, 0, sizeof(int), st));
  for (long long off = 0; off < count; off += f->n_max) {
    const int nb = (int)std::min<long long>(f->n_max, count - off);
    PV_KLAUNCH(&c->kprof, st, "k_fconfigs", 0.0, 0.0,
               k_fconfigs<<<(nb + 127) / 128, 128, 0, st>>>(nb, c->P.L1, c->P.L2, dS + off * N,
                                                           f->d_S32, f->d_csign, f->d_bad));
    const int chunk = c->batch->chunk;
    for (int o2 = 0; o2 < nb; o2 += chunk) {
      const int n = std::min(chunk, nb - o2);
      if (f->b64)
        plain_amplitude(f->b64->run, f->d_S32 + (long long)o2 * N, n, la + off + o2, sg + off + o2);
      else
        plain_amplitude(f->b32->run, f->d_S32 + (long long)o2 * N, n, la + off + o2, sg + off + o2);
    }
    PV_KLAUNCH(&c->kprof, st, "k_fapply", 0.0, 0.0,
               k_fapply<<<(nb + 127) / 128, 128, 0, st>>>(nb, f->d_csign, sg + off, la + off));
  }
  PV_CUDA(c, cudaGetLastError());
  if (!check) return PEPS_OK;
  int bad = 0;
  PV_CUDA(c, cudaMemcpyAsync(&bad, f->d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  PV_CUDA(c, cudaStreamSynchronize(st));
  if (bad) return fail(c, PEPS_EINVAL, "famp: a local index exceeds 15");
  return batch_status(c);
}

// theta (host, sixteen slices per site) into the signed slices on the device
int famp_theta(peps_famp* f, const double* theta) {
  peps_ctx* c = f->c;
  const int N = c->N;
  cudaStream_t st = c->stream;
  PV_CUDA(c, cudaMemcpyAsync(f->d_th16, theta, (size_t)f->n16 * sizeof(double), cudaMemcpyHostToDevice, st));
  long long big = 0;
  for (int i = 0; i < N; ++i) big = std::max(big, f->toff32[i + 1] - f->toff32[i]);
  dim3 g((unsigned)std::min<long long>((big + 255) / 256, 1024), (unsigned)N);
  if (f->b64)
    PV_KLAUNCH(&c->kprof, st, "k_fsigned", 0.0, 0.0,
               k_fsigned<double><<<g, 256, 0, st>>>(c->P.L1, c->P.L2, c->P.D, f->d_th16, f->d_toff16,
                                                    (double*)f->d_th32, f->d_toff32));
  else
    PV_KLAUNCH(&c->kprof, st, "k_fsigned", 0.0, 0.0,
               k_fsigned<float><<<g, 256, 0, st>>>(c->P.L1, c->P.L2, c->P.D, f->d_th16, f->d_toff16,
                                                   (float*)f->d_th32, f->d_toff32));
  if (f->strips) {
    dim3 g64((unsigned)std::min<long long>((2 * big + 255) / 256, 1024), (unsigned)N);
    if (f->b64)
      PV_KLAUNCH(&c->kprof, st, "k_fsigned64", 0.0, 0.0,
                 k_fsigned64<double><<<g64, 256, 0, st>>>(c->P.L1, c->P.L2, c->P.D, f->d_th16, f->d_toff16,
                                                          (double*)f->d_th64, f->d_toff64));
    else
      PV_KLAUNCH(&c->kprof, st, "k_fsigned64", 0.0, 0.0,
                 k_fsigned64<float><<<g64, 256, 0, st>>>(c->P.L1, c->P.L2, c->P.D, f->d_th16, f->d_toff16,
                                                         (float*)f->d_th64, f->d_toff64));
  }
  PV_CUDA(c, cudaGetLastError());
  return PEPS_OK;
}

// The strip forms on the engine's runner, pointed at the 64 slices for the call: one sweep
// (fermion_mc), the local energies (fermion_eloc) or the local energies with the O rows
// (fermion_eval) of the nb chains in d_S16, chunk by chunk.
enum { FAMP_SWEEP = 0, FAMP_ELOC = 1, FAMP_EVAL = 2 };

template <typename T>
int famp_strips_t(peps_famp* f, BatchImpl<T>* bi, int nb, int what, int p, uint64_t seed,
                  uint32_t sweep_no, double t_hop, double U, double mu) {
  peps_ctx* c = f->c;
  const int N = c->N;
  auto& run = bi->run;
  const T* th_old = run.theta;
  const std::vector<long long> toff_old = run.toff;
  run.theta = (const T*)f->d_th64;
  run.toff = f->toff64;
  const int chunk = c->batch->chunk;
  for (int off = 0; off < nb; off += chunk) {
    const int n = std::min(chunk, nb - off);
    if (what == FAMP_SWEEP)
      fermion_mc(run, f->d_S16 + (long long)off * N, f->d_S32 + (long long)off * N, n, p, seed,
                 sweep_no, f->d_acc + off, off);
    else if (what == FAMP_ELOC)
      fermion_eloc(run, f->d_S16 + (long long)off * N, f->d_S32 + (long long)off * N, n, t_hop, U, mu,
                   f->d_la + off, f->d_sg + off, f->d_es + off, f->d_ea + off);
    else
      fermion_eval(run, f->d_S16 + (long long)off * N, f->d_S32 + (long long)off * N, n, t_hop, U, mu,
                   f->d_la + off, f->d_sg + off, f->d_es + off, f->d_ea + off,
                   (T*)f->d_O + (long long)off * c->No, c->No, f->d_ooff);
  }
  run.theta = th_old;
  run.toff = toff_old;
  PV_CUDA(c, cudaGetLastError());
  return PEPS_OK;
}

int famp_strips(peps_famp* f, int nb, int what, int p, uint64_t seed, uint32_t sweep_no,
                double t_hop, double U, double mu) {
  return f->b64 ? famp_strips_t(f, f->b64, nb, what, p, seed, sweep_no, t_hop, U, mu)
                : famp_strips_t(f, f->b32, nb, what, p, seed, sweep_no, t_hop, U, mu);
}

// log|psi|, sign, E_sys and E_anc of the nb configurations in d_S16 (theta's slices made):
// the amplitudes, the configurations one hop away with their Jordan-Wigner coefficients, their
// amplitudes, the sums.
int famp_energies(peps_famp* f, int nb, double t_hop, double U, double mu) {
  peps_ctx* c = f->c;
  const int N = c->N;
  cudaStream_t st = c->stream;
  if (!f->d_bi) {
    std::vector<int> bi, bj;
    for (int r = 0; r < c->P.L1; ++r)
      for (int q = 0; q < c->P.L2; ++q) {
        const int i = r * c->P.L2 + q;
        if (q + 1 < c->P.L2) {
          bi.push_back(i);
          bj.push_back(i + 1);
        }
        if (r + 1 < c->P.L1) {
          bi.push_back(i);
          bj.push_back(i + c->P.L2);
        }
      }
    f->nbonds = (int)bi.size();
    PV_TRY(dalloc(c, &f->d_bi, bi.size() * sizeof(int)));
    PV_TRY(dalloc(c, &f->d_bj, bj.size() * sizeof(int)));
    PV_CUDA(c, cudaMemcpy(f->d_bi, bi.data(), bi.size() * sizeof(int), cudaMemcpyHostToDevice));
    PV_CUDA(c, cudaMemcpy(f->d_bj, bj.data(), bj.size() * sizeof(int), cudaMemcpyHostToDevice));
    PV_TRY(dalloc(c, &f->d_es, (size_t)f->n_max * sizeof(double)));
    PV_TRY(dalloc(c, &f->d_ea, (size_t)f->n_max * sizeof(double)));
    PV_TRY(dalloc(c, &f->d_cnt, (size_t)f->n_max * sizeof(int)));
    PV_TRY(dalloc(c, &f->d_off, (size_t)(f->n_max + 1) * sizeof(int)));
    // at most one allowed hop per bond and mode: four per bond and chain
    const long long cap = (long long)f->n_max * 4 * f->nbonds;
    PV_TRY(dalloc(c, &f->d_Sx, (size_t)cap * N));
    PV_TRY(dalloc(c, &f->d_coef, (size_t)cap * sizeof(double)));
    PV_TRY(dalloc(c, &f->d_slot, (size_t)cap * sizeof(int)));
    PV_TRY(dalloc(c, &f->d_lax, (size_t)cap * sizeof(double)));
    PV_TRY(dalloc(c, &f->d_sgx, (size_t)cap));
    f->x_cap = cap;
  }
  PV_TRY(famp_amplitudes(f, f->d_S16, nb, f->d_la, f->d_sg));   // also checks the entries
  if (f->strips) return famp_strips(f, nb, FAMP_ELOC, 2, 0, 0, t_hop, U, mu);
  const unsigned gb = (unsigned)((nb + 127) / 128);
  PV_KLAUNCH(&c->kprof, st, "k_fhop_count", 0.0, 0.0,
             k_fhop_count<<<gb, 128, 0, st>>>(nb, N, f->d_S16, f->d_bi, f->d_bj, f->nbonds, f->d_cnt));
  PV_KLAUNCH(&c->kprof, st, "k_fscan", 0.0, 0.0, k_fscan<<<1, 1024, 0, st>>>(nb, f->d_cnt, f->d_off));
  PV_KLAUNCH(&c->kprof, st, "k_fhops", 0.0, 0.0,
             k_fhops<<<gb, 128, 0, st>>>(nb, N, f->d_S16, f->d_bi, f->d_bj, f->nbonds, t_hop, f->d_off,
                                         f->d_Sx, f->d_coef, f->d_slot));
  int nx = 0;
  PV_CUDA(c, cudaMemcpyAsync(&nx, f->d_off + nb, sizeof(int), cudaMemcpyDeviceToHost, st));
  PV_CUDA(c, cudaStreamSynchronize(st));
  if (nx < 0 || nx > f->x_cap) return fail(c, PEPS_ECUDA, "famp: hop count out of range");
  PV_TRY(famp_amplitudes(f, f->d_Sx, nx, f->d_lax, f->d_sgx, false));
  PV_KLAUNCH(&c->kprof, st, "k_fsum", 0.0, 0.0,
             k_fsum<<<gb, 128, 0, st>>>(nb, N, f->d_S16, U, mu, f->d_off, f->d_coef, f->d_slot, f->d_lax,
                                        f->d_sgx, f->d_la, f->d_sg, f->d_es, f->d_ea));
  PV_CUDA(c, cudaGetLastError());
  return PEPS_OK;
}

// O rows of the nb configurations in d_S16 into d_O (theta's slices made): the plain rows of
// the signed slices, then the per-entry signs.
// The O-row buffer of n_max configurations and the site offsets of a row, made once.
int famp_orows_alloc(peps_famp* f) {
  if (f->d_O) return PEPS_OK;
  peps_ctx* c = f->c;
  const int N = c->N;
  const size_t real = f->b64 ? sizeof(double) : sizeof(float);
  PV_TRY(dalloc(c, (unsigned char**)&f->d_O, (size_t)f->n_max * c->No * real));
  PV_TRY(dalloc(c, &f->d_ooff, (N + 1) * sizeof(long long)));
  PV_CUDA(c, cudaMemcpy(f->d_ooff, c->ooff.data(), (N + 1) * sizeof(long long), cudaMemcpyHostToDevice));
  return PEPS_OK;
}

int famp_orows(peps_famp* f, int nb) {
  peps_ctx* c = f->c;
  const int N = c->N;
  const long long No = c->No;
  cudaStream_t st = c->stream;
  PV_TRY(famp_orows_alloc(f));
  PV_CUDA(c, cudaMemsetAsync(f->d_bad, 0, sizeof(int), st));
  PV_KLAUNCH(&c->kprof, st, "k_fconfigs", 0.0, 0.0,
             k_fconfigs<<<(nb + 127) / 128, 128, 0, st>>>(nb, c->P.L1, c->P.L2, f->d_S16, f->d_S32,
                                                         f->d_csign, f->d_bad));
  int bad = 0;
  PV_CUDA(c, cudaMemcpyAsync(&bad, f->d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  PV_CUDA(c, cudaStreamSynchronize(st));
  if (bad) return fail(c, PEPS_EINVAL, "famp: a local index exceeds 15");
  const int chunk = c->batch->chunk;
  for (int off = 0; off < nb; off += chunk) {
    const int n = std::min(chunk, nb - off);
    if (f->b64)
      plain_log_derivative(f->b64->run, f->d_S32 + (long long)off * N, n, (double*)f->d_O + (long long)off * No, No);
    else
      plain_log_derivative(f->b32->run, f->d_S32 + (long long)off * N, n, (float*)f->d_O + (long long)off * No, No);
  }
  long long big = 0;
  for (int i = 0; i < N; ++i) big = std::max(big, c->ooff[i + 1] - c->ooff[i]);
  dim3 g((unsigned)std::min<long long>(((long long)nb * big + 255) / 256, 4096), (unsigned)N);
  if (f->b64)
    PV_KLAUNCH(&c->kprof, st, "k_fosign", 0.0, 0.0,
               k_fosign<double><<<g, 256, 0, st>>>(nb, c->P.L1, c->P.L2, c->P.D, (double*)f->d_O, No,
                                                   f->d_ooff, f->d_S16));
  else
    PV_KLAUNCH(&c->kprof, st, "k_fosign", 0.0, 0.0,
               k_fosign<float><<<g, 256, 0, st>>>(nb, c->P.L1, c->P.L2, c->P.D, (float*)f->d_O, No,
                                                  f->d_ooff, f->d_S16));
  PV_CUDA(c, cudaGetLastError());
  return PEPS_OK;
}

// The sampling buffers (n_max chains), made once.
int famp_sweep_buffers(peps_famp* f) {
  if (f->d_Sp) return PEPS_OK;
  peps_ctx* c = f->c;
  const size_t n = (size_t)f->n_max;
  PV_TRY(dalloc(c, &f->d_Sp, n * c->N));
  PV_TRY(dalloc(c, &f->d_Sc, n * c->N));
  PV_TRY(dalloc(c, &f->d_act, n * sizeof(int)));
  PV_TRY(dalloc(c, &f->d_pos, (n + 1) * sizeof(int)));
  PV_TRY(dalloc(c, &f->d_la2, n * sizeof(double)));
  PV_TRY(dalloc(c, &f->d_sg2, n));
  PV_TRY(dalloc(c, &f->d_acc, n * sizeof(int)));
  return PEPS_OK;
}

// The SR buffers (n_max samples, the sixteen-slice parameters), made once.
int famp_sr_buffers(peps_famp* f) {
  if (f->d_sc) return PEPS_OK;
  peps_ctx* c = f->c;
  const int N = c->N;
  const long long Np = f->n16, No = c->No;
  const size_t n = (size_t)f->n_max;
  const size_t nch = (n + OTV_CHUNK - 1) / OTV_CHUNK, nyb = (n + SR_THREADS / 32 - 1) / (SR_THREADS / 32);
  f->nvb = grid_for(Np, SR_THREADS, 1024);
  std::vector<int> o2s((size_t)No);
  for (int i = 0; i < N; ++i)
    for (long long o = c->ooff[i]; o < c->ooff[i + 1]; ++o) o2s[(size_t)o] = i;
  PV_TRY(dalloc(c, &f->d_o2site, (size_t)No * sizeof(int)));
  PV_CUDA(c, cudaMemcpy(f->d_o2site, o2s.data(), (size_t)No * sizeof(int), cudaMemcpyHostToDevice));
  for (double** v : {&f->d_w, &f->d_E, &f->d_y}) PV_TRY(dalloc(c, v, n * sizeof(double)));
  PV_TRY(dalloc(c, &f->d_ypart, nyb * sizeof(double)));
  for (double** v : {&f->d_obar, &f->d_g, &f->d_x, &f->d_r, &f->d_p, &f->d_q})
    PV_TRY(dalloc(c, v, (size_t)Np * sizeof(double)));
  PV_TRY(dalloc(c, &f->d_part, nch * Np * sizeof(double)));
  PV_TRY(dalloc(c, &f->d_part2, nch * Np * sizeof(double)));
  for (double** v : {&f->d_bp1, &f->d_bp2, &f->d_pqpart}) PV_TRY(dalloc(c, v, (size_t)f->nvb * sizeof(double)));
  PV_TRY(dalloc(c, &f->d_fo, sizeof(FObs)));
  PV_TRY(dalloc(c, &f->d_sc, sizeof(SRScalars)));
  return PEPS_OK;
}

}  // namespace

extern "C" {

int peps_famp_create(int L1, int L2, int D, int chi, int n_max, int precision, void* stream,
                     peps_famp** out) {
  if (!out) return PEPS_EINVAL;
  *out = nullptr;
  if (L1 < 2 || L2 < 2 || L1 > MAX_L || L2 > MAX_L || D < 1 || D > 8 || chi < 1 || chi > 64 ||
      n_max < 1 || (precision != PEPS_FP64 && precision != PEPS_FP32 && precision != PEPS_TF32))
    return PEPS_EINVAL;
  std::unique_ptr<peps_famp> f(new peps_famp());
  peps_ctx* c = new peps_ctx();
  f->c = c;
  c->P.L1 = L1;
  c->P.L2 = L2;
  c->P.D = D;
  c->P.chi = chi;
  c->P.n_chains = n_max;
  c->P.precision = precision;
  c->P.model = PEPS_MODEL_J1J2;
  c->P.block_mode = PEPS_BLOCKS_BATCHED;
  c->stream = (cudaStream_t)stream;
  const int N = L1 * L2;
  c->N = N;
  f->n_max = n_max;
  f->toff16.assign(N + 1, 0);
  f->toff32.assign(N + 1, 0);
  c->ooff.assign(N + 1, 0);
  for (int i = 0; i < N; ++i) {
    const int r = i / L2, q = i % L2;
    const long long sz = (long long)(q == 0 ? 1 : D) * (q == L2 - 1 ? 1 : D) * (r == 0 ? 1 : D) *
                         (r == L1 - 1 ? 1 : D);
    f->toff16[i + 1] = f->toff16[i] + 16 * sz;
    f->toff32[i + 1] = f->toff32[i] + 32 * sz;
    c->ooff[i + 1] = c->ooff[i] + sz;
  }
  c->No = c->ooff[N];
  f->n16 = f->toff16[N];
  f->moves = fermion_moves(L1, L2);
  f->toff64.assign(N + 1, 0);
  for (int i = 0; i < N; ++i) f->toff64[i + 1] = f->toff64[i] + 2 * (f->toff32[i + 1] - f->toff32[i]);
  const size_t real = precision == PEPS_FP64 ? sizeof(double) : sizeof(float);
  auto bail = [&](int rc) {
    peps_free(c);
    f->c = nullptr;
    return rc;
  };
  int rc;
  if ((rc = dalloc(c, &f->d_toff16, (N + 1) * sizeof(long long)))) return bail(rc);
  if ((rc = dalloc(c, &f->d_toff32, (N + 1) * sizeof(long long)))) return bail(rc);
  if ((rc = dalloc(c, &f->d_th16, (size_t)f->n16 * sizeof(double)))) return bail(rc);
  if ((rc = dalloc(c, (unsigned char**)&f->d_th32, (size_t)f->toff32[N] * real))) return bail(rc);
  if ((rc = dalloc(c, &f->d_S16, (size_t)n_max * N))) return bail(rc);
  if ((rc = dalloc(c, &f->d_S32, (size_t)n_max * N))) return bail(rc);
  if ((rc = dalloc(c, &f->d_csign, (size_t)n_max))) return bail(rc);
  if ((rc = dalloc(c, &f->d_sg, (size_t)n_max))) return bail(rc);
  if ((rc = dalloc(c, &f->d_la, (size_t)n_max * sizeof(double)))) return bail(rc);
  if ((rc = dalloc(c, &f->d_bad, sizeof(int)))) return bail(rc);
  if ((rc = dalloc(c, &c->d_jsw, sizeof(unsigned long long)))) return bail(rc);
  if (cudaMemcpy(f->d_toff16, f->toff16.data(), (N + 1) * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(f->d_toff32, f->toff32.data(), (N + 1) * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(PEPS_ECUDA);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (precision == PEPS_FP64) {
    f->b64 = new BatchImpl<double>();
    c->batch.reset(f->b64);
    rc = init_runner_t<double>(c, sms, f->b64, D, (const double*)f->d_th32, f->toff32);
  } else {
    f->b32 = new BatchImpl<float>();
    c->batch.reset(f->b32);
    rc = init_runner_t<float>(c, sms, f->b32, D, (const float*)f->d_th32, f->toff32);
  }
  if (rc != PEPS_OK) return bail(rc);
  *out = f.release();
  return PEPS_OK;
}

int peps_famp_eval(peps_famp* f, const double* theta, size_t n_theta, const uint8_t* S, int nb,
                   double* log_abs, int8_t* sign) {
  if (!f || !f->c) return PEPS_EINVAL;
  peps_ctx* c = f->c;
  if (!theta || n_theta != (size_t)f->n16 || nb < 0 || nb > f->n_max || (nb > 0 && !S))
    return fail(c, PEPS_EINVAL, "famp_eval: args");
  if (nb == 0) return PEPS_OK;
  cudaStream_t st = c->stream;
  PV_TRY(famp_theta(f, theta));
  PV_CUDA(c, cudaMemcpyAsync(f->d_S16, S, (size_t)nb * c->N, cudaMemcpyHostToDevice, st));
  PV_TRY(famp_amplitudes(f, f->d_S16, nb, f->d_la, f->d_sg));
  if (log_abs) PV_CUDA(c, cudaMemcpyAsync(log_abs, f->d_la, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (sign) PV_CUDA(c, cudaMemcpyAsync(sign, f->d_sg, (size_t)nb, cudaMemcpyDeviceToHost, st));
  PV_CUDA(c, cudaStreamSynchronize(st));
  return PEPS_OK;
}

int peps_famp_local_energy(peps_famp* f, const double* theta, size_t n_theta, const uint8_t* S,
                           int nb, double t_hop, double U, double mu, double* log_abs,
                           int8_t* sign, double* e_sys, double* e_anc) {
  if (!f || !f->c) return PEPS_EINVAL;
  peps_ctx* c = f->c;
  if (!theta || n_theta != (size_t)f->n16 || nb < 0 || nb > f->n_max || (nb > 0 && !S) ||
      !std::isfinite(t_hop) || !std::isfinite(U) || !std::isfinite(mu))
    return fail(c, PEPS_EINVAL, "famp_local_energy: args");
  if (nb == 0) return PEPS_OK;
  cudaStream_t st = c->stream;
  PV_TRY(famp_theta(f, theta));
  PV_CUDA(c, cudaMemcpyAsync(f->d_S16, S, (size_t)nb * c->N, cudaMemcpyHostToDevice, st));
  PV_TRY(famp_energies(f, nb, t_hop, U, mu));
  if (log_abs) PV_CUDA(c, cudaMemcpyAsync(log_abs, f->d_la, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (sign) PV_CUDA(c, cudaMemcpyAsync(sign, f->d_sg, (size_t)nb, cudaMemcpyDeviceToHost, st));
  if (e_sys) PV_CUDA(c, cudaMemcpyAsync(e_sys, f->d_es, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (e_anc) PV_CUDA(c, cudaMemcpyAsync(e_anc, f->d_ea, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  PV_CUDA(c, cudaStreamSynchronize(st));
  return batch_status(c);
}

int peps_famp_log_derivative(peps_famp* f, const double* theta, size_t n_theta, const uint8_t* S,
                             int nb, void* O) {
  if (!f || !f->c) return PEPS_EINVAL;
  peps_ctx* c = f->c;
  if (!theta || n_theta != (size_t)f->n16 || nb < 0 || nb > f->n_max || (nb > 0 && (!S || !O)))
    return fail(c, PEPS_EINVAL, "famp_log_derivative: args");
  if (nb == 0) return PEPS_OK;
  cudaStream_t st = c->stream;
  const size_t real = f->b64 ? sizeof(double) : sizeof(float);
  PV_TRY(famp_theta(f, theta));
  PV_CUDA(c, cudaMemcpyAsync(f->d_S16, S, (size_t)nb * c->N, cudaMemcpyHostToDevice, st));
  PV_TRY(famp_orows(f, nb));
  PV_CUDA(c, cudaMemcpyAsync(O, f->d_O, (size_t)nb * c->No * real, cudaMemcpyDeviceToHost, st));
  PV_CUDA(c, cudaStreamSynchronize(st));
  return batch_status(c);
}

int peps_famp_set_strips(peps_famp* f, int enable) {
  if (!f || !f->c || enable < 0 || enable > 1) return PEPS_EINVAL;
  peps_ctx* c = f->c;
  if (enable && !f->d_th64) {
    const int N = c->N;
    const size_t real = f->b64 ? sizeof(double) : sizeof(float);
    PV_TRY(dalloc(c, (unsigned char**)&f->d_th64, (size_t)f->toff64[N] * real));
    PV_TRY(dalloc(c, &f->d_toff64, (N + 1) * sizeof(long long)));
    PV_CUDA(c, cudaMemcpy(f->d_toff64, f->toff64.data(), (N + 1) * sizeof(long long), cudaMemcpyHostToDevice));
  }
  f->strips = enable != 0;
  return PEPS_OK;
}

int peps_famp_n_moves(const peps_famp* f) {
  if (!f || !f->c) return PEPS_EINVAL;
  return (int)f->moves.size();
}

int peps_famp_sweep(peps_famp* f, const double* theta, size_t n_theta, uint8_t* S, int nb, int p,
                    int n_sweeps, uint64_t seed, uint64_t sweep0, const double* u, int* accepted,
                    double* log_abs, int8_t* sign) {
  if (!f || !f->c) return PEPS_EINVAL;
  peps_ctx* c = f->c;
  if (!theta || n_theta != (size_t)f->n16 || nb < 0 || nb > f->n_max || (nb > 0 && !S) ||
      (p != 1 && p != 2) || n_sweeps < 0 || sweep0 + (uint64_t)n_sweeps > 0xFFFFFFFFull)
    return fail(c, PEPS_EINVAL, "famp_sweep: args");
  if (u && f->strips) return fail(c, PEPS_EINVAL, "famp_sweep: given uniforms need the full-contraction sweep");
  if (nb == 0) return PEPS_OK;
  const int N = c->N, M = (int)f->moves.size();
  cudaStream_t st = c->stream;
  PV_TRY(famp_sweep_buffers(f));
  const size_t nu = (size_t)n_sweeps * nb * M;
  if (u && nu > f->u_cap) {
    PV_TRY(dalloc(c, &f->d_u, nu * sizeof(double)));
    f->u_cap = nu;
  }
  PV_TRY(famp_theta(f, theta));
  PV_CUDA(c, cudaMemcpyAsync(f->d_S16, S, (size_t)nb * N, cudaMemcpyHostToDevice, st));
  if (u && nu) PV_CUDA(c, cudaMemcpyAsync(f->d_u, u, nu * sizeof(double), cudaMemcpyHostToDevice, st));
  PV_TRY(famp_amplitudes(f, f->d_S16, nb, f->d_la, f->d_sg));   // also checks the entries
  PV_CUDA(c, cudaMemsetAsync(f->d_acc, 0, (size_t)nb * sizeof(int), st));
  const unsigned gb = (unsigned)((nb + 127) / 128);
  for (int k = 0; k < n_sweeps && f->strips; ++k)
    PV_TRY(famp_strips(f, nb, FAMP_SWEEP, p, seed, (uint32_t)(sweep0 + k), 0.0, 0.0, 0.0));
  if (f->strips && n_sweeps > 0) PV_TRY(famp_amplitudes(f, f->d_S16, nb, f->d_la, f->d_sg, false));
  for (int k = 0; k < n_sweeps && !f->strips; ++k) {
    const double* uk = u ? f->d_u + (size_t)k * nb * M : nullptr;
    for (int m = 0; m < M; ++m) {
      // the proposal per chain; only the chains where it applies are packed and contracted
      PV_KLAUNCH(&c->kprof, st, "k_fpropose", 0.0, 0.0,
                 k_fpropose<<<gb, 128, 0, st>>>(nb, N, f->d_S16, f->d_Sp, f->moves[m], f->d_act));
      PV_KLAUNCH(&c->kprof, st, "k_fscan", 0.0, 0.0, k_fscan<<<1, 1024, 0, st>>>(nb, f->d_act, f->d_pos));
      int na = 0;
      PV_CUDA(c, cudaMemcpyAsync(&na, f->d_pos + nb, sizeof(int), cudaMemcpyDeviceToHost, st));
      PV_CUDA(c, cudaStreamSynchronize(st));
      if (na < 0 || na > nb) return fail(c, PEPS_ECUDA, "famp_sweep: proposal count out of range");
      if (na == 0) continue;
      PV_KLAUNCH(&c->kprof, st, "k_fgather", 0.0, 0.0,
                 k_fgather<<<(unsigned)(((long long)nb * N + 255) / 256), 256, 0, st>>>(
                     nb, N, f->d_Sp, f->d_act, f->d_pos, f->d_Sc));
      PV_TRY(famp_amplitudes(f, f->d_Sc, na, f->d_la2, f->d_sg2, false));
      PV_KLAUNCH(&c->kprof, st, "k_faccept", 0.0, 0.0,
                 k_faccept<<<gb, 128, 0, st>>>(nb, N, m, M, p, seed, (uint32_t)(sweep0 + k), uk,
                                               f->d_act, f->d_pos, f->d_la2, f->d_sg2, f->d_S16,
                                               f->d_Sp, f->d_la, f->d_sg, f->d_acc));
    }
    PV_CUDA(c, cudaGetLastError());
  }
  PV_CUDA(c, cudaMemcpyAsync(S, f->d_S16, (size_t)nb * N, cudaMemcpyDeviceToHost, st));
  if (accepted) PV_CUDA(c, cudaMemcpyAsync(accepted, f->d_acc, (size_t)nb * sizeof(int), cudaMemcpyDeviceToHost, st));
  if (log_abs) PV_CUDA(c, cudaMemcpyAsync(log_abs, f->d_la, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (sign) PV_CUDA(c, cudaMemcpyAsync(sign, f->d_sg, (size_t)nb, cudaMemcpyDeviceToHost, st));
  PV_CUDA(c, cudaStreamSynchronize(st));
  return batch_status(c);
}

int peps_famp_sr_step(peps_famp* f, double* theta, size_t n_theta, const uint8_t* S, int nb,
                      double t_hop, double U, double mu, int p, double tau, double eps,
                      int max_cg, double cg_tol, peps_fstats* out) {
  if (!f || !f->c) return PEPS_EINVAL;
  peps_ctx* c = f->c;
  if (!theta || n_theta != (size_t)f->n16 || nb < 1 || nb > f->n_max || !S || (p != 1 && p != 2) ||
      !std::isfinite(t_hop) || !std::isfinite(U) || !std::isfinite(mu) || !std::isfinite(tau) ||
      !(eps >= 0) || !(cg_tol >= 0) || max_cg < 0)
    return fail(c, PEPS_EINVAL, "famp_sr_step: args");
  const int N = c->N;
  const long long Np = f->n16, No = c->No;
  cudaStream_t st = c->stream;
  PV_TRY(famp_sr_buffers(f));
  PV_TRY(famp_theta(f, theta));
  PV_CUDA(c, cudaMemcpyAsync(f->d_S16, S, (size_t)nb * N, cudaMemcpyHostToDevice, st));
  if (f->strips) {
    // local energies and O rows in one pass over the rows (the hop buffers are not needed)
    PV_TRY(famp_orows_alloc(f));
    if (!f->d_es) {
      PV_TRY(dalloc(c, &f->d_es, (size_t)f->n_max * sizeof(double)));
      PV_TRY(dalloc(c, &f->d_ea, (size_t)f->n_max * sizeof(double)));
    }
    PV_TRY(famp_amplitudes(f, f->d_S16, nb, f->d_la, f->d_sg));   // checks the entries
    PV_TRY(famp_strips(f, nb, FAMP_EVAL, 2, 0, 0, t_hop, U, mu));
  } else {
    PV_TRY(famp_energies(f, nb, t_hop, U, mu));
    PV_TRY(famp_orows(f, nb));
  }
  PV_KLAUNCH(&c->kprof, st, "k_fweights", 0.0, 0.0,
             k_fweights<<<1, SR_WEIGHT_THREADS, 0, st>>>(nb, N, p, f->d_la, f->d_sg, f->d_es, f->d_ea,
                                                         f->d_S16, f->d_w, f->d_E, f->d_sc, f->d_fo));
  FObs fo;
  PV_CUDA(c, cudaMemcpyAsync(&fo, f->d_fo, sizeof(fo), cudaMemcpyDeviceToHost, st));
  PV_CUDA(c, cudaStreamSynchronize(st));
  if (fo.zero) return fail(c, PEPS_EINVAL, "famp_sr_step: a configuration has psi = 0");
  // mean and gradient: one pass over the rows, then the chunk sums
  const int nch = (nb + OTV_CHUNK - 1) / OTV_CHUNK, nyb = (nb + SR_THREADS / 32 - 1) / (SR_THREADS / 32);
  const int nvb = f->nvb;
  const dim3 cgrid((unsigned)((No + SR_THREADS - 1) / SR_THREADS), (unsigned)nch);
  const bool f64 = f->b64 != nullptr;
  if (f64)
    PV_KLAUNCH(&c->kprof, st, "k_fcolsum1", 0.0, 0.0,
               k_fcolsum1<double, true><<<cgrid, SR_THREADS, 0, st>>>(
                   nb, N, No, (const double*)f->d_O, f->d_S16, f->d_o2site, f->d_toff16, f->d_ooff,
                   f->d_w, f->d_E, &f->d_sc->Ebar, f->d_part, f->d_part2, Np, nullptr));
  else
    PV_KLAUNCH(&c->kprof, st, "k_fcolsum1", 0.0, 0.0,
               k_fcolsum1<float, true><<<cgrid, SR_THREADS, 0, st>>>(
                   nb, N, No, (const float*)f->d_O, f->d_S16, f->d_o2site, f->d_toff16, f->d_ooff,
                   f->d_w, f->d_E, &f->d_sc->Ebar, f->d_part, f->d_part2, Np, nullptr));
  PV_KLAUNCH(&c->kprof, st, "k_colsum2_grad", 0.0, 0.0,
             k_colsum2_grad<<<grid_for(Np, SR_THREADS, 1 << 20), SR_THREADS, 0, st>>>(
                 Np, nch, f->d_part, f->d_part2, f->d_obar, f->d_g));
  // CG from x = 0 (Eq. 10 products as two passes over the rows)
  PV_KLAUNCH(&c->kprof, st, "k_dot_part", 0.0, 0.0,
             k_dot_part<<<nvb, SR_THREADS, 0, st>>>(Np, f->d_g, f->d_g, f->d_bp1, nullptr));
  PV_KLAUNCH(&c->kprof, st, "k_cg_init", 0.0, 0.0,
             k_cg_init<<<nvb, SR_THREADS, 0, st>>>(Np, f->d_g, f->d_x, f->d_r, f->d_p, nvb, f->d_bp1,
                                                   f->d_sc, max_cg, cg_tol, eps));
  PV_KLAUNCH(&c->kprof, st, "k_dot_part", 0.0, 0.0,
             k_dot_part<<<nvb, SR_THREADS, 0, st>>>(Np, f->d_obar, f->d_p, f->d_bp2, nullptr));
  PV_CUDA(c, cudaGetLastError());
  for (int it = 0; it < max_cg; ++it) {
    if (f64) {
      PV_KLAUNCH(&c->kprof, st, "k_ov", 0.0, 0.0,
                 k_ov<double><<<nyb, SR_THREADS, 0, st>>>(nb, N, No, (const double*)f->d_O, f->d_S16,
                                                          f->d_toff16, f->d_ooff, f->d_p, f->d_w, f->d_y,
                                                          f->d_ypart, nvb, f->d_bp2, f->d_sc));
      PV_KLAUNCH(&c->kprof, st, "k_fcolsum1", 0.0, 0.0,
                 k_fcolsum1<double, false><<<cgrid, SR_THREADS, 0, st>>>(
                     nb, N, No, (const double*)f->d_O, f->d_S16, f->d_o2site, f->d_toff16, f->d_ooff,
                     f->d_y, nullptr, nullptr, f->d_part, nullptr, Np, &f->d_sc->done));
    } else {
      PV_KLAUNCH(&c->kprof, st, "k_ov", 0.0, 0.0,
                 k_ov<float><<<nyb, SR_THREADS, 0, st>>>(nb, N, No, (const float*)f->d_O, f->d_S16,
                                                         f->d_toff16, f->d_ooff, f->d_p, f->d_w, f->d_y,
                                                         f->d_ypart, nvb, f->d_bp2, f->d_sc));
      PV_KLAUNCH(&c->kprof, st, "k_fcolsum1", 0.0, 0.0,
                 k_fcolsum1<float, false><<<cgrid, SR_THREADS, 0, st>>>(
                     nb, N, No, (const float*)f->d_O, f->d_S16, f->d_o2site, f->d_toff16, f->d_ooff,
                     f->d_y, nullptr, nullptr, f->d_part, nullptr, Np, &f->d_sc->done));
    }
    PV_KLAUNCH(&c->kprof, st, "k_otv2", 0.0, 0.0,
               k_otv2<<<nvb, SR_THREADS, 0, st>>>(Np, nch, f->d_part, f->d_obar, f->d_p, f->d_q, nyb,
                                                  f->d_ypart, f->d_pqpart, f->d_sc));
    PV_KLAUNCH(&c->kprof, st, "k_cg_a", 0.0, 0.0,
               k_cg_a<<<nvb, SR_THREADS, 0, st>>>(Np, f->d_x, f->d_r, f->d_p, f->d_q, nvb, f->d_pqpart,
                                                  f->d_bp1, f->d_sc));
    PV_KLAUNCH(&c->kprof, st, "k_cg_b", 0.0, 0.0,
               k_cg_b<<<nvb, SR_THREADS, 0, st>>>(Np, f->d_r, f->d_p, f->d_obar, nvb, f->d_bp1,
                                                  f->d_bp2, f->d_sc));
    PV_KLAUNCH(&c->kprof, st, "k_cg_scalars", 0.0, 0.0,
               k_cg_scalars<<<1, 1, 0, st>>>(nvb, f->d_bp1, f->d_sc));
    PV_CUDA(c, cudaGetLastError());
    if ((it & 7) == 7) {
      int done = 0;
      PV_CUDA(c, cudaMemcpyAsync(&done, &f->d_sc->done, sizeof(int), cudaMemcpyDeviceToHost, st));
      PV_CUDA(c, cudaStreamSynchronize(st));
      if (done) break;
    }
  }
  PV_KLAUNCH(&c->kprof, st, "k_update", 0.0, 0.0,
             k_update<<<grid_for(Np, 256), 256, 0, st>>>(Np, tau, f->d_x, f->d_th16, nullptr));
  PV_CUDA(c, cudaGetLastError());
  SRScalars h;
  PV_CUDA(c, cudaMemcpyAsync(&h, f->d_sc, sizeof(h), cudaMemcpyDeviceToHost, st));
  PV_CUDA(c, cudaMemcpyAsync(theta, f->d_th16, (size_t)Np * sizeof(double), cudaMemcpyDeviceToHost, st));
  PV_CUDA(c, cudaStreamSynchronize(st));
  PV_TRY(batch_status(c));
  if (out) {
    out->E_site = fo.H1 / N;
    out->E_err = fo.Eerr / N;
    out->docc = fo.docc / N;
    out->density = fo.dens / N;
    out->cg_iters = h.iters;
    out->cg_resid = h.gnorm > 0 ? std::sqrt(h.rr) / h.gnorm : 0.0;
  }
  if (!std::isfinite(h.rr) || !std::isfinite(fo.H1))
    return fail(c, PEPS_ENOTFINITE, "famp_sr_step: non-finite energy or residual");
  return (h.iters >= max_cg && max_cg > 0 && h.gnorm > 0 && std::sqrt(h.rr) > cg_tol * h.gnorm)
             ? PEPS_WARN_CG_MAXIT
             : PEPS_OK;
}

int peps_famp_profile(peps_famp* f, int enable) {
  if (!f || !f->c) return PEPS_EINVAL;
  return peps_profile(f->c, enable);
}

int peps_famp_profile_read(peps_famp* f, peps_kernel_stat* out, int cap, int* n_out) {
  if (!f || !f->c) return PEPS_EINVAL;
  return peps_profile_read(f->c, out, cap, n_out);
}

long long peps_famp_launches(const peps_famp* f) { return f && f->c ? f->c->kprof.launches : 0; }

int peps_famp_move_table(int L1, int L2, int* table, int cap) {
  if (L1 < 1 || L2 < 1 || L1 > MAX_L || L2 > MAX_L || cap < 0 || (cap > 0 && !table)) return PEPS_EINVAL;
  const std::vector<FMove> mv = fermion_moves(L1, L2);
  for (int m = 0; m < (int)mv.size() && m < cap; ++m) {
    table[4 * m] = mv[m].kind;
    table[4 * m + 1] = mv[m].i;
    table[4 * m + 2] = mv[m].j;
    table[4 * m + 3] = mv[m].k;
  }
  return (int)mv.size();
}

int peps_famp_init_theta(int L1, int L2, int D, double noise, uint64_t seed, double* theta,
                         size_t n_theta) {
  if (L1 < 1 || L2 < 1 || D < 1 || !(noise >= 0) || !theta) return PEPS_EINVAL;
  size_t need = 0;
  for (int i = 0; i < L1 * L2; ++i) {
    const int r = i / L2, q = i % L2;
    need += 16 * (size_t)(q == 0 ? 1 : D) * (q == L2 - 1 ? 1 : D) * (r == 0 ? 1 : D) * (r == L1 - 1 ? 1 : D);
  }
  if (n_theta != need) return PEPS_EINVAL;
  size_t off = 0;
  for (int i = 0; i < L1 * L2; ++i) {
    const int r = i / L2, q = i % L2;
    const int dl = q == 0 ? 1 : D, dr = q == L2 - 1 ? 1 : D, du = r == 0 ? 1 : D, dd = r == L1 - 1 ? 1 : D;
    const size_t sz = (size_t)dl * dr * du * dd;
    for (size_t e = 0; e < 16 * sz; ++e) {
      const int S = (int)(e / sz);
      size_t k = e % sz;
      const int d = (int)(k % dd);
      k /= dd;
      const int u = (int)(k % du);
      k /= du;
      const int rr = (int)(k % dr);
      const int l = (int)(k / dr);
      const int par = ((S & 1) + ((S >> 1) & 1) + ((S >> 2) & 1) + ((S >> 3) & 1) + l + rr + u + d) & 1;
      double v = 0.0;
      if (!par && noise > 0)
        v = noise * (2.0 * philox_uniform(seed, (uint32_t)i, (uint32_t)e, 0u, TAG_FINIT) - 1.0);
      if (e % sz == 0 && (S & 3) == (S >> 2)) v = S == 15 ? -1.0 : 1.0;
      theta[off + e] = v;
    }
    off += 16 * sz;
  }
  return PEPS_OK;
}

const char* peps_famp_last_error(const peps_famp* f) { return f && f->c ? f->c->err.c_str() : ""; }

void peps_famp_free(peps_famp* f) {
  if (!f) return;
  if (f->c) peps_free(f->c);
  delete f;
}

}  // extern "C"

// ------------------------------------------------------------------ group evaluation

struct peps_group {
  std::vector<peps_ctx*> ctxs;
  bool f64 = true;
  long long total = 0, sreal = 0, sint = 0;
  int nblk = 0, smem = 0;
  GroupItem* d_items = nullptr;
  void* d_scr = nullptr;
  int* d_iscr = nullptr;
  double* d_flops = nullptr;
  unsigned long long* d_jsw = nullptr;
  std::string err;
  ~peps_group() {
    if (d_items) cudaFree(d_items);
    if (d_scr) cudaFree(d_scr);
    if (d_iscr) cudaFree(d_iscr);
    if (d_flops) cudaFree(d_flops);
    if (d_jsw) cudaFree(d_jsw);
  }
};

namespace {

int gfail(peps_group* g, int code, const std::string& msg) {
  g->err = msg;
  return code;
}

template <typename P>
cudaError_t galloc(P** p, size_t bytes) {
  return cudaMalloc((void**)p, bytes ? bytes : 16);
}

}  // namespace

extern "C" {

int peps_group_create(peps_ctx* const* ctxs, int n, peps_group** out) {
  if (!out) return PEPS_EINVAL;
  *out = nullptr;
  if (!ctxs || n < 1) return PEPS_EINVAL;
  std::unique_ptr<peps_group> g(new peps_group());
  for (int i = 0; i < n; ++i) {
    peps_ctx* c = ctxs[i];
    if (!c) return PEPS_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return PEPS_EINVAL;   // each context once
    // the per-block engine's narrow blocks, one arithmetic for the whole group
    if (c->batch || c->wide) return PEPS_EINVAL;
    if (i > 0 && fp64(c) != fp64(ctxs[0])) return PEPS_EINVAL;
    g->ctxs.push_back(c);
  }
  peps_group* G = g.get();
  G->f64 = fp64(ctxs[0]);
  const size_t real = G->f64 ? sizeof(double) : sizeof(float);
  std::vector<GroupItem> items;
  for (peps_ctx* c : G->ctxs) {
    GroupItem it;
    it.g = make_geom(c);
    it.theta = G->f64 ? (const void*)c->d_theta : (const void*)c->d_theta_f;
    it.S = c->d_S;
    it.first = G->total;
    it.n = c->P.n_chains;
    it.log_abs = c->d_log_abs;
    it.es = c->d_es;
    it.ea = c->d_ea;
    it.sign = c->d_sign;
    it.O = c->d_O;
    it.No = c->No;
    items.push_back(it);
    G->total += it.n;
    G->sreal = std::max(G->sreal, c->sreal);
    G->sint = std::max(G->sint, c->sint);
    G->smem = std::max(G->smem, c->smem_bytes);
  }
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  G->nblk = (int)std::min<long long>(G->total, 4LL * sms);
  cudaError_t e = galloc(&G->d_items, items.size() * sizeof(GroupItem));
  if (e == cudaSuccess) e = galloc(&G->d_scr, (size_t)G->nblk * G->sreal * real);
  if (e == cudaSuccess) e = galloc(&G->d_iscr, (size_t)G->nblk * G->sint * sizeof(int));
  if (e == cudaSuccess) e = galloc(&G->d_flops, sizeof(double));
  if (e == cudaSuccess) e = galloc(&G->d_jsw, sizeof(unsigned long long));
  if (e == cudaSuccess)
    e = cudaMemcpy(G->d_items, items.data(), items.size() * sizeof(GroupItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && G->smem > 48 * 1024)
    e = G->f64 ? cudaFuncSetAttribute(k_eval_group<double, SAMPLE_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024)
               : cudaFuncSetAttribute(k_eval_group<float, SAMPLE_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? PEPS_ENOMEM : PEPS_ECUDA;
  }
  *out = g.release();
  return PEPS_OK;
}

int peps_group_eval(peps_group* G) {
  if (!G) return PEPS_EINVAL;
  // every context's earlier work (sweeps, parameter updates) has finished
  for (peps_ctx* c : G->ctxs) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return gfail(G, PEPS_ECUDA, std::string("group_eval: ") + cudaGetErrorString(e));
  }
  peps_ctx* c0 = G->ctxs[0];
  cudaStream_t st = c0->stream;
  cudaMemsetAsync(G->d_flops, 0, sizeof(double), st);
  cudaMemsetAsync(G->d_jsw, 0, sizeof(unsigned long long), st);
  if (G->f64)
    PV_KLAUNCH(&c0->kprof, st, "k_eval_group", 0.0, 0.0,
               (k_eval_group<double, SAMPLE_THREADS><<<G->nblk, SAMPLE_THREADS, G->smem, st>>>(
                   G->d_items, (int)G->ctxs.size(), G->total, (double*)G->d_scr, G->d_iscr, G->sreal,
                   G->sint, (double)JTOL_F64, JAC_MAX_SWEEPS, G->d_flops, G->d_jsw, G->smem)));
  else
    PV_KLAUNCH(&c0->kprof, st, "k_eval_group", 0.0, 0.0,
               (k_eval_group<float, SAMPLE_THREADS><<<G->nblk, SAMPLE_THREADS, G->smem, st>>>(
                   G->d_items, (int)G->ctxs.size(), G->total, (float*)G->d_scr, G->d_iscr, G->sreal,
                   G->sint, (float)JTOL_F32, JAC_MAX_SWEEPS, G->d_flops, G->d_jsw, G->smem)));
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return gfail(G, PEPS_ECUDA, std::string("group_eval: ") + cudaGetErrorString(e));
  for (peps_ctx* c : G->ctxs) c->have_eval = true;
  return PEPS_OK;
}

const char* peps_group_last_error(const peps_group* G) { return G ? G->err.c_str() : ""; }

void peps_group_free(peps_group* G) {
  if (!G) return;
  if (!G->ctxs.empty()) cudaStreamSynchronize(G->ctxs[0]->stream);
  delete G;
}

}  // extern "C"

// ------------------------------------------------------------------ allocation-free evaluation
//
// Work space of peps_eval_batch_noalloc: one file-scope device array, looked up once per
// device.  Layout: [0, 256) counters | toff, ooff tables | float32 theta (FP32 path) |
// per-block real scratch | per-block int scratch.

#include <mutex>

static __device__ __align__(256) unsigned char g_noalloc_scratch[PEPS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {nullptr};
constexpr int NOALLOC_SMEM_MAX = 96 * 1024;

// toff / ooff of the trimmed open-boundary layout, written on the device.
__global__ void k_noalloc_tables(int L1, int L2, int D, long long* toff, long long* ooff) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  toff[0] = ooff[0] = 0;
  for (int i = 0; i < L1 * L2; ++i) {
    int r = i / L2, c = i % L2;
    long long sz = (long long)(c == 0 ? 1 : D) * (c == L2 - 1 ? 1 : D) * (r == 0 ? 1 : D) *
                   (r == L1 - 1 ? 1 : D);
    toff[i + 1] = toff[i] + 4 * sz;
    ooff[i + 1] = ooff[i] + sz;
  }
}

long long align_up(long long x, long long a) { return (x + a - 1) / a * a; }

int noalloc_fail(int code, const std::string& msg) {
  g_noalloc_err = msg;
  return code;
}

// One-time set-up on the current device: device address of the array and the dynamic
// shared-memory attribute of the evaluation kernels.
int noalloc_setup(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(PEPS_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return noalloc_fail(PEPS_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess)
      return noalloc_fail(PEPS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    e = cudaFuncSetAttribute(k_eval<double, double, SAMPLE_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             NOALLOC_SMEM_MAX);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_eval<float, float, SAMPLE_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               NOALLOC_SMEM_MAX);
    if (e != cudaSuccess)
      return noalloc_fail(PEPS_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = (unsigned char*)ptr;
  }
  *out = g_noalloc_addr[dev];
  return PEPS_OK;
}

}  // namespace

extern "C" int peps_eval_batch_noalloc(const peps_params* P, const double* theta,
                                       const uint8_t* S, int nb, double* log_abs, int8_t* sign,
                                       double* e_sys, double* e_anc, void* O, void* stream) {
  g_noalloc_err.clear();
  if (!P || nb < 0 || (nb > 0 && (!theta || !S)))
    return noalloc_fail(PEPS_EINVAL, "eval_batch_noalloc: null argument or nb < 0");
  if (P->L1 < 2 || P->L2 < 2 || P->L1 > MAX_L || P->L2 > MAX_L || P->D < 1 || P->D > 8 ||
      P->chi < 1 || P->chi > 64 || P->model != PEPS_MODEL_J1J2 ||
      (P->precision != PEPS_FP64 && P->precision != PEPS_FP32))
    return noalloc_fail(PEPS_EINVAL, "eval_batch_noalloc: problem outside the library limits");
  unsigned char* base = nullptr;
  int rc = noalloc_setup(&base);
  if (rc != PEPS_OK) return rc;
  if (nb == 0) return PEPS_OK;
  const bool f64 = P->precision == PEPS_FP64;
  const long long real = f64 ? 8 : 4;
  const int N = P->L1 * P->L2;
  long long Np = 0, No = 0;
  for (int i = 0; i < N; ++i) {
    int r = i / P->L2, c = i % P->L2;
    long long sz = (long long)(c == 0 ? 1 : P->D) * (c == P->L2 - 1 ? 1 : P->D) *
                   (r == 0 ? 1 : P->D) * (r == P->L1 - 1 ? 1 : P->D);
    Np += 4 * sz;
    No += sz;
  }
  ScratchDims sd = scratch_dims(P->L1, P->L2, P->D, P->chi);
  const long long sreal = (sd.n_real + 31) & ~31LL, sint = (sd.n_int + 31) & ~31LL;
  const long long off_tab = 256;
  const long long off_thf = align_up(off_tab + 2LL * (N + 1) * 8, 256);
  const long long off_blk = align_up(off_thf + (f64 ? 0 : Np * 4), 256);
  const long long per_block = align_up(sreal * real, 256) + align_up(sint * 4, 256);
  const long long avail = (long long)PEPS_NOALLOC_SCRATCH_BYTES - off_blk;
  if (avail < per_block)
    return noalloc_fail(PEPS_EINVAL,
                        "eval_batch_noalloc: one block needs " + std::to_string(off_blk + per_block) +
                            " bytes of work space, above PEPS_NOALLOC_SCRATCH_BYTES = " +
                            std::to_string((long long)PEPS_NOALLOC_SCRATCH_BYTES));
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long nblk = std::min<long long>(avail / per_block, (long long)sms * 4);
  nblk = std::min<long long>(nblk, nb);
  unsigned char* rbase = base + off_blk;
  int* ibase = (int*)(rbase + nblk * align_up(sreal * real, 256));
  cudaStream_t st = (cudaStream_t)stream;
  long long* toff = (long long*)(base + off_tab);
  long long* ooff = toff + (N + 1);
  // counters start at zero on every call
  cudaError_t e = cudaMemsetAsync(base, 0, 256, st);
  if (e != cudaSuccess) return noalloc_fail(PEPS_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  k_noalloc_tables<<<1, 32, 0, st>>>(P->L1, P->L2, P->D, toff, ooff);
  Geom g;
  g.L1 = P->L1;
  g.L2 = P->L2;
  g.D = P->D;
  g.chi = P->chi;
  g.J1 = P->J1;
  g.J2 = P->J2;
  g.theta_off = toff;
  g.o_off = ooff;
  long long cD = (long long)P->chi * P->D;
  long long need = cD * (cD + 1) * 2 * real;
  int smem = need <= NOALLOC_SMEM_MAX ? (int)need : 0;
  double* flops = (double*)base;
  unsigned long long* jsw = (unsigned long long*)(base + 8);
  long long rstride = align_up(sreal * real, 256) / real;   // elements between blocks
  long long istride = align_up(sint * 4, 256) / 4;
  if (f64) {
    k_eval<double, double, SAMPLE_THREADS><<<(int)nblk, SAMPLE_THREADS, smem, st>>>(
        g, theta, S, nb, (double*)rbase, ibase, rstride, istride, log_abs, sign, e_sys, e_anc,
        (double*)O, No, JTOL_F64, JAC_MAX_SWEEPS, flops, jsw, smem, nullptr, nullptr, 0, 0);
  } else {
    float* thf = (float*)(base + off_thf);
    k_to_real<float><<<grid_for(Np, 256), 256, 0, st>>>(Np, theta, thf);
    k_eval<float, float, SAMPLE_THREADS><<<(int)nblk, SAMPLE_THREADS, smem, st>>>(
        g, thf, S, nb, (float*)rbase, ibase, rstride, istride, log_abs, sign, e_sys, e_anc,
        (float*)O, No, JTOL_F32, JAC_MAX_SWEEPS, flops, jsw, smem, nullptr, nullptr, 0, 0);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(PEPS_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return PEPS_OK;
}

namespace {
void tc_selftest_no_mma(TcSpec& t) { t.no_mma = 1; }
}  // namespace

// Failure-detection self-test of the tensor-core kernels' bounded waits (the paper has no
// counterpart).  A small contraction is launched with its MMAs withheld, so no arrival
// ever reaches the completion barrier: every wait must give up after its time limit, the
// kernel must free its tensor memory and raise its error flag, and a normal contraction on
// the same stream must then succeed and match a host product.
extern "C" int peps_selftest_tc_timeout(void) {
  const int n = 4, M = 128, N = 16, K = 16;
  cudaStream_t st = nullptr;
  if (cudaStreamCreate(&st) != cudaSuccess) return PEPS_ECUDA;
  float *dA = nullptr, *dB = nullptr, *dC = nullptr;
  int* derr = nullptr;
  int rc = PEPS_OK;
  std::vector<float> A((size_t)n * M * K), B((size_t)n * N * K), Cg((size_t)n * M * N);
  for (size_t i = 0; i < A.size(); ++i) A[i] = (float)((i * 37) % 17) / 17.0f - 0.5f;
  for (size_t i = 0; i < B.size(); ++i) B[i] = (float)((i * 11) % 13) / 13.0f - 0.5f;
  auto done = [&](int code) {
    cudaStreamSynchronize(st);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dC);
    cudaFree(derr);
    cudaStreamDestroy(st);
    return code;
  };
  if (cudaMalloc(&dA, A.size() * 4) != cudaSuccess || cudaMalloc(&dB, B.size() * 4) != cudaSuccess ||
      cudaMalloc(&dC, Cg.size() * 4) != cudaSuccess || cudaMalloc(&derr, sizeof(int)) != cudaSuccess)
    return done(PEPS_ENOMEM);
  cudaMemcpy(dA, A.data(), A.size() * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(dB, B.data(), B.size() * 4, cudaMemcpyHostToDevice);
  cudaMemset(derr, 0, sizeof(int));
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  CudaBE<float, float> be;
  be.st = st;
  be.sms = sms;
  be.tc = true;
  be.tc_err = derr;
  Dims d;
  d.set('x', M).set('y', N).set('k', K);
  Spec raw = make_spec("xy", "xk", "yk", d);
  MSpec m = merge_spec(raw);
  for (int pass = 0; pass < 2 && rc == PEPS_OK; ++pass) {
    be.tc_form_override = pass == 0 ? tc_selftest_no_mma : nullptr;
    cudaMemsetAsync(dC, 0, Cg.size() * 4, st);
    be.ein(raw, m, dC, (long long)M * N, batch_op<float>(dA, (long long)M * K),
           batch_op<float>(dB, (long long)N * K), n);
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return done(PEPS_ECUDA);
    int h = -1;
    cudaMemcpy(&h, derr, sizeof(int), cudaMemcpyDeviceToHost);
    cudaMemset(derr, 0, sizeof(int));
    // the withheld MMAs must be noticed (with no MMA issued the grace wait runs out too,
    // so bit 2 is set as well)
    if (pass == 0 && h != 3) rc = PEPS_ESTATE;
    if (pass == 1 && h != 0) rc = PEPS_ETIMEOUT;     // a normal contraction timed out
  }
  if (rc != PEPS_OK) return done(rc);
  cudaMemcpy(Cg.data(), dC, Cg.size() * 4, cudaMemcpyDeviceToHost);
  for (int s = 0; s < n; ++s)
    for (int x = 0; x < M; ++x)
      for (int y = 0; y < N; ++y) {
        double ref = 0, mag = 0;
        for (int k = 0; k < K; ++k) {
          const double p = (double)A[((size_t)s * M + x) * K + k] * B[((size_t)s * N + y) * K + k];
          ref += p;
          mag += std::fabs(p);
        }
        if (std::fabs(Cg[((size_t)s * M + x) * N + y] - ref) > 2e-3 * mag + 1e-6) rc = PEPS_ENOTFINITE;
      }
  return done(rc);
}
