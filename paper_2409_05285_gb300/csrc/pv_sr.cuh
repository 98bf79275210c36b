// Stochastic-reconfiguration kernels (Sec. II, Eqs. 5-7 and 10): sample weights and
// observables, the log-derivative mean and gradient, and the CG solve of
// (G + eps I) x = g with G applied as two passes over the O rows.
//
// O rows are compressed: row i holds, per site j, the slice S_ij of the derivative, so
// the full-space index of column o (site j, offset k) is theta_off[j] + S_ij sz_j + k.
// Every reduction has a fixed order (deterministic results for a fixed launch shape).
#pragma once

#include <cstdint>

namespace pv {

struct SRScalars {
  // sample statistics
  double Ebar;       // sum_i w_i E_i (E = E_sys + E_anc)
  double H1, H2;     // <H>, <H^2> of Eq. 11 (symmetrised over the two layers)
  double M2;         // <Mz^2>
  double diag;       // fraction of diagonal samples
  double Eerr;       // standard error of <H>
  // CG state
  double rr, gnorm, pq, obp, sumy;
  int iters, done, maxit, pad;
  double tol, eps;
};

constexpr int SR_THREADS = 256;
constexpr int SR_WEIGHT_THREADS = 1024;
constexpr int OTV_CHUNK = 128;   // samples per partial sum of the O^T y pass

template <typename T>
__device__ __forceinline__ T blk_sum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = 0;
  int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) s += red[i];
  __syncthreads();
  return s;
}

// Log of the unnormalised weight of sample i: p = 2 (samples of |rho|^2) 0; p = 1 (samples
// of |rho|, Eq. A1) log|rho|; p = 0 (direct draws of probability q, App. A Eq. A7 with
// r_4 = p_0 / q) 2 log|rho| - log q.
__device__ __forceinline__ double sr_log_weight(int p, const double* log_abs, const double* logq,
                                                int i) {
  return p == 2 ? 0.0 : p == 1 ? log_abs[i] : 2.0 * log_abs[i] - logq[i];
}

// Weights and sample statistics (one block): w_i = exp(lw_i) / sum_j exp(lw_j) with lw of
// sr_log_weight.  Observables: <H> = 1/2 sum w (Es + Ea), <H^2> = 1/2 sum w (Es^2 + Ea^2),
// <Mz^2> = 1/2 sum w (M(s)^2 + M(s')^2).
__global__ void k_sr_weights(int n, int N, int p, const double* __restrict__ log_abs,
                             const double* __restrict__ logq,
                             const double* __restrict__ es, const double* __restrict__ ea,
                             const uint8_t* __restrict__ S, double* __restrict__ w,
                             double* __restrict__ E, SRScalars* sc) {
  __shared__ double red[32];
  double mx = -INFINITY;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, sr_log_weight(p, log_abs, logq, i));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ double redm[32];
  if ((threadIdx.x & 31) == 0) redm[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = redm[0];
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) mx = fmax(mx, redm[i]);
  double zs = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    zs += (p == 2) ? 1.0 : exp(sr_log_weight(p, log_abs, logq, i) - mx);
  double Z = blk_sum(zs, red);
  double e1 = 0, h1 = 0, h2 = 0, m2 = 0, dg = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double wi = ((p == 2) ? 1.0 : exp(sr_log_weight(p, log_abs, logq, i) - mx)) / Z;
    w[i] = wi;
    double a = es[i], b = ea[i];
    E[i] = a + b;
    e1 += wi * (a + b);
    h1 += wi * 0.5 * (a + b);
    h2 += wi * 0.5 * (a * a + b * b);
    int ms = 0, ma = 0, dd = 1;
    for (int j = 0; j < N; ++j) {
      int s = S[(long long)i * N + j];
      ms += (s >> 1) ? -1 : 1;
      ma += (s & 1) ? -1 : 1;
      dd &= ((s >> 1) == (s & 1));
    }
    m2 += wi * 0.5 * (0.25 * ms * ms + 0.25 * ma * ma);
    dg += dd;
  }
  e1 = blk_sum(e1, red);
  h1 = blk_sum(h1, red);
  h2 = blk_sum(h2, red);
  m2 = blk_sum(m2, red);
  dg = blk_sum(dg, red);
  double ve = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double d = 0.5 * (es[i] + ea[i]) - h1;
    ve += w[i] * w[i] * d * d;
  }
  ve = blk_sum(ve, red);
  if (threadIdx.x == 0) {
    sc->Ebar = e1;
    sc->H1 = h1;
    sc->H2 = h2;
    sc->M2 = m2;
    sc->diag = dg / n;
    sc->Eerr = sqrt(ve);
  }
}

// Stage 1 of a segmented column sum over samples: for each column o of the O rows and
// each chunk of OTV_CHUNK samples, acc[S_ij] += c_i O[i][o] for the four values of S_ij,
// written to part[chunk][theta index].  Two coefficient vectors at once (c1 = y or w,
// c2 = w (E - Ebar) or unused).
template <typename OT, bool TWO>
__global__ void k_colsum1(int n, int N, long long No, const OT* __restrict__ O,
                          const uint8_t* __restrict__ S, const int* __restrict__ o2site,
                          const long long* __restrict__ toff, const long long* __restrict__ ooff,
                          const double* __restrict__ c1, const double* __restrict__ c2,
                          const double* __restrict__ shift, double* __restrict__ part1,
                          double* __restrict__ part2, long long Np, const int* done) {
  if (done && *done) return;
  const double Ebar_shift = TWO ? *shift : 0.0;
  long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= No) return;
  int ch = blockIdx.y;
  int i0 = ch * OTV_CHUNK, i1 = min(n, i0 + OTV_CHUNK);
  int j = o2site[o];
  long long k = o - ooff[j];
  long long sz = (ooff[j + 1] - ooff[j]);
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0;
  for (int i = i0; i < i1; ++i) {
    double v = (double)O[(long long)i * No + o];
    int s = S[(long long)i * N + j];
    double x = c1[i] * v;
    double y = TWO ? c1[i] * (c2[i] - Ebar_shift) * v : 0.0;
    if (s == 0) { a0 += x; if (TWO) b0 += y; }
    else if (s == 1) { a1 += x; if (TWO) b1 += y; }
    else if (s == 2) { a2 += x; if (TWO) b2 += y; }
    else { a3 += x; if (TWO) b3 += y; }
  }
  long long t = toff[j] + k;
  double* p1 = part1 + (long long)ch * Np;
  p1[t] = a0;
  p1[t + sz] = a1;
  p1[t + 2 * sz] = a2;
  p1[t + 3 * sz] = a3;
  if (TWO) {
    double* p2 = part2 + (long long)ch * Np;
    p2[t] = b0;
    p2[t + sz] = b1;
    p2[t + 2 * sz] = b2;
    p2[t + 3 * sz] = b3;
  }
}

// Float rows: each float32 entry is widened and multiplied and summed in float64.
template <bool TWO>
__global__ void k_colsum1_f32(int n, int N, long long No, const float* __restrict__ O,
                              const uint8_t* __restrict__ S, const int* __restrict__ o2site,
                              const long long* __restrict__ toff,
                              const long long* __restrict__ ooff, const double* __restrict__ c1,
                              const double* __restrict__ c2, const double* __restrict__ shift,
                              double* __restrict__ part1, double* __restrict__ part2,
                              long long Np, const int* done) {
  if (done && *done) return;
  const double Ebar_shift = TWO ? *shift : 0.0;
  long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= No) return;
  int ch = blockIdx.y;
  int i0 = ch * OTV_CHUNK, i1 = min(n, i0 + OTV_CHUNK);
  int j = o2site[o];
  long long k = o - ooff[j];
  long long sz = (ooff[j + 1] - ooff[j]);
  double a[4] = {0, 0, 0, 0}, b[4] = {0, 0, 0, 0};
  for (int i = i0; i < i1; ++i) {
    const double v = (double)O[(long long)i * No + o];
    const int s = S[(long long)i * N + j];
    const double x = c1[i] * v;
    const double y = TWO ? c1[i] * (c2[i] - Ebar_shift) * v : 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (s == q) {
        a[q] += x;
        if (TWO) b[q] += y;
      }
    }
  }
  long long t = toff[j] + k;
  double* p1 = part1 + (long long)ch * Np;
#pragma unroll
  for (int q = 0; q < 4; ++q) p1[t + q * sz] = a[q];
  if (TWO) {
    double* p2 = part2 + (long long)ch * Np;
#pragma unroll
    for (int q = 0; q < 4; ++q) p2[t + q * sz] = b[q];
  }
}

// Four consecutive O entries as float64: a 16-byte float32 load widened (exactly), or the
// float64 copy of the rows (two 16-byte loads, no conversion in the pass).
struct OV4 {
  double x, y, z, w;
};
__device__ __forceinline__ OV4 ov_ld4(const float* p) {
  const float4 f = __ldg((const float4*)p);
  return OV4{(double)f.x, (double)f.y, (double)f.z, (double)f.w};
}
__device__ __forceinline__ OV4 ov_ld4(const double* p) {
  const double2 a = __ldg((const double2*)p), b = __ldg((const double2*)p + 1);
  return OV4{a.x, a.y, b.x, b.y};
}

// float32 rows widened into a float64 copy (one pass per SR step; the CG passes then read
// the copy and spend no float64 issue on conversions)
__global__ void k_widen_o(long long n4, const float* __restrict__ O, double* __restrict__ O64) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n4;
       e += (long long)gridDim.x * blockDim.x) {
    const float4 f = __ldg((const float4*)O + e);
    ((double2*)O64)[2 * e] = make_double2(f.x, f.y);
    ((double2*)O64)[2 * e + 1] = make_double2(f.z, f.w);
  }
}

// Float rows, 16-byte vectors: every site slice holds a multiple of four entries, so each
// thread takes four consecutive columns of one site; four rows are loaded before they are
// accumulated.  Products and sums in float64, one FMA per entry: the per-state sums live in
// shared memory, [sum][state][column][thread], and each row adds into the four sums of its
// state (float64 issue, about 1/60 of float32 on GB300, bounds this pass).
template <bool TWO, typename OT = float>
__global__ void __launch_bounds__(SR_THREADS) k_colsum1_f32v(
    int n, int N, long long No, const OT* __restrict__ O, const uint8_t* __restrict__ S,
    const int* __restrict__ o2site, const long long* __restrict__ toff,
    const long long* __restrict__ ooff, const double* __restrict__ c1,
    const double* __restrict__ c2, const double* __restrict__ shift, double* __restrict__ part1,
    double* __restrict__ part2, long long Np, const int* done) {
  if (done && *done) return;
  extern __shared__ double cs_acc[];   // [TWO ? 2 : 1][4 states][4 columns][SR_THREADS]
  __shared__ double cx[OTV_CHUNK], cy[OTV_CHUNK];
  const int ch = blockIdx.y, tid = threadIdx.x;
  const int i0 = ch * OTV_CHUNK, i1 = min(n, i0 + OTV_CHUNK);
  const double Ebar_shift = TWO ? *shift : 0.0;
  for (int i = tid; i < i1 - i0; i += blockDim.x) {
    cx[i] = c1[i0 + i];
    cy[i] = TWO ? c1[i0 + i] * (c2[i0 + i] - Ebar_shift) : 0.0;
  }
  for (int e = tid; e < (TWO ? 32 : 16) * SR_THREADS; e += SR_THREADS) cs_acc[e] = 0.0;
  __syncthreads();
  const long long o = 4 * ((long long)blockIdx.x * blockDim.x + tid);
  if (o >= No) return;
  const int j = o2site[o];
  const long long k = o - ooff[j], sz = ooff[j + 1] - ooff[j];
  double* A = cs_acc + tid;                       // A[(q * 4 + c) * SR_THREADS]
  double* B = cs_acc + 16 * SR_THREADS + tid;
  int i = i0;
  for (; i + 4 <= i1; i += 4) {
    OV4 v[4];
    int st[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      v[u] = ov_ld4(O + (long long)(i + u) * No + o);
      st[u] = S[(long long)(i + u) * N + j];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      double* a = A + st[u] * 4 * SR_THREADS;
      const double x = cx[i + u - i0];
      a[0] += x * v[u].x;
      a[SR_THREADS] += x * v[u].y;
      a[2 * SR_THREADS] += x * v[u].z;
      a[3 * SR_THREADS] += x * v[u].w;
      if (TWO) {
        double* b = B + st[u] * 4 * SR_THREADS;
        const double y = cy[i + u - i0];
        b[0] += y * v[u].x;
        b[SR_THREADS] += y * v[u].y;
        b[2 * SR_THREADS] += y * v[u].z;
        b[3 * SR_THREADS] += y * v[u].w;
      }
    }
  }
  for (; i < i1; ++i) {
    const OV4 v = ov_ld4(O + (long long)i * No + o);
    const int s0 = S[(long long)i * N + j];
    double* a = A + s0 * 4 * SR_THREADS;
    const double x = cx[i - i0];
    a[0] += x * v.x;
    a[SR_THREADS] += x * v.y;
    a[2 * SR_THREADS] += x * v.z;
    a[3 * SR_THREADS] += x * v.w;
    if (TWO) {
      double* b = B + s0 * 4 * SR_THREADS;
      const double y = cy[i - i0];
      b[0] += y * v.x;
      b[SR_THREADS] += y * v.y;
      b[2 * SR_THREADS] += y * v.z;
      b[3 * SR_THREADS] += y * v.w;
    }
  }
  const long long t = toff[j] + k;
  double* p1 = part1 + (long long)ch * Np;
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int c = 0; c < 4; ++c) p1[t + q * sz + c] = A[(q * 4 + c) * SR_THREADS];
  if (TWO) {
    double* p2 = part2 + (long long)ch * Np;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < 4; ++c) p2[t + q * sz + c] = B[(q * 4 + c) * SR_THREADS];
  }
}

// Stage 2 for the mean and gradient: obar = sum_ch part1, g = sum_ch part2.
__global__ void k_colsum2_grad(long long Np, int nch, const double* __restrict__ part1,
                               const double* __restrict__ part2, double* __restrict__ obar,
                               double* __restrict__ g) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Np) return;
  double a = 0, b = 0;
  for (int c = 0; c < nch; ++c) {
    a += part1[(long long)c * Np + t];
    b += part2[(long long)c * Np + t];
  }
  obar[t] = a;
  g[t] = b;
}

// Block-partial dot products of length-Np vectors: part[block] = sum over the block.
__global__ void k_dot_part(long long Np, const double* __restrict__ a,
                           const double* __restrict__ b, double* __restrict__ part,
                           const SRScalars* sc) {
  __shared__ double red[32];
  if (sc && sc->done) return;
  double s = 0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < Np;
       t += (long long)gridDim.x * blockDim.x)
    s += a[t] * b[t];
  s = blk_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__device__ __forceinline__ double sum_parts(const double* part, int n) {
  double s = 0;
  for (int i = 0; i < n; ++i) s += part[i];
  return s;
}

// The same sum formed by the whole block (strided partials, then a tree): every thread of
// the block must call it; all blocks get the same value.
__device__ __forceinline__ double blk_sum_parts(const double* part, int n, double* red) {
  double s = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  return blk_sum(s, red);
}

// CG set-up: x = 0, r = p = g, rr = g.g, gnorm, done flag.
__global__ void k_cg_init(long long Np, const double* __restrict__ g, double* __restrict__ x,
                          double* __restrict__ r, double* __restrict__ p,
                          int ndp, const double* __restrict__ dpart, SRScalars* sc, int maxit,
                          double tol, double eps) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < Np;
       t += (long long)gridDim.x * blockDim.x) {
    x[t] = 0;
    r[t] = g[t];
    p[t] = g[t];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double rr = sum_parts(dpart, ndp);
    sc->rr = rr;
    sc->gnorm = sqrt(rr);
    sc->iters = 0;
    sc->maxit = maxit;
    sc->tol = tol;
    sc->eps = eps;
    sc->done = (maxit <= 0 || !(sqrt(rr) > tol * sqrt(rr))) ? 1 : 0;
  }
}

// y_i = w_i [ (O_i . p) - obar . p ], one warp per sample; per-block partials of sum y.
template <typename OT>
__global__ void k_ov(int n, int N, long long No, const OT* __restrict__ O,
                     const uint8_t* __restrict__ S, const long long* __restrict__ toff,
                     const long long* __restrict__ ooff, const double* __restrict__ p,
                     const double* __restrict__ w,
                     double* __restrict__ y, double* __restrict__ ypart, int ndp,
                     const double* __restrict__ dpart, const SRScalars* sc) {
  __shared__ double red[32];
  if (sc->done) return;
  double obp = blk_sum_parts(dpart, ndp, red);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int i = blockIdx.x * (blockDim.x >> 5) + warp;
  double yi = 0;
  if (i < n) {
    const OT* row = O + (long long)i * No;
    double acc = 0;
    for (int j = 0; j < N; ++j) {
      int s = S[(long long)i * N + j];
      long long o0 = ooff[j], sz = ooff[j + 1] - o0;
      long long t0 = toff[j] + (long long)s * sz;
      for (long long k = lane; k < sz; k += 32) acc += (double)row[o0 + k] * p[t0 + k];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    yi = w[i] * (acc - obp);
    if (lane == 0) y[i] = yi;
  }
  double contrib = (lane == 0) ? yi : 0.0;
  double s = blk_sum(contrib, red);
  if (threadIdx.x == 0) ypart[blockIdx.x] = s;
}

// Float rows, 16-byte vectors (site slices of multiples of four entries): y_i = w_i (O_i.p - obar.p),
// every entry widened to float64.  One warp per sample; the lanes walk the row's 16-byte column
// groups directly (site and state looked up per group), four groups in flight per lane.
template <typename OT = float>
__global__ void __launch_bounds__(SR_THREADS) k_ov_f32v(
    int n, int N, long long No, const OT* __restrict__ O, const uint8_t* __restrict__ S,
    const int* __restrict__ o2site, const long long* __restrict__ toff,
    const long long* __restrict__ ooff, const double* __restrict__ p, const double* __restrict__ w,
    double* __restrict__ y, double* __restrict__ ypart, int ndp, const double* __restrict__ dpart,
    const SRScalars* sc) {
  __shared__ double red[32];
  if (sc->done) return;
  double obp = blk_sum_parts(dpart, ndp, red);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int i = blockIdx.x * (blockDim.x >> 5) + warp;
  double yi = 0;
  if (i < n) {
    const OT* row = O + (long long)i * No;
    const uint8_t* Si = S + (long long)i * N;
    const long long nq = No >> 2;
    double acc = 0.0;
    long long q = lane;
    for (; q + 96 < nq; q += 128) {
      OV4 r[4];
      const double* pp[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long o = (q + 32 * u) << 2;
        const int j = o2site[o];
        const long long o0 = ooff[j];
        pp[u] = p + toff[j] + (long long)Si[j] * (ooff[j + 1] - o0) + (o - o0);
        r[u] = ov_ld4(row + ((q + 32 * u) << 2));
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double2 a = __ldg((const double2*)pp[u]), b = __ldg((const double2*)pp[u] + 1);
        acc += r[u].x * a.x + r[u].y * a.y + r[u].z * b.x + r[u].w * b.y;
      }
    }
    for (; q < nq; q += 32) {
      const long long o = q << 2;
      const int j = o2site[o];
      const long long o0 = ooff[j];
      const double* pp = p + toff[j] + (long long)Si[j] * (ooff[j + 1] - o0) + (o - o0);
      const OV4 r = ov_ld4(row + (q << 2));
      const double2 a = __ldg((const double2*)pp), b = __ldg((const double2*)pp + 1);
      acc += r.x * a.x + r.y * a.y + r.z * b.x + r.w * b.y;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    yi = w[i] * (acc - obp);
    if (lane == 0) y[i] = yi;
  }
  double contrib = (lane == 0) ? yi : 0.0;
  double sm = blk_sum(contrib, red);
  if (threadIdx.x == 0) ypart[blockIdx.x] = sm;
}

// q = sum_ch part - (sum y) obar + eps p ; block partials of p.q.
__global__ void k_otv2(long long Np, int nch, const double* __restrict__ part,
                       const double* __restrict__ obar, const double* __restrict__ p,
                       double* __restrict__ q, int nyp, const double* __restrict__ ypart,
                       double* __restrict__ pqpart, SRScalars* sc) {
  __shared__ double red[32];
  if (sc->done) return;
  double sumy = blk_sum_parts(ypart, nyp, red);
  double eps = sc->eps;
  double s = 0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < Np;
       t += (long long)gridDim.x * blockDim.x) {
    // eight chunk partials in flight at a time (fixed order: the sum is reproducible)
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int c = 0;
    for (; c + 8 <= nch; c += 8)
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] += part[(long long)(c + u) * Np + t];
    for (; c < nch; ++c) acc[0] += part[(long long)c * Np + t];
    double a = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
    double qt = a - sumy * obar[t] + eps * p[t];
    q[t] = qt;
    s += p[t] * qt;
  }
  s = blk_sum(s, red);
  if (threadIdx.x == 0) pqpart[blockIdx.x] = s;
}

// alpha = rr / p.q ; x += alpha p ; r -= alpha q ; block partials of r.r
__global__ void k_cg_a(long long Np, double* __restrict__ x, double* __restrict__ r,
                       const double* __restrict__ p, const double* __restrict__ q, int npq,
                       const double* __restrict__ pqpart, double* __restrict__ rrpart,
                       SRScalars* sc) {
  __shared__ double red[32];
  if (sc->done) return;
  double alpha = sc->rr / blk_sum_parts(pqpart, npq, red);
  double s = 0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < Np;
       t += (long long)gridDim.x * blockDim.x) {
    x[t] += alpha * p[t];
    double rt = r[t] - alpha * q[t];
    r[t] = rt;
    s += rt * rt;
  }
  s = blk_sum(s, red);
  if (threadIdx.x == 0) rrpart[blockIdx.x] = s;
}

// beta = rr_new / rr ; p = r + beta p ; block partials of obar.p for the next pass.
// The last block to finish updates the scalars (iteration count, convergence flag).
__global__ void k_cg_b(long long Np, const double* __restrict__ r, double* __restrict__ p,
                       const double* __restrict__ obar, int nrr,
                       const double* __restrict__ rrpart, double* __restrict__ obpart,
                       SRScalars* sc) {
  __shared__ double red[32];
  if (sc->done) return;
  double rr_new = blk_sum_parts(rrpart, nrr, red);
  double beta = rr_new / sc->rr;
  double s = 0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < Np;
       t += (long long)gridDim.x * blockDim.x) {
    double pt = r[t] + beta * p[t];
    p[t] = pt;
    s += obar[t] * pt;
  }
  s = blk_sum(s, red);
  if (threadIdx.x == 0) obpart[blockIdx.x] = s;
}

// Scalars after an iteration (one thread): rr <- rr_new, iteration count, stop test.
__global__ void k_cg_scalars(int nrr, const double* __restrict__ rrpart, SRScalars* sc) {
  if (sc->done) return;
  double rr_new = sum_parts(rrpart, nrr);
  sc->rr = rr_new;
  sc->iters += 1;
  if (sc->iters >= sc->maxit || !(sqrt(rr_new) > sc->tol * sc->gnorm)) sc->done = 1;
}

// ---------------------------------------------------------------- fused CG product
//
// q = (G + eps) p = sum_i y_i O_i - (sum_i y_i) obar + eps p with y_i = w_i (O_i.p - obar.p)
// (Eq. 10, two passes over the O rows), formed with one read of O from DRAM.  Every block
// owns a fixed slice of the compressed columns (and the four q entries of each) for the
// whole product.  The samples are taken in chunks of R = gridDim.x * rpb rows, small enough
// to stay in L2: in phase A every block forms the complete dot products of its own rpb rows
// of the chunk; after a grid barrier every block, in phase B, adds y_i O_i[o] over the
// chunk's rows for its own columns o, rows that the chunk's phase A has just brought into
// L2.  Products and sums are float64 (float32 entries are widened); every sum has a fixed
// order, so the result does not depend on timing.  The kernel must run with every block
// resident (cooperative launch); its barrier waits are bounded (GV_WAIT_NS), and a wait that
// runs out raises *err and makes every block return.

constexpr int GV_THREADS = 1024;
constexpr unsigned long long GV_WAIT_NS = 1000000000ull;

__device__ __forceinline__ unsigned long long gv_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier over the resident blocks: bar[0] counts arrivals, bar[1] is the generation
// (both zero at launch).  Returns false when a wait ran out here or in another block.
__device__ __forceinline__ bool gv_barrier(unsigned* bar, unsigned& gen, int* err, int* ok_sh) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g = gen;
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicExch(bar + 1, g + 1);
    } else {
      volatile unsigned* vg = bar + 1;
      volatile int* ve = err;
      const unsigned long long t0 = gv_now();
      while (*vg == g) {
        if (*ve) { ok = 0; break; }
        if (gv_now() - t0 > GV_WAIT_NS) {
          atomicOr(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    gen = g + 1;
    *ok_sh = ok;
  }
  __syncthreads();
  return *ok_sh != 0;
}

// Entry of p / q (full parameter space) of compressed column o for state s.
__device__ __forceinline__ long long gv_tidx(long long o, int s, const int* __restrict__ o2site,
                                             const long long* __restrict__ toff,
                                             const long long* __restrict__ ooff, int& j) {
  j = o2site[o];
  const long long o0 = ooff[j];
  return toff[j] + (long long)s * (ooff[j + 1] - o0) + (o - o0);
}

template <typename OT, bool VEC>
__global__ void __launch_bounds__(GV_THREADS) k_gv(
    int n, int N, long long No, const OT* __restrict__ O, const uint8_t* __restrict__ S,
    const int* __restrict__ o2site, const long long* __restrict__ toff,
    const long long* __restrict__ ooff, const double* __restrict__ p,
    const double* __restrict__ obar, const double* __restrict__ w, int ndp,
    const double* __restrict__ dpart, double* __restrict__ y, double* __restrict__ q,
    double* __restrict__ pqpart, int rpb, unsigned* bar, int* err, const SRScalars* sc) {
  __shared__ double red[32];
  __shared__ int ok_sh;
  extern __shared__ double gacc[];   // phase B: [4][blockDim] partial sums of the row groups
  if (sc->done) return;
  const int tid = threadIdx.x, nt = blockDim.x, G = gridDim.x, b = blockIdx.x;
  const double obp = blk_sum_parts(dpart, ndp, red);
  const double eps = sc->eps;
  // this block's columns [c0, c1)
  const long long segw = (No + G - 1) / G;
  const long long c0 = min(No, (long long)b * segw), c1 = min(No, c0 + segw);
  const int ncol = (int)(c1 - c0);
  // phase B layout: thread (col, rg); ncolp column slots of nrg row groups
  const int nrg = ncol > 0 ? max(1, nt / ncol) : 1;
  const int ncolp = ncol > 0 ? (nt / nrg) : 0;
  const int mycol = tid % max(1, ncolp), rg = tid / max(1, ncolp);
  const bool bthread = ncol > 0 && rg < nrg;
  // q for this block's columns starts at zero
  for (long long o = c0 + tid; o < c1; o += nt) {
    int j;
    const long long t = gv_tidx(o, 0, o2site, toff, ooff, j);
    const long long sz = ooff[j + 1] - ooff[j];
    q[t] = 0.0;
    q[t + sz] = 0.0;
    q[t + 2 * sz] = 0.0;
    q[t + 3 * sz] = 0.0;
  }
  const long long R = (long long)G * rpb;
  unsigned gen = 0;
  for (long long cbase = 0; cbase < n; cbase += R) {
    // ---- phase A: dot products of this block's rows of the chunk
    for (int r = 0; r < rpb; ++r) {
      const long long i = cbase + (long long)b * rpb + r;
      if (i >= n) break;
      const OT* row = O + i * No;
      const uint8_t* Si = S + i * N;
      double acc = 0.0;
      if (VEC) {   // four columns of one site per thread (site slices of multiples of four)
        for (long long o = 4LL * tid; o < No; o += 4LL * nt) {
          int j;
          const long long t = gv_tidx(o, 0, o2site, toff, ooff, j);
          const long long sz = ooff[j + 1] - ooff[j];
          const double* pp = p + t + (long long)Si[j] * sz;
          if (sizeof(OT) == 4) {
            const float4 v = __ldg((const float4*)(row + o));
            acc += (double)v.x * pp[0] + (double)v.y * pp[1] + (double)v.z * pp[2] + (double)v.w * pp[3];
          } else {
            const double2 v0 = __ldg((const double2*)(row + o)), v1 = __ldg((const double2*)(row + o + 2));
            acc += v0.x * pp[0] + v0.y * pp[1] + v1.x * pp[2] + v1.y * pp[3];
          }
        }
      } else {
        for (long long o = tid; o < No; o += nt) {
          int j;
          const long long t = gv_tidx(o, 0, o2site, toff, ooff, j);
          const long long sz = ooff[j + 1] - ooff[j];
          acc += (double)row[o] * p[t + (long long)Si[j] * sz];
        }
      }
      acc = blk_sum(acc, red);
      if (tid == 0) y[i] = w[i] * (acc - obp);
    }
    if (!gv_barrier(bar, gen, err, &ok_sh)) return;
    // ---- phase B: this block's columns, summed over the chunk's rows
    const long long cend = min((long long)n, cbase + R);
    if (bthread) {
      for (int col = mycol; col < ncol; col += ncolp) {
        const long long o = c0 + col;
        int j;
        const long long t = gv_tidx(o, 0, o2site, toff, ooff, j);
        const long long sz = ooff[j + 1] - ooff[j];
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        long long i = cbase + rg;
        // eight rows' loads in flight before they are accumulated (the rows come from L2)
        for (; i + 7LL * nrg < cend; i += 8LL * nrg) {
          OT v[8];
          double yy[8];
          int st[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const long long iu = i + (long long)u * nrg;
            v[u] = O[iu * No + o];
            yy[u] = __ldcg(y + iu);
            st[u] = S[iu * N + j];
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {   // one FMA per entry: the state selects the sum
            const double vv = (double)v[u];
            if (st[u] == 0) a0 += vv * yy[u];
            else if (st[u] == 1) a1 += vv * yy[u];
            else if (st[u] == 2) a2 += vv * yy[u];
            else a3 += vv * yy[u];
          }
        }
        for (; i < cend; i += nrg) {
          const double x = (double)O[i * No + o] * __ldcg(y + i);
          const int st = S[i * N + j];
          a0 += st == 0 ? x : 0.0;
          a1 += st == 1 ? x : 0.0;
          a2 += st == 2 ? x : 0.0;
          a3 += st == 3 ? x : 0.0;
        }
        if (nrg == 1) {
          q[t] += a0;
          q[t + sz] += a1;
          q[t + 2 * sz] += a2;
          q[t + 3 * sz] += a3;
        } else {
          // row groups of this column meet in shared memory (this column slot's entries only)
          gacc[0 * nt + tid] = a0;
          gacc[1 * nt + tid] = a1;
          gacc[2 * nt + tid] = a2;
          gacc[3 * nt + tid] = a3;
        }
        if (nrg > 1) break;   // with several row groups every slot holds exactly one column
      }
    }
    if (nrg > 1) {
      __syncthreads();
      if (bthread && rg == 0 && mycol < ncol) {
        const long long o = c0 + mycol;
        int j;
        const long long t = gv_tidx(o, 0, o2site, toff, ooff, j);
        const long long sz = ooff[j + 1] - ooff[j];
        double a[4] = {0, 0, 0, 0};
        for (int g2 = 0; g2 < nrg; ++g2)
#pragma unroll
          for (int s4 = 0; s4 < 4; ++s4) a[s4] += gacc[s4 * nt + g2 * ncolp + mycol];
        q[t] += a[0];
        q[t + sz] += a[1];
        q[t + 2 * sz] += a[2];
        q[t + 3 * sz] += a[3];
      }
      __syncthreads();
    }
  }
  // sum_i y_i in one fixed order (the same value in every block)
  double sy = 0.0;
  for (int i = tid; i < n; i += nt) sy += __ldcg(y + i);
  sy = blk_sum(sy, red);
  // q = sum y O - (sum y) obar + eps p on this block's entries; partial p.q
  double pq = 0.0;
  for (long long o = c0 + tid; o < c1; o += nt) {
    int j;
    const long long t = gv_tidx(o, 0, o2site, toff, ooff, j);
    const long long sz = ooff[j + 1] - ooff[j];
#pragma unroll
    for (int s4 = 0; s4 < 4; ++s4) {
      const long long ts = t + s4 * sz;
      const double qt = q[ts] - sy * obar[ts] + eps * p[ts];
      q[ts] = qt;
      pq += p[ts] * qt;
    }
  }
  pq = blk_sum(pq, red);
  if (tid == 0) pqpart[b] = pq;
}

// theta -= tau x (and the float32 copy).
__global__ void k_update(long long Np, double tau, const double* __restrict__ x,
                         double* __restrict__ theta, float* __restrict__ theta_f) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < Np;
       t += (long long)gridDim.x * blockDim.x) {
    double v = theta[t] - tau * x[t];
    theta[t] = v;
    if (theta_f) theta_f[t] = (float)v;
  }
}

}  // namespace pv
