// CTA-cooperative building blocks for the per-sample PEPS contraction.
//
// Every routine here is executed by all threads of one thread block on data in global
// memory (the block's scratch) and ends with the block synchronised.  The same source
// compiles for the host with a single "thread" (used by offline checks of the index
// arithmetic); the device build is the product path.
#pragma once

#include <cstdint>
#include <cmath>

#if defined(__CUDACC__)
#define PV_HD __host__ __device__ __forceinline__
#define PV_HDN __host__ __device__ __noinline__
#else
#define PV_HD inline
#define PV_HDN inline
#endif

#if defined(__CUDA_ARCH__)
#define PV_TID ((int)threadIdx.x)
#define PV_NTHR ((int)blockDim.x)
#define PV_LANE ((int)(threadIdx.x & 31u))
#define PV_WARP ((int)(threadIdx.x >> 5))
#define PV_NWARP ((int)(blockDim.x >> 5))
#define PV_WSIZE 32
#define PV_SYNC() __syncthreads()
#else
#define PV_TID 0
#define PV_NTHR 1
#define PV_LANE 0
#define PV_WARP 0
#define PV_NWARP 1
#define PV_WSIZE 1
#define PV_SYNC() ((void)0)
#endif

namespace pv {

template <typename T>
PV_HD T warp_sum(T v) {
#if defined(__CUDA_ARCH__)
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
#endif
  return v;
}

template <typename T>
PV_HD T warp_max(T v) {
#if defined(__CUDA_ARCH__)
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
#endif
  return v;
}

// Block-wide sum; every thread gets the same value (fixed summation order).  `red` is a
// shared array of at least PV_NWARP entries.
template <typename T>
PV_HD T cta_sum(T v, T* red) {
#if defined(__CUDA_ARCH__)
  v = warp_sum(v);
  __syncthreads();
  if (PV_LANE == 0) red[PV_WARP] = v;
  __syncthreads();
  T s = 0;
  for (int i = 0; i < PV_NWARP; ++i) s += red[i];
  return s;
#else
  (void)red;
  return v;
#endif
}

template <typename T>
PV_HD T cta_max(T v, T* red) {
#if defined(__CUDA_ARCH__)
  v = warp_max(v);
  __syncthreads();
  if (PV_LANE == 0) red[PV_WARP] = v;
  __syncthreads();
  T s = red[0];
  for (int i = 1; i < PV_NWARP; ++i) s = red[i] > s ? red[i] : s;
  return s;
#else
  (void)red;
  return v;
#endif
}

// ---------------------------------------------------------------------------------------
// A small einsum: out[o...] = sum_k A[..] * B[..] with single-letter labels.  Operands
// are dense row-major in their label order; `dims` maps 'a'..'z' to extents.

struct Dims {
  int v[26];
  PV_HD Dims() {
    for (int i = 0; i < 26; ++i) v[i] = 1;
  }
  PV_HD Dims& set(char c, int d) {
    v[c - 'a'] = d;
    return *this;
  }
  PV_HD int operator[](char c) const { return v[c - 'a']; }
};

struct Spec {
  int no, nk;
  int os[6], ks[3];
  long long ao[6], bo[6], ak[3], bk[3];
  long long total;   // number of output elements
  long long kprod;   // contraction length
};

PV_HD int pv_strlen(const char* s) {
  int n = 0;
  while (s[n]) ++n;
  return n;
}

PV_HD bool pv_has(const char* s, char c) {
  for (int i = 0; s[i]; ++i)
    if (s[i] == c) return true;
  return false;
}

PV_HD long long pv_stride(const char* s, char c, const Dims& d) {
  int n = pv_strlen(s);
  long long st = 1;
  for (int i = n - 1; i >= 0; --i) {
    if (s[i] == c) return st;
    st *= d[s[i]];
  }
  return 0;
}

PV_HD Spec make_spec(const char* out, const char* a, const char* b, const Dims& d) {
  Spec s;
  s.no = pv_strlen(out);
  s.total = 1;
  for (int i = 0; i < s.no; ++i) {
    char c = out[i];
    s.os[i] = d[c];
    s.ao[i] = pv_has(a, c) ? pv_stride(a, c, d) : 0;
    s.bo[i] = pv_has(b, c) ? pv_stride(b, c, d) : 0;
    s.total *= s.os[i];
  }
  s.nk = 0;
  s.kprod = 1;
  for (int i = 0; a[i]; ++i) {
    char c = a[i];
    if (pv_has(out, c)) continue;
    s.ks[s.nk] = d[c];
    s.ak[s.nk] = pv_stride(a, c, d);
    s.bk[s.nk] = pv_stride(b, c, d);
    s.kprod *= d[c];
    ++s.nk;
  }
  for (int i = s.nk; i < 3; ++i) {
    s.ks[i] = 1;
    s.ak[i] = s.bk[i] = 0;
  }
  return s;
}

// Executes the contraction with the whole block (grid-stride over output elements).
// Adjacent output (and contraction) dimensions whose strides chain in both operands are
// merged first; the index arithmetic is 32-bit and the contraction loop keeps four
// independent accumulators.
template <typename T, typename TA, typename TB>
PV_HDN void contract(T* out, const TA* A, const TB* B, const Spec& s) {
  int no = 0, os[6], ao[6], bo[6];
  for (int d = 0; d < s.no; ++d) {
    int n = s.os[d], a = (int)s.ao[d], b = (int)s.bo[d];
    if (n == 1) continue;
    if (no > 0 && ao[no - 1] == a * n && bo[no - 1] == b * n) {
      os[no - 1] *= n;
      ao[no - 1] = a;
      bo[no - 1] = b;
    } else {
      os[no] = n;
      ao[no] = a;
      bo[no] = b;
      ++no;
    }
  }
  int nk = 0, ks[3], ak[3], bk[3];
  for (int d = 0; d < s.nk; ++d) {
    int n = s.ks[d], a = (int)s.ak[d], b = (int)s.bk[d];
    if (n == 1) continue;
    if (nk > 0 && ak[nk - 1] == a * n && bk[nk - 1] == b * n) {
      ks[nk - 1] *= n;
      ak[nk - 1] = a;
      bk[nk - 1] = b;
    } else {
      ks[nk] = n;
      ak[nk] = a;
      bk[nk] = b;
      ++nk;
    }
  }
  for (int d = nk; d < 3; ++d) {
    ks[d] = 1;
    ak[d] = bk[d] = 0;
  }
  const int total = (int)s.total;
  const int K0 = ks[0], a0 = ak[0], b0 = bk[0];
  // Register blocking: when the last (merged) output dimension is a multiple of 4, each
  // thread computes 4 consecutive outputs along it, sharing the index arithmetic and the
  // operand loads that do not depend on that dimension.
  const int nlast = no > 0 ? os[no - 1] : 1;
  if (no > 0 && (nlast & 3) == 0 && total >= 4 * PV_NTHR / 2) {
    const int la = ao[no - 1], lb = bo[no - 1];
    const int quads = total >> 2;
    for (int qd = PV_TID; qd < quads; qd += PV_NTHR) {
      int idx = qd << 2;
      int rem = idx, oa = 0, ob = 0;
      for (int d = no - 1; d >= 0; --d) {
        int q = rem / os[d];
        int i = rem - q * os[d];
        rem = q;
        oa += i * ao[d];
        ob += i * bo[d];
      }
      T c0 = 0, c1 = 0, c2 = 0, c3 = 0;
      for (int k2 = 0; k2 < ks[2]; ++k2)
        for (int k1 = 0; k1 < ks[1]; ++k1) {
          const TA* pa = A + oa + k1 * ak[1] + k2 * ak[2];
          const TB* pb = B + ob + k1 * bk[1] + k2 * bk[2];
          if (la == 0) {
#pragma unroll 4
            for (int k0 = 0; k0 < K0; ++k0) {
              T av = (T)pa[k0 * a0];
              const TB* q = pb + k0 * b0;
              c0 += av * (T)q[0];
              c1 += av * (T)q[lb];
              c2 += av * (T)q[2 * lb];
              c3 += av * (T)q[3 * lb];
            }
          } else if (lb == 0) {
#pragma unroll 4
            for (int k0 = 0; k0 < K0; ++k0) {
              T bv = (T)pb[k0 * b0];
              const TA* q = pa + k0 * a0;
              c0 += (T)q[0] * bv;
              c1 += (T)q[la] * bv;
              c2 += (T)q[2 * la] * bv;
              c3 += (T)q[3 * la] * bv;
            }
          } else {
#pragma unroll 4
            for (int k0 = 0; k0 < K0; ++k0) {
              const TA* qa = pa + k0 * a0;
              const TB* qb = pb + k0 * b0;
              c0 += (T)qa[0] * (T)qb[0];
              c1 += (T)qa[la] * (T)qb[lb];
              c2 += (T)qa[2 * la] * (T)qb[2 * lb];
              c3 += (T)qa[3 * la] * (T)qb[3 * lb];
            }
          }
        }
      out[idx] = c0;
      out[idx + 1] = c1;
      out[idx + 2] = c2;
      out[idx + 3] = c3;
    }
    PV_SYNC();
    return;
  }
  for (int idx = PV_TID; idx < total; idx += PV_NTHR) {
    int rem = idx, oa = 0, ob = 0;
    for (int d = no - 1; d >= 0; --d) {
      int q = rem / os[d];
      int i = rem - q * os[d];
      rem = q;
      oa += i * ao[d];
      ob += i * bo[d];
    }
    T acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
    for (int k2 = 0; k2 < ks[2]; ++k2)
      for (int k1 = 0; k1 < ks[1]; ++k1) {
        const TA* pa = A + oa + k1 * ak[1] + k2 * ak[2];
        const TB* pb = B + ob + k1 * bk[1] + k2 * bk[2];
        int k0 = 0;
        for (; k0 + 4 <= K0; k0 += 4) {
          acc0 += (T)pa[k0 * a0] * (T)pb[k0 * b0];
          acc1 += (T)pa[(k0 + 1) * a0] * (T)pb[(k0 + 1) * b0];
          acc2 += (T)pa[(k0 + 2) * a0] * (T)pb[(k0 + 2) * b0];
          acc3 += (T)pa[(k0 + 3) * a0] * (T)pb[(k0 + 3) * b0];
        }
        for (; k0 < K0; ++k0) acc0 += (T)pa[k0 * a0] * (T)pb[k0 * b0];
      }
    out[idx] = (acc0 + acc1) + (acc2 + acc3);
  }
  PV_SYNC();
}

template <typename T, typename TA, typename TB>
PV_HD double einsum(T* out, const char* so, const TA* A, const char* sa, const TB* B,
                    const char* sb, const Dims& d) {
  Spec s = make_spec(so, sa, sb, d);
  contract<T>(out, A, B, s);
  return 2.0 * (double)s.total * (double)s.kprod;   // flops
}

// Block-wide dot product of two length-n vectors.
template <typename T>
PV_HD T dot(const T* x, const T* y, long long n, T* red) {
  T acc = 0;
  for (long long i = PV_TID; i < n; i += PV_NTHR) acc += x[i] * y[i];
  return cta_sum(acc, red);
}

template <typename T>
PV_HD void copy(T* dst, const T* src, long long n) {
  for (long long i = PV_TID; i < n; i += PV_NTHR) dst[i] = src[i];
  PV_SYNC();
}

template <typename T>
PV_HD void fill(T* dst, T v, long long n) {
  for (long long i = PV_TID; i < n; i += PV_NTHR) dst[i] = v;
  PV_SYNC();
}

// Divides x by max|x| (when non-zero) and returns log(max|x|) (0 when x == 0).
template <typename T>
PV_HD double normalize_maxabs(T* x, long long n, T* red) {
  T m = 0;
  for (long long i = PV_TID; i < n; i += PV_NTHR) {
    T a = x[i] < 0 ? -x[i] : x[i];
    m = a > m ? a : m;
  }
  m = cta_max(m, red);
  if (!(m > 0)) {
    PV_SYNC();
    return 0.0;
  }
  T inv = (T)1 / m;
  for (long long i = PV_TID; i < n; i += PV_NTHR) x[i] *= inv;
  PV_SYNC();
  return log((double)m);
}

// ---------------------------------------------------------------------------------------
// Householder triangular factor.  W holds an m x n matrix M row-major (row a contiguous,
// i.e. the columns of M^T).  On return Lout (m x K, row-major, K = min(m, n)) satisfies
// M = Lout Q with Q row-orthonormal (L = R^T from the QR factorisation of M^T).  W is
// overwritten.  `red` needs PV_NWARP entries, `sh` 2 entries of shared scratch.
template <typename T>
PV_HDN double lq_factor(T* Lout, T* W, int m, int n, T* red, T* sh) {
  int K = m < n ? m : n;
  double flops = 0;
  for (long long i = PV_TID; i < (long long)m * K; i += PV_NTHR) Lout[i] = 0;
  PV_SYNC();
  for (int j = 0; j < K; ++j) {
    T* x = W + (long long)j * n;   // column j of M^T, rows j..n-1 active
    T part = 0;
    for (int i = j + PV_TID; i < n; i += PV_NTHR) part += x[i] * x[i];
    T nrm2 = cta_sum(part, red);
    T x0 = x[j];
    T nrm = sqrt(nrm2);
    T alpha = x0 >= 0 ? -nrm : nrm;
    T v0 = x0 - alpha;
    T ax0 = x0 < 0 ? -x0 : x0;
    T vn2 = (T)2 * (nrm2 + nrm * ax0);   // |v|^2 = 2 (|x|^2 - alpha x0), v = x - alpha e_j
    PV_SYNC();
    if (PV_TID == 0) {
      x[j] = v0;
      Lout[(long long)j * K + j] = alpha;   // R[j][j]
    }
    PV_SYNC();
    bool active = nrm2 > 0 && vn2 > 0;
    // columns jj > j: a -= (2/|v|^2) (v.a) v ; then R[j][jj] = a[j]
    for (int jj = j + 1 + PV_WARP; jj < m; jj += PV_NWARP) {
      T* a = W + (long long)jj * n;
      if (active) {
        T p = 0;
        for (int i = j + PV_LANE; i < n; i += PV_WSIZE) p += x[i] * a[i];
        p = warp_sum(p);
        T g = (T)2 * p / vn2;
        for (int i = j + PV_LANE; i < n; i += PV_WSIZE) a[i] -= g * x[i];
      }
#if defined(__CUDA_ARCH__)
      __syncwarp();
#endif
      if (PV_LANE == 0) Lout[(long long)jj * K + j] = a[j];   // L[jj][j] = R[j][jj]
    }
    flops += 4.0 * (double)(n - j) * (double)(m - j);
    PV_SYNC();
  }
  (void)sh;
  return flops;
}

// ---------------------------------------------------------------------------------------
// One-sided (Hestenes) Jacobi: rotates the `nc` columns of Y (column j at Y + j*ldy, length
// len) until they are mutually orthogonal; when V is given the same rotations are applied
// to its nc columns (column j at V + j*ldv, length vlen).  Columns are paired in parallel
// round-robin order; each pair is handled by a group of G lanes (G a power of two, as many
// lanes as a block of `gref` threads allows, gref = 0: this block; the groups take the pairs
// of a round in turn, so a smaller block with the same gref computes the same bits).
// Returns the flop count; *sweeps_out receives the number of sweeps.  `flag` is one shared
// int, `red` PV_NWARP shared entries.
template <typename T>
PV_HD T group_sum(T v, int G) {
#if defined(__CUDA_ARCH__)
  for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
#else
  (void)G;
#endif
  return v;
}

template <typename T>
PV_HDN double jacobi(T* Y, int ldy, int nc, int len, T* V, int ldv, int vlen, T tol,
                     int max_sweeps, int* flag, int* sweeps_out, T* red, int gref = 0) {
  int np = nc + (nc & 1);   // even number of positions; position nc is empty when nc is odd
  double flops = 0;
  int sweep = 0;
  if (nc < 2) {
    if (sweeps_out) *sweeps_out = 0;
    return 0;
  }
  // Stopping test |x_p.x_q| <= tol |x_p||x_q| with tol no finer than the rounding of a
  // length-len dot product; columns below eps*len of the matrix norm are treated as zero
  // (their directions carry no weight and rounding keeps them from converging).
  const T eps = sizeof(T) == 4 ? (T)1.1920929e-7 : (T)2.220446049250313e-16;
  const T tol_eff = tol > (T)4 * len * eps ? tol : (T)4 * len * eps;
  // squared norm of the matrix, by the first warp in a fixed order (the same in any block)
  T nf2 = 0;
  if (PV_WARP == 0) {
    for (int j = 0; j < nc; ++j)
      for (int i = PV_LANE; i < len; i += PV_WSIZE) nf2 += Y[(long long)j * ldy + i] * Y[(long long)j * ldy + i];
    nf2 = warp_sum(nf2);
  }
  PV_SYNC();
  if (PV_TID == 0) red[0] = nf2;
  PV_SYNC();
  nf2 = red[0];
  PV_SYNC();
  const T tiny = (eps * len) * (eps * len) * nf2;
  const int npair = np / 2;
  int G = 1;
#if defined(__CUDA_ARCH__)
  const int gthr = gref > 0 ? gref : PV_NTHR;
  while (G < 32 && G * 2 * npair <= gthr) G *= 2;
  if (G > PV_NTHR) G = PV_NTHR;
#else
  (void)gref;
#endif
  const int ngroups = PV_NTHR / G;
  const int grp = PV_TID / G, gl = PV_TID % G;
  const int iters = (npair + ngroups - 1) / ngroups;
  for (; sweep < max_sweeps; ++sweep) {
    if (PV_TID == 0) *flag = 0;
    PV_SYNC();
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      for (int it = 0; it < iters; ++it) {
        int pr = grp + it * ngroups;
        int p = 0, q = 0;
        bool act = pr < npair;
        if (act) {
          if (pr == 0) {
            p = np - 1;
            q = rnd;
          } else {
            p = (rnd + pr) % (np - 1);
            q = (rnd - pr + (np - 1)) % (np - 1);
          }
          if (p > q) {
            int t = p;
            p = q;
            q = t;
          }
          act = q < nc;
        }
        T* xp = Y + (long long)p * ldy;
        T* xq = Y + (long long)q * ldy;
        T a = 0, b = 0, g = 0;
        if (act)
          for (int i = gl; i < len; i += G) {
            T u = xp[i], w = xq[i];
            a += u * u;
            b += w * w;
            g += u * w;
          }
        a = group_sum(a, G);
        b = group_sum(b, G);
        g = group_sum(g, G);
        T ag = g < 0 ? -g : g;
        if (act && ag > tol_eff * sqrt(a) * sqrt(b) && a > tiny && b > tiny) {
          T zeta = (b - a) / ((T)2 * g);
          T az = zeta < 0 ? -zeta : zeta;
          T t = (T)1 / (az + sqrt((T)1 + az * az));
          if (zeta < 0) t = -t;
          T c = (T)1 / sqrt((T)1 + t * t);
          T sn = c * t;
          for (int i = gl; i < len; i += G) {
            T u = xp[i], w = xq[i];
            xp[i] = c * u - sn * w;
            xq[i] = sn * u + c * w;
          }
          if (V) {
            T* vp = V + (long long)p * ldv;
            T* vq = V + (long long)q * ldv;
            for (int i = gl; i < vlen; i += G) {
              T u = vp[i], w = vq[i];
              vp[i] = c * u - sn * w;
              vq[i] = sn * u + c * w;
            }
          }
          if (gl == 0) {
#if defined(__CUDA_ARCH__)
            atomicAdd(flag, 1);
#else
            *flag += 1;
#endif
          }
        }
      }
      PV_SYNC();
    }
    int f = *flag;   // rotations applied in this sweep
    flops += (double)nc * (nc - 1) / 2 * 6.0 * len + (double)f * (6.0 * len + (V ? 6.0 * vlen : 0.0));
    PV_SYNC();
    if (!f) break;
  }
  if (sweeps_out) *sweeps_out = sweep + 1;
  return flops;
}

}  // namespace pv
