// Batched engine: the per-sample work of the cooling step (boundary-MPS environments,
// amplitude, E_loc, O rows, Metropolis sweep) executed in lockstep over a batch of chains.
// Every contraction, truncation, dot product and update is one operation over the whole
// batch (a kernel launch on the GPU), so the work streams through memory with the
// parallelism of the batch instead of one thread block walking one chain.
//
// The arithmetic is that of the per-sample engine (pv_sample.cuh): the same contractions
// in the same order, the same Householder and Jacobi routines, the same Philox draws.
// Bond dimensions depend only on the position, so all shapes are known on the host.
#pragma once

#include <cstdint>
#include <cmath>
#include <vector>
#include <type_traits>

#include "pv_coop.cuh"
#include "pv_philox.cuh"
#include "pv_sample.cuh"

namespace pv {

// Operand of a batched contraction: a per-sample tensor (base + s * stride) or a slice of
// the parameter vector T_i^{S} with S taken per sample from the configurations or from a
// per-sample selection array.
enum OpMode { OP_BATCH = 0, OP_SITE_S = 1, OP_SITE_SEL = 2 };

template <typename T>
struct Operand {
  const T* base;
  long long stride;      // OP_BATCH: elements between samples
  int mode;
  long long site_off;    // OP_SITE_*: theta offset of the site
  long long site_sz;     //            elements of one slice
  const uint8_t* S;      // OP_SITE_S: configurations [n][N]
  int site;              //            site index
  int N;
  const int8_t* sel;     // OP_SITE_SEL: local index per sample

  PV_HD const T* at(int s) const {
    if (mode == OP_BATCH) return base + (long long)s * stride;
    int v = mode == OP_SITE_S ? (int)S[(long long)s * N + site] : (int)sel[s];
    return base + site_off + (long long)v * site_sz;
  }
};

template <typename T>
PV_HD Operand<T> batch_op(const T* base, long long stride) {
  Operand<T> o;
  o.base = base;
  o.stride = stride;
  o.mode = OP_BATCH;
  o.site_off = o.site_sz = 0;
  o.S = nullptr;
  o.site = o.N = 0;
  o.sel = nullptr;
  return o;
}

// Merged-dimension form of a contraction (as in contract()).
struct MSpec {
  int no, nk;
  int os[6], ao[6], bo[6];
  int ks[3], ak[3], bk[3];
  int total;
  double flops;
};

inline MSpec merge_spec(const Spec& s) {
  MSpec m;
  m.no = 0;
  for (int d = 0; d < s.no; ++d) {
    int n = s.os[d], a = (int)s.ao[d], b = (int)s.bo[d];
    if (n == 1) continue;
    if (m.no > 0 && m.ao[m.no - 1] == a * n && m.bo[m.no - 1] == b * n) {
      m.os[m.no - 1] *= n;
      m.ao[m.no - 1] = a;
      m.bo[m.no - 1] = b;
    } else {
      m.os[m.no] = n;
      m.ao[m.no] = a;
      m.bo[m.no] = b;
      ++m.no;
    }
  }
  m.nk = 0;
  for (int d = 0; d < s.nk; ++d) {
    int n = s.ks[d], a = (int)s.ak[d], b = (int)s.bk[d];
    if (n == 1) continue;
    if (m.nk > 0 && m.ak[m.nk - 1] == a * n && m.bk[m.nk - 1] == b * n) {
      m.ks[m.nk - 1] *= n;
      m.ak[m.nk - 1] = a;
      m.bk[m.nk - 1] = b;
    } else {
      m.ks[m.nk] = n;
      m.ak[m.nk] = a;
      m.bk[m.nk] = b;
      ++m.nk;
    }
  }
  for (int d = m.nk; d < 3; ++d) {
    m.ks[d] = 1;
    m.ak[d] = m.bk[d] = 0;
  }
  m.total = (int)s.total;
  m.flops = 2.0 * (double)s.total * (double)s.kprod;
  return m;
}

// Four consecutive outputs (along the last merged dimension) of one sample's contraction.
template <typename T>
PV_HD void ein_quad(const MSpec& m, T* out, const T* A, const T* B, int idx) {
  int rem = idx, oa = 0, ob = 0;
  for (int d = m.no - 1; d >= 0; --d) {
    int q = rem / m.os[d];
    int i = rem - q * m.os[d];
    rem = q;
    oa += i * m.ao[d];
    ob += i * m.bo[d];
  }
  const int la = m.no > 0 ? m.ao[m.no - 1] : 0, lb = m.no > 0 ? m.bo[m.no - 1] : 0;
  const int K0 = m.ks[0], a0 = m.ak[0], b0 = m.bk[0];
  T c0 = 0, c1 = 0, c2 = 0, c3 = 0;
  for (int k2 = 0; k2 < m.ks[2]; ++k2)
    for (int k1 = 0; k1 < m.ks[1]; ++k1) {
      const T* pa = A + oa + k1 * m.ak[1] + k2 * m.ak[2];
      const T* pb = B + ob + k1 * m.bk[1] + k2 * m.bk[2];
#pragma unroll 4
      for (int k0 = 0; k0 < K0; ++k0) {
        const T* qa = pa + k0 * a0;
        const T* qb = pb + k0 * b0;
        c0 += qa[0] * qb[0];
        c1 += qa[la] * qb[lb];
        c2 += qa[2 * la] * qb[2 * lb];
        c3 += qa[3 * la] * qb[3 * lb];
      }
    }
  out[idx] = c0;
  out[idx + 1] = c1;
  out[idx + 2] = c2;
  out[idx + 3] = c3;
}

template <typename T>
PV_HD void ein_one(const MSpec& m, T* out, const T* A, const T* B, int idx) {
  int rem = idx, oa = 0, ob = 0;
  for (int d = m.no - 1; d >= 0; --d) {
    int q = rem / m.os[d];
    int i = rem - q * m.os[d];
    rem = q;
    oa += i * m.ao[d];
    ob += i * m.bo[d];
  }
  T acc = 0;
  for (int k2 = 0; k2 < m.ks[2]; ++k2)
    for (int k1 = 0; k1 < m.ks[1]; ++k1) {
      const T* pa = A + oa + k1 * m.ak[1] + k2 * m.ak[2];
      const T* pb = B + ob + k1 * m.bk[1] + k2 * m.bk[2];
      for (int k0 = 0; k0 < m.ks[0]; ++k0) acc += pa[k0 * m.ak[0]] * pb[k0 * m.bk[0]];
    }
  out[idx] = acc;
}

PV_HD bool quad_ok(const MSpec& m) { return m.no > 0 && (m.os[m.no - 1] & 3) == 0; }

// GEMM form of a contraction: every output label belongs to exactly one operand, so
// out = C[M][N] with the M index made of A's output labels and N of B's, both with the
// strides of the row-major output.  ok == false when some output label is in both
// operands (not used by this engine).
struct GSpec {
  int nm, nn, nk;
  int ms[4], mA[4], mC[4];
  int ns[4], nB[4], nC[4];
  int ks[4], kA[4], kB[4];
  int M, N, K;
  bool ok;
};

inline GSpec gemm_spec(const Spec& s) {
  GSpec g;
  g.nm = g.nn = g.nk = 0;
  g.M = g.N = g.K = 1;
  g.ok = true;
  long long cstride[6];
  long long st = 1;
  for (int d = s.no - 1; d >= 0; --d) {
    cstride[d] = st;
    st *= s.os[d];
  }
  for (int d = 0; d < s.no; ++d) {
    if (s.os[d] == 1) continue;
    bool inA = s.ao[d] != 0, inB = s.bo[d] != 0;
    if (inA == inB) {
      g.ok = false;
      return g;
    }
    if (inA) {
      if (g.nm == 4) { g.ok = false; return g; }
      g.ms[g.nm] = s.os[d];
      g.mA[g.nm] = (int)s.ao[d];
      g.mC[g.nm] = (int)cstride[d];
      g.M *= s.os[d];
      ++g.nm;
    } else {
      if (g.nn == 4) { g.ok = false; return g; }
      g.ns[g.nn] = s.os[d];
      g.nB[g.nn] = (int)s.bo[d];
      g.nC[g.nn] = (int)cstride[d];
      g.N *= s.os[d];
      ++g.nn;
    }
  }
  for (int d = 0; d < s.nk; ++d) {
    if (s.ks[d] == 1) continue;
    if (g.nk == 4) { g.ok = false; return g; }
    g.ks[g.nk] = s.ks[d];
    g.kA[g.nk] = (int)s.ak[d];
    g.kB[g.nk] = (int)s.bk[d];
    g.K *= s.ks[d];
    ++g.nk;
  }
  return g;
}

// Offsets of a row-major multi-index over dims (sz, stride1, stride2).
PV_HD void gemm_offsets(int idx, int n, const int* sz, const int* s1, const int* s2, int& o1,
                        int& o2) {
  o1 = o2 = 0;
  for (int d = n - 1; d >= 0; --d) {
    int q = idx / sz[d];
    int i = idx - q * sz[d];
    idx = q;
    o1 += i * s1[d];
    o2 += i * s2[d];
  }
}

// ------------------------------------------------------------------------ shapes

// Bond dimensions of every environment and of the truncation steps, from the geometry.
struct Shapes {
  int L1, L2, D, chi;
  // env bonds: down[r][c] (r = 1..L1), up[r][c] (r = 0..L1-1)
  std::vector<std::vector<int>> down, up;

  int dl(int c) const { return c == 0 ? 1 : D; }
  int dr(int c) const { return c == L2 - 1 ? 1 : D; }
  int du(int r) const { return r == 0 ? 1 : D; }
  int dd(int r) const { return r == L1 - 1 ? 1 : D; }

  // Output bonds of compressing (env with bonds `in`) x row r.
  std::vector<int> compress_bonds(const std::vector<int>& in, int p) const {
    std::vector<int> bc(L2 + 1), out(L2 + 1);
    int maxb = 0;
    for (int c = 0; c < L2; ++c) bc[c] = in[c] * dl(c);
    bc[L2] = 1;
    for (int c = 0; c <= L2; ++c) maxb = bc[c] > maxb ? bc[c] : maxb;
    if (maxb <= chi) return bc;
    std::vector<int> kf(L2 + 1);
    kf[L2] = 1;
    for (int c = L2 - 1; c >= 1; --c) kf[c] = bc[c] < p * kf[c + 1] ? bc[c] : p * kf[c + 1];
    out[0] = 1;
    int bprev = 1;
    for (int c = 0; c < L2 - 1; ++c) {
      int m = bprev * p, k = kf[c + 1];
      int kmax = m < k ? m : k;
      int kk = chi < kmax ? chi : kmax;
      out[c + 1] = kk;
      bprev = kk;
    }
    out[L2] = 1;
    return out;
  }

  void build(int L1_, int L2_, int D_, int chi_) {
    L1 = L1_;
    L2 = L2_;
    D = D_;
    chi = chi_;
    down.assign(L1 + 1, std::vector<int>(L2 + 1, 1));
    up.assign(L1, std::vector<int>(L2 + 1, 1));
    for (int r = L1 - 1; r >= 1; --r) down[r] = compress_bonds(down[r + 1], du(r));
    for (int r = 1; r < L1; ++r) up[r] = compress_bonds(up[r - 1], dd(r - 1));
  }
};

}  // namespace pv

namespace pv {

// ------------------------------------------------------------ per-sample operations
// Each functor does one sample's share of an operation; the GPU backend runs one thread
// block per sample, the host backend a plain loop.

template <typename T>
struct OpLq {   // Lf[s] = triangular factor of W[s] (m x nn); W overwritten
  T* Lf;
  long long ls;
  T* W;
  long long ws;
  int m, nn;
  T* red;
  PV_HD void operator()(int s, T* redbuf) const {
    lq_factor(Lf + (long long)s * ls, W + (long long)s * ws, m, nn, redbuf, redbuf);
  }
};

// Truncation of one bond: Jacobi on Y (nc columns of length len, or the m rows when not
// tall), the kk leading left singular vectors into Uk and the environment tensor `out`,
// which is max-abs normalised with the logarithm added to ls[s].
template <typename T>
struct OpTrunc {
  const T* Y;
  long long ys;
  bool tall;
  int nc, len, m, kk;
  T* Uk;
  long long uks;
  T* out;
  long long outs;
  double* lsv;
  int lstride;
  T jtol;
  int max_sweeps;
  unsigned long long* sweeps;
  double* jflops;   // when set: += flops of the Jacobi sweeps this matrix took
  PV_HD void operator()(int s, T* red, int* flag, T* smem, long long smem_cap, int* order,
                        T* sig, int gref = 0) const {
    run<T>(s, red, flag, smem, order, sig, gref, jtol);
    (void)smem_cap;
  }
  // The truncation with working type W (T, or double for float data: the rotations, the
  // singular values and the vectors in float64, the results stored as T).  smem holds the
  // working matrices, red 32 entries of W, sig nc + 4 of W.
  template <typename W>
  PV_HD void run(int s, W* red, int* flag, W* smem, int* order, W* sig, int gref, W tol) const {
    const T* Ys = Y + (long long)s * ys;
    int ldy = len | 1, ldv = m | 1;
    W* Yw = smem;
    W* Vw = smem + (long long)nc * ldy;
    for (long long i = PV_TID; i < (long long)nc * len; i += PV_NTHR)
      Yw[(i / len) * ldy + i % len] = (W)Ys[i];
    if (!tall)
      for (long long i = PV_TID; i < (long long)m * m; i += PV_NTHR)
        Vw[(i / m) * ldv + i % m] = (i / m == i % m) ? (W)1 : (W)0;
    PV_SYNC();
    int sw = 0;
    jacobi(Yw, ldy, nc, len, tall ? (W*)nullptr : Vw, ldv, m, tol, max_sweeps, flag, &sw, red, gref);
    for (int j = PV_WARP; j < nc; j += PV_NWARP) {
      W s2 = 0;
      const W* y = Yw + (long long)j * ldy;
      for (int i = PV_LANE; i < len; i += PV_WSIZE) s2 += y[i] * y[i];
      s2 = warp_sum(s2);
      if (PV_LANE == 0) sig[j] = sqrt(s2);
    }
    PV_SYNC();
    for (int j = PV_TID; j < nc; j += PV_NTHR) {
      int rank = 0;
      W sj = sig[j];
      for (int i = 0; i < nc; ++i) {
        W si = sig[i];
        rank += (si > sj || (si == sj && i < j)) ? 1 : 0;
      }
      order[rank] = j;
    }
    PV_SYNC();
    W zero2 = 0;
    if (tall) {
      W nf2 = 0;
      for (int j = 0; j < nc; ++j) nf2 += sig[j] * sig[j];
      const W eps = sizeof(W) == 4 ? (W)1.1920929e-7 : (W)2.220446049250313e-16;
      zero2 = (eps * len) * (eps * len) * nf2;
    }
    T* U = Uk + (long long)s * uks;
    for (long long idx = PV_TID; idx < (long long)m * kk; idx += PV_NTHR) {
      int q = (int)(idx / kk), jp = (int)(idx % kk);
      int j = order[jp];
      W v;
      if (tall) {
        W sg = sig[j];
        v = sg * sg > zero2 ? Yw[(long long)j * ldy + q] / sg : (W)0;
      } else {
        v = Vw[(long long)j * ldv + q];
      }
      U[idx] = (T)v;
    }
    PV_SYNC();
    T* o = out + (long long)s * outs;
    copy(o, U, (long long)m * kk);
    double l = normalize_maxabs(o, (long long)m * kk, (T*)red);
    if (PV_TID == 0) {
      lsv[(long long)s * lstride] += l;
      // a sweep visits nc (nc - 1) / 2 column pairs: three dot products and a rotation of two
      // columns of length len, and of two columns of V when it is accumulated
      const double jf = (double)sw * 0.5 * nc * (nc - 1) * (12.0 * len + (tall ? 0.0 : 6.0 * m));
#if defined(__CUDA_ARCH__)
      atomicAdd(sweeps, (unsigned long long)sw);
      if (jflops) atomicAdd(jflops, jf);
#else
      *sweeps += (unsigned long long)sw;
      if (jflops) *jflops += jf;
#endif
    }
    PV_SYNC();
  }
};

template <typename T>
struct OpChol {   // Lf[s] (m x m, lower) with Lf Lf^T = G[s] (symmetric positive semidefinite)
  const T* G;
  long long gs;
  T* Lf;
  long long ls;
  int m;
};

template <typename T>
struct OpNorm {   // x[s] /= max|x[s]|, ls[s] += log max
  T* x;
  long long xs, len;
  double* lsv;
  int lstride;
  PV_HD void operator()(int s, T* red) const {
    double l = normalize_maxabs(x + (long long)s * xs, len, red);
    if (PV_TID == 0) lsv[(long long)s * lstride] += l;
    PV_SYNC();
  }
};

template <typename T>
struct OpDot {   // out[s] = a[s] . b[s]
  const T* a;
  long long as;
  const T* b;
  long long bs, len;
  T* out;
  PV_HD void operator()(int s, T* red) const {
    T v = dot(a + (long long)s * as, b + (long long)s * bs, len, red);
    if (PV_TID == 0) out[s] = v;
    PV_SYNC();
  }
};

// --------------------------------------------------------------- elementwise per sample

template <typename T>
struct ElemSet {   // x[s][off] = v
  T* x;
  long long xs, off;
  T v;
  PV_HD void operator()(int s) const { x[(long long)s * xs + off] = v; }
};

template <typename T>
struct ElemCopyMasked {   // dst[s][:len] = src[s][:len] where mask[s] (all when mask null)
  T* dst;
  long long ds;
  const T* src;
  long long ss, len;
  const int8_t* mask;
};

// Local indices of a proposal: flip of site i, or exchange of layer (0 system, 1 ancilla)
// between sites i and j; valid = the move changes the configuration.
struct ElemSel {
  const uint8_t* S;
  int N, i, j, kind;   // kind 0 flip, 1 system exchange, 2 ancilla exchange
  int8_t *si, *sj, *valid;
  PV_HD void operator()(int s) const {
    int a = S[(long long)s * N + i];
    if (kind == 0) {
      si[s] = (int8_t)(3 - a);
      valid[s] = 1;
      return;
    }
    int b = S[(long long)s * N + j];
    int sa = a >> 1, sb = b >> 1, aa = a & 1, ab = b & 1;
    if (kind == 1) {
      si[s] = (int8_t)(2 * sb + aa);
      sj[s] = (int8_t)(2 * sa + ab);
      valid[s] = sa != sb;
    } else {
      si[s] = (int8_t)(2 * sa + ab);
      sj[s] = (int8_t)(2 * sb + aa);
      valid[s] = aa != ab;
    }
  }
};

// E += coef * num/den where valid (local-energy ratio terms).
template <typename T>
struct ElemRatio {
  const T* num;
  const T* den;
  long long dens;   // stride of den (0: per-sample scalar array)
  const int8_t* valid;
  double coef;
  double* e;
  PV_HD void operator()(int s) const {
    if (valid[s]) e[s] += coef * (double)num[s] / (double)den[(long long)s * dens];
  }
};

// Diagonal part of E_sys, E_anc: sum over bonds J S^z_i S^z_j on each layer.
struct ElemDiag {
  const uint8_t* S;
  int N, nb;
  const int* bi;
  const int* bj;
  const double* bJ;
  double *es, *ea;
  PV_HD void operator()(int s) const {
    const uint8_t* x = S + (long long)s * N;
    double a = 0, b = 0;
    for (int k = 0; k < nb; ++k) {
      int p = x[bi[k]], q = x[bj[k]];
      double zs = ((p >> 1) ? -0.5 : 0.5) * ((q >> 1) ? -0.5 : 0.5);
      double za = ((p & 1) ? -0.5 : 0.5) * ((q & 1) ? -0.5 : 0.5);
      a += bJ[k] * zs;
      b += bJ[k] * za;
    }
    es[s] = a;
    ea[s] = b;
  }
};

// Amplitude from the row-0 strip value and the down log-scale.
template <typename T>
struct ElemAmp {
  const T* val;
  long long vs;
  const double* lsd;
  int lstride;
  double* log_abs;
  int8_t* sign;
  PV_HD void operator()(int s) const {
    T v = val[(long long)s * vs];
    T av = v < 0 ? -v : v;
    if (log_abs) log_abs[s] = (av > 0 ? log((double)av) : -INFINITY) + lsd[(long long)s * lstride];
    if (sign) sign[s] = (int8_t)(v > 0 ? 1 : (v < 0 ? -1 : 0));
  }
};

// Metropolis test of a proposal: u = Philox(seed; chain, sweep, id, TAG_MC) < |num/den|^p.
// On acceptance the configuration takes the proposed local indices and `den` the
// numerator; acc/prop count the proposals made.
template <typename T>
struct ElemAccept {
  uint8_t* S;
  int N, i, j;   // j < 0: single-site move
  const int8_t *si, *sj, *valid;
  const T* num;
  T* den;
  int p;
  uint64_t seed;
  int chain0;
  uint32_t sweep, id;
  int *acc, *prop;
  int8_t* accepted;
  const uint32_t* sweep_dev;   // when set, the sweep number is read here (graph replays)
  PV_HD void operator()(int s) const {
    accepted[s] = 0;
    if (!valid[s]) return;
    const uint32_t sw = sweep_dev ? *sweep_dev : sweep;
    double u = philox_uniform(seed, (uint32_t)(chain0 + s), sw, id, TAG_MC);
    double ratio = (double)num[s] / (double)den[s];
    double q = p == 2 ? ratio * ratio : (ratio < 0 ? -ratio : ratio);
    prop[s] += 1;
    if (u < q) {
      acc[s] += 1;
      accepted[s] = 1;
      S[(long long)s * N + i] = (uint8_t)si[s];
      if (j >= 0) S[(long long)s * N + j] = (uint8_t)sj[s];
      den[s] = num[s];
    }
  }
};

// O row entries of one site: O[s][o_off + k] = env[s][k] / val[s].
template <typename T, typename OT>
struct ElemO {
  OT* O;
  long long No, o_off, sz;
  const T* env;
  long long es;
  const T* val;
  long long vs;
};

}  // namespace pv

namespace pv {

// ------------------------------------------------------------------ the batched runner

template <typename T>
struct BatchBufs {
  long long ENV, CB, LB, P1, P2, TMP, D4;
  T *envD, *envU, *Cs, *W, *Lf, *Am, *Y, *carry, *Uk;
  T *p1R, *p1L, *p2R, *p2L, *t0, *t1, *m0, *m1, *m2, *m3, *envo;
  T *val, *num, *den, *val2;
  double *lsD, *lsU;
  int8_t *si, *sj, *valid, *accepted;
  long long sD, sU, sLf, sp1R, sp1L, sp2R, sp2L;   // per-sample strides of the multi-slot buffers

  // Element counts per sample of every buffer, in allocation order.
  static void sizes(int L1, int L2, int D, int chi, std::vector<long long>& real_sz,
                    long long& int8_per_sample, long long& dbl_per_sample) {
    ScratchDims d = scratch_dims(L1, L2, D, chi);
    long long cD = (long long)chi * D;
    real_sz = {(long long)(L1 + 1) * L2 * d.ENV,   // envD
               (long long)L1 * L2 * d.ENV,         // envU
               d.CB, d.CB,                         // Cs, W
               (long long)(L2 + 1) * d.LB,         // Lf
               d.P2,                               // Am
               d.LB,                               // Y
               cD * chi, cD * chi,                 // carry, Uk
               (long long)(L2 + 1) * d.P1, 2 * d.P1,
               (long long)(L2 + 1) * d.P2, 2 * d.P2,
               d.TMP, d.TMP,
               d.P2, d.P2, d.P2, d.P2,
               (long long)D * D * D * D,
               1, 1, 1, 1};                        // val, num, den, val2
    int8_per_sample = 4;
    dbl_per_sample = (long long)(L1 + 1) + 1;
  }

  void bind(T* real, long long n, int8_t* i8, double* dbl, int L1, int L2, int D, int chi) {
    ScratchDims d = scratch_dims(L1, L2, D, chi);
    ENV = d.ENV;
    CB = d.CB;
    LB = d.LB;
    P1 = d.P1;
    P2 = d.P2;
    TMP = d.TMP;
    D4 = (long long)D * D * D * D;
    std::vector<long long> sz;
    long long n8, nd;
    sizes(L1, L2, D, chi, sz, n8, nd);
    T** dst[] = {&envD, &envU, &Cs, &W, &Lf, &Am, &Y, &carry, &Uk, &p1R, &p1L, &p2R, &p2L,
                 &t0, &t1, &m0, &m1, &m2, &m3, &envo, &val, &num, &den, &val2};
    T* p = real;
    for (size_t k = 0; k < sz.size(); ++k) {
      *dst[k] = p;
      p += sz[k] * n;
    }
    sD = sz[0];
    sU = sz[1];
    sLf = sz[4];
    sp1R = sz[9];
    sp1L = sz[10];
    sp2R = sz[11];
    sp2L = sz[12];
    si = i8;
    sj = i8 + n;
    valid = i8 + 2 * n;
    accepted = i8 + 3 * n;
    lsD = dbl;
    lsU = dbl + (L1 + 1) * n;
  }
};

// Buffer slot stride helper: per-sample tensors of size `sz` packed [n][sz].
template <typename T, typename BE, typename OT>
struct BatchRunner {
  BE& be;
  Shapes shp;
  int L1, L2, D, chi, N;
  double J1, J2;
  const T* theta;
  std::vector<long long> toff, ooff;
  BatchBufs<T> b;
  T jtol;
  int max_sweeps;
  double flops = 0;
  bool gram_lq = false;   // right factors from the Gram matrix (the TF32 path)
  const uint32_t* sweep_dev = nullptr;   // Metropolis sweep number in device memory, if set
  unsigned long long* sweeps;   // Jacobi sweep counter (device or host)
  double* jflops = nullptr;     // Jacobi flop counter (profiling), or none

  BatchRunner(BE& be_) : be(be_) {}

  int dl(int c) const { return c == 0 ? 1 : D; }
  int dr(int c) const { return c == L2 - 1 ? 1 : D; }
  int du(int r) const { return r == 0 ? 1 : D; }
  int dd(int r) const { return r == L1 - 1 ? 1 : D; }
  long long szs(int r, int c) const { return (long long)dl(c) * dr(c) * du(r) * dd(r); }

  Operand<T> site(int r, int c, const uint8_t* S) const {
    Operand<T> o = batch_op<T>(theta, 0);
    o.mode = OP_SITE_S;
    o.site_off = toff[r * L2 + c];
    o.site_sz = szs(r, c);
    o.S = S;
    o.site = r * L2 + c;
    o.N = N;
    return o;
  }
  Operand<T> site_sel(int r, int c, const int8_t* sel) const {
    Operand<T> o = site(r, c, nullptr);
    o.mode = OP_SITE_SEL;
    o.sel = sel;
    return o;
  }
  static Operand<T> bat(const T* base, long long stride) { return batch_op<T>(base, stride); }

  void ein(T* out, long long os, const char* so, Operand<T> A, const char* sa, Operand<T> B,
           const char* sb, const Dims& d, int n, bool exact = false) {
    Spec raw = make_spec(so, sa, sb, d);
    MSpec m = merge_spec(raw);
    flops += m.flops * n;
    be.ein(raw, m, out, os, A, B, n, exact);
  }

  // ---------------------------------------------------------------- environments
  // env tensor c of a multi-row environment array
  Operand<T> envt(const T* rowbase, long long stride, int c) const {
    return bat(rowbase + (long long)c * b.ENV, stride);
  }

  void absorb_site(const T* envrow, long long es, const std::vector<int>& bond, bool down, int r,
                   int c, const uint8_t* S, T* out, long long os, int n) {
    Dims dm;
    dm.set('a', bond[c]).set('b', bond[c + 1]).set('l', dl(c)).set('r', dr(c));
    dm.set('u', du(r)).set('d', dd(r));
    if (down)
      ein(out, os, "alubr", envt(envrow, es, c), "adb", site(r, c, S), "lrud", dm, n);
    else
      ein(out, os, "aldbr", envt(envrow, es, c), "aub", site(r, c, S), "lrud", dm, n);
  }

  // out[x][p][(b,r)] = sum_(a,l) carry[x][(a,l)] (env_c x site)[(a,l)][p][(b,r)] for column c
  // of row r, contracted as (carry . env_c) . site: the absorbed tensor (bond x D x D x bond x D)
  // is never formed, only the bprev x D x D x bond intermediate (in the Cs work buffer)
  void carry_absorb(const T* envrow, long long es, const std::vector<int>& bond, bool down, int r,
                    int c, const uint8_t* S, int bprev, T* out, long long os, int n) {
    Dims dm;
    dm.set('x', bprev).set('a', bond[c]).set('b', bond[c + 1]).set('l', dl(c)).set('r', dr(c));
    dm.set('u', du(r)).set('d', dd(r));
    const Operand<T> cy = bat(b.carry, (long long)chi * chi * D);
    if (down) {
      ein(b.Cs, b.CB, "xldb", cy, "xal", envt(envrow, es, c), "adb", dm, n);
      ein(out, os, "xubr", bat(b.Cs, b.CB), "xldb", site(r, c, S), "lrud", dm, n);
    } else {
      ein(b.Cs, b.CB, "xlub", cy, "xal", envt(envrow, es, c), "aub", dm, n);
      ein(out, os, "xdbr", bat(b.Cs, b.CB), "xlub", site(r, c, S), "lrud", dm, n);
    }
  }

  // Compress (env x row r) into outrow (same stride es); log-scales ls[s*lstride] += ...
  void compress(const T* envrow, long long es, const std::vector<int>& bond, bool down, int r,
                const uint8_t* S, T* outrow, long long os, double* ls, int lstride, int n) {
    const int p = down ? du(r) : dd(r);
    std::vector<int> bc(L2 + 1);
    int maxb = 0;
    for (int c = 0; c < L2; ++c) bc[c] = bond[c] * dl(c);
    bc[L2] = 1;
    for (int c = 0; c <= L2; ++c) maxb = bc[c] > maxb ? bc[c] : maxb;
    if (maxb <= chi) {
      for (int c = 0; c < L2; ++c) {
        T* o = outrow + (long long)c * b.ENV;
        absorb_site(envrow, es, bond, down, r, c, S, o, os, n);
        be.norm(OpNorm<T>{o, os, (long long)bc[c] * p * bc[c + 1], ls, lstride}, n);
      }
      return;
    }
    std::vector<int> kf(L2 + 1);
    kf[L2] = 1;
    be.set(b.Lf, b.sLf, (long long)L2 * b.LB, (T)1, n);
    for (int c = L2 - 1; c >= 1; --c) {
      absorb_site(envrow, es, bond, down, r, c, S, b.Cs, b.CB, n);
      Dims dm;
      dm.set('a', bc[c]).set('p', p).set('b', bc[c + 1]).set('k', kf[c + 1]);
      ein(b.W, b.CB, "apk", bat(b.Cs, b.CB), "apb", bat(b.Lf + (long long)(c + 1) * b.LB, b.sLf),
          "bk", dm, n);
      int m = bc[c], nn = p * kf[c + 1];
      if (gram_lq && nn >= m && m >= 16 && be.chol_fits(m)) {
        // a factor of the right Gram matrix W W^T (float32 products, semidefinite Cholesky)
        Dims dg;
        dg.set('a', m).set('e', m).set('p', p).set('k', kf[c + 1]);
        ein(b.Y, b.LB, "ae", bat(b.W, b.CB), "apk", bat(b.W, b.CB), "epk", dg, n, true);
        be.chol(OpChol<T>{b.Y, b.LB, b.Lf + (long long)c * b.LB, b.sLf, m}, n);
        flops += (double)m * m * m / 3.0 * n;
      } else {
        be.lq(OpLq<T>{b.Lf + (long long)c * b.LB, b.sLf, b.W, b.CB, m, nn, nullptr}, n);
        flops += lq_flops(m, nn) * n;
      }
      kf[c] = m < nn ? m : nn;
    }
    be.set(b.carry, (long long)chi * (chi * D), 0, (T)1, n);
    int bprev = 1;
    for (int c = 0; c < L2 - 1; ++c) {
      int bb = bc[c + 1], k = kf[c + 1];
      carry_absorb(envrow, es, bond, down, r, c, S, bprev, b.Am, b.P2, n);
      int m = bprev * p;
      bool tall = k <= m;
      Dims dq;
      dq.set('q', m).set('b', bb).set('k', k);
      const T* Lc = b.Lf + (long long)(c + 1) * b.LB;
      ein(b.Y, b.LB, tall ? "kq" : "qk", bat(b.Am, b.P2), "qb", bat(Lc, b.sLf), "bk", dq, n);
      int nc = tall ? k : m, len = tall ? m : k;
      int kmax = m < k ? m : k;
      int kk = chi < kmax ? chi : kmax;
      T* o = outrow + (long long)c * b.ENV;
      be.trunc(OpTrunc<T>{b.Y, b.LB, tall, nc, len, m, kk, b.Uk, (long long)chi * chi * D, o, os,
                          ls, lstride, jtol, max_sweeps, sweeps, jflops},
               n);
      Dims dc;
      dc.set('q', m).set('j', kk).set('b', bb);
      ein(b.carry, (long long)chi * chi * D, "jb", bat(b.Uk, (long long)chi * chi * D), "qj",
          bat(b.Am, b.P2), "qb", dc, n);
      bprev = kk;
    }
    {
      int c = L2 - 1;
      T* o = outrow + (long long)c * b.ENV;
      carry_absorb(envrow, es, bond, down, r, c, S, bprev, o, os, n);
      be.norm(OpNorm<T>{o, os, (long long)bprev * p * bc[c + 1], ls, lstride}, n);
    }
  }

  static double lq_flops(int m, int n) {
    int K = m < n ? m : n;
    double f = 0;
    for (int j = 0; j < K; ++j) f += 4.0 * (double)(n - j) * (double)(m - j);
    return f;
  }

  T* downrow(int r) const { return b.envD + (long long)r * L2 * b.ENV; }
  T* uprow(int r) const { return b.envU + (long long)r * L2 * b.ENV; }

  void trivial(T* row, long long stride, int n) {
    for (int c = 0; c < L2; ++c) be.set(row, stride, (long long)c * b.ENV, (T)1, n);
  }

  void build_down(const uint8_t* S, int n) {
    trivial(downrow(L1), b.sD, n);
    be.setd(b.lsD, L1 + 1, L1, 0.0, n);
    for (int r = L1 - 1; r >= 1; --r) {
      be.copyd(b.lsD, L1 + 1, r, r + 1, n);   // lsD[r] = lsD[r+1]
      compress(downrow(r + 1), b.sD, shp.down[r + 1], true, r, S, downrow(r), b.sD, b.lsD + r,
               L1 + 1, n);
    }
  }

  // Down environments that are the same for every chain (direct sampling's all-summed
  // rows): chain 0's, with its log scales, copied to chains 1..n-1.
  void broadcast_down(int n) {
    if (n <= 1) return;
    be.copy_masked(b.envD + b.sD, b.sD, b.envD, 0, b.sD, nullptr, n - 1);
    be.bcastd(b.lsD, L1 + 1, L1 + 1, n);
  }

  // ----------------------------------------------------------------- strips
  // one-row strip pieces (U row = up env of row r, Dn row = down env r+1)
  void s1_left(int r, int c, T* Lout, long long los, Operand<T> Lin, Operand<T> A, int n) {
    const std::vector<int>&bu = shp.up[r], &bd = shp.down[r + 1];
    Dims dm;
    dm.set('a', bu[c]).set('x', bu[c + 1]).set('b', bd[c]).set('y', bd[c + 1]);
    dm.set('l', dl(c)).set('r', dr(c)).set('u', du(r)).set('d', dd(r));
    ein(b.t0, b.TMP, "lbux", Lin, "alb", envt(uprow(r), b.sU, c), "aux", dm, n);
    ein(b.t1, b.TMP, "bxrd", bat(b.t0, b.TMP), "lbux", A, "lrud", dm, n);
    ein(Lout, los, "xry", bat(b.t1, b.TMP), "bxrd", envt(downrow(r + 1), b.sD, c), "bdy", dm, n);
  }
  void s1_right(int r, int c, T* Rout, long long ros, Operand<T> Rin, Operand<T> A, int n) {
    const std::vector<int>&bu = shp.up[r], &bd = shp.down[r + 1];
    Dims dm;
    dm.set('a', bu[c]).set('x', bu[c + 1]).set('b', bd[c]).set('y', bd[c + 1]);
    dm.set('l', dl(c)).set('r', dr(c)).set('u', du(r)).set('d', dd(r));
    ein(b.t0, b.TMP, "bdxr", envt(downrow(r + 1), b.sD, c), "bdy", Rin, "xry", dm, n);
    ein(b.t1, b.TMP, "lubx", A, "lrud", bat(b.t0, b.TMP), "bdxr", dm, n);
    ein(Rout, ros, "alb", envt(uprow(r), b.sU, c), "aux", bat(b.t1, b.TMP), "lubx", dm, n);
  }
  void s1_env(int r, int c, Operand<T> L, Operand<T> R, int n) {
    const std::vector<int>&bu = shp.up[r], &bd = shp.down[r + 1];
    Dims dm;
    dm.set('a', bu[c]).set('x', bu[c + 1]).set('b', bd[c]).set('y', bd[c + 1]);
    dm.set('l', dl(c)).set('r', dr(c)).set('u', du(r)).set('d', dd(r));
    ein(b.t0, b.TMP, "lbux", L, "alb", envt(uprow(r), b.sU, c), "aux", dm, n);
    ein(b.t1, b.TMP, "lbury", bat(b.t0, b.TMP), "lbux", R, "xry", dm, n);
    ein(b.envo, b.D4, "lrud", bat(b.t1, b.TMP), "lbury", envt(downrow(r + 1), b.sD, c), "bdy", dm, n);
  }
  long long s1_len(int r, int c) const {
    return (long long)shp.up[r][c] * (c < L2 ? dl(c) : 1) * shp.down[r + 1][c];
  }
  // two-row strip pieces (U = up env of row r, rows r and r+1, Dn = down env r+2)
  void s2_left(int r, int c, T* Lout, long long los, Operand<T> Lin, Operand<T> A1, Operand<T> A2,
               int n) {
    const std::vector<int>&bu = shp.up[r], &bd = shp.down[r + 2];
    Dims dm;
    dm.set('a', bu[c]).set('x', bu[c + 1]).set('b', bd[c]).set('y', bd[c + 1]);
    dm.set('i', dl(c)).set('r', dr(c)).set('j', dl(c)).set('s', dr(c));
    dm.set('u', du(r)).set('m', dd(r)).set('d', dd(r + 1));
    ein(b.t0, b.TMP, "ijbux", Lin, "aijb", envt(uprow(r), b.sU, c), "aux", dm, n);
    ein(b.t1, b.TMP, "jbxrm", bat(b.t0, b.TMP), "ijbux", A1, "irum", dm, n);
    ein(b.t0, b.TMP, "bxrsd", bat(b.t1, b.TMP), "jbxrm", A2, "jsmd", dm, n);
    ein(Lout, los, "xrsy", bat(b.t0, b.TMP), "bxrsd", envt(downrow(r + 2), b.sD, c), "bdy", dm, n);
  }
  void s2_right(int r, int c, T* Rout, long long ros, Operand<T> Rin, Operand<T> A1,
                Operand<T> A2, int n) {
    const std::vector<int>&bu = shp.up[r], &bd = shp.down[r + 2];
    Dims dm;
    dm.set('a', bu[c]).set('x', bu[c + 1]).set('b', bd[c]).set('y', bd[c + 1]);
    dm.set('i', dl(c)).set('r', dr(c)).set('j', dl(c)).set('s', dr(c));
    dm.set('u', du(r)).set('m', dd(r)).set('d', dd(r + 1));
    ein(b.t0, b.TMP, "bdxrs", envt(downrow(r + 2), b.sD, c), "bdy", Rin, "xrsy", dm, n);
    ein(b.t1, b.TMP, "jmbxr", A2, "jsmd", bat(b.t0, b.TMP), "bdxrs", dm, n);
    ein(b.t0, b.TMP, "iujbx", A1, "irum", bat(b.t1, b.TMP), "jmbxr", dm, n);
    ein(Rout, ros, "aijb", envt(uprow(r), b.sU, c), "aux", bat(b.t0, b.TMP), "iujbx", dm, n);
  }
  long long s2_len(int r, int c) const {
    long long l = c < L2 ? dl(c) : 1;
    return (long long)shp.up[r][c] * l * l * shp.down[r + 2][c];
  }

  T* p1R(int c) const { return b.p1R + (long long)c * b.P1; }
  T* p2R(int c) const { return b.p2R + (long long)c * b.P2; }

  // ------------------------------------------------------------------- evaluation
  void eval(const uint8_t* S, int n, double* log_abs, int8_t* sign, double* es, double* ea,
            OT* O, long long No, bool cached) {
    build_down(S, n);
    // diagonal energies
    be.diag(S, n, es, ea);
    if (!cached) trivial(uprow(0), b.sU, n);
    for (int r = 0; r < L1; ++r) {
      // one-row strip: right partials, value, O, horizontal ratios with a rolling left partial
      be.set(b.p1R, b.sp1R, (long long)L2 * b.P1, (T)1, n);
      for (int c = L2 - 1; c >= 0; --c)
        s1_right(r, c, p1R(c), b.sp1R, bat(p1R(c + 1), b.sp1R), site(r, c, S), n);
      if (r == 0) be.amp(b.p1R, b.sp1R, b.lsD + 1, L1 + 1, log_abs, sign, n);
      T* Lc = b.p1L;
      T* Ln = b.p1L + b.P1;
      be.set(b.p1L, b.sp1L, 0, (T)1, n);
      for (int c = 0; c < L2; ++c) {
        if (O) {
          s1_env(r, c, bat(Lc, b.sp1L), bat(p1R(c + 1), b.sp1R), n);
          be.writeO(O, No, ooff[r * L2 + c], b.envo, b.D4, szs(r, c), b.p1R, b.sp1R, n);
        }
        if (c + 1 < L2) {
          for (int layer = 0; layer < 2; ++layer) {
            be.sel(ElemSel{S, N, r * L2 + c, r * L2 + c + 1, 1 + layer, b.si, b.sj, b.valid}, n);
            s1_left(r, c, b.m0, b.P2, bat(Lc, b.sp1L), site_sel(r, c, b.si), n);
            s1_left(r, c + 1, b.m1, b.P2, bat(b.m0, b.P2), site_sel(r, c + 1, b.sj), n);
            be.dot(OpDot<T>{b.m1, b.P2, p1R(c + 2), b.sp1R, s1_len(r, c + 2), b.num}, n);
            be.ratio(b.num, b.p1R, b.sp1R, b.valid, 0.5 * J1, layer == 0 ? es : ea, n);
          }
          s1_left(r, c, Ln, b.sp1L, bat(Lc, b.sp1L), site(r, c, S), n);
          T* t = Lc;
          Lc = Ln;
          Ln = t;
        }
      }
      if (r + 1 < L1) {
        be.set(b.p2R, b.sp2R, (long long)L2 * b.P2, (T)1, n);
        for (int c = L2 - 1; c >= 0; --c)
          s2_right(r, c, p2R(c), b.sp2R, bat(p2R(c + 1), b.sp2R), site(r, c, S), site(r + 1, c, S), n);
        T* L2c = b.p2L;
        T* L2n = b.p2L + b.P2;
        be.set(b.p2L, b.sp2L, 0, (T)1, n);
        for (int c = 0; c < L2; ++c) {
          int i = r * L2 + c, j = i + L2;
          for (int layer = 0; layer < 2; ++layer) {
            be.sel(ElemSel{S, N, i, j, 1 + layer, b.si, b.sj, b.valid}, n);
            s2_left(r, c, b.m0, b.P2, bat(L2c, b.sp2L), site_sel(r, c, b.si), site_sel(r + 1, c, b.sj), n);
            be.dot(OpDot<T>{b.m0, b.P2, p2R(c + 1), b.sp2R, s2_len(r, c + 1), b.num}, n);
            be.ratio(b.num, b.p2R, b.sp2R, b.valid, 0.5 * J1, layer == 0 ? es : ea, n);
          }
          if (J2 != 0.0 && c + 1 < L2) {
            for (int diag = 0; diag < 2; ++diag) {
              int a = diag == 0 ? r * L2 + c : r * L2 + c + 1;
              int bb = diag == 0 ? (r + 1) * L2 + c + 1 : (r + 1) * L2 + c;
              for (int layer = 0; layer < 2; ++layer) {
                be.sel(ElemSel{S, N, a, bb, 1 + layer, b.si, b.sj, b.valid}, n);
                // columns c and c+1 of both rows with the two changed sites
                Operand<T> s00 = diag == 0 ? site_sel(r, c, b.si) : site(r, c, S);
                Operand<T> s10 = diag == 0 ? site(r + 1, c, S) : site_sel(r + 1, c, b.sj);
                Operand<T> s01 = diag == 0 ? site(r, c + 1, S) : site_sel(r, c + 1, b.si);
                Operand<T> s11 = diag == 0 ? site_sel(r + 1, c + 1, b.sj) : site(r + 1, c + 1, S);
                s2_left(r, c, b.m0, b.P2, bat(L2c, b.sp2L), s00, s10, n);
                s2_left(r, c + 1, b.m1, b.P2, bat(b.m0, b.P2), s01, s11, n);
                be.dot(OpDot<T>{b.m1, b.P2, p2R(c + 2), b.sp2R, s2_len(r, c + 2), b.num}, n);
                be.ratio(b.num, b.p2R, b.sp2R, b.valid, 0.5 * J2, layer == 0 ? es : ea, n);
              }
            }
          }
          s2_left(r, c, L2n, b.sp2L, bat(L2c, b.sp2L), site(r, c, S), site(r + 1, c, S), n);
          T* t = L2c;
          L2c = L2n;
          L2n = t;
        }
        if (!cached)
          compress(uprow(r), b.sU, shp.up[r], false, r, S, uprow(r + 1), b.sU, b.lsU, 1, n);
      }
    }
  }

  // -------------------------------------------------------------------- Metropolis
  void mc(uint8_t* S, int n, int p, uint64_t seed, int chain0, uint32_t sweep, int* acc,
          int* prop) {
    build_down(S, n);
    trivial(uprow(0), b.sU, n);
    for (int r = 0; r < L1; ++r) {
      be.set(b.p1R, b.sp1R, (long long)L2 * b.P1, (T)1, n);
      for (int c = L2 - 1; c >= 0; --c)
        s1_right(r, c, p1R(c), b.sp1R, bat(p1R(c + 1), b.sp1R), site(r, c, S), n);
      T* Lc = b.p1L;
      T* Ln = b.p1L + b.P1;
      be.set(b.p1L, b.sp1L, 0, (T)1, n);
      // P = Lc x column c at the current S (m0); X, Y proposals (m2, m3); Q = P x column c+1 (m1)
      s1_left(r, 0, b.m0, b.P2, bat(Lc, b.sp1L), site(r, 0, S), n);
      for (int c = 0; c < L2; ++c) {
        int i = r * L2 + c;
        be.dot(OpDot<T>{b.m0, b.P2, p1R(c + 1), b.sp1R, s1_len(r, c + 1), b.den}, n);
        be.sel(ElemSel{S, N, i, -1, 0, b.si, b.sj, b.valid}, n);
        s1_left(r, c, b.m2, b.P2, bat(Lc, b.sp1L), site_sel(r, c, b.si), n);
        be.dot(OpDot<T>{b.m2, b.P2, p1R(c + 1), b.sp1R, s1_len(r, c + 1), b.num}, n);
        be.accept(ElemAccept<T>{S, N, i, -1, b.si, b.sj, b.valid, b.num, b.den, p, seed, chain0,
                                sweep, (uint32_t)(8 * i), acc, prop, b.accepted, sweep_dev}, n);
        be.copy_masked(b.m0, b.P2, b.m2, b.P2, s1_len(r, c + 1), b.accepted, n);
        if (c + 1 < L2) {
          s1_left(r, c + 1, b.m1, b.P2, bat(b.m0, b.P2), site(r, c + 1, S), n);
          be.dot(OpDot<T>{b.m1, b.P2, p1R(c + 2), b.sp1R, s1_len(r, c + 2), b.den}, n);
          for (int layer = 0; layer < 2; ++layer) {
            be.sel(ElemSel{S, N, i, i + 1, 1 + layer, b.si, b.sj, b.valid}, n);
            s1_left(r, c, b.m2, b.P2, bat(Lc, b.sp1L), site_sel(r, c, b.si), n);
            s1_left(r, c + 1, b.m3, b.P2, bat(b.m2, b.P2), site_sel(r, c + 1, b.sj), n);
            be.dot(OpDot<T>{b.m3, b.P2, p1R(c + 2), b.sp1R, s1_len(r, c + 2), b.num}, n);
            be.accept(ElemAccept<T>{S, N, i, i + 1, b.si, b.sj, b.valid, b.num, b.den, p, seed,
                                    chain0, sweep, (uint32_t)(8 * i + 1 + layer), acc, prop,
                                    b.accepted, sweep_dev}, n);
            be.copy_masked(b.m0, b.P2, b.m2, b.P2, s1_len(r, c + 1), b.accepted, n);
            be.copy_masked(b.m1, b.P2, b.m3, b.P2, s1_len(r, c + 2), b.accepted, n);
          }
        }
        // advance: left partial past column c is P; the next P is Q
        be.copy_masked(Ln, b.sp1L, b.m0, b.P2, s1_len(r, c + 1), nullptr, n);
        T* t = Lc;
        Lc = Ln;
        Ln = t;
        if (c + 1 < L2) be.copy_masked(b.m0, b.P2, b.m1, b.P2, s1_len(r, c + 2), nullptr, n);
      }
      if (r + 1 < L1) {
        be.set(b.p2R, b.sp2R, (long long)L2 * b.P2, (T)1, n);
        for (int c = L2 - 1; c >= 0; --c)
          s2_right(r, c, p2R(c), b.sp2R, bat(p2R(c + 1), b.sp2R), site(r, c, S), site(r + 1, c, S), n);
        T* L2c = b.p2L;
        T* L2n = b.p2L + b.P2;
        be.set(b.p2L, b.sp2L, 0, (T)1, n);
        for (int c = 0; c < L2; ++c) {
          int i = r * L2 + c, j = i + L2;
          s2_left(r, c, b.m0, b.P2, bat(L2c, b.sp2L), site(r, c, S), site(r + 1, c, S), n);
          be.dot(OpDot<T>{b.m0, b.P2, p2R(c + 1), b.sp2R, s2_len(r, c + 1), b.den}, n);
          for (int layer = 0; layer < 2; ++layer) {
            be.sel(ElemSel{S, N, i, j, 1 + layer, b.si, b.sj, b.valid}, n);
            s2_left(r, c, b.m1, b.P2, bat(L2c, b.sp2L), site_sel(r, c, b.si), site_sel(r + 1, c, b.sj), n);
            be.dot(OpDot<T>{b.m1, b.P2, p2R(c + 1), b.sp2R, s2_len(r, c + 1), b.num}, n);
            be.accept(ElemAccept<T>{S, N, i, j, b.si, b.sj, b.valid, b.num, b.den, p, seed, chain0,
                                    sweep, (uint32_t)(8 * i + 3 + layer), acc, prop, b.accepted, sweep_dev}, n);
            be.copy_masked(b.m0, b.P2, b.m1, b.P2, s2_len(r, c + 1), b.accepted, n);
          }
          be.copy_masked(L2n, b.sp2L, b.m0, b.P2, s2_len(r, c + 1), nullptr, n);
          T* t = L2c;
          L2c = L2n;
          L2n = t;
        }
        compress(uprow(r), b.sU, shp.up[r], false, r, S, uprow(r + 1), b.sU, b.lsU, 1, n);
      }
    }
  }
};

}  // namespace pv

namespace pv {

// Bonds of Eq. 12 as (site i, site j, coupling) lists, the diagonal part of E_loc.
inline void bond_lists(int L1, int L2, double J1, double J2, std::vector<int>& bi,
                       std::vector<int>& bj, std::vector<double>& bJ) {
  bi.clear();
  bj.clear();
  bJ.clear();
  for (int r = 0; r < L1; ++r)
    for (int c = 0; c + 1 < L2; ++c) {
      bi.push_back(r * L2 + c);
      bj.push_back(r * L2 + c + 1);
      bJ.push_back(J1);
    }
  for (int r = 0; r + 1 < L1; ++r)
    for (int c = 0; c < L2; ++c) {
      bi.push_back(r * L2 + c);
      bj.push_back((r + 1) * L2 + c);
      bJ.push_back(J1);
    }
  if (J2 != 0.0)
    for (int r = 0; r + 1 < L1; ++r)
      for (int c = 0; c + 1 < L2; ++c) {
        bi.push_back(r * L2 + c);
        bj.push_back((r + 1) * L2 + c + 1);
        bJ.push_back(J2);
        bi.push_back(r * L2 + c + 1);
        bj.push_back((r + 1) * L2 + c);
        bJ.push_back(J2);
      }
}

}  // namespace pv

#include "pv_tc.cuh"
#include "pv_tc2.cuh"

#if defined(__CUDACC__)
#include "pv_prof.cuh"
namespace pv {

constexpr int BT = 256;   // threads of the per-sample blocks
constexpr int LQ_THREADS = 512;   // threads of the shared-memory Householder kernel

template <typename T>
__global__ void __launch_bounds__(256) kb_ein(MSpec m, T* out, long long os, Operand<T> A,
                                              Operand<T> B, int n, int quad) {
  int s = blockIdx.y;
  if (s >= n) return;
  const T* pa = A.at(s);
  const T* pb = B.at(s);
  T* po = out + (long long)s * os;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (quad) {
    int idx = t << 2;
    if (idx < m.total) ein_quad(m, po, pa, pb, idx);
  } else {
    if (t < m.total) ein_one(m, po, pa, pb, t);
  }
}

// Batched strided GEMM: one thread block computes a TM x TN tile of G samples'
// contractions (G > 1 when one sample's tile is smaller than the block); operand chunks
// of KC contraction indices are gathered into shared memory (each element loaded once per
// tile) and every thread accumulates a 4 x 4 register tile.  The index maps are the same
// for every sample and are built once per block.
template <typename T>
__global__ void __launch_bounds__(256) kb_gemm(GSpec g, T* C, long long cs, Operand<T> A,
                                               Operand<T> B, int n, int TM, int TN, int KC,
                                               int tilesN, int G) {
  extern __shared__ __align__(16) unsigned char dyn[];
  const int tid = threadIdx.x;
  const int tm = blockIdx.x / tilesN, tn = blockIdx.x % tilesN;
  const int m0 = tm * TM, n0 = tn * TN;
  const int chunkA = KC * TM, chunkB = KC * TN;
  T* As = (T*)dyn;                  // [G][KC][TM]
  T* Bs = As + G * chunkA;          // [G][KC][TN]
  int* rowA = (int*)(Bs + G * chunkB);
  int* rowC = rowA + TM;
  int* colB = rowC + TM;
  int* colC = colB + TN;
  int* kAo = colC + TN;
  int* kBo = kAo + g.K;
  for (int i = tid; i < TM; i += 256) {
    int m = m0 + i;
    if (m < g.M) gemm_offsets(m, g.nm, g.ms, g.mA, g.mC, rowA[i], rowC[i]);
    else rowA[i] = rowC[i] = -1;
  }
  for (int i = tid; i < TN; i += 256) {
    int c = n0 + i;
    if (c < g.N) gemm_offsets(c, g.nn, g.ns, g.nB, g.nC, colB[i], colC[i]);
    else colB[i] = colC[i] = -1;
  }
  for (int k = tid; k < g.K; k += 256) gemm_offsets(k, g.nk, g.ks, g.kA, g.kB, kAo[k], kBo[k]);
  __syncthreads();
  const int tnx = TN >> 2;
  const int per = (TM >> 2) * tnx;          // compute threads per sample
  const int slot = tid / per, loc = tid - slot * per;
  const int tx = loc % tnx, ty = loc / tnx;
  for (int sbase = blockIdx.y * G; sbase < n; sbase += gridDim.y * G) {
    const int ns = min(G, n - sbase);
    const int s = sbase + slot;
    const bool comp = slot < ns;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0;
    for (int k0 = 0; k0 < g.K; k0 += KC) {
      // four independent loads per thread before the stores
      const int totA = ns * chunkA, totB = ns * chunkB;
      for (int i0 = tid; i0 < totA; i0 += 1024) {
        T v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int idx = i0 + u * 256;
          v[u] = (T)0;
          if (idx < totA) {
            int gs = idx / chunkA, r = idx - gs * chunkA;
            int kk = r / TM, mm = r - kk * TM, k = k0 + kk;
            if (k < g.K && rowA[mm] >= 0) v[u] = A.at(sbase + gs)[rowA[mm] + kAo[k]];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (i0 + u * 256 < totA) As[i0 + u * 256] = v[u];
      }
      for (int i0 = tid; i0 < totB; i0 += 1024) {
        T v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int idx = i0 + u * 256;
          v[u] = (T)0;
          if (idx < totB) {
            int gs = idx / chunkB, r = idx - gs * chunkB;
            int kk = r / TN, nn = r - kk * TN, k = k0 + kk;
            if (k < g.K && colB[nn] >= 0) v[u] = B.at(sbase + gs)[colB[nn] + kBo[k]];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (i0 + u * 256 < totB) Bs[i0 + u * 256] = v[u];
      }
      __syncthreads();
      if (comp) {
        const T* as = As + slot * chunkA;
        const T* bs = Bs + slot * chunkB;
        const int kend = min(KC, g.K - k0);
        for (int kk = 0; kk < kend; ++kk) {
          T a[4], b[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = as[kk * TM + ty * 4 + i];
#pragma unroll
          for (int j = 0; j < 4; ++j) b[j] = bs[kk * TN + tx * 4 + j];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
      }
      __syncthreads();
    }
    if (comp) {
      T* pc = C + (long long)s * cs;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        int r = rowC[ty * 4 + i];
        if (r < 0) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          int c = colC[tx * 4 + j];
          if (c >= 0) pc[r + c] = acc[i][j];
        }
      }
    }
  }
}

// Householder factor per sample; the sample's matrix is first copied to shared memory
// when it fits (use_smem), so the column sweeps run out of shared memory.
template <typename T>
__global__ void __launch_bounds__(BT) kb_lq(OpLq<T> op, int n, int use_smem) {
  __shared__ T red[32];
  extern __shared__ __align__(16) unsigned char dyn[];
  T* Ws = (T*)dyn;
  const long long len = (long long)op.m * op.nn;
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    T* W = op.W + (long long)s * op.ws;
    if (use_smem) {
      for (long long i = threadIdx.x; i < len; i += blockDim.x) Ws[i] = W[i];
      __syncthreads();
      W = Ws;
    }
    lq_factor(op.Lf + (long long)s * op.ls, W, op.m, op.nn, red, red);
    __syncthreads();
  }
}

// Householder factor with the chain's matrix in shared memory (row stride ld, chosen so
// that the row groups of one warp fall on disjoint banks), 4-wide vector accesses.  Step j
// reflects the tail of row j onto e_j: alpha = -sign(x0) |x|, v = x - alpha e_j; v is kept
// in place of row j (its entries left of column j zeroed inside the first vector, so whole
// 4-wide vectors can be used).  Every later row jj is updated by a group of G threads (a
// partial dot v.a over the group's vectors, a shuffle reduction inside the group, then
// a -= (2 v.a / |v|^2) v) and L[jj][j] = a_j.  The group holding row j+1 also forms that
// row's tail norm and its reflector for step j+1, so each step costs one barrier.
// Needs nn and ld multiples of 4.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) kb_lq2(OpLq<T> op, int n, int ld, int G) {
  typedef typename std::conditional<sizeof(T) == 8, double2, float4>::type V2;
  extern __shared__ __align__(16) unsigned char dyn[];
  T* Wm = (T*)dyn;
  __shared__ T s_alpha[2], s_vn2[2];
  const int m = op.m, nn = op.nn, K = m < nn ? m : nn;
  const int tid = threadIdx.x, grp = tid / G, gl = tid - grp * G, ngrp = NT / G;
  const int nq = nn >> 2;   // 4-wide vectors per row
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    const T* W = op.W + (long long)s * op.ws;
    T* Lo = op.Lf + (long long)s * op.ls;
    for (int i = tid; i < m * nn; i += NT) {
      const int r = i / nn;
      Wm[r * ld + (i - r * nn)] = W[i];
    }
    for (int i = tid; i < m * K; i += NT) Lo[i] = (T)0;
    __syncthreads();
    if (tid < 32) {   // reflector of row 0
      T p = 0;
      for (int c = tid; c < nn; c += 32) p += Wm[c] * Wm[c];
      p = warp_sum(p);
      if (tid == 0) {
        const T x0 = Wm[0], nrm = sqrt(p), ax0 = x0 < 0 ? -x0 : x0;
        const T alpha = x0 >= 0 ? -nrm : nrm;
        s_alpha[0] = alpha;
        s_vn2[0] = (p > 0) ? (T)2 * (p + nrm * ax0) : (T)0;
        Wm[0] = x0 - alpha;
      }
    }
    __syncthreads();
    for (int j = 0; j < K; ++j) {
      const T* x = Wm + (long long)j * ld;
      const T vn2 = s_vn2[j & 1];
      const bool active = vn2 > 0;
      if (tid == 0) Lo[(long long)j * K + j] = s_alpha[j & 1];
      const int q0 = j >> 2;
      for (int base = j + 1; base < m; base += ngrp) {   // uniform trip count: shuffles below
        const int jj = base + grp;
        const bool valid = jj < m;
        T* a = Wm + (long long)(valid ? jj : j) * ld;
        T p0 = 0, p1 = 0;
        if (valid && active) {
#pragma unroll 2
          for (int q = q0 + gl; q < nq; q += G) {
            V2 xv, av;
            if constexpr (sizeof(T) == 8) {
              xv = *(const V2*)(x + 4 * q);
              av = *(const V2*)(a + 4 * q);
              p0 += xv.x * av.x + xv.y * av.y;
              xv = *(const V2*)(x + 4 * q + 2);
              av = *(const V2*)(a + 4 * q + 2);
              p1 += xv.x * av.x + xv.y * av.y;
            } else {
              xv = *(const V2*)(x + 4 * q);
              av = *(const V2*)(a + 4 * q);
              p0 += xv.x * av.x + xv.y * av.y;
              p1 += xv.z * av.z + xv.w * av.w;
            }
          }
        }
        T p = p0 + p1;
        for (int o = G >> 1; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
        const T g = active ? (T)2 * p / vn2 : (T)0;
        const bool first = base == j + 1;   // group 0 of the first pass holds row j + 1
        T t2 = 0;
        if (valid) {
          for (int q = q0 + gl; q < nq; q += G) {
            T* ap = a + 4 * q;
            T e[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) e[u] = ap[u] - g * x[4 * q + u];
            if constexpr (sizeof(T) == 8) {
              *(V2*)ap = V2{e[0], e[1]};
              *(V2*)(ap + 2) = V2{e[2], e[3]};
            } else {
              *(V2*)ap = V2{e[0], e[1], e[2], e[3]};
            }
            if (first)
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (4 * q + u > j) t2 += e[u] * e[u];
          }
          if (gl == 0) Lo[(long long)jj * K + j] = a[j];
        }
        if (first) {
          for (int o = G >> 1; o > 0; o >>= 1) t2 += __shfl_xor_sync(0xffffffffu, t2, o);
          // the lane holding column j + 1 of row j + 1 forms the next reflector
          const int c1 = j + 1;
          if (grp == 0 && c1 < nn && jj < m && gl == (c1 >> 2) - q0) {
            const T x0 = a[c1], nrm = sqrt(t2), ax0 = x0 < 0 ? -x0 : x0;
            const T alpha = x0 >= 0 ? -nrm : nrm;
            s_alpha[c1 & 1] = alpha;
            s_vn2[c1 & 1] = (t2 > 0) ? (T)2 * (t2 + nrm * ax0) : (T)0;
            a[c1] = x0 - alpha;
            for (int c = c1 & ~3; c < c1; ++c) a[c] = (T)0;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Semidefinite Cholesky factor of each chain's m x m Gram matrix in shared memory (row
// stride m + 1): pivots below m eps max(diag) zero their column (rank-deficient Grams).
template <typename T, int NT = BT>
__global__ void __launch_bounds__(NT) kb_chol(OpChol<T> op, int n) {
  extern __shared__ __align__(16) unsigned char dyn[];
  T* A = (T*)dyn;
  __shared__ T red[32];
  __shared__ T s_piv[2];
  const int m = op.m, ld = m + 1;
  const T eps = sizeof(T) == 4 ? (T)1.1920929e-7 : (T)2.220446049250313e-16;
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    const T* G = op.G + (long long)s * op.gs;
    T* L = op.Lf + (long long)s * op.ls;
    T dmax = 0;
    for (int i = threadIdx.x; i < m * m; i += NT) {
      const int r = i / m, c = i - r * m;
      const T v = G[i];
      A[r * ld + c] = v;
      if (r == c) dmax = v > dmax ? v : dmax;
    }
    dmax = cta_max(dmax, red);
    const T tol = (T)m * eps * dmax;
    __syncthreads();
    if (threadIdx.x == 0) {
      const T d = A[0];
      s_piv[0] = d > tol ? sqrt(d) : (T)0;
    }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
      const T l = s_piv[j & 1], inv = l > 0 ? (T)1 / l : (T)0;
      for (int i = j + threadIdx.x; i < m; i += NT) A[i * ld + j] = i == j ? l : A[i * ld + j] * inv;
      __syncthreads();
      // trailing update on a TW x TW thread grid (TW = 16 for 256 threads, 32 for 1024);
      // thread 0 updates the next diagonal entry and forms the next pivot, so a column costs
      // two barriers
      constexpr int TW = NT >= 1024 ? 32 : 16;
      const int ty = threadIdx.x / TW, tx = threadIdx.x % TW;
      for (int i = j + 1 + ty; i < m; i += TW) {
        const T lij = A[i * ld + j];
        for (int k = j + 1 + tx; k < m; k += TW) A[i * ld + k] -= lij * A[k * ld + j];
      }
      if (threadIdx.x == 0 && j + 1 < m) {
        const T d = A[(j + 1) * ld + j + 1];
        s_piv[(j + 1) & 1] = d > tol ? sqrt(d) : (T)0;
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < m * m; i += NT) {
      const int r = i / m, c = i - r * m;
      L[i] = c <= r ? A[r * ld + c] : (T)0;
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(BT) kb_trunc(OpTrunc<T> op, int n, long long cap, T* gwork) {
  __shared__ T red[32];
  __shared__ int flag;
  extern __shared__ __align__(16) unsigned char dyn[];
  // Jacobi matrices in shared memory, or, when they do not fit (gwork given), in this
  // block's slice of a global work area (cached in L2)
  T* smem = gwork ? gwork + (long long)blockIdx.x * cap : (T*)dyn;
  T* sig = gwork ? (T*)dyn : smem + cap;
  int* order = (int*)(sig + op.nc + 4);
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    op(s, red, &flag, smem, cap, order, sig, BT);   // the pairing of a 256-thread block
    __syncthreads();
  }
}

// The truncation of float data with a float64 working copy (rotations, singular values and
// vectors in float64): the matrices in shared memory, or, with gwork, in this block's slice
// of a global float64 work area.
template <typename T>
__global__ void __launch_bounds__(BT) kb_trunc64(OpTrunc<T> op, int n, long long cap, double* gwork,
                                                 double tol) {
  __shared__ double red[32];
  __shared__ int flag;
  extern __shared__ __align__(16) unsigned char dyn[];
  double* smem = gwork ? gwork + (long long)blockIdx.x * cap : (double*)dyn;
  double* sig = gwork ? (double*)dyn : smem + cap;
  int* order = (int*)(sig + op.nc + 4);
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    op.template run<double>(s, red, &flag, smem, order, sig, BT, tol);
    __syncthreads();
  }
}

// Truncation of a tall bond (no rotations to accumulate) with its Jacobi matrix in shared
// memory, one 1024-thread block per SM: the column pairs of a round are spread over all
// threads and every round runs at shared-memory latency.
template <typename T>
__global__ void __launch_bounds__(1024) kb_trunc_wide(OpTrunc<T> op, int n) {
  __shared__ T red[32];
  __shared__ int flag;
  extern __shared__ __align__(16) unsigned char dyn[];
  const long long cap = (long long)op.nc * (op.len | 1);
  T* smem = (T*)dyn;
  T* sig = smem + cap;
  int* order = (int*)(sig + op.nc + 4);
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    op(s, red, &flag, smem, cap, order, sig);
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(BT) kb_norm(OpNorm<T> op, int n) {
  __shared__ T red[32];
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    op(s, red);
    __syncthreads();
  }
}

// One warp per sample.
template <typename T>
__global__ void __launch_bounds__(256) kb_dot(OpDot<T> op, int n) {
  int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (s >= n) return;
  const T* a = op.a + (long long)s * op.as;
  const T* b = op.b + (long long)s * op.bs;
  T acc = 0;
  for (long long k = lane; k < op.len; k += 32) acc += a[k] * b[k];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) op.out[s] = acc;
}

template <typename F>
__global__ void kb_elem(F f, int n) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) f(s);
}

template <typename T>
__global__ void kb_set(T* x, long long xs, long long off, T v, int n) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) x[(long long)s * xs + off] = v;
}

__global__ void kb_fill_u8(uint8_t* x, uint8_t v, long long count) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < count;
       k += (long long)gridDim.x * blockDim.x)
    x[k] = v;
}

__global__ void kb_bcastd(double* x, long long xs, long long len, int n) {
  const int s = blockIdx.y + 1;
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n && k < len) x[(long long)s * xs + k] = x[k];
}

__global__ void kb_copyd(double* x, long long xs, int dst, int src, int n) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) x[(long long)s * xs + dst] = x[(long long)s * xs + src];
}

template <typename T>
__global__ void kb_copy(T* dst, long long ds, const T* src, long long ss, long long len,
                        const int8_t* mask, int n) {
  int s = blockIdx.y;
  if (s >= n || (mask && !mask[s])) return;
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < len) dst[(long long)s * ds + k] = src[(long long)s * ss + k];
}

template <typename T, typename OT>
__global__ void kb_O(OT* O, long long No, long long o_off, const T* env, long long es,
                     long long sz, const T* val, long long vs, int n) {
  int s = blockIdx.y;
  if (s >= n) return;
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < sz) O[(long long)s * No + o_off + k] = (OT)((double)env[(long long)s * es + k] / (double)val[(long long)s * vs]);
}

// Longest contraction of the FFMA GEMM: its per-K offset tables and 24 KB of operand tiles
// stay within the 96 KB of dynamic shared memory the kernel is given (kb_ein otherwise).
constexpr int FFMA_K_MAX = 8192;

// Launch-shape parameters of the batched engine, chosen by the autotuner; none of them
// changes any result (each chain's arithmetic is the same in every choice).
struct BatchTune {
  int grid_pct = 100;          // persistent tensor-core grid, per cent of the resident CTAs
  int db_bytes = 12 * 1024;    // largest operand stage that gets two stages
  int ffma_g = 256;            // most chains per block of the FFMA GEMM
  int kc_max = 64;             // largest contraction chunk of the tensor-core GEMM
  int pipelined = 1;           // tensor-core GEMM on the cp.async pipeline (kb_gemm_tc2): 0 none,
                               // 1 short vector contractions (K <= 64), 2 every vector one
  int stage_budget = 96 * 1024;   // ... bytes of copy stages per CTA
  int trunc_threads = 64;      // threads of a Jacobi truncation block (32..256) when its
                               // matrix is in shared memory (the same bits for each)
};

// Whether two operands address the same values for every chain.
template <typename T>
inline bool op_same(const Operand<T>& a, const Operand<T>& b) {
  if (a.base != b.base || a.mode != b.mode) return false;
  if (a.mode == OP_BATCH) return a.stride == b.stride;
  return a.site_off == b.site_off && a.site_sz == b.site_sz && a.S == b.S && a.site == b.site &&
         a.N == b.N && a.sel == b.sel;
}

// Whether every chain's slice of a float operand starts on a 16-byte boundary.
inline bool op_al16(const Operand<float>& o) {
  if ((uintptr_t)o.base % 16) return false;
  if (o.mode == OP_BATCH) return o.stride % 4 == 0;
  return o.site_off % 4 == 0 && o.site_sz % 4 == 0;
}

// Launch back end of the batched runner: one kernel per batched operation on `stream`.
template <typename T, typename OT>
struct CudaBE {
  cudaStream_t st;
  const int *bi, *bj;
  const double* bJ;
  int nb, N;
  long long trunc_cap;   // elements of the Jacobi work area of one block
  bool trunc64 = false;          // float data truncated with a float64 working copy
  double* trunc_g64 = nullptr;   // its global work area (8 blocks per SM x trunc_cap)
  double jtol64 = 1e-15;         // its Jacobi tolerance
  T* trunc_g = nullptr;  // global Jacobi work area (gblocks(n) blocks) when shared memory is too small
  int sms;
  int lq_smem_max = 0;   // bytes of shared memory the Householder kernel may take
  int lq2_smem_max = 0;  // ... and its shared-memory variant (kb_lq2; 0: not used)
  int trunc_wide_max = 0;  // shared memory kb_trunc_wide may take (0: not used)
  int chol_wide_max = 0;   // shared memory the 1024-thread kb_chol may take (0: not used)
  bool tc = false;       // float32: GEMM-shaped contractions on the tensor cores (TF32)
  bool tc_split = false; // ... with every operand split into two TF32 parts (3xTF32)
  int tc_min_rows = 64;  // smallest larger free side sent to the tensor cores
  BatchTune tune;        // launch shapes (autotuned; results do not depend on them)
  int* tc_err = nullptr; // raised by a tensor-core kernel whose completion wait ran out
  void (*tc_form_override)(TcSpec&) = nullptr;   // test hook: restrict the operand forms
  KProf* prof = nullptr; // launch counter and optional per-kernel timing

  // Algorithmic bytes of one batched contraction: each chain's operand slices read once
  // (a site tensor once per local index in use), the output written once.
  static double ein_bytes(const Spec& s, const Operand<T>& A, const Operand<T>& B, int n) {
    double a = 1, b = 1, c = 1;
    for (int d = 0; d < s.no; ++d) {
      c *= s.os[d];
      if (s.ao[d]) a *= s.os[d];
      if (s.bo[d]) b *= s.os[d];
    }
    for (int d = 0; d < s.nk; ++d) {
      a *= s.ks[d];
      b *= s.ks[d];
    }
    const double sites = n < 4 ? n : 4;
    if (op_same(A, B) && a == b) b = 0;   // a Gram product reads its operand once
    return (a * (A.mode == OP_BATCH ? n : sites) + b * (B.mode == OP_BATCH ? n : sites) + c * n) *
           sizeof(T);
  }
  int tc2_regs = 0;
  int tc2_reg_limit() {
    if (!tc2_regs) {
      cudaFuncAttributes fa;
      int regs = 64;
      if (cudaFuncGetAttributes(&fa, kb_gemm_tc2) == cudaSuccess && fa.numRegs > 0) regs = fa.numRegs;
      else cudaGetLastError();
      regs = (regs + 7) & ~7;
      int lim = 65536 / (regs * TC_THREADS);
      lim = lim > 2048 / TC_THREADS ? 2048 / TC_THREADS : lim;
      tc2_regs = lim < 1 ? 1 : lim;
    }
    return tc2_regs;
  }
  // resident tensor-core GEMM CTAs per SM allowed by registers and threads (cached)
  int tc_by_regs[2] = {0, 0};
  int tc_reg_limit(bool pref) {
    int& lim = tc_by_regs[pref ? 1 : 0];
    if (!lim) {
      cudaFuncAttributes fa;
      int regs = 64;
      cudaError_t e = pref ? cudaFuncGetAttributes(&fa, kb_gemm_tc<true>)
                           : cudaFuncGetAttributes(&fa, kb_gemm_tc<false>);
      if (e == cudaSuccess && fa.numRegs > 0) regs = fa.numRegs;
      else cudaGetLastError();
      regs = (regs + 7) & ~7;   // per-warp allocation granularity
      lim = 65536 / (regs * TC_THREADS);
      if (lim > 2048 / TC_THREADS) lim = 2048 / TC_THREADS;
      if (lim < 1) lim = 1;
    }
    return lim;
  }

  static int gx(long long n, int t) { return (int)((n + t - 1) / t); }
  int gblocks(int n) const { return n < 8 * sms ? n : 8 * sms; }

  void ein(const Spec& raw, const MSpec& m, T* out, long long os, Operand<T> A, Operand<T> B,
           int n, bool exact = false) {
    GSpec gs = gemm_spec(raw);
    if constexpr (std::is_same<T, float>::value) {
      TcSpec t;
      bool swap = false;
      if (tc && tc_plan(gs, t, swap, tc_min_rows)) {
        tc_forms(t, op_al16(swap ? B : A), op_al16(swap ? A : B),
                 ((uintptr_t)out % 16 == 0) && os % 4 == 0);
        t.split = (exact || tc_split) ? 1 : 0;   // float32-accurate products (3xTF32)
        if (tc_form_override) tc_form_override(t);
        t.sym = tc_symmetric(t, op_same(A, B)) ? 1 : 0;
        if (t.Kc > tune.kc_max) {   // smaller chunks: smaller stages, more resident CTAs
          t.Kc = tune.kc_max;
          if (t.K > t.Kc) t.pref = 0;
        }
        // the pipelined kernel wins (measured at the 10x10 D=6 chi=36 shapes) on short
        // contractions (K <= 64) whose operands are both vector copies, and on those of at most
        // 8 indices; element-wise gathers, long and split contractions stay on the
        // register-staged kernel
        const bool vec = t.modeP != TC_SCALAR && t.modeQ != TC_SCALAR;
        if (tune.pipelined && ((vec && !t.split && (t.K <= 64 || tune.pipelined == 2)) || t.K <= 8)) {
          // pipelined kernel: cp.async ring of stages over (chain, contraction chunk) items
          if (t.Kc > tune.kc_max) t.Kc = tune.kc_max;
          tc2_shape(t, (size_t)tune.stage_budget);
          const int tilesM = (t.M + TC_ROWS - 1) / TC_ROWS, tilesN = (t.N + t.TN - 1) / t.TN;
          const size_t bytes = tc2_smem_bytes(t);
          int per_sm = (int)((size_t)(227 * 1024) / (bytes + 1024));
          const int by_tmem = 512 / tc_cols(t.TN * t.nacc);
          const int by_regs = tc2_reg_limit();
          per_sm = per_sm < by_tmem ? per_sm : by_tmem;
          per_sm = per_sm < by_regs ? per_sm : by_regs;
          per_sm = per_sm < 16 ? per_sm : 16;
          per_sm = per_sm < 1 ? 1 : per_sm;
          long long gy = (long long)sms * per_sm * tune.grid_pct / (100LL * tilesM * tilesN);
          gy = gy < 1 ? 1 : (gy > n ? n : gy);
          gy = gy > 65535 ? 65535 : gy;
          dim3 gr(tilesM * tilesN, (unsigned)gy);
          PV_KLAUNCH(prof, st, "kb_gemm_tc2", ein_bytes(raw, A, B, n), 2.0 * raw.total * raw.kprod * n,
                     kb_gemm_tc2<<<gr, TC_THREADS, bytes, st>>>(t, out, os, swap ? B : A, swap ? A : B, n,
                                                                tilesN, tc_err));
          return;
        }
        // stay within the 200 KB of shared memory the kernel is configured for
        const size_t smem_cap = 200 * 1024;
        while (tc_smem_bytes(t) > smem_cap && t.Kc > 8) {
          t.Kc -= 8;
          t.pref = 0;
        }
        {
          // two operand stages and accumulators (consecutive chains pipelined) only for small
          // single-chunk stages: larger ones cost more in resident CTAs than they gain
          t.nst = (t.K <= t.Kc && tc_stage_bytes(t) <= (size_t)tune.db_bytes) ? 2 : 1;
          if (tc_smem_bytes(t) > smem_cap) t.nst = 1;
        }
        if (tc_smem_bytes(t) <= smem_cap) {
          const int tilesM = (t.M + TC_ROWS - 1) / TC_ROWS, tilesN = (t.N + t.TN - 1) / t.TN;
          const size_t bytes = tc_smem_bytes(t);
          // persistent grid of the CTAs that can be resident at once (shared memory, tensor
          // memory columns, registers)
          int per_sm = (int)((size_t)(227 * 1024) / (bytes + 1024));
          int by_tmem = 512 / tc_cols(t.TN * tc_stages(t));
          int by_regs = tc_reg_limit(t.pref != 0);
          per_sm = per_sm < by_tmem ? per_sm : by_tmem;
          per_sm = per_sm < by_regs ? per_sm : by_regs;
          per_sm = per_sm < 16 ? per_sm : 16;
          per_sm = per_sm < 1 ? 1 : per_sm;
          long long gy = (long long)sms * per_sm * tune.grid_pct / (100LL * tilesM * tilesN);
          gy = gy < 1 ? 1 : (gy > n ? n : gy);
          gy = gy > 65535 ? 65535 : gy;
          dim3 gr(tilesM * tilesN, (unsigned)gy);
          if (t.pref)
            PV_KLAUNCH(prof, st, "kb_gemm_tc", ein_bytes(raw, A, B, n), 2.0 * raw.total * raw.kprod * n,
                       kb_gemm_tc<true><<<gr, TC_THREADS, bytes, st>>>(t, out, os, swap ? B : A,
                                                                       swap ? A : B, n, tilesN, tc_err));
          else
            PV_KLAUNCH(prof, st, "kb_gemm_tc", ein_bytes(raw, A, B, n), 2.0 * raw.total * raw.kprod * n,
                       kb_gemm_tc<false><<<gr, TC_THREADS, bytes, st>>>(t, out, os, swap ? B : A,
                                                                        swap ? A : B, n, tilesN, tc_err));
          return;
        }
      }
    }
    if (gs.ok && gs.K > 1 && gs.K <= FFMA_K_MAX) {
      int Np = ((gs.N + 3) / 4) * 4;
      int TN = 4;
      while (TN < Np && TN < 64) TN <<= 1;
      int TM = 4096 / TN;
      int Mp = ((gs.M + 3) / 4) * 4;
      if (Mp < TM) TM = Mp;
      int G = 256 / ((TM / 4) * (TN / 4));   // samples per block when one tile is small
      if (G > tune.ffma_g) G = tune.ffma_g;
      if (G < 1) G = 1;
      int budget = (int)(6144 * 4 / sizeof(T));   // 24 KB of operand tiles
      int KC = budget / (G * (TM + TN));
      KC = KC < 1 ? 1 : (KC > 32 ? 32 : KC);
      if (KC > gs.K) KC = gs.K;
      int tilesN = (gs.N + TN - 1) / TN, tilesM = (gs.M + TM - 1) / TM;
      size_t bytes = (size_t)G * KC * (TM + TN) * sizeof(T) +
                     (size_t)(2 * TM + 2 * TN + 2 * gs.K) * 4;
      int gy = (n + G - 1) / G;
      if (gy > 65535) gy = 65535;
      dim3 gr(tilesN * tilesM, gy);
      PV_KLAUNCH(prof, st, "kb_gemm", ein_bytes(raw, A, B, n), 2.0 * raw.total * raw.kprod * n,
                 kb_gemm<T><<<gr, 256, bytes, st>>>(gs, out, os, A, B, n, TM, TN, KC, tilesN, G));
      return;
    }
    int quad = quad_ok(m) ? 1 : 0;
    long long work = quad ? (m.total >> 2) : m.total;
    dim3 g(gx(work, 256), n);
    PV_KLAUNCH(prof, st, "kb_ein", ein_bytes(raw, A, B, n), 2.0 * raw.total * raw.kprod * n,
               kb_ein<T><<<g, 256, 0, st>>>(m, out, os, A, B, n, quad));
  }
  void lq(OpLq<T> op, int n) {
    const int K = op.m < op.nn ? op.m : op.nn;
    double fl = 0;
    for (int j = 0; j < K; ++j) fl += 4.0 * (op.nn - j) * (op.m - j);
    const double lq_bytes = (double)n * ((double)op.m * op.nn + (double)op.m * K) * sizeof(T);
    // shared-memory factorisation: G threads per row, row stride ld = G (mod 32)
    const int G = op.nn >= 128 ? 16 : (op.nn >= 32 ? 8 : 4);
    const int ld = op.nn + ((G - op.nn % 32) % 32 + 32) % 32;
    const size_t bytes2 = (size_t)op.m * ld * sizeof(T);
    if (op.nn % 4 == 0 && bytes2 <= (size_t)lq2_smem_max) {
      int per_sm = (int)((size_t)(227 * 1024) / (bytes2 + 1024));
      per_sm = per_sm < 2048 / LQ_THREADS ? per_sm : 2048 / LQ_THREADS;
      per_sm = per_sm < 1 ? 1 : per_sm;
      const int grid = n < sms * per_sm ? n : sms * per_sm;
      PV_KLAUNCH(prof, st, "kb_lq", lq_bytes, fl * n,
                 (kb_lq2<T, LQ_THREADS><<<grid, LQ_THREADS, bytes2, st>>>(op, n, ld, G)));
      return;
    }
    size_t bytes = (size_t)op.m * op.nn * sizeof(T);
    int use = bytes <= (size_t)lq_smem_max ? 1 : 0;
    PV_KLAUNCH(prof, st, "kb_lq", lq_bytes, fl * n,
               kb_lq<T><<<gblocks(n), BT, use ? bytes : 0, st>>>(op, n, use));
  }
  void trunc(OpTrunc<T> op, int n) {
    if (trunc64) {
      const long long need = (long long)op.nc * (op.len | 1) + (op.tall ? 0 : (long long)op.m * (op.m | 1));
      const size_t bytes = (size_t)need * 8 + (size_t)(op.nc + 4) * (8 + sizeof(int)) + 16;
      if (bytes <= 200 * 1024 || !trunc_g64) {
        const int tt = tune.trunc_threads;
        int per_sm = (int)((size_t)(227 * 1024) / (bytes + 1024));
        per_sm = per_sm < 2048 / tt ? per_sm : 2048 / tt;
        per_sm = per_sm < 32 ? per_sm : 32;
        per_sm = per_sm < 1 ? 1 : per_sm;
        const int grid = n < sms * per_sm ? n : sms * per_sm;
        PV_KLAUNCH(prof, st, "kb_trunc", (double)n * 2.0 * op.nc * op.len * sizeof(T), 0.0,
                   kb_trunc64<T><<<grid, tt, bytes, st>>>(op, n, need, nullptr, jtol64));
      } else {
        const size_t b = (size_t)(op.nc + 4) * (8 + sizeof(int)) + 16;
        PV_KLAUNCH(prof, st, "kb_trunc", (double)n * 2.0 * op.nc * op.len * sizeof(T), 0.0,
                   kb_trunc64<T><<<gblocks(n), BT, b, st>>>(op, n, trunc_cap, trunc_g64, jtol64));
      }
      return;
    }
    if (op.tall && trunc_g) {
      // matrices too large for the shared-memory work area of the 256-thread kernel (which
      // would keep them in global memory): one 1024-thread block per SM holds one in shared
      // memory; smaller ones keep eight 256-thread blocks per SM
      const size_t wb = (size_t)op.nc * (op.len | 1) * sizeof(T) + (size_t)(op.nc + 4) * (sizeof(T) + sizeof(int)) + 16;
      if (wb <= (size_t)trunc_wide_max) {
        const int grid = n < sms ? n : sms;
        PV_KLAUNCH(prof, st, "kb_trunc", (double)n * 2.0 * op.nc * op.len * sizeof(T), 0.0,
                   kb_trunc_wide<T><<<grid, 1024, wb, st>>>(op, n));
        return;
      }
    }
    if (!trunc_g) {
      // the matrix (and, for a wide bond, its accumulated right vectors) in shared memory:
      // as many blocks per SM as that memory and the block size allow
      const long long need = (long long)op.nc * (op.len | 1) + (op.tall ? 0 : (long long)op.m * (op.m | 1));
      const size_t bytes = (size_t)need * sizeof(T) + (size_t)(op.nc + 4) * (sizeof(T) + sizeof(int)) + 16;
      const int tt = tune.trunc_threads;
      int per_sm = (int)((size_t)(227 * 1024) / (bytes + 1024));
      per_sm = per_sm < 2048 / tt ? per_sm : 2048 / tt;
      per_sm = per_sm < 32 ? per_sm : 32;
      per_sm = per_sm < 1 ? 1 : per_sm;
      const int grid = n < sms * per_sm ? n : sms * per_sm;
      PV_KLAUNCH(prof, st, "kb_trunc", (double)n * 2.0 * op.nc * op.len * sizeof(T), 0.0,
                 kb_trunc<T><<<grid, tt, bytes, st>>>(op, n, need, nullptr));
      return;
    }
    size_t bytes = (size_t)(op.nc + 4) * sizeof(T) + (size_t)(op.nc + 4) * sizeof(int) + 16;
    PV_KLAUNCH(prof, st, "kb_trunc", (double)n * 2.0 * op.nc * op.len * sizeof(T), 0.0,
               kb_trunc<T><<<gblocks(n), BT, bytes, st>>>(op, n, trunc_cap, trunc_g));
  }
  // Whether an m x m Gram factorisation fits the shared memory of one kb_chol block (the
  // compression takes the Householder factors otherwise).
  bool chol_fits(int m) const {
    const size_t bytes = (size_t)m * (m + 1) * sizeof(T);
    return bytes <= 200 * 1024 || (int)bytes <= chol_wide_max;
  }
  void chol(OpChol<T> op, int n) {
    const size_t bytes = (size_t)op.m * (op.m + 1) * sizeof(T);
    if (bytes > 96 * 1024 && (int)bytes <= chol_wide_max) {
      // at most one block fits per SM: 1024 threads share the trailing updates
      const int grid = n < sms ? n : sms;
      PV_KLAUNCH(prof, st, "kb_chol", (double)n * 2.0 * op.m * op.m * sizeof(T),
                 (double)op.m * op.m * op.m / 3.0 * n,
                 (kb_chol<T, 1024><<<grid, 1024, bytes, st>>>(op, n)));
      return;
    }
    PV_KLAUNCH(prof, st, "kb_chol", (double)n * 2.0 * op.m * op.m * sizeof(T),
               (double)op.m * op.m * op.m / 3.0 * n,
               kb_chol<T><<<gblocks(n), BT, bytes, st>>>(op, n));
  }
  void norm(OpNorm<T> op, int n) { PV_KLAUNCH(prof, st, "kb_norm", 0.0, 0.0, kb_norm<T><<<gblocks(n), BT, 0, st>>>(op, n)); }
  void dot(OpDot<T> op, int n) { PV_KLAUNCH(prof, st, "kb_dot", 0.0, 0.0, kb_dot<T><<<gx(n, 8), 256, 0, st>>>(op, n)); }
  void set(T* x, long long xs, long long off, T v, int n) { PV_KLAUNCH(prof, st, "kb_set", 0.0, 0.0, kb_set<T><<<gx(n, 256), 256, 0, st>>>(x, xs, off, v, n)); }
  void setd(double* x, long long xs, long long off, double v, int n) {
    PV_KLAUNCH(prof, st, "kb_set", 0.0, 0.0, kb_set<double><<<gx(n, 256), 256, 0, st>>>(x, xs, off, v, n));
  }
  // x[s][0..len) = x[0][0..len) for s = 1..n-1
  void bcastd(double* x, long long xs, long long len, int n) {
    if (n <= 1) return;
    dim3 g(gx(len, 128), n - 1);
    PV_KLAUNCH(prof, st, "kb_copyd", 0.0, 0.0, kb_bcastd<<<g, 128, 0, st>>>(x, xs, len, n));
  }
  void copyd(double* x, long long xs, int dst, int src, int n) {
    PV_KLAUNCH(prof, st, "kb_copyd", 0.0, 0.0, kb_copyd<<<gx(n, 256), 256, 0, st>>>(x, xs, dst, src, n));
  }
  void copy_masked(T* dst, long long ds, const T* src, long long ss, long long len,
                   const int8_t* mask, int n) {
    dim3 g(gx(len, 256), n);
    PV_KLAUNCH(prof, st, "kb_copy", 0.0, 0.0, kb_copy<T><<<g, 256, 0, st>>>(dst, ds, src, ss, len, mask, n));
  }
  void diag(const uint8_t* S, int n, double* es, double* ea) {
    PV_KLAUNCH(prof, st, "kb_elem_diag", 0.0, 0.0, kb_elem<<<gx(n, 128), 128, 0, st>>>(ElemDiag{S, N, nb, bi, bj, bJ, es, ea}, n));
  }
  void amp(const T* val, long long vs, const double* lsd, int lstride, double* la, int8_t* sg, int n) {
    PV_KLAUNCH(prof, st, "kb_elem_amp", 0.0, 0.0, kb_elem<<<gx(n, 128), 128, 0, st>>>(ElemAmp<T>{val, vs, lsd, lstride, la, sg}, n));
  }
  void writeO(OT* O, long long No, long long o_off, const T* env, long long es, long long sz,
              const T* val, long long vs, int n) {
    dim3 g(gx(sz, 256), n);
    PV_KLAUNCH(prof, st, "kb_O", 0.0, 0.0, kb_O<T, OT><<<g, 256, 0, st>>>(O, No, o_off, env, es, sz, val, vs, n));
  }
  void sel(ElemSel f, int n) { PV_KLAUNCH(prof, st, "kb_elem_sel", 0.0, 0.0, kb_elem<<<gx(n, 128), 128, 0, st>>>(f, n)); }
  void ratio(const T* num, const T* den, long long dens, const int8_t* valid, double coef,
             double* e, int n) {
    PV_KLAUNCH(prof, st, "kb_elem_ratio", 0.0, 0.0, kb_elem<<<gx(n, 128), 128, 0, st>>>(ElemRatio<T>{num, den, dens, valid, coef, e}, n));
  }
  void accept(ElemAccept<T> f, int n) { PV_KLAUNCH(prof, st, "kb_elem_accept", 0.0, 0.0, kb_elem<<<gx(n, 128), 128, 0, st>>>(f, n)); }
  // direct sampling (pv_direct.cuh): configuration fill, the candidate selector of every
  // chain, and one draw
  void fill_u8(uint8_t* x, uint8_t v, long long count) {
    const long long g = std::min<long long>((count + 255) / 256, 4LL * sms > 0 ? 4LL * sms : 1);
    PV_KLAUNCH(prof, st, "kb_fill", 0.0, 0.0, kb_fill_u8<<<(unsigned)(g > 0 ? g : 1), 256, 0, st>>>(x, v, count));
  }
  void set_i8(int8_t* x, int8_t v, int n) {
    PV_KLAUNCH(prof, st, "kb_set", 0.0, 0.0, kb_set<int8_t><<<gx(n, 256), 256, 0, st>>>(x, 1, 0, v, n));
  }
  template <typename F>
  void draw(F f, int n) { PV_KLAUNCH(prof, st, "kb_elem_draw", 0.0, 0.0, kb_elem<<<gx(n, 128), 128, 0, st>>>(f, n)); }
};

}  // namespace pv
#endif
