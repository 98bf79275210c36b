// Simple-update warm start on the device (arXiv:2409.05285, App. A: near beta = 0 a bond's
// environment is replaced by bond weights, the scheme of PRL 101, 090603).
//
// The same bond update as the host version (pv_su.cuh): weights of the two sites' other
// bonds multiplied into their legs and the bond's weight into the first site; each side
// reduced to its (local index, shared leg) part by one-sided Jacobi, X = Y V^T, R = sig V^T;
// the gate e^{-tau calH_ij} (Eq. 3 for one bond of Eq. 12) on R_A R_B^T; its SVD keeps the D
// largest singular values (above 1e-14 of the largest), which divided by the largest become
// the bond's new weights; the outer weights are divided back out.
//
// Batching: in the horizontal half of a step the bonds of different rows share no site and
// no weight that changes (a row's bonds read only the vertical weights), so every row is one
// thread block that takes its bonds left to right; in the vertical half every column is one
// block that takes its bonds top to bottom.  This is the host's order (horizontal bonds row
// by row, then vertical bonds), so the two give the same state up to the summation order of
// the Jacobi dot products.  A block's work arrays live in global memory (SuScratch).
#ifndef PV_SU_DEV_CUH
#define PV_SU_DEV_CUH
#include <cstdint>

#include "pv_coop.cuh"

#if defined(__CUDACC__)
namespace pv {

// Device state of the simple update: per site a tensor [4][d0][d1][d2][d3] (current leg
// dimensions in dims[4 i + k]) in a slot of 4 D^4 doubles; per bond a weight vector in a
// slot of D doubles and its length.
struct SuDev {
  int L1, L2, D;
  double* T;      // [N][4 D^4]
  int* dims;      // [N][4]
  double* lh;     // [N][D]  bond (r,c)-(r,c+1)
  int* nlh;       // [N]
  double* lv;     // [N][D]  bond (r,c)-(r+1,c)
  int* nlv;       // [N]
  double* gate;   // [256] e^{-tau calH_ij} on (S_i, S_j), row 4 S_i' + S_j'
};

// Work arrays of one block (all sizes from D: rows <= D^3, cols <= 4 D, core <= 16 D square).
struct SuScratch {
  double *XA, *XB, *YA, *YB, *VA, *VB, *sA, *sB, *Tc, *C, *YC, *VC, *sC, *lam;
  int *oA, *oB, *oC;
  static long long doubles(int D) {
    const long long rows = (long long)D * D * D, cols = 4LL * D, core = 16LL * D;
    return 4 * rows * cols + 2 * cols * cols + 2 * cols + 3 * core * core + core * core + core + D;
  }
  static long long ints(int D) { return 2 * 4LL * D + 16LL * D; }
  __device__ void bind(double* d, int* i, int D) {
    const long long rows = (long long)D * D * D, cols = 4LL * D, core = 16LL * D;
    XA = d; d += rows * cols;
    XB = d; d += rows * cols;
    YA = d; d += rows * cols;
    YB = d; d += rows * cols;
    VA = d; d += cols * cols;
    VB = d; d += cols * cols;
    sA = d; d += cols;
    sB = d; d += cols;
    Tc = d; d += core * core;
    C = d; d += core * core;
    YC = d; d += core * core;
    VC = d; d += core * core;
    sC = d; d += core;
    lam = d;
    oA = i; i += 4 * D;
    oB = i; i += 4 * D;
    oC = i;
  }
};

struct SuSide {
  int site, sh, rows, cols, outer[3];
  int d[4];
  const double* w[4];   // weight vectors of the four legs (a unit vector on open edges)
};

__device__ double su_unit_weight = 1.0;   // weight of an open leg (dimension 1)

__device__ const double* su_one() { return &su_unit_weight; }

__device__ void su_weights(const SuDev& s, int r, int c, const double** w) {
  const int L2 = s.L2;
  w[0] = c > 0 ? s.lh + (long long)(r * L2 + c - 1) * s.D : su_one();
  w[1] = c + 1 < L2 ? s.lh + (long long)(r * L2 + c) * s.D : su_one();
  w[2] = r > 0 ? s.lv + (long long)((r - 1) * L2 + c) * s.D : su_one();
  w[3] = r + 1 < s.L1 ? s.lv + (long long)(r * L2 + c) * s.D : su_one();
}

// X[o][(S, k)] of a site: rows the three outer legs (in leg order), columns the local index
// and the shared leg; outer legs times their weights, the shared leg times wk (if given).
__device__ void su_side_matrix(const SuDev& s, SuSide& sd, const double* wk, double* X) {
  const double* t = s.T + (long long)sd.site * 4 * s.D * s.D * s.D * s.D;
  int m = 0;
  for (int k = 0; k < 4; ++k)
    if (k != sd.sh) sd.outer[m++] = k;
  const int* d = sd.d;
  sd.rows = d[sd.outer[0]] * d[sd.outer[1]] * d[sd.outer[2]];
  const int dk = d[sd.sh];
  sd.cols = 4 * dk;
  const int tot = 4 * d[0] * d[1] * d[2] * d[3];
  for (int e = PV_TID; e < tot; e += PV_NTHR) {
    int ix[4], rem = e;
    ix[3] = rem % d[3]; rem /= d[3];
    ix[2] = rem % d[2]; rem /= d[2];
    ix[1] = rem % d[1]; rem /= d[1];
    ix[0] = rem % d[0];
    const int S = rem / d[0];
    const int o = (ix[sd.outer[0]] * d[sd.outer[1]] + ix[sd.outer[1]]) * d[sd.outer[2]] + ix[sd.outer[2]];
    double v = t[e];
    v *= sd.w[sd.outer[0]][ix[sd.outer[0]]] * sd.w[sd.outer[1]][ix[sd.outer[1]]] *
         sd.w[sd.outer[2]][ix[sd.outer[2]]];
    if (wk) v *= wk[ix[sd.sh]];
    X[(long long)o * sd.cols + S * dk + ix[sd.sh]] = v;
  }
  PV_SYNC();
}

// One-sided Jacobi of the columns of X (rows x cols, row-major): X = Y V^T with orthogonal
// columns Y_j (column j at Y + j rows) of norms sig_j; ord lists the columns by decreasing
// norm (ties in index order).
__device__ void su_jacobi_cols(const double* X, int rows, int cols, double* Y, double* V,
                               double* sig, int* ord, int* flag, double* red) {
  for (int e = PV_TID; e < rows * cols; e += PV_NTHR) {
    const int i = e / cols, j = e % cols;
    Y[(long long)j * rows + i] = X[e];
  }
  for (int e = PV_TID; e < cols * cols; e += PV_NTHR) V[e] = (e / cols == e % cols) ? 1.0 : 0.0;
  PV_SYNC();
  int sw = 0;
  jacobi(Y, rows, cols, rows, V, cols, cols, 1e-15, 60, flag, &sw, red);
  for (int j = PV_WARP; j < cols; j += PV_NWARP) {
    double s2 = 0;
    for (int i = PV_LANE; i < rows; i += PV_WSIZE) s2 += Y[(long long)j * rows + i] * Y[(long long)j * rows + i];
    s2 = warp_sum(s2);
    if (PV_LANE == 0) sig[j] = sqrt(s2);
  }
  PV_SYNC();
  for (int j = PV_TID; j < cols; j += PV_NTHR) {
    int rank = 0;
    for (int i = 0; i < cols; ++i) rank += (sig[i] > sig[j] || (sig[i] == sig[j] && i < j)) ? 1 : 0;
    ord[rank] = j;
  }
  PV_SYNC();
}

__device__ int su_rank(const double* s, const int* o, int n) {
  int k = 0;
  while (k < n && s[o[k]] > 1e-14 * s[o[0]] && s[o[k]] > 0) ++k;
  return k;
}

// New tensor of one side: X'[o][(S, k')] = sum_a Q[o][a] F[(S, a)][k'], Q = Y / sig, outer
// weights divided back out; F = U (left side) or V (right side) of the core's SVD.
__device__ void su_rebuild(const SuDev& s, const SuSide& sd, const double* Ys, const double* ss,
                           const int* os, int nr, const SuScratch& w, int m, int n, int kk,
                           bool left) {
  double* t = s.T + (long long)sd.site * 4 * s.D * s.D * s.D * s.D;
  int d[4] = {sd.d[0], sd.d[1], sd.d[2], sd.d[3]};
  d[sd.sh] = kk;
  const int rows = sd.rows;
  const int tot = 4 * kk * rows;
  // the old tensor enters only through Ys (the rotated copy of its side matrix), so the
  // site's slot is overwritten in place
  for (int e = PV_TID; e < tot; e += PV_NTHR) {
    const int o = e % rows, kp = (e / rows) % kk, S = e / (rows * kk);
    double v = 0;
    for (int a = 0; a < nr; ++a) {
      const double q = Ys[(long long)os[a] * rows + o] / ss[os[a]];
      const double f = left ? w.YC[(long long)w.oC[kp] * m + S * nr + a] / w.sC[w.oC[kp]]
                            : w.VC[(long long)w.oC[kp] * n + S * nr + a];
      v += q * f;
    }
    int ix[4];
    ix[sd.outer[2]] = o % d[sd.outer[2]];
    ix[sd.outer[1]] = (o / d[sd.outer[2]]) % d[sd.outer[1]];
    ix[sd.outer[0]] = o / (d[sd.outer[2]] * d[sd.outer[1]]);
    ix[sd.sh] = kp;
    const double wdiv = sd.w[sd.outer[0]][ix[sd.outer[0]]] * sd.w[sd.outer[1]][ix[sd.outer[1]]] *
                        sd.w[sd.outer[2]][ix[sd.outer[2]]];
    t[(((S * d[0] + ix[0]) * d[1] + ix[1]) * d[2] + ix[2]) * d[3] + ix[3]] = wdiv > 0 ? v / wdiv : 0.0;
  }
  PV_SYNC();
  if (PV_TID == 0)
    for (int k = 0; k < 4; ++k) s.dims[4 * sd.site + k] = d[k];
  PV_SYNC();
}

// The gate on one bond (r, c)-(r, c+1) (horizontal) or (r, c)-(r+1, c), by the whole block.
__device__ void su_bond(const SuDev& s, const SuScratch& w, int r, int c, bool horizontal,
                        int* flag, double* red) {
  const int L2 = s.L2;
  const int ia = r * L2 + c, ib = horizontal ? ia + 1 : ia + L2;
  const int rb = horizontal ? r : r + 1, cb = horizontal ? c + 1 : c;
  double* lam = (horizontal ? s.lh : s.lv) + (long long)ia * s.D;
  int* nlam = (horizontal ? s.nlh : s.nlv) + ia;
  SuSide A, B;
  A.site = ia;
  B.site = ib;
  A.sh = horizontal ? 1 : 3;
  B.sh = horizontal ? 0 : 2;
  su_weights(s, r, c, A.w);
  su_weights(s, rb, cb, B.w);
  for (int k = 0; k < 4; ++k) {
    A.d[k] = s.dims[4 * ia + k];
    B.d[k] = s.dims[4 * ib + k];
  }
  const int dk = A.d[A.sh];
  su_side_matrix(s, A, lam, w.XA);
  su_side_matrix(s, B, nullptr, w.XB);
  su_jacobi_cols(w.XA, A.rows, A.cols, w.YA, w.VA, w.sA, w.oA, flag, red);
  su_jacobi_cols(w.XB, B.rows, B.cols, w.YB, w.VB, w.sB, w.oB, flag, red);
  const int na = su_rank(w.sA, w.oA, A.cols), nb = su_rank(w.sB, w.oB, B.cols);
  if (na == 0 || nb == 0) return;   // a vanishing side: the gate leaves the product zero
  const int m = 4 * na, n = 4 * nb;
  // core Tc[(S0, a)][(T0, b)] = sum_k R_A[a][(S0, k)] R_B[b][(T0, k)], then C = gate . Tc
  for (int e = PV_TID; e < m * n; e += PV_NTHR) {
    const int row = e / n, col = e % n;
    const int S0 = row / na, a = row % na, T0 = col / nb, b = col % nb;
    const int ja = w.oA[a], jb = w.oB[b];
    double v = 0;
    for (int k = 0; k < dk; ++k)
      v += w.sA[ja] * w.VA[(long long)ja * A.cols + S0 * dk + k] * w.sB[jb] *
           w.VB[(long long)jb * B.cols + T0 * dk + k];
    w.Tc[e] = v;
  }
  PV_SYNC();
  for (int e = PV_TID; e < m * n; e += PV_NTHR) {
    const int row = e / n, col = e % n;
    const int S = row / na, a = row % na, T = col / nb, b = col % nb;
    double v = 0;
    for (int S0 = 0; S0 < 4; ++S0)
      for (int T0 = 0; T0 < 4; ++T0) {
        const double g = s.gate[(S * 4 + T) * 16 + S0 * 4 + T0];
        if (g != 0.0) v += g * w.Tc[(long long)(S0 * na + a) * n + T0 * nb + b];
      }
    w.C[e] = v;
  }
  PV_SYNC();
  su_jacobi_cols(w.C, m, n, w.YC, w.VC, w.sC, w.oC, flag, red);
  int kk = 0;
  const int kmax = s.D < n ? s.D : n;
  while (kk < kmax && kk < m && w.sC[w.oC[kk]] > 1e-14 * w.sC[w.oC[0]]) ++kk;
  kk = kk > 1 ? kk : 1;
  const double s0 = w.sC[w.oC[0]] > 0 ? w.sC[w.oC[0]] : 1.0;
  su_rebuild(s, A, w.YA, w.sA, w.oA, na, w, m, n, kk, true);
  su_rebuild(s, B, w.YB, w.sB, w.oB, nb, w, m, n, kk, false);
  for (int j = PV_TID; j < kk; j += PV_NTHR) lam[j] = w.sC[w.oC[j]] / s0;
  if (PV_TID == 0) *nlam = kk;
  PV_SYNC();
}

constexpr int SU_THREADS = 256;

// One half of an SU step: block b takes row b's horizontal bonds (horizontal) or column b's
// vertical bonds, in order.
__global__ void __launch_bounds__(SU_THREADS) k_su_half(SuDev s, double* wd, int* wi,
                                                        long long wds, long long wis,
                                                        int horizontal) {
  __shared__ double red[SU_THREADS / 32];
  __shared__ int flag;
  SuScratch w;
  w.bind(wd + (long long)blockIdx.x * wds, wi + (long long)blockIdx.x * wis, s.D);
  if (horizontal) {
    const int r = blockIdx.x;
    for (int c = 0; c + 1 < s.L2; ++c) su_bond(s, w, r, c, true, &flag, red);
  } else {
    const int c = blockIdx.x;
    for (int r = 0; r + 1 < s.L1; ++r) su_bond(s, w, r, c, false, &flag, red);
  }
}

// The beta = 0 state: every leg of dimension 1, G^S = delta_{s s'}, unit weights.
__global__ void k_su_init(SuDev s) {
  const int N = s.L1 * s.L2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double* t = s.T + (long long)i * 4 * s.D * s.D * s.D * s.D;
    t[0] = 1.0;   // S = 0: s = s' = up
    t[1] = 0.0;
    t[2] = 0.0;
    t[3] = 1.0;   // S = 3: s = s' = down
    for (int k = 0; k < 4; ++k) s.dims[4 * i + k] = 1;
    s.lh[(long long)i * s.D] = 1.0;
    s.lv[(long long)i * s.D] = 1.0;
    s.nlh[i] = 1;
    s.nlv[i] = 1;
  }
}

// Parameters of the lattice layout (per site [4][dl][dr][du][dd], open legs of dimension 1,
// legs zero-padded to D): sqrt of every bond weight multiplied into both of its tensors.
__global__ void k_su_theta(SuDev s, const long long* __restrict__ toff, double* __restrict__ theta) {
  const int N = s.L1 * s.L2;
  const int i = blockIdx.x;
  if (i >= N) return;
  const int r = i / s.L2, c = i % s.L2;
  const int P[4] = {c == 0 ? 1 : s.D, c == s.L2 - 1 ? 1 : s.D, r == 0 ? 1 : s.D, r == s.L1 - 1 ? 1 : s.D};
  const int sz = P[0] * P[1] * P[2] * P[3];
  const double* w[4];
  su_weights(s, r, c, w);
  const int* d = s.dims + 4 * i;
  const double* t = s.T + (long long)i * 4 * s.D * s.D * s.D * s.D;
  double* out = theta + toff[i];
  for (int e = threadIdx.x; e < 4 * sz; e += blockDim.x) {
    int ix[4], rem = e;
    ix[3] = rem % P[3]; rem /= P[3];
    ix[2] = rem % P[2]; rem /= P[2];
    ix[1] = rem % P[1]; rem /= P[1];
    ix[0] = rem % P[0];
    const int S = rem / P[0];
    double v = 0.0;
    if (ix[0] < d[0] && ix[1] < d[1] && ix[2] < d[2] && ix[3] < d[3]) {
      const double f = sqrt(w[0][ix[0]] * w[1][ix[1]] * w[2][ix[2]] * w[3][ix[3]]);
      v = t[(((S * d[0] + ix[0]) * d[1] + ix[1]) * d[2] + ix[2]) * d[3] + ix[3]] * f;
    }
    out[e] = v;
  }
}

}  // namespace pv
#endif  // __CUDACC__
#endif
