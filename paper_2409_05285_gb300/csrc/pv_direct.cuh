// Reweighted direct sampling (arXiv:2409.05285, App. A, Eqs. A2-A7) on the batched engine.
//
// The sums of rho(S)^2 over unsampled sites are contractions of the double-layer network,
// which is a single-layer network with bonds D^2 and five local tensors per site: the four
// T^S (x) T^S of a sampled site and their sum for an unsampled one (double_layer_theta).  So
// a BatchRunner built for bond dimension D^2 over those tensors draws the samples with the
// operations it already has:
//   * the down environments of the all-summed rows (local index 4 everywhere; the same for
//     every chain, so built for one and copied);
//   * row by row, the right partials of the one-row strip with the row still summed, then
//     per site the four candidates' strip values (left partial x candidate x right partial),
//     one elementwise draw (ElemDraw), and the left partial extended by the drawn tensor;
//   * the sampled row absorbed into the up environment and truncated to chi.
// Site order is row-major.  p_4c(s) = b(s) p_2c(s)^exponent (exponent 1/2 in Eq. A4, 1 for
// plain direct sampling; b = b_d on the diagonal states s = s', 1 otherwise, Eq. A5); a
// site is drawn from p_4c normalised over its four states by inverse CDF with the caller's
// uniform, and log q(S) (the sum of the logs of the normalised probabilities drawn) is
// returned for the weight r_4 = p_0 / q of Eq. A7.  Candidate values that truncation leaves
// slightly negative count as zero.
//
// This header holds the orchestration and the per-chain functor; a back end provides
// fill_u8(x, v, count), set_i8(x, v, n) and draw(ElemDraw, n) besides the BatchRunner
// operations, and every pointer handed to direct_draw lives where its kernels run.
#ifndef PV_DIRECT_CUH
#define PV_DIRECT_CUH
#include <cmath>
#include <vector>

#include "pv_batch.cuh"

namespace pv {

// Double-layer site tensors: per site [5][dl^2][dr^2][du^2][dd^2], slice s < 4 the product
// T^s (x) T^s with fused legs (a, a') -> a * d + a', slice 4 the sum of the four.  `theta`
// and `out` in the lattice layouts at D and at D^2 (offsets toff and toff2).
template <typename T>
inline void double_layer_theta(int L1, int L2, int D, const T* theta, T* out) {
  long long off = 0, off2 = 0;
  for (int r = 0; r < L1; ++r)
    for (int c = 0; c < L2; ++c) {
      const int d[4] = {c == 0 ? 1 : D, c == L2 - 1 ? 1 : D, r == 0 ? 1 : D, r == L1 - 1 ? 1 : D};
      const long long sz = (long long)d[0] * d[1] * d[2] * d[3], sz2 = sz * sz;
      for (long long e = 0; e < 5 * sz2; ++e) out[off2 + e] = 0;
      for (int s = 0; s < 4; ++s)
        for (int l = 0; l < d[0]; ++l)
          for (int L = 0; L < d[0]; ++L)
            for (int rr = 0; rr < d[1]; ++rr)
              for (int R = 0; R < d[1]; ++R)
                for (int u = 0; u < d[2]; ++u)
                  for (int U = 0; U < d[2]; ++U)
                    for (int dd = 0; dd < d[3]; ++dd)
                      for (int DD = 0; DD < d[3]; ++DD) {
                        const T a = theta[off + s * sz + ((l * d[1] + rr) * d[2] + u) * d[3] + dd];
                        const T b = theta[off + s * sz + ((L * d[1] + R) * d[2] + U) * d[3] + DD];
                        const long long i2 = (((long long)(l * d[0] + L) * (d[1] * d[1]) + rr * d[1] + R) *
                                                  (d[2] * d[2]) + u * d[2] + U) * (d[3] * d[3]) + dd * d[3] + DD;
                        out[off2 + s * sz2 + i2] = a * b;
                        out[off2 + 4 * sz2 + i2] += a * b;
                      }
      off += 4 * sz;
      off2 += 5 * sz2;
    }
}

// Draw of site i for every chain from the four candidate values w0..w3 (see the header).
template <typename T>
struct ElemDraw {
  uint8_t* S;
  int N, i;
  const T *w0, *w1, *w2, *w3;
  double b_d, expo;
  const double* u;   // [n][N] uniforms
  double* logq;
  PV_HD void operator()(int s) const {
    double w[4] = {(double)w0[s], (double)w1[s], (double)w2[s], (double)w3[s]};
    double tot = 0;
    for (int k = 0; k < 4; ++k) tot += w[k] > 0 ? w[k] : 0.0;
    double p[4], z = 0;
    for (int k = 0; k < 4; ++k) {
      const double p2 = tot > 0 && w[k] > 0 ? w[k] / tot : 0.0;
      p[k] = (k == 0 || k == 3 ? b_d : 1.0) * (p2 > 0 ? pow(p2, expo) : 0.0);
      z += p[k];
    }
    int pick = 3;
    if (z > 0) {
      const double x = u[(long long)s * N + i] * z;
      double acc = 0;
      pick = -1;
      for (int k = 0; k < 4; ++k) {
        acc += p[k];
        if (pick < 0 && x < acc) pick = k;
      }
      if (pick < 0) pick = 3;
      while (pick > 0 && p[pick] == 0.0) --pick;
      logq[s] += log(p[pick] / z);
    }
    S[(long long)s * N + i] = (uint8_t)pick;
  }
};

// One direct draw of every chain.  `run` is a BatchRunner built for bond dimension D^2 over
// double-layer tensors (its theta and toff); S [n][N] is overwritten with the samples (local
// indices 0..3), logq [n] receives log q(S).
template <typename T, typename BE, typename OT>
void direct_draw(BatchRunner<T, BE, OT>& run, uint8_t* S, int n, const double* u, double b_d,
                 double expo, double* logq) {
  BE& be = run.be;
  auto& b = run.b;
  const int L1 = run.L1, L2 = run.L2, N = run.N;
  be.fill_u8(S, 4, (long long)n * N);   // every site summed
  be.setd(logq, 1, 0, 0.0, n);
  run.build_down(S, 1);   // every chain's down environments are the same: build one, copy
  run.broadcast_down(n);
  run.trivial(run.uprow(0), b.sU, n);
  be.setd(b.lsU, 1, 0, 0.0, n);
  T* cand[4] = {b.val, b.num, b.den, b.val2};
  for (int r = 0; r < L1; ++r) {
    be.set(b.p1R, b.sp1R, (long long)L2 * b.P1, (T)1, n);
    for (int c = L2 - 1; c >= 0; --c)
      run.s1_right(r, c, run.p1R(c), b.sp1R, run.bat(run.p1R(c + 1), b.sp1R), run.site(r, c, S), n);
    T* Lc = b.p1L;
    T* Ln = b.p1L + b.P1;
    be.set(b.p1L, b.sp1L, 0, (T)1, n);
    for (int c = 0; c < L2; ++c) {
      const int i = r * L2 + c;
      for (int s = 0; s < 4; ++s) {
        be.set_i8(b.si, (int8_t)s, n);
        run.s1_left(r, c, b.m2, b.P2, run.bat(Lc, b.sp1L), run.site_sel(r, c, b.si), n);
        be.dot(OpDot<T>{b.m2, b.P2, run.p1R(c + 1), b.sp1R, run.s1_len(r, c + 1), cand[s]}, n);
      }
      be.draw(ElemDraw<T>{S, N, i, cand[0], cand[1], cand[2], cand[3], b_d, expo, u, logq}, n);
      run.s1_left(r, c, Ln, b.sp1L, run.bat(Lc, b.sp1L), run.site(r, c, S), n);
      T* t = Lc;
      Lc = Ln;
      Ln = t;
    }
    if (r + 1 < L1)
      run.compress(run.uprow(r), b.sU, run.shp.up[r], false, r, S, run.uprow(r + 1), b.sU, b.lsU, 1, n);
  }
}

}  // namespace pv
#endif
