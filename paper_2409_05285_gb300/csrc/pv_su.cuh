// Simple-update (SU) warm start of the doubled-lattice PEPS at very high temperature
// (arXiv:2409.05285, App. A: near beta = 0 the state is close to the product state |I>, so a
// bond's environment can be replaced by bond weights, the scheme of PRL 101, 090603; after
// tens to hundreds of SU steps the SR cooling takes over).
//
// Runs on the host: it evolves one state, bond by bond, through small dense factorisations
// (at D = 4 a 64 x 16 reduction per side and a 64 x 64 SVD per bond), work that a GPU would
// spend in launch latency.  The factorisations are the library's one-sided Jacobi
// (pv_coop.cuh) compiled for the host.
//
// One step of length tau applies the bond gate e^{-tau calH_ij} (Eq. 3 for one Heisenberg bond
// of Eq. 12: e^{-tau h} on the system spins times e^{-tau h^T} on the ancilla spins) to every
// nearest-neighbour bond, horizontal bonds row by row and then vertical bonds.  Per bond: the
// weights of the two sites' other bonds are multiplied into their legs and the bond's weight
// into the first site; each side is reduced to its (local index, shared leg) part by a
// one-sided Jacobi factorisation X = Q R; the gate acts on R_A R_B^T; its SVD keeps the D
// largest singular values (above 1e-14 of the largest), which divided by the largest become
// the bond's new weights; the outer weights are divided back out.  theta() multiplies the
// square root of every bond weight into both of its tensors and zero-pads the legs to D.
#ifndef PV_SU_CUH
#define PV_SU_CUH
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "pv_coop.cuh"

namespace pv {

class SimpleUpdate {
 public:
  SimpleUpdate(int L1, int L2, int D, double J1) : L1_(L1), L2_(L2), D_(D), J1_(J1) {
    const int N = L1 * L2;
    site_.resize(N);
    for (Site& s : site_) {
      s.d[0] = s.d[1] = s.d[2] = s.d[3] = 1;
      s.t.assign(4, 0.0);
      s.t[0] = 1.0;   // S = 0: s = s' = up
      s.t[3] = 1.0;   // S = 3: s = s' = down
    }
    lh_.assign((size_t)L1 * L2, std::vector<double>(1, 1.0));
    lv_.assign((size_t)L1 * L2, std::vector<double>(1, 1.0));
  }

  void step(double tau) {
    double gate[256];
    bond_gate(J1_, tau, gate);
    for (int r = 0; r < L1_; ++r)
      for (int c = 0; c + 1 < L2_; ++c) apply_bond(r, c, true, gate);
    for (int r = 0; r + 1 < L1_; ++r)
      for (int c = 0; c < L2_; ++c) apply_bond(r, c, false, gate);
  }

  // Parameters in the lattice layout: per site [4][dl][dr][du][dd], open legs of dimension 1.
  void theta(double* out) const {
    long long off = 0;
    for (int r = 0; r < L1_; ++r)
      for (int c = 0; c < L2_; ++c) {
        const Site& s = site_[r * L2_ + c];
        const int P[4] = {c == 0 ? 1 : D_, c == L2_ - 1 ? 1 : D_, r == 0 ? 1 : D_, r == L1_ - 1 ? 1 : D_};
        const long long sz = (long long)P[0] * P[1] * P[2] * P[3];
        std::fill(out + off, out + off + 4 * sz, 0.0);
        const std::vector<double>* w[4];
        weights(r, c, w);
        for (int S = 0; S < 4; ++S)
          for (int l = 0; l < s.d[0]; ++l)
            for (int rr = 0; rr < s.d[1]; ++rr)
              for (int u = 0; u < s.d[2]; ++u)
                for (int d = 0; d < s.d[3]; ++d) {
                  const double f = std::sqrt((*w[0])[l] * (*w[1])[rr] * (*w[2])[u] * (*w[3])[d]);
                  out[off + (((S * P[0] + l) * P[1] + rr) * P[2] + u) * P[3] + d] =
                      s.at(S, l, rr, u, d) * f;
                }
        off += 4 * sz;
      }
  }

  // Gate e^{-tau calH_ij} on (S_i, S_j), row (S_i', S_j') = 4 S_i' + S_j', S = 2 s + s'.
  // h = J S_i.S_j has eigenvalue J/4 on the triplet and -3J/4 on the singlet, so
  // e^{-tau h} = e^{-tau J/4} (3/4 + S.S) + e^{3 tau J/4} (1/4 - S.S).
  static void bond_gate(double J, double tau, double* G) {
    const double SS[4][4] = {{0.25, 0, 0, 0}, {0, -0.25, 0.5, 0}, {0, 0.5, -0.25, 0}, {0, 0, 0, 0.25}};
    const double et = std::exp(-0.25 * tau * J), es = std::exp(0.75 * tau * J);
    double g[4][4];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        g[a][b] = et * ((a == b ? 0.75 : 0.0) + SS[a][b]) + es * ((a == b ? 0.25 : 0.0) - SS[a][b]);
    for (int Si = 0; Si < 4; ++Si)
      for (int Sj = 0; Sj < 4; ++Sj)
        for (int Ti = 0; Ti < 4; ++Ti)
          for (int Tj = 0; Tj < 4; ++Tj) {
            const int sys = (Si >> 1) * 2 + (Sj >> 1), sys0 = (Ti >> 1) * 2 + (Tj >> 1);
            const int anc = (Si & 1) * 2 + (Sj & 1), anc0 = (Ti & 1) * 2 + (Tj & 1);
            G[(Si * 4 + Sj) * 16 + Ti * 4 + Tj] = g[sys][sys0] * g[anc][anc0];
          }
  }

 private:
  struct Site {
    int d[4];                 // current leg dimensions (l, r, u, d)
    std::vector<double> t;    // [4][d0][d1][d2][d3]
    double at(int S, int l, int r, int u, int d) const {
      return t[(((S * this->d[0] + l) * this->d[1] + r) * this->d[2] + u) * this->d[3] + d];
    }
  };
  int L1_, L2_, D_;
  double J1_;
  std::vector<Site> site_;
  std::vector<std::vector<double>> lh_, lv_;   // bond (r,c)-(r,c+1) and (r,c)-(r+1,c)
  const std::vector<double> one_ = std::vector<double>(1, 1.0);

  void weights(int r, int c, const std::vector<double>** w) const {
    w[0] = c > 0 ? &lh_[r * L2_ + c - 1] : &one_;
    w[1] = c + 1 < L2_ ? &lh_[r * L2_ + c] : &one_;
    w[2] = r > 0 ? &lv_[(r - 1) * L2_ + c] : &one_;
    w[3] = r + 1 < L1_ ? &lv_[r * L2_ + c] : &one_;
  }

  // X[o][(S, k)] of a site: rows the three outer legs (in leg order), columns the local index
  // and the shared leg `sh`; outer legs times their weights, the shared leg times `wk`.
  static void side_matrix(const Site& s, int sh, const std::vector<double>* const* w,
                          const std::vector<double>* wk, std::vector<double>& X, int& rows,
                          int& cols, int* outer) {
    int m = 0;
    for (int k = 0; k < 4; ++k)
      if (k != sh) outer[m++] = k;
    rows = s.d[outer[0]] * s.d[outer[1]] * s.d[outer[2]];
    const int dk = s.d[sh];
    cols = 4 * dk;
    X.assign((size_t)rows * cols, 0.0);
    int ix[4];
    for (int S = 0; S < 4; ++S)
      for (ix[0] = 0; ix[0] < s.d[0]; ++ix[0])
        for (ix[1] = 0; ix[1] < s.d[1]; ++ix[1])
          for (ix[2] = 0; ix[2] < s.d[2]; ++ix[2])
            for (ix[3] = 0; ix[3] < s.d[3]; ++ix[3]) {
              const int o = (ix[outer[0]] * s.d[outer[1]] + ix[outer[1]]) * s.d[outer[2]] + ix[outer[2]];
              double v = s.at(S, ix[0], ix[1], ix[2], ix[3]);
              v *= (*w[outer[0]])[ix[outer[0]]] * (*w[outer[1]])[ix[outer[1]]] * (*w[outer[2]])[ix[outer[2]]];
              if (wk) v *= (*wk)[ix[sh]];
              X[(size_t)o * cols + S * dk + ix[sh]] = v;
            }
  }

  // One-sided Jacobi of the columns of X (rows x cols, row-major): X = Y V^T with orthogonal
  // columns Y_j of norms sig_j.  Returns the columns in order of decreasing norm.
  static void jacobi_cols(const std::vector<double>& X, int rows, int cols, std::vector<double>& Y,
                          std::vector<double>& V, std::vector<double>& sig, std::vector<int>& ord) {
    Y.assign((size_t)cols * rows, 0.0);   // column j at Y + j * rows
    for (int i = 0; i < rows; ++i)
      for (int j = 0; j < cols; ++j) Y[(size_t)j * rows + i] = X[(size_t)i * cols + j];
    V.assign((size_t)cols * cols, 0.0);   // column j at V + j * cols
    for (int j = 0; j < cols; ++j) V[(size_t)j * cols + j] = 1.0;
    int flag = 0, sw = 0;
    double red[2] = {0, 0};
    jacobi(Y.data(), rows, cols, rows, V.data(), cols, cols, 1e-15, 60, &flag, &sw, red);
    sig.assign(cols, 0.0);
    for (int j = 0; j < cols; ++j) {
      double s2 = 0;
      for (int i = 0; i < rows; ++i) s2 += Y[(size_t)j * rows + i] * Y[(size_t)j * rows + i];
      sig[j] = std::sqrt(s2);
    }
    ord.resize(cols);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return sig[a] > sig[b]; });
  }

  void apply_bond(int r, int c, bool horizontal, const double* gate) {
    const int ia = r * L2_ + c, ib = horizontal ? ia + 1 : ia + L2_;
    const int ra_ = horizontal ? r : r + 1, cb = horizontal ? c + 1 : c;
    const int sha = horizontal ? 1 : 3, shb = horizontal ? 0 : 2;
    std::vector<double>& lam = horizontal ? lh_[ia] : lv_[ia];
    const std::vector<double>* wa[4];
    const std::vector<double>* wb[4];
    weights(r, c, wa);
    weights(ra_, cb, wb);
    Site& A = site_[ia];
    Site& B = site_[ib];
    const int dk = A.d[sha];
    // each side reduced to its (S, k) part: X = Q R, R = sig V^T
    std::vector<double> XA, XB, YA, VA, YB, VB, sA, sB;
    std::vector<int> oA, oB;
    int rowsA, colsA, rowsB, colsB, outA[3], outB[3];
    side_matrix(A, sha, wa, &lam, XA, rowsA, colsA, outA);
    side_matrix(B, shb, wb, nullptr, XB, rowsB, colsB, outB);
    jacobi_cols(XA, rowsA, colsA, YA, VA, sA, oA);
    jacobi_cols(XB, rowsB, colsB, YB, VB, sB, oB);
    auto rank = [](const std::vector<double>& s, const std::vector<int>& o) {
      int k = 0;
      while (k < (int)o.size() && s[o[k]] > 1e-14 * s[o[0]] && s[o[k]] > 0) ++k;
      return k;
    };
    const int na = rank(sA, oA), nb = rank(sB, oB);
    if (na == 0 || nb == 0) return;   // a vanishing side: the gate leaves the product zero
    // core: T[(S_A0, a)][(S_B0, b)] = sum_k R_A[a][(S_A0, k)] R_B[b][(S_B0, k)], then the gate
    const int m = 4 * na, n = 4 * nb;
    std::vector<double> Tc((size_t)m * n, 0.0), C((size_t)m * n, 0.0);
    for (int S0 = 0; S0 < 4; ++S0)
      for (int a = 0; a < na; ++a)
        for (int T0 = 0; T0 < 4; ++T0)
          for (int b = 0; b < nb; ++b) {
            double v = 0;
            for (int k = 0; k < dk; ++k)
              v += sA[oA[a]] * VA[(size_t)oA[a] * colsA + S0 * dk + k] * sB[oB[b]] *
                   VB[(size_t)oB[b] * colsB + T0 * dk + k];
            Tc[(size_t)(S0 * na + a) * n + T0 * nb + b] = v;
          }
    for (int S = 0; S < 4; ++S)
      for (int T = 0; T < 4; ++T)
        for (int S0 = 0; S0 < 4; ++S0)
          for (int T0 = 0; T0 < 4; ++T0) {
            const double g = gate[(S * 4 + T) * 16 + S0 * 4 + T0];
            if (g == 0.0) continue;
            for (int a = 0; a < na; ++a)
              for (int b = 0; b < nb; ++b)
                C[(size_t)(S * na + a) * n + T * nb + b] += g * Tc[(size_t)(S0 * na + a) * n + T0 * nb + b];
          }
    // SVD of the core: C = Y V^T, U = Y / sig
    std::vector<double> YC, VC, sC;
    std::vector<int> oC;
    jacobi_cols(C, m, n, YC, VC, sC, oC);
    int kk = 0;
    while (kk < std::min(D_, n) && kk < m && sC[oC[kk]] > 1e-14 * sC[oC[0]]) ++kk;
    kk = std::max(kk, 1);
    const double s0 = sC[oC[0]] > 0 ? sC[oC[0]] : 1.0;
    std::vector<double> lam_new(kk);
    for (int j = 0; j < kk; ++j) lam_new[j] = sC[oC[j]] / s0;
    // new tensors: X_A'[o][(S, k')] = sum_a Q_A[o][a] U[(S, a)][k'], same for B with V
    rebuild(A, sha, outA, wa, rowsA, YA, sA, oA, na, YC, sC, oC, m, kk, true, n, VC);
    rebuild(B, shb, outB, wb, rowsB, YB, sB, oB, nb, YC, sC, oC, m, kk, false, n, VC);
    lam = lam_new;
  }

  void rebuild(Site& s, int sh, const int* outer, const std::vector<double>* const* w, int rows,
               const std::vector<double>& Ys, const std::vector<double>& ss,
               const std::vector<int>& os, int nr, const std::vector<double>& YC,
               const std::vector<double>& sC, const std::vector<int>& oC, int m, int kk, bool left,
               int n, const std::vector<double>& VC) {
    Site out;
    for (int k = 0; k < 4; ++k) out.d[k] = s.d[k];
    out.d[sh] = kk;
    out.t.assign((size_t)4 * out.d[0] * out.d[1] * out.d[2] * out.d[3], 0.0);
    int ix[4];
    for (int S = 0; S < 4; ++S)
      for (int kp = 0; kp < kk; ++kp)
        for (int o = 0; o < rows; ++o) {
          double v = 0;
          for (int a = 0; a < nr; ++a) {
            const double q = Ys[(size_t)os[a] * rows + o] / ss[os[a]];
            const double f = left ? YC[(size_t)oC[kp] * m + S * nr + a] / sC[oC[kp]]
                                  : VC[(size_t)oC[kp] * n + S * nr + a];
            v += q * f;
          }
          ix[outer[2]] = o % s.d[outer[2]];
          ix[outer[1]] = (o / s.d[outer[2]]) % s.d[outer[1]];
          ix[outer[0]] = o / (s.d[outer[2]] * s.d[outer[1]]);
          ix[sh] = kp;
          double wdiv = (*w[outer[0]])[ix[outer[0]]] * (*w[outer[1]])[ix[outer[1]]] *
                        (*w[outer[2]])[ix[outer[2]]];
          out.t[(((S * out.d[0] + ix[0]) * out.d[1] + ix[1]) * out.d[2] + ix[2]) * out.d[3] + ix[3]] =
              wdiv > 0 ? v / wdiv : 0.0;
        }
    s = out;
  }
};

}  // namespace pv
#endif
