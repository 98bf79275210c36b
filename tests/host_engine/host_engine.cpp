// Host build of the batched engine's orchestration (BatchRunner from pv_batch.cuh) over a
// plain-loop back end, in float64.  Test infrastructure only: it runs the engine's sequence of
// batched operations (environments, compression, strips, ratios, O rows, Metropolis moves) on
// the CPU so that tests/test_host_engine.py can check that sequence against the oracle
// without a GPU.  The operations use the same per-chain functors the device kernels call
// (ein_one, OpLq, OpTrunc, OpNorm, OpDot, Elem*); the GPU-only kernels (tensor-core and FFMA
// GEMMs, shared-memory Householder, Cholesky) are not part of this build (the Gram path's
// Cholesky is a plain loop here).
//
// Usage: host_engine <in.bin> <out.bin>
//   in:  int32 mode (0 eval, 1 one Metropolis sweep, 2 one direct draw, 3 eval with the
//        compression's right factors from Gram matrices, 4 plain amplitude and O rows of a
//        PEPS of 32 slices per site, the fermionic engine's form, 5 one fermionic Metropolis
//        sweep on cached strips over 64 slices per site, 6 fermionic local energies on
//        strips over 64 slices per site, 7 as 6 with the O rows in the same pass; t, U, mu in
//        place of J1, J2 and seed), L1, L2, D, chi, n, p;
//        float64 J1, J2; uint64 seed; int32 sweep; float64 theta[N_p]; uint8 S[n][N];
//        mode 2 only: float64 b_d, exponent, u[n][N]
//   out: eval: float64 log_abs[n], int8 sign[n], float64 e_sys[n], e_anc[n], O[n][N_o]
//        mc:   uint8 S[n][N], int32 acc[n], int32 prop[n]
//        draw: uint8 S[n][N], float64 log_q[n]  (direct sampling, pv_direct.cuh)
//        mode 4: float64 log_abs[n], int8 sign[n], O[n][N_o]  (pv_fermion.cuh)
//        mode 5: uint8 S[n][N], int32 acc[n]  (fermion_mc, pv_fermion.cuh)
//        mode 6: float64 log_abs[n], int8 sign[n], float64 e_sys[n], e_anc[n]  (fermion_eloc)
//        mode 7: as mode 6, then float64 O[n][N_o]  (fermion_eval)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "pv_direct.cuh"
#include "pv_fermion.cuh"

using namespace pv;
using T = double;

struct HostBE {
  static constexpr bool host_loops = true;   // per-chain functors run as plain loops
  int N = 0, nb = 0;
  const int* bi = nullptr;
  const int* bj = nullptr;
  const double* bJ = nullptr;
  long long trunc_cap = 0;
  std::vector<T> red = std::vector<T>(64), work, sig;
  std::vector<int> order;

  void ein(const Spec&, const MSpec& m, T* out, long long os, Operand<T> A, Operand<T> B, int n,
           bool) {
    for (int s = 0; s < n; ++s)
      for (int idx = 0; idx < m.total; ++idx) ein_one(m, out + (long long)s * os, A.at(s), B.at(s), idx);
  }
  void lq(OpLq<T> op, int n) {
    for (int s = 0; s < n; ++s) op(s, red.data());
  }
  void trunc(OpTrunc<T> op, int n) {
    work.assign((size_t)trunc_cap, 0.0);
    sig.assign((size_t)op.nc + 4, 0.0);
    order.assign((size_t)op.nc + 4, 0);
    int flag = 0;
    for (int s = 0; s < n; ++s) op(s, red.data(), &flag, work.data(), trunc_cap, order.data(), sig.data());
  }
  // Semidefinite Cholesky of each chain's m x m Gram matrix, lower factor Lf (pivots below
  // m eps max(diag) zero their column), as the Gram path of the compression expects.
  bool chol_fits(int) const { return true; }
  void chol(OpChol<T> op, int n) {
    const int m = op.m;
    const T eps = 2.220446049250313e-16;
    std::vector<T> A((size_t)m * m);
    for (int s = 0; s < n; ++s) {
      const T* G = op.G + (long long)s * op.gs;
      T dmax = 0;
      for (int i = 0; i < m * m; ++i) A[i] = G[i];
      for (int i = 0; i < m; ++i) dmax = std::max(dmax, A[(size_t)i * m + i]);
      const T tol = (T)m * eps * dmax;
      for (int j = 0; j < m; ++j) {
        const T d = A[(size_t)j * m + j];
        const T l = d > tol ? std::sqrt(d) : (T)0, inv = l > 0 ? (T)1 / l : (T)0;
        for (int i = j; i < m; ++i) A[(size_t)i * m + j] = i == j ? l : A[(size_t)i * m + j] * inv;
        for (int i = j + 1; i < m; ++i)   // trailing update of the lower triangle
          for (int k = j + 1; k <= i; ++k) A[(size_t)i * m + k] -= A[(size_t)i * m + j] * A[(size_t)k * m + j];
      }
      T* L = op.Lf + (long long)s * op.ls;
      for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c) L[(size_t)r * m + c] = c <= r ? A[(size_t)r * m + c] : (T)0;
    }
  }
  void norm(OpNorm<T> op, int n) {
    for (int s = 0; s < n; ++s) op(s, red.data());
  }
  void dot(OpDot<T> op, int n) {
    for (int s = 0; s < n; ++s) op(s, red.data());
  }
  void set(T* x, long long xs, long long off, T v, int n) {
    for (int s = 0; s < n; ++s) x[(long long)s * xs + off] = v;
  }
  void setd(double* x, long long xs, long long off, double v, int n) {
    for (int s = 0; s < n; ++s) x[(long long)s * xs + off] = v;
  }
  void bcastd(double* x, long long xs, long long len, int n) {
    for (int s = 1; s < n; ++s)
      for (long long k = 0; k < len; ++k) x[(long long)s * xs + k] = x[k];
  }
  void copyd(double* x, long long xs, int dst, int src, int n) {
    for (int s = 0; s < n; ++s) x[(long long)s * xs + dst] = x[(long long)s * xs + src];
  }
  void copy_masked(T* dst, long long ds, const T* src, long long ss, long long len,
                   const int8_t* mask, int n) {
    for (int s = 0; s < n; ++s)
      if (!mask || mask[s])
        for (long long k = 0; k < len; ++k) dst[(long long)s * ds + k] = src[(long long)s * ss + k];
  }
  void diag(const uint8_t* S, int n, double* es, double* ea) {
    ElemDiag f{S, N, nb, bi, bj, bJ, es, ea};
    for (int s = 0; s < n; ++s) f(s);
  }
  void amp(const T* val, long long vs, const double* lsd, int lstride, double* la, int8_t* sg,
           int n) {
    ElemAmp<T> f{val, vs, lsd, lstride, la, sg};
    for (int s = 0; s < n; ++s) f(s);
  }
  void writeO(T* O, long long No, long long o_off, const T* env, long long es, long long sz,
              const T* val, long long vs, int n) {
    for (int s = 0; s < n; ++s)
      for (long long k = 0; k < sz; ++k)
        O[(long long)s * No + o_off + k] = env[(long long)s * es + k] / val[(long long)s * vs];
  }
  void sel(ElemSel f, int n) {
    for (int s = 0; s < n; ++s) f(s);
  }
  void ratio(const T* num, const T* den, long long dens, const int8_t* valid, double coef,
             double* e, int n) {
    ElemRatio<T> f{num, den, dens, valid, coef, e};
    for (int s = 0; s < n; ++s) f(s);
  }
  void accept(ElemAccept<T> f, int n) {
    for (int s = 0; s < n; ++s) f(s);
  }
  void set_i8(int8_t* x, int8_t v, int n) {
    for (int s = 0; s < n; ++s) x[s] = v;
  }
  void fill_u8(uint8_t* x, uint8_t v, long long count) {
    for (long long k = 0; k < count; ++k) x[k] = v;
  }
  void draw(ElemDraw<T> f, int n) {
    for (int s = 0; s < n; ++s) f(s);
  }
};

template <typename X>
static void rd(FILE* f, X* p, size_t n) {
  if (std::fread(p, sizeof(X), n, f) != n) {
    std::fprintf(stderr, "host_engine: short input\n");
    std::exit(2);
  }
}

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* fi = std::fopen(argv[1], "rb");
  if (!fi) return 2;
  int32_t hdr[7];
  rd(fi, hdr, 7);
  const int mode = hdr[0], L1 = hdr[1], L2 = hdr[2], D = hdr[3], chi = hdr[4], n = hdr[5], p = hdr[6];
  double J[2];
  rd(fi, J, 2);
  uint64_t seed;
  rd(fi, &seed, 1);
  int32_t sweep;
  rd(fi, &sweep, 1);
  const int N = L1 * L2;
  std::vector<long long> toff(N + 1, 0), ooff(N + 1, 0);
  const int slices = mode == 4 ? 32 : (mode >= 5 && mode <= 7) ? 64 : 4;
  for (int i = 0; i < N; ++i) {
    const int r = i / L2, c = i % L2;
    const long long sz = (long long)(c == 0 ? 1 : D) * (c == L2 - 1 ? 1 : D) * (r == 0 ? 1 : D) *
                         (r == L1 - 1 ? 1 : D);
    toff[i + 1] = toff[i] + slices * sz;
    ooff[i + 1] = ooff[i] + sz;
  }
  std::vector<T> theta((size_t)toff[N]);
  rd(fi, theta.data(), theta.size());
  std::vector<uint8_t> S((size_t)n * N);
  rd(fi, S.data(), S.size());
  double bx[2] = {1.0, 0.5};
  std::vector<double> u;
  if (mode == 2) {
    rd(fi, bx, 2);
    u.resize((size_t)n * N);
    rd(fi, u.data(), u.size());
  }
  std::fclose(fi);
  // direct sampling contracts the double-layer network: bond D^2, five local tensors per site
  const int Dn = mode == 2 ? D * D : D;
  std::vector<T> theta2;
  if (mode == 2) {
    toff.assign(N + 1, 0);
    for (int i = 0; i < N; ++i) {
      const int r = i / L2, c = i % L2;
      const long long sz = (long long)(c == 0 ? 1 : Dn) * (c == L2 - 1 ? 1 : Dn) * (r == 0 ? 1 : Dn) *
                           (r == L1 - 1 ? 1 : Dn);
      toff[i + 1] = toff[i] + 5 * sz;
    }
    theta2.resize((size_t)toff[N]);
    double_layer_theta(L1, L2, D, theta.data(), theta2.data());
  }

  HostBE be;
  std::vector<int> bi, bj;
  std::vector<double> bJ;
  bond_lists(L1, L2, J[0], J[1], bi, bj, bJ);
  be.N = N;
  be.nb = (int)bi.size();
  be.bi = bi.data();
  be.bj = bj.data();
  be.bJ = bJ.data();
  const long long cD = (long long)chi * Dn;
  be.trunc_cap = 2 * cD * (cD + 1);

  BatchRunner<T, HostBE, T> run(be);
  std::vector<long long> sz;
  long long n8 = 0, nd = 0, per = 0;
  BatchBufs<T>::sizes(L1, L2, Dn, chi, sz, n8, nd);
  for (long long x : sz) per += x;
  std::vector<T> real((size_t)per * n, 0.0);
  std::vector<int8_t> i8((size_t)n8 * n, 0);
  std::vector<double> dbl((size_t)nd * n, 0.0);
  unsigned long long jsw = 0;
  run.shp.build(L1, L2, Dn, chi);
  run.L1 = L1;
  run.L2 = L2;
  run.D = Dn;
  run.chi = chi;
  run.N = N;
  run.J1 = J[0];
  run.J2 = J[1];
  run.theta = mode == 2 ? theta2.data() : theta.data();
  run.toff = toff;
  run.ooff = ooff;
  run.jtol = 1e-15;
  run.max_sweeps = 60;
  run.sweeps = &jsw;
  run.b.bind(real.data(), n, i8.data(), dbl.data(), L1, L2, Dn, chi);
  run.gram_lq = mode == 3;

  FILE* fo = std::fopen(argv[2], "wb");
  if (!fo) return 2;
  if (mode == 4) {
    const long long No = ooff[N];
    std::vector<double> la(n);
    std::vector<int8_t> sg(n);
    std::vector<T> O((size_t)n * No);
    plain_amplitude(run, S.data(), n, la.data(), sg.data());
    plain_log_derivative(run, S.data(), n, O.data(), No);
    std::fwrite(la.data(), 8, n, fo);
    std::fwrite(sg.data(), 1, n, fo);
    std::fwrite(O.data(), 8, O.size(), fo);
  } else if (mode == 7) {
    double mu;
    std::memcpy(&mu, &seed, sizeof(mu));
    const long long No = ooff[N];
    std::vector<uint8_t> S32((size_t)n * N, 0);
    std::vector<double> la(n), es(n), ea(n);
    std::vector<int8_t> sg(n);
    std::vector<T> O((size_t)n * No);
    fermion_eval(run, S.data(), S32.data(), n, J[0], J[1], mu, la.data(), sg.data(), es.data(),
                 ea.data(), O.data(), No, ooff.data());
    std::fwrite(la.data(), 8, n, fo);
    std::fwrite(sg.data(), 1, n, fo);
    std::fwrite(es.data(), 8, n, fo);
    std::fwrite(ea.data(), 8, n, fo);
    std::fwrite(O.data(), 8, O.size(), fo);
  } else if (mode == 6) {
    // the couplings arrive in J1 (t), J2 (U) and the seed's bits (mu, a float64)
    double mu;
    std::memcpy(&mu, &seed, sizeof(mu));
    std::vector<uint8_t> S32((size_t)n * N, 0);
    std::vector<double> la(n), es(n), ea(n);
    std::vector<int8_t> sg(n);
    fermion_eloc(run, S.data(), S32.data(), n, J[0], J[1], mu, la.data(), sg.data(), es.data(), ea.data());
    std::fwrite(la.data(), 8, n, fo);
    std::fwrite(sg.data(), 1, n, fo);
    std::fwrite(es.data(), 8, n, fo);
    std::fwrite(ea.data(), 8, n, fo);
  } else if (mode == 5) {
    std::vector<uint8_t> S32((size_t)n * N, 0);
    std::vector<int> acc(n, 0);
    fermion_mc(run, S.data(), S32.data(), n, p, seed, (uint32_t)sweep, acc.data());
    std::fwrite(S.data(), 1, S.size(), fo);
    std::fwrite(acc.data(), 4, n, fo);
  } else if (mode == 0 || mode == 3) {
    const long long No = ooff[N];
    std::vector<double> la(n), es(n), ea(n);
    std::vector<int8_t> sg(n);
    std::vector<T> O((size_t)n * No);
    run.eval(S.data(), n, la.data(), sg.data(), es.data(), ea.data(), O.data(), No, false);
    std::fwrite(la.data(), 8, n, fo);
    std::fwrite(sg.data(), 1, n, fo);
    std::fwrite(es.data(), 8, n, fo);
    std::fwrite(ea.data(), 8, n, fo);
    std::fwrite(O.data(), 8, O.size(), fo);
  } else if (mode == 2) {
    std::vector<double> logq(n, 0.0);
    direct_draw(run, S.data(), n, u.data(), bx[0], bx[1], logq.data());
    std::fwrite(S.data(), 1, S.size(), fo);
    std::fwrite(logq.data(), 8, n, fo);
  } else {
    std::vector<int> acc(n, 0), prop(n, 0);
    run.mc(S.data(), n, p, seed, 0, (uint32_t)sweep, acc.data(), prop.data());
    std::fwrite(S.data(), 1, S.size(), fo);
    std::fwrite(acc.data(), 4, n, fo);
    std::fwrite(prop.data(), 4, n, fo);
  }
  std::fclose(fo);
  return 0;
}
