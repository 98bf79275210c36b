// A fermionic PEPS of the doubled Hubbard lattice (Sec. II, Fig. 1b; Sec. III.B) on the batched
// engine: amplitudes and O rows (plain_amplitude, plain_log_derivative and the sign kernels
// below), the Metropolis sweep and the local energies on cached strips (fermion_mc,
// fermion_eloc), and the kernels of the local energies with one full contraction per hop.
//
// The tensors are parity even with sixteen local states per site (system and ancilla modes
// c_up, c_dn, d_up, d_dn; parity of a local index = popcount mod 2, of a virtual index = its
// value mod 2) and the Fermi arrows order their Grassmann letters per site as l, u, P, d, r.
// By parity evenness the sign of that order reduces to
//     sign(S) * prod_i (-1)^((p(S_i) + p(d_i)) (p(l_i) + p(u_i)) + p(d_i) b_i),
// with sign(S) = (-1)^(sum_(i<j) p_i p_j + sum_R P_(R-1) P_R) (P_R the parity of the physical
// indices of rows 0..R) and b_i the parity of those left of site i in its row.  So the
// amplitude is sign(S) times the plain contraction of 32 signed slices per site (slice
// S_i + 16 b_i): the engine's own boundary-MPS contraction, unchanged.
#ifndef PV_FERMION_CUH
#define PV_FERMION_CUH
#include <cstdint>

#include "pv_batch.cuh"

namespace pv {

// log|psi| and the sign of the plain PEPS over `run`'s site tensors for the (extended)
// local indices S: the down environments, the right partials of row 0, the amplitude.
template <typename T, typename BE, typename OT>
void plain_amplitude(BatchRunner<T, BE, OT>& run, const uint8_t* S, int n, double* la, int8_t* sg) {
  auto& b = run.b;
  run.build_down(S, n);
  run.trivial(run.uprow(0), b.sU, n);
  run.be.set(b.p1R, b.sp1R, (long long)run.L2 * b.P1, (T)1, n);
  for (int c = run.L2 - 1; c >= 0; --c)
    run.s1_right(0, c, run.p1R(c), b.sp1R, run.bat(run.p1R(c + 1), b.sp1R), run.site(0, c, S), n);
  run.be.amp(b.p1R, b.sp1R, b.lsD + 1, run.L1 + 1, la, sg, n);
}

// O rows of the plain PEPS (d log / d of the site tensor at its slice, Eq. 8): per row the
// right partials, a rolling left partial, the environment of every site divided by the row
// strip's value, then the row absorbed into the up environment (the evaluation's own steps).
template <typename T, typename BE, typename OT>
void plain_log_derivative(BatchRunner<T, BE, OT>& run, const uint8_t* S, int n, OT* O, long long No) {
  auto& b = run.b;
  run.build_down(S, n);
  run.trivial(run.uprow(0), b.sU, n);
  run.be.setd(b.lsU, 1, 0, 0.0, n);
  for (int r = 0; r < run.L1; ++r) {
    run.be.set(b.p1R, b.sp1R, (long long)run.L2 * b.P1, (T)1, n);
    for (int c = run.L2 - 1; c >= 0; --c)
      run.s1_right(r, c, run.p1R(c), b.sp1R, run.bat(run.p1R(c + 1), b.sp1R), run.site(r, c, S), n);
    T* Lc = b.p1L;
    T* Ln = b.p1L + b.P1;
    run.be.set(b.p1L, b.sp1L, 0, (T)1, n);
    for (int c = 0; c < run.L2; ++c) {
      run.s1_env(r, c, run.bat(Lc, b.sp1L), run.bat(run.p1R(c + 1), b.sp1R), n);
      run.be.writeO(O, No, run.ooff[r * run.L2 + c], b.envo, b.D4, run.szs(r, c), b.p1R, b.sp1R, n);
      if (c + 1 < run.L2) {
        run.s1_left(r, c, Ln, b.sp1L, run.bat(Lc, b.sp1L), run.site(r, c, S), n);
        T* t = Lc;
        Lc = Ln;
        Ln = t;
      }
    }
    if (r + 1 < run.L1)
      run.compress(run.uprow(r), b.sU, run.shp.up[r], false, r, S, run.uprow(r + 1), b.sU, b.lsU, 1, n);
  }
}

// ---------------------------------------------------------------- Metropolis on cached strips
//
// One sweep in the row phases of fermion_moves (Sec. II, MCMC; target |psi|^p) with the
// proposals' amplitudes from one- and two-row strips between cached environments, as the
// spin sweep does, instead of a contraction of the whole lattice per proposal.  The site
// tensors carry 64 slices: S + 16 b (the signed slices) and S + 16 b + 32 (the same with a
// parity (-1)^(p(r)) on the right leg).  A pair keeps its site's parity; a horizontal hop (c,
// c+1) flips b of c+1 only; so the one-row strips of a row carry over with the actual bits.  A
// vertical hop at column c flips b of every site right of c in both rows, which equals a
// parity on the right leg of (r+1, c) times a sign (the right-leg parity of the lower site):
// the two-row phase keeps the bits of its start for the columns ahead, and an accepted hop
// carries the parity in its lower site's slice.  Only |psi'/psi| enters the decision, so the
// signs drop out.  S32 holds every chain's current slice indices; FConf resets them to the
// actual bits.

// Applies a per-chain functor to chains 0..n-1 on a back end that runs plain host loops (a
// device back end needs its own launch of the functor).
template <typename BE, typename F>
inline void fv_apply(BE& be, const F& f, int n) {
  static_assert(BE::host_loops, "fv_apply: this back end needs its own launch");
  (void)be;
  for (int s = 0; s < n; ++s) f(s);
}

PV_HD int fv_parity4(int v) { return (v ^ (v >> 1) ^ (v >> 2) ^ (v >> 3)) & 1; }

// S32 = S + 16 b with b the parity of the physical indices left of each site in its row.
struct FConf {
  const uint8_t* S16;
  uint8_t* S32;
  int L1, L2;
  PV_HD void operator()(int s) const {
    const long long N = (long long)L1 * L2;
    for (int r = 0; r < L1; ++r) {
      int b = 0;
      for (int c = 0; c < L2; ++c) {
        const int v = S16[s * N + r * L2 + c];
        S32[s * N + r * L2 + c] = (uint8_t)(v + 16 * b);
        b ^= fv_parity4(v);
      }
    }
  }
};

// The proposal's slice indices per chain.  kind 0: pair of spin k at site i; 1: hop of mode k
// across the horizontal bond (i, i+1) (b of i+1 flips); 2: hop of mode k across the vertical
// bond (i, j) in the two-row phase (frame bits; the lower site's right-leg parity toggles when
// `twist`, the site having a right neighbour).  valid = 0 where the move does not apply.
struct FSel {
  const uint8_t* S16;
  const uint8_t* S32;
  int N, kind, i, j, k, twist;
  int8_t *si, *sj, *valid;
  PV_HD void operator()(int s) const {
    const uint8_t* x = S16 + (long long)s * N;
    const uint8_t* y = S32 + (long long)s * N;
    const int a = x[i];
    if (kind == 0) {
      valid[s] = (int8_t)(((a >> k) & 1) == ((a >> (2 + k)) & 1));
      si[s] = (int8_t)((a ^ ((1 << k) | (1 << (2 + k)))) + (y[i] & 48));
      return;
    }
    const int bb = x[j];
    valid[s] = (int8_t)(((a >> k) & 1) != ((bb >> k) & 1));
    const int a2 = a ^ (1 << k), b2 = bb ^ (1 << k);
    si[s] = (int8_t)(a2 + (y[i] & 48));
    if (kind == 1)
      sj[s] = (int8_t)(b2 + ((y[j] & 48) ^ 16));
    else
      sj[s] = (int8_t)(b2 + ((y[j] & 48) ^ (twist ? 32 : 0)));
  }
};

// Metropolis decision: u = Philox(seed; chain0 + chain, sweep, m, TAG_FMC); accept iff log u < p
// log|num / den| (float64).  On acceptance the chain takes the proposed slices (and physical
// indices) and den the numerator.
template <typename T>
struct FAccept {
  uint8_t* S16;
  uint8_t* S32;
  int N, i, j;   // j < 0: one site
  const int8_t *si, *sj, *valid;
  const T* num;
  T* den;
  int p;
  uint64_t seed;
  int chain0;
  uint32_t sweep, m;
  int* acc;
  int8_t* accepted;
  PV_HD void operator()(int s) const {
    accepted[s] = 0;
    if (!valid[s]) return;
    const double u = philox_uniform(seed, (uint32_t)(chain0 + s), sweep, m, TAG_FMC);
    const double ratio = (double)num[s] / (double)den[s];
    const double d = log(u) - p * log(ratio < 0 ? -ratio : ratio);
    if (d < 0.0) {
      acc[s] += 1;
      accepted[s] = 1;
      S32[(long long)s * N + i] = (uint8_t)si[s];
      S16[(long long)s * N + i] = (uint8_t)(si[s] & 15);
      if (j >= 0) {
        S32[(long long)s * N + j] = (uint8_t)sj[s];
        S16[(long long)s * N + j] = (uint8_t)(sj[s] & 15);
      }
      den[s] = num[s];
    }
  }
};

// One sweep of every chain (`run` over the 64-slice tensors; S16 in and out, S32 work space
// for the slice indices; acc counts accepted proposals; chain s draws as chain chain0 + s).
// Move m draws counter m of the sweep, in the order of fermion_moves.
template <typename T, typename BE, typename OT>
void fermion_mc(BatchRunner<T, BE, OT>& run, uint8_t* S16, uint8_t* S32, int n, int p,
                uint64_t seed, uint32_t sweep, int* acc, int chain0 = 0) {
  auto& b = run.b;
  auto& be = run.be;
  const int L1 = run.L1, L2 = run.L2, N = run.N;
  fv_apply(be, FConf{S16, S32, L1, L2}, n);
  run.build_down(S32, n);
  run.trivial(run.uprow(0), b.sU, n);
  uint32_t m = 0;
  for (int r = 0; r < L1; ++r) {
    // one-row phase: each column's pairs, then the hops of its horizontal bond
    be.set(b.p1R, b.sp1R, (long long)L2 * b.P1, (T)1, n);
    for (int c = L2 - 1; c >= 0; --c)
      run.s1_right(r, c, run.p1R(c), b.sp1R, run.bat(run.p1R(c + 1), b.sp1R), run.site(r, c, S32), n);
    T* Lc = b.p1L;
    T* Ln = b.p1L + b.P1;
    be.set(b.p1L, b.sp1L, 0, (T)1, n);
    run.s1_left(r, 0, b.m0, b.P2, run.bat(Lc, b.sp1L), run.site(r, 0, S32), n);
    for (int c = 0; c < L2; ++c) {
      const int i = r * L2 + c;
      be.dot(OpDot<T>{b.m0, b.P2, run.p1R(c + 1), b.sp1R, run.s1_len(r, c + 1), b.den}, n);
      for (int sp = 0; sp < 2; ++sp, ++m) {
        fv_apply(be, FSel{S16, S32, N, 0, i, i, sp, 0, b.si, b.sj, b.valid}, n);
        run.s1_left(r, c, b.m2, b.P2, run.bat(Lc, b.sp1L), run.site_sel(r, c, b.si), n);
        be.dot(OpDot<T>{b.m2, b.P2, run.p1R(c + 1), b.sp1R, run.s1_len(r, c + 1), b.num}, n);
        fv_apply(be, FAccept<T>{S16, S32, N, i, -1, b.si, b.sj, b.valid, b.num, b.den, p, seed,
                                chain0, sweep, m, acc, b.accepted}, n);
        be.copy_masked(b.m0, b.P2, b.m2, b.P2, run.s1_len(r, c + 1), b.accepted, n);
      }
      if (c + 1 < L2) {
        run.s1_left(r, c + 1, b.m1, b.P2, run.bat(b.m0, b.P2), run.site(r, c + 1, S32), n);
        be.dot(OpDot<T>{b.m1, b.P2, run.p1R(c + 2), b.sp1R, run.s1_len(r, c + 2), b.den}, n);
        for (int k = 0; k < 4; ++k, ++m) {
          fv_apply(be, FSel{S16, S32, N, 1, i, i + 1, k, 0, b.si, b.sj, b.valid}, n);
          run.s1_left(r, c, b.m2, b.P2, run.bat(Lc, b.sp1L), run.site_sel(r, c, b.si), n);
          run.s1_left(r, c + 1, b.m3, b.P2, run.bat(b.m2, b.P2), run.site_sel(r, c + 1, b.sj), n);
          be.dot(OpDot<T>{b.m3, b.P2, run.p1R(c + 2), b.sp1R, run.s1_len(r, c + 2), b.num}, n);
          fv_apply(be, FAccept<T>{S16, S32, N, i, i + 1, b.si, b.sj, b.valid, b.num, b.den, p,
                                  seed, chain0, sweep, m, acc, b.accepted}, n);
          be.copy_masked(b.m0, b.P2, b.m2, b.P2, run.s1_len(r, c + 1), b.accepted, n);
          be.copy_masked(b.m1, b.P2, b.m3, b.P2, run.s1_len(r, c + 2), b.accepted, n);
        }
      }
      // advance: the left partial past column c is P; the next P is Q
      be.copy_masked(Ln, b.sp1L, b.m0, b.P2, run.s1_len(r, c + 1), nullptr, n);
      T* t = Lc;
      Lc = Ln;
      Ln = t;
      if (c + 1 < L2) be.copy_masked(b.m0, b.P2, b.m1, b.P2, run.s1_len(r, c + 2), nullptr, n);
    }
    if (r + 1 < L1) {
      // two-row phase: the hops of the vertical bonds to row r+1, column by column
      be.set(b.p2R, b.sp2R, (long long)L2 * b.P2, (T)1, n);
      for (int c = L2 - 1; c >= 0; --c)
        run.s2_right(r, c, run.p2R(c), b.sp2R, run.bat(run.p2R(c + 1), b.sp2R), run.site(r, c, S32),
                     run.site(r + 1, c, S32), n);
      T* L2c = b.p2L;
      T* L2n = b.p2L + b.P2;
      be.set(b.p2L, b.sp2L, 0, (T)1, n);
      for (int c = 0; c < L2; ++c) {
        const int i = r * L2 + c, j = i + L2;
        run.s2_left(r, c, b.m0, b.P2, run.bat(L2c, b.sp2L), run.site(r, c, S32), run.site(r + 1, c, S32), n);
        be.dot(OpDot<T>{b.m0, b.P2, run.p2R(c + 1), b.sp2R, run.s2_len(r, c + 1), b.den}, n);
        for (int k = 0; k < 4; ++k, ++m) {
          fv_apply(be, FSel{S16, S32, N, 2, i, j, k, c + 1 < L2, b.si, b.sj, b.valid}, n);
          run.s2_left(r, c, b.m1, b.P2, run.bat(L2c, b.sp2L), run.site_sel(r, c, b.si),
                      run.site_sel(r + 1, c, b.sj), n);
          be.dot(OpDot<T>{b.m1, b.P2, run.p2R(c + 1), b.sp2R, run.s2_len(r, c + 1), b.num}, n);
          fv_apply(be, FAccept<T>{S16, S32, N, i, j, b.si, b.sj, b.valid, b.num, b.den, p, seed,
                                  chain0, sweep, m, acc, b.accepted}, n);
          be.copy_masked(b.m0, b.P2, b.m1, b.P2, run.s2_len(r, c + 1), b.accepted, n);
        }
        be.copy_masked(L2n, b.sp2L, b.m0, b.P2, run.s2_len(r, c + 1), nullptr, n);
        T* t = L2c;
        L2c = L2n;
        L2n = t;
      }
      // the actual bits again (the phase's frame and parities dropped), then row r joins the
      // up environment
      fv_apply(be, FConf{S16, S32, L1, L2}, n);
      run.compress(run.uprow(r), b.sU, run.shp.up[r], false, r, S32, run.uprow(r + 1), b.sU, b.lsU, 1, n);
    }
  }
}

// ---------------------------------------------------------------- local energies on strips
//
// E_sys and E_anc (Eq. 9 with the Hubbard terms of Eq. 14 on the system and ancilla modes) from
// the same strips: the ratio psi(S')/psi(S) of a hop is cs(S')/cs(S) (the configuration signs)
// times the plain strip ratio, times, for a vertical hop at column c, the sign
// prod_(c' > c) (-1)^(p(S_(r+1, c'))) of its right-leg parity.

// (-1)^(sum_(i<j) p_i p_j + sum_R P_(R-1) P_R) of a configuration's physical indices.
PV_HD int fv_config_sign(const uint8_t* x, int L1, int L2) {
  int e = 0, pre = 0, prevP = 0, accP = 0;
  for (int r = 0; r < L1; ++r) {
    int row = 0;
    for (int c = 0; c < L2; ++c) {
      const int p = fv_parity4(x[r * L2 + c]);
      e += p * pre;
      pre ^= p;
      row ^= p;
    }
    accP ^= row;
    e += prevP * accP;
    prevP = accP;
  }
  return (e & 1) ? -1 : 1;
}

// Diagonal terms U n_up n_dn - mu (n_up + n_dn) per site, on each layer.
struct FDiag {
  const uint8_t* S16;
  int N;
  double U, mu;
  double *es, *ea;
  PV_HD void operator()(int s) const {
    double e[2] = {0.0, 0.0};
    for (int q = 0; q < N; ++q) {
      const int x = S16[(long long)s * N + q];
      for (int layer = 0; layer < 2; ++layer) {
        const int nu = (x >> (2 * layer)) & 1, nd = (x >> (2 * layer + 1)) & 1;
        e[layer] += U * nu * nd - mu * (nu + nd);
      }
    }
    es[s] = e[0];
    ea[s] = e[1];
  }
};

// sign *= cs(S): the plain amplitude's sign into the fermionic one.
struct FSignApply {
  const uint8_t* S16;
  int L1, L2;
  int8_t* sign;
  PV_HD void operator()(int s) const {
    sign[s] = (int8_t)(sign[s] * fv_config_sign(S16 + (long long)s * L1 * L2, L1, L2));
  }
};

// The hop of mode k across the bond (i, j) (one direction allowed where the occupations
// differ): E[layer of k] += -t JW(c+_a c_b) cs(S')/cs(S) twist num/den, with a the empty and b
// the occupied site, JW the Jordan-Wigner sign of the modes ordered site by site, and twist
// the right-leg sign of a vertical hop (vrow: the lower row, col: the hop's column; -1: none).
template <typename T>
struct FRatio {
  const uint8_t* S16;
  int L1, L2, i, j, k, vrow, col;
  const int8_t* valid;
  const T* num;
  const T* den;
  long long dens;
  double t_hop;
  double *es, *ea;
  PV_HD void operator()(int s) const {
    if (!valid[s]) return;
    const int N = L1 * L2;
    const uint8_t* x = S16 + (long long)s * N;
    const int bit = 1 << k;
    const int a = (x[i] & bit) ? j : i, b = (x[i] & bit) ? i : j;   // c+_a c_b
    uint8_t y[256];   // N <= 16 x 16 sites
    for (int q = 0; q < N; ++q) y[q] = x[q];
    // occupied modes below mode k of site b in x, then below mode k of site a after removal
    int cnt = 0;
    for (int q = 0; q < b; ++q) cnt += (x[q] & 1) + ((x[q] >> 1) & 1) + ((x[q] >> 2) & 1) + ((x[q] >> 3) & 1);
    for (int q = 0; q < k; ++q) cnt += (x[b] >> q) & 1;
    y[b] = (uint8_t)(x[b] & ~bit);
    for (int q = 0; q < a; ++q) cnt += (y[q] & 1) + ((y[q] >> 1) & 1) + ((y[q] >> 2) & 1) + ((y[q] >> 3) & 1);
    for (int q = 0; q < k; ++q) cnt += (y[a] >> q) & 1;
    y[a] = (uint8_t)(x[a] | bit);
    double f = (cnt & 1) ? t_hop : -t_hop;
    f *= fv_config_sign(y, L1, L2) * fv_config_sign(x, L1, L2);
    if (vrow >= 0)
      for (int c2 = col + 1; c2 < L2; ++c2)
        if (fv_parity4(y[vrow * L2 + c2])) f = -f;
    const double r = (double)num[s] / (double)den[(long long)s * dens];
    if (k < 2)
      es[s] += f * r;
    else
      ea[s] += f * r;
  }
};

// log|psi|, sign, E_sys and E_anc of every chain (`run` over the 64-slice tensors; S32 work
// space), each hop's ratio from a one-row (horizontal) or two-row (vertical) strip.
template <typename T, typename BE, typename OT>
void fermion_eloc(BatchRunner<T, BE, OT>& run, const uint8_t* S16, uint8_t* S32, int n,
                  double t_hop, double U, double mu, double* la, int8_t* sg, double* es,
                  double* ea) {
  auto& b = run.b;
  auto& be = run.be;
  const int L1 = run.L1, L2 = run.L2, N = run.N;
  fv_apply(be, FConf{S16, S32, L1, L2}, n);
  run.build_down(S32, n);
  fv_apply(be, FDiag{S16, N, U, mu, es, ea}, n);
  run.trivial(run.uprow(0), b.sU, n);
  for (int r = 0; r < L1; ++r) {
    be.set(b.p1R, b.sp1R, (long long)L2 * b.P1, (T)1, n);
    for (int c = L2 - 1; c >= 0; --c)
      run.s1_right(r, c, run.p1R(c), b.sp1R, run.bat(run.p1R(c + 1), b.sp1R), run.site(r, c, S32), n);
    if (r == 0) {
      be.amp(b.p1R, b.sp1R, b.lsD + 1, L1 + 1, la, sg, n);
      fv_apply(be, FSignApply{S16, L1, L2, sg}, n);
    }
    T* Lc = b.p1L;
    T* Ln = b.p1L + b.P1;
    be.set(b.p1L, b.sp1L, 0, (T)1, n);
    for (int c = 0; c + 1 < L2; ++c) {
      const int i = r * L2 + c;
      for (int k = 0; k < 4; ++k) {
        fv_apply(be, FSel{S16, S32, N, 1, i, i + 1, k, 0, b.si, b.sj, b.valid}, n);
        run.s1_left(r, c, b.m0, b.P2, run.bat(Lc, b.sp1L), run.site_sel(r, c, b.si), n);
        run.s1_left(r, c + 1, b.m1, b.P2, run.bat(b.m0, b.P2), run.site_sel(r, c + 1, b.sj), n);
        be.dot(OpDot<T>{b.m1, b.P2, run.p1R(c + 2), b.sp1R, run.s1_len(r, c + 2), b.num}, n);
        fv_apply(be, FRatio<T>{S16, L1, L2, i, i + 1, k, -1, c, b.valid, b.num, b.p1R, b.sp1R,
                               t_hop, es, ea}, n);
      }
      run.s1_left(r, c, Ln, b.sp1L, run.bat(Lc, b.sp1L), run.site(r, c, S32), n);
      T* t = Lc;
      Lc = Ln;
      Ln = t;
    }
    if (r + 1 < L1) {
      be.set(b.p2R, b.sp2R, (long long)L2 * b.P2, (T)1, n);
      for (int c = L2 - 1; c >= 0; --c)
        run.s2_right(r, c, run.p2R(c), b.sp2R, run.bat(run.p2R(c + 1), b.sp2R), run.site(r, c, S32),
                     run.site(r + 1, c, S32), n);
      T* L2c = b.p2L;
      T* L2n = b.p2L + b.P2;
      be.set(b.p2L, b.sp2L, 0, (T)1, n);
      for (int c = 0; c < L2; ++c) {
        const int i = r * L2 + c, j = i + L2;
        for (int k = 0; k < 4; ++k) {
          fv_apply(be, FSel{S16, S32, N, 2, i, j, k, c + 1 < L2, b.si, b.sj, b.valid}, n);
          run.s2_left(r, c, b.m0, b.P2, run.bat(L2c, b.sp2L), run.site_sel(r, c, b.si),
                      run.site_sel(r + 1, c, b.sj), n);
          be.dot(OpDot<T>{b.m0, b.P2, run.p2R(c + 1), b.sp2R, run.s2_len(r, c + 1), b.num}, n);
          fv_apply(be, FRatio<T>{S16, L1, L2, i, j, k, r + 1, c, b.valid, b.num, b.p2R, b.sp2R,
                                 t_hop, es, ea}, n);
        }
        run.s2_left(r, c, L2n, b.sp2L, run.bat(L2c, b.sp2L), run.site(r, c, S32), run.site(r + 1, c, S32), n);
        T* t = L2c;
        L2c = L2n;
        L2n = t;
      }
      run.compress(run.uprow(r), b.sU, run.shp.up[r], false, r, S32, run.uprow(r + 1), b.sU, b.lsU, 1, n);
    }
  }
}

// The plain O rows of one chain into those of the fermionic tensors: entry (l, r, u, d) of site
// i times (-1)^((p(S_i) + p(d)) (p(l) + p(u)) + p(d) b_i) (as k_fosign, one chain per call).
template <typename OT>
struct FOSign {
  const uint8_t* S16;
  int L1, L2, D;
  OT* O;
  long long No;
  const long long* ooff;
  PV_HD void operator()(int s) const {
    const uint8_t* x = S16 + (long long)s * L1 * L2;
    for (int i = 0; i < L1 * L2; ++i) {
      const int r = i / L2, c = i % L2;
      const int dr = c == L2 - 1 ? 1 : D, du = r == 0 ? 1 : D, dd = r == L1 - 1 ? 1 : D;
      int bb = 0;
      for (int q = 0; q < c; ++q) bb ^= fv_parity4(x[r * L2 + q]);
      const int pS = fv_parity4(x[i]);
      const long long sz = ooff[i + 1] - ooff[i];
      for (long long k = 0; k < sz; ++k) {
        long long t = k;
        const int d = (int)(t % dd);
        t /= dd;
        const int u = (int)(t % du);
        t /= du;
        t /= dr;
        const int l = (int)t;
        const int ex = (pS + (d & 1)) * ((l & 1) + (u & 1)) + (d & 1) * bb;
        if (ex & 1) {
          OT* q = O + (long long)s * No + ooff[i] + k;
          *q = -*q;
        }
      }
    }
  }
};

// One pass per chain over the rows (`run` over the 64-slice tensors; S32 work space): log|psi|,
// the sign, E_sys and E_anc (as fermion_eloc) and the O rows (Eq. 8: every site's environment
// over the strip value, then the Fermi-arrow signs; `ooff_dev` the site offsets of the rows as
// the functors read them).
template <typename T, typename BE, typename OT>
void fermion_eval(BatchRunner<T, BE, OT>& run, const uint8_t* S16, uint8_t* S32, int n,
                  double t_hop, double U, double mu, double* la, int8_t* sg, double* es,
                  double* ea, OT* O, long long No, const long long* ooff_dev) {
  auto& b = run.b;
  auto& be = run.be;
  const int L1 = run.L1, L2 = run.L2, N = run.N;
  fv_apply(be, FConf{S16, S32, L1, L2}, n);
  run.build_down(S32, n);
  fv_apply(be, FDiag{S16, N, U, mu, es, ea}, n);
  run.trivial(run.uprow(0), b.sU, n);
  for (int r = 0; r < L1; ++r) {
    be.set(b.p1R, b.sp1R, (long long)L2 * b.P1, (T)1, n);
    for (int c = L2 - 1; c >= 0; --c)
      run.s1_right(r, c, run.p1R(c), b.sp1R, run.bat(run.p1R(c + 1), b.sp1R), run.site(r, c, S32), n);
    if (r == 0) {
      be.amp(b.p1R, b.sp1R, b.lsD + 1, L1 + 1, la, sg, n);
      fv_apply(be, FSignApply{S16, L1, L2, sg}, n);
    }
    T* Lc = b.p1L;
    T* Ln = b.p1L + b.P1;
    be.set(b.p1L, b.sp1L, 0, (T)1, n);
    for (int c = 0; c < L2; ++c) {
      const int i = r * L2 + c;
      run.s1_env(r, c, run.bat(Lc, b.sp1L), run.bat(run.p1R(c + 1), b.sp1R), n);
      be.writeO(O, No, run.ooff[i], b.envo, b.D4, run.szs(r, c), b.p1R, b.sp1R, n);
      if (c + 1 < L2) {
        for (int k = 0; k < 4; ++k) {
          fv_apply(be, FSel{S16, S32, N, 1, i, i + 1, k, 0, b.si, b.sj, b.valid}, n);
          run.s1_left(r, c, b.m0, b.P2, run.bat(Lc, b.sp1L), run.site_sel(r, c, b.si), n);
          run.s1_left(r, c + 1, b.m1, b.P2, run.bat(b.m0, b.P2), run.site_sel(r, c + 1, b.sj), n);
          be.dot(OpDot<T>{b.m1, b.P2, run.p1R(c + 2), b.sp1R, run.s1_len(r, c + 2), b.num}, n);
          fv_apply(be, FRatio<T>{S16, L1, L2, i, i + 1, k, -1, c, b.valid, b.num, b.p1R, b.sp1R,
                                 t_hop, es, ea}, n);
        }
        run.s1_left(r, c, Ln, b.sp1L, run.bat(Lc, b.sp1L), run.site(r, c, S32), n);
        T* t = Lc;
        Lc = Ln;
        Ln = t;
      }
    }
    if (r + 1 < L1) {
      be.set(b.p2R, b.sp2R, (long long)L2 * b.P2, (T)1, n);
      for (int c = L2 - 1; c >= 0; --c)
        run.s2_right(r, c, run.p2R(c), b.sp2R, run.bat(run.p2R(c + 1), b.sp2R), run.site(r, c, S32),
                     run.site(r + 1, c, S32), n);
      T* L2c = b.p2L;
      T* L2n = b.p2L + b.P2;
      be.set(b.p2L, b.sp2L, 0, (T)1, n);
      for (int c = 0; c < L2; ++c) {
        const int i = r * L2 + c, j = i + L2;
        for (int k = 0; k < 4; ++k) {
          fv_apply(be, FSel{S16, S32, N, 2, i, j, k, c + 1 < L2, b.si, b.sj, b.valid}, n);
          run.s2_left(r, c, b.m0, b.P2, run.bat(L2c, b.sp2L), run.site_sel(r, c, b.si),
                      run.site_sel(r + 1, c, b.sj), n);
          be.dot(OpDot<T>{b.m0, b.P2, run.p2R(c + 1), b.sp2R, run.s2_len(r, c + 1), b.num}, n);
          fv_apply(be, FRatio<T>{S16, L1, L2, i, j, k, r + 1, c, b.valid, b.num, b.p2R, b.sp2R,
                                 t_hop, es, ea}, n);
        }
        run.s2_left(r, c, L2n, b.sp2L, run.bat(L2c, b.sp2L), run.site(r, c, S32), run.site(r + 1, c, S32), n);
        T* t = L2c;
        L2c = L2n;
        L2n = t;
      }
      run.compress(run.uprow(r), b.sU, run.shp.up[r], false, r, S32, run.uprow(r + 1), b.sU, b.lsU, 1, n);
    }
  }
  fv_apply(be, FOSign<OT>{S16, L1, L2, run.D, O, No, ooff_dev}, n);
}

#if defined(__CUDACC__)

// The plain O rows into those of the fermionic tensors: entry (l, r, u, d) of site i times
// (-1)^((p(S_i) + p(d)) (p(l) + p(u)) + p(d) b_i), the derivative of the signed slice with
// respect to the slice of theta.  Block y = site, threads over chains x entries.
template <typename OT>
__global__ void k_fosign(int n, int L1, int L2, int D, OT* __restrict__ O, long long No,
                         const long long* __restrict__ ooff, const uint8_t* __restrict__ S) {
  const int i = blockIdx.y, r = i / L2, c = i % L2, N = L1 * L2;
  const int dr = c == L2 - 1 ? 1 : D, du = r == 0 ? 1 : D, dd = r == L1 - 1 ? 1 : D;
  const long long sz = ooff[i + 1] - ooff[i];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)n * sz;
       e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / sz);
    const long long k = e - (long long)s * sz;
    long long t = k;
    const int d = (int)(t % dd);
    t /= dd;
    const int u = (int)(t % du);
    t /= du;
    t /= dr;
    const int l = (int)t;
    const uint8_t* x = S + (long long)s * N;
    int bb = 0;
    for (int q = 0; q < c; ++q) bb ^= __popc(x[r * L2 + q]) & 1;
    const int pS = __popc(x[i]) & 1;
    const int ex = (pS + (d & 1)) * ((l & 1) + (u & 1)) + (d & 1) * bb;
    if (ex & 1) {
      OT* p = O + (long long)s * No + ooff[i] + k;
      *p = -*p;
    }
  }
}

// The 32 signed slices per site from the sixteen of theta (float64, per site
// [16][dl][dr][du][dd]): block y = site, threads over slice x element.
template <typename T>
__global__ void k_fsigned(int L1, int L2, int D, const double* __restrict__ th16,
                          const long long* __restrict__ toff16, T* __restrict__ th32,
                          const long long* __restrict__ toff32) {
  const int i = blockIdx.y, r = i / L2, c = i % L2;
  const int dl = c == 0 ? 1 : D, dr = c == L2 - 1 ? 1 : D, du = r == 0 ? 1 : D, dd = r == L1 - 1 ? 1 : D;
  const long long sz = (long long)dl * dr * du * dd;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < 32 * sz;
       e += (long long)gridDim.x * blockDim.x) {
    const int slice = (int)(e / sz), S = slice & 15, bb = slice >> 4;
    const long long k = e - (long long)slice * sz;
    long long t = k;
    const int d = (int)(t % dd);
    t /= dd;
    const int u = (int)(t % du);
    t /= du;
    t /= dr;
    const int l = (int)t;
    const int pS = __popc(S) & 1;
    const int ex = (pS + (d & 1)) * ((l & 1) + (u & 1)) + (d & 1) * bb;
    const double v = th16[toff16[i] + (long long)S * sz + k];
    th32[toff32[i] + e] = (T)((ex & 1) ? -v : v);
  }
}

// Per chain: the extended local indices S_i + 16 b_i and sign(S); an entry above 15 raises
// `bad` (the chain's sign is 0 and its indices are left at 0).
__global__ void k_fconfigs(int n, int L1, int L2, const uint8_t* __restrict__ S,
                           uint8_t* __restrict__ S32, int8_t* __restrict__ csign, int* bad) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int N = L1 * L2;
  const uint8_t* x = S + (long long)s * N;
  uint8_t* y = S32 + (long long)s * N;
  int e = 0, pre = 0, prevP = 0, accP = 0, invalid = 0;
  for (int r = 0; r < L1; ++r) {
    int row = 0;
    for (int c = 0; c < L2; ++c) {
      const int v = x[r * L2 + c];
      invalid |= v > 15;
      const int p = __popc(v & 15) & 1;
      y[r * L2 + c] = (uint8_t)(v > 15 ? 0 : v + 16 * row);
      e += p * pre;
      pre ^= p;
      row ^= p;
    }
    accP ^= row;
    e += prevP * accP;
    prevP = accP;
  }
  csign[s] = invalid ? 0 : ((e & 1) ? -1 : 1);
  if (invalid) atomicOr(bad, 1);
}

__global__ void k_fapply(int n, const int8_t* __restrict__ csign, int8_t* __restrict__ sign,
                         double* __restrict__ la) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  sign[s] = (int8_t)(sign[s] * csign[s]);
  if (csign[s] == 0) la[s] = NAN;
}

// Exclusive prefix sums of n counts (one block): out[i] = in[0] + ... + in[i-1], out[n] the
// total.  Each thread sums a contiguous segment, the segment sums are scanned in shared
// memory, then each thread writes its segment's prefixes (a fixed order).
__global__ void k_fscan(int n, const int* __restrict__ in, int* __restrict__ out) {
  __shared__ int part[1024];
  const int T = blockDim.x, t = threadIdx.x;
  const int seg = (n + T - 1) / T, i0 = min(n, t * seg), i1 = min(n, i0 + seg);
  int sum = 0;
  for (int i = i0; i < i1; ++i) sum += in[i];
  part[t] = sum;
  __syncthreads();
  if (t == 0) {
    int acc = 0;
    for (int k = 0; k < T; ++k) {
      const int v = part[k];
      part[k] = acc;
      acc += v;
    }
    out[n] = acc;
  }
  __syncthreads();
  int acc = part[t];
  for (int i = i0; i < i1; ++i) {
    out[i] = acc;
    acc += in[i];
  }
}

// Allowed hops of the Hubbard terms of Eq. 14 per chain: for every bond and mode (layer,
// spin) exactly one direction is allowed where the two occupations differ, none otherwise.
__global__ void k_fhop_count(int nb, int N, const uint8_t* __restrict__ S, const int* __restrict__ bi,
                             const int* __restrict__ bj, int nbonds, int* __restrict__ cnt) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nb) return;
  const uint8_t* x = S + (long long)s * N;
  int c = 0;
  for (int b = 0; b < nbonds; ++b) c += __popc((x[bi[b]] ^ x[bj[b]]) & 15);
  cnt[s] = c;
}

// The configurations one allowed hop away (system: layer 0, ancilla: layer 1) written
// compactly: chain s's hops at off[s], off[s] + 1, ..., in the order of the slots k = ((bond
// * 2 + spin) * 2 + direction) * 2 + layer, each with the coefficient -t times its
// Jordan-Wigner sign (c+_a c_b with a, b the bond's sites in the slot's direction; modes
// ordered site by site, c_up c_dn d_up d_dn within a site) and its slot.
__global__ void k_fhops(int nb, int N, const uint8_t* __restrict__ S, const int* __restrict__ bi,
                        const int* __restrict__ bj, int nbonds, double t_hop,
                        const int* __restrict__ off, uint8_t* __restrict__ Sx,
                        double* __restrict__ coef, int* __restrict__ slot) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nb) return;
  const uint8_t* x = S + (long long)s * N;
  // occupied modes below mode (site, pos) of configuration z
  auto below = [&](const uint8_t* z, int site, int pos, int skip, uint8_t zskip) {
    int cnt = 0;
    for (int i = 0; i < site; ++i) cnt += __popc(i == skip ? zskip : z[i]);
    return cnt + __popc((site == skip ? zskip : z[site]) & ((1 << pos) - 1));
  };
  long long e = off[s];
  for (int k = 0; k < nbonds * 8; ++k) {
    const int layer = k & 1, dir = (k >> 1) & 1, spin = (k >> 2) & 1, bond = k >> 3;
    const int a = dir ? bi[bond] : bj[bond], b = dir ? bj[bond] : bi[bond];   // c+_a c_b
    const int pos = 2 * layer + spin, bit = 1 << pos;
    if (!(x[b] & bit) || (x[a] & bit)) continue;
    const uint8_t xb = (uint8_t)(x[b] & ~bit);
    const int js = below(x, b, pos, -1, 0) + below(x, a, pos, b, xb);
    uint8_t* y = Sx + e * N;
    for (int i = 0; i < N; ++i) y[i] = x[i];
    y[b] = xb;
    y[a] = (uint8_t)(x[a] | bit);
    coef[e] = -t_hop * ((js & 1) ? -1.0 : 1.0);
    slot[e] = k;
    ++e;
  }
}

// E_sys and E_anc per chain: the diagonal terms (U n_up n_dn - mu (n_up + n_dn) per site and
// layer) plus sum coef psi(S') / psi(S) over the chain's hops of that layer, in slot order.
__global__ void k_fsum(int nb, int N, const uint8_t* __restrict__ S, double U, double mu,
                       const int* __restrict__ off, const double* __restrict__ coef,
                       const int* __restrict__ slot, const double* __restrict__ la_x,
                       const int8_t* __restrict__ sg_x, const double* __restrict__ la,
                       const int8_t* __restrict__ sg, double* __restrict__ es,
                       double* __restrict__ ea) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nb) return;
  double e[2] = {0.0, 0.0};
  const uint8_t* x = S + (long long)s * N;
  for (int i = 0; i < N; ++i)
    for (int layer = 0; layer < 2; ++layer) {
      const int nu = (x[i] >> (2 * layer)) & 1, nd = (x[i] >> (2 * layer + 1)) & 1;
      e[layer] += U * nu * nd - mu * (nu + nd);
    }
  if (sg[s] == 0) {
    es[s] = NAN;
    ea[s] = NAN;
    return;
  }
  for (int q = off[s]; q < off[s + 1]; ++q) {
    if (sg_x[q] == 0) continue;
    e[slot[q] & 1] += coef[q] * (double)(sg_x[q] * sg[s]) * exp(la_x[q] - la[s]);
  }
  es[s] = e[0];
  ea[s] = e[1];
}

#endif  // __CUDACC__

}  // namespace pv
#endif
