// Per-sample work of the cooling step, executed by one thread block per configuration:
// boundary-MPS environments of the single-layer network rho_theta(S) (Sec. III.A, bond
// D_c = chi), amplitude, local energy from amplitude ratios (Eq. 9), log-derivatives
// (Eq. 8), and the Metropolis sweep (Sec. II MCMC, App. A reweighting).
//
// Conventions (shared with the C ABI):
//  * lattice L1 x L2 (rows x columns), site i = r*L2 + c; local index S = 2 s + s'.
//  * site tensor T_i^S[l][r][u][d], open legs of dimension 1; theta = concatenation of the
//    site blocks [4][dl][dr][du][dd]; O row = concatenation of the [dl][dr][du][dd] slices.
//  * environment = MPS over the columns, tensor c is [bond c][phys][bond c+1]; down env
//    at row boundary r contracts rows r..L1-1, up env rows 0..r-1.
//  * compression to chi (only when a bond exceeds chi): right-to-left triangular factors
//    L_c (C_{>=c} = L_c Q_{>=c}, Q row-orthonormal, Householder), then left-to-right
//    singular vectors of X_c = (carry C_c) L_{c+1} (one-sided Jacobi), keeping the chi
//    largest; carry' = U_chi^T (carry C_c).  Every env tensor is max-abs normalised with
//    the logarithm accumulated in a float64 log-scale.
//  * one-row strip of row r: up[r], row r, down[r+1]; horizontal-bond ratios and O.
//    two-row strip of rows r, r+1: up[r], the two rows, down[r+2]; vertical and
//    next-nearest-neighbour ratios.  A ratio is strip(S')/strip(S) with the same envs.
#pragma once

#include "pv_coop.cuh"
#include "pv_philox.cuh"

namespace pv {

constexpr int MAX_L = 16;   // lattice side limit (rows and columns)
constexpr int MAX_N = MAX_L * MAX_L;

struct Geom {
  int L1, L2, D, chi;
  double J1, J2;
  const long long* theta_off;   // N+1 entries
  const long long* o_off;       // N+1 entries
  PV_HD int N() const { return L1 * L2; }
  PV_HD int dl(int c) const { return c == 0 ? 1 : D; }
  PV_HD int dr(int c) const { return c == L2 - 1 ? 1 : D; }
  PV_HD int du(int r) const { return r == 0 ? 1 : D; }
  PV_HD int dd(int r) const { return r == L1 - 1 ? 1 : D; }
  PV_HD long long sz(int r, int c) const {
    return (long long)dl(c) * dr(c) * du(r) * dd(r);
  }
};

// Element counts of the per-block scratch.
struct ScratchDims {
  long long ENV, CB, LB, P1, P2, TMP;
  long long n_real, n_int;
};

PV_HD ScratchDims scratch_dims(int L1, int L2, int D, int chi) {
  ScratchDims s;
  long long cD = (long long)chi * D;
  s.ENV = (long long)chi * D * chi;
  s.CB = cD * D * cD;
  s.LB = cD * cD;
  s.P1 = (long long)chi * D * chi;
  s.P2 = (long long)chi * D * D * chi;
  s.TMP = (long long)chi * chi * D * D * D;
  s.n_real = (long long)(L1 + 1) * L2 * s.ENV   // down envs
             + 2LL * L2 * s.ENV                 // up envs (ping-pong)
             + s.CB                             // one site of the product MPS
             + (long long)(L2 + 1) * s.LB       // right factors
             + s.CB                             // Householder work
             + s.CB                             // carry * C_c
             + 2 * s.LB                         // Jacobi matrix + accumulated rotations
             + cD * chi                         // kept singular vectors
             + cD * chi                         // carry
             + cD                               // singular values
             + 2LL * (L2 + 1) * s.P1            // one-row partials
             + 2LL * (L2 + 1) * s.P2            // two-row partials
             + 2 * s.TMP                        // temporaries (ping-pong)
             + 4 * s.P2                         // modified / cached partials
             + (long long)D * D * D * D;        // site environment
  s.n_int = (long long)(L1 + 1) * (L2 + 1) + 2LL * (L2 + 1) + (L2 + 1) + (L2 + 1) + cD;
  return s;
}

template <typename T>
struct Scratch {
  ScratchDims d;
  T *envD, *envU[2], *Cs, *Lf, *W, *Am, *Y, *V, *Uk, *carry, *sig;
  T *p1L, *p1R, *p2L, *p2R, *t0, *t1, *m0, *m1, *m2, *m3, *envo;
  int *bondD, *bondU[2], *bondC, *kf, *order;
  T* smem = nullptr;        // optional fast buffer for the Jacobi matrices
  long long smem_cap = 0;   // its capacity in elements

  // Narrow layout in global memory: buffers that are never live at the same time share
  // space, so fewer distinct cache lines are touched per block (W and Cs share the
  // temporaries, Am / carry / Uk the partial buffers).
  PV_HD void alias_global() {
    W = t0;
    Cs = t1;
    Am = m0;
    carry = m2;
    Uk = m3;
  }

  // Elements of shared memory that hold every short-lived buffer (bind_shared).
  PV_HD static long long shared_elems(int D, int chi) {
    ScratchDims q = scratch_dims(1, 1, D, chi);
    long long cD = (long long)chi * D;
    long long jac = 2 * cD * (cD + 1);
    return 2 * q.TMP + 4 * q.P2 + (long long)D * D * D * D + (jac <= q.TMP ? 0 : jac);
  }

  // Places the temporaries, the partial buffers, the one-site product MPS, the
  // Householder work matrix, carry, kept vectors and the Jacobi matrices in shared
  // memory.  Buffers that are never live at the same time share space: W and the Jacobi
  // matrices (step (i) vs step (ii) of the truncation), Cs and t1, Am and m0/m1, carry/Uk
  // and m2/m3.
  PV_HD void bind_shared(T* sm, int D, int chi) {
    long long cD = (long long)chi * D;
    T* q = sm;
    t0 = q; q += d.TMP;
    t1 = q; q += d.TMP;
    m0 = q; q += d.P2;
    m1 = q; q += d.P2;
    m2 = q; q += d.P2;
    m3 = q; q += d.P2;
    envo = q; q += (long long)D * D * D * D;
    W = t0;
    Cs = t1;
    Am = m0;      // Am: chi*D*cD <= 2 * P2
    carry = m2;   // chi*cD <= P2
    Uk = m3;
    long long jac = 2 * cD * (cD + 1);
    if (jac <= d.TMP) {
      smem = t0;
      smem_cap = d.TMP;
    } else {
      smem = q;
      smem_cap = jac;
    }
  }

  PV_HD void bind(T* base, int* ibase, int L1, int L2, int D, int chi) {
    d = scratch_dims(L1, L2, D, chi);
    long long cD = (long long)chi * D;
    T* p = base;
    envD = p; p += (long long)(L1 + 1) * L2 * d.ENV;
    envU[0] = p; p += (long long)L2 * d.ENV;
    envU[1] = p; p += (long long)L2 * d.ENV;
    Cs = p; p += d.CB;
    Lf = p; p += (long long)(L2 + 1) * d.LB;
    W = p; p += d.CB;
    Am = p; p += d.CB;
    Y = p; p += d.LB;
    V = p; p += d.LB;
    Uk = p; p += cD * chi;
    carry = p; p += cD * chi;
    sig = p; p += cD;
    p1L = p; p += (long long)(L2 + 1) * d.P1;
    p1R = p; p += (long long)(L2 + 1) * d.P1;
    p2L = p; p += (long long)(L2 + 1) * d.P2;
    p2R = p; p += (long long)(L2 + 1) * d.P2;
    t0 = p; p += d.TMP;
    t1 = p; p += d.TMP;
    m0 = p; p += d.P2;
    m1 = p; p += d.P2;
    m2 = p; p += d.P2;
    m3 = p; p += d.P2;
    envo = p; p += (long long)D * D * D * D;
    int* q = ibase;
    bondD = q; q += (L1 + 1) * (L2 + 1);
    bondU[0] = q; q += L2 + 1;
    bondU[1] = q; q += L2 + 1;
    bondC = q; q += L2 + 1;
    kf = q; q += L2 + 1;
    order = q; q += (int)cD;
  }
};

// Shared-memory block state of the sample pass.
template <typename T>
struct Shared {
  T red[32];
  double redd[32];
  int flag;
  unsigned char S[MAX_N];
  double lsD[MAX_L + 1];
  double lsU[2];
  double flops;
  int jac_sweeps;
};

// Tensor T_i^{S} (row-major [dl][dr][du][dd]).
template <typename TT>
PV_HD const TT* site_tensor(const Geom& g, const TT* theta, int r, int c, int S) {
  int i = r * g.L2 + c;
  return theta + g.theta_off[i] + (long long)S * g.sz(r, c);
}

// ---------------------------------------------------------------- environments

// Site c of row r absorbed into an environment, into Cout.  down: env below row r
// (phys = dd(r)); the result has phys du(r).  up: env above row r (phys = du(r)); result
// phys dd(r).  Bond (a, l) of the product is fused as a*dl + l.
template <typename T, typename TT>
PV_HDN double absorb_site(const Geom& g, Scratch<T>& sc, const T* env, const int* bond, bool down,
                          int r, int c, const TT* theta, const unsigned char* S, T* Cout) {
  const TT* A = site_tensor(g, theta, r, c, S[r * g.L2 + c]);
  Dims dm;
  dm.set('a', bond[c]).set('b', bond[c + 1]).set('l', g.dl(c)).set('r', g.dr(c));
  dm.set('u', g.du(r)).set('d', g.dd(r));
  const T* E = env + (long long)c * sc.d.ENV;
  if (down) return einsum(Cout, "alubr", E, "adb", A, "lrud", dm);
  return einsum(Cout, "aldbr", E, "aub", A, "lrud", dm);
}

// Bonds of the product MPS of `bond` and row r (bond c fused with the row's left leg).
template <typename T>
PV_HD void product_bonds(const Geom& g, Scratch<T>& sc, const int* bond) {
  if (PV_TID == 0) {
    for (int c = 0; c < g.L2; ++c) sc.bondC[c] = bond[c] * g.dl(c);
    sc.bondC[g.L2] = 1;
  }
  PV_SYNC();
}

// Product MPS producer: the environment and row whose product is compressed.
template <typename T, typename TT>
struct Product {
  const T* env;
  const int* bond;
  bool down;
  int r;
  const TT* theta;
  const unsigned char* S;
};

// Compresses the product MPS of pr (bonds sc.bondC, phys p) into `out` (bonds out_bond),
// normalising and accumulating the log-scale into *ls (thread 0 writes).  The product is
// formed one site at a time (into sc.Cs) when a site is needed.
template <typename T, typename TT>
PV_HDN double compress(const Geom& g, Scratch<T>& sc, Shared<T>& sh, int p, const Product<T, TT>& pr,
                       T* out, int* out_bond, double* ls, T jtol, int max_sweeps) {
  const int n = g.L2;
  const int chi = g.chi;
  double fl = 0;
  product_bonds(g, sc, pr.bond);
  auto site = [&](int c) {
    fl += absorb_site(g, sc, pr.env, pr.bond, pr.down, pr.r, c, pr.theta, pr.S, sc.Cs);
  };
  int maxb = 0;
  for (int c = 0; c <= n; ++c) maxb = sc.bondC[c] > maxb ? sc.bondC[c] : maxb;
  double lsum = 0;
  if (maxb <= chi) {
    for (int c = 0; c < n; ++c) {
      long long len = (long long)sc.bondC[c] * p * sc.bondC[c + 1];
      T* o = out + (long long)c * sc.d.ENV;
      fl += absorb_site(g, sc, pr.env, pr.bond, pr.down, pr.r, c, pr.theta, pr.S, o);
      lsum += normalize_maxabs(o, len, sh.red);
    }
    if (PV_TID == 0) {
      for (int c = 0; c <= n; ++c) out_bond[c] = sc.bondC[c];
      *ls += lsum;
    }
    PV_SYNC();
    return fl;
  }
  // (i) right-to-left triangular factors
  if (PV_TID == 0) {
    sc.Lf[(long long)n * sc.d.LB] = 1;
    sc.kf[n] = 1;
  }
  PV_SYNC();
  for (int c = n - 1; c >= 1; --c) {
    Dims dm;
    dm.set('a', sc.bondC[c]).set('p', p).set('b', sc.bondC[c + 1]).set('k', sc.kf[c + 1]);
    site(c);
    fl += einsum(sc.W, "apk", sc.Cs, "apb", sc.Lf + (long long)(c + 1) * sc.d.LB, "bk", dm);
    int m = sc.bondC[c], nn = p * sc.kf[c + 1];
    fl += lq_factor(sc.Lf + (long long)c * sc.d.LB, sc.W, m, nn, sh.red, sh.red);
    if (PV_TID == 0) sc.kf[c] = m < nn ? m : nn;
    PV_SYNC();
  }
  // (ii) left-to-right truncation
  if (PV_TID == 0) {
    sc.carry[0] = 1;
    out_bond[0] = 1;
  }
  PV_SYNC();
  int bprev = 1;
  for (int c = 0; c < n - 1; ++c) {
    int a = sc.bondC[c], b = sc.bondC[c + 1], k = sc.kf[c + 1];
    Dims dm;
    dm.set('x', bprev).set('a', a).set('p', p).set('b', b);
    site(c);
    fl += einsum(sc.Am, "xpb", sc.carry, "xa", sc.Cs, "apb", dm);
    int m = bprev * p;
    Dims dq;
    dq.set('q', m).set('b', b).set('k', k);
    const T* Lc = sc.Lf + (long long)(c + 1) * sc.d.LB;
    bool tall = k <= m;   // Jacobi on the k columns of X; else on its m rows with rotations kept
    int nc, len;
    if (tall) {
      fl += einsum(sc.Y, "kq", sc.Am, "qb", Lc, "bk", dq);
      nc = k;
      len = m;
    } else {
      fl += einsum(sc.Y, "qk", sc.Am, "qb", Lc, "bk", dq);
      nc = m;
      len = k;
    }
    // work copy: shared memory (columns padded to an odd stride) when it fits
    T* Yw = sc.Y;
    T* Vw = sc.V;
    int ldy = len, ldv = m;
    long long need = (long long)nc * (len + 1) + (tall ? 0 : (long long)m * (m + 1));
    if (sc.smem && need <= sc.smem_cap) {
      ldy = len | 1;
      ldv = m | 1;
      Yw = sc.smem;
      Vw = sc.smem + (long long)nc * ldy;
      for (long long i = PV_TID; i < (long long)nc * len; i += PV_NTHR)
        Yw[(i / len) * ldy + i % len] = sc.Y[i];
    }
    if (!tall) {
      for (long long i = PV_TID; i < (long long)m * m; i += PV_NTHR)
        Vw[(i / m) * ldv + i % m] = (i / m == i % m) ? (T)1 : (T)0;
    }
    PV_SYNC();
    int sweeps = 0;
    fl += jacobi(Yw, ldy, nc, len, tall ? (T*)nullptr : Vw, ldv, m, jtol, max_sweeps, &sh.flag,
                 &sweeps, sh.red);
    if (PV_TID == 0) sh.jac_sweeps += sweeps;
    // singular values (column norms) and their descending order (ties by index)
    for (int j = PV_WARP; j < nc; j += PV_NWARP) {
      T s2 = 0;
      const T* y = Yw + (long long)j * ldy;
      for (int i = PV_LANE; i < len; i += PV_WSIZE) s2 += y[i] * y[i];
      s2 = warp_sum(s2);
      if (PV_LANE == 0) sc.sig[j] = sqrt(s2);
    }
    PV_SYNC();
    for (int j = PV_TID; j < nc; j += PV_NTHR) {
      int rank = 0;
      T sj = sc.sig[j];
      for (int i = 0; i < nc; ++i) {
        T si = sc.sig[i];
        rank += (si > sj || (si == sj && i < j)) ? 1 : 0;
      }
      sc.order[rank] = j;
    }
    PV_SYNC();
    int kmax = m < k ? m : k;
    int kk = chi < kmax ? chi : kmax;
    // Columns below the rounding floor of the Jacobi (norm^2 <= (eps len)^2 |X|^2) were not
    // orthogonalised; they are zero singular values and give zero vectors, never
    // normalised noise (which would not be orthogonal to the kept directions).
    T zero2 = 0;
    if (tall) {
      T nf2 = 0;
      for (int j = 0; j < nc; ++j) nf2 += sc.sig[j] * sc.sig[j];
      const T eps = sizeof(T) == 4 ? (T)1.1920929e-7 : (T)2.220446049250313e-16;
      zero2 = (eps * len) * (eps * len) * nf2;
    }
    // kept left singular vectors Uk[q][j']
    for (long long idx = PV_TID; idx < (long long)m * kk; idx += PV_NTHR) {
      int q = (int)(idx / kk), jp = (int)(idx % kk);
      int j = sc.order[jp];
      T v;
      if (tall) {
        T s = sc.sig[j];
        v = s * s > zero2 ? Yw[(long long)j * ldy + q] / s : (T)0;
      } else {
        v = Vw[(long long)j * ldv + q];
      }
      sc.Uk[idx] = v;
    }
    PV_SYNC();
    T* o = out + (long long)c * sc.d.ENV;
    copy(o, sc.Uk, (long long)m * kk);
    Dims dc;
    dc.set('q', m).set('j', kk).set('b', b);
    fl += einsum(sc.carry, "jb", sc.Uk, "qj", sc.Am, "qb", dc);
    if (PV_TID == 0) out_bond[c + 1] = kk;
    PV_SYNC();
    lsum += normalize_maxabs(o, (long long)m * kk, sh.red);
    bprev = kk;
  }
  {
    int c = n - 1;
    Dims dm;
    dm.set('x', bprev).set('a', sc.bondC[c]).set('p', p).set('b', sc.bondC[c + 1]);
    T* o = out + (long long)c * sc.d.ENV;
    site(c);
    fl += einsum(o, "xpb", sc.carry, "xa", sc.Cs, "apb", dm);
    lsum += normalize_maxabs(o, (long long)bprev * p * sc.bondC[c + 1], sh.red);
    if (PV_TID == 0) {
      out_bond[n] = 1;
      *ls += lsum;
    }
    PV_SYNC();
  }
  return fl;
}

template <typename T>
PV_HD void trivial_env(const Geom& g, Scratch<T>& sc, T* env, int* bond) {
  for (int c = PV_TID; c < g.L2; c += PV_NTHR) env[(long long)c * sc.d.ENV] = 1;
  for (int c = PV_TID; c <= g.L2; c += PV_NTHR) bond[c] = 1;
  PV_SYNC();
}

// ---------------------------------------------------------------- one-row strips

struct Strip1 {
  const void* U;
  const int* bu;
  const void* Dn;
  const int* bd;
  int r;
};

// Lout[x,r,y] = sum L[a,l,b] U[a,u,x] A[l,r,u,d] Dn[b,d,y]
template <typename T, typename TT>
PV_HDN double s1_left(const Geom& g, Scratch<T>& sc, const Strip1& st, int c, T* Lout,
                     const T* Lin, const TT* A) {
  Dims dm;
  dm.set('a', st.bu[c]).set('x', st.bu[c + 1]).set('b', st.bd[c]).set('y', st.bd[c + 1]);
  dm.set('l', g.dl(c)).set('r', g.dr(c)).set('u', g.du(st.r)).set('d', g.dd(st.r));
  const T* U = (const T*)st.U + (long long)c * sc.d.ENV;
  const T* Dn = (const T*)st.Dn + (long long)c * sc.d.ENV;
  double fl = einsum(sc.t0, "lbux", Lin, "alb", U, "aux", dm);
  fl += einsum(sc.t1, "bxrd", sc.t0, "lbux", A, "lrud", dm);
  fl += einsum(Lout, "xry", sc.t1, "bxrd", Dn, "bdy", dm);
  return fl;
}

// Rout[a,l,b] = sum U[a,u,x] A[l,r,u,d] Dn[b,d,y] Rin[x,r,y]
template <typename T, typename TT>
PV_HDN double s1_right(const Geom& g, Scratch<T>& sc, const Strip1& st, int c, T* Rout,
                      const T* Rin, const TT* A) {
  Dims dm;
  dm.set('a', st.bu[c]).set('x', st.bu[c + 1]).set('b', st.bd[c]).set('y', st.bd[c + 1]);
  dm.set('l', g.dl(c)).set('r', g.dr(c)).set('u', g.du(st.r)).set('d', g.dd(st.r));
  const T* U = (const T*)st.U + (long long)c * sc.d.ENV;
  const T* Dn = (const T*)st.Dn + (long long)c * sc.d.ENV;
  double fl = einsum(sc.t0, "bdxr", Dn, "bdy", Rin, "xry", dm);
  fl += einsum(sc.t1, "lubx", A, "lrud", sc.t0, "bdxr", dm);
  fl += einsum(Rout, "alb", U, "aux", sc.t1, "lubx", dm);
  return fl;
}

// Env[l,r,u,d] = sum L[a,l,b] U[a,u,x] Dn[b,d,y] R[x,r,y]  (into sc.envo)
template <typename T>
PV_HDN double s1_env(const Geom& g, Scratch<T>& sc, const Strip1& st, int c, const T* L,
                    const T* R) {
  Dims dm;
  dm.set('a', st.bu[c]).set('x', st.bu[c + 1]).set('b', st.bd[c]).set('y', st.bd[c + 1]);
  dm.set('l', g.dl(c)).set('r', g.dr(c)).set('u', g.du(st.r)).set('d', g.dd(st.r));
  const T* U = (const T*)st.U + (long long)c * sc.d.ENV;
  const T* Dn = (const T*)st.Dn + (long long)c * sc.d.ENV;
  double fl = einsum(sc.t0, "lbux", L, "alb", U, "aux", dm);
  fl += einsum(sc.t1, "lbury", sc.t0, "lbux", R, "xry", dm);
  fl += einsum(sc.envo, "lrud", sc.t1, "lbury", Dn, "bdy", dm);
  return fl;
}

// Length of the right partial R_c of a one-row strip: [bu[c]][dl(c)][bd[c]] (R_{L2} is 1).
template <typename T>
PV_HD long long s1_len(const Strip1& st, const Geom& g, int c) {
  return (long long)st.bu[c] * (c < g.L2 ? g.dl(c) : 1) * st.bd[c];
}

// ---------------------------------------------------------------- two-row strips

struct Strip2 {
  const void* U;
  const int* bu;
  const void* Dn;
  const int* bd;
  int r;   // upper row
};

// Lout[x,r,s,y] = sum L[a,i,j,b] U[a,u,x] A1[i,r,u,m] A2[j,s,m,d] Dn[b,d,y]
template <typename T, typename TT>
PV_HDN double s2_left(const Geom& g, Scratch<T>& sc, const Strip2& st, int c, T* Lout,
                     const T* Lin, const TT* A1, const TT* A2) {
  Dims dm;
  dm.set('a', st.bu[c]).set('x', st.bu[c + 1]).set('b', st.bd[c]).set('y', st.bd[c + 1]);
  dm.set('i', g.dl(c)).set('r', g.dr(c)).set('j', g.dl(c)).set('s', g.dr(c));
  dm.set('u', g.du(st.r)).set('m', g.dd(st.r)).set('d', g.dd(st.r + 1));
  const T* U = (const T*)st.U + (long long)c * sc.d.ENV;
  const T* Dn = (const T*)st.Dn + (long long)c * sc.d.ENV;
  double fl = einsum(sc.t0, "ijbux", Lin, "aijb", U, "aux", dm);
  fl += einsum(sc.t1, "jbxrm", sc.t0, "ijbux", A1, "irum", dm);
  fl += einsum(sc.t0, "bxrsd", sc.t1, "jbxrm", A2, "jsmd", dm);
  fl += einsum(Lout, "xrsy", sc.t0, "bxrsd", Dn, "bdy", dm);
  return fl;
}

// Rout[a,i,j,b] = sum U[a,u,x] A1[i,r,u,m] A2[j,s,m,d] Dn[b,d,y] Rin[x,r,s,y]
template <typename T, typename TT>
PV_HDN double s2_right(const Geom& g, Scratch<T>& sc, const Strip2& st, int c, T* Rout,
                      const T* Rin, const TT* A1, const TT* A2) {
  Dims dm;
  dm.set('a', st.bu[c]).set('x', st.bu[c + 1]).set('b', st.bd[c]).set('y', st.bd[c + 1]);
  dm.set('i', g.dl(c)).set('r', g.dr(c)).set('j', g.dl(c)).set('s', g.dr(c));
  dm.set('u', g.du(st.r)).set('m', g.dd(st.r)).set('d', g.dd(st.r + 1));
  const T* U = (const T*)st.U + (long long)c * sc.d.ENV;
  const T* Dn = (const T*)st.Dn + (long long)c * sc.d.ENV;
  double fl = einsum(sc.t0, "bdxrs", Dn, "bdy", Rin, "xrsy", dm);
  fl += einsum(sc.t1, "jmbxr", A2, "jsmd", sc.t0, "bdxrs", dm);
  fl += einsum(sc.t0, "iujbx", A1, "irum", sc.t1, "jmbxr", dm);
  fl += einsum(Rout, "aijb", U, "aux", sc.t0, "iujbx", dm);
  return fl;
}

// Length of the right partial of a two-row strip: [bu[c]][dl(c)][dl(c)][bd[c]].
template <typename T>
PV_HD long long s2_len(const Strip2& st, const Geom& g, int c) {
  long long l = c < g.L2 ? g.dl(c) : 1;
  return (long long)st.bu[c] * l * l * st.bd[c];
}

// ---------------------------------------------------------------- per-sample driver

// Up environments of one chain kept between the Metropolis sweep and the evaluation:
// row boundaries 0..L1-1, tensors [L1][L2][ENV], bonds [L1][L2+1] (null when unused).
template <typename T>
struct UCache {
  T* env;
  int* bond;
};

template <typename T>
PV_HD void ucache_store(const Geom& g, Scratch<T>& sc, UCache<T> uc, int rb, const T* env,
                        const int* bond) {
  if (!uc.env) return;
  copy(uc.env + (long long)rb * g.L2 * sc.d.ENV, env, (long long)g.L2 * sc.d.ENV);
  for (int c = PV_TID; c <= g.L2; c += PV_NTHR) uc.bond[rb * (g.L2 + 1) + c] = bond[c];
  PV_SYNC();
}

struct SampleOut {
  double log_abs;
  int sign;
  double e_sys, e_anc;
};

template <typename T>
PV_HD double sz_of(int s) {
  return s == 0 ? 0.5 : -0.5;
}

// Builds all down environments (row boundaries L1-1 .. 1) for configuration sh.S.
template <typename T, typename TT>
PV_HDN double build_down(const Geom& g, Scratch<T>& sc, Shared<T>& sh, const TT* theta, T jtol,
                        int max_sweeps) {
  double fl = 0;
  T* envL = sc.envD + (long long)g.L1 * g.L2 * sc.d.ENV;
  int* bL = sc.bondD + g.L1 * (g.L2 + 1);
  trivial_env(g, sc, envL, bL);
  if (PV_TID == 0) sh.lsD[g.L1] = 0;
  PV_SYNC();
  for (int r = g.L1 - 1; r >= 1; --r) {
    T* envN = sc.envD + (long long)(r + 1) * g.L2 * sc.d.ENV;
    int* bN = sc.bondD + (r + 1) * (g.L2 + 1);
    if (PV_TID == 0) sh.lsD[r] = sh.lsD[r + 1];
    PV_SYNC();
    Product<T, TT> pr{envN, bN, true, r, theta, sh.S};
    fl += compress(g, sc, sh, g.du(r), pr, sc.envD + (long long)r * g.L2 * sc.d.ENV,
                   sc.bondD + r * (g.L2 + 1), &sh.lsD[r], jtol, max_sweeps);
  }
  return fl;
}

template <typename T>
PV_HD T* down_env(const Geom& g, Scratch<T>& sc, int r) {
  return sc.envD + (long long)r * g.L2 * sc.d.ENV;
}
template <typename T>
PV_HD int* down_bond(const Geom& g, Scratch<T>& sc, int r) {
  return sc.bondD + r * (g.L2 + 1);
}

// Evaluation of one configuration (already in sh.S): amplitude, E_sys, E_anc and, when
// O is non-null, the compressed O row.
// With uc.env set, the up environments come from the cache written by the sweep that
// produced this configuration (same contractions of the same rows: identical values).
template <typename T, typename TT, typename OT>
PV_HDN SampleOut eval_sample(const Geom& g, Scratch<T>& sc, Shared<T>& sh, const TT* theta,
                            OT* O, T jtol, int max_sweeps, UCache<T> uc) {
  SampleOut res;
  res.e_sys = res.e_anc = 0;
  double fl = build_down(g, sc, sh, theta, jtol, max_sweeps);
  const int L2 = g.L2;
  const unsigned char* S = sh.S;
  int cur = 0;
  trivial_env(g, sc, sc.envU[cur], sc.bondU[cur]);
  if (PV_TID == 0) sh.lsU[cur] = 0;
  PV_SYNC();
  for (int r = 0; r < g.L1; ++r) {
    const T* Uenv = uc.env ? uc.env + (long long)r * L2 * sc.d.ENV : sc.envU[cur];
    const int* Ubond = uc.env ? uc.bond + r * (L2 + 1) : sc.bondU[cur];
    Strip1 st{Uenv, Ubond, down_env(g, sc, r + 1), down_bond(g, sc, r + 1), r};
    // left and right partials of the one-row strip
    if (PV_TID == 0) {
      sc.p1L[0] = 1;
      sc.p1R[(long long)L2 * sc.d.P1] = 1;
    }
    PV_SYNC();
    for (int c = L2 - 1; c >= 0; --c)
      fl += s1_right(g, sc, st, c, sc.p1R + (long long)c * sc.d.P1,
                     sc.p1R + (long long)(c + 1) * sc.d.P1,
                     site_tensor(g, theta, r, c, S[r * L2 + c]));
    // the strip value is R_0 (a 1x1x1 tensor); left partials are rolled below
    T val = sc.p1R[0];
    if (r == 0) {
      T av = val < 0 ? -val : val;
      res.log_abs = (av > 0 ? log((double)av) : -INFINITY) + sh.lsD[1];
      res.sign = val > 0 ? 1 : (val < 0 ? -1 : 0);
    }
    // O rows of the sites of row r and horizontal bonds, with a rolling left partial Lc
    T* Lc = sc.p1L;
    T* Lnext = sc.p1L + sc.d.P1;
    for (int c = 0; c < L2; ++c) {
      if (O) {
        fl += s1_env(g, sc, st, c, Lc, sc.p1R + (long long)(c + 1) * sc.d.P1);
        long long n = g.sz(r, c);
        OT* o = O + g.o_off[r * L2 + c];
        double inv = 1.0 / (double)val;
        for (long long k = PV_TID; k < n; k += PV_NTHR) o[k] = (OT)((double)sc.envo[k] * inv);
        PV_SYNC();
      }
      if (c + 1 >= L2) break;
      int i = r * L2 + c, j = i + 1;
      int si = S[i] >> 1, sj = S[j] >> 1, ai = S[i] & 1, aj = S[j] & 1;
      res.e_sys += g.J1 * sz_of<T>(si) * sz_of<T>(sj);
      res.e_anc += g.J1 * sz_of<T>(ai) * sz_of<T>(aj);
      for (int layer = 0; layer < 2; ++layer) {
        int Si2, Sj2;
        if (layer == 0) {
          if (si == sj) continue;
          Si2 = 2 * sj + ai;
          Sj2 = 2 * si + aj;
        } else {
          if (ai == aj) continue;
          Si2 = 2 * si + aj;
          Sj2 = 2 * sj + ai;
        }
        fl += s1_left(g, sc, st, c, sc.m0, Lc, site_tensor(g, theta, r, c, Si2));
        fl += s1_left(g, sc, st, c + 1, sc.m1, sc.m0, site_tensor(g, theta, r, c + 1, Sj2));
        T num = dot(sc.m1, sc.p1R + (long long)(c + 2) * sc.d.P1, s1_len<T>(st, g, c + 2), sh.red);
        double ratio = (double)num / (double)val;
        if (layer == 0)
          res.e_sys += 0.5 * g.J1 * ratio;
        else
          res.e_anc += 0.5 * g.J1 * ratio;
      }
      fl += s1_left(g, sc, st, c, Lnext, Lc, site_tensor(g, theta, r, c, S[r * L2 + c]));
      T* tmp = Lc;
      Lc = Lnext;
      Lnext = tmp;
    }
    // two-row strip: vertical and next-nearest-neighbour bonds between rows r and r+1
    if (r + 1 < g.L1) {
      Strip2 s2{Uenv, Ubond, down_env(g, sc, r + 2), down_bond(g, sc, r + 2), r};
      if (PV_TID == 0) {
        sc.p2L[0] = 1;
        sc.p2R[(long long)L2 * sc.d.P2] = 1;
      }
      PV_SYNC();
      for (int c = L2 - 1; c >= 0; --c)
        fl += s2_right(g, sc, s2, c, sc.p2R + (long long)c * sc.d.P2,
                       sc.p2R + (long long)(c + 1) * sc.d.P2,
                       site_tensor(g, theta, r, c, S[r * L2 + c]),
                       site_tensor(g, theta, r + 1, c, S[(r + 1) * L2 + c]));
      T val2 = sc.p2R[0];
      T* L2c = sc.p2L;              // rolling left partial of the two-row strip
      T* L2n = sc.p2L + sc.d.P2;
      for (int c = 0; c < L2; ++c) {
        // vertical bond (r,c)-(r+1,c)
        {
          int i = r * L2 + c, j = i + L2;
          int si = S[i] >> 1, sj = S[j] >> 1, ai = S[i] & 1, aj = S[j] & 1;
          res.e_sys += g.J1 * sz_of<T>(si) * sz_of<T>(sj);
          res.e_anc += g.J1 * sz_of<T>(ai) * sz_of<T>(aj);
          for (int layer = 0; layer < 2; ++layer) {
            int Si2, Sj2;
            if (layer == 0) {
              if (si == sj) continue;
              Si2 = 2 * sj + ai;
              Sj2 = 2 * si + aj;
            } else {
              if (ai == aj) continue;
              Si2 = 2 * si + aj;
              Sj2 = 2 * sj + ai;
            }
            fl += s2_left(g, sc, s2, c, sc.m0, L2c, site_tensor(g, theta, r, c, Si2),
                          site_tensor(g, theta, r + 1, c, Sj2));
            T num = dot(sc.m0, sc.p2R + (long long)(c + 1) * sc.d.P2, s2_len<T>(s2, g, c + 1),
                        sh.red);
            double ratio = (double)num / (double)val2;
            if (layer == 0)
              res.e_sys += 0.5 * g.J1 * ratio;
            else
              res.e_anc += 0.5 * g.J1 * ratio;
          }
        }
        // next-nearest neighbours (r,c)-(r+1,c+1) and (r,c+1)-(r+1,c)
        if (g.J2 != 0.0 && c + 1 < L2) {
          for (int diag = 0; diag < 2; ++diag) {
            int i = diag == 0 ? r * L2 + c : r * L2 + c + 1;
            int j = diag == 0 ? (r + 1) * L2 + c + 1 : (r + 1) * L2 + c;
            int si = S[i] >> 1, sj = S[j] >> 1, ai = S[i] & 1, aj = S[j] & 1;
            res.e_sys += g.J2 * sz_of<T>(si) * sz_of<T>(sj);
            res.e_anc += g.J2 * sz_of<T>(ai) * sz_of<T>(aj);
            for (int layer = 0; layer < 2; ++layer) {
              int Si2, Sj2;
              if (layer == 0) {
                if (si == sj) continue;
                Si2 = 2 * sj + ai;
                Sj2 = 2 * si + aj;
              } else {
                if (ai == aj) continue;
                Si2 = 2 * si + aj;
                Sj2 = 2 * sj + ai;
              }
              // modified local indices of the four sites of columns c, c+1
              int s00 = S[r * L2 + c], s01 = S[r * L2 + c + 1];
              int s10 = S[(r + 1) * L2 + c], s11 = S[(r + 1) * L2 + c + 1];
              if (diag == 0) {
                s00 = Si2;
                s11 = Sj2;
              } else {
                s01 = Si2;
                s10 = Sj2;
              }
              fl += s2_left(g, sc, s2, c, sc.m0, L2c, site_tensor(g, theta, r, c, s00),
                            site_tensor(g, theta, r + 1, c, s10));
              fl += s2_left(g, sc, s2, c + 1, sc.m1, sc.m0, site_tensor(g, theta, r, c + 1, s01),
                            site_tensor(g, theta, r + 1, c + 1, s11));
              T num = dot(sc.m1, sc.p2R + (long long)(c + 2) * sc.d.P2, s2_len<T>(s2, g, c + 2),
                          sh.red);
              double ratio = (double)num / (double)val2;
              if (layer == 0)
                res.e_sys += 0.5 * g.J2 * ratio;
              else
                res.e_anc += 0.5 * g.J2 * ratio;
            }
          }
        }
        // advance the left partial past column c
        fl += s2_left(g, sc, s2, c, L2n, L2c, site_tensor(g, theta, r, c, S[r * L2 + c]),
                      site_tensor(g, theta, r + 1, c, S[(r + 1) * L2 + c]));
        T* t2p = L2c;
        L2c = L2n;
        L2n = t2p;
      }
      // absorb row r into the up environment (unless the cache holds it)
      if (!uc.env) {
        int nxt = cur ^ 1;
        if (PV_TID == 0) sh.lsU[nxt] = sh.lsU[cur];
        PV_SYNC();
        Product<T, TT> pr{sc.envU[cur], sc.bondU[cur], false, r, theta, S};
        fl += compress(g, sc, sh, g.dd(r), pr, sc.envU[nxt], sc.bondU[nxt], &sh.lsU[nxt], jtol,
                       max_sweeps);
        cur = nxt;
      }
    }
  }
  if (PV_TID == 0) sh.flops += fl;
  PV_SYNC();
  return res;
}

// Metropolis test for target |rho|^p.
PV_HD bool mc_accept(double u, double ratio, int p) {
  double q = p == 2 ? ratio * ratio : (ratio < 0 ? -ratio : ratio);
  return u < q;
}

// One Metropolis sweep of one chain (configuration in sh.S, updated in place).
// Move m at site i has counter (chain, sweep, 8 i + m, TAG_MC).  The strip value of the
// current configuration (the ratio's denominator) and the advanced left partial are kept
// between proposals: they are the same contractions of the same operands, so reusing them
// changes no value.
template <typename T, typename TT>
PV_HDN void mc_sweep(const Geom& g, Scratch<T>& sc, Shared<T>& sh, const TT* theta, int p,
                     uint64_t seed, uint32_t chain, uint32_t sweep, T jtol, int max_sweeps,
                     int* n_acc, int* n_prop, UCache<T> uc) {
  double fl = build_down(g, sc, sh, theta, jtol, max_sweeps);
  const int L2 = g.L2;
  unsigned char* S = sh.S;
  int cur = 0;
  trivial_env(g, sc, sc.envU[cur], sc.bondU[cur]);
  if (PV_TID == 0) sh.lsU[cur] = 0;
  PV_SYNC();
  ucache_store(g, sc, uc, 0, sc.envU[cur], sc.bondU[cur]);
  int acc = 0, prop = 0;
  auto take = [&](bool accepted, int i, int Si2, int j, int Sj2) {
    if (accepted) {
      ++acc;
      PV_SYNC();
      if (PV_TID == 0) {
        S[i] = (unsigned char)Si2;
        if (j >= 0) S[j] = (unsigned char)Sj2;
      }
      PV_SYNC();
    }
  };
  for (int r = 0; r < g.L1; ++r) {
    Strip1 st{sc.envU[cur], sc.bondU[cur], down_env(g, sc, r + 1), down_bond(g, sc, r + 1), r};
    if (PV_TID == 0) {
      sc.p1L[0] = 1;
      sc.p1R[(long long)L2 * sc.d.P1] = 1;
    }
    PV_SYNC();
    for (int c = L2 - 1; c >= 0; --c)
      fl += s1_right(g, sc, st, c, sc.p1R + (long long)c * sc.d.P1,
                     sc.p1R + (long long)(c + 1) * sc.d.P1,
                     site_tensor(g, theta, r, c, S[r * L2 + c]));
    // Lc: left partial up to column c; P = Lc x column c (current S); Q = P x column c+1.
    T* Lc = sc.p1L;
    T* P = sc.m0;
    T* Q = sc.m1;
    T* X = sc.m2;
    T* Y = sc.m3;
    fl += s1_left(g, sc, st, 0, P, Lc, site_tensor(g, theta, r, 0, S[r * L2]));
    for (int c = 0; c < L2; ++c) {
      int i = r * L2 + c;
      const T* R1 = sc.p1R + (long long)(c + 1) * sc.d.P1;
      long long n1 = s1_len<T>(st, g, c + 1);
      // move 0: both-flip of site i
      {
        T den = dot(P, R1, n1, sh.red);
        fl += s1_left(g, sc, st, c, X, Lc, site_tensor(g, theta, r, c, 3 - S[i]));
        T num = dot(X, R1, n1, sh.red);
        double u = philox_uniform(seed, chain, sweep, (uint32_t)(8 * i + 0), TAG_MC);
        ++prop;
        bool a = mc_accept(u, (double)num / (double)den, p);
        take(a, i, 3 - S[i], -1, 0);
        if (a) {
          T* t = P;
          P = X;
          X = t;
        }
      }
      // moves 1, 2: system / ancilla exchange with (r, c+1)
      bool q_valid = false;   // Q == P x column c+1 at the current S
      if (c + 1 < L2) {
        const T* R2 = sc.p1R + (long long)(c + 2) * sc.d.P1;
        long long n2 = s1_len<T>(st, g, c + 2);
        for (int layer = 0; layer < 2; ++layer) {
          int j = i + 1;
          int si = S[i] >> 1, sj = S[j] >> 1, ai = S[i] & 1, aj = S[j] & 1;
          int Si2, Sj2;
          if (layer == 0) {
            if (si == sj) continue;
            Si2 = 2 * sj + ai;
            Sj2 = 2 * si + aj;
          } else {
            if (ai == aj) continue;
            Si2 = 2 * si + aj;
            Sj2 = 2 * sj + ai;
          }
          if (!q_valid) {
            fl += s1_left(g, sc, st, c + 1, Q, P, site_tensor(g, theta, r, c + 1, S[j]));
            q_valid = true;
          }
          T den = dot(Q, R2, n2, sh.red);
          fl += s1_left(g, sc, st, c, X, Lc, site_tensor(g, theta, r, c, Si2));
          fl += s1_left(g, sc, st, c + 1, Y, X, site_tensor(g, theta, r, c + 1, Sj2));
          T num = dot(Y, R2, n2, sh.red);
          double u = philox_uniform(seed, chain, sweep, (uint32_t)(8 * i + 1 + layer), TAG_MC);
          ++prop;
          bool a = mc_accept(u, (double)num / (double)den, p);
          take(a, i, Si2, j, Sj2);
          if (a) {
            T* t = P;
            P = X;
            X = t;
            t = Q;
            Q = Y;
            Y = t;
          }
        }
      }
      // advance: the left partial past column c is P
      T* Ln = (Lc == sc.p1L) ? sc.p1L + sc.d.P1 : sc.p1L;
      copy(Ln, P, s1_len<T>(st, g, c + 1));
      Lc = Ln;
      if (c + 1 < L2) {
        if (q_valid) {
          T* t = P;
          P = Q;
          Q = t;
        } else {
          fl += s1_left(g, sc, st, c + 1, P, Lc, site_tensor(g, theta, r, c + 1, S[i + 1]));
        }
      }
    }
    if (r + 1 < g.L1) {
      Strip2 s2{sc.envU[cur], sc.bondU[cur], down_env(g, sc, r + 2), down_bond(g, sc, r + 2), r};
      if (PV_TID == 0) {
        sc.p2L[0] = 1;
        sc.p2R[(long long)L2 * sc.d.P2] = 1;
      }
      PV_SYNC();
      for (int c = L2 - 1; c >= 0; --c)
        fl += s2_right(g, sc, s2, c, sc.p2R + (long long)c * sc.d.P2,
                       sc.p2R + (long long)(c + 1) * sc.d.P2,
                       site_tensor(g, theta, r, c, S[r * L2 + c]),
                       site_tensor(g, theta, r + 1, c, S[(r + 1) * L2 + c]));
      T* L2c = sc.p2L;
      T* P2 = sc.m0;
      T* X2 = sc.m1;
      for (int c = 0; c < L2; ++c) {
        int i = r * L2 + c, j = i + L2;
        const T* R = sc.p2R + (long long)(c + 1) * sc.d.P2;
        long long n = s2_len<T>(s2, g, c + 1);
        fl += s2_left(g, sc, s2, c, P2, L2c, site_tensor(g, theta, r, c, S[i]),
                      site_tensor(g, theta, r + 1, c, S[j]));
        T den = 0;
        bool den_valid = false;
        for (int layer = 0; layer < 2; ++layer) {
          int si = S[i] >> 1, sj = S[j] >> 1, ai = S[i] & 1, aj = S[j] & 1;
          int Si2, Sj2;
          if (layer == 0) {
            if (si == sj) continue;
            Si2 = 2 * sj + ai;
            Sj2 = 2 * si + aj;
          } else {
            if (ai == aj) continue;
            Si2 = 2 * si + aj;
            Sj2 = 2 * sj + ai;
          }
          if (!den_valid) {
            den = dot(P2, R, n, sh.red);
            den_valid = true;
          }
          fl += s2_left(g, sc, s2, c, X2, L2c, site_tensor(g, theta, r, c, Si2),
                        site_tensor(g, theta, r + 1, c, Sj2));
          T num = dot(X2, R, n, sh.red);
          double u = philox_uniform(seed, chain, sweep, (uint32_t)(8 * i + 3 + layer), TAG_MC);
          ++prop;
          bool a = mc_accept(u, (double)num / (double)den, p);
          take(a, i, Si2, j, Sj2);
          if (a) {
            T* t = P2;
            P2 = X2;
            X2 = t;
            den = num;
          }
        }
        T* Ln = (L2c == sc.p2L) ? sc.p2L + sc.d.P2 : sc.p2L;
        copy(Ln, P2, s2_len<T>(s2, g, c + 1));
        L2c = Ln;
      }
      int nxt = cur ^ 1;
      if (PV_TID == 0) sh.lsU[nxt] = sh.lsU[cur];
      PV_SYNC();
      Product<T, TT> pr{sc.envU[cur], sc.bondU[cur], false, r, theta, S};
      fl += compress(g, sc, sh, g.dd(r), pr, sc.envU[nxt], sc.bondU[nxt], &sh.lsU[nxt], jtol,
                     max_sweeps);
      cur = nxt;
      ucache_store(g, sc, uc, r + 1, sc.envU[cur], sc.bondU[cur]);
    }
  }
  if (PV_TID == 0) sh.flops += fl;
  PV_SYNC();
  *n_acc = acc;
  *n_prop = prop;
}

}  // namespace pv
