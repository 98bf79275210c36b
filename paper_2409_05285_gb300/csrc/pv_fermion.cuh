// Amplitudes of a fermionic PEPS of the doubled Hubbard lattice (Sec. II, Fig. 1b; Sec. III.B)
// on the batched engine.
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
