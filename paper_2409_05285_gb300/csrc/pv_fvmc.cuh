// Metropolis sampling and stochastic reconfiguration of the fermionic thermal state (Sec. II,
// MCMC and Eqs. 5-10, on the fermionic PEPS of Fig. 1b for the Hubbard model of Sec. III.B):
// proposals and acceptance decisions per chain, the sample weights and observables, and the
// column sums of O rows over sixteen local states.  The CG kernels of pv_sr.cuh serve
// unchanged: they address theta through the slice S_ij times the slice size.
//
// Moves of one sweep (fermion_moves, in row phases): per row, for every column the
// system-ancilla pairs of its site created or removed (spin up, then down; only where c_s and
// d_s are equally occupied) and one electron of mode k = 0..3 hopping across its horizontal
// bond (only where the two occupations differ); then the hops across the vertical bonds to
// the next row, column by column.  A move that does not apply is skipped.  Both kinds keep the total
// parity even and N_s(c) - N_s(d) fixed, and each is its own inverse (symmetric proposals).
#ifndef PV_FVMC_CUH
#define PV_FVMC_CUH
#include <cstdint>
#include <vector>

#include "pv_fermion.cuh"
#include "pv_philox.cuh"
#include "pv_sr.cuh"

namespace pv {

// kind 0: pair of spin k at site i; kind 1: mode k across the bond (i, j)
struct FMove {
  int kind, i, j, k;
};

// The moves of one sweep in order: per row, for every column the pairs of its site (spin up,
// then down) and the hops of its horizontal bond (modes 0..3); then the hops of the vertical
// bonds to the next row, column by column.
inline std::vector<FMove> fermion_moves(int L1, int L2) {
  std::vector<FMove> out;
  for (int r = 0; r < L1; ++r) {
    for (int q = 0; q < L2; ++q) {
      const int i = r * L2 + q;
      for (int sp = 0; sp < 2; ++sp) out.push_back(FMove{0, i, i, sp});
      if (q + 1 < L2)
        for (int k = 0; k < 4; ++k) out.push_back(FMove{1, i, i + 1, k});
    }
    if (r + 1 < L1)
      for (int q = 0; q < L2; ++q)
        for (int k = 0; k < 4; ++k) out.push_back(FMove{1, r * L2 + q, (r + 1) * L2 + q, k});
  }
  return out;
}

// Observables of the samples: <H> per lattice (Eq. 11), its standard error, the double
// occupancy and the density summed over the sites (both layers averaged), and the number
// of samples whose amplitude vanishes.
struct FObs {
  double H1, Eerr, docc, dens;
  int zero, pad;
};

#if defined(__CUDACC__)

// The strip forms' per-chain functors (fermion_mc, fermion_eloc) on the device: one thread per
// chain through the batched engine's element kernel.
template <typename T, typename OT, typename F>
inline void fv_apply(CudaBE<T, OT>& be, const F& f, int n) {
  PV_KLAUNCH(be.prof, be.st, "kb_elem_fermion", 0.0, 0.0,
             kb_elem<<<CudaBE<T, OT>::gx(n, 128), 128, 0, be.st>>>(f, n));
}

// The 64 slices per site of the strip forms from the sixteen of theta (float64, per site
// [16][dl][dr][du][dd]): slice S + 16 b + 32 x is T[S] times (-1)^((p(S) + p(d)) (p(l) + p(u))
// + p(d) b + x p(r)).  Block y = site, threads over slice x element.
template <typename T>
__global__ void k_fsigned64(int L1, int L2, int D, const double* __restrict__ th16,
                            const long long* __restrict__ toff16, T* __restrict__ th64,
                            const long long* __restrict__ toff64) {
  const int i = blockIdx.y, r = i / L2, c = i % L2;
  const int dl = c == 0 ? 1 : D, dr = c == L2 - 1 ? 1 : D, du = r == 0 ? 1 : D, dd = r == L1 - 1 ? 1 : D;
  const long long sz = (long long)dl * dr * du * dd;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < 64 * sz;
       e += (long long)gridDim.x * blockDim.x) {
    const int slice = (int)(e / sz), S = slice & 15, bb = (slice >> 4) & 1, x = slice >> 5;
    const long long k = e - (long long)slice * sz;
    long long t = k;
    const int d = (int)(t % dd);
    t /= dd;
    const int u = (int)(t % du);
    t /= du;
    const int rr = (int)(t % dr);
    t /= dr;
    const int l = (int)t;
    const int pS = __popc(S) & 1;
    const int ex = (pS + (d & 1)) * ((l & 1) + (u & 1)) + (d & 1) * bb + x * (rr & 1);
    const double v = th16[toff16[i] + (long long)S * sz + k];
    th64[toff64[i] + e] = (T)((ex & 1) ? -v : v);
  }
}

// Sp = S with move mv applied, per chain; act = 1 where the move applies (else 0, Sp = S).
__global__ void k_fpropose(int nb, int N, const uint8_t* __restrict__ S, uint8_t* __restrict__ Sp,
                           FMove mv, int* __restrict__ act) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nb) return;
  const uint8_t* x = S + (long long)s * N;
  uint8_t* y = Sp + (long long)s * N;
  for (int q = 0; q < N; ++q) y[q] = x[q];
  int ok;
  if (mv.kind == 0) {
    ok = ((x[mv.i] >> mv.k) & 1) == ((x[mv.i] >> (2 + mv.k)) & 1);
    if (ok) y[mv.i] = (uint8_t)(x[mv.i] ^ ((1 << mv.k) | (1 << (2 + mv.k))));
  } else {
    ok = ((x[mv.i] >> mv.k) & 1) != ((x[mv.j] >> mv.k) & 1);
    if (ok) {
      y[mv.i] = (uint8_t)(x[mv.i] ^ (1 << mv.k));
      y[mv.j] = (uint8_t)(x[mv.j] ^ (1 << mv.k));
    }
  }
  act[s] = ok;
}

// The proposed rows of the chains where the move applies, packed: row s to position pos[s].
__global__ void k_fgather(int nb, int N, const uint8_t* __restrict__ Sp, const int* __restrict__ act,
                          const int* __restrict__ pos, uint8_t* __restrict__ Sc) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nb * N) return;
  const int s = (int)(e / N), q = (int)(e % N);
  if (act[s]) Sc[(long long)pos[s] * N + q] = Sp[e];
}

// The decision on move m for every chain where it applies, target |psi|^p: accept iff log u <
// p (log|psi'| - log|psi|) in float64, psi' = 0 rejected; psi' of chain s at the packed
// position pos[s].  u from the caller ([chain][move]) or from Philox4x32-10 (seed; counter
// chain, sweep, m, TAG_FMC).
__global__ void k_faccept(int nb, int N, int m, int n_moves, int p, uint64_t seed, uint32_t sweep,
                          const double* __restrict__ u, const int* __restrict__ act,
                          const int* __restrict__ pos, const double* __restrict__ la2,
                          const int8_t* __restrict__ sg2, uint8_t* __restrict__ S,
                          const uint8_t* __restrict__ Sp, double* __restrict__ la,
                          int8_t* __restrict__ sg, int* __restrict__ acc) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nb || !act[s]) return;
  const int c = pos[s];
  if (sg2[c] == 0) return;
  const double us = u ? u[(long long)s * n_moves + m]
                      : philox_uniform(seed, (uint32_t)s, sweep, (uint32_t)m, TAG_FMC);
  const double d = log(us) - p * (la2[c] - la[s]);
  if (d < 0.0) {
    for (int q = 0; q < N; ++q) S[(long long)s * N + q] = Sp[(long long)s * N + q];
    la[s] = la2[c];
    sg[s] = sg2[c];
    acc[s] += 1;
  }
}

// Weights and observables (one block): w_i = 1/n (p = 2, samples of |psi|^2) or |psi_i| /
// sum_j |psi_j| (p = 1, samples of |psi|, Eq. A1); E_i = E_sys + E_anc and Ebar = sum w E
// for the gradient; <H> = sum w (E_sys + E_anc)/2 with the delta-method error sqrt(sum w^2
// (h - <H>)^2); the double occupancy and density per configuration (n_up n_dn and n_up +
// n_dn summed over the sites, the two layers averaged).  Samples with psi = 0 are counted.
__global__ void k_fweights(int n, int N, int p, const double* __restrict__ la,
                           const int8_t* __restrict__ sg, const double* __restrict__ es,
                           const double* __restrict__ ea, const uint8_t* __restrict__ S,
                           double* __restrict__ w, double* __restrict__ E, SRScalars* sc,
                           FObs* fo) {
  __shared__ double red[32];
  double mx = -INFINITY;
  if (p == 1)
    for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, la[i]);
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ double redm[32];
  if ((threadIdx.x & 31) == 0) redm[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = redm[0];
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) mx = fmax(mx, redm[i]);
  double zs = 0, zero = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    zs += (p == 2) ? 1.0 : exp(la[i] - mx);
    zero += sg[i] == 0;
  }
  const double Z = blk_sum(zs, red);
  zero = blk_sum(zero, red);
  double e1 = 0, h1 = 0, dc = 0, dn = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double wi = ((p == 2) ? 1.0 : exp(la[i] - mx)) / Z;
    w[i] = wi;
    const double a = es[i], b = ea[i];
    E[i] = a + b;
    e1 += wi * (a + b);
    h1 += wi * 0.5 * (a + b);
    int d2 = 0, nn = 0;
    for (int j = 0; j < N; ++j) {
      const int x = S[(long long)i * N + j];
      d2 += (x & 1) * ((x >> 1) & 1) + ((x >> 2) & 1) * ((x >> 3) & 1);
      nn += __popc(x & 15);
    }
    dc += wi * 0.5 * d2;
    dn += wi * 0.5 * nn;
  }
  e1 = blk_sum(e1, red);
  h1 = blk_sum(h1, red);
  dc = blk_sum(dc, red);
  dn = blk_sum(dn, red);
  double ve = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = 0.5 * (es[i] + ea[i]) - h1;
    ve += w[i] * w[i] * d * d;
  }
  ve = blk_sum(ve, red);
  if (threadIdx.x == 0) {
    sc->Ebar = e1;
    sc->H1 = h1;
    fo->H1 = h1;
    fo->Eerr = sqrt(ve);
    fo->docc = dc;
    fo->dens = dn;
    fo->zero = (int)zero;
  }
}

// Stage 1 of the segmented column sums over samples with sixteen local states: for column o
// of the O rows and the chunk of OTV_CHUNK samples of block y, acc[S_ij] += c1_i O[i][o] (and
// c1_i (c2_i - shift) O[i][o] for TWO), in sample order, written to part[chunk][theta index]
// for all sixteen slices of the column (k_colsum2_grad or k_otv2 then sums the chunks).
template <typename OT, bool TWO>
__global__ void k_fcolsum1(int n, int N, long long No, const OT* __restrict__ O,
                           const uint8_t* __restrict__ S, const int* __restrict__ o2site,
                           const long long* __restrict__ toff, const long long* __restrict__ ooff,
                           const double* __restrict__ c1, const double* __restrict__ c2,
                           const double* __restrict__ shift, double* __restrict__ part1,
                           double* __restrict__ part2, long long Np, const int* done) {
  if (done && *done) return;
  const double sh = TWO ? *shift : 0.0;
  const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= No) return;
  const int ch = blockIdx.y;
  const int i0 = ch * OTV_CHUNK, i1 = min(n, i0 + OTV_CHUNK);
  const int j = o2site[o];
  const long long k = o - ooff[j], sz = ooff[j + 1] - ooff[j];
  double a[16], b[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    a[q] = 0.0;
    b[q] = 0.0;
  }
  for (int i = i0; i < i1; ++i) {
    const double v = (double)O[(long long)i * No + o];
    const int s = S[(long long)i * N + j];
    const double x = c1[i] * v;
    const double y = TWO ? c1[i] * (c2[i] - sh) * v : 0.0;
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (s == q) {
        a[q] += x;
        if (TWO) b[q] += y;
      }
  }
  const long long t = toff[j] + k;
  double* p1 = part1 + (long long)ch * Np;
#pragma unroll
  for (int q = 0; q < 16; ++q) p1[t + q * sz] = a[q];
  if (TWO) {
    double* p2 = part2 + (long long)ch * Np;
#pragma unroll
    for (int q = 0; q < 16; ++q) p2[t + q * sz] = b[q];
  }
}

#endif  // __CUDACC__

}  // namespace pv
#endif
