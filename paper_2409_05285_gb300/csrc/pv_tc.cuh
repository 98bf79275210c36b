// Tensor-core contractions of the batched engine (float32 storage, TF32 multiplies, FP32
// accumulation): one strided GEMM per chain, C[m][n] = sum_k P[m][k] Q[n][k], where the row,
// column and contraction indices are multi-indices with arbitrary strides (the transfer
// contractions of the boundary-MPS environments and strips, Sec. II).
//
// A CTA of four warps owns one 128-row tile of one chain at a time and loops over chains.
// Per contraction chunk of Kc (<= 64) indices every thread gathers operand elements from
// global memory, rounds them to TF32 and writes them into shared memory in the canonical
// K-major layout without swizzle (core matrices of 8 rows x 16 bytes stored as 128
// contiguous bytes); one thread issues Kc/8 `tcgen05.mma.kind::tf32` instructions
// (M = 128, N = the tile width) into an accumulator in tensor memory and commits them to an
// mbarrier; after the last chunk each warp reads its 32 accumulator lanes with
// `tcgen05.ld` and scatters them to C.  Rows of a chunk past the edge of C are not gathered
// (they only reach accumulator rows and columns that are not stored), and a Gram product
// C = P P^T that one tile covers gathers P once: the B descriptor points at the A stage.
// Every wait on the mbarrier is bounded: when it runs out the kernel raises `err`, waits once
// more, frees its tensor memory and returns (err bit 2 when that second wait ran out too).
#ifndef PV_TC_CUH
#define PV_TC_CUH
#include <cstdint>

namespace pv {

// Index plan of one tensor-core contraction; rows are the larger of the two free sides.
struct TcSpec {
  int nr, nc, nk;
  int rs[4], rP[4], rC[4];   // row dims: sizes, strides in P, strides in C
  int cs[4], cQ[4], cC[4];   // column dims: sizes, strides in Q, strides in C
  int ks[4], kP[4], kQ[4];   // contraction dims: sizes, strides in P and in Q
  int M, N, K;
  int TN;                    // tile width: a multiple of 16, at most 256
  int Kc;                    // contraction chunk: a multiple of 8, at most 64
  int modeP, modeQ;          // operand gather forms (TC_SCALAR, TC_VEC_K, TC_VEC_T)
  int vecC;                  // 16-byte stores of four consecutive columns of C
  int pref;                  // one chunk small enough to stage in registers (next chain prefetched)
  int split;                 // 3xTF32: operands as hi + lo TF32 parts, products hi.hi + hi.lo + lo.hi
  int nst;                   // operand stages / accumulators: 2 pipelines consecutive chains
  int sym;                   // Q is P with the same index maps (C = P P^T, one tile): the B
                             // operand is read from the A stage instead of being gathered
  int no_mma;                // self-test only: issue no MMA and no commit, so every wait runs out
  int ns;                    // pipelined kernel: shared-memory stages of the copy ring
  int nacc;                  // pipelined kernel: accumulators in tensor memory (1 or 2)
};

constexpr int TC_ROWS = 128;
constexpr int TC_THREADS = 128;
constexpr int TC_KMAX = 64;
constexpr unsigned long long TC_WAIT_NS = 1000000000ull;   // bound of one completion wait (1 s)
constexpr int TC_SCALAR = 0, TC_VEC_K = 1, TC_VEC_T = 2;

// Plans C = A.B of a GEMM-shaped contraction for the tensor cores; false when the shape
// does not suit them (no contraction worth the name, or both free sides small).
inline bool tc_plan(const GSpec& g, TcSpec& t, bool& swap, int tc_min_rows = 64) {
  if (!g.ok || g.K < 4 || g.K > 4096) return false;
  swap = g.N > g.M;
  const int M = swap ? g.N : g.M, N = swap ? g.M : g.N;
  if (M < tc_min_rows) return false;
  t.M = M;
  t.N = N;
  t.K = g.K;
  t.nr = swap ? g.nn : g.nm;
  t.nc = swap ? g.nm : g.nn;
  t.nk = g.nk;
  for (int d = 0; d < 4; ++d) {
    t.rs[d] = swap ? g.ns[d] : g.ms[d];
    t.rP[d] = swap ? g.nB[d] : g.mA[d];
    t.rC[d] = swap ? g.nC[d] : g.mC[d];
    t.cs[d] = swap ? g.ms[d] : g.ns[d];
    t.cQ[d] = swap ? g.mA[d] : g.nB[d];
    t.cC[d] = swap ? g.mC[d] : g.nC[d];
    t.ks[d] = g.ks[d];
    t.kP[d] = swap ? g.kB[d] : g.kA[d];
    t.kQ[d] = swap ? g.kA[d] : g.kB[d];
  }
  int n16 = ((N + 15) / 16) * 16;
  t.TN = n16 < 256 ? n16 : 256;
  int k8 = ((g.K + 7) / 8) * 8;
  t.Kc = k8 < TC_KMAX ? k8 : TC_KMAX;
  t.modeP = t.modeQ = TC_SCALAR;
  t.vecC = 0;
  // register staging holds 16 values of P and 8 of Q per thread
  t.pref = (g.K <= t.Kc && t.Kc <= 16 && t.TN * t.Kc <= 1024) ? 1 : 0;
  t.split = 0;
  t.nst = 1;
  t.sym = 0;
  t.no_mma = 0;
  t.ns = 2;
  t.nacc = 1;
  return true;
}

// Whether C = P Q^T is a Gram product P P^T that one tile covers: the column side and its
// strides in Q are the row side and its strides in P, the contraction strides agree, and the
// caller passes the same operand twice (`same`).
inline bool tc_symmetric(const TcSpec& t, bool same) {
  if (!same || t.M != t.N || t.M > TC_ROWS || t.TN < t.N || t.nr != t.nc) return false;
  for (int d = 0; d < t.nr; ++d)
    if (t.rs[d] != t.cs[d] || t.rP[d] != t.cQ[d]) return false;
  for (int d = 0; d < t.nk; ++d)
    if (t.kP[d] != t.kQ[d]) return false;
  return t.modeP == t.modeQ;
}

inline bool tc_all4(const int* st, int n) {
  for (int d = 0; d < n; ++d)
    if (st[d] % 4) return false;
  return true;
}

// Operand form: 16-byte loads along the contraction index or along the rows when the
// operand is unit-stride there in blocks of four and every other stride keeps 16-byte
// alignment (`al`: the operand's base and per-chain offsets are multiples of 16 bytes).
inline int tc_mode(bool al, int nr, const int* rsz, const int* rst, int nk, const int* ksz,
                   const int* kst) {
  if (!al) return TC_SCALAR;
  if (nk > 0 && kst[nk - 1] == 1 && ksz[nk - 1] % 4 == 0 && tc_all4(kst, nk - 1) &&
      tc_all4(rst, nr))
    return TC_VEC_K;
  if (nr > 0 && rst[nr - 1] == 1 && rsz[nr - 1] % 4 == 0 && tc_all4(rst, nr - 1) &&
      tc_all4(kst, nk))
    return TC_VEC_T;
  return TC_SCALAR;
}

inline void tc_forms(TcSpec& t, bool p_al, bool q_al, bool c_al) {
  t.modeP = tc_mode(p_al, t.nr, t.rs, t.rP, t.nk, t.ks, t.kP);
  t.modeQ = tc_mode(q_al, t.nc, t.cs, t.cQ, t.nk, t.ks, t.kQ);
  t.vecC = (c_al && t.nc > 0 && t.cC[t.nc - 1] == 1 && t.cs[t.nc - 1] % 4 == 0 &&
            tc_all4(t.cC, t.nc - 1) && tc_all4(t.rC, t.nr)) ? 1 : 0;
  if (t.modeP == TC_SCALAR || t.modeQ == TC_SCALAR) t.pref = 0;
}

// Operand stages: two (double buffering across chains) when the planner chose it (one
// chunk per chain, small stages), else one.
PV_HD int tc_stages(const TcSpec& t) { return t.nst; }

// Bytes of one operand stage: the A chunk (128 rows), the B chunk (TN rows) unless B is read
// from A, both twice for split operands.
inline size_t tc_stage_bytes(const TcSpec& t) {
  return (size_t)(TC_ROWS + (t.sym ? 0 : t.TN)) * t.Kc * sizeof(float) * (t.split ? 2 : 1);
}

inline size_t tc_smem_bytes(const TcSpec& t) {
  return tc_stage_bytes(t) * tc_stages(t) + (size_t)(2 * TC_ROWS + 2 * t.TN + 2 * t.K) * sizeof(int);
}

PV_HD int tc_cols(int TN) {
  int c = 32;
  while (c < TN) c <<= 1;
  return c;
}

#if defined(__CUDACC__)

__device__ __forceinline__ uint32_t tc_smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading-dimension byte offset (between
// core matrices along K), stride-dimension byte offset (between 8-row groups), descriptor
// version 1 (bits 46-47), base offset 0, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32: D float32 (bits 4-5 = 1), A and B TF32 (bits 7-9 and
// 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float tc_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ unsigned long long tc_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the phase `parity` of an mbarrier to complete; false after TC_WAIT_NS.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = tc_now();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (tc_now() - t0 > TC_WAIT_NS) return false;
  }
}

// 16 consecutive accumulator columns of this thread's lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Operand chunk (rows x Kc) to shared memory, rounded to TF32, in the canonical K-major
// layout without swizzle: core matrix (g, q) of rows 8g..8g+7 and contraction indices
// 4q..4q+3 at element offset (g * Kc/4 + q) * 32, row-major inside (16 bytes per row).
// Three gather forms fill it:
//  TC_SCALAR  element loads;
//  TC_VEC_K   16-byte loads of four consecutive contraction indices (the operand is
//             unit-stride in its innermost contraction index), one 16-byte store each;
//  TC_VEC_T   16-byte loads of four consecutive rows (the operand is unit-stride in its
//             innermost row index): four lanes load a 4 x 4 block at four contraction
//             indices, transpose it with shuffles and store one row each.
// Each thread issues TC_UNROLL independent loads before it stores.
constexpr int TC_UNROLL = 4;

__device__ __forceinline__ float4 tc_round4(float4 v) {
  return make_float4(tc_round(v.x), tc_round(v.y), tc_round(v.z), tc_round(v.w));
}

// Stores the TF32 rounding of v, and, for split operands, the rounding of the remainder.
__device__ __forceinline__ void tc_st(float* hi, float* lo, int e, float v) {
  const float h = tc_round(v);
  hi[e] = h;
  if (lo) lo[e] = tc_round(v - h);
}
__device__ __forceinline__ void tc_st4(float* hi, float* lo, int e, float4 v) {
  const float4 h = tc_round4(v);
  ((float4*)hi)[e] = h;
  if (lo) ((float4*)lo)[e] = tc_round4(make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w));
}

__device__ __forceinline__ void tc_gather(float* dst, float* dlo, const float* __restrict__ src,
                                          int mode, int rows, int Kc, int k0, int K,
                                          const int* roff, const int* koff, int tid) {
  if (mode == TC_SCALAR) {
    const int qn = Kc >> 2, total = rows * Kc;
    for (int e0 = tid; e0 < total; e0 += TC_THREADS * TC_UNROLL) {
      float v[TC_UNROLL];
#pragma unroll
      for (int u = 0; u < TC_UNROLL; ++u) {
        const int e = e0 + u * TC_THREADS;
        v[u] = 0.f;
        if (e < total) {
          const int cm = e >> 5, j = e & 31;
          const int g = cm / qn, q = cm - g * qn;
          const int ro = roff[g * 8 + (j >> 2)], k = k0 + q * 4 + (j & 3);
          if (ro >= 0 && k < K) v[u] = __ldg(src + ro + koff[k]);
        }
      }
#pragma unroll
      for (int u = 0; u < TC_UNROLL; ++u) {
        const int e = e0 + u * TC_THREADS;
        if (e < total) tc_st(dst, dlo, e, v[u]);
      }
    }
  } else if (mode == TC_VEC_K) {
    const int qn = Kc >> 2, total = (rows * Kc) >> 2;
    for (int e0 = tid; e0 < total; e0 += TC_THREADS * TC_UNROLL) {
      float4 v[TC_UNROLL];
#pragma unroll
      for (int u = 0; u < TC_UNROLL; ++u) {
        const int e = e0 + u * TC_THREADS;
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < total) {
          const int cm = e >> 3;
          const int g = cm / qn, q = cm - g * qn;
          const int ro = roff[g * 8 + (e & 7)], k = k0 + q * 4;
          if (ro >= 0 && k < K) v[u] = __ldg((const float4*)(src + ro + koff[k]));
        }
      }
#pragma unroll
      for (int u = 0; u < TC_UNROLL; ++u) {
        const int e = e0 + u * TC_THREADS;
        if (e < total) tc_st4(dst, dlo, e, v[u]);
      }
    }
  } else {
    // blocks of 4 rows x 4 contraction indices; lane j of a quad holds index 4kq + j
    const int qn = Kc >> 2, nrb = rows >> 2, total = nrb * qn;
    const int lane = tid & 31, j = lane & 3;
    for (int b0 = tid >> 2; b0 - (lane >> 2) < total; b0 += (TC_THREADS / 4) * TC_UNROLL) {
      float4 v[TC_UNROLL];
#pragma unroll
      for (int u = 0; u < TC_UNROLL; ++u) {
        const int blk = b0 + u * (TC_THREADS / 4);
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (blk < total) {
          const int kq = blk / nrb, rb = blk - kq * nrb;
          const int ro = roff[rb * 4], k = k0 + kq * 4 + j;
          if (ro >= 0 && k < K) v[u] = __ldg((const float4*)(src + ro + koff[k]));
        }
      }
#pragma unroll
      for (int u = 0; u < TC_UNROLL; ++u) {
        const int blk = b0 + u * (TC_THREADS / 4);
        float o0 = 0.f, o1 = 0.f, o2 = 0.f, o3 = 0.f;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int c = (j - r) & 3;   // component this lane sends: row c of its column
          const float send = c == 0 ? v[u].x : (c == 1 ? v[u].y : (c == 2 ? v[u].z : v[u].w));
          const float got = __shfl_sync(0xffffffffu, send, (lane & ~3) | ((j + r) & 3));
          const int idx = (j + r) & 3;   // row j at contraction index 4kq + idx
          o0 = idx == 0 ? got : o0;
          o1 = idx == 1 ? got : o1;
          o2 = idx == 2 ? got : o2;
          o3 = idx == 3 ? got : o3;
        }
        if (blk < total) {
          const int kq = blk / nrb, rb = blk - kq * nrb;
          const int r = rb * 4 + j;
          tc_st4(dst, dlo, ((r >> 3) * qn + kq) * 8 + (r & 7), make_float4(o0, o1, o2, o3));
        }
      }
    }
  }
}

// Register-staged gather for chunks small enough to prefetch (at most 4 * NV elements or
// NV 16-byte vectors per thread): tc_pload issues the global loads of one chunk into
// registers, tc_pstore rounds them and writes the canonical layout, so the loads of the
// next chain can be in flight while the current chain's MMA and epilogue run.
template <int NV>
__device__ __forceinline__ void tc_pload(float4 (&r)[NV], const float* __restrict__ src, int mode,
                                         int rows, int Kc, int K, const int* roff,
                                         const int* koff, int tid) {
  const int qn = Kc >> 2;
  if (mode == TC_VEC_K) {
    const int total = (rows * Kc) >> 2;
#pragma unroll
    for (int u = 0; u < NV; ++u) {
      const int e = tid + u * TC_THREADS;
      r[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (e < total) {
        const int cm = e >> 3;
        const int g = cm / qn, q = cm - g * qn;
        const int ro = roff[g * 8 + (e & 7)], k = q * 4;
        if (ro >= 0 && k < K) r[u] = __ldg((const float4*)(src + ro + koff[k]));
      }
    }
  } else {
    const int nrb = rows >> 2, total = nrb * qn, j = tid & 3;
#pragma unroll
    for (int u = 0; u < NV; ++u) {
      const int blk = (tid >> 2) + u * (TC_THREADS / 4);
      r[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (blk < total) {
        const int kq = blk / nrb, rb = blk - kq * nrb;
        const int ro = roff[rb * 4], k = kq * 4 + j;
        if (ro >= 0 && k < K) r[u] = __ldg((const float4*)(src + ro + koff[k]));
      }
    }
  }
}

template <int NV>
__device__ __forceinline__ void tc_pstore(const float4 (&r)[NV], float* dst, float* dlo, int mode,
                                          int rows, int Kc, int tid) {
  const int qn = Kc >> 2;
  if (mode == TC_VEC_K) {
    const int total = (rows * Kc) >> 2;
#pragma unroll
    for (int u = 0; u < NV; ++u) {
      const int e = tid + u * TC_THREADS;
      if (e < total) tc_st4(dst, dlo, e, r[u]);
    }
  } else {
    const int nrb = rows >> 2, total = nrb * qn, lane = tid & 31, j = lane & 3;
#pragma unroll
    for (int u = 0; u < NV; ++u) {
      const int blk = (tid >> 2) + u * (TC_THREADS / 4);
      float o0 = 0.f, o1 = 0.f, o2 = 0.f, o3 = 0.f;
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const int c = (j - rr) & 3;
        const float send = c == 0 ? r[u].x : (c == 1 ? r[u].y : (c == 2 ? r[u].z : r[u].w));
        const float got = __shfl_sync(0xffffffffu, send, (lane & ~3) | ((j + rr) & 3));
        const int idx = (j + rr) & 3;
        o0 = idx == 0 ? got : o0;
        o1 = idx == 1 ? got : o1;
        o2 = idx == 2 ? got : o2;
        o3 = idx == 3 ? got : o3;
      }
      if (blk < total) {
        const int kq = blk / nrb, rb = blk - kq * nrb;
        const int row = rb * 4 + j;
        tc_st4(dst, dlo, ((row >> 3) * qn + kq) * 8 + (row & 7), make_float4(o0, o1, o2, o3));
      }
    }
  }
}

// Descriptor of k-block kb (8 contraction indices = two core matrices along K).
__device__ __forceinline__ uint64_t tc_kdesc(uint32_t base, int Kc, int kb) {
  return tc_desc(base + kb * 256, 128, (uint32_t)Kc * 32u);
}

// The MMAs of k-block kb: hi.hi, and for split operands also hi.lo and lo.hi.
__device__ __forceinline__ void tc_mma_k(int split, uint32_t tmem, uint32_t a, uint32_t b,
                                         uint32_t al, uint32_t bl, int Kc, int kb,
                                         uint32_t idesc, bool accumulate) {
  tc_mma(tmem, tc_kdesc(a, Kc, kb), tc_kdesc(b, Kc, kb), idesc, accumulate ? 1 : 0);
  if (split) {
    tc_mma(tmem, tc_kdesc(a, Kc, kb), tc_kdesc(bl, Kc, kb), idesc, 1);
    tc_mma(tmem, tc_kdesc(al, Kc, kb), tc_kdesc(b, Kc, kb), idesc, 1);
  }
}

// Accumulator rows of this warp's lane quarter to C (16-byte stores when C is unit-stride
// in its columns).
__device__ __forceinline__ void tc_epilogue(const TcSpec& t, uint32_t tmem, float* pc,
                                            const int* rowC, const int* colC, int warp, int lane) {
  const int oc = rowC[warp * 32 + lane];
  for (int c0 = 0; c0 < t.TN; c0 += 16) {
    uint32_t v[16];
    tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
    if (oc >= 0) {
      if (t.vecC) {
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
          const int cc = colC[c0 + j];
          if (cc >= 0)
            *(float4*)(pc + oc + cc) = make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                                                   __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int cc = colC[c0 + j];
          if (cc >= 0) pc[oc + cc] = __uint_as_float(v[j]);
        }
      }
    }
  }
}

template <bool PREF>
__global__ void __launch_bounds__(TC_THREADS) kb_gemm_tc(TcSpec t, float* C, long long cs,
                                                         Operand<float> P, Operand<float> Q,
                                                         int n, int tilesN, int* err) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  __shared__ int stuck;   // a grace wait ran out too: an MMA may still be writing tensor memory
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tm = blockIdx.x / tilesN, tn = blockIdx.x - (blockIdx.x / tilesN) * tilesN;
  const int TN = t.TN, Kc = t.Kc;
  const int m0 = tm * TC_ROWS, n0 = tn * TN;
  const int nst = tc_stages(t);
  // per stage: A hi, B hi, then (split) A lo, B lo; no B chunks when B is read from A
  const int sa = TC_ROWS * Kc, sb = t.sym ? 0 : TN * Kc, sst = (sa + sb) * (t.split ? 2 : 1);
  // rows of the chunks that hold data; the rows past the edge of C are left as they are
  // (they only feed accumulator rows and columns that the epilogue does not store)
  const int rowsA = min(TC_ROWS, ((t.M - m0 + 7) >> 3) << 3);
  const int rowsB = min(TN, ((t.N - n0 + 7) >> 3) << 3);
  float* stage0 = (float*)dyn;
  int* rowP = (int*)(stage0 + (long long)nst * sst);
  int* rowC = rowP + TC_ROWS;
  int* colQ = rowC + TC_ROWS;
  int* colC = colQ + TN;
  int* kPo = colC + TN;
  int* kQo = kPo + t.K;
  for (int i = tid; i < TC_ROWS; i += TC_THREADS) {
    int m = m0 + i;
    if (m < t.M) gemm_offsets(m, t.nr, t.rs, t.rP, t.rC, rowP[i], rowC[i]);
    else rowP[i] = rowC[i] = -1;
  }
  for (int i = tid; i < TN; i += TC_THREADS) {
    int c = n0 + i;
    if (c < t.N) gemm_offsets(c, t.nc, t.cs, t.cQ, t.cC, colQ[i], colC[i]);
    else colQ[i] = colC[i] = -1;
  }
  for (int k = tid; k < t.K; k += TC_THREADS) gemm_offsets(k, t.nk, t.ks, t.kP, t.kQ, kPo[k], kQo[k]);
  const uint32_t ncols = (uint32_t)tc_cols(TN * nst);
  const uint32_t bar0 = tc_smem_addr(&bar[0]), bar1 = tc_smem_addr(&bar[1]);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc_smem_addr(&tslot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    abort_flag = 0;
    stuck = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0), "r"(1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar1), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  const uint32_t idesc = tc_idesc(TC_ROWS, TN);
  const int Kp = ((t.K + 7) >> 3) << 3;
  uint32_t ph = 0u;   // phase bits of the two barriers (bit i: barrier i)

  if (nst == 2) {
    // One contraction chunk per chain, two operand stages and two accumulators: the MMA of
    // chain i runs while the operands of chain i+1 are gathered (or, with PREF, while
    // their prefetched registers are stored), and chain i's epilogue follows the next MMA.
    float4 ra[PREF ? 4 : 1], rb[PREF ? 2 : 1];
    int it = 0, prev = -1;
    int s = blockIdx.y;
    if constexpr (PREF) {
      if (s < n) {
        tc_pload(ra, P.at(s), t.modeP, rowsA, Kc, t.K, rowP, kPo, tid);
        if (!t.sym) tc_pload(rb, Q.at(s), t.modeQ, rowsB, Kc, t.K, colQ, kQo, tid);
      }
    }
    for (; s < n; s += gridDim.y, ++it) {
      const int st = it & 1;
      float* As = stage0 + (long long)st * sst;
      float* Bs = t.sym ? As : As + sa;
      float* Al = t.split ? As + sa + sb : nullptr;
      float* Bl = t.split ? (t.sym ? Al : Al + sa) : nullptr;
      if constexpr (PREF) {
        tc_pstore(ra, As, Al, t.modeP, rowsA, Kc, tid);
        if (!t.sym) tc_pstore(rb, Bs, Bl, t.modeQ, rowsB, Kc, tid);
      } else {
        tc_gather(As, Al, P.at(s), t.modeP, rowsA, Kc, 0, t.K, rowP, kPo, tid);
        if (!t.sym) tc_gather(Bs, Bl, Q.at(s), t.modeQ, rowsB, Kc, 0, t.K, colQ, kQo, tid);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      __syncthreads();
      if (abort_flag) break;
      if (tid == 0 && !t.no_mma) {
        tc_fence_after();
        const uint32_t a = tc_smem_addr(As), b = tc_smem_addr(Bs);
        const uint32_t al = t.split ? tc_smem_addr(Al) : 0, bl = t.split ? tc_smem_addr(Bl) : 0;
        for (int kb = 0; kb < (Kp >> 3); ++kb)
          tc_mma_k(t.split, tmem + (uint32_t)(st * TN), a, b, al, bl, Kc, kb, idesc, kb > 0);
        tc_commit(st ? bar1 : bar0);
      }
      if constexpr (PREF) {
        const int sn = s + gridDim.y;
        if (sn < n) {
          tc_pload(ra, P.at(sn), t.modeP, rowsA, Kc, t.K, rowP, kPo, tid);
          if (!t.sym) tc_pload(rb, Q.at(sn), t.modeQ, rowsB, Kc, t.K, colQ, kQo, tid);
        }
      }
      if (it > 0) {   // the previous chain: its MMA was issued one iteration ago
        const int ps = st ^ 1;
        const uint32_t pb = (ph >> ps) & 1u;
        bool good = tc_wait(ps ? bar1 : bar0, pb);
        if (!good) {
          if (!tc_wait(ps ? bar1 : bar0, pb)) stuck = 1;
          abort_flag = 1;
        }
        good = __all_sync(0xffffffffu, good);   // tcgen05.ld below is warp-collective
        ph ^= 1u << ps;
        if (good) {
          tc_fence_after();
          tc_epilogue(t, tmem + (uint32_t)(ps * TN), C + (long long)prev * cs, rowC, colC, warp, lane);
        }
      }
      prev = s;
    }
    // the last MMA issued (iteration it - 1) has not been waited for yet
    if (it > 0) {
      const int ls = (it - 1) & 1;
      const uint32_t pb = (ph >> ls) & 1u;
      if (!tc_wait(ls ? bar1 : bar0, pb)) {
        if (!tc_wait(ls ? bar1 : bar0, pb)) stuck = 1;
        abort_flag = 1;
      }
      ph ^= 1u << ls;
      __syncthreads();
      if (!abort_flag) {
        tc_fence_after();
        tc_epilogue(t, tmem + (uint32_t)(ls * TN), C + (long long)prev * cs, rowC, colC, warp, lane);
      }
    }
    tc_fence_before();
  } else {
    // several chunks per chain: one stage, accumulate over the chunks, then the epilogue
    float* As = stage0;
    float* Bs = t.sym ? As : As + sa;
    float* Al = t.split ? As + sa + sb : nullptr;
    float* Bl = t.split ? (t.sym ? Al : Al + sa) : nullptr;
    const uint32_t a = tc_smem_addr(As), b = tc_smem_addr(Bs);
    const uint32_t al = t.split ? tc_smem_addr(Al) : 0, bl = t.split ? tc_smem_addr(Bl) : 0;
    bool ok = true;
    for (int s = blockIdx.y; s < n && ok; s += gridDim.y) {
      const float* pp = P.at(s);
      const float* pq = Q.at(s);
      for (int k0 = 0; k0 < t.K; k0 += Kc) {
        tc_gather(As, Al, pp, t.modeP, rowsA, Kc, k0, t.K, rowP, kPo, tid);
        if (!t.sym) tc_gather(Bs, Bl, pq, t.modeQ, rowsB, Kc, k0, t.K, colQ, kQo, tid);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && !t.no_mma) {
          tc_fence_after();
          const int nkb = (Kp - k0 < Kc ? Kp - k0 : Kc) >> 3;
          for (int kb = 0; kb < nkb; ++kb)
            tc_mma_k(t.split, tmem, a, b, al, bl, Kc, kb, idesc, k0 > 0 || kb > 0);
          tc_commit(bar0);
        }
        if (!tc_wait(bar0, ph & 1u)) {
          if (!tc_wait(bar0, ph & 1u)) stuck = 1;
          abort_flag = 1;
        }
        ph ^= 1u;
        __syncthreads();
        if (abort_flag) {
          ok = false;
          break;
        }
      }
      if (!ok) break;
      tc_fence_after();
      tc_epilogue(t, tmem, C + (long long)s * cs, rowC, colC, warp, lane);
      tc_fence_before();
    }
  }
  __syncthreads();
  // Tensor memory must be released before the CTA exits.  After a timeout whose grace wait
  // also ran out, an MMA may still be writing it: the flag then carries bit 2, and the
  // host reports that every result of the context is undefined from this call on.
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
  }
  if (tid == 0 && abort_flag) atomicOr(err, stuck ? 3 : 1);
}

#endif  // __CUDACC__

}  // namespace pv
#endif
