// Pipelined tensor-core contraction of the batched engine: the same strided GEMM per chain as
// kb_gemm_tc (C[m][n] = sum_k P[m][k] Q[n][k] with multi-index rows, columns and contraction
// indices of arbitrary strides, TF32 operands rounded to nearest, FP32 accumulation), with
// every operand element fetched asynchronously.
//
// A CTA of four warps owns one 128-row x TN tile position and walks the items (chain,
// contraction chunk) of the chains assigned to it.  Each item's operand chunks are copied
// from global memory straight into the canonical K-major no-swizzle layout of a ring of
// `ns` shared-memory stages with cp.async (16-byte copies of four consecutive contraction
// indices when the operand is unit-stride there, 4-byte copies otherwise; out-of-range rows
// and indices are zero-filled), so the copies of the next ns - 1 items are in flight while
// the current item's MMAs run.  When an item's copies have landed, every thread rounds the
// elements it copied to TF32 (round to nearest; for split operands also forms the TF32
// remainder), then one thread issues the item's `tcgen05.mma.kind::tf32` (M = 128, N = TN,
// K = 8 per instruction) into the chain's accumulator in tensor memory and commits them to
// the stage's mbarrier.  The wait for the previous item's MMAs (which frees its stage for the
// next copy) comes after the current item's MMAs have been issued.  With two accumulators a
// chain's epilogue (tcgen05.ld, then 16-byte or scalar stores to C) runs while the next
// chain's MMAs accumulate into the other one; with one (wide tiles), before them.
// Every wait is bounded as in kb_gemm_tc (err bit 1; bit 2 when the grace wait also ran out).
#ifndef PV_TC2_CUH
#define PV_TC2_CUH
#include <cstdint>

namespace pv {

constexpr int TC2_MAXST = 6;   // most pipeline stages

// Bytes of one stage of the pipelined kernel (as tc_stage_bytes).
inline size_t tc2_stage_bytes(const TcSpec& t) { return tc_stage_bytes(t); }

inline size_t tc2_smem_bytes(const TcSpec& t) {
  return tc2_stage_bytes(t) * t.ns + (size_t)(2 * TC_ROWS + 2 * t.TN + 2 * t.K) * sizeof(int) + 128;
}

// Chooses the contraction chunk, the number of stages and of accumulators of the pipelined
// kernel: about `budget` bytes of stages per CTA, at least three stages where chunks of 8
// allow it, two accumulators when their columns fit in 256 (two CTAs per SM), or in 512 when
// the stages take more than half the shared memory (one CTA per SM anyway).
inline void tc2_shape(TcSpec& t, size_t budget) {
  // the stages and the offset tables stay within the 200 KB the kernel is configured for
  const size_t tables = (size_t)(2 * TC_ROWS + 2 * t.TN + 2 * t.K) * sizeof(int) + 128;
  const size_t cap = 200 * 1024 > tables ? 200 * 1024 - tables : 0;
  budget = budget < cap ? budget : cap;
  const int k8 = ((t.K + 7) / 8) * 8;
  t.Kc = k8 < t.Kc ? k8 : t.Kc;
  if (t.Kc > 32) t.Kc = 32;
  for (;;) {
    const size_t sb = tc2_stage_bytes(t);
    int ns = (int)(budget / sb);
    if (ns >= 3 || t.Kc <= 8) {
      t.ns = ns < 2 ? 2 : (ns > TC2_MAXST ? TC2_MAXST : ns);
      break;
    }
    t.Kc -= 8;
  }
  t.nacc = tc_cols(2 * t.TN) <= (budget > 114 * 1024 ? 512 : 256) ? 2 : 1;
}

#if defined(__CUDACC__)

__device__ __forceinline__ void tc2_cp16(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void tc2_cp4(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void tc2_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void tc2_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void tc2_wait_groups(int n) {
  switch (n) {   // the count must be an immediate
    case 0: tc2_wait_group<0>(); break;
    case 1: tc2_wait_group<1>(); break;
    case 2: tc2_wait_group<2>(); break;
    case 3: tc2_wait_group<3>(); break;
    case 4: tc2_wait_group<4>(); break;
    default: tc2_wait_group<5>(); break;
  }
}

// Asynchronous copy of one operand chunk (rows x Kc at contraction offset k0) into the
// canonical layout at `dst`; with `round` set the same elements are instead rounded in place
// (hi) and their remainders written to `dlo` (split operands).  The element-to-thread map is
// the same in both calls, so a thread rounds exactly what it copied.
__device__ __forceinline__ void tc2_chunk(float* dst, float* dlo, const float* __restrict__ src,
                                          int mode, int rows, int Kc, int k0, int K,
                                          const int* roff, const int* koff, int tid, bool round) {
  const int qn = Kc >> 2;
  if (mode == TC_VEC_K) {
    const int total = (rows * Kc) >> 2;   // 16-byte pieces: one core-matrix row each
    for (int e = tid; e < total; e += TC_THREADS) {
      if (round) {
        const float4 v = ((const float4*)dst)[e];
        const float4 h = tc_round4(v);
        ((float4*)dst)[e] = h;
        if (dlo) ((float4*)dlo)[e] = tc_round4(make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w));
      } else {
        const int cm = e >> 3;
        const int g = cm / qn, q = cm - g * qn;
        const int ro = roff[g * 8 + (e & 7)], k = k0 + q * 4;
        const bool ok = ro >= 0 && k < K;
        tc2_cp16(tc_smem_addr(dst + 4 * e), ok ? (const void*)(src + ro + koff[k]) : (const void*)src, ok);
      }
    }
  } else {
    // element copies; consecutive threads take consecutive rows of one contraction index
    // (coalesced when the operand is unit-stride in its rows), a core matrix holds rows
    // 8g..8g+7 x indices 4q..4q+3 at element offset (g * qn + q) * 32 + (row & 7) * 4 + (k & 3)
    const int total = rows * Kc;
    for (int e = tid; e < total; e += TC_THREADS) {
      const int kk = e / rows, r = e - kk * rows;
      const int off = ((r >> 3) * qn + (kk >> 2)) * 32 + (r & 7) * 4 + (kk & 3);
      if (round) {
        const float v = dst[off];
        const float h = tc_round(v);
        dst[off] = h;
        if (dlo) dlo[off] = tc_round(v - h);
      } else {
        const int ro = roff[r], k = k0 + kk;
        const bool ok = ro >= 0 && k < K;
        tc2_cp4(tc_smem_addr(dst + off), ok ? (const void*)(src + ro + koff[k]) : (const void*)src, ok);
      }
    }
  }
}

__global__ void __launch_bounds__(TC_THREADS) kb_gemm_tc2(TcSpec t, float* C, long long cs,
                                                          Operand<float> P, Operand<float> Q, int n,
                                                          int tilesN, int* err) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ __align__(8) uint64_t mbar[TC2_MAXST];
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  __shared__ int stuck;   // a grace wait ran out too: an MMA may still be writing tensor memory
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tm = blockIdx.x / tilesN, tn = blockIdx.x - tm * tilesN;
  const int TN = t.TN, Kc = t.Kc, ns = t.ns, nacc = t.nacc;
  const int m0 = tm * TC_ROWS, n0 = tn * TN;
  const int sa = TC_ROWS * Kc, sb = t.sym ? 0 : TN * Kc, sst = (sa + sb) * (t.split ? 2 : 1);
  const int rowsA = min(TC_ROWS, ((t.M - m0 + 7) >> 3) << 3);
  const int rowsB = min(TN, ((t.N - n0 + 7) >> 3) << 3);
  float* stage0 = (float*)dyn;
  int* rowP = (int*)(stage0 + (long long)ns * sst);
  int* rowC = rowP + TC_ROWS;
  int* colQ = rowC + TC_ROWS;
  int* colC = colQ + TN;
  int* kPo = colC + TN;
  int* kQo = kPo + t.K;
  for (int i = tid; i < TC_ROWS; i += TC_THREADS) {
    const int m = m0 + i;
    if (m < t.M) gemm_offsets(m, t.nr, t.rs, t.rP, t.rC, rowP[i], rowC[i]);
    else rowP[i] = rowC[i] = -1;
  }
  for (int i = tid; i < TN; i += TC_THREADS) {
    const int c = n0 + i;
    if (c < t.N) gemm_offsets(c, t.nc, t.cs, t.cQ, t.cC, colQ[i], colC[i]);
    else colQ[i] = colC[i] = -1;
  }
  for (int k = tid; k < t.K; k += TC_THREADS) gemm_offsets(k, t.nk, t.ks, t.kP, t.kQ, kPo[k], kQo[k]);
  const uint32_t ncols = (uint32_t)tc_cols(TN * nacc);
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
    for (int s = 0; s < ns; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem_addr(&mbar[s])), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  const uint32_t idesc = tc_idesc(TC_ROWS, TN);
  const int Kp = ((t.K + 7) >> 3) << 3;
  const int nk = (t.K + Kc - 1) / Kc;
  const int gy = gridDim.y;
  const int nch = blockIdx.y < n ? (n - 1 - blockIdx.y) / gy + 1 : 0;
  const long long total = (long long)nch * nk;

  auto stA = [&](long long j) { return stage0 + (long long)(j % ns) * sst; };
  // copies (round = false) or rounding (round = true) of item j's operand chunks
  auto chunk = [&](long long j, bool round) {
    const int c = (int)(j / nk), kc = (int)(j - (long long)c * nk);
    const int s = blockIdx.y + c * gy;
    float* As = stA(j);
    float* Bs = t.sym ? As : As + sa;
    float* Al = t.split ? As + sa + sb : nullptr;
    float* Bl = t.split ? (t.sym ? Al : Al + sa) : nullptr;
    tc2_chunk(As, Al, P.at(s), t.modeP, rowsA, Kc, kc * Kc, t.K, rowP, kPo, tid, round);
    if (!t.sym) tc2_chunk(Bs, Bl, Q.at(s), t.modeQ, rowsB, Kc, kc * Kc, t.K, colQ, kQo, tid, round);
  };
  // waits for item j's MMAs; false when the wait ran out (abort raised)
  auto wait_mma = [&](long long j) {
    const uint32_t bar = tc_smem_addr(&mbar[j % ns]);
    const uint32_t par = (uint32_t)((j / ns) & 1);
    if (tc_wait(bar, par)) return true;
    if (!tc_wait(bar, par)) stuck = 1;
    abort_flag = 1;
    return false;
  };
  auto epilogue = [&](long long j) {   // chain of item j, accumulator of that chain
    const int c = (int)(j / nk);
    const int s = blockIdx.y + c * gy;
    tc_fence_after();
    tc_epilogue(t, tmem + (uint32_t)((c % nacc) * TN), C + (long long)s * cs, rowC, colC, warp, lane);
    tc_fence_before();
  };

  for (int i = 0; i < ns - 1; ++i) {
    if (i < total) chunk(i, false);
    tc2_commit_group();
  }
  long long waited = -1;   // last item whose MMAs have been waited for
  for (long long j = 0; j < total; ++j) {
    tc2_wait_groups(ns - 2);   // item j's copies (groups complete in order)
    chunk(j, true);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    const int kc = (int)(j % nk);
    if (abort_flag) break;
    if (nacc == 1 && kc == 0 && j > 0) {
      // one accumulator: the previous chain's epilogue must read it before it is overwritten
      wait_mma(j - 1);
      waited = j - 1;
      __syncthreads();
      if (abort_flag) break;
      epilogue(j - 1);
      __syncthreads();
    }
    if (tid == 0 && !t.no_mma) {
      tc_fence_after();
      float* As = stA(j);
      float* Bs = t.sym ? As : As + sa;
      float* Al = t.split ? As + sa + sb : nullptr;
      float* Bl = t.split ? (t.sym ? Al : Al + sa) : nullptr;
      const uint32_t a = tc_smem_addr(As), b = tc_smem_addr(Bs);
      const uint32_t al = t.split ? tc_smem_addr(Al) : 0, bl = t.split ? tc_smem_addr(Bl) : 0;
      const int k0 = kc * Kc;
      const int nkb = (Kp - k0 < Kc ? Kp - k0 : Kc) >> 3;
      const uint32_t acc = tmem + (uint32_t)(((j / nk) % nacc) * TN);
      for (int kb = 0; kb < nkb; ++kb) tc_mma_k(t.split, acc, a, b, al, bl, Kc, kb, idesc, kc > 0 || kb > 0);
      tc_commit(tc_smem_addr(&mbar[j % ns]));
    }
    if (j >= 1 && waited < j - 1) {
      // the previous item's MMAs: their stage is refilled below; their chain's epilogue
      // (two accumulators) overlaps the MMAs just issued
      wait_mma(j - 1);
      waited = j - 1;
      __syncthreads();   // every thread sees the same abort flag (tcgen05.ld is warp-collective)
      if (abort_flag) break;
      if (nacc == 2 && (j - 1) % nk == nk - 1) epilogue(j - 1);
    }
    if (j + ns - 1 < total) chunk(j + ns - 1, false);
    tc2_commit_group();
  }
  // the last item
  __syncthreads();
  if (!abort_flag && total > 0 && waited < total - 1) {
    wait_mma(total - 1);
    __syncthreads();
    if (!abort_flag) epilogue(total - 1);
  }
  tc2_wait_group<0>();   // no copy may land after the CTA has left
  __syncthreads();
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
