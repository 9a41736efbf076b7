// Device-side helpers: TMA bulk copies with mbarriers (bounded waits),
// deterministic reductions, structured-grid element products.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ddel_internal.h"
#include "ddel_launch.h"

namespace ddel {

// Upper bound on mbarrier try_wait polls before a kernel gives up (each poll
// suspends for a hardware-defined interval; this bounds a wait to seconds).
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// 1D bulk copy global -> shared, completion signalled on `bar` (16-byte
// aligned addresses, size a multiple of 16 bytes).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  uint64_t g;
  asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(src));
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(g), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: returns false (and the caller reports kErrTimeout) instead of
// spinning forever.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = kWaitLimit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Asynchronous 8-byte copy global -> shared (cp.async, sm_80 and later);
// cp_async_commit closes a group, cp_async_wait_all waits for all groups of
// the thread.  Addresses 8-byte aligned.
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  uint64_t g;
  asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(src));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of NV values (fixed reduction tree: deterministic).
template <int NV, int THREADS>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* scratch /* NV*32 */) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) scratch[i * 32 + w] = v[i];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double t = lane < THREADS / 32 ? scratch[i * 32 + lane] : 0.0;
      v[i] = warp_sum(t);
    }
  }
  __syncthreads();
}

// Grid-level deterministic reduction: every block stores its partials, the
// last block to arrive (atomic ticket) sums all partials in block order.
// Returns true in the last block (thread 0 then holds the totals in v).
template <int NV, int THREADS>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double* partials /* NV*gridDim */,
                                         unsigned* ticket, double* scratch) {
  block_sum<NV, THREADS>(v, scratch);
  __shared__ bool last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) partials[i * gridDim.x + blockIdx.x] = v[i];
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    acc[i] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += THREADS)
      acc[i] += __ldcg(&partials[i * gridDim.x + b]);
  }
  block_sum<NV, THREADS>(acc, scratch);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = acc[i];
    *ticket = 0u;  // ready for the next launch
  }
  return true;
}

// Local node index of grid offset (dx, dy, dz) in {0,1}^3 within an element
// (order (0,0),(1,0),(1,1),(0,1), then +4 for dz = 1).
__device__ __forceinline__ int elem_local_node(int dx, int dy, int dz) {
  const int q = dy ? (dx ? 2 : 3) : (dx ? 1 : 0);
  return q + 4 * dz;
}

__device__ __forceinline__ void elem_node_offset(int a, int& dx, int& dy, int& dz) {
  const int q = a & 3;
  dx = (q == 1 || q == 2);
  dy = (q >= 2);
  dz = a >> 2;
}

// ---- double-float arithmetic (value = hi + lo, two FP32 numbers) ----------
// Error-free transformations with explicitly rounded intrinsics (the compiler
// may not contract them into FMAs, which would break them): Dekker's product
// split via FMA and Knuth's TwoSum, about 48 significant bits on the FP32
// pipes (this GPU issues 2 FP64 multiply-adds per clock per SM).
__device__ __forceinline__ void df_add(float& hi, float& lo, float p) {
  const float s = __fadd_rn(hi, p);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// (hi, lo) += (p_hi, p_lo): double-float addition (Knuth's TwoSum on the high
// parts, low parts added, renormalised).
__device__ __forceinline__ void df_add2(float& hi, float& lo, float phi, float plo) {
  const float s = __fadd_rn(hi, phi);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(phi, bp));
  const float t = __fadd_rn(__fadd_rn(lo, plo), err);
  hi = __fadd_rn(s, t);
  lo = __fsub_rn(t, __fsub_rn(hi, s));
}

// (hi, lo) += s * x for double-float s and x: the high product p = s.hi x.hi,
// its exact rounding error by FMA and the hi*lo cross terms go to lo.
__device__ __forceinline__ void df_mad(float& hi, float& lo, float2 s, float2 x) {
  const float p = __fmul_rn(s.x, x.x);
  lo = __fadd_rn(lo, __fadd_rn(__fmaf_rn(s.x, x.x, -p), __fmaf_rn(s.x, x.y, __fmul_rn(s.y, x.x))));
  df_add(hi, lo, p);
}

__device__ __forceinline__ float2 df_from(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

// Warp-wide double-float sum (the same bits in every lane).
__device__ __forceinline__ void df_warp_sum(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ph = __shfl_xor_sync(0xffffffffu, hi, o), pl = __shfl_xor_sync(0xffffffffu, lo, o);
    df_add2(hi, lo, ph, pl);
  }
}

// Sum of src[0..n) by one warp in a fixed order (lane-strided with four
// independent accumulators, so that the loads overlap, then the warp tree);
// every lane returns the total, and every block that calls it on the same
// data obtains the same bits.
__device__ __forceinline__ double reduce_partials_warp(const double* __restrict__ src, int n) {
  const int lane = threadIdx.x & 31;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int b = lane;
  for (; b + 96 < n; b += 128) {
    a0 += __ldcg(src + b);
    a1 += __ldcg(src + b + 32);
    a2 += __ldcg(src + b + 64);
    a3 += __ldcg(src + b + 96);
  }
  for (; b < n; b += 32) a0 += __ldcg(src + b);
  return warp_sum((a0 + a1) + (a2 + a3));
}

// Fixed-order sum over the block of nv <= NV values per thread: a binary tree
// in shared memory in which every addition is useful (FP64 is scarce on this
// GPU: two DFMA per clock per SM).  red: NV * blockDim.x doubles, blockDim.x a
// power of two.  On return (block synchronised) red[v * blockDim.x] holds sum v.
template <int NV>
__device__ __forceinline__ void block_tree_sum(const double (&a)[NV], int nv, double* red) {
  const int tid = threadIdx.x, T = blockDim.x;
#pragma unroll
  for (int v = 0; v < NV; ++v)
    if (v < nv) red[v * T + tid] = a[v];
  __syncthreads();
  // each level's nv * s additions are spread over all threads (the same
  // additions in the same order as one tree per value)
  int ls = 0;
  while ((1 << ls) < T) ++ls;
  for (int s = T / 2, l = ls - 1; s > 0; s >>= 1, --l) {
    for (int e = tid; e < nv * s; e += T) {
      const int v = e >> l, i = e & (s - 1);
      red[v * T + i] += red[v * T + i + s];
    }
    __syncthreads();
  }
}

// Schur kernel of a PCG iteration: record the iteration index for the update
// kernel.  (With a coarse space the Schur kernels apply S to the face-local
// part of u only; the update kernel adds S Q cc from the stored S Q.)
__device__ __forceinline__ void schur_pcg_prologue(const SchurIO& io, int bid) {
  if (io.pcg && bid == 0 && threadIdx.x == 0) io.pcg->kU = io.pcg->kS;
}
__device__ __forceinline__ void schur_pcg_prologue(const SchurIO& io) { schur_pcg_prologue(io, blockIdx.x); }

// The block's share of delta = (S u, u): the values d of warps [0, NW) summed,
// written by thread 0 to pd[blockIdx.x].  All threads call it.
template <int NW>
__device__ __forceinline__ void schur_pcg_epilogue(const SchurIO& io, double d, double* red, int bid) {
  if (!io.pcg) return;
  const int w = threadIdx.x >> 5;
  if (w < NW) {
    const double s = warp_sum(d);
    if ((threadIdx.x & 31) == 0) red[w] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
#pragma unroll
    for (int i = 0; i < NW; ++i) tot += red[i];
    io.pd[bid] = tot;
  }
}
template <int NW>
__device__ __forceinline__ void schur_pcg_epilogue(const SchurIO& io, double d, double* red) {
  schur_pcg_epilogue<NW>(io, d, red, blockIdx.x);
}

// 1 / sqrt(d), d > 0: Newton's iteration for f(r) = 1 / r^2 - d,
// r <- r (3 - d r^2) / 2, from the single-precision estimate; each step
// doubles the correct bits, two take the estimate's 23 past double precision
// (a few units in the last place).  Outside the single-precision range the
// library square root and division serve.  (FP64 only.)
__device__ __forceinline__ double pivot_rsqrt(double d) {
  if (d > 1e-36 && d < 1e36) {
    double r = (double)rsqrtf((float)d);
    r = r * fma(-0.5 * d, r * r, 1.5);
    r = r * fma(-0.5 * d, r * r, 1.5);
    return r;
  }
  return 1.0 / sqrt(d);
}

}  // namespace ddel
