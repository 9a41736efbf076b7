// Residual check that allocates nothing: ddel_residual_norm_noalloc.
//
// For callers that cannot allocate device memory themselves (for example code
// running under an allocator that forbids cudaMalloc, or a host process that
// only receives device pointers from another component).  Everything the
// kernel needs besides its inputs and outputs -- one pair of FP64 partial sums
// per thread block and the arrival counter of the two-level reduction -- lives
// in a fixed file-scope device array, so the call makes no cudaMalloc, no
// cudaFree and no allocating library call.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/ddel.h"
#include "ddel_device.cuh"

namespace {

constexpr int kThreads = 256;
// One block per kThreads grid nodes, at most kMaxBlocks blocks: grids of up to
// kMaxBlocks * kThreads = 1,048,576 nodes.
constexpr int kMaxBlocks = 4096;

// Scratch shared by every call on a device: partial sums (2 per block) and the
// arrival counter.  64 KB + 256 B, held by every GPU that loads the library
// until the process exits.
struct NoAllocScratch {
  double partials[2 * kMaxBlocks];
  unsigned ticket;
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

template <int DIM>
__global__ void __launch_bounds__(kThreads) residual_noalloc_kernel(
    int nx, int ny, int nz, const double* __restrict__ Ke, const double* __restrict__ factors,
    const uint8_t* __restrict__ fixed, const double* __restrict__ f, const double* __restrict__ u,
    double* r, double* norms, NoAllocScratch* scr) {
  constexpr int NN = 1 << DIM, ND = DIM * NN;
  __shared__ double ke[ND * ND];
  __shared__ double red[64];
  for (int i = threadIdx.x; i < ND * ND; i += kThreads) ke[i] = Ke[i];
  __syncthreads();
  const int ne[3] = {nx, ny, DIM == 3 ? nz : 1};
  const int nn1 = ny + 1, nn2 = DIM == 3 ? nz + 1 : 1;
  const int64_t n_nodes = (int64_t)(nx + 1) * nn1 * nn2;
  double acc[2] = {0.0, 0.0};
  const int64_t n = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (n < n_nodes) {
    const int k = DIM == 3 ? (int)(n % nn2) : 0;
    const int64_t ij = n / nn2;
    const int j = (int)(ij % nn1), i = (int)(ij / nn1);
    double out[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) out[c] = 0.0;
    for (int ox = 0; ox < 2; ++ox) {
      const int ex = i - ox;
      if (ex < 0 || ex >= ne[0]) continue;
      for (int oy = 0; oy < 2; ++oy) {
        const int ey = j - oy;
        if (ey < 0 || ey >= ne[1]) continue;
        for (int oz = 0; oz < (DIM == 3 ? 2 : 1); ++oz) {
          const int ez = k - oz;
          if (DIM == 3 && (ez < 0 || ez >= ne[2])) continue;
          const int64_t e = ((int64_t)ex * ne[1] + ey) * ne[2] + ez;
          const int ln = ddel::elem_local_node(ox, oy, oz);
          double part[DIM];
#pragma unroll
          for (int c = 0; c < DIM; ++c) part[c] = 0.0;
#pragma unroll
          for (int a = 0; a < NN; ++a) {
            int dx, dy, dz;
            ddel::elem_node_offset(a, dx, dy, dz);
            const int64_t nb = ((int64_t)(ex + dx) * nn1 + (ey + dy)) * nn2 + (ez + dz);
#pragma unroll
            for (int c2 = 0; c2 < DIM; ++c2) {
              const int64_t d2 = DIM * nb + c2;
              const double xv = (fixed && fixed[d2]) ? 0.0 : u[d2];
#pragma unroll
              for (int c = 0; c < DIM; ++c) part[c] += ke[(ln * DIM + c) * ND + a * DIM + c2] * xv;
            }
          }
          const double sc = factors[e];
#pragma unroll
          for (int c = 0; c < DIM; ++c) out[c] += sc * part[c];
        }
      }
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const int64_t d = DIM * n + c;
      if (fixed && fixed[d]) {
        if (r) r[d] = 0.0;
        continue;
      }
      const double fv = f[d], rv = fv - out[c];
      if (r) r[d] = rv;
      acc[0] += rv * rv;
      acc[1] += fv * fv;
    }
  }
  // deterministic two-level sum: block partials in the scratch array, the
  // last block to arrive adds them in block order
  if (ddel::grid_sum<2, kThreads>(acc, scr->partials, &scr->ticket, red) && threadIdx.x == 0) {
    norms[0] = sqrt(acc[0]);
    norms[1] = sqrt(acc[1]);
  }
}

}  // namespace

extern "C" int ddel_residual_norm_noalloc(int dim, int nx, int ny, int nz, const double* Ke,
                                          const double* factors, const uint8_t* fixed,
                                          const double* f, const double* u, double* r,
                                          double* norms, void* cuda_stream) {
  if ((dim != 2 && dim != 3) || nx < 1 || ny < 1 || (dim == 3 && nz < 1)) return DDEL_EINVAL;
  if (!Ke || !factors || !f || !u || !norms) return DDEL_EINVAL;
  const int64_t n_nodes = (int64_t)(nx + 1) * (ny + 1) * (dim == 3 ? (int64_t)(nz + 1) : 1);
  if (n_nodes > (int64_t)kMaxBlocks * kThreads) return DDEL_EINVAL;  // beyond the scratch capacity
  // the device address of the scratch array on the current device (its
  // host-side name is only a stand-in), looked up on every call: the lookup
  // allocates nothing, and no address outlives a cudaDeviceReset or a reload
  // of the library
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DDEL_ECUDA;
  NoAllocScratch* scr = static_cast<NoAllocScratch*>(p);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // the arrival counter must start at zero
  if (cudaMemsetAsync(&scr->ticket, 0, sizeof(unsigned), s) != cudaSuccess) return DDEL_ECUDA;
  const int blocks = (int)((n_nodes + kThreads - 1) / kThreads);
  if (dim == 2)
    residual_noalloc_kernel<2><<<blocks, kThreads, 0, s>>>(nx, ny, 0, Ke, factors, fixed, f, u, r,
                                                           norms, scr);
  else
    residual_noalloc_kernel<3><<<blocks, kThreads, 0, s>>>(nx, ny, nz, Ke, factors, fixed, f, u, r,
                                                           norms, scr);
  return cudaGetLastError() == cudaSuccess ? DDEL_OK : DDEL_ECUDA;
}
