// Topology-optimisation kernels for the Picard loop of Sec. 5 (eq. NumberTen
// with SIMP exponent p): density filter, compliance, adjoint sensitivities and
// the optimality-criteria update with its volume multiplier found by
// bisection inside one cooperative launch.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "ddel_device.cuh"
#include "ddel_launch.h"
#include "ddel_topopt.h"

namespace cg = cooperative_groups;

namespace ddel {
namespace {

constexpr int kThreads = 256;

struct Grid3 {
  int ne[3];
  int dim;
  __device__ __forceinline__ int64_t index(int a, int b, int c) const {
    return ((int64_t)a * ne[1] + b) * ne[2] + c;
  }
};

__device__ __forceinline__ void decompose(const Grid3& g, int64_t e, int& a, int& b, int& c) {
  c = (int)(e % g.ne[2]);
  const int64_t ab = e / g.ne[2];
  b = (int)(ab % g.ne[1]);
  a = (int)(ab / g.ne[1]);
}

// Sum of the hat weights max(0, r_min - |d|) over the neighbours of element
// (a, b, c) inside the grid.
__device__ double weight_sum(const Grid3& g, int R, double r_min, int a, int b, int c) {
  double s = 0.0;
  const int Rz = g.dim == 3 ? R : 0;
  for (int da = -R; da <= R; ++da)
    for (int db = -R; db <= R; ++db)
      for (int dc = -Rz; dc <= Rz; ++dc) {
        const int x = a + da, y = b + db, z = c + dc;
        if (x < 0 || x >= g.ne[0] || y < 0 || y >= g.ne[1] || z < 0 || z >= g.ne[2]) continue;
        const double w = r_min - sqrt((double)(da * da + db * db + dc * dc));
        if (w > 0.0) s += w;
      }
  return s;
}

// out_i = sum_j w_ij in_j / sum_j w_ij  (transpose = 0), or
// out_j = sum_i w_ij / W_i in_i         (transpose = 1, chain rule of the filter)
__global__ void filter_kernel(Grid3 g, int R, double r_min, const double* __restrict__ in,
                              double* __restrict__ out, int transpose, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int a, b, c;
    decompose(g, e, a, b, c);
    const int Rz = g.dim == 3 ? R : 0;
    double acc = 0.0, wsum = 0.0;
    for (int da = -R; da <= R; ++da)
      for (int db = -R; db <= R; ++db)
        for (int dc = -Rz; dc <= Rz; ++dc) {
          const int x = a + da, y = b + db, z = c + dc;
          if (x < 0 || x >= g.ne[0] || y < 0 || y >= g.ne[1] || z < 0 || z >= g.ne[2]) continue;
          const double w = r_min - sqrt((double)(da * da + db * db + dc * dc));
          if (w <= 0.0) continue;
          const int64_t j = g.index(x, y, z);
          if (transpose) {
            acc += w / weight_sum(g, R, r_min, x, y, z) * in[j];
          } else {
            acc += w * in[j];
            wsum += w;
          }
        }
    out[e] = transpose ? acc : acc / wsum;
  }
}

// dc/drho~_e = -p E rho~_e^(p-1) u_e^T K_e u_e  (E folded into the unit-E K_e scale)
template <int DIM>
__global__ void sensitivity_kernel(Grid3 g, const double* __restrict__ Ke, double E, double p,
                                   const double* __restrict__ rho_f, const double* __restrict__ u,
                                   double* __restrict__ dcf, int64_t n) {
  constexpr int NN = 1 << DIM, ND = DIM * NN;
  __shared__ double ke[ND * ND];
  for (int i = threadIdx.x; i < ND * ND; i += blockDim.x) ke[i] = Ke[i];
  __syncthreads();
  const int nn1 = g.ne[1] + 1, nn2 = DIM == 3 ? g.ne[2] + 1 : 1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int a, b, c;
    decompose(g, e, a, b, c);
    double ue[ND];
#pragma unroll
    for (int q = 0; q < NN; ++q) {
      int dx, dy, dz;
      elem_node_offset(q, dx, dy, dz);
      const int64_t node = ((int64_t)(a + dx) * nn1 + (b + dy)) * nn2 + (DIM == 3 ? c + dz : 0);
#pragma unroll
      for (int k = 0; k < DIM; ++k) ue[q * DIM + k] = u[DIM * node + k];
    }
    double en = 0.0;
#pragma unroll
    for (int i = 0; i < ND; ++i) {
      double row = 0.0;
#pragma unroll
      for (int j = 0; j < ND; ++j) row += ke[i * ND + j] * ue[j];
      en += ue[i] * row;
    }
    dcf[e] = -p * E * pow(rho_f[e], p - 1.0) * en;
  }
}

__global__ void dot_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                           double* partials, unsigned* ticket, double* out) {
  __shared__ double red[32];
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc[0] += a[i] * b[i];
  if (grid_sum<1, kThreads>(acc, partials, ticket, red) && threadIdx.x == 0) *out = acc[0];
}

// Optimality-criteria update:
//   B_e = max(-dc_e, 0) / dv_e,
//   rho_new(lambda) = clamp(rho sqrt(B / lambda), max(rho_min, rho - m), min(1, rho + m)),
// lambda by 64 bisection steps on [0, 1e9] so that dv . rho_new = target.
// Every block sums the per-block partials of a step in block order, so all
// blocks take the same decision (deterministic, no atomics).
__global__ void __launch_bounds__(kThreads) oc_kernel(double* rho, const double* __restrict__ dc,
                                                      const double* __restrict__ dv, int64_t n,
                                                      double target, double rho_min, double move,
                                                      double* partials, double* out) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double red[32];
  __shared__ double total_s;
  double lo = 0.0, hi = 1e9;
  auto newval = [&](int64_t e, double lam) {
    const double r = rho[e];
    const double lower = fmax(rho_min, r - move), upper = fmin(1.0, r + move);
    if (!(lam > 0.0)) return upper;
    const double B = fmax(-dc[e], 0.0) / dv[e];
    return fmin(fmax(r * sqrt(B / lam), lower), upper);
  };
  for (int step = 0; step < 64; ++step) {
    const double lam = 0.5 * (lo + hi);
    double acc[1] = {0.0};
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
      acc[0] += dv[e] * newval(e, lam);
    block_sum<1, kThreads>(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc[0];
    grid.sync();
    if (threadIdx.x < 32) {
      double t = 0.0;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) t += __ldcg(&partials[b]);
      t = warp_sum(t);
      if (threadIdx.x == 0) total_s = t;
    }
    __syncthreads();
    if (total_s > target)
      lo = lam;
    else
      hi = lam;
    grid.sync();  // partials are rewritten by the next step
  }
  const double lam = 0.5 * (lo + hi);
  double acc[2] = {0.0, 0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double v = newval(e, lam);
    acc[0] += dv[e] * v;
    acc[1] = fmax(acc[1], fabs(v - rho[e]));
    rho[e] = v;
  }
  // volume (sum) and change (max) of this block; block 0 gathers after a sync
  acc[0] = warp_sum(acc[0]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc[1] = fmax(acc[1], __shfl_xor_sync(0xffffffffu, acc[1], o));
  __shared__ double wv[32], wm[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    wv[w] = acc[0];
    wm[w] = acc[1];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0, m = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) {
      v += wv[i];
      m = fmax(m, wm[i]);
    }
    partials[blockIdx.x] = v;
    partials[gridDim.x + blockIdx.x] = m;
  }
  grid.sync();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double v = 0.0, m = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
      v += __ldcg(&partials[b]);
      m = fmax(m, __ldcg(&partials[gridDim.x + b]));
    }
    out[0] = lam;
    out[1] = v;
    out[2] = m;
  }
}

__global__ void fill_kernel(double* x, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

int blocks_for(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  return (int)(b < 1 ? 1 : (b > 152 * 8 ? 152 * 8 : b));
}

Grid3 make_grid(const DevTables& t) {
  Grid3 g;
  g.dim = t.dim;
  g.ne[0] = t.ne[0];
  g.ne[1] = t.ne[1];
  g.ne[2] = t.dim == 3 ? t.ne[2] : 1;
  return g;
}

}  // namespace

int filter_radius_cells(double r_min) { return (int)ceil(r_min) - 1; }

void launch_filter(const DevTables& t, double r_min, const double* in, double* out, int transpose,
                   cudaStream_t st) {
  filter_kernel<<<blocks_for(t.n_elem), kThreads, 0, st>>>(make_grid(t), filter_radius_cells(r_min),
                                                           r_min, in, out, transpose, t.n_elem);
}

void launch_sensitivity(const DevTables& t, double E, double p, const double* rho_f, const double* u,
                        double* dcf, cudaStream_t st) {
  if (t.dim == 2)
    sensitivity_kernel<2><<<blocks_for(t.n_elem), kThreads, 0, st>>>(make_grid(t), t.Ke64, E, p,
                                                                     rho_f, u, dcf, t.n_elem);
  else
    sensitivity_kernel<3><<<blocks_for(t.n_elem), kThreads, 0, st>>>(make_grid(t), t.Ke64, E, p,
                                                                     rho_f, u, dcf, t.n_elem);
}

void launch_dot(const double* a, const double* b, int64_t n, double* partials, unsigned* ticket,
                double* out, cudaStream_t st) {
  dot_kernel<<<blocks_for(n), kThreads, 0, st>>>(a, b, n, partials, ticket, out);
}

void launch_fill(double* x, int64_t n, double v, cudaStream_t st) {
  fill_kernel<<<blocks_for(n), kThreads, 0, st>>>(x, n, v);
}

cudaError_t launch_oc(double* rho, const double* dc, const double* dv, int64_t n, double target,
                      double rho_min, double move, double* partials, double* out, cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, oc_kernel, kThreads, 0);
  int blocks = sms * (per_sm > 2 ? 2 : per_sm);
  const int need = (int)((n + kThreads - 1) / kThreads);
  if (blocks > need) blocks = need < 1 ? 1 : need;
  void* args[] = {&rho, (void*)&dc, (void*)&dv, &n, &target, &rho_min, &move, &partials, &out};
  return cudaLaunchCooperativeKernel((void*)oc_kernel, blocks, kThreads, args, 0, st);
}

}  // namespace ddel
