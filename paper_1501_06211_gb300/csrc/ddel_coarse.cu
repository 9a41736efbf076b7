// Coarse space of the interface PCG (an addition to the paper's face-local
// preconditioner of Sec. 4): orthonormal basis by Cholesky QR, the k x k
// Galerkin matrix E = Q^T S Q and its inverse, and the Galerkin initial guess.
#include "ddel_device.cuh"
#include "ddel_launch.h"

namespace ddel {
namespace {

constexpr int kGramThreads = 256;
constexpr int kGramBlocks = 64;
constexpr int kPairs = kMaxCoarse * kMaxCoarse;

// out = A^T B for k <= kMaxCoarse columns of length n (column-major), every
// entry a deterministic grid reduction.
__global__ void __launch_bounds__(kGramThreads) gram_kernel(const double* __restrict__ A,
                                                            const double* __restrict__ B, int k,
                                                            int64_t n, double* out,
                                                            double* partials, unsigned* ticket) {
  __shared__ double scratch[kPairs * 32];
  double acc[kPairs];
#pragma unroll
  for (int q = 0; q < kPairs; ++q) acc[q] = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n;
       g += (int64_t)gridDim.x * blockDim.x) {
    double a[kMaxCoarse], b[kMaxCoarse];
#pragma unroll
    for (int i = 0; i < kMaxCoarse; ++i) {
      a[i] = i < k ? A[i * n + g] : 0.0;
      b[i] = i < k ? B[i * n + g] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < kMaxCoarse; ++i)
#pragma unroll
      for (int j = 0; j < kMaxCoarse; ++j) acc[i * kMaxCoarse + j] += a[i] * b[j];
  }
  if (grid_sum<kPairs, kGramThreads>(acc, partials, ticket, scratch) && threadIdx.x == 0)
    for (int q = 0; q < kPairs; ++q) out[q] = acc[q];
}

// Cholesky G = R^T R of the Gram matrix, in column order; a column whose
// pivot is below drop * max(diag G) depends on the earlier ones and is left
// out.  T = R^-1 restricted to the kept columns, so that Z T has orthonormal
// columns (one thread: k <= 8).
__global__ void cholqr_factor_kernel(const double* __restrict__ G, int k, double drop, double* T,
                                     int* k_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double R[kMaxCoarse][kMaxCoarse] = {};
  int keep[kMaxCoarse];
  double gmax = 0.0;
  for (int i = 0; i < k; ++i) gmax = fmax(gmax, G[i * kMaxCoarse + i]);
  int m = 0;  // kept columns so far
  for (int j = 0; j < k; ++j) {
    // column j against the kept ones: R[.][m] = R_kept^-T G[kept][j]
    double col[kMaxCoarse];
    double d = G[j * kMaxCoarse + j];
    for (int a = 0; a < m; ++a) {
      double v = G[keep[a] * kMaxCoarse + j];
      for (int b = 0; b < a; ++b) v -= R[b][a] * col[b];
      col[a] = v / R[a][a];
      d -= col[a] * col[a];
    }
    if (!(d > drop * gmax) || !isfinite(d)) continue;
    for (int a = 0; a < m; ++a) R[a][m] = col[a];
    R[m][m] = sqrt(d);
    keep[m++] = j;
  }
  // T (k x m): rows index the original columns, T[keep[a]][.] = (R^-1)[a][.]
  double Rinv[kMaxCoarse][kMaxCoarse] = {};
  for (int c = 0; c < m; ++c) {
    Rinv[c][c] = 1.0 / R[c][c];
    for (int a = c - 1; a >= 0; --a) {
      double v = 0.0;
      for (int b = a + 1; b <= c; ++b) v += R[a][b] * Rinv[b][c];
      Rinv[a][c] = -v / R[a][a];
    }
  }
  for (int i = 0; i < kMaxCoarse * kMaxCoarse; ++i) T[i] = 0.0;
  for (int a = 0; a < m; ++a)
    for (int c = 0; c < m; ++c) T[keep[a] * kMaxCoarse + c] = Rinv[a][c];
  *k_out = m;
}

__global__ void apply_T_kernel(const double* __restrict__ Z, const double* __restrict__ T, int k,
                               const int* __restrict__ k_out, int64_t n, double* out) {
  const int m = *k_out;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n;
       g += (int64_t)gridDim.x * blockDim.x) {
    double z[kMaxCoarse];
#pragma unroll
    for (int i = 0; i < kMaxCoarse; ++i) z[i] = i < k ? Z[i * n + g] : 0.0;
    for (int c = 0; c < m; ++c) {
      double v = 0.0;
#pragma unroll
      for (int i = 0; i < kMaxCoarse; ++i) v += z[i] * T[i * kMaxCoarse + c];
      out[c * n + g] = v;
    }
  }
}

// Einv = E^-1 via Cholesky of the symmetrised E; flag = 0 when a pivot is not
// positive (E not SPD: the coarse space is not used).
__global__ void coarse_invert_kernel(const double* __restrict__ E, int k, double* Einv, int* flag) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double L[kMaxCoarse][kMaxCoarse] = {};
  int ok = 1;
  for (int j = 0; j < k && ok; ++j) {
    for (int i = j; i < k; ++i) {
      double v = 0.5 * (E[i * kMaxCoarse + j] + E[j * kMaxCoarse + i]);
      for (int q = 0; q < j; ++q) v -= L[i][q] * L[j][q];
      if (i == j) {
        if (!(v > 0.0) || !isfinite(v)) {
          ok = 0;
          break;
        }
        L[j][j] = sqrt(v);
      } else {
        L[i][j] = v / L[j][j];
      }
    }
  }
  for (int i = 0; i < kMaxCoarse * kMaxCoarse; ++i) Einv[i] = 0.0;
  *flag = ok;
  if (!ok) return;
  // columns of E^-1: solve L L^T x = e_c
  for (int c = 0; c < k; ++c) {
    double y[kMaxCoarse];
    for (int i = 0; i < k; ++i) {
      double v = i == c ? 1.0 : 0.0;
      for (int q = 0; q < i; ++q) v -= L[i][q] * y[q];
      y[i] = v / L[i][i];
    }
    for (int i = k - 1; i >= 0; --i) {
      double v = y[i];
      for (int q = i + 1; q < k; ++q) v -= L[q][i] * Einv[q * kMaxCoarse + c];
      Einv[i * kMaxCoarse + c] = v / L[i][i];
    }
  }
}

// Galerkin initial guess: y = Q^T g, v = (S Q)^T g, c0 = E^-1 y, and
// ||g - S Q c0||^2 = ||g||^2 - 2 c0^T v + c0^T G c0; c0 = 0 when that exceeds
// ||g||^2 (the guess would raise the residual).
__global__ void __launch_bounds__(kGramThreads) coarse_x0_kernel(CoarseDev cd, const double* __restrict__ g,
                                                                 int64_t n, PcgState* st) {
  constexpr int NV = 2 * kMaxCoarse + 1;
  __shared__ double scratch[NV * 32];
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0.0;
  const int k = cd.k;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const double gv = g[q];
    acc[0] += gv * gv;
#pragma unroll
    for (int i = 0; i < kMaxCoarse; ++i)
      if (i < k) {
        acc[1 + i] += cd.Q[i * n + q] * gv;
        acc[1 + kMaxCoarse + i] += cd.SQ[i * n + q] * gv;
      }
  }
  if (grid_sum<NV, kGramThreads>(acc, st->partials, &st->ticket[2], scratch) && threadIdx.x == 0) {
    double c[kMaxCoarse] = {};
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) c[i] += cd.Einv[i * kMaxCoarse + j] * acc[1 + j];
    double r2 = acc[0];
    for (int i = 0; i < k; ++i) {
      r2 -= 2.0 * c[i] * acc[1 + kMaxCoarse + i];
      for (int j = 0; j < k; ++j) r2 += c[i] * cd.G[i * kMaxCoarse + j] * c[j];
    }
    const int use = isfinite(r2) && r2 <= acc[0];
    for (int i = 0; i < kMaxCoarse; ++i) st->c0[i] = use && i < k ? c[i] : 0.0;
    st->x0_used = use;
  }
}

int grid_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 4 * 152 ? 4 * 152 : b));
}

}  // namespace

void launch_gram(const double* A, const double* B, int k, int64_t n, double* out, double* partials,
                 unsigned* ticket, cudaStream_t st) {
  gram_kernel<<<kGramBlocks, kGramThreads, 0, st>>>(A, B, k, n, out, partials, ticket);
}

void launch_cholqr_factor(const double* G, int k, double drop, double* T, int* k_out, cudaStream_t st) {
  cholqr_factor_kernel<<<1, 32, 0, st>>>(G, k, drop, T, k_out);
}

void launch_apply_T(const double* Z, const double* T, int k, const int* k_out, int64_t n, double* out,
                    cudaStream_t st) {
  apply_T_kernel<<<grid_for(n), 256, 0, st>>>(Z, T, k, k_out, n, out);
}

void launch_coarse_invert(const double* E, int k, double* Einv, int* flag, cudaStream_t st) {
  coarse_invert_kernel<<<1, 32, 0, st>>>(E, k, Einv, flag);
}

void launch_coarse_x0(const CoarseDev& cd, const double* g, int64_t n, PcgState* s, cudaStream_t st) {
  coarse_x0_kernel<<<kGramBlocks, kGramThreads, 0, st>>>(cd, g, n, s);
}

}  // namespace ddel
