// Global interface preconditioner of Sec. 3 applied by inverse Lanczos, and
// the full-system flexible GMRES of the paper's Table 1 (Sec. 3-4).
//
//  * global_prec_kernel: z = S~^-1 r with S~ = W H~_theta W per displacement
//    component, H~_theta = M (M^-1 L)^(1 - theta) (eq. NumberEight and
//    NumberNine on the whole interface Gamma).  One CTA per component runs the
//    whole application: b = M^-1 r by Jacobi-preconditioned CG, k steps of
//    Lanczos for L^-1 M in the M inner product (each step an inner PCG on L,
//    preconditioned by L on each face with the cross points removed), the
//    eigen-decomposition of the k x k tridiagonal T_k by one warp (cyclic
//    Jacobi rotations) and z = ||b||_M Q_k f(T_k) e_1, f(t) = t^(1 - theta).
//    The interface of one component holds a few thousand to a few tens of
//    thousands of DOFs and every step depends on the previous one's sums, so
//    one CTA with block-wide reductions (no grid-wide synchronisation) is the
//    launch shape; the vectors live in global memory (L2-resident).
//  * multi_dot / multi_axpy: the classical Gram-Schmidt passes of FGMRES over
//    the stored Krylov basis (deterministic two-level sums).
#include <cuda_runtime.h>

#include <cmath>

#include "ddel_device.cuh"
#include "ddel_globalprec.h"

namespace ddel {
namespace {

constexpr int kGpThreads = 1024;

// Block-wide sum in a fixed order (warp butterflies, then warp 0 over the
// warp totals); every thread returns the same bits.  sh: 33 doubles.
__device__ __forceinline__ double cta_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = lane < nw ? sh[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) sh[32] = t;
  }
  __syncthreads();
  const double tot = sh[32];
  __syncthreads();  // sh is reused by the next call
  return tot;
}

// y = A x for one component's CSR matrix (rows of this thread); returns the
// thread's share of x . y.
__device__ __forceinline__ double spmv_dot(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                           const double* __restrict__ val, const double* x, double* y) {
  double d = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double acc = 0.0;
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) acc += val[q] * x[col[q]];
    y[i] = acc;
    d += x[i] * acc;
  }
  return d;
}

// Inner preconditioner of the solve with L (Sec. 4): the inverse of L
// restricted to each face (cross points removed) and 1 / L_ii at cross
// points.  Returns the thread's share of r . z.
__device__ __forceinline__ double precond_L(const GPComp& c, const double* r, double* z) {
  double d = 0.0;
  for (int i = threadIdx.x; i < c.n; i += blockDim.x) {
    const int f = c.row_face[i];
    double zi;
    if (f < 0) {
      zi = r[i] * c.cross_inv[i];
    } else {
      const int l0 = c.face_l0[f], nf = c.face_n[f], a = i - l0;
      const double* A = c.face_inv + c.face_inv_off[f] + (int64_t)a * nf;
      zi = 0.0;
      for (int b = 0; b < nf; ++b) zi += A[b] * r[l0 + b];
    }
    z[i] = zi;
    d += r[i] * zi;
  }
  return d;
}

// PCG on A x = b for one component (x, r, z, p, q: work vectors of length n;
// x starts at 0): stops when ||r|| <= tol ||b|| or after max_it iterations,
// the order of operations of textbook PCG with the test at the top of the
// loop.  prec: 0 Jacobi (1 / diag), 1 the face-block preconditioner of L.
// Returns the iteration count.  All threads of the block call it.
__device__ int cta_pcg(const GPComp& c, const int64_t* rp, const int32_t* col, const double* val,
                       const double* dinv, int prec, const double* b, double* x, double* r, double* z,
                       double* p, double* q, double tol, int max_it, double* sh) {
  const int n = c.n;
  double rz = 0.0, bb = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    x[i] = 0.0;
    r[i] = b[i];
    bb += b[i] * b[i];
  }
  __syncthreads();
  if (prec == 1) {
    rz = precond_L(c, r, z);
  } else {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      z[i] = r[i] * dinv[i];
      rz += r[i] * z[i];
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = z[i];
  rz = cta_sum(rz, sh);
  const double nb = sqrt(cta_sum(bb, sh));
  double rr = nb * nb;
  int k = 0;
  while (sqrt(rr) > tol * nb && k < max_it) {
    const double pq = cta_sum(spmv_dot(n, rp, col, val, p, q), sh);
    const double a = rz / pq;
    double rl = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      x[i] += a * p[i];
      const double ri = r[i] - a * q[i];
      r[i] = ri;
      rl += ri * ri;
    }
    rr = cta_sum(rl, sh);  // also orders the r writes before the preconditioner
    double rzl = 0.0;
    if (prec == 1) {
      rzl = precond_L(c, r, z);
    } else {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        z[i] = r[i] * dinv[i];
        rzl += r[i] * z[i];
      }
    }
    const double rz_new = cta_sum(rzl, sh);
    const double beta = rz_new / rz;
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = z[i] + beta * p[i];
    rz = rz_new;
    ++k;
    __syncthreads();  // p complete before the next product reads it
  }
  __syncthreads();
  return k;
}

// Eigen-decomposition of the symmetric m x m matrix A (row-major, shared
// memory, destroyed) by cyclic Jacobi rotations in warp 0: on return the
// diagonal of A holds the eigenvalues and the columns of V (row-major m x m)
// the eigenvectors.  Lane l updates row / column l of each rotation.
__device__ void warp_jacobi_eig(int m, double* A, double* V) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < m * m; i += 32) V[i] = (i / m == i % m) ? 1.0 : 0.0;
  __syncwarp();
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = lane; i < m * m; i += 32) {
      const double v = A[i] * A[i];
      tot += v;
      if (i / m != i % m) off += v;
    }
    off = warp_sum(off);
    tot = warp_sum(tot);
    if (!(off > 1e-32 * tot)) break;
    for (int pp = 0; pp < m - 1; ++pp)
      for (int qq = pp + 1; qq < m; ++qq) {
        const double apq = A[pp * m + qq];
        if (apq == 0.0) continue;  // uniform: every lane reads the same value
        const double app = A[pp * m + pp], aqq = A[qq * m + qq];
        const double th = (aqq - app) / (2.0 * apq);
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        __syncwarp();
        if (lane < m) {  // columns p, q of A J
          const double akp = A[lane * m + pp], akq = A[lane * m + qq];
          A[lane * m + pp] = cs * akp - sn * akq;
          A[lane * m + qq] = sn * akp + cs * akq;
        }
        __syncwarp();
        if (lane < m) {  // rows p, q of J^T (A J)
          const double apk = A[pp * m + lane], aqk = A[qq * m + lane];
          A[pp * m + lane] = cs * apk - sn * aqk;
          A[qq * m + lane] = sn * apk + cs * aqk;
          const double vkp = V[lane * m + pp], vkq = V[lane * m + qq];
          V[lane * m + pp] = cs * vkp - sn * vkq;
          V[lane * m + qq] = sn * vkp + cs * vkq;
        }
        __syncwarp();
      }
  }
}

// z = S~^-1 r on the interface, one CTA per displacement component c.
// Work vectors of component c (n = its Gamma DOFs): rc, b, w, x, r, zz, pp,
// qq, then Q_0..Q_k and t_j = M Q_j (j < k).  out (may be NULL): per
// component [m, mass iterations, alpha (kLz), beta (kLz), inner its (kLz)].
__global__ void __launch_bounds__(kGpThreads) global_prec_kernel(GPDev gd, const double* __restrict__ rg,
                                                                  double* __restrict__ zg,
                                                                  const double* __restrict__ diagG, double theta,
                                                                  int ksteps, double inner_tol, double mass_tol,
                                                                  int scaling, double* out) {
  const GPComp& c = gd.c[blockIdx.x];
  const int n = c.n, tid = threadIdx.x, T = blockDim.x;
  __shared__ double sh[33];
  __shared__ double Tm[kLz * kLz], Vm[kLz * kLz];
  __shared__ double alpha[kLz], beta[kLz], yv[kLz];
  __shared__ int inner_its[kLz];
  double* rc = c.work;
  double* b = rc + n;
  double* w = b + n;
  double* xx = w + n;
  double* rr = xx + n;
  double* zz = rr + n;
  double* pp = zz + n;
  double* qq = pp + n;
  double* Q = qq + n;              // (ksteps + 1) x n
  double* Tv = Q + (size_t)(ksteps + 1) * n;  // ksteps x n: M Q_j
  // scaled right-hand side: rc = W^-1 r on this component
  for (int i = tid; i < n; i += T) {
    double wi = 1.0;
    if (scaling) wi = sqrt(diagG[c.pos[i]] / (pow(c.Mdiag[i], theta) * pow(c.Ldiag[i], 1.0 - theta)));
    c.w[i] = wi;
    rc[i] = rg[c.pos[i]] / wi;
  }
  __syncthreads();
  // b = M^-1 rc
  const int mass_its = cta_pcg(c, c.rowptr, c.col, c.M, c.Minv_diag, 0, rc, b, rr, zz, pp, qq, mass_tol, 500, sh);
  // ||b||_M
  const double nb = sqrt(cta_sum(spmv_dot(n, c.rowptr, c.col, c.M, b, qq), sh));
  if (!(nb > 0.0)) {
    for (int i = tid; i < n; i += T) zg[c.pos[i]] = 0.0;
    if (out && tid == 0) {
      double* o = out + blockIdx.x * (2 + 3 * kLz);
      o[0] = 0;
      o[1] = mass_its;
    }
    return;
  }
  for (int i = tid; i < n; i += T) Q[i] = b[i] / nb;
  __syncthreads();
  int m = ksteps;
  double amax = 0.0;
  for (int j = 0; j < ksteps; ++j) {
    const double* qj = Q + (size_t)j * n;
    double* tj = Tv + (size_t)j * n;
    // t_j = M q_j; w = L^-1 t_j by the inner PCG of Sec. 4
    for (int i = tid; i < n; i += T) {
      double acc = 0.0;
      for (int64_t e = c.rowptr[i]; e < c.rowptr[i + 1]; ++e) acc += c.M[e] * qj[c.col[e]];
      tj[i] = acc;
    }
    __syncthreads();
    const int its = cta_pcg(c, c.rowptr, c.col, c.L, nullptr, 1, tj, w, rr, zz, pp, qq, inner_tol, 1000, sh);
    // alpha_j = (q_j, w)_M = t_j . w
    double a = 0.0;
    for (int i = tid; i < n; i += T) a += tj[i] * w[i];
    a = cta_sum(a, sh);
    // full M-orthogonalisation against q_0 .. q_j (modified Gram-Schmidt)
    for (int l = 0; l <= j; ++l) {
      const double* ql = Q + (size_t)l * n;
      const double* tl = Tv + (size_t)l * n;
      double h = 0.0;
      for (int i = tid; i < n; i += T) h += tl[i] * w[i];
      h = cta_sum(h, sh);
      for (int i = tid; i < n; i += T) w[i] -= h * ql[i];
      __syncthreads();
    }
    const double bt = sqrt(fmax(cta_sum(spmv_dot(n, c.rowptr, c.col, c.M, w, qq), sh), 0.0));
    if (tid == 0) {
      alpha[j] = a;
      beta[j] = bt;
      inner_its[j] = its;
    }
    amax = fmax(amax, fabs(a));
    if (j + 1 < ksteps) {
      if (bt <= 1e-14 * fmax(amax, 1e-300)) {  // invariant subspace: exact
        m = j + 1;
        break;
      }
      double* qn = Q + (size_t)(j + 1) * n;
      for (int i = tid; i < n; i += T) qn[i] = w[i] / bt;
      __syncthreads();
    }
  }
  __syncthreads();
  // f(T_m) e_1 with f(t) = max(t, 0)^(1 - theta) from the eigenpairs of T_m
  if (threadIdx.x < 32) {
    for (int i = threadIdx.x; i < m * m; i += 32) {
      const int r0 = i / m, c0 = i % m;
      Tm[i] = r0 == c0 ? alpha[r0] : (r0 == c0 + 1 ? beta[c0] : (c0 == r0 + 1 ? beta[r0] : 0.0));
    }
    __syncwarp();
    warp_jacobi_eig(m, Tm, Vm);
    __syncwarp();
    if (threadIdx.x < m) {
      const int i = threadIdx.x;
      double y = 0.0;
      for (int l = 0; l < m; ++l) y += Vm[i * m + l] * pow(fmax(Tm[l * m + l], 0.0), 1.0 - theta) * Vm[l];
      yv[i] = y;
    }
  }
  __syncthreads();
  // z = W^-1 ||b||_M Q_m y
  for (int i = tid; i < n; i += T) {
    double acc = 0.0;
    for (int l = 0; l < m; ++l) acc += yv[l] * Q[(size_t)l * n + i];
    zg[c.pos[i]] = nb * acc / c.w[i];
  }
  if (out && tid == 0) {
    double* o = out + blockIdx.x * (2 + 3 * kLz);
    o[0] = m;
    o[1] = mass_its;
    for (int l = 0; l < m; ++l) {
      o[2 + l] = alpha[l];
      if (l + 1 < m) o[2 + kLz + l] = beta[l];
      o[2 + 2 * kLz + l] = inner_its[l];
    }
  }
}

// ---- FGMRES vector kernels ------------------------------------------------
constexpr int kMdBlocks = 2 * 152;  // partial sums per dot product
constexpr int kMdThreads = 256;

// partial[j * kMdBlocks + bx] = the block's share of V_j . w, j = blockIdx.y.
__global__ void __launch_bounds__(kMdThreads) multi_dot_kernel(const double* __restrict__ V, int64_t ld,
                                                               const double* __restrict__ w, int64_t n,
                                                               double* __restrict__ partial) {
  __shared__ double sh[33];
  const double* v = V + (int64_t)blockIdx.y * ld;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += v[i] * w[i];
  acc = cta_sum(acc, sh);
  if (threadIdx.x == 0) partial[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = acc;
}

// h[j] = sum of the partials of dot product j (one warp each), added to h
// when accumulate != 0.
__global__ void multi_dot_finish(const double* __restrict__ partial, int nb, int nv, double* h, int accumulate) {
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= nv) return;
  const double s = reduce_partials_warp(partial + (int64_t)j * nb, nb);
  if ((threadIdx.x & 31) == 0) h[j] = accumulate ? h[j] + s : s;
}

// w -= sum_j h[j] V_j  (sign = -1), or u = sum_j h[j] V_j (sign = 0: overwrite).
__global__ void multi_axpy_kernel(const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ h,
                                  double* w, int64_t n, int overwrite) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < nv; ++j) acc += h[j] * V[(int64_t)j * ld + i];
    w[i] = overwrite ? acc : w[i] - acc;
  }
}

// out = in * (1 / h[idx]) (the new Krylov vector), or out = in / s0 (idx < 0).
__global__ void scale_kernel_gm(const double* __restrict__ in, double* __restrict__ out, int64_t n,
                                const double* __restrict__ h, int idx, double s0) {
  const double s = idx >= 0 ? h[idx] : s0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i] / s;
}

// out[g] = in[gamma_dof[g]]
__global__ void gather_gamma_kernel(const int64_t* __restrict__ gd, int64_t ng, const double* __restrict__ in,
                                    double* __restrict__ out) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x)
    out[g] = in[gd[g]];
}

int grid_of(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : g > 152 * 8 ? 152 * 8 : g);
}

}  // namespace

size_t global_prec_work_elems(int n, int ksteps) { return (size_t)(2 * ksteps + 9) * n; }

cudaError_t launch_global_prec(const GPDev& gd, const double* r, double* z, const double* diagG, double theta,
                               int ksteps, double inner_tol, double mass_tol, int scaling, double* out,
                               cudaStream_t st) {
  global_prec_kernel<<<gd.ncomp, kGpThreads, 0, st>>>(gd, r, z, diagG, theta, ksteps, inner_tol, mass_tol,
                                                      scaling, out);
  return cudaGetLastError();
}

void launch_multi_dot(const double* V, int64_t ld, int nv, const double* w, int64_t n, double* partial,
                      double* h, int accumulate, cudaStream_t st) {
  multi_dot_kernel<<<dim3(kMdBlocks, nv), kMdThreads, 0, st>>>(V, ld, w, n, partial);
  multi_dot_finish<<<(nv + 7) / 8, 256, 0, st>>>(partial, kMdBlocks, nv, h, accumulate);
}

size_t multi_dot_partials(int nv) { return (size_t)kMdBlocks * nv; }

void launch_multi_axpy(const double* V, int64_t ld, int nv, const double* h, double* w, int64_t n, int overwrite,
                       cudaStream_t st) {
  multi_axpy_kernel<<<grid_of(n), 256, 0, st>>>(V, ld, nv, h, w, n, overwrite);
}

void launch_scale_gm(const double* in, double* out, int64_t n, const double* h, int idx, double s0,
                     cudaStream_t st) {
  scale_kernel_gm<<<grid_of(n), 256, 0, st>>>(in, out, n, h, idx, s0);
}

void launch_gather_gamma(const int64_t* gd, int64_t ng, const double* in, double* out, cudaStream_t st) {
  gather_gamma_kernel<<<grid_of(ng), 256, 0, st>>>(gd, ng, in, out);
}

}  // namespace ddel
