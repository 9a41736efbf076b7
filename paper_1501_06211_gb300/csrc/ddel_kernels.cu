// CUDA kernels of the hot path for sm_103a (2D Q1 path; the 3D H8 path lives in
// ddel_kernels3d.cu).
//
//  * factor2d_kernel  : fused assembly of the interior line blocks of every
//                       K_{I_i I_i} (eq. NumberFive) and its block-tridiagonal
//                       Cholesky factorisation, one CTA per subdomain.
//  * schur2d_kernel   : per-subdomain solve with the factor (eq. 3MatSplit2):
//                       w = f_I - K_IG x, t = K_II^-1 w by block forward and
//                       backward substitution, y = (K^(i) [t; x])_G.  Factor
//                       blocks stream from HBM through a TMA bulk-copy ring
//                       buffer; one warp per subdomain.
//  * pcg_*_kernel     : interface PCG with the face-local preconditioner of
//                       Sec. 3-4; deterministic two-level FP64 dot products.
//  * apply_K_kernel   : global element-by-element K x / f - K x in FP64.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>

#include "ddel_device.cuh"
#include "ddel_launch.h"

namespace ddel {
namespace {

constexpr int kRedThreads = 256;

__device__ __forceinline__ int64_t node2(const DevTables& t, int i, int j) {
  return (int64_t)i * t.nn[1] + j;
}

// ============================================================ assembly
__global__ void scale_kernel(const double* __restrict__ rho, int64_t n, double E, double p,
                             double* s64, float* s32, int* err) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double r = rho[e];
    if (!(r > 0.0) || !isfinite(r)) {
      atomicExch(err, kErrBadRho);
      r = 1.0;
    }
    const double v = E * pow(r, p);
    s64[e] = v;
    s32[e] = (float)v;
  }
}

// diag(K_GG) at every Gamma DOF: sum over the elements touching the node.
template <int DIM>
__global__ void gamma_diag_kernel(DevTables t, DevFields fld) {
  constexpr int ND = DIM << DIM;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < t.n_gamma;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t dof = t.gamma_dof[g];
    const int64_t n = dof / DIM;
    const int c = (int)(dof % DIM);
    const int k = DIM == 3 ? (int)(n % t.nn[2]) : 0;
    const int64_t ij = DIM == 3 ? n / t.nn[2] : n;
    const int j = (int)(ij % t.nn[1]), i = (int)(ij / t.nn[1]);
    double acc = 0.0;
    for (int ox = 0; ox < 2; ++ox) {
      const int ex = i - ox;
      if (ex < 0 || ex >= t.ne[0]) continue;
      for (int oy = 0; oy < 2; ++oy) {
        const int ey = j - oy;
        if (ey < 0 || ey >= t.ne[1]) continue;
        for (int oz = 0; oz < (DIM == 3 ? 2 : 1); ++oz) {
          const int ez = k - oz;
          if (DIM == 3 && (ez < 0 || ez >= t.ne[2])) continue;
          const int64_t e = DIM == 3 ? ((int64_t)ex * t.ne[1] + ey) * t.ne[2] + ez
                                     : (int64_t)ex * t.ne[1] + ey;
          const int ln = elem_local_node(ox, oy, oz);
          acc += fld.scale64[e] * t.Ke64[(ln * DIM + c) * ND + ln * DIM + c];
        }
      }
    }
    fld.diagG[g] = acc;
  }
}

// Face scaling (one warp per face block) and cross-point diagonal.  Each face
// block is applied as S~_f^-1 r = W^-1 H_f^-1 W^-1 r with a diagonal W:
//   mode 0: W = I (paper-literal);
//   mode 1: W = sqrt(alpha) I, alpha = mean diag(K_GG) / mean diag(H_f);
//   mode 2: W_ii = sqrt(diag(K_GG)_i / diag(H_f)_i), so diag(S~_f) = diag(K_GG).
__global__ void face_scale_kernel(DevTables t, DevFields fld, int face_scaling, int cross_mode) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int b = gw; b < t.n_blocks; b += nw) {
    const int off = t.blk_off[b], n = t.blk_n[b];
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += fld.diagG[off + i];
    s = warp_sum(s);
    const double alpha = (s / n) / t.blk_hmean[b];
    if (lane == 0) fld.blk_alpha[b] = face_scaling == 1 ? alpha : 1.0;
    for (int i = lane; i < n; i += 32) {
      double w = 1.0;
      if (face_scaling == 1) w = sqrt(alpha);
      if (face_scaling == 2) w = sqrt(fld.diagG[off + i] / t.hdiag[off + i]);
      fld.face_w[off + i] = 1.0 / w;  // stored as the reciprocal: products, no divisions later
    }
  }
  const int64_t ncross = t.n_gamma - t.n_face_dofs;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncross;
       c += (int64_t)gridDim.x * blockDim.x)
    fld.cross_scale[c] = cross_mode == 0 ? 1.0 / fld.diagG[t.n_face_dofs + c] : 1.0;
}

// ============================================================ factorisation
// Entry ((kr, r), (kc, c)) of K_{I_i I_i}: rows r of interior plane kr, columns
// c of plane kc.  Rows beyond the block size and fixed DOFs form identity rows,
// which keeps every block of a uniform padded size BP.
template <typename T>
__device__ __forceinline__ T entry2d(const DevTables& t, const SubInfo& si, const T* ke,
                                     const T* __restrict__ scale, int kr, int r, int kc, int c) {
  const bool vr = r < si.bsz, vc = c < si.bsz;
  const int xr = si.ilo[0] + kr, yr = si.ilo[1] + (r >> 1), cr = r & 1;
  const int xc = si.ilo[0] + kc, yc = si.ilo[1] + (c >> 1), cc = c & 1;
  const bool fr = !vr || t.fixed[2 * node2(t, xr, yr) + cr];
  const bool fc = !vc || t.fixed[2 * node2(t, xc, yc) + cc];
  if (fr || fc) return (kr == kc && r == c) ? T(1) : T(0);
  if (abs(yr - yc) > 1 || abs(xr - xc) > 1) return T(0);
  T sum = T(0);
  const int s = t.s;
  for (int ex = max(xr, xc) - 1; ex <= min(xr, xc); ++ex) {
    const int ea = ex - si.lo[0];
    if (ea < 0 || ea >= s) continue;
    for (int ey = max(yr, yc) - 1; ey <= min(yr, yc); ++ey) {
      const int eb = ey - si.lo[1];
      if (eb < 0 || eb >= s) continue;
      const int la = elem_local_node(xr - ex, yr - ey, 0);
      const int lb = elem_local_node(xc - ex, yc - ey, 0);
      sum += scale[(int64_t)ex * t.ne[1] + ey] * ke[(la * 2 + cr) * 8 + lb * 2 + cc];
    }
  }
  return sum;
}

// Block step k of the block-tridiagonal Cholesky factorisation of K_{I_i I_i}
// over the planes of interior nodes (eq. NumberFive): A_kk -= C_k C_k^T;
// L_kk = chol(A_kk); D_k = L_kk^-1; C_{k+1} = A_{k+1,k} D_k^T.  Stored per
// subdomain as [C_k | D_k] for every k (C_k dense column-major BP x BP, D_k
// packed lower column-major), so that one forward step reads one contiguous
// [C_k D_k] and one backward step one contiguous [D_k C_{k+1}].
//
// One CTA of kFacThreads threads per subdomain, every block in shared memory:
//  (a) the lower triangle of A_kk (nonzero only where the nodes' y differ by
//      at most one) minus C_k C_k^T, in TS x TS register tiles, over the
//      columns where C_k does not vanish;
//  (b) blocked right-looking Cholesky with PW-wide panels: the diagonal block
//      by one warp (one lane per entry of each column step's update), each
//      panel row by one thread, the trailing update in TS x TS tiles -- three
//      CTA barriers per panel;
//  (c) D_k = L_kk^-1 by 8 x 8 blocks: the diagonal blocks inverted by one
//      thread per column, then block row p from the rows above,
//      D_pq = -D_pp sum_{q <= m < p} L_pm D_mq, every entry one thread;
//  (e) C_{k+1} = A_{k+1,k} D_k^T using the sparsity of A_{k+1,k}: a row
//      couples only to the nodes y - 1, y, y + 1 of the plane before, six
//      consecutive columns, assembled once per row.
// The FP64 pipe of this GPU retires one warp instruction per 16 clocks per SM
// whatever the number of active lanes, so the sequential parts are laid out
// to keep the lanes of each FP64 instruction busy, and the FP64 pivots take one
// reciprocal square root (Newton) instead of a square root and divisions.
// A pivot that is not positive is replaced by 1 and reported (kErrPivot, the
// lowest such subdomain in bad_sub).
constexpr int kFacThreads = 256;


template <typename T>
__device__ __forceinline__ void lds4(const T* p, T (&v)[4]) {
  if constexpr (sizeof(T) == 8) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  } else {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
  }
}

// tile q of the lower block triangle of an nt x nt tiling -> (ti, tj), tj <= ti
__device__ __forceinline__ void lower_tile(int q, int nt, int& ti, int& tj) {
  tj = 0;
  while (q >= nt - tj) {
    q -= nt - tj;
    ++tj;
  }
  ti = tj + q;
}

template <typename T, int BP>
size_t factor2d_smem() {
  return (size_t)(2 * BP * (BP + 1) + BP * BP + 64 + BP + 6 * BP) * sizeof(T);
}

template <typename T, int BP>
__global__ void __launch_bounds__(kFacThreads, BP == 32 ? 4 : 1)
    factor2d_kernel(DevTables t, const T* __restrict__ Ke_g, const T* __restrict__ scale, T* __restrict__ factor,
                    int* err, int* bad_sub) {
  constexpr int LD = BP + 1, PC = BP * BP, PD = BP * (BP + 1) / 2, STAGE = PC + PD;
  constexpr int TS = BP == 32 ? 2 : 4;                   // register tile edge
  constexpr int NT = BP / TS;                            // tiles per edge
  constexpr int PW = BP == 32 ? 8 : 16;                  // Cholesky panel width
  constexpr int NJ = kFacThreads / BP;                   // column groups of the C product
  const int sub = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const SubInfo si = t.subs[sub];
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);  // BP x LD, lower part: A_kk, then L_kk
  T* Dm = A + BP * LD;                    // BP x LD, lower part: D_k
  T* CT = Dm + BP * LD;                   // BP x BP: CT[m * BP + i] = C_k(i, m)
  T* ke = CT + BP * BP;                   // 64
  T* rdiag = ke + 64;                     // BP: 1 / L_kk(j, j)
  T* anz = rdiag + BP;                    // BP x 6: the nonzeros of a row of A_{k+1,k}
  __shared__ int s_bad;
  for (int i = tid; i < 64; i += kFacThreads) ke[i] = Ke_g[i];
  if (tid == 0) s_bad = 0;
  __syncthreads();
  const int nb = si.nb;
  T* fb = factor + si.factor_off;
  for (int k = 0; k < nb; ++k) {
    // (a) lower triangle of A_kk - C_k C_k^T.  C_k(i, m) vanishes below the
    // lowest column row i couples to, 2 (i / 2) - 2 (the coupling computed in
    // (e) adds no term there), so a tile row's products start at TS ti - 2;
    // the tiles go row by row so that the lanes of a warp share that start.
    for (int q = tid; q < NT * (NT + 1) / 2; q += kFacThreads) {
      int ti = 0, tj = q;
      while (tj > ti) {
        tj -= ti + 1;
        ++ti;
      }
      T acc[TS][TS];
#pragma unroll
      for (int u = 0; u < TS; ++u)
#pragma unroll
        for (int v = 0; v < TS; ++v) acc[u][v] = T(0);
      if (k > 0) {
#pragma unroll 4
        for (int m = max(0, TS * ti - 2); m < BP; ++m) {
          T a[TS], b[TS];
          if constexpr (TS == 4) {
            lds4(CT + m * BP + 4 * ti, a);
            lds4(CT + m * BP + 4 * tj, b);
          } else {
#pragma unroll
            for (int u = 0; u < TS; ++u) a[u] = CT[m * BP + TS * ti + u], b[u] = CT[m * BP + TS * tj + u];
          }
#pragma unroll
          for (int u = 0; u < TS; ++u)
#pragma unroll
            for (int v = 0; v < TS; ++v) acc[u][v] += a[u] * b[v];
        }
      }
#pragma unroll
      for (int u = 0; u < TS; ++u)
#pragma unroll
        for (int v = 0; v < TS; ++v) {
          const int i = TS * ti + u, j = TS * tj + v;
          if (j <= i) {
            const T e = abs((i >> 1) - (j >> 1)) <= 1 ? entry2d<T>(t, si, ke, scale, k, i, k, j) : T(0);
            A[i * LD + j] = e - acc[u][v];
          }
        }
    }
    __syncthreads();
    // (b) blocked right-looking Cholesky, lower, in place
    for (int j0 = 0; j0 < BP; j0 += PW) {
      if (warp == 0) {
        for (int j = j0; j < j0 + PW; ++j) {
          T d = A[j * LD + j];
          if (!(d > T(0)) || !isfinite((double)d)) {
            if (lane == 0) s_bad = 1;
            d = T(1);
          }
          // FP64: one reciprocal square root, products; FP32 (cheap divisions
          // on this GPU): the correctly rounded square root and quotients
          T ljj, rj;
          if constexpr (sizeof(T) == 8) {
            rj = pivot_rsqrt(d);
            ljj = d * rj;
          } else {
            ljj = sqrt(d);
            rj = T(1) / ljj;
          }
          __syncwarp();
          if (lane == 0) {
            A[j * LD + j] = ljj;
            rdiag[j] = rj;
          }
          const int i = j + 1 + lane;
          if (i < j0 + PW) {
            if constexpr (sizeof(T) == 8)
              A[i * LD + j] *= rj;
            else
              A[i * LD + j] /= ljj;
          }
          __syncwarp();
          // update of the block's trailing lower triangle (m rows), one lane per entry
          const int m = j0 + PW - 1 - j;
          for (int e = lane; e < m * (m + 1) / 2; e += 32) {
            int r = 0, c = e;
            while (c > r) {
              c -= r + 1;
              ++r;
            }
            const int ii = j + 1 + r, cc = j + 1 + c;
            A[ii * LD + cc] -= A[ii * LD + j] * A[cc * LD + j];
          }
          __syncwarp();
        }
      }
      __syncthreads();
      const int r0 = j0 + PW;
      if (r0 < BP) {
        // panel rows below the diagonal block: X L_pp^T = A_ip
        for (int i = r0 + tid; i < BP; i += kFacThreads) {
          T x[PW];
#pragma unroll
          for (int c = 0; c < PW; ++c) x[c] = A[i * LD + j0 + c];
#pragma unroll
          for (int c = 0; c < PW; ++c) {
            T v = x[c];
#pragma unroll
            for (int m = 0; m < c; ++m) v -= x[m] * A[(j0 + c) * LD + j0 + m];
            if constexpr (sizeof(T) == 8)
              x[c] = v * rdiag[j0 + c];
            else
              x[c] = v / A[(j0 + c) * LD + j0 + c];
          }
#pragma unroll
          for (int c = 0; c < PW; ++c) A[i * LD + j0 + c] = x[c];
        }
        __syncthreads();
        // trailing update of the lower triangle of rows / columns [r0, BP)
        const int ntr = (BP - r0) / TS;
        for (int q = tid; q < ntr * (ntr + 1) / 2; q += kFacThreads) {
          int ti, tj;
          lower_tile(q, ntr, ti, tj);
          const int i0 = r0 + TS * ti, c0 = r0 + TS * tj;
          T acc[TS][TS];
#pragma unroll
          for (int u = 0; u < TS; ++u)
#pragma unroll
            for (int v = 0; v < TS; ++v) acc[u][v] = T(0);
#pragma unroll
          for (int m = 0; m < PW; ++m) {
            T a[TS], b[TS];
#pragma unroll
            for (int u = 0; u < TS; ++u) a[u] = A[(i0 + u) * LD + j0 + m], b[u] = A[(c0 + u) * LD + j0 + m];
#pragma unroll
            for (int u = 0; u < TS; ++u)
#pragma unroll
              for (int v = 0; v < TS; ++v) acc[u][v] += a[u] * b[v];
          }
#pragma unroll
          for (int u = 0; u < TS; ++u)
#pragma unroll
            for (int v = 0; v < TS; ++v)
              if (c0 + v <= i0 + u) A[(i0 + u) * LD + c0 + v] -= acc[u][v];
        }
      }
      __syncthreads();
    }
    // (c) D = L^-1 by 8 x 8 blocks.  Diagonal blocks: thread (p, c) inverts
    // column c of L_pp by forward substitution (zeros above the diagonal).
    if (tid < BP) {
      const int p0 = tid & ~7, c = tid & 7;
      T x[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        T v = r == c ? T(1) : T(0);
#pragma unroll
        for (int m = 0; m < r; ++m) v -= A[(p0 + r) * LD + p0 + m] * x[m];
        if constexpr (sizeof(T) == 8)
          x[r] = r >= c ? v * rdiag[p0 + r] : T(0);
        else
          x[r] = r >= c ? v / A[(p0 + r) * LD + p0 + r] : T(0);
      }
#pragma unroll
      for (int r = 0; r < 8; ++r) Dm[(p0 + r) * LD + p0 + c] = x[r];
    }
    __syncthreads();
    // block row p: T_pq = sum_{q <= m < p} L_pm D_mq (into CT, free until (e)),
    // then D_pq = -D_pp T_pq
    for (int p = 1; p < BP / 8; ++p) {
      for (int e = tid; e < p * 64; e += kFacThreads) {
        const int q = e >> 6, r = (e >> 3) & 7, c = e & 7;
        const T* Lrow = A + (8 * p + r) * LD;
        T v = T(0);
        for (int m = 8 * q; m < 8 * p; ++m) v += Lrow[m] * Dm[m * LD + 8 * q + c];
        CT[e] = v;
      }
      __syncthreads();
      for (int e = tid; e < p * 64; e += kFacThreads) {
        const int q = e >> 6, r = (e >> 3) & 7, c = e & 7;
        T v = T(0);
#pragma unroll
        for (int s2 = 0; s2 < 8; ++s2) v += Dm[(8 * p + r) * LD + 8 * p + s2] * CT[(q << 6) + (s2 << 3) + c];
        Dm[(8 * p + r) * LD + 8 * q + c] = -v;
      }
      __syncthreads();
    }
    // (d) store D_k packed lower column-major
    T* Dg = fb + (int64_t)k * STAGE + PC;
    for (int idx = tid; idx < BP * BP; idx += kFacThreads) {
      const int j = idx / BP, r = idx % BP;
      if (r >= j) Dg[j * BP - j * (j - 1) / 2 + (r - j)] = Dm[r * LD + j];
    }
    // (e) C_{k+1} = A_{k+1,k} D_k^T
    if (k + 1 < nb) {
      for (int e = tid; e < 6 * BP; e += kFacThreads) {
        const int i = e / 6, m = 2 * (i >> 1) - 2 + e % 6;
        anz[e] = (m >= 0 && m < BP) ? entry2d<T>(t, si, ke, scale, k + 1, i, k, m) : T(0);
      }
      __syncthreads();
      const int i = tid % BP, jg = tid / BP;
      if (jg < NJ) {
        const int m0 = 2 * (i >> 1) - 2;
        T a[6];
#pragma unroll
        for (int w = 0; w < 6; ++w) a[w] = anz[6 * i + w];
        T* Cg = fb + (int64_t)(k + 1) * STAGE;
        for (int j = jg; j < BP; j += NJ) {
          T c = T(0);
#pragma unroll
          for (int w = 0; w < 6; ++w) {
            const int m = m0 + w;
            if (m >= 0 && m <= j) c += a[w] * Dm[j * LD + m];
          }
          CT[j * BP + i] = c;
          Cg[j * BP + i] = c;
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0 && s_bad) {
    atomicExch(err, kErrPivot);
    atomicMin(bad_sub, sub);
  }
}

// ============================================================ subdomain solve
// K^(i) xloc at local closure node (a, b), component c (element by element,
// only elements of this subdomain).
template <typename T>
__device__ __forceinline__ T ebe_local2d(const T* ke, const T* sc, const T* xloc, int s, int a,
                                         int b, int c) {
  const int s1 = s + 1;
  T acc = T(0);
#pragma unroll
  for (int dx = 0; dx < 2; ++dx) {
    const int ea = a - dx;
    if (ea < 0 || ea >= s) continue;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const int eb = b - dy;
      if (eb < 0 || eb >= s) continue;
      const T* krow = ke + (elem_local_node(dx, dy, 0) * 2 + c) * 8;
      const T* x00 = xloc + (ea * s1 + eb) * 2;
      const T* x10 = x00 + 2 * s1;
      T part = krow[0] * x00[0] + krow[1] * x00[1];  // node (0,0)
      part += krow[2] * x10[0] + krow[3] * x10[1];   // node (1,0)
      part += krow[4] * x10[2] + krow[5] * x10[3];   // node (1,1)
      part += krow[6] * x00[2] + krow[7] * x00[3];   // node (0,1)
      acc += sc[ea * s + eb] * part;
    }
  }
  return acc;
}

template <typename T, int BP, int NS>
__global__ void __launch_bounds__(32) schur2d_kernel(DevTables t, const T* __restrict__ Ke_g,
                                                     const T* __restrict__ scale,
                                                     const T* __restrict__ factor, SchurIO io) {
  if (io.done && *io.done) return;
  schur_pcg_prologue(io);
  constexpr int PC = BP * BP, PD = BP * (BP + 1) / 2, STAGE = PC + PD, R = BP / 32;
  const int sub = blockIdx.x, lane = threadIdx.x;
  const SubInfo si = t.subs[sub];
  const int s = t.s, s1 = s + 1, nloc = s1 * s1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* stage = reinterpret_cast<T*>(smem_raw);
  T* ybuf = stage + NS * STAGE;
  T* vbuf = ybuf + t.nb_max * BP;
  T* xloc = vbuf + BP;
  T* ke = xloc + 2 * nloc;
  T* sc = ke + 64;
  uint64_t* bar = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(sc + s * s) + 15) & ~uintptr_t(15));
  const int nb = si.nb, nchunks = 2 * nb;
  const T* fbase = factor + si.factor_off;

  auto issue = [&](int c) {
    const int st = c % NS;
    T* dst = stage + st * STAGE;
    const T* src;
    uint32_t elems;
    if (c < nb) {  // forward step k = c: [C_k D_k] (k = 0: D_0 only, placed after C)
      const int k = c;
      if (k == 0) {
        src = fbase + PC;
        elems = PD;
        dst += PC;
      } else {
        src = fbase + (int64_t)k * STAGE;
        elems = STAGE;
      }
    } else {  // backward step k: [D_k C_{k+1}] (last block: D only)
      const int k = 2 * nb - 1 - c;
      src = fbase + (int64_t)k * STAGE + PC;
      elems = (k < nb - 1) ? STAGE : PD;
    }
    const uint32_t bytes = elems * (uint32_t)sizeof(T);
    mbar_expect_tx(&bar[st], bytes);
    bulk_load(dst, src, bytes, &bar[st]);
  };

  if (lane == 0) {
    for (int i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
    fence_mbar_init();
    for (int c = 0; c < NS && c < nchunks; ++c) issue(c);
  }
  for (int i = lane; i < 64; i += 32) ke[i] = Ke_g[i];
  for (int i = lane; i < s * s; i += 32)
    sc[i] = scale[(int64_t)(si.lo[0] + i / s) * t.ne[1] + si.lo[1] + i % s];
  for (int i = lane; i < 2 * nloc; i += 32) xloc[i] = T(0);
  __syncwarp();
  const bool have_x = io.x != nullptr;
  if (have_x) {
    for (int r = lane; r < si.n_ring; r += 32) {
      const int g = t.ring_gidx[si.ring_off + r];
      xloc[t.ring_loc[si.ring_off + r]] = (T)io.x[g];
    }
  }
  __syncwarp();

  bool ok = true;
  int cfail = 0;  // the chunk whose wait ran out
  // ---- forward substitution: y_k = D_k (w_k - C_k y_{k-1})
  for (int k = 0; k < nb; ++k) {
    const int st = k % NS;
    ok = __all_sync(0xffffffffu, mbar_wait(&bar[st], (k / NS) & 1));
    cfail = k;
    if (!ok) break;
    const T* Cs = stage + st * STAGE;
    const T* Ds = Cs + PC;
    T w[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int r = lane + 32 * m;
      T v = T(0);
      if (r < si.bsz) {
        const int x = si.ilo[0] + k, y = si.ilo[1] + (r >> 1), c = r & 1;
        const int64_t dof = 2 * node2(t, x, y) + c;
        if (!t.fixed[dof]) {
          if (io.f) v = (T)io.f[dof];
          if (have_x) v -= ebe_local2d<T>(ke, sc, xloc, s, x - si.lo[0], y - si.lo[1], c);
        }
      }
      w[m] = v;
    }
    if (k > 0) {
      const T* yp = ybuf + (k - 1) * BP;
#pragma unroll 8
      for (int j = 0; j < BP; ++j) {
        const T yj = yp[j];
#pragma unroll
        for (int m = 0; m < R; ++m) w[m] -= Cs[j * BP + lane + 32 * m] * yj;
      }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) vbuf[lane + 32 * m] = w[m];
    __syncwarp();
    T y[R];
#pragma unroll
    for (int m = 0; m < R; ++m) y[m] = T(0);
#pragma unroll 4
    for (int j = 0; j < BP; ++j) {
      const T vj = vbuf[j];
      const T* col = Ds + (j * BP - j * (j - 1) / 2 - j);
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int r = lane + 32 * m;
        if (r >= j) y[m] += col[r] * vj;
      }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) ybuf[k * BP + lane + 32 * m] = y[m];
    __syncwarp();
    if (lane == 0 && k + NS < nchunks) {
      fence_proxy_async_smem();
      issue(k + NS);
    }
  }
  // ---- backward substitution: t_k = D_k^T (y_k - C_{k+1}^T t_{k+1})
  for (int kk = 0; ok && kk < nb; ++kk) {
    const int k = nb - 1 - kk, c = nb + kk, st = c % NS;
    ok = __all_sync(0xffffffffu, mbar_wait(&bar[st], (c / NS) & 1));
    cfail = c;
    if (!ok) break;
    const T* Ds = stage + st * STAGE;
    const T* Cs = Ds + PD;
    T v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = ybuf[k * BP + lane + 32 * m];
    if (k + 1 < nb) {
      const T* tn = ybuf + (k + 1) * BP;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int r = lane + 32 * m;
        T acc = T(0);
#pragma unroll
        for (int h = 0; h < R; ++h)
#pragma unroll 8
          for (int rr = 0; rr < 32; ++rr) {
            const int r2 = (rr ^ lane) + 32 * h;  // bank-conflict-free transposed read
            acc += Cs[r * BP + r2] * tn[r2];
          }
        v[m] -= acc;
      }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) vbuf[lane + 32 * m] = v[m];
    __syncwarp();
    T tk[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int r = lane + 32 * m;
      const T* col = Ds + (r * BP - r * (r - 1) / 2);
      T acc = T(0);
      for (int o = 0; r + o < BP; ++o) acc += col[o] * vbuf[r + o];
      tk[m] = acc;
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < R; ++m) ybuf[k * BP + lane + 32 * m] = tk[m];
    __syncwarp();
    if (lane == 0 && c + NS < nchunks) {
      fence_proxy_async_smem();
      issue(c + NS);
    }
  }
  if (!ok) {
    // bounded wait for this CTA's copies still in flight (chunks cfail ..
    // cfail + NS - 1 were issued), then report
    if (lane == 0) {
      for (int c = cfail; c < cfail + NS && c < nchunks; ++c) mbar_wait(&bar[c % NS], (c / NS) & 1);
      if (io.err) atomicExch(io.err, kErrTimeout);
    }
    return;
  }
  // ---- outputs
  if (io.u_out || io.ring_out) {
    for (int k = 0; k < nb; ++k)
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int r = lane + 32 * m;
        if (r >= si.bsz) continue;
        const int x = si.ilo[0] + k, y = si.ilo[1] + (r >> 1), c = r & 1;
        const int64_t dof = 2 * node2(t, x, y) + c;
        if (t.fixed[dof]) continue;
        const T tv = ybuf[k * BP + r];
        if (io.u_out) io.u_out[dof] = (double)tv;
        xloc[((x - si.lo[0]) * s1 + (y - si.lo[1])) * 2 + c] = tv;
      }
    __syncwarp();
  }
  double d[1] = {0.0};
  if (io.ring_out) {
    T* out = reinterpret_cast<T*>(io.ring_out);
    for (int r = lane; r < si.n_ring; r += 32) {
      const int loc = t.ring_loc[si.ring_off + r];
      const int node = loc >> 1, c = loc & 1;
      const T y = ebe_local2d<T>(ke, sc, xloc, s, node / s1, node % s1, c);
      out[t.ring_dst[si.ring_off + r]] = y;
      d[0] += (double)xloc[loc] * (double)y;
    }
  }
  __shared__ double red[1];  // delta = (S u, u) = sum over subdomains of u_i^T S_i u_i
  schur_pcg_epilogue<1>(io, d[0], red);
}

// ============================================================ explicit local Schur
// S_i = K_GG^(i) - K_GI^(i) K_II^-1 K_IG^(i) = K_GG^(i) - W^T W with W = L^-1 K_IG^(i)
// (block forward substitution with the n_ring right-hand sides of the ring).
// One CTA of 256 threads per subdomain; the NR x NR result is accumulated in
// registers as 16 x 16 thread tiles across all block steps and stored dense
// (symmetric, so row- and column-major coincide).
template <typename T>
__device__ __forceinline__ T kig_entry2d(const DevTables& t, const SubInfo& si, const T* ke,
                                         const T* sc, int k, int r, int loc) {
  // K^(i)[interior (block k, row r)][ring DOF with local closure index loc]
  if (r >= si.bsz || loc < 0) return T(0);
  const int s = t.s, s1 = s + 1;
  const int x = si.ilo[0] + k, y = si.ilo[1] + (r >> 1), c = r & 1;
  if (t.fixed[2 * node2(t, x, y) + c]) return T(0);
  const int a = x - si.lo[0], b = y - si.lo[1];
  const int nj = loc >> 1, cj = loc & 1, aj = nj / s1, bj = nj % s1;
  if (abs(a - aj) > 1 || abs(b - bj) > 1) return T(0);
  T sum = T(0);
  for (int ea = max(a, aj) - 1; ea <= min(a, aj); ++ea) {
    if (ea < 0 || ea >= s) continue;
    for (int eb = max(b, bj) - 1; eb <= min(b, bj); ++eb) {
      if (eb < 0 || eb >= s) continue;
      const int la = elem_local_node(a - ea, b - eb, 0), lb = elem_local_node(aj - ea, bj - eb, 0);
      sum += sc[ea * s + eb] * ke[(la * 2 + c) * 8 + lb * 2 + cj];
    }
  }
  return sum;
}

template <typename T>
__device__ __forceinline__ T kgg_entry2d(int s, const T* ke, const T* sc, int li, int lj) {
  // K^(i)[ring li][ring lj], both local closure DOF indices
  if (li < 0 || lj < 0) return T(0);
  const int s1 = s + 1;
  const int ni = li >> 1, ci = li & 1, ai = ni / s1, bi = ni % s1;
  const int nj = lj >> 1, cj = lj & 1, aj = nj / s1, bj = nj % s1;
  if (abs(ai - aj) > 1 || abs(bi - bj) > 1) return T(0);
  T sum = T(0);
  for (int ea = max(ai, aj) - 1; ea <= min(ai, aj); ++ea) {
    if (ea < 0 || ea >= s) continue;
    for (int eb = max(bi, bj) - 1; eb <= min(bi, bj); ++eb) {
      if (eb < 0 || eb >= s) continue;
      const int la = elem_local_node(ai - ea, bi - eb, 0), lb = elem_local_node(aj - ea, bj - eb, 0);
      sum += sc[ea * s + eb] * ke[(la * 2 + ci) * 8 + lb * 2 + cj];
    }
  }
  return sum;
}

template <typename T, int BP, int NR>
__global__ void __launch_bounds__(256) schur_form2d_kernel(DevTables t, const T* __restrict__ Ke_g,
                                                           const T* __restrict__ scale,
                                                           const T* __restrict__ factor,
                                                           T* __restrict__ Sexp) {
  constexpr int PC = BP * BP, PD = BP * (BP + 1) / 2, STAGE = PC + PD, TL = NR / 16;
  const int sub = blockIdx.x, tid = threadIdx.x;
  const SubInfo si = t.subs[sub];
  const int s = t.s;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* Wb = reinterpret_cast<T*>(smem_raw);  // BP x NR
  T* Tb = Wb + BP * NR;                     // BP x NR
  T* Cs = Tb + BP * NR;                     // PC
  T* Ds = Cs + PC;                          // PD
  T* ke = Ds + PD;                          // 64
  T* sc = ke + 64;                          // s*s
  int* rloc = reinterpret_cast<int*>(sc + s * s);  // NR
  for (int i = tid; i < 64; i += 256) ke[i] = Ke_g[i];
  for (int i = tid; i < s * s; i += 256)
    sc[i] = scale[(int64_t)(si.lo[0] + i / s) * t.ne[1] + si.lo[1] + i % s];
  for (int j = tid; j < NR; j += 256) rloc[j] = j < si.n_ring ? t.ring_loc[si.ring_off + j] : -1;
  for (int i = tid; i < BP * NR; i += 256) Wb[i] = T(0);
  __syncthreads();
  // S is symmetric: threads 0..135 own the 136 upper tiles (ty <= tx) of the
  // 16 x 16 grid of TL x TL tiles; the other warps sit out the SYRK.
  int ty = 0, tx = 0;
  const bool owner = tid < 136;
  if (owner) {
    int q = tid;
    while (q >= 16 - ty) {
      q -= 16 - ty;
      ++ty;
    }
    tx = ty + q;
  }
  T acc[TL][TL];
#pragma unroll
  for (int a = 0; a < TL; ++a)
#pragma unroll
    for (int b = 0; b < TL; ++b)
      acc[a][b] = owner ? kgg_entry2d<T>(s, ke, sc, rloc[ty * TL + a], rloc[tx * TL + b]) : T(0);
  const T* fb = factor + si.factor_off;
  for (int k = 0; k < si.nb; ++k) {
    const T* src = fb + (int64_t)k * STAGE;
    for (int i = tid; i < STAGE; i += 256) {
      if (i < PC) {
        if (k > 0) Cs[i] = src[i];
      } else {
        Ds[i - PC] = src[i];
      }
    }
    for (int i = tid; i < BP * NR; i += 256) {
      const int r = i / NR, j = i % NR;
      Tb[i] = kig_entry2d<T>(t, si, ke, sc, k, r, rloc[j]);
    }
    __syncthreads();
    if (k > 0) {  // T = B_k - C_k W_{k-1}
      for (int i = tid; i < BP * NR; i += 256) {
        const int r = i / NR, j = i % NR;
        T v = Tb[i];
#pragma unroll 8
        for (int m = max(0, 2 * (r >> 1) - 2); m < BP; ++m) v -= Cs[m * BP + r] * Wb[m * NR + j];  // C_k's band
        Tb[i] = v;
      }
      __syncthreads();
    }
    for (int i = tid; i < BP * NR; i += 256) {  // W_k = D_k T
      const int r = i / NR, j = i % NR;
      T v = T(0);
      for (int m = 0; m <= r; ++m) v += Ds[m * BP - m * (m - 1) / 2 + (r - m)] * Tb[m * NR + j];
      Wb[i] = v;
    }
    __syncthreads();
    if (owner)
#pragma unroll 2
      for (int m = 0; m < BP; ++m) {  // S -= W_k^T W_k (upper tiles)
      T wi[TL], wj[TL];
#pragma unroll
      for (int a = 0; a < TL; ++a) {
        wi[a] = Wb[m * NR + ty * TL + a];
        wj[a] = Wb[m * NR + tx * TL + a];
      }
#pragma unroll
      for (int a = 0; a < TL; ++a)
#pragma unroll
        for (int b = 0; b < TL; ++b) acc[a][b] -= wi[a] * wj[b];
    }
    __syncthreads();
  }
  T* out = Sexp + (int64_t)sub * NR * NR;
  if (owner) {
#pragma unroll
    for (int a = 0; a < TL; ++a)
#pragma unroll
      for (int b = 0; b < TL; ++b) {
        out[(ty * TL + a) * NR + tx * TL + b] = acc[a][b];
        out[(tx * TL + b) * NR + ty * TL + a] = acc[a][b];  // mirror
      }
  }
}

// ---- double-float formation --------------------------------------------------
// schur_form2d_kernel<double> with every product and sum in double-float
// arithmetic (FP32 (hi, lo) pairs, about 48 significant bits) on the FP32
// pipes (this GPU issues 2 DFMA per clock per SM): the factor blocks and the
// K_IG, K_GG entries (computed in FP64) are split once, T, W and the S tiles
// live as pairs, S_i is stored as FP64 (hi + lo).  Serves the double-float
// PCG apply, whose operator is rounded to pairs anyway; the FP64 kernel
// serves the EXPLICIT form.
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

template <int BP, int NR>
__global__ void __launch_bounds__(256) schur_form2d_df_kernel(DevTables t, const double* __restrict__ Ke_g,
                                                              const double* __restrict__ scale,
                                                              const double* __restrict__ factor,
                                                              double* __restrict__ Sexp) {
  constexpr int PC = BP * BP, PD = BP * (BP + 1) / 2, STAGE = PC + PD, TL = NR / 16;
  const int sub = blockIdx.x, tid = threadIdx.x;
  const SubInfo si = t.subs[sub];
  const int s = t.s;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* Wb = reinterpret_cast<float2*>(smem_raw);  // BP x NR
  float2* Tb = Wb + BP * NR;                          // BP x NR
  float2* Cs = Tb + BP * NR;                          // PC
  float2* Ds = Cs + PC;                               // PD
  double* ke = reinterpret_cast<double*>(Ds + PD);    // 64
  double* sc = ke + 64;                               // s*s
  int* rloc = reinterpret_cast<int*>(sc + s * s);     // NR
  for (int i = tid; i < 64; i += 256) ke[i] = Ke_g[i];
  for (int i = tid; i < s * s; i += 256)
    sc[i] = scale[(int64_t)(si.lo[0] + i / s) * t.ne[1] + si.lo[1] + i % s];
  for (int j = tid; j < NR; j += 256) rloc[j] = j < si.n_ring ? t.ring_loc[si.ring_off + j] : -1;
  for (int i = tid; i < BP * NR; i += 256) Wb[i] = make_float2(0.f, 0.f);
  __syncthreads();
  // threads 0..135 own the 136 upper tiles (ty <= tx) of the 16 x 16 grid
  int ty = 0, tx = 0;
  const bool owner = tid < 136;
  if (owner) {
    int q = tid;
    while (q >= 16 - ty) {
      q -= 16 - ty;
      ++ty;
    }
    tx = ty + q;
  }
  float ah[TL][TL], al[TL][TL];
#pragma unroll
  for (int a = 0; a < TL; ++a)
#pragma unroll
    for (int b = 0; b < TL; ++b) {
      const float2 v = owner ? df_from(kgg_entry2d<double>(s, ke, sc, rloc[ty * TL + a], rloc[tx * TL + b]))
                             : make_float2(0.f, 0.f);
      ah[a][b] = v.x;
      al[a][b] = v.y;
    }
  const double* fb = factor + si.factor_off;
  for (int k = 0; k < si.nb; ++k) {
    const double* src = fb + (int64_t)k * STAGE;
    for (int i = tid; i < STAGE; i += 256) {
      if (i < PC) {
        if (k > 0) Cs[i] = df_neg(df_from(src[i]));  // -C_k
      } else {
        Ds[i - PC] = df_from(src[i]);
      }
    }
    for (int i = tid; i < BP * NR; i += 256) {
      const int r = i / NR, j = i % NR;
      Tb[i] = df_from(kig_entry2d<double>(t, si, ke, sc, k, r, rloc[j]));
    }
    __syncthreads();
    if (k > 0) {  // T = B_k - C_k W_{k-1}
      for (int i = tid; i < BP * NR; i += 256) {
        const int r = i / NR, j = i % NR;
        float2 v = Tb[i];
#pragma unroll 8
        for (int m = max(0, 2 * (r >> 1) - 2); m < BP; ++m)  // C_k vanishes below its band
          df_mad(v.x, v.y, Cs[m * BP + r], Wb[m * NR + j]);
        Tb[i] = v;
      }
      __syncthreads();
    }
    for (int i = tid; i < BP * NR; i += 256) {  // W_k = D_k T
      const int r = i / NR, j = i % NR;
      float h = 0.f, l = 0.f;
      for (int m = 0; m <= r; ++m) df_mad(h, l, Ds[m * BP - m * (m - 1) / 2 + (r - m)], Tb[m * NR + j]);
      Wb[i] = make_float2(h, l);
    }
    __syncthreads();
    if (owner)
#pragma unroll 2
      for (int m = 0; m < BP; ++m) {  // S -= W_k^T W_k (upper tiles)
        float2 wi[TL], wj[TL];
#pragma unroll
        for (int a = 0; a < TL; ++a) {
          wi[a] = df_neg(Wb[m * NR + ty * TL + a]);
          wj[a] = Wb[m * NR + tx * TL + a];
        }
#pragma unroll
        for (int a = 0; a < TL; ++a)
#pragma unroll
          for (int b = 0; b < TL; ++b) df_mad(ah[a][b], al[a][b], wi[a], wj[b]);
      }
    __syncthreads();
  }
  double* out = Sexp + (int64_t)sub * NR * NR;
  if (owner) {
#pragma unroll
    for (int a = 0; a < TL; ++a)
#pragma unroll
      for (int b = 0; b < TL; ++b) {
        const double v = (double)ah[a][b] + (double)al[a][b];
        out[(ty * TL + a) * NR + tx * TL + b] = v;
        out[(tx * TL + b) * NR + ty * TL + a] = v;  // mirror
      }
  }
}

// Explicit S_i for rings too wide for one CTA's registers and shared memory
// (NR = 256: up to 32 x 32-element subdomains, planes of BP = 64 or 96 rows), in two
// passes through a global scratch W (per subdomain nb_max planes of BP x NR):
//  1. form_w2d_kernel, one CTA per (subdomain, group of GC ring columns):
//     W_k = D_k (B_k - C_k W_{k-1}) with B_k the K_IG rows of plane k, the block
//     forward substitution of schur_form2d_kernel restricted to GC columns;
//  2. form_syrk2d_kernel, one CTA per (subdomain, TQ x TQ tile (qa <= qb)):
//     S tile = K_GG tile - sum_k W_k[:, qa]^T W_k[:, qb], mirrored below the
//     diagonal.
template <typename T, int BP, int NR, int GC>
__global__ void __launch_bounds__(256) form_w2d_kernel(DevTables t, const T* __restrict__ Ke_g,
                                                       const T* __restrict__ scale,
                                                       const T* __restrict__ factor, T* __restrict__ W) {
  constexpr int PC = BP * BP, PD = BP * (BP + 1) / 2, STAGE = PC + PD;
  const int sub = blockIdx.x, g = blockIdx.y, tid = threadIdx.x;
  const SubInfo si = t.subs[sub];
  const int s = t.s;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* Cs = reinterpret_cast<T*>(smem_raw);  // PC
  T* Ds = Cs + PC;                          // PD
  T* Wp = Ds + PD;                          // BP x GC: W_{k-1}, then W_k
  T* Tb = Wp + BP * GC;                     // BP x GC
  T* ke = Tb + BP * GC;                     // 64
  T* sc = ke + 64;                          // s*s
  int* rloc = reinterpret_cast<int*>(sc + s * s);  // GC
  for (int i = tid; i < 64; i += 256) ke[i] = Ke_g[i];
  for (int i = tid; i < s * s; i += 256)
    sc[i] = scale[(int64_t)(si.lo[0] + i / s) * t.ne[1] + si.lo[1] + i % s];
  for (int j = tid; j < GC; j += 256) {
    const int jr = g * GC + j;
    rloc[j] = jr < si.n_ring ? t.ring_loc[si.ring_off + jr] : -1;
  }
  for (int i = tid; i < BP * GC; i += 256) Wp[i] = T(0);
  __syncthreads();
  const T* fb = factor + si.factor_off;
  T* Wout = W + (int64_t)sub * t.nb_max * BP * NR;
  for (int k = 0; k < si.nb; ++k) {
    const T* src = fb + (int64_t)k * STAGE;
    for (int i = tid; i < STAGE; i += 256) {
      if (i < PC) {
        if (k > 0) Cs[i] = src[i];
      } else {
        Ds[i - PC] = src[i];
      }
    }
    for (int i = tid; i < BP * GC; i += 256) Tb[i] = kig_entry2d<T>(t, si, ke, sc, k, i / GC, rloc[i % GC]);
    __syncthreads();
    if (k > 0) {  // T = B_k - C_k W_{k-1}
      // C_k(r, m) vanishes below the lowest column row r couples to in plane
      // k - 1, 2 (r / 2) - 2: the products start there (a warp shares r)
      for (int i = tid; i < BP * GC; i += 256) {
        const int r = i / GC, j = i % GC;
        T v = Tb[i];
#pragma unroll 8
        for (int m = max(0, 2 * (r >> 1) - 2); m < BP; ++m) v -= Cs[m * BP + r] * Wp[m * GC + j];
        Tb[i] = v;
      }
      __syncthreads();
    }
    for (int i = tid; i < BP * GC; i += 256) {  // W_k = D_k T
      const int r = i / GC, j = i % GC;
      T v = T(0);
      for (int m = 0; m <= r; ++m) v += Ds[m * BP - m * (m - 1) / 2 + (r - m)] * Tb[m * GC + j];
      Wp[i] = v;
      Wout[((int64_t)k * BP + r) * NR + g * GC + j] = v;
    }
    __syncthreads();
  }
}

template <typename T, int BP, int NR, int TQ>
__global__ void __launch_bounds__(256) form_syrk2d_kernel(DevTables t, const T* __restrict__ Ke_g,
                                                          const T* __restrict__ scale,
                                                          const T* __restrict__ W, T* __restrict__ Sexp) {
  constexpr int NQ = NR / TQ, TA = TQ / 16;
  const int sub = blockIdx.x, tid = threadIdx.x;
  int qa = 0, q = blockIdx.y;  // tile index -> (qa, qb), qa <= qb
  while (q >= NQ - qa) {
    q -= NQ - qa;
    ++qa;
  }
  const int qb = qa + q;
  const SubInfo si = t.subs[sub];
  const int s = t.s;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* Wa = reinterpret_cast<T*>(smem_raw);  // BP x TQ
  T* Wb = Wa + BP * TQ;                     // BP x TQ
  T* ke = Wb + BP * TQ;                     // 64
  T* sc = ke + 64;                          // s*s
  int* rl = reinterpret_cast<int*>(sc + s * s);  // 2 TQ: ring rows of qa, then of qb
  for (int i = tid; i < 64; i += 256) ke[i] = Ke_g[i];
  for (int i = tid; i < s * s; i += 256)
    sc[i] = scale[(int64_t)(si.lo[0] + i / s) * t.ne[1] + si.lo[1] + i % s];
  for (int j = tid; j < 2 * TQ; j += 256) {
    const int jr = (j < TQ ? qa : qb) * TQ + j % TQ;
    rl[j] = jr < si.n_ring ? t.ring_loc[si.ring_off + jr] : -1;
  }
  __syncthreads();
  // thread (ty, tx) owns rows ty + 16 a of block qa and columns tx + 16 b of qb
  const int ty = tid / 16, tx = tid % 16;
  T acc[TA][TA];
#pragma unroll
  for (int a = 0; a < TA; ++a)
#pragma unroll
    for (int b = 0; b < TA; ++b) acc[a][b] = kgg_entry2d<T>(s, ke, sc, rl[ty + 16 * a], rl[TQ + tx + 16 * b]);
  const T* Win = W + (int64_t)sub * t.nb_max * BP * NR;
  for (int k = 0; k < si.nb; ++k) {
    for (int i = tid; i < BP * TQ; i += 256) {
      const int m = i / TQ, j = i % TQ;
      const T* row = Win + ((int64_t)k * BP + m) * NR;
      Wa[i] = row[qa * TQ + j];
      Wb[i] = row[qb * TQ + j];
    }
    __syncthreads();
#pragma unroll 4
    for (int m = 0; m < BP; ++m) {
      T wi[TA], wj[TA];
#pragma unroll
      for (int a = 0; a < TA; ++a) {
        wi[a] = Wa[m * TQ + ty + 16 * a];
        wj[a] = Wb[m * TQ + tx + 16 * a];
      }
#pragma unroll
      for (int a = 0; a < TA; ++a)
#pragma unroll
        for (int b = 0; b < TA; ++b) acc[a][b] -= wi[a] * wj[b];
    }
    __syncthreads();
  }
  T* out = Sexp + (int64_t)sub * NR * NR;
#pragma unroll
  for (int a = 0; a < TA; ++a)
#pragma unroll
    for (int b = 0; b < TA; ++b) {
      const int i = qa * TQ + ty + 16 * a, j = qb * TQ + tx + 16 * b;
      out[(int64_t)i * NR + j] = acc[a][b];
      if (qa != qb) out[(int64_t)j * NR + i] = acc[a][b];
    }
}

#include "ddel_ozaki.cuh"

// Tile policy of the 2D formation: S_i = K_GG - W^T W, K_GG by element
// entries of the ring, the result into the dense NR x NR S_i (FP64 or FP32).
template <int NR, typename TO>
struct FormTile {
  const double* Ke;
  const double* scale;
  TO* Sexp;
  static size_t smem(const DevTables& t) { return (64 + (size_t)t.s * t.s) * 8 + 2 * kOzTile * 4; }
  __device__ int rows(const DevTables& t, const SubInfo& si) const { return si.nb * t.BP; }
  __device__ void setup(const DevTables& t, const SubInfo& si, int ta, int tb, unsigned char* sm) const {
    double* ke = reinterpret_cast<double*>(sm);
    double* sc = ke + 64;
    int* rl = reinterpret_cast<int*>(sc + t.s * t.s);
    const int s = t.s;
    for (int i = threadIdx.x; i < 64; i += blockDim.x) ke[i] = Ke[i];
    for (int i = threadIdx.x; i < s * s; i += blockDim.x)
      sc[i] = scale[(int64_t)(si.lo[0] + i / s) * t.ne[1] + si.lo[1] + i % s];
    for (int j = threadIdx.x; j < 2 * kOzTile; j += blockDim.x) {
      const int jr = (j < kOzTile ? ta : tb) * kOzTile + j % kOzTile;
      rl[j] = jr < si.n_ring ? t.ring_loc[si.ring_off + jr] : -1;
    }
  }
  __device__ double value(const DevTables& t, const SubInfo&, const unsigned char* sm, int, int, int li,
                          int lj) const {
    const double* ke = reinterpret_cast<const double*>(sm);
    const double* sc = ke + 64;
    const int* rl = reinterpret_cast<const int*>(sc + t.s * t.s);
    return kgg_entry2d<double>(t.s, ke, sc, rl[li], rl[kOzTile + lj]);
  }
  __device__ void store(const DevTables&, const SubInfo&, int sub, int gi, int gj, double v) const {
    Sexp[(int64_t)sub * NR * NR + (int64_t)gi * NR + gj] = (TO)v;
  }
};

// y_ring = S_i x_ring for every subdomain.
template <typename T, int NR>
__global__ void __launch_bounds__(256) schur_explicit_kernel(DevTables t, const T* __restrict__ Sexp,
                                                             SchurIO io) {
  if (io.done && *io.done) return;
  // two CTAs per subdomain (rows [half * RH, half * RH + RH)), H column groups
  // per row: 2 * n_sub CTAs balance the SMs better than one CTA per subdomain
  constexpr int RH = NR / 2, H = 256 / RH;
  const int sub = blockIdx.x >> 1, half = blockIdx.x & 1, tid = threadIdx.x;
  const SubInfo si = t.subs[sub];
  __shared__ T xr[NR];
  __shared__ T part[256];
  __shared__ double red[RH / 32];
  schur_pcg_prologue(io);
  for (int j = tid; j < NR; j += 256) {
    T v = T(0);
    if (j < si.n_ring) v = (T)io.x[t.ring_gidx[si.ring_off + j]];
    xr[j] = v;
  }
  __syncthreads();
  const int r = half * RH + tid % RH, h = tid / RH;
  const T* Sc = Sexp + (int64_t)sub * NR * NR;
  T acc0 = T(0), acc1 = T(0);
  const int j0 = h * (NR / H), j1 = j0 + NR / H;
#pragma unroll 4
  for (int j = j0; j < j1; j += 2) {
    acc0 += Sc[j * NR + r] * xr[j];
    acc1 += Sc[(j + 1) * NR + r] * xr[j + 1];
  }
  part[tid] = acc0 + acc1;
  __syncthreads();
  double d[1] = {0.0};
  const int row = half * RH + tid;
  if (tid < RH && row < si.n_ring) {
    T y = T(0);
#pragma unroll
    for (int q = 0; q < H; ++q) y += part[q * RH + tid];
    reinterpret_cast<T*>(io.ring_out)[t.ring_dst[si.ring_off + row]] = y;
    d[0] = (double)xr[row] * (double)y;
  }
  schur_pcg_epilogue<RH / 32>(io, d[0], red);  // delta: rows of this CTA
}

// Native FP64 form of the explicit apply, laid out like the double-float one:
// each thread owns two adjacent rows and JN columns, reading both rows' entries
// of a column as one 16-byte load (S_i column-major FP64), with one
// accumulator per row; the H column groups of a row are added in group order.
// GB300 issues two DFMA per clock per SM, so this product is bound by the FP64
// pipe (2 n_ring^2 flop per subdomain) rather than by the bytes it streams.
// SPLIT CTAs share a subdomain, NR / SPLIT rows each (the tile shape the
// autotuner chooses: fewer, longer column groups with SPLIT = 1, more CTAs
// with SPLIT = 4).
template <int NR, int SPLIT>
__global__ void __launch_bounds__(256, NR <= 128 ? 7 : 5) schur_explicit_f64_kernel(DevTables t,
                                                                                   const double* __restrict__ Sexp,
                                                                                   SchurIO io) {
  const int done = io.done ? *io.done : 0;
  constexpr int RH = NR / SPLIT, RP = RH / 2, H = 256 / RP, JN = NR / H;
  static_assert(RH >= 32 && RP <= 256 && H * RP == 256 && H * JN == NR, "tile shape");
  const int sub = blockIdx.x / SPLIT, half = blockIdx.x % SPLIT, tid = threadIdx.x;
  const SubInfo si = t.subs[sub];
  __shared__ double xr[NR];
  __shared__ double part[2 * 256];
  __shared__ double red[RH / 32];
  for (int j = tid; j < NR; j += 256) {
    double v = 0.0;
    if (j < si.n_ring) v = io.x[t.ring_gidx[si.ring_off + j]];
    xr[j] = v;
  }
  if (done) return;  // uniform over the grid: converged in an earlier iteration
  schur_pcg_prologue(io);
  __syncthreads();
  const int rp = tid % RP, h = tid / RP;
  const int r0 = half * RH + 2 * rp;
  const double2* Sc = reinterpret_cast<const double2*>(Sexp + (int64_t)sub * NR * NR);
  // one accumulator per row: with dozens of warps sharing an SM's FP64 pipe a
  // warp's FMAs are issued far enough apart to need no second chain, and the
  // extra additions would cost pipe cycles.  Column groups wholly beyond the
  // ring (zero padding of subdomains at the domain boundary) are skipped.
  double a0 = 0.0, a1 = 0.0;
  if (h * JN < si.n_ring) {
#pragma unroll 16
    for (int q = 0; q < JN; ++q) {
      const int j = h * JN + q;
      const double2 s0 = Sc[(j * NR + r0) >> 1];
      const double x0 = xr[j];
      a0 = fma(s0.x, x0, a0);
      a1 = fma(s0.y, x0, a1);
    }
  }
  part[2 * tid] = a0;
  part[2 * tid + 1] = a1;
  __syncthreads();
  double d[1] = {0.0};
  const int row = half * RH + tid;
  if (tid < RH && row < si.n_ring) {
    double y = 0.0;
#pragma unroll
    for (int q = 0; q < H; ++q) y += part[2 * (q * RP + (tid >> 1)) + (tid & 1)];
    reinterpret_cast<double*>(io.ring_out)[t.ring_dst[si.ring_off + row]] = y;
    d[0] = xr[row] * y;
  }
  schur_pcg_epilogue<RH / 32>(io, d[0], red);
}

// ---- double-float form of the explicit apply --------------------------------
// S_i is stored as pairs (hi, lo) of FP32 with hi + lo = S to 2^-48 relative,
// the ring vector likewise, and each row sum is accumulated as a pair with the
// error-free transformations of df_mad / df_add2, so the arithmetic runs on
// the FP32 pipes (GB300: 128 lanes/clk/SM) instead of the FP64 pipe
// (2 DFMA/clk/SM) while keeping about 48 significant bits.

__global__ void split_df_kernel(const double* __restrict__ in, float2* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = in[i];
    const float hi = (float)v;
    out[i] = make_float2(hi, (float)(v - (double)hi));
  }
}


// One CTA per half of a subdomain's rows; each thread owns two adjacent rows
// and JN columns, loading both rows' entries of a column as one 16-byte
// float4 (S_i stored column-major as (hi, lo) pairs); the H column groups of a
// row are combined in double-float as well, so FP64 work is left to the
// final row values.  Up to 128 ring rows, registers are capped so that 7 CTAs
// fit an SM: the 1024 CTAs of 512 subdomains then run in one wave (rings of
// 256: 6 CTAs, 40 registers; more registers made that form slower).
// The body as a device function of the block index bid: the kernel below,
// and the batched persistent kernel, which runs it for other problems'
// blocks within one launch (CG: the vectors written earlier in that launch
// by other blocks are read through L2, bypassing the non-coherent L1).
template <int NR, bool CG, int SPLIT = 2>
__device__ __forceinline__ void schur_df_tile(const DevTables& t, const float2* __restrict__ Sexp, const SchurIO& io,
                                              int bid) {
  // the flag's load overlaps the gather; nothing is written before the test
  const int done = io.done ? (CG ? __ldcg(io.done) : *io.done) : 0;
  constexpr int RH = NR / SPLIT, RP = RH / 2, H = 256 / RP, JN = NR / H;
  static_assert(RH >= 32 && RP <= 256 && H * RP == 256 && H * JN == NR, "tile shape");
  const int sub = bid / SPLIT, half = bid % SPLIT, tid = threadIdx.x;
  const SubInfo si = t.subs[sub];
  __shared__ float2 xr[NR];
  __shared__ double xd[NR];
  __shared__ float2 part[2 * 256];
  __shared__ double red[RH / 32];
  for (int j = tid; j < NR; j += 256) {
    double v = 0.0;
    if (j < si.n_ring) {
      const double* xp = io.x + t.ring_gidx[si.ring_off + j];
      v = CG ? __ldcg(xp) : *xp;
    }
    const float hi = (float)v;
    xr[j] = make_float2(hi, (float)(v - (double)hi));
    xd[j] = v;
  }
  if (done) return;  // uniform over the grid: converged in an earlier iteration
  schur_pcg_prologue(io, bid);
  __syncthreads();
  const int rp = tid % RP, h = tid / RP;
  const int r0 = half * RH + 2 * rp;
  const float4* Sc = reinterpret_cast<const float4*>(Sexp + (int64_t)sub * NR * NR);
  float hi0 = 0.f, lo0 = 0.f, hi1 = 0.f, lo1 = 0.f;
  auto term = [](float& hi, float& lo, float sx, float sy, float2 x) {
    const float p = __fmul_rn(sx, x.x);
    // low-order part: product error (exact via FMA) and the hi*lo cross terms
    lo = __fadd_rn(lo, __fadd_rn(__fmaf_rn(sx, x.x, -p), __fmaf_rn(sx, x.y, __fmul_rn(sy, x.x))));
    df_add(hi, lo, p);
  };
#pragma unroll 8
  for (int q = 0; q < JN; ++q) {
    const int j = h * JN + q;
    const float4 sv4 = Sc[(j * NR + r0) >> 1];
    const float2 x = xr[j];
    term(hi0, lo0, sv4.x, sv4.y, x);
    term(hi1, lo1, sv4.z, sv4.w, x);
  }
  part[2 * tid] = make_float2(hi0, lo0);
  part[2 * tid + 1] = make_float2(hi1, lo1);
  __syncthreads();
  double d[1] = {0.0};
  const int row = half * RH + tid;
  if (tid < RH && row < si.n_ring) {
    float yh = 0.f, yl = 0.f;
#pragma unroll
    for (int q = 0; q < H; ++q) {
      const float2 pq = part[2 * (q * RP + (tid >> 1)) + (tid & 1)];
      df_add2(yh, yl, pq.x, pq.y);
    }
    const double y = (double)yh + (double)yl;
    reinterpret_cast<double*>(io.ring_out)[t.ring_dst[si.ring_off + row]] = y;
    d[0] = xd[row] * y;
  }
  schur_pcg_epilogue<RH / 32>(io, d[0], red, bid);
}

// SPLIT CTAs per subdomain (NR / SPLIT rows each; the persistent batch uses 2).
template <int NR, int SPLIT>
__global__ void __launch_bounds__(256, NR <= 128 ? 7 : 6) schur_explicit_df_kernel(DevTables t, const float2* __restrict__ Sexp,
                                                                SchurIO io) {
  schur_df_tile<NR, false, SPLIT>(t, Sexp, io, blockIdx.x);
}

// ============================================================ Gamma sums
// Sum of the owners' contributions to Gamma DOF g, in owner (subdomain) order;
// the owner-major layout makes them one contiguous, aligned vector load.
template <typename T, bool CG = false>
__device__ __forceinline__ double ring_sum(const DevTables& t, const T* __restrict__ ring, int64_t g) {
  if (t.max_owners == 4) {
    if constexpr (sizeof(T) == 8) {
      const double2* q = reinterpret_cast<const double2*>(ring) + 2 * g;
      const double2 a = CG ? __ldcg(q) : q[0];
      const double2 b = CG ? __ldcg(q + 1) : q[1];
      return ((a.x + a.y) + b.x) + b.y;
    } else {
      const float4* q = reinterpret_cast<const float4*>(ring) + g;
      const float4 v = CG ? __ldcg(q) : q[0];
      return (((double)v.x + (double)v.y) + (double)v.z) + (double)v.w;
    }
  }
  double acc = 0.0;
  for (int k = 0; k < t.max_owners; ++k) {
    const T* q = ring + g * t.max_owners + k;
    acc += (double)(CG ? __ldcg(q) : *q);
  }
  return acc;
}

template <typename T>
__global__ void gamma_sum_kernel(DevTables t, const T* __restrict__ ring,
                                 const double* __restrict__ base, double sign,
                                 double* __restrict__ out) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < t.n_gamma;
       g += (int64_t)gridDim.x * blockDim.x)
    out[g] = (base ? base[t.gamma_dof[g]] : 0.0) + sign * ring_sum<T>(t, ring, g);
}

// ============================================================ PCG
// Face blocks: one warp per (face, component) block, z = W^-1 P W^-1 r with P
// symmetric, read by columns (coalesced); cross points: one thread per DOF.
// INIT: x = x0, r = g - S x0, p = s = 0 (x0 = 0 without a coarse space).
// Update j: every block first reduces the partials of the Schur apply
// (delta_j) and of update j-1 (gamma_j, rr_j, coarse sums), tests
// convergence, and forms alpha_j, beta_j itself (the same bits in every
// block); then w_g = sum of the ring entries of the owning subdomains,
// p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s.
// Both: u^ = S~^-1 r and the block's partials of gamma^ = (r, u^), rr = (r, r).
// Coarse space (KC > 0, k <= KC columns): u = u^ + Q cc with cc = E^-1 Q^T r
// (additive correction) or cc = E^-1 (Q^T r - (S Q)^T u^) (deflation,
// u = Q E^-1 Q^T r + (I - Q E^-1 Q^T S) u^).  The array u and the Schur
// kernels see only u^; the update adds Q cc to u and S Q cc to w = S u^, and
// forms gamma = gamma^ + (Q^T r)^T cc and delta = (S u, u) = delta^ +
// 2 cc^T (S Q)^T u^ + cc^T E cc from the partial sums of Q^T r and (S Q)^T u^.
// REPL (with INIT, no coarse space): the reliable update of the relaxed
// mixed-precision PCG -- r = g - (S x from the ring of an accurate apply of
// the current x), x, p and s kept, u = S~^-1 r with the partials of gamma and
// rr, and two more rows: (u, s) and (p, s) for the corrected step length
// (pcg_replace_fix_kernel).
template <typename T, bool INIT, int KC, bool REPL = false>
__global__ void __launch_bounds__(kRedThreads) pcg_cg_kernel(DevTables t, DevFields fld,
                                                             const double* __restrict__ gin,
                                                             const T* __restrict__ ring, double* x,
                                                             double* r, double* u, double* p,
                                                             double* sv, PcgState* st, CoarseDev cd,
                                                             const double* __restrict__ pd, int nd,
                                                             const double* __restrict__ pu_in,
                                                             double* __restrict__ pu_out, int par) {
  static_assert(!REPL || (INIT && KC == 0), "the replacement runs without a coarse space");
  const int done = st->done;  // tested once the prologue's loads are in flight
  constexpr int NV = 2 + 2 * KC + (REPL ? 2 : 0), NP = 3 + 2 * KC + (REPL ? 1 : 0);
  extern __shared__ double rw_all[];  // (blockDim/32) * max_blk_n doubles, then as many float2
  __shared__ double red[NP * kRedThreads];  // tree sums (prologue NP values, epilogue NV)
  __shared__ double sums[NP];               // delta^, gamma^, rr, Q^T r, (S Q)^T u^
  __shared__ double sab[2 + kMaxCoarse];    // alpha, beta, cc
  __shared__ int sflag;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* rw = rw_all + wib * t.max_blk_n;
  float2* rwf = reinterpret_cast<float2*>(rw_all + (blockDim.x >> 5) * t.max_blk_n) + wib * t.max_blk_n;
  const int k = KC > 0 ? cd.k : 0;  // coarse columns
  const bool deflate = KC > 0 && cd.correct == 2;
  const int j = INIT ? -1 : st->kU;
  double alpha = 0.0, beta = 0.0;
  double cc[KC > 0 ? KC : 1];  // INIT: x0 coefficients; else coarse coefficients of u_j
  if (!INIT) {
    // E^-1 and E staged in shared memory by all threads at once (thread 0's
    // scalar phase below would otherwise wait on a chain of global loads)
    __shared__ double sEinv[KC > 0 ? KC * KC : 1], sE[KC > 0 ? KC * KC : 1];
    constexpr int KD = KC > 0 ? KC : 1;  // divisor (no coarse rows when KC = 0)
    for (int i = threadIdx.x; i < KC * KC; i += blockDim.x) {
      const int a = i / KD, b = i % KD;
      if (a < k && b < k) {
        sEinv[i] = cd.Einv[a * kMaxCoarse + b];
        sE[i] = 0.5 * (cd.E[a * kMaxCoarse + b] + cd.E[b * kMaxCoarse + a]);
      }
    }
    // scalars of thread 0 loaded first, so that their latency overlaps the sums
    double tol2 = 0.0, ginv = 0.0, ainv = 0.0;
    int max_it = 0;
    if (threadIdx.x == 0) {
      tol2 = st->tol2;
      max_it = st->max_it;
      ginv = st->ginv_s[par ^ 1];
      ainv = st->ainv_s[par ^ 1];
    }
    // every thread loads its strided share of all partial vectors at once
    // (independent loads in flight), then one tree sum per value
    const double* U = pu_in;
    const int nu = gridDim.x;
    double a[NP];
#pragma unroll
    for (int v = 0; v < NP; ++v) {
      a[v] = 0.0;
      if (v >= 3 && (v - 3) % (KC > 0 ? KC : 1) >= k) continue;  // coarse rows beyond k
      const double* src = v == 0 ? pd : U + (size_t)(v - 1) * nu;
      const int n = v == 0 ? nd : nu;
      for (int b = threadIdx.x; b < n; b += kRedThreads) a[v] += __ldcg(src + b);
    }
    if (done) return;  // uniform over the grid
    block_tree_sum<NP>(a, NP, red);
    if (threadIdx.x < NP) sums[threadIdx.x] = red[threadIdx.x * kRedThreads];
    __syncthreads();
    if (threadIdx.x == 0) {
      double gamma = sums[1], delta = sums[0];
      const double rr = sums[2];
      const double* y = sums + 3;       // Q^T r_j
      const double* vq = sums + 3 + KC;  // (S Q)^T u^_j
      for (int i = 0; i < k; ++i) {
        double c = 0.0;
        for (int q = 0; q < k; ++q) c += sEinv[i * KC + q] * (y[q] - (deflate ? vq[q] : 0.0));
        sab[2 + i] = c;
      }
      for (int i = 0; i < k; ++i) {
        const double ci = sab[2 + i];
        gamma += y[i] * ci;
        double ec = 0.0;
        for (int q = 0; q < k; ++q) ec += sE[i * KC + q] * sab[2 + q];
        delta += ci * (2.0 * vq[i] + ec);
      }
      int status = 1;  // 1: iterate
      double a_ = 0.0, b_ = 0.0, den = delta;  // den = p^T S p (Chronopoulos-Gear)
      const double gi = 1.0 / gamma;          // independent of the division below
      if (rr <= tol2) {
        status = 0;
      } else if (!isfinite(rr) || !isfinite(gamma)) {
        status = -6;
      } else if (j >= max_it) {
        status = -5;
      } else {
        if (j > 0) {
          b_ = gamma * ginv;  // gamma_j / gamma_{j-1}
          den = delta - b_ * gamma * ainv;
        }
        if (!(den > 0.0) || !isfinite(den)) status = -6;  // breakdown
        else a_ = gamma / den;
      }
      sab[0] = a_;
      sab[1] = b_;
      sflag = status;
      if (blockIdx.x == 0) {
        st->rr = rr;
        st->it = j;
        if (status != 1) {
          st->done = 1;
          st->status = status;
        } else {
          st->ainv_s[par] = den * gi;  // 1 / alpha_j = den / gamma_j
          st->ginv_s[par] = gi;
          st->kS = j + 1;
        }
      }
    }
    __syncthreads();
    if (sflag != 1) return;
    alpha = sab[0];
    beta = sab[1];
#pragma unroll
    for (int i = 0; i < KC; ++i) cc[i] = i < k ? sab[2 + i] : 0.0;
  } else {
    if (done) return;
#pragma unroll
    for (int i = 0; i < KC; ++i) cc[i] = (i < k && cd.x0) ? st->c0[i] : 0.0;
    if (!REPL && blockIdx.x == 0 && threadIdx.x == 0) st->kS = 0;
  }
  auto coarse = [&](const double* V, int64_t g) -> double {
    double v = 0.0;
#pragma unroll
    for (int i = 0; i < KC; ++i)
      if (i < k) v += V[i * t.n_gamma + g] * cc[i];
    return v;
  };
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0.0;
  auto step = [&](int64_t g) -> double {
    double rg;
    if constexpr (REPL) {
      rg = gin[g] - ring_sum<T>(t, ring, g);
    } else if (INIT) {
      p[g] = 0.0;
      sv[g] = 0.0;
      if (KC > 0) {
        x[g] = coarse(cd.Q, g);
        rg = gin[g] - coarse(cd.SQ, g);
      } else {
        x[g] = 0.0;
        rg = gin[g];
      }
    } else {
      // S u at this DOF: the ring entries of its owners (fixed-width table,
      // subdomain order, so the sum order is fixed), plus S Q cc
      const double w = ring_sum<T>(t, ring, g) + (KC > 0 ? coarse(cd.SQ, g) : 0.0);
      const double pg = u[g] + (KC > 0 ? coarse(cd.Q, g) : 0.0) + beta * p[g];
      const double sg = w + beta * sv[g];
      p[g] = pg;
      sv[g] = sg;
      x[g] += alpha * pg;
      rg = r[g] - alpha * sg;
    }
    r[g] = rg;
    acc[1] += rg * rg;
#pragma unroll
    for (int i = 0; i < KC; ++i)
      if (i < k) acc[2 + i] += cd.Q[i * t.n_gamma + g] * rg;
    return rg;
  };
  auto local = [&](int64_t g, double ri, double ui) {  // u^ at g: store and sum
    u[g] = ui;
    acc[0] += ri * ui;
#pragma unroll
    for (int i = 0; i < KC; ++i)
      if (i < k) acc[2 + KC + i] += cd.SQ[i * t.n_gamma + g] * ui;
    if constexpr (REPL) {
      const double sg = sv[g];
      acc[NV - 2] += ui * sg;
      acc[NV - 1] += p[g] * sg;
    }
  };
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int b = gw; b < t.n_blocks; b += nw) {
    const int off = t.blk_off[b], n = t.blk_n[b];
    for (int i = lane; i < n; i += 32) {
      const double ri = step(off + i);
      const double v = ri * fld.face_w[off + i];  // W^-1 r (face_w holds 1 / W_ii)
      rw[i] = v;
      const float hi = (float)v;
      rwf[i] = make_float2(hi, (float)(v - (double)hi));
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      // column i of the symmetric P in double-float arithmetic on the FP32
      // pipes (about 48 significant bits; this GPU issues 2 DFMA per clock per
      // SM), the same error-free transformations as the explicit Schur apply
      const float2* Pc = t.ptab_df + t.blk_poff[b] + i;
      float hi = 0.f, lo = 0.f;
#pragma unroll 4
      for (int q = 0; q < n; ++q) {
        const float2 s = Pc[q * n], xq = rwf[q];
        const float pr = __fmul_rn(s.x, xq.x);
        lo = __fadd_rn(lo, __fadd_rn(__fmaf_rn(s.x, xq.x, -pr), __fmaf_rn(s.x, xq.y, __fmul_rn(s.y, xq.x))));
        df_add(hi, lo, pr);
      }
      const double zi = (double)hi + (double)lo;
      // u^_i = W^-1 zi; r_i (this thread wrote it in the first loop)
      local(off + i, r[off + i], zi * fld.face_w[off + i]);
    }
    __syncwarp();
  }
  for (int64_t g = t.n_face_dofs + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < t.n_gamma;
       g += (int64_t)gridDim.x * blockDim.x) {
    const double ri = step(g);
    local(g, ri, ri * fld.cross_scale[g - t.n_face_dofs]);
  }
  // this block's partials of iteration j + 1 (gamma^, rr, Q^T r, (S Q)^T u^)
  block_tree_sum<NV>(acc, NV, red);
  if (threadIdx.x < NV) pu_out[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = red[threadIdx.x * kRedThreads];
}

// Update j of the PCG (the non-INIT form of pcg_cg_kernel: the same
// arithmetic on every interface DOF, so the iterates agree with that kernel's
// to rounding of the grid-wide sums) laid out for latency:
//  * face blocks are packed UL lanes apiece (UL = the power of two >= the
//    largest block, at most 32), so a warp serves 32 / UL blocks at once;
//  * before the partial sums are reduced, every lane issues the loads that
//    need no scalar -- for its DOFs of its first face block and its first
//    cross-point DOF: the owners' ring entries of S u, u, p, s, x, r and the
//    face weight -- and, where it fits, the face block's dense H~^-1 table is
//    copied into shared memory (cp.async), so that their latency overlaps the
//    reduction's;
//  * without a coarse space the three grid-wide sums (delta, gamma, rr) are
//    reduced by one warp each (lane-strided loads, then a shuffle tree; every
//    block forms bitwise the same totals) instead of a block-wide tree.
// Further blocks of a warp (more face blocks than lanes) load as they come.
// The body as a device function of the block index bid of nblk blocks: the
// kernel below, and the batched persistent kernel (CG: values written earlier
// in that launch by other blocks are read through L2; the convergence flag,
// which block 0 of the same iteration may be setting meanwhile, is read once
// per block and shared, so that every thread of a block takes the same path).
template <typename T, int KC, bool CG>
__device__ __forceinline__ void pcg_update_tile(const DevTables& t, const DevFields& fld, const T* __restrict__ ring,
                                                double* x, double* r, double* u, double* p, double* sv, PcgState* st,
                                                const CoarseDev& cd, const double* __restrict__ pd, int nd,
                                                const double* __restrict__ pu_in, double* __restrict__ pu_out,
                                                int par, int bid, int nblk) {
  __shared__ int s_done;
  int done = 0;
  if constexpr (CG) {
    if (threadIdx.x == 0) s_done = __ldcg(&st->done);
  } else {
    done = st->done;
  }
  auto ld = [](const double* q) -> double { return CG ? __ldcg(q) : *q; };
  constexpr int NV = 2 + 2 * KC, NP = 3 + 2 * KC, PE = 2;
  // dynamic shared memory: per warp UG * max_blk_n doubles (W^-1 r), as many
  // float2 (its double-float split), then, when staged, UG * max_blk_n^2
  // float2 per warp (the face tables)
  extern __shared__ double rw_all[];
  __shared__ double red[NP * kRedThreads];
  __shared__ double sums[NP];
  __shared__ double sab[2 + kMaxCoarse];
  __shared__ int sflag;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  const int UL = t.upd_lanes, UG = 32 / UL, mbn = t.max_blk_n;
  const int grp = lane / UL, gl = lane % UL;
  double* rw = rw_all + (wib * UG + grp) * mbn;
  float2* rwf = reinterpret_cast<float2*>(rw_all + nwb * UG * mbn) + (wib * UG + grp) * mbn;
  float2* ptile = reinterpret_cast<float2*>(rw_all + 2 * nwb * UG * mbn) + (size_t)(wib * UG + grp) * mbn * mbn;
  const int k = KC > 0 ? cd.k : 0;
  const bool deflate = KC > 0 && cd.correct == 2;
  const int j = CG ? __ldcg(&st->kU) : st->kU;
  const int gw = (bid * blockDim.x + threadIdx.x) >> 5;
  const int nw = (nblk * blockDim.x) >> 5;
  struct Dof {
    double w, u, p, s, x, r, fw;
  };
  auto load_dof = [&](int64_t g, double fw) -> Dof {
    Dof d;
    d.w = ring_sum<T, CG>(t, ring, g);
    d.u = ld(u + g);
    d.p = ld(p + g);
    d.s = ld(sv + g);
    d.x = ld(x + g);
    d.r = ld(r + g);
    d.fw = fw;
    return d;
  };
  // --- loads that need no scalar, issued first
  const int b0 = gw * UG + grp;
  int off0 = 0, n0 = 0, poff0 = 0;
  if (b0 < t.n_blocks) {
    off0 = t.blk_off[b0];
    n0 = t.blk_n[b0];
    poff0 = t.blk_poff[b0];
  }
  const bool pre_ok = n0 <= UL * PE;
  Dof pre[PE];
#pragma unroll
  for (int e = 0; e < PE; ++e) {
    const int i = gl + UL * e;
    if (pre_ok && i < n0) pre[e] = load_dof(off0 + i, fld.face_w[off0 + i]);
  }
  if (t.upd_stage_p && n0 > 0) {
    const float2* src = t.ptab_df + poff0;
    for (int i = gl; i < n0 * n0; i += UL) cp_async8(ptile + i, src + i);
  }
  cp_async_commit();
  const int64_t gc0 = t.n_face_dofs + bid * (int64_t)blockDim.x + threadIdx.x;
  Dof prc;
  if (gc0 < t.n_gamma) prc = load_dof(gc0, fld.cross_scale[gc0 - t.n_face_dofs]);
  // --- partial sums of the Schur apply (delta) and of update j-1 (gamma, rr,
  //     coarse sums), then alpha_j, beta_j and the coarse coefficients
  double alpha = 0.0, beta = 0.0;
  double cc[KC > 0 ? KC : 1];
  {
    __shared__ double sEinv[KC > 0 ? KC * KC : 1], sE[KC > 0 ? KC * KC : 1];
    constexpr int KD = KC > 0 ? KC : 1;
    for (int i = threadIdx.x; i < KC * KC; i += blockDim.x) {
      const int a = i / KD, b = i % KD;
      if (a < k && b < k) {
        sEinv[i] = cd.Einv[a * kMaxCoarse + b];
        sE[i] = 0.5 * (cd.E[a * kMaxCoarse + b] + cd.E[b * kMaxCoarse + a]);
      }
    }
    double tol2 = 0.0, ginv = 0.0, ainv = 0.0;
    int max_it = 0;
    if (threadIdx.x == 0) {
      tol2 = st->tol2;
      max_it = st->max_it;
      ginv = ld(&st->ginv_s[par ^ 1]);
      ainv = ld(&st->ainv_s[par ^ 1]);
    }
    const int nu = nblk;
    if constexpr (KC == 0) {
      // delta, gamma, rr: one warp each
      if (wib < 3) {
        const double* src = wib == 0 ? pd : pu_in + (size_t)(wib - 1) * nu;
        const double v = reduce_partials_warp(src, wib == 0 ? nd : nu);
        if (lane == 0) sums[wib] = v;
      }
      if constexpr (CG) {
        __syncthreads();
        done = s_done;
      }
      if (done) {  // uniform over the grid; no copy outlives the block
        cp_async_wait_all();
        return;
      }
      __syncthreads();
    } else {
      // delta, gamma, rr and the coarse sums: the warps take the values in
      // turn, each reduced by one warp as above
      for (int v = wib; v < NP; v += nwb) {
        double tot = 0.0;
        if (!(v >= 3 && (v - 3) % KD >= k)) {  // coarse rows beyond k stay 0
          const double* src = v == 0 ? pd : pu_in + (size_t)(v - 1) * nu;
          tot = reduce_partials_warp(src, v == 0 ? nd : nu);
        }
        if (lane == 0) sums[v] = tot;
      }
      if constexpr (CG) {
        __syncthreads();
        done = s_done;
      }
      if (done) {  // uniform over the grid; no copy outlives the block
        cp_async_wait_all();
        return;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      double gamma = sums[1], delta = sums[0];
      const double rr = sums[2];
      const double* y = sums + 3;
      const double* vq = sums + 3 + KC;
      for (int i = 0; i < k; ++i) {
        double c = 0.0;
        for (int q = 0; q < k; ++q) c += sEinv[i * KC + q] * (y[q] - (deflate ? vq[q] : 0.0));
        sab[2 + i] = c;
      }
      for (int i = 0; i < k; ++i) {
        const double ci = sab[2 + i];
        gamma += y[i] * ci;
        double ec = 0.0;
        for (int q = 0; q < k; ++q) ec += sE[i * KC + q] * sab[2 + q];
        delta += ci * (2.0 * vq[i] + ec);
      }
      int status = 1;
      double a_ = 0.0, b_ = 0.0, den = delta;
      const double gi = 1.0 / gamma;
      if (rr <= tol2) {
        status = 0;
      } else if (!isfinite(rr) || !isfinite(gamma)) {
        status = -6;
      } else if (j >= max_it) {
        status = -5;
      } else {
        if (j > 0) {
          b_ = gamma * ginv;
          den = delta - b_ * gamma * ainv;
        }
        if (!(den > 0.0) || !isfinite(den)) status = -6;
        else a_ = gamma / den;
      }
      sab[0] = a_;
      sab[1] = b_;
      sflag = status;
      if (bid == 0) {
        st->rr = rr;
        st->it = j;
        if (status != 1) {
          st->done = 1;
          st->status = status;
        } else {
          st->ainv_s[par] = den * gi;
          st->ginv_s[par] = gi;
          st->kS = j + 1;
        }
      }
    }
    __syncthreads();
    if (sflag != 1) {
      cp_async_wait_all();  // no copy outlives the block
      return;
    }
    alpha = sab[0];
    beta = sab[1];
#pragma unroll
    for (int i = 0; i < KC; ++i) cc[i] = i < k ? sab[2 + i] : 0.0;
  }
  auto coarse = [&](const double* V, int64_t g) -> double {
    double v = 0.0;
#pragma unroll
    for (int i = 0; i < KC; ++i)
      if (i < k) v += V[i * t.n_gamma + g] * cc[i];
    return v;
  };
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0.0;
  auto step = [&](int64_t g, const Dof& d) -> double {
    const double w = d.w + (KC > 0 ? coarse(cd.SQ, g) : 0.0);
    const double pg = d.u + (KC > 0 ? coarse(cd.Q, g) : 0.0) + beta * d.p;
    const double sg = w + beta * d.s;
    p[g] = pg;
    sv[g] = sg;
    x[g] = d.x + alpha * pg;
    const double rg = d.r - alpha * sg;
    r[g] = rg;
    acc[1] += rg * rg;
#pragma unroll
    for (int i = 0; i < KC; ++i)
      if (i < k) acc[2 + i] += cd.Q[i * t.n_gamma + g] * rg;
    return rg;
  };
  auto local = [&](int64_t g, double ri, double ui) {
    u[g] = ui;
    acc[0] += ri * ui;
#pragma unroll
    for (int i = 0; i < KC; ++i)
      if (i < k) acc[2 + KC + i] += cd.SQ[i * t.n_gamma + g] * ui;
  };
  cp_async_wait_all();
  double rkeep[PE];
  for (int base = gw * UG; base < t.n_blocks; base += nw * UG) {
    const int b = base + grp;
    const bool first = base == gw * UG;
    const bool has = b < t.n_blocks;
    const int off = first ? off0 : (has ? t.blk_off[b] : 0);
    const int n = first ? n0 : (has ? t.blk_n[b] : 0);
    const bool fast = n <= UL * PE;
    if (fast) {
#pragma unroll
      for (int e = 0; e < PE; ++e) {
        const int i = gl + UL * e;
        if (i < n) {
          Dof d;
          if (first) d = pre[e];
          else d = load_dof(off + i, fld.face_w[off + i]);
          const double ri = step(off + i, d);
          rkeep[e] = ri;
          const double v = ri * d.fw;  // W^-1 r (face_w holds 1 / W_ii)
          rw[i] = v;
          const float hi = (float)v;
          rwf[i] = make_float2(hi, (float)(v - (double)hi));
        }
      }
    } else {
      for (int i = gl; i < n; i += UL) {
        const double ri = step(off + i, load_dof(off + i, fld.face_w[off + i]));
        const double v = ri * fld.face_w[off + i];
        rw[i] = v;
        const float hi = (float)v;
        rwf[i] = make_float2(hi, (float)(v - (double)hi));
      }
    }
    __syncwarp();
    const float2* Ptab = (first && t.upd_stage_p) ? ptile : t.ptab_df + (has ? t.blk_poff[b] : 0);
    for (int i = gl; i < n; i += UL) {
      // column i of the symmetric P in double-float arithmetic on the FP32
      // pipes, the same error-free transformations as the explicit Schur apply
      const float2* Pc = Ptab + i;
      float hi = 0.f, lo = 0.f;
#pragma unroll 4
      for (int q = 0; q < n; ++q) {
        const float2 sq = Pc[q * n], xq = rwf[q];
        const float pr = __fmul_rn(sq.x, xq.x);
        lo = __fadd_rn(lo, __fadd_rn(__fmaf_rn(sq.x, xq.x, -pr), __fmaf_rn(sq.x, xq.y, __fmul_rn(sq.y, xq.x))));
        df_add(hi, lo, pr);
      }
      const double zi = (double)hi + (double)lo;
      const int e = (i - gl) / UL;
      const double ri = fast ? (e == 0 ? rkeep[0] : rkeep[PE - 1]) : ld(r + off + i);
      local(off + i, ri, zi * fld.face_w[off + i]);
    }
    __syncwarp();
  }
  for (int64_t g = gc0; g < t.n_gamma; g += (int64_t)nblk * blockDim.x) {
    Dof d;
    if (g == gc0) d = prc;
    else d = load_dof(g, fld.cross_scale[g - t.n_face_dofs]);
    const double ri = step(g, d);
    local(g, ri, ri * d.fw);
  }
  block_tree_sum<NV>(acc, NV, red);
  if (threadIdx.x < NV) pu_out[(size_t)threadIdx.x * nblk + bid] = red[threadIdx.x * kRedThreads];
}

template <typename T, int KC>
__global__ void __launch_bounds__(kRedThreads, 2) pcg_update_kernel(DevTables t, DevFields fld,
                                                                    const T* __restrict__ ring, double* x,
                                                                    double* r, double* u, double* p,
                                                                    double* sv, PcgState* st, CoarseDev cd,
                                                                    const double* __restrict__ pd, int nd,
                                                                    const double* __restrict__ pu_in,
                                                                    double* __restrict__ pu_out, int par) {
  pcg_update_tile<T, KC, false>(t, fld, ring, x, r, u, p, sv, st, cd, pd, nd, pu_in, pu_out, par, blockIdx.x,
                                gridDim.x);
}

// ---- batched persistent PCG ------------------------------------------------
constexpr uint32_t kBatchWaitPolls = 1u << 24;  // x 64 ns sleeps: about a second
constexpr int kBatchSchurGroup = 4;  // Schur blocks per tile of the persistent kernel

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// pre: prefix sums of the problems' Schur blocks (pre[0 .. nprob]) and of
// their update blocks (pre[nprob + 1 .. 2 nprob + 1]).  cnt[2 P] counts the
// finished Schur blocks of problem P, cnt[2 P + 1] its finished update blocks,
// cnt[2 nprob] is the queue head, cnt[2 nprob + 1] the abort flag.
__global__ void __launch_bounds__(kRedThreads, 2) batch_pcg_kernel(const BatchProb* __restrict__ probs, int nprob,
                                                                   const int* __restrict__ pre, int iters,
                                                                   unsigned* cnt, int* err) {
  __shared__ int s_q, s_ok;
  const int* preS = pre;
  const int* preU = pre + nprob + 1;
  const int totS = preS[nprob], totU = preU[nprob], per = totS + totU;
  const long long total = (long long)iters * per;
  unsigned* head = cnt + 2 * nprob;
  unsigned* abort_flag = head + 1;
  int next = 0;  // thread 0: the queue entry taken ahead of time
  if (threadIdx.x == 0) next = (int)atomicAdd(head, 1u);
  for (;;) {
    __syncthreads();  // the previous tile's shared memory is free
    if (threadIdx.x == 0) {
      s_q = ld_acquire_u32(abort_flag) ? -1 : next;
      if (s_q >= 0 && s_q < total) next = (int)atomicAdd(head, 1u);  // overlaps this tile's work
    }
    __syncthreads();
    const long long q = s_q;
    if (q < 0 || q >= total) break;
    const int it = (int)(q / per), rr = (int)(q % per);
    const bool schur = rr < totS;
    const int* pref = schur ? preS : preU;
    const int key = schur ? rr : rr - totS;
    int P = 0;
    while (P + 1 < nprob && pref[P + 1] <= key) ++P;
    const int b = key - pref[P];  // tile of this problem's phase
    const BatchProb& bp = probs[P];
    const int nts = (bp.n_schur + kBatchSchurGroup - 1) / kBatchSchurGroup;  // Schur tiles
    // wait for the phase this tile depends on (earlier in the queue)
    unsigned target = 0;
    const unsigned* c = nullptr;
    if (schur && it > 0) {
      c = cnt + 2 * P + 1;
      target = (unsigned)it * bp.n_upd;
    } else if (!schur) {
      c = cnt + 2 * P;
      target = (unsigned)(it + 1) * nts;
    }
    if (threadIdx.x == 0) {
      int ok = 1;
      if (c) {
        uint32_t polls = 0;
        while (ld_acquire_u32(c) < target) {
          if (++polls > kBatchWaitPolls) {
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
      }
      if (!ok) {
        atomicExch(err, kErrTimeout);
        atomicExch(abort_flag, 1u);
      }
      __threadfence();
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    if (schur) {
      SchurIO io;
      io.x = bp.u;
      io.ring_out = bp.ring;
      io.done = &bp.st->done;
      io.pcg = bp.st;
      io.pd = bp.pd;
      io.err = err;
      const int b1 = min((b + 1) * kBatchSchurGroup, bp.n_schur);
      for (int bb = b * kBatchSchurGroup; bb < b1; ++bb) {
        if (bp.nr == 64) schur_df_tile<64, true, 1>(bp.t, bp.sexp_df, io, bb);
        else if (bp.nr == 128) schur_df_tile<128, true>(bp.t, bp.sexp_df, io, bb);
        else schur_df_tile<256, true>(bp.t, bp.sexp_df, io, bb);
        __syncthreads();
      }
    } else {
      const int par = it & 1;
      const size_t rows = (size_t)kPcgRows * bp.n_upd;
      pcg_update_tile<double, 0, true>(bp.t, bp.f, bp.ring, bp.x, bp.r, bp.u, bp.p, bp.sv, bp.st, CoarseDev(), bp.pd,
                                       bp.n_schur, bp.pu + par * rows, bp.pu + (par ^ 1) * rows, par, b,
                                       bp.n_upd);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // this tile's results before its count
      atomicAdd(cnt + 2 * P + (schur ? 0 : 1), 1u);
    }
  }
}

__global__ void precond_kernel(DevTables t, DevFields fld, const double* __restrict__ r,
                               double* __restrict__ z) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int b = gw; b < t.n_blocks; b += nw) {
    const int off = t.blk_off[b], n = t.blk_n[b];
    const double* P = t.ptab + t.blk_poff[b];
    for (int i = lane; i < n; i += 32) {
      double zi = 0.0;
      for (int j = 0; j < n; ++j) zi += P[j * n + i] * (r[off + j] * fld.face_w[off + j]);
      z[off + i] = zi * fld.face_w[off + i];
    }
  }
  for (int64_t g = t.n_face_dofs + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < t.n_gamma;
       g += (int64_t)gridDim.x * blockDim.x)
    z[g] = r[g] * fld.cross_scale[g - t.n_face_dofs];
}

// ============================================================ global K x
template <int DIM>
__global__ void __launch_bounds__(kRedThreads) apply_K_kernel(DevTables t, DevFields fld, const double* __restrict__ x,
                                                     const double* __restrict__ f, double* y,
                                                     int mode, double* partials, unsigned* ticket,
                                                     double* nrm) {
  constexpr int NN = 1 << DIM, ND = DIM * NN;
  __shared__ double ke[ND * ND];
  __shared__ double scratch[64];
  for (int i = threadIdx.x; i < ND * ND; i += blockDim.x) ke[i] = t.Ke64[i];
  __syncthreads();
  double acc[2] = {0.0, 0.0};
  const int64_t n_nodes = t.n_dof / DIM;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < n_nodes;
       n += (int64_t)gridDim.x * blockDim.x) {
    const int k = DIM == 3 ? (int)(n % t.nn[2]) : 0;
    const int64_t ij = DIM == 3 ? n / t.nn[2] : n;
    const int j = (int)(ij % t.nn[1]), i = (int)(ij / t.nn[1]);
    double out[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) out[c] = 0.0;
    for (int ox = 0; ox < 2; ++ox) {
      const int ex = i - ox;
      if (ex < 0 || ex >= t.ne[0]) continue;
      for (int oy = 0; oy < 2; ++oy) {
        const int ey = j - oy;
        if (ey < 0 || ey >= t.ne[1]) continue;
        for (int oz = 0; oz < (DIM == 3 ? 2 : 1); ++oz) {
          const int ez = k - oz;
          if (DIM == 3 && (ez < 0 || ez >= t.ne[2])) continue;
          const int64_t e = DIM == 3 ? ((int64_t)ex * t.ne[1] + ey) * t.ne[2] + ez
                                     : (int64_t)ex * t.ne[1] + ey;
          const int ln = elem_local_node(ox, oy, oz);
          double part[DIM];
#pragma unroll
          for (int c = 0; c < DIM; ++c) part[c] = 0.0;
#pragma unroll
          for (int a = 0; a < NN; ++a) {
            int dx, dy, dz;
            elem_node_offset(a, dx, dy, dz);
            const int64_t nb = DIM == 3
                                   ? ((int64_t)(ex + dx) * t.nn[1] + (ey + dy)) * t.nn[2] + (ez + dz)
                                   : (int64_t)(ex + dx) * t.nn[1] + (ey + dy);
#pragma unroll
            for (int c2 = 0; c2 < DIM; ++c2) {
              const int64_t d2 = DIM * nb + c2;
              const double xv = t.fixed[d2] ? 0.0 : x[d2];
#pragma unroll
              for (int c = 0; c < DIM; ++c) part[c] += ke[(ln * DIM + c) * ND + a * DIM + c2] * xv;
            }
          }
          const double sc = fld.scale64[e];
#pragma unroll
          for (int c = 0; c < DIM; ++c) out[c] += sc * part[c];
        }
      }
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const int64_t d = DIM * n + c;
      if (t.fixed[d]) {
        y[d] = 0.0;
        continue;
      }
      if (mode == 0) {
        y[d] = out[c];
      } else {
        const double fv = f[d];
        const double rv = fv - out[c];
        y[d] = rv;
        acc[0] += rv * rv;
        acc[1] += fv * fv;
      }
    }
  }
  if (mode == 1) {
    if (grid_sum<2, kRedThreads>(acc, partials, ticket, scratch) && threadIdx.x == 0) {
      nrm[0] = sqrt(acc[0]);
      nrm[1] = sqrt(acc[1]);
    }
  }
}

__global__ void scatter_gamma_kernel(DevTables t, const double* __restrict__ xg, double* u) {
  const int64_t n = t.n_dof > t.n_gamma ? t.n_dof : t.n_gamma;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < t.n_gamma) u[t.gamma_dof[i]] = xg[i];
    if (i < t.n_dof && t.fixed[i]) u[i] = 0.0;
  }
}

__global__ void axpy_kernel(int64_t n, double a, const double* __restrict__ x, double* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

int grid_for(int64_t n, int threads, int cap = 152 * 8) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

template <typename T, int BP, int NS>
size_t schur_smem(const DevTables& t) {
  constexpr int PC = BP * BP, PD = BP * (BP + 1) / 2, STAGE = PC + PD;
  const int s = t.s, nloc = (s + 1) * (s + 1);
  size_t elems = (size_t)NS * STAGE + (size_t)t.nb_max * BP + BP + 2 * nloc + 64 + s * s;
  return elems * sizeof(T) + 16 + NS * sizeof(uint64_t) + 16;
}

template <typename T, int BP, int NS>
void run_schur(const DevTables& t, const DevFields& fld, const void* factor, const SchurIO& io,
               cudaStream_t st) {
  const size_t smem = schur_smem<T, BP, NS>(t);
  auto kern = schur2d_kernel<T, BP, NS>;
  DevFields f2 = fld;
  const T* ke = nullptr;
  const T* sc = nullptr;
  if constexpr (sizeof(T) == 8) {
    ke = reinterpret_cast<const T*>(t.Ke64);
    sc = reinterpret_cast<const T*>(f2.scale64);
  } else {
    ke = reinterpret_cast<const T*>(t.Ke32);
    sc = reinterpret_cast<const T*>(f2.scale32);
  }
  kern<<<t.n_sub, 32, smem, st>>>(t, ke, sc, reinterpret_cast<const T*>(factor), io);
}

template <typename T, int BP>
void run_factor(const DevTables& t, const DevFields& fld, void* factor, int* err, int* bad_sub,
                cudaStream_t st) {
  const size_t smem = factor2d_smem<T, BP>();
  auto kern = factor2d_kernel<T, BP>;
  const T* ke;
  const T* sc;
  if constexpr (sizeof(T) == 8) {
    ke = reinterpret_cast<const T*>(t.Ke64);
    sc = reinterpret_cast<const T*>(fld.scale64);
  } else {
    ke = reinterpret_cast<const T*>(t.Ke32);
    sc = reinterpret_cast<const T*>(fld.scale32);
  }
  kern<<<t.n_sub, kFacThreads, smem, st>>>(t, ke, sc, reinterpret_cast<T*>(factor), err, bad_sub);
}

template <typename T, int BP, int NR>
size_t form_smem(const DevTables& t) {
  constexpr int PC = BP * BP, PD = BP * (BP + 1) / 2;
  return (size_t)(2 * BP * NR + PC + PD + 64 + t.s * t.s) * sizeof(T) + NR * sizeof(int) + 16;
}

constexpr int kFormGC = 32, kFormTQ = 64;  // NR = 256 formation: W column group, S tile

template <typename T, int BP, int NR>
size_t form_w_smem(const DevTables& t) {
  constexpr int PC = BP * BP, PD = BP * (BP + 1) / 2;
  return (size_t)(PC + PD + 2 * BP * kFormGC + 64 + t.s * t.s) * sizeof(T) + kFormGC * sizeof(int) + 16;
}

template <typename T, int BP, int NR>
size_t form_syrk_smem(const DevTables& t) {
  return (size_t)(2 * BP * kFormTQ + 64 + t.s * t.s) * sizeof(T) + 2 * kFormTQ * sizeof(int) + 16;
}

template <typename T, int BP, int NR>
void run_form_wide(const DevTables& t, const DevFields& fld, const void* factor, void* work, void* Sexp,
                   cudaStream_t st) {
  const T* ke;
  const T* sc;
  if constexpr (sizeof(T) == 8) {
    ke = reinterpret_cast<const T*>(t.Ke64);
    sc = reinterpret_cast<const T*>(fld.scale64);
  } else {
    ke = reinterpret_cast<const T*>(t.Ke32);
    sc = reinterpret_cast<const T*>(fld.scale32);
  }
  constexpr int NQ = NR / kFormTQ;
  form_w2d_kernel<T, BP, NR, kFormGC><<<dim3(t.n_sub, NR / kFormGC), 256, form_w_smem<T, BP, NR>(t), st>>>(
      t, ke, sc, reinterpret_cast<const T*>(factor), reinterpret_cast<T*>(work));
  form_syrk2d_kernel<T, BP, NR, kFormTQ><<<dim3(t.n_sub, NQ * (NQ + 1) / 2), 256, form_syrk_smem<T, BP, NR>(t),
                                          st>>>(t, ke, sc, reinterpret_cast<const T*>(work),
                                                reinterpret_cast<T*>(Sexp));
}

template <int BP, int NR>
void run_form_df(const DevTables& t, const DevFields& fld, const void* factor, void* Sexp, cudaStream_t st) {
  schur_form2d_df_kernel<BP, NR><<<t.n_sub, 256, form_smem<double, BP, NR>(t), st>>>(
      t, t.Ke64, fld.scale64, reinterpret_cast<const double*>(factor), reinterpret_cast<double*>(Sexp));
}

template <typename T, int BP, int NR>
void run_form(const DevTables& t, const DevFields& fld, const void* factor, void* Sexp,
              cudaStream_t st) {
  const T* ke;
  const T* sc;
  if constexpr (sizeof(T) == 8) {
    ke = reinterpret_cast<const T*>(t.Ke64);
    sc = reinterpret_cast<const T*>(fld.scale64);
  } else {
    ke = reinterpret_cast<const T*>(t.Ke32);
    sc = reinterpret_cast<const T*>(fld.scale32);
  }
  schur_form2d_kernel<T, BP, NR><<<t.n_sub, 256, form_smem<T, BP, NR>(t), st>>>(
      t, ke, sc, reinterpret_cast<const T*>(factor), reinterpret_cast<T*>(Sexp));
}

}  // namespace

size_t ozaki_smem_bytes(const DevTables& t) {
  return (size_t)kOzStages * 32768 + 2 * kOzTile * 4 + FormTile<128, double>::smem(t) + 64;
}

int ozaki_kp(const DevTables& t) { return ((t.nb_max * t.BP + kOzKC - 1) / kOzKC) * kOzKC; }

// Slices of the FP64 form (54 bits; enough buffer for the FP32 form too).
size_t ozaki_slice_elems(const DevTables& t, int NR) {
  const int Kp = ozaki_kp(t);
  const int bits = Kp <= 1489 ? 6 : 5;
  return (size_t)t.n_sub * oz_slices(bits, 54) * NR * Kp;
}

int explicit_ring_size(const DevTables& t) {
  // NR: padded ring size of the explicit form (0 = explicit form unavailable)
  if (t.dim != 2) return 0;
  if (t.BP == 32) return t.s <= 8 ? 64 : (t.s <= 16 ? 128 : 0);
  if ((t.BP == 64 || t.BP == 96) && t.s <= 32) return 256;
  return 0;
}

size_t explicit_form_work_elems(const DevTables& t) {
  // W = L^-1 K_IG of every subdomain: the NR = 256 formation, and the
  // tensor-core formation of NR = 128
  const int NR = explicit_ring_size(t);
  return NR >= 128 ? (size_t)t.n_sub * t.nb_max * t.BP * NR : 0;
}

bool tensor_form_available(const DevTables& t) {
  const int NR = explicit_ring_size(t);
  return NR == 128 || NR == 256;
}

size_t tensor_form_work_bytes(const DevTables& t) {
  const int NR = explicit_ring_size(t);
  if (NR != 128 && NR != 256) return 0;
  return ozaki_slice_elems(t, NR) * sizeof(__nv_bfloat16) + (size_t)t.n_sub * NR * sizeof(int) + 256;
}

void launch_schur_form_tc(const DevTables& t, const DevFields& fld, int precision, const void* factor, void* work,
                          void* tc_work, void* Sexp, int* err, cudaStream_t st) {
  const int NR = explicit_ring_size(t);
  const int Kp = ozaki_kp(t);
  const int bits = Kp <= 1489 ? 6 : 5;
  // slices to 54 bits in both precisions: W^T W to FP64 accuracy, and for
  // the FP32 form S_i rounded once to FP32.  (Slices to only 24 bits, the
  // FP32 significand, cut the small entries of a column to the bits left
  // below its largest one: on the 512 x 256 cantilever at 1e9 stiffness
  // contrast the refined FP32 solve then took 13 cycles and 13.5 k PCG
  // iterations instead of 9 and 7.2 k.)
  const int S = oz_slices(bits, 54);
  __nv_bfloat16* Wsl = reinterpret_cast<__nv_bfloat16*>(tc_work);
  int* expo = reinterpret_cast<int*>(reinterpret_cast<char*>(tc_work) + ozaki_slice_elems(t, NR) * 2 + 128);
  const size_t sm = ozaki_smem_bytes(t);
  if (precision == 0) {
    double* W = reinterpret_cast<double*>(work);
    const double* fac = reinterpret_cast<const double*>(factor);
    if (NR == 128)
      form_w2d_kernel<double, 32, 128, kFormGC><<<dim3(t.n_sub, 128 / kFormGC), 256, form_w_smem<double, 32, 128>(t),
                                                  st>>>(t, t.Ke64, fld.scale64, fac, W);
    else if (t.BP == 64)
      form_w2d_kernel<double, 64, 256, kFormGC><<<dim3(t.n_sub, 256 / kFormGC), 256, form_w_smem<double, 64, 256>(t),
                                                  st>>>(t, t.Ke64, fld.scale64, fac, W);
    else
      form_w2d_kernel<double, 96, 256, kFormGC><<<dim3(t.n_sub, 256 / kFormGC), 256, form_w_smem<double, 96, 256>(t),
                                                  st>>>(t, t.Ke64, fld.scale64, fac, W);
    const OzSlab src{(int64_t)t.nb_max * t.BP * NR, 0, NR, -1, NR};
    launch_ozaki_slice<double>(dim3(t.n_sub, NR / 32), st, t, W, src, NR, Kp, Wsl, expo);
    if (NR == 128)
      ozaki_syrk_kernel<128, FormTile<128, double>><<<dim3(t.n_sub, 1), kOzThreads, sm, st>>>(
          t, FormTile<128, double>{t.Ke64, fld.scale64, reinterpret_cast<double*>(Sexp)}, Wsl, expo, Kp, S, err);
    else
      ozaki_syrk_kernel<256, FormTile<256, double>><<<dim3(t.n_sub, 3), kOzThreads, sm, st>>>(
          t, FormTile<256, double>{t.Ke64, fld.scale64, reinterpret_cast<double*>(Sexp)}, Wsl, expo, Kp, S, err);
  } else {
    float* W = reinterpret_cast<float*>(work);
    const float* fac = reinterpret_cast<const float*>(factor);
    if (NR == 128)
      form_w2d_kernel<float, 32, 128, kFormGC><<<dim3(t.n_sub, 128 / kFormGC), 256, form_w_smem<float, 32, 128>(t),
                                                 st>>>(t, t.Ke32, fld.scale32, fac, W);
    else if (t.BP == 64)
      form_w2d_kernel<float, 64, 256, kFormGC><<<dim3(t.n_sub, 256 / kFormGC), 256, form_w_smem<float, 64, 256>(t),
                                                 st>>>(t, t.Ke32, fld.scale32, fac, W);
    else
      form_w2d_kernel<float, 96, 256, kFormGC><<<dim3(t.n_sub, 256 / kFormGC), 256, form_w_smem<float, 96, 256>(t),
                                                 st>>>(t, t.Ke32, fld.scale32, fac, W);
    const OzSlab src{(int64_t)t.nb_max * t.BP * NR, 0, NR, -1, NR};
    launch_ozaki_slice<float>(dim3(t.n_sub, NR / 32), st, t, W, src, NR, Kp, Wsl, expo);
    if (NR == 128)
      ozaki_syrk_kernel<128, FormTile<128, float>><<<dim3(t.n_sub, 1), kOzThreads, sm, st>>>(
          t, FormTile<128, float>{t.Ke64, fld.scale64, reinterpret_cast<float*>(Sexp)}, Wsl, expo, Kp, S, err);
    else
      ozaki_syrk_kernel<256, FormTile<256, float>><<<dim3(t.n_sub, 3), kOzThreads, sm, st>>>(
          t, FormTile<256, float>{t.Ke64, fld.scale64, reinterpret_cast<float*>(Sexp)}, Wsl, expo, Kp, S, err);
  }
}

void launch_schur_form(const DevTables& t, const DevFields& fld, int precision, bool df, const void* factor,
                       void* work, void* Sexp, cudaStream_t st) {
  const int NR = explicit_ring_size(t);
  // rings of 256 (32 x 32 subdomains: 31 planes, sums of about 2000 terms)
  // keep the FP64 formation: formed in double-float their PCG needed half as
  // many iterations again
  if (precision == 0 && df && NR <= 128) {
    if (NR == 64) run_form_df<32, 64>(t, fld, factor, Sexp, st);
    else run_form_df<32, 128>(t, fld, factor, Sexp, st);
  } else if (precision == 0) {
    if (NR == 64) run_form<double, 32, 64>(t, fld, factor, Sexp, st);
    else if (NR == 128) run_form<double, 32, 128>(t, fld, factor, Sexp, st);
    else if (t.BP == 64) run_form_wide<double, 64, 256>(t, fld, factor, work, Sexp, st);
    else run_form_wide<double, 96, 256>(t, fld, factor, work, Sexp, st);
  } else {
    if (NR == 64) run_form<float, 32, 64>(t, fld, factor, Sexp, st);
    else if (NR == 128) run_form<float, 32, 128>(t, fld, factor, Sexp, st);
    else if (t.BP == 64) run_form_wide<float, 64, 256>(t, fld, factor, work, Sexp, st);
    else run_form_wide<float, 96, 256>(t, fld, factor, work, Sexp, st);
  }
}

void launch_split_df(const double* in, float2* out, int64_t n, cudaStream_t st) {
  split_df_kernel<<<grid_for(n, 256), 256, 0, st>>>(in, out, n);
}

template <int NR>
void run_explicit_df(const DevTables& t, const float2* S, const SchurIO& io, int split, cudaStream_t st) {
  if (split == 1)
    schur_explicit_df_kernel<NR, 1><<<t.n_sub, 256, 0, st>>>(t, S, io);
  else if (split == 4 && NR >= 128)
    schur_explicit_df_kernel<NR, (NR >= 128 ? 4 : 2)><<<4 * t.n_sub, 256, 0, st>>>(t, S, io);
  else
    schur_explicit_df_kernel<NR, 2><<<2 * t.n_sub, 256, 0, st>>>(t, S, io);
}

int launch_schur_explicit_df(const DevTables& t, const float2* Sexp, const SchurIO& io, int split,
                             cudaStream_t st) {
  const int NR = explicit_ring_size(t);
  split = explicit_split(t, split);
  if (NR == 64) run_explicit_df<64>(t, Sexp, io, split, st);
  else if (NR == 128) run_explicit_df<128>(t, Sexp, io, split, st);
  else run_explicit_df<256>(t, Sexp, io, split, st);
  return split * t.n_sub;
}

int explicit_split(const DevTables& t, int split) {
  // CTAs per subdomain of the explicit apply: 1, 2 or 4, at least 32 rows
  // each; 0 (and anything else) by ring size: one CTA for rings of 64 (8 x 8
  // subdomains on a 512 x 256 grid, per PCG iteration: native FP64 33.1
  // against 40.8 us, double-float 21.6 against 27.2 us), two for the larger
  // ones (128: FP64 28.9 against 30.7 with one and 31.6 with four, double-float
  // equal with one; 256: FP64 equal, double-float 19.7 against 21.6 and 20.8)
  const int NR = explicit_ring_size(t);
  if (split != 1 && split != 2 && split != 4) split = NR <= 64 ? 1 : 2;
  if (NR / split < 32) split = NR <= 64 ? 1 : 2;
  return split;
}

template <int NR>
void run_explicit_f64(const DevTables& t, const double* S, const SchurIO& io, int split, cudaStream_t st) {
  if (split == 1)
    schur_explicit_f64_kernel<NR, 1><<<t.n_sub, 256, 0, st>>>(t, S, io);
  else if (split == 4 && NR >= 128)
    schur_explicit_f64_kernel<NR, (NR >= 128 ? 4 : 2)><<<4 * t.n_sub, 256, 0, st>>>(t, S, io);
  else
    schur_explicit_f64_kernel<NR, 2><<<2 * t.n_sub, 256, 0, st>>>(t, S, io);
}

int launch_schur_explicit(const DevTables& t, int precision, const void* Sexp, const SchurIO& io, int split,
                          cudaStream_t st) {
  const int NR = explicit_ring_size(t);
  if (precision == 0) {
    const double* S = (const double*)Sexp;
    split = explicit_split(t, split);
    if (NR == 64) run_explicit_f64<64>(t, S, io, split, st);
    else if (NR == 128) run_explicit_f64<128>(t, S, io, split, st);
    else run_explicit_f64<256>(t, S, io, split, st);
    return split * t.n_sub;
  } else {
    const float* S = (const float*)Sexp;
    if (NR == 64) schur_explicit_kernel<float, 64><<<2 * t.n_sub, 256, 0, st>>>(t, S, io);
    else if (NR == 128) schur_explicit_kernel<float, 128><<<2 * t.n_sub, 256, 0, st>>>(t, S, io);
    else schur_explicit_kernel<float, 256><<<2 * t.n_sub, 256, 0, st>>>(t, S, io);
  }
  return 2 * t.n_sub;
}

// ============================================================ launchers
cudaError_t configure_kernels() {
  int dev = 0, big = 232448;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&big, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaError_t e = cudaSuccess;
  // dynamic opt-in = device maximum minus the kernel's static shared memory
#define DDEL_CFG(k)                                                                   \
  do {                                                                                \
    cudaFuncAttributes fa;                                                            \
    cudaError_t e2 = cudaFuncGetAttributes(&fa, k);                                   \
    if (e2 == cudaSuccess)                                                            \
      e2 = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                                big - (int)fa.sharedSizeBytes);                       \
    if (e2 != cudaSuccess) e = e2;                                                    \
  } while (0)
  DDEL_CFG((schur2d_kernel<double, 32, 3>));
  DDEL_CFG((schur2d_kernel<double, 64, 2>));
  DDEL_CFG((schur2d_kernel<double, 96, 1>));
  DDEL_CFG((schur2d_kernel<float, 32, 4>));
  DDEL_CFG((schur2d_kernel<float, 64, 2>));
  DDEL_CFG((schur2d_kernel<float, 96, 2>));
  DDEL_CFG((factor2d_kernel<double, 32>));
  DDEL_CFG((factor2d_kernel<double, 64>));
  DDEL_CFG((factor2d_kernel<double, 96>));
  DDEL_CFG((factor2d_kernel<float, 32>));
  DDEL_CFG((factor2d_kernel<float, 64>));
  DDEL_CFG((factor2d_kernel<float, 96>));
  DDEL_CFG((schur_form2d_kernel<double, 32, 64>));
  DDEL_CFG((schur_form2d_kernel<double, 32, 128>));
  DDEL_CFG((schur_form2d_kernel<float, 32, 64>));
  DDEL_CFG((schur_form2d_kernel<float, 32, 128>));
  DDEL_CFG((form_w2d_kernel<double, 64, 256, kFormGC>));
  DDEL_CFG((form_w2d_kernel<float, 64, 256, kFormGC>));
  DDEL_CFG((form_syrk2d_kernel<double, 64, 256, kFormTQ>));
  DDEL_CFG((form_syrk2d_kernel<float, 64, 256, kFormTQ>));
  DDEL_CFG((schur_form2d_df_kernel<32, 64>));
  DDEL_CFG((schur_form2d_df_kernel<32, 128>));
  DDEL_CFG((form_w2d_kernel<double, 96, 256, kFormGC>));
  DDEL_CFG((form_w2d_kernel<float, 96, 256, kFormGC>));
  DDEL_CFG((form_syrk2d_kernel<double, 96, 256, kFormTQ>));
  DDEL_CFG((form_syrk2d_kernel<float, 96, 256, kFormTQ>));
  // the update kernel's staged face tables plus the coarse variants' static
  // reduction arrays exceed the default 48 KB
  DDEL_CFG((ozaki_syrk_kernel<128, FormTile<128, double>>));
  DDEL_CFG((ozaki_syrk_kernel<256, FormTile<256, double>>));
  DDEL_CFG((ozaki_syrk_kernel<128, FormTile<128, float>>));
  DDEL_CFG((ozaki_syrk_kernel<256, FormTile<256, float>>));
  DDEL_CFG((form_w2d_kernel<double, 32, 128, kFormGC>));
  DDEL_CFG((form_w2d_kernel<float, 32, 128, kFormGC>));
  DDEL_CFG((batch_pcg_kernel));
  DDEL_CFG((pcg_update_kernel<double, 0>));
  DDEL_CFG((pcg_update_kernel<double, 4>));
  DDEL_CFG((pcg_update_kernel<double, 8>));
  DDEL_CFG((pcg_update_kernel<float, 0>));
  DDEL_CFG((pcg_update_kernel<float, 4>));
  DDEL_CFG((pcg_update_kernel<float, 8>));
#undef DDEL_CFG
  cudaError_t e3 = configure_kernels3d();
  return e != cudaSuccess ? e : e3;
}

void launch_assemble(const DevTables& t, const DevFields& fld, const double* rho, double E, double p,
                     int face_scaling, int crosspoint_mode, int* err, cudaStream_t st) {
  scale_kernel<<<grid_for(t.n_elem, 256), 256, 0, st>>>(rho, t.n_elem, E, p, fld.scale64,
                                                        fld.scale32, err);
  if (t.dim == 2)
    gamma_diag_kernel<2><<<grid_for(t.n_gamma, 256), 256, 0, st>>>(t, fld);
  else
    gamma_diag_kernel<3><<<grid_for(t.n_gamma, 256), 256, 0, st>>>(t, fld);
  face_scale_kernel<<<grid_for((int64_t)t.n_blocks * 32 + t.n_gamma, 256), 256, 0, st>>>(
      t, fld, face_scaling, crosspoint_mode);
}

int launch_factor(const DevTables& t, const DevFields& fld, int precision, void* factor, void* work,
                  int* err, int* bad_sub, int tensor, cudaStream_t st) {
  if (t.dim == 3) return launch_factor3d(t, fld, precision, factor, work, err, bad_sub, tensor, st);
  if (precision == 0) {
    if (t.BP == 32) run_factor<double, 32>(t, fld, factor, err, bad_sub, st);
    else if (t.BP == 64) run_factor<double, 64>(t, fld, factor, err, bad_sub, st);
    else run_factor<double, 96>(t, fld, factor, err, bad_sub, st);
  } else {
    if (t.BP == 32) run_factor<float, 32>(t, fld, factor, err, bad_sub, st);
    else if (t.BP == 64) run_factor<float, 64>(t, fld, factor, err, bad_sub, st);
    else run_factor<float, 96>(t, fld, factor, err, bad_sub, st);
  }
  return 1;
}

size_t schur_smem_bytes(const DevTables& t, int precision) {
  if (precision == 0) {
    if (t.BP == 32) return schur_smem<double, 32, 3>(t);
    if (t.BP == 64) return schur_smem<double, 64, 2>(t);
    return schur_smem<double, 96, 1>(t);
  }
  if (t.BP == 32) return schur_smem<float, 32, 4>(t);
  if (t.BP == 64) return schur_smem<float, 64, 2>(t);
  return schur_smem<float, 96, 2>(t);
}

void launch_schur(const DevTables& t, const DevFields& fld, int precision, const void* factor,
                  const SchurIO& io, cudaStream_t st) {
  if (t.dim == 3) {
    launch_schur3d(t, fld, precision, factor, io, st);
    return;
  }
  if (precision == 0) {
    if (t.BP == 32) run_schur<double, 32, 3>(t, fld, factor, io, st);
    else if (t.BP == 64) run_schur<double, 64, 2>(t, fld, factor, io, st);
    else run_schur<double, 96, 1>(t, fld, factor, io, st);
  } else {
    if (t.BP == 32) run_schur<float, 32, 4>(t, fld, factor, io, st);
    else if (t.BP == 64) run_schur<float, 64, 2>(t, fld, factor, io, st);
    else run_schur<float, 96, 2>(t, fld, factor, io, st);
  }
}

void launch_gamma_sum(const DevTables& t, int precision, const void* ring, const double* base,
                      double sign, double* out, cudaStream_t st) {
  const int g = grid_for(t.n_gamma, 256);
  if (precision == 0)
    gamma_sum_kernel<double><<<g, 256, 0, st>>>(t, (const double*)ring, base, sign, out);
  else
    gamma_sum_kernel<float><<<g, 256, 0, st>>>(t, (const float*)ring, base, sign, out);
}

static size_t update_smem(const DevTables& t) {
  return (size_t)(kRedThreads / 32) * t.max_blk_n * (sizeof(double) + sizeof(float2));
}

// The update kernel's shared memory: per warp (32 / upd_lanes) face blocks of
// W^-1 r as doubles and float pairs, plus their H~^-1 tables when staged.
static size_t update_kernel_smem(const DevTables& t) {
  const size_t ug = 32 / t.upd_lanes, w = kRedThreads / 32;
  size_t b = w * ug * t.max_blk_n * (sizeof(double) + sizeof(float2));
  if (t.upd_stage_p) b += w * ug * (size_t)t.max_blk_n * t.max_blk_n * sizeof(float2);
  return b;
}

// Coarse columns padded to 4 or 8 (template width of the coarse sums).
static int coarse_width(int k) { return k <= 0 ? 0 : k <= 4 ? 4 : 8; }

void launch_pcg_init(const DevTables& t, const DevFields& fld, const double* g, double* x, double* r,
                     double* u, double* p, double* sv, PcgState* s, double* pu_out, cudaStream_t st,
                     int nblk, const CoarseDev& cd) {
  const size_t sm = update_smem(t);
  switch (coarse_width(cd.k)) {  // x0 = Q c0 and the coarse sums of iteration 0
    case 4:
      pcg_cg_kernel<double, true, 4><<<nblk, kRedThreads, sm, st>>>(t, fld, g, nullptr, x, r, u, p, sv, s, cd,
                                                                     nullptr, 0, nullptr, pu_out, 1);
      break;
    case 8:
      pcg_cg_kernel<double, true, 8><<<nblk, kRedThreads, sm, st>>>(t, fld, g, nullptr, x, r, u, p, sv, s, cd,
                                                                     nullptr, 0, nullptr, pu_out, 1);
      break;
    default:
      pcg_cg_kernel<double, true, 0><<<nblk, kRedThreads, sm, st>>>(t, fld, g, nullptr, x, r, u, p, sv, s, cd,
                                                                     nullptr, 0, nullptr, pu_out, 1);
  }
}

// Step length after a reliable update.  The Chronopoulos-Gear denominator
// delta - beta gamma / alpha_prev equals (p, S p) only while the new residual
// is orthogonal to the previous search direction, which a replaced residual
// is not; the exact value is delta + 2 beta (u, s_prev) + beta^2 (p_prev,
// s_prev).  Stores the 1 / alpha that makes the next update's formula give
// it.  The replacement follows a whole batch of an even number of iterations
// (the relaxed PCG runs its low-precision phase with a zero device
// tolerance, so no batch stops early): the last update wrote slot 1, which
// the next batch's first update reads.  Also the true rr and whether it meets
// tol2 (replaced_ok); an error status (done) is kept.  One block.
__global__ void __launch_bounds__(kRedThreads) pcg_replace_fix_kernel(PcgState* st, const double* __restrict__ pu,
                                                                      int nblk, double tol2) {
  __shared__ double red[4 * kRedThreads];
  double a[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    a[v] = 0.0;
    for (int b = threadIdx.x; b < nblk; b += kRedThreads) a[v] += pu[(size_t)v * nblk + b];
  }
  block_tree_sum<4>(a, 4, red);
  if (threadIdx.x != 0) return;
  const double gamma = red[0], rr = red[kRedThreads], us = red[2 * kRedThreads], ps = red[3 * kRedThreads];
  st->rr = rr;
  st->replaced_ok = rr <= tol2 ? 1 : 0;
  if (st->done) return;  // breakdown or iteration cap: the host stops
  const double beta = gamma * st->ginv_s[1];
  const double ainv = -(2.0 * us + beta * ps) / gamma;
  if (st->kS <= 0 || !isfinite(rr) || !(gamma > 0.0) || !isfinite(ainv)) {
    st->done = 1;
    st->status = -6;  // breakdown
    return;
  }
  st->ainv_s[1] = ainv;
}

void launch_pcg_replace(const DevTables& t, const DevFields& fld, const double* g, const double* ring, double* x,
                        double* r, double* u, double* p, double* sv, PcgState* s, double* pu_out, cudaStream_t st,
                        int nblk, double tol2) {
  pcg_cg_kernel<double, true, 0, true><<<nblk, kRedThreads, update_smem(t), st>>>(
      t, fld, g, ring, x, r, u, p, sv, s, CoarseDev(), nullptr, 0, nullptr, pu_out, 1);
  pcg_replace_fix_kernel<<<1, kRedThreads, 0, st>>>(s, pu_out, nblk, tol2);
}

template <typename T>
static void launch_update_t(const DevTables& t, const DevFields& fld, const T* ring, double* x, double* r,
                            double* u, double* p, double* sv, PcgState* s, const double* pd, int nd,
                            const double* pu_in, double* pu_out, int par, cudaStream_t st, int nblk,
                            const CoarseDev& cd) {
  const size_t sm = update_kernel_smem(t);
  switch (cd.correct ? coarse_width(cd.k) : 0) {
    case 4:
      pcg_update_kernel<T, 4><<<nblk, kRedThreads, sm, st>>>(t, fld, ring, x, r, u, p, sv, s, cd, pd, nd, pu_in,
                                                             pu_out, par);
      break;
    case 8:
      pcg_update_kernel<T, 8><<<nblk, kRedThreads, sm, st>>>(t, fld, ring, x, r, u, p, sv, s, cd, pd, nd, pu_in,
                                                             pu_out, par);
      break;
    default:
      pcg_update_kernel<T, 0><<<nblk, kRedThreads, sm, st>>>(t, fld, ring, x, r, u, p, sv, s, cd, pd, nd, pu_in,
                                                             pu_out, par);
  }
}

void launch_pcg_update(const DevTables& t, const DevFields& fld, int precision, const void* ring,
                       double* x, double* r, double* u, double* p, double* sv, PcgState* s,
                       const double* pd, int nd, const double* pu_in, double* pu_out, int par,
                       cudaStream_t st, int nblk, const CoarseDev& cd) {
  if (precision == 0)
    launch_update_t(t, fld, (const double*)ring, x, r, u, p, sv, s, pd, nd, pu_in, pu_out, par, st, nblk, cd);
  else
    launch_update_t(t, fld, (const float*)ring, x, r, u, p, sv, s, pd, nd, pu_in, pu_out, par, st, nblk, cd);
}

size_t batch_pcg_smem(const DevTables& t) { return update_kernel_smem(t); }

int batch_schur_tiles(int n_schur_blocks) { return (n_schur_blocks + kBatchSchurGroup - 1) / kBatchSchurGroup; }

int batch_pcg_blocks_per_sm(size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_pcg_kernel, kRedThreads, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_batch_pcg(const BatchProb* probs, int nprob, const int* pre, int iters, unsigned* cnt, int* err,
                             int grid, size_t smem, cudaStream_t st) {
  void* args[] = {(void*)&probs, (void*)&nprob, (void*)&pre, (void*)&iters, (void*)&cnt, (void*)&err};
  // a cooperative launch: every block is resident at once, which the waits
  // on earlier queue entries rely on
  return cudaLaunchCooperativeKernel((const void*)batch_pcg_kernel, dim3(grid), dim3(kRedThreads), args, smem, st);
}

void launch_precond(const DevTables& t, const DevFields& fld, const double* r, double* z,
                    cudaStream_t st) {
  precond_kernel<<<grid_for((int64_t)t.n_blocks * 32 + t.n_gamma, 256), 256, 0, st>>>(t, fld, r, z);
}

void launch_apply_K(const DevTables& t, const DevFields& fld, const double* x, const double* f,
                    double* y, int mode, double* partials, unsigned* ticket, double* nrm,
                    cudaStream_t st, int nblk) {
  if (t.dim == 2)
    apply_K_kernel<2><<<nblk, kRedThreads, 0, st>>>(t, fld, x, f, y, mode, partials, ticket, nrm);
  else
    apply_K_kernel<3><<<nblk, kRedThreads, 0, st>>>(t, fld, x, f, y, mode, partials, ticket, nrm);
}

void launch_scatter_gamma(const DevTables& t, const double* xg, double* u, cudaStream_t st) {
  scatter_gamma_kernel<<<grid_for(t.n_dof > t.n_gamma ? t.n_dof : t.n_gamma, 256), 256, 0, st>>>(
      t, xg, u);
}

__global__ void round_f32_kernel(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

void launch_round_f32(const double* in, float* out, int64_t n, cudaStream_t st) {
  round_f32_kernel<<<grid_for(n, 256), 256, 0, st>>>(in, out, n);
}

void launch_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t st) {
  axpy_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, a, x, y);
}

}  // namespace ddel
