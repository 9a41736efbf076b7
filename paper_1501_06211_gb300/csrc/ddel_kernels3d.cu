// 3D H8 path: factorisation and per-subdomain solve for blocks too large for
// shared memory (interior planes of up to 8 x 8 nodes x 3 components).
//
//  * factor3d_kernel: one CTA per subdomain; per interior plane k the block
//    A_kk - C_k C_k^T is assembled in a global scratch matrix (the product
//    over C_k's nonzero band only; optionally on the tensor cores, one launch
//    per plane), factorised by a blocked right-looking Cholesky (32-wide
//    panels through shared memory), inverted by blocked forward substitution
//    (D_k = L_kk^-1), and C_{k+1} = A_{k+1,k} D_k^T is formed from the 27
//    nonzeros per row of the plane coupling A_{k+1,k}.  The factor layout
//    is the one of the 2D path: [C_k (column-major) | D_k (packed lower,
//    column-major)] per plane.
//  * schur3d_kernel: one CTA per subdomain: w = f_I - K_IG x element by element,
//    block forward/backward substitution with coalesced column reads of the
//    factor, t into the local closure, y = (K^(i) [t; x])_G on the ring.
#include <cuda_bf16.h>

#include <cmath>

#include "ddel_device.cuh"
#include "ddel_launch.h"

namespace ddel {
namespace {

constexpr int kT3 = 256;  // threads per CTA
constexpr int TB = 32;    // tile edge

__device__ __forceinline__ int64_t node3(const DevTables& t, int i, int j, int k) {
  return ((int64_t)i * t.nn[1] + j) * t.nn[2] + k;
}

// Interior row r of plane k -> grid node and component (3D): rows enumerate
// (y, z) of the plane with z fastest, then the 3 components.
__device__ __forceinline__ void row_node3(const SubInfo& si, int k, int r, int& x, int& y, int& z,
                                          int& c) {
  c = r % 3;
  const int q = r / 3;
  x = si.ilo[0] + k;
  y = si.ilo[1] + q / si.icnt[2];
  z = si.ilo[2] + q % si.icnt[2];
}

template <typename T>
__device__ T entry3d(const DevTables& t, const SubInfo& si, const T* ke, const T* __restrict__ scale,
                     int kr, int r, int kc, int c) {
  const bool vr = r < si.bsz, vc = c < si.bsz;
  if (!vr || !vc) return (kr == kc && r == c) ? T(1) : T(0);
  int xr, yr, zr, cr, xc, yc, zc, cc;
  row_node3(si, kr, r, xr, yr, zr, cr);
  row_node3(si, kc, c, xc, yc, zc, cc);
  // nodes more than one element apart do not couple (checked before any load)
  if (abs(xr - xc) > 1 || abs(yr - yc) > 1 || abs(zr - zc) > 1) return T(0);
  const bool fr = t.fixed[3 * node3(t, xr, yr, zr) + cr];
  const bool fc = t.fixed[3 * node3(t, xc, yc, zc) + cc];
  if (fr || fc) return (kr == kc && r == c) ? T(1) : T(0);
  T sum = T(0);
  const int s = t.s;
  for (int ex = max(xr, xc) - 1; ex <= min(xr, xc); ++ex) {
    if (ex - si.lo[0] < 0 || ex - si.lo[0] >= s) continue;
    for (int ey = max(yr, yc) - 1; ey <= min(yr, yc); ++ey) {
      if (ey - si.lo[1] < 0 || ey - si.lo[1] >= s) continue;
      for (int ez = max(zr, zc) - 1; ez <= min(zr, zc); ++ez) {
        if (ez - si.lo[2] < 0 || ez - si.lo[2] >= s) continue;
        const int la = elem_local_node(xr - ex, yr - ey, zr - ez);
        const int lb = elem_local_node(xc - ex, yc - ey, zc - ez);
        const int64_t e = ((int64_t)ex * t.ne[1] + ey) * t.ne[2] + ez;
        sum += scale[e] * ke[(la * 3 + cr) * 24 + lb * 3 + cc];
      }
    }
  }
  return sum;
}

// Column of the w-th possible nonzero of row i of the plane coupling
// A_{k+1,k} (w = 9 (dy + 1) + 3 (dz + 1) + component, node (y + dy, z + dz) of
// the plane before), or -1 when that node lies outside the interior plane or
// row i is a padding row.
__device__ __forceinline__ int nz_col3(const SubInfo& si, int i, int w, int BP) {
  if (i >= si.bsz) return -1;
  const int q = i / 3, y = q / si.icnt[2] + w / 9 - 1, z = q % si.icnt[2] + (w / 3) % 3 - 1;
  if (y < 0 || y >= si.icnt[1] || z < 0 || z >= si.icnt[2]) return -1;
  const int m = 3 * (y * si.icnt[2] + z) + w % 3;
  return m < BP ? m : -1;
}

// C(i, j) += alpha * sum_m A(i, m) B(j, m) for i < M, j < N (j <= i when lower;
// with b_tri the caller guarantees B(j, m) = 0 for m < j, with a_band >= 0
// that A(i, m) = 0 for m < i - a_band, which a lower product also needs of B),
// with general strides A(i, m) = A[i * ai + m * am], B(j, m) = B[j * bj + m * bm],
// C(i, j) = C[i * ci + j * cj].  32 x 32 x 32 tiles through shared memory.
template <typename T>
__device__ void cta_gemm(int M, int N, int K, const T* A, int ai, int am, const T* B, int bj, int bm,
                         T* C, int ci, int cj, T alpha, bool lower, T* sA, T* sB, bool b_tri = false,
                         int a_band = -1) {
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;  // each thread: rows ty, ty+16; cols tx, tx+16
  for (int i0 = 0; i0 < M; i0 += TB)
    for (int j0 = 0; j0 < N; j0 += TB) {
      if (lower && j0 > i0 + TB - 1) continue;
      T acc[2][2] = {{T(0), T(0)}, {T(0), T(0)}};
      // b_tri: B(j, m) = 0 for m < j, so the tile's products start at m = j0;
      // a_band >= 0: A(i, m) = 0 for m < i - a_band, and with j <= i (lower)
      // the tile's products start at the chunk holding i0 - a_band
      int m_start = b_tri ? j0 : 0;
      if (a_band >= 0 && lower) m_start = max(m_start, ((i0 - a_band) / TB) * TB);
      for (int m0 = m_start; m0 < K; m0 += TB) {
        for (int q = tid; q < TB * TB; q += kT3) {
          const int a = q / TB, b = q % TB;  // a: row in tile, b: m in tile
          const int i = i0 + a, j = j0 + a, m = m0 + b;
          sA[a * (TB + 1) + b] = (i < M && m < K) ? A[(int64_t)i * ai + (int64_t)m * am] : T(0);
          sB[a * (TB + 1) + b] = (j < N && m < K) ? B[(int64_t)j * bj + (int64_t)m * bm] : T(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int b = 0; b < TB; ++b) {
          const T a0 = sA[ty * (TB + 1) + b], a1 = sA[(ty + 16) * (TB + 1) + b];
          const T b0 = sB[tx * (TB + 1) + b], b1 = sB[(tx + 16) * (TB + 1) + b];
          acc[0][0] += a0 * b0;
          acc[0][1] += a0 * b1;
          acc[1][0] += a1 * b0;
          acc[1][1] += a1 * b1;
        }
        __syncthreads();
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
          if (i < M && j < N && (!lower || j <= i))
            C[(int64_t)i * ci + (int64_t)j * cj] += alpha * acc[u][v];
        }
    }
  __syncthreads();
}

// Blocked right-looking Cholesky of the row-major n x n matrix A (lower part);
// pivots that are not positive set *bad and are replaced by 1.
template <typename T>
__device__ void cta_cholesky(T* A, int n, T* sA, T* sB, bool* bad) {
  const int tid = threadIdx.x;
  for (int jb = 0; jb < n; jb += TB) {
    const int w = min(TB, n - jb);
    // diagonal tile in shared memory
    for (int q = tid; q < TB * TB; q += kT3) {
      const int a = q / TB, b = q % TB;
      sA[a * (TB + 1) + b] = (a < w && b < w) ? A[(int64_t)(jb + a) * n + jb + b] : T(0);
    }
    __syncthreads();
    for (int j = 0; j < w; ++j) {
      // the pivot, and its reciprocal in sB[j] for the panel below; FP64 by
      // one Newton reciprocal square root (the FP64 pipe retires a warp
      // instruction per 16 clocks however few lanes are active), FP32 by the
      // correctly rounded square root and quotients
      if (tid == 0) {
        T d = sA[j * (TB + 1) + j];
        if (!(d > T(0)) || !isfinite((double)d)) {
          *bad = true;
          d = T(1);
        }
        if constexpr (sizeof(T) == 8) {
          const T r = pivot_rsqrt(d);
          sA[j * (TB + 1) + j] = d * r;
          sB[j] = r;
        } else {
          const T l = sqrt(d);
          sA[j * (TB + 1) + j] = l;
          sB[j] = T(1) / l;
        }
      }
      __syncthreads();
      if (tid > j && tid < w) {
        if constexpr (sizeof(T) == 8)
          sA[tid * (TB + 1) + j] *= sB[j];
        else
          sA[tid * (TB + 1) + j] /= sA[j * (TB + 1) + j];
      }
      __syncthreads();
      for (int q = tid; q < TB * TB; q += kT3) {
        const int a = q / TB, b = q % TB;
        if (a > j && b > j && b <= a && a < w) sA[a * (TB + 1) + b] -= sA[a * (TB + 1) + j] * sA[b * (TB + 1) + j];
      }
      __syncthreads();
    }
    for (int q = tid; q < TB * TB; q += kT3) {
      const int a = q / TB, b = q % TB;
      if (a < w && b <= a) A[(int64_t)(jb + a) * n + jb + b] = sA[a * (TB + 1) + b];
    }
    __syncthreads();
    // panel: rows below, X L11^T = A21 (forward substitution across the w columns)
    for (int i = jb + w + tid; i < n; i += kT3) {
      T* row = A + (int64_t)i * n + jb;
      for (int c = 0; c < w; ++c) {
        T v = row[c];
        for (int m = 0; m < c; ++m) v -= row[m] * sA[c * (TB + 1) + m];
        if constexpr (sizeof(T) == 8)
          row[c] = v * sB[c];
        else
          row[c] = v / sA[c * (TB + 1) + c];
      }
    }
    __syncthreads();
    // trailing update A22 -= L21 L21^T (lower)
    const int r0 = jb + w;
    if (r0 < n)
      cta_gemm<T>(n - r0, n - r0, w, A + (int64_t)r0 * n + jb, n, 1, A + (int64_t)r0 * n + jb, n, 1,
                  A + (int64_t)r0 * n + r0, n, 1, T(-1), true, sA, sB);
  }
}

// D = L^-1 (both row-major n x n, lower) by block rows:
// D_i,: = L_ii^-1 (E_i - L_i,<i D_<i,:).
template <typename T>
__device__ void cta_tri_inverse(const T* L, T* D, int n, T* sA, T* sB) {
  const int tid = threadIdx.x;
  for (int q = tid; q < n * n; q += kT3) D[q] = T(0);
  __syncthreads();
  for (int ib = 0; ib < n; ib += TB) {
    const int w = min(TB, n - ib);
    // R = E_i - L_i,<i D_<i,: for columns 0 .. ib+w-1 (stored into D's block row)
    for (int q = tid; q < w * (ib + w); q += kT3) {
      const int a = q / (ib + w), j = q % (ib + w);
      D[(int64_t)(ib + a) * n + j] = (ib + a == j) ? T(1) : T(0);
    }
    __syncthreads();
    if (ib > 0)
      cta_gemm<T>(w, ib, ib, L + (int64_t)ib * n, n, 1, D, 1, n, D + (int64_t)ib * n, n, 1, T(-1),
                  false, sA, sB, true);
    // solve L_ii X = R in place (forward substitution down the w rows)
    for (int q = tid; q < TB * TB; q += kT3) {
      const int a = q / TB, b = q % TB;
      sA[a * (TB + 1) + b] = (a < w && b < w) ? L[(int64_t)(ib + a) * n + ib + b] : T(0);
    }
    if (sizeof(T) == 8 && tid < w) sB[tid] = T(1) / L[(int64_t)(ib + tid) * n + ib + tid];
    __syncthreads();
    for (int a = 0; a < w; ++a) {
      for (int j = tid; j < ib + w; j += kT3) {
        T v = D[(int64_t)(ib + a) * n + j];
        for (int m = 0; m < a; ++m) v -= sA[a * (TB + 1) + m] * D[(int64_t)(ib + m) * n + j];
        if constexpr (sizeof(T) == 8)
          D[(int64_t)(ib + a) * n + j] = v * sB[a];
        else
          D[(int64_t)(ib + a) * n + j] = v / sA[a * (TB + 1) + a];
      }
      __syncthreads();
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kT3) factor3d_kernel(DevTables t, const T* __restrict__ Ke_g,
                                                       const T* __restrict__ scale,
                                                       T* __restrict__ factor, T* __restrict__ work,
                                                       int* err, int* bad_sub, int k0, int k1, int prepared) {
  const int BP = t.BP, PC = BP * BP, PD = BP * (BP + 1) / 2, STAGE = PC + PD;
  const int sub = blockIdx.x, tid = threadIdx.x;
  const SubInfo si = t.subs[sub];
  __shared__ T ke[576];
  __shared__ T sA[TB * (TB + 1)], sB[TB * (TB + 1)];
  __shared__ bool bad;
  for (int i = tid; i < 576; i += kT3) ke[i] = Ke_g[i];
  if (tid == 0) bad = false;
  __syncthreads();
  T* A = work + (int64_t)sub * 2 * PC;  // A_kk, then L_kk, then A_{k+1,k}
  T* D = A + PC;                         // dense D_k
  T* fb = factor + si.factor_off;
  for (int k = k0; k < min(k1, si.nb); ++k) {
    // A_kk - C_k C_k^T, unless an earlier launch (the tensor-core product)
    // left it in A already
    if (!(prepared && k > 0)) {
      for (int q = tid; q < PC; q += kT3) {
        const int i = q / BP, j = q % BP;
        A[q] = j <= i ? entry3d<T>(t, si, ke, scale, k, i, k, j) : T(0);
      }
      __syncthreads();
      if (k > 0) {  // A -= C_k C_k^T, C_k column-major in the factor
        const T* Ck = fb + (int64_t)k * STAGE;
        // C_k(i, m) = 0 below the lowest column row i couples to in plane
        // k - 1, 3 (i / 3) - 3 icnt_2 - 3 >= i - 3 icnt_2 - 5: the product
        // skips those chunks
        cta_gemm<T>(BP, BP, BP, Ck, 1, BP, Ck, 1, BP, A, BP, 1, T(-1), true, sA, sB, false,
                    3 * si.icnt[2] + 5);
      }
    }
    cta_cholesky<T>(A, BP, sA, sB, &bad);
    cta_tri_inverse<T>(A, D, BP, sA, sB);
    __syncthreads();
    T* Dg = fb + (int64_t)k * STAGE + PC;
    for (int q = tid; q < PC; q += kT3) {
      const int j = q / BP, r = q % BP;  // column-major walk
      if (r >= j) Dg[j * BP - j * (j - 1) / 2 + (r - j)] = D[(int64_t)r * BP + j];
    }
    if (k + 1 < si.nb) {
      // C_{k+1} = A_{k+1,k} D_k^T.  Row i of A_{k+1,k} (node (y, z) of plane
      // k + 1) couples only to the nodes (y + dy, z + dz), |dy|, |dz| <= 1, of
      // plane k: 27 columns w = 9 (dy + 1) + 3 (dz + 1) + component.  Their
      // entries go to anz[w * BP + i] (the scratch A, free after the inverse).
      T* anz = A;
      for (int q = tid; q < 27 * BP; q += kT3) {
        const int w = q / BP, i = q % BP;
        const int m = nz_col3(si, i, w, BP);
        anz[q] = m >= 0 ? entry3d<T>(t, si, ke, scale, k + 1, i, k, m) : T(0);
      }
      __syncthreads();
      // C stored column-major: Cg[j * BP + i] = sum_w anz(i, w) D(j, m_w), m_w <= j
      T* Cg = fb + (int64_t)(k + 1) * STAGE;
      const int cy = 3 * si.icnt[2];
      for (int q = tid; q < PC; q += kT3) {
        const int j = q / BP, i = q % BP;
        T c = T(0);
        // the lowest column row i couples to is 3 n - cy - 3: below it C vanishes
        if (i < si.bsz && j >= 3 * (i / 3) - cy - 3) {
          const int n = i / 3, y = n / si.icnt[2], z = n - y * si.icnt[2], base = 3 * n;
          const bool y0 = y > 0, y2 = y + 1 < si.icnt[1], z0 = z > 0, z2 = z + 1 < si.icnt[2];
          const T* Dj = D + (int64_t)j * BP;
#pragma unroll
          for (int w = 0; w < 27; ++w) {
            const int dy = w / 9 - 1, dz = (w / 3) % 3 - 1;
            const bool ok = (dy < 0 ? y0 : (dy > 0 ? y2 : true)) && (dz < 0 ? z0 : (dz > 0 ? z2 : true));
            const int m = base + dy * cy + 3 * dz + w % 3;
            if (ok && m <= j) c += anz[w * BP + i] * Dj[m];
          }
        }
        Cg[q] = c;
      }
    }
    __syncthreads();
  }
  if (tid == 0 && bad) {
    atomicExch(err, kErrPivot);
    atomicMin(bad_sub, sub);
  }
}

// K^(i) xloc at local closure node (a, b, c), component comp (3D).
template <typename T>
__device__ __forceinline__ T ebe_local3d(const T* ke, const T* sc, const T* xloc, int s, int a, int b,
                                         int c, int comp) {
  const int s1 = s + 1;
  T acc = T(0);
  for (int dx = 0; dx < 2; ++dx) {
    const int ea = a - dx;
    if (ea < 0 || ea >= s) continue;
    for (int dy = 0; dy < 2; ++dy) {
      const int eb = b - dy;
      if (eb < 0 || eb >= s) continue;
      for (int dz = 0; dz < 2; ++dz) {
        const int ec = c - dz;
        if (ec < 0 || ec >= s) continue;
        const T* krow = ke + (elem_local_node(dx, dy, dz) * 3 + comp) * 24;
        T part = T(0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          int ox, oy, oz;
          elem_node_offset(q, ox, oy, oz);
          const T* xn = xloc + (((ea + ox) * s1 + (eb + oy)) * s1 + (ec + oz)) * 3;
          part += krow[3 * q] * xn[0] + krow[3 * q + 1] * xn[1] + krow[3 * q + 2] * xn[2];
        }
        acc += sc[(ea * s + eb) * s + ec] * part;
      }
    }
  }
  return acc;
}

// ebe_local3d in double-float arithmetic: (hi, lo) += (K^(i) xloc) at local
// node (a, b, c), component comp (ke, sc, xloc as FP32 pairs).
__device__ __forceinline__ void ebe_local3d_df(const float2* ke, const float2* sc, const float2* xloc, int s,
                                               int a, int b, int c, int comp, float& hi, float& lo) {
  const int s1 = s + 1;
  for (int dx = 0; dx < 2; ++dx) {
    const int ea = a - dx;
    if (ea < 0 || ea >= s) continue;
    for (int dy = 0; dy < 2; ++dy) {
      const int eb = b - dy;
      if (eb < 0 || eb >= s) continue;
      for (int dz = 0; dz < 2; ++dz) {
        const int ec = c - dz;
        if (ec < 0 || ec >= s) continue;
        const float2* krow = ke + (elem_local_node(dx, dy, dz) * 3 + comp) * 24;
        float ph = 0.f, pl = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          int ox, oy, oz;
          elem_node_offset(q, ox, oy, oz);
          const float2* xn = xloc + (((ea + ox) * s1 + (eb + oy)) * s1 + (ec + oz)) * 3;
          df_mad(ph, pl, krow[3 * q], xn[0]);
          df_mad(ph, pl, krow[3 * q + 1], xn[1]);
          df_mad(ph, pl, krow[3 * q + 2], xn[2]);
        }
        df_mad(hi, lo, sc[(ea * s + eb) * s + ec], make_float2(ph, pl));
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kT3) schur3d_kernel(DevTables t, const T* __restrict__ Ke_g,
                                                      const T* __restrict__ scale,
                                                      const T* __restrict__ factor, SchurIO io) {
  if (io.done && *io.done) return;
  schur_pcg_prologue(io);
  const int BP = t.BP, PC = BP * BP, PD = BP * (BP + 1) / 2, STAGE = PC + PD;
  const int sub = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const SubInfo si = t.subs[sub];
  const int s = t.s, s1 = s + 1, nloc = s1 * s1 * s1;
  extern __shared__ __align__(128) unsigned char smem_raw3[];
  T* ybuf = reinterpret_cast<T*>(smem_raw3);  // nb_max * BP
  T* vbuf = ybuf + t.nb_max * BP;             // BP
  T* xloc = vbuf + BP;                        // 3 * nloc
  T* ke = xloc + 3 * nloc;                    // 576
  T* sc = ke + 576;                           // s^3
  for (int i = tid; i < 576; i += kT3) ke[i] = Ke_g[i];
  for (int i = tid; i < s * s * s; i += kT3) {
    const int a = i / (s * s), b = (i / s) % s, c = i % s;
    sc[i] = scale[((int64_t)(si.lo[0] + a) * t.ne[1] + si.lo[1] + b) * t.ne[2] + si.lo[2] + c];
  }
  for (int i = tid; i < 3 * nloc; i += kT3) xloc[i] = T(0);
  __syncthreads();
  const bool have_x = io.x != nullptr;
  if (have_x)
    for (int r = tid; r < si.n_ring; r += kT3)
      xloc[t.ring_loc[si.ring_off + r]] = (T)io.x[t.ring_gidx[si.ring_off + r]];
  __syncthreads();
  const int nb = si.nb;
  const T* fb = factor + si.factor_off;
  // forward: y_k = D_k (w_k - C_k y_{k-1})
  for (int k = 0; k < nb; ++k) {
    const T* Ck = fb + (int64_t)k * STAGE;
    const T* Dk = Ck + PC;
    for (int r = tid; r < BP; r += kT3) {
      T v = T(0);
      if (r < si.bsz) {
        int x, y, z, c;
        row_node3(si, k, r, x, y, z, c);
        const int64_t dof = 3 * node3(t, x, y, z) + c;
        if (!t.fixed[dof]) {
          if (io.f) v = (T)io.f[dof];
          if (have_x) v -= ebe_local3d<T>(ke, sc, xloc, s, x - si.lo[0], y - si.lo[1], z - si.lo[2], c);
        }
      }
      if (k > 0) {  // C_k(r, j) = 0 below column 3 (r / 3) - 3 icnt_2 - 3
        const T* yp = ybuf + (k - 1) * BP;
        for (int j = max(0, 3 * (r / 3) - 3 * si.icnt[2] - 3); j < BP; ++j) v -= Ck[(int64_t)j * BP + r] * yp[j];
      }
      vbuf[r] = v;
    }
    __syncthreads();
    for (int r = tid; r < BP; r += kT3) {
      T acc = T(0);
      for (int j = 0; j <= r; ++j) acc += Dk[j * BP - j * (j - 1) / 2 + (r - j)] * vbuf[j];
      ybuf[k * BP + r] = acc;
    }
    __syncthreads();
  }
  // backward: t_k = D_k^T (y_k - C_{k+1}^T t_{k+1}); one warp per output entry
  for (int k = nb - 1; k >= 0; --k) {
    const T* Dk = fb + (int64_t)k * STAGE + PC;
    const T* Cn = fb + (int64_t)(k + 1) * STAGE;
    for (int j = warp; j < BP; j += kT3 / 32) {
      T acc = T(0);
      if (k + 1 < nb) {
        const T* tn = ybuf + (k + 1) * BP;
        // C_{k+1}(r, j) = 0 for r > j + 3 icnt_2 + 5
        for (int r = lane; r < min(BP, j + 3 * si.icnt[2] + 6); r += 32) acc += Cn[(int64_t)j * BP + r] * tn[r];
      }
      acc = warp_sum(acc);
      if (lane == 0) vbuf[j] = ybuf[k * BP + j] - acc;
    }
    __syncthreads();
    for (int j = warp; j < BP; j += kT3 / 32) {
      const T* col = Dk + (j * BP - j * (j - 1) / 2);
      T acc = T(0);
      for (int i = j + lane; i < BP; i += 32) acc += col[i - j] * vbuf[i];
      acc = warp_sum(acc);
      if (lane == 0) ybuf[k * BP + j] = acc;
    }
    __syncthreads();
  }
  // outputs
  if (io.u_out || io.ring_out) {
    for (int k = 0; k < nb; ++k)
      for (int r = tid; r < si.bsz; r += kT3) {
        int x, y, z, c;
        row_node3(si, k, r, x, y, z, c);
        const int64_t dof = 3 * node3(t, x, y, z) + c;
        if (t.fixed[dof]) continue;
        const T tv = ybuf[k * BP + r];
        if (io.u_out) io.u_out[dof] = (double)tv;
        xloc[(((x - si.lo[0]) * s1 + (y - si.lo[1])) * s1 + (z - si.lo[2])) * 3 + c] = tv;
      }
    __syncthreads();
  }
  double d[1] = {0.0};
  if (io.ring_out) {
    T* out = reinterpret_cast<T*>(io.ring_out);
    for (int r = tid; r < si.n_ring; r += kT3) {
      const int loc = t.ring_loc[si.ring_off + r];
      const int node = loc / 3, c = loc % 3;
      const int a = node / (s1 * s1), b = (node / s1) % s1, cc = node % s1;
      const T y = ebe_local3d<T>(ke, sc, xloc, s, a, b, cc, c);
      out[t.ring_dst[si.ring_off + r]] = y;
      d[0] += (double)xloc[loc] * (double)y;
    }
  }
  __shared__ double red[kT3 / 32];
  schur_pcg_epilogue<kT3 / 32>(io, d[0], red);
}

// --- Double-float PCG apply --------------------------------------------------
// The FP64 operator of schur3d_kernel<double> with every product in
// double-float arithmetic on the FP32 pipes (the FP64 form keeps this GPU's
// FP64 pipe 84 % busy).  The factor is the stream-ordered copy of
// launch_build_df3 (no padding rows; a row-major copy for the backward sweep),
// read once per apply in the order of use with streaming (evict-first) loads.
// Each warp serves 16 rows: lanes l and l + 16 take the two halves of a row's
// dot product (coalesced over the rows) and add them by one shuffle; each
// thread keeps eight loads in flight ahead of its products.  (An L2 bulk prefetch of the next block step,
// 75 MB over all subdomains, evicted lines before their use: slower.)
constexpr int kT3D = 384;  // 12 warps x 16 rows: blocks of up to 192 rows in one pass
constexpr int kTriSlots = 4;  // chunks of a triangular pass

__host__ __device__ __forceinline__ int64_t pad16(int64_t v) { return (v + 15) & ~int64_t(15); }

// (hi, lo) += sum_{j = j0}^{j1 - 1} M[a_j] v[j] with a_{j0} = a, a_{j+1} = a_j + st_j,
// st_{j+1} = st_j + dst (dst 0: a strided column; -1, +1: the packed triangles).
// Software-pipelined: the loads of the next group of eight entries are issued
// before the products of the current group, so a thread always has loads in
// flight while it computes (the products of one row form a dependent chain).
__device__ __forceinline__ void df_dot(const float2* __restrict__ M, int a, int st, int dst,
                                       const float2* v, int j0, int j1, float& hi, float& lo) {
  constexpr int U = 8;
  int j = j0;
  if (j + U <= j1) {
    float2 e[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      e[u] = __ldcs(M + a);
      a += st;
      st += dst;
    }
    for (; j + 2 * U <= j1; j += U) {
      float2 nx[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        nx[u] = __ldcs(M + a);
        a += st;
        st += dst;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) df_mad(hi, lo, e[u], v[j + u]);
#pragma unroll
      for (int u = 0; u < U; ++u) e[u] = nx[u];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) df_mad(hi, lo, e[u], v[j + u]);
    j += U;
  }
  for (; j < j1; ++j) {
    df_mad(hi, lo, __ldcs(M + a), v[j]);
    a += st;
    st += dst;
  }
}

// Sum of the partials of lanes l and l ^ 16 (lanes 0-15 hold the result used).
__device__ __forceinline__ void df_half_sum(float& hi, float& lo) {
  const float ph = __shfl_xor_sync(0xffffffffu, hi, 16), pl = __shfl_xor_sync(0xffffffffu, lo, 16);
  df_add2(hi, lo, ph, pl);
}

__global__ void __launch_bounds__(kT3D, 3) schur3d_df_kernel(DevTables t, const double* __restrict__ Ke_g,
                                                             const double* __restrict__ scale,
                                                             const float2* __restrict__ factor,
                                                             const int64_t* __restrict__ off, SchurIO io) {
  if (io.done && *io.done) return;
  schur_pcg_prologue(io);
  const int sub = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int hh = lane >> 4, hl = lane & 15;
  const SubInfo si = t.subs[sub];
  const int s = t.s, s1 = s + 1, nloc = s1 * s1 * s1, NM = t.BP;
  const int n = si.bsz, nb = si.nb, cy = 3 * si.icnt[2];
  // triangular passes: kTriSlots column (forward) / row (backward) chunks of
  // width wc, chunk c serving the rows r >= c wc (forward) or the outputs
  // j < (c + 1) wc (backward)
  const int wc = (n + kTriSlots - 1) / kTriSlots;
  int tri_f = 0, tri_b = 0;  // work items of the forward and backward passes
  for (int c = 0; c * wc < n; ++c) {
    tri_f += n - c * wc;
    tri_b += min(n, (c + 1) * wc);
  }
  const int szC = (int)pad16((int64_t)n * n), szD = (int)pad16((int64_t)n * (n + 1) / 2);
  const float2* fw = factor + off[sub];
  const float2* bw = fw + (int64_t)nb * szD + (int64_t)(nb - 1) * szC;
  extern __shared__ __align__(128) unsigned char smem_df3[];
  float2* ybuf = reinterpret_cast<float2*>(smem_df3);  // nb_max * NM: w_k, then y_k, then t_k
  float2* vbuf = ybuf + t.nb_max * NM;                  // NM
  float2* xloc = vbuf + NM;                             // 3 * nloc
  float2* ke = xloc + 3 * nloc;                         // 576
  float2* sc = ke + 576;                                // s^3
  float2* part = sc + s * s * s;                        // kTriSlots * NM: triangular-pass partials
  for (int i = tid; i < 576; i += kT3D) ke[i] = df_from(Ke_g[i]);
  for (int i = tid; i < s * s * s; i += kT3D) {
    const int a = i / (s * s), b = (i / s) % s, c = i % s;
    sc[i] = df_from(scale[((int64_t)(si.lo[0] + a) * t.ne[1] + si.lo[1] + b) * t.ne[2] + si.lo[2] + c]);
  }
  for (int i = tid; i < 3 * nloc; i += kT3D) xloc[i] = make_float2(0.f, 0.f);
  __syncthreads();
  const bool have_x = io.x != nullptr;
  if (have_x)
    for (int r = tid; r < si.n_ring; r += kT3D)
      xloc[t.ring_loc[si.ring_off + r]] = df_from(io.x[t.ring_gidx[si.ring_off + r]]);
  __syncthreads();
  // w_k = f_I - K_IG x for every plane (K_IG x vanishes on rows with no
  // neighbour on the subdomain boundary)
  for (int q = tid; q < nb * n; q += kT3D) {
    const int k = q / n, r = q % n;
    int x, y, z, c;
    row_node3(si, k, r, x, y, z, c);
    const int64_t dof = 3 * node3(t, x, y, z) + c;
    float2 v = make_float2(0.f, 0.f);
    if (!t.fixed[dof]) {
      if (io.f) v = df_from(io.f[dof]);
      const int a = x - si.lo[0], b = y - si.lo[1], cz = z - si.lo[2];
      const bool near = a <= 1 || a >= s - 1 || b <= 1 || b >= s - 1 || cz <= 1 || cz >= s - 1;
      if (have_x && near) {
        float eh = 0.f, el = 0.f;
        ebe_local3d_df(ke, sc, xloc, s, a, b, cz, c, eh, el);
        df_add2(v.x, v.y, -eh, -el);
      }
    }
    ybuf[k * NM + r] = v;
  }
  __syncthreads();
  // forward: y_k = D_k (w_k - C_k y_{k-1})
  for (int k = 0; k < nb; ++k) {
    const float2* D = fw + (int64_t)k * (szC + szD);
    for (int r0 = 0; r0 < n; r0 += kT3D / 2) {
      const int rg = r0 + warp * 16, r = rg + hl;
      float ah = 0.f, al = 0.f;
      if (k > 0 && r < n) {
        // C_k(r, m) = 0 for m < 3 (r / 3) - cy - 3 (below the lowest node of
        // plane k - 1 that row r couples to): the 16 rows of this group read
        // the columns from their first row's bound on, two halves per row
        const int jl = max(0, 3 * (rg / 3) - cy - 3), jm = jl + (n - jl + 1) / 2;
        const int j0 = hh ? jm : jl, j1 = hh ? n : jm;
        df_dot(D - szC, j0 * n + r, n, 0, ybuf + (k - 1) * NM, j0, j1, ah, al);
      }
      df_half_sum(ah, al);
      if (r < n && hh == 0) {
        float2 w = ybuf[k * NM + r];
        df_add2(w.x, w.y, -ah, -al);
        vbuf[r] = w;
      }
    }
    __syncthreads();
    // triangular pass y_r = sum_{j <= r} D_k(r, j) v_j: column chunk c of
    // width wc for every row r >= c wc, consecutive threads on consecutive
    // rows of one chunk (coalesced); partials summed in chunk order
    for (int q = tid; q < tri_f; q += kT3D) {
      int c = 0, r = q;
      while (r >= n - c * wc) {
        r -= n - c * wc;
        ++c;
      }
      r += c * wc;
      const int j0 = c * wc, j1 = min(j0 + wc, r + 1);
      float ah = 0.f, al = 0.f;
      df_dot(D, j0 * n - j0 * (j0 - 1) / 2 + (r - j0), n - j0 - 1, -1, vbuf, j0, j1, ah, al);
      part[c * NM + r] = make_float2(ah, al);
    }
    __syncthreads();
    for (int r = tid; r < n; r += kT3D) {
      float2 y = part[r];
      for (int c = 1; c * wc <= r; ++c) df_add2(y.x, y.y, part[c * NM + r].x, part[c * NM + r].y);
      ybuf[k * NM + r] = y;
    }
    __syncthreads();
  }
  // backward: t_k = D_k^T (y_k - C_{k+1}^T t_{k+1}), one thread pair per output
  for (int k = nb - 1; k >= 0; --k) {
    const float2* Db = bw + (int64_t)(nb - 1 - k) * (szC + szD);
    for (int j0 = 0; j0 < n; j0 += kT3D / 2) {
      const int jg = j0 + warp * 16, j = jg + hl;
      float ah = 0.f, al = 0.f;
      if (k + 1 < nb && j < n) {
        // C_{k+1}(i, j) = 0 for i > j + cy + 5: the group's 16 outputs read
        // the rows up to its last output's bound, two halves per output
        const int ie = min(n, jg + cy + 21), im = (ie + 1) / 2;
        const int i0 = hh ? im : 0, i1 = hh ? ie : im;
        df_dot(Db - szC, i0 * n + j, n, 0, ybuf + (k + 1) * NM, i0, i1, ah, al);
      }
      df_half_sum(ah, al);
      if (j < n && hh == 0) {
        float2 w = ybuf[k * NM + j];
        df_add2(w.x, w.y, -ah, -al);
        vbuf[j] = w;
      }
    }
    __syncthreads();
    // triangular pass t_j = sum_{i >= j} D_k(i, j) v_i over the row-major
    // copy: row chunk c (rows [c wc, c wc + wc)) for every output j below its
    // end, consecutive threads on consecutive outputs (coalesced)
    for (int q = tid; q < tri_b; q += kT3D) {
      int c = 0, j = q;
      while (j >= min(n, (c + 1) * wc)) {
        j -= min(n, (c + 1) * wc);
        ++c;
      }
      const int i0 = max(j, c * wc), i1 = min(n, (c + 1) * wc);
      float ah = 0.f, al = 0.f;
      df_dot(Db, i0 * (i0 + 1) / 2 + j, i0 + 1, 1, vbuf, i0, i1, ah, al);
      part[c * NM + j] = make_float2(ah, al);
    }
    __syncthreads();
    for (int j = tid; j < n; j += kT3D) {
      const int c0 = j / wc;
      float2 y = part[c0 * NM + j];
      for (int c = c0 + 1; c * wc < n; ++c) df_add2(y.x, y.y, part[c * NM + j].x, part[c * NM + j].y);
      ybuf[k * NM + j] = y;
    }
    __syncthreads();
  }
  // outputs: t into the local closure, y = (K^(i) [t; x])_G on the ring
  if (io.u_out || io.ring_out) {
    for (int q = tid; q < nb * n; q += kT3D) {
      const int k = q / n, r = q % n;
      int x, y, z, c;
      row_node3(si, k, r, x, y, z, c);
      const int64_t dof = 3 * node3(t, x, y, z) + c;
      if (t.fixed[dof]) continue;
      const float2 tv = ybuf[k * NM + r];
      if (io.u_out) io.u_out[dof] = (double)tv.x + (double)tv.y;
      xloc[(((x - si.lo[0]) * s1 + (y - si.lo[1])) * s1 + (z - si.lo[2])) * 3 + c] = tv;
    }
    __syncthreads();
  }
  double d[1] = {0.0};
  if (io.ring_out) {
    double* out = reinterpret_cast<double*>(io.ring_out);
    for (int r = tid; r < si.n_ring; r += kT3D) {
      const int loc = t.ring_loc[si.ring_off + r];
      const int node = loc / 3, c = loc % 3;
      const int a = node / (s1 * s1), b = (node / s1) % s1, cc = node % s1;
      float yh = 0.f, yl = 0.f;
      ebe_local3d_df(ke, sc, xloc, s, a, b, cc, c, yh, yl);
      const double y = (double)yh + (double)yl;
      out[t.ring_dst[si.ring_off + r]] = y;
      d[0] += ((double)xloc[loc].x + (double)xloc[loc].y) * y;
    }
  }
  __shared__ double red[kT3D / 32];
  schur_pcg_epilogue<kT3D / 32>(io, d[0], red);
}

// FP64 factor (padded planes of launch_factor3d) -> the stream-ordered
// double-float copy; one CTA per subdomain.
__global__ void __launch_bounds__(256) build_df3_kernel(DevTables t, const double* __restrict__ factor,
                                                        const int64_t* __restrict__ off,
                                                        float2* __restrict__ out) {
  const SubInfo si = t.subs[blockIdx.x];
  const int BP = t.BP, PC = BP * BP, STAGE = PC + BP * (BP + 1) / 2;
  const int n = si.bsz, nb = si.nb;
  const int64_t szC = pad16((int64_t)n * n), szD = pad16((int64_t)n * (n + 1) / 2);
  float2* fw = out + off[blockIdx.x];
  float2* bw = fw + nb * szD + (nb - 1) * szC;
  const double* fb = factor + si.factor_off;
  for (int k = 0; k < nb; ++k) {
    const double* Ck = fb + (int64_t)k * STAGE;
    const double* Dk = Ck + PC;
    float2* Df = fw + k * (szC + szD);
    float2* Cf = Df - szC;
    float2* Db = bw + (nb - 1 - k) * (szC + szD);
    float2* Cb = bw + (nb - k) * (szC + szD) - szC;  // used by the backward step k - 1
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
      const int j = q / n, r = q % n;
      if (k > 0) {
        const float2 c = df_from(Ck[(int64_t)j * BP + r]);
        Cf[(int64_t)j * n + r] = c;
        Cb[(int64_t)r * n + j] = c;
      }
      if (r >= j) {
        const float2 d = df_from(Dk[(int64_t)j * BP - j * (j - 1) / 2 + (r - j)]);
        Df[(int64_t)j * n - j * (j - 1) / 2 + (r - j)] = d;
        Db[(int64_t)r * (r + 1) / 2 + j] = d;
      }
    }
  }
}

#include "ddel_ozaki.cuh"

// Tile policy of the FP64 3D factorisation's C_k C_k^T on the tensor cores:
// the product of plane k is taken from the assembled A_kk (element entries)
// and the result A_kk - C_k C_k^T written, both triangles, into the
// subdomain's scratch block A (row-major BP x BP), where factor3d_kernel
// picks it up.  W is the block C_k itself (its column-major storage is W^T
// row-major), sliced per row of C_k.
struct Factor3Tile {
  const double* Ke;
  const double* scale;
  double* work;
  int plane;
  static size_t smem(const DevTables&) { return 576 * 8; }
  __device__ int rows(const DevTables& t, const SubInfo& si) const {
    return plane >= 1 && plane < si.nb ? t.BP : 0;
  }
  __device__ void setup(const DevTables&, const SubInfo&, int, int, unsigned char* sm) const {
    double* ke = reinterpret_cast<double*>(sm);
    for (int i = threadIdx.x; i < 576; i += blockDim.x) ke[i] = Ke[i];
  }
  __device__ double value(const DevTables& t, const SubInfo& si, const unsigned char* sm, int gi, int gj, int,
                          int) const {
    return gi < t.BP && gj < t.BP
               ? entry3d<double>(t, si, reinterpret_cast<const double*>(sm), scale, plane, gi, plane, gj)
               : 0.0;
  }
  __device__ void store(const DevTables& t, const SubInfo&, int sub, int gi, int gj, double v) const {
    if (gi < t.BP && gj < t.BP) work[(int64_t)sub * 2 * t.BP * t.BP + (int64_t)gi * t.BP + gj] = v;
  }
};

}  // namespace

// The tensor-core product serves FP64 contexts with planes of up to 256 rows
// when asked for with tensor = 2.  It does not pay at these sizes: on
// 96 x 48 x 48 (160-row planes, 432 subdomains) it takes 3.9 ms per plane plus
// 0.55 ms of slicing against about 3 ms for the FP64-pipe product inside the
// fused kernel -- 135 bulk-copy steps of 32 KB for 1 M multiply-adds each
// (the 45 slice pairs of 3 chunks) leave the tensor cores waiting on L2.
static bool factor3d_tc(const DevTables& t, int precision, int tensor) {
  return tensor == 2 && precision == 0 && t.BP <= 256;
}
static int f3_nr(const DevTables& t) { return t.BP <= 128 ? 128 : 256; }
static int f3_kp(const DevTables& t) { return ((t.BP + 63) / 64) * 64; }
static size_t f3_slice_bytes(const DevTables& t) {
  const int Kp = f3_kp(t);
  return (size_t)t.n_sub * oz_slices(oz_bits(Kp), 54) * (f3_nr(t) / 128) * (Kp / 64) * 16384;
}

size_t factor3d_work_elems(const DevTables& t, int precision, int tensor) {
  size_t e = (size_t)t.n_sub * 2 * t.BP * t.BP;
  if (factor3d_tc(t, precision, tensor))  // slices and exponents of C_k (FP64 elements)
    e += (f3_slice_bytes(t) + (size_t)t.n_sub * f3_nr(t) * 4 + 256 + 7) / 8;
  return e;
}

int launch_factor3d(const DevTables& t, const DevFields& fld, int precision, void* factor, void* work, int* err,
                    int* bad_sub, int tensor, cudaStream_t st) {
  if (precision != 0) {
    factor3d_kernel<float><<<t.n_sub, kT3, 0, st>>>(t, t.Ke32, fld.scale32, (float*)factor, (float*)work, err,
                                                    bad_sub, 0, t.nb_max, 0);
    return 1;
  }
  if (!factor3d_tc(t, precision, tensor)) {
    factor3d_kernel<double><<<t.n_sub, kT3, 0, st>>>(t, t.Ke64, fld.scale64, (double*)factor, (double*)work, err,
                                                     bad_sub, 0, t.nb_max, 0);
    return 1;
  }
  // plane by plane: slices of C_k, A_kk - C_k C_k^T on the tensor cores
  // (FP64 accuracy), then the plane's Cholesky, inverse and C_{k+1}
  const int NR = f3_nr(t), Kp = f3_kp(t), S = oz_slices(oz_bits(Kp), 54);
  const int64_t PC = (int64_t)t.BP * t.BP, STAGE = PC + (int64_t)t.BP * (t.BP + 1) / 2;
  double* wd = reinterpret_cast<double*>(work);
  __nv_bfloat16* Wsl = reinterpret_cast<__nv_bfloat16*>(wd + (size_t)t.n_sub * 2 * PC);
  int* expo = reinterpret_cast<int*>(reinterpret_cast<char*>(Wsl) + f3_slice_bytes(t) + 128);
  const size_t sm = (size_t)kOzStages * 32768 + 2 * kOzTile * 4 + Factor3Tile::smem(t) + 64;
  int launches = 0;
  for (int k = 0; k < t.nb_max; ++k) {
    if (k > 0) {
      const OzSlab src{0, k * STAGE, t.BP, k, t.BP};
      launch_ozaki_slice<double>(dim3(t.n_sub, NR / 32), st, t, (const double*)factor, src, NR, Kp, Wsl, expo);
      const Factor3Tile tile{t.Ke64, fld.scale64, wd, k};
      if (NR == 128)
        ozaki_syrk_kernel<128, Factor3Tile><<<dim3(t.n_sub, 1), kOzThreads, sm, st>>>(t, tile, Wsl, expo, Kp, S, err);
      else
        ozaki_syrk_kernel<256, Factor3Tile><<<dim3(t.n_sub, 3), kOzThreads, sm, st>>>(t, tile, Wsl, expo, Kp, S, err);
      launches += 2;
    }
    factor3d_kernel<double><<<t.n_sub, kT3, 0, st>>>(t, t.Ke64, fld.scale64, (double*)factor, wd, err, bad_sub, k,
                                                     k + 1, 1);
    ++launches;
  }
  return launches;
}

size_t schur3d_smem(const DevTables& t, int precision);

int64_t df3_layout(const SubInfo* subs, int n_sub, int64_t* off) {
  int64_t tot = 0;
  for (int i = 0; i < n_sub; ++i) {
    const int64_t n = subs[i].bsz, nb = subs[i].nb;
    off[i] = tot;
    if (nb > 0) tot += 2 * (nb * pad16(n * (n + 1) / 2) + (nb - 1) * pad16(n * n));
  }
  return tot;
}

void launch_build_df3(const DevTables& t, const double* factor, const int64_t* off, float2* out,
                      cudaStream_t st) {
  build_df3_kernel<<<t.n_sub, 256, 0, st>>>(t, factor, off, out);
}

size_t schur3d_df_smem(const DevTables& t);

void launch_schur3d_df(const DevTables& t, const DevFields& fld, const float2* factor, const int64_t* off,
                       const SchurIO& io, cudaStream_t st) {
  schur3d_df_kernel<<<t.n_sub, kT3D, schur3d_df_smem(t), st>>>(t, t.Ke64, fld.scale64, factor, off, io);
}

size_t schur3d_df_smem(const DevTables& t) { return schur3d_smem(t, 0) + (size_t)kTriSlots * t.BP * 8; }

size_t schur3d_smem(const DevTables& t, int precision) {
  const int s = t.s, nloc = (s + 1) * (s + 1) * (s + 1);
  const size_t elems = (size_t)t.nb_max * t.BP + t.BP + 3 * nloc + 576 + s * s * s;
  return elems * (precision ? 4 : 8) + 16;
}

void launch_schur3d(const DevTables& t, const DevFields& fld, int precision, const void* factor,
                    const SchurIO& io, cudaStream_t st) {
  const size_t smem = schur3d_smem(t, precision);
  if (precision == 0)
    schur3d_kernel<double><<<t.n_sub, kT3, smem, st>>>(t, t.Ke64, fld.scale64,
                                                       (const double*)factor, io);
  else
    schur3d_kernel<float><<<t.n_sub, kT3, smem, st>>>(t, t.Ke32, fld.scale32, (const float*)factor,
                                                      io);
}

cudaError_t configure_kernels3d() {
  int dev = 0, big = 232448;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&big, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaError_t e = cudaSuccess;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, schur3d_df_kernel) == cudaSuccess) {
    cudaError_t e2 = cudaFuncSetAttribute(schur3d_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          big - (int)fa.sharedSizeBytes);
    if (e2 != cudaSuccess) e = e2;
  }
  for (auto k : {ozaki_syrk_kernel<128, Factor3Tile>, ozaki_syrk_kernel<256, Factor3Tile>})
    if (cudaFuncGetAttributes(&fa, k) == cudaSuccess) {
      cudaError_t e2 = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            big - (int)fa.sharedSizeBytes);
      if (e2 != cudaSuccess) e = e2;
    }
  if (cudaFuncGetAttributes(&fa, schur3d_kernel<double>) == cudaSuccess)
    e = cudaFuncSetAttribute(schur3d_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             big - (int)fa.sharedSizeBytes);
  if (cudaFuncGetAttributes(&fa, schur3d_kernel<float>) == cudaSuccess) {
    cudaError_t e2 = cudaFuncSetAttribute(schur3d_kernel<float>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          big - (int)fa.sharedSizeBytes);
    if (e2 != cudaSuccess) e = e2;
  }
  return e;
}

}  // namespace ddel
