// Kernel launchers (host functions) shared by the API translation unit.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ddel_internal.h"

namespace ddel {

// Device-resident copy of the static tables of a Setup.
struct DevTables {
  int dim, s, n_sub, BP, nb_max;
  int ne[3], nn[3];
  int64_t n_dof, n_elem, n_gamma;
  int n_face_dofs, n_blocks, max_blk_n;
  int upd_lanes;    // lanes per face block in the PCG update (power of two >= max_blk_n, <= 32)
  int upd_stage_p;  // 1: the update kernel stages face tables in shared memory
  SubInfo* subs;
  uint8_t* fixed;
  int32_t* ring_gidx;
  int32_t* ring_loc;
  int64_t n_ring;
  int32_t* owner_ptr;
  int32_t* owner_idx;
  int32_t* owner_pad;  // n_gamma x max_owners, -1 padded (16-byte aligned rows in 2D)
  // Ring entries are stored owner-major: the contribution of ring slot q lives
  // at ring[ring_dst[q]] = ring[g * max_owners + k]; a Gamma DOF reads its
  // max_owners entries contiguously (unused entries hold 0).
  int32_t* ring_dst;
  int max_owners;
  int64_t* gamma_dof;
  int32_t* blk_off;
  int32_t* blk_n;
  int32_t* blk_poff;
  double* blk_hmean;
  double* hdiag;  // n_face_dofs: diag(H_f)
  double* ptab;
  float2* ptab_df;  // ptab as FP32 (hi, lo) pairs for the double-float preconditioner product
  double* Ke64;
  float* Ke32;
};

// PCG state kept on the device (read by the host only at check points).
// Chronopoulos-Gear form of PCG: gamma = (r, u), delta = (S u, u) with
// u = S~^-1 r; one Schur apply and one update kernel per iteration.  Grid-wide
// sums have no single-block tail: every block of a kernel writes its partial
// sums, and every block of the next kernel reduces them itself in a fixed
// order (all blocks obtain bitwise the same totals), so each kernel starts
// with the scalars it needs.  Iteration j: the Schur kernel reads kS = j and
// records kU = j; the update kernel reads kU, stores 1/alpha_j, 1/gamma_j in
// slot j & 1 and sets kS = j + 1; the update partials are double-buffered by
// parity (the buffers are kernel arguments).
constexpr int kMaxCoarse = 8;
constexpr int kPcgRows = 2 + 2 * kMaxCoarse;  // gamma, rr, Q^T r (k), (S Q)^T u^ (k)

struct PcgState {
  double tol2, rr;
  int it, max_it, done, status;
  int kS, kU;
  double ainv_s[2], ginv_s[2];  // 1 / alpha_j and 1 / gamma_j in slot j & 1
  unsigned ticket[4];
  double* partials;  // scratch of grid_sum-based one-off kernels
  double c0[kMaxCoarse];  // coefficients of the initial guess x0 = Q c0
  int x0_used;
  int replaced_ok;  // relaxed PCG: the last reliable update met the tolerance
};

// Coarse space of the interface PCG: orthonormal Q (k columns of n_gamma,
// column-major), S Q, E^-1 = (Q^T S Q)^-1 and G = (S Q)^T (S Q), k x k
// row-major with leading dimension kMaxCoarse.
struct CoarseDev {
  const double* Q = nullptr;
  const double* SQ = nullptr;
  const double* Einv = nullptr;
  const double* E = nullptr;  // Q^T S Q (as formed; symmetrised where used)
  const double* G = nullptr;
  int k = 0;
  int correct = 1;  // 0: initial guess only; 1: additive correction; 2: deflation
  int x0 = 1;       // start from the Galerkin guess Q c0 (else from 0)
};

// Per-assembly fields.
struct DevFields {
  double* scale64;  // n_elem: E rho^p
  float* scale32;
  double* diagG;    // n_gamma: diag(K_GG)
  double* blk_alpha;
  double* face_w;       // n_face_dofs: S~_f^-1 = W^-1 H_f^-1 W^-1; stores 1 / W_ii
  double* cross_scale;  // n_gamma - n_face_dofs
};

struct SchurIO {
  const double* x = nullptr;      // Gamma input (nullptr = 0)
  const double* f = nullptr;      // global right-hand side for the interior (nullptr = 0)
  void* ring_out = nullptr;       // per ring slot output (T), nullptr = skip
  double* u_out = nullptr;        // global vector, interior DOFs written, nullptr = skip
  const int* done = nullptr;      // early exit flag
  PcgState* pcg = nullptr;        // PCG form: also write this block's share of delta = (S u, u)
  double* pd = nullptr;           // PCG form: the delta partials (one per block)
  int* err = nullptr;
};

// Opt-in shared memory sizes for every kernel instantiation (call once).
cudaError_t configure_kernels();

// Assembly: element factors from densities, diag(K_GG), face scales.
void launch_assemble(const DevTables& t, const DevFields& fld, const double* rho, double E, double p,
                     int face_scaling, int crosspoint_mode, int* err, cudaStream_t st);
// Fused interior assembly + block-tridiagonal Cholesky; factor in T.  work:
// 3D scratch of factor3d_work_elems() elements of the precision (unused in 2D).
// tensor: FP64 3D planes take C_k C_k^T on the tensor cores.  Returns the
// number of kernel launches.
int launch_factor(const DevTables& t, const DevFields& fld, int precision, void* factor, void* work,
                  int* err, int* bad_sub, int tensor, cudaStream_t st);
// 3D path (ddel_kernels3d.cu)
size_t factor3d_work_elems(const DevTables& t, int precision, int tensor);
int launch_factor3d(const DevTables& t, const DevFields& fld, int precision, void* factor, void* work, int* err,
                    int* bad_sub, int tensor, cudaStream_t st);
void launch_schur3d(const DevTables& t, const DevFields& fld, int precision, const void* factor,
                    const SchurIO& io, cudaStream_t st);
// FP64 operator in double-float arithmetic on a stream-ordered copy of the
// FP64 factor as FP32 (hi, lo) pairs: per subdomain (n = bsz rows per plane, nb
// planes, blocks padded to 16 pairs) the forward sweep's blocks D_0, C_1, D_1,
// ..., C_{nb-1}, D_{nb-1} (C column-major n x n, D packed lower column-major),
// then the backward sweep's D_{nb-1}, C_{nb-1}, D_{nb-2}, ..., C_1, D_0 (C
// row-major, D packed lower row-major), so that both sweeps read it in order
// with one thread per output row.  df3_layout fills the per-subdomain offsets
// (n_sub entries) and returns the total number of pairs.
int64_t df3_layout(const SubInfo* subs, int n_sub, int64_t* off);
void launch_build_df3(const DevTables& t, const double* factor, const int64_t* off, float2* out,
                      cudaStream_t st);
void launch_schur3d_df(const DevTables& t, const DevFields& fld, const float2* factor, const int64_t* off,
                       const SchurIO& io, cudaStream_t st);
cudaError_t configure_kernels3d();
// Per-subdomain solve kernel (condense / Schur / back-substitution forms).
void launch_schur(const DevTables& t, const DevFields& fld, int precision, const void* factor,
                  const SchurIO& io, cudaStream_t st);
size_t schur_smem_bytes(const DevTables& t, int precision);
// Explicit local Schur complements (2D, ring size NR <= 256): formation after the
// factorisation, and the batched dense apply used inside PCG.
int explicit_ring_size(const DevTables& t);
// work: scratch of explicit_form_work_elems() elements of the precision (the
// per-plane W = L^-1 K_IG of the NR = 256 formation; 0 otherwise).  df (FP64,
// rings up to 128): every product and sum of the formation in double-float
// arithmetic on the FP32 pipes (about 48 significant bits), S_i still stored
// in FP64.
size_t explicit_form_work_elems(const DevTables& t);
void launch_schur_form(const DevTables& t, const DevFields& fld, int precision, bool df, const void* factor,
                       void* work, void* Sexp, cudaStream_t st);
// Tensor-core formation (rings of 128 and 256): W = L^-1 K_IG in the
// factor's precision into work (explicit_form_work_elems elements), then
// S_i = K_GG - W^T W with the product on tcgen05 from the Ozaki splitting of
// W into BF16 slices (tc_work: tensor_form_work_bytes) -- to FP64 accuracy
// (precision 0) or to the 24 bits of the FP32 operator (precision 1).  err: kErrTimeout if a bounded
// wait on the tensor-core completion ran out.
bool tensor_form_available(const DevTables& t);
size_t tensor_form_work_bytes(const DevTables& t);
void launch_schur_form_tc(const DevTables& t, const DevFields& fld, int precision, const void* factor, void* work,
                          void* tc_work, void* Sexp, int* err, cudaStream_t st);
// Double-float form: S_i split into FP32 (hi, lo) pairs; the apply runs on the
// FP32 pipes with about 48 significant bits (ring output FP64).
void launch_split_df(const double* in, float2* out, int64_t n, cudaStream_t st);
// Returns the number of blocks; split as for launch_schur_explicit.
int launch_schur_explicit_df(const DevTables& t, const float2* Sexp, const SchurIO& io, int split,
                             cudaStream_t st);
// Returns the number of blocks (one delta partial each); split: CTAs per
// subdomain of the native FP64 form (1, 2 or 4; others mean 2).
int launch_schur_explicit(const DevTables& t, int precision, const void* Sexp, const SchurIO& io, int split,
                          cudaStream_t st);
int explicit_split(const DevTables& t, int split);
// Sum ring contributions: out[g] = sign * sum(ring) + (base ? base[gamma_dof[g]] : 0)
void launch_gamma_sum(const DevTables& t, int precision, const void* ring, const double* base,
                      double sign, double* out, cudaStream_t st);
// PCG kernels (Chronopoulos-Gear form).  init: x = 0, r = g, p = s = 0,
// u = S~^-1 r, gamma.  update: w = sum(ring), p = u + beta p, s = w + beta s,
// x += alpha p, r -= alpha s, u = S~^-1 r, gamma; convergence test.
// With a coarse space (cd.k > 0) the preconditioner is S~^-1 r + Q E^-1 Q^T r
// (u keeps the face-local part; the coarse part lives in PcgState::cc), and
// init starts from x0 = Q c0 (PcgState::c0, set by launch_coarse_x0).
// pu_out: the update partials written (kPcgRows x nblk).
void launch_pcg_init(const DevTables& t, const DevFields& fld, const double* g, double* x, double* r,
                     double* u, double* p, double* sv, PcgState* s, double* pu_out, cudaStream_t st,
                     int nblk, const CoarseDev& cd = CoarseDev());
// Reliable update of the relaxed mixed-precision PCG (no coarse space), after
// a whole batch of iterations and an accurate Schur apply of x into the FP64
// ring: r = g - S x, u = S~^-1 r and its partials (x, p, s kept), then the
// step-length correction, the true rr and replaced_ok = (rr <= tol2) in the
// state.  Nothing changes once the state is done (an error status).  Two
// launches.
void launch_pcg_replace(const DevTables& t, const DevFields& fld, const double* g, const double* ring, double* x,
                        double* r, double* u, double* p, double* sv, PcgState* s, double* pu_out, cudaStream_t st,
                        int nblk, double tol2);
// Update j: pd holds the nd delta partials of the Schur kernel, pu_in the
// update partials of iteration j (written by update j-1 or init), pu_out
// receives those of j + 1; par = j & 1 (recurrence scalar slots).  Passing
// them as arguments keeps a dependent load off the start of the kernel.
void launch_pcg_update(const DevTables& t, const DevFields& fld, int precision, const void* ring,
                       double* x, double* r, double* u, double* p, double* sv, PcgState* s,
                       const double* pd, int nd, const double* pu_in, double* pu_out, int par,
                       cudaStream_t st, int nblk, const CoarseDev& cd = CoarseDev());
// Batched persistent PCG: one problem of a batch (the double-float explicit
// form, no coarse space).  The kernel runs `iters` PCG iterations of every
// problem in one launch: a device work queue hands out, in order, per
// iteration the Schur blocks of every problem and then their update blocks
// (the blocks of schur_explicit_df_kernel and pcg_update_kernel, computing
// exactly what those kernels compute); a block waits, bounded, until the
// blocks its problem's phase depends on have completed (per-problem
// counters).  pre: prefix sums of the problems' Schur tiles, then of their
// update blocks.  cnt: 2 counters per problem, the queue head and an abort
// flag, zeroed before each launch.
struct BatchProb {
  DevTables t;
  DevFields f;
  const float2* sexp_df;
  double* ring;
  double *x, *r, *u, *p, *sv;
  PcgState* st;
  double* pd;
  double* pu;       // 2 x kPcgRows x n_upd partials (by iteration parity)
  int nr;           // ring size of the explicit form (64, 128 or 256)
  int n_schur;      // Schur blocks (2 per subdomain)
  int n_upd;        // update blocks
  int pad;
};
// Blocks per SM of the persistent kernel for the given dynamic shared memory.
int batch_pcg_blocks_per_sm(size_t smem);
size_t batch_pcg_smem(const DevTables& t);
// Queue tiles of a problem's Schur phase (several Schur blocks per tile).
int batch_schur_tiles(int n_schur_blocks);
cudaError_t launch_batch_pcg(const BatchProb* probs, int nprob, const int* pre, int iters, unsigned* cnt,
                             int* err, int grid, size_t smem, cudaStream_t st);

// Coarse-space set-up (ddel_coarse.cu).  Gram matrix out = A^T B (k x k,
// leading dimension kMaxCoarse) of k <= kMaxCoarse columns of length n.
void launch_gram(const double* A, const double* B, int k, int64_t n, double* out, double* partials,
                 unsigned* ticket, cudaStream_t st);
// Cholesky QR step on the Gram matrix G of k columns: T (k x k) with Z T
// orthonormal, columns whose pivot falls below drop * max pivot removed;
// *k_out = number kept.
void launch_cholqr_factor(const double* G, int k, double drop, double* T, int* k_out, cudaStream_t st);
// out (k_out columns) = Z (k columns) T
void launch_apply_T(const double* Z, const double* T, int k, const int* k_out, int64_t n, double* out,
                    cudaStream_t st);
// E = Q^T S Q (symmetrised) -> Einv, and flag = 1 when E is SPD (else 0).
void launch_coarse_invert(const double* E, int k, double* Einv, int* flag, cudaStream_t st);
// c0 = E^-1 Q^T g, or 0 when ||g - S Q c0|| > ||g|| (PcgState::x0_used).
void launch_coarse_x0(const CoarseDev& cd, const double* g, int64_t n, PcgState* s, cudaStream_t st);
void launch_precond(const DevTables& t, const DevFields& fld, const double* r, double* z,
                    cudaStream_t st);
// Global element-by-element product / residual in FP64 (node-centric, no atomics).
// mode 0: y = K x (free rows); mode 1: y = f - K x (free rows), norms into nrm[0..1]
void launch_apply_K(const DevTables& t, const DevFields& fld, const double* x, const double* f,
                    double* y, int mode, double* partials, unsigned* ticket, double* nrm,
                    cudaStream_t st, int nblk);
// u[gamma_dof[g]] = xg[g]; u = 0 on fixed DOFs
void launch_scatter_gamma(const DevTables& t, const double* xg, double* u, cudaStream_t st);
// out = (float) in, n elements
void launch_round_f32(const double* in, float* out, int64_t n, cudaStream_t st);
// y += a * x (n)
void launch_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t st);

}  // namespace ddel
