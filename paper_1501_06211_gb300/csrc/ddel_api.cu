// C ABI of libddel (declared in include/ddel.h): context life cycle, device
// memory, the solve driver (eq. 3MatSplit2 + interface PCG + FP64 iterative
// refinement) and the step-level entry points.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ddel.h"
#include "../../include/ddel_learn.h"
#include "ddel_internal.h"
#include "ddel_globalprec.h"
#include "ddel_launch.h"
#include "ddel_topopt.h"

using namespace ddel;

struct ddel_ctx {
  Setup S;
  DevTables T{};
  DevFields F{};
  ddel_mesh mesh{};
  ddel_material mat{};
  ddel_options opt{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<void*> allocs;
  void* factor[2] = {nullptr, nullptr};
  void* work3d[2] = {nullptr, nullptr};  // 3D factorisation scratch
  size_t work3d_bytes[2] = {0, 0};
  void* sexp[2] = {nullptr, nullptr};  // explicit local Schur complements (2D)
  void* form_work[2] = {nullptr, nullptr};  // W = L^-1 K_IG scratch of the widest rings
  void* tc_work = nullptr;             // BF16 slices of W and column exponents (tensor-core formation)
  float* sexp32 = nullptr;             // MIXED: FP64-formed S_i rounded to FP32
  bool mixed_ready = false;
  float2* sexp_df = nullptr;           // FP64 S_i as FP32 (hi, lo) pairs (double-float apply)
  bool df_ok = false;
  float2* factor_df = nullptr;         // 3D: FP64 factor as FP32 pairs (double-float apply)
  int64_t* df3_off = nullptr;          // 3D: per-subdomain offsets into factor_df
  bool df3_ok = false;
  bool graph_df = false;
  bool pending_explicit = false;
  bool explicit_ok[2] = {false, false};
  bool factored[2] = {false, false};
  int active_prec = 0;
  bool assembled = false;
  // owner-major ring buffers, one per precision: their zero padding must not see
  // writes of the other element size
  void* ring = nullptr;    // FP64
  void* ring32 = nullptr;  // FP32
  double *d_f = nullptr, *d_load = nullptr, *d_u = nullptr, *d_r = nullptr, *d_d = nullptr;
  double *g = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  double* sv = nullptr;  // s = S p of the Chronopoulos-Gear recurrence
  double* rho = nullptr;
  PcgState* st = nullptr;
  PcgState* h_st = nullptr;
  double* partials = nullptr;
  double* pcg_pd = nullptr;  // PCG partial sums: Schur kernel (delta), update kernel (2 parities)
  double* pcg_pu = nullptr;
  unsigned* ticketK = nullptr;
  double* nrm = nullptr;
  double* h_nrm = nullptr;
  int* err = nullptr;
  int* bad_sub = nullptr;
  int* h_err = nullptr;
  int nblk = 0;
  int nupd = 0;  // blocks of the PCG init / update kernels (their partial-sum count)
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool graph_explicit[2] = {false, false};
  bool graph_apply32[2] = {false, false};
  int graph_iters = 0;
  // relaxed MIXED PCG: iterations with the FP32-stored S_i (FP64 factors, no
  // coarse space), captured beside graph[0]
  cudaGraphExec_t graph_lo = nullptr;
  int graph_lo_iters = 0, graph_lo_split = 0;
  int64_t launches = 0;           // kernel launches issued (graph-contained ones included)
  int64_t launches_at_assemble = 0;
  cudaEvent_t ev[11] = {};        // [8], [9]: around the last ddel_factor; [7], [10]: PCG state copies
  double t_factor_ms = 0.0;       // device time of the last ddel_factor (with S_i formation)
  // topology optimisation buffers (allocated on first use)
  double *rho_f = nullptr, *dcf = nullptr, *dc = nullptr, *dv = nullptr, *topo_u = nullptr;
  double* topo_out = nullptr;    // device: lambda, volume, change, compliance
  double* h_topo = nullptr;      // pinned copy
  double dv_rmin = -1.0;         // filter radius dv was computed for
  // coarse space of the interface PCG (ddel_set_coarse; allocated on first use)
  double *cZ = nullptr, *cQ1 = nullptr, *cQ = nullptr, *cSQ = nullptr;
  double* csmall = nullptr;      // 6 k x k blocks: G1 T1 G2 T2 E Einv | Gsq
  int* cflags = nullptr;         // k after pass 1, k after pass 2, E SPD
  unsigned* cticket = nullptr;
  int* h_cflags = nullptr;
  int ck_in = 0;                 // columns given
  int ck = 0;                    // usable coarse dimension (0: plain PCG)
  int coarse_flags = 0;          // DDEL_COARSE_* bits
  int coarse_prec = -1;          // precision whose S formed E (-1: stale)
  int graph_ck[2] = {0, 0};      // coarse dimension captured in graph[prec]
  int graph_split[2] = {0, 0};   // CTAs per subdomain of the FP64 explicit apply captured
  bool u_valid = false;          // d_u holds a converged solution (x0_mode WARM)
  // global interface preconditioner and full-system FGMRES (first use)
  GPDev gp{};
  int gp_state = 0;               // 0 not built, 1 ready, -1 singular interface Laplacian
  double* gp_out = nullptr;       // device: Lanczos record of the last application
  double* h_gp_out = nullptr;     // pinned copy
  double *gm_V = nullptr, *gm_Z = nullptr, *gm_w = nullptr, *gm_h = nullptr, *gm_part = nullptr;
  double *gm_vg = nullptr, *gm_zg = nullptr, *h_gm = nullptr;
  int gm_cap = 0;                 // iterations the FGMRES buffers hold
  std::vector<ddel_learner*> learners;  // attached learners (detached on destroy)
  std::string last_error;
};

namespace ddel {
cudaStream_t ctx_stream(const ddel_ctx* ctx) { return ctx->stream; }
ddel_mesh ctx_mesh(const ddel_ctx* ctx) { return ctx->mesh; }
void ctx_attach_learner(ddel_ctx* ctx, ddel_learner* L) { ctx->learners.push_back(L); }
void ctx_detach_learner(ddel_ctx* ctx, ddel_learner* L) {
  auto& v = ctx->learners;
  v.erase(std::remove(v.begin(), v.end(), L), v.end());
}
void learner_context_gone(ddel_learner* L);  // ddel_learner.cu
}  // namespace ddel

namespace {

std::string g_create_error;  // message of the last failed ddel_create (ddel_last_error(NULL))

int fail(ddel_ctx* c, int code, const std::string& msg) {
  if (c) c->last_error = msg;
  return code;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(ctx, DDEL_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename P>
cudaError_t dalloc(ddel_ctx* ctx, P** p, size_t bytes) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, bytes < 16 ? 16 : bytes);
  if (e == cudaSuccess) {
    ctx->allocs.push_back(v);
    *p = static_cast<P*>(v);
  }
  return e;
}

template <typename V>
cudaError_t upload(ddel_ctx* ctx, const std::vector<V>& h, V** d) {
  cudaError_t e = dalloc(ctx, d, h.size() * sizeof(V));
  if (e != cudaSuccess) return e;
  if (!h.empty()) e = cudaMemcpy(*d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice);
  return e;
}

// Kernel-side PCG configuration: tolerance from the device-resident norms.
__global__ void set_tol_kernel(PcgState* st, const double* nrm, double tol, double inner_tol,
                               int mixed, int max_it) {
  const double fnorm = nrm[1], rnorm = nrm[0];
  double t = 0.5 * tol * fnorm;
  if (mixed) t = fmax(t, inner_tol * rnorm);
  st->tol2 = t * t;
  st->max_it = max_it;
  st->done = 0;
  st->status = 0;
  st->it = 0;
  st->replaced_ok = 0;
}

__global__ void set_tol_abs_kernel(PcgState* st, double tol_abs, int max_it) {
  st->tol2 = tol_abs * tol_abs;
  st->max_it = max_it;
  st->done = 0;
  st->status = 0;
  st->it = 0;
}

int check_kernel_err(ddel_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->h_err, ctx->err, 4 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return DDEL_OK;
}

void* ring_of(ddel_ctx* ctx, int prec) { return prec ? ctx->ring32 : ctx->ring; }

SchurIO make_io(ddel_ctx* ctx) {
  SchurIO io;
  io.err = ctx->err;
  return io;
}

// The Schur apply that the PCG of precision prec uses (double-float explicit,
// explicit, or implicit block substitution), into the ring of that precision.
int apply_prec(ddel_ctx* ctx, int prec, bool apply32) {
  const bool expl = ctx->explicit_ok[prec];
  return expl ? (apply32 ? 1 : prec) : prec;
}

// Returns the number of blocks launched (one delta partial each in a PCG).
int schur_dispatch(ddel_ctx* ctx, int prec, bool apply32, SchurIO& io, cudaStream_t s) {
  const bool expl = ctx->explicit_ok[prec];
  io.ring_out = ring_of(ctx, apply_prec(ctx, prec, apply32));
  const void* smat = apply32 ? (const void*)ctx->sexp32 : ctx->sexp[prec];
  if (expl && prec == 0 && !apply32 && ctx->df_ok)
    return launch_schur_explicit_df(ctx->T, ctx->sexp_df, io, ctx->opt.schur_split, s);
  if (expl) return launch_schur_explicit(ctx->T, apply32 ? 1 : prec, smat, io, ctx->opt.schur_split, s);
  if (ctx->T.dim == 3 && prec == 0 && !apply32 && ctx->df3_ok)
    launch_schur3d_df(ctx->T, ctx->F, ctx->factor_df, ctx->df3_off, io, s);
  else
    launch_schur(ctx->T, ctx->F, prec, ctx->factor[prec], io, s);
  return ctx->T.n_sub;
}

CoarseDev coarse_dev(ddel_ctx* ctx) {
  CoarseDev cd;
  if (ctx->ck <= 0) return cd;
  const int KK = kMaxCoarse * kMaxCoarse;
  cd.Q = ctx->cQ;
  cd.SQ = ctx->cSQ;
  cd.Einv = ctx->csmall + 5 * KK;
  cd.E = ctx->csmall + 4 * KK;
  cd.G = ctx->csmall + 6 * KK;
  cd.k = ctx->ck;
  cd.correct = (ctx->coarse_flags & DDEL_COARSE_CORRECT) ? 1 : (ctx->coarse_flags & DDEL_COARSE_DEFLATE) ? 2 : 0;
  cd.x0 = (ctx->coarse_flags & DDEL_COARSE_X0) ? 1 : 0;
  return cd;
}

// Iterations issued between host checks: even, so that the parity of the
// double-buffered partial sums repeats across graph launches.
int pcg_per(const ddel_ctx* ctx) {
  const int per = ctx->opt.check_every > 0 ? ctx->opt.check_every : 16;
  return per + (per & 1);
}

double* pcg_partials(ddel_ctx* ctx, int par) { return ctx->pcg_pu + (size_t)par * kPcgRows * ctx->nupd; }

// One PCG iteration: w = S u (ring) with the partials of delta = (S u, u);
// then alpha, beta, the vector updates and u = S~^-1 r (+ the coarse part)
// with the partials of gamma = (r, u).  par = iteration parity.
void pcg_iteration(ddel_ctx* ctx, int prec, bool apply32, int par) {
  cudaStream_t s = ctx->stream;
  const CoarseDev cd = coarse_dev(ctx);
  SchurIO io = make_io(ctx);
  io.x = ctx->z;
  io.done = &ctx->st->done;
  io.pcg = ctx->st;
  io.pd = ctx->pcg_pd;
  const int nd = schur_dispatch(ctx, prec, apply32, io, s);
  launch_pcg_update(ctx->T, ctx->F, apply_prec(ctx, prec, apply32), io.ring_out, ctx->x, ctx->r,
                    ctx->z, ctx->p, ctx->sv, ctx->st, ctx->pcg_pd, nd, pcg_partials(ctx, par),
                    pcg_partials(ctx, par ^ 1), par, s, ctx->nupd, cd);
}

// PCG initialisation (asynchronous) and, with use_graph, the CUDA graph of
// check_every iterations for this precision and form.
int pcg_start(ddel_ctx* ctx, int prec, const double* g, bool apply32) {
  cudaStream_t s = ctx->stream;
  const CoarseDev cd = coarse_dev(ctx);
  if (cd.k > 0 && cd.x0) {
    launch_coarse_x0(cd, g, ctx->T.n_gamma, ctx->st, s);
    ctx->launches += 1;
  }
  launch_pcg_init(ctx->T, ctx->F, g, ctx->x, ctx->r, ctx->z, ctx->p, ctx->sv, ctx->st, pcg_partials(ctx, 0), s,
                  ctx->nupd, cd);
  ctx->launches += 1;
  const int per = pcg_per(ctx);
  const bool expl = ctx->explicit_ok[prec];
  const bool df = prec == 0 && ctx->df_ok;
  const int gck = cd.k > 0 && cd.correct ? cd.k : 0;
  const int gsplit = explicit_split(ctx->T, ctx->opt.schur_split);
  if (ctx->graph[prec] && (ctx->graph_explicit[prec] != expl || ctx->graph_apply32[prec] != apply32 ||
                           ctx->graph_iters != per || (prec == 0 && ctx->graph_df != df) ||
                           ctx->graph_ck[prec] != gck || ctx->graph_split[prec] != gsplit)) {
    cudaGraphExecDestroy(ctx->graph[prec]);
    ctx->graph[prec] = nullptr;
  }
  if (ctx->opt.use_graph && !ctx->graph[prec]) {
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < per; ++i) pcg_iteration(ctx, prec, apply32, i & 1);
    CK(cudaStreamEndCapture(s, &graph));
    CK(cudaGraphInstantiate(&ctx->graph[prec], graph, 0));
    cudaGraphDestroy(graph);
    ctx->graph_iters = per;
    ctx->graph_explicit[prec] = expl;
    ctx->graph_apply32[prec] = apply32;
    ctx->graph_ck[prec] = gck;
    ctx->graph_split[prec] = gsplit;
    if (prec == 0) ctx->graph_df = df;
  }
  return DDEL_OK;
}

// Issues check_every iterations and the copy of the PCG state to the host
// into h_st[slot] (asynchronous; ctx->ev[7] for slot 0, ctx->ev[10] for slot
// 1, is recorded after the copy).  lo_graph: the relaxed PCG's FP32 graph.
int pcg_issue(ddel_ctx* ctx, int prec, bool apply32, int slot = 0, bool lo_graph = false) {
  cudaStream_t s = ctx->stream;
  const int per = pcg_per(ctx);
  if (ctx->opt.use_graph) {
    CK(cudaGraphLaunch(lo_graph ? ctx->graph_lo : ctx->graph[prec], s));
  } else {
    for (int i = 0; i < per; ++i) pcg_iteration(ctx, prec, apply32, i & 1);
  }
  ctx->launches += 2 * per;
  CK(cudaMemcpyAsync(ctx->h_st + slot, ctx->st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(ctx->ev[slot ? 10 : 7], s));
  return DDEL_OK;
}

// Batches of `per` iterations until the state read back says done.  The next
// batch is issued before the state of the current one is read (two in
// flight, their states in h_st[0] / h_st[1]), so the GPU does not idle while
// the host waits and decides; a batch issued after convergence exits at once
// in every kernel (the done flag) and leaves the state as it was.  The final
// state ends in h_st[0].
int pcg_run(ddel_ctx* ctx, int prec, const double* g, int* iters, int* status,
            bool apply32 = false) {
  int rc = pcg_start(ctx, prec, g, apply32);
  if (rc) return rc;
  const int per = pcg_per(ctx);
  const int max_checks = ctx->opt.max_it / per + 2;
  rc = pcg_issue(ctx, prec, apply32, 0);
  if (rc) return rc;
  int issued = 1, last = 0;
  for (int chk = 0; chk < max_checks; ++chk) {
    if (issued < max_checks) {
      rc = pcg_issue(ctx, prec, apply32, issued & 1);
      if (rc) return rc;
      ++issued;
    }
    last = chk & 1;
    CK(cudaEventSynchronize(ctx->ev[last ? 10 : 7]));
    if (ctx->h_st[last].done) break;
  }
  // no state copy stays in flight past this point
  CK(cudaEventSynchronize(ctx->ev[((issued - 1) & 1) ? 10 : 7]));
  if (last) ctx->h_st[0] = ctx->h_st[1];
  *iters = ctx->h_st->it;
  *status = ctx->h_st->done ? ctx->h_st->status : DDEL_ENOCONV;
  return DDEL_OK;
}

// The relaxed PCG's graph: check_every iterations with the FP32-stored S_i
// of a FP64 context (no coarse space), kept beside graph[0].
int ensure_graph_lo(ddel_ctx* ctx) {
  const int per = pcg_per(ctx);
  const int split = explicit_split(ctx->T, ctx->opt.schur_split);
  if (ctx->graph_lo && (ctx->graph_lo_iters != per || ctx->graph_lo_split != split)) {
    cudaGraphExecDestroy(ctx->graph_lo);
    ctx->graph_lo = nullptr;
  }
  if (ctx->graph_lo) return DDEL_OK;
  cudaGraph_t graph;
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < per; ++i) pcg_iteration(ctx, 0, true, i & 1);
  CK(cudaStreamEndCapture(ctx->stream, &graph));
  CK(cudaGraphInstantiate(&ctx->graph_lo, graph, 0));
  cudaGraphDestroy(graph);
  ctx->graph_lo_iters = per;
  ctx->graph_lo_split = split;
  return DDEL_OK;
}

__global__ void set_tol2_kernel(PcgState* st, double tol2) { st->tol2 = tol2; }

// Reliable update after a whole batch: y = S x with the FP64 operator (into
// the FP64 ring), then r = g - y, u = S~^-1 r and the corrected step length
// (launch_pcg_replace); waits for the state.
int pcg_replace(ddel_ctx* ctx, const double* g, double tol2) {
  cudaStream_t s = ctx->stream;
  SchurIO io = make_io(ctx);
  io.x = ctx->x;
  schur_dispatch(ctx, 0, false, io, s);
  launch_pcg_replace(ctx->T, ctx->F, g, (const double*)ring_of(ctx, 0), ctx->x, ctx->r, ctx->z, ctx->p, ctx->sv,
                     ctx->st, pcg_partials(ctx, 0), s, ctx->nupd, tol2);
  ctx->launches += 3;
  CK(cudaMemcpyAsync(ctx->h_st, ctx->st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(ctx->ev[7], s));
  CK(cudaEventSynchronize(ctx->ev[7]));
  return DDEL_OK;
}

// Relaxed mixed-precision PCG on S x = g: the Schur apply may lose accuracy
// as the residual falls (relaxation of inexact Krylov methods, van den Eshof
// and Sleijpen 2004), so the FP64 S_i serve until the recursive residual is
// below relax_switch ||f|| and their FP32 copies after; the recursive residual
// is replaced by the true one, computed with the FP64 operator, whenever it
// has fallen by relax_delta since the last replacement or meets the
// tolerance (reliable updates, Sleijpen and van der Vorst 1996), and the
// iteration stops only on a replaced residual.  The FP32 phase runs with a
// zero device tolerance, so that its batches never stop early and each
// replacement follows a whole batch; decisions are taken between batches of
// check_every iterations, each read back before the next is issued.  Three
// replacements in a row without a new low of the true residual return the
// iteration to the FP64 operator (and the device tolerance) for good.
int pcg_run_relaxed(ddel_ctx* ctx, const double* g, int* iters, int* status, int* low_iters, int* replacements) {
  int rc = pcg_start(ctx, 0, g, false);
  if (rc) return rc;
  const bool use_graph = ctx->opt.use_graph != 0;
  if (use_graph) {
    rc = ensure_graph_lo(ctx);
    if (rc) return rc;
  }
  cudaStream_t s = ctx->stream;
  const int per = pcg_per(ctx);
  const int max_checks = ctx->opt.max_it / per + 2;
  const double delta = ctx->opt.relax_delta > 0.0 && ctx->opt.relax_delta < 1.0 ? ctx->opt.relax_delta : 0.1;
  bool lo = false, allow_lo = true;
  double tol2 = -1.0, tau = 0.0, r_max = 0.0, best = INFINITY;
  int stall = 0, it_prev = 0;
  *low_iters = 0;
  *replacements = 0;
  *status = DDEL_ENOCONV;
  for (int chk = 0; chk < max_checks; ++chk) {
    rc = pcg_issue(ctx, 0, lo, 0, lo && use_graph);
    if (rc) return rc;
    CK(cudaEventSynchronize(ctx->ev[7]));
    const PcgState h = ctx->h_st[0];
    if (lo) *low_iters += h.it - it_prev;
    it_prev = h.it;
    if (tol2 < 0.0) {
      // the device tolerance of this cycle, tol2 = (tol ||f|| / 2)^2
      tol2 = h.tol2;
      tau = ctx->opt.tol > 0.0 ? ctx->opt.relax_switch * 2.0 * std::sqrt(tol2) / ctx->opt.tol : 0.0;
    }
    if (h.done) {
      // FP64 phase: converged (the textbook stop) or an error status; FP32
      // phase (zero tolerance): an error status, or an exactly zero recursive
      // residual, which says nothing of the true one
      *status = (lo && h.status == 0) ? DDEL_ENOCONV : h.status;
      break;
    }
    const double rn = std::sqrt(h.rr);
    if (!lo) {
      if (allow_lo && rn <= tau) {
        lo = true;
        r_max = rn;
        set_tol2_kernel<<<1, 1, 0, s>>>(ctx->st, 0.0);
        ctx->launches += 1;
      }
      continue;
    }
    if (rn * rn <= tol2 || rn < delta * r_max) {
      rc = pcg_replace(ctx, g, tol2);
      if (rc) return rc;
      ++*replacements;
      const PcgState h2 = ctx->h_st[0];
      if (h2.done) {  // breakdown in the corrected step
        *status = h2.status;
        break;
      }
      if (h2.replaced_ok) {
        *status = DDEL_OK;
        break;
      }
      const double rt = std::sqrt(h2.rr);
      r_max = rt;
      if (rt < best) {
        best = rt;
        stall = 0;
      } else if (++stall >= 3) {
        lo = false;
        allow_lo = false;
        set_tol2_kernel<<<1, 1, 0, s>>>(ctx->st, tol2);
        ctx->launches += 1;
      }
      continue;
    }
    r_max = std::max(r_max, rn);
  }
  CK(cudaGetLastError());
  *iters = ctx->h_st->it;
  return DDEL_OK;
}

void condense(ddel_ctx* ctx, int prec, const double* f, double* g) {
  SchurIO io = make_io(ctx);
  io.f = f;
  io.ring_out = ring_of(ctx, prec);
  launch_schur(ctx->T, ctx->F, prec, ctx->factor[prec], io, ctx->stream);
  launch_gamma_sum(ctx->T, prec, io.ring_out, f, -1.0, g, ctx->stream);
  ctx->launches += 2;
}

void back_substitute(ddel_ctx* ctx, int prec, const double* f, const double* xg, double* u) {
  SchurIO io = make_io(ctx);
  io.f = f;
  io.x = xg;
  io.u_out = u;
  launch_schur(ctx->T, ctx->F, prec, ctx->factor[prec], io, ctx->stream);
  launch_scatter_gamma(ctx->T, xg, u, ctx->stream);
  ctx->launches += 2;
}


// Factor (and, where available, form the explicit local Schur complements) in
// one precision: launch (asynchronous) and check (ENOTSPD on a failed pivot,
// EINVAL on a bad density).
int factor_launch(ddel_ctx* ctx, int prec) {
  if (!ctx->factor[prec]) {
    cudaError_t e = cudaMalloc(&ctx->factor[prec], ctx->S.factor_elems * (prec ? 4 : 8) + 256);
    if (e != cudaSuccess) return fail(ctx, DDEL_ENOMEM, "factor allocation");
  }
  const int init[2] = {0, 0x7fffffff};
  CK(cudaMemcpyAsync(ctx->err, init, sizeof(init), cudaMemcpyHostToDevice, ctx->stream));
  if (ctx->T.dim == 3) {
    // the scratch grows when the tensor-core planes are switched on later
    const size_t need = factor3d_work_elems(ctx->T, prec, ctx->opt.tensor_form) * (prec ? 4 : 8);
    if (ctx->work3d[prec] && ctx->work3d_bytes[prec] < need) {
      CK(cudaStreamSynchronize(ctx->stream));
      cudaFree(ctx->work3d[prec]);
      ctx->work3d[prec] = nullptr;
    }
    if (!ctx->work3d[prec]) {
      cudaError_t e = cudaMalloc(&ctx->work3d[prec], need);
      if (e != cudaSuccess) return fail(ctx, DDEL_ENOMEM, "3D factor scratch");
      ctx->work3d_bytes[prec] = need;
    }
  }
  ctx->launches += launch_factor(ctx->T, ctx->F, prec, ctx->factor[prec], ctx->work3d[prec], ctx->err,
                                 ctx->bad_sub, ctx->opt.tensor_form, ctx->stream);
  CK(cudaGetLastError());
  ctx->factored[prec] = false;
  ctx->explicit_ok[prec] = false;
  const int NR = explicit_ring_size(ctx->T);
  const bool want_explicit = NR > 0 && ctx->opt.schur_mode != DDEL_SCHUR_IMPLICIT;
  if (want_explicit) {
    if (!ctx->sexp[prec]) {
      cudaError_t e = cudaMalloc(&ctx->sexp[prec], (size_t)ctx->T.n_sub * NR * NR * (prec ? 4 : 8));
      if (e != cudaSuccess) return fail(ctx, DDEL_ENOMEM, "explicit Schur allocation");
    }
    const size_t we = explicit_form_work_elems(ctx->T);
    if (we && !ctx->form_work[prec]) {
      cudaError_t e = cudaMalloc(&ctx->form_work[prec], we * (prec ? 4 : 8));
      if (e != cudaSuccess) return fail(ctx, DDEL_ENOMEM, "explicit Schur scratch allocation");
    }
    // S_i with W^T W on the tensor cores, FP64-accurate: for the native FP64
    // form and the double-float form's rings of 256 (for rings of 128 the
    // double-float form keeps its own, faster double-float formation); the
    // FP32 form only with tensor_form = 2 (its FP32-pipe formation is the
    // faster one, the FP32 pipes being wide)
    const int tf = ctx->opt.tensor_form;
    const bool tc = (tf == 2 || (tf == 1 && prec == 0)) && tensor_form_available(ctx->T) &&
                    !(prec == 0 && ctx->opt.schur_mode == DDEL_SCHUR_AUTO && NR <= 128);
    if (tc) {
      if (!ctx->form_work[prec]) {
        cudaError_t e = cudaMalloc(&ctx->form_work[prec], explicit_form_work_elems(ctx->T) * (prec ? 4 : 8));
        if (e != cudaSuccess) return fail(ctx, DDEL_ENOMEM, "explicit Schur scratch allocation");
      }
      if (!ctx->tc_work && cudaMalloc(&ctx->tc_work, tensor_form_work_bytes(ctx->T)) != cudaSuccess)
        return fail(ctx, DDEL_ENOMEM, "tensor-core formation scratch allocation");
      launch_schur_form_tc(ctx->T, ctx->F, prec, ctx->factor[prec], ctx->form_work[prec], ctx->tc_work,
                           ctx->sexp[prec], ctx->err, ctx->stream);
      ctx->launches += 3;
    } else {
      // AUTO applies S_i in double-float arithmetic, so it is formed that way too
      const bool df = prec == 0 && ctx->opt.schur_mode == DDEL_SCHUR_AUTO;
      launch_schur_form(ctx->T, ctx->F, prec, df, ctx->factor[prec], ctx->form_work[prec], ctx->sexp[prec],
                        ctx->stream);
      ctx->launches += 1;
    }
    CK(cudaGetLastError());
  }
  ctx->pending_explicit = want_explicit;
  return DDEL_OK;
}

// Reads the error words of a launched factorisation (synchronises the stream).
int factor_check(ddel_ctx* ctx, int prec) {
  int rc = check_kernel_err(ctx);
  if (rc) return rc;
  if (ctx->h_err[2] == kErrBadRho) return fail(ctx, DDEL_EINVAL, "density must be > 0");
  if (ctx->h_err[0] == kErrPivot)
    return fail(ctx, DDEL_ENOTSPD, "pivot failure in subdomain " + std::to_string(ctx->h_err[1]));
  if (ctx->h_err[0] == kErrTimeout)
    return fail(ctx, DDEL_ETIMEOUT, "a bounded wait of the tensor-core formation ran out");
  ctx->factored[prec] = true;
  ctx->explicit_ok[prec] = ctx->pending_explicit;
  ctx->coarse_prec = -1;  // E must be formed again with the new S (next ddel_solve)
  ctx->ck = 0;
  if (prec == 0) ctx->df_ok = ctx->df3_ok = false;
  if (prec == 0 && ctx->T.dim == 3 && ctx->opt.schur_mode == DDEL_SCHUR_AUTO) {
    // 3D: the FP64 factor as FP32 (hi, lo) pairs, in the order of the sweeps,
    // for the double-float PCG apply
    if (!ctx->factor_df) {
      std::vector<int64_t> off(ctx->S.n_sub);
      const int64_t tot = df3_layout(ctx->S.subs.data(), ctx->S.n_sub, off.data());
      if (cudaMalloc(&ctx->factor_df, tot * sizeof(float2) + 256) != cudaSuccess ||
          cudaMalloc(&ctx->df3_off, off.size() * sizeof(int64_t)) != cudaSuccess) {
        if (ctx->factor_df) cudaFree(ctx->factor_df);
        ctx->factor_df = nullptr;
        ctx->df3_off = nullptr;
        return fail(ctx, DDEL_ENOMEM, "double-float factor allocation");
      }
      CK(cudaMemcpy(ctx->df3_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
      CK(cudaMemsetAsync(ctx->factor_df, 0, tot * sizeof(float2), ctx->stream));
    }
    launch_build_df3(ctx->T, (const double*)ctx->factor[0], ctx->df3_off, ctx->factor_df, ctx->stream);
    ctx->launches += 1;
    CK(cudaGetLastError());
    ctx->df3_ok = true;
  }
  if (prec == 0 && ctx->explicit_ok[0] && ctx->opt.schur_mode == DDEL_SCHUR_AUTO) {
    // FP64 local Schur complements as FP32 (hi, lo) pairs for the double-float apply
    const int NR = explicit_ring_size(ctx->T);
    const int64_t n = (int64_t)ctx->T.n_sub * NR * NR;
    if (!ctx->sexp_df && cudaMalloc(&ctx->sexp_df, n * sizeof(float2)) != cudaSuccess)
      return fail(ctx, DDEL_ENOMEM, "double-float Schur allocation");
    launch_split_df((const double*)ctx->sexp[0], ctx->sexp_df, n, ctx->stream);
    ctx->launches += 1;
    CK(cudaGetLastError());
    ctx->df_ok = true;
  }
  return DDEL_OK;
}

int factor_prec(ddel_ctx* ctx, int prec) {
  int rc = factor_launch(ctx, prec);
  return rc ? rc : factor_check(ctx, prec);
}

// Coarse space for the PCG of precision prec (and apply32): Cholesky QR of Z
// twice, S Q with the same Schur apply as the PCG, E = Q^T S Q and its
// inverse, G = (S Q)^T S Q.  Synchronises (three small read-backs).
int coarse_build(ddel_ctx* ctx, int prec, bool apply32) {
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->T.n_gamma;
  const int KK = kMaxCoarse * kMaxCoarse;
  double* cs = ctx->csmall;
  ctx->ck = 0;
  launch_gram(ctx->cZ, ctx->cZ, ctx->ck_in, n, cs, ctx->partials, ctx->cticket, s);
  launch_cholqr_factor(cs, ctx->ck_in, 1e-10, cs + KK, ctx->cflags, s);
  launch_apply_T(ctx->cZ, cs + KK, ctx->ck_in, ctx->cflags, n, ctx->cQ1, s);
  ctx->launches += 3;
  int k1 = 0;
  CK(cudaMemcpyAsync(ctx->h_cflags, ctx->cflags, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  k1 = ctx->h_cflags[0];
  ctx->coarse_prec = prec * 2 + (apply32 ? 1 : 0);
  if (k1 <= 0) return DDEL_OK;
  launch_gram(ctx->cQ1, ctx->cQ1, k1, n, cs + 2 * KK, ctx->partials, ctx->cticket, s);
  launch_cholqr_factor(cs + 2 * KK, k1, 1e-10, cs + 3 * KK, ctx->cflags + 1, s);
  launch_apply_T(ctx->cQ1, cs + 3 * KK, k1, ctx->cflags + 1, n, ctx->cQ, s);
  ctx->launches += 3;
  CK(cudaMemcpyAsync(ctx->h_cflags + 1, ctx->cflags + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int k2 = ctx->h_cflags[1];
  if (k2 <= 0) return DDEL_OK;
  const int ap = apply_prec(ctx, prec, apply32);
  for (int i = 0; i < k2; ++i) {
    SchurIO io = make_io(ctx);
    io.x = ctx->cQ + i * n;
    schur_dispatch(ctx, prec, apply32, io, s);
    launch_gamma_sum(ctx->T, ap, io.ring_out, nullptr, 1.0, ctx->cSQ + i * n, s);
    ctx->launches += 2;
  }
  launch_gram(ctx->cQ, ctx->cSQ, k2, n, cs + 4 * KK, ctx->partials, ctx->cticket, s);
  launch_gram(ctx->cSQ, ctx->cSQ, k2, n, cs + 6 * KK, ctx->partials, ctx->cticket, s);
  launch_coarse_invert(cs + 4 * KK, k2, cs + 5 * KK, ctx->cflags + 2, s);
  ctx->launches += 3;
  CK(cudaMemcpyAsync(ctx->h_cflags + 2, ctx->cflags + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  ctx->ck = ctx->h_cflags[2] ? k2 : 0;
  return DDEL_OK;
}

// Global interface preconditioner: host set-up of every displacement
// component (interface M, L, face inverses of L) and device copies with a
// workspace for the most Lanczos steps.  Returns DDEL_EINVAL for a singular
// interface Laplacian (a part of Gamma that meets no clamped node).
int gp_build(ddel_ctx* ctx) {
  if (ctx->gp_state == 1) return DDEL_OK;
  if (ctx->gp_state == -1) return fail(ctx, DDEL_EINVAL, "global preconditioner: singular interface Laplacian");
  const int dim = ctx->S.dim;
  GPDev gd{};
  for (int c = 0; c < dim; ++c) {
    GPHost h;
    const std::string msg = build_global_prec(ctx->S, c, &h);
    if (!msg.empty()) return fail(ctx, DDEL_EINVAL, "global preconditioner: " + msg);
    if (h.singular || h.pos.empty()) {
      ctx->gp_state = -1;
      return fail(ctx, DDEL_EINVAL,
                  "global preconditioner: singular interface Laplacian (a part of the interface meets no "
                  "clamped node)");
    }
    GPComp& g = gd.c[c];
    g.n = (int)h.pos.size();
    int32_t *pos, *col, *rf, *fl0, *fn;
    int64_t *rp, *fio;
    double *M, *L, *Md, *Ld, *Mi, *ci, *fi, *w, *work;
    CK(upload(ctx, h.pos, &pos));
    CK(upload(ctx, h.rowptr, &rp));
    CK(upload(ctx, h.col, &col));
    CK(upload(ctx, h.M, &M));
    CK(upload(ctx, h.L, &L));
    CK(upload(ctx, h.Mdiag, &Md));
    CK(upload(ctx, h.Ldiag, &Ld));
    CK(upload(ctx, h.Minv_diag, &Mi));
    CK(upload(ctx, h.cross_inv, &ci));
    CK(upload(ctx, h.row_face, &rf));
    CK(upload(ctx, h.face_l0, &fl0));
    CK(upload(ctx, h.face_n, &fn));
    CK(upload(ctx, h.face_inv_off, &fio));
    CK(upload(ctx, h.face_inv, &fi));
    CK(dalloc(ctx, &w, (size_t)g.n * 8));
    CK(dalloc(ctx, &work, global_prec_work_elems(g.n, kLz) * 8));
    g.pos = pos;
    g.rowptr = rp;
    g.col = col;
    g.M = M;
    g.L = L;
    g.Mdiag = Md;
    g.Ldiag = Ld;
    g.Minv_diag = Mi;
    g.cross_inv = ci;
    g.row_face = rf;
    g.face_l0 = fl0;
    g.face_n = fn;
    g.face_inv_off = fio;
    g.face_inv = fi;
    g.w = w;
    g.work = work;
  }
  gd.ncomp = dim;
  CK(dalloc(ctx, &ctx->gp_out, (size_t)3 * (2 + 3 * kLz) * 8));
  CK(cudaMallocHost(&ctx->h_gp_out, (size_t)3 * (2 + 3 * kLz) * 8));
  ctx->gp = gd;
  ctx->gp_state = 1;
  return DDEL_OK;
}

int gp_check_options(ddel_ctx* ctx, const ddel_gmres_options* o) {
  if (o->precond < DDEL_PREC_IDENTITY || o->precond > DDEL_PREC_GLOBAL)
    return fail(ctx, DDEL_EINVAL, "precond must be IDENTITY, FACE or GLOBAL");
  if (o->precond == DDEL_PREC_GLOBAL &&
      (o->lanczos_steps < 1 || o->lanczos_steps > kLz || !(o->inner_tol > 0.0 && o->inner_tol < 1.0) ||
       !(o->mass_tol > 0.0 && o->mass_tol < 1.0)))
    return fail(ctx, DDEL_EINVAL, "lanczos_steps in 1..32, inner_tol and mass_tol in (0, 1)");
  return DDEL_OK;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

}  // namespace

extern "C" {

void ddel_default_options(ddel_options* o) {
  if (!o) return;
  o->precision = DDEL_FP64;
  o->theta = 0.5;
  o->face_scaling = 2;
  o->crosspoint_mode = 0;
  o->tol = 1e-8;
  o->max_it = 5000;
  o->max_cycles = 10;
  o->inner_tol = 1e-6;
  o->x0_mode = DDEL_X0_ZERO;
  o->schur_mode = DDEL_SCHUR_AUTO;
  o->use_graph = 1;
  o->check_every = 16;
  o->tensor_form = 1;
  o->schur_split = 0;
  o->relax_switch = 0.0;
  o->relax_delta = 0.1;
}

const char* ddel_strerror(int s) {
  switch (s) {
    case DDEL_OK: return "ok";
    case DDEL_EINVAL: return "invalid argument";
    case DDEL_ENOMEM: return "out of memory";
    case DDEL_ECUDA: return "CUDA error";
    case DDEL_ENOTSPD: return "subdomain matrix not positive definite";
    case DDEL_ENOCONV: return "no convergence within the iteration limits";
    case DDEL_EBREAKDOWN: return "Krylov breakdown";
    case DDEL_ESTATE: return "call order violated";
    case DDEL_ETIMEOUT: return "bounded device wait ran out";
    default: return "unknown status";
  }
}

const char* ddel_last_error(const ddel_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : g_create_error.c_str();
}

int ddel_create(const ddel_mesh* mesh, const ddel_material* mat, const ddel_bc* bc,
                const ddel_options* opt, void* cuda_stream, ddel_ctx** out) {
  if (!mesh || !mat || !bc || !out) return DDEL_EINVAL;
  *out = nullptr;
  ddel_ctx* ctx = new (std::nothrow) ddel_ctx();
  if (!ctx) return DDEL_ENOMEM;
  ctx->mesh = *mesh;
  ctx->mat = *mat;
  if (opt) {
    if (!(opt->relax_switch >= 0.0) || !std::isfinite(opt->relax_switch)) {
      g_create_error = "relax_switch must be a finite value >= 0";
      delete ctx;
      return DDEL_EINVAL;
    }
    ctx->opt = *opt;
  } else {
    ddel_default_options(&ctx->opt);
  }
  const int ne[3] = {mesh->nx, mesh->ny, mesh->nz};
  std::string msg = build_setup(mesh->dim, ne, mesh->sub, mat->E, mat->nu, mat->plane_stress,
                                bc->clamp_faces, bc->fixed_dof, bc->n_point, bc->point_node,
                                bc->point_force, bc->traction_face, bc->traction, bc->body_force, ctx->opt.theta,
                                &ctx->S);
  if (!msg.empty()) {
    g_create_error = msg;
    delete ctx;
    return DDEL_EINVAL;
  }
  if (!(mat->simp_p > 0)) {
    delete ctx;
    return DDEL_EINVAL;
  }
  Setup& S = ctx->S;
  int rc = DDEL_OK;
  auto bad = [&](cudaError_t e) {
    if (e != cudaSuccess) {
      rc = e == cudaErrorMemoryAllocation ? DDEL_ENOMEM : DDEL_ECUDA;
      ctx->last_error = cudaGetErrorString(e);
      return true;
    }
    return false;
  };
  if (bad(configure_kernels())) {
    ctx->last_error = "kernel configuration: " + ctx->last_error;
    goto fail_out;
  }
  if (cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (bad(cudaStreamCreate(&ctx->stream))) goto fail_out;
    ctx->own_stream = true;
  }
  {
    DevTables& T = ctx->T;
    T.dim = S.dim;
    T.s = S.sub;
    T.n_sub = S.n_sub;
    T.BP = S.BP;
    T.nb_max = S.nb_max;
    for (int a = 0; a < 3; ++a) {
      T.ne[a] = S.ne[a] ? S.ne[a] : 1;
      T.nn[a] = S.nn[a];
    }
    T.n_dof = S.n_dof;
    T.n_elem = S.n_elem;
    T.n_gamma = (int64_t)S.gamma_dof.size();
    T.n_face_dofs = S.n_face_dofs;
    T.n_blocks = (int)S.blk_off.size();
    T.max_blk_n = S.max_blk_n > 0 ? S.max_blk_n : 1;
    T.upd_lanes = 1;
    while (T.upd_lanes < T.max_blk_n && T.upd_lanes < 32) T.upd_lanes *= 2;
    // face tables staged in shared memory when the update kernel's dynamic
    // shared memory stays within 40 KB (eight warps, 32 / upd_lanes blocks each)
    {
      const size_t ug = 32 / T.upd_lanes, mb = T.max_blk_n;
      T.upd_stage_p = 8 * ug * mb * (16 + 8 * mb) <= 40 * 1024 ? 1 : 0;
    }
    T.n_ring = (int64_t)S.ring_gidx.size();
    T.max_owners = S.max_owners;
    std::vector<float> ke32(S.Ke.begin(), S.Ke.end());
    if (bad(upload(ctx, S.subs, &T.subs)) || bad(upload(ctx, S.fixed, &T.fixed)) ||
        bad(upload(ctx, S.ring_gidx, &T.ring_gidx)) || bad(upload(ctx, S.ring_loc, &T.ring_loc)) ||
        bad(upload(ctx, S.owner_ptr, &T.owner_ptr)) || bad(upload(ctx, S.owner_idx, &T.owner_idx)) ||
        bad(upload(ctx, S.owner_pad, &T.owner_pad)) || bad(upload(ctx, S.ring_dst, &T.ring_dst)) ||
        bad(upload(ctx, S.gamma_dof, &T.gamma_dof)) || bad(upload(ctx, S.blk_off, &T.blk_off)) ||
        bad(upload(ctx, S.blk_n, &T.blk_n)) || bad(upload(ctx, S.blk_poff, &T.blk_poff)) ||
        bad(upload(ctx, S.blk_hmean, &T.blk_hmean)) || bad(upload(ctx, S.ptab, &T.ptab)) ||
        bad(upload(ctx, S.hdiag, &T.hdiag)) ||
        bad(upload(ctx, S.Ke, &T.Ke64)) || bad(upload(ctx, ke32, &T.Ke32)))
      goto fail_out;
    // face preconditioner blocks also as FP32 (hi, lo) pairs (see pcg_cg_kernel)
    if (bad(dalloc(ctx, &T.ptab_df, S.ptab.size() * sizeof(float2)))) goto fail_out;
    if (!S.ptab.empty()) launch_split_df(T.ptab, T.ptab_df, (int64_t)S.ptab.size(), nullptr);
    if (bad(cudaDeviceSynchronize()) || bad(cudaGetLastError())) goto fail_out;
    const int64_t ng = T.n_gamma, nd = S.n_dof;
    // owner-major ring (ng x max_owners entries of up to 8 bytes), zero padded
    const size_t ring_bytes = (size_t)(ng * S.max_owners + 4) * 8;
    DevFields& F = ctx->F;
    if (bad(dalloc(ctx, &F.scale64, S.n_elem * 8)) || bad(dalloc(ctx, &F.scale32, S.n_elem * 4)) ||
        bad(dalloc(ctx, &F.diagG, ng * 8)) || bad(dalloc(ctx, &F.blk_alpha, (T.n_blocks + 1) * 8)) ||
        bad(dalloc(ctx, &F.face_w, (T.n_face_dofs + 1) * 8)) ||
        bad(dalloc(ctx, &F.cross_scale, (ng - T.n_face_dofs + 1) * 8)) ||
        bad(dalloc(ctx, &ctx->ring, ring_bytes)) || bad(dalloc(ctx, &ctx->ring32, ring_bytes)) ||
        bad(dalloc(ctx, &ctx->d_f, nd * 8)) ||
        bad(dalloc(ctx, &ctx->d_load, nd * 8)) || bad(dalloc(ctx, &ctx->d_u, nd * 8)) ||
        bad(dalloc(ctx, &ctx->d_r, nd * 8)) || bad(dalloc(ctx, &ctx->d_d, nd * 8)) ||
        bad(dalloc(ctx, &ctx->g, ng * 8)) || bad(dalloc(ctx, &ctx->x, ng * 8)) ||
        bad(dalloc(ctx, &ctx->r, ng * 8)) || bad(dalloc(ctx, &ctx->z, ng * 8)) ||
        bad(dalloc(ctx, &ctx->p, ng * 8)) || bad(dalloc(ctx, &ctx->q, ng * 8)) ||
        bad(dalloc(ctx, &ctx->sv, ng * 8)) ||
        bad(dalloc(ctx, &ctx->rho, S.n_elem * 8)) || bad(dalloc(ctx, &ctx->st, sizeof(PcgState))) ||
        bad(dalloc(ctx, &ctx->partials, (size_t)(4 * 152 * (2 + 2 * kMaxCoarse) + 2 * T.n_sub + 64) * 8)) ||
        bad(dalloc(ctx, &ctx->pcg_pd, (size_t)(4 * T.n_sub + 64) * 8)) ||
        bad(dalloc(ctx, &ctx->pcg_pu, (size_t)2 * kPcgRows * 2 * 152 * 8)) ||
        bad(dalloc(ctx, &ctx->ticketK, 16)) || bad(dalloc(ctx, &ctx->nrm, 16)) ||
        bad(dalloc(ctx, &ctx->err, 4 * sizeof(int))))
      goto fail_out;
    ctx->bad_sub = ctx->err + 1;
    if (bad(cudaMallocHost(&ctx->h_st, 2 * sizeof(PcgState))) ||
        bad(cudaMallocHost(&ctx->h_nrm, 2 * sizeof(double))) ||
        bad(cudaMallocHost(&ctx->h_err, 4 * sizeof(int))))
      goto fail_out;
    ctx->nblk = 2 * 152;
    PcgState st0{};
    st0.partials = ctx->partials;

    if (bad(cudaMemcpy(ctx->st, &st0, sizeof(PcgState), cudaMemcpyHostToDevice)) ||
        bad(cudaMemset(ctx->ticketK, 0, 16)) || bad(cudaMemset(ctx->ring, 0, ring_bytes)) ||
        bad(cudaMemset(ctx->ring32, 0, ring_bytes)) ||
        bad(cudaMemcpy(ctx->d_load, S.f.data(), nd * 8, cudaMemcpyHostToDevice)))
      goto fail_out;
    const int zero_err[4] = {0, 0x7fffffff, 0, 0};
    if (bad(cudaMemcpy(ctx->err, zero_err, sizeof(zero_err), cudaMemcpyHostToDevice))) goto fail_out;
    ctx->nblk = 2 * 152;
    {
      // PCG update: enough blocks of eight warps for the packed face blocks
      // and one thread per cross-point DOF, at most two per SM
      const int64_t ug = 32 / T.upd_lanes, n_cross = T.n_gamma - T.n_face_dofs;
      const int64_t need = std::max((T.n_blocks + 8 * ug - 1) / (8 * ug), (n_cross + 255) / 256);
      ctx->nupd = (int)std::min<int64_t>(std::max<int64_t>(need, 1), 2 * 152);
    }
    for (auto& e : ctx->ev)
      if (bad(cudaEventCreate(&e))) goto fail_out;
  }
  *out = ctx;
  return DDEL_OK;
fail_out:
  g_create_error = ctx->last_error;
  ddel_destroy(ctx);
  return rc != DDEL_OK ? rc : DDEL_ECUDA;
}

void ddel_destroy(ddel_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (ddel_learner* L : ctx->learners) learner_context_gone(L);  // they must not touch ctx again
  ctx->learners.clear();
  for (auto& g : ctx->graph)
    if (g) cudaGraphExecDestroy(g);
  if (ctx->graph_lo) cudaGraphExecDestroy(ctx->graph_lo);
  for (void* p : ctx->allocs) cudaFree(p);
  for (void* p : ctx->factor)
    if (p) cudaFree(p);
  for (void* p : ctx->sexp)
    if (p) cudaFree(p);
  for (void* p : ctx->form_work)
    if (p) cudaFree(p);
  if (ctx->tc_work) cudaFree(ctx->tc_work);
  for (void* p : ctx->work3d)
    if (p) cudaFree(p);
  if (ctx->sexp32) cudaFree(ctx->sexp32);
  if (ctx->sexp_df) cudaFree(ctx->sexp_df);
  if (ctx->factor_df) cudaFree(ctx->factor_df);
  if (ctx->df3_off) cudaFree(ctx->df3_off);
  if (ctx->h_st) cudaFreeHost(ctx->h_st);
  if (ctx->h_nrm) cudaFreeHost(ctx->h_nrm);
  if (ctx->h_err) cudaFreeHost(ctx->h_err);
  if (ctx->h_topo) cudaFreeHost(ctx->h_topo);
  if (ctx->h_cflags) cudaFreeHost(ctx->h_cflags);
  if (ctx->h_gp_out) cudaFreeHost(ctx->h_gp_out);
  if (ctx->h_gm) cudaFreeHost(ctx->h_gm);
  for (double* p : {ctx->gm_V, ctx->gm_Z, ctx->gm_w, ctx->gm_h, ctx->gm_part, ctx->gm_vg, ctx->gm_zg})
    if (p) cudaFree(p);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

int ddel_get_info(const ddel_ctx* ctx, ddel_info_t* info) {
  if (!ctx || !info) return DDEL_EINVAL;
  const Setup& S = ctx->S;
  info->dim = S.dim;
  info->n_sub = S.n_sub;
  info->n_elem = (int)S.n_elem;
  info->max_block = S.BP;
  info->max_blocks_per_sub = S.nb_max;
  info->n_nodes = S.n_nodes;
  info->n_dof = S.n_dof;
  info->n_gamma = (int64_t)S.gamma_dof.size();
  int64_t nf = 0;
  for (auto v : S.fixed) nf += v;
  info->n_fixed = nf;
  info->factor_bytes = S.factor_elems * 8;
  info->n_face_blocks = (int)S.blk_off.size();
  info->n_cross = (int)(S.gamma_dof.size() - S.n_face_dofs);
  return DDEL_OK;
}

int ddel_set_options(ddel_ctx* ctx, const ddel_options* opt) {
  if (!ctx || !opt) return DDEL_EINVAL;
  if (opt->theta != ctx->opt.theta) return fail(ctx, DDEL_EINVAL, "theta is fixed at creation");
  if (!(opt->relax_switch >= 0.0) || !std::isfinite(opt->relax_switch))
    return fail(ctx, DDEL_EINVAL, "relax_switch must be a finite value >= 0");
  if (opt->schur_mode != ctx->opt.schur_mode || opt->precision != ctx->opt.precision)
    ctx->factored[0] = ctx->factored[1] = false;  // refactor to switch forms
  ctx->opt = *opt;
  return DDEL_OK;
}

int ddel_assemble(ddel_ctx* ctx, const double* rho, int on_device) {
  if (!ctx || !rho) return DDEL_EINVAL;
  const int64_t ne = ctx->S.n_elem;
  if (!on_device) {
    for (int64_t e = 0; e < ne; ++e)
      if (!(rho[e] > 0) || !std::isfinite(rho[e])) return fail(ctx, DDEL_EINVAL, "density must be > 0");
    CK(cudaMemcpyAsync(ctx->rho, rho, ne * 8, cudaMemcpyHostToDevice, ctx->stream));
  } else {
    CK(cudaMemcpyAsync(ctx->rho, rho, ne * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  CK(cudaMemsetAsync(ctx->err + 2, 0, sizeof(int), ctx->stream));
  ctx->launches_at_assemble = ctx->launches;
  ctx->launches += 3;
  launch_assemble(ctx->T, ctx->F, ctx->rho, ctx->mat.E, ctx->mat.simp_p, ctx->opt.face_scaling,
                  ctx->opt.crosspoint_mode, ctx->err + 2, ctx->stream);
  CK(cudaGetLastError());
  ctx->assembled = true;
  ctx->factored[0] = ctx->factored[1] = false;
  return DDEL_OK;
}

int ddel_factor(ddel_ctx* ctx) {
  if (!ctx) return DDEL_EINVAL;
  if (!ctx->assembled) return fail(ctx, DDEL_ESTATE, "assemble before factor");
  const int want = ctx->opt.precision == DDEL_FP32 ? 1 : 0;
  CK(cudaEventRecord(ctx->ev[8], ctx->stream));
  int rc = factor_prec(ctx, want);
  if (rc == DDEL_ENOTSPD && want == 1) rc = factor_prec(ctx, 0);  // FP32 pivot failed: FP64
  if (rc == DDEL_OK) ctx->active_prec = ctx->factored[want] ? want : 0;
  ctx->mixed_ready = false;
  if (rc == DDEL_OK && ctx->opt.precision == DDEL_MIXED && ctx->explicit_ok[0]) {
    // FP64-formed local Schur complements, stored (and applied) in FP32
    const int NR = explicit_ring_size(ctx->T);
    const int64_t n = (int64_t)ctx->T.n_sub * NR * NR;
    if (!ctx->sexp32 && cudaMalloc(&ctx->sexp32, n * 4) != cudaSuccess)
      return fail(ctx, DDEL_ENOMEM, "mixed Schur allocation");
    launch_round_f32((const double*)ctx->sexp[0], ctx->sexp32, n, ctx->stream);
    ctx->launches += 1;
    CK(cudaGetLastError());
    ctx->mixed_ready = true;
  }
  if (rc == DDEL_OK) {
    CK(cudaEventRecord(ctx->ev[9], ctx->stream));
    CK(cudaEventSynchronize(ctx->ev[9]));
    ctx->t_factor_ms = elapsed(ctx->ev[8], ctx->ev[9]);
  }
  return rc;
}

int ddel_solve(ddel_ctx* ctx, const double* f, double* u, int on_device, ddel_stats* stats) {
  if (!ctx || !u) return DDEL_EINVAL;
  if (!ctx->factored[ctx->active_prec]) return fail(ctx, DDEL_ESTATE, "factor before solve");
  cudaStream_t s = ctx->stream;
  const int64_t nd = ctx->S.n_dof;
  ddel_stats st{};
  st.bad_subdomain = -1;
  CK(cudaEventRecord(ctx->ev[0], s));
  if (!f)
    CK(cudaMemcpyAsync(ctx->d_f, ctx->d_load, nd * 8, cudaMemcpyDeviceToDevice, s));
  else
    CK(cudaMemcpyAsync(ctx->d_f, f, nd * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  // ZERO: u = 0; WARM: u = the previous solution (d_u keeps it between solves)
  if (!(ctx->opt.x0_mode == DDEL_X0_WARM && ctx->u_valid)) CK(cudaMemsetAsync(ctx->d_u, 0, nd * 8, s));
  const int init[2] = {0, 0x7fffffff};
  CK(cudaMemcpyAsync(ctx->err, init, sizeof(init), cudaMemcpyHostToDevice, s));
  // r = f - K u and ||f||
  launch_apply_K(ctx->T, ctx->F, ctx->d_u, ctx->d_f, ctx->d_r, 1, ctx->partials, ctx->ticketK,
                 ctx->nrm, s, ctx->nblk);
  ctx->launches += 1;
  int status = DDEL_ENOCONV;
  double t_cond = 0, t_pcg = 0, t_back = 0, t_ver = 0;
  double prev_relres = INFINITY;
  int prec = ctx->active_prec;
  bool apply32 = ctx->mixed_ready && prec == 0;
  for (int cyc = 0; cyc < ctx->opt.max_cycles; ++cyc) {
    // relaxed MIXED: one PCG to the final tolerance (no inner tolerance)
    const bool relaxed = apply32 && ctx->opt.relax_switch > 0.0 && ctx->ck_in == 0;
    set_tol_kernel<<<1, 1, 0, s>>>(ctx->st, ctx->nrm, ctx->opt.tol, ctx->opt.inner_tol,
                                   (prec == 1 || (apply32 && !relaxed)) ? 1 : 0, ctx->opt.max_it);
    ctx->launches += 1;
    CK(cudaEventRecord(ctx->ev[1], s));
    if (ctx->ck_in > 0 && ctx->coarse_prec != prec * 2 + (apply32 ? 1 : 0)) {
      int rc = coarse_build(ctx, prec, apply32);
      if (rc) return rc;
    }
    condense(ctx, prec, ctx->d_r, ctx->g);
    CK(cudaEventRecord(ctx->ev[2], s));
    int it = 0, pst = 0, low_it = 0, n_repl = 0;
    int rc = relaxed ? pcg_run_relaxed(ctx, ctx->g, &it, &pst, &low_it, &n_repl)
                     : pcg_run(ctx, prec, ctx->g, &it, &pst, apply32);
    if (rc) return rc;
    st.iters += it;
    st.low_iters += low_it;
    st.replacements += n_repl;
    st.coarse_k = ctx->ck;
    if (ctx->ck > 0 && (ctx->coarse_flags & DDEL_COARSE_X0)) st.x0_used += ctx->h_st->x0_used;
    if (pst == DDEL_EBREAKDOWN && ctx->ck > 0) {
      // The coarse-corrected recurrence lost definiteness (rounding with an
      // ill-conditioned or inaccurate coarse space): drop the coarse space for
      // the rest of this solve and redo the cycle with plain PCG.
      ctx->ck = 0;
      st.coarse_k = 0;
      st.fallback |= 2;
      continue;
    }
    CK(cudaEventRecord(ctx->ev[3], s));
    back_substitute(ctx, prec, ctx->d_r, ctx->x, ctx->d_d);
    launch_axpy(nd, 1.0, ctx->d_d, ctx->d_u, s);
    ctx->launches += 1;
    CK(cudaEventRecord(ctx->ev[4], s));
    launch_apply_K(ctx->T, ctx->F, ctx->d_u, ctx->d_f, ctx->d_r, 1, ctx->partials, ctx->ticketK,
                   ctx->nrm, s, ctx->nblk);
    ctx->launches += 1;
    CK(cudaMemcpyAsync(ctx->h_nrm, ctx->nrm, 16, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ctx->h_err, ctx->err, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(ctx->ev[5], s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    t_cond += elapsed(ctx->ev[1], ctx->ev[2]);
    t_pcg += elapsed(ctx->ev[2], ctx->ev[3]);
    t_back += elapsed(ctx->ev[3], ctx->ev[4]);
    t_ver += elapsed(ctx->ev[4], ctx->ev[5]);
    st.cycles = cyc + 1;
    const double fn = ctx->h_nrm[1];
    st.relres = fn > 0 ? ctx->h_nrm[0] / fn : 0.0;
    st.pcg_relres = fn > 0 ? std::sqrt(ctx->h_st->rr) / fn : 0.0;
    if (ctx->h_err[0] == kErrTimeout) {
      status = DDEL_ETIMEOUT;
      break;
    }
    const bool diverged = pst == DDEL_EBREAKDOWN || !std::isfinite(st.relres) ||
                          st.relres > (cyc == 0 ? 1.0 : prev_relres);
    if (diverged && apply32) {  // FP32-stored Schur complements: continue with FP64 ones
      launch_axpy(nd, -1.0, ctx->d_d, ctx->d_u, s);
      launch_apply_K(ctx->T, ctx->F, ctx->d_u, ctx->d_f, ctx->d_r, 1, ctx->partials, ctx->ticketK,
                     ctx->nrm, s, ctx->nblk);
      ctx->launches += 2;
      apply32 = false;
      st.fallback = 1;
      prev_relres = INFINITY;
      continue;
    }
    if (diverged && prec == 1) {
      // The FP32 operator lost definiteness or the correction diverged
      // (possible at high stiffness contrast): discard this correction and
      // continue the refinement with the FP64 factorisation.
      launch_axpy(nd, -1.0, ctx->d_d, ctx->d_u, s);
      launch_apply_K(ctx->T, ctx->F, ctx->d_u, ctx->d_f, ctx->d_r, 1, ctx->partials, ctx->ticketK,
                     ctx->nrm, s, ctx->nblk);
      ctx->launches += 2;
      if (!ctx->factored[0]) {
        int rc2 = factor_prec(ctx, 0);
        if (rc2) return rc2;
      }
      prec = 0;
      st.fallback = 1;
      prev_relres = INFINITY;
      continue;
    }
    if (pst == DDEL_EBREAKDOWN || !std::isfinite(st.relres)) {
      status = DDEL_EBREAKDOWN;
      break;
    }
    if (st.relres <= ctx->opt.tol || fn == 0.0) {
      status = DDEL_OK;
      break;
    }
    if (cyc > 0 && st.relres > 0.5 * prev_relres) {
      if (apply32) {  // stalled above the target: finish with the FP64 Schur complements
        apply32 = false;
        st.fallback = 1;
        prev_relres = st.relres;
        continue;
      }
      if (prec == 1) {  // FP32 refinement stalls above the target: finish in FP64
        if (!ctx->factored[0]) {
          int rc2 = factor_prec(ctx, 0);
          if (rc2) return rc2;
        }
        prec = 0;
        st.fallback = 1;
        prev_relres = st.relres;
        continue;
      }
      break;  // FP64 refinement at its rounding floor: the tolerance is unattainable
    }
    prev_relres = st.relres;
  }
  if (on_device)
    CK(cudaMemcpyAsync(u, ctx->d_u, nd * 8, cudaMemcpyDeviceToDevice, s));
  else
    CK(cudaMemcpyAsync(u, ctx->d_u, nd * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(ctx->ev[6], s));
  CK(cudaStreamSynchronize(s));
  st.t_factor_ms = ctx->t_factor_ms;
  st.t_condense_ms = t_cond;
  st.t_pcg_ms = t_pcg;
  st.t_backsub_ms = t_back;
  st.t_verify_ms = t_ver;
  st.t_total_ms = elapsed(ctx->ev[0], ctx->ev[6]);
  st.status = status;
  ctx->u_valid = status == DDEL_OK;
  if (stats) *stats = st;
  return status;
}


int ddel_topopt_step(ddel_ctx* ctx, ddel_topopt_state* ts, ddel_stats* stats) {
  if (!ctx || !ts || !ts->rho) return DDEL_EINVAL;
  if (!(ts->volfrac > 0.0 && ts->volfrac <= 1.0) || !(ts->r_min > 0.0) || !(ts->move > 0.0))
    return fail(ctx, DDEL_EINVAL, "topopt: need 0 < volfrac <= 1, r_min > 0, move > 0");
  if (ts->r_min > 8.0) return fail(ctx, DDEL_EINVAL, "topopt: r_min above 8 elements");
  cudaStream_t s = ctx->stream;
  const int64_t ne = ctx->S.n_elem, nd = ctx->S.n_dof;
  if (!ctx->rho_f) {
    if (dalloc(ctx, &ctx->rho_f, ne * 8) || dalloc(ctx, &ctx->dcf, ne * 8) ||
        dalloc(ctx, &ctx->dc, ne * 8) || dalloc(ctx, &ctx->dv, ne * 8) ||
        dalloc(ctx, &ctx->topo_u, nd * 8) || dalloc(ctx, &ctx->topo_out, 8 * 8))
      return fail(ctx, DDEL_ENOMEM, "topopt buffers");
    CK(cudaMallocHost(&ctx->h_topo, 8 * 8));
  }
  if (ctx->dv_rmin != ts->r_min) {  // dV/drho = Hbar^T 1
    launch_fill(ctx->dcf, ne, 1.0, s);
    launch_filter(ctx->T, ts->r_min, ctx->dcf, ctx->dv, 1, s);
    ctx->launches += 2;
    ctx->dv_rmin = ts->r_min;
  }
  launch_filter(ctx->T, ts->r_min, ts->rho, ctx->rho_f, 0, s);
  ctx->launches += 1;
  int rc = ddel_assemble(ctx, ctx->rho_f, 1);
  if (rc) return rc;
  rc = ddel_factor(ctx);
  if (rc) return rc;
  ddel_learner* learner = static_cast<ddel_learner*>(ts->learner);
  if (learner && (rc = ddel_learner_predict(learner, ctx->rho_f))) return rc;
  double* u = ts->u ? ts->u : ctx->topo_u;
  // adaptive tolerance from the last two compliances (Sec. 5, Table 3)
  const double tol0 = ctx->opt.tol;
  double tol = tol0;
  if (ts->tol_eta > 0.0) {
    const double tmax = std::max(ts->tol_max > 0.0 ? ts->tol_max : 1e-3, tol0);
    if (ts->iteration < 2 || !(ts->compliance != 0.0)) {
      tol = tmax;
    } else {
      const double d = ts->tol_eta * std::fabs(ts->compliance - ts->compliance_prev) / std::fabs(ts->compliance);
      tol = std::min(tmax, std::max(tol0, d));
    }
  }
  ctx->opt.tol = tol;
  rc = ddel_solve(ctx, nullptr, u, 1, stats);
  ctx->opt.tol = tol0;
  if (rc) return rc;
  ts->tol_used = tol;
  if (learner && (rc = ddel_learner_observe(learner, ctx->rho_f, u))) return rc;
  launch_dot(ctx->d_load, u, nd, ctx->partials, ctx->ticketK, ctx->topo_out + 3, s);
  launch_sensitivity(ctx->T, ctx->mat.E, ctx->mat.simp_p, ctx->rho_f, u, ctx->dcf, s);
  launch_filter(ctx->T, ts->r_min, ctx->dcf, ctx->dc, 1, s);
  if (ts->rho_phys)
    CK(cudaMemcpyAsync(ts->rho_phys, ctx->rho_f, ne * 8, cudaMemcpyDeviceToDevice, s));
  CK(launch_oc(ts->rho, ctx->dc, ctx->dv, ne, ts->volfrac * (double)ne, ctx->mat.rho_min, ts->move,
               ctx->partials, ctx->topo_out, s));
  ctx->launches += 4;
  CK(cudaMemcpyAsync(ctx->h_topo, ctx->topo_out, 4 * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  ts->lambda = ctx->h_topo[0];
  ts->volume = ctx->h_topo[1] / (double)ne;
  ts->change = ctx->h_topo[2];
  ts->compliance_prev = ts->compliance;
  ts->compliance = ctx->h_topo[3];
  ts->iteration += 1;
  return DDEL_OK;
}


namespace {
// Checkpoint file: header, densities, checksum (little-endian host layout).
struct CkpHeader {
  char magic[8];  // "DDELCKP1"
  uint32_t version, dim;
  int32_t nx, ny, nz, sub, plane_stress, pad;
  double E, nu, simp_p, rho_min;
  int64_t n_elem;
  double volfrac, r_min, move, compliance, volume, change, lambda;
  int64_t iteration;
  double tol_eta, tol_max, compliance_prev;  // version 2
};
constexpr char kCkpMagic[8] = {'D', 'D', 'E', 'L', 'C', 'K', 'P', '1'};
constexpr size_t kCkpHeaderV1 = offsetof(CkpHeader, tol_eta);

uint64_t fnv1a(const unsigned char* p, size_t n, uint64_t h = 1469598103934665603ull) {
  for (size_t i = 0; i < n; ++i) h = (h ^ p[i]) * 1099511628211ull;
  return h;
}

CkpHeader ckp_identity(const ddel_ctx* ctx) {
  CkpHeader h{};
  std::memcpy(h.magic, kCkpMagic, 8);
  h.version = 2;
  h.dim = (uint32_t)ctx->mesh.dim;
  h.nx = ctx->mesh.nx;
  h.ny = ctx->mesh.ny;
  h.nz = ctx->mesh.dim == 3 ? ctx->mesh.nz : 0;
  h.sub = ctx->mesh.sub;
  h.plane_stress = ctx->mat.plane_stress;
  h.E = ctx->mat.E;
  h.nu = ctx->mat.nu;
  h.simp_p = ctx->mat.simp_p;
  h.rho_min = ctx->mat.rho_min;
  h.n_elem = ctx->S.n_elem;
  return h;
}
}  // namespace

int ddel_checkpoint_save(const ddel_ctx* cctx, const ddel_topopt_state* ts, const char* path) {
  ddel_ctx* ctx = const_cast<ddel_ctx*>(cctx);
  if (!ctx || !ts || !ts->rho || !path) return DDEL_EINVAL;
  CkpHeader h = ckp_identity(ctx);
  h.volfrac = ts->volfrac;
  h.r_min = ts->r_min;
  h.move = ts->move;
  h.compliance = ts->compliance;
  h.volume = ts->volume;
  h.change = ts->change;
  h.lambda = ts->lambda;
  h.iteration = ts->iteration;
  h.tol_eta = ts->tol_eta;
  h.tol_max = ts->tol_max;
  h.compliance_prev = ts->compliance_prev;
  std::vector<double> rho(ctx->S.n_elem);
  CK(cudaMemcpyAsync(rho.data(), ts->rho, rho.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  uint64_t sum = fnv1a(reinterpret_cast<const unsigned char*>(&h), sizeof(h));
  sum = fnv1a(reinterpret_cast<const unsigned char*>(rho.data()), rho.size() * 8, sum);
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return fail(ctx, DDEL_EINVAL, "checkpoint: cannot write " + tmp);
  bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 && std::fwrite(rho.data(), 8, rho.size(), f) == rho.size() &&
            std::fwrite(&sum, sizeof(sum), 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return fail(ctx, DDEL_EINVAL, std::string("checkpoint: cannot write ") + path);
  }
  return DDEL_OK;
}

int ddel_checkpoint_load(ddel_ctx* ctx, ddel_topopt_state* ts, const char* path) {
  if (!ctx || !ts || !ts->rho || !path) return DDEL_EINVAL;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(ctx, DDEL_EINVAL, std::string("checkpoint: cannot read ") + path);
  CkpHeader h{};
  const CkpHeader want = ckp_identity(ctx);
  std::vector<double> rho;
  uint64_t sum = 0;
  // version 1 files end their header before the adaptive-tolerance fields
  bool ok = std::fread(&h, kCkpHeaderV1, 1, f) == 1 && std::memcmp(h.magic, kCkpMagic, 8) == 0 &&
            (h.version == 1 || h.version == 2) &&
            (h.version == 1 ||
             std::fread(reinterpret_cast<char*>(&h) + kCkpHeaderV1, sizeof(h) - kCkpHeaderV1, 1, f) == 1) &&
            h.n_elem == want.n_elem;
  const size_t hbytes = h.version == 1 ? kCkpHeaderV1 : sizeof(h);
  if (ok) {
    rho.resize(h.n_elem);
    ok = std::fread(rho.data(), 8, rho.size(), f) == rho.size() && std::fread(&sum, sizeof(sum), 1, f) == 1;
  }
  ok = ok && std::fgetc(f) == EOF;
  std::fclose(f);
  if (!ok) return fail(ctx, DDEL_EINVAL, std::string("checkpoint: not a checkpoint of this size: ") + path);
  uint64_t chk = fnv1a(reinterpret_cast<const unsigned char*>(&h), hbytes);
  chk = fnv1a(reinterpret_cast<const unsigned char*>(rho.data()), rho.size() * 8, chk);
  if (chk != sum) return fail(ctx, DDEL_EINVAL, "checkpoint: checksum mismatch");
  if (h.dim != want.dim || h.nx != want.nx || h.ny != want.ny || h.nz != want.nz || h.sub != want.sub ||
      h.plane_stress != want.plane_stress || h.E != want.E || h.nu != want.nu || h.simp_p != want.simp_p ||
      h.rho_min != want.rho_min)
    return fail(ctx, DDEL_EINVAL, "checkpoint: written for another mesh or material");
  CK(cudaMemcpyAsync(ts->rho, rho.data(), rho.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ts->volfrac = h.volfrac;
  ts->r_min = h.r_min;
  ts->move = h.move;
  ts->compliance = h.compliance;
  ts->volume = h.volume;
  ts->change = h.change;
  ts->lambda = h.lambda;
  ts->iteration = (int)h.iteration;
  if (h.version >= 2) {
    ts->tol_eta = h.tol_eta;
    ts->tol_max = h.tol_max;
    ts->compliance_prev = h.compliance_prev;
  } else {
    ts->compliance_prev = h.compliance;
  }
  ctx->u_valid = false;  // a WARM start must not pick up an unrelated solution
  return DDEL_OK;
}


int ddel_batch_solve(ddel_ctx* const* ctxs, int n, double* const* u, ddel_stats* stats) {
  if (!ctxs || n <= 0) return DDEL_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i] || !ctxs[i]->assembled) return ctxs[i] ? fail(ctxs[i], DDEL_ESTATE, "assemble first") : DDEL_EINVAL;
  std::vector<int> prec(n), checks(n, 0), state(n, 0);  // state: 0 PCG running, 1 finished
  std::vector<bool> a32(n, false);
  // 1. all factorisations in flight at once (one stream per context)
  for (int i = 0; i < n; ++i) {
    ddel_ctx* c = ctxs[i];
    prec[i] = c->opt.precision == DDEL_FP32 ? 1 : 0;
    int rc = factor_launch(c, prec[i]);
    if (rc) return rc;
  }
  for (int i = 0; i < n; ++i) {
    ddel_ctx* c = ctxs[i];
    int rc = factor_check(c, prec[i]);
    if (rc == DDEL_ENOTSPD && prec[i] == 1) {
      prec[i] = 0;
      rc = factor_prec(c, 0);
    }
    if (rc) return rc;
    c->active_prec = prec[i];
    c->mixed_ready = false;
  }
  // 2. right-hand sides, condensation, PCG start
  for (int i = 0; i < n; ++i) {
    ddel_ctx* ctx = ctxs[i];
    cudaStream_t s = ctx->stream;
    const int64_t nd = ctx->S.n_dof;
    CK(cudaEventRecord(ctx->ev[0], s));
    CK(cudaMemcpyAsync(ctx->d_f, ctx->d_load, nd * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(ctx->d_u, 0, nd * 8, s));
    launch_apply_K(ctx->T, ctx->F, ctx->d_u, ctx->d_f, ctx->d_r, 1, ctx->partials, ctx->ticketK,
                   ctx->nrm, s, ctx->nblk);
    set_tol_kernel<<<1, 1, 0, s>>>(ctx->st, ctx->nrm, ctx->opt.tol, ctx->opt.inner_tol, prec[i],
                                   ctx->opt.max_it);
    ctx->launches += 2;
    condense(ctx, prec[i], ctx->d_r, ctx->g);
    int rc = pcg_start(ctx, prec[i], ctx->g, false);
    if (rc) return rc;
    rc = pcg_issue(ctx, prec[i], false);
    if (rc) return rc;
  }
  // 3. round robin: relaunch each unfinished context as soon as its last
  //    batch of iterations has reported, finish the others
  int remaining = n;
  while (remaining > 0) {
    bool progressed = false;
    for (int i = 0; i < n; ++i) {
      if (state[i]) continue;
      ddel_ctx* ctx = ctxs[i];
      const cudaError_t q = cudaEventQuery(ctx->ev[7]);
      if (q == cudaErrorNotReady) continue;
      CK(q);
      progressed = true;
      const int per = pcg_per(ctx);
      if (!ctx->h_st->done && ++checks[i] < ctx->opt.max_it / per + 2) {
        int rc = pcg_issue(ctx, prec[i], false);
        if (rc) return rc;
        continue;
      }
      state[i] = 1;
      --remaining;
      cudaStream_t s = ctx->stream;
      back_substitute(ctx, prec[i], ctx->d_r, ctx->x, ctx->d_d);
      launch_axpy(ctx->S.n_dof, 1.0, ctx->d_d, ctx->d_u, s);
      launch_apply_K(ctx->T, ctx->F, ctx->d_u, ctx->d_f, ctx->d_r, 1, ctx->partials, ctx->ticketK,
                     ctx->nrm, s, ctx->nblk);
      ctx->launches += 2;
      CK(cudaMemcpyAsync(ctx->h_nrm, ctx->nrm, 16, cudaMemcpyDeviceToHost, s));
      CK(cudaEventRecord(ctx->ev[6], s));
    }
    if (!progressed) std::this_thread::yield();
  }
  // 4. statistics; a context that missed the tolerance is finished by the
  //    ordinary refinement loop
  int status = DDEL_OK;
  for (int i = 0; i < n; ++i) {
    ddel_ctx* ctx = ctxs[i];
    CK(cudaEventSynchronize(ctx->ev[6]));
    ddel_stats st{};
    st.bad_subdomain = -1;
    st.iters = ctx->h_st->it;
    st.cycles = 1;
    const double fn = ctx->h_nrm[1];
    st.relres = fn > 0 ? ctx->h_nrm[0] / fn : 0.0;
    st.pcg_relres = fn > 0 ? std::sqrt(ctx->h_st->rr) / fn : 0.0;
    st.t_total_ms = elapsed(ctx->ev[0], ctx->ev[6]);
    st.status = DDEL_OK;
    if (!(st.relres <= ctx->opt.tol) && fn > 0) {
      const int rc = ddel_solve(ctx, nullptr, u && u[i] ? u[i] : ctx->d_d, 1, &st);
      if (rc && status == DDEL_OK) status = rc;
      if (u && u[i]) {
        if (stats) stats[i] = st;
        continue;
      }
      CK(cudaMemcpyAsync(ctx->d_u, ctx->d_d, ctx->S.n_dof * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    if (u && u[i])
      CK(cudaMemcpyAsync(u[i], ctx->d_u, ctx->S.n_dof * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    if (stats) stats[i] = st;
  }
  for (int i = 0; i < n; ++i) {
    ddel_ctx* ctx = ctxs[i];
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return status;
}

int ddel_batch_solve_persistent(ddel_ctx* const* ctxs, int n, double* const* u, ddel_stats* stats) {
  if (!ctxs || n <= 0) return DDEL_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i] || !ctxs[i]->assembled) return ctxs[i] ? fail(ctxs[i], DDEL_ESTATE, "assemble first") : DDEL_EINVAL;
  // 1. every factorisation in flight at once (one stream per context)
  for (int i = 0; i < n; ++i) {
    int rc = factor_launch(ctxs[i], 0);
    if (rc) return rc;
  }
  for (int i = 0; i < n; ++i) {
    ddel_ctx* c = ctxs[i];
    int rc = factor_check(c, 0);
    if (rc) return rc;
    c->active_prec = 0;
    c->mixed_ready = false;
    // the persistent form runs the double-float explicit apply without a
    // coarse space; any other configuration takes the stream-per-problem path
    // ... and with the tile shape of its own launches (by ring size), so that
    // its results equal those of single solves bit for bit
    const int nr = explicit_ring_size(c->T);
    if (c->T.dim != 2 || !c->explicit_ok[0] || !c->df_ok || c->ck_in > 0 ||
        explicit_split(c->T, c->opt.schur_split) != (nr <= 64 ? 1 : 2))
      return ddel_batch_solve(ctxs, n, u, stats);
  }
  // 2. right-hand sides, condensation, PCG start on each context's stream
  size_t smem = 0;
  std::vector<BatchProb> hp(n);
  std::vector<int> pre(2 * n + 2, 0);
  int max_it = 0;
  for (int i = 0; i < n; ++i) {
    ddel_ctx* ctx = ctxs[i];
    cudaStream_t s = ctx->stream;
    const int64_t nd = ctx->S.n_dof;
    CK(cudaEventRecord(ctx->ev[0], s));
    CK(cudaMemcpyAsync(ctx->d_f, ctx->d_load, nd * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(ctx->d_u, 0, nd * 8, s));
    launch_apply_K(ctx->T, ctx->F, ctx->d_u, ctx->d_f, ctx->d_r, 1, ctx->partials, ctx->ticketK, ctx->nrm, s,
                   ctx->nblk);
    set_tol_kernel<<<1, 1, 0, s>>>(ctx->st, ctx->nrm, ctx->opt.tol, ctx->opt.inner_tol, 0, ctx->opt.max_it);
    condense(ctx, 0, ctx->d_r, ctx->g);
    launch_pcg_init(ctx->T, ctx->F, ctx->g, ctx->x, ctx->r, ctx->z, ctx->p, ctx->sv, ctx->st, pcg_partials(ctx, 0), s,
                    ctx->nupd, CoarseDev());
    ctx->launches += 3;
    BatchProb& b = hp[i];
    b.t = ctx->T;
    b.f = ctx->F;
    b.sexp_df = ctx->sexp_df;
    b.ring = reinterpret_cast<double*>(ctx->ring);
    b.x = ctx->x;
    b.r = ctx->r;
    b.u = ctx->z;
    b.p = ctx->p;
    b.sv = ctx->sv;
    b.st = ctx->st;
    b.pd = ctx->pcg_pd;
    b.pu = ctx->pcg_pu;
    b.nr = explicit_ring_size(ctx->T);
    b.n_schur = (b.nr <= 64 ? 1 : 2) * ctx->T.n_sub;  // one CTA per ring of 64
    b.n_upd = ctx->nupd;
    pre[i + 1] = pre[i] + batch_schur_tiles(b.n_schur);
    pre[n + 2 + i] = pre[n + 1 + i] + b.n_upd;
    smem = std::max(smem, batch_pcg_smem(ctx->T));
    max_it = std::max(max_it, ctx->opt.max_it);
  }
  ddel_ctx* c0 = ctxs[0];
  ddel_ctx* ctx = c0;  // where the error checks record their message
  for (int i = 0; i < n; ++i) CK(cudaStreamSynchronize(ctxs[i]->stream));
  cudaStream_t s0 = c0->stream;
  const int per = pcg_per(c0);
  const int bps = batch_pcg_blocks_per_sm(smem);
  int dev = 0, nsm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (bps < 1) return fail(c0, DDEL_ECUDA, "persistent batch kernel does not fit an SM");
  BatchProb* d_probs = nullptr;
  int* d_pre = nullptr;
  unsigned* d_cnt = nullptr;
  std::vector<PcgState> hst(n);
  auto cleanup = [&]() {
    if (d_probs) cudaFree(d_probs);
    if (d_pre) cudaFree(d_pre);
    if (d_cnt) cudaFree(d_cnt);
  };
  if (cudaMalloc(&d_probs, n * sizeof(BatchProb)) != cudaSuccess || cudaMalloc(&d_pre, pre.size() * 4) != cudaSuccess ||
      cudaMalloc(&d_cnt, (2 * n + 2) * 4) != cudaSuccess) {
    cleanup();
    return fail(c0, DDEL_ENOMEM, "persistent batch tables");
  }
  const int init[2] = {0, 0x7fffffff};
  CK(cudaMemcpyAsync(c0->err, init, sizeof(init), cudaMemcpyHostToDevice, s0));
  // 3. launches of `per` iterations of every problem until all have stopped
  const int max_launch = max_it / per + 2;
  int launches = 0;
  std::vector<int> active(n);
  for (int i = 0; i < n; ++i) active[i] = i;
  std::vector<BatchProb> ap;
  std::vector<int> apre;
  for (; launches < max_launch; ++launches) {
    // the problems still iterating, in batch order (finished ones leave the queue)
    const int na = (int)active.size();
    ap.assign(na, BatchProb{});
    apre.assign(2 * na + 2, 0);
    for (int a = 0; a < na; ++a) {
      ap[a] = hp[active[a]];
      apre[a + 1] = apre[a] + batch_schur_tiles(ap[a].n_schur);
      apre[na + 2 + a] = apre[na + 1 + a] + ap[a].n_upd;
    }
    CK(cudaMemcpyAsync(d_probs, ap.data(), na * sizeof(BatchProb), cudaMemcpyHostToDevice, s0));
    CK(cudaMemcpyAsync(d_pre, apre.data(), apre.size() * 4, cudaMemcpyHostToDevice, s0));
    CK(cudaMemsetAsync(d_cnt, 0, (2 * na + 2) * 4, s0));
    cudaError_t e = launch_batch_pcg(d_probs, na, d_pre, per, d_cnt, c0->err, bps * nsm, smem, s0);
    if (e != cudaSuccess) {
      cleanup();
      return fail(c0, DDEL_ECUDA, std::string("persistent batch launch: ") + cudaGetErrorString(e));
    }
    for (int i : active)
      CK(cudaMemcpyAsync(&hst[i], ctxs[i]->st, sizeof(PcgState), cudaMemcpyDeviceToHost, s0));
    CK(cudaMemcpyAsync(c0->h_err, c0->err, 8, cudaMemcpyDeviceToHost, s0));
    CK(cudaStreamSynchronize(s0));
    for (int i : active) ctxs[i]->launches += 2 * per;
    if (c0->h_err[0] == kErrTimeout) {
      cleanup();
      return fail(c0, DDEL_ETIMEOUT, "a bounded wait of the persistent batch kernel ran out");
    }
    std::vector<int> still;
    for (int i : active)
      if (!hst[i].done) still.push_back(i);
    active.swap(still);
    if (active.empty()) break;
  }
  cleanup();
  // 4. back-substitution and the FP64 residual of every problem; a problem
  //    that missed its tolerance is finished by the refinement loop
  int status = DDEL_OK;
  for (int i = 0; i < n; ++i) {
    ddel_ctx* ctx = ctxs[i];
    cudaStream_t s = ctx->stream;
    *ctx->h_st = hst[i];
    back_substitute(ctx, 0, ctx->d_r, ctx->x, ctx->d_d);
    launch_axpy(ctx->S.n_dof, 1.0, ctx->d_d, ctx->d_u, s);
    launch_apply_K(ctx->T, ctx->F, ctx->d_u, ctx->d_f, ctx->d_r, 1, ctx->partials, ctx->ticketK, ctx->nrm, s,
                   ctx->nblk);
    ctx->launches += 3;
    CK(cudaMemcpyAsync(ctx->h_nrm, ctx->nrm, 16, cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(ctx->ev[6], s));
  }
  for (int i = 0; i < n; ++i) {
    ddel_ctx* ctx = ctxs[i];
    CK(cudaEventSynchronize(ctx->ev[6]));
    ddel_stats st{};
    st.bad_subdomain = -1;
    st.iters = hst[i].it;
    st.cycles = 1;
    const double fn = ctx->h_nrm[1];
    st.relres = fn > 0 ? ctx->h_nrm[0] / fn : 0.0;
    st.pcg_relres = fn > 0 ? std::sqrt(hst[i].rr) / fn : 0.0;
    st.t_total_ms = elapsed(ctx->ev[0], ctx->ev[6]);
    st.t_factor_ms = ctx->t_factor_ms;
    st.status = DDEL_OK;
    if (!(st.relres <= ctx->opt.tol) && fn > 0) {
      const int rc2 = ddel_solve(ctx, nullptr, u && u[i] ? u[i] : ctx->d_d, 1, &st);
      if (rc2 && status == DDEL_OK) status = rc2;
      if (u && u[i]) {
        if (stats) stats[i] = st;
        continue;
      }
      CK(cudaMemcpyAsync(ctx->d_u, ctx->d_d, ctx->S.n_dof * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    if (u && u[i])
      CK(cudaMemcpyAsync(u[i], ctx->d_u, ctx->S.n_dof * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    if (stats) stats[i] = st;
  }
  for (int i = 0; i < n; ++i) CK(cudaStreamSynchronize(ctxs[i]->stream));
  return status;
}

int ddel_autotune(ddel_ctx* ctx, const char* cache_path, int* chosen_mode, int* chosen_check,
                  int* from_cache) {
  if (!ctx) return DDEL_EINVAL;
  if (!ctx->assembled) return fail(ctx, DDEL_ESTATE, "assemble before autotune");
  const int prec = ctx->opt.precision == DDEL_FP32 ? 1 : 0;
  char key[128];
  std::snprintf(key, sizeof(key), "%d %d %d %d %d", ctx->S.dim, ctx->S.sub, ctx->S.BP, ctx->S.n_sub,
                ctx->opt.precision);
  if (from_cache) *from_cache = 0;
  auto apply = [&](int mode, int check, int tf, int split) {
    ctx->opt.schur_mode = mode;
    ctx->opt.check_every = check;
    ctx->opt.tensor_form = tf;
    ctx->opt.schur_split = split;
    ctx->factored[0] = ctx->factored[1] = false;
    if (chosen_mode) *chosen_mode = mode;
    if (chosen_check) *chosen_check = check;
  };
  if (cache_path) {
    if (FILE* fp = std::fopen(cache_path, "r")) {
      char line[256];
      int mode = -1, check = 0, tform = ctx->opt.tensor_form, split = ctx->opt.schur_split;
      while (std::fgets(line, sizeof(line), fp)) {
        int d, s, b, n, p, m, c, tf = ctx->opt.tensor_form, sp = ctx->opt.schur_split;
        const int got = std::sscanf(line, "%d %d %d %d %d %d %d %d %d", &d, &s, &b, &n, &p, &m, &c, &tf, &sp);
        if (got >= 7) {  // lines without the last fields keep the context's settings
          char k2[128];
          std::snprintf(k2, sizeof(k2), "%d %d %d %d %d", d, s, b, n, p);
          if (std::strcmp(k2, key) == 0) {
            mode = m;
            check = c;
            tform = tf;
            split = sp;
          }
        }
      }
      std::fclose(fp);
      if (mode >= 0) {
        apply(mode, check, tform, split);
        if (from_cache) *from_cache = 1;
        return DDEL_OK;
      }
    }
  }
  // iteration count of the problem: one solve in the current configuration
  ddel_options saved = ctx->opt;
  int rc = ddel_factor(ctx);
  if (rc) return rc;
  ddel_stats st{};
  rc = ddel_solve(ctx, nullptr, ctx->d_d, 1, &st);
  if (rc != DDEL_OK && rc != DDEL_ENOCONV) return rc;
  const double n_iter = st.iters > 0 ? st.iters : 1;
  const bool has_explicit = explicit_ring_size(ctx->T) > 0;
  // candidates: Schur form, S_i formation on the tensor cores or the FP64
  // pipe, and for the native FP64 explicit apply its tile shape (CTAs per
  // subdomain)
  struct Cand {
    int mode, tf, split;
  };
  const bool tc_ok = tensor_form_available(ctx->T);
  std::vector<Cand> forms = {{DDEL_SCHUR_IMPLICIT, saved.tensor_form, saved.schur_split}};
  if (has_explicit && prec == 0) {
    forms.push_back({DDEL_SCHUR_AUTO, 0, saved.schur_split});
    if (tc_ok && explicit_ring_size(ctx->T) > 128) forms.push_back({DDEL_SCHUR_AUTO, 1, saved.schur_split});
  }
  if (has_explicit) {
    for (int split : {1, 2, 4}) {
      if (prec == 0 ? explicit_split(ctx->T, split) != split : split != 2) continue;
      forms.push_back({DDEL_SCHUR_EXPLICIT, 0, split});
      if (tc_ok) forms.push_back({DDEL_SCHUR_EXPLICIT, prec ? 2 : 1, split});
    }
  }
  const int checks[3] = {8, 16, 32};
  double best = 1e300;
  int best_mode = saved.schur_mode, best_check = saved.check_every, best_tf = saved.tensor_form,
      best_split = saved.schur_split;
  cudaStream_t s = ctx->stream;
  for (const auto& fm : forms)
    for (int check : checks) {
      const int mode = fm.mode;
      ctx->opt = saved;
      ctx->opt.schur_mode = mode;
      ctx->opt.check_every = check;
      ctx->opt.tensor_form = fm.tf;
      ctx->opt.schur_split = fm.split;
      CK(cudaEventRecord(ctx->ev[0], s));
      rc = ddel_factor(ctx);
      if (rc) return rc;
      CK(cudaEventRecord(ctx->ev[1], s));
      // 48 iterations of this form (tolerance 0: nothing converges early)
      set_tol_abs_kernel<<<1, 1, 0, s>>>(ctx->st, 0.0, 48);
      const int p = ctx->active_prec;
      launch_apply_K(ctx->T, ctx->F, ctx->d_u, ctx->d_load, ctx->d_r, 1, ctx->partials,
                     ctx->ticketK, ctx->nrm, s, ctx->nblk);
      condense(ctx, p, ctx->d_load, ctx->g);
      rc = pcg_start(ctx, p, ctx->g, false);
      if (rc) return rc;
      CK(cudaEventRecord(ctx->ev[2], s));
      int done_it = 0;
      while (done_it < 48) {
        rc = pcg_issue(ctx, p, false);
        if (rc) return rc;
        done_it += check;
      }
      CK(cudaEventRecord(ctx->ev[3], s));
      CK(cudaEventSynchronize(ctx->ev[3]));
      const double t_fact = elapsed(ctx->ev[0], ctx->ev[1]);
      const double it_done = ctx->h_st->it > 0 ? ctx->h_st->it : 1;
      const double t_it = elapsed(ctx->ev[2], ctx->ev[3]) / it_done;
      // graph launches cover whole batches: add the expected idle tail
      const double predicted = t_fact + (n_iter + 0.5 * check) * t_it;
      if (predicted < best) {
        best = predicted;
        best_mode = mode;
        best_check = check;
        best_tf = fm.tf;
        best_split = fm.split;
      }
    }
  ctx->opt = saved;
  apply(best_mode, best_check, best_tf, best_split);
  if (cache_path) {
    if (FILE* fp = std::fopen(cache_path, "a")) {
      std::fprintf(fp, "%s %d %d %d %d\n", key, best_mode, best_check, best_tf, best_split);
      std::fclose(fp);
    }
  }
  return DDEL_OK;
}

void ddel_default_gmres_options(ddel_gmres_options* o) {
  if (!o) return;
  o->precond = DDEL_PREC_GLOBAL;
  o->lanczos_steps = 8;
  o->inner_tol = 1e-3;
  o->mass_tol = 1e-13;
  o->global_scaling = 1;
  o->tol = 1e-6;
  o->max_it = 300;
}

int ddel_global_precond_apply(ddel_ctx* ctx, const ddel_gmres_options* opt, const double* r, double* z,
                              double* lanczos_out) {
  if (!ctx || !opt || !r || !z) return DDEL_EINVAL;
  if (!ctx->assembled) return fail(ctx, DDEL_ESTATE, "assemble first");
  ddel_gmres_options o = *opt;
  o.precond = DDEL_PREC_GLOBAL;
  int rc = gp_check_options(ctx, &o);
  if (rc) return rc;
  if ((rc = gp_build(ctx))) return rc;
  CK(launch_global_prec(ctx->gp, r, z, ctx->F.diagG, ctx->opt.theta, o.lanczos_steps, o.inner_tol, o.mass_tol,
                        o.global_scaling ? 1 : 0, ctx->gp_out, ctx->stream));
  ctx->launches += 1;
  if (lanczos_out) {
    const size_t per = 2 + 3 * kLz;
    CK(cudaMemcpyAsync(ctx->h_gp_out, ctx->gp_out, ctx->gp.ncomp * per * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    std::memcpy(lanczos_out, ctx->h_gp_out, ctx->gp.ncomp * per * 8);
  }
  return DDEL_OK;
}

int ddel_gmres_solve(ddel_ctx* ctx, const ddel_gmres_options* opt, const double* f, double* u, int on_device,
                     ddel_gmres_stats* stats) {
  if (!ctx || !opt || !u) return DDEL_EINVAL;
  const int prec = ctx->active_prec;
  if (!ctx->factored[prec]) return fail(ctx, DDEL_ESTATE, "factor before solve");
  int rc = gp_check_options(ctx, opt);
  if (rc) return rc;
  if (!(opt->tol > 0.0) || opt->max_it < 1 || opt->max_it > 2000)
    return fail(ctx, DDEL_EINVAL, "tol > 0 and max_it in 1..2000");
  if (opt->precond == DDEL_PREC_GLOBAL && (rc = gp_build(ctx))) return rc;
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->S.n_dof, ng = ctx->T.n_gamma;
  const int cap = opt->max_it;
  if (ctx->gm_cap < cap) {
    for (double** p : {&ctx->gm_V, &ctx->gm_Z, &ctx->gm_w, &ctx->gm_h, &ctx->gm_part, &ctx->gm_vg, &ctx->gm_zg})
      if (*p) {
        cudaFree(*p);
        *p = nullptr;
      }
    if (ctx->h_gm) cudaFreeHost(ctx->h_gm);
    ctx->h_gm = nullptr;
    ctx->gm_cap = 0;
    if (cudaMalloc(&ctx->gm_V, (size_t)(cap + 1) * n * 8) != cudaSuccess ||
        cudaMalloc(&ctx->gm_Z, (size_t)cap * n * 8) != cudaSuccess ||
        cudaMalloc(&ctx->gm_w, (size_t)n * 8) != cudaSuccess ||
        cudaMalloc(&ctx->gm_h, (size_t)(2 * cap + 8) * 8) != cudaSuccess ||
        cudaMalloc(&ctx->gm_part, multi_dot_partials(cap + 1) * 8) != cudaSuccess ||
        cudaMalloc(&ctx->gm_vg, (size_t)(ng + 1) * 8) != cudaSuccess ||
        cudaMalloc(&ctx->gm_zg, (size_t)(ng + 1) * 8) != cudaSuccess ||
        cudaMallocHost(&ctx->h_gm, (size_t)(2 * cap + 8) * 8) != cudaSuccess)
      return fail(ctx, DDEL_ENOMEM, "FGMRES basis allocation");
    ctx->gm_cap = cap;
  }
  double *V = ctx->gm_V, *Z = ctx->gm_Z, *w = ctx->gm_w, *h = ctx->gm_h, *h2 = ctx->gm_h + cap + 2;
  ddel_gmres_stats st{};
  st.inner_min = 1 << 30;
  long long inner_sum = 0, inner_cnt = 0;
  CK(cudaEventRecord(ctx->ev[0], s));
  if (!f)
    CK(cudaMemcpyAsync(ctx->d_f, ctx->d_load, n * 8, cudaMemcpyDeviceToDevice, s));
  else
    CK(cudaMemcpyAsync(ctx->d_f, f, n * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  launch_multi_dot(ctx->d_f, 0, 1, ctx->d_f, n, ctx->gm_part, h, 0, s);
  CK(cudaMemcpyAsync(ctx->h_gm, h, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double beta0 = std::sqrt(ctx->h_gm[0]);
  std::vector<double> H((size_t)(cap + 1) * cap, 0.0), cs(cap), sn(cap), e(cap + 1, 0.0);
  int k_done = 0;
  st.status = DDEL_ENOCONV;
  if (beta0 == 0.0) {
    CK(cudaMemsetAsync(ctx->d_u, 0, n * 8, s));
    st.status = DDEL_OK;
  } else {
    launch_scale_gm(ctx->d_f, V, n, nullptr, -1, beta0, s);
    e[0] = beta0;
    const int per = 2 + 3 * kLz;
    for (int k = 0; k < cap; ++k) {
      double* vk = V + (size_t)k * n;
      double* zk = Z + (size_t)k * n;
      // z_k = P~^-1 v_k: S~^-1 on the interface part, then the interior solves
      launch_gather_gamma(ctx->T.gamma_dof, ng, vk, ctx->gm_vg, s);
      if (opt->precond == DDEL_PREC_IDENTITY) {
        CK(cudaMemcpyAsync(ctx->gm_zg, ctx->gm_vg, ng * 8, cudaMemcpyDeviceToDevice, s));
      } else if (opt->precond == DDEL_PREC_FACE) {
        launch_precond(ctx->T, ctx->F, ctx->gm_vg, ctx->gm_zg, s);
      } else {
        CK(launch_global_prec(ctx->gp, ctx->gm_vg, ctx->gm_zg, ctx->F.diagG, ctx->opt.theta, opt->lanczos_steps,
                              opt->inner_tol, opt->mass_tol, opt->global_scaling ? 1 : 0, ctx->gp_out, s));
      }
      back_substitute(ctx, prec, vk, ctx->gm_zg, zk);
      // w = K z_k, then classical Gram-Schmidt twice against v_0 .. v_k
      launch_apply_K(ctx->T, ctx->F, zk, nullptr, w, 0, ctx->partials, ctx->ticketK, ctx->nrm, s, ctx->nblk);
      launch_multi_dot(V, n, k + 1, w, n, ctx->gm_part, h, 0, s);
      launch_multi_axpy(V, n, k + 1, h, w, n, 0, s);
      launch_multi_dot(V, n, k + 1, w, n, ctx->gm_part, h2, 0, s);
      launch_multi_axpy(V, n, k + 1, h2, w, n, 0, s);
      launch_multi_dot(w, 0, 1, w, n, ctx->gm_part, h2 + k + 1, 0, s);
      ctx->launches += 12;
      CK(cudaMemcpyAsync(ctx->h_gm, h, (size_t)(2 * cap + 4) * 8, cudaMemcpyDeviceToHost, s));
      if (opt->precond == DDEL_PREC_GLOBAL)
        CK(cudaMemcpyAsync(ctx->h_gp_out, ctx->gp_out, (size_t)ctx->gp.ncomp * per * 8, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      CK(cudaGetLastError());
      if (opt->precond == DDEL_PREC_GLOBAL) {
        for (int c = 0; c < ctx->gp.ncomp; ++c) {
          const double* o = ctx->h_gp_out + c * per;
          const int m = (int)o[0];
          st.lanczos_m = m;
          for (int j = 0; j < m; ++j) {
            const int it = (int)o[2 + 2 * kLz + j];
            st.inner_min = std::min(st.inner_min, it);
            st.inner_max = std::max(st.inner_max, it);
            inner_sum += it;
            inner_cnt += 1;
          }
        }
      }
      const double* hh = ctx->h_gm;
      const double* hh2 = ctx->h_gm + cap + 2;
      for (int j = 0; j <= k; ++j) H[(size_t)j * cap + k] = hh[j] + hh2[j];
      const double hn = std::sqrt(std::max(hh2[k + 1], 0.0));
      H[(size_t)(k + 1) * cap + k] = hn;
      if (hn > 0.0 && k + 1 <= cap) launch_scale_gm(w, V + (size_t)(k + 1) * n, n, nullptr, -1, hn, s);
      // Givens rotations of the Hessenberg column (Saad)
      for (int j = 0; j < k; ++j) {
        const double a = H[(size_t)j * cap + k], b = H[(size_t)(j + 1) * cap + k];
        H[(size_t)j * cap + k] = cs[j] * a + sn[j] * b;
        H[(size_t)(j + 1) * cap + k] = -sn[j] * a + cs[j] * b;
      }
      const double a = H[(size_t)k * cap + k], b = H[(size_t)(k + 1) * cap + k];
      const double den = std::hypot(a, b);
      cs[k] = a / den;
      sn[k] = b / den;
      H[(size_t)k * cap + k] = den;
      H[(size_t)(k + 1) * cap + k] = 0.0;
      e[k + 1] = -sn[k] * e[k];
      e[k] = cs[k] * e[k];
      k_done = k + 1;
      st.est_relres = std::fabs(e[k + 1]) / beta0;
      if (std::fabs(e[k + 1]) <= opt->tol * beta0 || !(hn > 0.0)) {
        st.status = DDEL_OK;
        break;
      }
    }
    // y = R^-1 e, u = Z y
    std::vector<double> y(k_done, 0.0);
    for (int i = k_done - 1; i >= 0; --i) {
      double v = e[i];
      for (int j = i + 1; j < k_done; ++j) v -= H[(size_t)i * cap + j] * y[j];
      y[i] = v / H[(size_t)i * cap + i];
    }
    std::memcpy(ctx->h_gm, y.data(), k_done * 8);
    CK(cudaMemcpyAsync(h, ctx->h_gm, k_done * 8, cudaMemcpyHostToDevice, s));
    launch_multi_axpy(Z, n, k_done, h, ctx->d_u, n, 1, s);
  }
  st.iters = k_done;
  // the FP64 residual of the result
  launch_apply_K(ctx->T, ctx->F, ctx->d_u, ctx->d_f, ctx->d_r, 1, ctx->partials, ctx->ticketK, ctx->nrm, s,
                 ctx->nblk);
  ctx->launches += 2;
  CK(cudaMemcpyAsync(ctx->h_nrm, ctx->nrm, 16, cudaMemcpyDeviceToHost, s));
  if (on_device)
    CK(cudaMemcpyAsync(u, ctx->d_u, n * 8, cudaMemcpyDeviceToDevice, s));
  else
    CK(cudaMemcpyAsync(u, ctx->d_u, n * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(ctx->ev[6], s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  st.relres = ctx->h_nrm[1] > 0 ? ctx->h_nrm[0] / ctx->h_nrm[1] : 0.0;
  st.t_ms = elapsed(ctx->ev[0], ctx->ev[6]);
  if (inner_cnt == 0) st.inner_min = 0;
  st.inner_mean = inner_cnt ? (double)inner_sum / inner_cnt : 0.0;
  ctx->u_valid = false;
  if (stats) *stats = st;
  return st.status;
}

int ddel_apply_K(ddel_ctx* ctx, const double* x, double* y) {
  if (!ctx || !x || !y) return DDEL_EINVAL;
  if (!ctx->assembled) return fail(ctx, DDEL_ESTATE, "assemble first");
  launch_apply_K(ctx->T, ctx->F, x, nullptr, y, 0, ctx->partials, ctx->ticketK, ctx->nrm,
                 ctx->stream, ctx->nblk);
  ctx->launches += 1;
  CK(cudaGetLastError());
  return DDEL_OK;
}

int ddel_condense(ddel_ctx* ctx, const double* f, double* g) {
  if (!ctx || !f || !g) return DDEL_EINVAL;
  if (!ctx->factored[ctx->active_prec]) return fail(ctx, DDEL_ESTATE, "factor first");
  condense(ctx, ctx->active_prec, f, g);
  CK(cudaGetLastError());
  return DDEL_OK;
}

int ddel_schur_apply(ddel_ctx* ctx, const double* x, double* y) {
  if (!ctx || !x || !y) return DDEL_EINVAL;
  const int prec = ctx->active_prec;
  if (!ctx->factored[prec]) return fail(ctx, DDEL_ESTATE, "factor first");
  SchurIO io = make_io(ctx);
  io.x = x;
  schur_dispatch(ctx, prec, false, io, ctx->stream);
  launch_gamma_sum(ctx->T, apply_prec(ctx, prec, false), io.ring_out, nullptr, 1.0, y, ctx->stream);
  ctx->launches += 2;
  CK(cudaGetLastError());
  return DDEL_OK;
}

int ddel_schur_apply_ring(ddel_ctx* ctx, const double* x) {
  if (!ctx || !x) return DDEL_EINVAL;
  const int prec = ctx->active_prec;
  if (!ctx->factored[prec]) return fail(ctx, DDEL_ESTATE, "factor first");
  SchurIO io = make_io(ctx);
  io.x = x;
  schur_dispatch(ctx, prec, false, io, ctx->stream);
  ctx->launches += 1;
  CK(cudaGetLastError());
  return DDEL_OK;
}

int ddel_set_coarse(ddel_ctx* ctx, const double* Z, int k, int flags, int on_device) {
  if (!ctx) return DDEL_EINVAL;
  if (k < 0 || k > kMaxCoarse || (k > 0 && !Z))
    return fail(ctx, DDEL_EINVAL, "coarse space: need 0 <= k <= DDEL_MAX_COARSE and Z");
  if (k > 0 && (flags <= 0 || (flags & ~(DDEL_COARSE_X0 | DDEL_COARSE_CORRECT | DDEL_COARSE_DEFLATE)) ||
                ((flags & DDEL_COARSE_CORRECT) && (flags & DDEL_COARSE_DEFLATE))))
    return fail(ctx, DDEL_EINVAL,
                "coarse space: flags = DDEL_COARSE_X0 and/or one of DDEL_COARSE_CORRECT, DDEL_COARSE_DEFLATE");
  ctx->ck = 0;
  ctx->coarse_prec = -1;
  ctx->ck_in = k;
  ctx->coarse_flags = k > 0 ? flags : 0;
  if (k == 0) return DDEL_OK;
  const int64_t n = ctx->T.n_gamma;
  if (!ctx->cZ) {
    const size_t vb = (size_t)kMaxCoarse * n * 8;
    if (dalloc(ctx, &ctx->cZ, vb) || dalloc(ctx, &ctx->cQ1, vb) || dalloc(ctx, &ctx->cQ, vb) ||
        dalloc(ctx, &ctx->cSQ, vb) || dalloc(ctx, &ctx->csmall, 7 * kMaxCoarse * kMaxCoarse * 8) ||
        dalloc(ctx, &ctx->cflags, 4 * sizeof(int)) || dalloc(ctx, &ctx->cticket, 16)) {
      ctx->ck_in = 0;
      return fail(ctx, DDEL_ENOMEM, "coarse space allocation");
    }
    if (cudaMallocHost(&ctx->h_cflags, 4 * sizeof(int)) != cudaSuccess) {
      ctx->ck_in = 0;
      return fail(ctx, DDEL_ENOMEM, "coarse space allocation");
    }
    CK(cudaMemsetAsync(ctx->cticket, 0, 16, ctx->stream));
  }
  CK(cudaMemcpyAsync(ctx->cZ, Z, (size_t)k * n * 8,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  if (!on_device) CK(cudaStreamSynchronize(ctx->stream));
  return DDEL_OK;
}

int ddel_precond_apply(ddel_ctx* ctx, const double* r, double* z) {
  if (!ctx || !r || !z) return DDEL_EINVAL;
  if (!ctx->assembled) return fail(ctx, DDEL_ESTATE, "assemble first");
  launch_precond(ctx->T, ctx->F, r, z, ctx->stream);
  ctx->launches += 1;
  CK(cudaGetLastError());
  return DDEL_OK;
}

int ddel_back_substitute(ddel_ctx* ctx, const double* f, const double* uG, double* u) {
  if (!ctx || !f || !uG || !u) return DDEL_EINVAL;
  if (!ctx->factored[ctx->active_prec]) return fail(ctx, DDEL_ESTATE, "factor first");
  back_substitute(ctx, ctx->active_prec, f, uG, u);
  CK(cudaGetLastError());
  return DDEL_OK;
}

int ddel_pcg(ddel_ctx* ctx, const double* g, double* x, double tol_abs, ddel_stats* stats) {
  if (!ctx || !g || !x) return DDEL_EINVAL;
  const int prec = ctx->active_prec;
  if (!ctx->factored[prec]) return fail(ctx, DDEL_ESTATE, "factor first");
  if (ctx->ck_in > 0 && ctx->coarse_prec != prec * 2) {
    int rc = coarse_build(ctx, prec, false);
    if (rc) return rc;
  }
  set_tol_abs_kernel<<<1, 1, 0, ctx->stream>>>(ctx->st, tol_abs, ctx->opt.max_it);
  ctx->launches += 1;
  int it = 0, pst = 0;
  int rc = pcg_run(ctx, prec, g, &it, &pst);
  if (rc) return rc;
  CK(cudaMemcpyAsync(x, ctx->x, ctx->T.n_gamma * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->iters = it;
    stats->status = pst;
    stats->pcg_relres = std::sqrt(ctx->h_st->rr);
    stats->cycles = 1;
    stats->bad_subdomain = -1;
  }
  return pst;
}

int ddel_residual_norm(ddel_ctx* ctx, const double* f, const double* u, double* r_norm,
                       double* f_norm) {
  if (!ctx || !f || !u) return DDEL_EINVAL;
  if (!ctx->assembled) return fail(ctx, DDEL_ESTATE, "assemble first");
  launch_apply_K(ctx->T, ctx->F, u, f, ctx->d_r, 1, ctx->partials, ctx->ticketK, ctx->nrm,
                 ctx->stream, ctx->nblk);
  ctx->launches += 1;
  CK(cudaMemcpyAsync(ctx->h_nrm, ctx->nrm, 16, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (r_norm) *r_norm = ctx->h_nrm[0];
  if (f_norm) *f_norm = ctx->h_nrm[1];
  return DDEL_OK;
}

int ddel_gamma_dofs(const ddel_ctx* ctx, int64_t* out) {
  if (!ctx || !out) return DDEL_EINVAL;
  std::memcpy(out, ctx->S.gamma_dof.data(), ctx->S.gamma_dof.size() * sizeof(int64_t));
  return DDEL_OK;
}

int ddel_load_vector(const ddel_ctx* ctx, double* out) {
  if (!ctx || !out) return DDEL_EINVAL;
  std::memcpy(out, ctx->S.f.data(), ctx->S.f.size() * sizeof(double));
  return DDEL_OK;
}

int ddel_fixed_mask(const ddel_ctx* ctx, uint8_t* out) {
  if (!ctx || !out) return DDEL_EINVAL;
  std::memcpy(out, ctx->S.fixed.data(), ctx->S.fixed.size());
  return DDEL_OK;
}

int ddel_kernel_info(const ddel_ctx* ctx, ddel_kernel_info_t* out) {
  if (!ctx || !out) return DDEL_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->launches_total = ctx->launches;
  out->launches_since_assemble = ctx->launches - ctx->launches_at_assemble;
  const int prec = ctx->active_prec;
  const int64_t tb = prec ? 4 : 8;
  out->precision = prec;
  out->schur_form = ctx->explicit_ok[prec] ? 1 : 0;
  out->double_float = (prec == 0 && ctx->df_ok) ? 1 : 0;
  int64_t mat = 0, ring = 0;
  for (const SubInfo& si : ctx->S.subs) {
    ring += si.n_ring;
    if (ctx->explicit_ok[prec]) {
      mat += (int64_t)si.n_ring * si.n_ring;
    } else {
      // the D_k triangles and the nonzeros of the C_k: C_k(i, m) = 0 below the
      // lowest column row i couples to in the plane before
      const int64_t b = si.bsz;
      int64_t cnz = 0;
      for (int64_t i = 0; i < b; ++i) {
        const int64_t lo = ctx->S.dim == 3 ? 3 * (i / 3) - 3 * si.icnt[2] - 3 : 2 * (i / 2) - 2;
        cnz += b - std::max<int64_t>(0, lo);
      }
      mat += 2 * (si.nb * b * (b + 1) / 2 + (si.nb > 0 ? si.nb - 1 : 0) * cnz);
    }
  }
  // matrix entries read once, plus the ring gather (z and p, FP64) and the ring output
  out->schur_apply_bytes = mat * tb + ring * (16 + tb);
  out->schur_apply_flops = 2 * mat;
  return DDEL_OK;
}

struct ddel_plan {
  Setup S;
};

int ddel_plan_create(const ddel_mesh* mesh, const ddel_material* mat, const ddel_bc* bc,
                     double theta, ddel_plan** out) {
  if (!mesh || !mat || !bc || !out) return DDEL_EINVAL;
  *out = nullptr;
  ddel_plan* p = new (std::nothrow) ddel_plan();
  if (!p) return DDEL_ENOMEM;
  const int ne[3] = {mesh->nx, mesh->ny, mesh->nz};
  std::string msg = build_setup(mesh->dim, ne, mesh->sub, mat->E, mat->nu, mat->plane_stress,
                                bc->clamp_faces, bc->fixed_dof, bc->n_point, bc->point_node,
                                bc->point_force, bc->traction_face, bc->traction, bc->body_force, theta, &p->S);
  if (!msg.empty()) {
    delete p;
    return DDEL_EINVAL;
  }
  *out = p;
  return DDEL_OK;
}

void ddel_plan_destroy(ddel_plan* plan) { delete plan; }

int ddel_plan_info(const ddel_plan* plan, ddel_info_t* info) {
  if (!plan || !info) return DDEL_EINVAL;
  const Setup& S = plan->S;
  info->dim = S.dim;
  info->n_sub = S.n_sub;
  info->n_elem = (int)S.n_elem;
  info->max_block = S.BP;
  info->max_blocks_per_sub = S.nb_max;
  info->n_nodes = S.n_nodes;
  info->n_dof = S.n_dof;
  info->n_gamma = (int64_t)S.gamma_dof.size();
  int64_t nf = 0;
  for (auto v : S.fixed) nf += v;
  info->n_fixed = nf;
  info->factor_bytes = S.factor_elems * 8;
  info->n_face_blocks = (int)S.blk_off.size();
  info->n_cross = (int)(S.gamma_dof.size() - S.n_face_dofs);
  return DDEL_OK;
}

int ddel_plan_gamma_dofs(const ddel_plan* plan, int64_t* out) {
  if (!plan || !out) return DDEL_EINVAL;
  std::memcpy(out, plan->S.gamma_dof.data(), plan->S.gamma_dof.size() * sizeof(int64_t));
  return DDEL_OK;
}

int ddel_plan_face_block(const ddel_plan* plan, int b, int32_t* off, int32_t* n, double* P,
                         double* hmean) {
  if (!plan || b < 0 || b >= (int)plan->S.blk_off.size()) return DDEL_EINVAL;
  const Setup& S = plan->S;
  const int nb = S.blk_n[b];
  if (off) *off = S.blk_off[b];
  if (n) *n = nb;
  if (hmean) *hmean = S.blk_hmean[b];
  if (P) std::memcpy(P, S.ptab.data() + S.blk_poff[b], (size_t)nb * nb * sizeof(double));
  return DDEL_OK;
}

int ddel_plan_element_matrix(const ddel_plan* plan, double* Ke) {
  if (!plan || !Ke) return DDEL_EINVAL;
  std::memcpy(Ke, plan->S.Ke.data(), plan->S.Ke.size() * sizeof(double));
  return DDEL_OK;
}

int ddel_plan_interface_operator(const ddel_plan* plan, int comp, int32_t* n, int64_t* nnz, int32_t* pos,
                                 int64_t* rowptr, int32_t* col, double* M, double* L) {
  if (!plan || !n || !nnz || comp < 0 || comp >= plan->S.dim) return DDEL_EINVAL;
  std::vector<int32_t> p, c;
  std::vector<int64_t> rp;
  std::vector<double> m, l;
  interface_operator(plan->S, comp, &p, &rp, &c, &m, &l);
  *n = (int32_t)p.size();
  *nnz = (int64_t)c.size();
  if (!pos) return DDEL_OK;
  if (!rowptr || !col || !M || !L) return DDEL_EINVAL;
  std::memcpy(pos, p.data(), p.size() * sizeof(int32_t));
  std::memcpy(rowptr, rp.data(), rp.size() * sizeof(int64_t));
  std::memcpy(col, c.data(), c.size() * sizeof(int32_t));
  std::memcpy(M, m.data(), m.size() * sizeof(double));
  std::memcpy(L, l.data(), l.size() * sizeof(double));
  return DDEL_OK;
}

int ddel_plan_subdomain(const ddel_plan* plan, int i, int32_t* ilo, int32_t* icnt) {
  if (!plan || i < 0 || i >= plan->S.n_sub || !ilo || !icnt) return DDEL_EINVAL;
  for (int a = 0; a < 3; ++a) {
    ilo[a] = plan->S.subs[i].ilo[a];
    icnt[a] = plan->S.subs[i].icnt[a];
  }
  return DDEL_OK;
}

}  // extern "C"
