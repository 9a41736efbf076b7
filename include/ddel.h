/*
 * ddel.h -- C ABI of libddel: GB300-native non-overlapping domain-decomposition
 * solve of discretised linear elasticity, inside the Picard loop of topology
 * optimisation (Turner, Kocvara, Loghin, arXiv:1501.06211).
 *
 * Conventions (apply to every call):
 *  - Every function returns a ddel_status (0 = success, < 0 = error).  No call
 *    aborts the process and no C++ exception crosses this boundary.
 *    ddel_strerror() gives a message; ddel_last_error() the context's last one.
 *    Besides the errors a call lists: DDEL_EINVAL for a null context or a null
 *    required pointer, DDEL_ESTATE for a call before its prerequisite (see the
 *    step-level section), DDEL_ECUDA when a CUDA runtime call fails.
 *  - Plain pointers and sizes only.  "device" pointers are CUDA device memory
 *    of the current device (e.g. from torch); "host" pointers are ordinary (or
 *    pinned) host memory.  Every pointer argument says which it is.
 *  - Inputs are read, never retained: the context copies what it needs.
 *    Outputs go to caller-allocated buffers; the caller keeps ownership.
 *  - Global vectors have n_dof = dim * n_nodes entries in node-interleaved order:
 *    2D node (i, j) has index n = i*(ny+1) + j, 3D node (i, j, k) has
 *    n = (i*(ny+1) + j)*(nz+1) + k, and DOF d*n + c holds component c.
 *    Element (ex, ey[, ez]) has index ex*ny + ey (2D), (ex*ny + ey)*nz + ez (3D).
 *    Dirichlet (clamped) DOFs are eliminated (Sec. 1, Sec. 2): outputs hold 0.
 *  - Interface ("Gamma") vectors have n_gamma entries in the library's own order
 *    (face blocks first, then cross-point DOFs); ddel_gamma_dofs() maps them to
 *    global DOFs.
 *  - Calls are asynchronous on the context's stream except those that return
 *    statistics or status read from the device (ddel_solve, ddel_pcg,
 *    ddel_residual_norm, ddel_topopt_step), which synchronise that stream.
 *  - A context is not thread-safe; use one context per host thread.
 *  - Memory: the context allocates all its device workspace in ddel_create /
 *    ddel_factor and frees it in ddel_destroy.
 */
#ifndef DDEL_H
#define DDEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DDEL_OK = 0,
  DDEL_EINVAL = -1,      /* bad argument (sizes, material range, null pointer) */
  DDEL_ENOMEM = -2,      /* device or host allocation failed */
  DDEL_ECUDA = -3,       /* a CUDA runtime call failed */
  DDEL_ENOTSPD = -4,     /* a subdomain pivot was <= 0 or not finite; stats.bad_subdomain */
  DDEL_ENOCONV = -5,     /* max_it / max_cycles reached before the tolerance */
  DDEL_EBREAKDOWN = -6,  /* Krylov breakdown (p^T S p <= 0 or not finite) */
  DDEL_ESTATE = -7,      /* call order violated (e.g. solve before factor) */
  DDEL_ETIMEOUT = -8     /* a bounded device wait ran out; the kernel returned */
} ddel_status;

/* FP64: factors and local Schur complements formed in FP64.  How S_i is
 *       applied inside PCG depends on schur_mode: EXPLICIT and IMPLICIT apply
 *       it in native FP64 arithmetic (the plain FP64 method); AUTO (the
 *       default) forms S_i in double-float arithmetic and applies it as FP32
 *       (hi, lo) pairs, about 48 significant bits -- a reduced-precision
 *       operator inside an FP64 Krylov iteration, FP64 residual and FP64
 *       refinement (ddel_kernel_info_t.double_float reports it).
 * FP32: factors and applications in FP32 (FP64 Krylov vectors and dot
 *       products, FP64 residual and refinement).
 * MIXED: FP64 factors and local Schur complements, which are stored and
 *       applied in FP32 inside PCG (FP64 vectors and dot products); condensation,
 *       back-substitution and the refinement residual stay FP64.  Where the
 *       explicit form is unavailable it behaves as FP64.  With
 *       ddel_options.relax_switch > 0 the FP32 copies enter only the late
 *       iterations of one PCG that stops on an FP64 residual (relaxed form). */
typedef enum { DDEL_FP64 = 0, DDEL_FP32 = 1, DDEL_MIXED = 2 } ddel_precision;
typedef enum { DDEL_SCHUR_IMPLICIT = 0, DDEL_SCHUR_EXPLICIT = 1, DDEL_SCHUR_AUTO = 2 } ddel_schur_mode;
/* Initial iterate of ddel_solve: ZERO (u = 0), WARM (the previous converged
 * solution of this context, e.g. of the last Picard step; 0 before the first). */
typedef enum { DDEL_X0_ZERO = 0, DDEL_X0_WARM = 1 } ddel_x0_mode;
/* Coarse-space use (ddel_set_coarse).  Not in the paper, whose preconditioner
 * is face-local only. */
typedef enum { DDEL_COARSE_X0 = 1, DDEL_COARSE_CORRECT = 2, DDEL_COARSE_DEFLATE = 4 } ddel_coarse_flags;
#define DDEL_MAX_COARSE 8

/* Structured grid of unit elements, split into sub^dim-element subdomains
 * (Sec. 1: N non-overlapping subdomains).  dim = 2 (Q1 bilinear, 2 DOF/node)
 * or 3 (H8 trilinear, 3 DOF/node).  sub must divide nx, ny (, nz). */
typedef struct {
  int dim;
  int nx, ny, nz; /* elements per axis; nz ignored in 2D */
  int sub;        /* subdomain edge in elements */
} ddel_mesh;

/* Isotropic material of Sec. 1: Young's modulus E > 0 and Poisson ratio
 * -1 < nu < 1/2 give the Lame constants mu, lambda.  2D uses plane stress when
 * plane_stress != 0 (lambda* = 2 mu lambda / (lambda + 2 mu)), else plane strain.
 * Element stiffness is E_e = E * rho_e^simp_p times the unit-E element matrix
 * (eq. NumberTen with exponent p; p = 1 is the paper's variable-thickness sheet). */
typedef struct {
  double E, nu;
  int plane_stress;
  double simp_p;
  double rho_min; /* lower density bound used by topology optimisation */
} ddel_material;

/* Boundary conditions of Sec. 1: clamped (u = 0) parts and loads.
 * clamp_faces: bit (2*axis + side) fixes every DOF on grid face axis = 0
 * (side 0) or axis = n_axis (side 1).  fixed_dof: optional host array of
 * n_dof bytes, nonzero = DOF fixed (OR'ed with clamp_faces).  Point loads:
 * n_point nodes (host int64 node indices) with dim force components each (host
 * doubles).  traction_face = 2*axis + side applies the uniform surface
 * traction `traction` (force per unit area) on that face as consistent nodal
 * loads, or -1 for none.  body_force: uniform force per unit volume (the f of
 * the mixed problem of Sec. 1) as consistent nodal loads, each unit element
 * giving 1/2^dim of its force to each of its nodes (zeros for none). */
typedef struct {
  uint32_t clamp_faces;
  const uint8_t* fixed_dof;
  int n_point;
  const int64_t* point_node;
  const double* point_force;
  int traction_face;
  double traction[3];
  double body_force[3];
} ddel_bc;

/* Solver options.  ddel_default_options() fills documented defaults. */
typedef struct {
  int precision;       /* ddel_precision of the subdomain factors and Schur applies (FP64) */
  double theta;        /* fractional index theta of eq. NumberEight (0.5) */
  int face_scaling;    /* face block S~_f = W H_f W (reading of Sec. 3 for heterogeneous
                          material): 0 W = I; 1 W = sqrt(mean diag K_GG / mean diag H_f) I;
                          2 W_ii = sqrt(diag(K_GG)_ii / diag(H_f)_ii)  (2) */
  int crosspoint_mode; /* 0: z = r / diag(K_GG) at cross points; 1: identity (0) */
  double tol;          /* target ||f - K u||_2 / ||f||_2 (1e-8) */
  int max_it;          /* PCG iteration cap per cycle (5000) */
  int max_cycles;      /* refinement cycles cap (10) */
  double inner_tol;    /* per-cycle PCG reduction in FP32 mode (1e-6) */
  int x0_mode;         /* ddel_x0_mode of ddel_solve (ZERO) */
  int schur_mode;      /* ddel_schur_mode (AUTO): EXPLICIT/AUTO form each local Schur
                          complement S_i after the factorisation where the ring fits
                          (2D, sub <= 32) and apply it as one dense product per PCG
                          iteration; IMPLICIT applies it by block substitution */
  int use_graph;       /* capture PCG iterations in a CUDA graph (1) */
  int check_every;     /* PCG iterations between host convergence checks (16) */
  int tensor_form;     /* 1: form the FP64 local Schur complements with W^T W on the
                          tensor cores at FP64 accuracy (Ozaki splitting into BF16 slices,
                          FP32 accumulation): rings of 128 and 256 in the EXPLICIT form,
                          rings of 256 in the AUTO form (whose rings of 128 keep the
                          faster double-float formation); FP32 contexts form theirs on
                          the FP32 pipes; 2: as 1, and also FP32 contexts on the tensor
                          cores (W from the FP32 factors, S_i rounded once to FP32) and
                          the C_k C_k^T of each plane of the FP64 3D factorisation (FP64
                          accuracy; slower than the FP64 pipe at these sizes);
                          0: every formation on the FP64 / FP32 pipes (1) */
  int schur_split;     /* CTAs per subdomain of the explicit apply (native FP64 and
                          double-float): 1, 2 or 4 (rows per CTA = ring / split, at least
                          32); 0: by ring size, one for rings of 64, two for 128 and 256
                          (0); the persistent batch runs the default shape only */
  double relax_switch; /* MIXED precision, explicit 2D form, no coarse space: > 0 runs
                          one relaxed PCG instead of refinement cycles -- the FP64 Schur
                          complements until the recursive residual is below
                          relax_switch * ||f||, then their FP32 copies, with reliable
                          updates (r = g - S x with the FP64 operator) whenever the
                          residual has fallen by relax_delta since the last one and when
                          it converges; it stops only on such a true residual, and goes
                          back to the FP64 operator if three updates in a row bring no
                          new low.  0: refinement cycles as described under MIXED (0) */
  double relax_delta;  /* residual reduction between reliable updates (0.1) */
} ddel_options;

typedef struct {
  int status;          /* ddel_status of the solve */
  int iters;           /* total PCG iterations (all cycles) */
  int cycles;          /* refinement cycles (1 for a converged FP64 solve) */
  double relres;       /* final ||f - K u||_2 / ||f||_2 computed in FP64 */
  double pcg_relres;   /* last interface residual ||r_G|| / ||f|| of the recurrence */
  int bad_subdomain;   /* first subdomain with a failed pivot, or -1 */
  int fallback;        /* bit 0: an FP32 solve switched to the FP64 factors; bit 1: the
                          coarse space was dropped after a Krylov breakdown */
  double t_factor_ms;  /* device time of the context's last ddel_factor (with S_i formation) */
  double t_condense_ms, t_pcg_ms, t_backsub_ms, t_verify_ms, t_total_ms;
  int coarse_k;        /* coarse dimension used by the interface PCG (0: none) */
  int x0_used;         /* cycles whose PCG started from the Galerkin guess */
  int low_iters;       /* relaxed PCG: iterations with the FP32 Schur complements */
  int replacements;    /* relaxed PCG: reliable updates (FP64 residual replacements) */
} ddel_stats;

typedef struct {
  int dim, n_sub, n_elem, max_block, max_blocks_per_sub;
  int64_t n_nodes, n_dof, n_gamma, n_fixed, factor_bytes;
  int n_face_blocks, n_cross;
} ddel_info_t;

typedef struct ddel_ctx ddel_ctx;

void ddel_default_options(ddel_options* opt);
const char* ddel_strerror(int status);
/* Message of the context's last error; with ctx == NULL, of the last failed ddel_create. */
const char* ddel_last_error(const ddel_ctx* ctx);

/* Set up mesh, DOF classification (Gamma = nodes in two or more subdomain
 * closures; interior = the rest, per subdomain; Sec. 1 and eq. NumberFive),
 * the face-local interface preconditioner (Sec. 3-4) and device workspace.
 * cuda_stream: a cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream) or
 * NULL for a stream owned by the context.  Errors: EINVAL (sizes, nu outside
 * (-1, 1/2), E <= 0, sub not dividing the grid), ENOMEM, ECUDA. */
int ddel_create(const ddel_mesh* mesh, const ddel_material* mat, const ddel_bc* bc,
                const ddel_options* opt, void* cuda_stream, ddel_ctx** out);
void ddel_destroy(ddel_ctx* ctx);
int ddel_get_info(const ddel_ctx* ctx, ddel_info_t* info);
/* Changing precision or schur_mode requires a new ddel_factor (ESTATE until then);
 * theta is fixed at creation (EINVAL). */
int ddel_set_options(ddel_ctx* ctx, const ddel_options* opt);

/* Element densities rho (n_elem doubles; host when on_device == 0, else device):
 * element stiffness factors E * rho_e^p (eq. NumberTen), the diagonal of K_GG
 * and the face scales.  Values must be > 0 and finite (EINVAL otherwise,
 * detected on the host for host input, on the device for device input). */
int ddel_assemble(ddel_ctx* ctx, const double* rho, int on_device);

/* Batched factorisation of every K_{I_i I_i} (eq. NumberFive) in the context's
 * precision: interior DOFs ordered by grid plane give a block-tridiagonal
 * matrix; each block step is SYRK update, dense Cholesky, explicit inverse of
 * the diagonal factor, and the off-diagonal factor (the banded O(k^2 n) solve
 * of Sec. 4).  ENOTSPD when a pivot fails (stats via ddel_solve). */
int ddel_factor(ddel_ctx* ctx);

/* Whole solve of K u = f by the three steps of eq. 3MatSplit2 with interface
 * PCG (reading of Sec. 3: S~ SPD, applied exactly), repeated as FP64 iterative
 * refinement until ||f - K u|| <= tol ||f||.  f: n_dof doubles or NULL for the
 * loads of ddel_bc; u: n_dof doubles (output).  Both host when on_device == 0,
 * else device.  st may be NULL.  Synchronises the stream. */
int ddel_solve(ddel_ctx* ctx, const double* f, double* u, int on_device, ddel_stats* st);

/* Coarse space for the interface PCG (an addition to the paper's face-local
 * preconditioner of Sec. 3-4).  Z: k vectors over the Gamma DOFs (column-major,
 * k x n_gamma doubles in ddel_gamma_dofs order; host when on_device == 0, else
 * device), 0 <= k <= DDEL_MAX_COARSE; k == 0 removes the coarse space.  The
 * library orthonormalises Z (Cholesky QR, twice; numerically dependent columns
 * are dropped), forms E = Q^T S Q with the context's Schur apply after each
 * factorisation (lazily, at the next solve) and, with flags:
 *   DDEL_COARSE_X0:      each PCG starts from the Galerkin guess
 *                        x0 = Q E^-1 Q^T g (kept only if ||g - S x0|| <= ||g||);
 *   DDEL_COARSE_CORRECT: preconditioner S~^-1 r + Q E^-1 Q^T r (additive, SPD);
 *   DDEL_COARSE_DEFLATE: instead, Q E^-1 Q^T r + (I - Q E^-1 Q^T S) S~^-1 r
 *                        (deflation in the "A-DEF2" form of Tang, Nabben, Vuik
 *                        and Erlangga 2009; eigenvalue 1 on span(Q)).
 * If E is not SPD the solve runs plain PCG (stats.coarse_k = 0).  Z is copied;
 * the caller keeps ownership.  Errors: EINVAL (k or flags out of range, or
 * CORRECT together with DEFLATE). */
int ddel_set_coarse(ddel_ctx* ctx, const double* Z, int k, int flags, int on_device);

/* --- Topology optimisation (Sec. 5) ------------------------------------------
 * One Picard step of the variable-thickness-sheet / SIMP problem of
 * eq. NumberTen: density filter rho~ = Hbar rho (hat weights
 * max(0, r_min - distance), rows normalised), finite-element analysis with
 * element factors E rho~^p (assemble + factor + solve of this library),
 * compliance c = f^T u, adjoint sensitivities dc/drho~_e = -p E rho~_e^(p-1)
 * u_e^T K_e u_e, filter chain rule, and the optimality-criteria update
 * rho_new = clamp(rho (-dc / (lambda dV))^(1/2), max(rho_min, rho - move),
 * min(1, rho + move)) with lambda found by 64 bisection steps on [0, 1e9] so
 * that sum(rho~_new) = volfrac * n_elem.  The paper names OC without formulas
 * (Sec. 5); these are the standard optimality conditions of the Lagrangian. */
typedef struct {
  double* rho;        /* device, n_elem: design densities, updated in place */
  double volfrac;     /* target volume fraction of the filtered densities */
  double r_min;       /* filter radius in elements (e.g. 1.5) */
  double move;        /* OC move limit (e.g. 0.2) */
  int iteration;      /* incremented by every step */
  double compliance;  /* out: f^T u of this step's analysis */
  double volume;      /* out: sum of the filtered new densities / n_elem */
  double change;      /* out: max |rho_new - rho| */
  double lambda;      /* out: OC volume multiplier */
  double* u;          /* device, n_dof, or NULL: displacement of this step */
  double* rho_phys;   /* device, n_elem, or NULL: filtered densities of this step */
  void* learner;      /* a ddel_learner of this context (ddel_learn.h) or NULL: coarse
                         space predicted before the solve, observation after it */
  /* Adaptive tolerance of the analysis (Sec. 5, Table 3: "based on successive
   * compliance values"; the formula is this library's reading): with
   * tol_eta > 0 a step solves to tol = clamp(tol_eta |c_k - c_(k-1)| / |c_k|,
   * ctx tol, tol_max) where c_k = compliance, c_(k-1) = compliance_prev (the
   * last two steps' compliances), and to tol_max in the first two steps;
   * tol_eta = 0: the context's tol. */
  double tol_eta;         /* e.g. 0.1; 0 = off */
  double tol_max;         /* cap of the adaptive tolerance (0: 1e-3) */
  double tol_used;        /* out: the tolerance of this step's solve */
  double compliance_prev; /* kept by ddel_topopt_step: the compliance of the step before */
} ddel_topopt_state;
/* Densities must lie in [rho_min, 1]; the loads are those of ddel_bc.
 * Synchronises the stream.  st (may be NULL) receives the solve statistics. */
int ddel_topopt_step(ddel_ctx* ctx, ddel_topopt_state* state, ddel_stats* st);

/* Checkpoint / resume of a topology-optimisation run (the paper has no
 * counterpart).  save writes the design densities (state->rho, device), the
 * state scalars (volfrac, r_min, move, iteration, compliance, volume, change,
 * lambda, tol_eta, tol_max, compliance_prev; files of version 1 hold the first
 * eight and load as compliance_prev = compliance) and the identity of the
 * problem (mesh and material) to `path`,
 * through a temporary file renamed into place, with a 64-bit FNV-1a checksum.
 * load checks magic, version, problem identity and checksum, then copies the
 * densities into state->rho (device, n_elem doubles, caller-owned) and sets the
 * scalars; it leaves u, rho_phys and learner untouched.  A resumed run repeats
 * the original bitwise (every reduction has a fixed order), except that a
 * WARM or coarse-space initial guess restarts from nothing.
 * Errors: EINVAL (bad arguments, unreadable or foreign file, checksum or
 * identity mismatch), ECUDA.  Both synchronise the stream. */
int ddel_checkpoint_save(const ddel_ctx* ctx, const ddel_topopt_state* state, const char* path);
int ddel_checkpoint_load(ddel_ctx* ctx, ddel_topopt_state* state, const char* path);

/* --- Batched independent problems ---------------------------------------------
 * Solves n independent, assembled problems (each its own context: any grid,
 * subdomain size, material) for their ddel_bc loads, concurrently: all
 * factorisations are launched before any is checked, and the PCG iterations of
 * every context are issued in batches of check_every as soon as that
 * context's previous batch has reported, so kernels of different problems run
 * side by side (contexts need distinct streams: create them with
 * cuda_stream = NULL).  u: array of n device pointers (n_dof of each problem)
 * or NULL entries; stats: n entries or NULL.  A problem that misses its
 * tolerance after one cycle is finished by the refinement loop of
 * ddel_solve.  The result of every problem is bitwise the one of ddel_solve
 * in FP64 (same kernels, same order).  Synchronises all streams. */
int ddel_batch_solve(ddel_ctx* const* ctxs, int n, double* const* u, ddel_stats* stats);

/* The same batch in one persistent launch per check_every iterations: a
 * device work queue hands out, in order, for every PCG iteration the Schur
 * blocks of every problem and then their update blocks (per-problem PCG
 * scalars stay in each context's device state); a block that depends on
 * another problem phase waits for it, bounded (a lost arrival returns
 * DDEL_ETIMEOUT instead of hanging); the blocks compute exactly what the
 * kernels of ddel_solve compute, so every problem's result is bitwise that of
 * ddel_solve.  For the default FP64 double-float explicit form in 2D without
 * a coarse space; other configurations take ddel_batch_solve's path.  The
 * factorisations, condensation and back-substitution run on each context's
 * stream as in ddel_batch_solve; the persistent launches use the first
 * context's stream.  Synchronises all streams. */
int ddel_batch_solve_persistent(ddel_ctx* const* ctxs, int n, double* const* u, ddel_stats* stats);

/* --- Autotuner ------------------------------------------------------------------
 * Chooses the Schur form (IMPLICIT block substitution, EXPLICIT FP64, or AUTO =
 * explicit applied in double-float arithmetic), the formation of S_i (tensor
 * cores or FP64 pipe, ddel_options.tensor_form, where both exist), the tile
 * shape of the native FP64 explicit apply (ddel_options.schur_split: 1, 2 or 4
 * CTAs per subdomain) and the PCG graph batch size (check_every in
 * {8, 16, 32}) for an assembled context by timing them on this
 * GPU: one solve gives the iteration count N, then each candidate is
 * factorised and runs 48 PCG iterations; the predicted solve time is
 * factor (+ formation) time + N x time per iteration.  The winner is applied
 * to the context (ddel_set_options semantics: refactor before solving) and,
 * with cache_path != NULL, appended to that text file under the key
 * "dim sub BP n_sub precision" (fields: mode, check_every, tensor_form,
 * schur_split; lines without the last fields keep the context's settings); a
 * later call with the same key reads the file
 * and applies the cached choice without timing (*from_cache = 1).
 * chosen_mode / chosen_check: outputs (may be NULL).  Synchronises. */
int ddel_autotune(ddel_ctx* ctx, const char* cache_path, int* chosen_mode, int* chosen_check,
                  int* from_cache);

/* --- Full-system flexible GMRES with the block-triangular preconditioner -------
 * The Krylov method of the paper's Table 1 (Sec. 3-4): GMRES on the whole
 * system K u = f (interior and interface DOFs), right-preconditioned by
 * P~ = [[K_II, K_IG], [0, S~]], whose inverse is applied as
 * P~^-1 v = (K_II^-1 (v_I - K_IG S~^-1 v_G), S~^-1 v_G) with the context's
 * subdomain factors (eq. 3MatSplit2).  Flexible (Saad's FGMRES: the
 * preconditioned directions are stored) because the inverse-Lanczos S~^-1 is
 * not a fixed linear map.  The interface preconditioner S~ is one of
 *   DDEL_PREC_IDENTITY  S~ = I (Table 1's first columns);
 *   DDEL_PREC_FACE      the face-local H~_theta of ddel_precond_apply (the
 *                       preconditioner of the interface PCG);
 *   DDEL_PREC_GLOBAL    H~_theta = M (M^-1 L)^(1 - theta) of eq. NumberEight
 *                       and NumberNine on the whole interface, per displacement
 *                       component, applied by inverse Lanczos (Sec. 3): k steps
 *                       of Lanczos for L^-1 M in the M inner product from
 *                       b = M^-1 r give S~^-1 r ~ ||b||_M Q_k T_k^(1-theta) e_1;
 *                       each step solves with L by the inner PCG of Sec. 4
 *                       (relative tolerance inner_tol, preconditioned by L on
 *                       each face with the cross points removed, diagonal at
 *                       cross points); b = M^-1 r by Jacobi-preconditioned CG
 *                       to mass_tol.  Needs a nonsingular interface Laplacian
 *                       per component (every connected part of the interface
 *                       meets a clamped node; EINVAL otherwise).
 * theta is the context's (ddel_options.theta at creation): the H_OPT columns of
 * Table 1 use one context per theta.  Iterations are capped at max_it (no
 * restart); the stopping test is the GMRES residual estimate
 * ||f - K u|| <= tol ||f||; stats.relres is then recomputed in FP64. */
typedef enum { DDEL_PREC_IDENTITY = 0, DDEL_PREC_FACE = 1, DDEL_PREC_GLOBAL = 2 } ddel_interface_prec;
#define DDEL_MAX_LANCZOS 32
typedef struct {
  int precond;          /* ddel_interface_prec (DDEL_PREC_GLOBAL) */
  int lanczos_steps;    /* GLOBAL: inverse Lanczos steps k, 1..DDEL_MAX_LANCZOS (8) */
  double inner_tol;     /* GLOBAL: relative residual of the inner PCG on L (1e-3) */
  double mass_tol;      /* GLOBAL: relative residual of the CG solve with M (1e-13) */
  int global_scaling;   /* GLOBAL: 0 none (paper-literal, homogeneous material);
                           1 W_ii = (diag(K_GG)_ii / (M_ii^theta L_ii^(1-theta)))^(1/2),
                           S~ = W H~ W (this library's reading for heterogeneous
                           material) (1) */
  double tol;           /* relative residual target (1e-6, Table 1's) */
  int max_it;           /* iteration cap, 1..2000 (300) */
} ddel_gmres_options;
typedef struct {
  int status;           /* DDEL_OK, or DDEL_ENOCONV at max_it */
  int iters;            /* FGMRES iterations (preconditioner applications) */
  double est_relres;    /* GMRES residual estimate at exit */
  double relres;        /* ||f - K u|| / ||f|| recomputed in FP64 */
  int inner_min, inner_max;  /* GLOBAL: inner PCG iterations per solve with L */
  double inner_mean;
  int lanczos_m;        /* GLOBAL: Lanczos steps of the last application (< k on breakdown) */
  double t_ms;          /* device time of the solve */
} ddel_gmres_stats;
void ddel_default_gmres_options(ddel_gmres_options* opt);
/* f: n_dof doubles or NULL for the loads of ddel_bc; u: n_dof doubles (output);
 * host when on_device == 0, else device.  Needs ddel_factor (ESTATE).
 * Allocates its Krylov basis (2 max_it + 1 vectors of n_dof doubles) on first
 * use.  Synchronises the stream (one small read-back per iteration). */
int ddel_gmres_solve(ddel_ctx* ctx, const ddel_gmres_options* opt, const double* f, double* u,
                     int on_device, ddel_gmres_stats* st);
/* Step level: z = S~^-1 r with the global interface preconditioner above
 * (device n_gamma vectors, ddel_gamma_dofs order).  lanczos_out (host, may be
 * NULL): per component c < dim, 2 + 3 DDEL_MAX_LANCZOS doubles at
 * c (2 + 3 DDEL_MAX_LANCZOS): [m, mass-CG iterations, alpha_0..alpha_{m-1} at
 * 2.., beta_0..beta_{m-2} at 2 + DDEL_MAX_LANCZOS.., inner PCG iterations of
 * step j at 2 + 2 DDEL_MAX_LANCZOS + j] (the tridiagonal T_m of the last
 * application and its iteration counts).  Synchronises when lanczos_out is
 * given.  Errors: EINVAL (steps or tolerances out of range, a singular
 * interface Laplacian), ESTATE before ddel_assemble. */
int ddel_global_precond_apply(ddel_ctx* ctx, const ddel_gmres_options* opt, const double* r, double* z,
                              double* lanczos_out);

/* --- Step-level entry points (device pointers; asynchronous) ---------------
 * Prerequisites (DDEL_ESTATE otherwise): ddel_assemble for apply_K,
 * precond_apply and residual_norm; ddel_factor for condense, schur_apply,
 * schur_apply_ring, back_substitute and pcg. */
/* y = K(rho) x over all free DOFs (fixed rows 0), element by element, FP64. */
int ddel_apply_K(ddel_ctx* ctx, const double* x, double* y);
/* g = f_G - sum_i K_{G I_i} K_{I_i I_i}^-1 f_{I_i} (eq. 3MatSplit2, second line). */
int ddel_condense(ddel_ctx* ctx, const double* f, double* g);
/* y = S x = sum_i (K_GG^(i) x_i - K_{G I_i} K_{I_i I_i}^-1 K_{I_i G} x_i) without forming S
 * (Sec. 3: "avoid the direct construction"); x, y: n_gamma. */
int ddel_schur_apply(ddel_ctx* ctx, const double* x, double* y);
/* The per-subdomain half of ddel_schur_apply alone: y_i = S_i x_i for every
 * subdomain into the context's ring buffer, no sum over the subdomains (the
 * PCG update kernel forms that sum itself).  For timing the Schur kernel as the
 * PCG runs it; x: n_gamma (device).  ESTATE before ddel_factor. */
int ddel_schur_apply_ring(ddel_ctx* ctx, const double* x);
/* z = S~^-1 r: face-local H~_theta^-1 per component (eq. NumberEight/NumberNine,
 * cross points removed as in Sec. 4) and a diagonal at cross points. */
int ddel_precond_apply(ddel_ctx* ctx, const double* r, double* z);
/* u_I = K_II^-1 (f_I - K_IG u_G), u_G = uG, u = 0 on fixed DOFs (eq. 3MatSplit2). */
int ddel_back_substitute(ddel_ctx* ctx, const double* f, const double* uG, double* u);
/* Interface PCG on S x = g from x = 0 (from the Galerkin guess, and with the
 * coarse correction, when ddel_set_coarse gave a coarse space); stops at
 * ||r|| <= tol_abs.  g, x: device n_gamma.  Synchronises. */
int ddel_pcg(ddel_ctx* ctx, const double* g, double* x, double tol_abs, ddel_stats* st);
/* ||f - K u||_2 and ||f||_2 over free DOFs in FP64 (device f, u; host outputs). */
int ddel_residual_norm(ddel_ctx* ctx, const double* f, const double* u, double* r_norm,
                       double* f_norm);
/* Gamma index -> global DOF (host int64 array of n_gamma). */
int ddel_gamma_dofs(const ddel_ctx* ctx, int64_t* out);
/* Load vector assembled from ddel_bc (host, n_dof doubles). */
int ddel_load_vector(const ddel_ctx* ctx, double* out);
/* Fixed-DOF mask (host, n_dof bytes). */
int ddel_fixed_mask(const ddel_ctx* ctx, uint8_t* out);

/* Counters and work estimates for profiling (host output).  schur_apply_bytes:
 * algorithmic bytes of one Schur application in the active form and precision
 * (explicit: sum of n_ring_i^2 matrix entries; implicit: the nonzero entries of
 * the block factors -- the D_k triangles and the C_k without their zero band
 * below each row's lowest coupled column -- read twice, forward and backward)
 * plus the ring vectors. */
typedef struct {
  int64_t launches_total;          /* kernel launches issued by the context */
  int64_t launches_since_assemble; /* launches since the last ddel_assemble */
  int64_t schur_apply_bytes;
  int64_t schur_apply_flops;
  int schur_form;                  /* 0 implicit (block substitution), 1 explicit */
  int precision;                   /* active ddel_precision */
  int double_float;                /* 1: explicit FP64 apply in FP32-pair (double-float)
                                      arithmetic, the default with schur_mode AUTO */
} ddel_kernel_info_t;
int ddel_kernel_info(const ddel_ctx* ctx, ddel_kernel_info_t* out);

/* Self-test of failure detection without a fault: a kernel waits on a device
 * barrier that nothing completes, through the same bounded wait (poll_limit
 * polls, 1 <= poll_limit <= 2^22) and error word as the solver's bulk-copy
 * waits, and gives up; *status = DDEL_ETIMEOUT when the timeout was detected
 * and reported (DDEL_OK would mean the wait completed, which cannot happen).
 * The paper has no counterpart.  Synchronises the device. */
int ddel_selftest_wait_timeout(unsigned int poll_limit, int* status);

/* --- Residual check without allocation ----------------------------------------
 * The paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory themselves -- code running under an allocator or
 * runtime that forbids cudaMalloc, or a component that is handed device
 * buffers by someone else and must not own any.  It computes the same FP64
 * quantities as ddel_residual_norm without a context and without allocating:
 * r = f - K(rho) u on the free DOFs (0 on fixed ones) and
 * norms[0] = ||r||_2, norms[1] = ||f||_2 over the free DOFs.
 *
 * Arguments (all device pointers except the sizes and the stream):
 *   dim, nx, ny, nz  grid of unit elements (nz ignored in 2D), node-interleaved
 *                    DOFs as everywhere in this header;
 *   Ke               unit-E element stiffness, (dim 2^dim)^2 doubles, row-major,
 *                    local node order (0,0),(1,0),(1,1),(0,1) [then z = 1];
 *   factors          n_elem doubles: the element stiffness factors E rho_e^p;
 *   fixed            n_dof bytes, nonzero = fixed DOF, or NULL for none;
 *   f, u             n_dof doubles; r: n_dof doubles output or NULL;
 *   norms            2 doubles, written on the device;
 *   cuda_stream      the stream to run on (NULL = legacy default stream).
 * The call is asynchronous on the stream; read norms after synchronising it.
 *
 * Scratch: a fixed 64 KB device array inside the library (one pair of partial
 * sums per thread block plus an arrival counter), present on every GPU that
 * loads the library until the process exits.  It caps the grid at 1,048,576
 * nodes; larger grids return DDEL_EINVAL without launching.  Every call looks
 * up the array's device address on the current device (the first call on a
 * device may load the library's device code there: make it before any stream
 * capture).  Every call on a device
 * shares the one array: calls whose kernels overlap on the GPU (different
 * streams, no ordering between them) race and may return wrong norms;
 * serialise them.  The call clears the counter itself; no other state carries
 * over between calls.  Errors: EINVAL (sizes, null inputs, grid too large),
 * ECUDA (device address lookup or launch failed). */
int ddel_residual_norm_noalloc(int dim, int nx, int ny, int nz, const double* Ke,
                               const double* factors, const uint8_t* fixed, const double* f,
                               const double* u, double* r, double* norms, void* cuda_stream);

/* --- Host-only plan (no CUDA call; for inspection and tests) --------------- */
/* The set-up of ddel_create without any device work: DOF classification,
 * interface ordering, face blocks and element matrix.  Errors as ddel_create. */
typedef struct ddel_plan ddel_plan;
int ddel_plan_create(const ddel_mesh* mesh, const ddel_material* mat, const ddel_bc* bc,
                     double theta, ddel_plan** out);
void ddel_plan_destroy(ddel_plan* plan);
int ddel_plan_info(const ddel_plan* plan, ddel_info_t* info);
/* Gamma index -> global DOF (host int64, n_gamma). */
int ddel_plan_gamma_dofs(const ddel_plan* plan, int64_t* out);
/* Face block b of the preconditioner: first Gamma index, size n, and the n x n
 * row-major matrix H^-1 of eq. NumberEight/NumberNine restricted to the face
 * (host; P may be NULL to query n), mean of diag(H) in *hmean. */
int ddel_plan_face_block(const ddel_plan* plan, int b, int32_t* off, int32_t* n, double* P,
                         double* hmean);
/* Unit-E element stiffness (host, (dim 2^dim)^2 doubles, row-major). */
int ddel_plan_element_matrix(const ddel_plan* plan, double* Ke);
/* The interface mass M and Laplacian L of eq. NumberEight assembled on all of
 * Gamma (the global form of the paper's Tables 1-3, not the face-local one of
 * the preconditioner) for displacement component comp, restricted to that
 * component's free Gamma DOFs: CSR matrices of *n rows with *nnz entries,
 * ascending columns, rows and columns in Gamma order (pos[r] = the Gamma
 * position of row r).  Host arrays: pos (n), rowptr (n + 1), col, M, L (nnz);
 * with pos == NULL only *n and *nnz are returned.  Errors: EINVAL (null plan,
 * comp outside [0, dim), null n or nnz). */
int ddel_plan_interface_operator(const ddel_plan* plan, int comp, int32_t* n, int64_t* nnz, int32_t* pos,
                                 int64_t* rowptr, int32_t* col, double* M, double* L);
/* Interior box of subdomain i: ilo[3], icnt[3] (host int32). */
int ddel_plan_subdomain(const ddel_plan* plan, int i, int32_t* ilo, int32_t* icnt);

#ifdef __cplusplus
}
#endif
#endif /* DDEL_H */
