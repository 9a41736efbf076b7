/* Learned initial guess and coarse space for the interface PCG of ddel.h.
 *
 * Not part of the paper's method: arXiv:1501.06211 preconditions the
 * interface problem with face-local operators only (Sec. 3-4) and solves each
 * Picard step of the topology optimisation (Sec. 5) from scratch.  This header
 * adds
 *   - ddel_cnn: a 4-level U-Net (3x3 convolutions, 2x2 average pooling, 2x
 *     nearest upsampling, skip concatenation, 1x1 head) with forward, backward
 *     (mean-squared-error loss) and Adam, all in CUDA kernels, FP32 storage and
 *     accumulation, deterministic reductions;
 *   - ddel_learner: per solver context, it maps the filtered densities and the
 *     loads on the node grid to coarse fields (ddel_set_coarse) before each
 *     solve, and trains online on the converged displacements of the last
 *     Picard steps; or, in HISTORY mode, uses the last k interface solutions
 *     themselves as the coarse space (no network).
 *
 * Status codes are those of ddel.h.  Every device pointer argument is a CUDA
 * device address; every call is asynchronous on the object's stream unless it
 * says that it synchronises. */
#ifndef DDEL_LEARN_H
#define DDEL_LEARN_H

#include <stdint.h>

#include "ddel.h"

#ifdef __cplusplus
extern "C" {
#endif

/* --- U-Net ---------------------------------------------------------------------
 * Tensors are NCHW float32 on the device: input [n][in_ch][H][W], output
 * [n][out_ch][H][W], H and W multiples of 8 (three 2x poolings), n <= max_batch.
 * widths: channels of the four levels (NULL: 16, 32, 48, 64; each 1..256).
 * Parameters (ddel_cnn_num_params floats) are packed layer by layer as
 * (W[Cout][Cin][k][k], b[Cout]) in the order e0a e0b e1a e1b e2a e2b e3a e3b d2 d1
 * d0 head; initial weights He-uniform U(-a, a), a = sqrt(6 / fan_in), from
 * SplitMix64 of (seed, index), biases 0.  cuda_stream: a cudaStream_t or NULL
 * for an owned stream.  Errors: EINVAL (sizes), ENOMEM, ECUDA. */
typedef struct ddel_cnn ddel_cnn;
int ddel_cnn_create(int in_ch, int out_ch, int H, int W, int max_batch, const int* widths, uint64_t seed,
                    void* cuda_stream, ddel_cnn** out);
void ddel_cnn_destroy(ddel_cnn* net);
const char* ddel_cnn_last_error(const ddel_cnn* net);
int64_t ddel_cnn_num_params(const ddel_cnn* net);
/* Copy the parameters out / in (host when on_device == 0); set_params also
 * resets the Adam moments and step count.  Both synchronise. */
int ddel_cnn_get_params(ddel_cnn* net, float* out, int on_device);
int ddel_cnn_set_params(ddel_cnn* net, const float* in, int on_device);
/* y = net(x) for n samples (device x, y). */
int ddel_cnn_forward(ddel_cnn* net, const float* x, int n, float* y);
/* loss = 0.5 * mean((net(x) - target)^2) and its parameter gradient, kept in
 * the object for ddel_cnn_adam_step and copied to grad (device, may be NULL).
 * Synchronises (loss to the host). */
int ddel_cnn_loss_grad(ddel_cnn* net, const float* x, const float* target, int n, double* loss, float* grad);
/* One Adam step (Kingma and Ba, bias-corrected) with the last gradient. */
int ddel_cnn_adam_step(ddel_cnn* net, double lr, double beta1, double beta2, double eps);

/* --- Learned coarse space of a solver context (2D) --------------------------------
 * Node grid (nx+1) x (ny+1), zero-padded to multiples of 8.  Network input (3
 * channels): nodal filtered density (mean of the adjacent elements), and the
 * two load components divided by max |f|.  Output / training target (4
 * channels): rho_n u^_x, rho_n u^_y, (1 - rho_n) u^_x, (1 - rho_n) u^_y with
 * u^ = u / max |u| of a converged solution: the displacement shape split by
 * component and into its stiff and soft parts.  The coarse space is these four
 * fields on the Gamma DOFs (each nonzero in one component), so its span holds
 * the predicted displacement field itself; with DDEL_COARSE_X0 the PCG starts
 * from the best (energy-norm) combination of them.
 * mode CNN: before each solve, fields of the network (once min_samples
 * observations are stored); after it, the observation joins a replay buffer of
 * the last `replay` steps and train_steps Adam steps run on its `batch` newest
 * observations.
 * mode HISTORY: the coarse space is the last k_history interface solutions.
 * mode CNN_HISTORY: both, the k_history solutions first (k_history <= 4). */
typedef enum { DDEL_LEARN_CNN = 0, DDEL_LEARN_HISTORY = 1, DDEL_LEARN_CNN_HISTORY = 2 } ddel_learn_mode;
typedef struct {
  int mode;           /* ddel_learn_mode (CNN) */
  int coarse_flags;   /* ddel_coarse_flags for ddel_set_coarse (X0 | CORRECT) */
  int k_history;      /* HISTORY, CNN_HISTORY: solutions kept (4; at most DDEL_MAX_COARSE,
                         or DDEL_MAX_COARSE - 4 with the network) */
  int replay;         /* CNN: observations kept (16) */
  int train_steps;    /* CNN: Adam steps per observation (4) */
  int batch;          /* CNN: minibatch, the newest observations of the replay buffer (8) */
  int min_samples;    /* CNN: observations before the first prediction (2) */
  double lr;          /* CNN: Adam learning rate (1e-3) */
  int widths[4];      /* CNN: level widths (16, 32, 48, 64) */
  uint64_t seed;      /* CNN: initial weights (1) */
} ddel_learner_options;
typedef struct {
  int samples;        /* observations stored (replay buffer; HISTORY: solutions) */
  int predictions;    /* coarse spaces set from the network or the history */
  int64_t adam_steps;
  double last_loss;   /* loss before the last training step (-1: none) */
  double t_train_ms;  /* device time of the last training (all steps) */
  double t_predict_ms;
} ddel_learner_info;
typedef struct ddel_learner ddel_learner;
void ddel_learner_default_options(ddel_learner_options* opt);
/* For a 2D context; runs on the context's stream.  EINVAL for 3D or bad
 * options, ENOMEM, ECUDA. */
int ddel_learner_create(ddel_ctx* ctx, const ddel_learner_options* opt, ddel_learner** out);
void ddel_learner_destroy(ddel_learner* L);
/* Coarse space for the next solve from the filtered densities rho_f (device,
 * n_elem); with too few observations it removes the coarse space instead. */
int ddel_learner_predict(ddel_learner* L, const double* rho_f);
/* Stores (rho_f, u) (device: n_elem, n_dof; u a converged solution) and trains.
 * Synchronises. */
int ddel_learner_observe(ddel_learner* L, const double* rho_f, const double* u);
int ddel_learner_get_info(const ddel_learner* L, ddel_learner_info* info);
/* Network input / target of one observation (device float, [3][H][W] and
 * [4][H][W]; u may be NULL for the input only), H and W as ddel_learner_grid. */
int ddel_learner_features(ddel_learner* L, const double* rho_f, const double* u, float* x, float* target);
int ddel_learner_grid(const ddel_learner* L, int* H, int* W);
ddel_cnn* ddel_learner_network(ddel_learner* L);

#ifdef __cplusplus
}
#endif

#endif /* DDEL_LEARN_H */
