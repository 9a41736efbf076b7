// Learned (or history) coarse space for the interface PCG of a solver
// context: node-grid features, training targets, replay buffer and the map of
// the network's fields onto the Gamma DOFs.  Not part of the paper's method.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/ddel.h"
#include "../../include/ddel_learn.h"
#include "ddel_device.cuh"

namespace ddel {
cudaStream_t ctx_stream(const ddel_ctx* ctx);
ddel_mesh ctx_mesh(const ddel_ctx* ctx);
void ctx_attach_learner(ddel_ctx* ctx, ddel_learner* L);
void ctx_detach_learner(ddel_ctx* ctx, ddel_learner* L);
void cnn_stream_gone(ddel_cnn* net);  // ddel_cnn.cu

namespace {

// Network input [3][H][W] (nodal filtered density, loads / max|f|) and, with u,
// the target [4][H][W] (rho_n u^_x, rho_n u^_y, (1 - rho_n) u^_x,
// (1 - rho_n) u^_y, u^ = u / max|u|); zero outside the node grid.
__global__ void features_kernel(const double* __restrict__ rho_f, int nx, int ny,
                                const double* __restrict__ f, double inv_fmax,
                                const double* __restrict__ u, const double* __restrict__ umax, int H,
                                int W, float* __restrict__ x, float* __restrict__ t) {
  const int64_t plane = (int64_t)H * W;
  const double inv_u = (u && *umax > 0.0) ? 1.0 / *umax : 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < plane;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(p / W), j = (int)(p % W);
    float v[3] = {0.f, 0.f, 0.f}, tv[4] = {0.f, 0.f, 0.f, 0.f};
    if (i <= nx && j <= ny) {
      double rs = 0.0;
      int cnt = 0;
      for (int a = i - 1; a <= i; ++a)
        for (int b = j - 1; b <= j; ++b)
          if (a >= 0 && a < nx && b >= 0 && b < ny) {
            rs += rho_f[(int64_t)a * ny + b];
            ++cnt;
          }
      const double rn = rs / cnt;
      const int64_t node = (int64_t)i * (ny + 1) + j;
      v[0] = (float)rn;
      v[1] = (float)(f[2 * node] * inv_fmax);
      v[2] = (float)(f[2 * node + 1] * inv_fmax);
      if (u) {
        const double ux = u[2 * node] * inv_u, uy = u[2 * node + 1] * inv_u;
        tv[0] = (float)(rn * ux);
        tv[1] = (float)(rn * uy);
        tv[2] = (float)((1.0 - rn) * ux);
        tv[3] = (float)((1.0 - rn) * uy);
      }
    }
    for (int c = 0; c < 3; ++c) x[c * plane + p] = v[c];
    if (t)
      for (int c = 0; c < 4; ++c) t[c * plane + p] = tv[c];
  }
}

// out = max_i |u_i| (one block, fixed order).
__global__ void __launch_bounds__(1024) absmax_kernel(const double* __restrict__ u, int64_t n, double* out) {
  __shared__ double red[32];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(u[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) *out = m;
  }
}

// Z[q][g] = field q at the node of Gamma DOF g when q % 2 is its component, else 0.
__global__ void zfields_kernel(const float* __restrict__ y, int H, int W, int ny,
                               const int64_t* __restrict__ gamma_dof, int64_t n_gamma, double* __restrict__ Z) {
  const int64_t plane = (int64_t)H * W;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_gamma;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t dof = gamma_dof[g], node = dof / 2;
    const int c = (int)(dof % 2);
    const int64_t p = (node / (ny + 1)) * W + node % (ny + 1);
    for (int q = 0; q < 4; ++q) Z[q * n_gamma + g] = (q % 2 == c) ? (double)y[q * plane + p] : 0.0;
  }
}

__global__ void gather_gamma_kernel(const double* __restrict__ u, const int64_t* __restrict__ gamma_dof,
                                    int64_t n_gamma, double* __restrict__ out) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_gamma;
       g += (int64_t)gridDim.x * blockDim.x)
    out[g] = u[gamma_dof[g]];
}

int grid1(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 4 * 152 ? 4 * 152 : b));
}

}  // namespace
}  // namespace ddel

using namespace ddel;

struct ddel_learner {
  ddel_ctx* ctx = nullptr;
  ddel_learner_options opt{};
  cudaStream_t s = nullptr;
  int nx = 0, ny = 0, H = 0, W = 0;
  int64_t n_elem = 0, n_dof = 0, n_gamma = 0;
  ddel_cnn* net = nullptr;
  int64_t* d_gamma = nullptr;
  double* d_load = nullptr;
  double inv_fmax = 0.0;
  float *rx = nullptr, *rt = nullptr, *xin = nullptr, *yout = nullptr;
  double *Z = nullptr, *hist = nullptr, *umax = nullptr;
  int count = 0, next = 0;  // replay buffer: stored observations, next slot
  int hcount = 0;           // history ring: stored interface solutions
  ddel_learner_info info{};
  cudaEvent_t ev[4] = {};
  std::vector<void*> allocs;
};

namespace ddel {
// The context is being destroyed (its stream already synchronised): the
// learner keeps only its own memory and refuses further work.
void learner_context_gone(ddel_learner* L) {
  L->ctx = nullptr;
  L->s = nullptr;
  if (L->net) cnn_stream_gone(L->net);
}
}  // namespace ddel

namespace {

template <typename P>
bool lalloc(ddel_learner* L, P** p, int64_t elems) {
  void* v = nullptr;
  if (cudaMalloc(&v, (size_t)(elems > 1 ? elems : 1) * sizeof(P)) != cudaSuccess) return false;
  L->allocs.push_back(v);
  *p = static_cast<P*>(v);
  return true;
}

}  // namespace

extern "C" {

void ddel_learner_default_options(ddel_learner_options* o) {
  if (!o) return;
  o->mode = DDEL_LEARN_CNN;
  o->coarse_flags = DDEL_COARSE_X0 | DDEL_COARSE_CORRECT;
  o->k_history = 4;
  o->replay = 16;
  o->train_steps = 4;
  o->batch = 8;
  o->min_samples = 2;
  o->lr = 1e-3;
  const int w[4] = {16, 32, 48, 64};
  for (int i = 0; i < 4; ++i) o->widths[i] = w[i];
  o->seed = 1;
}

int ddel_learner_create(ddel_ctx* ctx, const ddel_learner_options* opt, ddel_learner** out) {
  if (!ctx || !out) return DDEL_EINVAL;
  *out = nullptr;
  ddel_learner_options o;
  if (opt) o = *opt;
  else ddel_learner_default_options(&o);
  const ddel_mesh m = ctx_mesh(ctx);
  if (m.dim != 2) return DDEL_EINVAL;
  if (o.mode != DDEL_LEARN_CNN && o.mode != DDEL_LEARN_HISTORY && o.mode != DDEL_LEARN_CNN_HISTORY)
    return DDEL_EINVAL;
  const int kmax = o.mode == DDEL_LEARN_HISTORY ? DDEL_MAX_COARSE : DDEL_MAX_COARSE - 4;
  if (o.mode != DDEL_LEARN_CNN && (o.k_history < 1 || o.k_history > kmax)) return DDEL_EINVAL;
  if (o.mode != DDEL_LEARN_HISTORY &&
      (o.replay < 1 || o.train_steps < 0 || o.min_samples < 1 || !(o.lr > 0) || o.batch < 1))
    return DDEL_EINVAL;
  ddel_info_t info;
  if (int rc = ddel_get_info(ctx, &info)) return rc;
  ddel_learner* L = new (std::nothrow) ddel_learner();
  if (!L) return DDEL_ENOMEM;
  L->ctx = ctx;
  L->opt = o;
  L->s = ctx_stream(ctx);
  L->nx = m.nx;
  L->ny = m.ny;
  L->H = (m.nx + 1 + 7) / 8 * 8;
  L->W = (m.ny + 1 + 7) / 8 * 8;
  L->n_elem = info.n_elem;
  L->n_dof = info.n_dof;
  L->n_gamma = info.n_gamma;
  L->info.last_loss = -1.0;
  std::vector<int64_t> gd(L->n_gamma);
  std::vector<double> load(L->n_dof);
  int rc = ddel_gamma_dofs(ctx, gd.data());
  if (!rc) rc = ddel_load_vector(ctx, load.data());
  double fmax = 0.0;
  for (double v : load) fmax = std::max(fmax, std::fabs(v));
  L->inv_fmax = fmax > 0 ? 1.0 / fmax : 0.0;
  const int64_t plane = (int64_t)L->H * L->W;
  const int R = o.mode != DDEL_LEARN_HISTORY ? o.replay : 1;
  bool ok = !rc && lalloc(L, &L->d_gamma, L->n_gamma) && lalloc(L, &L->d_load, L->n_dof) &&
            lalloc(L, &L->Z, (int64_t)DDEL_MAX_COARSE * L->n_gamma) &&
            lalloc(L, &L->hist, (int64_t)DDEL_MAX_COARSE * L->n_gamma) && lalloc(L, &L->umax, 1) &&
            lalloc(L, &L->rx, (int64_t)R * 3 * plane) && lalloc(L, &L->rt, (int64_t)R * 4 * plane) &&
            lalloc(L, &L->xin, 3 * plane) && lalloc(L, &L->yout, 4 * plane);
  for (auto& e : L->ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
  ok = ok && cudaMemcpy(L->d_gamma, gd.data(), gd.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(L->d_load, load.data(), load.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok && o.mode != DDEL_LEARN_HISTORY) {
    rc = ddel_cnn_create(3, 4, L->H, L->W, R, o.widths, o.seed, L->s, &L->net);
    ok = rc == DDEL_OK;
  }
  if (!ok) {
    ddel_learner_destroy(L);
    return rc ? rc : DDEL_ENOMEM;
  }
  ctx_attach_learner(ctx, L);
  *out = L;
  return DDEL_OK;
}

void ddel_learner_destroy(ddel_learner* L) {
  if (!L) return;
  if (L->ctx) {  // else the context (and its stream) is gone and was synchronised
    cudaStreamSynchronize(L->s);
    ctx_detach_learner(L->ctx, L);
  }
  if (L->net) ddel_cnn_destroy(L->net);
  for (auto e : L->ev)
    if (e) cudaEventDestroy(e);
  for (void* p : L->allocs) cudaFree(p);
  delete L;
}

int ddel_learner_grid(const ddel_learner* L, int* H, int* W) {
  if (!L) return DDEL_EINVAL;
  if (H) *H = L->H;
  if (W) *W = L->W;
  return DDEL_OK;
}

ddel_cnn* ddel_learner_network(ddel_learner* L) { return L ? L->net : nullptr; }

int ddel_learner_features(ddel_learner* L, const double* rho_f, const double* u, float* x, float* target) {
  if (!L || !rho_f || !x || (u && !target)) return DDEL_EINVAL;
  if (!L->ctx) return DDEL_ESTATE;
  if (u) absmax_kernel<<<1, 1024, 0, L->s>>>(u, L->n_dof, L->umax);
  features_kernel<<<grid1((int64_t)L->H * L->W), 256, 0, L->s>>>(rho_f, L->nx, L->ny, L->d_load, L->inv_fmax,
                                                                 u, L->umax, L->H, L->W, x, u ? target : nullptr);
  return cudaGetLastError() == cudaSuccess ? DDEL_OK : DDEL_ECUDA;
}

int ddel_learner_predict(ddel_learner* L, const double* rho_f) {
  if (!L || !rho_f) return DDEL_EINVAL;
  if (!L->ctx) return DDEL_ESTATE;
  const int flags = L->opt.coarse_flags;
  const bool use_hist = L->opt.mode != DDEL_LEARN_CNN, use_net = L->opt.mode != DDEL_LEARN_HISTORY;
  const int kh = use_hist ? std::min(L->hcount, L->opt.k_history) : 0;
  const bool net_ready = use_net && L->count >= L->opt.min_samples;
  const int k = kh + (net_ready ? 4 : 0);
  if (k == 0) return ddel_set_coarse(L->ctx, nullptr, 0, 0, 1);
  // Z = [the kh latest interface solutions, the network's four fields]
  if (kh > 0 && cudaMemcpyAsync(L->Z, L->hist, (size_t)kh * L->n_gamma * 8, cudaMemcpyDeviceToDevice, L->s) !=
                    cudaSuccess)
    return DDEL_ECUDA;
  if (net_ready) {
    cudaEventRecord(L->ev[2], L->s);
    int rc = ddel_learner_features(L, rho_f, nullptr, L->xin, nullptr);
    if (!rc) rc = ddel_cnn_forward(L->net, L->xin, 1, L->yout);
    if (rc) return rc;
    zfields_kernel<<<grid1(L->n_gamma), 256, 0, L->s>>>(L->yout, L->H, L->W, L->ny, L->d_gamma, L->n_gamma,
                                                       L->Z + (int64_t)kh * L->n_gamma);
    if (cudaGetLastError() != cudaSuccess) return DDEL_ECUDA;
    cudaEventRecord(L->ev[3], L->s);
  }
  const int rc = ddel_set_coarse(L->ctx, L->Z, k, flags, 1);
  if (!rc) {
    L->info.predictions += 1;
    if (net_ready) {
      cudaEventSynchronize(L->ev[3]);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, L->ev[2], L->ev[3]);
      L->info.t_predict_ms = ms;
    }
  }
  return rc;
}

int ddel_learner_observe(ddel_learner* L, const double* rho_f, const double* u) {
  if (!L || !rho_f || !u) return DDEL_EINVAL;
  if (!L->ctx) return DDEL_ESTATE;
  if (L->opt.mode != DDEL_LEARN_CNN) {
    // history ring, newest first: shift so that column 0 is the latest solution
    const int k = L->opt.k_history;
    for (int q = std::min(L->hcount, k - 1); q > 0; --q)
      if (cudaMemcpyAsync(L->hist + q * L->n_gamma, L->hist + (q - 1) * L->n_gamma, L->n_gamma * 8,
                          cudaMemcpyDeviceToDevice, L->s) != cudaSuccess)
        return DDEL_ECUDA;
    gather_gamma_kernel<<<grid1(L->n_gamma), 256, 0, L->s>>>(u, L->d_gamma, L->n_gamma, L->hist);
    L->hcount = std::min(L->hcount + 1, k);
  }
  if (L->opt.mode == DDEL_LEARN_HISTORY) {
    L->info.samples = L->hcount;
    return cudaStreamSynchronize(L->s) == cudaSuccess ? DDEL_OK : DDEL_ECUDA;
  }
  const int64_t plane = (int64_t)L->H * L->W;
  const int slot = L->next;
  int rc = ddel_learner_features(L, rho_f, u, L->rx + (int64_t)slot * 3 * plane,
                                 L->rt + (int64_t)slot * 4 * plane);
  if (rc) return rc;
  L->next = (L->next + 1) % L->opt.replay;
  L->count = std::min(L->count + 1, L->opt.replay);
  L->info.samples = L->count;
  cudaEventRecord(L->ev[0], L->s);
  // minibatch: the `batch` newest observations as one contiguous run of slots
  // (when the newest lie at the start of the ring, the first `batch` slots)
  const int nb = std::min(L->count, L->opt.batch);
  const int first = L->next >= nb ? L->next - nb : 0;
  const float* bx = L->rx + (int64_t)first * 3 * plane;
  const float* bt = L->rt + (int64_t)first * 4 * plane;
  for (int step = 0; step < L->opt.train_steps; ++step) {
    double loss = 0.0;
    rc = ddel_cnn_loss_grad(L->net, bx, bt, nb, &loss, nullptr);
    if (!rc) rc = ddel_cnn_adam_step(L->net, L->opt.lr, 0.9, 0.999, 1e-8);
    if (rc) return rc;
    if (step == 0) L->info.last_loss = loss;
    L->info.adam_steps += 1;
  }
  cudaEventRecord(L->ev[1], L->s);
  if (cudaEventSynchronize(L->ev[1]) != cudaSuccess) return DDEL_ECUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, L->ev[0], L->ev[1]);
  L->info.t_train_ms = ms;
  return DDEL_OK;
}

int ddel_learner_get_info(const ddel_learner* L, ddel_learner_info* info) {
  if (!L || !info) return DDEL_EINVAL;
  *info = L->info;
  return DDEL_OK;
}

}  // extern "C"
