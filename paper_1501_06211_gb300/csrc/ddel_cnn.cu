// U-Net of the learned initial guess / coarse space (an addition to the
// paper's method, which has no learned part): forward, backward and Adam, all
// in FP32 with FP32 accumulation, NCHW tensors, deterministic reductions.
//
// Architecture (4 levels, widths C0..C3, 3x3 convolutions with zero padding,
// bias and ReLU; 2x2 average pooling; 2x nearest upsampling; skip
// concatenation; 1x1 head without activation):
//   e0 = c(c(x)), e1 = c(c(pool e0)), e2 = c(c(pool e1)), e3 = c(c(pool e2)),
//   d2 = c([up e3, e2]), d1 = c([up d2, e1]), d0 = c([up d1, e0]), y = head(d0).
// Parameters are packed layer by layer as (W[Cout][Cin][k][k], b[Cout]) in the
// order e0a e0b e1a e1b e2a e2b e3a e3b d2 d1 d0 head.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/ddel_learn.h"
#include "ddel_device.cuh"

namespace ddel {
namespace {

constexpr int kTile = 16;     // output tile edge of the convolution kernel
constexpr int kCo = 16;       // output channels per thread
constexpr int kCi = 8;        // input channels per shared-memory stage
constexpr int kGy = 8, kGx = 32;  // pixel tile of the weight-gradient kernel

// out[n][co][p] = bias[co] + sum_ci sum_taps w[co][ci][tap] in[n][ci][p + tap]
// (K = 3: zero padding 1; K = 1: pointwise), optional ReLU.  One thread per
// output pixel computes kCo output channels; input tiles and weights staged in
// shared memory kCi channels at a time.
template <int K, bool RELU>
__global__ void __launch_bounds__(kTile* kTile) conv_kernel(const float* __restrict__ in, int Cin, int H,
                                                            int W, const float* __restrict__ w,
                                                            const float* __restrict__ bias,
                                                            float* __restrict__ out, int Cout) {
  constexpr int P = K / 2, TE = kTile + 2 * P, KK = K * K;
  __shared__ float tin[kCi][TE][TE];
  __shared__ float tw[kCo][kCi][KK];
  const int tilesx = (W + kTile - 1) / kTile;
  const int ty0 = (blockIdx.x / tilesx) * kTile, tx0 = (blockIdx.x % tilesx) * kTile;
  const int co0 = blockIdx.y * kCo, n = blockIdx.z;
  const int tid = threadIdx.x, ly = tid / kTile, lx = tid % kTile;
  const int64_t plane = (int64_t)H * W;
  const float* inn = in + (int64_t)n * Cin * plane;
  float acc[kCo];
#pragma unroll
  for (int o = 0; o < kCo; ++o) acc[o] = 0.f;
  for (int c0 = 0; c0 < Cin; c0 += kCi) {
    for (int i = tid; i < kCi * TE * TE; i += kTile * kTile) {
      const int c = i / (TE * TE), r = (i / TE) % TE, q = i % TE;
      const int gy = ty0 + r - P, gx = tx0 + q - P;
      float v = 0.f;
      if (c0 + c < Cin && gy >= 0 && gy < H && gx >= 0 && gx < W) v = inn[(c0 + c) * plane + gy * W + gx];
      tin[c][r][q] = v;
    }
    for (int i = tid; i < kCo * kCi * KK; i += kTile * kTile) {
      const int o = i / (kCi * KK), c = (i / KK) % kCi, t = i % KK;
      float v = 0.f;
      if (co0 + o < Cout && c0 + c < Cin) v = w[((int64_t)(co0 + o) * Cin + c0 + c) * KK + t];
      tw[o][c][t] = v;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kCi; ++c)
#pragma unroll
      for (int t = 0; t < KK; ++t) {
        const float v = tin[c][ly + t / K][lx + t % K];
#pragma unroll
        for (int o = 0; o < kCo; ++o) acc[o] = fmaf(tw[o][c][t], v, acc[o]);
      }
    __syncthreads();
  }
  const int y = ty0 + ly, x = tx0 + lx;
  if (y >= H || x >= W) return;
  float* outn = out + (int64_t)n * Cout * plane + y * W + x;
#pragma unroll
  for (int o = 0; o < kCo; ++o) {
    if (co0 + o >= Cout) break;
    float v = acc[o] + (bias ? bias[co0 + o] : 0.f);
    if (RELU) v = fmaxf(v, 0.f);
    outn[(int64_t)(co0 + o) * plane] = v;
  }
}

// Partial weight and bias gradients over a share of the pixel tiles:
// part[s][co][ci][tap] = sum_{n,p} g[n][co][p] in[n][ci][p + tap],
// bpart[s][co] = sum_{n,p} g[n][co][p].  Thread (o, c) of a 16 x 16 block
// owns one (co, ci) pair and its K*K taps.
template <int K>
__global__ void __launch_bounds__(256) wgrad_kernel(const float* __restrict__ g, const float* __restrict__ in,
                                                    int N, int Cin, int H, int W, int Cout,
                                                    float* __restrict__ part, float* __restrict__ bpart) {
  constexpr int P = K / 2, KK = K * K, EY = kGy + 2 * P, EX = kGx + 2 * P;
  __shared__ float tg[16][kGy][kGx];
  __shared__ float tin[16][EY][EX + 1];
  const int co0 = blockIdx.x * 16, ci0 = blockIdx.y * 16, s = blockIdx.z, S = gridDim.z;
  const int tid = threadIdx.x, o = tid / 16, c = tid % 16;
  const int tly = (H + kGy - 1) / kGy, tlx = (W + kGx - 1) / kGx, per = tly * tlx;
  const int64_t plane = (int64_t)H * W;
  float acc[KK];
#pragma unroll
  for (int t = 0; t < KK; ++t) acc[t] = 0.f;
  float bacc = 0.f;
  for (int tile = s; tile < N * per; tile += S) {
    const int n = tile / per, ty0 = ((tile % per) / tlx) * kGy, tx0 = (tile % tlx) * kGx;
    for (int i = tid; i < 16 * kGy * kGx; i += 256) {
      const int oo = i / (kGy * kGx), r = (i / kGx) % kGy, q = i % kGx;
      const int y = ty0 + r, x = tx0 + q;
      float v = 0.f;
      if (co0 + oo < Cout && y < H && x < W) v = g[((int64_t)n * Cout + co0 + oo) * plane + y * W + x];
      tg[oo][r][q] = v;
    }
    for (int i = tid; i < 16 * EY * EX; i += 256) {
      const int cc = i / (EY * EX), r = (i / EX) % EY, q = i % EX;
      const int y = ty0 + r - P, x = tx0 + q - P;
      float v = 0.f;
      if (ci0 + cc < Cin && y >= 0 && y < H && x >= 0 && x < W)
        v = in[((int64_t)n * Cin + ci0 + cc) * plane + y * W + x];
      tin[cc][r][q] = v;
    }
    __syncthreads();
    for (int r = 0; r < kGy; ++r)
      for (int q = 0; q < kGx; ++q) {
        const float gv = tg[o][r][q];
        if (c == 0) bacc += gv;
#pragma unroll
        for (int t = 0; t < KK; ++t) acc[t] = fmaf(gv, tin[c][r + t / K][q + t % K], acc[t]);
      }
    __syncthreads();
  }
  if (co0 + o < Cout && ci0 + c < Cin) {
    float* dst = part + (((int64_t)s * Cout + co0 + o) * Cin + ci0 + c) * KK;
#pragma unroll
    for (int t = 0; t < KK; ++t) dst[t] = acc[t];
  }
  if (blockIdx.y == 0 && c == 0 && co0 + o < Cout) bpart[(int64_t)s * Cout + co0 + o] = bacc;
}

// gw[i] = sum_s part[s][i] in split order; gb likewise.
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, const float* __restrict__ bpart, int S,
                                    int64_t nw, int nb, float* __restrict__ gw, float* __restrict__ gb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nw + nb;
       i += (int64_t)gridDim.x * blockDim.x) {
    float a = 0.f;
    if (i < nw) {
      for (int s = 0; s < S; ++s) a += part[s * nw + i];
      gw[i] = a;
    } else {
      const int64_t j = i - nw;
      for (int s = 0; s < S; ++s) a += bpart[s * nb + j];
      gb[j] = a;
    }
  }
}

// wt[ci][co][K-1-dy][K-1-dx] = w[co][ci][dy][dx]: the weights of the
// transposed convolution (gradient with respect to the input).
__global__ void flip_transpose_kernel(const float* __restrict__ w, int Cout, int Cin, int KK,
                                      float* __restrict__ wt) {
  const int64_t n = (int64_t)Cout * Cin * KK;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(i % KK), ci = (int)((i / KK) % Cin), co = (int)(i / ((int64_t)KK * Cin));
    wt[((int64_t)ci * Cout + co) * KK + (KK - 1 - t)] = w[i];
  }
}

__global__ void pool_kernel(const float* __restrict__ in, int NC, int H, int W, float* __restrict__ out) {
  const int h = H / 2, w = W / 2;
  const int64_t n = (int64_t)NC * h * w;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / ((int64_t)h * w);
    const int y = (int)((i / w) % h), x = (int)(i % w);
    const float* p = in + c * H * W + (2 * y) * W + 2 * x;
    out[i] = 0.25f * ((p[0] + p[1]) + (p[W] + p[W + 1]));
  }
}

// g_in[2y+i][2x+j] += g[y][x] / 4
__global__ void pool_bwd_acc_kernel(const float* __restrict__ g, int NC, int H, int W, float* __restrict__ gin) {
  const int64_t n = (int64_t)NC * H * W;
  const int h = H / 2, w = W / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / ((int64_t)H * W);
    const int y = (int)((i / W) % H), x = (int)(i % W);
    gin[i] += 0.25f * g[c * h * w + (y / 2) * w + x / 2];
  }
}

// cat[n] = [up(a[n]) (ca channels), b[n] (cb channels)] at H x W
__global__ void upcat_kernel(const float* __restrict__ a, int ca, const float* __restrict__ b, int cb, int N,
                             int H, int W, float* __restrict__ cat) {
  const int C = ca + cb;
  const int64_t plane = (int64_t)H * W, n = (int64_t)N * C * plane;
  const int h = H / 2, w = W / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / (C * plane);
    const int c = (int)((i / plane) % C);
    const int y = (int)((i / W) % H), x = (int)(i % W);
    cat[i] = c < ca ? a[(s * ca + c) * h * w + (y / 2) * w + x / 2]
                    : b[(s * cb + c - ca) * plane + (int64_t)y * W + x];
  }
}

// From g_cat: g_a[y][x] = sum of the 2x2 block of the first ca channels (the
// adjoint of nearest upsampling), g_b = the last cb channels.
__global__ void upcat_bwd_kernel(const float* __restrict__ gcat, int ca, int cb, int N, int H, int W,
                                 float* __restrict__ ga, float* __restrict__ gb) {
  const int C = ca + cb, h = H / 2, w = W / 2;
  const int64_t plane = (int64_t)H * W;
  const int64_t na = (int64_t)N * ca * h * w, nb = (int64_t)N * cb * plane;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < na + nb;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < na) {
      const int64_t s = i / ((int64_t)ca * h * w);
      const int c = (int)((i / ((int64_t)h * w)) % ca);
      const int y = (int)((i / w) % h), x = (int)(i % w);
      const float* p = gcat + (s * C + c) * plane + (2 * y) * W + 2 * x;
      ga[i] = (p[0] + p[1]) + (p[W] + p[W + 1]);
    } else {
      const int64_t j = i - na;
      const int64_t s = j / (cb * plane), r = j % (cb * plane);
      gb[j] = gcat[(s * C + ca) * plane + r];
    }
  }
}

__global__ void relu_mask_kernel(float* __restrict__ g, const float* __restrict__ a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!(a[i] > 0.f)) g[i] = 0.f;
}

// loss = 0.5 * mean((y - t)^2) (FP64 reduction), gy = (y - t) / n
__global__ void __launch_bounds__(256) mse_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                                  int64_t n, float* __restrict__ gy, double* partials,
                                                  unsigned* ticket, double* loss) {
  __shared__ double scratch[32];
  double acc[1] = {0.0};
  const float inv = (float)(1.0 / (double)n);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    acc[0] += (double)d * (double)d;
    if (gy) gy[i] = d * inv;
  }
  if (grid_sum<1, 256>(acc, partials, ticket, scratch) && threadIdx.x == 0) *loss = 0.5 * acc[0] / (double)n;
}

// Adam (Kingma and Ba) with bias correction; c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t).
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// He-uniform initial weights U(-a, a), a = sqrt(6 / fan_in), zero biases, from
// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) of (seed, parameter index).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void init_kernel(float* __restrict__ p, int64_t off, int64_t nw, int64_t nb, float a,
                            uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nw + nb;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nw) {
      const uint64_t r = splitmix64(seed ^ splitmix64((uint64_t)(off + i)));
      const double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);  // [0, 1)
      p[off + i] = (float)((2.0 * u - 1.0) * a);
    } else {
      p[off + i] = 0.f;
    }
  }
}

int grid1(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 8 * 152 ? 8 * 152 : b));
}

}  // namespace
}  // namespace ddel

using namespace ddel;

struct ddel_cnn;
namespace ddel {
void cnn_stream_gone(ddel_cnn* net);
}

struct ddel_cnn {
  int in_ch = 0, out_ch = 0, H = 0, W = 0, nmax = 0;
  int C[4] = {0, 0, 0, 0};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  struct Layer {
    int cout, cin, k;
    int64_t off;  // weights at off, bias at off + cout * cin * k * k
  };
  std::vector<Layer> L;
  int64_t n_params = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr, *wt = nullptr;
  int64_t t = 0;  // Adam steps taken
  // activations (nmax samples) and their gradients
  float *x = nullptr, *a0a = nullptr, *a0b = nullptr, *p1 = nullptr, *a1a = nullptr, *a1b = nullptr;
  float *p2 = nullptr, *a2a = nullptr, *a2b = nullptr, *p3 = nullptr, *a3a = nullptr, *a3b = nullptr;
  float *cat2 = nullptr, *d2 = nullptr, *cat1 = nullptr, *d1 = nullptr, *cat0 = nullptr, *d0 = nullptr;
  float *y = nullptr, *gy = nullptr, *gA = nullptr, *gB = nullptr, *gC = nullptr;
  float *g0b = nullptr, *g1b = nullptr, *g2b = nullptr;
  float *part = nullptr, *bpart = nullptr;
  int64_t part_elems = 0;
  double* partials = nullptr;
  unsigned* ticket = nullptr;
  double* loss = nullptr;
  double* h_loss = nullptr;
  std::vector<void*> allocs;
  std::string last_error;
};

namespace ddel {
// The borrowed stream's owner has synchronised and destroyed it.
void cnn_stream_gone(ddel_cnn* net) {
  if (!net->own_stream) net->stream = nullptr;
}
}  // namespace ddel

namespace {

int cnn_fail(ddel_cnn* c, int code, const std::string& msg) {
  if (c) c->last_error = msg;
  return code;
}

#define CKC(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return cnn_fail(net, DDEL_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename P>
bool nalloc(ddel_cnn* net, P** p, int64_t elems) {
  void* v = nullptr;
  if (cudaMalloc(&v, (size_t)(elems > 4 ? elems : 4) * sizeof(P)) != cudaSuccess) return false;
  net->allocs.push_back(v);
  *p = static_cast<P*>(v);
  return true;
}

int splits_for(int tiles, int blocks_per_split) {
  int s = (2 * 152 + blocks_per_split - 1) / blocks_per_split;
  if (s > tiles) s = tiles;
  return s < 1 ? 1 : s;
}

void conv(ddel_cnn* net, int li, const float* in, int N, int H, int W, float* out, bool relu) {
  const auto& l = net->L[li];
  const float* w = net->p + l.off;
  const float* b = w + (int64_t)l.cout * l.cin * l.k * l.k;
  dim3 grid(((W + kTile - 1) / kTile) * ((H + kTile - 1) / kTile), (l.cout + kCo - 1) / kCo, N);
  if (l.k == 3) {
    if (relu) conv_kernel<3, true><<<grid, kTile * kTile, 0, net->stream>>>(in, l.cin, H, W, w, b, out, l.cout);
    else conv_kernel<3, false><<<grid, kTile * kTile, 0, net->stream>>>(in, l.cin, H, W, w, b, out, l.cout);
  } else {
    conv_kernel<1, false><<<grid, kTile * kTile, 0, net->stream>>>(in, l.cin, H, W, w, b, out, l.cout);
  }
}

// Gradient of layer li from the gradient gz at its pre-activation output:
// weights/bias into net->g, and (if gin) the input gradient.
void conv_backward(ddel_cnn* net, int li, const float* in, const float* gz, int N, int H, int W, float* gin) {
  const auto& l = net->L[li];
  const int KK = l.k * l.k;
  const int64_t nw = (int64_t)l.cout * l.cin * KK;
  const int tiles = N * ((H + kGy - 1) / kGy) * ((W + kGx - 1) / kGx);
  const int bps = ((l.cout + 15) / 16) * ((l.cin + 15) / 16);
  int S = splits_for(tiles, bps);
  while ((int64_t)S * (nw + l.cout) > net->part_elems && S > 1) S /= 2;
  dim3 grid((l.cout + 15) / 16, (l.cin + 15) / 16, S);
  if (l.k == 3)
    wgrad_kernel<3><<<grid, 256, 0, net->stream>>>(gz, in, N, l.cin, H, W, l.cout, net->part,
                                                   net->part + (int64_t)S * nw);
  else
    wgrad_kernel<1><<<grid, 256, 0, net->stream>>>(gz, in, N, l.cin, H, W, l.cout, net->part,
                                                   net->part + (int64_t)S * nw);
  wgrad_reduce_kernel<<<grid1(nw + l.cout), 256, 0, net->stream>>>(
      net->part, net->part + (int64_t)S * nw, S, nw, l.cout, net->g + l.off, net->g + l.off + nw);
  if (!gin) return;
  flip_transpose_kernel<<<grid1(nw), 256, 0, net->stream>>>(net->p + l.off, l.cout, l.cin, KK, net->wt);
  dim3 g2(((W + kTile - 1) / kTile) * ((H + kTile - 1) / kTile), (l.cin + kCo - 1) / kCo, N);
  if (l.k == 3)
    conv_kernel<3, false><<<g2, kTile * kTile, 0, net->stream>>>(gz, l.cout, H, W, net->wt, nullptr, gin, l.cin);
  else
    conv_kernel<1, false><<<g2, kTile * kTile, 0, net->stream>>>(gz, l.cout, H, W, net->wt, nullptr, gin, l.cin);
}

void relu_mask(ddel_cnn* net, float* g, const float* a, int64_t n) {
  relu_mask_kernel<<<grid1(n), 256, 0, net->stream>>>(g, a, n);
}

void forward(ddel_cnn* net, int N) {
  const int H0 = net->H, W0 = net->W, H1 = H0 / 2, W1 = W0 / 2, H2 = H1 / 2, W2 = W1 / 2, H3 = H2 / 2,
            W3 = W2 / 2;
  const int* C = net->C;
  cudaStream_t s = net->stream;
  conv(net, 0, net->x, N, H0, W0, net->a0a, true);
  conv(net, 1, net->a0a, N, H0, W0, net->a0b, true);
  pool_kernel<<<grid1((int64_t)N * C[0] * H1 * W1), 256, 0, s>>>(net->a0b, N * C[0], H0, W0, net->p1);
  conv(net, 2, net->p1, N, H1, W1, net->a1a, true);
  conv(net, 3, net->a1a, N, H1, W1, net->a1b, true);
  pool_kernel<<<grid1((int64_t)N * C[1] * H2 * W2), 256, 0, s>>>(net->a1b, N * C[1], H1, W1, net->p2);
  conv(net, 4, net->p2, N, H2, W2, net->a2a, true);
  conv(net, 5, net->a2a, N, H2, W2, net->a2b, true);
  pool_kernel<<<grid1((int64_t)N * C[2] * H3 * W3), 256, 0, s>>>(net->a2b, N * C[2], H2, W2, net->p3);
  conv(net, 6, net->p3, N, H3, W3, net->a3a, true);
  conv(net, 7, net->a3a, N, H3, W3, net->a3b, true);
  upcat_kernel<<<grid1((int64_t)N * (C[3] + C[2]) * H2 * W2), 256, 0, s>>>(net->a3b, C[3], net->a2b, C[2], N,
                                                                          H2, W2, net->cat2);
  conv(net, 8, net->cat2, N, H2, W2, net->d2, true);
  upcat_kernel<<<grid1((int64_t)N * (C[2] + C[1]) * H1 * W1), 256, 0, s>>>(net->d2, C[2], net->a1b, C[1], N,
                                                                          H1, W1, net->cat1);
  conv(net, 9, net->cat1, N, H1, W1, net->d1, true);
  upcat_kernel<<<grid1((int64_t)N * (C[1] + C[0]) * H0 * W0), 256, 0, s>>>(net->d1, C[1], net->a0b, C[0], N,
                                                                          H0, W0, net->cat0);
  conv(net, 10, net->cat0, N, H0, W0, net->d0, true);
  conv(net, 11, net->d0, N, H0, W0, net->y, false);
}

// Backward pass from net->gy (gradient at y); parameter gradients into net->g.
void backward(ddel_cnn* net, int N) {
  const int H0 = net->H, W0 = net->W, H1 = H0 / 2, W1 = W0 / 2, H2 = H1 / 2, W2 = W1 / 2, H3 = H2 / 2,
            W3 = W2 / 2;
  const int* C = net->C;
  cudaStream_t s = net->stream;
  const int64_t P0 = (int64_t)N * H0 * W0, P1 = (int64_t)N * H1 * W1, P2 = (int64_t)N * H2 * W2,
                P3 = (int64_t)N * H3 * W3;
  float *gA = net->gA, *gB = net->gB, *gC = net->gC;
  // head and d0
  conv_backward(net, 11, net->d0, net->gy, N, H0, W0, gA);  // gA = g(d0)
  relu_mask(net, gA, net->d0, P0 * C[0]);
  conv_backward(net, 10, net->cat0, gA, N, H0, W0, gB);      // gB = g(cat0)
  upcat_bwd_kernel<<<grid1(P1 * C[1] + P0 * C[0]), 256, 0, s>>>(gB, C[1], C[0], N, H0, W0, gA, net->g0b);
  // d1
  relu_mask(net, gA, net->d1, P1 * C[1]);
  conv_backward(net, 9, net->cat1, gA, N, H1, W1, gB);       // g(cat1)
  upcat_bwd_kernel<<<grid1(P2 * C[2] + P1 * C[1]), 256, 0, s>>>(gB, C[2], C[1], N, H1, W1, gA, net->g1b);
  // d2
  relu_mask(net, gA, net->d2, P2 * C[2]);
  conv_backward(net, 8, net->cat2, gA, N, H2, W2, gB);       // g(cat2)
  upcat_bwd_kernel<<<grid1(P3 * C[3] + P2 * C[2]), 256, 0, s>>>(gB, C[3], C[2], N, H2, W2, gA, net->g2b);
  // level 3: gA = g(a3b)
  relu_mask(net, gA, net->a3b, P3 * C[3]);
  conv_backward(net, 7, net->a3a, gA, N, H3, W3, gB);        // g(a3a)
  relu_mask(net, gB, net->a3a, P3 * C[3]);
  conv_backward(net, 6, net->p3, gB, N, H3, W3, gC);         // g(p3)
  pool_bwd_acc_kernel<<<grid1(P2 * C[2]), 256, 0, s>>>(gC, N * C[2], H2, W2, net->g2b);
  // level 2
  relu_mask(net, net->g2b, net->a2b, P2 * C[2]);
  conv_backward(net, 5, net->a2a, net->g2b, N, H2, W2, gB);
  relu_mask(net, gB, net->a2a, P2 * C[2]);
  conv_backward(net, 4, net->p2, gB, N, H2, W2, gC);         // g(p2)
  pool_bwd_acc_kernel<<<grid1(P1 * C[1]), 256, 0, s>>>(gC, N * C[1], H1, W1, net->g1b);
  // level 1
  relu_mask(net, net->g1b, net->a1b, P1 * C[1]);
  conv_backward(net, 3, net->a1a, net->g1b, N, H1, W1, gB);
  relu_mask(net, gB, net->a1a, P1 * C[1]);
  conv_backward(net, 2, net->p1, gB, N, H1, W1, gC);         // g(p1)
  pool_bwd_acc_kernel<<<grid1(P0 * C[0]), 256, 0, s>>>(gC, N * C[0], H0, W0, net->g0b);
  // level 0
  relu_mask(net, net->g0b, net->a0b, P0 * C[0]);
  conv_backward(net, 1, net->a0a, net->g0b, N, H0, W0, gB);
  relu_mask(net, gB, net->a0a, P0 * C[0]);
  conv_backward(net, 0, net->x, gB, N, H0, W0, nullptr);
}

int check_n(ddel_cnn* net, int n) {
  if (n < 1 || n > net->nmax) return cnn_fail(net, DDEL_EINVAL, "batch outside [1, max_batch]");
  return DDEL_OK;
}

}  // namespace

extern "C" {

int ddel_cnn_create(int in_ch, int out_ch, int H, int W, int max_batch, const int* widths, uint64_t seed,
                    void* cuda_stream, ddel_cnn** out) {
  if (!out) return DDEL_EINVAL;
  *out = nullptr;
  if (in_ch < 1 || out_ch < 1 || H < 8 || W < 8 || H % 8 || W % 8 || max_batch < 1) return DDEL_EINVAL;
  ddel_cnn* net = new (std::nothrow) ddel_cnn();
  if (!net) return DDEL_ENOMEM;
  net->in_ch = in_ch;
  net->out_ch = out_ch;
  net->H = H;
  net->W = W;
  net->nmax = max_batch;
  const int defw[4] = {16, 32, 48, 64};
  for (int i = 0; i < 4; ++i) {
    net->C[i] = widths ? widths[i] : defw[i];
    if (net->C[i] < 1 || net->C[i] > 256) {
      delete net;
      return DDEL_EINVAL;
    }
  }
  const int* C = net->C;
  const int convs[11][2] = {{C[0], in_ch}, {C[0], C[0]}, {C[1], C[0]}, {C[1], C[1]},
                            {C[2], C[1]},  {C[2], C[2]}, {C[3], C[2]}, {C[3], C[3]},
                            {C[2], C[3] + C[2]}, {C[1], C[2] + C[1]}, {C[0], C[1] + C[0]}};
  int64_t off = 0, maxw = 0;
  for (auto& cv : convs) {
    net->L.push_back({cv[0], cv[1], 3, off});
    off += (int64_t)cv[0] * cv[1] * 9 + cv[0];
    maxw = std::max<int64_t>(maxw, (int64_t)cv[0] * cv[1] * 9);
  }
  net->L.push_back({out_ch, C[0], 1, off});
  off += (int64_t)out_ch * C[0] + out_ch;
  net->n_params = off;
  if (cuda_stream) {
    net->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete net;
      return DDEL_ECUDA;
    }
    net->own_stream = true;
  }
  const int64_t N = max_batch, P0 = N * H * W, P1 = P0 / 4, P2 = P1 / 4, P3 = P2 / 4;
  const int64_t gmax = std::max({P0 * (C[1] + C[0]), P1 * (C[2] + C[1]), P2 * (C[3] + C[2]), P0 * out_ch});
  net->part_elems = 2 * 152 * (maxw + 256) + (int64_t)64 * 1024;
  bool ok = nalloc(net, &net->p, off) && nalloc(net, &net->g, off) && nalloc(net, &net->m, off) &&
            nalloc(net, &net->v, off) && nalloc(net, &net->wt, maxw) && nalloc(net, &net->x, P0 * in_ch) &&
            nalloc(net, &net->a0a, P0 * C[0]) && nalloc(net, &net->a0b, P0 * C[0]) &&
            nalloc(net, &net->p1, P1 * C[0]) && nalloc(net, &net->a1a, P1 * C[1]) &&
            nalloc(net, &net->a1b, P1 * C[1]) && nalloc(net, &net->p2, P2 * C[1]) &&
            nalloc(net, &net->a2a, P2 * C[2]) && nalloc(net, &net->a2b, P2 * C[2]) &&
            nalloc(net, &net->p3, P3 * C[2]) && nalloc(net, &net->a3a, P3 * C[3]) &&
            nalloc(net, &net->a3b, P3 * C[3]) && nalloc(net, &net->cat2, P2 * (C[3] + C[2])) &&
            nalloc(net, &net->d2, P2 * C[2]) && nalloc(net, &net->cat1, P1 * (C[2] + C[1])) &&
            nalloc(net, &net->d1, P1 * C[1]) && nalloc(net, &net->cat0, P0 * (C[1] + C[0])) &&
            nalloc(net, &net->d0, P0 * C[0]) && nalloc(net, &net->y, P0 * out_ch) &&
            nalloc(net, &net->gy, P0 * out_ch) && nalloc(net, &net->gA, gmax) && nalloc(net, &net->gB, gmax) &&
            nalloc(net, &net->gC, gmax) && nalloc(net, &net->g0b, P0 * C[0]) &&
            nalloc(net, &net->g1b, P1 * C[1]) && nalloc(net, &net->g2b, P2 * C[2]) &&
            nalloc(net, &net->part, net->part_elems) && nalloc(net, &net->partials, 8 * 152 + 64) &&
            nalloc(net, &net->ticket, 4) && nalloc(net, &net->loss, 2);
  if (!ok || cudaMallocHost(&net->h_loss, sizeof(double)) != cudaSuccess) {
    ddel_cnn_destroy(net);
    return DDEL_ENOMEM;
  }
  cudaMemsetAsync(net->ticket, 0, 16, net->stream);
  cudaMemsetAsync(net->m, 0, off * 4, net->stream);
  cudaMemsetAsync(net->v, 0, off * 4, net->stream);
  for (const auto& l : net->L) {
    const int64_t nw = (int64_t)l.cout * l.cin * l.k * l.k;
    const float a = (float)std::sqrt(6.0 / (double)(l.cin * l.k * l.k));
    init_kernel<<<grid1(nw + l.cout), 256, 0, net->stream>>>(net->p, l.off, nw, l.cout, a, seed);
  }
  if (cudaStreamSynchronize(net->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    ddel_cnn_destroy(net);
    return DDEL_ECUDA;
  }
  *out = net;
  return DDEL_OK;
}

void ddel_cnn_destroy(ddel_cnn* net) {
  if (!net) return;
  if (net->stream) cudaStreamSynchronize(net->stream);  // null once a borrowed stream is gone
  for (void* p : net->allocs) cudaFree(p);
  if (net->h_loss) cudaFreeHost(net->h_loss);
  if (net->own_stream && net->stream) cudaStreamDestroy(net->stream);
  delete net;
}

const char* ddel_cnn_last_error(const ddel_cnn* net) { return net ? net->last_error.c_str() : ""; }

int64_t ddel_cnn_num_params(const ddel_cnn* net) { return net ? net->n_params : -1; }

int ddel_cnn_get_params(ddel_cnn* net, float* out, int on_device) {
  if (!net || !out) return DDEL_EINVAL;
  CKC(cudaMemcpyAsync(out, net->p, net->n_params * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                      net->stream));
  CKC(cudaStreamSynchronize(net->stream));
  return DDEL_OK;
}

int ddel_cnn_set_params(ddel_cnn* net, const float* in, int on_device) {
  if (!net || !in) return DDEL_EINVAL;
  CKC(cudaMemcpyAsync(net->p, in, net->n_params * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      net->stream));
  CKC(cudaMemsetAsync(net->m, 0, net->n_params * 4, net->stream));
  CKC(cudaMemsetAsync(net->v, 0, net->n_params * 4, net->stream));
  net->t = 0;
  CKC(cudaStreamSynchronize(net->stream));
  return DDEL_OK;
}

int ddel_cnn_forward(ddel_cnn* net, const float* x, int n, float* y) {
  if (!net || !x || !y) return DDEL_EINVAL;
  if (int rc = check_n(net, n)) return rc;
  const int64_t P0 = (int64_t)n * net->H * net->W;
  if (x != net->x) CKC(cudaMemcpyAsync(net->x, x, P0 * net->in_ch * 4, cudaMemcpyDeviceToDevice, net->stream));
  forward(net, n);
  if (y != net->y) CKC(cudaMemcpyAsync(y, net->y, P0 * net->out_ch * 4, cudaMemcpyDeviceToDevice, net->stream));
  CKC(cudaGetLastError());
  return DDEL_OK;
}

int ddel_cnn_loss_grad(ddel_cnn* net, const float* x, const float* target, int n, double* loss, float* grad) {
  if (!net || !x || !target) return DDEL_EINVAL;
  if (int rc = check_n(net, n)) return rc;
  const int64_t P0 = (int64_t)n * net->H * net->W, ny = P0 * net->out_ch;
  if (x != net->x) CKC(cudaMemcpyAsync(net->x, x, P0 * net->in_ch * 4, cudaMemcpyDeviceToDevice, net->stream));
  forward(net, n);
  mse_kernel<<<grid1(ny) < 4 * 152 ? grid1(ny) : 4 * 152, 256, 0, net->stream>>>(
      net->y, target, ny, net->gy, net->partials, net->ticket, net->loss);
  backward(net, n);
  if (grad) CKC(cudaMemcpyAsync(grad, net->g, net->n_params * 4, cudaMemcpyDeviceToDevice, net->stream));
  CKC(cudaMemcpyAsync(net->h_loss, net->loss, 8, cudaMemcpyDeviceToHost, net->stream));
  CKC(cudaStreamSynchronize(net->stream));
  CKC(cudaGetLastError());
  if (loss) *loss = *net->h_loss;
  return DDEL_OK;
}

int ddel_cnn_adam_step(ddel_cnn* net, double lr, double beta1, double beta2, double eps) {
  if (!net || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return DDEL_EINVAL;
  net->t += 1;
  const double c1 = 1.0 / (1.0 - std::pow(beta1, (double)net->t));
  const double c2 = 1.0 / (1.0 - std::pow(beta2, (double)net->t));
  adam_kernel<<<grid1(net->n_params), 256, 0, net->stream>>>(net->p, net->g, net->m, net->v, net->n_params,
                                                             (float)lr, (float)beta1, (float)beta2, (float)eps,
                                                             (float)c1, (float)c2);
  CKC(cudaGetLastError());
  return DDEL_OK;
}

}  // extern "C"
