// Tensor-core (tcgen05) formation of the local Schur complements at FP64
// accuracy; included by ddel_kernels.cu inside its anonymous namespace, after
// the element helpers (kgg_entry2d) it uses.
#pragma once

// Local Schur complements S_i = K_GG^(i) - W^T W (W = L^-1 K_IG^(i), FP64)
// with the product W^T W on the tensor cores (tcgen05, BF16 operands, FP32
// accumulation in tensor memory) at FP64 accuracy by error-free splitting:
// the Ozaki scheme (Ozaki, Ogita, Oishi, Rump 2012).  Each column j of W is
// scaled by 2^-e_j (e_j: the exponent of its largest entry) and cut into S
// slices of B bits, W[:, j] = 2^e_j sum_p 2^(-B p) D_p[:, j], every D_p an
// integer matrix with |entries| <= 2^B (exact in BF16).  Then
//   (W^T W)_ij = 2^(e_i + e_j) sum_{p, q} 2^(-B (p + q)) (D_p^T D_q)_ij,
// and every integer product sum D_p^T D_q is exact in FP32 as long as its
// magnitude stays below 2^24, which B is chosen for (B = 6 up to 1489 rows of
// W, else 5); the pairs of one d = p + q share a scale and one accumulator.
// Dropped pairs (p + q > S + 1) leave a relative truncation below 2^-(B (S+1)),
// S B >= 54 bits.  The accumulators are drained into FP64 (smallest d
// first) on top of K_GG.
//
// ozaki_slice_kernel: per subdomain and ring column, e_j and the slices
//   (BF16, stored [slice][column][row] with the rows contiguous, zero padded
//   to a multiple of 64 rows).
// ozaki_syrk_kernel: one CTA of 128 threads per (subdomain, 128 x 128 tile of
//   S); per K chunk of 64 rows the two operand tiles are copied to shared
//   memory in the canonical K-major no-swizzle layout (8 x 8 core matrices of
//   128 bytes, K-adjacent core matrices 128 B apart, 8-row groups 256 B
//   apart) and thread 0 issues four 128 x 128 x 16 MMAs into a 128-column
//   accumulator in tensor memory; completion is signalled on an mbarrier
//   (bounded wait).  The four warps then read the accumulator (each its 32
//   lanes = rows) and add it, scaled, into the FP64 tile in shared memory.


constexpr int kOzThreads = 128;
constexpr int kOzKC = 64;      // rows of W per operand chunk
constexpr int kOzTile = 128;   // output tile edge (MMA M = N)
constexpr int kOzLd = kOzTile + 1;  // FP64 tile row stride (rows in distinct banks)

__device__ __forceinline__ int oz_bits(int K) { return K <= 1489 ? 6 : 5; }
__device__ __host__ __forceinline__ int oz_slices(int bits) { return (54 + bits - 1) / bits; }

// Slices of W for every subdomain.  W: per subdomain nb_max * BP rows of NR
// doubles; Wsl: per subdomain S * NR * Kp BF16 values (Kp = rows rounded up to
// kOzKC); expo: per subdomain NR ints.  One thread per (subdomain, column).
__global__ void ozaki_slice_kernel(DevTables t, const double* __restrict__ W, int NR, int Kp,
                                   __nv_bfloat16* __restrict__ Wsl, int* __restrict__ expo) {
  const int sub = blockIdx.x, j = threadIdx.x + blockIdx.y * blockDim.x;
  if (j >= NR) return;
  const SubInfo si = t.subs[sub];
  const int K = si.nb * t.BP;  // rows of this subdomain's W (the rest are zero)
  const int bits = oz_bits(Kp), S = oz_slices(bits);
  const double* Wc = W + (int64_t)sub * t.nb_max * t.BP * NR + j;
  double mx = 0.0;
  for (int k = 0; k < K; ++k) mx = fmax(mx, fabs(Wc[(int64_t)k * NR]));
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);  // mx = f 2^e, 0.5 <= f < 1: |W_kj| 2^-e < 1
  expo[(int64_t)sub * NR + j] = e;
  __nv_bfloat16* out = Wsl + (int64_t)sub * S * NR * Kp;
  const double up = ldexp(1.0, bits);
  for (int k = 0; k < Kp; ++k) {
    double v = k < K ? ldexp(Wc[(int64_t)k * NR], -e) : 0.0;
    for (int p = 0; p < S; ++p) {
      const double tv = v * up;    // exact: a power-of-two scaling
      const double dv = rint(tv);  // |dv| <= 2^bits, an integer
      v = tv - dv;                 // exact: |v| <= 1/2
      out[((int64_t)p * NR + j) * Kp + k] = __double2bfloat16(dv);
    }
  }
}

// ---- tcgen05 helpers (single-CTA forms) ------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major without swizzling: start address,
// leading-dimension (K-direction) and stride-dimension (M/N-direction) byte
// offsets between core matrices, descriptor version 1 (bits 46-47).
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
  const uint64_t a = smem_addr(p);
  return ((a >> 4) & 0x3FFFull) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 D, both
// operands K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

// 32 consecutive FP32 columns of this thread's lane (tensor-memory row).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Copies rows [r0, r0 + 128) x chunk rows [k0, k0 + 64) of one slice (stored
// [column][row], rows contiguous) into the operand layout: K slab s (16 rows
// of W) at s * 4096 bytes, in it the core matrix of 8-column group g and
// 8-row half h at g * 256 + h * 128, each core-matrix row 16 bytes.
__device__ __forceinline__ void oz_load_tile(const __nv_bfloat16* __restrict__ sl, int Kp, int c0, int k0,
                                             unsigned char* dst) {
  for (int v = threadIdx.x; v < kOzTile * (kOzKC / 8); v += blockDim.x) {
    const int c = v / (kOzKC / 8), kq = v % (kOzKC / 8);  // column, 8-row octet
    const uint4 val = *reinterpret_cast<const uint4*>(sl + (int64_t)(c0 + c) * Kp + k0 + 8 * kq);
    const int s = kq >> 1, h = kq & 1;
    *reinterpret_cast<uint4*>(dst + s * 4096 + (c >> 3) * 256 + h * 128 + (c & 7) * 16) = val;
  }
}

// S tile (ta, tb) of one subdomain: K_GG entries plus -2^(e_i + e_j) sum_d
// 2^(-B d) C_d, C_d = sum_{p + q = d} D_p^T D_q accumulated in tensor memory.
// Dynamic shared memory: the FP64 tile (128 x 128), two operand tiles (16 KB
// each), column scales, the element data of K_GG.  err: set to kErrTimeout
// when a bounded wait runs out (the kernel then skips the remaining work,
// still frees its tensor memory and returns).
template <int NR>
__global__ void __launch_bounds__(kOzThreads, 1) ozaki_syrk_kernel(DevTables t, const double* __restrict__ Ke_g,
                                                                   const double* __restrict__ scale,
                                                                   const __nv_bfloat16* __restrict__ Wsl,
                                                                   const int* __restrict__ expo, int Kp,
                                                                   double* __restrict__ Sexp, int* err) {
  constexpr int NT = NR / kOzTile;
  const int sub = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int ta = 0, q = blockIdx.y;  // tile index -> (ta, tb), ta <= tb
  while (q >= NT - ta) {
    q -= NT - ta;
    ++ta;
  }
  const int tb = ta + q;
  const SubInfo si = t.subs[sub];
  const int s = t.s;
  const int bits = oz_bits(Kp), S = oz_slices(bits);
  extern __shared__ __align__(1024) unsigned char oz_smem[];
  double* St = reinterpret_cast<double*>(oz_smem);                 // 128 x kOzLd FP64
  unsigned char* At = oz_smem + kOzTile * kOzLd * 8;               // 16 KB
  unsigned char* Bt = At + kOzTile * kOzKC * 2;                     // 16 KB
  double* colsc = reinterpret_cast<double*>(Bt + kOzTile * kOzKC * 2);  // 128: 2^e_j of tile tb
  float* rowsc = reinterpret_cast<float*>(colsc + kOzTile);         // 128: 2^(e_i - B d) of tile ta
  double* ke = reinterpret_cast<double*>(rowsc + kOzTile);          // 64
  double* sc = ke + 64;                                             // s * s
  int* rl = reinterpret_cast<int*>(sc + s * s);                     // 256: ring locs of ta, tb
  int* erow = rl + 2 * kOzTile;                                     // 128
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  for (int i = tid; i < 64; i += kOzThreads) ke[i] = Ke_g[i];
  for (int i = tid; i < s * s; i += kOzThreads)
    sc[i] = scale[(int64_t)(si.lo[0] + i / s) * t.ne[1] + si.lo[1] + i % s];
  for (int j = tid; j < 2 * kOzTile; j += kOzThreads) {
    const int jr = (j < kOzTile ? ta : tb) * kOzTile + j % kOzTile;
    rl[j] = jr < si.n_ring ? t.ring_loc[si.ring_off + jr] : -1;
  }
  const int* ex = expo + (int64_t)sub * NR;
  for (int j = tid; j < kOzTile; j += kOzThreads) {
    colsc[j] = ldexp(1.0, ex[tb * kOzTile + j]);
    erow[j] = ex[ta * kOzTile + j];
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    s_fail = 0;
  }
  if (warp == 0) tmem_alloc(&tmem_base, 128);
  __syncthreads();
  // K_GG part of the tile (FP64)
  for (int v = tid; v < kOzTile * kOzTile; v += kOzThreads) {
    const int i = v / kOzTile, j = v % kOzTile;
    St[i * kOzLd + j] = kgg_entry2d<double>(s, ke, sc, rl[i], rl[kOzTile + j]);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t dt = tmem_base;
  constexpr uint32_t idesc = idesc_bf16_f32(kOzTile, kOzTile);
  const __nv_bfloat16* base = Wsl + (int64_t)sub * S * NR * Kp;
  const int Kv = ((si.nb * t.BP + kOzKC - 1) / kOzKC) * kOzKC;  // rows holding data
  uint32_t phase = 0;
  for (int d = S + 1; d >= 2; --d) {
    int first = 1;
    for (int p = d - 1 < S ? d - 1 : S; p >= 1 && d - p <= S; --p) {
      const int qq = d - p;
      const __nv_bfloat16* sa = base + (int64_t)(p - 1) * NR * Kp;
      const __nv_bfloat16* sb = base + (int64_t)(qq - 1) * NR * Kp;
      for (int k0 = 0; k0 < Kv; k0 += kOzKC) {
        oz_load_tile(sa, Kp, ta * kOzTile, k0, At);
        oz_load_tile(sb, Kp, tb * kOzTile, k0, Bt);
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0 && !s_fail) {
          tc_fence_after();
#pragma unroll
          for (int ks = 0; ks < kOzKC / 16; ++ks)
            mma_bf16(dt, smem_desc(At + ks * 4096, 128, 256), smem_desc(Bt + ks * 4096, 128, 256), idesc,
                     (first && ks == 0) ? 0 : 1);
          mma_commit(&bar);
        }
        // every thread waits for the products that read the operand tiles
        if (!s_fail && !mbar_wait(&bar, phase)) s_fail = 1;
        phase ^= 1;
        first = 0;
        __syncthreads();
      }
    }
    if (s_fail) break;
    // drain C_d: row i = this thread's lane of its warp's 32 tensor-memory lanes
    tc_fence_after();
    const int i = warp * 32 + lane;
    const float rs = ldexpf(1.0f, erow[i] - bits * d);
#pragma unroll 1
    for (int c0 = 0; c0 < kOzTile; c0 += 32) {
      float v[32];
      tmem_ld32(dt + ((uint32_t)(warp * 32) << 16) + c0, v);
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int j = c0 + c;
        // 2^(e_i - B d) C exact in FP32 (a power-of-two scaling), then 2^e_j in FP64
        St[i * kOzLd + j] = fma(-(double)__fmul_rn(v[c], rs), colsc[j], St[i * kOzLd + j]);
      }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (s_fail && tid == 0) atomicExch(err, kErrTimeout);
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem_base, 128);
  // the tile and, off the diagonal, its mirror
  double* out = Sexp + (int64_t)sub * NR * NR;
  for (int v = tid; v < kOzTile * kOzTile; v += kOzThreads) {
    const int i = v / kOzTile, j = v % kOzTile;
    const int gi = ta * kOzTile + i, gj = tb * kOzTile + j;
    out[(int64_t)gi * NR + gj] = St[i * kOzLd + j];
    if (ta != tb) out[(int64_t)gj * NR + gi] = St[i * kOzLd + j];
  }
}

