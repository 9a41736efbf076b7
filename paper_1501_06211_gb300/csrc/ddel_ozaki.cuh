// Tensor-core (tcgen05) products W^T W at FP64 accuracy: the formation of
// the local Schur complements, and (opt-in) the C_k C_k^T of the 3D factor
// planes.  Included inside the anonymous namespace of ddel_kernels.cu and of
// ddel_kernels3d.cu, each of which defines the tile policy (what the product
// is subtracted from, where it goes) it instantiates the SYRK kernel with.
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
// S B >= 54 bits.  The accumulators are drained into an FP64 sum over d
// (smallest d first), scaled by 2^(e_i + e_j) and subtracted from K_GG once.
//
// Both precisions slice to 54 bits: the FP32 form rounds the FP64-accurate
// S_i once to FP32.
//
// ozaki_slice_kernel: per subdomain and ring column, e_j and the slices, each
//   stored as ready-made 16 KB operand images (below).
// ozaki_syrk_kernel: one CTA of 256 threads per (subdomain, 128 x 128 tile of
//   the product, upper triangle of tiles); one thread streams operand images
//   into shared memory by bulk copies and issues the MMAs, all eight warps
//   drain the accumulator into the FP64 tile they keep in registers.


constexpr int kOzThreads = 256;
constexpr int kOzKC = 64;      // rows of W per operand chunk
constexpr int kOzTile = 128;   // output tile edge (MMA M = N)

__device__ __host__ __forceinline__ int oz_bits(int K) { return K <= 1489 ? 6 : 5; }
// Slices for a target of `target` significant bits.
__device__ __host__ __forceinline__ int oz_slices(int bits, int target) { return (target + bits - 1) / bits; }

// Byte offset of element (c, k) (c < 128 ring columns of a row tile, k < 64
// rows of a chunk) in a 16 KB operand image: the canonical K-major layout
// without swizzling -- K slab k / 16 at 4096 B, in it the 8 x 8 core matrix
// of column group c / 8 and row half (k % 16) / 8 at 256 B and 128 B steps,
// 16 bytes per core-matrix row.  The slices are stored as these images, so a
// chunk reaches shared memory by one bulk copy.
__device__ __forceinline__ int oz_img_off(int c, int k) {
  return (k >> 4) * 4096 + (c >> 3) * 256 + ((k >> 3) & 1) * 128 + (c & 7) * 16 + (k & 7) * 2;
}

// Where a subdomain's matrix W (K rows of ncols columns, row stride ld) lies.
//  plane < 0: W = L^-1 K_IG of the 2D formation, sub_stride elements per
//    subdomain, K = nb BP rows of NR columns (ld = ncols = NR);
//  plane >= 0: the block C_plane of a subdomain's factor (at factor_off +
//    off, column-major BP x BP, i.e. W(m, i) = C(i, m): K = BP rows of BP
//    columns), for the product C C^T; K = 0 (nothing) unless 1 <= plane < nb.
struct OzSlab {
  int64_t sub_stride;
  int64_t off;
  int ld;
  int plane;
  int ncols;
};

// Slices of W for every subdomain.  Wsl: per subdomain, slice p, row tile rt
// (NR / 128) and chunk kc (Kp / 64) one 16 KB image (oz_img_off); expo: per
// subdomain NR ints.  Block (subdomain, 32 columns) of 256 threads: the
// column maxima, then per thread one column and 8 consecutive rows, written as
// one 16-byte unit per slice.  Columns from ncols to NR and rows from K to Kp
// are zero.
template <typename TW, int B, int S>
__global__ void __launch_bounds__(256) ozaki_slice_kernel(DevTables t, const TW* __restrict__ W, OzSlab src, int NR,
                                                          int Kp, __nv_bfloat16* __restrict__ Wsl,
                                                          int* __restrict__ expo) {
  static_assert(B * S >= 54 && B * S <= 55 && 30 % B == 0, "slice shape");
  constexpr int NLO = 30 / B, HALF = 1 << (B - 1), MASK = (1 << B) - 1;
  const int sub = blockIdx.x, j0 = blockIdx.y * 32, tid = threadIdx.x;
  const int jl = tid & 31, ko = tid >> 5;  // column in the block, row offset
  const SubInfo si = t.subs[sub];
  const int K = src.plane < 0 ? si.nb * t.BP : (src.plane >= 1 && src.plane < si.nb ? t.BP : 0);
  const int ld = src.ld, jv = j0 + jl < src.ncols;  // this column holds data
  const TW* Wb = W + (src.plane < 0 ? (int64_t)sub * src.sub_stride : si.factor_off) + src.off;
  __shared__ double mx_s[8][32];
  __shared__ int e_s[32];
  double mx = 0.0;
  if (jv)
    for (int k = ko; k < K; k += 8) mx = fmax(mx, fabs((double)Wb[(int64_t)k * ld + j0 + jl]));
  mx_s[ko][jl] = mx;
  __syncthreads();
  if (tid < 32) {
    double m = 0.0;
    for (int q = 0; q < 8; ++q) m = fmax(m, mx_s[q][tid]);
    int e = 0;
    if (m > 0.0) frexp(m, &e);  // m = f 2^e, 0.5 <= f < 1: |W_kj| 2^-e < 1
    e_s[tid] = e;
    expo[(int64_t)sub * NR + j0 + tid] = e;
  }
  __syncthreads();
  const int e = e_s[jl];
  const int j = j0 + jl, rt = j >> 7, c = j & 127;
  const int NRT = NR / 128, NKC = Kp / 64;
  unsigned char* img0 = reinterpret_cast<unsigned char*>(Wsl) + (int64_t)sub * S * NRT * NKC * 16384;
  for (int k8 = ko * 8; k8 < Kp; k8 += 64) {
    // m = W 2^(B S - e) rounded to an integer (|m| < 2^(B S), B S <= 55 bits);
    // its balanced base-2^B digits are the slices, m = sum_p d_p 2^(B (S-1-p)):
    // every digit but the top one in [-2^(B-1), 2^(B-1)), the top one
    // |d_0| <= 2^B, all exact in BF16.  They are taken least significant
    // first in 32-bit integers: the low 30 bits (NLO digits), then the high
    // part plus the carry.
    __align__(16) __nv_bfloat16 h[S][8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const long long m =
          jv && k8 + r < K ? __double2ll_rn(ldexp((double)Wb[(int64_t)(k8 + r) * ld + j], B * S - e)) : 0ll;
      int lo = (int)(m & ((1ll << 30) - 1)), y = (int)(m >> 30);  // m = y 2^30 + lo, 0 <= lo < 2^30
#pragma unroll
      for (int q = 0; q < NLO; ++q) {
        const int d = ((lo + HALF) & MASK) - HALF;
        lo = (lo - d) >> B;  // exact: lo - d is a non-negative multiple of 2^B
        h[S - 1 - q][r] = __float2bfloat16_rn((float)d);
      }
      y += lo;  // the carry out of the low part, 0 or 1
#pragma unroll
      for (int p = S - 1 - NLO; p > 0; --p) {
        const int d = ((y + HALF) & MASK) - HALF;
        y = (y - d) >> B;  // exact: a multiple of 2^B
        h[p][r] = __float2bfloat16_rn((float)d);
      }
      h[0][r] = __float2bfloat16_rn((float)y);
    }
    const int kc = k8 >> 6;
    const int off = oz_img_off(c, k8 & 63);
#pragma unroll
    for (int p = 0; p < S; ++p) {
      unsigned char* img = img0 + ((int64_t)(p * NRT + rt) * NKC + kc) * 16384;
      *reinterpret_cast<uint4*>(img + off) = *reinterpret_cast<const uint4*>(h[p]);
    }
  }
}

// Slices of a matrix for the tensor-core products (the digit width B and count
// S follow from the rows Kp: B = 6, S = 9 up to 1489 rows, else B = 5, S = 11).
template <typename TW>
void launch_ozaki_slice(dim3 grid, cudaStream_t st, const DevTables& t, const TW* W, const OzSlab& src, int NR, int Kp,
                        __nv_bfloat16* Wsl, int* expo) {
  if (oz_bits(Kp) == 6)
    ozaki_slice_kernel<TW, 6, 9><<<grid, 256, 0, st>>>(t, W, src, NR, Kp, Wsl, expo);
  else
    ozaki_slice_kernel<TW, 5, 11><<<grid, 256, 0, st>>>(t, W, src, NR, Kp, Wsl, expo);
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

// Tile (ta, tb) of one subdomain: the tile's own entries (K_GG for S_i) minus 2^(e_i + e_j) sum_d
// 2^(-B d) C_d, C_d = sum_{p + q = d} D_p^T D_q accumulated in tensor memory,
// d from S + 1 down to 2 (small terms first), the sum over d in FP64.  256 threads: thread (w, l)
// keeps row 32 (w % 4) + l, columns 64 (w / 4) .. + 63 of the FP64 tile in
// registers (warp w reads tensor-memory lanes 32 (w % 4) ..).  Thread 0
// drives a pipeline of kOzStages stages: per step (pair, chunk) one bulk copy
// of the A and one of the B image (16 KB each) completing on the stage's
// full barrier, four 128 x 128 x 16 MMAs committed to the stage's empty
// barrier, after which the stage is refilled with the step kOzStages ahead
// (the sequence runs on across groups, so the loads of the next group overlap
// the drain of this one).  Every wait is bounded; on a timeout the kernel
// records kErrTimeout in err, stops issuing work, still frees its tensor
// memory and returns.
constexpr int kOzStages = 6;

// Tile: what the product is subtracted from and where the result goes --
//   int rows(t, si): rows of W holding data (0: the CTA has nothing to do);
//   void setup(t, si, ta, tb, sm): stage what value() reads (all threads);
//   double value(t, si, sm, gi, gj, li, lj): the entry the product is taken
//     from (global indices gi, gj; li, lj within the tiles ta, tb);
//   void store(t, si, sub, gi, gj, v): write the result entry;
//   static size_t smem(t) on the host: bytes of sm.
template <int NR, class Tile>
__global__ void __launch_bounds__(kOzThreads, 1) ozaki_syrk_kernel(DevTables t, Tile tile,
                                                                   const __nv_bfloat16* __restrict__ Wsl,
                                                                   const int* __restrict__ expo, int Kp, int S,
                                                                   int* err) {
  constexpr int NT = NR / kOzTile, NST = kOzStages;
  const int sub = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int ta = 0, q = blockIdx.y;  // tile index -> (ta, tb), ta <= tb
  while (q >= NT - ta) {
    q -= NT - ta;
    ++ta;
  }
  const int tb = ta + q;
  const SubInfo si = t.subs[sub];
  const int K = tile.rows(t, si);
  if (K <= 0) return;  // uniform over the CTA, before any barrier or tensor memory
  const int bits = oz_bits(Kp);
  extern __shared__ __align__(1024) unsigned char oz_smem[];
  unsigned char* stage = oz_smem;                                // NST x (A 16 KB, B 16 KB)
  int* ex = reinterpret_cast<int*>(oz_smem + NST * 32768);      // 256: exponents of ta, tb
  unsigned char* tsm = oz_smem + NST * 32768 + 2 * kOzTile * 4;  // the tile's own data
  __shared__ __align__(8) uint64_t full[NST], empty[NST];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  tile.setup(t, si, ta, tb, tsm);
  for (int j = tid; j < 2 * kOzTile; j += kOzThreads) {
    const int jr = (j < kOzTile ? ta : tb) * kOzTile + j % kOzTile;
    ex[j] = expo[(int64_t)sub * NR + jr];
  }
  if (tid == 0) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    fence_mbar_init();
    s_fail = 0;
  }
  if (warp == 0) tmem_alloc(&tmem_base, 128);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // this thread's part of the tile: row i, columns jc .. jc + 63.  acc sums
  // T = sum_d 2^(-B d) C_d in FP64 (each term exact: an integer-valued FP32
  // sum times a power of two); the tile's own entries and the column scales
  // 2^(e_i + e_j) join once, at the end
  const int i = 32 * (warp & 3) + lane, jc = 64 * (warp >> 2);
  double acc[64];
#pragma unroll
  for (int c = 0; c < 64; ++c) acc[c] = 0.0;
  const uint32_t dt = tmem_base;
  constexpr uint32_t idesc = idesc_bf16_f32(kOzTile, kOzTile);
  const int NRT = NR / 128, NKC = Kp / 64;
  const int nkc = (K + 63) / 64;  // chunks holding data
  const unsigned char* img0 = reinterpret_cast<const unsigned char*>(Wsl) + (int64_t)sub * S * NRT * NKC * 16384;
  auto img = [&](int p, int rt, int kc) { return img0 + ((int64_t)((p - 1) * NRT + rt) * NKC + kc) * 16384; };
  // step sequence: d from S + 1 down to 2; p from min(d - 1, S) down to
  // max(1, d - S) (q = d - p); chunks kc < nkc
  auto p_hi = [&](int d) { return d - 1 < S ? d - 1 : S; };
  auto p_lo = [&](int d) { return d - S > 1 ? d - S : 1; };
  int ld_d = S + 1, ld_p = p_hi(S + 1), ld_kc = 0, ld_n = 0;  // thread 0: the next step to load
  auto produce = [&]() {
    if (ld_d < 2 || s_fail) return;
    const int st = ld_n % NST;
    if (ld_n >= NST && !mbar_wait(&empty[st], ((ld_n / NST) - 1) & 1)) {
      s_fail = 1;
      return;
    }
    mbar_expect_tx(&full[st], 32768);
    bulk_load(stage + st * 32768, img(ld_p, ta, ld_kc), 16384, &full[st]);
    bulk_load(stage + st * 32768 + 16384, img(ld_d - ld_p, tb, ld_kc), 16384, &full[st]);
    ++ld_n;
    if (++ld_kc == nkc) {
      ld_kc = 0;
      if (--ld_p < p_lo(ld_d)) {
        --ld_d;
        ld_p = p_hi(ld_d);
      }
    }
  };
  if (tid == 0)
    for (int k = 0; k < NST; ++k) produce();
  int n = 0;  // steps issued so far (the same count in every thread)
  for (int d = S + 1; d >= 2; --d) {
    const int steps = (p_hi(d) - p_lo(d) + 1) * nkc;
    if (tid == 0) {
      for (int k = 0; k < steps; ++k) {
        const int st = (n + k) % NST;
        if (s_fail || !mbar_wait(&full[st], ((n + k) / NST) & 1)) {
          s_fail = 1;
          break;
        }
        tc_fence_after();
        const unsigned char* A = stage + st * 32768;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
          mma_bf16(dt, smem_desc(A + ks * 4096, 128, 256), smem_desc(A + 16384 + ks * 4096, 128, 256), idesc,
                   (k == 0 && ks == 0) ? 0 : 1);
        mma_commit(&empty[st]);
        produce();
      }
    }
    n += steps;
    __syncthreads();
    // the group's last products complete (its commit: step n - 1)
    if (!s_fail && !mbar_wait(&empty[(n - 1) % NST], ((n - 1) / NST) & 1)) s_fail = 1;
    __syncthreads();
    if (s_fail) break;
    tc_fence_after();
    const double rsd = ldexp(1.0, -bits * d);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float v[32];
      tmem_ld32(dt + ((uint32_t)(32 * (warp & 3)) << 16) + jc + 32 * h, v);
#pragma unroll
      for (int c = 0; c < 32; ++c) acc[32 * h + c] = fma((double)v[c], rsd, acc[32 * h + c]);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (s_fail && tid == 0) atomicExch(err, kErrTimeout);
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem_base, 128);
  const int gi = ta * kOzTile + i;
#pragma unroll
  for (int c = 0; c < 64; ++c) {
    const int gj = tb * kOzTile + jc + c;
    // the tile's entry minus 2^(e_i + e_j) T (an exact power-of-two scaling)
    const double v = tile.value(t, si, tsm, gi, gj, i, jc + c) - ldexp(acc[c], ex[i] + ex[kOzTile + jc + c]);
    tile.store(t, si, sub, gi, gj, v);
    if (ta != tb) tile.store(t, si, sub, gj, gi, v);
  }
}
