// Limb -> RNS lift (Sec. 5 "Limb-to-RNS Conversion"): for each coefficient
// A (L little-endian 32-bit limbs) and each prime q_i,
//     a_i = A mod q_i = sum_l limb_l (2^(32 l) mod q_i)  (mod q_i),
// by limb-wise accumulation with the precomputed constants 2^(32 l) mod q_i
// (Sec. 5 "Precomputed RNS Conversion Constants") and one final reduction.
//
// One thread owns one coefficient: its limbs sit in registers (read once,
// coalesced across the warp), and it loops over all primes, writing one
// coalesced residue row per prime.  The constant table of the CTA's primes is
// staged in shared memory and read as warp-wide broadcasts.
#include "common.cuh"

namespace fhe {

constexpr int kLiftThreads = 128;

// (hi:lo) 96-bit accumulator -> value mod q.  a2 < 2^8.
__device__ __forceinline__ uint32_t reduce96(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t q, uint32_t r32,
                                             uint32_t r32s, uint32_t r64) {
  // v = a2 2^64 + a1 2^32 + a0 == a2 r64 + a1 r32 + a0 (mod q), < 2^64
  uint64_t v = (uint64_t)a2 * r64 + (uint64_t)a1 * r32 + a0;
  uint32_t vh = (uint32_t)(v >> 32), vl = (uint32_t)v;
  uint32_t t = shoup_mul(vh, r32, r32s, q);  // vh 2^32 mod q
  if (vl >= 2 * q) vl -= 2 * q;
  if (vl >= q) vl -= q;
  return add_mod(t, vl, q);
}

template <int LB>
__global__ void __launch_bounds__(kLiftThreads) k_lift(const uint32_t* __restrict__ src, int L, size_t src_pstride,
                                                       size_t src_bstride, uint32_t* __restrict__ dst,
                                                       size_t dst_pstride, size_t dst_bstride, int npoly, int r,
                                                       int N, const uint32_t* __restrict__ pow2,
                                                       const uint32_t* __restrict__ qtab,
                                                       const uint32_t* __restrict__ red) {
  extern __shared__ uint32_t sc[];  // [r][Lp], Lp = L rounded up to 4, zero padded
  const int Lp = (L + 3) & ~3;
  for (int idx = threadIdx.x; idx < r * Lp; idx += blockDim.x) {
    const int i = idx / Lp, l = idx % Lp;
    sc[idx] = l < L ? pow2[(size_t)i * kMaxLiftLimbs + l] : 0u;
  }
  __syncthreads();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int poly = blockIdx.y % npoly, b = blockIdx.y / npoly;
  const uint32_t* s = src + (size_t)b * src_bstride + (size_t)poly * src_pstride + n;
  uint32_t x[LB];
#pragma unroll
  for (int l = 0; l < LB; ++l) x[l] = (l < L) ? __ldg(s + (size_t)l * N) : 0u;
  uint32_t* d = dst + (size_t)b * dst_bstride + (size_t)poly * dst_pstride + n;
  for (int i = 0; i < r; ++i) {
    const uint4* c4 = reinterpret_cast<const uint4*>(sc + i * Lp);
    uint64_t acc = 0;
    uint32_t a2 = 0;
#pragma unroll
    for (int l4 = 0; l4 < LB / 4; ++l4) {
      if (4 * l4 < L) {
        // 128-bit broadcast of four constants; two products < 2^63 sum below 2^64
        const uint4 c = c4[l4];
        uint64_t p = (uint64_t)x[4 * l4] * c.x + (uint64_t)x[4 * l4 + 1] * c.y;
        acc += p;
        a2 += (acc < p);
        p = (uint64_t)x[4 * l4 + 2] * c.z + (uint64_t)x[4 * l4 + 3] * c.w;
        acc += p;
        a2 += (acc < p);
      }
    }
    const uint32_t q = __ldg(qtab + i);
    d[(size_t)i * N] = reduce96((uint32_t)acc, (uint32_t)(acc >> 32), a2, q, __ldg(red + 4 * i),
                                __ldg(red + 4 * i + 1), __ldg(red + 4 * i + 2));
  }
}


// Digit lift for operands of up to 48 limbs: the coefficient is re-read as
// 24-bit digits z_m (A = sum_m z_m 2^(24 m)), so every product z_m (2^(24 m)
// mod q_i) is below 2^55 and up to 256 of them add up in one 64-bit register
// without any overflow handling: one 32x32->64 multiply-add per digit.
template <int LB>
__global__ void __launch_bounds__(kLiftThreads) k_lift_digits(const uint32_t* __restrict__ src, int L,
                                                              size_t src_pstride, size_t src_bstride,
                                                              uint32_t* __restrict__ dst, size_t dst_pstride,
                                                              size_t dst_bstride, int npoly, int r, int N,
                                                              const uint32_t* __restrict__ pow24,
                                                              const uint32_t* __restrict__ qtab,
                                                              const uint32_t* __restrict__ red) {
  constexpr int MD = (32 * LB + 23) / 24;  // digits covering LB limbs
  constexpr int MP = (MD + 3) & ~3;        // padded to 128-bit loads
  static_assert(MP <= kLiftDigits, "digit table too short");
  extern __shared__ uint32_t sc[];  // [r][MP]
  for (int idx = threadIdx.x; idx < r * MP; idx += blockDim.x) {
    const int i = idx / MP, m = idx % MP;
    sc[idx] = m < MD ? pow24[(size_t)i * kLiftDigits + m] : 0u;
  }
  __syncthreads();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int poly = blockIdx.y % npoly, b = blockIdx.y / npoly;
  const uint32_t* s = src + (size_t)b * src_bstride + (size_t)poly * src_pstride + n;
  uint32_t x[LB + 1];
#pragma unroll
  for (int l = 0; l < LB; ++l) x[l] = (l < L) ? __ldg(s + (size_t)l * N) : 0u;
  x[LB] = 0;
  uint32_t z[MP];
#pragma unroll
  for (int m = 0; m < MP; ++m) {
    const int o = 24 * m, l = o >> 5, sh = o & 31;
    z[m] = (m < MD && l < LB) ? (__funnelshift_r(x[l], x[l + 1], sh) & 0xFFFFFFu) : 0u;
  }
  uint32_t* d = dst + (size_t)b * dst_bstride + (size_t)poly * dst_pstride + n;
  const int md_live = (32 * L + 23) / 24;  // digits of the live limbs
  for (int i = 0; i < r; ++i) {
    const uint4* c4 = reinterpret_cast<const uint4*>(sc + i * MP);
    uint64_t acc = 0;
#pragma unroll
    for (int m4 = 0; m4 < MP / 4; ++m4) {
      if (4 * m4 < md_live) {
        const uint4 c = c4[m4];
        acc += (uint64_t)z[4 * m4] * c.x;
        acc += (uint64_t)z[4 * m4 + 1] * c.y;
        acc += (uint64_t)z[4 * m4 + 2] * c.z;
        acc += (uint64_t)z[4 * m4 + 3] * c.w;
      }
    }
    const uint32_t q = __ldg(qtab + i);
    d[(size_t)i * N] = reduce96((uint32_t)acc, (uint32_t)(acc >> 32), 0u, q, __ldg(red + 4 * i),
                                __ldg(red + 4 * i + 1), __ldg(red + 4 * i + 2));
  }
}

// Small signed coefficients (secret, ephemeral, error polynomials).
template <typename T>
__global__ void k_lift_small(const T* __restrict__ src, size_t src_bstride, uint32_t* __restrict__ dst,
                             size_t dst_bstride, int r, int N, const uint32_t* __restrict__ qtab) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int b = blockIdx.y;
  const int32_t v = (int32_t)src[(size_t)b * src_bstride + n];
  const uint32_t av = v < 0 ? (uint32_t)(-(int64_t)v) : (uint32_t)v;  // < 2^31 < 2q
  for (int i = 0; i < r; ++i) {
    const uint32_t q = __ldg(qtab + i);
    uint32_t m = av >= q ? av - q : av;
    if (v < 0 && m != 0) m = q - m;
    dst[(size_t)b * dst_bstride + (size_t)i * N + n] = m;
  }
}

template <int LB>
static void lift_launch(const fhe_ctx* ctx, const uint32_t* src, int L, size_t sp, size_t sb, uint32_t* dst,
                        size_t dp, size_t db, int npoly, int nbatch, int r, cudaStream_t st) {
  const int N = ctx->N;
  const int threads = N < kLiftThreads ? N : kLiftThreads;
  dim3 grid((N + threads - 1) / threads, npoly * nbatch);
  if constexpr (LB <= 48) {
    constexpr int MP = (((32 * LB + 23) / 24) + 3) & ~3;
    const size_t smem = (size_t)r * MP * sizeof(uint32_t);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_lift_digits<LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_lift_digits<LB><<<grid, threads, smem, st>>>(src, L, sp, sb, dst, dp, db, npoly, r, N, ctx->d_pow24, ctx->d_q,
                                                    ctx->d_red);
    return;
  }
  size_t smem = (size_t)r * ((L + 3) & ~3) * sizeof(uint32_t);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_lift<LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_lift<LB><<<grid, threads, smem, st>>>(src, L, sp, sb, dst, dp, db, npoly, r, N, ctx->d_pow2, ctx->d_q,
                                           ctx->d_red);
}

int launch_lift(const fhe_ctx* ctx, const uint32_t* src, int L, size_t src_pstride, size_t src_bstride,
                uint32_t* dst, size_t dst_pstride, size_t dst_bstride, int npoly, int nbatch, int r,
                cudaStream_t st) {
  if (L < 1 || L > kMaxLiftLimbs || r < 1 || r > ctx->R || nbatch < 1 || npoly < 1 ||
      (size_t)npoly * nbatch > 65535u) {
    set_error("lift: bad sizes L=%d r=%d", L, r);
    return FHE_EINVAL;
  }
  if ((size_t)r * ((L + 3) & ~3) * 4 > 200 * 1024) {
    set_error("lift: constant table of %d x %d words exceeds 200 KB", r, L);
    return FHE_EINVAL;
  }
  ProfScope ps(ctx, FHE_K_LIFT, 1, st);
#define FHE_LIFT_CASE(B)                                                                 \
  if (L <= B) {                                                                          \
    lift_launch<B>(ctx, src, L, src_pstride, src_bstride, dst, dst_pstride, dst_bstride, \
                   npoly, nbatch, r, st);                                                \
    return FHE_OK;                                                                       \
  }
  FHE_LIFT_CASE(4)
  FHE_LIFT_CASE(8)
  FHE_LIFT_CASE(16)
  FHE_LIFT_CASE(24)
  FHE_LIFT_CASE(32)
  FHE_LIFT_CASE(40)
  FHE_LIFT_CASE(48)
  FHE_LIFT_CASE(64)
  FHE_LIFT_CASE(80)
  FHE_LIFT_CASE(104)
  FHE_LIFT_CASE(128)
#undef FHE_LIFT_CASE
  return FHE_EINVAL;
}

int launch_lift_small(const fhe_ctx* ctx, const void* src, bool is_i8, size_t src_bstride, uint32_t* dst,
                      size_t dst_bstride, int nbatch, int r, cudaStream_t st) {
  const int N = ctx->N;
  const int threads = N < 256 ? N : 256;
  dim3 grid((N + threads - 1) / threads, nbatch);
  ProfScope ps(ctx, FHE_K_LIFT, 1, st);
  if (is_i8)
    k_lift_small<int8_t><<<grid, threads, 0, st>>>((const int8_t*)src, src_bstride, dst, dst_bstride, r, N,
                                                   ctx->d_q);
  else
    k_lift_small<int32_t><<<grid, threads, 0, st>>>((const int32_t*)src, src_bstride, dst, dst_bstride, r, N,
                                                    ctx->d_q);
  return FHE_OK;
}

}  // namespace fhe
