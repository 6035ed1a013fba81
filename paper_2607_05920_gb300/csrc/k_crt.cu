// RNS -> limb reconstruction (Sec. 5 "RNS-to-Limb Reconstruction", "Signed
// Representation Handling") with a fused epilogue (relinearisation rounding,
// rescale, additions, centring), in four forms that give identical results:
//  - k_crt_tc (the default, FHE_CRT_DIRECT / _CVT): the exact direct CRT with
//    a rounded quotient, its dense sum a byte-digit f16 GEMM on the tcgen05
//    tensor cores (persistent, warp-specialised; third section below);
//  - k_crt_direct (FHE_CRT_DIRECT_INT): the same CRT with the dense sum on the
//    integer pipe (second section);
//  - k_garner (FHE_CRT_GARNER): Garner's mixed-radix conversion in the nested
//    order of Sec. 2 Eq. garner_mrc (this section), described below.
//
// Garner, per coefficient (one thread each):
//  1. digits  v_k = | ((x_k - v_0) c_{0,k} - v_1) c_{1,k} - ... ) c_{k-1,k} |_{q_k},
//     c_{j,k} = [q_j^-1]_{q_k}, in the nested order of Eq. garner_mrc, with
//     Shoup multiplications by the precomputed constants; digits are kept in
//     the thread's shared-memory column.
//  2. X = v_0 + q_0 (v_1 + q_1 (v_2 + ...)) evaluated by Horner from the top
//     digit, modulo 2^(32 LB) only (LB register limbs).  The value after the
//     digits k..r-1 is below 2^(31 (r-k)), so only that many limbs are touched.
//  3. sign: the prime count leaves the top prime spare (prod_{i<r-1} q_i
//     exceeds the bound), so the top digit is 0 for a non-negative result and
//     q_{r-1} - 1 for a negative one; negative results get M = prod q_i
//     subtracted (mod 2^(32 LB)), giving the two's complement of the signed
//     exact product.
//  4. epilogue on the thread's limb column (see Epi in common.cuh).
#include <type_traits>

#include <cuda.h>  // CUtensorMap (the encoder is reached through the runtime)

#include "common.cuh"

namespace fhe {
__device__ unsigned int g_fhe_dev_status = 0;  // set when a bounded device wait gives up
}
#define FHE_TC_STATUS fhe::g_fhe_dev_status
#include "tc.cuh"

namespace fhe {

constexpr int kCrtThreads = 128;

#define COL(l) sv[(size_t)(l) * cstride + tid]

// out_bits-bit mask for limb l
__device__ __forceinline__ uint32_t limb_mask(int l, int bits) {
  const int rem = bits - 32 * l;
  if (rem >= 32) return 0xFFFFFFFFu;
  if (rem <= 0) return 0u;
  return (1u << rem) - 1u;
}

// column += 2^pos (mod 2^(32 nl))
__device__ __forceinline__ void col_add_pow2(uint32_t* sv, int tid, int cstride, int nl, int pos) {
  int l = pos >> 5;
  uint32_t add = 1u << (pos & 31);
  for (; l < nl && add; ++l) {
    uint32_t v = COL(l) + add;
    add = (v < add) ? 1u : 0u;
    COL(l) = v;
  }
}

// column[l] <- (column >> sh)[l] for l < nl_out, reading limbs < nl_in (zero above)
__device__ __forceinline__ void col_shift_right(uint32_t* sv, int tid, int cstride, int nl_in, int nl_out, int sh) {
  const int sl = sh >> 5, sb = sh & 31;
  for (int l = 0; l < nl_out; ++l) {
    const int a = l + sl;
    uint32_t lo = a < nl_in ? COL(a) : 0u;
    uint32_t hi = (a + 1) < nl_in ? COL(a + 1) : 0u;
    COL(l) = sb ? __funnelshift_r(lo, hi, sb) : lo;
  }
}

// Epilogue on the thread's limb column, which holds X mod 2^(32 LB) in rows
// [0, LB): relinearisation rounding / rescale / additions / centring per
// EpiArgs, then the store of epi.out_limbs limbs.  add_s, when given, holds
// the addend limbs already staged in shared memory (limb l at l * add_sstride).
__device__ __noinline__ void crt_epilogue(uint32_t* __restrict__ sv, int tid, int cstride, int LB, const EpiArgs& epi,
                                          int poly, int b, int n, int N, uint32_t* __restrict__ out,
                                          size_t out_pstride, size_t out_bstride,
                                          const uint32_t* add_s = nullptr, int add_sstride = 0) {

  const int ob = epi.item_bits ? __ldg(epi.item_bits + b) : epi.out_bits;
  int nl = LB;  // live limbs in the column
  if (epi.kind == Epi::kRelin) {
    if (epi.shift > 0) col_add_pow2(sv, tid, cstride, LB, epi.shift - 1);
    const int nz = (ob + 31) >> 5;
    col_shift_right(sv, tid, cstride, LB, nz, epi.shift);
    nl = nz;
  } else if (epi.kind == Epi::kAddSmall && epi.negate) {
    uint32_t c = 1;
    for (int l = 0; l < LB; ++l) {  // -X = ~X + 1
      const uint32_t v = ~COL(l) + c;
      c = (c && v == 0) ? 1u : 0u;
      COL(l) = v;
    }
  }
  const int nlo = (ob + 31) >> 5;  // limbs of the mod-2^ob value
  if (epi.add && poly < epi.add_polys) {
    const uint32_t* ad = epi.add + (size_t)b * epi.add_bstride + (size_t)poly * epi.add_pstride + n;
    uint32_t c = 0;
    for (int l = 0; l < nlo; ++l) {
      const uint32_t a = l < epi.add_limbs ? (add_s ? add_s[(size_t)l * add_sstride] : __ldg(ad + (size_t)l * N)) : 0u;
      const uint32_t x = l < nl ? COL(l) : 0u;
      const uint64_t s = (uint64_t)x + a + c;
      COL(l) = (uint32_t)s;
      c = (uint32_t)(s >> 32);
    }
    nl = nlo;
  }
  const int32_t* sm = poly == 0 ? epi.small : (poly == 1 ? epi.small1 : nullptr);
  if (sm) {
    const int32_t e = __ldg(sm + (size_t)b * epi.small_bstride + n);
    const uint32_t ext = e < 0 ? 0xFFFFFFFFu : 0u;
    uint32_t c = 0;
    for (int l = 0; l < nlo; ++l) {
      const uint32_t a = l == 0 ? (uint32_t)e : ext;
      const uint32_t x = l < nl ? COL(l) : 0u;
      const uint64_t s = (uint64_t)x + a + c;
      COL(l) = (uint32_t)s;
      c = (uint32_t)(s >> 32);
    }
    nl = nlo;
  }
  for (int l = 0; l < nlo; ++l) COL(l) = (l < nl ? COL(l) : 0u) & limb_mask(l, ob);
  nl = nlo;

  int fb = ob;  // bits of the final modulus
  if (epi.kind == Epi::kRelin && epi.k2 > 0) {
    col_add_pow2(sv, tid, cstride, nl, epi.k2 - 1);
    fb = ob - epi.k2;
    const int nf = (fb + 31) >> 5;
    col_shift_right(sv, tid, cstride, nl, nf, epi.k2);
    for (int l = 0; l < nf; ++l) COL(l) &= limb_mask(l, fb);
    nl = nf;
  }
  uint32_t ext = 0;
  if (epi.kind == Epi::kDecrypt) {
    // centred (Sec. 5): x > Q/2 -> x - Q, i.e. top bit set and any lower bit set
    const int tb = fb - 1;
    const bool top = (COL(tb >> 5) >> (tb & 31)) & 1u;
    bool low = false;
    for (int l = 0; l <= (tb >> 5) && !low; ++l) {
      uint32_t v = COL(l);
      if (l == (tb >> 5)) v &= (1u << (tb & 31)) - 1u;
      low = v != 0;
    }
    if (top && low) ext = 0xFFFFFFFFu;
  }
  uint32_t* dst = out + (size_t)b * out_bstride + (size_t)poly * out_pstride + n;
  for (int l = 0; l < epi.out_limbs; ++l) {
    uint32_t v = l < nl ? COL(l) : 0u;
    if (ext) v |= ~limb_mask(l, fb);
    dst[(size_t)l * N] = v;
  }
}


template <int LB>
__global__ void __launch_bounds__(kCrtThreads) k_garner(const uint32_t* __restrict__ in, size_t in_pstride,
                                                        size_t in_bstride, int r, int npoly,
                                                        uint32_t* __restrict__ out, size_t out_pstride,
                                                        size_t out_bstride, EpiArgs epi, int N,
                                                        const uint32_t* __restrict__ qtab,
                                                        const uint2* __restrict__ gtab, int R,
                                                        const uint32_t* __restrict__ mprod,
                                                        const uint32_t* __restrict__ nscale,
                                                        const uint32_t* __restrict__ nscale_sh) {
  extern __shared__ uint32_t sv[];  // [rows][kCrtThreads], one column per thread
  const int tid = threadIdx.x;
  constexpr int cstride = kCrtThreads;
  const int n = blockIdx.x * blockDim.x + tid;
  if (n >= N) return;  // columns are private: no block-wide barrier below
  const int poly = blockIdx.y % npoly, b = blockIdx.y / npoly;
  const uint32_t* src = in + (size_t)b * in_bstride + (size_t)poly * in_pstride + n;

  // 1. mixed-radix digits
  for (int k = 0; k < r; ++k) {
    const uint32_t qk = __ldg(qtab + k), twoq = 2u * qk;
    // the inverse transform's N^-1 2^32 scale, left out there
    uint32_t x = shoup_mul(__ldg(src + (size_t)k * N), __ldg(nscale + k), __ldg(nscale_sh + k), qk);
    const uint2* crow = gtab + (size_t)k * R;
    int j = 0;
    for (; j + 4 <= k; j += 4) {
      const uint2 c0 = __ldg(crow + j), c1 = __ldg(crow + j + 1), c2 = __ldg(crow + j + 2), c3 = __ldg(crow + j + 3);
      uint32_t d;
      d = x - COL(j);     if ((int32_t)d < 0) d += twoq; x = shoup_mul(d, c0.x, c0.y, qk);
      d = x - COL(j + 1); if ((int32_t)d < 0) d += twoq; x = shoup_mul(d, c1.x, c1.y, qk);
      d = x - COL(j + 2); if ((int32_t)d < 0) d += twoq; x = shoup_mul(d, c2.x, c2.y, qk);
      d = x - COL(j + 3); if ((int32_t)d < 0) d += twoq; x = shoup_mul(d, c3.x, c3.y, qk);
    }
    for (; j < k; ++j) {
      const uint2 c = __ldg(crow + j);
      uint32_t d = x - COL(j);
      if ((int32_t)d < 0) d += twoq;  // x - v_j + 2 q_k in (0, 2^32)
      x = shoup_mul(d, c.x, c.y, qk);
    }
    COL(k) = x;
  }

  // 2. Horner from the top digit, mod 2^(32 LB)
  uint32_t X[LB];
#pragma unroll
  for (int l = 0; l < LB; ++l) X[l] = 0;
  const uint32_t vtop = COL(r - 1);
  X[0] = vtop;
  for (int k = r - 2; k >= 0; --k) {
    const uint32_t qk = __ldg(qtab + k);
    uint32_t carry = COL(k);
    const int act = (31 * (r - k) + 31) >> 5;  // limbs of the running value
#pragma unroll
    for (int c = 0; c < LB; c += 8) {
      if (c < act) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const uint64_t t = (uint64_t)X[c + u] * qk + carry;
          X[c + u] = (uint32_t)t;
          carry = (uint32_t)(t >> 32);
        }
      }
    }
  }

  // 3. sign from the spare top digit
  if (vtop > (__ldg(qtab + r - 1) >> 1)) {
    const uint32_t* M = mprod + (size_t)r * kMaxLimbs;
    uint32_t borrow = 0;
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      const uint64_t d = (uint64_t)X[l] - __ldg(M + l) - borrow;
      X[l] = (uint32_t)d;
      borrow = (uint32_t)(d >> 63);
    }
  }

  // 4. epilogue on the column
#pragma unroll
  for (int l = 0; l < LB; ++l) COL(l) = X[l];
  crt_epilogue(sv, tid, kCrtThreads, LB, epi, poly, b, n, N, out, out_pstride, out_bstride);
}


// ------------------------------------------------------------- direct CRT
// Exact CRT with a rounded quotient (the floating-point quotient of
// Halevi-Polyakov-Shoup 2019, "An improved RNS variant of the BFV scheme"):
//   y_i = [x_i (M/q_i)^-1]_{q_i},   X = sum_i y_i (M/q_i) - kappa M,
//   kappa = round(sum_i y_i / q_i).
// sum_i y_i / q_i = kappa + X/M exactly, and |X| < prod_{i<r-1} q_i = M/q_{r-1}
// (the prime count's spare prime) gives |X/M| < 2^-30; the fp32 sum has an
// absolute error below 2^-8 for r <= 256 terms, so round() returns kappa
// exactly and X comes out signed (two's complement mod 2^(32 LB)).  The
// dense part sum_i y_i (M/q_i) is a [coefficients x r] by [r x LB-limbs]
// product: one 32x32->64 multiply-add per (prime, limb), with the constant
// rows staged in shared memory and read as 128-bit broadcasts.
// Column form of the dense product: the constants are held as 24-bit digits,
// so each product y_i d (y_i < q < 2^30, d < 2^24) is below 2^54 and a whole
// column sum over r + 1 <= 257 terms fits one 64-bit register -- one
// 32x32->64 multiply-add per (prime, digit), no carry chain.  The y_i sit in
// the thread's shared-memory column; columns are taken 8 at a time (192 bits
// = 6 limbs), normalised into limbs kept in registers, the block's carry
// passed on.  kappa enters as one more term with the digits of -M.
template <int LB>
__global__ void __launch_bounds__(kCrtThreads, 3) k_crt_direct(const uint32_t* __restrict__ in, size_t in_pstride,
                                                               size_t in_bstride, int r, int npoly,
                                                               uint32_t* __restrict__ out, size_t out_pstride,
                                                               size_t out_bstride, EpiArgs epi, int N,
                                                               const uint32_t* __restrict__ qtab,
                                                               const uint2* __restrict__ cinv,
                                                               const uint32_t* __restrict__ dig,
                                                               const float* __restrict__ invq) {
  constexpr int NBLK = (LB + 5) / 6;  // 6-limb blocks of 8 digit columns
  static_assert(8 * NBLK <= kCrtDigits, "digit table too short");
  extern __shared__ uint32_t sv[];  // [rows][kCrtThreads] y_0..y_{r-1}, kappa (later the limb column),
                                    // then [2][r+1][8] digit columns of the current block
  const int tid = threadIdx.x;
  constexpr int cstride = kCrtThreads;
  const int rows = (r + 1) > (LB + 2) ? (r + 1) : (LB + 2);
  uint32_t* cbase = sv + (size_t)rows * kCrtThreads;
  const int n = blockIdx.x * blockDim.x + tid;
  const bool active = n < N;
  const int poly = blockIdx.y % npoly, b = blockIdx.y / npoly;
  // 1. y_i = [x_i (M/q_i)^-1]_{q_i} and the fp32 quotient estimate
  if (active) {
    const uint32_t* src = in + (size_t)b * in_bstride + (size_t)poly * in_pstride + n;
    float fs = 0.f;
    constexpr int PF = 8;  // residue loads kept in flight
    uint32_t xb[PF];
#pragma unroll
    for (int k = 0; k < PF; ++k) xb[k] = k < r ? __ldg(src + (size_t)k * N) : 0u;
    for (int i0 = 0; i0 < r; i0 += PF) {
#pragma unroll
      for (int k = 0; k < PF; ++k) {
        const int i = i0 + k;
        if (i < r) {
          const uint32_t x = xb[k];
          if (i + PF < r) xb[k] = __ldg(src + (size_t)(i + PF) * N);
          const uint2 ci = __ldg(cinv + i);
          const uint32_t y = shoup_mul(x, ci.x, ci.y, __ldg(qtab + i));
          fs = fmaf(__uint2float_rn(y), __ldg(invq + i), fs);
          COL(i) = y;
        }
      }
    }
    COL(r) = (uint32_t)__float2int_rn(fs);  // kappa, multiplies the -M row
  }
  // 2. column sums, 8 digit columns per block; each block's constants staged in shared memory
  uint32_t X[6 * NBLK];
  uint64_t carry = 0;
  const int terms = r + 1;
#pragma unroll
  for (int blk = 0; blk < NBLK; ++blk) {
    uint32_t* cb = cbase + (size_t)(blk & 1) * terms * 8;
    for (int idx = tid; idx < terms * 8; idx += blockDim.x)
      cb[idx] = __ldg(dig + (size_t)(idx >> 3) * kCrtDigits + 8 * blk + (idx & 7));
    __syncthreads();
    uint64_t s0 = carry, s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0, s6 = 0, s7 = 0;
#pragma unroll 4
    for (int i = 0; i < terms; ++i) {
      const uint32_t y = COL(i);
      const uint4 d0 = *reinterpret_cast<const uint4*>(cb + 8 * i);
      const uint4 d1 = *reinterpret_cast<const uint4*>(cb + 8 * i + 4);
      s0 += (uint64_t)y * d0.x;
      s1 += (uint64_t)y * d0.y;
      s2 += (uint64_t)y * d0.z;
      s3 += (uint64_t)y * d0.w;
      s4 += (uint64_t)y * d1.x;
      s5 += (uint64_t)y * d1.y;
      s6 += (uint64_t)y * d1.z;
      s7 += (uint64_t)y * d1.w;
    }
    // normalise 8 digit columns into 6 limbs; the rest carries into the next block
    uint32_t dd[8];
    s1 += s0 >> 24; dd[0] = (uint32_t)s0 & 0xFFFFFFu;
    s2 += s1 >> 24; dd[1] = (uint32_t)s1 & 0xFFFFFFu;
    s3 += s2 >> 24; dd[2] = (uint32_t)s2 & 0xFFFFFFu;
    s4 += s3 >> 24; dd[3] = (uint32_t)s3 & 0xFFFFFFu;
    s5 += s4 >> 24; dd[4] = (uint32_t)s4 & 0xFFFFFFu;
    s6 += s5 >> 24; dd[5] = (uint32_t)s5 & 0xFFFFFFu;
    s7 += s6 >> 24; dd[6] = (uint32_t)s6 & 0xFFFFFFu;
    dd[7] = (uint32_t)s7 & 0xFFFFFFu;
    carry = s7 >> 24;
    X[6 * blk + 0] = dd[0] | (dd[1] << 24);
    X[6 * blk + 1] = (dd[1] >> 8) | (dd[2] << 16);
    X[6 * blk + 2] = (dd[2] >> 16) | (dd[3] << 8);
    X[6 * blk + 3] = dd[4] | (dd[5] << 24);
    X[6 * blk + 4] = (dd[5] >> 8) | (dd[6] << 16);
    X[6 * blk + 5] = (dd[6] >> 16) | (dd[7] << 8);
  }
  if (!active) return;
  // 3. epilogue on the limb column (the y rows are dead)
#pragma unroll
  for (int l = 0; l < LB; ++l) COL(l) = X[l];
  crt_epilogue(sv, tid, kCrtThreads, LB, epi, poly, b, n, N, out, out_pstride, out_bstride);
}

// ------------------------------------------------- direct CRT, tensor cores
// The dense part of the direct CRT, sum_i y_i C_i (C_i = M/q_i, and kappa
// times C_r = -M), as an fp16 GEMM on the tcgen05 tensor cores.  y_i and C_i
// are split into balanced bytes (digits in [-128, 128]), so every product is
// an integer of magnitude <= 2^14 and a column sum over 4 (r + 1) <= 1020
// terms stays below 2^24: the fp32 accumulator is exact.  Output byte column
// p is S_p = sum_{i,a} d_{i,a} c_{i,p-a}: D[128 coefficients][P] =
// A[128][K] B[P][K]^T with K = 4 i + a, the byte digits of y_i in A and the
// Toeplitz-shifted digits c_{i,p-a} in B (host-built, build_crt_tc).
//
// A tile = 128 coefficients of one polynomial = the MMA's M = the 128 TMEM
// lanes.  The kernel is persistent (one CTA per SM walks the tiles) and warp
// specialised, every hand-off an mbarrier:
//   warps 0-7   (Y) y_i = [x_i (M/q_i)^-1]_{q_i} and kappa from the staged
//               residues (two threads per row), as f16 digits into an A stage;
//   warps 8-15  (E) two groups of four: S_p from each thread's own TMEM lane,
//               carried into 32-bit limbs, then the epilogue; the groups take
//               alternate tiles, or (one accumulator, relinearisation) both
//               drain every tile, a column half each;
//   warp 16     residues by TMA tensor loads (16 primes x 128 coefficients)
//               and an L2 prefetch of the next tile's;
//   warp 17     TMEM allocation and the MMA issue (one thread);
//   warp 18     B: streamed in K 64 stages, or loaded once when resident;
//   warp 19     the staged addend of each tile (TMA tensor load).
// With P <= 256 two accumulators alternate, so the epilogue of one tile runs
// under the GEMM of the next.  K runs in chunks of 64 (16 primes), or 128
// with B resident.  Every wait is bounded and reports a timeout through
// fhe_sync.
constexpr int kTcRows = 128;
constexpr int kTcYWarps = 8;                // two threads per coefficient row
constexpr int kTcEWarps = 8;                // two groups of four
constexpr int kTcWarpProd = kTcYWarps + kTcEWarps;  // residues
constexpr int kTcWarpMma = kTcWarpProd + 1;         // TMEM owner, MMA issue
constexpr int kTcWarpProdB = kTcWarpMma + 1;        // B slices
constexpr int kTcWarpProdAdd = kTcWarpProdB + 1;    // staged addends
constexpr int kTcThreads = 32 * (kTcWarpProdAdd + 1);
constexpr int kTcNX = 3;                    // residue stages
constexpr int kTcXStage = 16 * kTcRows * 4; // bytes: 16 primes x 128 coefficients
constexpr int kTcAStage = kTcRows * 64 * 2; // bytes: 128 rows x K 64 f16
constexpr int kTcHead = 1024;               // mbarriers + TMEM address
constexpr int kTcFsx = 4096;                // quotient partial sums [tile parity][half][row] (floats),
                                            // then epilogue carries [tile parity][row] (int64)

// Balanced bytes of y < 2^31 (y < q) as two f16x2 registers {d0, d1}, {d2, d3}:
// e = y + 0x808080, d_a = byte_a(e) - 128 for a < 3, d_3 = byte_3(e) <= 128.
// A byte b is placed under the f16 exponent of 1024 (bits 0x6400 | b = 1024 + b),
// then 1152 (or 1024) is subtracted exactly.
__device__ __forceinline__ void y_digits(uint32_t y, uint32_t& lo, uint32_t& hi) {
  const uint32_t e = y + 0x00808080u;
  const uint32_t l = __byte_perm(e, 0x64646464u, 0x5140);
  const uint32_t h = __byte_perm(e, 0x64646464u, 0x5342);
  asm("sub.rn.f16x2 %0, %1, %2;\n" : "=r"(lo) : "r"(l), "r"(0x64806480u));
  asm("sub.rn.f16x2 %0, %1, %2;\n" : "=r"(hi) : "r"(h), "r"(0x64006480u));
}

// Streaming forms of the two hot epilogues, fed limb by limb (low to high)
// straight from the carry of the column sums, so no limb column is stored.
// They compute exactly what crt_epilogue computes for these kinds:
//  kStore: X mod 2^ob;
//  kRelin: Y = ((X + 2^(s-1)) >> s) + A mod 2^ob, then, if k2 > 0,
//          (Y + 2^(k2-1)) >> k2 mod 2^(ob-k2).
// (X + 2^(s-1)) >> s = (X >> s) + bit_{s-1}(X): the rounding bit sits in a
// limb that arrives before the first shifted limb, and every later stage only
// needs the limb after the current one, so each arriving limb moves every
// stage by at most one limb.
struct RelinStream {
  // configuration
  int sl, sb, rl, rbit;  // relin shift s in limbs / bits, limb and bit of bit s-1
  int nz;                // limbs of the mod-2^ob value
  uint32_t zmask;        // mask of its top limb
  const uint32_t* add;   // addend limbs (stride add_stride), or null
  int add_limbs, add_stride;
  int k2, kl, kb, rl2, rbit2, nf;  // rescale shift, limbs of the mod-2^(ob-k2) value
  uint32_t wmask;
  int out_limbs;
  uint32_t* dst;
  int N;
  // state
  uint32_t xprev = 0, cA = 0, cB = 0, zprev = 0, cC = 0;
  int j = 0, zi = 0, i = 0;

  __device__ __forceinline__ void store(uint32_t w) {
    if (i < out_limbs) dst[(size_t)i * N] = w;
    ++i;
  }
  __device__ __forceinline__ void push_z(uint32_t z) {
    if (k2 == 0) {
      if (zi < nz) store(z);
      ++zi;
      return;
    }
    if (zi == rl2) cC = (z >> rbit2) & 1u;
    if (zi >= kl + 1 && i < nf) {
      uint32_t w = __funnelshift_r(zprev, z, kb) + cC;
      cC = (w < cC) ? 1u : 0u;
      if (i == nf - 1) w &= wmask;
      store(w);
    }
    zprev = z;
    ++zi;
  }
  __device__ __forceinline__ void push_x(int l, uint32_t x) {
    if (l == rl) cA = (x >> rbit) & 1u;
    if (l >= sl + 1 && j < nz) {
      uint32_t y = __funnelshift_r(xprev, x, sb) + cA;
      cA = (y < cA) ? 1u : 0u;
      const uint32_t a = (add && j < add_limbs) ? add[(size_t)j * add_stride] : 0u;
      const uint64_t zz = (uint64_t)y + a + cB;
      cB = (uint32_t)(zz >> 32);
      uint32_t z = (uint32_t)zz;
      if (j == nz - 1) z &= zmask;
      ++j;
      push_z(z);
    }
    xprev = x;
  }
  // after the last limb: the stages drain on zero limbs, then the store is padded
  __device__ __forceinline__ void finish(int l) {
    while (j < nz) push_x(l++, 0u);
    if (k2 > 0)
      while (i < nf) push_z(0u);
    while (i < out_limbs) store(0u);
  }
};

// Configures the relinearisation stream of one coefficient (kRelin epilogue):
// shift s = epi.shift (round at bit s - 1), result mod 2^ob plus the addend
// (staged in shared memory with row stride kTcRows when add_s is given, else
// read from global), then the rescale by epi.k2 bits.
__device__ __forceinline__ void relin_setup(RelinStream& rs, const EpiArgs& epi, int ob, bool has_add,
                                            const uint32_t* add_s, int b, int poly, int n, int N, uint32_t* dst) {
  const int sft = epi.shift;
  rs.sl = sft >> 5;
  rs.sb = sft & 31;
  rs.rl = (sft - 1) >> 5;
  rs.rbit = (sft - 1) & 31;
  const int nlo = (ob + 31) >> 5;
  rs.nz = nlo;
  rs.zmask = limb_mask(nlo - 1, ob);
  rs.add = has_add ? (add_s ? add_s : epi.add + (size_t)b * epi.add_bstride + (size_t)poly * epi.add_pstride + n)
                   : nullptr;
  rs.add_limbs = epi.add_limbs;
  rs.add_stride = add_s ? kTcRows : N;
  rs.k2 = epi.k2;
  rs.kl = epi.k2 >> 5;
  rs.kb = epi.k2 & 31;
  rs.rl2 = epi.k2 > 0 ? (epi.k2 - 1) >> 5 : 0;
  rs.rbit2 = epi.k2 > 0 ? (epi.k2 - 1) & 31 : 0;
  const int fb = ob - epi.k2;
  rs.nf = (fb + 31) >> 5;
  rs.wmask = limb_mask(rs.nf - 1, fb);
  rs.out_limbs = epi.out_limbs;
  rs.dst = dst;
  rs.N = N;
}

// The relinearisation epilogue of one coefficient in one pass over its limb column held in
// shared memory (col[l kTcRows] for l in [min(rl, sl), nx): the column sums after their
// carries, the high half still without the low half's carry), with the
// low half's carry c0 rippled in from limb lsplit up as the limbs are read (limbs at and above
// nx read as zero):
//   X' = X + c0 2^(32 lsplit) mod 2^(32 nx),
//   Z  = ((X' + 2^(s-1)) >> s) + A mod 2^ob,
//   W  = (Z + 2^(k2-1)) >> k2 mod 2^(ob-k2)   (W = Z when k2 = 0),
// stored as out_limbs limbs (zeros above W).  The rounding carry of the shift and the carry of
// the addend travel as one carry in {0, 1, 2} (f + a + c0 + c1 has the same low word as
// ((f + c0) mod 2^32) + a + c1, and the two carries out add up to its high word), so a limb of
// Z costs one funnel shift and one three-input add.  Limbs between the first output limb and
// the top one take a branch-free loop; the first limbs (rounding bits) and the top limb (masks)
// take the general step.
__device__ __forceinline__ void relin_column(const uint32_t* col, int nx, int lsplit, int c0, const EpiArgs& epi,
                                             int ob, const uint32_t* add, int add_stride, uint32_t* dst, int N) {
  const int s = epi.shift, sl = s >> 5, sb = s & 31, rl = (s - 1) >> 5, rbit = (s - 1) & 31;
  const int nz = (ob + 31) >> 5;
  const uint32_t zmask = limb_mask(nz - 1, ob);
  const int na = add ? epi.add_limbs : 0;
  const int out_limbs = epi.out_limbs;
  const int k2 = epi.k2, kl = k2 >> 5, kb = k2 & 31;
  const int rl2 = k2 > 0 ? (k2 - 1) >> 5 : -1, rbit2 = (k2 - 1) & 31;
  const int fb = ob - k2, nf = k2 > 0 ? (fb + 31) >> 5 : nz;
  const uint32_t wmask = limb_mask(nf - 1, fb);
  const int wfirst = k2 > 0 ? kl + 1 : 0;  // z limb that completes w limb 0
  // X' limbs in ascending order: every limb from lsplit up passes through `ripple` exactly once
  int rc = 0;  // carry entering the next rippled limb (c0 at limb lsplit)
  auto ripple = [&](int l, uint32_t x) -> uint32_t {
    if (l == lsplit) rc = c0;
    const long long t = (long long)x + rc;
    rc = (int)(t >> 32);
    return l < nx ? (uint32_t)t : 0u;
  };
  auto xload = [&](int l) -> uint32_t { return l < nx ? col[(size_t)l * kTcRows] : 0u; };
  for (int l = lsplit; l < rl; ++l) ripple(l, xload(l));  // limbs below the rounding limb only carry
  const uint32_t xr = ripple(rl, xload(rl));
  uint32_t c = (xr >> rbit) & 1u;  // the rounding bit, then the combined carry
  uint32_t xprev = sl == rl ? xr : ripple(sl, xload(sl));
  uint32_t zprev = 0u, cC = 0u;
  int i = 0;  // next output limb
  // the general step for z limb j: every mask, rounding bit and bound checked
  auto step = [&](int j, uint32_t x, uint32_t a) {
    const uint64_t zz = (uint64_t)__funnelshift_r(xprev, x, sb) + a + c;
    c = (uint32_t)(zz >> 32);
    uint32_t z = (uint32_t)zz;
    if (j == nz - 1) z &= zmask;
    if (j == rl2) cC = (z >> rbit2) & 1u;
    if (j >= wfirst) {
      uint32_t w = z;
      if (k2 > 0) {
        w = __funnelshift_r(zprev, z, kb) + cC;
        cC = w < cC ? 1u : 0u;
        if (i == nf - 1) w &= wmask;
      }
      if (i < nf && i < out_limbs) dst[(size_t)i * N] = w;
      ++i;
    }
    zprev = z;
    xprev = x;
  };
  // z limbs [0, ja): the general step; [ja, nz - 1): no mask, no rounding bit, w limb i < nf - 1
  const int ja = min(nz - 1, max(wfirst, rl2 + 1));
  int j = 0;
  for (; j < ja; ++j) step(j, ripple(sl + j + 1, xload(sl + j + 1)), j < na ? add[(size_t)j * add_stride] : 0u);
  for (; j < nz - 1; j += 8) {
    uint32_t xv[8], av[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      xv[q] = xload(sl + j + q + 1);
      av[q] = j + q < na ? add[(size_t)(j + q) * add_stride] : 0u;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (j + q >= nz - 1) break;
      const uint32_t x = ripple(sl + j + q + 1, xv[q]);
      const uint64_t zz = (uint64_t)__funnelshift_r(xprev, x, sb) + av[q] + c;
      c = (uint32_t)(zz >> 32);
      const uint32_t z = (uint32_t)zz;
      uint32_t w = z;
      if (k2 > 0) {
        w = __funnelshift_r(zprev, z, kb) + cC;
        cC = w < cC ? 1u : 0u;
      }
      if (i < out_limbs) dst[(size_t)i * N] = w;
      ++i;
      zprev = z;
      xprev = x;
    }
  }
  j = nz - 1;
  step(j, ripple(sl + j + 1, xload(sl + j + 1)), j < na ? add[(size_t)j * add_stride] : 0u);
  // w limbs whose upper z limb lies above Z: z_{nz-1} (when it is their lower limb) and zeros
  for (; i < nf; ++i) {
    uint32_t w = (kl + i == nz - 1 ? (zprev >> kb) : 0u) + cC;
    cC = w < cC ? 1u : 0u;
    if (i == nf - 1) w &= wmask;
    if (i < out_limbs) dst[(size_t)i * N] = w;
  }
  for (; i < out_limbs; ++i) dst[(size_t)i * N] = 0u;
}

// Limb partial S0 + 2^8 S1 + 2^16 S2 + 2^24 S3 of four exact column sums
// |S_u| < 2^22 held as fp32 in v: the bits of S + 1.5 2^23 are 0x4B400000 + S,
// so two 32-bit wrap-around sums (each exact as int32) and one 64-bit
// combine give it; K = -257 * 0x4B400000 mod 2^32 removes the offsets.
__device__ __forceinline__ long long limb_partial_exact(const uint32_t* v) {
  uint32_t a[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) a[u] = __float_as_uint(__uint_as_float(v[u]) + 12582912.0f);
  const uint32_t lo = a[0] + (a[1] << 8) + 0x74C00000u;
  const uint32_t hi = a[2] + (a[3] << 8) + 0x74C00000u;
  return (long long)(int32_t)lo + ((long long)(int32_t)hi << 16);
}
__device__ __forceinline__ long long limb_partial_cvt(const uint32_t* v) {
  return (long long)__float2int_rn(__uint_as_float(v[0])) + (long long)__float2int_rn(__uint_as_float(v[1])) * 256LL +
         (long long)__float2int_rn(__uint_as_float(v[2])) * 65536LL +
         (long long)__float2int_rn(__uint_as_float(v[3])) * 16777216LL;
}

struct TcShape {
  int r, MT, nblk, npoly, ntiles;  // primes, output m-tiles, 128-blocks per polynomial, tiles
  int acc_cols, nacc;              // TMEM columns per accumulator, accumulators
  int nadd;                        // staged addend buffers (0: the epilogue reads the addend from global)
  int const_bytes;                 // shared bytes of the per-prime constants
  int limb;                        // 1: a limb column per epilogue group (some tile drains TMEM first)
  int exact22;                     // 1: every column sum is below 2^22 (fp32 -> int by one exact addition)
  int lbase;                       // first limb a limb column holds (limbs below only feed the carry)
  int split;                       // 1: both epilogue groups drain every tile (relinearisation, one accumulator)
};

// Shared memory of k_crt_tc: header, prime constants, quotient partial sums
// and epilogue carries, residue stages, two A stages (K 64, or K 128 with B
// resident), B (two stages of two K 32 slices, one stage per chunk, or all of
// it resident), one limb column per epilogue group (per tile parity when both
// groups drain every tile) when some tile needs it, and the staged addends.
static size_t tc_b_bytes(const TcShape& sh, bool res) {
  const int KS = (sh.r + 4) >> 2;
  return (size_t)(res ? (KS + 1) / 2 : 4) * sh.MT * 16 * 64;
}
static size_t tc_smem_bytes(const TcShape& sh, int add_limbs, bool res) {
  return (size_t)kTcHead + sh.const_bytes + kTcFsx + (size_t)kTcNX * kTcXStage + 2 * (size_t)kTcAStage * (res ? 2 : 1) +
         tc_b_bytes(sh, res) + (sh.limb ? 2 * (size_t)(4 * sh.MT - sh.lbase) * kTcRows * 4 : 0) +
         (size_t)sh.nadd * add_limbs * 512;
}

// RES: B (all 4(r + 1) digits of every output column) stays in shared memory
// for the whole persistent kernel and an A chunk spans two residue chunks
// (K 128), so the MMA thread polls one barrier per eight k-steps; each of its
// barrier polls, MMAs and commits costs it 100-250 cycles, which otherwise
// bounds the tile rate.  Used when B fits (the tensor-product shape).
template <bool RES>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_crt_tc(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_xp,
             const __grid_constant__ CUtensorMap tm_add, TcShape sh,
             uint32_t* __restrict__ out, size_t out_pstride, size_t out_bstride, EpiArgs epi, int N,
             const uint32_t* __restrict__ qtab, const uint2* __restrict__ cinv, const float* __restrict__ invq,
             const uint16_t* __restrict__ bmat, int pmax) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (smem_addr(smem) & 1023u) {  // TMA boxes and MMA operands assume 1 KB alignment
    if (tid == 0) atomicOr(&g_fhe_dev_status, 2u);
    return;
  }
  const int r = sh.r, MT = sh.MT;
  const int P = 16 * MT;
  const int KS = (r + 4) >> 2;    // k-steps of 16 over the 4 (r + 1) digits
  const int nch = (KS + 3) >> 2;  // chunks of 4 k-steps (16 primes)
  const uint32_t bslice = (uint32_t)P * 64u;  // bytes of a K-32 slice of B
  constexpr int CPA = RES ? 2 : 1;             // residue chunks per A chunk
  constexpr uint32_t kAStage = (uint32_t)kTcAStage * CPA, kASbo = 1024u * CPA;
  const int nchA = (nch + CPA - 1) / CPA;      // A chunks per tile
  const int add_limbs = epi.add ? epi.add_limbs : 0;
  uint4* CONST = reinterpret_cast<uint4*>(smem + kTcHead);
  float* FSX = reinterpret_cast<float*>(smem + kTcHead + sh.const_bytes);
  uint8_t* X = smem + kTcHead + sh.const_bytes + kTcFsx;
  uint8_t* A = X + kTcNX * kTcXStage;
  uint8_t* B = A + 2 * kAStage;
  uint32_t* LIMB = reinterpret_cast<uint32_t*>(B + (size_t)(RES ? (KS + 1) / 2 : 4) * bslice);
  const int lcol = 4 * MT - sh.lbase;  // limbs held per coefficient in a limb column
  uint8_t* ADD = reinterpret_cast<uint8_t*>(LIMB + (sh.limb ? (size_t)2 * lcol * kTcRows : 0));
  const uint32_t bar0 = smem_addr(smem);
  auto x_full = [&](int s) { return bar0 + 8u * s; };
  auto x_empty = [&](int s) { return bar0 + 8u * (3 + s); };
  auto a_full = [&](int s) { return bar0 + 8u * (6 + s); };
  auto a_empty = [&](int s) { return bar0 + 8u * (8 + s); };
  auto b_full = [&](int s) { return bar0 + 8u * (10 + s); };
  // per tile parity (= epilogue group): each completes once every two tiles
  auto acc_full = [&](int s) { return bar0 + 8u * (14 + s); };
  auto acc_empty = [&](int s) { return bar0 + 8u * (16 + s); };
  auto add_full = [&](int s) { return bar0 + 8u * (18 + s); };
  auto add_empty = [&](int s) { return bar0 + 8u * (20 + s); };
  auto fsx_bar = [&](int s) { return bar0 + 8u * (22 + s); };  // per tile parity: Y partial sums written
  auto limb_full = [&](int s) { return bar0 + 8u * (24 + s); };   // split: both halves of a limb column written
  auto limb_empty = [&](int s) { return bar0 + 8u * (26 + s); };  // split: the column has been streamed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 512);
  auto tile_of = [&](int t, int& n0, int& poly, int& b) {
    const int py = t / sh.nblk;
    n0 = (t - py * sh.nblk) * kTcRows;
    poly = py % sh.npoly;
    b = py / sh.npoly;
  };

  if (tid == 0) {
    for (int s = 0; s < kTcNX; ++s) {
      mbar_init(x_full(s), 1);
      mbar_init(x_empty(s), 32 * kTcYWarps);
    }
    for (int s = 0; s < 2; ++s) {
      // streamed B shares the A stage barriers: full after the digit warps and the
      // B copies (one arrival with its bytes), empty after one MMA commit
      mbar_init(a_full(s), 32 * kTcYWarps + (RES ? 0 : 1));
      mbar_init(a_empty(s), 1);
      mbar_init(b_full(s), 1);  // resident B: all of it, once
      mbar_init(acc_full(s), 1);
      mbar_init(acc_empty(s), sh.split ? 2 * kTcRows : kTcRows);
      mbar_init(limb_full(s), 2 * kTcRows);
      mbar_init(limb_empty(s), kTcRows);
      mbar_init(add_full(s), 1);
      mbar_init(add_empty(s), kTcRows);
      mbar_init(fsx_bar(s), 32 * kTcYWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  for (int i = tid; i < r; i += kTcThreads) {
    const uint2 ci = __ldg(cinv + i);
    CONST[i] = make_uint4(__ldg(qtab + i), ci.x, ci.y, __float_as_uint(__ldg(invq + i)));
  }
  if (warp == kTcWarpMma) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(tmem_slot)),
                 "r"(sh.acc_cols * sh.nacc)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == kTcWarpProd) {
    if (lane == 0) {
      // producer: one TMA box (128 coefficients x 16 primes) per chunk; at
      // each tile start the next tile's residues are prefetched into L2
      int g = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < sh.ntiles && ok; t += gridDim.x) {
        int n0, poly, b;
        tile_of(t, n0, poly, b);
        if (t + (int)gridDim.x < sh.ntiles) {
          int n0n, polyn, bn;
          tile_of(t + gridDim.x, n0n, polyn, bn);
          tma_prefetch_4d(&tm_xp, n0n, 0, polyn, bn);
        }
        for (int c = 0; c < nch && ok; ++c, ++g) {
          const int sx = g % kTcNX;
          if (g >= kTcNX && !(ok = mbar_wait(x_empty(sx), (uint32_t)((g / kTcNX) - 1) & 1u))) break;
          mbar_expect_tx(x_full(sx), (uint32_t)kTcXStage);
          tma_load_4d(smem_addr(X + sx * kTcXStage), &tm_x, n0, 16 * c, poly, b, x_full(sx));
        }
      }
    }
  } else if (warp == kTcWarpProdAdd) {
    if (lane == 0 && sh.nadd) {
      // addend limbs of each tile, nadd stages ahead of the epilogue
      int tl = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < sh.ntiles && ok; t += gridDim.x, ++tl) {
        int n0, poly, b;
        tile_of(t, n0, poly, b);
        const int s = tl % sh.nadd;
        if (tl >= sh.nadd &&
            !(ok = mbar_wait(add_empty((tl - sh.nadd) & 1), (uint32_t)((tl - sh.nadd) >> 1) & 1u)))
          break;
        const bool has = add_limbs > 0 && poly < epi.add_polys;
        mbar_expect_tx(add_full(tl & 1), has ? (uint32_t)add_limbs * 512u : 0u);
        if (has)
          tma_load_4d(smem_addr(ADD + (size_t)s * add_limbs * 512), &tm_add, n0, 0, poly, b, add_full(tl & 1));
      }
    }
  } else if (warp == kTcWarpProdB) {
    if (RES) {
      if (lane == 0) {  // all of B once, on barrier b_full(0)
        const int nsl = (KS + 1) / 2;
        mbar_expect_tx(b_full(0), (uint32_t)nsl * bslice);
        for (int c2 = 0; c2 < nsl; ++c2)
          bulk_g2s(smem_addr(B + (size_t)c2 * bslice), bmat + (size_t)c2 * pmax * 32, bslice, b_full(0));
      }
    } else if (lane == 0) {
      // B: per chunk one stage of two K 32 slices (K 64), the same sequence for every tile
      int gb = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < sh.ntiles && ok; t += gridDim.x)
        for (int c = 0; c < nch; ++c, ++gb) {
          const int sb = gb & 1;
          if (gb >= 2 && !(ok = mbar_wait(a_empty(sb), (uint32_t)((gb >> 1) - 1) & 1u))) break;
          mbar_expect_tx(a_full(sb), 2u * bslice);
          for (int h = 0; h < 2; ++h)
            bulk_g2s(smem_addr(B + (size_t)(2 * sb + h) * bslice), bmat + (size_t)(2 * c + h) * pmax * 32, bslice,
                     a_full(sb));
        }
    }
  } else if (warp == kTcWarpMma) {
    if (lane == 0) {
      // MMA issue: D[128][P] += A_chunk B_slice^T, output columns in pieces of at most 256.
      // This one thread's instruction latency bounds the MMA rate: everything per
      // split is precomputed, descriptors advance by adding to the address field.
      const int nsplit = (MT + 15) / 16;  // 1 or 2 (P <= 512)
      const int mh = nsplit > 1 ? MT / 2 : MT;  // m-tiles of the first piece
      const uint32_t col1 = 16u * (uint32_t)mh;
      const uint64_t boff1 = (uint64_t)((2u * (uint32_t)mh * 512u) >> 4);
      const uint32_t idesc0 = (1u << 4) | ((16u * (uint32_t)mh >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
      const uint32_t idesc1 = (1u << 4) | ((16u * (uint32_t)(MT - mh) >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
      const uint64_t adesc0 = tc_desc(smem_addr(A), 128u, kASbo);
      const uint64_t bdesc0 = tc_desc(smem_addr(B), 128u, 512u);
      int g = 0, tl = 0;
      bool ok = true;
      if (RES) ok = mbar_wait(b_full(0), 0u);
      for (int t = blockIdx.x; t < sh.ntiles && ok; t += gridDim.x, ++tl) {
        const int ab = tl % sh.nacc;
        if (tl >= sh.nacc &&
            !(ok = mbar_wait(acc_empty((tl - sh.nacc) & 1), (uint32_t)((tl - sh.nacc) >> 1) & 1u)))
          break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t dbase = tmem + (uint32_t)(ab * sh.acc_cols);
        if (RES) {
          // B resident: k-step j of the tile reads slice j / 2 at 256 B (j odd)
          uint64_t db = bdesc0;
          for (int c = 0; c < nchA && ok; ++c, ++g) {
            const int s = g & 1;
            if (!(ok = mbar_wait(a_full(s), (uint32_t)(g >> 1) & 1u))) break;
            const uint64_t adesc = adesc0 + (uint64_t)((s * kAStage) >> 4);
            const int nks = min(8, KS - 8 * c);
            for (int ks = 0; ks < nks; ++ks) {
              const uint32_t accum = (c > 0 || ks > 0) ? 1u : 0u;
              const uint64_t da = adesc + (uint64_t)(16 * ks);
              tc_mma(dbase, da, db, idesc0, accum);
              if (nsplit > 1) tc_mma(dbase + col1, da, db + boff1, idesc1, accum);
              db += (ks & 1) ? (uint64_t)((bslice - 256u) >> 4) : (uint64_t)16;
            }
            tc_commit(a_empty(s));
          }
        } else {
          for (int c = 0; c < nch && ok; ++c, ++g) {
            const int s = g & 1;
            if (!(ok = mbar_wait(a_full(s), (uint32_t)(g >> 1) & 1u))) break;
            const uint64_t adesc = adesc0 + (uint64_t)((s * kAStage) >> 4);
            const int nks = min(4, KS - 4 * c);
            const uint64_t bdesc = bdesc0 + (uint64_t)((2u * (uint32_t)s * bslice) >> 4);  // B stage = A stage
            for (int ks = 0; ks < nks; ++ks) {
              const uint32_t accum = (c > 0 || ks > 0) ? 1u : 0u;
              const uint64_t da = adesc + (uint64_t)(16 * ks);  // + 256 B per k-step
              const uint64_t db = bdesc + (uint64_t)((ks >> 1) * (bslice >> 4) + 16 * (ks & 1));
              tc_mma(dbase, da, db, idesc0, accum);
              if (nsplit > 1) tc_mma(dbase + col1, da, db + boff1, idesc1, accum);
            }
            tc_commit(a_empty(s));
          }
        }
        if (!ok) break;
        tc_commit(acc_full(tl & 1));
      }
    }
  } else if (warp < kTcYWarps) {
    // Y: digits of y_i (and kappa); thread (t, h) handles primes 8h .. 8h + 7 of every chunk of row t
    const int t0 = tid & (kTcRows - 1), h = tid >> 7;
    int g = 0, tly = 0, ga = 0;  // residue chunks, tiles, A chunks
    bool ok = true;
    for (int t = blockIdx.x; t < sh.ntiles && ok; t += gridDim.x, ++tly) {
      float fs = 0.f;
      for (int c = 0; c < nch; ++c, ++g) {
        const int sx = g % kTcNX, u = c % CPA, sa = ga & 1;
        if (!(ok = mbar_wait(x_full(sx), (uint32_t)(g / kTcNX) & 1u))) break;
        if (u == 0 && ga >= 2 && !(ok = mbar_wait(a_empty(sa), (uint32_t)((ga >> 1) - 1) & 1u))) break;
        const uint32_t* xs = reinterpret_cast<const uint32_t*>(X + sx * kTcXStage) + 8 * h * kTcRows + t0;
        uint8_t* arow = A + sa * kAStage + (t0 >> 3) * kASbo + (t0 & 7) * 16 + (8 * u + 4 * h) * 128;
        const int i0 = 16 * c + 8 * h;
        uint32_t yv[8];
        if (16 * c + 16 <= r) {
          // eight real primes: every load first, then the arithmetic
          uint32_t xv[8];
          uint4 kq[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) xv[j] = xs[j * kTcRows];
#pragma unroll
          for (int j = 0; j < 8; ++j) kq[j] = CONST[i0 + j];
#pragma unroll
          for (int j = 0; j < 8; ++j) yv[j] = shoup_mul(xv[j], kq[j].y, kq[j].z, kq[j].x);
#pragma unroll
          for (int j = 0; j < 8; ++j) fs = fmaf(__uint2float_rn(yv[j]), __uint_as_float(kq[j].w), fs);
        } else {
          // the chunk holding kappa (i = r): both halves exchange their partial quotient sums
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int i = i0 + j;
            yv[j] = 0u;
            if (i < r) {
              const uint4 k = CONST[i];
              yv[j] = shoup_mul(xs[j * kTcRows], k.y, k.z, k.x);
              fs = fmaf(__uint2float_rn(yv[j]), __uint_as_float(k.w), fs);
            }
          }
          float* fx = FSX + (tly & 1) * 2 * kTcRows;
          fx[h * kTcRows + t0] = fs;
          mbar_arrive(fsx_bar(tly & 1));
          if (!(ok = mbar_wait(fsx_bar(tly & 1), (uint32_t)(tly >> 1) & 1u))) break;
          if (r >= i0 && r < i0 + 8) {
            const uint32_t kappa = (uint32_t)__float2int_rn(fx[t0] + fx[kTcRows + t0]);
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (i0 + j == r) yv[j] = kappa;
          }
        }
#pragma unroll
        for (int jp = 0; jp < 4; ++jp) {
          uint32_t d[4];
          y_digits(yv[2 * jp], d[0], d[1]);
          y_digits(yv[2 * jp + 1], d[2], d[3]);
          *reinterpret_cast<uint4*>(arow + jp * 128) = make_uint4(d[0], d[1], d[2], d[3]);
        }
        mbar_arrive(x_empty(sx));
        if (u == CPA - 1 || c == nch - 1) {
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          mbar_arrive(a_full(sa));
          ++ga;
        }
      }
    }
  } else {
    // E: two groups of four warps take alternate tiles; warp w reads TMEM lanes 32 (w % 4) .. + 31
    const int e = tid - 32 * kTcYWarps;
    const int eg = e >> 7, ec = e & (kTcRows - 1);
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
    uint32_t* limb = LIMB + (size_t)eg * lcol * kTcRows + ec - (size_t)sh.lbase * kTcRows;  // index by limb l
    int tl = 0;
    bool ok = true;
    // column sums (exact integers in fp32) -> 32-bit limbs, 16 columns (4 limbs) per TMEM load:
    // limb l = sum_u S_{4l+u} 256^u + carry.  With |S| < 2^22 the low mantissa bits of
    // S + 1.5 2^23 are S (one FADD), else cvt.rni.
    auto limbs16 = [&](auto exact, uint32_t taddr, long long& carry, auto&& emit, int m) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long val =
            carry + (decltype(exact)::value ? limb_partial_exact(v + 4 * q) : limb_partial_cvt(v + 4 * q));
        carry = val >> 32;
        emit(4 * m + q, (uint32_t)val);
      }
    };
    if (sh.split) {
      // Relinearisation with one accumulator: both groups drain every tile, group 0 the low
      // column half (its carry out goes through shared memory), group 1 the high half with a
      // zero carry in.  Group (tile & 1) then streams the tile's limb column, adding that carry
      // at limb lsplit, while the MMAs fill the accumulator again: the MMAs wait for half a
      // drain instead of a whole one.
      const int mh = min(MT, max((MT + 1) >> 1, (sh.lbase + 3) >> 2));  // limbs >= 4 mh >= lbase are stored
      const int lsplit = 4 * mh;
      const int m0 = eg ? mh : 0, m1 = eg ? MT : mh;
      long long* CAR = reinterpret_cast<long long*>(FSX + 4 * kTcRows);  // [tile parity][row]
      for (int t = blockIdx.x; t < sh.ntiles; t += gridDim.x, ++tl) {
        const int par = tl & 1;
        ok = ok && mbar_wait(acc_full(par), (uint32_t)(tl >> 1) & 1u);
        if (tl >= 2) ok = ok && mbar_wait(limb_empty(par), (uint32_t)((tl >> 1) - 1) & 1u);
        ok = __all_sync(0xFFFFFFFFu, ok);  // tcgen05.ld is warp-collective
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t base = tmem + lane_off;  // the single accumulator
        uint32_t* col = LIMB + (size_t)par * lcol * kTcRows + ec - (size_t)sh.lbase * kTcRows;
        long long carry = 0;
        auto emit = [&](int l, uint32_t x) {
          if (l >= sh.lbase) col[(size_t)l * kTcRows] = x;
        };
        for (int m = m0; m < m1; ++m) {
          if (sh.exact22)
            limbs16(std::true_type{}, base + 16u * (uint32_t)m, carry, emit, m);
          else
            limbs16(std::false_type{}, base + 16u * (uint32_t)m, carry, emit, m);
        }
        if (eg == 0) CAR[par * kTcRows + ec] = carry;
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        mbar_arrive(acc_empty(par));
        mbar_arrive(limb_full(par));
        if (par != eg) continue;
        int n0, poly, b;
        tile_of(t, n0, poly, b);
        if (!(ok = mbar_wait(limb_full(par), (uint32_t)(tl >> 1) & 1u))) break;
        if (sh.nadd && !(ok = mbar_wait(add_full(eg), (uint32_t)(tl >> 1) & 1u))) break;
        const int ob = epi.item_bits ? __ldg(epi.item_bits + b) : epi.out_bits;
        const bool has_add = epi.add && poly < epi.add_polys;
        const uint32_t* add_s =
            sh.nadd ? reinterpret_cast<const uint32_t*>(ADD + (size_t)(tl % sh.nadd) * add_limbs * 512) + ec : nullptr;
        uint32_t* dst = out + (size_t)b * out_bstride + (size_t)poly * out_pstride + n0 + ec;
        const uint32_t* add = has_add ? (add_s ? add_s
                                               : epi.add + (size_t)b * epi.add_bstride +
                                                     (size_t)poly * epi.add_pstride + n0 + ec)
                                      : nullptr;
        // group 0's carry enters the high half at limb lsplit, rippled in as the epilogue reads it
        relin_column(col, 4 * MT, lsplit, (int)CAR[par * kTcRows + ec], epi, ob, add, add_s ? kTcRows : N, dst, N);
        if (sh.nadd) mbar_arrive(add_empty(eg));
        mbar_arrive(limb_empty(par));
      }
    }
    for (int t = blockIdx.x; t < sh.ntiles && !sh.split; t += gridDim.x, ++tl) {
      if ((tl & 1) != eg) continue;
      int n0, poly, b;
      tile_of(t, n0, poly, b);
      const int ab = tl % sh.nacc;
      ok = ok && mbar_wait(acc_full(eg), (uint32_t)(tl >> 1) & 1u);
      ok = __all_sync(0xFFFFFFFFu, ok);  // tcgen05.ld is warp-collective
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t base = tmem + lane_off + (uint32_t)(ab * sh.acc_cols);
      const int ob = epi.item_bits ? __ldg(epi.item_bits + b) : epi.out_bits;
      const bool has_add = epi.add && poly < epi.add_polys;
      const int32_t* smallp = poly == 0 ? epi.small : (poly == 1 ? epi.small1 : nullptr);
      // 0: limb column + crt_epilogue, 1: masked store, 2: relinearisation stream
      const int mode = (epi.kind == Epi::kStore && !has_add && !smallp) ? 1
                       : (epi.kind == Epi::kRelin && epi.shift > 0 && !smallp) ? 2 : 0;
      // with two accumulators the stream runs off TMEM directly; with one the
      // accumulator is drained into the limb column first and released
      const bool direct = sh.nacc == 2 && mode != 0;
      const uint32_t* add_s =
          sh.nadd ? reinterpret_cast<const uint32_t*>(ADD + (size_t)(tl % sh.nadd) * add_limbs * 512) + ec : nullptr;
      uint32_t* dst = out + (size_t)b * out_bstride + (size_t)poly * out_pstride + n0 + ec;
      const int nlo = (ob + 31) >> 5;
      RelinStream rs;
      if (mode == 2) relin_setup(rs, epi, ob, has_add, add_s, b, poly, n0 + ec, N, dst);
      bool have_add_stage = false;
      if (direct && mode == 2 && sh.nadd) {
        if (!(ok = mbar_wait(add_full(eg), (uint32_t)(tl >> 1) & 1u))) break;
        have_add_stage = true;
      }
      // limbs below the relinearisation's rounding bit only feed the carry
      const int lfirst = mode == 2 ? min(rs.rl, rs.sl) : 0;
      long long carry = 0;
      // column sums (exact integers in fp32) -> 32-bit limbs: limb l = sum_u S_{4l+u} 256^u + carry.
      // With |S| < 2^22 the low mantissa bits of S + 1.5 2^23 are S (one FADD), else cvt.rni.
      auto drain = [&](auto exact, auto&& emit) {
        for (int m = 0; m < MT; ++m) {
          uint32_t v[16];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(base + 16u * (uint32_t)m));
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const long long val =
                carry + (decltype(exact)::value ? limb_partial_exact(v + 4 * q) : limb_partial_cvt(v + 4 * q));
            carry = val >> 32;
            emit(4 * m + q, (uint32_t)val);
          }
        }
      };
      // the limb consumer is chosen once per tile
      auto run = [&](auto&& emit) {
        if (sh.exact22)
          drain(std::true_type{}, emit);
        else
          drain(std::false_type{}, emit);
      };
      if (!direct) {
        run([&](int l, uint32_t x) {
          if (l >= lfirst) limb[(size_t)l * kTcRows] = x;
        });
      } else if (mode == 1) {
        // X mod 2^ob: full limbs below the top one, the top one masked, zeros above
        const uint32_t topmask = limb_mask(nlo - 1, ob);
        const int olim = epi.out_limbs;
        run([&](int l, uint32_t x) {
          if (l < olim) dst[(size_t)l * N] = l < nlo - 1 ? x : (l == nlo - 1 ? (x & topmask) : 0u);
        });
      } else {
        run([&](int l, uint32_t x) { rs.push_x(l, x); });
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      mbar_arrive(acc_empty(eg));
      if (sh.nadd && !have_add_stage && !(ok = mbar_wait(add_full(eg), (uint32_t)(tl >> 1) & 1u))) break;
      if (direct) {
        if (mode == 2) rs.finish(4 * MT);
      } else if (mode == 1) {
        for (int l0 = 0; l0 < epi.out_limbs; l0 += 8) {
          uint32_t xv[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) xv[q] = (l0 + q < nlo) ? limb[(size_t)(l0 + q) * kTcRows] : 0u;
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (l0 + q < epi.out_limbs) dst[(size_t)(l0 + q) * N] = xv[q] & limb_mask(l0 + q, ob);
        }
      } else if (mode == 2) {
        for (int l0 = lfirst; l0 < 4 * MT; l0 += 8) {
          uint32_t xv[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) xv[q] = (l0 + q < 4 * MT) ? limb[(size_t)(l0 + q) * kTcRows] : 0u;
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (l0 + q < 4 * MT) rs.push_x(l0 + q, xv[q]);
        }
        rs.finish(4 * MT);
      } else {
        crt_epilogue(LIMB + (size_t)eg * lcol * kTcRows, ec, kTcRows, 4 * MT, epi, poly, b, n0 + ec, N, out,
                     out_pstride, out_bstride, add_s, kTcRows);
      }
      if (sh.nadd) mbar_arrive(add_empty(eg));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == kTcWarpMma) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(sh.acc_cols * sh.nacc)
                 : "memory");
  }
}

// Runs the tensor-core form when it applies; returns 1 if launched, 0 if the
// caller must use the integer form (nothing enqueued).
// Tensor maps for the TMA loads: 4-D u32 tensors [d3][d2][d1][d0] with element
// strides s1, s2, s3 and a box of b0 x b1.  cuTensorMapEncodeTiled comes from
// the driver through the runtime's entry-point query (no link to libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}
static bool tmap_4d(CUtensorMap* m, const void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t d3, size_t s1,
                    size_t s2, size_t s3, uint32_t b0, uint32_t b1) {
  const EncodeTiledFn fn = encode_tiled();
  if (!fn || s1 == 0 || s2 == 0 || s3 == 0) return false;
  const cuuint64_t dims[4] = {d0, d1, d2, d3};
  const cuuint64_t strides[3] = {(cuuint64_t)s1 * 4, (cuuint64_t)s2 * 4, (cuuint64_t)s3 * 4};
  const cuuint32_t box[4] = {b0, b1, 1, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int tc_launch(const fhe_ctx* ctx, const uint32_t* in, size_t ip, size_t ib, int r, int npoly, int nbatch,
                     uint32_t* out, size_t op, size_t ob, const EpiArgs& epi, int need, cudaStream_t st) {
  const int N = ctx->N;
  const int MT = (need + 3) / 4;
  if (!ctx->d_crt_tc || r + 1 > 255 || N % kTcRows != 0 || MT > ctx->crt_tc_mt || (ip & 3) || (ib & 3) ||
      ((uintptr_t)in & 15))
    return 0;
  TcShape sh;
  sh.r = r;
  sh.MT = MT;
  sh.nblk = N / kTcRows;
  sh.npoly = npoly;
  sh.ntiles = sh.nblk * npoly * nbatch;
  sh.acc_cols = 32;
  while (sh.acc_cols < 16 * MT) sh.acc_cols <<= 1;
  sh.nacc = 2 * sh.acc_cols <= 512 ? 2 : 1;
  sh.const_bytes = (r * 16 + 1023) & ~1023;
  sh.exact22 = ctx->crt_mode == FHE_CRT_DIRECT && ctx->crt_tc_exact22.size() > (size_t)r ? ctx->crt_tc_exact22[r] : 0;
  const int add_limbs = epi.add ? epi.add_limbs : 0;
  const bool stageable = add_limbs > 0 && !((uintptr_t)epi.add & 15) && !(epi.add_pstride & 3) &&
                         !(epi.add_bstride & 3) && !(N & 3);
  // the epilogue streams straight from TMEM unless the accumulator is single or
  // some polynomial takes the general epilogue (the kernel's own rule)
  sh.limb = sh.nacc == 1;
  for (int p = 0; p < npoly && !sh.limb; ++p) {
    const bool has_add = epi.add && p < epi.add_polys;
    const bool smallp = p == 0 ? epi.small != nullptr : (p == 1 ? epi.small1 != nullptr : false);
    const bool streamed = (epi.kind == Epi::kStore && !has_add && !smallp) ||
                          (epi.kind == Epi::kRelin && epi.shift > 0 && !smallp);
    if (!streamed) sh.limb = 1;
  }
  // when every tile is a relinearisation stream, a limb column starts at its rounding limb
  sh.lbase = 0;
  if (epi.kind == Epi::kRelin && epi.shift > 0) {
    bool all_stream = true;
    for (int p = 0; p < npoly; ++p)
      if (p == 0 ? epi.small != nullptr : (p == 1 ? epi.small1 != nullptr : false)) all_stream = false;
    if (all_stream) sh.lbase = min((epi.shift - 1) >> 5, epi.shift >> 5);
  }
  // one accumulator and every tile a relinearisation stream: both epilogue groups drain each tile
  sh.split = (sh.nacc == 1 && sh.lbase > 0) ? 1 : 0;
  constexpr size_t kSmemMax = 227 * 1024;
  sh.nadd = 0;
  const bool res = tc_smem_bytes(sh, add_limbs, true) <= kSmemMax;
  if (stageable) {
    for (int na = 2; na >= 1 && !sh.nadd; --na) {
      sh.nadd = na;
      if (tc_smem_bytes(sh, add_limbs, res) > kSmemMax) sh.nadd = 0;
    }
  }
  // residues [nbatch][npoly][r][N]: boxes of 128 x 16 for the stages, 128 x r for the L2 prefetch.
  // A zero stride over a dimension longer than one (a broadcast) has no tensor map: such
  // calls take the integer form, and such addends are read from global memory.
  auto stride_or = [](size_t s, uint64_t extent, size_t dflt) -> size_t { return s ? s : (extent == 1 ? dflt : 0); };
  CUtensorMap tm_x, tm_xp, tm_add;
  memset(&tm_add, 0, sizeof(tm_add));
  const size_t ipx = stride_or(ip, npoly, (size_t)r * N);
  const size_t ibx = stride_or(ib, nbatch, ipx * npoly);
  if (!tmap_4d(&tm_x, in, N, r, npoly, nbatch, N, ipx, ibx, kTcRows, 16) ||
      !tmap_4d(&tm_xp, in, N, r, npoly, nbatch, N, ipx, ibx, kTcRows, (uint32_t)(r < 256 ? r : 256)))
    return 0;
  if (sh.nadd) {
    const int apolys = epi.add_polys < npoly ? epi.add_polys : npoly;
    const size_t apx = stride_or(epi.add_pstride, apolys, (size_t)add_limbs * N);
    const size_t abx = stride_or(epi.add_bstride, nbatch, apx * apolys);
    if (add_limbs > 256 || apolys < 1 ||
        !tmap_4d(&tm_add, epi.add, N, add_limbs, apolys, nbatch, N, apx, abx, kTcRows, (uint32_t)add_limbs))
      sh.nadd = 0;
  }
  const size_t smem = tc_smem_bytes(sh, add_limbs, res);
  if (smem > kSmemMax) return 0;
  static thread_local int configured_dev = -1, nsm = 0;
  if (configured_dev != ctx->device) {
    cudaFuncSetAttribute(k_crt_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
    cudaFuncSetAttribute(k_crt_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    configured_dev = ctx->device;
  }
  const int grid = sh.ntiles < nsm ? sh.ntiles : nsm;
  ProfScope ps(ctx, FHE_K_CRT, 1, st);
  const size_t off = (size_t)r * (r - 1) / 2;
  auto kern = res ? k_crt_tc<true> : k_crt_tc<false>;
  kern<<<grid, kTcThreads, smem, st>>>(tm_x, tm_xp, tm_add, sh, out, op, ob, epi, N, ctx->d_q, ctx->d_crt_inv + off,
                                       ctx->d_invq, ctx->d_crt_tc + ctx->crt_tc_off[r], 16 * ctx->crt_tc_mt);
  return 1;
}

// Self-test of the timeout path: one thread waits on a shared-memory mbarrier that nothing
// arrives on, with at most `tries` polls of a short suspend hint; when they run out it records the
// timeout in the status word (as every pipeline wait of the tensor-core kernels does) and returns.
__global__ void k_wait_selftest(int tries) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = smem_addr(&bar);
  mbar_init(b, 1);
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  for (int it = 0; it < tries; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(b), "r"(0u), "r"(1000u)
        : "memory");
    if (ok) return;  // cannot happen: no thread arrives
  }
  atomicOr(&FHE_TC_STATUS, 1u);
}

// Device status word: nonzero after a bounded wait gave up.  Read and cleared.
unsigned int read_dev_status() {
  unsigned int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_fhe_dev_status, sizeof(v)) != cudaSuccess) v = 0;
  if (v) cudaMemcpyToSymbol(g_fhe_dev_status, &z, sizeof(z));
  return v | read_lift_status();
}

template <int LB>
static int direct_launch(const fhe_ctx* ctx, const uint32_t* in, size_t ip, size_t ib, int r, int npoly, int nbatch,
                         uint32_t* out, size_t op, size_t ob, const EpiArgs& epi, cudaStream_t st) {
  const int N = ctx->N;
  const int threads = kCrtThreads;
  const int rows = (r + 1) > (LB + 2) ? (r + 1) : (LB + 2);
  const size_t smem = (size_t)rows * threads * 4 + 2 * (size_t)(r + 1) * 8 * 4;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_crt_direct<LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((N + threads - 1) / threads, npoly * nbatch);
  ProfScope ps(ctx, FHE_K_CRT, 1, st);
  const size_t off = (size_t)r * (r - 1) / 2;
  const size_t dbase = (size_t)(r - 1) * (r + 2) / 2;
  k_crt_direct<LB><<<grid, threads, smem, st>>>(in, ip, ib, r, npoly, out, op, ob, epi, N, ctx->d_q,
                                                 ctx->d_crt_inv + off, ctx->d_crt_dig + dbase * kCrtDigits,
                                                 ctx->d_invq);
  return FHE_OK;
}

template <int LB>
static int garner_launch(const fhe_ctx* ctx, const uint32_t* in, size_t ip, size_t ib, int r, int npoly, int nbatch,
                         uint32_t* out, size_t op, size_t ob, const EpiArgs& epi, cudaStream_t st) {
  const int N = ctx->N;
  const int threads = kCrtThreads;
  const int rows = r > LB + 2 ? r : LB + 2;
  const size_t smem = (size_t)rows * threads * 4;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_garner<LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((N + threads - 1) / threads, npoly * nbatch);
  ProfScope ps(ctx, FHE_K_CRT, 1, st);
  k_garner<LB><<<grid, threads, smem, st>>>(in, ip, ib, r, npoly, out, op, ob, epi, N, ctx->d_q, ctx->d_garner,
                                             ctx->R, ctx->d_mprod, ctx->d_nscale, ctx->d_nscale_sh);
  return FHE_OK;
}

int launch_garner(const fhe_ctx* ctx, const uint32_t* in, size_t in_pstride, size_t in_bstride, int r, int npoly,
                  int nbatch, uint32_t* out, size_t out_pstride, size_t out_bstride, const EpiArgs& epi,
                  cudaStream_t st) {
  if (r < 2 || r > ctx->R || npoly < 1 || nbatch < 1 || (size_t)npoly * nbatch > 65535u || epi.out_bits < 1) {
    set_error("garner: bad sizes r=%d", r);
    return FHE_EINVAL;
  }
  // limbs the reconstruction must carry: enough for the epilogue's reads
  int need_bits = epi.out_bits + (epi.kind == Epi::kRelin ? epi.shift : 0);
  int need = (need_bits + 31) / 32;
  if (epi.out_limbs > need) need = epi.out_limbs;
  if (need > kMaxLimbs) {
    set_error("garner: %d limbs exceed %d", need, kMaxLimbs);
    return FHE_EINVAL;
  }
  if ((ctx->crt_mode == FHE_CRT_DIRECT || ctx->crt_mode == FHE_CRT_DIRECT_CVT) &&
      tc_launch(ctx, in, in_pstride, in_bstride, r, npoly, nbatch, out, out_pstride, out_bstride, epi, need, st))
    return FHE_OK;
#define FHE_GARNER_CASE(B)                                                                                       \
  if (need <= B)                                                                                                 \
    return ctx->crt_mode == 1                                                                                    \
               ? garner_launch<B>(ctx, in, in_pstride, in_bstride, r, npoly, nbatch, out, out_pstride, out_bstride, \
                                  epi, st)                                                                       \
               : direct_launch<B>(ctx, in, in_pstride, in_bstride, r, npoly, nbatch, out, out_pstride, out_bstride, \
                                  epi, st);
  FHE_GARNER_CASE(8)
  FHE_GARNER_CASE(16)
  FHE_GARNER_CASE(24)
  FHE_GARNER_CASE(32)
  FHE_GARNER_CASE(40)
  FHE_GARNER_CASE(48)
  FHE_GARNER_CASE(56)
  FHE_GARNER_CASE(64)
  FHE_GARNER_CASE(80)
  FHE_GARNER_CASE(96)
  FHE_GARNER_CASE(112)
  FHE_GARNER_CASE(128)
#undef FHE_GARNER_CASE
  return FHE_EINVAL;
}

}  // namespace fhe

extern "C" int fhe_selftest_wait_timeout(int tries, void* stream) {
  if (tries < 1 || tries > 100000) {
    fhe::set_error("selftest_wait_timeout: tries %d out of 1..100000", tries);
    return FHE_EINVAL;
  }
  fhe::k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(tries);
  FHE_CHECK_CUDA(cudaGetLastError());
  return FHE_OK;
}
