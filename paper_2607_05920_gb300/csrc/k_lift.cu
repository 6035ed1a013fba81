// Limb -> RNS lift (Sec. 5 "Limb-to-RNS Conversion"): for each coefficient
// A (L little-endian 32-bit limbs) and each prime q_i,
//     a_i = A mod q_i = sum_l limb_l (2^(32 l) mod q_i)  (mod q_i),
// by limb-wise accumulation with the precomputed constants 2^(32 l) mod q_i
// (Sec. 5 "Precomputed RNS Conversion Constants") and one final reduction.
//
// Integer form (the Garner and integer-pipe reconstruction modes): one thread
// owns one coefficient: its limbs sit in registers (read once, coalesced
// across the warp), and it loops over all primes, writing one coalesced
// residue row per prime.  The constant table of the CTA's primes is staged in
// shared memory and read as warp-wide broadcasts.  The default form,
// k_lift_tc below, runs the same sum as a byte-digit GEMM on the tensor cores.
#include "common.cuh"

namespace fhe {
__device__ unsigned int g_lift_dev_status = 0;  // set when a bounded device wait gives up
}
#define FHE_TC_STATUS fhe::g_lift_dev_status
#include "tc.cuh"

namespace fhe {

constexpr int kLiftThreads = 128;

// Signed lift: the value of batch item b is the two's-complement integer of sb bits held in
// the low sb bits of its limbs (sb = 0: unsigned).  sign_of gives its sign bit; sext_limb gives
// limb l of the same value sign-extended to every limb (limbs at and above bit sb ignored).
__device__ __forceinline__ int item_sbits(int sbits, const int32_t* __restrict__ item_bits, int b, int L) {
  // per-item widths are clamped to the limbs present (a signed launch stays signed for every item)
  return item_bits ? min(max(__ldg(item_bits + b), 1), 32 * L) : sbits;
}
__device__ __forceinline__ uint32_t sign_of(const uint32_t* __restrict__ s, int N, int sb) {
  return (__ldg(s + (size_t)((sb - 1) >> 5) * N) >> ((sb - 1) & 31)) & 1u;
}
__device__ __forceinline__ uint32_t sext_limb(uint32_t x, int l, int sb, uint32_t sgn) {
  const int lo = 32 * l;
  if (lo >= sb) return sgn ? 0xFFFFFFFFu : 0u;
  const int tb = sb - lo;
  if (tb >= 32) return x;
  const uint32_t m = (1u << tb) - 1u;
  return sgn ? (x | ~m) : (x & m);
}

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
                                                       const uint32_t* __restrict__ red, int sbits,
                                                       const int32_t* __restrict__ item_bits) {
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
  // signed: x - sgn 2^sb = (x sign-extended to 32 L bits) - sgn 2^(32 L)
  const int sb = item_sbits(sbits, item_bits, b, L);
  const uint32_t sgn = sb > 0 ? sign_of(s, N, sb) : 0u;
  if (sb > 0) {
#pragma unroll
    for (int l = 0; l < LB; ++l)
      if (l < L) x[l] = sext_limb(x[l], l, sb, sgn);
  }
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
    uint32_t res = reduce96((uint32_t)acc, (uint32_t)(acc >> 32), a2, q, __ldg(red + 4 * i), __ldg(red + 4 * i + 1),
                            __ldg(red + 4 * i + 2));
    if (sgn) res = sub_mod(res, __ldg(pow2 + (size_t)i * kMaxLiftLimbs + L), q);
    d[(size_t)i * N] = res;
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
                                                              const uint32_t* __restrict__ red,
                                                              const uint32_t* __restrict__ pow2, int sbits,
                                                              const int32_t* __restrict__ item_bits) {
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
  const int sb = item_sbits(sbits, item_bits, b, L);
  const uint32_t sgn = sb > 0 ? sign_of(s, N, sb) : 0u;
  if (sb > 0) {
#pragma unroll
    for (int l = 0; l < LB; ++l)
      if (l < L) x[l] = sext_limb(x[l], l, sb, sgn);
  }
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
    uint32_t res = reduce96((uint32_t)acc, (uint32_t)(acc >> 32), 0u, q, __ldg(red + 4 * i), __ldg(red + 4 * i + 1),
                            __ldg(red + 4 * i + 2));
    if (sgn) res = sub_mod(res, __ldg(pow2 + (size_t)i * kMaxLiftLimbs + L), q);
    d[(size_t)i * N] = res;
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
  const uint32_t av = v < 0 ? (uint32_t)(-(int64_t)v) : (uint32_t)v;  // <= 2^31
  for (int i = 0; i < r; ++i) {
    const uint32_t q = __ldg(qtab + i);
    uint32_t m = av < q ? av : av % q;
    if (v < 0 && m != 0) m = q - m;
    dst[(size_t)b * dst_bstride + (size_t)i * N + n] = m;
  }
}

// ------------------------------------------------------ lift, tensor cores
// The lift is a dense contraction too: with the limbs' bytes b_k and
// d_k = b_k - 128 in [-128, 127], and C_{i,k} = 2^(8k) 2^32 mod q_i split into
// digits c_{i,k,a} (|c| <= 128),
//   T_i = sum_a 256^a S_{i,a},  S_{i,a} = sum_k d_k c_{i,k,a},
// is congruent to (x - 128 sum_k 256^k) 2^32 mod q_i.  S = A B^T with A the
// digits of the 128 coefficients of a tile ([128][K = 4L]) and B the
// constants ([4r][K]); |S| <= 4L 2^14 < 2^22 for L < 64, exact in fp32.  One
// more K column (A: 2048, B: 6144, both exact in f16) adds 1.5 2^23 to every
// sum inside the GEMM, so the accumulators hold integers in [2^23, 2^24),
// exact at every partial sum, whose bits are 0x4B400000 + S: the epilogue
// reads the integers off the bit patterns without a conversion.  Adding the
// folded offset (and 2^17 q_i) and one Montgomery reduction gives x mod q_i,
// written as a representative below 2q (the forward transform that follows
// every lift takes inputs below 4q).
// The constants stay resident in shared memory for the whole (persistent)
// kernel; the output columns are split into two TMEM accumulators (residue
// halves) so each half's drain overlaps the other half's MMAs.  Warp roles:
//   warps 0-7   limbs -> digit tile A (two threads per coefficient row),
//               the next tile's limbs loaded while the MMAs read A;
//   warps 8-23  four epilogue groups that drain the first half, then the
//               second, each taking every fourth 4-residue column block:
//               TMEM -> integers -> Montgomery -> residue rows;
//   warp 24     TMEM allocation and the MMA issue (one thread).
constexpr int kLtRows = 128;
constexpr int kLtYWarps = 8, kLtEWarps = 16;
constexpr int kLtWarpMma = kLtYWarps + kLtEWarps;
constexpr int kLtThreads = 32 * (kLtWarpMma + 1);

struct LtShape {
  int r, L, Kpad;          // primes, limbs, K padded to 16
  int r0, n0, n1;          // residues of the first half; MMA N of each half (n1 = 0: one half)
  int acc_cols;            // TMEM columns per accumulator
  int nblk, npoly, ntiles;
};

static size_t lt_smem_bytes(const LtShape& sh) {
  return 512 + 16 * 128 + (size_t)(sh.n0 + sh.n1) * sh.Kpad * 2 + (size_t)kLtRows * sh.Kpad * 2;
}

template <bool SIGNED>
__global__ void __launch_bounds__(kLtThreads, 1)
    k_lift_tc(const uint32_t* __restrict__ src, size_t src_pstride, size_t src_bstride, uint32_t* __restrict__ dst,
              size_t dst_pstride, size_t dst_bstride, LtShape sh, int N, const uint16_t* __restrict__ bmat,
              const uint32_t* __restrict__ qtab, const uint32_t* __restrict__ qinv,
              const uint64_t* __restrict__ offL, int sbits, const int32_t* __restrict__ item_bits) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = sh.r, L = sh.L, Kpad = sh.Kpad;
  const int kcols = Kpad / 8;                       // core-matrix columns along K
  const uint32_t sbo = (uint32_t)kcols * 128u;      // bytes between 8-row groups
  const int nrows = sh.n0 + sh.n1;
  const int nh = sh.n1 > 0 ? 2 : 1;
  uint4* PC = reinterpret_cast<uint4*>(smem + 512);            // per prime {q, q^-1 mod 2^32, K lo, K hi}
  uint8_t* B = smem + 512 + 16 * 128;
  uint8_t* A = B + (size_t)nrows * Kpad * 2;
  const uint32_t bar0 = smem_addr(smem);
  const uint32_t a_full = bar0, a_empty = bar0 + 8;
  auto acc_full = [&](int h) { return bar0 + 16u + 8u * h; };
  auto acc_empty = [&](int h) { return bar0 + 32u + 8u * h; };
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 256);
  auto tile_of = [&](int t, int& n0, int& poly, int& b) {
    const int py = t / sh.nblk;
    n0 = (t - py * sh.nblk) * kLtRows;
    poly = py % sh.npoly;
    b = py / sh.npoly;
  };

  if (tid == 0) {
    mbar_init(a_full, 32 * kLtYWarps);
    mbar_init(a_empty, 1);
    for (int h = 0; h < 2; ++h) {
      mbar_init(acc_full(h), 1);
      mbar_init(acc_empty(h), 32 * kLtEWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // resident constants: B rows (i, a) for i < r (zero above), per-prime reduction constants
  for (int idx = tid; idx < nrows * kcols; idx += kLtThreads) {
    const int p = idx / kcols, kc = idx - p * kcols;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (p < 4 * r) {
      v = __ldg(reinterpret_cast<const uint4*>(bmat) + (((size_t)(p >> 3) * (4 * kMaxLiftLimbs / 8) + kc) * 8 + (p & 7)));
      // K = 4L (limb L's digit 0) carries the conversion constant: every B row holds 6144 there, every
      // A row 2048, so each sum gains 2048 * 6144 = 1.5 2^23 (below)
      if (kc == L / 2) {
        if (L & 1)
          v.z = (v.z & 0xFFFF0000u) | 0x6E00u;
        else
          v.x = (v.x & 0xFFFF0000u) | 0x6E00u;
      }
    }
    *reinterpret_cast<uint4*>(B + ((size_t)((p >> 3) * kcols + kc) * 8 + (p & 7)) * 16) = v;
  }
  for (int i = tid; i < r; i += kLtThreads) {
    const uint64_t k = __ldg(offL + i);
    PC[i] = make_uint4(__ldg(qtab + i), __ldg(qinv + i), (uint32_t)k, (uint32_t)(k >> 32));
  }
  // K padding of the digit tile stays zero, but for the constant 2048 (f16 0x6800) at K = 4L when L is
  // even (for odd L the digit producers write it with limb L's digits)
  for (int idx = tid; idx < kLtRows * kcols; idx += kLtThreads) {
    const int t = idx / kcols, kc = idx - t * kcols;
    if (kc >= (L + 1) / 2)
      *reinterpret_cast<uint4*>(A + (size_t)(t >> 3) * sbo + kc * 128 + (t & 7) * 16) =
          make_uint4(kc == L / 2 ? 0x6800u : 0u, 0u, 0u, 0u);
  }
  if (warp == kLtWarpMma) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(tmem_slot)),
                 "r"(sh.acc_cols * nh)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == kLtWarpMma) {
    if (lane == 0) {
      const int KS = Kpad / 16;
      const uint32_t idesc0 = (1u << 4) | (((uint32_t)sh.n0 >> 3) << 17) | ((uint32_t)(kLtRows >> 4) << 24);
      const uint32_t idesc1 = (1u << 4) | (((uint32_t)sh.n1 >> 3) << 17) | ((uint32_t)(kLtRows >> 4) << 24);
      const uint64_t adesc = tc_desc(smem_addr(A), 128u, sbo);
      const uint64_t bdesc0 = tc_desc(smem_addr(B), 128u, sbo);
      const uint64_t bdesc1 = bdesc0 + (uint64_t)(((uint32_t)(sh.n0 >> 3) * sbo) >> 4);
      int tl = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < sh.ntiles && ok; t += gridDim.x, ++tl) {
        if (!(ok = mbar_wait(a_full, (uint32_t)tl & 1u))) break;
        for (int h = 0; h < nh; ++h) {
          if (tl >= 1 && !(ok = mbar_wait(acc_empty(h), (uint32_t)(tl - 1) & 1u))) break;
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t d = tmem + (uint32_t)(h * sh.acc_cols);
          const uint64_t bd = h ? bdesc1 : bdesc0;
          const uint32_t id = h ? idesc1 : idesc0;
          for (int ks = 0; ks < KS; ++ks)
            tc_mma(d, adesc + (uint64_t)(16 * ks), bd + (uint64_t)(16 * ks), id, ks > 0 ? 1u : 0u);
          tc_commit(acc_full(h));
        }
        if (!ok) break;
        tc_commit(a_empty);
      }
    }
  } else if (warp < kLtYWarps) {
    // Y: thread (t, hh) owns limb pairs [hh PH, min(P2, (hh + 1) PH)) of coefficient t
    const int t0 = tid & (kLtRows - 1), hh = tid >> 7;
    const int P2 = (L + 1) / 2, PH = (P2 + 1) / 2;
    const int p0 = hh * PH, np = max(0, min(P2, p0 + PH) - p0);
    uint8_t* arow = A + (size_t)(t0 >> 3) * sbo + (t0 & 7) * 16;
    uint32_t xv[32];
    int ysb = 0;        // signed: the loaded tile's value width and sign
    uint32_t ysgn = 0;
    auto load = [&](int t) {
      int n0, poly, b;
      tile_of(t, n0, poly, b);
      const uint32_t* s = src + (size_t)b * src_bstride + (size_t)poly * src_pstride + n0 + t0;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int l = 2 * p0 + j;
        xv[j] = (j < 2 * np && l < L) ? __ldg(s + (size_t)l * N) : 0u;
      }
      if constexpr (SIGNED) {
        ysb = item_sbits(sbits, item_bits, b, L);
        ysgn = sign_of(s, N, ysb);
      }
    };
    // the tile after next: its L limb rows of 512 B into L2, one 128-byte line per thread, so
    // the register loads of the next tile (issued while the MMAs read A) find them there
    auto prefetch = [&](int t) {
      if (t >= sh.ntiles) return;
      int n0, poly, b;
      tile_of(t, n0, poly, b);
      const int l = tid >> 2;
      if (l < L) {
        const uint32_t* a =
            src + (size_t)b * src_bstride + (size_t)poly * src_pstride + (size_t)l * N + n0 + 32 * (tid & 3);
        asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a));
      }
    };
    int tl = 0;
    bool ok = true;
    if (blockIdx.x < sh.ntiles) load(blockIdx.x);
    prefetch(blockIdx.x + gridDim.x);
    for (int t = blockIdx.x; t < sh.ntiles && ok; t += gridDim.x, ++tl) {
      if (tl >= 1 && !(ok = mbar_wait(a_empty, (uint32_t)(tl - 1) & 1u))) break;
#pragma unroll
      for (int jp = 0; jp < 16; ++jp) {
        if (jp < np) {
          uint32_t d[4];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            // byte b -> f16 (1024 + b) - 1152 = b - 128; a limb beyond L contributes no digits.  Signed:
            // the value sign-extended to 32 L bits, its top byte fed as the signed digit (b ^ 0x80) - 128
            uint32_t x = xv[2 * jp + u];
            if constexpr (SIGNED) {
              const int l = 2 * (p0 + jp) + u;
              x = sext_limb(x, l, ysb, ysgn) ^ (l == L - 1 ? 0x80000000u : 0u);
            }
            const uint32_t lo = __byte_perm(x, 0x64646464u, 0x5140), hi = __byte_perm(x, 0x64646464u, 0x5342);
            asm("sub.rn.f16x2 %0, %1, %2;\n" : "=r"(d[2 * u]) : "r"(lo), "r"(0x64806480u));
            asm("sub.rn.f16x2 %0, %1, %2;\n" : "=r"(d[2 * u + 1]) : "r"(hi), "r"(0x64806480u));
            if (2 * (p0 + jp) + u >= L) {  // no limb: no digits; limb L: the conversion constant
              d[2 * u] = 2 * (p0 + jp) + u == L ? 0x6800u : 0u;
              d[2 * u + 1] = 0u;
            }
          }
          *reinterpret_cast<uint4*>(arow + (p0 + jp) * 128) = make_uint4(d[0], d[1], d[2], d[3]);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_arrive(a_full);
      prefetch(t + 2 * (int)gridDim.x);
      if (t + (int)gridDim.x < sh.ntiles) load(t + gridDim.x);  // in flight while the MMAs read A
    }
  } else {
    // E: all four groups drain half 0, then half 1, each taking every fourth 4-residue column
    // block, so a half's accumulator is released after a quarter of its work per group and the
    // next tile's MMAs into it wait less
    const int e = tid - 32 * kLtYWarps;
    const int g = e >> 7, ec = e & (kLtRows - 1);
    const int nb0 = (min(r, sh.r0) + 3) / 4;  // 4-residue column blocks of half 0
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
    int tl = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < sh.ntiles && ok; t += gridDim.x, ++tl) {
     int n0, poly, b;
     tile_of(t, n0, poly, b);
     uint32_t* d = dst + (size_t)b * dst_bstride + (size_t)poly * dst_pstride + n0 + ec;
     for (int h = 0; h < nh; ++h) {
      const int i0 = h ? sh.r0 : 0, i1 = h ? r : min(r, sh.r0);
      ok = ok && mbar_wait(acc_full(h), (uint32_t)tl & 1u);
      ok = __all_sync(0xFFFFFFFFu, ok);  // tcgen05.ld is warp-collective
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t base = tmem + lane_off + (uint32_t)(h * sh.acc_cols);
      // blocks are numbered across both halves (half 1 after half 0's nb0) and dealt round-robin,
      // starting one group later each tile, so no group drains more than its share every tile
      const int first = (g - (h ? nb0 : 0) - (tl & 3)) & 3;
      for (int q4 = first; 4 * q4 < i1 - i0; q4 += 4) {
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(base + 16u * (uint32_t)q4));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int i = i0 + 4 * q4 + j;
          if (i < i1) {
            // the accumulators hold S + 1.5 2^23 (the constant column), integers in [2^23, 2^24) as
            // |S| < 2^22, so every partial sum was exact and the bits are 0x4B400000 + S; thus
            // lo = S0 + 256 S1 = a0 + 256 a1 - 257 * 0x4B400000 (mod 2^32, exact as int32)
            const uint32_t* sa = v + 4 * j;
            const int lo = (int)(sa[0] + (sa[1] << 8) + 0x74C00000u), hi = (int)(sa[2] + (sa[3] << 8) + 0x74C00000u);
            const uint4 k = PC[i];
            const uint64_t u = (uint64_t)((long long)lo + ((long long)hi << 16)) +
                               (((uint64_t)k.w << 32) | k.z);  // >= 0, < 2^49
            // Montgomery: (u - m q) / 2^32 with m = u q^-1 mod 2^32, in (-q, 2^17); left as that plus
            // q, in (0, q + 2^17), below 2q: the forward transform that every lift feeds accepts it
            const uint32_t m = (uint32_t)u * k.y;
            d[(size_t)i * N] = (uint32_t)(u >> 32) - __umulhi(m, k.x) + k.x;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      mbar_arrive(acc_empty(h));
     }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == kLtWarpMma) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(sh.acc_cols * nh)
                 : "memory");
  }
}

// Tensor-core lift when it applies (L < 64, r <= 128, N a multiple of 128, shared memory fits);
// returns 1 if launched, 0 if the caller must use the integer form.
static int lift_tc_launch(const fhe_ctx* ctx, const uint32_t* src, int L, size_t sp, size_t sb, uint32_t* dst,
                          size_t dp, size_t db, int npoly, int nbatch, int r, int sbits, const int32_t* item_bits,
                          cudaStream_t st) {
  const int N = ctx->N;
  const bool want_tc = ctx->lift_form == FHE_LIFT_TC ||
                       (ctx->lift_form == FHE_LIFT_AUTO &&
                        (ctx->crt_mode == FHE_CRT_DIRECT || ctx->crt_mode == FHE_CRT_DIRECT_CVT));
  if (!ctx->d_lift_tc || !want_tc || L >= 64 || r > 128 || N % kLtRows != 0) return 0;
  LtShape sh;
  sh.r = r;
  sh.L = L;
  sh.Kpad = 16 * ((4 * L + 1 + 15) / 16);  // the digits and the conversion constant's column
  sh.r0 = 4 * ((r + 7) / 8);  // a multiple of 4, so the first half's N is a multiple of 16
  sh.n0 = 4 * sh.r0;
  sh.n1 = r > sh.r0 ? 16 * ((4 * (r - sh.r0) + 15) / 16) : 0;
  sh.acc_cols = 32;
  while (sh.acc_cols < sh.n0 || sh.acc_cols < sh.n1) sh.acc_cols <<= 1;
  sh.nblk = N / kLtRows;
  sh.npoly = npoly;
  sh.ntiles = sh.nblk * npoly * nbatch;
  if (sh.n0 % 16 || sh.n0 > 256 || sh.n1 > 256) return 0;
  const size_t smem = lt_smem_bytes(sh);
  if (smem > 227 * 1024) return 0;
  static thread_local int configured_dev = -1, nsm = 0;
  if (configured_dev != ctx->device) {
    cudaFuncSetAttribute(k_lift_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_lift_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    configured_dev = ctx->device;
  }
  const int grid = sh.ntiles < nsm ? sh.ntiles : nsm;
  if (sbits > 0 || item_bits)
    k_lift_tc<true><<<grid, kLtThreads, smem, st>>>(src, sp, sb, dst, dp, db, sh, N, ctx->d_lift_tc, ctx->d_q,
                                                    ctx->d_qinv, ctx->d_lift_off_s + (size_t)L * ctx->R, sbits,
                                                    item_bits);
  else
    k_lift_tc<false><<<grid, kLtThreads, smem, st>>>(src, sp, sb, dst, dp, db, sh, N, ctx->d_lift_tc, ctx->d_q,
                                                     ctx->d_qinv, ctx->d_lift_off + (size_t)L * ctx->R, 0, nullptr);
  return 1;
}

// Device status word of this file's kernels: nonzero (then cleared) after a bounded wait gave up.
unsigned int read_lift_status() {
  unsigned int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_lift_dev_status, sizeof(v)) != cudaSuccess) return 0;
  if (v) cudaMemcpyToSymbol(g_lift_dev_status, &z, sizeof(z));
  return v;
}

template <int LB>
static void lift_launch(const fhe_ctx* ctx, const uint32_t* src, int L, size_t sp, size_t sb, uint32_t* dst,
                        size_t dp, size_t db, int npoly, int nbatch, int r, int sbits, const int32_t* item_bits,
                        cudaStream_t st) {
  const int N = ctx->N;
  const int threads = N < kLiftThreads ? N : kLiftThreads;
  dim3 grid((N + threads - 1) / threads, npoly * nbatch);
  if constexpr (LB <= 48) {
    constexpr int MP = (((32 * LB + 23) / 24) + 3) & ~3;
    const size_t smem = (size_t)r * MP * sizeof(uint32_t);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_lift_digits<LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_lift_digits<LB><<<grid, threads, smem, st>>>(src, L, sp, sb, dst, dp, db, npoly, r, N, ctx->d_pow24, ctx->d_q,
                                                    ctx->d_red, ctx->d_pow2, sbits, item_bits);
    return;
  }
  size_t smem = (size_t)r * ((L + 3) & ~3) * sizeof(uint32_t);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_lift<LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_lift<LB><<<grid, threads, smem, st>>>(src, L, sp, sb, dst, dp, db, npoly, r, N, ctx->d_pow2, ctx->d_q,
                                           ctx->d_red, sbits, item_bits);
}

static int lift_any(const fhe_ctx* ctx, const uint32_t* src, int L, size_t src_pstride, size_t src_bstride,
                    uint32_t* dst, size_t dst_pstride, size_t dst_bstride, int npoly, int nbatch, int r, int sbits,
                    const int32_t* item_bits, cudaStream_t st) {
  if (L < 1 || L > kMaxLiftLimbs || r < 1 || r > ctx->R || nbatch < 1 || npoly < 1 ||
      (size_t)npoly * nbatch > 65535u || sbits < 0 || sbits > 32 * L ||
      ((sbits > 0 || item_bits) && L >= kMaxLiftLimbs)) {
    set_error("lift: bad sizes L=%d r=%d sbits=%d", L, r, sbits);
    return FHE_EINVAL;
  }
  if ((size_t)r * ((L + 3) & ~3) * 4 > 200 * 1024) {
    set_error("lift: constant table of %d x %d words exceeds 200 KB", r, L);
    return FHE_EINVAL;
  }
  ProfScope ps(ctx, FHE_K_LIFT, 1, st);
  if (lift_tc_launch(ctx, src, L, src_pstride, src_bstride, dst, dst_pstride, dst_bstride, npoly, nbatch, r, sbits,
                     item_bits, st))
    return FHE_OK;
#define FHE_LIFT_CASE(B)                                                                 \
  if (L <= B) {                                                                          \
    lift_launch<B>(ctx, src, L, src_pstride, src_bstride, dst, dst_pstride, dst_bstride, \
                   npoly, nbatch, r, sbits, item_bits, st);                              \
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

int launch_lift(const fhe_ctx* ctx, const uint32_t* src, int L, size_t src_pstride, size_t src_bstride,
                uint32_t* dst, size_t dst_pstride, size_t dst_bstride, int npoly, int nbatch, int r,
                cudaStream_t st) {
  return lift_any(ctx, src, L, src_pstride, src_bstride, dst, dst_pstride, dst_bstride, npoly, nbatch, r, 0, nullptr,
                  st);
}

int launch_lift_signed(const fhe_ctx* ctx, const uint32_t* src, int L, size_t src_pstride, size_t src_bstride,
                       uint32_t* dst, size_t dst_pstride, size_t dst_bstride, int npoly, int nbatch, int r, int sbits,
                       const int32_t* item_bits, cudaStream_t st) {
  if (sbits < 1 && !item_bits) {
    set_error("lift (signed): no sign bit position");
    return FHE_EINVAL;
  }
  return lift_any(ctx, src, L, src_pstride, src_bstride, dst, dst_pstride, dst_bstride, npoly, nbatch, r, sbits,
                  item_bits, st);
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
