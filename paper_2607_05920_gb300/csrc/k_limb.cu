// Transform-domain pointwise products and the limb-domain kernels.
//
// Pointwise (Sec. 5 "element-wise arithmetic in the NTT domain"): Montgomery
// products a b 2^-32 (Montgomery 1985); the 2^-32 is undone by the inverse
// transform's scale N^-1 2^32 (applied in the reconstruction), so every
// transform-domain product below is exactly one Montgomery product deep.  The tensor product uses Karatsuba (Sec. 5
// "Karatsuba Polynomial Multiplication") on the transformed operands:
// D0 = B1 B2, D2 = A1 A2, D1 = (A1 + B1)(A2 + B2) - D0 - D2.
//
// Limb-domain kernels (Sec. 5: add, subtract, negate stay in limb form;
// rescale is a rounded right shift; the automorphism is a signed gather).
// Every limb kernel gives one thread one coefficient and walks its limbs,
// so each limb row is read and written with coalesced accesses.
#include "common.cuh"

namespace fhe {

// -------------------------------------------------------------- pointwise
__global__ void k_pw_tensor(uint32_t* __restrict__ X, int r, int N, const uint32_t* __restrict__ qtab,
                            const uint32_t* __restrict__ qinv) {
  const int k = blockIdx.y, b = blockIdx.z;
  const int n4 = blockIdx.x * blockDim.x + threadIdx.x;
  if (n4 * 4 >= N) return;
  const uint32_t q = __ldg(qtab + k), qi = __ldg(qinv + k);
  const size_t rowN = (size_t)r * N;
  uint32_t* base = X + (size_t)b * 4 * rowN + (size_t)k * N;
  uint4* pb1 = (uint4*)(base) + n4;
  uint4* pa1 = (uint4*)(base + rowN) + n4;
  uint4* pb2 = (uint4*)(base + 2 * rowN) + n4;
  const uint4* pa2 = (const uint4*)(base + 3 * rowN) + n4;
  uint4 B1 = *pb1, A1 = *pa1, B2 = *pb2, A2 = *pa2;
  uint4 D0, D1, D2;
#define FHE_KARA(c)                                                             \
  {                                                                             \
    const uint32_t d0 = mont_mul(B1.c, B2.c, q, qi);                            \
    const uint32_t d2 = mont_mul(A1.c, A2.c, q, qi);                            \
    const uint32_t s = mont_mul(add_mod(A1.c, B1.c, q), add_mod(A2.c, B2.c, q), q, qi); \
    D0.c = d0;                                                                  \
    D2.c = d2;                                                                  \
    D1.c = sub_mod(sub_mod(s, d0, q), d2, q);                                   \
  }
  FHE_KARA(x) FHE_KARA(y) FHE_KARA(z) FHE_KARA(w)
#undef FHE_KARA
  *pb1 = D0;
  *pa1 = D1;
  *pb2 = D2;
}

__global__ void k_pw_key(uint32_t* __restrict__ Y, const uint32_t* __restrict__ K, int krows, int r, int N,
                         const uint32_t* __restrict__ qtab, const uint32_t* __restrict__ qinv) {
  const int k = blockIdx.y, b = blockIdx.z;
  const int n4 = blockIdx.x * blockDim.x + threadIdx.x;
  if (n4 * 4 >= N) return;
  const uint32_t q = __ldg(qtab + k), qi = __ldg(qinv + k);
  uint4* y0 = (uint4*)(Y + (size_t)b * 2 * r * N + (size_t)k * N) + n4;
  uint4* y1 = (uint4*)(Y + (size_t)b * 2 * r * N + (size_t)(r + k) * N) + n4;
  const uint4 kb = __ldg((const uint4*)(K + (size_t)k * N) + n4);
  const uint4 ka = __ldg((const uint4*)(K + (size_t)(krows + k) * N) + n4);
  const uint4 d = *y0;
  uint4 o0, o1;
  o0.x = mont_mul(d.x, kb.x, q, qi); o1.x = mont_mul(d.x, ka.x, q, qi);
  o0.y = mont_mul(d.y, kb.y, q, qi); o1.y = mont_mul(d.y, ka.y, q, qi);
  o0.z = mont_mul(d.z, kb.z, q, qi); o1.z = mont_mul(d.z, ka.z, q, qi);
  o0.w = mont_mul(d.w, kb.w, q, qi); o1.w = mont_mul(d.w, ka.w, q, qi);
  *y0 = o0;
  *y1 = o1;
}

__global__ void k_pw_mul(uint32_t* __restrict__ Z, size_t z_bstride, const uint32_t* __restrict__ A, size_t a_bstride,
                         const uint32_t* __restrict__ B, size_t b_bstride, int r, int N,
                         const uint32_t* __restrict__ qtab, const uint32_t* __restrict__ qinv) {
  const int k = blockIdx.y, b = blockIdx.z;
  const int n4 = blockIdx.x * blockDim.x + threadIdx.x;
  if (n4 * 4 >= N) return;
  const uint32_t q = __ldg(qtab + k), qi = __ldg(qinv + k);
  const uint4 a = *((const uint4*)(A + (size_t)b * a_bstride + (size_t)k * N) + n4);
  const uint4 c = *((const uint4*)(B + (size_t)b * b_bstride + (size_t)k * N) + n4);
  uint4 o;
  o.x = mont_mul(a.x, c.x, q, qi);
  o.y = mont_mul(a.y, c.y, q, qi);
  o.z = mont_mul(a.z, c.z, q, qi);
  o.w = mont_mul(a.w, c.w, q, qi);
  *((uint4*)(Z + (size_t)b * z_bstride + (size_t)k * N) + n4) = o;
}

static dim3 pw_grid(int N, int r, int nbatch, int threads) {
  return dim3((N / 4 + threads - 1) / threads, r, nbatch);
}

int launch_pointwise_tensor(const fhe_ctx* ctx, uint32_t* X, int r, int nbatch, cudaStream_t st) {
  const int threads = 128;
  if (r > 65535 || nbatch > 65535 || ctx->N < 4) return FHE_EINVAL;
  ProfScope ps(ctx, FHE_K_POINTWISE, 1, st);
  k_pw_tensor<<<pw_grid(ctx->N, r, nbatch, threads), threads, 0, st>>>(X, r, ctx->N, ctx->d_q, ctx->d_qinv);
  return FHE_OK;
}
int launch_pointwise_key(const fhe_ctx* ctx, uint32_t* Y, const uint32_t* K, int krows, int r, int nbatch,
                         cudaStream_t st) {
  const int threads = 128;
  if (r > krows || nbatch > 65535 || ctx->N < 4) return FHE_EINVAL;
  ProfScope ps(ctx, FHE_K_POINTWISE, 1, st);
  k_pw_key<<<pw_grid(ctx->N, r, nbatch, threads), threads, 0, st>>>(Y, K, krows, r, ctx->N, ctx->d_q, ctx->d_qinv);
  return FHE_OK;
}
int launch_pointwise_mul(const fhe_ctx* ctx, uint32_t* Z, const uint32_t* A, size_t a_bstride, const uint32_t* B,
                         size_t b_bstride, int r, int nbatch, cudaStream_t st) {
  const int threads = 128;
  if (nbatch > 65535 || ctx->N < 4) return FHE_EINVAL;
  ProfScope ps(ctx, FHE_K_POINTWISE, 1, st);
  k_pw_mul<<<pw_grid(ctx->N, r, nbatch, threads), threads, 0, st>>>(Z, (size_t)r * ctx->N, A, a_bstride, B,
                                                                     b_bstride, r, ctx->N, ctx->d_q, ctx->d_qinv);
  return FHE_OK;
}
int launch_pointwise_mul_strided(const fhe_ctx* ctx, uint32_t* Z, size_t z_bstride, const uint32_t* A,
                                 size_t a_bstride, const uint32_t* B, size_t b_bstride, int r, int nbatch,
                                 cudaStream_t st) {
  const int threads = 128;
  if (nbatch > 65535 || ctx->N < 4) return FHE_EINVAL;
  ProfScope ps(ctx, FHE_K_POINTWISE, 1, st);
  k_pw_mul<<<pw_grid(ctx->N, r, nbatch, threads), threads, 0, st>>>(Z, z_bstride, A, a_bstride, B, b_bstride, r,
                                                                     ctx->N, ctx->d_q, ctx->d_qinv);
  return FHE_OK;
}

// ----------------------------------------------------------- limb kernels
__device__ __forceinline__ uint32_t mask_of(int l, int bits) {
  const int rem = bits - 32 * l;
  return rem >= 32 ? 0xFFFFFFFFu : (rem <= 0 ? 0u : ((1u << rem) - 1u));
}

// out = round(in / 2^k) mod 2^(logQ - k): (x + 2^(k-1)) >> k, halves up (rescaleBy, Sec. 6)
__global__ void k_rescale(const uint32_t* __restrict__ in, int Lin, uint32_t* __restrict__ out, int Lout, int k,
                          int out_bits, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const uint32_t* x = in + (size_t)blockIdx.y * Lin * N + n;
  uint32_t* y = out + (size_t)blockIdx.y * Lout * N + n;
  // carry of x + 2^(k-1) into limb kl = k / 32 and above
  const int kl = k >> 5, kb = k & 31;
  const int rl = (k - 1) >> 5;
  const uint32_t radd = 1u << ((k - 1) & 31);
  uint32_t carry = 0;
  for (int l = rl; l < kl; ++l) {  // limbs below the cut: only their carry matters
    const uint32_t v = __ldg(x + (size_t)l * N);
    const uint32_t a = (l == rl) ? radd : 0u;
    const uint64_t s = (uint64_t)v + a + carry;
    carry = (uint32_t)(s >> 32);
  }
  // limbs from kl upward of (x + 2^(k-1)), shifted right by kb
  uint32_t cur;
  {
    const uint32_t v = kl < Lin ? __ldg(x + (size_t)kl * N) : 0u;
    const uint32_t a = (kl == rl) ? radd : 0u;
    const uint64_t s = (uint64_t)v + a + carry;
    cur = (uint32_t)s;
    carry = (uint32_t)(s >> 32);
  }
  for (int l = 0; l < Lout; ++l) {
    const int src = kl + l + 1;
    const uint32_t v = src < Lin ? __ldg(x + (size_t)src * N) : 0u;
    const uint64_t s = (uint64_t)v + carry;
    const uint32_t nxt = (uint32_t)s;
    carry = (uint32_t)(s >> 32);
    const uint32_t o = kb ? __funnelshift_r(cur, nxt, kb) : cur;
    y[(size_t)l * N] = o & mask_of(l, out_bits);
    cur = nxt;
  }
}

__global__ void k_moddown(const uint32_t* __restrict__ in, int Lin, uint32_t* __restrict__ out, int Lout,
                          int out_bits, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const uint32_t* x = in + (size_t)blockIdx.y * Lin * N + n;
  uint32_t* y = out + (size_t)blockIdx.y * Lout * N + n;
  for (int l = 0; l < Lout; ++l) y[(size_t)l * N] = (l < Lin ? __ldg(x + (size_t)l * N) : 0u) & mask_of(l, out_bits);
}

// mode 0: a + b, 1: a - b, 2: -a  (mod 2^bits)
__global__ void k_addsub(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b, uint32_t* __restrict__ out,
                         int L, int bits, int mode, int N, int b_polys) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const size_t off = (size_t)blockIdx.y * L * N + n;
  // b_polys > 0: b holds that many polynomials, reused for every ciphertext (broadcast mode)
  const size_t boff = b_polys > 0 ? (size_t)(blockIdx.y % b_polys) * L * N + n : off;
  uint32_t c = (mode == 0) ? 0u : 1u;  // subtraction: x + ~y + 1
  for (int l = 0; l < L; ++l) {
    const size_t i = off + (size_t)l * N;
    uint32_t x, y;
    if (mode == 2) {
      x = 0;
      y = ~a[i];
    } else {
      const uint32_t bv = b[boff + (size_t)l * N];
      x = a[i];
      y = (mode == 0) ? bv : ~bv;
    }
    const uint64_t s = (uint64_t)x + y + c;
    c = (uint32_t)(s >> 32);
    out[i] = (uint32_t)s & mask_of(l, bits);
  }
}

__global__ void k_mult_const(const uint32_t* __restrict__ in, int32_t cst, uint32_t* __restrict__ out, int L,
                             int bits, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const size_t off = (size_t)blockIdx.y * L * N + n;
  const uint32_t m = cst < 0 ? (uint32_t)(-(int64_t)cst) : (uint32_t)cst;
  // |c| x, then negate if c < 0 (two's complement mod 2^bits)
  uint32_t carry = 0, neg = cst < 0 ? 1u : 0u;
  for (int l = 0; l < L; ++l) {
    const size_t i = off + (size_t)l * N;
    const uint64_t t = (uint64_t)in[i] * m + carry;
    carry = (uint32_t)(t >> 32);
    uint32_t v = (uint32_t)t;
    if (cst < 0) {
      const uint64_t s = (uint64_t)(~v) + neg;
      v = (uint32_t)s;
      neg = (uint32_t)(s >> 32);
    }
    out[i] = v & mask_of(l, bits);
  }
}

// kappa_g on limb polynomials: output coefficient e receives +-input i with i g = e (mod 2N)
__global__ void k_automorph(const uint32_t* __restrict__ in, size_t in_pstride, uint32_t* __restrict__ out,
                            size_t out_pstride, int L, int bits, uint32_t ginv, int logN) {
  const int N = 1 << logN;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N) return;
  const uint32_t i2 = (uint32_t)(((uint64_t)e * ginv) & (uint64_t)(2 * N - 1));  // source exponent mod 2N
  const bool neg = i2 >= (uint32_t)N;
  const uint32_t i = neg ? i2 - N : i2;
  const uint32_t* x = in + (size_t)blockIdx.y * in_pstride + i;
  uint32_t* y = out + (size_t)blockIdx.y * out_pstride + e;
  uint32_t c = 1;
  for (int l = 0; l < L; ++l) {
    uint32_t v = __ldg(x + (size_t)l * N);
    if (neg) {
      const uint64_t s = (uint64_t)(~v) + c;
      v = (uint32_t)s;
      c = (uint32_t)(s >> 32);
    }
    y[(size_t)l * N] = v & mask_of(l, bits);
  }
}

__global__ void k_automorph_small(const int32_t* __restrict__ in, int32_t* __restrict__ out, uint32_t ginv,
                                  int logN) {
  const int N = 1 << logN;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N) return;
  const uint32_t i2 = (uint32_t)(((uint64_t)e * ginv) & (uint64_t)(2 * N - 1));
  out[e] = i2 >= (uint32_t)N ? -in[i2 - N] : in[i2];
}

// out = (-t + e + (sf << logP)) mod 2^bits; t: Lt two's complement limbs, sf: Ls two's complement limbs
__global__ void k_key_combine(const uint32_t* __restrict__ t, int Lt, const int32_t* __restrict__ e,
                              const uint32_t* __restrict__ sf, int Ls, int logP, uint32_t* __restrict__ out,
                              int bits, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int L = (bits + 31) / 32;
  const int32_t ev = e[n];
  const uint32_t text = Lt > 0 && (t[(size_t)(Lt - 1) * N + n] >> 31) ? 0xFFFFFFFFu : 0u;
  const uint32_t sext = Ls > 0 && (sf[(size_t)(Ls - 1) * N + n] >> 31) ? 0xFFFFFFFFu : 0u;
  const int pl = logP >> 5, pb = logP & 31;
  uint32_t c1 = 1, c2 = 0, c3 = 0;  // -t = ~t + 1 ; + e ; + sf << logP
  for (int l = 0; l < L; ++l) {
    const uint32_t tv = l < Lt ? t[(size_t)l * N + n] : text;
    uint64_t s = (uint64_t)(~tv) + c1;
    uint32_t v = (uint32_t)s;
    c1 = (uint32_t)(s >> 32);
    const uint32_t ew = l == 0 ? (uint32_t)ev : (ev < 0 ? 0xFFFFFFFFu : 0u);
    s = (uint64_t)v + ew + c2;
    v = (uint32_t)s;
    c2 = (uint32_t)(s >> 32);
    // limb l of (sf << logP)
    const int a = l - pl;
    uint32_t lo = (a >= 0) ? (a < Ls ? sf[(size_t)a * N + n] : sext) : 0u;
    uint32_t lo1 = (a - 1 >= 0) ? (a - 1 < Ls ? sf[(size_t)(a - 1) * N + n] : sext) : 0u;
    const uint32_t sw = pb ? __funnelshift_l(lo1, lo, pb) : lo;
    s = (uint64_t)v + sw + c3;
    v = (uint32_t)s;
    c3 = (uint32_t)(s >> 32);
    out[(size_t)l * N + n] = v & mask_of(l, bits);
  }
}

// b_0 += value 2^shift (mod 2^bits) for each ciphertext of the batch (addconst)
__global__ void k_add_const(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t value,
                            const int64_t* __restrict__ values, int shift, int L, int bits, int N, int cnum) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cnum) return;
  if (values) value = values[c];  // pairwise: one constant per ciphertext
  const size_t base = (size_t)c * 2 * L * N;  // coefficient 0 of poly 0
  const int sl = shift >> 5, sb = shift & 31;
  const uint64_t v = (uint64_t)value;
  const uint32_t ext = value < 0 ? 0xFFFFFFFFu : 0u;
  // limb j of value << shift: bits of the sign-extended value
  uint32_t carry = 0;
  for (int l = 0; l < L; ++l) {
    const int a = l - sl;
    auto word = [&](int w) -> uint32_t {
      if (w < 0) return 0u;
      if (w == 0) return (uint32_t)v;
      if (w == 1) return (uint32_t)(v >> 32);
      return ext;
    };
    const uint32_t hi = word(a), lo = word(a - 1);
    const uint32_t add = sb ? __funnelshift_l(lo, hi, sb) : hi;
    const uint64_t s = (uint64_t)in[base + (size_t)l * N] + add + carry;
    carry = (uint32_t)(s >> 32);
    out[base + (size_t)l * N] = (uint32_t)s & mask_of(l, bits);
  }
}

static dim3 limb_grid(int N, int y, int threads) { return dim3((N + threads - 1) / threads, y); }

int launch_add_const(const fhe_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t value, const int64_t* values,
                     int shift, int logQ, int cnum, cudaStream_t st) {
  ProfScope ps(ctx, FHE_K_LIMB, 1, st);
  k_add_const<<<(cnum + 127) / 128, 128, 0, st>>>(in, out, value, values, shift, limbs_for_bits(logQ), logQ, ctx->N,
                                                  cnum);
  return FHE_OK;
}

// Multiplication by the monomial X^k (0 <= k < N) in Z_Q[X]/(X^N + 1): coefficient i moves to
// i + k, negated (two's complement mod 2^bits) when it wraps past X^N = -1.  k = N/2 is imult
// (X^(N/2) evaluates to the imaginary unit at every slot's root).
__global__ void k_monomial(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int L, int bits, int k,
                           int logN) {
  const int N = 1 << logN;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N) return;
  const bool neg = e < k;
  const int i = neg ? e - k + N : e - k;
  const uint32_t* x = in + (size_t)blockIdx.y * L * N + i;
  uint32_t* y = out + (size_t)blockIdx.y * L * N + e;
  uint32_t c = 1;
  for (int l = 0; l < L; ++l) {
    uint32_t v = __ldg(x + (size_t)l * N);
    if (neg) {
      const uint64_t s = (uint64_t)(~v) + c;
      v = (uint32_t)s;
      c = (uint32_t)(s >> 32);
    }
    y[(size_t)l * N] = v & mask_of(l, bits);
  }
}

int launch_monomial(const fhe_ctx* ctx, const uint32_t* in, uint32_t* out, int logQ, int k, int npolys,
                    cudaStream_t st) {
  if (npolys > 65535 || k < 0 || k >= ctx->N || in == out) return FHE_EINVAL;
  ProfScope ps(ctx, FHE_K_LIMB, 1, st);
  k_monomial<<<limb_grid(ctx->N, npolys, 128), 128, 0, st>>>(in, out, limbs_for_bits(logQ), logQ, k, ctx->prm.logN);
  return FHE_OK;
}

int launch_rescale(const fhe_ctx* ctx, const uint32_t* in, int logQ_in, uint32_t* out, int k, int npolys,
                   cudaStream_t st) {
  if (k < 1 || k >= logQ_in || npolys > 65535) return FHE_EINVAL;
  const int Lin = limbs_for_bits(logQ_in), Lout = limbs_for_bits(logQ_in - k);
  ProfScope ps(ctx, FHE_K_LIMB, 1, st);
  k_rescale<<<limb_grid(ctx->N, npolys, 128), 128, 0, st>>>(in, Lin, out, Lout, k, logQ_in - k, ctx->N);
  return FHE_OK;
}
int launch_moddown(const fhe_ctx* ctx, const uint32_t* in, int logQ_in, uint32_t* out, int logQ_out, int npolys,
                   cudaStream_t st) {
  if (logQ_out < 1 || logQ_out > logQ_in || npolys > 65535) return FHE_EINVAL;
  ProfScope ps(ctx, FHE_K_LIMB, 1, st);
  k_moddown<<<limb_grid(ctx->N, npolys, 128), 128, 0, st>>>(in, limbs_for_bits(logQ_in), out,
                                                            limbs_for_bits(logQ_out), logQ_out, ctx->N);
  return FHE_OK;
}
int launch_addsub(const fhe_ctx* ctx, const uint32_t* a, const uint32_t* b, uint32_t* out, int logQ, int npolys,
                  int mode, cudaStream_t st, int b_polys) {
  if (npolys > 65535) return FHE_EINVAL;
  ProfScope ps(ctx, FHE_K_LIMB, 1, st);
  k_addsub<<<limb_grid(ctx->N, npolys, 128), 128, 0, st>>>(a, b, out, limbs_for_bits(logQ), logQ, mode, ctx->N,
                                                           b_polys);
  return FHE_OK;
}
int launch_mult_const(const fhe_ctx* ctx, const uint32_t* in, int32_t c, uint32_t* out, int logQ, int npolys,
                      cudaStream_t st) {
  if (npolys > 65535) return FHE_EINVAL;
  ProfScope ps(ctx, FHE_K_LIMB, 1, st);
  k_mult_const<<<limb_grid(ctx->N, npolys, 128), 128, 0, st>>>(in, c, out, limbs_for_bits(logQ), logQ, ctx->N);
  return FHE_OK;
}
static uint32_t inv_mod_pow2(uint32_t g, uint32_t two_n) {
  // g odd: inverse mod 2N by Newton iteration mod 2^32, then reduce
  uint32_t x = 1;
  for (int i = 0; i < 5; ++i) x *= 2u - g * x;
  return x & (two_n - 1);
}
int launch_automorph(const fhe_ctx* ctx, const uint32_t* in, size_t in_pstride, uint32_t* out, size_t out_pstride,
                     int L, int logQ, uint32_t g, int npolys, cudaStream_t st) {
  if (npolys > 65535 || (g & 1u) == 0) return FHE_EINVAL;
  const uint32_t ginv = inv_mod_pow2(g, 2u * ctx->N);
  ProfScope ps(ctx, FHE_K_LIMB, 1, st);
  k_automorph<<<limb_grid(ctx->N, npolys, 128), 128, 0, st>>>(in, in_pstride, out, out_pstride, L, logQ, ginv,
                                                              ctx->prm.logN);
  return FHE_OK;
}
int launch_automorph_small(const fhe_ctx* ctx, const int32_t* in, int32_t* out, uint32_t g, cudaStream_t st) {
  const uint32_t ginv = inv_mod_pow2(g, 2u * ctx->N);
  ProfScope ps(ctx, FHE_K_LIMB, 1, st);
  k_automorph_small<<<limb_grid(ctx->N, 1, 128), 128, 0, st>>>(in, out, ginv, ctx->prm.logN);
  return FHE_OK;
}
int launch_key_combine(const fhe_ctx* ctx, const uint32_t* t, int Lt, const int32_t* e, const uint32_t* sfrom,
                       int Ls, int logP, uint32_t* out, int bits, cudaStream_t st) {
  ProfScope ps(ctx, FHE_K_LIMB, 1, st);
  k_key_combine<<<limb_grid(ctx->N, 1, 128), 128, 0, st>>>(t, Lt, e, sfrom, Ls, logP, out, bits, ctx->N);
  return FHE_OK;
}

}  // namespace fhe
