// BGV on one odd big modulus (no RNS at rest): reduction modulo the chain
// moduli Q_l = q0 r^l, the delta-corrected division by P of the key switch,
// the modulus switch Q_l -> Q_{l-1}, and decryption modulo t.
//
// The paper runs one CKKS-BGV abstraction (Sec. 6) without printing BGV's
// formulas; these kernels implement the standard BGV definitions on big
// integers:
//   key switch   KS(y) = (y + delta) / P,  delta = t [(-y) t^-1]_P  (centred)
//   mod switch   c' = (c + delta') / r,     delta' = t [(-c) t^-1]_r (centred)
//   decrypt      [[b + a s]_{Q_l}]_t with the centred representative.
//
// Ring products (tensor, key switching, encryption, decryption) run through
// the same lift / NTT / CRT kernels as CKKS; the CRT emits the exact signed
// product (two's complement limbs) and the kernels here finish modulo Q_l.
// One thread owns one coefficient; big integers of up to kBgvLimbs limbs
// live in registers.
//
// Reduction of an n-limb value X modulo Q (Q of up to 16 limbs): with the
// precomputed R_j = 2^(32 j) mod Q, S = sum_j X_j R_j (+ (-2^(32 n)) mod Q
// when X is negative) is congruent to X and below (n + 1) 2^32 Q; its
// quotient by Q (< 2^38) is estimated from the top limbs in double precision
// (error at most one) and corrected with one conditional add or subtract.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "bgv.cuh"

namespace fhe {

constexpr int KB = kBgvLimbs;

// S (KB + 2 limbs) += v * R (KB limbs)
__device__ __forceinline__ void acc_mul_word(uint32_t (&S)[KB + 2], uint32_t v, const uint32_t* __restrict__ R) {
  uint32_t c = 0;
#pragma unroll
  for (int l = 0; l < KB; ++l) {
    uint64_t t = (uint64_t)v * __ldg(R + l) + S[l];
    t += c;
    S[l] = (uint32_t)t;
    c = (uint32_t)(t >> 32);
  }
  uint64_t t = (uint64_t)S[KB] + c;
  S[KB] = (uint32_t)t;
  S[KB + 1] += (uint32_t)(t >> 32);
}

// S += W (KB limbs), W in global memory
__device__ __forceinline__ void acc_add(uint32_t (&S)[KB + 2], const uint32_t* __restrict__ W) {
  uint32_t c = 0;
#pragma unroll
  for (int l = 0; l < KB; ++l) {
    const uint64_t t = (uint64_t)S[l] + __ldg(W + l) + c;
    S[l] = (uint32_t)t;
    c = (uint32_t)(t >> 32);
  }
  const uint64_t t = (uint64_t)S[KB] + c;
  S[KB] = (uint32_t)t;
  S[KB + 1] += (uint32_t)(t >> 32);
}

// S mod Q for S < 2^38 Q; result in out[0, KB)
__device__ __forceinline__ void finish_mod(uint32_t (&S)[KB + 2], const BgvLevel& L, uint32_t (&out)[KB]) {
  const int nq = L.nl;
  // top limbs of S at the position of Q's top limb
  uint32_t s2 = 0, s1 = 0, s0 = 0, sm = 0;
#pragma unroll
  for (int l = 0; l < KB + 2; ++l) {
    if (l == nq + 1) s2 = S[l];
    if (l == nq) s1 = S[l];
    if (l == nq - 1) s0 = S[l];
    if (l == nq - 2) sm = S[l];
  }
  const double sd = ((double)s2 * 4294967296.0 + (double)s1) * 4294967296.0 + (double)s0 + (double)sm * 2.3283064365386963e-10;
  double qd = floor(sd / L.qtop);
  if (qd < 0) qd = 0;
  const uint64_t qh = (uint64_t)qd;
  const uint32_t q0 = (uint32_t)qh, q1 = (uint32_t)(qh >> 32);
  // S -= qh * Q
  uint32_t borrow = 0, c0 = 0, c1 = 0;
#pragma unroll
  for (int l = 0; l < KB + 2; ++l) {
    const uint32_t ql = l < KB ? L.q[l] : 0u;
    const uint32_t qlm1 = (l >= 1 && l - 1 < KB) ? L.q[l - 1] : 0u;
    // limb l of qh * Q = lo(q0 ql) + hi(q0 q_{l-1}) + lo(q1 q_{l-1}) + hi(q1 q_{l-2}) + carries
    const uint64_t p0 = (uint64_t)q0 * ql + c0;
    c0 = (uint32_t)(p0 >> 32);
    const uint64_t p1 = (uint64_t)q1 * qlm1 + c1 + (uint32_t)p0;
    c1 = (uint32_t)(p1 >> 32);
    const uint32_t tl = (uint32_t)p1;
    const uint64_t d = (uint64_t)S[l] - tl - borrow;
    S[l] = (uint32_t)d;
    borrow = (uint32_t)(d >> 63);
  }
  if (borrow) {  // over-estimated: add Q back
    uint32_t c = 0;
#pragma unroll
    for (int l = 0; l < KB + 2; ++l) {
      const uint64_t t = (uint64_t)S[l] + (l < KB ? L.q[l] : 0u) + c;
      S[l] = (uint32_t)t;
      c = (uint32_t)(t >> 32);
    }
  }
  // S >= Q ?
  bool ge = true;
#pragma unroll
  for (int l = KB + 1; l >= 0; --l) {
    const uint32_t ql = l < KB ? L.q[l] : 0u;
    if (S[l] != ql) {
      ge = S[l] > ql;
      break;
    }
  }
  if (ge) {
    uint32_t bo = 0;
#pragma unroll
    for (int l = 0; l < KB + 2; ++l) {
      const uint64_t d = (uint64_t)S[l] - (l < KB ? L.q[l] : 0u) - bo;
      S[l] = (uint32_t)d;
      bo = (uint32_t)(d >> 63);
    }
  }
#pragma unroll
  for (int l = 0; l < KB; ++l) out[l] = S[l];
}

// value (nx limbs at x[j * stride], two's complement if is_signed) + small, reduced mod Q_l
__device__ void mod_q(const uint32_t* __restrict__ x, size_t stride, int nx, bool is_signed, int64_t small,
                      const BgvLevel& L, uint32_t (&out)[KB]) {
  uint32_t S[KB + 2];
#pragma unroll
  for (int l = 0; l < KB + 2; ++l) S[l] = 0;
  uint32_t top = 0;
  for (int j = 0; j < nx; ++j) {
    const uint32_t v = __ldg(x + (size_t)j * stride);
    top = v;
    acc_mul_word(S, v, L.R[j]);
  }
  if (is_signed && (top >> 31)) acc_add(S, L.negR[nx]);
  if (small != 0) {
    const uint64_t a = small < 0 ? (uint64_t)(-small) : (uint64_t)small;
    if (small > 0) {
      acc_mul_word(S, (uint32_t)a, L.R[0]);
      acc_mul_word(S, (uint32_t)(a >> 32), L.R[1]);
    } else {  // add Q - |small| mod Q = |small| * (-1 mod Q): use the -R_0 row
      acc_mul_word(S, (uint32_t)a, L.negR[0]);
      acc_mul_word(S, (uint32_t)(a >> 32), L.negR[1]);
    }
  }
  finish_mod(S, L, out);
}

// out = (a + b) mod Q for canonical a, b
__device__ __forceinline__ void add_mod_q(uint32_t (&a)[KB], const uint32_t (&b)[KB], const BgvLevel& L) {
  uint32_t S[KB + 2];
  uint32_t c = 0;
#pragma unroll
  for (int l = 0; l < KB; ++l) {
    const uint64_t t = (uint64_t)a[l] + b[l] + c;
    S[l] = (uint32_t)t;
    c = (uint32_t)(t >> 32);
  }
  S[KB] = c;
  S[KB + 1] = 0;
  bool ge = true;
#pragma unroll
  for (int l = KB + 1; l >= 0; --l) {
    const uint32_t ql = l < KB ? L.q[l] : 0u;
    if (S[l] != ql) {
      ge = S[l] > ql;
      break;
    }
  }
  uint32_t bo = 0;
#pragma unroll
  for (int l = 0; l < KB; ++l) {
    if (ge) {
      const uint64_t d = (uint64_t)S[l] - L.q[l] - bo;
      a[l] = (uint32_t)d;
      bo = (uint32_t)(d >> 63);
    } else {
      a[l] = S[l];
    }
  }
}

__device__ __forceinline__ void neg_mod_q(uint32_t (&a)[KB], const BgvLevel& L) {
  bool zero = true;
#pragma unroll
  for (int l = 0; l < KB; ++l) zero = zero && a[l] == 0;
  if (zero) return;
  uint32_t bo = 0;
#pragma unroll
  for (int l = 0; l < KB; ++l) {
    const uint64_t d = (uint64_t)L.q[l] - a[l] - bo;
    a[l] = (uint32_t)d;
    bo = (uint32_t)(d >> 63);
  }
}

__device__ __forceinline__ void load_canon(const uint32_t* __restrict__ p, size_t stride, int nl, uint32_t (&a)[KB]) {
#pragma unroll
  for (int l = 0; l < KB; ++l) a[l] = l < nl ? __ldg(p + (size_t)l * stride) : 0u;
}

// -------------------------------------------------------------- kernels
// out = (sign X + t e + add) mod Q_level; X two's complement (nx limbs) or unsigned
__global__ void k_bgv_reduce(const uint32_t* __restrict__ X, int nx, size_t x_pstride, size_t x_bstride, int npoly,
                             bool is_signed, bool negate, const int32_t* __restrict__ e0, const int32_t* __restrict__ e1,
                             size_t e_bstride, const uint32_t* __restrict__ add, int add_polys, size_t add_pstride,
                             size_t add_bstride, uint32_t* __restrict__ out, size_t o_pstride, size_t o_bstride, int N,
                             const BgvLevel* __restrict__ lv, uint32_t t) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int poly = blockIdx.y % npoly, b = blockIdx.y / npoly;
  const BgvLevel& L = *lv;
  uint32_t c[KB];
  mod_q(X + (size_t)b * x_bstride + (size_t)poly * x_pstride + n, N, nx, is_signed, 0, L, c);
  if (negate) neg_mod_q(c, L);
  const int32_t* e = poly == 0 ? e0 : (poly == 1 ? e1 : nullptr);
  if (e) {
    const int64_t te = (int64_t)t * __ldg(e + (size_t)b * e_bstride + n);
    if (te != 0) {
      uint32_t w[KB];
      // (t e) mod Q as a canonical value
      const uint64_t a = te < 0 ? (uint64_t)(-te) : (uint64_t)te;
#pragma unroll
      for (int l = 0; l < KB; ++l) w[l] = l == 0 ? (uint32_t)a : (l == 1 ? (uint32_t)(a >> 32) : 0u);
      if (te < 0) neg_mod_q(w, L);
      add_mod_q(c, w, L);
    }
  }
  if (add && poly < add_polys) {
    uint32_t w[KB];
    load_canon(add + (size_t)b * add_bstride + (size_t)poly * add_pstride + n, N, L.nl, w);
    add_mod_q(c, w, L);
  }
  uint32_t* o = out + (size_t)b * o_bstride + (size_t)poly * o_pstride + n;
#pragma unroll
  for (int l = 0; l < KB; ++l)
    if (l < L.nl) o[(size_t)l * N] = c[l];
}

// (d + (Y + delta) / P) mod Q_level; Y two's complement (ny limbs), d canonical
__global__ void k_bgv_keyswitch(const uint32_t* __restrict__ Y, int ny, size_t y_pstride, size_t y_bstride,
                                const uint32_t* __restrict__ d, int add_polys, size_t d_pstride, size_t d_bstride,
                                uint32_t* __restrict__ out, size_t o_pstride, size_t o_bstride, int N,
                                const BgvLevel* __restrict__ lv, const BgvConsts* __restrict__ cs,
                                uint32_t* __restrict__ scratch, size_t s_pstride, size_t s_bstride) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int poly = blockIdx.y % 2, b = blockIdx.y / 2;
  const BgvLevel& L = *lv;
  const int logP = cs->logP, lp = (logP + 31) >> 5;
  const uint32_t t = cs->t;
  const uint32_t* y = Y + (size_t)b * y_bstride + (size_t)poly * y_pstride + n;
  // low logP bits of Y, u = [(-Y) t^-1] mod 2^logP
  uint32_t lo[KB], w[KB], u[KB];
  const uint32_t topmask = (logP & 31) ? ((1u << (logP & 31)) - 1u) : 0xFFFFFFFFu;
#pragma unroll
  for (int l = 0; l < KB; ++l) lo[l] = l < lp ? __ldg(y + (size_t)l * N) : 0u;
#pragma unroll
  for (int l = 0; l < KB; ++l)
    if (l == lp - 1) lo[l] &= topmask;
  uint32_t cneg = 1;
#pragma unroll
  for (int l = 0; l < KB; ++l) {  // w = -lo mod 2^(32 lp), masked to logP bits
    const uint64_t s = (uint64_t)(~lo[l]) + cneg;
    w[l] = l < lp ? (uint32_t)s : 0u;
    cneg = (uint32_t)(s >> 32);
  }
#pragma unroll
  for (int l = 0; l < KB; ++l)
    if (l == lp - 1) w[l] &= topmask;
#pragma unroll
  for (int l = 0; l < KB; ++l) u[l] = 0;
#pragma unroll
  for (int i = 0; i < KB; ++i) {  // u = w * tinvP mod 2^(32 lp)
    if (i < lp) {
      uint32_t c = 0;
#pragma unroll
      for (int j = 0; j < KB; ++j) {
        if (i + j < lp) {
          uint64_t tt = (uint64_t)w[i] * __ldg(cs->tinvP + j) + u[i + j];
          tt += c;
          u[i + j] = (uint32_t)tt;
          c = (uint32_t)(tt >> 32);
        }
      }
    }
  }
#pragma unroll
  for (int l = 0; l < KB; ++l)
    if (l == lp - 1) u[l] &= topmask;
  // sign of the centred u: bit logP - 1
  uint32_t ubit = 0;
#pragma unroll
  for (int l = 0; l < KB; ++l)
    if (l == ((logP - 1) >> 5)) ubit = (u[l] >> ((logP - 1) & 31)) & 1u;
  // h = (lo + t u) >> logP, exact small integer
  uint32_t v[KB + 1];
  {
    uint32_t c = 0;
#pragma unroll
    for (int l = 0; l < KB; ++l) {
      uint64_t tt = (uint64_t)t * u[l] + lo[l];
      tt += c;
      v[l] = (uint32_t)tt;
      c = (uint32_t)(tt >> 32);
    }
    v[KB] = c;
  }
  uint64_t h = 0;
#pragma unroll
  for (int l = 0; l < KB; ++l) {
    if (l == (logP >> 5)) {
      const int sb = logP & 31;
      const uint64_t w2 = ((uint64_t)v[l + 1] << 32) | v[l];
      h = sb ? (w2 >> sb) : v[l];
    }
  }
  const int64_t eps = (int64_t)h - (ubit ? (int64_t)t : 0);
  // Z = (Y >> logP) + eps: the shifted limbs go through scratch (two's complement, sign-extended)
  const int sl = logP >> 5, sb = logP & 31;
  const int nz = ny - sl;
  uint32_t* z = scratch + (size_t)b * s_bstride + (size_t)poly * s_pstride + n;
  const uint32_t ytop = __ldg(y + (size_t)(ny - 1) * N);
  const uint32_t ext = (ytop >> 31) ? 0xFFFFFFFFu : 0u;
  for (int j = 0; j < nz; ++j) {
    const uint32_t a0 = __ldg(y + (size_t)(j + sl) * N);
    const uint32_t a1 = (j + sl + 1 < ny) ? __ldg(y + (size_t)(j + sl + 1) * N) : ext;
    z[(size_t)j * N] = sb ? __funnelshift_r(a0, a1, sb) : a0;
  }
  uint32_t c[KB];
  mod_q(z, N, nz, true, eps, L, c);
  if (d && poly < add_polys) {
    uint32_t dd[KB];
    load_canon(d + (size_t)b * d_bstride + (size_t)poly * d_pstride + n, N, L.nl, dd);
    add_mod_q(c, dd, L);
  }
  uint32_t* o = out + (size_t)b * o_bstride + (size_t)poly * o_pstride + n;
#pragma unroll
  for (int l = 0; l < KB; ++l)
    if (l < L.nl) o[(size_t)l * N] = c[l];
}

// Q_l -> Q_{l-1}: c' = (c + t [(-c) t^-1]_r) / r, canonical in, canonical out
__global__ void k_bgv_modswitch(const uint32_t* __restrict__ in, size_t i_pstride, uint32_t* __restrict__ out,
                                size_t o_pstride, int N, const BgvLevel* __restrict__ lv_in,
                                const BgvLevel* __restrict__ lv_out, const BgvConsts* __restrict__ cs) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const BgvLevel& Li = *lv_in;
  const BgvLevel& Lo = *lv_out;
  const uint32_t* x = in + (size_t)blockIdx.y * i_pstride + n;
  uint32_t c[KB];
  load_canon(x, N, Li.nl, c);
  const uint64_t r = cs->r;
  // c mod r
  unsigned __int128 acc = 0;
#pragma unroll
  for (int l = 0; l < KB; ++l) acc += (unsigned __int128)c[l] * Li.rpow[l];
  const uint64_t cr = (uint64_t)(acc % r);
  const uint64_t wneg = cr == 0 ? 0 : r - cr;
  uint64_t uu = (uint64_t)(((unsigned __int128)wneg * cs->tinv_r) % r);
  __int128 us = (__int128)uu;
  if (2 * (unsigned __int128)uu >= r) us -= (__int128)r;  // centred
  const __int128 delta = (__int128)cs->t * us;
  // z = c + delta over KB + 2 limbs, two's complement
  uint32_t z[KB + 2];
  {
    unsigned __int128 dv = (unsigned __int128)delta;  // two's complement bits
    uint32_t carry = 0;
#pragma unroll
    for (int l = 0; l < KB + 2; ++l) {
      const uint32_t dl = l < 4 ? (uint32_t)(dv >> (32 * l)) : (delta < 0 ? 0xFFFFFFFFu : 0u);
      const uint64_t s = (uint64_t)(l < KB ? c[l] : 0u) + dl + carry;
      z[l] = (uint32_t)s;
      carry = (uint32_t)(s >> 32);
    }
  }
  // exact quotient q = z r^-1 mod 2^(32 (KB + 2))
  uint32_t q[KB + 2];
#pragma unroll
  for (int l = 0; l < KB + 2; ++l) q[l] = 0;
#pragma unroll
  for (int i = 0; i < KB + 2; ++i) {
    uint32_t cc = 0;
#pragma unroll
    for (int j = 0; j < KB + 2; ++j) {
      if (i + j < KB + 2) {
        uint64_t tt = (uint64_t)z[i] * __ldg(Li.rinv + j) + q[i + j];
        tt += cc;
        q[i + j] = (uint32_t)tt;
        cc = (uint32_t)(tt >> 32);
      }
    }
  }
  // into [0, Q_{l-1}): the quotient lies in (-t/2, Q_{l-1} + t/2)
  uint32_t res[KB];
  if (q[KB + 1] >> 31) {  // negative: add Q_{l-1}
    uint32_t cc = 0;
#pragma unroll
    for (int l = 0; l < KB; ++l) {
      const uint64_t s = (uint64_t)q[l] + Lo.q[l] + cc;
      res[l] = (uint32_t)s;
      cc = (uint32_t)(s >> 32);
    }
  } else {
#pragma unroll
    for (int l = 0; l < KB; ++l) res[l] = q[l];
    uint32_t zero[KB];
#pragma unroll
    for (int l = 0; l < KB; ++l) zero[l] = 0;
    add_mod_q(res, zero, Lo);  // one conditional subtraction of Q_{l-1}
  }
  uint32_t* o = out + (size_t)blockIdx.y * o_pstride + n;
#pragma unroll
  for (int l = 0; l < KB; ++l)
    if (l < Lo.nl) o[(size_t)l * N] = res[l];
}

// m = [[X + b]_{Q_l}]_t: X two's complement product a s, b canonical; one word per coefficient
__global__ void k_bgv_decrypt(const uint32_t* __restrict__ X, int nx, size_t x_bstride,
                              const uint32_t* __restrict__ bpoly, size_t b_bstride, uint32_t* __restrict__ out,
                              size_t o_bstride, int N, const BgvLevel* __restrict__ lv,
                              const BgvConsts* __restrict__ cs) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int b = blockIdx.y;
  const BgvLevel& L = *lv;
  uint32_t c[KB], w[KB];
  mod_q(X + (size_t)b * x_bstride + n, N, nx, true, 0, L, c);
  load_canon(bpoly + (size_t)b * b_bstride + n, N, L.nl, w);
  add_mod_q(c, w, L);
  // centred: c > Q/2 (Q odd) -> c - Q
  uint32_t dbl[KB + 1];
  uint32_t carry = 0;
#pragma unroll
  for (int l = 0; l < KB; ++l) {
    dbl[l] = (c[l] << 1) | carry;
    carry = c[l] >> 31;
  }
  dbl[KB] = carry;
  bool gt = false;
  {
    bool decided = false;
#pragma unroll
    for (int l = KB; l >= 0; --l) {
      const uint32_t ql = l < KB ? L.q[l] : 0u;
      if (!decided && dbl[l] != ql) {
        gt = dbl[l] > ql;
        decided = true;
      }
    }
  }
  const uint32_t t = cs->t;
  uint64_t m = 0;
#pragma unroll
  for (int l = 0; l < KB; ++l) m = (m + (uint64_t)c[l] * cs->tpow[l]) % t;
  if (gt) m = (m + t - L.q_mod_t) % t;
  out[(size_t)b * o_bstride + n] = (uint32_t)m;
}

// V = sign X + t e + s2 2^logP, out = V mod P Q_top = (V mod P) + P ((V >> logP) mod Q_top)
__global__ void k_bgv_modpq(const uint32_t* __restrict__ X, int nx, bool is_signed, bool negate,
                            const int32_t* __restrict__ e, const int32_t* __restrict__ s2, uint32_t* __restrict__ out,
                            int nout, int N, const BgvLevel* __restrict__ ltop, const BgvConsts* __restrict__ cs,
                            uint32_t* __restrict__ scratch) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const uint32_t t = cs->t;
  const int logP = cs->logP;
  const int nv = nx + 2;
  // V into scratch (two's complement, nv limbs)
  uint32_t* v = scratch + n;
  const uint32_t xtop = __ldg(X + (size_t)(nx - 1) * N + n);
  const uint32_t xext = (is_signed && (xtop >> 31)) ? 0xFFFFFFFFu : 0u;
  const int64_t te = e ? (int64_t)t * __ldg(e + n) : 0;
  const int32_t sq = s2 ? __ldg(s2 + n) : 0;
  const int pl = logP >> 5, pb = logP & 31;
  const uint64_t tu = (uint64_t)te;
  const uint32_t te_ext = te < 0 ? 0xFFFFFFFFu : 0u;
  const uint32_t sq_ext = sq < 0 ? 0xFFFFFFFFu : 0u;
  uint32_t cx = negate ? 1u : 0u, c2 = 0, c3 = 0;
  for (int l = 0; l < nv; ++l) {
    uint32_t xv = l < nx ? __ldg(X + (size_t)l * N + n) : xext;
    if (negate) {
      const uint64_t s = (uint64_t)(~xv) + cx;
      xv = (uint32_t)s;
      cx = (uint32_t)(s >> 32);
    }
    const uint32_t tw = l == 0 ? (uint32_t)tu : (l == 1 ? (uint32_t)(tu >> 32) : te_ext);
    uint64_t s = (uint64_t)xv + tw + c2;
    uint32_t acc = (uint32_t)s;
    c2 = (uint32_t)(s >> 32);
    // limb l of sq << logP
    const int a = l - pl;
    const uint32_t hi = a >= 0 ? (a == 0 ? (uint32_t)sq : sq_ext) : 0u;
    const uint32_t lo = (a - 1) >= 0 ? ((a - 1) == 0 ? (uint32_t)sq : sq_ext) : 0u;
    const uint32_t sw = pb ? __funnelshift_l(lo, hi, pb) : hi;
    s = (uint64_t)acc + sw + c3;
    v[(size_t)l * N] = (uint32_t)s;
    c3 = (uint32_t)(s >> 32);
  }
  // high part V >> logP (arithmetic) into scratch rows [nv, nv + nh)
  const uint32_t vext = (v[(size_t)(nv - 1) * N] >> 31) ? 0xFFFFFFFFu : 0u;
  const int nh = nv - pl;
  uint32_t* hpart = scratch + (size_t)nv * N + n;
  for (int j = 0; j < nh; ++j) {
    const uint32_t a0 = v[(size_t)(j + pl) * N];
    const uint32_t a1 = (j + pl + 1 < nv) ? v[(size_t)(j + pl + 1) * N] : vext;
    hpart[(size_t)j * N] = pb ? __funnelshift_r(a0, a1, pb) : a0;
  }
  uint32_t c[KB];
  mod_q(hpart, N, nh, true, 0, *ltop, c);
  // out = low logP bits of V, then c << logP
  for (int l = 0; l < nout; ++l) {
    uint32_t lowv = 0;
    if (l < pl) lowv = v[(size_t)l * N];
    else if (l == pl && pb) lowv = v[(size_t)l * N] & ((1u << pb) - 1u);
    const int a = l - pl;
    uint32_t chi = 0, clo = 0;
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      if (k == a) chi = c[k];
      if (k == a - 1) clo = c[k];
    }
    const uint32_t cw = pb ? __funnelshift_l(clo, chi, pb) : chi;
    out[(size_t)l * N + n] = lowv | cw;
  }
}

// (a +- b) mod Q_l or -a mod Q_l on canonical operands
__global__ void k_bgv_addsub(const uint32_t* __restrict__ a, const uint32_t* __restrict__ bb, uint32_t* __restrict__ out,
                             int mode, int N, const BgvLevel* __restrict__ lv) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const BgvLevel& L = *lv;
  const size_t off = (size_t)blockIdx.y * L.nl * N + n;
  uint32_t x[KB], y[KB];
  load_canon(a + off, N, L.nl, x);
  if (mode == 2) {
    neg_mod_q(x, L);
  } else {
    load_canon(bb + off, N, L.nl, y);
    if (mode == 1) neg_mod_q(y, L);
    add_mod_q(x, y, L);
  }
#pragma unroll
  for (int l = 0; l < KB; ++l)
    if (l < L.nl) out[off + (size_t)l * N] = x[l];
}

// ------------------------------------------------------------ launchers
static dim3 g1(int N, int y) { return dim3((N + 127) / 128, y); }

int launch_bgv_reduce(const fhe_ctx* ctx, const uint32_t* X, int nx, size_t xp, size_t xb, int npoly, int nbatch,
                      bool is_signed, bool negate, const int32_t* e0, const int32_t* e1, size_t eb, const uint32_t* add,
                      int add_polys, size_t ap, size_t ab, uint32_t* out, size_t op, size_t ob, int level,
                      cudaStream_t st) {
  if (nx < 1 || nx > kBgvInLimbs || level < 0 || level > ctx->prm.bgv_levels) return FHE_EINVAL;
  ProfScope ps(ctx, FHE_K_LIMB, 1, st);
  k_bgv_reduce<<<g1(ctx->N, npoly * nbatch), 128, 0, st>>>(X, nx, xp, xb, npoly, is_signed, negate, e0, e1, eb, add,
                                                           add_polys, ap, ab, out, op, ob, ctx->N,
                                                           ctx->d_bgv_levels + level, ctx->prm.t);
  return FHE_OK;
}

int launch_bgv_keyswitch(const fhe_ctx* ctx, const uint32_t* Y, int ny, size_t yp, size_t yb, const uint32_t* d,
                         int add_polys, size_t dp, size_t db, uint32_t* out, size_t op, size_t ob, int nbatch,
                         int level, uint32_t* scratch, size_t sp, size_t sb, cudaStream_t st) {
  if (ny < 1 || ny - (ctx->prm.logP >> 5) > kBgvInLimbs || level < 0 || level > ctx->prm.bgv_levels)
    return FHE_EINVAL;
  ProfScope ps(ctx, FHE_K_LIMB, 1, st);
  k_bgv_keyswitch<<<g1(ctx->N, 2 * nbatch), 128, 0, st>>>(Y, ny, yp, yb, d, add_polys, dp, db, out, op, ob, ctx->N,
                                                          ctx->d_bgv_levels + level, ctx->d_bgv_consts, scratch, sp,
                                                          sb);
  return FHE_OK;
}

int launch_bgv_modswitch(const fhe_ctx* ctx, const uint32_t* in, size_t ip, uint32_t* out, size_t op, int npolys,
                         int level, cudaStream_t st) {
  if (level < 1 || level > ctx->prm.bgv_levels) return FHE_EINVAL;
  ProfScope ps(ctx, FHE_K_LIMB, 1, st);
  k_bgv_modswitch<<<g1(ctx->N, npolys), 128, 0, st>>>(in, ip, out, op, ctx->N, ctx->d_bgv_levels + level,
                                                      ctx->d_bgv_levels + level - 1, ctx->d_bgv_consts);
  return FHE_OK;
}

int launch_bgv_decrypt(const fhe_ctx* ctx, const uint32_t* X, int nx, size_t xb, const uint32_t* b, size_t bb,
                       uint32_t* out, size_t ob, int nbatch, int level, cudaStream_t st) {
  if (nx < 1 || nx > kBgvInLimbs || level < 0 || level > ctx->prm.bgv_levels) return FHE_EINVAL;
  ProfScope ps(ctx, FHE_K_LIMB, 1, st);
  k_bgv_decrypt<<<g1(ctx->N, nbatch), 128, 0, st>>>(X, nx, xb, b, bb, out, ob, ctx->N, ctx->d_bgv_levels + level,
                                                    ctx->d_bgv_consts);
  return FHE_OK;
}

int launch_bgv_modpq(const fhe_ctx* ctx, const uint32_t* X, int nx, bool is_signed, bool negate, const int32_t* e,
                     const int32_t* s2, uint32_t* out, int nout, uint32_t* scratch, cudaStream_t st) {
  if (nx < 1 || nx + 2 - (ctx->prm.logP >> 5) > kBgvInLimbs) return FHE_EINVAL;
  ProfScope ps(ctx, FHE_K_LIMB, 1, st);
  k_bgv_modpq<<<g1(ctx->N, 1), 128, 0, st>>>(X, nx, is_signed, negate, e, s2, out, nout, ctx->N,
                                             ctx->d_bgv_levels + ctx->prm.bgv_levels, ctx->d_bgv_consts, scratch);
  return FHE_OK;
}

int launch_bgv_addsub(const fhe_ctx* ctx, const uint32_t* a, const uint32_t* b, uint32_t* out, int npolys, int mode,
                      int level, cudaStream_t st) {
  ProfScope ps(ctx, FHE_K_LIMB, 1, st);
  k_bgv_addsub<<<g1(ctx->N, npolys), 128, 0, st>>>(a, b, out, mode, ctx->N, ctx->d_bgv_levels + level);
  return FHE_OK;
}

}  // namespace fhe

// ------------------------------------------------------- host: the tables
namespace fhe {
namespace {

using Big = std::vector<uint32_t>;  // little-endian limbs

void big_mul_u64(Big& x, uint64_t m) {
  const uint32_t m0 = (uint32_t)m, m1 = (uint32_t)(m >> 32);
  Big out(x.size() + 2, 0);
  for (size_t i = 0; i < x.size(); ++i) {
    uint64_t c = 0;
    uint64_t t = (uint64_t)x[i] * m0 + out[i] + c;
    out[i] = (uint32_t)t;
    c = t >> 32;
    t = (uint64_t)x[i] * m1 + out[i + 1] + c;
    out[i + 1] = (uint32_t)t;
    c = t >> 32;
    for (size_t k = i + 2; c && k < out.size(); ++k) {
      t = (uint64_t)out[k] + c;
      out[k] = (uint32_t)t;
      c = t >> 32;
    }
  }
  while (out.size() > 1 && out.back() == 0) out.pop_back();
  x = out;
}
int big_bits(const Big& x) {
  for (int i = (int)x.size() - 1; i >= 0; --i)
    if (x[i]) return 32 * i + (32 - __builtin_clz(x[i]));
  return 0;
}
int big_cmp(const Big& a, const Big& b) {  // same length
  for (int i = (int)a.size() - 1; i >= 0; --i)
    if (a[i] != b[i]) return a[i] > b[i] ? 1 : -1;
  return 0;
}
void big_sub(Big& a, const Big& b) {  // a -= b, same length, a >= b
  uint32_t bo = 0;
  for (size_t i = 0; i < a.size(); ++i) {
    const uint64_t d = (uint64_t)a[i] - b[i] - bo;
    a[i] = (uint32_t)d;
    bo = (uint32_t)(d >> 63);
  }
}
// (x * 2) mod Q for x < Q (same length as Q, one spare limb)
void big_double_mod(Big& x, const Big& Q) {
  uint32_t c = 0;
  for (size_t i = 0; i < x.size(); ++i) {
    const uint32_t nc = x[i] >> 31;
    x[i] = (x[i] << 1) | c;
    c = nc;
  }
  if (big_cmp(x, Q) >= 0) big_sub(x, Q);
}
// x^-1 mod 2^(32 n) for odd x given as a u64
Big inv_pow2(uint64_t x, int n) {
  uint64_t y = 1;  // inverse mod 2^64 by Newton
  for (int i = 0; i < 6; ++i) y *= 2 - x * y;
  Big r(n, 0);
  r[0] = (uint32_t)y;
  if (n > 1) r[1] = (uint32_t)(y >> 32);
  // Newton on limbs: r <- r (2 - x r) mod 2^(32 n), doubling the correct bits each round
  for (int round = 0; round < 6; ++round) {
    Big xr(n, 0);  // x * r mod 2^(32n)
    for (int i = 0; i < n; ++i) {
      uint64_t c = 0;
      for (int k = 0; k < 2 && i + k < n; ++k) {
        const uint32_t xk = k == 0 ? (uint32_t)x : (uint32_t)(x >> 32);
        uint64_t t = (uint64_t)r[i] * xk + xr[i + k] + c;
        xr[i + k] = (uint32_t)t;
        c = t >> 32;
        if (k == 1)
          for (int m = i + 2; c && m < n; ++m) {
            t = (uint64_t)xr[m] + c;
            xr[m] = (uint32_t)t;
            c = t >> 32;
          }
      }
      if (i + 1 >= n) continue;
      (void)c;
    }
    // e = 2 - xr mod 2^(32n)
    Big e(n, 0);
    uint32_t bo = 0;
    for (int i = 0; i < n; ++i) {
      const uint64_t d = (uint64_t)(i == 0 ? 2u : 0u) - xr[i] - bo;
      e[i] = (uint32_t)d;
      bo = (uint32_t)(d >> 63);
    }
    Big nr(n, 0);
    for (int i = 0; i < n; ++i) {
      uint64_t c = 0;
      for (int j = 0; i + j < n; ++j) {
        const uint64_t t = (uint64_t)r[i] * e[j] + nr[i + j] + c;
        nr[i + j] = (uint32_t)t;
        c = t >> 32;
      }
    }
    r = nr;
  }
  return r;
}
uint64_t inv_mod_u64(uint64_t a, uint64_t m) {  // extended Euclid, gcd(a, m) = 1
  __int128 t = 0, nt = 1, rr = m, nr = a % m;
  while (nr) {
    const __int128 q = rr / nr;
    __int128 tmp = t - q * nt;
    t = nt;
    nt = tmp;
    tmp = rr - q * nr;
    rr = nr;
    nr = tmp;
  }
  if (t < 0) t += m;
  return (uint64_t)t;
}

}  // namespace

int build_bgv_tables(fhe_ctx* ctx) {
  const fhe_params& p = ctx->prm;
  const int L = p.bgv_levels;
  std::vector<BgvLevel> lv(L + 1);
  memset(lv.data(), 0, sizeof(BgvLevel) * lv.size());
  ctx->bgv_bits.assign(L + 1, 0);
  Big Q{(uint32_t)p.bgv_q0, (uint32_t)(p.bgv_q0 >> 32)};
  while (Q.size() > 1 && Q.back() == 0) Q.pop_back();
  for (int l = 0; l <= L; ++l) {
    if (l > 0) big_mul_u64(Q, p.bgv_r);
    const int bits = big_bits(Q);
    const int nl = (bits + 31) / 32;
    if (nl > kBgvLimbs) {
      set_error("bgv: Q_%d has %d bits, more than %d", l, bits, 32 * kBgvLimbs);
      return FHE_EINVAL;
    }
    ctx->bgv_bits[l] = bits;
    BgvLevel& B = lv[l];
    B.nl = nl;
    for (int i = 0; i < nl; ++i) B.q[i] = Q[i];
    Big Qp(kBgvLimbs + 1, 0), x(kBgvLimbs + 1, 0);
    for (int i = 0; i < nl; ++i) Qp[i] = Q[i];
    x[0] = 1;
    if (big_cmp(x, Qp) >= 0) big_sub(x, Qp);
    for (int j = 0; j <= kBgvInLimbs; ++j) {
      bool zero = true;
      for (int i = 0; i < kBgvLimbs; ++i) {
        B.R[j][i] = x[i];
        zero = zero && x[i] == 0;
      }
      Big ng = Qp;
      if (!zero) big_sub(ng, x); else std::fill(ng.begin(), ng.end(), 0u);
      for (int i = 0; i < kBgvLimbs; ++i) B.negR[j][i] = ng[i];
      for (int k = 0; k < 32; ++k) big_double_mod(x, Qp);
    }
    double qt = 0.0;
    for (int k = 0; k < 3 && nl - 1 - k >= 0; ++k) qt += (double)Q[nl - 1 - k] * pow(2.0, -32.0 * k);
    B.qtop = qt;
    uint64_t qm = 0, pw = 1;
    for (int i = 0; i < nl; ++i) {
      qm = (qm + (uint64_t)Q[i] % p.t * pw) % p.t;
      pw = pw * (((uint64_t)1 << 32) % p.t) % p.t;
    }
    B.q_mod_t = (uint32_t)qm;
    unsigned __int128 rp = 1;
    for (int i = 0; i < kBgvLimbs; ++i) {
      B.rpow[i] = (uint64_t)rp;
      rp = (rp << 32) % p.bgv_r;
    }
    Big ri = inv_pow2(p.bgv_r, kBgvLimbs + 2);
    for (int i = 0; i < kBgvLimbs + 2; ++i) B.rinv[i] = ri[i];
  }
  BgvConsts C;
  memset(&C, 0, sizeof(C));
  C.t = p.t;
  C.logP = p.logP;
  C.r = p.bgv_r;
  C.tinv_r = inv_mod_u64(p.t % p.bgv_r, p.bgv_r);
  uint64_t pw = 1;
  for (int i = 0; i < kBgvLimbs; ++i) {
    C.tpow[i] = (uint32_t)pw;
    pw = pw * (((uint64_t)1 << 32) % p.t) % p.t;
  }
  Big ti = inv_pow2(p.t, kBgvLimbs);
  const int lp = (p.logP + 31) / 32;
  for (int i = 0; i < kBgvLimbs; ++i) C.tinvP[i] = i < lp ? ti[i] : 0u;
  if (p.logP & 31) C.tinvP[lp - 1] &= (1u << (p.logP & 31)) - 1u;
  ctx->d_bgv_levels = (BgvLevel*)ctx_alloc(ctx, sizeof(BgvLevel) * lv.size());
  ctx->d_bgv_consts = (BgvConsts*)ctx_alloc(ctx, sizeof(BgvConsts));
  if (!ctx->d_bgv_levels || !ctx->d_bgv_consts) return FHE_ENOMEM;
  if (cudaMemcpy(ctx->d_bgv_levels, lv.data(), sizeof(BgvLevel) * lv.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ctx->d_bgv_consts, &C, sizeof(C), cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("bgv: table upload failed");
    return FHE_ECUDA;
  }
  return FHE_OK;
}

}  // namespace fhe
