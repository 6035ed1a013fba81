// Host side of the context: NTT-friendly primes, the precomputed tables of
// Sec. 5 "Precomputation for GPU-Accelerated Negacyclic NTT", allocation and
// error reporting.  Host arithmetic only; uploads with cudaMemcpy.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "common.cuh"

namespace fhe {

// ------------------------------------------------------------- errors
static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
const char* last_error() { return g_err; }

// ------------------------------------------------------- host modular math
static uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((unsigned __int128)a * b % m); }
static uint64_t powmod64(uint64_t a, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m;
  a %= m;
  while (e) {
    if (e & 1) r = mulmod64(r, a, m);
    a = mulmod64(a, a, m);
    e >>= 1;
  }
  return r;
}
static bool is_prime32(uint32_t n) {
  if (n < 2) return false;
  // deterministic Miller-Rabin for 32-bit n: bases 2, 7, 61
  const uint32_t bases[3] = {2, 7, 61};
  for (uint32_t b : bases)
    if (n % b == 0) return n == b;
  uint32_t d = n - 1;
  int s = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    ++s;
  }
  for (uint32_t b : bases) {
    uint64_t x = powmod64(b, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int i = 1; i < s; ++i) {
      x = mulmod64(x, x, n);
      if (x == n - 1) {
        comp = false;
        break;
      }
    }
    if (comp) return false;
  }
  return true;
}
static uint32_t inv_mod(uint32_t a, uint32_t q) { return (uint32_t)powmod64(a, q - 2, q); }
static uint32_t shoup_of(uint32_t w, uint32_t q) { return (uint32_t)(((uint64_t)w << 32) / q); }

// Primes q = 1 (mod 2^17), 2^29 < q < 2^30, largest first: NTT-friendly for
// every N <= 2^16 (Sec. 2: q = 1 mod 2N; Sec. 4: 30-bit primes).  Below 2^30,
// 4q fits 32 bits, which the lazy NTT butterflies use.
const std::vector<uint32_t>& global_primes() {
  static std::vector<uint32_t> primes;
  static std::once_flag once;
  std::call_once(once, [] {
    const uint32_t step = 1u << 17;
    for (uint32_t c = 0x40000000u - step + 1; c > 0x20000000u && (int)primes.size() < kMaxPrimes; c -= step)
      if (is_prime32(c)) primes.push_back(c);
  });
  return primes;
}

// Smallest r with prod_{i<r-1} q_i >= 2^bound_bits: the product is exact and
// the top prime is a spare whose mixed-radix digit carries the sign.
int primes_for_bound_global(int bound_bits) {
  const auto& p = global_primes();
  double acc = 0.0;
  for (int r = 1; r <= (int)p.size(); ++r) {
    // acc = sum_{i<r-1} log2 q_i
    if (acc >= (double)bound_bits + 1e-6) return r;
    acc += log2((double)p[r - 1]);
  }
  return -1;
}
int primes_for_bound(const fhe_ctx* ctx, int bound_bits) {
  int r = primes_for_bound_global(bound_bits);
  return (r < 0 || r > ctx->R) ? -1 : r;
}

void* ctx_alloc(fhe_ctx* ctx, size_t bytes) {
  bytes = align256(bytes);
  void* p = nullptr;
  if (ctx->alloc) {
    p = ctx->alloc(bytes, ctx->alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (p) ctx->owned.emplace_back(p, bytes);
  return p;
}

cudaEvent_t Profile::get_event() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
void Profile::reset(bool enable) {
  for (int k = 0; k < FHE_K_COUNT; ++k) {
    launches[k] = 0;
    for (auto& pr : ev[k]) {
      pool.push_back(pr.first);
      pool.push_back(pr.second);
    }
    ev[k].clear();
  }
  timing = enable;
}
Profile::~Profile() {
  reset(false);
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

ProfScope::ProfScope(const fhe_ctx* ctx, int kclass, int kernels, cudaStream_t st) : p_(&ctx->prof), k_(kclass), st_(st) {
  p_->launches[k_] += kernels;
  if (p_->timing) {
    cudaEvent_t start = p_->get_event();
    stop_ = p_->get_event();
    if (start && stop_) {
      cudaEventRecord(start, st_);
      p_->ev[k_].emplace_back(start, stop_);
    } else {
      stop_ = nullptr;
    }
  }
}
ProfScope::~ProfScope() {
  if (stop_) cudaEventRecord(stop_, st_);
}

void ctx_free(fhe_ctx* ctx, void* p) {
  for (size_t i = 0; i < ctx->owned.size(); ++i) {
    if (ctx->owned[i].first == p) {
      if (ctx->free_)
        ctx->free_(p, ctx->owned[i].second, ctx->alloc_user);
      else
        cudaFree(p);
      ctx->owned.erase(ctx->owned.begin() + i);
      return;
    }
  }
}

static unsigned bitrev(unsigned x, int bits) {
  unsigned r = 0;
  for (int i = 0; i < bits; ++i) {
    r = (r << 1) | (x & 1);
    x >>= 1;
  }
  return r;
}

// Upload helper: allocate + copy, returns nullptr on failure (error set).
template <typename T>
static T* upload(fhe_ctx* ctx, const std::vector<T>& h) {
  T* d = (T*)ctx_alloc(ctx, h.size() * sizeof(T));
  if (!d) {
    set_error("device allocation of %zu bytes failed", h.size() * sizeof(T));
    return nullptr;
  }
  if (cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("table upload failed");
    return nullptr;
  }
  return d;
}

// (value, Shoup companion) pairs, one 64-bit word per twiddle.
static std::vector<uint2> interleave(const std::vector<uint32_t>& w, const std::vector<uint32_t>& wp) {
  std::vector<uint2> out(w.size());
  for (size_t i = 0; i < w.size(); ++i) out[i] = make_uint2(w[i], wp[i]);
  return out;
}

// fp16 bit pattern of a small integer, |v| <= 2048 (exact).
static uint16_t half_of_int(int v) {
  if (v == 0) return 0;
  const uint16_t sign = v < 0 ? 0x8000u : 0u;
  const unsigned a = (unsigned)(v < 0 ? -v : v);
  int e = 0;
  while ((a >> (e + 1)) != 0) ++e;
  const unsigned mant = (a << (10 - e)) & 0x3FFu;
  return (uint16_t)(sign | (unsigned)((e + 15) << 10) | mant);
}

// Balanced base-256 digits c_p in [-128, 127] of x mod 2^(32 kMaxLimbs):
// sum_p c_p 256^p = x (mod 2^(32 kMaxLimbs)); the carry out of the top is dropped.
static void balanced_bytes(const uint32_t* limbs, int8_t* out) {
  int carry = 0;
  for (int p = 0; p < 4 * kMaxLimbs; ++p) {
    const int v = (int)((limbs[p >> 2] >> (8 * (p & 3))) & 0xFFu) + carry;
    carry = v >= 128 ? 1 : 0;
    out[p] = (int8_t)(v - 256 * carry);
  }
}

// Tensor-core form of the direct CRT's dense product (k_crt_tc).  Output
// byte column p of sum_i y_i C_i (C_i = M_r/q_i, C_r = -M_r with y_r = kappa)
// is S_p = sum_i sum_a d_{i,a} c_{i,p-a}, d_{i,a} the balanced bytes of y_i,
// c_{i,.} those of C_i: a GEMM with K = 4 i + a and the B operand
// B[p][4 i + a] = c_{i,p-a}, stored per slice of 32 k as K-major core
// matrices (8 rows x 8 f16) in the order [p/8][k/8][p%8][k%8].
static int build_crt_tc(fhe_ctx* ctx, const std::vector<uint32_t>& qhat, const std::vector<uint32_t>& negm) {
  const int R = ctx->R;
  const int lmax = (R + 4 < kMaxLimbs) ? R + 4 : kMaxLimbs;
  const int MT = (lmax + 3) / 4;
  const int P = 16 * MT;
  ctx->crt_tc_mt = MT;
  ctx->crt_tc_off.assign(R + 1, 0);
  ctx->crt_tc_exact22.assign(R + 1, 0);
  size_t total = 0;
  for (int r = 1; r <= R; ++r) {
    ctx->crt_tc_off[r] = total;
    total += (size_t)((r + 16) / 16) * P * 64;
  }
  std::vector<uint16_t> mat(total, 0);
  std::vector<int8_t> dig((size_t)(R + 1) * 4 * kMaxLimbs);
  uint16_t h16[256];
  for (int v = -128; v < 128; ++v) h16[v + 128] = half_of_int(v);
  for (int r = 1; r <= R; ++r) {
    const size_t off = (size_t)r * (r - 1) / 2;
    for (int i = 0; i < r; ++i) balanced_bytes(&qhat[(off + i) * kMaxLimbs], &dig[(size_t)i * 4 * kMaxLimbs]);
    balanced_bytes(&negm[(size_t)r * kMaxLimbs], &dig[(size_t)r * 4 * kMaxLimbs]);
    // largest possible |S_p| over the columns: digits of y_i (< q < 2^30) are at
    // most 128 in magnitude (64 for the top one), kappa's single digit at most r
    int64_t smax = 0;
    for (int p = 0; p < P; ++p) {
      int64_t sp = 0;
      for (int i = 0; i <= r; ++i)
        for (int a = 0; a < 4 && a <= p; ++a) {
          const int64_t c = dig[(size_t)i * 4 * kMaxLimbs + p - a];
          const int64_t dm = i == r ? (a == 0 ? r : 0) : (a < 3 ? 128 : 64);
          sp += dm * (c < 0 ? -c : c);
        }
      smax = sp > smax ? sp : smax;
    }
    ctx->crt_tc_exact22[r] = smax < ((int64_t)1 << 22) ? 1 : 0;
    const int nch = (r + 16) / 16;
    uint16_t* base = mat.data() + ctx->crt_tc_off[r];
    for (int c = 0; c < nch; ++c)
      for (int p = 0; p < P; ++p)
        for (int k = 0; k < 64; ++k) {
          const int kg = 64 * c + k, i = kg >> 2, a = kg & 3, pa = p - a;
          if (i > r || pa < 0) continue;
          const int kh = kg >> 5, kk = kg & 31;
          base[(size_t)kh * P * 32 + ((size_t)(p >> 3) * 4 + (kk >> 3)) * 64 + (p & 7) * 8 + (kk & 7)] =
              h16[dig[(size_t)i * 4 * kMaxLimbs + pa] + 128];
        }
  }
  return (ctx->d_crt_tc = upload(ctx, mat)) ? FHE_OK : FHE_ENOMEM;
}

// Tensor-core form of the lift (k_lift_tc).  With x = sum_k b_k 256^k (bytes
// b_k of the limbs) and d_k = b_k - 128, the residue row i of the GEMM output
// is T_i = sum_a 256^a sum_k d_k c_{i,k,a}, c_{i,k,a} the digits of
// C_{i,k} = 2^(8k) 2^32 mod q_i; T_i = (x - 128 sum_k 256^k) 2^32 (mod q_i), so
// adding off_i(L) = (128 sum_{k<4L} 256^k) 2^32 mod q_i (and 2^17 q_i to make
// it non-negative) and one Montgomery reduction give x mod q_i.  The signed
// form (a two's-complement value of 32 L bits) feeds the top byte as the
// signed digit (b ^ 0x80) - 128 and so takes offs_i(L), the same sum without
// the top byte's term.
static int build_lift_tc(fhe_ctx* ctx) {
  const int R = ctx->R, KMAX = 4 * kMaxLiftLimbs;
  const std::vector<uint32_t>& q = ctx->q;
  const size_t rows8 = (size_t)((4 * R + 7) / 8) * 8;  // whole 8-row core-matrix groups
  std::vector<uint16_t> mat(rows8 * KMAX, 0);
  std::vector<uint64_t> off((size_t)(kMaxLiftLimbs + 1) * R, 0), offs((size_t)(kMaxLiftLimbs + 1) * R, 0);
  for (int i = 0; i < R; ++i) {
    const uint64_t qi = q[i];
    uint64_t c = ((uint64_t)1 << 32) % qi;  // C_{i,0} = 2^32 mod q
    uint64_t offacc = 0;                    // (128 sum_{k' < k} 256^k') 2^32 mod q
    for (int k = 0; k < KMAX; ++k) {
      if ((k & 3) == 0) off[(size_t)(k >> 2) * R + i] = offacc + (qi << 17);
      // signed form of L = (k + 1) / 4 limbs: the top byte is a signed digit, no offset for it
      if ((k & 3) == 3) offs[(size_t)((k + 1) >> 2) * R + i] = offacc + (qi << 17);
      // digits of C: bytes 0..2 balanced with carry, byte 3 takes the carry (C < q < 2^30)
      int carry = 0, dg[4];
      for (int a = 0; a < 3; ++a) {
        const int v = (int)((c >> (8 * a)) & 0xFF) + carry;
        carry = v >= 128 ? 1 : 0;
        dg[a] = v - 256 * carry;
      }
      dg[3] = (int)((c >> 24) & 0xFF) + carry;
      for (int a = 0; a < 4; ++a) {
        const int row = 4 * i + a;
        mat[(((size_t)(row >> 3) * (KMAX / 8) + (k >> 3)) * 8 + (row & 7)) * 8 + (k & 7)] = half_of_int(dg[a]);
      }
      offacc = (offacc + 128 * c) % qi;
      c = (c << 8) % qi;
    }
    off[(size_t)kMaxLiftLimbs * R + i] = offacc + (qi << 17);
  }
  if (!(ctx->d_lift_tc = upload(ctx, mat)) || !(ctx->d_lift_off = upload(ctx, off)) ||
      !(ctx->d_lift_off_s = upload(ctx, offs)))
    return FHE_ENOMEM;
  return FHE_OK;
}

int build_tables(fhe_ctx* ctx) {
  const int N = ctx->N, logN = ctx->prm.logN, R = ctx->R;
  const auto& gp = global_primes();
  ctx->q.assign(gp.begin(), gp.begin() + R);
  const std::vector<uint32_t>& q = ctx->q;

  std::vector<uint32_t> qinv(R), nscale(R), nscale_sh(R), red(4 * (size_t)R);
  std::vector<uint32_t> psi((size_t)R * N), psi_sh((size_t)R * N), ipsi((size_t)R * N), ipsi_sh((size_t)R * N);
  std::vector<uint32_t> pow2((size_t)R * kMaxLiftLimbs), pow24((size_t)R * kLiftDigits);
  std::vector<uint2> garner((size_t)R * R, make_uint2(0, 0));
  std::vector<uint32_t> mprod((size_t)(R + 1) * kMaxLimbs, 0);

  for (int i = 0; i < R; ++i) {
    const uint32_t qi = q[i];
    uint32_t inv = 1;  // Newton iteration for q^-1 mod 2^32
    for (int it = 0; it < 5; ++it) inv *= 2u - qi * inv;
    qinv[i] = inv;
    // psi: order exactly 2N (psi^N = -1)
    uint32_t ps = 0;
    for (uint32_t x = 2;; ++x) {
      uint32_t c = (uint32_t)powmod64(x, (qi - 1) / (2ull * N), qi);
      if (powmod64(c, N, qi) == qi - 1) {
        ps = c;
        break;
      }
    }
    const uint32_t ips = inv_mod(ps, qi);
    for (int k = 0; k < N; ++k) {
      unsigned e = bitrev((unsigned)k, logN);
      uint32_t w = (uint32_t)powmod64(ps, e, qi);
      uint32_t iw = (uint32_t)powmod64(ips, e, qi);
      psi[(size_t)i * N + k] = w;
      psi_sh[(size_t)i * N + k] = shoup_of(w, qi);
      ipsi[(size_t)i * N + k] = iw;
      ipsi_sh[(size_t)i * N + k] = shoup_of(iw, qi);
    }
    // N^-1 * 2^32 mod q: the INTT scale also removes the 2^-32 of one Montgomery product
    uint32_t ninv = inv_mod((uint32_t)(N % qi), qi);
    nscale[i] = (uint32_t)mulmod64(ninv, ((uint64_t)1 << 32) % qi, qi);
    nscale_sh[i] = shoup_of(nscale[i], qi);
    for (int l = 0; l < kMaxLiftLimbs; ++l) pow2[(size_t)i * kMaxLiftLimbs + l] = (uint32_t)powmod64(2, 32ull * l, qi);
    for (int m = 0; m < kLiftDigits; ++m) pow24[(size_t)i * kLiftDigits + m] = (uint32_t)powmod64(2, 24ull * m, qi);
    uint32_t r32 = (uint32_t)(((uint64_t)1 << 32) % qi);
    uint32_t r64 = (uint32_t)mulmod64(r32, r32, qi);
    red[4 * i + 0] = r32;
    red[4 * i + 1] = shoup_of(r32, qi);
    red[4 * i + 2] = r64;
    red[4 * i + 3] = shoup_of(r64, qi);
  }
  // Garner constants c_{j,k} = [q_j^-1]_{q_k}, j < k (Sec. 2 Eq. garner_mrc; Sec. 5 CRT constants)
  for (int k = 0; k < R; ++k)
    for (int j = 0; j < k; ++j) {
      uint32_t c = inv_mod(q[j] % q[k], q[k]);
      garner[(size_t)k * R + j] = make_uint2(c, shoup_of(c, q[k]));
    }
  // M_k = prod_{i<k} q_i mod 2^(32 kMaxLimbs) (Sec. 5 CRT constants)
  std::vector<uint32_t> acc(kMaxLimbs, 0);
  acc[0] = 1;
  for (int k = 0; k <= R; ++k) {
    memcpy(&mprod[(size_t)k * kMaxLimbs], acc.data(), kMaxLimbs * sizeof(uint32_t));
    if (k == R) break;
    uint64_t carry = 0;
    for (int l = 0; l < kMaxLimbs; ++l) {
      uint64_t t = (uint64_t)acc[l] * q[k] + carry;
      acc[l] = (uint32_t)t;
      carry = t >> 32;
    }
  }

  // Direct CRT constants for every prime-prefix size r (built incrementally:
  // adding prime q_r multiplies each M_r / q_i by q_r and appends M_r itself).
  const size_t nrows = (size_t)R * (R + 1) / 2;
  std::vector<uint32_t> qhat(nrows * kMaxLimbs, 0), negm((size_t)(R + 1) * kMaxLimbs, 0);
  std::vector<uint2> crt_inv(nrows);
  std::vector<float> invq(R);
  {
    std::vector<uint32_t> cur((size_t)R * kMaxLimbs, 0);  // cur[i] = prod_{j<r, j!=i} q_j mod 2^4096
    std::vector<uint32_t> Mr(kMaxLimbs, 0);               // M_r mod 2^4096
    std::vector<uint64_t> pm(R, 1);                       // prod_{j<r, j!=i} q_j mod q_i
    Mr[0] = 1;
    auto mul_word = [](uint32_t* x, uint32_t w) {
      uint64_t c = 0;
      for (int l = 0; l < kMaxLimbs; ++l) {
        uint64_t t = (uint64_t)x[l] * w + c;
        x[l] = (uint32_t)t;
        c = t >> 32;
      }
    };
    for (int r = 1; r <= R; ++r) {
      // extend from r-1 primes to r primes: new prime q_{r-1}
      const uint32_t qn = q[r - 1];
      for (int i = 0; i < r - 1; ++i) {
        mul_word(&cur[(size_t)i * kMaxLimbs], qn);
        pm[i] = pm[i] * (qn % q[i]) % q[i];
      }
      memcpy(&cur[(size_t)(r - 1) * kMaxLimbs], Mr.data(), kMaxLimbs * 4);  // M_{r-1} = prod_{j<r-1} q_j
      uint64_t pr = 1;
      for (int j = 0; j < r - 1; ++j) pr = pr * (q[j] % qn) % qn;
      pm[r - 1] = pr;
      mul_word(Mr.data(), qn);  // M_r
      const size_t off = (size_t)r * (r - 1) / 2;
      for (int i = 0; i < r; ++i) {
        memcpy(&qhat[(off + i) * kMaxLimbs], &cur[(size_t)i * kMaxLimbs], kMaxLimbs * 4);
        // the inverse transforms leave out their N^-1 2^32 scale (see k_ntt.cu): it is folded in here
        const uint32_t inv = (uint32_t)mulmod64(inv_mod((uint32_t)pm[i], q[i]), nscale[i], q[i]);
        crt_inv[off + i] = make_uint2(inv, shoup_of(inv, q[i]));
      }
      uint64_t c = 1;  // -M_r = ~M_r + 1
      for (int l = 0; l < kMaxLimbs; ++l) {
        uint64_t t = (uint64_t)(uint32_t)~Mr[l] + c;
        negm[(size_t)r * kMaxLimbs + l] = (uint32_t)t;
        c = t >> 32;
      }
    }
    for (int i = 0; i < R; ++i) invq[i] = (float)(1.0 / (double)q[i]);
  }

  // the same constants as 24-bit digit columns: set r occupies rows [r(r+1)/2 - 1 ...] -> offset
  // sum_{r'<r} (r'+1) = r(r+1)/2 - 1 rows... kept simple: rows of set r start at (r-1)(r+2)/2
  std::vector<uint32_t> dig((size_t)((R) * (R + 3) / 2 + 2) * kCrtDigits, 0);
  auto digits_of = [](const uint32_t* limbs, uint32_t* out) {
    for (int m = 0; m < kCrtDigits; ++m) {
      const int o = 24 * m, l = o >> 5, sh = o & 31;
      uint64_t w = 0;
      if (l < kMaxLimbs) w = limbs[l];
      if (l + 1 < kMaxLimbs) w |= (uint64_t)limbs[l + 1] << 32;
      out[m] = (uint32_t)(w >> sh) & 0xFFFFFFu;
    }
  };
  for (int r = 1; r <= R; ++r) {
    const size_t base = (size_t)(r - 1) * (r + 2) / 2;  // sum_{r'=1}^{r-1} (r'+1)
    const size_t off = (size_t)r * (r - 1) / 2;
    for (int i = 0; i < r; ++i) digits_of(&qhat[(off + i) * kMaxLimbs], &dig[(base + i) * kCrtDigits]);
    digits_of(&negm[(size_t)r * kMaxLimbs], &dig[(base + r) * kCrtDigits]);
  }
  if (!(ctx->d_crt_dig = upload(ctx, dig))) return FHE_ENOMEM;
  if (build_crt_tc(ctx, qhat, negm) != FHE_OK) return FHE_ENOMEM;
  if (build_lift_tc(ctx) != FHE_OK) return FHE_ENOMEM;
  if (!(ctx->d_crt_qhat = upload(ctx, qhat)) || !(ctx->d_crt_inv = upload(ctx, crt_inv)) ||
      !(ctx->d_crt_negm = upload(ctx, negm)) || !(ctx->d_invq = upload(ctx, invq)))
    return FHE_ENOMEM;
  if (!(ctx->d_q = upload(ctx, q)) || !(ctx->d_qinv = upload(ctx, qinv)) || !(ctx->d_psi2 = upload(ctx, interleave(psi, psi_sh))) ||
      !(ctx->d_ipsi2 = upload(ctx, interleave(ipsi, ipsi_sh))) || !(ctx->d_nscale = upload(ctx, nscale)) ||
      !(ctx->d_nscale_sh = upload(ctx, nscale_sh)) || !(ctx->d_pow2 = upload(ctx, pow2)) || !(ctx->d_pow24 = upload(ctx, pow24)) ||
      !(ctx->d_red = upload(ctx, red)) || !(ctx->d_garner = upload(ctx, garner)) ||
      !(ctx->d_mprod = upload(ctx, mprod)))
    return FHE_ENOMEM;
  return FHE_OK;
}

void free_all(fhe_ctx* ctx) {
  for (auto& pr : ctx->owned) {
    if (ctx->free_)
      ctx->free_(pr.first, pr.second, ctx->alloc_user);
    else
      cudaFree(pr.first);
  }
  ctx->owned.clear();
}

}  // namespace fhe
