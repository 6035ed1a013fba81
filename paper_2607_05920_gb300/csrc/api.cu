// The C ABI of include/fhe.h: argument checks, workspace carving and the
// kernel sequence of each homomorphic operation.
//
// Ring product (Sec. 5 pipeline): limb -> RNS lift -> forward NTT ->
// pointwise -> INTT -> Garner -> limb, with the prime count sized to the
// exact product's bound so the CRT result is the exact integer product.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "bgv.cuh"
#include "common.cuh"

using namespace fhe;

namespace {

constexpr int kMaxCnum = 1 << 14;

int check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("kernel launch failed: %s", cudaGetErrorString(e));
    return FHE_ECUDA;
  }
  return FHE_OK;
}

#define RET_IF(x)           \
  do {                      \
    int _rc = (x);          \
    if (_rc != FHE_OK) return _rc; \
  } while (0)

// bump allocator over the caller's workspace
struct Carve {
  uint8_t* base;
  size_t size, used = 0;
  bool ok = true;
  Carve(void* p, size_t s) : base((uint8_t*)p), size(s) {}
  uint32_t* take(size_t words) {
    size_t b = align256(words * 4);
    if (!base || used + b > size) {
      ok = false;
      return nullptr;
    }
    uint32_t* p = (uint32_t*)(base + used);
    used += b;
    return p;
  }
};

// prime counts of the products (exact bounds; Sec. 5 signed handling needs the spare prime)
int r_tensor(const fhe_ctx* c, int logQ) { return primes_for_bound(c, c->prm.logN + 2 * logQ + 1); }
int r_keyswitch(const fhe_ctx* c, int logQ) {
  return primes_for_bound(c, c->prm.logN + logQ + c->prm.logP + c->prm.logQ);
}
int r_enc(const fhe_ctx* c) { return primes_for_bound(c, c->prm.logN + c->prm.logQ); }
int r_dec(const fhe_ctx* c, int logQ) { return primes_for_bound(c, c->prm.logN + logQ); }

size_t words_mult(const fhe_ctx* c, int logQ, int cnum) {
  const size_t N = c->N;
  const int rt = r_tensor(c, logQ), rk = r_keyswitch(c, logQ), L = limbs_for_bits(logQ);
  if (rt < 0 || rk < 0) return 0;
  return (size_t)cnum * N * (4 * (size_t)rt + 3 * (size_t)L + 2 * (size_t)rk) + 3 * 64;
}
size_t words_rotate(const fhe_ctx* c, int logQ, int cnum) {
  const size_t N = c->N;
  const int rk = r_keyswitch(c, logQ), L = limbs_for_bits(logQ);
  if (rk < 0) return 0;
  // transform of the centred a, the key products, kappa(b)
  return (size_t)cnum * N * ((size_t)L + 3 * (size_t)rk) + 3 * 64;
}
size_t words_encrypt(const fhe_ctx* c, int cnum) {
  const int re = r_enc(c);
  if (re < 0) return 0;
  return (size_t)cnum * c->N * 2 * (size_t)re + 64;
}
size_t words_decrypt(const fhe_ctx* c, int logQ, int cnum) {
  const int rd = r_dec(c, logQ);
  if (rd < 0) return 0;
  return (size_t)cnum * c->N * (size_t)rd + 64;
}
size_t words_ringmul(const fhe_ctx* c, int bits, int cnum) {
  const int r = primes_for_bound(c, c->prm.logN + 2 * bits);
  if (r < 0) return 0;
  return (size_t)cnum * c->N * 2 * (size_t)r + 2 * 64;
}

// the seeded encryption's v (int8), e0, e1 (int32) ahead of the rest of the workspace
size_t enc_sampler_bytes(const fhe_ctx* c, int cnum) {
  const size_t n = (size_t)cnum * c->N;
  return align256(n) + 2 * align256(4 * n);
}
size_t enc_sampler_words(const fhe_ctx* c, int cnum) { return enc_sampler_bytes(c, cnum) / 4; }

bool is_bgv(const fhe_ctx* ctx) { return ctx->prm.scheme == FHE_SCHEME_BGV; }

bool ct_ok(const fhe_ctx* ctx, const fhe_ct* ct) {
  if (!ct || !ct->data || ct->cnum < 1 || ct->cnum > kMaxCnum || ct->logQ < 1 || ct->logQ > ctx->prm.logQ) return false;
  if (is_bgv(ctx))
    return ct->level >= 0 && ct->level <= ctx->prm.bgv_levels && ct->logQ == ctx->bgv_bits[ct->level];
  return true;
}

// BGV: limbs of the exact signed product emitted by the CRT (bound + sign + headroom)
int bgv_prod_limbs(int bound_bits) { return limbs_for_bits(bound_bits + 2); }

size_t words_mult_bgv(const fhe_ctx* c, int bits, int cnum) {
  const size_t N = c->N;
  const int rt = r_tensor(c, bits), rk = r_keyswitch(c, bits), L = limbs_for_bits(bits);
  if (rt < 0 || rk < 0) return 0;
  const int nxt = bgv_prod_limbs(c->prm.logN + 2 * bits + 1);
  const int nxk = bgv_prod_limbs(c->prm.logN + bits + c->prm.logP + c->prm.logQ);
  const int nz = nxk - (c->prm.logP >> 5);
  return (size_t)cnum * N *
             (4 * (size_t)rt + 3 * (size_t)nxt + 3 * (size_t)L + 2 * (size_t)rk + 2 * (size_t)nxk + 2 * (size_t)nz) +
         6 * 64;
}

// One ring product C = A * B into limbs through `epi`.  A: La limbs or small
// int32 (As) / int8 (As8); B: the same.  ws: 2 r N words.  nbatch = 1.
int ring_product(fhe_ctx* ctx, const uint32_t* A, int La, const int32_t* As, const uint32_t* B, int Lb,
                 const int32_t* Bs, int r, uint32_t* out, const EpiArgs& epi, uint32_t* ws, cudaStream_t st) {
  const size_t N = ctx->N;
  uint32_t* RA = ws;
  uint32_t* RB = ws + (size_t)r * N;
  if (A)
    RET_IF(launch_lift(ctx, A, La, 0, 0, RA, 0, 0, 1, 1, r, st));
  else
    RET_IF(launch_lift_small(ctx, As, false, 0, RA, 0, 1, r, st));
  if (B)
    RET_IF(launch_lift(ctx, B, Lb, 0, 0, RB, 0, 0, 1, 1, r, st));
  else
    RET_IF(launch_lift_small(ctx, Bs, false, 0, RB, 0, 1, r, st));
  RET_IF(launch_ntt(ctx, ws, 2, r, r, r, false, st));
  RET_IF(launch_pointwise_mul(ctx, RA, RA, 0, RB, 0, r, 1, st));
  RET_IF(launch_ntt(ctx, RA, 1, r, r, r, true, st));
  RET_IF(launch_garner(ctx, RA, 0, 0, r, 1, 1, out, 0, 0, epi, st));
  return check_launch();
}

// limbs -> resident NTT form over `rows` primes: dst [npoly][rows][N]
int to_ntt_form(fhe_ctx* ctx, const uint32_t* src, int L, int npoly, int rows, uint32_t* dst, cudaStream_t st) {
  const size_t N = ctx->N;
  RET_IF(launch_lift(ctx, src, L, (size_t)L * N, 0, dst, (size_t)rows * N, 0, npoly, 1, rows, st));
  RET_IF(launch_ntt(ctx, dst, npoly, rows, rows, rows, false, st));
  return check_launch();
}

// Shared body of relinearisation and rotation key switching (Sec. 6):
// Y = [nbatch][2][rk][N] whose block 0 holds the lifted c (limb poly to switch),
// key K = [2][krows][N]; result (add + round(Y / P)) mod 2^logQ into out.
// The reconstruction of a key switch: (add + round(Y / P)) mod 2^(logQ - k2) from the coefficient-form
// products Y = [nbatch][2][rk][N].
int key_switch_epilogue(fhe_ctx* ctx, const uint32_t* Y, int rk, int nbatch, int logQ, int k2, const uint32_t* add,
                        size_t add_pstride, size_t add_bstride, int add_polys, uint32_t* out, cudaStream_t st,
                        const int32_t* item_bits = nullptr, int out_limbs_pad = 0) {
  const size_t N = ctx->N;
  EpiArgs epi;
  epi.kind = Epi::kRelin;
  epi.out_bits = logQ;
  epi.shift = ctx->prm.logP;
  epi.k2 = k2;
  epi.out_limbs = limbs_for_bits(logQ - k2);
  epi.add = add;
  epi.add_limbs = limbs_for_bits(logQ);
  epi.add_pstride = add_pstride;
  epi.add_bstride = add_bstride;
  epi.add_polys = add_polys;
  epi.item_bits = item_bits;
  if (out_limbs_pad > 0) epi.out_limbs = out_limbs_pad;
  const size_t Lo = epi.out_limbs;
  RET_IF(launch_garner(ctx, Y, (size_t)rk * N, 2 * (size_t)rk * N, rk, 2, nbatch, out, Lo * N, 2 * Lo * N, epi, st));
  return check_launch();
}

int key_switch_tail(fhe_ctx* ctx, uint32_t* Y, const SwitchKey& K, int rk, int nbatch, int logQ, int k2,
                    const uint32_t* add, size_t add_pstride, size_t add_bstride, int add_polys, uint32_t* out,
                    cudaStream_t st, const int32_t* item_bits = nullptr, int out_limbs_pad = 0) {
  RET_IF(launch_ring_key(ctx, Y, K.ntt, K.rows, rk, nbatch, st));
  return key_switch_epilogue(ctx, Y, rk, nbatch, logQ, k2, add, add_pstride, add_bstride, add_polys, out, st,
                             item_bits, out_limbs_pad);
}

// Automorphisms with key switching (Sec. 6 leftrotate_broadcast_into, conjugate_pairwise_into) of one
// ciphertext batch for n Galois elements gs[s] -> outs[s]:
//   outs[s] = (kappa(b), 0) + round(P^-1 kappa(centred a) rtk mod P Q)  (mod Q),
// kappa taken over Z on the centred representative of a (two's complement of logQ bits).  The
// centred a is lifted and transformed once; each kappa is then a row gather in the transform
// domain in front of the key products (hoisting), so n rotations cost one lift and one forward
// transform in all, plus per step the key products, two inverse transforms and the reconstruction.
int rotate_many(fhe_ctx* ctx, const fhe_ct* in, const uint32_t* gs, int n, fhe_ct* const* outs, void* ws,
                size_t ws_bytes, cudaStream_t st) {
  const int cnum = in->cnum, logQ = in->logQ, L = limbs_for_bits(logQ), rk = r_keyswitch(ctx, logQ);
  const size_t N = ctx->N;
  std::vector<const SwitchKey*> keys(n);
  for (int s = 0; s < n; ++s) {
    auto it = ctx->rtk.find(gs[s]);
    if (it == ctx->rtk.end()) {
      set_error("rotate: no switching key for the Galois element %u", gs[s]);
      return FHE_ENOKEY;
    }
    keys[s] = &it->second;
  }
  Carve cv(ws, ws_bytes);
  uint32_t* AH = cv.take((size_t)cnum * rk * N);
  uint32_t* Y = cv.take((size_t)cnum * 2 * rk * N);
  uint32_t* KB = cv.take((size_t)cnum * L * N);
  if (!cv.ok || ((uintptr_t)ws & 255)) {
    set_error("rotate: workspace of %zu bytes too small or misaligned", ws_bytes);
    return FHE_EWORKSPACE;
  }
  RET_IF(launch_lift_signed(ctx, in->data + (size_t)L * N, L, 0, 2 * (size_t)L * N, AH, 0, (size_t)rk * N, 1, cnum,
                            rk, logQ, nullptr, st));
  RET_IF(launch_ntt(ctx, AH, cnum, rk, rk, rk, false, st));
  for (int s = 0; s < n; ++s) {
    RET_IF(launch_automorph(ctx, in->data, 2 * (size_t)L * N, KB, (size_t)L * N, L, logQ, gs[s], cnum, st));
    RET_IF(launch_key_perm(ctx, AH, Y, keys[s]->ntt, keys[s]->rows, rk, cnum, gs[s], st));
    RET_IF(key_switch_epilogue(ctx, Y, rk, cnum, logQ, 0, KB, 0, (size_t)L * N, 1, outs[s]->data, st));
    outs[s]->log_scale = in->log_scale;
  }
  return FHE_OK;
}

int rotate_checks(fhe_ctx* ctx, const fhe_ct* in, fhe_ct* const* outs, int n, const char* who) {
  if (ctx && is_bgv(ctx)) {
    set_error("%s: CKKS only", who);
    return FHE_EINVAL;
  }
  if (!ctx || !ct_ok(ctx, in) || n < 1 || !outs) {
    set_error("%s: bad arguments", who);
    return FHE_EINVAL;
  }
  for (int s = 0; s < n; ++s) {
    const fhe_ct* o = outs[s];
    if (!ct_ok(ctx, o) || o->logQ != in->logQ || o->cnum != in->cnum || o->data == in->data) {
      set_error("%s: output %d malformed, of another level or batch size, or aliasing the input", who, s);
      return FHE_EINVAL;
    }
    for (int t = 0; t < s; ++t)
      if (outs[t]->data == o->data) {
        set_error("%s: outputs %d and %d alias", who, t, s);
        return FHE_EINVAL;
      }
  }
  return FHE_OK;
}

// BGV multiplication at level l: exact tensor product reduced mod Q_l, then the
// key switch (d2 evk, divided by P with the t-multiple correction) added to (d0, d1).
int mult_bgv(fhe_ctx* ctx, const fhe_ct* a, const fhe_ct* b, fhe_ct* out, void* ws, size_t ws_bytes,
             cudaStream_t st) {
  const int bits = a->logQ, level = a->level, cnum = a->cnum, L = limbs_for_bits(bits);
  const int rt = r_tensor(ctx, bits), rk = r_keyswitch(ctx, bits);
  const int nxt = bgv_prod_limbs(ctx->prm.logN + 2 * bits + 1);
  const int nxk = bgv_prod_limbs(ctx->prm.logN + bits + ctx->prm.logP + ctx->prm.logQ);
  const int nz = nxk - (ctx->prm.logP >> 5);
  const size_t N = ctx->N;
  Carve cv(ws, ws_bytes);
  uint32_t* X = cv.take((size_t)cnum * 4 * rt * N);
  uint32_t* T1 = cv.take((size_t)cnum * 3 * nxt * N);
  uint32_t* D = cv.take((size_t)cnum * 3 * L * N);
  uint32_t* Y = cv.take((size_t)cnum * 2 * rk * N);
  uint32_t* T2 = cv.take((size_t)cnum * 2 * nxk * N);
  uint32_t* Z = cv.take((size_t)cnum * 2 * nz * N);
  if (!cv.ok || ((uintptr_t)ws & 255)) {
    set_error("mult (BGV): workspace of %zu bytes too small or misaligned", ws_bytes);
    return FHE_EWORKSPACE;
  }
  const size_t ctw = 2 * (size_t)L * N;
  RET_IF(launch_lift(ctx, a->data, L, (size_t)L * N, ctw, X, (size_t)rt * N, 4 * (size_t)rt * N, 2, cnum, rt, st));
  RET_IF(launch_lift(ctx, b->data, L, (size_t)L * N, b->cnum == 1 ? 0 : ctw, X + 2 * (size_t)rt * N, (size_t)rt * N,
                     4 * (size_t)rt * N, 2, cnum, rt, st));
  RET_IF(launch_ring_tensor(ctx, X, rt, cnum, st));
  EpiArgs e0;
  e0.kind = Epi::kStore;
  e0.out_bits = 32 * nxt;
  e0.out_limbs = nxt;
  RET_IF(launch_garner(ctx, X, (size_t)rt * N, 4 * (size_t)rt * N, rt, 3, cnum, T1, (size_t)nxt * N,
                       3 * (size_t)nxt * N, e0, st));
  RET_IF(launch_bgv_reduce(ctx, T1, nxt, (size_t)nxt * N, 3 * (size_t)nxt * N, 3, cnum, true, false, nullptr, nullptr,
                           0, nullptr, 0, 0, 0, D, (size_t)L * N, 3 * (size_t)L * N, level, st));
  RET_IF(launch_lift(ctx, D + 2 * (size_t)L * N, L, 0, 3 * (size_t)L * N, Y, 0, 2 * (size_t)rk * N, 1, cnum, rk,
                     st));
  RET_IF(launch_ring_key(ctx, Y, ctx->evk.ntt, ctx->evk.rows, rk, cnum, st));
  EpiArgs e1;
  e1.kind = Epi::kStore;
  e1.out_bits = 32 * nxk;
  e1.out_limbs = nxk;
  RET_IF(launch_garner(ctx, Y, (size_t)rk * N, 2 * (size_t)rk * N, rk, 2, cnum, T2, (size_t)nxk * N,
                       2 * (size_t)nxk * N, e1, st));
  RET_IF(launch_bgv_keyswitch(ctx, T2, nxk, (size_t)nxk * N, 2 * (size_t)nxk * N, D, 2, (size_t)L * N,
                              3 * (size_t)L * N, out->data, (size_t)L * N, 2 * (size_t)L * N, cnum, level, Z,
                              (size_t)nz * N, 2 * (size_t)nz * N, st));
  return check_launch();
}

// Ragged batch: item i at modulus 2^item_bits[i] (device array), all stored in
// L_pad limbs; prime counts and key rows from the largest level (exact for all).
int mult_ragged(fhe_ctx* ctx, const uint32_t* a, const uint32_t* b, uint32_t* out, int cnum, int L_pad,
                const int32_t* item_bits, int logQ_max, int k2, void* ws, size_t ws_bytes, cudaStream_t st) {
  const int L = L_pad;
  const int rt = r_tensor(ctx, logQ_max), rk = r_keyswitch(ctx, logQ_max);
  const size_t N = ctx->N;
  Carve cv(ws, ws_bytes);
  uint32_t* X = cv.take((size_t)cnum * 4 * rt * N);
  uint32_t* D = cv.take((size_t)cnum * 3 * L * N);
  uint32_t* Y = cv.take((size_t)cnum * 2 * rk * N);
  if (!cv.ok || ((uintptr_t)ws & 255)) {
    set_error("mult_ragged: workspace of %zu bytes too small or misaligned", ws_bytes);
    return FHE_EWORKSPACE;
  }
  const size_t ctw = 2 * (size_t)L * N;
  RET_IF(launch_lift(ctx, a, L, (size_t)L * N, ctw, X, (size_t)rt * N, 4 * (size_t)rt * N, 2, cnum, rt, st));
  RET_IF(launch_lift(ctx, b, L, (size_t)L * N, ctw, X + 2 * (size_t)rt * N, (size_t)rt * N, 4 * (size_t)rt * N, 2,
                     cnum, rt, st));
  RET_IF(launch_ring_tensor(ctx, X, rt, cnum, st));
  EpiArgs e0;
  e0.kind = Epi::kStore;
  e0.out_bits = logQ_max;
  e0.item_bits = item_bits;
  e0.out_limbs = L;
  RET_IF(launch_garner(ctx, X, (size_t)rt * N, 4 * (size_t)rt * N, rt, 3, cnum, D, (size_t)L * N,
                       3 * (size_t)L * N, e0, st));
  RET_IF(launch_lift_signed(ctx, D + 2 * (size_t)L * N, L, 0, 3 * (size_t)L * N, Y, 0, 2 * (size_t)rk * N, 1, cnum,
                            rk, 0, item_bits, st));
  return key_switch_tail(ctx, Y, ctx->evk, rk, cnum, logQ_max, k2, D, (size_t)L * N, 3 * (size_t)L * N, 2, out, st,
                         item_bits, L);
}

// Ragged batches of several rings (groups): the steps of mult_ragged, with each transform stage
// of all groups at N >= 2^13 launched once over a work table (one segment per group).
int mult_batch(const fhe_batch_group* gs, int ng, int k2, const fhe_batch_sched& sc, cudaStream_t st) {
  struct Bufs {
    int rt, rk, L;
    size_t N;
    uint32_t *X, *D, *Y;
  };
  std::vector<Bufs> v(ng);
  for (int i = 0; i < ng; ++i) {
    fhe_ctx* ctx = gs[i].ctx;
    Bufs& b = v[i];
    b.rt = r_tensor(ctx, gs[i].logQ_max);
    b.rk = r_keyswitch(ctx, gs[i].logQ_max);
    b.L = gs[i].L_pad;
    b.N = ctx->N;
    const size_t cnum = gs[i].cnum;
    Carve cv(gs[i].ws, gs[i].ws_bytes);
    b.X = cv.take(cnum * 4 * b.rt * b.N);
    b.D = cv.take(cnum * 3 * b.L * b.N);
    b.Y = cv.take(cnum * 2 * b.rk * b.N);
    if (!cv.ok || ((uintptr_t)gs[i].ws & 255)) {
      set_error("mult_relin_rescale_batch: workspace of group %d (%zu bytes) too small or misaligned", i,
                gs[i].ws_bytes);
      return FHE_EWORKSPACE;
    }
  }
  // groups at N <= 2^12 run their ring products per group (single-CTA transforms)
  auto tabled = [&](int i) { return gs[i].ctx->prm.logN >= 13; };
  int ntab = 0;
  for (int i = 0; i < ng; ++i) ntab += tabled(i);
  const fhe_ctx* pctx = gs[0].ctx;
  // one stage over every tabled group; rows of the column stages as in launch_ring_tensor / _key:
  //  tensor X = [nb][4][r][N]: forward over blocks 0..3 (row map {r, r}, 4 r nb rows), inverse over
  //  blocks 0..2 (row map {3r, 4r}, 3 r nb rows); key Y = [nb][2][r][N]: forward over block 0 (row
  //  map {r, 2r}, r nb rows), inverse over blocks 0..1 (row map {r, r}, 2 r nb rows)
  auto stage = [&](bool key, int stg) -> int {
    NttTable t{};
    t.unit_rows = sc.col_unit_rows;
    for (int i = 0; i < ng; ++i) {
      if (!tabled(i)) continue;
      const fhe_ctx* ctx = gs[i].ctx;
      NttSeg& g = t.seg[t.nseg++];
      const int r = key ? v[i].rk : v[i].rt, nb = gs[i].cnum;
      g.data = key ? v[i].Y : v[i].X;
      g.key = key ? ctx->evk.ntt : nullptr;
      g.krows = key ? ctx->evk.rows : 0;
      g.tw = stg == kTableColsInv ? ctx->d_ipsi2 : ctx->d_psi2;
      g.itw = ctx->d_ipsi2;
      g.q = ctx->d_q;
      g.qinv = ctx->d_qinv;
      g.r = r;
      g.logN = ctx->prm.logN;
      g.nb = nb;
      if (stg == kTableColsFwd) {
        g.group_rows = r;
        g.group_stride = key ? 2 * r : r;
        g.rows = (key ? 1 : 4) * r * nb;
      } else if (stg == kTableColsInv) {
        g.group_rows = key ? r : 3 * r;
        g.group_stride = key ? r : 4 * r;
        g.rows = (key ? 2 : 3) * r * nb;
      }
    }
    const int per_sm = stg == kTableColsFwd || stg == kTableColsInv ? sc.col_ctas_per_sm : sc.row_ctas_per_sm;
    return launch_ntt_table(pctx, t, stg, per_sm, st);
  };
  // tensor products: lifts per group, the three transform stages over the table, reconstructions
  for (int i = 0; i < ng; ++i) {
    const fhe_batch_group& g = gs[i];
    const Bufs& b = v[i];
    const size_t ctw = 2 * (size_t)b.L * b.N;
    RET_IF(launch_lift(g.ctx, g.a, b.L, (size_t)b.L * b.N, ctw, b.X, (size_t)b.rt * b.N, 4 * (size_t)b.rt * b.N, 2,
                       g.cnum, b.rt, st));
    RET_IF(launch_lift(g.ctx, g.b, b.L, (size_t)b.L * b.N, ctw, b.X + 2 * (size_t)b.rt * b.N, (size_t)b.rt * b.N,
                       4 * (size_t)b.rt * b.N, 2, g.cnum, b.rt, st));
    if (!tabled(i)) RET_IF(launch_ring_tensor(g.ctx, b.X, b.rt, g.cnum, st));
  }
  if (ntab) {
    RET_IF(stage(false, kTableColsFwd));
    RET_IF(stage(false, kTableRowsTensor));
    RET_IF(stage(false, kTableColsInv));
  }
  for (int i = 0; i < ng; ++i) {
    const fhe_batch_group& g = gs[i];
    const Bufs& b = v[i];
    EpiArgs e0;
    e0.kind = Epi::kStore;
    e0.out_bits = g.logQ_max;
    e0.item_bits = g.item_logQ;
    e0.out_limbs = b.L;
    RET_IF(launch_garner(g.ctx, b.X, (size_t)b.rt * b.N, 4 * (size_t)b.rt * b.N, b.rt, 3, g.cnum, b.D,
                         (size_t)b.L * b.N, 3 * (size_t)b.L * b.N, e0, st));
    RET_IF(launch_lift_signed(g.ctx, b.D + 2 * (size_t)b.L * b.N, b.L, 0, 3 * (size_t)b.L * b.N, b.Y, 0,
                              2 * (size_t)b.rk * b.N, 1, g.cnum, b.rk, 0, g.item_logQ, st));
    if (!tabled(i)) RET_IF(launch_ring_key(g.ctx, b.Y, g.ctx->evk.ntt, g.ctx->evk.rows, b.rk, g.cnum, st));
  }
  // key switches: the three transform stages over the table, then each group's epilogue
  if (ntab) {
    RET_IF(stage(true, kTableColsFwd));
    RET_IF(stage(true, kTableRowsKey));
    RET_IF(stage(true, kTableColsInv));
  }
  for (int i = 0; i < ng; ++i) {
    const fhe_batch_group& g = gs[i];
    const Bufs& b = v[i];
    RET_IF(key_switch_epilogue(g.ctx, b.Y, b.rk, g.cnum, g.logQ_max, k2, b.D, (size_t)b.L * b.N,
                               3 * (size_t)b.L * b.N, 2, g.out, st, g.item_logQ, b.L));
  }
  return FHE_OK;
}

int mult_impl(fhe_ctx* ctx, const fhe_ct* a, const fhe_ct* b, int k2, fhe_ct* out, void* ws, size_t ws_bytes,
              void* stream) {
  if (!ctx || !ct_ok(ctx, a) || !ct_ok(ctx, b) || !ct_ok(ctx, out)) {
    set_error("mult: null or malformed argument");
    return FHE_EINVAL;
  }
  if (a->logQ != b->logQ || (a->cnum != b->cnum && b->cnum != 1) || out->cnum != a->cnum) {
    set_error("mult: operands differ in level or batch size (b->cnum must equal a->cnum, or be 1 to broadcast)");
    return FHE_ELEVEL;
  }
  if (k2 < 0 || out->logQ != a->logQ - k2 || out->logQ < 1) {
    set_error("mult: output level %d != %d - %d", out->logQ, a->logQ, k2);
    return FHE_ELEVEL;
  }
  if (!ctx->have_keys) {
    set_error("mult: no relinearisation key (call fhe_keygen)");
    return FHE_ENOKEY;
  }
  if (out->data == a->data || out->data == b->data) {
    set_error("mult: out aliases an input");
    return FHE_EINVAL;
  }
  if (is_bgv(ctx)) {
    if (k2 != 0 || a->level != b->level || out->level != a->level) {
      set_error("mult (BGV): operands and output must share one level; no rescale");
      return FHE_ELEVEL;
    }
    return mult_bgv(ctx, a, b, out, ws, ws_bytes, (cudaStream_t)stream);
  }
  const int logQ = a->logQ, cnum = a->cnum, L = limbs_for_bits(logQ);
  const int rt = r_tensor(ctx, logQ), rk = r_keyswitch(ctx, logQ);
  const size_t N = ctx->N;
  Carve cv(ws, ws_bytes);
  uint32_t* X = cv.take((size_t)cnum * 4 * rt * N);
  uint32_t* D = cv.take((size_t)cnum * 3 * L * N);
  uint32_t* Y = cv.take((size_t)cnum * 2 * rk * N);
  if (!cv.ok || ((uintptr_t)ws & 255)) {
    set_error("mult: workspace of %zu bytes too small or misaligned", ws_bytes);
    return FHE_EWORKSPACE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ctw = 2 * (size_t)L * N;  // words per input ciphertext
  // tensor product: lift (b1, a1) and (b2, a2), 4 forward NTTs, 3 products, 3 INTTs, reconstruction
  const size_t btw = b->cnum == 1 ? 0 : ctw;  // broadcast mode: every item reads the one b
  RET_IF(launch_lift(ctx, a->data, L, (size_t)L * N, ctw, X, (size_t)rt * N, 4 * (size_t)rt * N, 2, cnum, rt, st));
  RET_IF(launch_lift(ctx, b->data, L, (size_t)L * N, btw, X + 2 * (size_t)rt * N, (size_t)rt * N,
                     4 * (size_t)rt * N, 2, cnum, rt, st));
  RET_IF(launch_ring_tensor(ctx, X, rt, cnum, st));
  EpiArgs e0;
  e0.kind = Epi::kStore;
  e0.out_bits = logQ;
  e0.out_limbs = L;
  RET_IF(launch_garner(ctx, X, (size_t)rt * N, 4 * (size_t)rt * N, rt, 3, cnum, D, (size_t)L * N,
                       3 * (size_t)L * N, e0, st));
  // relinearisation: centred d2 -> rk primes, times evk, round(/P), + (d0, d1), optional rescale
  RET_IF(launch_lift_signed(ctx, D + 2 * (size_t)L * N, L, 0, 3 * (size_t)L * N, Y, 0, 2 * (size_t)rk * N, 1, cnum,
                            rk, logQ, nullptr, st));
  RET_IF(key_switch_tail(ctx, Y, ctx->evk, rk, cnum, logQ, k2, D, (size_t)L * N, 3 * (size_t)L * N, 2, out->data,
                         st));
  out->log_scale = a->log_scale + b->log_scale - k2;
  return FHE_OK;
}

}  // namespace

extern "C" {

const char* fhe_last_error(void) { return fhe::last_error(); }

int fhe_primes_for_bound(int bound_bits) { return primes_for_bound_global(bound_bits); }

int fhe_set_forms(fhe_ctx* ctx, int crt, int lift, int ntt) {
  if (!ctx || crt < FHE_CRT_DIRECT || crt > FHE_CRT_DIRECT_CVT || lift < FHE_LIFT_AUTO || lift > FHE_LIFT_TC ||
      (ntt != FHE_NTT_FUSED && ntt != FHE_NTT_SPLIT && ntt != FHE_NTT_FUSED_GROUPS)) {
    set_error("set_forms: bad arguments (crt %d, lift %d, ntt %d)", crt, lift, ntt);
    return FHE_EINVAL;
  }
  ctx->crt_mode = crt;
  ctx->lift_form = lift;
  ctx->ntt_form = ntt;
  return FHE_OK;
}

int fhe_profile_reset(fhe_ctx* ctx, int enable) {
  if (!ctx) {
    set_error("profile_reset: null context");
    return FHE_EINVAL;
  }
  ctx->prof.reset(enable != 0);
  return FHE_OK;
}

int fhe_profile_read(fhe_ctx* ctx, int kclass, int64_t* launches, double* ms) {
  if (!ctx || kclass < 0 || kclass >= FHE_K_COUNT) {
    set_error("profile_read: bad arguments");
    return FHE_EINVAL;
  }
  if (launches) *launches = ctx->prof.launches[kclass];
  if (ms) {
    double total = 0.0;
    for (auto& pr : ctx->prof.ev[kclass]) {
      FHE_CHECK_CUDA(cudaEventSynchronize(pr.second));
      float t = 0.f;
      FHE_CHECK_CUDA(cudaEventElapsedTime(&t, pr.first, pr.second));
      total += t;
    }
    *ms = total;
  }
  return FHE_OK;
}

size_t fhe_ct_bytes(int logN, int logQ, int cnum) {
  if (logN < 0 || logN > kMaxLogN || logQ < 1 || cnum < 1) return 0;
  return (size_t)cnum * 2 * limbs_for_bits(logQ) * ((size_t)1 << logN) * 4;
}

int fhe_ctx_create(const fhe_params* p, fhe_alloc_fn alloc, fhe_free_fn free_, void* user, fhe_ctx** out) {
  if (!p || !out) {
    set_error("ctx_create: null argument");
    return FHE_EINVAL;
  }
  *out = nullptr;
  if ((p->scheme != FHE_SCHEME_CKKS && p->scheme != FHE_SCHEME_BGV) || p->logN < 3 || p->logN > kMaxLogN ||
      p->logQ < 1 || p->logP < 1 ||
      p->logQ + p->logP > 32 * (kMaxLimbs - 3) || (alloc == nullptr) != (free_ == nullptr) ||
      (p->crt != FHE_CRT_DIRECT && p->crt != FHE_CRT_GARNER && p->crt != FHE_CRT_DIRECT_INT &&
       p->crt != FHE_CRT_DIRECT_CVT)) {
    set_error("ctx_create: parameters out of range (logN %d, logQ %d, logP %d)", p->logN, p->logQ, p->logP);
    return FHE_EINVAL;
  }
  if (p->scheme == FHE_SCHEME_BGV) {
    const bool ok = p->t >= 3 && (p->t & 1u) && p->t < (1u << 31) && p->bgv_levels >= 1 && p->bgv_levels <= 64 &&
                    (p->bgv_q0 & 1u) && (p->bgv_r & 1u) && p->bgv_q0 % p->t == 1 % p->t && p->bgv_r % p->t == 1 % p->t &&
                    p->bgv_q0 > p->t && p->bgv_r > 256 && p->bgv_r < ((uint64_t)1 << 62) && p->logP < 32 * kBgvLimbs &&
                    p->logP >= p->logQ;
    if (!ok) {
      set_error("ctx_create: BGV chain parameters out of range (t odd, q0 = r = 1 mod t, odd, logP >= logQ)");
      return FHE_EINVAL;
    }
  }
  if (p->hamming_weight < 0 || p->hamming_weight > (1 << p->logN) || p->sigma < 0.0 || p->sigma > kMaxGaussSigma) {
    set_error("ctx_create: hamming_weight %d (0..N) or sigma %g (0..%g) out of range", p->hamming_weight, p->sigma,
              kMaxGaussSigma);
    return FHE_EINVAL;
  }
  GaussTable gt;
  if (gauss_table(p->sigma > 0.0 ? p->sigma : kDefaultSigma, &gt) != FHE_OK) {
    set_error("ctx_create: sigma %g gives no usable rounded-Gaussian table", p->sigma);
    return FHE_EINVAL;
  }
  const int R = primes_for_bound_global(p->logN + 2 * p->logQ + p->logP);
  if (R < 0) {
    set_error("ctx_create: more than %d primes needed", kMaxPrimes);
    return FHE_EINVAL;
  }
  fhe_ctx* ctx = new fhe_ctx();
  ctx->prm = *p;
  ctx->N = 1 << p->logN;
  ctx->alloc = alloc;
  ctx->free_ = free_;
  ctx->alloc_user = user;
  ctx->R = R;
  ctx->crt_mode = p->crt;
  ctx->gauss = gt;
  cudaGetDevice(&ctx->device);
  int rc = build_tables(ctx);
  if (rc == FHE_OK && p->scheme == FHE_SCHEME_BGV) {
    rc = build_bgv_tables(ctx);
    if (rc == FHE_OK && ctx->bgv_bits[p->bgv_levels] != p->logQ) {
      set_error("ctx_create: logQ = %d but q0 r^L has %d bits", p->logQ, ctx->bgv_bits[p->bgv_levels]);
      rc = FHE_EINVAL;
    }
  }
  if (rc != FHE_OK) {
    free_all(ctx);
    delete ctx;
    return rc;
  }
  *out = ctx;
  return FHE_OK;
}

int fhe_ctx_destroy(fhe_ctx* ctx) {
  if (!ctx) return FHE_OK;
  cudaDeviceSynchronize();
  free_all(ctx);
  delete ctx;
  return FHE_OK;
}

int fhe_sync(fhe_ctx* ctx) {
  (void)ctx;
  FHE_CHECK_CUDA(cudaDeviceSynchronize());
  FHE_CHECK_CUDA(cudaGetLastError());
  if (read_dev_status()) {
    set_error("a bounded device-side wait gave up (results of the preceding work are invalid)");
    return FHE_ETIMEOUT;
  }
  return FHE_OK;
}

size_t fhe_workspace_bytes(const fhe_ctx* ctx, int op, int logQ, int cnum) {
  if (!ctx || cnum < 1 || cnum > kMaxCnum || logQ < 1) return 0;
  size_t w = 0;
  switch (op) {
    case FHE_OP_MULT:
      if (logQ > ctx->prm.logQ) return 0;
      w = is_bgv(ctx) ? words_mult_bgv(ctx, logQ, cnum) : words_mult(ctx, logQ, cnum);
      break;
    case FHE_OP_ROTATE:
      if (logQ > ctx->prm.logQ) return 0;
      w = words_rotate(ctx, logQ, cnum);
      break;
    case FHE_OP_ENCRYPT:
      w = words_encrypt(ctx, cnum);
      if (w) w += enc_sampler_words(ctx, cnum);
      if (w && is_bgv(ctx))
        w += (size_t)cnum * ctx->N * 2 * bgv_prod_limbs(ctx->prm.logN + ctx->prm.logQ) + 64;
      break;
    case FHE_OP_DECRYPT:
      if (logQ > ctx->prm.logQ) return 0;
      w = words_decrypt(ctx, logQ, cnum);
      if (w && is_bgv(ctx)) w += (size_t)cnum * ctx->N * bgv_prod_limbs(ctx->prm.logN + logQ) + 64;
      break;
    case FHE_OP_KEYGEN: {
      const int r = ctx->R;
      w = 2 * (size_t)r * ctx->N + 64;
      break;
    }
    case FHE_OP_RING_MUL:
      w = words_ringmul(ctx, logQ, cnum);
      break;
    case FHE_OP_MULT_PLAIN:
      if (logQ > ctx->prm.logQ || is_bgv(ctx)) return 0;
      {
        const int r = r_tensor(ctx, logQ);
        if (r < 0) return 0;
        w = (size_t)cnum * ctx->N * 3 * (size_t)r + 2 * 64;  // the batch's two polynomials and up to cnum plaintexts
      }
      break;
    case FHE_OP_ENCODE:
      w = (size_t)cnum * ctx->N * 8;  // two complex double buffers
      break;
    case FHE_OP_MULT_RAGGED:
      if (logQ > ctx->prm.logQ) return 0;
      w = words_mult(ctx, logQ, cnum);
      break;
    default:
      return 0;
  }
  return w ? w * 4 + 1024 : 0;
}

int fhe_keygen_inject(fhe_ctx* ctx, const int8_t* s, const uint32_t* a_pk, const int32_t* e_pk,
                      const uint32_t* a_ev, const int32_t* e_ev) {
  if (!ctx || !s || !a_pk || !e_pk || !a_ev || !e_ev) {
    set_error("keygen: null argument");
    return FHE_EINVAL;
  }
  const size_t N = ctx->N;
  const int logQ = ctx->prm.logQ, logP = ctx->prm.logP;
  const int Lq = limbs_for_bits(logQ), Lpq = limbs_for_bits(logQ + logP);
  const int re = r_enc(ctx), rd = r_dec(ctx, logQ), R = ctx->R;
  // host secret -> int32
  std::vector<int32_t> s32(N);
  for (size_t i = 0; i < N; ++i) {
    if (s[i] < -1 || s[i] > 1) {
      set_error("keygen: secret coefficient %d out of {-1,0,1}", (int)s[i]);
      return FHE_EINVAL;
    }
    s32[i] = s[i];
  }
  // resident key memory (allocated once)
  if (!ctx->d_s) {
    ctx->d_s = (int32_t*)ctx_alloc(ctx, N * 4);
    ctx->d_pk = (uint32_t*)ctx_alloc(ctx, 2 * (size_t)Lq * N * 4);
    ctx->d_pk_ntt = (uint32_t*)ctx_alloc(ctx, 2 * (size_t)re * N * 4);
    ctx->d_s_ntt = (uint32_t*)ctx_alloc(ctx, (size_t)rd * N * 4);
    ctx->evk.ntt = (uint32_t*)ctx_alloc(ctx, 2 * (size_t)R * N * 4);
    if (!ctx->d_s || !ctx->d_pk || !ctx->d_pk_ntt || !ctx->d_s_ntt || !ctx->evk.ntt) {
      set_error("keygen: key allocation failed");
      return FHE_ENOMEM;
    }
  }
  ctx->r_enc = re;
  ctx->r_dec = rd;
  ctx->evk.rows = R;
  // scratch: inputs, s^2, a s, ring-product workspace (+ BGV reduction scratch)
  const int nxb = bgv_prod_limbs(ctx->prm.logN + logQ + logP);
  const size_t bgv_extra = is_bgv(ctx) ? (size_t)N * (4 * (size_t)nxb + 8 + Lq) : 0;
  const size_t scratch_words =
      (size_t)N * (2 + 1 + 1 + Lq + Lpq + 1 + (size_t)(nxb > Lpq ? nxb : Lpq) + 2 * Lpq) + 2 * (size_t)R * N +
      bgv_extra;
  uint32_t* scratch = (uint32_t*)ctx_alloc(ctx, scratch_words * 4);
  if (!scratch) {
    set_error("keygen: scratch allocation failed");
    return FHE_ENOMEM;
  }
  int32_t* d_epk = (int32_t*)scratch;
  int32_t* d_eev = d_epk + N;
  uint32_t* d_apk = (uint32_t*)(d_eev + N);
  uint32_t* d_aev = d_apk + (size_t)Lq * N;
  uint32_t* d_s2 = d_aev + (size_t)Lpq * N;        // 1 limb two's complement
  uint32_t* d_t = d_s2 + N;                        // two's complement of a_ev s (Lpq, BGV nxb limbs)
  uint32_t* d_evl = d_t + (size_t)(nxb > Lpq ? nxb : Lpq) * N;  // [2][Lpq][N] evk limbs
  uint32_t* rws = d_evl + 2 * (size_t)Lpq * N;     // 2 R N
  uint32_t* bsc = rws + 2 * (size_t)R * N;         // BGV: reduction scratch, then canonical a_pk
  cudaStream_t st = 0;
  int rc = FHE_OK;
  auto fail = [&](int code) {
    ctx_free(ctx, scratch);
    return code;
  };
  if (cudaMemcpy(ctx->d_s, s32.data(), N * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_epk, e_pk, N * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_eev, e_ev, N * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_apk, a_pk, (size_t)Lq * N * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_aev, a_ev, (size_t)Lpq * N * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("keygen: upload failed");
    return fail(FHE_ECUDA);
  }
  if (is_bgv(ctx)) {
    // BGV: pk = (-a s + t e, a) mod Q_L; evk = (-a' s + t e' + P s^2, a') mod P Q_L; inputs reduced first
    const int L = ctx->prm.bgv_levels;
    uint32_t* d_apk_c = bsc + (size_t)N * (4 * (size_t)nxb + 8);
    if ((rc = launch_bgv_reduce(ctx, d_apk, Lq, 0, 0, 1, 1, false, false, nullptr, nullptr, 0, nullptr, 0, 0, 0,
                                d_apk_c, 0, 0, L, st)))
      return fail(rc);
    const int nx1 = bgv_prod_limbs(ctx->prm.logN + logQ);
    EpiArgs ek;
    ek.kind = Epi::kStore;
    ek.out_bits = 32 * nx1;
    ek.out_limbs = nx1;
    if ((rc = ring_product(ctx, d_apk_c, Lq, nullptr, nullptr, 0, ctx->d_s, re, d_t, ek, rws, st))) return fail(rc);
    if ((rc = launch_bgv_reduce(ctx, d_t, nx1, 0, 0, 1, 1, true, true, d_epk, nullptr, 0, nullptr, 0, 0, 0, ctx->d_pk,
                                0, 0, L, st)))
      return fail(rc);
    if (cudaMemcpy(ctx->d_pk + (size_t)Lq * N, d_apk_c, (size_t)Lq * N * 4, cudaMemcpyDeviceToDevice) != cudaSuccess)
      return fail(FHE_ECUDA);
    // a' canonical mod P Q_L into the second evk poly
    if ((rc = launch_bgv_modpq(ctx, d_aev, Lpq, false, false, nullptr, nullptr, d_evl + (size_t)Lpq * N, Lpq, bsc,
                               st)))
      return fail(rc);
    EpiArgs e1;
    e1.kind = Epi::kStore;
    e1.out_bits = 32;
    e1.out_limbs = 1;
    if ((rc = ring_product(ctx, nullptr, 0, ctx->d_s, nullptr, 0, ctx->d_s, primes_for_bound(ctx, ctx->prm.logN + 1),
                           d_s2, e1, rws, st)))
      return fail(rc);
    const int nx2 = bgv_prod_limbs(ctx->prm.logN + logQ + logP);
    EpiArgs e2;
    e2.kind = Epi::kStore;
    e2.out_bits = 32 * nx2;
    e2.out_limbs = nx2;
    if ((rc = ring_product(ctx, d_evl + (size_t)Lpq * N, Lpq, nullptr, nullptr, 0, ctx->d_s,
                           primes_for_bound(ctx, ctx->prm.logN + logQ + logP), d_t, e2, rws, st)))
      return fail(rc);
    if ((rc = launch_bgv_modpq(ctx, d_t, nx2, true, true, d_eev, (const int32_t*)d_s2, d_evl, Lpq, bsc, st)))
      return fail(rc);
  } else {
  // pk = (-a s + e, a) mod Q
  {
    EpiArgs e;
    e.kind = Epi::kAddSmall;
    e.negate = 1;
    e.small = d_epk;
    e.out_bits = logQ;
    e.out_limbs = Lq;
    rc = ring_product(ctx, d_apk, Lq, nullptr, nullptr, 0, ctx->d_s, re, ctx->d_pk, e, rws, st);
    if (rc) return fail(rc);
    if (cudaMemcpy(ctx->d_pk + (size_t)Lq * N, d_apk, (size_t)Lq * N * 4, cudaMemcpyDeviceToDevice) != cudaSuccess)
      return fail(FHE_ECUDA);
  }
  // s^2 (|.| <= N, one limb two's complement) and a_ev s mod 2^(32 Lpq)
  {
    EpiArgs e;
    e.kind = Epi::kStore;
    e.out_bits = 32;
    e.out_limbs = 1;
    rc = ring_product(ctx, nullptr, 0, ctx->d_s, nullptr, 0, ctx->d_s, primes_for_bound(ctx, ctx->prm.logN + 1),
                      d_s2, e, rws, st);
    if (rc) return fail(rc);
    EpiArgs e2;
    e2.kind = Epi::kStore;
    e2.out_bits = 32 * Lpq;
    e2.out_limbs = Lpq;
    rc = ring_product(ctx, d_aev, Lpq, nullptr, nullptr, 0, ctx->d_s,
                      primes_for_bound(ctx, ctx->prm.logN + logQ + logP), d_t, e2, rws, st);
    if (rc) return fail(rc);
  }
  // evk_b = -a s + e + P s^2 mod PQ ; evk_a = a
  rc = launch_key_combine(ctx, d_t, Lpq, d_eev, d_s2, 1, logP, d_evl, logQ + logP, st);
  if (rc) return fail(rc);
  if (cudaMemcpy(d_evl + (size_t)Lpq * N, d_aev, (size_t)Lpq * N * 4, cudaMemcpyDeviceToDevice) != cudaSuccess)
    return fail(FHE_ECUDA);
  }
  // resident NTT forms
  if ((rc = to_ntt_form(ctx, d_evl, Lpq, 2, R, ctx->evk.ntt, st))) return fail(rc);
  if ((rc = to_ntt_form(ctx, ctx->d_pk, Lq, 2, re, ctx->d_pk_ntt, st))) return fail(rc);
  if ((rc = launch_lift_small(ctx, ctx->d_s, false, 0, ctx->d_s_ntt, 0, 1, rd, st))) return fail(rc);
  if ((rc = launch_ntt(ctx, ctx->d_s_ntt, 1, rd, rd, rd, false, st))) return fail(rc);
  if (cudaDeviceSynchronize() != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    set_error("keygen: device error %s", cudaGetErrorString(cudaGetLastError()));
    return fail(FHE_ECUDA);
  }
  ctx_free(ctx, scratch);
  ctx->have_keys = true;
  return FHE_OK;
}

}  // extern "C"

namespace {

// Switching key of the automorphism X -> X^g (rotation or conjugation, Sec. 6 rtk / ck):
// (-a s + e + P s(X^g), a) mod P Q in NTT form, stored under g.
int keygen_switch(fhe_ctx* ctx, uint32_t g, const uint32_t* a, const int32_t* e, const char* who) {
  if (ctx && is_bgv(ctx)) {
    set_error("%s: CKKS only", who);
    return FHE_EINVAL;
  }
  if (!ctx || !a || !e) {
    set_error("%s: null argument", who);
    return FHE_EINVAL;
  }
  if (!ctx->have_keys) {
    set_error("%s: generate the key set first", who);
    return FHE_ENOKEY;
  }
  const size_t N = ctx->N;
  const int logQ = ctx->prm.logQ, logP = ctx->prm.logP;
  const int Lpq = limbs_for_bits(logQ + logP), R = ctx->R;
  SwitchKey& K = ctx->rtk[g];
  if (!K.ntt) {
    K.ntt = (uint32_t*)ctx_alloc(ctx, 2 * (size_t)R * N * 4);
    K.rows = R;
    if (!K.ntt) {
      ctx->rtk.erase(g);
      set_error("%s: allocation failed", who);
      return FHE_ENOMEM;
    }
  }
  const size_t scratch_words = (size_t)N * (1 + 1 + Lpq + Lpq + 2 * Lpq) + 2 * (size_t)R * N;
  uint32_t* scratch = (uint32_t*)ctx_alloc(ctx, scratch_words * 4);
  if (!scratch) {
    set_error("%s: scratch allocation failed", who);
    return FHE_ENOMEM;
  }
  auto fail = [&](int code) {
    ctx_free(ctx, scratch);
    return code;
  };
  int32_t* d_e = (int32_t*)scratch;
  int32_t* d_ks = d_e + N;  // kappa(s), one limb two's complement
  uint32_t* d_a = (uint32_t*)(d_ks + N);
  uint32_t* d_t = d_a + (size_t)Lpq * N;
  uint32_t* d_kl = d_t + (size_t)Lpq * N;
  uint32_t* rws = d_kl + 2 * (size_t)Lpq * N;
  cudaStream_t st = 0;
  if (cudaMemcpy(d_e, e, N * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_a, a, (size_t)Lpq * N * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("%s: upload failed", who);
    return fail(FHE_ECUDA);
  }
  int rc = launch_automorph_small(ctx, ctx->d_s, d_ks, g, st);
  if (rc) return fail(rc);
  EpiArgs e2;
  e2.kind = Epi::kStore;
  e2.out_bits = 32 * Lpq;
  e2.out_limbs = Lpq;
  rc = ring_product(ctx, d_a, Lpq, nullptr, nullptr, 0, ctx->d_s, primes_for_bound(ctx, ctx->prm.logN + logQ + logP),
                    d_t, e2, rws, st);
  if (rc) return fail(rc);
  if ((rc = launch_key_combine(ctx, d_t, Lpq, d_e, (const uint32_t*)d_ks, 1, logP, d_kl, logQ + logP, st)))
    return fail(rc);
  if (cudaMemcpy(d_kl + (size_t)Lpq * N, d_a, (size_t)Lpq * N * 4, cudaMemcpyDeviceToDevice) != cudaSuccess)
    return fail(FHE_ECUDA);
  if ((rc = to_ntt_form(ctx, d_kl, Lpq, 2, R, K.ntt, st))) return fail(rc);
  if (cudaDeviceSynchronize() != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    set_error("%s: device error", who);
    return fail(FHE_ECUDA);
  }
  ctx_free(ctx, scratch);
  return FHE_OK;
}

}  // namespace

extern "C" {

int fhe_keygen_rotation(fhe_ctx* ctx, int step, const uint32_t* a, const int32_t* e) {
  return keygen_switch(ctx, ctx ? galois_of_step(ctx->N, step) : 0u, a, e, "keygen_rotation");
}

int fhe_keygen_conjugation(fhe_ctx* ctx, const uint32_t* a, const int32_t* e) {
  return keygen_switch(ctx, ctx ? 2u * ctx->N - 1u : 0u, a, e, "keygen_conjugation");
}

int fhe_keygen(fhe_ctx* ctx, uint64_t seed, const int* rot_steps, int n_rot) {
  if (!ctx || n_rot < 0 || (n_rot > 0 && !rot_steps)) {
    set_error("keygen: null context or bad rotation-step list");
    return FHE_EINVAL;
  }
  const int N = ctx->N, logQ = ctx->prm.logQ, logP = ctx->prm.logP;
  const bool bgv = is_bgv(ctx);
  // BGV reduces the uniform parts modulo Q and P Q itself: draw whole limbs
  const int bq = bgv ? 32 * limbs_for_bits(logQ) : logQ;
  const int bpq = bgv ? 32 * limbs_for_bits(logQ + logP) : logQ + logP;
  std::vector<int8_t> s(N);
  if (ctx->prm.hamming_weight > 0)
    sample_sparse_ternary(seed, kTagSecret, 0, N, ctx->prm.hamming_weight, s.data());
  else
    sample_ternary(seed, kTagSecret, 0, N, s.data());
  std::vector<uint32_t> a_pk((size_t)limbs_for_bits(bq) * N), a_ev((size_t)limbs_for_bits(bpq) * N);
  std::vector<int32_t> e_pk(N), e_ev(N);
  sample_uniform_limbs(seed, kTagPkA, 0, N, bq, a_pk.data());
  sample_gaussian(seed, kTagPkE, 0, N, ctx->gauss, e_pk.data());
  sample_uniform_limbs(seed, kTagEvA, 0, N, bpq, a_ev.data());
  sample_gaussian(seed, kTagEvE, 0, N, ctx->gauss, e_ev.data());
  RET_IF(fhe_keygen_inject(ctx, s.data(), a_pk.data(), e_pk.data(), a_ev.data(), e_ev.data()));
  if (bgv) {
    if (n_rot > 0) {
      set_error("keygen: rotation keys are CKKS only");
      return FHE_EINVAL;
    }
    return FHE_OK;
  }
  std::vector<uint32_t> a((size_t)limbs_for_bits(logQ + logP) * N);
  std::vector<int32_t> e(N);
  auto one = [&](uint32_t g, const char* who) {
    sample_uniform_limbs(seed, kTagSwA, g, N, logQ + logP, a.data());
    sample_gaussian(seed, kTagSwE, g, N, ctx->gauss, e.data());
    return keygen_switch(ctx, g, a.data(), e.data(), who);
  };
  for (int i = 0; i < n_rot; ++i) RET_IF(one(galois_of_step(N, rot_steps[i]), "keygen (rotation key)"));
  return one(2u * N - 1u, "keygen (conjugation key)");
}

int fhe_encrypt_inject(fhe_ctx* ctx, const uint32_t* pt, const int8_t* v, const int32_t* e0, const int32_t* e1,
                       fhe_ct* out, void* ws, size_t ws_bytes, void* stream) {
  if (!ctx || !pt || !v || !e0 || !e1 || !ct_ok(ctx, out)) {
    set_error("encrypt: null or malformed argument");
    return FHE_EINVAL;
  }
  if (!ctx->have_keys) {
    set_error("encrypt: no public key");
    return FHE_ENOKEY;
  }
  const int cnum = out->cnum, re = ctx->r_enc, logQ = out->logQ, L = limbs_for_bits(logQ);
  const size_t N = ctx->N;
  Carve cv(ws, ws_bytes);
  uint32_t* Y = cv.take((size_t)cnum * 2 * re * N);
  if (!cv.ok || ((uintptr_t)ws & 255)) {
    set_error("encrypt: workspace too small or misaligned");
    return FHE_EWORKSPACE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int nxe = is_bgv(ctx) ? bgv_prod_limbs(ctx->prm.logN + ctx->prm.logQ) : 0;
  uint32_t* T = is_bgv(ctx) ? cv.take((size_t)cnum * 2 * nxe * N) : nullptr;
  if (!cv.ok) {
    set_error("encrypt: workspace too small");
    return FHE_EWORKSPACE;
  }
  RET_IF(launch_lift_small(ctx, v, true, N, Y, 2 * (size_t)re * N, cnum, re, st));
  SwitchKey pk{ctx->d_pk_ntt, re};
  RET_IF(launch_ring_key(ctx, Y, pk.ntt, pk.rows, re, cnum, st));
  if (is_bgv(ctx)) {  // exact v pk, then (+ m + t e) mod Q_l
    EpiArgs ex;
    ex.kind = Epi::kStore;
    ex.out_bits = 32 * nxe;
    ex.out_limbs = nxe;
    RET_IF(launch_garner(ctx, Y, (size_t)re * N, 2 * (size_t)re * N, re, 2, cnum, T, (size_t)nxe * N,
                         2 * (size_t)nxe * N, ex, st));
    RET_IF(launch_bgv_reduce(ctx, T, nxe, (size_t)nxe * N, 2 * (size_t)nxe * N, 2, cnum, true, false, e0, e1, N, pt, 1,
                             0, (size_t)L * N, out->data, (size_t)L * N, 2 * (size_t)L * N, out->level, st));
    return check_launch();
  }
  EpiArgs e;
  e.kind = Epi::kAddSmall;
  e.out_bits = logQ;
  e.out_limbs = L;
  e.add = pt;
  e.add_limbs = L;
  e.add_bstride = (size_t)L * N;
  e.add_polys = 1;
  e.small = e0;
  e.small1 = e1;
  e.small_bstride = N;
  RET_IF(launch_garner(ctx, Y, (size_t)re * N, 2 * (size_t)re * N, re, 2, cnum, out->data, (size_t)L * N,
                       2 * (size_t)L * N, e, st));
  return check_launch();
}

int fhe_encrypt(fhe_ctx* ctx, const uint32_t* pt, uint64_t seed, fhe_ct* out, void* ws, size_t ws_bytes,
                void* stream) {
  if (!ctx || !pt || !ct_ok(ctx, out)) {
    set_error("encrypt: null or malformed argument");
    return FHE_EINVAL;
  }
  const size_t head = enc_sampler_bytes(ctx, out->cnum);
  if (!ws || ((uintptr_t)ws & 255) || ws_bytes < head) {
    set_error("encrypt: workspace of %zu bytes too small or misaligned", ws_bytes);
    return FHE_EWORKSPACE;
  }
  const size_t n = (size_t)out->cnum * ctx->N;
  int8_t* v = (int8_t*)ws;
  int32_t* e0 = (int32_t*)((uint8_t*)ws + align256(n));
  int32_t* e1 = (int32_t*)((uint8_t*)ws + align256(n) + align256(4 * n));
  if (!ctx->have_keys) {
    set_error("encrypt: no public key");
    return FHE_ENOKEY;
  }
  RET_IF(launch_sample_enc(ctx, seed, out->cnum, v, e0, e1, (cudaStream_t)stream));
  RET_IF(check_launch());
  return fhe_encrypt_inject(ctx, pt, v, e0, e1, out, (uint8_t*)ws + head, ws_bytes - head, stream);
}

int fhe_decrypt(fhe_ctx* ctx, const fhe_ct* in, uint32_t* pt_out, void* ws, size_t ws_bytes, void* stream) {
  if (!ctx || !ct_ok(ctx, in) || !pt_out) {
    set_error("decrypt: null or malformed argument");
    return FHE_EINVAL;
  }
  if (!ctx->have_keys) {
    set_error("decrypt: no secret key");
    return FHE_ENOKEY;
  }
  const int cnum = in->cnum, logQ = in->logQ, L = limbs_for_bits(logQ), rd = r_dec(ctx, logQ);
  const size_t N = ctx->N;
  Carve cv(ws, ws_bytes);
  uint32_t* Y = cv.take((size_t)cnum * rd * N);
  if (!cv.ok || ((uintptr_t)ws & 255) || rd > ctx->r_dec) {
    set_error("decrypt: workspace too small or misaligned");
    return FHE_EWORKSPACE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int nxd = is_bgv(ctx) ? bgv_prod_limbs(ctx->prm.logN + logQ) : 0;
  uint32_t* T = is_bgv(ctx) ? cv.take((size_t)cnum * nxd * N) : nullptr;
  if (!cv.ok) {
    set_error("decrypt: workspace too small");
    return FHE_EWORKSPACE;
  }
  RET_IF(launch_lift(ctx, in->data + (size_t)L * N, L, 0, 2 * (size_t)L * N, Y, 0, (size_t)rd * N, 1, cnum, rd, st));
  RET_IF(launch_ntt(ctx, Y, cnum, rd, rd, rd, false, st));
  RET_IF(launch_pointwise_mul(ctx, Y, Y, (size_t)rd * N, ctx->d_s_ntt, 0, rd, cnum, st));
  RET_IF(launch_ntt(ctx, Y, cnum, rd, rd, rd, true, st));
  if (is_bgv(ctx)) {  // exact a s, then [[b + a s]_{Q_l}]_t, one word per coefficient
    EpiArgs ex;
    ex.kind = Epi::kStore;
    ex.out_bits = 32 * nxd;
    ex.out_limbs = nxd;
    RET_IF(launch_garner(ctx, Y, 0, (size_t)rd * N, rd, 1, cnum, T, 0, (size_t)nxd * N, ex, st));
    RET_IF(launch_bgv_decrypt(ctx, T, nxd, (size_t)nxd * N, in->data, 2 * (size_t)L * N, pt_out, N, cnum, in->level,
                              st));
    return check_launch();
  }
  EpiArgs e;
  e.kind = Epi::kDecrypt;
  e.out_bits = logQ;
  e.out_limbs = L;
  e.add = in->data;
  e.add_limbs = L;
  e.add_bstride = 2 * (size_t)L * N;
  RET_IF(launch_garner(ctx, Y, 0, (size_t)rd * N, rd, 1, cnum, pt_out, 0, (size_t)L * N, e, st));
  return check_launch();
}

int fhe_mult_relin(fhe_ctx* ctx, const fhe_ct* a, const fhe_ct* b, fhe_ct* out, void* ws, size_t ws_bytes,
                   void* stream) {
  return mult_impl(ctx, a, b, 0, out, ws, ws_bytes, stream);
}

int fhe_mult_relin_rescale_ragged(fhe_ctx* ctx, const uint32_t* a, const uint32_t* b, uint32_t* out, int cnum,
                                  int L_pad, const int32_t* item_logQ, int logQ_max, int k, void* ws, size_t ws_bytes,
                                  void* stream) {
  if (!ctx || !a || !b || !out || !item_logQ || cnum < 1 || cnum > kMaxCnum || logQ_max < 1 ||
      logQ_max > ctx->prm.logQ || L_pad < limbs_for_bits(logQ_max) || L_pad > kMaxLiftLimbs || k < 0 ||
      k >= logQ_max || is_bgv(ctx)) {
    set_error("mult_relin_rescale_ragged: bad arguments");
    return FHE_EINVAL;
  }
  if (!ctx->have_keys) {
    set_error("mult_relin_rescale_ragged: no relinearisation key");
    return FHE_ENOKEY;
  }
  if (out == a || out == b) {
    set_error("mult_relin_rescale_ragged: out aliases an input");
    return FHE_EINVAL;
  }
  return mult_ragged(ctx, a, b, out, cnum, L_pad, item_logQ, logQ_max, k, ws, ws_bytes, (cudaStream_t)stream);
}

int fhe_mult_relin_rescale_batch(const fhe_batch_group* groups, int ngroups, int k, const fhe_batch_sched* sched,
                                 void* stream) {
  if (!groups || ngroups < 1 || ngroups > kTableSegs || k < 0) {
    set_error("mult_relin_rescale_batch: bad arguments (%d groups, k %d)", ngroups, k);
    return FHE_EINVAL;
  }
  const fhe_batch_sched sc = sched ? *sched : fhe_batch_sched{0, 0, 1};
  if (sc.col_ctas_per_sm < 0 || sc.row_ctas_per_sm < 0 || sc.col_unit_rows < 1) {
    set_error("mult_relin_rescale_batch: bad schedule (%d, %d, %d)", sc.col_ctas_per_sm, sc.row_ctas_per_sm,
              sc.col_unit_rows);
    return FHE_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_error("mult_relin_rescale_batch: no current device");
    return FHE_ECUDA;
  }
  for (int i = 0; i < ngroups; ++i) {
    const fhe_batch_group& g = groups[i];
    fhe_ctx* ctx = g.ctx;
    if (!ctx || !g.a || !g.b || !g.out || !g.item_logQ || g.cnum < 1 || g.cnum > kMaxCnum || g.logQ_max < 1 ||
        g.logQ_max > ctx->prm.logQ || g.L_pad < limbs_for_bits(g.logQ_max) || g.L_pad > kMaxLiftLimbs ||
        k >= g.logQ_max || is_bgv(ctx) || ctx->device != dev) {
      set_error("mult_relin_rescale_batch: group %d: bad arguments, BGV context or another device", i);
      return FHE_EINVAL;
    }
    if (!ctx->have_keys) {
      set_error("mult_relin_rescale_batch: group %d: no relinearisation key", i);
      return FHE_ENOKEY;
    }
    if (g.out == g.a || g.out == g.b) {
      set_error("mult_relin_rescale_batch: group %d: out aliases an input", i);
      return FHE_EINVAL;
    }
    // the bytes mult_batch carves from a group's workspace: X, D, Y
    auto carved = [](const fhe_batch_group& h) {
      const size_t N = h.ctx->N, c = h.cnum;
      return align256(c * 4 * r_tensor(h.ctx, h.logQ_max) * N * 4) + align256(c * 3 * h.L_pad * N * 4) +
             align256(c * 2 * r_keyswitch(h.ctx, h.logQ_max) * N * 4);
    };
    for (int j = 0; j < i; ++j) {
      const uintptr_t a0 = (uintptr_t)g.ws, a1 = a0 + carved(g), b0 = (uintptr_t)groups[j].ws,
                      b1 = b0 + carved(groups[j]);
      if (a0 < b1 && b0 < a1) {
        set_error("mult_relin_rescale_batch: workspaces of groups %d and %d overlap", j, i);
        return FHE_EWORKSPACE;
      }
    }
  }
  return mult_batch(groups, ngroups, k, sc, (cudaStream_t)stream);
}

int fhe_mult_relin_rescale(fhe_ctx* ctx, const fhe_ct* a, const fhe_ct* b, int k, fhe_ct* out, void* ws,
                           size_t ws_bytes, void* stream) {
  if (k < 1 || (ctx && is_bgv(ctx))) {
    set_error("mult_relin_rescale: CKKS only, k >= 1 (k = %d)", k);
    return FHE_EINVAL;
  }
  return mult_impl(ctx, a, b, k, out, ws, ws_bytes, stream);
}

int fhe_rescale(fhe_ctx* ctx, const fhe_ct* in, int k, fhe_ct* out, void* stream) {
  if (ctx && is_bgv(ctx)) {
    set_error("rescale: CKKS only (BGV uses fhe_moddown)");
    return FHE_EINVAL;
  }
  if (!ctx || !ct_ok(ctx, in) || !ct_ok(ctx, out) || k < 1 || out->logQ != in->logQ - k || out->cnum != in->cnum) {
    set_error("rescale: bad arguments");
    return FHE_EINVAL;
  }
  if (out->data == in->data && limbs_for_bits(out->logQ) != limbs_for_bits(in->logQ)) {
    set_error("rescale: in-place rescale must keep the limb count");
    return FHE_EINVAL;
  }
  RET_IF(launch_rescale(ctx, in->data, in->logQ, out->data, k, in->cnum * 2, (cudaStream_t)stream));
  out->log_scale = in->log_scale - k;
  return check_launch();
}

int fhe_moddown(fhe_ctx* ctx, const fhe_ct* in, fhe_ct* out, void* stream) {
  if (!ctx || !ct_ok(ctx, in) || !ct_ok(ctx, out) || out->logQ > in->logQ || out->cnum != in->cnum) {
    set_error("moddown: bad arguments");
    return FHE_EINVAL;
  }
  if (is_bgv(ctx)) {  // modulus switch Q_l -> Q_{l-1}
    if (out->level != in->level - 1 || out->data == in->data) {
      set_error("moddown (BGV): one level per call (out->level = in->level - 1), no aliasing");
      return FHE_ELEVEL;
    }
    const size_t N = ctx->N;
    RET_IF(launch_bgv_modswitch(ctx, in->data, (size_t)limbs_for_bits(in->logQ) * N, out->data,
                                (size_t)limbs_for_bits(out->logQ) * N, in->cnum * 2, in->level, (cudaStream_t)stream));
    return check_launch();
  }
  if (out->data == in->data && limbs_for_bits(out->logQ) != limbs_for_bits(in->logQ)) {
    set_error("moddown: in-place drop must keep the limb count");
    return FHE_EINVAL;
  }
  RET_IF(launch_moddown(ctx, in->data, in->logQ, out->data, out->logQ, in->cnum * 2, (cudaStream_t)stream));
  out->log_scale = in->log_scale;
  return check_launch();
}

static int addsub(fhe_ctx* ctx, const fhe_ct* a, const fhe_ct* b, fhe_ct* out, int mode, void* stream) {
  if (!ctx || !ct_ok(ctx, a) || !ct_ok(ctx, out) || (mode != 2 && !ct_ok(ctx, b))) {
    set_error("add/sub/negate: bad arguments");
    return FHE_EINVAL;
  }
  const bool bcast = mode != 2 && b->cnum == 1 && a->cnum > 1;
  if ((mode != 2 && (b->logQ != a->logQ || (b->cnum != a->cnum && !bcast))) || out->logQ != a->logQ ||
      out->cnum != a->cnum) {
    set_error("add/sub/negate: operand levels or batch sizes differ (b->cnum must equal a->cnum, or be 1)");
    return FHE_ELEVEL;
  }
  if (bcast && (out->data == b->data || is_bgv(ctx))) {
    set_error("add/sub (broadcast): CKKS only, out must not alias the broadcast operand");
    return FHE_EINVAL;
  }
  if (is_bgv(ctx)) {
    if ((mode != 2 && b->level != a->level) || out->level != a->level) {
      set_error("add/sub/negate (BGV): levels differ");
      return FHE_ELEVEL;
    }
    RET_IF(launch_bgv_addsub(ctx, a->data, mode == 2 ? a->data : b->data, out->data, a->cnum * 2, mode, a->level,
                             (cudaStream_t)stream));
    return check_launch();
  }
  if (mode != 2 && fabs(a->log_scale - b->log_scale) > 1e-9) {
    set_error("add/sub: operand scales differ (2^%g vs 2^%g)", a->log_scale, b->log_scale);
    return FHE_ELEVEL;
  }
  RET_IF(launch_addsub(ctx, a->data, mode == 2 ? a->data : b->data, out->data, a->logQ, a->cnum * 2, mode,
                       (cudaStream_t)stream, bcast ? 2 : 0));
  out->log_scale = a->log_scale;
  return check_launch();
}
int fhe_add(fhe_ctx* ctx, const fhe_ct* a, const fhe_ct* b, fhe_ct* out, void* stream) {
  return addsub(ctx, a, b, out, 0, stream);
}
int fhe_sub(fhe_ctx* ctx, const fhe_ct* a, const fhe_ct* b, fhe_ct* out, void* stream) {
  return addsub(ctx, a, b, out, 1, stream);
}
int fhe_negate(fhe_ctx* ctx, const fhe_ct* in, fhe_ct* out, void* stream) {
  return addsub(ctx, in, nullptr, out, 2, stream);
}
int fhe_mult_const(fhe_ctx* ctx, const fhe_ct* in, int32_t c, fhe_ct* out, void* stream) {
  if (ctx && is_bgv(ctx)) {
    set_error("mult_const: CKKS only");
    return FHE_EINVAL;
  }
  if (!ctx || !ct_ok(ctx, in) || !ct_ok(ctx, out) || out->logQ != in->logQ || out->cnum != in->cnum ||
      c == INT32_MIN) {
    set_error("mult_const: bad arguments");
    return FHE_EINVAL;
  }
  RET_IF(launch_mult_const(ctx, in->data, c, out->data, in->logQ, in->cnum * 2, (cudaStream_t)stream));
  out->log_scale = in->log_scale;
  return check_launch();
}

int fhe_add_const(fhe_ctx* ctx, const fhe_ct* in, int64_t value, int shift, fhe_ct* out, void* stream) {
  if (!ctx || is_bgv(ctx) || !ct_ok(ctx, in) || !ct_ok(ctx, out) || out->logQ != in->logQ || out->cnum != in->cnum ||
      shift < 0 || shift >= in->logQ) {
    set_error("add_const: bad arguments (CKKS, 0 <= shift < logQ)");
    return FHE_EINVAL;
  }
  const size_t bytes = fhe_ct_bytes(ctx->prm.logN, in->logQ, in->cnum);
  if (out->data != in->data)
    FHE_CHECK_CUDA(cudaMemcpyAsync(out->data, in->data, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  RET_IF(launch_add_const(ctx, out->data, out->data, value, nullptr, shift, in->logQ, in->cnum,
                          (cudaStream_t)stream));
  out->log_scale = in->log_scale;
  return check_launch();
}

int fhe_add_const_vec(fhe_ctx* ctx, const fhe_ct* in, const int64_t* values, int shift, fhe_ct* out, void* stream) {
  if (!ctx || !values || is_bgv(ctx) || !ct_ok(ctx, in) || !ct_ok(ctx, out) || out->logQ != in->logQ ||
      out->cnum != in->cnum || shift < 0 || shift >= in->logQ) {
    set_error("add_const_vec: bad arguments (CKKS, values non-null, 0 <= shift < logQ)");
    return FHE_EINVAL;
  }
  const size_t bytes = fhe_ct_bytes(ctx->prm.logN, in->logQ, in->cnum);
  if (out->data != in->data)
    FHE_CHECK_CUDA(cudaMemcpyAsync(out->data, in->data, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  RET_IF(launch_add_const(ctx, out->data, out->data, 0, values, shift, in->logQ, in->cnum, (cudaStream_t)stream));
  out->log_scale = in->log_scale;
  return check_launch();
}

int fhe_imult(fhe_ctx* ctx, const fhe_ct* in, fhe_ct* out, void* stream) {
  if (!ctx || is_bgv(ctx) || !ct_ok(ctx, in) || !ct_ok(ctx, out) || out->logQ != in->logQ || out->cnum != in->cnum ||
      out->data == in->data) {
    set_error("imult: bad arguments (CKKS, same level and batch, no aliasing)");
    return FHE_EINVAL;
  }
  RET_IF(launch_monomial(ctx, in->data, out->data, in->logQ, ctx->N / 2, in->cnum * 2, (cudaStream_t)stream));
  out->log_scale = in->log_scale;
  return check_launch();
}

int fhe_mult_plain(fhe_ctx* ctx, const fhe_ct* in, const uint32_t* pt, int pt_cnum, double pt_log_scale, fhe_ct* out,
                   void* ws, size_t ws_bytes, void* stream) {
  if (!ctx || is_bgv(ctx) || !pt || !ct_ok(ctx, in) || !ct_ok(ctx, out) || out->logQ != in->logQ ||
      out->cnum != in->cnum || out->data == in->data || (pt_cnum != 1 && pt_cnum != in->cnum)) {
    set_error("mult_plain: bad arguments (CKKS, pt_cnum 1 or cnum, same level and batch, no aliasing)");
    return FHE_EINVAL;
  }
  const int cnum = in->cnum, logQ = in->logQ, L = limbs_for_bits(logQ), r = r_tensor(ctx, logQ);
  const size_t N = ctx->N;
  Carve cv(ws, ws_bytes);
  uint32_t* X = cv.take((size_t)cnum * 2 * r * N);
  uint32_t* M = cv.take((size_t)pt_cnum * r * N);
  if (!cv.ok || ((uintptr_t)ws & 255)) {
    set_error("mult_plain: workspace of %zu bytes too small or misaligned", ws_bytes);
    return FHE_EWORKSPACE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t rN = (size_t)r * N;
  RET_IF(launch_lift(ctx, in->data, L, (size_t)L * N, 2 * (size_t)L * N, X, rN, 2 * rN, 2, cnum, r, st));
  RET_IF(launch_lift(ctx, pt, L, 0, (size_t)L * N, M, 0, rN, 1, pt_cnum, r, st));
  RET_IF(launch_ntt(ctx, X, cnum * 2, r, r, r, false, st));
  RET_IF(launch_ntt(ctx, M, pt_cnum, r, r, r, false, st));
  for (int p = 0; p < 2; ++p)
    RET_IF(launch_pointwise_mul_strided(ctx, X + p * rN, 2 * rN, X + p * rN, 2 * rN, M, pt_cnum == 1 ? 0 : rN, r, cnum,
                                        st));
  RET_IF(launch_ntt(ctx, X, cnum * 2, r, r, r, true, st));
  EpiArgs e;
  e.kind = Epi::kStore;
  e.out_bits = logQ;
  e.out_limbs = L;
  RET_IF(launch_garner(ctx, X, rN, 2 * rN, r, 2, cnum, out->data, (size_t)L * N, 2 * (size_t)L * N, e, st));
  out->log_scale = in->log_scale + pt_log_scale;
  return check_launch();
}

int fhe_rotate(fhe_ctx* ctx, const fhe_ct* in, int step, fhe_ct* out, void* ws, size_t ws_bytes, void* stream) {
  fhe_ct* outs[1] = {out};
  RET_IF(rotate_checks(ctx, in, outs, 1, "rotate"));
  const uint32_t g = galois_of_step(ctx->N, step);
  return rotate_many(ctx, in, &g, 1, outs, ws, ws_bytes, (cudaStream_t)stream);
}

int fhe_rotate_hoisted(fhe_ctx* ctx, const fhe_ct* in, const int* steps, int nsteps, fhe_ct* const* outs, void* ws,
                       size_t ws_bytes, void* stream) {
  if (!steps || nsteps < 1 || nsteps > 4096) {
    set_error("rotate_hoisted: steps null or nsteps %d out of 1..4096", nsteps);
    return FHE_EINVAL;
  }
  RET_IF(rotate_checks(ctx, in, outs, nsteps, "rotate_hoisted"));
  std::vector<uint32_t> gs(nsteps);
  for (int s = 0; s < nsteps; ++s) gs[s] = galois_of_step(ctx->N, steps[s]);
  return rotate_many(ctx, in, gs.data(), nsteps, outs, ws, ws_bytes, (cudaStream_t)stream);
}

int fhe_conjugate(fhe_ctx* ctx, const fhe_ct* in, fhe_ct* out, void* ws, size_t ws_bytes, void* stream) {
  fhe_ct* outs[1] = {out};
  RET_IF(rotate_checks(ctx, in, outs, 1, "conjugate"));
  const uint32_t g = 2u * ctx->N - 1u;
  return rotate_many(ctx, in, &g, 1, outs, ws, ws_bytes, (cudaStream_t)stream);
}

int fhe_ring_mul(fhe_ctx* ctx, const uint32_t* a, int La, const uint32_t* b, int Lb, int logOut, uint32_t* out,
                 int cnum, void* ws, size_t ws_bytes, void* stream) {
  if (!ctx || !a || !b || !out || La < 1 || Lb < 1 || La > kMaxLiftLimbs || Lb > kMaxLiftLimbs || logOut < 1 ||
      cnum < 1 || cnum > kMaxCnum) {
    set_error("ring_mul: bad arguments");
    return FHE_EINVAL;
  }
  const int r = primes_for_bound(ctx, ctx->prm.logN + 32 * (La + Lb));
  if (r < 0) {
    set_error("ring_mul: operands too wide for this context's primes");
    return FHE_EINVAL;
  }
  if (limbs_for_bits(logOut) > kMaxLimbs) {
    set_error("ring_mul: output too wide");
    return FHE_EINVAL;
  }
  const size_t N = ctx->N;
  Carve cv(ws, ws_bytes);
  uint32_t* RA = cv.take((size_t)cnum * r * N);
  uint32_t* RB = cv.take((size_t)cnum * r * N);
  if (!cv.ok || ((uintptr_t)ws & 255)) {
    set_error("ring_mul: workspace too small or misaligned");
    return FHE_EWORKSPACE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  RET_IF(launch_lift(ctx, a, La, 0, (size_t)La * N, RA, 0, (size_t)r * N, 1, cnum, r, st));
  RET_IF(launch_lift(ctx, b, Lb, 0, (size_t)Lb * N, RB, 0, (size_t)r * N, 1, cnum, r, st));
  RET_IF(launch_ntt(ctx, RA, cnum, r, r, r, false, st));
  RET_IF(launch_ntt(ctx, RB, cnum, r, r, r, false, st));
  RET_IF(launch_pointwise_mul(ctx, RA, RA, (size_t)r * N, RB, (size_t)r * N, r, cnum, st));
  RET_IF(launch_ntt(ctx, RA, cnum, r, r, r, true, st));
  EpiArgs e;
  e.kind = Epi::kStore;
  e.out_bits = logOut;
  e.out_limbs = limbs_for_bits(logOut);
  RET_IF(launch_garner(ctx, RA, 0, (size_t)r * N, r, 1, cnum, out, 0, (size_t)e.out_limbs * N, e, st));
  return check_launch();
}

}  // extern "C"
