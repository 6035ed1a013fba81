// BGV constants and launchers (see k_bgv.cu).
#pragma once

#include "common.cuh"

namespace fhe {

constexpr int kBgvLimbs = 16;    // chain moduli up to 512 bits
constexpr int kBgvInLimbs = 48;  // two's-complement inputs of the reductions up to 1536 bits

// One level of the chain Q_l = q0 r^l, in device memory.
struct BgvLevel {
  uint32_t q[kBgvLimbs];                       // Q_l, zero padded
  uint32_t R[kBgvInLimbs + 1][kBgvLimbs];      // 2^(32 j) mod Q_l
  uint32_t negR[kBgvInLimbs + 1][kBgvLimbs];   // (-2^(32 j)) mod Q_l
  double qtop;                                 // Q_l / 2^(32 (nl - 1))
  int32_t nl;                                  // limbs of Q_l
  uint32_t q_mod_t;                            // Q_l mod t
  uint64_t rpow[kBgvLimbs];                    // 2^(32 j) mod r
  uint32_t rinv[kBgvLimbs + 2];                // r^-1 mod 2^(32 (kBgvLimbs + 2))
};

struct BgvConsts {
  uint32_t t;
  int32_t logP;
  uint64_t r;
  uint64_t tinv_r;              // t^-1 mod r
  uint32_t tpow[kBgvLimbs];     // 2^(32 j) mod t
  uint32_t tinvP[kBgvLimbs];    // t^-1 mod 2^logP
};

int build_bgv_tables(fhe_ctx* ctx);

int launch_bgv_reduce(const fhe_ctx* ctx, const uint32_t* X, int nx, size_t xp, size_t xb, int npoly, int nbatch,
                      bool is_signed, bool negate, const int32_t* e0, const int32_t* e1, size_t eb, const uint32_t* add,
                      int add_polys, size_t ap, size_t ab, uint32_t* out, size_t op, size_t ob, int level,
                      cudaStream_t st);
int launch_bgv_keyswitch(const fhe_ctx* ctx, const uint32_t* Y, int ny, size_t yp, size_t yb, const uint32_t* d,
                         int add_polys, size_t dp, size_t db, uint32_t* out, size_t op, size_t ob, int nbatch,
                         int level, uint32_t* scratch, size_t sp, size_t sb, cudaStream_t st);
int launch_bgv_modswitch(const fhe_ctx* ctx, const uint32_t* in, size_t ip, uint32_t* out, size_t op, int npolys,
                         int level, cudaStream_t st);
int launch_bgv_decrypt(const fhe_ctx* ctx, const uint32_t* X, int nx, size_t xb, const uint32_t* b, size_t bb,
                       uint32_t* out, size_t ob, int nbatch, int level, cudaStream_t st);
int launch_bgv_modpq(const fhe_ctx* ctx, const uint32_t* X, int nx, bool is_signed, bool negate, const int32_t* e,
                     const int32_t* s2, uint32_t* out, int nout, uint32_t* scratch, cudaStream_t st);
int launch_bgv_addsub(const fhe_ctx* ctx, const uint32_t* a, const uint32_t* b, uint32_t* out, int npolys, int mode,
                      int level, cudaStream_t st);

}  // namespace fhe
