/*
 * gapgen_core.h — per-edge arithmetic of the synthetic graph generators,
 * shared verbatim by the host library (gapgen.c) and the device library
 * (gapgen_cuda.cu) so that both produce bit-identical edge lists.
 *
 * Counter-based randomness: value(s, i) is the i-th output of a splitmix64
 * sequence whose state starts at s (Steele, Lea & Flood, OOPSLA 2014), so
 * every edge is a pure function of (seed, stream, index).  Only integer
 * arithmetic is used here, so x86, Arm and the GPU agree exactly.
 */
#ifndef GAPGEN_CORE_H
#define GAPGEN_CORE_H
#include <stdint.h>

#ifdef __CUDACC__
#define GAPGEN_HD __host__ __device__ __forceinline__
#else
#define GAPGEN_HD static inline
#endif

#define GAPGEN_GOLDEN 0x9E3779B97F4A7C15ULL

GAPGEN_HD uint64_t gapgen_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* i-th output (i >= 0) of splitmix64 whose state starts at `seed`. */
GAPGEN_HD uint64_t gapgen_sm64(uint64_t seed, uint64_t i) {
  return gapgen_mix64(seed + (i + 1) * GAPGEN_GOLDEN);
}

/* Independent stream key for (seed, stream id). */
GAPGEN_HD uint64_t gapgen_stream_key(uint64_t seed, uint64_t stream) {
  return gapgen_mix64(seed ^ gapgen_mix64(stream * GAPGEN_GOLDEN + 0x632BE59BD9B4E019ULL));
}

/* Uniform integer in [0, n) from the high 32 bits (multiply-shift). */
GAPGEN_HD uint32_t gapgen_bounded32(uint64_t r, uint64_t n) {
  return (uint32_t)(((r >> 32) * n) >> 32);
}

/* Keyed bijection on [0, 2^bits): four rounds of (x*odd + c) mod 2^bits and
 * an xorshift, each a bijection on bits-wide integers. */
typedef struct {
  int bits, shift;
  uint64_t mask, mul[4], add[4];
} gapgen_perm_t;

GAPGEN_HD void gapgen_perm_init(gapgen_perm_t* p, int bits, uint64_t seed) {
  p->bits = bits;
  p->mask = bits >= 64 ? ~0ULL : ((1ULL << bits) - 1);
  int sh = bits / 2 + 1;
  if (sh >= bits) sh = bits - 1;
  p->shift = sh < 1 ? 1 : sh;
  for (int r = 0; r < 4; ++r) {
    p->mul[r] = (gapgen_sm64(seed, 2 * r) | 1ULL) & p->mask;
    if (p->mul[r] == 0) p->mul[r] = 1;
    p->add[r] = gapgen_sm64(seed, 2 * r + 1) & p->mask;
  }
}

GAPGEN_HD uint64_t gapgen_perm(const gapgen_perm_t* p, uint64_t x) {
  if (p->bits <= 1) return x;
  for (int r = 0; r < 4; ++r) {
    x = (x * p->mul[r] + p->add[r]) & p->mask;
    x ^= x >> p->shift;
  }
  return x;
}

/* ---- uniform random draws ---- */
typedef struct {
  int64_t n;
  uint64_t ks, kd;
} gapgen_urand_t;

GAPGEN_HD void gapgen_urand_init(gapgen_urand_t* a, int64_t n, uint64_t seed) {
  a->n = n;
  a->ks = gapgen_stream_key(seed, 1);
  a->kd = gapgen_stream_key(seed, 2);
}

GAPGEN_HD void gapgen_urand_edge(const gapgen_urand_t* a, uint64_t i, int32_t* u, int32_t* v) {
  *u = (int32_t)gapgen_bounded32(gapgen_sm64(a->ks, i), (uint64_t)a->n);
  *v = (int32_t)gapgen_bounded32(gapgen_sm64(a->kd, i), (uint64_t)a->n);
}

/* ---- Kronecker / R-MAT draws ---- */
typedef struct {
  int scale, permute;
  uint64_t key;
  uint32_t tA, tAB, tABC;
  gapgen_perm_t perm;
} gapgen_kron_t;

/* Thresholds are floor(p * 2^32), computed by the caller (host) so the
 * device never touches floating point. */
GAPGEN_HD void gapgen_kron_init(gapgen_kron_t* a, int scale, uint32_t tA, uint32_t tAB,
                                uint32_t tABC, uint64_t seed, int permute) {
  a->scale = scale;
  a->permute = permute;
  a->key = gapgen_stream_key(seed, 3);
  a->tA = tA;
  a->tAB = tAB;
  a->tABC = tABC;
  gapgen_perm_init(&a->perm, scale, gapgen_stream_key(seed, 4));
}

/* Each level picks a quadrant: A -> (0,0), B -> (0,1), C -> (1,0), D -> (1,1);
 * two levels share one 64-bit draw (low half first). */
GAPGEN_HD void gapgen_kron_edge(const gapgen_kron_t* a, uint64_t i, int32_t* u_out, int32_t* v_out) {
  const uint64_t words = (uint64_t)((a->scale + 1) / 2);
  uint64_t u = 0, v = 0;
  for (int l = 0; l < a->scale; l += 2) {
    uint64_t w = gapgen_sm64(a->key, i * words + (uint64_t)(l >> 1));
    for (int h = 0; h < 2 && l + h < a->scale; ++h) {
      uint32_t r = h ? (uint32_t)(w >> 32) : (uint32_t)w;
      uint64_t bu = (r >= a->tAB) ? 1u : 0u;
      uint64_t bv = ((r >= a->tA && r < a->tAB) || r >= a->tABC) ? 1u : 0u;
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
  }
  if (a->permute) {
    u = gapgen_perm(&a->perm, u);
    v = gapgen_perm(&a->perm, v);
  }
  *u_out = (int32_t)u;
  *v_out = (int32_t)v;
}

/* ---- Chung-Lu draws from a prebuilt alias table ---- */
GAPGEN_HD uint32_t gapgen_alias_draw(const uint32_t* thresh, const uint32_t* alias, int64_t n,
                                     uint64_t r) {
  uint32_t col = gapgen_bounded32(r, (uint64_t)n);
  uint32_t coin = (uint32_t)r;
  return coin < thresh[col] ? col : alias[col];
}

typedef struct {
  int64_t n;
  uint64_t ks, kd;
  gapgen_perm_t ps, pd;
} gapgen_cl_t;

GAPGEN_HD void gapgen_cl_init(gapgen_cl_t* a, int64_t n, int bits, uint64_t seed) {
  a->n = n;
  a->ks = gapgen_stream_key(seed, 6);
  a->kd = gapgen_stream_key(seed, 7);
  gapgen_perm_init(&a->ps, bits, gapgen_stream_key(seed, 8));
  gapgen_perm_init(&a->pd, bits, gapgen_stream_key(seed, 9));
}

GAPGEN_HD void gapgen_cl_edge(const gapgen_cl_t* a, const uint32_t* thresh, const uint32_t* alias,
                              uint64_t i, int32_t* u, int32_t* v) {
  uint32_t s = gapgen_alias_draw(thresh, alias, a->n, gapgen_sm64(a->ks, i));
  uint32_t t = gapgen_alias_draw(thresh, alias, a->n, gapgen_sm64(a->kd, i));
  *u = (int32_t)gapgen_perm(&a->ps, s);
  *v = (int32_t)gapgen_perm(&a->pd, t);
}

#endif
