/*
 * gapgen — seeded synthetic input graphs shaped like the GAP benchmark's
 * inputs (paper §2.2): uniform random (Erdos-Renyi, "urand"), Kronecker /
 * R-MAT with the Graph 500 parameters ("kron"), road-like 2D grids with
 * random edge deletions, and Chung-Lu power-law digraphs.
 *
 * This module holds no PageRank arithmetic.  It only draws edge lists, and
 * both the CPU oracle and the CUDA path consume its output.  The per-edge
 * arithmetic lives in gapgen_core.h, shared with the device generator, so
 * host and device lists are bit-identical.  Results do not depend on the
 * thread count, as paper §3 asks of its generators.  The Chung-Lu weights use
 * libm pow(); tests compare GPU and oracle on edges drawn on one machine.
 */
#include "gapgen_core.h"

#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

uint64_t gapgen_splitmix64_at(uint64_t seed, uint64_t i) { return gapgen_sm64(seed, i); }

uint64_t gapgen_perm_apply(int bits, uint64_t seed, uint64_t x) {
  gapgen_perm_t p;
  gapgen_perm_init(&p, bits, seed);
  return gapgen_perm(&p, x);
}

uint32_t gapgen_prob_threshold(double p) {
  double t = floor(p * 4294967296.0);
  if (t < 0) return 0;
  return t >= 4294967296.0 ? 0xFFFFFFFFu : (uint32_t)t;
}

/* ---- thread fan-out over an index range ---- */
typedef struct {
  int kind;
  int64_t lo, hi;
  const void* args;
  const uint32_t *thresh, *alias;
  int32_t *src, *dst;
} job_t;

static void* job_main(void* p) {
  job_t* j = (job_t*)p;
  for (int64_t i = j->lo; i < j->hi; ++i) {
    if (j->kind == 0)
      gapgen_urand_edge((const gapgen_urand_t*)j->args, (uint64_t)i, &j->src[i], &j->dst[i]);
    else if (j->kind == 1)
      gapgen_kron_edge((const gapgen_kron_t*)j->args, (uint64_t)i, &j->src[i], &j->dst[i]);
    else
      gapgen_cl_edge((const gapgen_cl_t*)j->args, j->thresh, j->alias, (uint64_t)i, &j->src[i],
                     &j->dst[i]);
  }
  return NULL;
}

static int fan_out(int kind, int64_t m, const void* args, const uint32_t* thresh,
                   const uint32_t* alias, int32_t* src, int32_t* dst, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (m < 65536) nthreads = 1;
  job_t jobs[256];
  pthread_t th[256];
  int64_t per = (m + nthreads - 1) / nthreads;
  int started = 0;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].kind = kind;
    jobs[t].lo = (int64_t)t * per < m ? (int64_t)t * per : m;
    jobs[t].hi = (int64_t)(t + 1) * per < m ? (int64_t)(t + 1) * per : m;
    jobs[t].args = args;
    jobs[t].thresh = thresh;
    jobs[t].alias = alias;
    jobs[t].src = src;
    jobs[t].dst = dst;
  }
  for (int t = 1; t < nthreads; ++t) {
    if (pthread_create(&th[t], NULL, job_main, &jobs[t]) != 0) break;
    started = t;
  }
  job_main(&jobs[0]);
  for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
  for (int t = started + 1; t < nthreads; ++t) job_main(&jobs[t]);
  return 0;
}

/* Uniform random digraph draws: m pairs (u, v), u and v uniform in [0, n). */
int gapgen_urand(int64_t n, int64_t m, uint64_t seed, int32_t* src, int32_t* dst, int nthreads) {
  if (n <= 0 || n > 2147483647LL || m < 0) return -1;
  gapgen_urand_t a;
  gapgen_urand_init(&a, n, seed);
  return fan_out(0, m, &a, NULL, NULL, src, dst, nthreads);
}

/* Kronecker / R-MAT draws: m pairs on 2^scale vertices, quadrant
 * probabilities (A, B, C, 1-A-B-C) per level, then a seeded relabelling. */
int gapgen_kron(int scale, int64_t m, double A, double B, double C, uint64_t seed, int permute,
                int32_t* src, int32_t* dst, int nthreads) {
  if (scale < 1 || scale > 31 || m < 0) return -1;
  if (A < 0 || B < 0 || C < 0 || A + B + C > 1.0) return -1;
  gapgen_kron_t a;
  gapgen_kron_init(&a, scale, gapgen_prob_threshold(A), gapgen_prob_threshold(A + B),
                   gapgen_prob_threshold(A + B + C), seed, permute);
  return fan_out(1, m, &a, NULL, NULL, src, dst, nthreads);
}

/* Road-like grid: rows x cols lattice, vertex id r*cols + c, undirected
 * 4-neighbour edges (right and down neighbours listed once), each deleted
 * independently with probability p_del.  Capacity needed: 2*rows*cols. */
int gapgen_grid(int64_t rows, int64_t cols, double p_del, uint64_t seed, int32_t* src, int32_t* dst,
                int64_t* m_out) {
  if (rows <= 0 || cols <= 0 || rows * cols > 2147483647LL || p_del < 0 || p_del > 1) return -1;
  uint64_t key = gapgen_stream_key(seed, 5);
  double t = floor(p_del * 4294967296.0);
  uint64_t thr = t >= 4294967296.0 ? 0x100000000ULL : (uint64_t)t;
  int64_t k = 0;
  for (int64_t r = 0; r < rows; ++r) {
    for (int64_t c = 0; c < cols; ++c) {
      int64_t v = r * cols + c;
      for (int dir = 0; dir < 2; ++dir) {
        int64_t w;
        if (dir == 0) {
          if (c + 1 >= cols) continue;
          w = v + 1;
        } else {
          if (r + 1 >= rows) continue;
          w = v + cols;
        }
        uint64_t h = gapgen_sm64(key, (uint64_t)(2 * v + dir));
        if ((uint64_t)(uint32_t)(h >> 32) < thr) continue; /* deleted */
        src[k] = (int32_t)v;
        dst[k] = (int32_t)w;
        ++k;
      }
    }
  }
  *m_out = k;
  return 0;
}

/* Chung-Lu alias table: expected degrees w_i = s*(i+1)^(-1/(gamma-1)), capped
 * at `cap`, with s chosen by bisection so that sum_i w_i = m; Vose's alias
 * method (1991) turns w into (thresh, alias) for O(1) draws. */
int gapgen_chunglu_table(int64_t n, int64_t m, double gamma, double cap, uint32_t* thresh,
                         uint32_t* alias) {
  if (n <= 1 || n > 2147483647LL || m < 0 || gamma <= 1.0) return -1;
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  int64_t* small = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int64_t* large = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  double* prob = (double*)malloc(sizeof(double) * (size_t)n);
  if (!w || !small || !large || !prob) {
    free(w); free(small); free(large); free(prob);
    return -2;
  }
  double ex = -1.0 / (gamma - 1.0);
  for (int64_t i = 0; i < n; ++i) w[i] = pow((double)(i + 1), ex);
  double lo = 0.0, hi = 1.0;
  for (;;) {
    double tot = 0;
    for (int64_t i = 0; i < n; ++i) tot += fmin(hi * w[i], cap);
    if (tot >= (double)m || hi > 1e300) break;
    hi *= 2.0;
  }
  for (int it = 0; it < 64; ++it) {
    double mid = 0.5 * (lo + hi), tot = 0;
    for (int64_t i = 0; i < n; ++i) tot += fmin(mid * w[i], cap);
    if (tot < (double)m) lo = mid; else hi = mid;
  }
  double total = 0;
  for (int64_t i = 0; i < n; ++i) {
    w[i] = fmin(hi * w[i], cap);
    total += w[i];
  }
  int64_t ns = 0, nl = 0;
  for (int64_t i = 0; i < n; ++i) {
    prob[i] = w[i] * (double)n / total;
    if (prob[i] < 1.0) small[ns++] = i; else large[nl++] = i;
  }
  for (int64_t i = 0; i < n; ++i) alias[i] = (uint32_t)i;
  while (ns > 0 && nl > 0) {
    int64_t s = small[--ns], l = large[--nl];
    thresh[s] = gapgen_prob_threshold(prob[s]);
    alias[s] = (uint32_t)l;
    prob[l] = (prob[l] + prob[s]) - 1.0;
    if (prob[l] < 1.0) small[ns++] = l; else large[nl++] = l;
  }
  while (nl > 0) thresh[large[--nl]] = 0xFFFFFFFFu;
  while (ns > 0) thresh[small[--ns]] = 0xFFFFFFFFu;
  free(w); free(small); free(large); free(prob);
  return 0;
}

/* Chung-Lu digraph draws from a table made by gapgen_chunglu_table.  Sources
 * and targets are relabelled by two independent seeded bijections so that
 * out-degree and target popularity are uncorrelated and IDs carry no
 * locality.  n must be a power of two. */
int gapgen_chunglu_draw(int64_t n, int64_t m, uint64_t seed, const uint32_t* thresh,
                        const uint32_t* alias, int32_t* src, int32_t* dst, int nthreads) {
  if (n <= 1 || n > 2147483647LL || (n & (n - 1)) != 0 || m < 0) return -1;
  int bits = 0;
  while ((1LL << bits) < n) ++bits;
  gapgen_cl_t a;
  gapgen_cl_init(&a, n, bits, seed);
  return fan_out(2, m, &a, thresh, alias, src, dst, nthreads);
}
