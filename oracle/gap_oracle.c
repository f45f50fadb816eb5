/*
 * gap_oracle.c — TEST INFRASTRUCTURE ONLY.  A plain, slow, single-threaded
 * FP64 CPU statement of the GAP PageRank kernel, used to check the CUDA path.
 * Only the test suite, the smoke check and the CPU-baseline leg of the bench
 * may load it; the product library never links or calls it, and it shares no
 * code with the product (only the input generators feed both).
 *
 * Build flags: -O2 -ffp-contract=off (no fused multiply-add anywhere, so
 * every product and sum is rounded exactly as written).
 *
 * What it follows (GAP Benchmark Suite, Beamer, Asanovic & Patterson):
 *   - §2 notation: n = |V|, N+(v) out-neighbours, N-(v) in-neighbours.
 *   - §2.1 PageRank equation: PR(v) = (1-d)/|V| + d * sum_{u in N-(v)} PR(u)/|N+(u)|.
 *   - §2.1 tolerance equation: a result is correct when one more classical
 *     iteration changes the scores by a summed absolute change below 1e-4.
 *   - §2.3: duplicate edges and self-loops may be removed, neighbour lists
 *     may be reordered; the graph is held in CSR.
 *   - §3 PageRank verifier: serial, push direction, one extra iteration.
 *   - §2.1 Breadth-First Search: a parent array with parent[source] = source,
 *     -1 for unreachable vertices, an arc parent[v] -> v, and depth[v] =
 *     depth[parent[v]] + 1; §3 BFS verifier: serial BFS depths.
 *   - §2.1 Connected Components: vertices get the same label exactly when an
 *     undirected path joins them (weakly connected components of a digraph);
 *     §3 CC verifier: one traversal per label.
 * Readings where the paper is silent (dangling vertices drop their mass,
 * x0 = 1/n, strict '<', the newest iterate is returned) are listed at each
 * function below.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* qsort comparator for int32 neighbour ids */
static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/*
 * Build a CSR (row u lists the heads v of arcs u->v) from m draws (src[i],
 * dst[i]) — §2.3 allows dropping self-loops and duplicates and reordering
 * neighbours.  Textbook construction: count arcs per row, prefix-sum the
 * counts into offsets, scatter heads, sort each row ascending, then remove
 * repeated heads when `dedup`.  With `symmetrize`, each draw (u,v) also adds
 * (v,u).  The in-direction (CSC) is the same routine applied to (dst, src).
 *
 * offsets: int64[n+1] (out); idx: int32[capacity] (out), capacity must be at
 * least (symmetrize ? 2m : m); *m_out receives the number of arcs kept.
 * Returns 0, or -1 on a bad argument / vertex id, -2 on allocation failure.
 */
int oracle_build_csr(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int symmetrize,
                     int dedup, int drop_self_loops, int64_t* offsets, int32_t* idx,
                     int64_t* m_out) {
  if (n < 0 || m < 0) return -1;
  for (int64_t i = 0; i < m; ++i)
    if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return -1;
  int64_t* cursor = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!cursor) return -2;
  for (int64_t v = 0; v <= n; ++v) offsets[v] = 0;
  /* 1. count arcs per tail */
  for (int64_t i = 0; i < m; ++i) {
    int32_t u = src[i], v = dst[i];
    if (drop_self_loops && u == v) continue;
    offsets[u + 1] += 1;
    if (symmetrize) offsets[v + 1] += 1;
  }
  /* 2. inclusive scan of counts -> row starts */
  for (int64_t v = 0; v < n; ++v) offsets[v + 1] += offsets[v];
  for (int64_t v = 0; v < n; ++v) cursor[v] = offsets[v];
  /* 3. scatter heads */
  for (int64_t i = 0; i < m; ++i) {
    int32_t u = src[i], v = dst[i];
    if (drop_self_loops && u == v) continue;
    idx[cursor[u]++] = v;
    if (symmetrize) idx[cursor[v]++] = u;
  }
  /* 4. sort each row */
  for (int64_t v = 0; v < n; ++v) {
    int64_t len = offsets[v + 1] - offsets[v];
    if (len > 1) qsort(idx + offsets[v], (size_t)len, sizeof(int32_t), cmp_i32);
  }
  /* 5. remove repeated heads within a row, compacting in place */
  if (dedup) {
    int64_t w = 0;
    int64_t row_start = 0;
    for (int64_t v = 0; v < n; ++v) {
      int64_t b = row_start, e = offsets[v + 1];
      row_start = e;
      offsets[v] = w;
      for (int64_t j = b; j < e; ++j)
        if (j == b || idx[j] != idx[j - 1]) idx[w++] = idx[j];
    }
    offsets[n] = w;
  }
  *m_out = offsets[n];
  free(cursor);
  return 0;
}

/*
 * One classical push iteration (§2.1 equation, §3 verifier direction):
 *   c[u]   = x[u] / |N+(u)|   (0 when |N+(u)| = 0: a dangling vertex sends
 *                              nothing, so its mass leaves the system — the
 *                              equation sums only over real in-edges)
 *   s[v]   = sum over arcs u->v of c[u], accumulated by visiting u ascending
 *            and each row of the CSR in stored (ascending) order
 *   y[v]   = base[v] + d * s[v]
 * `base` is either the scalar (1-d)/n (plain PR, base_vec == NULL) or a
 * per-vertex vector (personalized PR).  Returns sum_v |y[v] - x[v]| summed in
 * ascending v.  `c` and `s` are caller scratch of length n.
 */
static double push_iteration(int64_t n, const int64_t* off, const int32_t* idx, double d,
                             double base, const double* base_vec, const double* x, double* y,
                             double* c, double* s) {
  for (int64_t u = 0; u < n; ++u) {
    int64_t deg = off[u + 1] - off[u];
    c[u] = deg > 0 ? x[u] / (double)deg : 0.0;
    s[u] = 0.0;
  }
  for (int64_t u = 0; u < n; ++u)
    for (int64_t j = off[u]; j < off[u + 1]; ++j) s[idx[j]] += c[u];
  double delta = 0.0;
  for (int64_t v = 0; v < n; ++v) {
    double b = base_vec ? base_vec[v] : base;
    double prod = d * s[v];
    y[v] = b + prod;
    double diff = y[v] - x[v];
    delta += diff < 0 ? -diff : diff;
  }
  return delta;
}

/*
 * Iterate the §2.1 equation from x0[v] = 1/n (reading: the paper does not
 * state x0; the uniform start has total mass 1).  After each iteration k the
 * summed change delta_k = sum_v |x_k[v] - x_{k-1}[v]| is recorded; the loop
 * stops after the first iteration with delta < tol (strict, as in the §2.1
 * tolerance equation) or after max_iters iterations.  The newest iterate is
 * returned (reading: since delta_{k+1} <= d * delta_k, the returned scores
 * also satisfy the §2.1 criterion).  tol = 0 gives a fixed iteration count.
 *
 * off/idx: out-CSR (push direction).  x: double[n] (out).  delta_hist:
 * double[max_iters] (out, may be NULL).  Returns the iteration count, or -1
 * on a bad argument, -2 on allocation failure.
 */
int oracle_pagerank(int64_t n, const int64_t* off, const int32_t* idx, double d, double tol,
                    int32_t max_iters, double* x, double* delta_hist) {
  if (n <= 0 || max_iters < 0) return -1;
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  double* c = (double*)malloc(sizeof(double) * (size_t)n);
  double* s = (double*)malloc(sizeof(double) * (size_t)n);
  if (!y || !c || !s) {
    free(y); free(c); free(s);
    return -2;
  }
  const double base = (1.0 - d) / (double)n;
  for (int64_t v = 0; v < n; ++v) x[v] = 1.0 / (double)n;
  int32_t k = 0;
  while (k < max_iters) {
    double delta = push_iteration(n, off, idx, d, base, NULL, x, y, c, s);
    memcpy(x, y, sizeof(double) * (size_t)n);
    if (delta_hist) delta_hist[k] = delta;
    ++k;
    if (delta < tol) break;
  }
  free(y); free(c); free(s);
  return k;
}

/*
 * oracle_pagerank continued from a given score vector: on entry x holds an
 * iterate x_k; up to max_iters further iterations are applied exactly as
 * oracle_pagerank applies them (the same push iteration, the same strict stop
 * test on each new delta).  So continuing x_k for j iterations gives
 * oracle_pagerank's x_{k+j} bit for bit, which lets one serial run serve
 * comparisons at several iteration counts.  Returns the iterations performed,
 * or -1 / -2 as oracle_pagerank.
 */
int oracle_pagerank_from(int64_t n, const int64_t* off, const int32_t* idx, double d, double tol,
                         int32_t max_iters, double* x, double* delta_hist) {
  if (n <= 0 || max_iters < 0) return -1;
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  double* c = (double*)malloc(sizeof(double) * (size_t)n);
  double* s = (double*)malloc(sizeof(double) * (size_t)n);
  if (!y || !c || !s) {
    free(y); free(c); free(s);
    return -2;
  }
  const double base = (1.0 - d) / (double)n;
  int32_t k = 0;
  while (k < max_iters) {
    double delta = push_iteration(n, off, idx, d, base, NULL, x, y, c, s);
    memcpy(x, y, sizeof(double) * (size_t)n);
    if (delta_hist) delta_hist[k] = delta;
    ++k;
    if (delta < tol) break;
  }
  free(y); free(c); free(s);
  return k;
}

/*
 * §3 verifier: one extra serial push iteration from a candidate score vector
 * y (e.g. a GPU result promoted to FP64); returns sum_v |y'[v] - y[v]| through
 * *delta.  The §2.1 criterion holds when *delta < 1e-4.
 */
int oracle_pr_verify(int64_t n, const int64_t* off, const int32_t* idx, double d, const double* y,
                     double* delta) {
  if (n <= 0) return -1;
  double* z = (double*)malloc(sizeof(double) * (size_t)n);
  double* c = (double*)malloc(sizeof(double) * (size_t)n);
  double* s = (double*)malloc(sizeof(double) * (size_t)n);
  if (!z || !c || !s) {
    free(z); free(c); free(s);
    return -2;
  }
  *delta = push_iteration(n, off, idx, d, (1.0 - d) / (double)n, NULL, y, z, c, s);
  free(z); free(c); free(s);
  return 0;
}

/*
 * The §2.1 equation evaluated for a few rows only, one by one, in pull form:
 * for each listed vertex v,
 *   out[i] = (1-d)/n + d * sum_{u in N-(v)} x[u] / |N+(u)|
 * with the in-neighbours u = in_idx[in_off[v] .. in_off[v+1]) taken in stored
 * order and x[u]/|N+(u)| = 0 for a vertex without out-neighbours (its mass is
 * dropped, as in push_iteration).  For a score vector y this gives y' on the
 * sampled rows, so sum |y'[v] - y[v]| over a uniform sample, scaled by n /
 * nrows, estimates the §3 verifier's summed change on graphs too large for a
 * full serial iteration.  Returns 0, or -1 on a bad argument.
 */
int oracle_pr_rows(int64_t n, const int64_t* in_off, const int32_t* in_idx, const int32_t* outdeg, double d,
                   const double* x, int64_t nrows, const int64_t* rows, double* out) {
  if (n <= 0 || nrows < 0) return -1;
  const double base = (1.0 - d) / (double)n;
  for (int64_t i = 0; i < nrows; ++i) {
    const int64_t v = rows[i];
    if (v < 0 || v >= n) return -1;
    double s = 0.0;
    for (int64_t j = in_off[v]; j < in_off[v + 1]; ++j) {
      const int32_t u = in_idx[j];
      if (u < 0 || u >= n) return -1;
      if (outdeg[u] > 0) s += x[u] / (double)outdeg[u];
    }
    double prod = d * s;
    out[i] = base + prod;
  }
  return 0;
}

/*
 * The personalized update (see oracle_ppr) for listed rows only, one by one:
 *   out[i] = (1-d) * t[v] + d * sum_{u in N-(v)} x[u] / |N+(u)|,
 * t uniform over the distinct seeds.  As oracle_pr_rows, it lets a sample of
 * rows check the one-more-iteration change of a score vector on graphs too
 * large for a serial run.  Returns 0, or -1 on a bad argument.
 */
int oracle_ppr_rows(int64_t n, const int64_t* in_off, const int32_t* in_idx, const int32_t* outdeg, double d,
                    const double* x, const int32_t* seeds, int32_t nseeds, int64_t nrows, const int64_t* rows,
                    double* out) {
  if (n <= 0 || nrows < 0 || nseeds <= 0) return -1;
  /* distinct seeds: sort a copy */
  int32_t* sd = (int32_t*)malloc(sizeof(int32_t) * (size_t)nseeds);
  if (!sd) return -1;
  memcpy(sd, seeds, sizeof(int32_t) * (size_t)nseeds);
  qsort(sd, (size_t)nseeds, sizeof(int32_t), cmp_i32);
  int32_t distinct = 0;
  for (int32_t i = 0; i < nseeds; ++i) {
    if (sd[i] < 0 || sd[i] >= n) { free(sd); return -1; }
    if (i == 0 || sd[i] != sd[i - 1]) sd[distinct++] = sd[i];
  }
  const double tval = 1.0 / (double)distinct;
  for (int64_t i = 0; i < nrows; ++i) {
    const int64_t v = rows[i];
    if (v < 0 || v >= n) { free(sd); return -1; }
    int seed = 0; /* binary search among the distinct seeds */
    int32_t lo = 0, hi = distinct - 1;
    while (lo <= hi) {
      const int32_t mid = (lo + hi) / 2;
      if (sd[mid] == v) { seed = 1; break; }
      if (sd[mid] < v) lo = mid + 1; else hi = mid - 1;
    }
    double s = 0.0;
    for (int64_t j = in_off[v]; j < in_off[v + 1]; ++j) {
      const int32_t u = in_idx[j];
      if (u < 0 || u >= n) { free(sd); return -1; }
      if (outdeg[u] > 0) s += x[u] / (double)outdeg[u];
    }
    const double b = seed ? (1.0 - d) * tval : 0.0;
    double prod = d * s;
    out[i] = b + prod;
  }
  free(sd);
  return 0;
}

/*
 * Personalized PageRank (not in the paper; the serving workload's variant of
 * the §2.1 equation): the teleport term (1-d)/n becomes (1-d) * t[v] with t
 * uniform over the seed set S (t[v] = 1/|S| for v in S, else 0).  Repeated
 * seeds count once.  Start x0 = t; stop rule and returned iterate as in
 * oracle_pagerank.  Returns the iteration count or a negative error.
 */
int oracle_ppr(int64_t n, const int64_t* off, const int32_t* idx, double d, double tol,
               int32_t max_iters, const int32_t* seeds, int32_t nseeds, double* x,
               double* delta_hist) {
  if (n <= 0 || max_iters < 0 || nseeds <= 0) return -1;
  for (int32_t i = 0; i < nseeds; ++i)
    if (seeds[i] < 0 || seeds[i] >= n) return -1;
  double* t = (double*)calloc((size_t)n, sizeof(double));
  double* bv = (double*)malloc(sizeof(double) * (size_t)n);
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  double* c = (double*)malloc(sizeof(double) * (size_t)n);
  double* s = (double*)malloc(sizeof(double) * (size_t)n);
  if (!t || !bv || !y || !c || !s) {
    free(t); free(bv); free(y); free(c); free(s);
    return -2;
  }
  int64_t distinct = 0;
  for (int32_t i = 0; i < nseeds; ++i)
    if (t[seeds[i]] == 0.0) {
      t[seeds[i]] = 1.0;
      ++distinct;
    }
  for (int64_t v = 0; v < n; ++v) {
    t[v] = t[v] != 0.0 ? 1.0 / (double)distinct : 0.0;
    bv[v] = (1.0 - d) * t[v];
    x[v] = t[v];
  }
  int32_t k = 0;
  while (k < max_iters) {
    double delta = push_iteration(n, off, idx, d, 0.0, bv, x, y, c, s);
    memcpy(x, y, sizeof(double) * (size_t)n);
    if (delta_hist) delta_hist[k] = delta;
    ++k;
    if (delta < tol) break;
  }
  free(t); free(bv); free(y); free(c); free(s);
  return k;
}

/* ------------------------------------------------ connected components --- */

/* Root of x in the union-find forest, halving the path on the way. */
static int32_t uf_find(int32_t* parent, int32_t x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]];
    x = parent[x];
  }
  return x;
}

/*
 * §2.1 Connected Components: label every vertex by its weakly connected
 * component (arcs read as undirected edges).  Textbook union-find: every arc
 * u->v of the CSR unites the sets of u and v; a union makes the smaller root
 * the parent, so each set's root is its smallest vertex id, and the label of
 * v is that root.  (The paper asks only for one distinct label per component;
 * the smallest member id is one such labelling, and it is unique, so a GPU
 * result can be compared with this one element by element.)
 * labels: int32[n] (out).  Returns 0, or -2 on allocation failure.
 */
int oracle_cc(int64_t n, const int64_t* off, const int32_t* idx, int32_t* labels) {
  for (int64_t v = 0; v < n; ++v) labels[v] = (int32_t)v;
  for (int64_t u = 0; u < n; ++u) {
    for (int64_t j = off[u]; j < off[u + 1]; ++j) {
      int32_t ru = uf_find(labels, (int32_t)u), rv = uf_find(labels, idx[j]);
      if (ru == rv) continue;
      if (ru < rv) labels[rv] = ru;
      else labels[ru] = rv;
    }
  }
  for (int64_t v = 0; v < n; ++v) labels[v] = uf_find(labels, (int32_t)v);
  return 0;
}

/*
 * §3 CC verifier: for each distinct label, one breadth-first traversal over
 * the undirected graph (out- and in-arcs) from a vertex carrying it; the
 * traversal must meet no other label, and after all traversals every vertex
 * must have been reached (two components sharing a label leave one of them
 * unreached).  Any labelling can be checked, not only smallest-id labels.
 * Returns 1 if `labels` passes, 0 if not, -1 on a label outside [0, n),
 * -2 on allocation failure.
 */
int oracle_cc_verify(int64_t n, const int64_t* off, const int32_t* idx, const int32_t* labels) {
  for (int64_t v = 0; v < n; ++v)
    if (labels[v] < 0 || labels[v] >= n) return -1;
  const int64_t m = off[n];
  /* reverse arcs: in-direction CSR */
  int64_t* roff = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int32_t* ridx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int32_t* first = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  uint8_t* seen = (uint8_t*)calloc((size_t)n + 1, 1);
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int ok = 1;
  if (!roff || !ridx || !cur || !first || !seen || !queue) {
    ok = -2;
    goto done;
  }
  for (int64_t j = 0; j < m; ++j) roff[idx[j] + 1] += 1;
  for (int64_t v = 0; v < n; ++v) roff[v + 1] += roff[v];
  for (int64_t v = 0; v < n; ++v) cur[v] = roff[v];
  for (int64_t u = 0; u < n; ++u)
    for (int64_t j = off[u]; j < off[u + 1]; ++j) ridx[cur[idx[j]]++] = (int32_t)u;
  /* one start vertex per label: the first vertex carrying it */
  for (int64_t v = 0; v < n; ++v) first[v] = -1;
  for (int64_t v = 0; v < n; ++v)
    if (first[labels[v]] < 0) first[labels[v]] = (int32_t)v;
  for (int64_t l = 0; l < n && ok == 1; ++l) {
    if (first[l] < 0) continue;
    int64_t head = 0, tail = 0;
    queue[tail++] = first[l];
    seen[first[l]] = 1;
    while (head < tail && ok == 1) {
      const int32_t u = queue[head++];
      for (int dir = 0; dir < 2 && ok == 1; ++dir) {
        const int64_t* o = dir ? roff : off;
        const int32_t* x = dir ? ridx : idx;
        for (int64_t j = o[u]; j < o[u + 1]; ++j) {
          const int32_t w = x[j];
          if (labels[w] != labels[u]) {
            ok = 0;
            break;
          }
          if (!seen[w]) {
            seen[w] = 1;
            queue[tail++] = w;
          }
        }
      }
    }
  }
  for (int64_t v = 0; v < n && ok == 1; ++v)
    if (!seen[v]) ok = 0;
done:
  free(roff);
  free(ridx);
  free(cur);
  free(first);
  free(seen);
  free(queue);
  return ok;
}

/* --------------------------------------------- breadth-first search --- */

/*
 * Depths from `source` by a plain FIFO breadth-first search over the out-arcs
 * of the CSR (§3: the BFS verifier's trivial serial BFS).  depth: int32[n]
 * (out), -1 where unreachable.  Returns the number of reached vertices, or -1
 * on a bad source, -2 on allocation failure.
 */
int64_t oracle_bfs_depths(int64_t n, const int64_t* off, const int32_t* idx, int32_t source, int32_t* depth) {
  if (source < 0 || source >= n) return -1;
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!queue) return -2;
  for (int64_t v = 0; v < n; ++v) depth[v] = -1;
  int64_t head = 0, tail = 0;
  depth[source] = 0;
  queue[tail++] = source;
  while (head < tail) {
    const int32_t u = queue[head++];
    for (int64_t j = off[u]; j < off[u + 1]; ++j) {
      const int32_t v = idx[j];
      if (depth[v] < 0) {
        depth[v] = depth[u] + 1;
        queue[tail++] = v;
      }
    }
  }
  free(queue);
  return tail;
}

/* Is there an arc u -> v?  Rows of the CSR are sorted ascending: binary search. */
static int has_arc(const int64_t* off, const int32_t* idx, int32_t u, int32_t v) {
  int64_t lo = off[u], hi = off[u + 1];
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (idx[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo < off[u + 1] && idx[lo] == v;
}

/*
 * §3 BFS verifier for a parent array (§2.1 BFS definition): parent[source] =
 * source; parent[v] = -1 exactly where v is unreachable; otherwise the arc
 * parent[v] -> v exists and depth[parent[v]] = depth[v] - 1, with depths
 * from oracle_bfs_depths.  The CSR rows must be sorted (as oracle_build_csr
 * makes them).  Returns 1 if `parent` passes, 0 if not, -1 on a bad source,
 * -2 on allocation failure.
 */
int oracle_bfs_verify(int64_t n, const int64_t* off, const int32_t* idx, int32_t source, const int32_t* parent) {
  int32_t* depth = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!depth) return -2;
  const int64_t reached = oracle_bfs_depths(n, off, idx, source, depth);
  if (reached < 0) {
    free(depth);
    return (int)reached;
  }
  int ok = parent[source] == source;
  for (int64_t v = 0; v < n && ok; ++v) {
    if (v == source) continue;
    const int32_t p = parent[v];
    if (depth[v] < 0) {
      ok = p == -1;
    } else {
      ok = p >= 0 && p < n && has_arc(off, idx, p, (int32_t)v) && depth[p] == depth[v] - 1;
    }
  }
  free(depth);
  return ok;
}
