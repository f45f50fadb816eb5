/*
 * cpu_pull_omp.c — a multi-core CPU baseline of the GAP PageRank kernel, for
 * the benchmark's CPU comparison only (TEST INFRASTRUCTURE, like the oracle;
 * shares no code with the CUDA path).  It runs the §2.1 PageRank equation in
 * the pull direction over the CSC (the §3 formulation), rows split across
 * OpenMP threads, FP64, until the summed change is below tol (§2.1 tolerance
 * equation).  Built without OpenMP it runs on one thread.
 */
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int cpu_pull_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* x: double[n] out.  Returns the iteration count, or -1 / -2 on a bad argument
 * / allocation failure. */
int cpu_pagerank_pull(int64_t n, const int64_t* in_off, const int32_t* in_idx, const int32_t* outdeg, double d,
                      double tol, int32_t max_iters, double* x) {
  if (n <= 0 || max_iters < 0) return -1;
  double* c = (double*)malloc(sizeof(double) * (size_t)n);
  if (!c) return -2;
  const double base = (1.0 - d) / (double)n;
  for (int64_t v = 0; v < n; ++v) x[v] = 1.0 / (double)n;
  int32_t k = 0;
  while (k < max_iters) {
    int64_t u;
#pragma omp parallel for schedule(static)
    for (u = 0; u < n; ++u) c[u] = outdeg[u] > 0 ? x[u] / (double)outdeg[u] : 0.0;
    double delta = 0.0;
    int64_t v;
#pragma omp parallel for schedule(dynamic, 4096) reduction(+ : delta)
    for (v = 0; v < n; ++v) {
      double s = 0.0;
      for (int64_t j = in_off[v]; j < in_off[v + 1]; ++j) s += c[in_idx[j]];
      const double y = base + d * s;
      const double diff = y - x[v];
      delta += diff < 0 ? -diff : diff;
      x[v] = y; /* in place is safe: this iteration reads only c */
    }
    ++k;
    if (delta < tol) break;
  }
  free(c);
  return k;
}
