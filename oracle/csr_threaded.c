/*
 * csr_threaded.c — TEST INFRASTRUCTURE ONLY.  A row-partitioned threaded twin
 * of oracle_build_csr (gap_oracle.c) for graphs whose serial build would take
 * many minutes (2^26 vertices, 2.1e9 arcs).  It performs the same textbook
 * construction (§2.3: self-loops and duplicates may be dropped, neighbour
 * lists may be reordered; the graph is held in CSR): count the arcs of every
 * row, prefix-sum the counts, scatter the heads, sort every row ascending,
 * drop repeated heads.  Thread t owns the rows [r0, r1) and reads every draw,
 * keeping the arcs whose tail is one of its rows, so no two threads write the
 * same memory and the result does not depend on the thread count.  Its output
 * equals oracle_build_csr's bit for bit (pinned by the CPU tests).
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the bench
 * load it; it shares no code with the product.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int cmp_i32_t(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

typedef struct {
  int64_t n, m;
  const int32_t* src;
  const int32_t* dst;
  int symmetrize, dedup, drop_self_loops;
  int64_t r0, r1;       /* rows owned */
  int64_t i0, i1;       /* draws checked for valid ids */
  int64_t* cnt;         /* [n]: arcs per row, then kept arcs per row */
  int64_t* start;       /* [n+1]: row starts in tmp */
  int32_t* tmp;         /* unsorted / sorted rows, before compaction */
  const int64_t* offsets; /* final row starts (phase 4) */
  int32_t* idx;         /* final heads */
  int phase;
  int bad;
} job_t;

static void* worker(void* p) {
  job_t* j = (job_t*)p;
  const int32_t* src = j->src;
  const int32_t* dst = j->dst;
  if (j->phase == 0) { /* ids in [0, n) */
    for (int64_t i = j->i0; i < j->i1; ++i)
      if (src[i] < 0 || src[i] >= j->n || dst[i] < 0 || dst[i] >= j->n) j->bad = 1;
  } else if (j->phase == 1) { /* 1. count arcs per owned tail */
    for (int64_t i = 0; i < j->m; ++i) {
      const int32_t u = src[i], v = dst[i];
      if (j->drop_self_loops && u == v) continue;
      if (u >= j->r0 && u < j->r1) j->cnt[u] += 1;
      if (j->symmetrize && v >= j->r0 && v < j->r1) j->cnt[v] += 1;
    }
  } else if (j->phase == 2) { /* 3. scatter heads of owned rows (cnt becomes a cursor) */
    /* touch the owned part of tmp in order first, so its pages are mapped by
       this thread in sequence rather than faulted in at random by the scatter */
    memset(j->tmp + j->start[j->r0], 0, sizeof(int32_t) * (size_t)(j->start[j->r1] - j->start[j->r0]));
    for (int64_t v = j->r0; v < j->r1; ++v) j->cnt[v] = j->start[v];
    for (int64_t i = 0; i < j->m; ++i) {
      const int32_t u = src[i], v = dst[i];
      if (j->drop_self_loops && u == v) continue;
      if (u >= j->r0 && u < j->r1) j->tmp[j->cnt[u]++] = v;
      if (j->symmetrize && v >= j->r0 && v < j->r1) j->tmp[j->cnt[v]++] = u;
    }
    /* 4. sort each owned row; 5. count the heads kept after dropping repeats */
    for (int64_t v = j->r0; v < j->r1; ++v) {
      int32_t* row = j->tmp + j->start[v];
      const int64_t len = j->start[v + 1] - j->start[v];
      if (len > 1) qsort(row, (size_t)len, sizeof(int32_t), cmp_i32_t);
      int64_t kept = len;
      if (j->dedup && len > 1) {
        kept = 1;
        for (int64_t k = 1; k < len; ++k)
          if (row[k] != row[k - 1]) row[kept++] = row[k];
      }
      j->cnt[v] = kept;
    }
  } else { /* copy the kept heads of owned rows to their final places */
    for (int64_t v = j->r0; v < j->r1; ++v)
      memcpy(j->idx + j->offsets[v], j->tmp + j->start[v], sizeof(int32_t) * (size_t)j->cnt[v]);
  }
  return NULL;
}

static int run_phase(job_t* jobs, int t, int phase) {
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)t);
  if (!th) return -2;
  int started = 0;
  for (int k = 0; k < t; ++k) {
    jobs[k].phase = phase;
    if (pthread_create(&th[k], NULL, worker, &jobs[k]) != 0) break;
    ++started;
  }
  for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
  free(th);
  return started == t ? 0 : -2;
}

/*
 * Same contract as oracle_build_csr: offsets int64[n+1] (out), idx
 * int32[capacity] with capacity >= (symmetrize ? 2m : m) (out), *m_out the
 * arcs kept.  nthreads >= 1.  Returns 0, -1 on a bad argument / vertex id,
 * -2 on allocation or thread failure.
 */
int oracle_build_csr_threaded(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int symmetrize,
                              int dedup, int drop_self_loops, int64_t* offsets, int32_t* idx, int64_t* m_out,
                              int nthreads) {
  if (n < 0 || m < 0 || nthreads < 1) return -1;
  int t = nthreads;
  if (n > 0 && t > n) t = (int)n;
  if (t < 1) t = 1;
  job_t* jobs = (job_t*)calloc((size_t)t, sizeof(job_t));
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t* start = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!jobs || !cnt || !start) {
    free(jobs); free(cnt); free(start);
    return -2;
  }
  for (int k = 0; k < t; ++k) {
    job_t* j = &jobs[k];
    j->n = n; j->m = m; j->src = src; j->dst = dst;
    j->symmetrize = symmetrize; j->dedup = dedup; j->drop_self_loops = drop_self_loops;
    j->r0 = n * k / t; j->r1 = n * (k + 1) / t;
    j->i0 = m * k / t; j->i1 = m * (k + 1) / t;
    j->cnt = cnt; j->start = start;
  }
  int rc = run_phase(jobs, t, 0);
  for (int k = 0; k < t && rc == 0; ++k)
    if (jobs[k].bad) rc = -1;
  if (rc == 0) rc = run_phase(jobs, t, 1);
  int32_t* tmp = NULL;
  if (rc == 0) { /* 2. row starts: exclusive prefix sum of the counts */
    start[0] = 0;
    for (int64_t v = 0; v < n; ++v) start[v + 1] = start[v] + cnt[v];
    tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(start[n] > 0 ? start[n] : 1));
    if (!tmp) rc = -2;
  }
  if (rc == 0) {
    for (int k = 0; k < t; ++k) jobs[k].tmp = tmp;
    rc = run_phase(jobs, t, 2);
  }
  if (rc == 0) { /* final offsets from the kept counts */
    offsets[0] = 0;
    for (int64_t v = 0; v < n; ++v) offsets[v + 1] = offsets[v] + cnt[v];
    for (int k = 0; k < t; ++k) {
      jobs[k].offsets = offsets;
      jobs[k].idx = idx;
    }
    rc = run_phase(jobs, t, 3);
  }
  if (rc == 0) *m_out = offsets[n];
  free(tmp); free(jobs); free(cnt); free(start);
  return rc;
}
