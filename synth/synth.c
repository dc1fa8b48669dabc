/*
 * Seeded synthetic inputs for the random-walk engine and its oracle.
 *
 * This module holds no arithmetic of the walk method itself: it only makes
 * graphs (R-MAT edge lists turned into sorted, de-duplicated CSR), per-edge
 * weights and labels, walk sources and MetaPath schemas.  Every value is a
 * pure function of (seed, tag, index) through a counter-based SplitMix64
 * mix (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014), so results do not depend on the thread count.
 *
 * Graph model: R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004) with
 * quadrant probabilities (a, b, c, 1-a-b-c), no noise and no vertex
 * permutation.  Self-loops are dropped, rows are sorted and de-duplicated.
 * An undirected graph stores each edge in both directions (the paper's
 * Section 2.1 convention); weights and labels are keyed on the unordered
 * pair so both directions agree.
 */
#define _GNU_SOURCE
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

#define SYN_TAG_RMAT 3u
#define SYN_TAG_WEIGHT 4u
#define SYN_TAG_LABEL 5u
#define SYN_TAG_SOURCE 1u
#define SYN_TAG_SCHEMA 2u

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* Counter-based draw: the i-th 64-bit value of stream (seed, tag). */
static inline uint64_t syn_u64(uint64_t seed, uint32_t tag, uint64_t i) {
  uint64_t k = mix64(seed ^ ((uint64_t)tag << 56) ^ 0x5851f42d4c957f2dULL);
  return mix64(k + (i + 1) * 0x9e3779b97f4a7c15ULL);
}

uint64_t syn_draw(uint64_t seed, uint32_t tag, uint64_t i) { return syn_u64(seed, tag, i); }

static int syn_threads(int nthreads) {
  if (nthreads > 0) return nthreads;
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  if (n < 1) n = 1;
  if (n > 64) n = 64;
  return (int)n;
}

/* ---------------------------------------------------------------- R-MAT */

typedef struct {
  int scale;
  uint64_t seed;
  uint32_t ta, tab, tabc; /* cumulative quadrant thresholds, floor(p * 2^32) */
} rmat_cfg;

static inline void rmat_edge(const rmat_cfg* c, uint64_t e, uint32_t* src, uint32_t* dst) {
  uint32_t u = 0, v = 0;
  const int words = (c->scale + 1) / 2;
  int level = 0;
  for (int k = 0; k < words; ++k) {
    uint64_t r = syn_u64(c->seed, SYN_TAG_RMAT, e * (uint64_t)words + (uint64_t)k);
    for (int h = 0; h < 2 && level < c->scale; ++h, ++level) {
      uint32_t x = (uint32_t)(r >> (32 * h));
      uint32_t bu, bv;
      if (x < c->ta) { bu = 0; bv = 0; }
      else if (x < c->tab) { bu = 0; bv = 1; }
      else if (x < c->tabc) { bu = 1; bv = 0; }
      else { bu = 1; bv = 1; }
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
  }
  *src = u;
  *dst = v;
}

typedef struct {
  const rmat_cfg* cfg;
  uint64_t e0, e1;
  int symmetric;
  int phase;              /* 0 = count degrees, 1 = scatter */
  uint32_t* cnt;          /* phase 0: per-vertex counters (atomic) */
  int64_t* fill;          /* phase 1: per-vertex next slot (atomic) */
  int32_t* tmp_col;
} rmat_job;

static void* rmat_worker(void* arg) {
  rmat_job* j = (rmat_job*)arg;
  for (uint64_t e = j->e0; e < j->e1; ++e) {
    uint32_t u, v;
    rmat_edge(j->cfg, e, &u, &v);
    if (u == v) continue;
    if (j->phase == 0) {
      __atomic_fetch_add(&j->cnt[u], 1u, __ATOMIC_RELAXED);
      if (j->symmetric) __atomic_fetch_add(&j->cnt[v], 1u, __ATOMIC_RELAXED);
    } else {
      int64_t p = __atomic_fetch_add(&j->fill[u], 1, __ATOMIC_RELAXED);
      j->tmp_col[p] = (int32_t)v;
      if (j->symmetric) {
        p = __atomic_fetch_add(&j->fill[v], 1, __ATOMIC_RELAXED);
        j->tmp_col[p] = (int32_t)u;
      }
    }
  }
  return NULL;
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

static inline void sort_row(int32_t* a, int64_t n) {
  if (n <= 24) {
    for (int64_t i = 1; i < n; ++i) {
      int32_t x = a[i];
      int64_t k = i - 1;
      while (k >= 0 && a[k] > x) { a[k + 1] = a[k]; --k; }
      a[k + 1] = x;
    }
  } else {
    qsort(a, (size_t)n, sizeof(int32_t), cmp_i32);
  }
}

typedef struct {
  int64_t nv;
  const int64_t* tmp_ptr;
  int32_t* tmp_col;
  int64_t* deg;          /* out: de-duplicated degree */
  int64_t* next;         /* shared work counter */
} dedup_job;

static void* dedup_worker(void* arg) {
  dedup_job* j = (dedup_job*)arg;
  const int64_t chunk = 4096;
  for (;;) {
    int64_t v0 = __atomic_fetch_add(j->next, chunk, __ATOMIC_RELAXED);
    if (v0 >= j->nv) break;
    int64_t v1 = v0 + chunk < j->nv ? v0 + chunk : j->nv;
    for (int64_t v = v0; v < v1; ++v) {
      int32_t* a = j->tmp_col + j->tmp_ptr[v];
      int64_t n = j->tmp_ptr[v + 1] - j->tmp_ptr[v];
      sort_row(a, n);
      int64_t m = 0;
      for (int64_t i = 0; i < n; ++i)
        if (m == 0 || a[i] != a[m - 1]) a[m++] = a[i];
      j->deg[v] = m;
    }
  }
  return NULL;
}

typedef struct {
  int64_t v0, v1;
  const int64_t* tmp_ptr;
  const int32_t* tmp_col;
  const int64_t* row_ptr;
  int32_t* col;
} copy_job;

static void* copy_worker(void* arg) {
  copy_job* j = (copy_job*)arg;
  for (int64_t v = j->v0; v < j->v1; ++v) {
    int64_t n = j->row_ptr[v + 1] - j->row_ptr[v];
    memcpy(j->col + j->row_ptr[v], j->tmp_col + j->tmp_ptr[v], (size_t)n * sizeof(int32_t));
  }
  return NULL;
}

/*
 * Build the CSR of an R-MAT graph with 2^scale vertices from edge_factor*2^scale
 * generated edges.  Writes row_ptr[nv+1] (int64, caller-owned), the edge count
 * through *ne_out and a malloc'd column array through *col_out, which the
 * caller releases with syn_free().  Returns 0, -1 on bad arguments, -2 on OOM.
 */
void syn_free(void* p) { free(p); }

int syn_rmat_build(int scale, int edge_factor, double a, double b, double c, uint64_t seed,
                   int symmetric, int nthreads, int64_t* row_ptr, int64_t* ne_out,
                   int32_t** col_out) {
  if (scale < 1 || scale > 30 || edge_factor < 1) return -1;
  if (!(a >= 0 && b >= 0 && c >= 0 && a + b + c <= 1.0)) return -1;
  const int64_t nv = (int64_t)1 << scale;
  const uint64_t ne_gen = (uint64_t)nv * (uint64_t)edge_factor;
  rmat_cfg cfg;
  cfg.scale = scale;
  cfg.seed = seed;
  cfg.ta = (uint32_t)(a * 4294967296.0 >= 4294967295.0 ? 4294967295.0 : a * 4294967296.0);
  cfg.tab = (uint32_t)((a + b) * 4294967296.0 >= 4294967295.0 ? 4294967295.0 : (a + b) * 4294967296.0);
  cfg.tabc = (uint32_t)((a + b + c) * 4294967296.0 >= 4294967295.0 ? 4294967295.0 : (a + b + c) * 4294967296.0);
  const int T = syn_threads(nthreads);

  uint32_t* cnt = (uint32_t*)calloc((size_t)nv, sizeof(uint32_t));
  int64_t* tmp_ptr = (int64_t*)malloc((size_t)(nv + 1) * sizeof(int64_t));
  if (!cnt || !tmp_ptr) { free(cnt); free(tmp_ptr); return -2; }

  pthread_t th[64];
  rmat_job jobs[64];
  for (int pass = 0; pass < 2; ++pass) {
    for (int t = 0; t < T; ++t) {
      jobs[t].cfg = &cfg;
      jobs[t].e0 = ne_gen * (uint64_t)t / (uint64_t)T;
      jobs[t].e1 = ne_gen * (uint64_t)(t + 1) / (uint64_t)T;
      jobs[t].symmetric = symmetric;
      jobs[t].phase = pass;
      jobs[t].cnt = cnt;
      jobs[t].fill = NULL;
      jobs[t].tmp_col = NULL;
    }
    if (pass == 1) {
      tmp_ptr[0] = 0;
      for (int64_t v = 0; v < nv; ++v) tmp_ptr[v + 1] = tmp_ptr[v] + cnt[v];
      free(cnt);
      cnt = NULL;
      int64_t* fill = (int64_t*)malloc((size_t)nv * sizeof(int64_t));
      int32_t* tmp_col = (int32_t*)malloc((size_t)(tmp_ptr[nv] > 0 ? tmp_ptr[nv] : 1) * sizeof(int32_t));
      if (!fill || !tmp_col) { free(fill); free(tmp_col); free(tmp_ptr); return -2; }
      memcpy(fill, tmp_ptr, (size_t)nv * sizeof(int64_t));
      for (int t = 0; t < T; ++t) { jobs[t].fill = fill; jobs[t].tmp_col = tmp_col; }
      for (int t = 0; t < T; ++t) pthread_create(&th[t], NULL, rmat_worker, &jobs[t]);
      for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
      free(fill);
      /* sort + dedup each row */
      int64_t* deg = (int64_t*)malloc((size_t)nv * sizeof(int64_t));
      if (!deg) { free(tmp_col); free(tmp_ptr); return -2; }
      int64_t next = 0;
      dedup_job dj = {nv, tmp_ptr, tmp_col, deg, &next};
      for (int t = 0; t < T; ++t) pthread_create(&th[t], NULL, dedup_worker, &dj);
      for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
      row_ptr[0] = 0;
      for (int64_t v = 0; v < nv; ++v) row_ptr[v + 1] = row_ptr[v] + deg[v];
      free(deg);
      const int64_t ne = row_ptr[nv];
      int32_t* col = (int32_t*)malloc((size_t)(ne > 0 ? ne : 1) * sizeof(int32_t));
      if (!col) { free(tmp_col); free(tmp_ptr); return -2; }
      copy_job cj[64];
      for (int t = 0; t < T; ++t) {
        cj[t].v0 = nv * t / T;
        cj[t].v1 = nv * (t + 1) / T;
        cj[t].tmp_ptr = tmp_ptr;
        cj[t].tmp_col = tmp_col;
        cj[t].row_ptr = row_ptr;
        cj[t].col = col;
        pthread_create(&th[t], NULL, copy_worker, &cj[t]);
      }
      for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
      free(tmp_col);
      free(tmp_ptr);
      *col_out = col;
      *ne_out = ne;
      return 0;
    }
    for (int t = 0; t < T; ++t) pthread_create(&th[t], NULL, rmat_worker, &jobs[t]);
    for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
  }
  return -3; /* unreachable */
}

/* ------------------------------------------------- per-edge attributes */

typedef struct {
  int64_t v0, v1;
  const int64_t* row_ptr;
  const int32_t* col;
  uint64_t seed;
  float lo, span;
  int nlabels;
  float* w;
  uint8_t* l;
} attr_job;

static inline uint64_t pair_key(int64_t u, int64_t v) {
  uint64_t a = (uint64_t)(u < v ? u : v), b = (uint64_t)(u < v ? v : u);
  return (a << 32) | b;
}

static void* attr_worker(void* arg) {
  attr_job* j = (attr_job*)arg;
  for (int64_t v = j->v0; v < j->v1; ++v) {
    for (int64_t e = j->row_ptr[v]; e < j->row_ptr[v + 1]; ++e) {
      uint64_t key = pair_key(v, j->col[e]);
      if (j->w) {
        uint64_t r = syn_u64(j->seed, SYN_TAG_WEIGHT, key);
        double u = (double)(r >> 40) * (1.0 / 16777216.0); /* 24 bits in [0,1) */
        j->w[e] = (float)((double)j->lo + (double)j->span * u);
      }
      if (j->l) {
        uint64_t r = syn_u64(j->seed, SYN_TAG_LABEL, key);
        j->l[e] = (uint8_t)(((r >> 32) * (uint64_t)j->nlabels) >> 32);
      }
    }
  }
  return NULL;
}

static void run_attr(int64_t nv, const int64_t* row_ptr, const int32_t* col, uint64_t seed,
                     float lo, float hi, int nlabels, float* w, uint8_t* l, int nthreads) {
  const int T = syn_threads(nthreads);
  pthread_t th[64];
  attr_job jobs[64];
  for (int t = 0; t < T; ++t) {
    jobs[t].v0 = nv * t / T;
    jobs[t].v1 = nv * (t + 1) / T;
    jobs[t].row_ptr = row_ptr;
    jobs[t].col = col;
    jobs[t].seed = seed;
    jobs[t].lo = lo;
    jobs[t].span = hi - lo;
    jobs[t].nlabels = nlabels;
    jobs[t].w = w;
    jobs[t].l = l;
    pthread_create(&th[t], NULL, attr_worker, &jobs[t]);
  }
  for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
}

/* fp32 weights uniform in [lo, hi), keyed on the unordered endpoint pair. */
int syn_edge_weights(int64_t nv, const int64_t* row_ptr, const int32_t* col, uint64_t seed,
                     float lo, float hi, float* w, int nthreads) {
  if (!(hi > lo)) return -1;
  run_attr(nv, row_ptr, col, seed, lo, hi, 0, w, NULL, nthreads);
  return 0;
}

/* uint8 labels uniform in [0, nlabels), keyed on the unordered endpoint pair. */
int syn_edge_labels(int64_t nv, const int64_t* row_ptr, const int32_t* col, uint64_t seed,
                    int nlabels, uint8_t* l, int nthreads) {
  if (nlabels < 1 || nlabels > 256) return -1;
  run_attr(nv, row_ptr, col, seed, 0.f, 1.f, nlabels, NULL, l, nthreads);
  return 0;
}

/* n sources uniform in [0, nv). */
int syn_sources(int64_t n, int64_t nv, uint64_t seed, int32_t* out) {
  if (nv < 1 || nv > 2147483647LL) return -1;
  for (int64_t i = 0; i < n; ++i) {
    uint64_t r = syn_u64(seed, SYN_TAG_SOURCE, (uint64_t)i);
    out[i] = (int32_t)(((r >> 32) * (uint64_t)nv) >> 32);
  }
  return 0;
}

/* A schema of len labels uniform in [0, nlabels). */
int syn_schema(int len, int nlabels, uint64_t seed, uint8_t* out) {
  if (len < 0 || nlabels < 1 || nlabels > 256) return -1;
  for (int i = 0; i < len; ++i) {
    uint64_t r = syn_u64(seed, SYN_TAG_SCHEMA, (uint64_t)i);
    out[i] = (uint8_t)(((r >> 32) * (uint64_t)nlabels) >> 32);
  }
  return 0;
}
