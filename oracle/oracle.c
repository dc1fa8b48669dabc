/*
 * ORACLE -- test infrastructure, not part of the product.
 *
 * A plain, slow, single-threaded CPU walker for ThunderRW's
 * Gather-Move-Update model (Section 4.2, Algorithm 2), written from the paper
 * so that the CUDA path can be checked against it bit for bit.  Only the
 * tests, the package's smoke check and the bench's CPU-baseline leg may load
 * this file; the product path never does.  It shares no code, header, table
 * or helper with the CUDA library.
 *
 * Every random number is drawn from Philox4x32-10 (Salmon, Moraes, Dror and
 * Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3", SC 2011), keyed on the
 * walk seed, with counter (walk index, step, draw, tag).  Real-valued draws
 * of the paper are replaced by fixed-point integers:
 *   - a uniform integer in [0, n) is the high 64 bits of r64 * n, where
 *     r64 = B0 | B1 << 32 of the Philox block;
 *   - a uniform real y in [0, 1) compared with a probability t is the 32-bit
 *     word B2 (or B3 for the PPR stop coin) compared with floor(t * 2^32).
 *
 * Readings of the paper that this file fixes (where the text is silent or
 * ambiguous):
 *   - max_len counts moves; a path holds at most max_len + 1 vertices.
 *   - PPR flips its stop coin before every move, the first one included, so
 *     the expected number of vertices is 1/stop (5 at stop 0.2, Section 6.2).
 *   - A vertex with no out-edge (or, for weighted walks, only zero-weight
 *     out-edges) ends the walk there.
 *   - MetaPath step s (0-based move index) uses label H[s mod |H|]; no
 *     matching edge ends the walk.
 *   - Rejection accepts when y < p_x, strictly (Section 2.3, REJ).
 *   - Node2Vec's IsNeighbor(c, u) means c is an out-neighbour of u.
 *   - Weighted Node2Vec multiplies Eq. 1 by the edge weight (Section 2.2).
 *     Its O-REJ dart hits when two independent words pass: y = B2 the class
 *     threshold of Eq. 1 (as unweighted Node2Vec) and z = B3 the weight
 *     threshold floor(W_x * 2^32 / P), so a candidate is taken with
 *     probability proportional to T_class * floor(W_x * 2^32 / P).  P is the
 *     caller's bound on the weights (quantised like a weight), or p*_v of the
 *     REJ table when the caller gives none.  With every weight equal to P the
 *     walk is unweighted Node2Vec's.
 *   - The alias table is built by Vose's method on integer weights, with
 *     first-in first-out work lists (the paper leaves the construction open).
 *   - Weighted DeepWalk may also sample by ITS, REJ or O-REJ (Section 2.3),
 *     all on the same integer weights W_e.  Static ITS stores the row's
 *     prefix sums P' and draws x uniform in [0, p'_{d-1}); static REJ stores
 *     p*_v = max W_e of the row; O-REJ takes a user bound P >= max W_e
 *     (MaxWeight, quantised like a weight) and has no initialisation.  A dart
 *     (x, y) hits when the 32-bit word y is below floor(W_x * 2^32 / p*),
 *     clamped to 2^32 when W_x >= p*.  A row whose weights are all zero is a
 *     dead end for ITS and REJ (their initialisation sees it); O-REJ cannot
 *     see it and runs into the trial cap.
 *
 * Pins: tests/oracle_pins.py holds every function here to something other
 * than itself: Philox known-answer vectors, closed forms of the fixed-point
 * conventions, exact rational laws of the alias tables, chi-square tests of
 * path laws against brute force on tiny graphs, the PPR chain's linear solve,
 * closed-form rejection trial counts, reductions to NAIVE, and hand counts
 * of the statistics' sector model (the distinct 32-byte sectors a move reads
 * in the device layout) on tiny graphs.  No function is unpinned.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

enum { ORC_DEEPWALK = 0, ORC_DEEPWALK_WEIGHTED = 1, ORC_PPR = 2, ORC_NODE2VEC = 3, ORC_METAPATH = 4,
       ORC_NODE2VEC_WEIGHTED = 5 };
enum { ORC_OK = 0, ORC_ERR_INVALID = -1, ORC_ERR_OOM = -2, ORC_ERR_REJECT_CAP = -6 };
/* Sampling method of weighted DeepWalk (the other walks take 0). */
enum { ORC_SAMPLER_DEFAULT = 0, ORC_SAMPLER_ITS = 1, ORC_SAMPLER_REJ = 2, ORC_SAMPLER_OREJ = 3 };

#define ORC_REJECT_CAP 65536

/* ------------------------------------------------------------------ Philox */

/* Philox4x32 with 10 rounds, as defined by Salmon et al. (SC 2011, Section 5):
 * each round multiplies words 0 and 2 by fixed constants, swaps the halves and
 * XORs in the round key; the key is bumped by the Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * x0;
    uint64_t p1 = (uint64_t)M1 * x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += W0;
    k1 += W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The block for draw `draw` of step `step` of walk `walk` under `seed`. */
static void draw_block(uint64_t seed, uint64_t walk, uint32_t step, uint32_t draw, uint32_t out[4]) {
  uint32_t ctr[4] = {(uint32_t)walk, step, draw, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* Uniform integer in [0, n): floor(r64 * n / 2^64). */
static uint64_t uniform_below(const uint32_t B[4], uint64_t n) {
  uint64_t r64 = (uint64_t)B[0] | ((uint64_t)B[1] << 32);
  return (uint64_t)(((unsigned __int128)r64 * n) >> 64);
}

/* Fixed-point threshold of a probability t in [0, 1]: floor(t * 2^32), so that
 * a 32-bit uniform word y succeeds (y < T) with probability exactly T / 2^32. */
uint64_t orc_threshold(double t) {
  if (!(t > 0.0)) return 0;
  if (t >= 1.0) return 4294967296ULL;
  return (uint64_t)floor(t * 4294967296.0);
}

/* -------------------------------------------------------- alias sampling */

/* Integer weight of an fp32 edge weight: round-half-even of w * 2^16, clamped
 * to [0, 2^32 - 1].  Negative or non-finite weights are rejected (-1). */
int64_t orc_quantize_weight(float w) {
  if (!isfinite(w) || w < 0.0f) return -1;
  double t = rint((double)w * 65536.0);
  if (t > 4294967295.0) t = 4294967295.0;
  return (int64_t)t;
}

/*
 * Initialisation phase of ALIAS (Section 2.3) for one vertex with d integer
 * weights W[0..d-1]: probability table H (fixed point, H[i] / 2^32 is the
 * chance of A[i].first) and alias table A (first = i, second = the donor or
 * -1 for a one-element bucket whose H is 2^32).  Vose's method on integers:
 * each item j carries q_j = d * W_j against a bucket capacity S = sum W, so
 * no rounding happens until H is written.  Returns 1 when S == 0 (no
 * distribution: the vertex is a dead end for weighted walks), else 0.
 */
int orc_alias_build(int64_t d, const uint32_t* W, uint64_t* H, int32_t* A_first, int32_t* A_second) {
  uint64_t S = 0;
  for (int64_t j = 0; j < d; ++j) S += W[j];
  if (d == 0) return 0;
  if (S == 0) {
    for (int64_t j = 0; j < d; ++j) { H[j] = 0; A_first[j] = (int32_t)j; A_second[j] = -1; }
    return 1;
  }
  uint64_t* q = (uint64_t*)malloc((size_t)d * sizeof(uint64_t));
  int64_t* small = (int64_t*)malloc((size_t)d * sizeof(int64_t));
  int64_t* large = (int64_t*)malloc((size_t)d * sizeof(int64_t));
  int64_t s_head = 0, s_tail = 0, l_head = 0, l_tail = 0;
  for (int64_t j = 0; j < d; ++j) {
    q[j] = (uint64_t)d * W[j];
    if (q[j] < S) small[s_tail++] = j; else large[l_tail++] = j;
  }
  while (s_head < s_tail && l_head < l_tail) {
    int64_t s = small[s_head++];
    int64_t l = large[l_head];
    H[s] = (uint64_t)(((unsigned __int128)q[s] << 32) / S);
    A_first[s] = (int32_t)s;
    A_second[s] = (int32_t)l;
    q[l] -= S - q[s];
    if (q[l] < S) {
      ++l_head;
      small[s_tail++] = l;
    }
  }
  /* Whatever is left holds exactly one full bucket. */
  while (l_head < l_tail) {
    int64_t j = large[l_head++];
    H[j] = 4294967296ULL;
    A_first[j] = (int32_t)j;
    A_second[j] = -1;
  }
  while (s_head < s_tail) {
    int64_t j = small[s_head++];
    H[j] = 4294967296ULL;
    A_first[j] = (int32_t)j;
    A_second[j] = -1;
  }
  free(q); free(small); free(large);
  return 0;
}

/*
 * Algorithm 3 (preprocessing for static RW): for every vertex, quantise the
 * weights of E_v, run the ALIAS initialisation and store C_v.  Tables are
 * indexed by edge slot (row_ptr[v] + i).  dead[v] = 1 when v has out-edges
 * but no positive integer weight.  Returns 0 or -1 on a bad weight.
 */
int orc_prepare_alias(int64_t nv, const int64_t* row_ptr, const float* weights, uint64_t* H,
                      int32_t* A_first, int32_t* A_second, uint8_t* dead) {
  int64_t dmax = 0;
  for (int64_t v = 0; v < nv; ++v) {
    int64_t d = row_ptr[v + 1] - row_ptr[v];
    if (d > dmax) dmax = d;
  }
  uint32_t* W = (uint32_t*)malloc((size_t)(dmax > 0 ? dmax : 1) * sizeof(uint32_t));
  for (int64_t v = 0; v < nv; ++v) {
    int64_t off = row_ptr[v], d = row_ptr[v + 1] - off;
    for (int64_t j = 0; j < d; ++j) {
      int64_t wq = orc_quantize_weight(weights[off + j]);
      if (wq < 0) { free(W); return ORC_ERR_INVALID; }
      W[j] = (uint32_t)wq;
    }
    dead[v] = (uint8_t)orc_alias_build(d, W, H + off, A_first + off, A_second + off);
  }
  free(W);
  return ORC_OK;
}

/*
 * Algorithm 3 with the ITS initialisation (Section 2.3): for every vertex v,
 * the cumulative sums of its integer weights, P'_i = W_0 + ... + W_i, stored
 * per edge slot (off + i).  Returns 0 or -1 on a bad weight.
 */
int orc_prepare_its(int64_t nv, const int64_t* row_ptr, const float* weights, uint64_t* cdf) {
  for (int64_t v = 0; v < nv; ++v) {
    uint64_t acc = 0;
    for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      int64_t wq = orc_quantize_weight(weights[e]);
      if (wq < 0) return ORC_ERR_INVALID;
      acc += (uint64_t)wq;
      cdf[e] = acc;
    }
  }
  return ORC_OK;
}

/*
 * Algorithm 3 with the REJ initialisation (Section 2.3): p*_v, the largest
 * integer weight of E_v (0 for a vertex without edges or with only zero
 * weights).  Returns 0 or -1 on a bad weight.
 */
int orc_prepare_rej(int64_t nv, const int64_t* row_ptr, const float* weights, uint32_t* pmax) {
  for (int64_t v = 0; v < nv; ++v) {
    uint32_t m = 0;
    for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      int64_t wq = orc_quantize_weight(weights[e]);
      if (wq < 0) return ORC_ERR_INVALID;
      if ((uint32_t)wq > m) m = (uint32_t)wq;
    }
    pmax[v] = m;
  }
  return ORC_OK;
}

/* Fixed-point acceptance threshold of a rejection dart with weight W under the
 * bound pstar > 0: floor(W / pstar * 2^32), exactly, and 2^32 once W >= pstar. */
uint64_t orc_rej_threshold(uint32_t W, uint64_t pstar) {
  if ((uint64_t)W >= pstar) return 4294967296ULL;
  return ((uint64_t)W << 32) / pstar;
}

/* ------------------------------------------------------------------ walks */

typedef struct {
  int64_t nv;
  const int64_t* row_ptr;
  const int32_t* col;
  const uint64_t* H;        /* ALIAS tables from orc_prepare_alias, or NULL */
  const int32_t* A_first;
  const int32_t* A_second;
  const uint8_t* dead;
  const uint8_t* labels;    /* MetaPath edge labels, or NULL */
  const float* weights;     /* edge weights (REJ, O-REJ darts), or NULL */
  const uint64_t* cdf;      /* ITS prefix sums from orc_prepare_its, or NULL */
  const uint32_t* pmax;     /* REJ bounds p*_v from orc_prepare_rej, or NULL */
} orc_graph;

typedef struct {
  int32_t algo;
  int32_t walks_per_source;   /* >= 1; walk i starts at sources[i / walks_per_source] */
  double ppr_stop;            /* PPR termination probability per step */
  double n2v_p, n2v_q;        /* Node2Vec return (a) and in-out (b) parameters, Eq. 1 */
  const uint8_t* schema;      /* MetaPath schema H */
  int32_t schema_len;
  int32_t endpoints_only;     /* 1: out_paths holds one vertex (the end) per walk */
  int64_t walk_offset;        /* index of the first walk in the Philox counter */
  int32_t sampler;            /* weighted DeepWalk: ORC_SAMPLER_* (0 = ALIAS); 0 for the others */
  double max_weight;          /* O-REJ, weighted Node2Vec: the caller's bound on the edge weights (MaxWeight) */
} orc_params;

typedef struct {
  int64_t moves;          /* total moves (steps) of all walks */
  int64_t attempts;       /* Node2Vec, REJ, O-REJ: total rejection trials */
  int64_t stop_len, stop_coin, stop_dead, stop_schema;
  int64_t sectors;        /* distinct 32-byte sectors read, summed over steps (layout model) */
  int64_t out_bytes;      /* bytes of path output written */
  int64_t checks;         /* Node2Vec: IsNeighbor results that decided an attempt (the dart fell
                             between the neighbour and far thresholds) */
  int64_t return_only;    /* unweighted Node2Vec: attempts after the first move whose word lies at or
                             past both non-return thresholds (only a return to prev accepts them) */
} orc_stats;

/* Sector model of the device layout, used only for the roofline: 4-byte
 * row offsets and column ids, 16-byte packed alias records, 1-byte labels,
 * 8-byte ITS prefix sums, 4-byte REJ bounds and edge weights. */
enum { SEC_ROW = 0, SEC_COL = 1, SEC_ALIAS = 2, SEC_LABEL = 3, SEC_CDF = 4, SEC_PMAX = 5, SEC_WEIGHT = 6 };
typedef struct { int64_t n; int64_t key[512]; } sector_set;
static void sec_touch(sector_set* s, int array, int64_t byte_off) {
  int64_t k = ((int64_t)array << 58) | (byte_off >> 5);
  for (int64_t i = 0; i < s->n; ++i) if (s->key[i] == k) return;
  if (s->n < 512) s->key[s->n++] = k;
}
static void sec_touch_range(sector_set* s, int array, int64_t byte_lo, int64_t byte_hi) {
  for (int64_t b = byte_lo & ~31LL; b < byte_hi; b += 32) sec_touch(s, array, b);
}

/* IsNeighbor(c, u) of the Node2Vec Weight function: is c in N_u?  Rows are
 * sorted, so a library binary search serves. */
static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}
static int is_neighbor(const orc_graph* g, int32_t c, int32_t u, sector_set* sec) {
  int64_t lo = g->row_ptr[u], hi = g->row_ptr[u + 1];
  if (sec) {
    sec_touch(sec, SEC_ROW, (int64_t)u * 4);
    sec_touch(sec, SEC_ROW, (int64_t)(u + 1) * 4);
    /* binary-search probes */
    int64_t a = lo, b = hi;
    while (a < b) {
      int64_t m = a + (b - a) / 2;
      sec_touch(sec, SEC_COL, m * 4);
      if (g->col[m] < c) a = m + 1; else b = m;
    }
  }
  return bsearch(&c, g->col + lo, (size_t)(hi - lo), sizeof(int32_t), cmp_i32) != NULL;
}

/*
 * Run n * walks_per_source walks (Algorithm 2: Gather, Move, Update per step).
 * out_paths has (max_len + 1) entries per walk (one when endpoints_only);
 * out_lengths[i] = number of vertices of walk i.  Returns ORC_OK,
 * ORC_ERR_INVALID or ORC_ERR_REJECT_CAP.
 */
int orc_walk(const orc_graph* g, const orc_params* p, const int32_t* sources, int64_t n_sources,
             int32_t max_len, uint64_t seed, int32_t* out_paths, int32_t* out_lengths, orc_stats* st) {
  if (max_len < 0 || p->walks_per_source < 1 || n_sources < 0 || p->walk_offset < 0) return ORC_ERR_INVALID;
  const int64_t wps = p->walks_per_source;
  const int64_t nwalks = n_sources * wps;
  if (p->walk_offset + nwalks > 4294967296LL) return ORC_ERR_INVALID; /* walk ids are 32-bit */
  const int64_t row = p->endpoints_only ? 1 : (int64_t)max_len + 1;
  const uint64_t T_stop = orc_threshold(p->ppr_stop);
  /* Node2Vec (Eq. 1): weight 1/a on the return edge, 1 at distance 1, 1/b at
   * distance 2; O-REJ bound p* = max{1, 1/a, 1/b} (Section 2.3, Section 4.2). */
  double w_ret = 0, w_nb = 0, w_far = 0, pstar = 1;
  if (p->algo == ORC_NODE2VEC || p->algo == ORC_NODE2VEC_WEIGHTED) {
    if (!(p->n2v_p > 0) || !(p->n2v_q > 0)) return ORC_ERR_INVALID;
    w_ret = 1.0 / p->n2v_p;
    w_nb = 1.0;
    w_far = 1.0 / p->n2v_q;
    pstar = w_ret > w_nb ? w_ret : w_nb;
    if (w_far > pstar) pstar = w_far;
  }
  const uint64_t T_ret = orc_threshold(w_ret / pstar);
  const uint64_t T_nb = orc_threshold(w_nb / pstar);
  const uint64_t T_far = orc_threshold(w_far / pstar);
  if (p->algo == ORC_METAPATH && (p->schema_len < 1 || !p->schema || !g->labels)) return ORC_ERR_INVALID;
  if (p->sampler != ORC_SAMPLER_DEFAULT && p->algo != ORC_DEEPWALK_WEIGHTED) return ORC_ERR_INVALID;
  if (p->sampler < ORC_SAMPLER_DEFAULT || p->sampler > ORC_SAMPLER_OREJ) return ORC_ERR_INVALID;
  if (p->algo == ORC_DEEPWALK_WEIGHTED) {
    if (p->sampler == ORC_SAMPLER_DEFAULT && !g->H) return ORC_ERR_INVALID;
    if (p->sampler == ORC_SAMPLER_ITS && !g->cdf) return ORC_ERR_INVALID;
    if (p->sampler == ORC_SAMPLER_REJ && (!g->pmax || !g->weights)) return ORC_ERR_INVALID;
    if (p->sampler == ORC_SAMPLER_OREJ && !g->weights) return ORC_ERR_INVALID;
  }
  /* O-REJ's bound P: round-half-even(MaxWeight * 2^16), clamped to 2^32 - 1
   * like a weight; it must be at least 1. */
  uint64_t P_user = 0;
  if (p->algo == ORC_NODE2VEC_WEIGHTED) {
    if (!g->weights) return ORC_ERR_INVALID;
    if (p->max_weight == 0.0 && !g->pmax) return ORC_ERR_INVALID;
    if (p->max_weight != 0.0) {
      if (!isfinite(p->max_weight) || !(p->max_weight > 0)) return ORC_ERR_INVALID;
      double t = rint(p->max_weight * 65536.0);
      if (t > 4294967295.0) t = 4294967295.0;
      if (t < 1.0) return ORC_ERR_INVALID;
      P_user = (uint64_t)t;
    }
  }
  if (p->algo == ORC_DEEPWALK_WEIGHTED && p->sampler == ORC_SAMPLER_OREJ) {
    if (!isfinite(p->max_weight) || !(p->max_weight > 0)) return ORC_ERR_INVALID;
    double t = rint(p->max_weight * 65536.0);
    if (t > 4294967295.0) t = 4294967295.0;
    if (t < 1.0) return ORC_ERR_INVALID;
    P_user = (uint64_t)t;
  }

  int32_t* path = (int32_t*)malloc(((size_t)max_len + 1) * sizeof(int32_t));
  int64_t dmax = 0;
  for (int64_t v = 0; v < g->nv; ++v)
    if (g->row_ptr[v + 1] - g->row_ptr[v] > dmax) dmax = g->row_ptr[v + 1] - g->row_ptr[v];
  int64_t* cdf = (int64_t*)malloc((size_t)(dmax > 0 ? dmax : 1) * sizeof(int64_t));
  sector_set* sec = st ? (sector_set*)malloc(sizeof(sector_set)) : NULL;
  int rc = ORC_OK;

  for (int64_t i = 0; i < nwalks && rc == ORC_OK; ++i) {
    const uint64_t w = (uint64_t)(p->walk_offset + i);
    int32_t cur = sources[i / wps];
    if (cur < 0 || cur >= g->nv) { rc = ORC_ERR_INVALID; break; }
    int32_t s = 0;
    path[0] = cur;
    for (;;) {
      if (sec) sec->n = 0;
      /* Update's termination test for the next step. */
      if (s == max_len) { if (st) st->stop_len++; break; }
      uint32_t B[4];
      draw_block(seed, w, (uint32_t)s, 0u, B);
      if (p->algo == ORC_PPR && (uint64_t)B[3] < T_stop) { if (st) st->stop_coin++; break; }
      const int64_t off = g->row_ptr[cur];
      const int64_t d = g->row_ptr[cur + 1] - off;
      if (sec) { sec_touch(sec, SEC_ROW, (int64_t)cur * 4); sec_touch(sec, SEC_ROW, (int64_t)(cur + 1) * 4); }
      if (d == 0) { if (st) st->stop_dead++; break; }
      int32_t next = -1;
      if (p->algo == ORC_DEEPWALK || p->algo == ORC_PPR) {
        /* NAIVE: x uniform in [0, d_v), pick E_v[x]. */
        const uint64_t x = uniform_below(B, (uint64_t)d);
        next = g->col[off + (int64_t)x];
        if (sec) sec_touch(sec, SEC_COL, (off + (int64_t)x) * 4);
      } else if (p->algo == ORC_DEEPWALK_WEIGHTED && p->sampler == ORC_SAMPLER_ITS) {
        /* Static walk, ITS generation from the stored P': x uniform in
         * [0, p'_{d-1}), then the smallest i with x < p'_i. */
        const uint64_t* P = g->cdf + off;
        if (sec) sec_touch(sec, SEC_CDF, (off + d - 1) * 8);
        if (P[d - 1] == 0) { if (st) st->stop_dead++; break; }
        const uint64_t x = uniform_below(B, P[d - 1]);
        int64_t lo = 0, hi = d - 1;
        while (lo < hi) {
          int64_t mid = lo + (hi - lo) / 2;
          if (sec) sec_touch(sec, SEC_CDF, (off + mid) * 8);
          if (x < P[mid]) hi = mid; else lo = mid + 1;
        }
        next = g->col[off + lo];
        if (sec) sec_touch(sec, SEC_COL, (off + lo) * 4);
      } else if (p->algo == ORC_DEEPWALK_WEIGHTED && p->sampler != ORC_SAMPLER_DEFAULT) {
        /* REJ (p* stored by the preprocessing) or O-REJ (the user's bound):
         * throw darts (x, y), x uniform in [0, d_v), until y < p_x / p*. */
        uint64_t pstar = P_user;
        if (p->sampler == ORC_SAMPLER_REJ) {
          pstar = g->pmax[cur];
          if (sec) sec_touch(sec, SEC_PMAX, (int64_t)cur * 4);
          if (pstar == 0) { if (st) st->stop_dead++; break; }
        }
        int accepted = 0;
        for (uint32_t a = 0; a < ORC_REJECT_CAP; ++a) {
          if (a > 0) draw_block(seed, w, (uint32_t)s, a, B);
          if (st) st->attempts++;
          const int64_t x = (int64_t)uniform_below(B, (uint64_t)d);
          const uint32_t Wx = (uint32_t)orc_quantize_weight(g->weights[off + x]);
          if (sec) { sec_touch(sec, SEC_WEIGHT, (off + x) * 4); sec_touch(sec, SEC_COL, (off + x) * 4); }
          if ((uint64_t)B[2] < orc_rej_threshold(Wx, pstar)) { next = g->col[off + x]; accepted = 1; break; }
        }
        if (!accepted) { rc = ORC_ERR_REJECT_CAP; break; }
      } else if (p->algo == ORC_DEEPWALK_WEIGHTED) {
        /* Static walk: C_v was stored by the preprocessing, no Gather. */
        if (g->dead[cur]) { if (st) st->stop_dead++; break; }
        /* ALIAS generation: x uniform in [0, d_v), y uniform in [0, 1);
         * y < H[x] picks A[x].first, otherwise A[x].second. */
        const int64_t x = (int64_t)uniform_below(B, (uint64_t)d);
        const uint64_t y = B[2];
        const int32_t pick = (y < g->H[off + x]) ? g->A_first[off + x] : g->A_second[off + x];
        next = g->col[off + pick];
        if (sec) sec_touch(sec, SEC_ALIAS, (off + x) * 16);
      } else if (p->algo == ORC_METAPATH) {
        /* Gather: Weight(Q, e) = 1 if l_e == H[s mod |H|] else 0, then the ITS
         * initialisation builds the CDF P'. */
        const uint8_t h = p->schema[s % p->schema_len];
        int64_t acc = 0;
        for (int64_t j = 0; j < d; ++j) {
          acc += (g->labels[off + j] == h) ? 1 : 0;
          cdf[j] = acc;
        }
        if (sec) sec_touch_range(sec, SEC_LABEL, off, off + d);
        if (acc == 0) { if (st) st->stop_schema++; break; }
        /* Move (ITS generation): x uniform in [0, p'_{d-1}), then the smallest
         * i with x < p'_i by binary search. */
        const int64_t x = (int64_t)uniform_below(B, (uint64_t)acc);
        int64_t lo = 0, hi = d - 1;
        while (lo < hi) {
          int64_t mid = lo + (hi - lo) / 2;
          if (x < cdf[mid]) hi = mid; else lo = mid + 1;
        }
        next = g->col[off + lo];
        if (sec) sec_touch(sec, SEC_COL, (off + lo) * 4);
      } else if (p->algo == ORC_NODE2VEC || p->algo == ORC_NODE2VEC_WEIGHTED) {
        /* O-REJ: throw darts (x, y) until y < p_x.  Weighted: the dart must
         * also pass the weight word, z < W_x / P. */
        uint64_t P = P_user;
        if (p->algo == ORC_NODE2VEC_WEIGHTED && P == 0) {
          P = g->pmax[cur];
          if (sec) sec_touch(sec, SEC_PMAX, (int64_t)cur * 4);
          if (P == 0) { if (st) st->stop_dead++; break; }
        }
        int accepted = 0;
        for (uint32_t a = 0; a < ORC_REJECT_CAP; ++a) {
          if (a > 0) draw_block(seed, w, (uint32_t)s, a, B);
          if (st) st->attempts++;
          if (st && p->algo == ORC_NODE2VEC && s > 0 && (uint64_t)B[2] >= (T_nb > T_far ? T_nb : T_far))
            st->return_only++;
          const int64_t x = (int64_t)uniform_below(B, (uint64_t)d);
          const int32_t c = g->col[off + x];
          if (sec) sec_touch(sec, SEC_COL, (off + x) * 4);
          if (p->algo == ORC_NODE2VEC_WEIGHTED) {
            const uint32_t Wx = (uint32_t)orc_quantize_weight(g->weights[off + x]);
            if (sec) sec_touch(sec, SEC_WEIGHT, (off + x) * 4);
            if (!((uint64_t)B[3] < orc_rej_threshold(Wx, P))) continue;
          }
          uint64_t T;
          if (s == 0) {
            T = 4294967296ULL; /* Weight = MaxWeight on the first step */
          } else {
            const int32_t u = path[s - 1];
            if (c == u) {
              T = T_ret;
            } else {
              const uint64_t lo = T_nb < T_far ? T_nb : T_far, hi = T_nb < T_far ? T_far : T_nb;
              if (st && (uint64_t)B[2] >= lo && (uint64_t)B[2] < hi) st->checks++;
              T = is_neighbor(g, c, u, sec) ? T_nb : T_far;
            }
          }
          if ((uint64_t)B[2] < T) { next = c; accepted = 1; break; }
        }
        if (!accepted) { rc = ORC_ERR_REJECT_CAP; break; }
      } else {
        rc = ORC_ERR_INVALID;
        break;
      }
      /* Update: append the vertex. */
      ++s;
      path[s] = next;
      cur = next;
      if (st) { st->moves++; st->sectors += sec->n; }
    }
    if (rc != ORC_OK) break;
    if (p->endpoints_only) {
      out_paths[i] = path[s];
      if (st) st->out_bytes += 4;
    } else {
      memcpy(out_paths + i * row, path, ((size_t)s + 1) * sizeof(int32_t));
      if (st) st->out_bytes += ((int64_t)s + 1) * 4;
    }
    out_lengths[i] = s + 1;
  }
  free(path);
  free(cdf);
  free(sec);
  return rc;
}

/* ------------------------------------------------------- user-defined walks */

/*
 * A walk given by user functions (Section 4.3, "APIs"): the sampling method
 * (0 NAIVE, 1 O-REJ), Weight and MaxWeight as fixed-point integers, and
 * Update, called after each move with the query already moved; a non-zero
 * return ends the walk.  Draws as every other walk: block (walk, step,
 * attempt, 0); NAIVE takes E_cur[x]; an O-REJ dart hits when the 32-bit word
 * B2 is below floor(Weight * 2^32 / MaxWeight) (2^32 once Weight >= MaxWeight).
 * A walk also ends after max_len moves and at a vertex without out-edges.
 */
typedef uint32_t (*orc_weight_fn)(void* user, int64_t walk, int32_t length, int32_t cur, int32_t prev, int32_t dst,
                                  int64_t edge);
typedef int (*orc_update_fn)(void* user, int64_t walk, int32_t length, int32_t cur, int32_t prev, int32_t dst,
                             int64_t edge);

int orc_walk_custom(const orc_graph* g, int32_t sampler, uint32_t max_weight, orc_weight_fn weight,
                    orc_update_fn update, void* user, const int32_t* sources, int64_t n_sources,
                    int32_t walks_per_source, int32_t max_len, uint64_t seed, int64_t walk_offset,
                    int32_t* out_paths, int32_t* out_lengths, orc_stats* st) {
  if (max_len < 0 || walks_per_source < 1 || n_sources < 0 || walk_offset < 0) return ORC_ERR_INVALID;
  if (sampler != 0 && sampler != 1) return ORC_ERR_INVALID;
  if (sampler == 1 && (max_weight == 0 || !weight)) return ORC_ERR_INVALID;
  const int64_t nwalks = n_sources * walks_per_source;
  if (walk_offset + nwalks > 4294967296LL) return ORC_ERR_INVALID;
  const int64_t row = (int64_t)max_len + 1;
  for (int64_t i = 0; i < nwalks; ++i) {
    const uint64_t w = (uint64_t)(walk_offset + i);
    int32_t cur = sources[i / walks_per_source], prev = -1;
    if (cur < 0 || cur >= g->nv) return ORC_ERR_INVALID;
    int32_t s = 0;
    out_paths[i * row] = cur;
    while (s < max_len) {
      const int64_t off = g->row_ptr[cur], d = g->row_ptr[cur + 1] - off;
      if (d == 0) { if (st) st->stop_dead++; break; }
      int64_t x = -1;
      for (uint32_t a = 0; a < ORC_REJECT_CAP; ++a) {
        uint32_t B[4];
        draw_block(seed, w, (uint32_t)s, a, B);
        if (st && sampler == 1) st->attempts++;
        const int64_t c = (int64_t)uniform_below(B, (uint64_t)d);
        if (sampler == 0) { x = c; break; }
        const uint32_t W = weight(user, (int64_t)w, s, cur, prev, g->col[off + c], off + c);
        if ((uint64_t)B[2] < orc_rej_threshold(W, max_weight)) { x = c; break; }
      }
      if (x < 0) return ORC_ERR_REJECT_CAP;
      const int32_t dst = g->col[off + x];
      prev = cur;
      cur = dst;
      ++s;
      out_paths[i * row + s] = cur;
      if (st) st->moves++;
      if (update && update(user, (int64_t)w, s, cur, prev, dst, off + x)) break;
    }
    out_lengths[i] = s + 1;
  }
  return ORC_OK;
}
