/*
 * trw.h -- C ABI of the GB300 random-walk engine (libtrw.so).
 *
 * The engine runs massive numbers of independent random-walk queries under
 * ThunderRW's step-centric Gather-Move-Update model (Section 4.2,
 * Algorithm 2): Gather reads (static walks) or builds (dynamic walks) the
 * transition weights of the current vertex's edges, Move samples the next
 * edge, Update appends the vertex and decides termination.  Every step runs
 * in CUDA kernels for sm_103a; the host side only validates, copies and
 * launches.
 *
 * Conventions common to every call:
 *  - Every call returns a trw_status; no C++ exception crosses this ABI.
 *    On a non-OK status, trw_last_error() returns a thread-local message.
 *  - The caller owns every input.  trw_graph_load copies the graph to the
 *    device, so the caller may free its arrays afterwards.  The library owns
 *    the device copies and the prepared tables until trw_graph_free.
 *  - Buffers marked "host or device" may be either; the library detects the
 *    kind with cudaPointerGetAttributes and copies host data through its own
 *    device staging buffers.
 *  - Randomness: walk i of a call draws every random number from
 *    Philox4x32-10 keyed on the 64-bit seed, with counter
 *    (walk_offset + i, step, draw, 0).  A walk therefore depends only on
 *    (graph, algorithm, parameters, seed, walk index): results do not depend
 *    on batching, kernel choice, launch shape or scheduling.
 *  - Fixed point replaces real-valued draws: a uniform integer in [0, n) is
 *    the high 64 bits of r64 * n (r64 = the block's first two words); a
 *    probability t is the threshold floor(t * 2^32) against a 32-bit word.
 *  - Graph sizes: nv < 2^31 and ne < 2^31 (int32 device offsets); walk
 *    indices walk_offset + i < 2^32.
 *  - A graph lives on the device that was current when it was loaded.  Every
 *    call that works on a graph (directly, or through a plan or a server)
 *    returns TRW_ERR_INVALID, before any copy or launch, when another device
 *    is current.
 *  - TRW_ERR_OOM reports a device or pinned host allocation that failed; the
 *    graph (or server) keeps the state it had before the call.
 */
#ifndef TRW_H
#define TRW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct trw_graph trw_graph;
typedef struct trw_server trw_server;

typedef enum {
  TRW_OK = 0,
  TRW_PENDING = 1,              /* serve: request still running */
  TRW_ERR_INVALID = -1,         /* bad argument; nothing was written */
  TRW_ERR_OOM = -2,             /* device or host allocation failed */
  TRW_ERR_NOT_PREPARED = -3,    /* weighted walk before trw_prepare of its sampler's table */
  TRW_ERR_CUDA = -4,            /* a CUDA runtime call failed */
  TRW_ERR_TIMEOUT = -5,         /* a bounded wait ran out */
  TRW_ERR_REJECT_CAP = -6,      /* a rejection step exceeded TRW_REJECT_CAP trials */
  TRW_ERR_BUSY = -7,            /* serve: no capacity to admit the request now */
  TRW_ERR_NOT_FOUND = -8,       /* serve: unknown request id */
  TRW_ERR_INTERNAL = -9,        /* a device-side consistency check failed */
  TRW_ERR_STOPPED = -10,        /* stream: the consumer asked to stop */
  TRW_ERR_IO = -11              /* stream to files: a file could not be opened or written */
} trw_status;

/* Walk algorithms of Section 2.2 and the sampler each uses (Section 4.3's
 * recommendation: unbiased -> NAIVE, static -> ALIAS, dynamic -> O-REJ when
 * a bound on the weights is known, else ITS). */
typedef enum {
  TRW_DEEPWALK = 0,             /* unbiased, NAIVE sampling */
  TRW_DEEPWALK_WEIGHTED = 1,    /* static biased by w_e, ALIAS sampling */
  TRW_PPR = 2,                  /* unbiased with a stop coin per step, NAIVE */
  TRW_NODE2VEC = 3,             /* dynamic second order (Eq. 1), O-REJ */
  TRW_METAPATH = 4,             /* dynamic label filter, ITS */
  TRW_NODE2VEC_WEIGHTED = 5     /* Node2Vec with Eq. 1 multiplied by w_e (Section 2.2), O-REJ: a dart
                                   passes the class threshold (word 2) and the weight threshold
                                   floor(W_x * 2^32 / P) (word 3); P = the caller's max_weight
                                   quantised, or the row's p*_v (TRW_PREP_REJ) when max_weight is 0 */
} trw_algo;

/* Kernel choice for trw_walk_ex. */
typedef enum {
  TRW_KERNEL_AUTO = 0,          /* the persistent kernel; the plain one for a batch that fits in one
                                   resident wave and needs no warp-cooperative path */
  TRW_KERNEL_PLAIN = 1,         /* baseline: one launch, one thread per walk, no refill */
  TRW_KERNEL_PERSISTENT = 2,    /* persistent kernel, device work queue, refill, staging */
  TRW_KERNEL_BSP = 3            /* baseline: step-synchronous (the BSP model of KnightKing and C-SAW,
                                   Section 3): one launch per step over the live walkers, walker state
                                   in device memory, the live count read back after every launch;
                                   synchronous calls only */
} trw_kernel;

#define TRW_OUT_PATHS 0u        /* out_paths[i * (max_len + 1) + k] = Q[k] */
#define TRW_OUT_ENDPOINTS 1u    /* out_paths[i] = the last vertex of walk i */
#define TRW_OUT_COMPACT 2u      /* trw_walk / trw_walk_ex only: the vertices of walk 0, then of walk 1, ...
                                   with no padding (out_paths[o_i + k] = Q_i[k], o_i the sum of the
                                   lengths of walks 0 .. i-1); out_paths needs room for the sum of the
                                   lengths, at most nwalks * (max_len + 1) */

/* Sampling method of TRW_DEEPWALK_WEIGHTED (Section 2.3); the other
 * algorithms take TRW_SAMPLER_DEFAULT.  All four draw from the same law
 * over the integer weights W_e = round-half-even(w_e * 2^16), within the
 * fixed-point rounding of each method's thresholds.
 *   DEFAULT  ALIAS over the tables of TRW_PREP_ALIAS: one record per move.
 *   ITS      static ITS over the prefix sums of TRW_PREP_ITS: x uniform in
 *            [0, p'_{d-1}), then the smallest i with x < p'_i (binary search;
 *            with TRW_PREP_ITS_GUIDE the same answer through guided records).
 *   REJ      rejection against p*_v = max W_e of the row (TRW_PREP_REJ):
 *            darts (x, y) with x uniform in [0, d_v) until y < W_x / p*_v,
 *            the 32-bit word y tested against floor(W_x * 2^32 / p*_v).
 *   OREJ     rejection against the caller's bound P = round-half-even(
 *            max_weight * 2^16); no preparation.  P should be >= every W_e:
 *            a larger W_e is accepted like W_e = P.  A row whose weights are
 *            all zero is a dead end for ALIAS, ITS and REJ; under O-REJ it
 *            exhausts the trial cap (TRW_ERR_REJECT_CAP).
 * Draw a of step s of walk i is Philox block (i, s, a, 0); REJ and O-REJ
 * take as many draws as darts. */
#define TRW_SAMPLER_DEFAULT 0
#define TRW_SAMPLER_ITS 1
#define TRW_SAMPLER_REJ 2
#define TRW_SAMPLER_OREJ 3

#define TRW_MAX_SCHEMA 16       /* longest MetaPath schema */
#define TRW_REJECT_CAP 65536    /* rejection trials per step before TRW_ERR_REJECT_CAP */

/* Per-call walk parameters. */
typedef struct {
  double ppr_stop;              /* PPR: termination probability, flipped before every move, in [0, 1] */
  double n2v_p;                 /* Node2Vec return parameter (the paper's a): weight 1/p on the edge back to prev, > 0 */
  double n2v_q;                 /* Node2Vec in-out parameter (the paper's b): weight 1/q at distance 2, > 0 */
  const uint8_t* schema;        /* MetaPath schema H (host memory), step s uses H[s mod schema_len] */
  int32_t schema_len;           /* 1 .. TRW_MAX_SCHEMA for MetaPath, ignored otherwise */
  uint32_t out_mode;            /* TRW_OUT_PATHS, TRW_OUT_ENDPOINTS or (trw_walk / trw_walk_ex) TRW_OUT_COMPACT */
  int32_t walks_per_source;     /* >= 1; walk i starts at sources[i / walks_per_source] */
  int32_t sampler;              /* TRW_SAMPLER_*: weighted DeepWalk's sampling method */
  int64_t walk_offset;          /* index of walk 0 in the Philox counter (for sharding a batch) */
  double max_weight;            /* TRW_SAMPLER_OREJ and TRW_NODE2VEC_WEIGHTED: MaxWeight, the caller's
                                   bound on w_e, finite and > 0 (weighted Node2Vec: 0 = the REJ bounds) */
} trw_params;

/* Fills *p with defaults: ppr_stop 0.2, p = q = 1, no schema, paths,
 * one walk per source, offset 0, the default sampler. */
void trw_params_default(trw_params* p);

#define TRW_LOAD_CHECK 1u        /* validate col ids and strictly increasing rows on the device */

/*
 * Load a CSR graph (Appendix B "graph storage": vertex array, edge array,
 * per-edge weight and label arrays; Section 2.1: an undirected edge is two
 * directed edges).
 *   nv, ne      vertex and edge counts, 0 <= nv, ne < 2^31.
 *   row_ptr     host, int64[nv + 1], row_ptr[0] = 0, non-decreasing, row_ptr[nv] = ne.
 *   col         host, int32[ne], destination of each edge, in [0, nv).
 *               Node2Vec's IsNeighbor needs every row sorted ascending without
 *               duplicates (checked under TRW_LOAD_CHECK, else assumed).
 *   weights     host, fp32[ne] edge weights (finite, >= 0, checked on the device) or NULL.
 *   labels      host, uint8[ne] edge labels or NULL.
 *   flags       TRW_LOAD_CHECK or 0.
 *   out         receives the handle.
 * Errors: TRW_ERR_INVALID (sizes, offsets, ids, weights), TRW_ERR_OOM, TRW_ERR_CUDA.
 */
trw_status trw_graph_load(int64_t nv, int64_t ne, const int64_t* row_ptr, const int32_t* col,
                          const float* weights, const uint8_t* labels, uint32_t flags, trw_graph** out);

/* Release every device buffer of the graph.  NULL is ignored. */
void trw_graph_free(trw_graph* g);

/* The device arrays of a loaded graph, for user-defined walks
 * (trw_custom.cuh): device pointers owned by the graph, valid until
 * trw_graph_free; the caller must not write through them. */
typedef struct {
  const int32_t* row_ptr;       /* [nv + 1] int32 offsets */
  const int32_t* col;           /* [ne] */
  const float* weights;         /* [ne] or NULL */
  const uint8_t* labels;        /* [ne] or NULL */
  int64_t nv, ne;
  int32_t sorted;               /* 1: every row strictly increasing */
  int32_t device;               /* CUDA device of the arrays */
} trw_graph_view;

/* Fills *out.  Errors: TRW_ERR_INVALID (NULL argument). */
trw_status trw_graph_get_view(const trw_graph* g, trw_graph_view* out);

#define TRW_PREP_ALIAS 1u        /* build the ALIAS tables for TRW_DEEPWALK_WEIGHTED */
#define TRW_PREP_LABEL_INDEX 2u  /* build the MetaPath label index (labelled graphs) */
#define TRW_LABEL_INDEX_MAX_LABELS 30
#define TRW_PREP_NEIGHBOR_HASH 4u /* build the neighbour hash for Node2Vec's IsNeighbor */
#define TRW_NEIGHBOR_HASH_MIN_DEGREE 8
#define TRW_PREP_ROW_RECORDS 8u   /* build row records for NAIVE moves and O-REJ candidates */
#define TRW_PREP_ITS 16u          /* build ITS prefix sums for TRW_SAMPLER_ITS */
#define TRW_PREP_REJ 32u          /* build REJ bounds p*_v for TRW_SAMPLER_REJ */
#define TRW_PREP_ITS_GUIDE 64u    /* build guided ITS records for TRW_SAMPLER_ITS */

/*
 * Preprocessing for static walks (Algorithm 3): for every vertex v, apply the
 * weight function to E_v and run the initialisation phase of ALIAS
 * (Section 2.3), storing C_v on the device.  Weights are quantised to
 * integers round-half-even(w * 2^16); the tables come from Vose's method on
 * those integers with first-in first-out work lists, so every table entry is
 * exact up to one floor of H.  A vertex whose edges all quantise to zero
 * becomes a dead end for weighted walks.
 *
 * TRW_PREP_LABEL_INDEX (not in the paper, whose MetaPath Gather scans the
 * labels of E_v at every step, Section 2.2): every row is stably partitioned
 * by edge label, and each edge slot gets a record holding its destination
 * and the bounds of the destination's label groups.  A MetaPath move then
 * reads one record instead of scanning the row; the r-th edge of a label
 * group is the row's r-th matching edge in CSR order, so every walk is
 * identical with and without the index.  Labels must lie in
 * [0, TRW_LABEL_INDEX_MAX_LABELS); the records take (NL + 2) int32 rounded up
 * to 8, 16 or 32 words per edge and per vertex (NL = largest label + 1).
 * Preparing an index that exists already does nothing.
 *
 * TRW_PREP_NEIGHBOR_HASH (not in the paper, whose Node2Vec IsNeighbor is a
 * binary search in the sorted row of the previous vertex, Section 4): every
 * row of at least TRW_NEIGHBOR_HASH_MIN_DEGREE entries gets an
 * open-addressing hash table of its neighbours (2 d slots at load 1/2, laid
 * out like the rows: 8 bytes of device memory per edge), and IsNeighbor(c,
 * prev) for such a row reads about one sector instead of log2(d_prev) row
 * entries.  Membership is exact, so every walk is identical with and without
 * it.  Preparing a hash that exists already does nothing.
 *
 * TRW_PREP_ROW_RECORDS (not in the paper, whose NAIVE move reads the row of
 * the current vertex and then one edge of it, Section 2.3): a 32-byte record
 * per edge slot e = (v -> dst) {destination, its row offset, its degree, W_e
 * (the integer weight, 0 without weights), the position of v in dst's row
 * (-1 when dst has no edge back to v, or the rows are not sorted), 0, 0, 0},
 * so that a NAIVE move (DeepWalk, PPR), an O-REJ candidate (Node2Vec), a REJ
 * or O-REJ dart or an ITS pick reads one record and the next step needs no
 * row-offset lookup: one dependent random read per move instead of two.  With
 * the records, an unweighted Node2Vec dart whose word lies at or past both
 * non-return thresholds (only a return to the previous vertex can accept it)
 * is decided from the previous vertex's position in the row, without reading
 * its candidate.  32 bytes of device memory per edge; every walk is identical
 * with and without them.  Preparing records that exist already does nothing.
 *
 * TRW_PREP_ITS and TRW_PREP_REJ: Algorithm 3 with the ITS and REJ
 * initialisations of Section 2.3, for the samplers of the same names: the
 * inclusive prefix sums of every row's integer weights (uint64, 8 bytes of
 * device memory per edge) and p*_v, every row's largest integer weight
 * (4 bytes per vertex).  Preparing a table that exists already does nothing.
 *
 * TRW_PREP_ITS_GUIDE (not in the paper, whose ITS generation is a binary
 * search over P', Section 2.3): a 32-byte record per edge slot with the
 * edge's ITS bound in draw space, its destination and the destination's row,
 * and the guide entries of Chen and Asau's guide table (one cell per edge, in
 * draw space), which bound the answer to a few candidates.  An ITS move then
 * reads the cell's record and usually one more instead of log2(d) prefix
 * sums and the edge.  The walks are those of TRW_PREP_ITS exactly; when both
 * exist the records are used.
 *
 * Runs on the device; synchronous.  Errors: TRW_ERR_INVALID (no weights, or
 * no labels, loaded for the requested table; a label too large for the
 * index; an unknown flag), TRW_ERR_OOM, TRW_ERR_CUDA.
 */
trw_status trw_prepare(trw_graph* g, uint32_t what);

/*
 * Run n_sources * walks_per_source walks to completion (Algorithm 2 for every
 * query; one persistent kernel with a device work queue).
 *   algo, params   algorithm and its parameters (params may be NULL for defaults).
 *   sources        host or device, int32[n_sources], each in [0, nv).
 *   max_len        moves per walk, >= 0: a path holds at most max_len + 1 vertices.
 *   seed           Philox key.
 *   out_paths      host or device, int32[nwalks * (max_len + 1)] (TRW_OUT_PATHS)
 *                  or int32[nwalks] (TRW_OUT_ENDPOINTS).  Entries past a walk's
 *                  length are left unspecified.
 *   out_lengths    host or device, int32[nwalks]: vertices in walk i (>= 1).
 * A walk stops after max_len moves, on PPR's stop coin (flipped before each
 * move), at a vertex without out-edges, or when no edge carries the MetaPath
 * label of the step.  Synchronous on the graph's stream.  Host outputs go
 * through device staging; a large batch walks in slices whose copy-out
 * overlaps the next slice's walk.
 * Errors: TRW_ERR_INVALID (a source out of range, max_len < 0, a missing
 * weight/label array, p or q <= 0, ppr_stop outside [0, 1], bad schema, a
 * sampler other than the default for an algorithm other than weighted
 * DeepWalk, an O-REJ max_weight that is not finite or quantises to 0),
 * TRW_ERR_NOT_PREPARED, TRW_ERR_REJECT_CAP, TRW_ERR_OOM, TRW_ERR_CUDA.
 */
trw_status trw_walk(trw_graph* g, trw_algo algo, const trw_params* params, const int32_t* sources,
                    int64_t n_sources, int32_t max_len, uint64_t seed, int32_t* out_paths,
                    int32_t* out_lengths);

/*
 * trw_walk with an explicit kernel and stream.
 *   kernel   TRW_KERNEL_AUTO, TRW_KERNEL_PLAIN or TRW_KERNEL_PERSISTENT.
 *   stream   a cudaStream_t (cudaStreamLegacy, i.e. (void*)1, names the legacy
 *            default stream), or NULL for the graph's own stream.
 *   sync     1: wait and return the device status (as trw_walk);
 *            0: device buffers only, return after the launch; collect the
 *               device status later with trw_sync.
 * Errors as trw_walk; with sync = 0, TRW_ERR_INVALID for host buffers.
 */
trw_status trw_walk_ex(trw_graph* g, trw_algo algo, const trw_params* params, const int32_t* sources,
                       int64_t n_sources, int32_t max_len, uint64_t seed, int32_t* out_paths,
                       int32_t* out_lengths, trw_kernel kernel, void* stream, int sync);

/* Wait for the stream (NULL: the graph's) and return, then clear, the status
 * that kernels launched with sync = 0 left on the device. */
trw_status trw_sync(trw_graph* g, void* stream);

/*
 * Streaming output (the paper's double-buffered dump of the walk paths,
 * Appendix "Input and output"): trw_walk's batch in source-aligned slices of
 * about slice_walks walks, each handed to fn on the calling thread as soon as
 * it is on the host.  Slice i walks into device staging buffer i % 2 while the
 * copy engine moves slice i - 1 into pinned host buffer (i - 1) % 2 and fn
 * consumes slice i - 2's: device and host memory stay O(slice) whatever the
 * batch size.
 *   fn(user, first_walk, n_walks, paths, lengths)
 *       paths    host, int32[n_walks * (max_len + 1)] (TRW_OUT_PATHS, rows
 *                padded as in trw_walk) or int32[n_walks] (TRW_OUT_ENDPOINTS);
 *       lengths  host, int32[n_walks];
 *       both valid only during the call.  Walk first_walk + k of the batch is
 *       row k.  Return 0 to continue, anything else to stop.  fn runs with
 *       the graph locked: it must not call the library on the same graph.
 *   slice_walks  walks per slice (rounded down to whole sources, at least one
 *                source).
 * Every slice is checked before fn sees it.  Synchronous; the other arguments
 * as trw_walk.  Errors: those of trw_walk, TRW_ERR_STOPPED (fn returned
 * non-zero; the slices before were delivered).
 */
typedef int (*trw_stream_fn)(void* user, int64_t first_walk, int64_t n_walks, const int32_t* paths,
                             const int32_t* lengths);
trw_status trw_walk_stream(trw_graph* g, trw_algo algo, const trw_params* params, const int32_t* sources,
                           int64_t n_sources, int32_t max_len, uint64_t seed, int64_t slice_walks, trw_stream_fn fn,
                           void* user);

/*
 * trw_walk_stream into two files, written on the calling thread while the
 * GPU walks the next slice: paths_file receives the vertices of walk 0, then
 * of walk 1, ... (lengths[i] int32 each, no padding; one int32 per walk with
 * TRW_OUT_ENDPOINTS) and lengths_file the int32 lengths, both in the host's
 * byte order.  Errors: those of trw_walk, TRW_ERR_IO.
 */
trw_status trw_walk_to_file(trw_graph* g, trw_algo algo, const trw_params* params, const int32_t* sources,
                            int64_t n_sources, int32_t max_len, uint64_t seed, const char* paths_file,
                            const char* lengths_file);

/*
 * Random-gather ceiling (measurement aid, no counterpart in the paper): the
 * rate at which this GPU serves dependent random loads of record_bytes-wide
 * records (4, 8 or 16) from a table of table_bytes, with the same occupancy
 * and chain length as a walk: every thread follows hops_per_chain dependent
 * random hops of chains_per_thread independent chains.  Allocates and frees
 * its own table.  Writes loads per second and the kernel time.
 * Errors: TRW_ERR_INVALID (sizes), TRW_ERR_OOM, TRW_ERR_CUDA.
 */
trw_status trw_gather_ceiling(int64_t table_bytes, int32_t record_bytes, int32_t hops_per_chain,
                              int32_t chains_per_thread, double* loads_per_s, double* kernel_ms);

/*
 * A mixed batch in ONE persistent launch (the paper's Algorithm 4 admits a new
 * query whenever one completes; here the device work queue does it across
 * requests of different algorithms and lengths).  Request r is described by
 * algos[r], params[r], sources[r] (n_sources[r] entries), max_lens[r],
 * seeds[r], out_paths[r], out_lengths[r], with the meaning of trw_walk.
 * Pointers are device pointers.  n_requests in 1 .. TRW_MAX_BATCH.
 * Synchronous when sync = 1 (see trw_walk_ex).
 */
#define TRW_MAX_BATCH 64
trw_status trw_walk_batch(trw_graph* g, int32_t n_requests, const trw_algo* algos, const trw_params* params,
                          const int32_t* const* sources, const int64_t* n_sources, const int32_t* max_lens,
                          const uint64_t* seeds, int32_t* const* out_paths, int32_t* const* out_lengths,
                          void* stream, int sync);

/*
 * Batch plans (no counterpart in the paper, whose executor is a CPU loop): the
 * mixed batch of trw_walk_batch, with the same arguments and the same device
 * buffers, captured once as a CUDA graph (control reset, one source check
 * over every request, the persistent walk launch) and
 * replayed by trw_plan_launch with a single graph launch.  Every replay
 * re-walks the batch into the same outputs; the walks of a replay are those
 * of trw_walk_batch with the plan's current seeds.  The plan keeps the
 * graph's launch configuration and prepared tables as they were at creation;
 * destroy plans before their graph.  The buffers must stay valid while the
 * plan exists.
 *   trw_plan_create   validates and captures; nothing runs.
 *                     Errors: those of trw_walk_batch, TRW_ERR_OOM, TRW_ERR_CUDA.
 *   trw_plan_set_seed changes request r's seed for the next launch (waits for
 *                     the previous launch of the plan to finish).
 *   trw_plan_launch   enqueues one replay on stream (NULL: the graph's
 *                     stream); asynchronous.
 *   trw_plan_sync     waits for the last launch and returns its status
 *                     (TRW_ERR_INVALID for a source outside [0, nv): nothing
 *                     was written; TRW_ERR_REJECT_CAP); *moves (may be NULL)
 *                     receives the moves it made.
 *   trw_plan_destroy  waits for the last launch and frees the plan.
 */
typedef struct trw_plan trw_plan;
trw_status trw_plan_create(trw_graph* g, int32_t n_requests, const trw_algo* algos, const trw_params* params,
                           const int32_t* const* sources, const int64_t* n_sources, const int32_t* max_lens,
                           const uint64_t* seeds, int32_t* const* out_paths, int32_t* const* out_lengths,
                           trw_plan** plan);
trw_status trw_plan_set_seed(trw_plan* plan, int32_t request, uint64_t seed);
trw_status trw_plan_launch(trw_plan* plan, void* stream);
trw_status trw_plan_sync(trw_plan* plan, int64_t* moves);
void trw_plan_destroy(trw_plan* plan);

/*
 * trw_walk_batch with no allocation (the paper has no counterpart: this is an
 * interface for callers that must not allocate device memory during the call,
 * e.g. code running while the caller's memory pool owns the free device
 * memory, code under an allocator that must see every allocation, or code
 * that must not let cudaMalloc/cudaFree synchronise the device).
 * Same requests, results and errors as trw_walk_batch (device buffers only),
 * on the caller's stream (NULL: the legacy default stream).  Synchronous on
 * that stream: the request table goes up from host memory on it, and the call
 * returns once the walks are done and their status is read back on it; it
 * waits for no other stream unless that stream is the legacy default stream,
 * which orders itself after every blocking stream of the device.  Refused
 * with TRW_ERR_INVALID when the current device is not the graph's.
 * Its scratch -- control block, request table, prefix sums, about 9 KB -- is a
 * fixed array in device memory that every GPU loading the library holds
 * until the process exits; n_requests above TRW_NOALLOC_MAX_REQUESTS is
 * refused with TRW_ERR_INVALID.  The first call on a device looks up the
 * array's device address: make it before any stream capture.  All calls share
 * the array (each clears what must start at zero); calls that overlap on the
 * GPU race on it.
 */
#define TRW_NOALLOC_MAX_REQUESTS 64
trw_status trw_walk_batch_noalloc(const trw_graph* g, int32_t n_requests, const trw_algo* algos,
                                  const trw_params* params, const int32_t* const* sources, const int64_t* n_sources,
                                  const int32_t* max_lens, const uint64_t* seeds, int32_t* const* out_paths,
                                  int32_t* const* out_lengths, void* stream);

/* Launch shape and tuning knobs of the persistent kernel (the GPU analogue of
 * the ring sizes k and k' of Section 5.4). */
typedef struct {
  int32_t block_threads;        /* threads per block, multiple of 32, 64..512 */
  int32_t blocks_per_sm;        /* resident blocks per SM requested (0: occupancy maximum) */
  int32_t chunk;                /* walks claimed from the work queue per warp claim, >= 1 */
  int32_t coop_degree;          /* MetaPath label rows at least this long: Gather by the whole warp, >= 1 */
  int32_t search_degree;        /* Node2Vec IsNeighbor in rows of prev at least this long: 32-way warp
                                   search, >= 33 (0x7fffffff: every search by its own lane) */
} trw_tuning;

/* Read or set the tuning of the graph's persistent kernel.  Setting checks ranges
 * (TRW_ERR_INVALID).  Results never depend on tuning. */
trw_status trw_get_tuning(const trw_graph* g, trw_tuning* t);
trw_status trw_set_tuning(trw_graph* g, const trw_tuning* t);

/*
 * Autotune (the analogue of Section 5.4's ring-size tuning): time short
 * pre-walks of the given algorithm from sampled sources over a grid of
 * tunings and keep the fastest.  Writes the choice to *best when non-NULL.
 */
trw_status trw_autotune(trw_graph* g, trw_algo algo, const trw_params* params, int32_t max_len,
                        trw_tuning* best);

/* Counters of the last completed call on this graph. */
typedef struct {
  int64_t walks;                /* walks run */
  int64_t moves;                /* total moves (steps) taken */
  double kernel_ms;             /* device time of the walk kernel (CUDA events) */
  int32_t grid_blocks;          /* launch shape used */
  int32_t block_threads;
  int32_t kernel;               /* TRW_KERNEL_PLAIN, _PERSISTENT or _BSP: the kernel that ran */
  int32_t launches;             /* walk-kernel launches of the call (BSP: one per step, plus one) */
} trw_stats;
trw_status trw_last_stats(const trw_graph* g, trw_stats* s);

/* Graph facts. */
int64_t trw_graph_nv(const trw_graph* g);
int64_t trw_graph_ne(const trw_graph* g);
/* Bytes of device memory the graph holds (CSR, weights, labels, tables). */
int64_t trw_graph_device_bytes(const trw_graph* g);

/* Copy the device ALIAS tables to host buffers of ne entries each:
 * H (probability threshold; 0xFFFFFFFF marks a one-element bucket),
 * first/second destination vertex (-1, -1 for a dead vertex).  For tests. */
trw_status trw_debug_alias(const trw_graph* g, uint32_t* H, int32_t* first, int32_t* second);

/* Copy the guided ITS records to host memory, 8 uint32 words per edge slot:
 * {U low, U high, destination, its row offset, its degree, first candidate of
 * the cell, last candidate of the cell, 0}.  For tests.  Errors:
 * TRW_ERR_INVALID (NULL argument), TRW_ERR_NOT_PREPARED, TRW_ERR_CUDA. */
trw_status trw_debug_its_records(const trw_graph* g, uint32_t* words);

/* Copy the row records to host memory, 4 int32 words per edge slot e = (v ->
 * dst): {dst, its row offset, its degree, aux}, aux the integer weight W_e on a
 * weighted graph, else the position of v in dst's row (-1: none, or rows not
 * sorted).  For tests.  Errors: TRW_ERR_INVALID (NULL argument),
 * TRW_ERR_NOT_PREPARED, TRW_ERR_CUDA. */
trw_status trw_debug_row_records(const trw_graph* g, int32_t* words);

/* Copy the ITS prefix sums (host uint64[ne]) and/or the REJ bounds (host
 * uint32[nv]) to host buffers; a NULL buffer is skipped.  For tests.
 * Errors: TRW_ERR_INVALID (NULL graph), TRW_ERR_NOT_PREPARED (a requested
 * table was not built), TRW_ERR_CUDA. */
trw_status trw_debug_sampler_tables(const trw_graph* g, uint64_t* cdf, uint32_t* pmax);

/*
 * Copy of the MetaPath label index (tests): *stride receives the words per
 * record (0 when not prepared); when vrec and erec are both non-NULL they
 * receive nv * stride and ne * stride int32 (host).  Errors: TRW_ERR_INVALID
 * (NULL graph or stride), TRW_ERR_CUDA.
 */
trw_status trw_debug_label_index(const trw_graph* g, int32_t* stride, int32_t* vrec, int32_t* erec);

/*
 * IsNeighbor(v[i], u[i]) for n pairs as the walk kernels evaluate it (the
 * neighbour hash where prepared, else the binary search of u's sorted row):
 * out[i] = 1 when v[i] is in N(u[i]).  Host arrays; every u[i] in [0, nv).
 * Errors: TRW_ERR_INVALID (NULL argument, n < 0, a u out of range),
 * TRW_ERR_OOM, TRW_ERR_CUDA.
 */
trw_status trw_debug_is_neighbor(const trw_graph* g, const int32_t* u, const int32_t* v, int64_t n, uint8_t* out);

/* Philox4x32-10 blocks computed on the device: out[4*i..4*i+3] for counter
 * ctr[4*i..4*i+3] and key (key0, key1).  Host buffers.  For tests. */
trw_status trw_debug_philox(const uint32_t* ctr, int64_t n, uint32_t key0, uint32_t key1, uint32_t* out);

/*
 * Test hook (the paper has no counterpart): after the next `after`
 * allocations of device or pinned host memory that the library makes, every
 * later one fails as if the device were out of memory, until the hook is
 * reset with a negative `after`.  Calls then return TRW_ERR_OOM and leave the
 * graph or server as it was.  Process-wide; for failure tests only.
 */
void trw_debug_fail_allocs(int64_t after);

/*
 * Test hook (the paper has no counterpart): the device checks of every call
 * compare the graph's device with `device` instead of the current device
 * (negative: the current device again).  It changes no launch: a call either
 * refuses with TRW_ERR_INVALID or runs on the current device as always.
 * Process-wide; lets a one-GPU test exercise the wrong-device refusal.
 */
void trw_debug_pretend_device(int32_t device);

/* ------------------------------------------------------------- serving */

/* Serving configuration. */
typedef struct {
  int64_t max_inflight_walks;   /* admission: walks admitted but not finished */
  int64_t max_inflight_bytes;   /* admission: output bytes admitted but not collected */
  int32_t max_requests;         /* request slots, 1 .. 4096 */
  int32_t idle_timeout_us;      /* the resident kernel exits after this long without work */
} trw_serve_config;

void trw_serve_config_default(trw_serve_config* c);

/*
 * Create a server over a loaded (and, for weighted walks, prepared) graph.
 * Requests that arrive while others run join the running device work queue
 * (continuous batching): a resident persistent kernel polls a request ring
 * with bounded waits and exits after idle_timeout_us without work; the next
 * submit relaunches it.
 */
trw_status trw_serve_create(trw_graph* g, const trw_serve_config* cfg, trw_server** out);

/*
 * Submit a request (same meaning as trw_walk; out_paths and out_lengths must be
 * DEVICE buffers that stay valid until poll returns TRW_OK or an error, and
 * that no other stream still writes when submit is called: the server runs
 * on its own streams and orders itself after the caller's only through
 * trw_serve_order_after).
 * sources may be host or device, and every source is range-checked before any
 * walk of the request runs.  Host sources, and device sources of requests with
 * more than TRW_SERVE_DEVICE_CHECK_MAX sources, are checked at submit
 * (TRW_ERR_INVALID for one outside [0, nv): nothing queued or written).  The
 * device sources of a smaller request are checked on the device when the
 * server admits it, which saves submit a copy to the host and a wait: one
 * outside [0, nv) completes the request with TRW_ERR_INVALID (reported by
 * poll or reap) and nothing is written.  Host sources are copied into the
 * server's pool before submit returns; device sources are read in place, so
 * they must stay valid and unchanged until the request is reported.  Submit does not wait for the walk kernel.  Returns TRW_ERR_BUSY when admitting it would exceed the
 * configured walk, byte or slot limits (nothing is queued), else queues it
 * and writes *req_id.
 */
#define TRW_SERVE_DEVICE_CHECK_MAX 1024
trw_status trw_serve_submit(trw_server* s, trw_algo algo, const trw_params* params, const int32_t* sources,
                            int64_t n_sources, int32_t max_len, uint64_t seed, int32_t* out_paths,
                            int32_t* out_lengths, uint64_t* req_id);

/*
 * Orders the server after a caller's stream without blocking the host: the
 * requests submitted after this call become visible to the device (and
 * their device sources are read for the range check) only once the work
 * queued on stream before this call has finished -- e.g. the allocation or
 * fill of a request's buffers.  stream is a cudaStream_t ((void*)1 names the
 * legacy default stream).  A stream with no work left orders nothing, and the
 * next submit publishes at once.  Errors: TRW_ERR_INVALID (NULL), TRW_ERR_CUDA.
 */
trw_status trw_serve_order_after(trw_server* s, void* stream);

/* TRW_OK when request req_id has finished (its slot is released), TRW_PENDING
 * while it runs, TRW_ERR_NOT_FOUND for an unknown or already collected id,
 * or the request's error status. */
trw_status trw_serve_poll(trw_server* s, uint64_t req_id);

/* Collect up to max finished requests (oldest first) in one call:
 * ids[i] and statuses[i] (TRW_OK or the request's error status) for
 * i < *n_out; each is released as by trw_serve_poll.  *n_out = 0 when none
 * has finished.  Errors: TRW_ERR_INVALID (bad arguments), TRW_ERR_CUDA,
 * TRW_ERR_INTERNAL (a failed device self-check). */
trw_status trw_serve_reap(trw_server* s, uint64_t* ids, int32_t* statuses, int32_t max, int32_t* n_out);

/* Device timeline of request req_id (tracing; the paper has no counterpart):
 * t_ns[0] when the kernel's dispatcher took it in, t_ns[1] when a worker
 * first loaded it (its walks start), t_ns[2] when its last walk finished, on
 * the device's global nanosecond clock (0: not reached yet).  Valid while the
 * request's slot has not been reused (fewer than max_requests later submits).
 * Errors: TRW_ERR_INVALID, TRW_ERR_NOT_FOUND, TRW_ERR_CUDA. */
trw_status trw_serve_trace(trw_server* s, uint64_t req_id, uint64_t* t_ns);

/* Wait (bounded by timeout_ms) until every submitted request has finished. */
trw_status trw_serve_drain(trw_server* s, int32_t timeout_ms);

/* Stop the resident kernel, wait for it and free the server. */
void trw_serve_destroy(trw_server* s);

/* Thread-local message describing the last non-OK status of this thread. */
const char* trw_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TRW_H */
