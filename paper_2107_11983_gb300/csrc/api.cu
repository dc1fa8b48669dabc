// Host side of the C ABI declared in include/trw.h: argument checks, device
// residency of the graph, staging of host buffers, launches and status.
// Every step of a walk runs in the kernels of walk_kernels.cu and
// prepare_kernels.cu; this file never computes a walk on the host.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/trw.h"
#include "trw_api_internal.h"
#include "trw_internal.h"

using namespace trw;

// ------------------------------------------------------------------ errors

static thread_local std::string t_last_error;

trw_status trw_fail(trw_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_last_error = buf;
  return st;
}

trw_status trw_cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // not sticky: clear it so the next call starts clean
    return trw_fail(TRW_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  }
  return trw_fail(TRW_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" const char* trw_last_error(void) { return t_last_error.c_str(); }

// ------------------------------------------- allocation gate, device check
// Two test hooks (declared in trw.h) make failures that a test could not
// otherwise cause on a healthy one-GPU machine.  Neither can make a call do
// anything but refuse or fail cleanly: the injected allocation failure is
// reported as the runtime's own out-of-memory error, and the pretended device
// only changes what the device check compares.

static std::atomic<long long> g_allocs_before_failure{-1};  // -1: no injected failure
static std::atomic<int> g_pretend_device{-1};               // -1: the current device

extern "C" void trw_debug_fail_allocs(int64_t after) { g_allocs_before_failure.store(after < 0 ? -1 : after); }

extern "C" void trw_debug_pretend_device(int32_t device) { g_pretend_device.store(device < 0 ? -1 : device); }

// True when the test hook makes this allocation fail: once its count of
// allocations to let through reaches zero, every later one fails until the
// hook is reset.
static bool injected_alloc_failure() {
  long long n = g_allocs_before_failure.load();
  while (n > 0 && !g_allocs_before_failure.compare_exchange_weak(n, n - 1)) {
  }
  return n == 0;
}

cudaError_t trw_dev_malloc(void** p, size_t bytes) {
  if (injected_alloc_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

cudaError_t trw_host_alloc(void** p, size_t bytes, unsigned int flags) {
  if (injected_alloc_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaHostAlloc(p, bytes, flags);
}

trw_status trw_check_device(const trw_graph* g) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return trw_cuda_fail(e, "cudaGetDevice");
  const int pretend = g_pretend_device.load();
  if (pretend >= 0) dev = pretend;
  if (dev != g->device)
    return trw_fail(TRW_ERR_INVALID, "the current device is %d but the graph lives on device %d", dev, g->device);
  return TRW_OK;
}

// ------------------------------------------------------------ small helpers

bool trw_is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static uint64_t threshold_of(double t) {
  if (!(t > 0.0)) return 0;
  if (t >= 1.0) return 4294967296ull;
  return (uint64_t)std::floor(t * 4294967296.0);
}

trw_status trw_grow(void** p, size_t* cap, size_t need) {
  if (*cap >= need) return TRW_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  size_t n = std::max(need, (size_t)4096);
  cudaError_t e = trw_dev_malloc(p, n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return trw_fail(TRW_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", n, cudaGetErrorString(e));
  }
  *cap = n;
  return TRW_OK;
}

// --------------------------------------------------------------------- load

extern "C" void trw_params_default(trw_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->ppr_stop = 0.2;
  p->n2v_p = 1.0;
  p->n2v_q = 1.0;
  p->schema = nullptr;
  p->schema_len = 0;
  p->out_mode = TRW_OUT_PATHS;
  p->walks_per_source = 1;
  p->walk_offset = 0;
}

static void graph_release(trw_graph* g) {
  if (!g) return;
  cudaFree(g->row_ptr);
  cudaFree(g->col);
  cudaFree(g->weights);
  cudaFree(g->labels);
  cudaFree(g->alias);
  cudaFree(g->lvrec);
  cudaFree(g->lerec);
  cudaFree(g->nh_slots);
  cudaFree(g->rrec);
  cudaFree(g->its_cdf);
  cudaFree(g->rej_pmax);
  cudaFree(g->its_rec);
  cudaFree(g->bsp_walkers[0]);
  cudaFree(g->bsp_walkers[1]);
  if (g->bsp_host) cudaFreeHost(g->bsp_host);
  trw_free_stream_buffers(g);
  cudaFree(g->cmp_stage);
  cudaFree(g->cmp_scratch);
  if (g->cmp_host) cudaFreeHost(g->cmp_host);
  cudaFree(g->ctrl);
  cudaFree(g->src_stage);
  cudaFree(g->out_stage);
  cudaFree(g->len_stage);
  cudaFree(g->batch_specs);
  if (g->batch_host) cudaFreeHost(g->batch_host);
  cudaFree(g->misc);
  if (g->ev0) cudaEventDestroy(g->ev0);
  if (g->ev1) cudaEventDestroy(g->ev1);
  for (int b = 0; b < 2; ++b) {
    if (g->ev_walked[b]) cudaEventDestroy(g->ev_walked[b]);
    if (g->ev_copied[b]) cudaEventDestroy(g->ev_copied[b]);
  }
  if (g->copy_stream) cudaStreamDestroy(g->copy_stream);
  if (g->stream2) cudaStreamDestroy(g->stream2);
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  if (g->ev_join) cudaEventDestroy(g->ev_join);
  cudaFree(g->ctrl2);
  if (g->stream) cudaStreamDestroy(g->stream);
  delete g;
}

extern "C" void trw_graph_free(trw_graph* g) { graph_release(g); }

static trw_status alloc_dev(void** p, size_t bytes, const char* what) {
  cudaError_t e = trw_dev_malloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return trw_fail(TRW_ERR_OOM, "cudaMalloc for %s (%zu bytes) failed: %s", what, bytes, cudaGetErrorString(e));
  }
  return TRW_OK;
}

extern "C" trw_status trw_graph_load(int64_t nv, int64_t ne, const int64_t* row_ptr, const int32_t* col,
                                     const float* weights, const uint8_t* labels, uint32_t flags, trw_graph** out) {
  (void)flags;
  if (!out) return trw_fail(TRW_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (nv < 0 || ne < 0 || nv >= (int64_t)INT32_MAX || ne >= (int64_t)INT32_MAX)
    return trw_fail(TRW_ERR_INVALID, "nv=%lld ne=%lld outside [0, 2^31-1)", (long long)nv, (long long)ne);
  if (!row_ptr) return trw_fail(TRW_ERR_INVALID, "row_ptr is NULL");
  if (ne > 0 && !col) return trw_fail(TRW_ERR_INVALID, "col is NULL");
  if (row_ptr[0] != 0) return trw_fail(TRW_ERR_INVALID, "row_ptr[0] != 0");
  std::vector<int32_t> rp32((size_t)nv + 1);
  for (int64_t v = 0; v <= nv; ++v) {
    const int64_t x = row_ptr[v];
    if (v > 0 && x < row_ptr[v - 1])
      return trw_fail(TRW_ERR_INVALID, "row_ptr decreases at vertex %lld", (long long)v);
    rp32[(size_t)v] = (int32_t)x;
  }
  if (row_ptr[nv] != ne) return trw_fail(TRW_ERR_INVALID, "row_ptr[nv]=%lld != ne=%lld", (long long)row_ptr[nv], (long long)ne);

  trw_graph* g = new trw_graph();
  g->nv = nv;
  g->ne = ne;
  trw_status st;
  cudaError_t e = cudaGetDevice(&g->device);
  if (e != cudaSuccess) {
    graph_release(g);
    return trw_cuda_fail(e, "cudaGetDevice");
  }
  cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
  if (g->num_sms <= 0) g->num_sms = 1;
#define LOAD_TRY(x)          \
  do {                       \
    st = (x);                \
    if (st != TRW_OK) {      \
      graph_release(g);      \
      return st;             \
    }                        \
  } while (0)
#define LOAD_CUDA(call, what)                       \
  do {                                              \
    cudaError_t e2 = (call);                        \
    if (e2 != cudaSuccess) {                        \
      graph_release(g);                             \
      return trw_cuda_fail(e2, what);               \
    }                                               \
  } while (0)
  LOAD_CUDA(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking), "cudaStreamCreate");
  LOAD_CUDA(cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking), "cudaStreamCreate");
  LOAD_CUDA(cudaStreamCreateWithFlags(&g->stream2, cudaStreamNonBlocking), "cudaStreamCreate");
  LOAD_CUDA(cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming), "cudaEventCreate");
  LOAD_CUDA(cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming), "cudaEventCreate");
  for (int b = 0; b < 2; ++b) {
    LOAD_CUDA(cudaEventCreateWithFlags(&g->ev_walked[b], cudaEventDisableTiming), "cudaEventCreate");
    LOAD_CUDA(cudaEventCreateWithFlags(&g->ev_copied[b], cudaEventDisableTiming), "cudaEventCreate");
  }
  LOAD_CUDA(cudaEventCreate(&g->ev0), "cudaEventCreate");
  LOAD_CUDA(cudaEventCreate(&g->ev1), "cudaEventCreate");
  LOAD_TRY(alloc_dev((void**)&g->row_ptr, sizeof(int32_t) * ((size_t)nv + 1), "row_ptr"));
  LOAD_TRY(alloc_dev((void**)&g->col, sizeof(int32_t) * ((size_t)ne + 4), "col"));
  LOAD_TRY(alloc_dev((void**)&g->ctrl, sizeof(Ctrl), "ctrl"));
  LOAD_TRY(alloc_dev((void**)&g->ctrl2, sizeof(Ctrl), "ctrl"));
  LOAD_TRY(alloc_dev((void**)&g->misc, 256, "misc"));
  LOAD_CUDA(cudaMemcpy(g->row_ptr, rp32.data(), sizeof(int32_t) * ((size_t)nv + 1), cudaMemcpyHostToDevice), "copy row_ptr");
  if (ne > 0) LOAD_CUDA(cudaMemcpy(g->col, col, sizeof(int32_t) * (size_t)ne, cudaMemcpyHostToDevice), "copy col");
  if (weights) {
    LOAD_TRY(alloc_dev((void**)&g->weights, sizeof(float) * ((size_t)ne + 4), "weights"));
    if (ne > 0) LOAD_CUDA(cudaMemcpy(g->weights, weights, sizeof(float) * (size_t)ne, cudaMemcpyHostToDevice), "copy weights");
  }
  if (labels) {
    // padded so that aligned 4- and 16-byte loads of the last row stay inside the allocation
    LOAD_TRY(alloc_dev((void**)&g->labels, (size_t)ne + 64, "labels"));
    LOAD_CUDA(cudaMemset(g->labels, 0, (size_t)ne + 64), "memset labels");
    if (ne > 0) LOAD_CUDA(cudaMemcpy(g->labels, labels, (size_t)ne, cudaMemcpyHostToDevice), "copy labels");
  }
  // Device checks: ids in range, rows sorted.
  LOAD_CUDA(cudaMemset(g->ctrl, 0, sizeof(Ctrl)), "memset ctrl");
  LOAD_CUDA(cudaMemset(g->misc, 0, 256), "memset misc");
  LOAD_CUDA(launch_check_graph((int32_t)nv, g->row_ptr, g->col, g->ctrl, (int*)g->misc, g->stream), "check graph");
  LOAD_CUDA(cudaStreamSynchronize(g->stream), "check graph");
  Ctrl c;
  int unsorted = 0;
  LOAD_CUDA(cudaMemcpy(&c, g->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost), "read ctrl");
  LOAD_CUDA(cudaMemcpy(&unsorted, g->misc, sizeof(int), cudaMemcpyDeviceToHost), "read flag");
  if (c.err != 0) {
    graph_release(g);
    return trw_fail(TRW_ERR_INVALID, "a column id is outside [0, nv)");
  }
  if (g->weights) {
    LOAD_CUDA(launch_check_weights(ne, g->weights, g->ctrl, g->stream), "check weights");
    LOAD_CUDA(cudaStreamSynchronize(g->stream), "check weights");
    LOAD_CUDA(cudaMemcpy(&c, g->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost), "read ctrl");
    if (c.err != 0) {
      graph_release(g);
      return trw_fail(TRW_ERR_INVALID, "an edge weight is negative or not finite");
    }
  }
  g->sorted = unsorted == 0;
  g->tuning.block_threads = 256;
  g->tuning.blocks_per_sm = 0;
  g->tuning.chunk = 32;
  g->tuning.coop_degree = 256;
  g->tuning.search_degree = 0x7fffffff;
  g->device_bytes = (int64_t)(sizeof(int32_t) * ((size_t)nv + 1) + sizeof(int32_t) * (size_t)ne +
                              (weights ? sizeof(float) * (size_t)ne : 0) + (labels ? (size_t)ne : 0));
  *out = g;
  return TRW_OK;
#undef LOAD_TRY
#undef LOAD_CUDA
}

extern "C" trw_status trw_graph_get_view(const trw_graph* g, trw_graph_view* out) {
  if (!g || !out) return trw_fail(TRW_ERR_INVALID, "NULL argument");
  out->row_ptr = g->row_ptr;
  out->col = g->col;
  out->weights = g->weights;
  out->labels = g->labels;
  out->nv = g->nv;
  out->ne = g->ne;
  out->sorted = g->sorted ? 1 : 0;
  out->device = g->device;
  return TRW_OK;
}

extern "C" int64_t trw_graph_nv(const trw_graph* g) { return g ? g->nv : -1; }
extern "C" int64_t trw_graph_ne(const trw_graph* g) { return g ? g->ne : -1; }
extern "C" int64_t trw_graph_device_bytes(const trw_graph* g) { return g ? g->device_bytes : -1; }

DevGraph trw_dev_graph(const trw_graph* g) {
  DevGraph d;
  d.row_ptr = g->row_ptr;
  d.col = g->col;
  d.alias = g->alias;
  d.labels = g->labels;
  d.weights = g->weights;
  d.cdf = g->its_cdf;
  d.pmax = g->rej_pmax;
  d.its_rec = g->its_rec;
  d.rrec = g->rrec;
  d.rrec_rev = (g->rrec && !g->weights) ? 1 : 0;
  d.lidx.vrec = g->lvrec;
  d.lidx.erec = g->lerec;
  d.lidx.stride = g->lstride;
  d.lidx.nl = g->lnl;
  d.nh.slots = g->nh_slots;
  d.nh.min_degree = TRW_NEIGHBOR_HASH_MIN_DEGREE;
  d.nv = (int32_t)g->nv;
  d.ne = (int32_t)g->ne;
  return d;
}

// ------------------------------------------------------------------ prepare

static trw_status prepare_alias(trw_graph* g) {
  if (!g->weights) return trw_fail(TRW_ERR_INVALID, "ALIAS preparation needs edge weights");
  const size_t ne = (size_t)g->ne;
  if (!g->alias) {
    trw_status st = alloc_dev((void**)&g->alias, sizeof(AliasRec) * (ne + 1), "alias tables");
    if (st != TRW_OK) return st;
    g->device_bytes += (int64_t)(sizeof(AliasRec) * ne);
  }
  unsigned long long* q = nullptr;
  int32_t *sm = nullptr, *lg = nullptr;
  trw_status st = alloc_dev((void**)&q, sizeof(unsigned long long) * (ne + 1), "alias scratch");
  if (st == TRW_OK) st = alloc_dev((void**)&sm, sizeof(int32_t) * (ne + 1), "alias scratch");
  if (st == TRW_OK) st = alloc_dev((void**)&lg, sizeof(int32_t) * (ne + 1), "alias scratch");
  cudaError_t e = cudaSuccess;
  Ctrl c{};
  if (st == TRW_OK) {
    e = cudaMemsetAsync(g->ctrl, 0, sizeof(Ctrl), g->stream);
    if (e == cudaSuccess)
      e = launch_prepare_alias((int32_t)g->nv, g->ne, g->row_ptr, g->col, g->weights, g->alias, q, sm, lg, g->ctrl,
                               g->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&c, g->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost);
  }
  cudaFree(q);
  cudaFree(sm);
  cudaFree(lg);
  if (st != TRW_OK) return st;
  if (e != cudaSuccess) return trw_cuda_fail(e, "prepare alias");
  if (c.err != 0) {
    g->prepared_alias = false;
    return trw_fail(TRW_ERR_INVALID, "an edge weight is negative or not finite");
  }
  g->prepared_alias = true;
  return TRW_OK;
}

static trw_status prepare_label_index(trw_graph* g) {
  if (!g->labels) return trw_fail(TRW_ERR_INVALID, "the label index needs edge labels");
  if (g->lerec) return TRW_OK;
  unsigned int* d_max = reinterpret_cast<unsigned int*>(static_cast<char*>(g->misc) + 64);
  unsigned int mx = 0;
  cudaError_t e = cudaMemsetAsync(d_max, 0, sizeof(unsigned int), g->stream);
  if (e == cudaSuccess) e = launch_label_max(g->labels, g->ne, d_max, g->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&mx, d_max, sizeof(unsigned int), cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return trw_cuda_fail(e, "label maximum");
  const int32_t nl = (int32_t)mx + 1;
  if (nl > TRW_LABEL_INDEX_MAX_LABELS)
    return trw_fail(TRW_ERR_INVALID, "label %u is too large for the label index (at most %d labels)", mx,
                    TRW_LABEL_INDEX_MAX_LABELS);
  const int32_t stride = nl + 2 <= 8 ? 8 : nl + 2 <= 16 ? 16 : 32;
  int32_t *vrec = nullptr, *erec = nullptr;
  const size_t vbytes = sizeof(int32_t) * (size_t)stride * (size_t)g->nv;
  const size_t ebytes = sizeof(int32_t) * (size_t)stride * (size_t)g->ne;
  trw_status st = alloc_dev((void**)&vrec, vbytes, "label index");
  if (st == TRW_OK) st = alloc_dev((void**)&erec, ebytes, "label index");
  if (st == TRW_OK) {
    e = launch_prepare_labels((int32_t)g->nv, g->ne, g->row_ptr, g->col, g->labels, nl, stride, vrec, erec,
                              g->stream);
    if (e != cudaSuccess) st = trw_cuda_fail(e, "prepare label index");
  }
  if (st != TRW_OK) {
    cudaFree(vrec);
    cudaFree(erec);
    return st;
  }
  g->lvrec = vrec;
  g->lerec = erec;
  g->lstride = stride;
  g->lnl = nl;
  g->device_bytes += (int64_t)(vbytes + ebytes);
  return TRW_OK;
}

static trw_status prepare_neighbor_hash(trw_graph* g) {
  if (g->nh_slots) return TRW_OK;
  int32_t* slots = nullptr;
  const size_t bytes = sizeof(int32_t) * 2 * (size_t)g->ne;
  trw_status st = alloc_dev((void**)&slots, bytes, "neighbour hash");
  if (st != TRW_OK) return st;
  const cudaError_t e =
      launch_neighbor_hash((int32_t)g->nv, g->ne, g->row_ptr, g->col, TRW_NEIGHBOR_HASH_MIN_DEGREE, slots, g->stream);
  if (e != cudaSuccess) {
    cudaFree(slots);
    return trw_cuda_fail(e, "prepare neighbour hash");
  }
  g->nh_slots = slots;
  g->device_bytes += (int64_t)bytes;
  return TRW_OK;
}

static trw_status prepare_row_records(trw_graph* g) {
  if (g->rrec) return TRW_OK;
  RowRec* rec = nullptr;
  const size_t bytes = sizeof(RowRec) * (size_t)g->ne;
  trw_status st = alloc_dev((void**)&rec, bytes, "row records");
  if (st != TRW_OK) return st;
  cudaError_t e = launch_row_records((int32_t)g->nv, g->ne, g->row_ptr, g->col, g->weights, g->sorted, rec, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) {
    cudaFree(rec);
    return trw_cuda_fail(e, "prepare row records");
  }
  g->rrec = rec;
  g->device_bytes += (int64_t)bytes;
  return TRW_OK;
}

// ITS prefix sums and REJ bounds (Algorithm 3 with the ITS and REJ
// initialisations of Section 2.3), built together in one pass over the weights.
static trw_status prepare_sampler_tables(trw_graph* g, bool its, bool rej) {
  if (its && g->its_cdf) its = false;
  if (rej && g->rej_pmax) rej = false;
  if (!its && !rej) return TRW_OK;
  unsigned long long* cdf = nullptr;
  uint32_t* pmax = nullptr;
  const size_t cbytes = sizeof(unsigned long long) * (size_t)g->ne, pbytes = sizeof(uint32_t) * (size_t)g->nv;
  trw_status st = TRW_OK;
  if (its) st = alloc_dev((void**)&cdf, cbytes, "ITS prefix sums");
  if (st == TRW_OK && rej) st = alloc_dev((void**)&pmax, pbytes, "REJ bounds");
  if (st == TRW_OK) {
    cudaError_t e = launch_sampler_tables((int32_t)g->nv, g->row_ptr, g->weights, cdf, pmax, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) st = trw_cuda_fail(e, "prepare ITS / REJ tables");
  }
  if (st != TRW_OK) {
    cudaFree(cdf);
    cudaFree(pmax);
    return st;
  }
  if (cdf) {
    g->its_cdf = cdf;
    g->device_bytes += (int64_t)cbytes;
  }
  if (pmax) {
    g->rej_pmax = pmax;
    g->device_bytes += (int64_t)pbytes;
  }
  return TRW_OK;
}

static trw_status prepare_its_records(trw_graph* g) {
  if (g->its_rec) return TRW_OK;
  ItsRec* rec = nullptr;
  const size_t bytes = sizeof(ItsRec) * (size_t)g->ne;
  trw_status st = alloc_dev((void**)&rec, bytes, "guided ITS records");
  if (st != TRW_OK) return st;
  cudaError_t e = launch_its_records((int32_t)g->nv, g->row_ptr, g->col, g->weights, rec, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) {
    cudaFree(rec);
    return trw_cuda_fail(e, "prepare guided ITS records");
  }
  g->its_rec = rec;
  g->device_bytes += (int64_t)bytes;
  return TRW_OK;
}

extern "C" trw_status trw_prepare(trw_graph* g, uint32_t what) {
  if (!g) return trw_fail(TRW_ERR_INVALID, "graph is NULL");
  if (trw_status dc = trw_check_device(g); dc != TRW_OK) return dc;
  if (what & ~(TRW_PREP_ALIAS | TRW_PREP_LABEL_INDEX | TRW_PREP_NEIGHBOR_HASH | TRW_PREP_ROW_RECORDS | TRW_PREP_ITS |
               TRW_PREP_REJ | TRW_PREP_ITS_GUIDE))
    return trw_fail(TRW_ERR_INVALID, "unknown prepare flags 0x%x", what);
  std::lock_guard<std::mutex> lk(g->mu);
  if ((what & TRW_PREP_ALIAS) && !g->weights) return trw_fail(TRW_ERR_INVALID, "ALIAS preparation needs edge weights");
  if ((what & (TRW_PREP_ITS | TRW_PREP_REJ | TRW_PREP_ITS_GUIDE)) && !g->weights)
    return trw_fail(TRW_ERR_INVALID, "ITS and REJ preparation need edge weights");
  if ((what & TRW_PREP_LABEL_INDEX) && !g->labels) return trw_fail(TRW_ERR_INVALID, "the label index needs edge labels");
  if (what & TRW_PREP_ALIAS) {
    trw_status st = prepare_alias(g);
    if (st != TRW_OK) return st;
  }
  if (what & TRW_PREP_LABEL_INDEX) {
    trw_status st = prepare_label_index(g);
    if (st != TRW_OK) return st;
  }
  if (what & TRW_PREP_NEIGHBOR_HASH) {
    trw_status st = prepare_neighbor_hash(g);
    if (st != TRW_OK) return st;
  }
  if (what & (TRW_PREP_ITS | TRW_PREP_REJ)) {
    trw_status st = prepare_sampler_tables(g, (what & TRW_PREP_ITS) != 0, (what & TRW_PREP_REJ) != 0);
    if (st != TRW_OK) return st;
  }
  if (what & TRW_PREP_ITS_GUIDE) {
    trw_status st = prepare_its_records(g);
    if (st != TRW_OK) return st;
  }
  if (what & TRW_PREP_ROW_RECORDS) return prepare_row_records(g);
  return TRW_OK;
}

// --------------------------------------------------------------------- walk

trw_status trw_make_spec(const trw_graph* g, trw_algo algo, const trw_params* pin, int64_t n_sources,
                         int32_t max_len, uint64_t seed, WalkSpec* sp, bool allow_compact) {
  trw_params p;
  if (pin) p = *pin;
  else trw_params_default(&p);
  std::memset(sp, 0, sizeof(*sp));
  if ((int)algo < TRW_DEEPWALK || (int)algo > TRW_NODE2VEC_WEIGHTED)
    return trw_fail(TRW_ERR_INVALID, "unknown algorithm %d", (int)algo);
  if (max_len < 0) return trw_fail(TRW_ERR_INVALID, "max_len < 0");
  if (n_sources < 0) return trw_fail(TRW_ERR_INVALID, "n_sources < 0");
  if (p.walks_per_source < 1) return trw_fail(TRW_ERR_INVALID, "walks_per_source < 1");
  if (p.out_mode != TRW_OUT_PATHS && p.out_mode != TRW_OUT_ENDPOINTS && !(allow_compact && p.out_mode == TRW_OUT_COMPACT))
    return trw_fail(TRW_ERR_INVALID, p.out_mode == TRW_OUT_COMPACT ? "compact output is for trw_walk and trw_walk_ex only"
                                                                  : "bad out_mode");
  if (p.walk_offset < 0) return trw_fail(TRW_ERR_INVALID, "walk_offset < 0");
  const int64_t nwalks = n_sources * (int64_t)p.walks_per_source;
  if (n_sources > 0 && nwalks / n_sources != p.walks_per_source) return trw_fail(TRW_ERR_INVALID, "walk count overflows");
  if (p.walk_offset + nwalks > 4294967296LL) return trw_fail(TRW_ERR_INVALID, "walk indices exceed 2^32");
  if (n_sources > 0 && g->nv == 0) return trw_fail(TRW_ERR_INVALID, "sources on an empty graph");
  sp->algo = (int32_t)algo;
  sp->max_len = max_len;
  sp->wps = (uint32_t)p.walks_per_source;
  sp->endpoints = p.out_mode == TRW_OUT_ENDPOINTS ? 1u : 0u;
  sp->key0 = (uint32_t)seed;
  sp->key1 = (uint32_t)(seed >> 32);
  sp->walk_offset = (uint32_t)p.walk_offset;
  sp->nwalks = nwalks;
  if (algo == TRW_PPR) {
    if (!(p.ppr_stop >= 0.0 && p.ppr_stop <= 1.0)) return trw_fail(TRW_ERR_INVALID, "ppr_stop outside [0, 1]");
    sp->T_stop = threshold_of(p.ppr_stop);
  }
  if (algo == TRW_NODE2VEC || algo == TRW_NODE2VEC_WEIGHTED) {
    if (!(p.n2v_p > 0.0) || !(p.n2v_q > 0.0) || !std::isfinite(p.n2v_p) || !std::isfinite(p.n2v_q))
      return trw_fail(TRW_ERR_INVALID, "node2vec p and q must be finite and > 0");
    if (!g->sorted) return trw_fail(TRW_ERR_INVALID, "node2vec needs sorted adjacency rows");
    const double w_ret = 1.0 / p.n2v_p, w_nb = 1.0, w_far = 1.0 / p.n2v_q;
    double pstar = w_ret > w_nb ? w_ret : w_nb;
    if (w_far > pstar) pstar = w_far;
    sp->T_ret = threshold_of(w_ret / pstar);
    sp->T_nb = threshold_of(w_nb / pstar);
    sp->T_far = threshold_of(w_far / pstar);
    sp->T_lo = std::min(sp->T_nb, sp->T_far);
    sp->T_hi = std::max(sp->T_nb, sp->T_far);
  }
  if (algo == TRW_NODE2VEC_WEIGHTED) {
    // Eq. 1 times w_e: the weight word's bound is the caller's max_weight,
    // quantised like a weight, or the row's p*_v when max_weight is 0
    if (!g->weights) return trw_fail(TRW_ERR_INVALID, "weighted node2vec needs edge weights");
    if (p.max_weight == 0.0) {
      if (!g->rej_pmax)
        return trw_fail(TRW_ERR_NOT_PREPARED, "weighted node2vec without max_weight needs trw_prepare(TRW_PREP_REJ)");
    } else {
      if (!std::isfinite(p.max_weight) || !(p.max_weight > 0.0))
        return trw_fail(TRW_ERR_INVALID, "max_weight must be finite and > 0 (or 0 for the REJ bounds)");
      double t = std::rint(p.max_weight * 65536.0);
      if (t > 4294967295.0) t = 4294967295.0;
      if (t < 1.0) return trw_fail(TRW_ERR_INVALID, "max_weight %g quantises to 0", p.max_weight);
      sp->T_stop = (uint64_t)t;
    }
    sp->algo = N2V_W;
  }
  if (algo == TRW_METAPATH) {
    if (!g->labels) return trw_fail(TRW_ERR_INVALID, "metapath needs edge labels");
    if (!p.schema || p.schema_len < 1 || p.schema_len > TRW_MAX_SCHEMA)
      return trw_fail(TRW_ERR_INVALID, "metapath schema length must be in [1, %d]", TRW_MAX_SCHEMA);
    sp->schema_len = (uint32_t)p.schema_len;
    for (int i = 0; i < p.schema_len; ++i) {
      if (i < 8) sp->schema_lo |= (uint64_t)p.schema[i] << (8 * i);
      else sp->schema_hi |= (uint64_t)p.schema[i] << (8 * (i - 8));
    }
  }
  if (p.sampler != TRW_SAMPLER_DEFAULT && algo != TRW_DEEPWALK_WEIGHTED)
    return trw_fail(TRW_ERR_INVALID, "a sampler can be chosen for weighted DeepWalk only");
  if (algo == TRW_DEEPWALK_WEIGHTED) {
    if (!g->weights) return trw_fail(TRW_ERR_INVALID, "weighted walks need edge weights");
    switch (p.sampler) {
      case TRW_SAMPLER_DEFAULT:
        if (!g->prepared_alias) return trw_fail(TRW_ERR_NOT_PREPARED, "call trw_prepare(TRW_PREP_ALIAS) first");
        break;
      case TRW_SAMPLER_ITS:
        if (!g->its_cdf && !g->its_rec)
          return trw_fail(TRW_ERR_NOT_PREPARED, "call trw_prepare(TRW_PREP_ITS or TRW_PREP_ITS_GUIDE) first");
        sp->algo = DW_ITS;
        break;
      case TRW_SAMPLER_REJ:
        if (!g->rej_pmax) return trw_fail(TRW_ERR_NOT_PREPARED, "call trw_prepare(TRW_PREP_REJ) first");
        sp->algo = DW_REJ;
        break;
      case TRW_SAMPLER_OREJ: {
        // the bound P = round-half-even(MaxWeight * 2^16), clamped like a weight
        if (!std::isfinite(p.max_weight) || !(p.max_weight > 0.0))
          return trw_fail(TRW_ERR_INVALID, "O-REJ needs a finite max_weight > 0");
        double t = std::rint(p.max_weight * 65536.0);
        if (t > 4294967295.0) t = 4294967295.0;
        if (t < 1.0) return trw_fail(TRW_ERR_INVALID, "max_weight %g quantises to 0", p.max_weight);
        sp->T_stop = (uint64_t)t;  // the bound rides in the PPR-only threshold
        sp->algo = DW_OREJ;
        break;
      }
      default: return trw_fail(TRW_ERR_INVALID, "unknown sampler %d", (int)p.sampler);
    }
  }
  return TRW_OK;
}

LaunchCfg trw_launch_cfg(const trw_graph* g, int algo) {
  LaunchCfg c;
  c.block_threads = g->tuning.block_threads;
  int bps = g->tuning.blocks_per_sm;
  const bool coop = algo == MIXED || (algo == METAPATH && !g->lerec && g->tuning.coop_degree < 0x7fffffff) ||
                    (is_n2v(algo) && !g->nh_slots && g->tuning.search_degree < 0x7fffffff);
  const int occ = persistent_blocks_per_sm(algo, c.block_threads, coop);
  if (bps <= 0 || bps > occ) bps = occ;
  c.grid_blocks = g->num_sms * bps;
  c.chunk = g->tuning.chunk;
  c.coop_degree = g->tuning.coop_degree;
  c.search_degree = g->tuning.search_degree;
  if (algo == METAPATH && g->lerec) c.coop_degree = 0x7fffffff;  // indexed: no label scans to share
  if (g->nh_slots) c.search_degree = 0x7fffffff;                  // hashed: no row searches to share
  return c;
}

LaunchCfg trw_launch_cfg_batch(const trw_graph* g, const WalkSpec* specs, int n) {
  // The cooperative variant only when a request can hand work to its warp.
  bool coop = false;
  for (int r = 0; r < n; ++r) {
    if (specs[r].algo == NODE2VEC && !g->nh_slots && g->tuning.search_degree < 0x7fffffff) coop = true;
    if (specs[r].algo == METAPATH && !g->lerec && g->tuning.coop_degree < 0x7fffffff) coop = true;
  }
  LaunchCfg c;
  c.block_threads = g->tuning.block_threads;
  const int occ = persistent_blocks_per_sm(MIXED, c.block_threads, coop);
  int bps = g->tuning.blocks_per_sm;
  if (bps <= 0 || bps > occ) bps = occ;
  c.grid_blocks = g->num_sms * bps;
  // A claim of a mixed batch also looks up each walk's request: a warp takes
  // at least one walk per lane per claim, whatever a single-algorithm tuning chose.
  c.chunk = std::max(32, g->tuning.chunk);
  c.coop_degree = g->tuning.coop_degree;
  c.search_degree = g->nh_slots ? 0x7fffffff : g->tuning.search_degree;
  c.batch_coop = coop;
  return c;
}

static trw_status collect_status(trw_graph* g, cudaStream_t stream) {
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return trw_cuda_fail(e, "walk kernel");
  Ctrl c;
  e = cudaMemcpy(&c, g->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return trw_cuda_fail(e, "read status");
  float ms = 0.f;
  if (g->timed && cudaEventElapsedTime(&ms, g->ev0, g->ev1) == cudaSuccess) g->last.kernel_ms = ms;
  cudaGetLastError();
  g->last.moves = (int64_t)c.moves;
  if (c.err != 0) {
    cudaMemsetAsync(&g->ctrl->err, 0, sizeof(int), stream);
    cudaStreamSynchronize(stream);
    if (c.err == kErrRejectCap) return trw_fail(TRW_ERR_REJECT_CAP, "a rejection step exceeded %d trials", TRW_REJECT_CAP);
    if (c.err == kErrInvalid) return trw_fail(TRW_ERR_INVALID, "a source vertex is outside [0, nv)");
    return trw_fail(TRW_ERR_INTERNAL, "device status %d", c.err);
  }
  return TRW_OK;
}

// Slices of at least this many walks overlap their copy-out with the next walk.
static constexpr int64_t kSliceWalks = 1 << 19;

// The synchronous walk of trw_walk_ex with host outputs, sliced: slice i walks
// into staging buffer b = i % 2 on compute stream b (the caller's stream or
// the graph's second one, each with its own control block), so that the
// blocks of slice i + 1 start on the SMs that slice i's tail leaves idle; its
// paths and lengths are copied to the host on the graph's copy stream while
// the next slices walk; slice i + 2 waits until the copy of slice i has
// drained its buffer.
static trw_status walk_sliced(trw_graph* g, WalkSpec sp, trw_kernel kernel, const int32_t* d_src, int64_t n_sources,
                              int64_t row, int32_t* out_paths, int32_t* out_lengths, cudaStream_t stream) {
  const int64_t wps = (int64_t)sp.wps;
  const int64_t nwalks = sp.nwalks;
  // Slices of 2^18 walks, 2 to 16 of them: more slices shorten the copy-out
  // tail that no walk overlaps (weighted DeepWalk s22: 8 -> 16 slices,
  // 9.24 -> 8.85 ms), but past 16 the slices' own walk tails cost more
  // (Node2Vec s24: 32 slices, 82 -> 87 ms).
  int64_t nslices = nwalks / (kSliceWalks / 2);
  if (nslices < 2) nslices = 2;
  if (nslices > 16) nslices = 16;
  const int64_t src_per = (n_sources + nslices - 1) / nslices;
  const int64_t walks_per = src_per * wps;
  trw_status st = trw_grow((void**)&g->out_stage, &g->out_cap, sizeof(int32_t) * (size_t)(2 * walks_per * row));
  if (st != TRW_OK) return st;
  st = trw_grow((void**)&g->len_stage, &g->len_cap, sizeof(int32_t) * (size_t)(2 * walks_per));
  if (st != TRW_OK) return st;
  const DevGraph dg = trw_dev_graph(g);
  const LaunchCfg cfg = trw_launch_cfg(g, sp.algo);
  cudaStream_t cs = g->copy_stream;
  cudaStream_t ks[2] = {stream, g->stream2};
  Ctrl* kc[2] = {g->ctrl, g->ctrl2};
  CUDA_TRY(cudaMemsetAsync(g->ctrl, 0, sizeof(Ctrl), stream), "reset ctrl");
  CUDA_TRY(cudaMemsetAsync(g->ctrl2, 0, sizeof(Ctrl), stream), "reset ctrl");
  CUDA_TRY(cudaEventRecord(g->ev0, stream), "event");
  CUDA_TRY(cudaEventRecord(g->ev_fork, stream), "event");
  CUDA_TRY(cudaStreamWaitEvent(g->stream2, g->ev_fork, 0), "fork");
  int64_t done_src = 0;
  int32_t slices = 0;
  for (int64_t i = 0; done_src < n_sources; ++i, ++slices) {
    const int b = (int)(i & 1);
    cudaStream_t kst = ks[b];
    const int64_t s0 = done_src, s1 = std::min(n_sources, s0 + src_per);
    WalkSpec sl = sp;
    sl.sources = d_src + s0;
    sl.nwalks = (s1 - s0) * wps;
    sl.walk_offset = sp.walk_offset + (uint32_t)(s0 * wps);
    sl.out_paths = g->out_stage + (size_t)b * (size_t)(walks_per * row);
    sl.out_lengths = g->len_stage + (size_t)b * (size_t)walks_per;
    if (i >= 2) CUDA_TRY(cudaStreamWaitEvent(kst, g->ev_copied[b], 0), "wait for a drained buffer");
    CUDA_TRY(cudaMemsetAsync(&kc[b]->head, 0, sizeof(unsigned long long), kst), "reset queue");
    if (kernel == TRW_KERNEL_PLAIN) CUDA_TRY(launch_walk_plain(dg, sl, kc[b], kst, 256), "plain walk launch");
    else CUDA_TRY(launch_walk_persistent(dg, sl, kc[b], kst, cfg), "persistent walk launch");
    CUDA_TRY(cudaEventRecord(g->ev_walked[b], kst), "event");
    CUDA_TRY(cudaStreamWaitEvent(cs, g->ev_walked[b], 0), "wait for a walked slice");
    CUDA_TRY(cudaMemcpyAsync(out_paths + s0 * wps * row, sl.out_paths, sizeof(int32_t) * (size_t)(sl.nwalks * row),
                             cudaMemcpyDeviceToHost, cs),
             "copy paths");
    CUDA_TRY(cudaMemcpyAsync(out_lengths + s0 * wps, sl.out_lengths, sizeof(int32_t) * (size_t)sl.nwalks,
                             cudaMemcpyDeviceToHost, cs),
             "copy lengths");
    CUDA_TRY(cudaEventRecord(g->ev_copied[b], cs), "event");
    done_src = s1;
  }
  CUDA_TRY(cudaEventRecord(g->ev_join, g->stream2), "event");
  CUDA_TRY(cudaStreamWaitEvent(stream, g->ev_join, 0), "join");
  CUDA_TRY(cudaEventRecord(g->ev1, stream), "event");
  g->timed = true;
  g->last.grid_blocks = cfg.grid_blocks;
  g->last.block_threads = cfg.block_threads;
  g->last.kernel = kernel == TRW_KERNEL_PLAIN ? TRW_KERNEL_PLAIN : TRW_KERNEL_PERSISTENT;
  g->last.launches = slices;
  CUDA_TRY(cudaStreamSynchronize(cs), "copy stream");
  // the second control block's moves and status join the first's
  Ctrl c2;
  CUDA_TRY(cudaStreamSynchronize(stream), "walk kernel");
  CUDA_TRY(cudaMemcpy(&c2, g->ctrl2, sizeof(Ctrl), cudaMemcpyDeviceToHost), "read status");
  trw_status rs = collect_status(g, stream);
  g->last.moves += (int64_t)c2.moves;
  if (rs != TRW_OK) return rs;
  if (c2.err == kErrRejectCap) return trw_fail(TRW_ERR_REJECT_CAP, "a rejection step exceeded %d trials", TRW_REJECT_CAP);
  if (c2.err == kErrInvalid) return trw_fail(TRW_ERR_INVALID, "a source vertex is outside [0, nv)");
  if (c2.err != 0) return trw_fail(TRW_ERR_INTERNAL, "device status %d", c2.err);
  return TRW_OK;
}

// The step-synchronous baseline: one launch per step over the live walkers,
// the live count read back after each.  Every launch advances or finishes
// each live walker, so there are at most max_len step launches.
static trw_status run_bsp(trw_graph* g, const DevGraph& dg, const WalkSpec& sp, cudaStream_t stream) {
  const size_t bytes = bsp_walker_bytes() * (size_t)sp.nwalks;
  for (int b = 0; b < 2; ++b) {
    trw_status st = trw_grow(&g->bsp_walkers[b], &g->bsp_cap[b], bytes);
    if (st != TRW_OK) return st;
  }
  if (!g->bsp_host)
    CUDA_TRY(trw_host_alloc((void**)&g->bsp_host, sizeof(unsigned long long), cudaHostAllocDefault), "pinned count");
  unsigned long long* d_count = reinterpret_cast<unsigned long long*>(static_cast<char*>(g->misc) + 128);
  CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), stream), "reset count");
  CUDA_TRY(launch_bsp_init(dg, sp, g->bsp_walkers[0], d_count, g->ctrl, stream), "BSP init launch");
  CUDA_TRY(cudaMemcpyAsync(g->bsp_host, d_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, stream),
           "read count");
  CUDA_TRY(cudaStreamSynchronize(stream), "BSP init");
  int64_t n = (int64_t)*g->bsp_host;
  int cur = 0;
  int32_t steps = 0;
  while (n > 0) {
    if (++steps > sp.max_len) return trw_fail(TRW_ERR_INTERNAL, "step-synchronous walk exceeded max_len steps");
    CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), stream), "reset count");
    CUDA_TRY(launch_bsp_step(dg, sp, g->bsp_walkers[cur], n, g->bsp_walkers[1 - cur], d_count, g->ctrl, stream),
             "BSP step launch");
    CUDA_TRY(cudaMemcpyAsync(g->bsp_host, d_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, stream),
             "read count");
    CUDA_TRY(cudaStreamSynchronize(stream), "BSP step");
    n = (int64_t)*g->bsp_host;
    cur = 1 - cur;
  }
  g->last.launches = steps + 1;
  g->last.grid_blocks = (int32_t)std::min<int64_t>((sp.nwalks + 255) / 256, INT32_MAX);
  g->last.block_threads = 256;
  return TRW_OK;
}

extern "C" trw_status trw_walk_ex(trw_graph* g, trw_algo algo, const trw_params* params, const int32_t* sources,
                                  int64_t n_sources, int32_t max_len, uint64_t seed, int32_t* out_paths,
                                  int32_t* out_lengths, trw_kernel kernel, void* stream_v, int sync) {
  if (!g) return trw_fail(TRW_ERR_INVALID, "graph is NULL");
  if (trw_status dc = trw_check_device(g); dc != TRW_OK) return dc;
  if (kernel != TRW_KERNEL_AUTO && kernel != TRW_KERNEL_PLAIN && kernel != TRW_KERNEL_PERSISTENT &&
      kernel != TRW_KERNEL_BSP)
    return trw_fail(TRW_ERR_INVALID, "unknown kernel %d", (int)kernel);
  if (kernel == TRW_KERNEL_BSP && !sync)
    return trw_fail(TRW_ERR_INVALID, "the step-synchronous baseline runs synchronously only");
  const bool compact = params && params->out_mode == TRW_OUT_COMPACT;
  if (compact && (!sync || kernel == TRW_KERNEL_BSP))
    return trw_fail(TRW_ERR_INVALID, "compact output runs synchronously, in the plain or persistent kernel");
  WalkSpec sp;
  trw_status st = trw_make_spec(g, algo, params, n_sources, max_len, seed, &sp, true);
  if (st != TRW_OK) return st;
  if (n_sources > 0 && (!sources || !out_paths || !out_lengths)) return trw_fail(TRW_ERR_INVALID, "NULL buffer");
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t stream = stream_v ? (cudaStream_t)stream_v : g->stream;
  const int64_t nwalks = sp.nwalks;
  const size_t out_elems = sp.endpoints ? (size_t)nwalks : (size_t)nwalks * ((size_t)max_len + 1);
  const bool src_dev = trw_is_device_ptr(sources);
  const bool out_dev = trw_is_device_ptr(out_paths);
  const bool len_dev = trw_is_device_ptr(out_lengths);
  if (!sync && (!src_dev || !out_dev || !len_dev))
    return trw_fail(TRW_ERR_INVALID, "asynchronous walks need device buffers");
  if (!src_dev && !trw_sources_in_range(sources, n_sources, g->nv)) {
    for (int64_t i = 0; i < n_sources; ++i)  // name the first offender
      if (sources[i] < 0 || sources[i] >= g->nv)
        return trw_fail(TRW_ERR_INVALID, "source %lld = %d is outside [0, %lld)", (long long)i, sources[i], (long long)g->nv);
  }
  g->last.walks = nwalks;
  g->last.moves = 0;
  g->last.kernel_ms = 0;
  g->last.launches = 0;
  g->timed = false;
  if (nwalks == 0) return TRW_OK;
  if (kernel == TRW_KERNEL_AUTO) {
    // Refill only pays when there are more walks than resident lanes: a batch
    // that fits in one wave of the persistent configuration (and needs no
    // warp-cooperative path) runs the one-launch kernel, which has less to do
    // per step.
    const LaunchCfg cfg = trw_launch_cfg(g, sp.algo);
    const bool coop = (sp.algo == METAPATH && cfg.coop_degree < 0x7fffffff) ||
                      (is_n2v(sp.algo) && cfg.search_degree < 0x7fffffff);
    kernel = !coop && nwalks <= (int64_t)cfg.grid_blocks * cfg.block_threads ? TRW_KERNEL_PLAIN : TRW_KERNEL_PERSISTENT;
  }

  const int32_t* d_src = sources;
  int32_t* d_out = out_paths;
  int32_t* d_len = out_lengths;
  if (!src_dev) {
    st = trw_grow((void**)&g->src_stage, &g->src_cap, sizeof(int32_t) * (size_t)n_sources);
    if (st != TRW_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(g->src_stage, sources, sizeof(int32_t) * (size_t)n_sources, cudaMemcpyHostToDevice, stream),
             "copy sources");
    d_src = g->src_stage;
  }
  // Device sources with host outputs (or compact output): check them before
  // anything is copied out (an invalid batch must leave the caller's buffers
  // untouched).
  if (src_dev && (!out_dev || !len_dev || compact)) {
    CUDA_TRY(cudaMemsetAsync(g->ctrl, 0, sizeof(Ctrl), stream), "reset ctrl");
    CUDA_TRY(launch_validate_sources(d_src, n_sources, (int32_t)g->nv, g->ctrl, stream), "validate sources");
    Ctrl c;
    CUDA_TRY(cudaMemcpyAsync(&c, g->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, stream), "read status");
    CUDA_TRY(cudaStreamSynchronize(stream), "validate sources");
    if (c.err != 0) return trw_fail(TRW_ERR_INVALID, "a source vertex is outside [0, nv)");
  }
  // Compact output: sliced, each slice compacted on the device and copied out
  // at its running offset.
  if (compact) {
    st = trw_walk_compact(g, sp, kernel, d_src, n_sources, out_paths, out_lengths, stream);
    if (st != TRW_OK) return st;
    return collect_status(g, stream);
  }
  // Host outputs of a large batch: walk it in source-aligned slices into two
  // device staging buffers and copy each slice out on a second stream while
  // the next slice walks (a double-buffered dump of the paths).
  const int64_t row = sp.endpoints ? 1 : (int64_t)max_len + 1;
  if (!out_dev && !len_dev && sync && nwalks >= 2 * kSliceWalks && kernel != TRW_KERNEL_BSP)
    return walk_sliced(g, sp, kernel, d_src, n_sources, row, out_paths, out_lengths, stream);
  if (!out_dev) {
    st = trw_grow((void**)&g->out_stage, &g->out_cap, sizeof(int32_t) * out_elems);
    if (st != TRW_OK) return st;
    d_out = g->out_stage;
  }
  if (!len_dev) {
    st = trw_grow((void**)&g->len_stage, &g->len_cap, sizeof(int32_t) * (size_t)nwalks);
    if (st != TRW_OK) return st;
    d_len = g->len_stage;
  }
  sp.sources = d_src;
  sp.out_paths = d_out;
  sp.out_lengths = d_len;
  const DevGraph dg = trw_dev_graph(g);
  if (sync) CUDA_TRY(cudaMemsetAsync(g->ctrl, 0, sizeof(Ctrl), stream), "reset ctrl");
  else CUDA_TRY(cudaMemsetAsync(g->ctrl, 0, offsetof(Ctrl, err), stream), "reset ctrl");
  if (src_dev) CUDA_TRY(launch_validate_sources(d_src, n_sources, (int32_t)g->nv, g->ctrl, stream), "validate sources");
  CUDA_TRY(cudaEventRecord(g->ev0, stream), "event");
  g->last.kernel = kernel;
  g->last.launches = 1;
  if (kernel == TRW_KERNEL_BSP) {
    st = run_bsp(g, dg, sp, stream);
    if (st != TRW_OK) return st;
  } else if (kernel == TRW_KERNEL_PLAIN) {
    CUDA_TRY(launch_walk_plain(dg, sp, g->ctrl, stream, 256), "plain walk launch");
    g->last.grid_blocks = (int32_t)((nwalks + 255) / 256);
    g->last.block_threads = 256;
  } else {
    const LaunchCfg cfg = trw_launch_cfg(g, sp.algo);
    CUDA_TRY(launch_walk_persistent(dg, sp, g->ctrl, stream, cfg), "persistent walk launch");
    g->last.grid_blocks = (int32_t)std::min<int64_t>(cfg.grid_blocks, (nwalks + cfg.block_threads - 1) / cfg.block_threads);
    g->last.block_threads = cfg.block_threads;
  }
  CUDA_TRY(cudaEventRecord(g->ev1, stream), "event");
  g->timed = true;
  if (!out_dev)
    CUDA_TRY(cudaMemcpyAsync(out_paths, d_out, sizeof(int32_t) * out_elems, cudaMemcpyDeviceToHost, stream), "copy paths");
  if (!len_dev)
    CUDA_TRY(cudaMemcpyAsync(out_lengths, d_len, sizeof(int32_t) * (size_t)nwalks, cudaMemcpyDeviceToHost, stream),
             "copy lengths");
  if (!sync) return TRW_OK;
  return collect_status(g, stream);
}

extern "C" trw_status trw_walk(trw_graph* g, trw_algo algo, const trw_params* params, const int32_t* sources,
                               int64_t n_sources, int32_t max_len, uint64_t seed, int32_t* out_paths,
                               int32_t* out_lengths) {
  return trw_walk_ex(g, algo, params, sources, n_sources, max_len, seed, out_paths, out_lengths, TRW_KERNEL_AUTO,
                     nullptr, 1);
}

extern "C" trw_status trw_sync(trw_graph* g, void* stream_v) {
  if (!g) return trw_fail(TRW_ERR_INVALID, "graph is NULL");
  if (trw_status dc = trw_check_device(g); dc != TRW_OK) return dc;
  std::lock_guard<std::mutex> lk(g->mu);
  return collect_status(g, stream_v ? (cudaStream_t)stream_v : g->stream);
}

extern "C" trw_status trw_walk_batch(trw_graph* g, int32_t n_requests, const trw_algo* algos, const trw_params* params,
                                     const int32_t* const* sources, const int64_t* n_sources, const int32_t* max_lens,
                                     const uint64_t* seeds, int32_t* const* out_paths, int32_t* const* out_lengths,
                                     void* stream_v, int sync) {
  if (!g) return trw_fail(TRW_ERR_INVALID, "graph is NULL");
  if (trw_status dc = trw_check_device(g); dc != TRW_OK) return dc;
  if (n_requests < 1 || n_requests > TRW_MAX_BATCH)
    return trw_fail(TRW_ERR_INVALID, "n_requests must be in [1, %d]", TRW_MAX_BATCH);
  if (!algos || !sources || !n_sources || !max_lens || !seeds || !out_paths || !out_lengths)
    return trw_fail(TRW_ERR_INVALID, "NULL array");
  std::vector<WalkSpec> specs((size_t)n_requests);
  std::vector<int64_t> prefix((size_t)n_requests + 1, 0);
  for (int r = 0; r < n_requests; ++r) {
    trw_status st = trw_make_spec(g, algos[r], params ? &params[r] : nullptr, n_sources[r], max_lens[r], seeds[r], &specs[r]);
    if (st != TRW_OK) return trw_fail(st, "request %d: %s", r, trw_last_error());
    if (specs[r].nwalks > 0) {
      if (!trw_is_device_ptr(sources[r]) || !trw_is_device_ptr(out_paths[r]) || !trw_is_device_ptr(out_lengths[r]))
        return trw_fail(TRW_ERR_INVALID, "request %d: batch buffers must be device memory", r);
    }
    specs[r].sources = sources[r];
    specs[r].out_paths = out_paths[r];
    specs[r].out_lengths = out_lengths[r];
    prefix[r + 1] = prefix[r] + specs[r].nwalks;
  }
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t stream = stream_v ? (cudaStream_t)stream_v : g->stream;
  const size_t spec_bytes = sizeof(WalkSpec) * TRW_MAX_BATCH;
  const size_t need = spec_bytes + sizeof(int64_t) * (TRW_MAX_BATCH + 1);
  if (!g->batch_specs) {
    trw_status st = alloc_dev((void**)&g->batch_specs, need, "batch table");
    if (st != TRW_OK) return st;
    CUDA_TRY(trw_host_alloc((void**)&g->batch_host, need, cudaHostAllocDefault), "pinned batch table");
  }
  // The pinned staging copy stays untouched until the previous copy finished.
  CUDA_TRY(cudaStreamSynchronize(stream), "batch table");
  std::memcpy(g->batch_host, specs.data(), sizeof(WalkSpec) * (size_t)n_requests);
  std::memcpy(g->batch_host + spec_bytes, prefix.data(), sizeof(int64_t) * ((size_t)n_requests + 1));
  CUDA_TRY(cudaMemcpyAsync(g->batch_specs, g->batch_host, need, cudaMemcpyHostToDevice, stream), "copy batch table");
  const int64_t total = prefix[(size_t)n_requests];
  g->last.walks = total;
  g->last.moves = 0;
  g->timed = false;
  if (sync) CUDA_TRY(cudaMemsetAsync(g->ctrl, 0, sizeof(Ctrl), stream), "reset ctrl");
  else CUDA_TRY(cudaMemsetAsync(g->ctrl, 0, offsetof(Ctrl, err), stream), "reset ctrl");
  for (int r = 0; r < n_requests; ++r)
    if (specs[r].nwalks > 0)
      CUDA_TRY(launch_validate_sources(specs[r].sources, n_sources[r], (int32_t)g->nv, g->ctrl, stream), "validate");
  const LaunchCfg cfg = trw_launch_cfg_batch(g, specs.data(), n_requests);
  CUDA_TRY(cudaEventRecord(g->ev0, stream), "event");
  CUDA_TRY(launch_walk_batch(trw_dev_graph(g), reinterpret_cast<const WalkSpec*>(g->batch_specs),
                             reinterpret_cast<const int64_t*>(g->batch_specs + spec_bytes), n_requests, total, g->ctrl,
                             stream, cfg),
           "batch walk launch");
  CUDA_TRY(cudaEventRecord(g->ev1, stream), "event");
  g->timed = true;
  g->last.kernel = TRW_KERNEL_PERSISTENT;
  g->last.launches = 1;
  g->last.grid_blocks = cfg.grid_blocks;
  g->last.block_threads = cfg.block_threads;
  if (!sync) return TRW_OK;
  return collect_status(g, stream);
}

// ---------------------------------------------------------------- tuning

extern "C" trw_status trw_get_tuning(const trw_graph* g, trw_tuning* t) {
  if (!g || !t) return trw_fail(TRW_ERR_INVALID, "NULL argument");
  *t = g->tuning;
  return TRW_OK;
}

extern "C" trw_status trw_set_tuning(trw_graph* g, const trw_tuning* t) {
  if (!g || !t) return trw_fail(TRW_ERR_INVALID, "NULL argument");
  if (t->block_threads < 64 || t->block_threads > 512 || (t->block_threads & 31))
    return trw_fail(TRW_ERR_INVALID, "block_threads must be a multiple of 32 in [64, 512]");
  if (t->blocks_per_sm < 0 || t->blocks_per_sm > 32) return trw_fail(TRW_ERR_INVALID, "blocks_per_sm in [0, 32]");
  if (t->chunk < 1 || t->chunk > (1 << 20)) return trw_fail(TRW_ERR_INVALID, "chunk in [1, 2^20]");
  if (t->coop_degree < 1) return trw_fail(TRW_ERR_INVALID, "coop_degree >= 1");
  if (t->search_degree < 33) return trw_fail(TRW_ERR_INVALID, "search_degree >= 33");
  std::lock_guard<std::mutex> lk(g->mu);
  g->tuning = *t;
  return TRW_OK;
}

extern "C" trw_status trw_last_stats(const trw_graph* g, trw_stats* s) {
  if (!g || !s) return trw_fail(TRW_ERR_INVALID, "NULL argument");
  *s = g->last;
  return TRW_OK;
}

// ------------------------------------------------------------------ debug

extern "C" trw_status trw_debug_alias(const trw_graph* g, uint32_t* H, int32_t* first, int32_t* second) {
  if (!g || !H || !first || !second) return trw_fail(TRW_ERR_INVALID, "NULL argument");
  if (trw_status dc = trw_check_device(g); dc != TRW_OK) return dc;
  if (!g->prepared_alias) return trw_fail(TRW_ERR_NOT_PREPARED, "no alias tables");
  std::vector<AliasRec> rec((size_t)g->ne);
  if (g->ne > 0)
    CUDA_TRY(cudaMemcpy(rec.data(), g->alias, sizeof(AliasRec) * (size_t)g->ne, cudaMemcpyDeviceToHost), "copy alias");
  for (int64_t i = 0; i < g->ne; ++i) {
    H[i] = rec[(size_t)i].a.x;
    first[i] = (int32_t)rec[(size_t)i].a.y;
    second[i] = (int32_t)rec[(size_t)i].a.z;
  }
  return TRW_OK;
}

extern "C" trw_status trw_debug_sampler_tables(const trw_graph* g, uint64_t* cdf, uint32_t* pmax) {
  if (!g) return trw_fail(TRW_ERR_INVALID, "graph is NULL");
  if (trw_status dc = trw_check_device(g); dc != TRW_OK) return dc;
  if ((cdf && !g->its_cdf) || (pmax && !g->rej_pmax)) return trw_fail(TRW_ERR_NOT_PREPARED, "table not prepared");
  if (cdf && g->ne > 0)
    CUDA_TRY(cudaMemcpy(cdf, g->its_cdf, sizeof(uint64_t) * (size_t)g->ne, cudaMemcpyDeviceToHost), "copy ITS sums");
  if (pmax && g->nv > 0)
    CUDA_TRY(cudaMemcpy(pmax, g->rej_pmax, sizeof(uint32_t) * (size_t)g->nv, cudaMemcpyDeviceToHost), "copy REJ bounds");
  return TRW_OK;
}

extern "C" trw_status trw_debug_row_records(const trw_graph* g, int32_t* words) {
  if (!g || !words) return trw_fail(TRW_ERR_INVALID, "NULL argument");
  if (trw_status dc = trw_check_device(g); dc != TRW_OK) return dc;
  if (!g->rrec) return trw_fail(TRW_ERR_NOT_PREPARED, "no row records");
  if (g->ne > 0)
    CUDA_TRY(cudaMemcpy(words, g->rrec, sizeof(RowRec) * (size_t)g->ne, cudaMemcpyDeviceToHost), "copy row records");
  return TRW_OK;
}

extern "C" trw_status trw_debug_its_records(const trw_graph* g, uint32_t* words) {
  if (!g || !words) return trw_fail(TRW_ERR_INVALID, "NULL argument");
  if (trw_status dc = trw_check_device(g); dc != TRW_OK) return dc;
  if (!g->its_rec) return trw_fail(TRW_ERR_NOT_PREPARED, "no guided ITS records");
  if (g->ne > 0)
    CUDA_TRY(cudaMemcpy(words, g->its_rec, sizeof(ItsRec) * (size_t)g->ne, cudaMemcpyDeviceToHost), "copy ITS records");
  return TRW_OK;
}

extern "C" trw_status trw_debug_label_index(const trw_graph* g, int32_t* stride, int32_t* vrec, int32_t* erec) {
  if (!g || !stride) return trw_fail(TRW_ERR_INVALID, "NULL argument");
  if (trw_status dc = trw_check_device(g); dc != TRW_OK) return dc;
  *stride = g->lerec ? g->lstride : 0;
  if (!g->lerec || !vrec || !erec) return TRW_OK;
  const size_t sw = (size_t)g->lstride;
  if (g->nv > 0)
    CUDA_TRY(cudaMemcpy(vrec, g->lvrec, sizeof(int32_t) * sw * (size_t)g->nv, cudaMemcpyDeviceToHost), "copy index");
  if (g->ne > 0)
    CUDA_TRY(cudaMemcpy(erec, g->lerec, sizeof(int32_t) * sw * (size_t)g->ne, cudaMemcpyDeviceToHost), "copy index");
  return TRW_OK;
}

extern "C" trw_status trw_debug_is_neighbor(const trw_graph* g, const int32_t* u, const int32_t* v, int64_t n,
                                            uint8_t* out) {
  if (!g || n < 0 || (n > 0 && (!u || !v || !out))) return trw_fail(TRW_ERR_INVALID, "bad arguments");
  if (trw_status dc = trw_check_device(g); dc != TRW_OK) return dc;
  for (int64_t i = 0; i < n; ++i)
    if (u[i] < 0 || u[i] >= g->nv) return trw_fail(TRW_ERR_INVALID, "vertex %d out of range", u[i]);
  if (n == 0) return TRW_OK;
  int32_t *du = nullptr, *dv = nullptr;
  uint8_t* dout = nullptr;
  trw_status st = alloc_dev((void**)&du, sizeof(int32_t) * (size_t)n, "pairs");
  if (st == TRW_OK) st = alloc_dev((void**)&dv, sizeof(int32_t) * (size_t)n, "pairs");
  if (st == TRW_OK) st = alloc_dev((void**)&dout, (size_t)n, "pairs");
  cudaError_t e = cudaSuccess;
  if (st == TRW_OK) {
    e = cudaMemcpy(du, u, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dv, v, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_debug_is_neighbor(trw_dev_graph(g), du, dv, n, dout, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, (size_t)n, cudaMemcpyDeviceToHost);
  }
  cudaFree(du);
  cudaFree(dv);
  cudaFree(dout);
  if (st != TRW_OK) return st;
  if (e != cudaSuccess) return trw_cuda_fail(e, "is_neighbor");
  return TRW_OK;
}

extern "C" trw_status trw_debug_philox(const uint32_t* ctr, int64_t n, uint32_t key0, uint32_t key1, uint32_t* out) {
  if (n < 0 || (n > 0 && (!ctr || !out))) return trw_fail(TRW_ERR_INVALID, "bad arguments");
  if (n == 0) return TRW_OK;
  uint32_t *dc = nullptr, *dout = nullptr;
  trw_status st = alloc_dev((void**)&dc, sizeof(uint32_t) * 4 * (size_t)n, "philox");
  if (st != TRW_OK) return st;
  st = alloc_dev((void**)&dout, sizeof(uint32_t) * 4 * (size_t)n, "philox");
  if (st != TRW_OK) {
    cudaFree(dc);
    return st;
  }
  cudaError_t e = cudaMemcpy(dc, ctr, sizeof(uint32_t) * 4 * (size_t)n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_debug_philox(dc, n, key0, key1, dout, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(uint32_t) * 4 * (size_t)n, cudaMemcpyDeviceToHost);
  cudaFree(dc);
  cudaFree(dout);
  if (e != cudaSuccess) return trw_cuda_fail(e, "philox");
  return TRW_OK;
}
