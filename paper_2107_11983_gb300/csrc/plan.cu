// Batch plans: one mixed-batch walk (the work-queue launch of
// trw_walk_batch) captured once as a CUDA graph and replayed by a single
// cudaGraphLaunch.  The graph holds three nodes: the reset of the plan's
// control block, the source check, and the persistent walk kernel.  A plan of
// several requests runs the mixed-batch kernel over a request table in device
// memory owned by the plan, and trw_plan_set_seed rewrites one entry there
// between launches.  A plan of one request runs that algorithm's own kernel
// (the one trw_walk's automatic choice would run) with the request passed by
// value, and a new seed re-captures the graph.
#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "trw_api_internal.h"
#include "walk_step.cuh"

using namespace trw;

struct trw_plan {
  trw_graph* g = nullptr;
  int32_t nreq = 0;
  int64_t n_src0 = 0;          // one-request plans: the request's source count
  trw::LaunchCfg cfg{};
  trw::DevGraph dg{};
  int64_t total = 0;
  char* d_table = nullptr;   // WalkSpec[nreq] then int64 prefix[nreq + 1]
  char* h_table = nullptr;   // pinned host copy
  size_t table_bytes = 0;
  Ctrl* ctrl = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;  // recorded after every launch
  bool launched = false;
};

namespace {

// Every request's sources in [0, nv): the batch form of the per-call check.
__global__ void validate_batch(const WalkSpec* __restrict__ specs, int nreq, int32_t nv, Ctrl* ctrl) {
  for (int r = 0; r < nreq; ++r) {
    const WalkSpec& sp = specs[r];
    const int64_t n = sp.wps ? sp.nwalks / (int64_t)sp.wps : 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      const int32_t v = sp.sources[i];
      if (v < 0 || v >= nv) step::set_err(ctrl, kErrInvalid);
    }
  }
}

void plan_release(trw_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->done) cudaEventDestroy(p->done);
  if (p->cap) cudaStreamDestroy(p->cap);
  cudaFree(p->d_table);
  cudaFree(p->ctrl);
  if (p->h_table) cudaFreeHost(p->h_table);
  delete p;
}

}  // namespace

#define PLAN_CUDA(expr, what)                          \
  do {                                                 \
    cudaError_t e_ = (expr);                           \
    if (e_ != cudaSuccess) {                           \
      plan_release(p);                                 \
      return trw_cuda_fail(e_, what);                  \
    }                                                  \
  } while (0)

// (Re)captures the plan's graph from its request table (host copy).
static cudaError_t capture(trw_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
  const WalkSpec* h_specs = reinterpret_cast<const WalkSpec*>(p->h_table);
  const size_t spec_bytes = sizeof(WalkSpec) * (size_t)p->nreq;
  const WalkSpec* d_specs = reinterpret_cast<const WalkSpec*>(p->d_table);
  const int64_t* d_prefix = reinterpret_cast<const int64_t*>(p->d_table + spec_bytes);
  int64_t max_src = 0;
  for (int r = 0; r < p->nreq; ++r)
    max_src = std::max<int64_t>(max_src, h_specs[r].wps ? h_specs[r].nwalks / (int64_t)h_specs[r].wps : 0);
  int64_t vblocks = (max_src + 255) / 256;
  if (vblocks < 1) vblocks = 1;
  if (vblocks > 4096) vblocks = 4096;
  cudaError_t e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(p->ctrl, 0, sizeof(Ctrl), p->cap);
  if (p->nreq == 1) {
    // the kernel trw_walk's automatic choice would run: the one-launch kernel
    // for a request that fits in one resident wave and needs no warp
    // cooperation, else the persistent one
    const WalkSpec& s0 = h_specs[0];
    const bool coop = (s0.algo == METAPATH && p->cfg.coop_degree < 0x7fffffff) ||
                      (is_n2v(s0.algo) && p->cfg.search_degree < 0x7fffffff);
    const bool one_wave = !coop && s0.nwalks <= (int64_t)p->cfg.grid_blocks * p->cfg.block_threads;
    if (e == cudaSuccess) e = launch_validate_sources(s0.sources, p->n_src0, p->dg.nv, p->ctrl, p->cap);
    if (e == cudaSuccess && s0.nwalks > 0)
      e = one_wave ? launch_walk_plain(p->dg, s0, p->ctrl, p->cap, 256)
                   : launch_walk_persistent(p->dg, s0, p->ctrl, p->cap, p->cfg);
  } else {
    if (e == cudaSuccess) {
      validate_batch<<<(unsigned)vblocks, 256, 0, p->cap>>>(d_specs, p->nreq, p->dg.nv, p->ctrl);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_walk_batch(p->dg, d_specs, d_prefix, p->nreq, p->total, p->ctrl, p->cap, p->cfg);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(p->cap, &graph);
  p->graph = graph;
  if (e != cudaSuccess) return e;
  if (ec != cudaSuccess) return ec;
  return cudaGraphInstantiate(&p->exec, p->graph, 0);
}

extern "C" trw_status trw_plan_create(trw_graph* g, int32_t n_requests, const trw_algo* algos,
                                      const trw_params* params, const int32_t* const* sources,
                                      const int64_t* n_sources, const int32_t* max_lens, const uint64_t* seeds,
                                      int32_t* const* out_paths, int32_t* const* out_lengths, trw_plan** out) {
  if (!out) return trw_fail(TRW_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!g) return trw_fail(TRW_ERR_INVALID, "graph is NULL");
  if (trw_status dc = trw_check_device(g); dc != TRW_OK) return dc;
  if (n_requests < 1 || n_requests > TRW_MAX_BATCH)
    return trw_fail(TRW_ERR_INVALID, "n_requests must be in [1, %d]", TRW_MAX_BATCH);
  if (!algos || !sources || !n_sources || !max_lens || !seeds || !out_paths || !out_lengths)
    return trw_fail(TRW_ERR_INVALID, "NULL array");
  std::vector<WalkSpec> specs((size_t)n_requests);
  std::vector<int64_t> prefix((size_t)n_requests + 1, 0);
  for (int r = 0; r < n_requests; ++r) {
    trw_status st = trw_make_spec(g, algos[r], params ? &params[r] : nullptr, n_sources[r], max_lens[r], seeds[r],
                                  &specs[r]);
    if (st != TRW_OK) return trw_fail(st, "request %d: %s", r, trw_last_error());
    if (specs[r].nwalks > 0 &&
        (!trw_is_device_ptr(sources[r]) || !trw_is_device_ptr(out_paths[r]) || !trw_is_device_ptr(out_lengths[r])))
      return trw_fail(TRW_ERR_INVALID, "request %d: plan buffers must be device memory", r);
    specs[r].sources = sources[r];
    specs[r].out_paths = out_paths[r];
    specs[r].out_lengths = out_lengths[r];
    prefix[r + 1] = prefix[r] + specs[r].nwalks;
  }
  trw_plan* p = new trw_plan;
  p->g = g;
  p->nreq = n_requests;
  p->total = prefix[(size_t)n_requests];
  const size_t spec_bytes = sizeof(WalkSpec) * (size_t)n_requests;
  p->table_bytes = spec_bytes + sizeof(int64_t) * ((size_t)n_requests + 1);
  PLAN_CUDA(trw_dev_malloc((void**)&p->d_table, p->table_bytes), "plan table");
  PLAN_CUDA(trw_host_alloc((void**)&p->h_table, p->table_bytes, cudaHostAllocDefault), "plan table");
  std::memcpy(p->h_table, specs.data(), spec_bytes);
  std::memcpy(p->h_table + spec_bytes, prefix.data(), sizeof(int64_t) * ((size_t)n_requests + 1));
  PLAN_CUDA(cudaMemcpy(p->d_table, p->h_table, p->table_bytes, cudaMemcpyHostToDevice), "plan table");
  PLAN_CUDA(trw_dev_malloc((void**)&p->ctrl, sizeof(Ctrl)), "plan control block");
  PLAN_CUDA(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking), "plan stream");
  PLAN_CUDA(cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming), "plan event");
  {
    std::lock_guard<std::mutex> lk(g->mu);
    p->cfg = n_requests == 1 ? trw_launch_cfg(g, specs[0].algo) : trw_launch_cfg_batch(g, specs.data(), n_requests);
    p->dg = trw_dev_graph(g);
  }
  p->n_src0 = n_sources[0];
  PLAN_CUDA(capture(p), "capture plan");
  *out = p;
  return TRW_OK;
}

extern "C" trw_status trw_plan_set_seed(trw_plan* p, int32_t request, uint64_t seed) {
  if (!p) return trw_fail(TRW_ERR_INVALID, "plan is NULL");
  if (trw_status dc = trw_check_device(p->g); dc != TRW_OK) return dc;
  if (request < 0 || request >= p->nreq) return trw_fail(TRW_ERR_INVALID, "request %d out of range", request);
  // The table is read by the last launch: wait for it before rewriting.
  if (p->launched) CUDA_TRY(cudaEventSynchronize(p->done), "plan wait");
  WalkSpec* sp = reinterpret_cast<WalkSpec*>(p->h_table) + request;
  sp->key0 = (uint32_t)seed;
  sp->key1 = (uint32_t)(seed >> 32);
  CUDA_TRY(cudaMemcpy(reinterpret_cast<WalkSpec*>(p->d_table) + request, sp, sizeof(WalkSpec), cudaMemcpyHostToDevice),
           "plan seed");
  if (p->nreq == 1) CUDA_TRY(capture(p), "plan re-capture");  // the request is a kernel argument
  return TRW_OK;
}

extern "C" trw_status trw_plan_launch(trw_plan* p, void* stream) {
  if (!p) return trw_fail(TRW_ERR_INVALID, "plan is NULL");
  if (trw_status dc = trw_check_device(p->g); dc != TRW_OK) return dc;
  cudaStream_t st = stream ? (cudaStream_t)stream : p->g->stream;
  CUDA_TRY(cudaGraphLaunch(p->exec, st), "plan launch");
  CUDA_TRY(cudaEventRecord(p->done, st), "plan event");
  p->launched = true;
  return TRW_OK;
}

extern "C" trw_status trw_plan_sync(trw_plan* p, int64_t* moves) {
  if (!p) return trw_fail(TRW_ERR_INVALID, "plan is NULL");
  if (trw_status dc = trw_check_device(p->g); dc != TRW_OK) return dc;
  if (p->launched) CUDA_TRY(cudaEventSynchronize(p->done), "plan wait");
  Ctrl c;
  CUDA_TRY(cudaMemcpy(&c, p->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost), "plan status");
  if (moves) *moves = (int64_t)c.moves;
  if (c.err == kErrRejectCap) return trw_fail(TRW_ERR_REJECT_CAP, "a rejection step exceeded %d trials", TRW_REJECT_CAP);
  if (c.err == kErrInvalid) return trw_fail(TRW_ERR_INVALID, "a source vertex is outside [0, nv)");
  if (c.err != 0) return trw_fail(TRW_ERR_INTERNAL, "device status %d", c.err);
  return TRW_OK;
}

extern "C" void trw_plan_destroy(trw_plan* p) {
  if (!p) return;
  if (p->launched) cudaEventSynchronize(p->done);
  plan_release(p);
}
