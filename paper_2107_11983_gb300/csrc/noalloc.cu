// trw_walk_batch_noalloc: the mixed-batch walk of trw_walk_batch for callers
// that must not allocate device memory during the call.
//
// Some callers can't call cudaMalloc at the point where they walk: code that
// runs while the caller's memory pool owns all free device memory, code that
// sits under an allocator that must see every allocation, or code paths that
// must not synchronise the device (cudaMalloc and cudaFree may).  This entry
// point needs nothing beyond the caller's inputs and outputs: its scratch --
// the work-queue control block, the request table and its prefix sums -- is a
// file-scope device array of fixed size, resident on every GPU that loads the
// library until the process exits.
//
// Its host code uses the array through the device address that
// cudaGetSymbolAddress returns; the host-side name of the array is only a
// stand-in and is never handed to a kernel.  The address is looked up once per
// device, by the first call on that device, with that device current; make that
// first call before any stream capture.
//
// All calls share the array and it keeps the last call's contents: each call
// clears the control block before its kernels run, and calls that overlap on
// the GPU (different streams, or host threads that do not serialise) race on
// it.
//
// The call is synchronous on the stream it is given: its request table goes
// up from host memory on that stream, and it returns once the walks are done
// and their status is read back on that stream.  It waits for no other
// stream, unless the stream given is the legacy default stream (NULL), which
// orders itself after every blocking stream of the device.
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "trw_api_internal.h"

using namespace trw;

namespace {

constexpr int kNoAllocMaxRequests = TRW_NOALLOC_MAX_REQUESTS;

// Layout of the scratch array: control block, request table, prefix sums.
constexpr size_t kCtrlOff = 0;
constexpr size_t kSpecOff = 256;
constexpr size_t kPrefixOff = kSpecOff + sizeof(WalkSpec) * kNoAllocMaxRequests;
constexpr size_t kScratchBytes = kPrefixOff + sizeof(int64_t) * (kNoAllocMaxRequests + 1);
static_assert(sizeof(Ctrl) <= kSpecOff, "control block fits its slot");
static_assert(kSpecOff % alignof(WalkSpec) == 0 && kPrefixOff % 8 == 0, "aligned sections");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_addr_mu;
void* g_addr[128] = {nullptr};  // device address of g_noalloc_scratch, per device ordinal

// Device address of the scratch array on the current device (looked up once).
trw_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return trw_cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 128) return trw_fail(TRW_ERR_INTERNAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return trw_cuda_fail(e, "cudaGetSymbolAddress of the no-alloc scratch");
    if (!p) return trw_fail(TRW_ERR_INTERNAL, "no device address for the no-alloc scratch");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return TRW_OK;
}

}  // namespace

extern "C" trw_status trw_walk_batch_noalloc(const trw_graph* g, int32_t n_requests, const trw_algo* algos,
                                             const trw_params* params, const int32_t* const* sources,
                                             const int64_t* n_sources, const int32_t* max_lens,
                                             const uint64_t* seeds, int32_t* const* out_paths,
                                             int32_t* const* out_lengths, void* stream_v) {
  if (!g) return trw_fail(TRW_ERR_INVALID, "graph is NULL");
  // The graph's arrays live on one device: refuse before any launch when
  // another one is current (its kernels would read another GPU's memory).
  if (trw_status dc = trw_check_device(g); dc != TRW_OK) return dc;
  if (n_requests < 1 || n_requests > kNoAllocMaxRequests)
    return trw_fail(TRW_ERR_INVALID, "n_requests must be in [1, %d] (the size of the no-alloc request table)",
                    kNoAllocMaxRequests);
  if (!algos || !sources || !n_sources || !max_lens || !seeds || !out_paths || !out_lengths)
    return trw_fail(TRW_ERR_INVALID, "NULL array");
  WalkSpec specs[kNoAllocMaxRequests];
  int64_t prefix[kNoAllocMaxRequests + 1];
  prefix[0] = 0;
  for (int r = 0; r < n_requests; ++r) {
    trw_status st = trw_make_spec(g, algos[r], params ? &params[r] : nullptr, n_sources[r], max_lens[r], seeds[r],
                                  &specs[r]);
    if (st != TRW_OK) return trw_fail(st, "request %d: %s", r, trw_last_error());
    if (specs[r].nwalks > 0 &&
        (!trw_is_device_ptr(sources[r]) || !trw_is_device_ptr(out_paths[r]) || !trw_is_device_ptr(out_lengths[r])))
      return trw_fail(TRW_ERR_INVALID, "request %d: buffers must be device memory", r);
    specs[r].sources = sources[r];
    specs[r].out_paths = out_paths[r];
    specs[r].out_lengths = out_lengths[r];
    prefix[r + 1] = prefix[r] + specs[r].nwalks;
  }
  void* base = nullptr;
  trw_status st = scratch_address(&base);
  if (st != TRW_OK) return st;
  unsigned char* b = static_cast<unsigned char*>(base);
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(b + kCtrlOff);
  WalkSpec* d_specs = reinterpret_cast<WalkSpec*>(b + kSpecOff);
  int64_t* d_prefix = reinterpret_cast<int64_t*>(b + kPrefixOff);
  cudaStream_t stream = stream_v ? (cudaStream_t)stream_v : (cudaStream_t)0;
  // Host arrays are pageable stack memory: these copies complete their reads of
  // them before returning.
  cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_specs, specs, sizeof(WalkSpec) * (size_t)n_requests, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_prefix, prefix, sizeof(int64_t) * ((size_t)n_requests + 1), cudaMemcpyHostToDevice, stream);
  for (int r = 0; r < n_requests && e == cudaSuccess; ++r)
    if (specs[r].nwalks > 0) e = launch_validate_sources(specs[r].sources, n_sources[r], (int32_t)g->nv, ctrl, stream);
  // the launch configuration of trw_walk_batch for the same requests
  const LaunchCfg cfg = trw_launch_cfg_batch(g, specs, n_requests);
  if (e == cudaSuccess)
    e = launch_walk_batch(trw_dev_graph(g), d_specs, d_prefix, n_requests, prefix[n_requests], ctrl, stream, cfg);
  Ctrl c;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&c, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return trw_cuda_fail(e, "no-alloc batch walk");
  if (c.err == kErrRejectCap) return trw_fail(TRW_ERR_REJECT_CAP, "a rejection step exceeded %d trials", TRW_REJECT_CAP);
  if (c.err == kErrInvalid) return trw_fail(TRW_ERR_INVALID, "a source vertex is outside [0, nv)");
  if (c.err != 0) return trw_fail(TRW_ERR_INTERNAL, "device status %d", c.err);
  return TRW_OK;
}
