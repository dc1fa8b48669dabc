// The opaque handles of the C ABI and helpers shared by api.cu, serve.cu and
// autotune.cu.
#pragma once

#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/trw.h"
#include "trw_internal.h"

struct trw_graph {
  int64_t nv = 0, ne = 0;
  int device = 0;
  int num_sms = 1;
  bool sorted = false;
  bool prepared_alias = false;
  int32_t* row_ptr = nullptr;        // [nv + 1]
  int32_t* col = nullptr;            // [ne]
  float* weights = nullptr;          // [ne] or null
  uint8_t* labels = nullptr;         // [ne + 64] or null
  trw::AliasRec* alias = nullptr;    // [ne] after trw_prepare(ALIAS)
  int32_t* lvrec = nullptr;          // MetaPath label index (trw_prepare(LABEL_INDEX)): vertex records
  int32_t* lerec = nullptr;          // and edge records, lstride words each
  int32_t lstride = 0;
  int32_t lnl = 0;                   // labels in the index (largest label + 1)
  trw::RowRec* rrec = nullptr;       // row records (trw_prepare(ROW_RECORDS))
  unsigned long long* its_cdf = nullptr;  // ITS prefix sums (trw_prepare(ITS)): ne
  uint32_t* rej_pmax = nullptr;      // REJ bounds p*_v (trw_prepare(REJ)): nv
  trw::ItsRec* its_rec = nullptr;    // guided ITS records (trw_prepare(ITS_GUIDE)): ne
  void* bsp_walkers[2] = {nullptr, nullptr};  // step-synchronous baseline: walker lists (grow-only)
  size_t bsp_cap[2] = {0, 0};
  unsigned long long* bsp_host = nullptr;     // pinned: the live count read back after each step
  int32_t* pin_paths[2] = {nullptr, nullptr}; // streaming output: pinned host slices (grow-only)
  size_t pin_paths_cap[2] = {0, 0};
  int32_t* pin_lens[2] = {nullptr, nullptr};
  size_t pin_lens_cap[2] = {0, 0};
  trw::Ctrl* pin_ctrl = nullptr;              // pinned copies of the two slices' control blocks
  int32_t* cmp_stage = nullptr;               // compact output: compacted slices (grow-only)
  size_t cmp_cap = 0;
  int64_t* cmp_scratch = nullptr;             // their scan offsets, block sums and totals
  size_t cmp_scratch_cap = 0;
  int64_t* cmp_host = nullptr;                // pinned: the two slices' totals
  int32_t* nh_slots = nullptr;       // neighbour hash (trw_prepare(NEIGHBOR_HASH)): 2 ne int32
  trw::Ctrl* ctrl = nullptr;         // per-call control block
  void* misc = nullptr;              // 256 bytes of flags
  int32_t* src_stage = nullptr;      // staging for host buffers (grow-only)
  size_t src_cap = 0;
  int32_t* out_stage = nullptr;
  size_t out_cap = 0;
  int32_t* len_stage = nullptr;
  size_t len_cap = 0;
  char* batch_specs = nullptr;       // device table of a mixed batch
  char* batch_host = nullptr;        // pinned staging of that table
  cudaStream_t stream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool timed = false;
  cudaStream_t copy_stream = nullptr;              // copy-out of sliced walks
  cudaStream_t stream2 = nullptr;                  // odd slices of sliced walks (tails overlap)
  trw::Ctrl* ctrl2 = nullptr;                      // their control block
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_walked[2] = {nullptr, nullptr};   // slice walked into staging buffer b
  cudaEvent_t ev_copied[2] = {nullptr, nullptr};   // staging buffer b copied out
  trw_tuning tuning{};
  trw_stats last{};
  int64_t device_bytes = 0;
  std::mutex mu;
};

trw_status trw_fail(trw_status st, const char* fmt, ...);
void trw_free_stream_buffers(trw_graph* g);

// Every id of src[0..n) in [0, nv) (branch-free, so the loop vectorises).
inline bool trw_sources_in_range(const int32_t* src, int64_t n, int64_t nv) {
  uint32_t bad = 0;
  for (int64_t i = 0; i < n; ++i) bad |= (uint32_t)((uint32_t)src[i] >= (uint32_t)nv);
  return bad == 0;
}
trw_status trw_cuda_fail(cudaError_t e, const char* what);
// Returns TRW_ERR_CUDA from the enclosing function, with `what` and CUDA's
// message in trw_last_error(), when the runtime call fails.
#define CUDA_TRY(call, what)                                 \
  do {                                                       \
    cudaError_t e__ = (call);                                \
    if (e__ != cudaSuccess) return trw_cuda_fail(e__, what); \
  } while (0)
bool trw_is_device_ptr(const void* p);
// TRW_ERR_INVALID unless the current device is the one the graph was loaded on.
trw_status trw_check_device(const trw_graph* g);
trw_status trw_grow(void** p, size_t* cap, size_t need);
trw_status trw_make_spec(const trw_graph* g, trw_algo algo, const trw_params* p, int64_t n_sources, int32_t max_len,
                         uint64_t seed, trw::WalkSpec* sp, bool allow_compact = false);
// The walk of trw_walk_ex with TRW_OUT_COMPACT (sources on the device and
// checked; outputs host or device).  Every slice runs on `stream` and reports
// its moves and status into the graph's control block.
trw_status trw_walk_compact(trw_graph* g, trw::WalkSpec sp, trw_kernel kernel, const int32_t* d_src,
                            int64_t n_sources, int32_t* out_paths, int32_t* out_lengths, cudaStream_t stream);
trw::LaunchCfg trw_launch_cfg(const trw_graph* g, int algo);
trw::LaunchCfg trw_launch_cfg_batch(const trw_graph* g, const trw::WalkSpec* specs, int n);
trw::DevGraph trw_dev_graph(const trw_graph* g);
