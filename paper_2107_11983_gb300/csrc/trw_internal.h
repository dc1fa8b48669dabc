// Host-side declarations shared by the translation units of libtrw.so.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "trw_device.cuh"

namespace trw {

struct LaunchCfg {
  int block_threads = 256;
  int grid_blocks = 0;       // persistent: resident blocks over all SMs
  int chunk = 32;            // walks per warp claim
  int coop_degree = 256;     // MetaPath label rows this long or longer: warp-cooperative Gather
  int search_degree = 0x7fffffff;  // Node2Vec rows of prev this long or longer: warp search
  bool batch_coop = true;    // mixed batches: the variant with the warp-cooperative scan and search
};

// Occupancy-derived resident blocks per SM of the persistent kernel for algo
// (coop: the variant with the warp-cooperative scan and search).
int persistent_blocks_per_sm(int algo, int block_threads, bool coop);

// Step-synchronous baseline: bytes of one stored walker, the launch that
// creates the walkers (all live unless max_len is 0) and one step launch over
// n live walkers; each appends the walkers still alive to out and counts them
// in *n_out.
size_t bsp_walker_bytes();
cudaError_t launch_bsp_init(const DevGraph& g, const WalkSpec& sp, void* out, unsigned long long* n_out, Ctrl* ctrl,
                            cudaStream_t st);
cudaError_t launch_bsp_step(const DevGraph& g, const WalkSpec& sp, const void* in, int64_t n, void* out,
                            unsigned long long* n_out, Ctrl* ctrl, cudaStream_t st);
cudaError_t launch_validate_sources(const int32_t* src, int64_t n, int32_t nv, Ctrl* ctrl, cudaStream_t st);
cudaError_t launch_walk_plain(const DevGraph& g, const WalkSpec& sp, Ctrl* ctrl, cudaStream_t st, int block);
cudaError_t launch_walk_persistent(const DevGraph& g, const WalkSpec& sp, Ctrl* ctrl, cudaStream_t st,
                                   const LaunchCfg& cfg);
cudaError_t launch_walk_batch(const DevGraph& g, const WalkSpec* d_specs, const int64_t* d_prefix, int nreq,
                              int64_t total, Ctrl* ctrl, cudaStream_t st, const LaunchCfg& cfg);

// ALIAS preprocessing (Algorithm 3) on the device; synchronises st.  The
// three scratch arrays hold ne elements each.
cudaError_t launch_prepare_alias(int32_t nv, int64_t ne, const int32_t* row_ptr, const int32_t* col,
                                 const float* weights, AliasRec* alias, unsigned long long* q_scratch,
                                 int32_t* idx_scratch, int32_t* part_scratch, Ctrl* ctrl, cudaStream_t st);

// MetaPath label index (LabelIndex): the largest label into *d_out (atomicMax;
// zero it first), then the vertex and edge records for nl labels at stride
// words per record; the second call synchronises st.
cudaError_t launch_label_max(const uint8_t* labels, int64_t ne, unsigned int* d_out, cudaStream_t st);
cudaError_t launch_prepare_labels(int32_t nv, int64_t ne, const int32_t* row_ptr, const int32_t* col,
                                  const uint8_t* labels, int32_t nl, int32_t stride, int32_t* vrec, int32_t* erec,
                                  cudaStream_t st);

// Neighbour hash (NeighborHash) of the rows of at least min_degree entries,
// built into slots (2 ne int32, allocated by the caller); synchronises st.
cudaError_t launch_neighbor_hash(int32_t nv, int64_t ne, const int32_t* row_ptr, const int32_t* col,
                                 int32_t min_degree, int32_t* slots, cudaStream_t st);

// Row records {col[e], row_ptr[col[e]], deg(col[e]), 0} of every edge slot.
cudaError_t launch_row_records(int32_t nv, int64_t ne, const int32_t* row_ptr, const int32_t* col,
                               const float* weights, bool sorted, RowRec* rec,
                               cudaStream_t st);
cudaError_t launch_sampler_tables(int32_t nv, const int32_t* row_ptr, const float* weights, unsigned long long* cdf,
                                  uint32_t* pmax, cudaStream_t st);
cudaError_t launch_its_records(int32_t nv, const int32_t* row_ptr, const int32_t* col, const float* weights,
                               ItsRec* rec, cudaStream_t st);
cudaError_t launch_check_weights(int64_t ne, const float* weights, Ctrl* ctrl, cudaStream_t st);

// Graph checks: ids in range, rows strictly increasing (sets *sorted_flag to 0 when not).
cudaError_t launch_check_graph(int32_t nv, const int32_t* row_ptr, const int32_t* col, Ctrl* ctrl,
                               int* d_unsorted, cudaStream_t st);

cudaError_t launch_debug_is_neighbor(const DevGraph& g, const int32_t* u, const int32_t* v, int64_t n, uint8_t* out,
                                     cudaStream_t st);
cudaError_t launch_debug_philox(const uint32_t* d_ctr, int64_t n, uint32_t k0, uint32_t k1, uint32_t* d_out,
                                cudaStream_t st);

}  // namespace trw

// Every device and pinned host allocation of the library goes through these
// two (the allocation-failure test hook of trw.h sits here).
cudaError_t trw_dev_malloc(void** p, size_t bytes);
cudaError_t trw_host_alloc(void** p, size_t bytes, unsigned int flags);
