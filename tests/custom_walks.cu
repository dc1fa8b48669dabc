// Walk types written against include/trw_custom.cuh, built by the tests into
// a small shared library (one extern "C" entry per walk type).  Each mirrors
// a user function set that the tests also give the oracle.
#include <cstdint>

#include "trw_custom.cuh"

namespace {

// DeepWalk restated: NAIVE, Update never ends the walk.
struct NaiveWalk {
  static constexpr trw_custom::Sampler sampler = trw_custom::Sampler::NAIVE;
  struct Params {};
  __device__ static uint32_t weight(const Params&, const trw_custom::Graph&, const trw_custom::Query&,
                                    const trw_custom::Edge&) {
    return 1;
  }
  __device__ static uint32_t max_weight(const Params&) { return 1; }
  __device__ static bool update(const Params&, const trw_custom::Graph&, const trw_custom::Query&,
                                const trw_custom::Edge&) {
    return false;
  }
};

// NAIVE; Update ends the walk on the first vertex divisible by `modulus`.
struct StopOnMultiple {
  static constexpr trw_custom::Sampler sampler = trw_custom::Sampler::NAIVE;
  struct Params {
    int32_t modulus;
  };
  __device__ static uint32_t weight(const Params&, const trw_custom::Graph&, const trw_custom::Query&,
                                    const trw_custom::Edge&) {
    return 1;
  }
  __device__ static uint32_t max_weight(const Params&) { return 1; }
  __device__ static bool update(const Params& p, const trw_custom::Graph&, const trw_custom::Query& q,
                                const trw_custom::Edge&) {
    return q.cur % p.modulus == 0;
  }
};

// Node2Vec in the paper's ten lines (Section 4.3, a = 0.5, b = 2): Eq. 1's
// weights 1/a, 1, 1/b in fixed point 4 / 2 / 1 over MaxWeight 4, times the
// integer edge weight when `weighted` (MaxWeight then 4 * the weight bound).
struct Node2VecWalk {
  static constexpr trw_custom::Sampler sampler = trw_custom::Sampler::OREJ;
  struct Params {
    int32_t weighted;
    uint32_t bound;   // integer weight bound when weighted
  };
  __device__ static uint32_t weight(const Params& p, const trw_custom::Graph& g, const trw_custom::Query& q,
                                    const trw_custom::Edge& e) {
    uint32_t c = 4;
    if (q.length > 0) c = e.dst == q.prev ? 4u : (g.is_neighbor(q.prev, e.dst) ? 2u : 1u);
    if (!p.weighted) return c;
    const float t = __ldg(g.weights + e.index) * 65536.0f;
    const uint32_t w = t >= 4294967296.0f ? 0xffffffffu : __float2uint_rn(t);
    return (uint32_t)min(0xffffffffull, (unsigned long long)c * w);
  }
  __device__ static uint32_t max_weight(const Params& p) { return p.weighted ? 4u * p.bound : 4u; }
  __device__ static bool update(const Params&, const trw_custom::Graph&, const trw_custom::Query&,
                                const trw_custom::Edge&) {
    return false;
  }
};

// A weight of both endpoints: 1 + 3 ((cur + 2 dst) mod 3) over MaxWeight 7.
struct EndpointWeight {
  static constexpr trw_custom::Sampler sampler = trw_custom::Sampler::OREJ;
  struct Params {};
  __device__ static uint32_t weight(const Params&, const trw_custom::Graph&, const trw_custom::Query& q,
                                    const trw_custom::Edge& e) {
    return 1u + 3u * (uint32_t)((q.cur + 2 * e.dst) % 3);
  }
  __device__ static uint32_t max_weight(const Params&) { return 7; }
  __device__ static bool update(const Params&, const trw_custom::Graph&, const trw_custom::Query&,
                                const trw_custom::Edge&) {
    return false;
  }
};

}  // namespace

extern "C" int tw_naive(const trw_graph* g, const int32_t* src, int64_t n, int32_t wps, int32_t max_len, uint64_t seed,
                        uint32_t offset, int32_t* paths, int32_t* lengths, int64_t* moves) {
  return trw_custom::walk<NaiveWalk>(g, NaiveWalk::Params{}, src, n, wps, max_len, seed, offset, paths, lengths,
                                     nullptr, moves);
}

extern "C" int tw_stop_on_multiple(const trw_graph* g, const int32_t* src, int64_t n, int32_t max_len, uint64_t seed,
                                   int32_t modulus, int32_t* paths, int32_t* lengths, int64_t* moves) {
  return trw_custom::walk<StopOnMultiple>(g, StopOnMultiple::Params{modulus}, src, n, 1, max_len, seed, 0, paths,
                                          lengths, nullptr, moves);
}

extern "C" int tw_node2vec(const trw_graph* g, const int32_t* src, int64_t n, int32_t max_len, uint64_t seed,
                           int32_t weighted, uint32_t bound, int32_t* paths, int32_t* lengths, int64_t* moves) {
  return trw_custom::walk<Node2VecWalk>(g, Node2VecWalk::Params{weighted, bound}, src, n, 1, max_len, seed, 0, paths,
                                        lengths, nullptr, moves);
}

extern "C" int tw_endpoint_weight(const trw_graph* g, const int32_t* src, int64_t n, int32_t wps, int32_t max_len,
                                  uint64_t seed, int32_t* paths, int32_t* lengths, int64_t* moves) {
  return trw_custom::walk<EndpointWeight>(g, EndpointWeight::Params{}, src, n, wps, max_len, seed, 0, paths, lengths,
                                          nullptr, moves);
}
