// Serving loop with continuous batching.
//
// Requests (any algorithm, any size) arrive while others run.  The host
// writes a request's descriptor into a ring of records in mapped host memory
// and publishes it by raising the request count: with a store into mapped
// memory, or, while the request must wait for a caller's stream (or its host
// sources go up first), with a copy of the count into a device counter on a
// copy stream (copy engines, no SM: the resident kernel holds every SM).  A
// submit never waits for the device.  A resident persistent kernel does the
// rest:
//   - warp 0 of block 0 is the dispatcher: it reads the two counts (the only
//     reader of the host ring), copies each new record into the device slot
//     table, cuts the request into chunks of walks and pushes them into a
//     device chunk queue;
//   - every other warp is a worker: it pops chunks (CAS on the queue head),
//     copies the request's descriptor into one of its two shared-memory slots
//     (field by field, past L1, so a reused table entry is never read stale),
//     runs the walks with the same step code as the batch kernels and refills
//     a lane as soon as its walk ends, from the newest request it holds;
//   - a warp counts the walks it finished per request and adds the count to
//     the request's completion word when it holds no more of its walks; the
//     add that completes the request writes its status and done flag, in one
//     word, to host-mapped memory.
// Every wait is bounded: with no work for idle_timeout_us the kernel exits,
// and the host relaunches it when work is pending (submit, poll, drain).
// Queue and dispatcher state live in device memory, so nothing is lost
// between launches.
#include <atomic>
#include <cmath>
#include <chrono>
#include <cstddef>
#include <cstring>
#include <cstdint>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "trw_api_internal.h"
#include "walk_step.cuh"

using namespace trw;

namespace {

constexpr uint32_t kQueueCap = 1u << 16;
constexpr int kServeThreads = 256;    // threads per block of the serving kernel
constexpr int kServeWarps = kServeThreads / 32;
constexpr int kMaxActive = 64;        // requests the dispatcher interleaves
constexpr int kPollSkip = 6;          // refills a walking warp skips after its first empty queue poll
constexpr int kPollSkipMax = 48;      // ... doubling after each further empty poll, up to this many
constexpr int64_t kDeviceCheckMax = TRW_SERVE_DEVICE_CHECK_MAX;  // device sources the dispatcher checks
// A request's completion word (SlotRec::finished): finished walks in the low
// 48 bits, one bit per error kind above them.  Recording an error and adding
// a warp's count are atomics on the same word, so the add that completes the
// request also returns every error recorded before it.
constexpr unsigned long long kCountMask = (1ull << 48) - 1;
constexpr int kErrBitRejectCap = 56, kErrBitInternal = 57;

struct Chunk {
  unsigned long long k;   // request number
  uint32_t begin, end;    // walk range within the request
  unsigned long long seq; // queue position it was written for (checked by the reader)
  unsigned long long pad;
};

// The counters that many warps touch at once sit on cache lines of their own
// (tickets on q_head, polls of q_tail, pops on q_consumed, the published
// count and the exit flag), so that polling one does not slow the atomics on
// another.
struct ServeState {       // device memory, persists across launches
  alignas(128) unsigned long long q_head;      // next queue entry to pop (tickets)
  alignas(128) unsigned long long q_tail;      // entries pushed
  alignas(128) unsigned long long q_consumed;  // entries popped and read
  alignas(128) unsigned long long published;   // requests 0..published-1 are visible: a copy-engine store of the
                                               // host's count (requests ordered after a caller's stream), raised
                                               // by the dispatcher to the host-mapped count
  alignas(128) int exit_now;      // set by the dispatcher: the launch is ending (cleared before each launch)
  alignas(128) unsigned long long disp_next;   // dispatcher: next published request to admit
  int n_act;                      // dispatcher: requests with walks not yet queued
  int rr;                         // (unused)
  unsigned long long act_k[kMaxActive];    // their request numbers
  unsigned long long act_pos[kMaxActive];  // next walk to queue
  unsigned long long act_n[kMaxActive];    // walks of the request
  unsigned long long act_cw[kMaxActive];   // walks per chunk
  unsigned long long act_w[kMaxActive];    // expected moves per walk
  unsigned long long moves;       // total moves of finished walks
  int live_workers;               // worker warps of the running launch
  int err;                        // first failed self-check (kernel-wide)
  unsigned long long bad[4];      // what that check saw
};

// Everything the device keeps per request slot: the host writes it into mapped
// memory at submit, the dispatcher copies it into the device table at admission.
struct SlotRec {
  WalkSpec spec;                  // the request
  unsigned long long finished;    // completion word: walks finished, error bits (zero at submit)
  uint32_t cw;                    // walks per chunk
  uint32_t exp_moves;             // expected moves per walk (the dispatcher's work estimate)
  uint32_t check_n;               // device sources the dispatcher range-checks at admission (0: none)
  uint32_t pad;
  unsigned long long t_admit;     // device clock (ns): the dispatcher took the request in
  unsigned long long t_first;     // a worker loaded its descriptor (first walks start)
  unsigned long long t_done;      // its last walk finished
};
// The dispatcher copies a record as 16-byte words, one per lane, and reads
// its own fields from the words it holds.
constexpr int kRecWords = (int)(sizeof(SlotRec) / 16);
static_assert(sizeof(SlotRec) % 16 == 0 && kRecWords <= 32, "slot record: whole 16-byte words, one per lane");
static_assert(offsetof(SlotRec, spec) + offsetof(WalkSpec, sources) == 5 * 16, "sources: word 5, x-y");
static_assert(offsetof(SlotRec, spec) + offsetof(WalkSpec, nwalks) == 6 * 16 + 8, "nwalks: word 6, z-w");
static_assert(offsetof(SlotRec, cw) == 8 * 16 + 8 && offsetof(SlotRec, exp_moves) == 8 * 16 + 12, "cw, exp_moves: word 8, z, w");
static_assert(offsetof(SlotRec, check_n) == 9 * 16 && offsetof(SlotRec, t_admit) == 9 * 16 + 8, "check_n, t_admit: word 9");

struct ServeHost {        // host-mapped pinned memory
  unsigned int stop;              // the host asks the kernel to end
  unsigned int pad;
  unsigned long long published;   // requests 0..published-1 are visible (host stores; see ServeState::published)
};

struct ServeDev {
  ServeState* state;
  Chunk* queue;                     // [kQueueCap]
  SlotRec* slots;                   // [R]
  const SlotRec* stage;             // [R] host-mapped: the records as the host wrote them
  volatile ServeHost* host;         // device pointer to host-mapped control
  volatile unsigned long long* done;// [R] host-mapped: (k + 1) << 8 | -status once request k finished
  int R;
  step::Coop coop;                  // rows this long go to the whole warp
  long long idle_ns;
  int32_t nv;                       // vertices of the graph (the dispatcher's source check)
  unsigned long long depth;         // queued chunks the dispatcher keeps ahead of the workers
};

// Polling uses relaxed loads: an acquire invalidates the SM's L1 cache, and
// warps that poll often would take the L1 hits of the warps that walk (the
// second half of an alias record, for one).  A poll that finds work takes
// the acquire as a fence before reading what it found.
__device__ __forceinline__ unsigned long long ld_relaxed_gpu(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void fence_acquire_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void fence_acquire_sys() { asm volatile("fence.acq_rel.sys;" ::: "memory"); }

// 16 bytes of host-mapped memory, read again on every call.
__device__ __forceinline__ uint4 ld_volatile_v4(const void* p) {
  uint4 v;
  asm volatile("ld.volatile.global.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (long long)t;
}

// Active-request set of the dispatcher, kept in shared memory during a launch
// and saved to the persistent state when the launch ends.
struct ActiveSet {
  unsigned long long k[kMaxActive];
  unsigned long long pos[kMaxActive];
  unsigned long long n[kMaxActive];
  unsigned long long cw[kMaxActive];
  unsigned long long w[kMaxActive];
};

// A worker warp's queue bookkeeping, kept in shared memory between refills so
// that none of it is live in registers while the lanes step their walks.
struct WarpState {
  unsigned long long ticket;      // lane 0: queue ticket held (has_ticket)
  unsigned long long pk;          // popped chunk not yet placed (pend): request
  unsigned long long fin[2];      // walks of key[e] finished here and not yet added to the request's count
  long long idle_since;           // when the warp ran out of walks (-1: it has some)
  uint32_t wlo, whi;              // unassigned walks of key[cur]
  uint32_t pb, pe;                // popped chunk not yet placed: walk range
  int cur;                        // slot receiving new walks
  int pend;
  int has_ticket;
  int empty_polls;                // empty polls in a row while some lanes walk
  int pad[2];
};

// Dispatcher: admits published requests into an active set and cuts them into
// chunks, shortest remaining work first (walks not yet queued times expected
// moves per walk), keeping at most sv.depth chunks queued: a request that
// arrives behind a large one waits for a bounded number of chunks, not for
// the large request, and of two large requests the one nearer completion
// finishes first instead of both finishing late.  It alone decides when the launch ends: after
// idle_timeout with nothing to hand out, or on the host's stop, it raises
// exit_now for the workers.  One warp; lane 0 works.
__device__ void dispatcher(const ServeDev& sv, ActiveSet* act) {
  const int lane = threadIdx.x & 31;
  ServeState* st = sv.state;
  int n_act = 0, rr = 0;
  if (lane == 0) {
    n_act = st->n_act;
    rr = st->rr;
    for (int i = 0; i < n_act; ++i) {
      act->k[i] = st->act_k[i];
      act->pos[i] = st->act_pos[i];
      act->n[i] = st->act_n[i];
      act->cw[i] = st->act_cw[i];
      act->w[i] = st->act_w[i];
    }
  }
  long long idle_since = now_ns();
  unsigned long long disp_next = st->disp_next;
  unsigned long long tail = st->q_tail;
  for (;;) {
    int go = 1;
    unsigned long long P = 0;
    int fresh = 0;
    if (lane == 0) {
      // the larger of the two counts; the device count is raised to the host's
      // (atomically: a copy-engine store may land at the same time) before any
      // of its requests' chunks are queued, so workers may check against it
      P = ld_relaxed_gpu(&st->published);
      const unsigned long long H = sv.host->published;
      if (H > P) {
        atomicMax(&st->published, H);
        P = H;
      }
      fresh = P > disp_next ? 1 : 0;
    }
    // every lane that reads the new requests' records (host memory) does so
    // after their count
    if (__shfl_sync(0xffffffffu, fresh, 0)) fence_acquire_sys();
    // Admission, one request at a time.  A small request with device sources
    // has its sources range-checked here by the whole warp; one out of range
    // completes the request with the invalid-argument status, and no walk runs.
    for (;;) {
      int adm = 0, slot = 0;
      if (lane == 0 && n_act < kMaxActive && disp_next < P) {
        adm = 1;
        slot = (int)(disp_next % (unsigned long long)sv.R);
      }
      if (!__shfl_sync(0xffffffffu, adm, 0)) break;
      slot = __shfl_sync(0xffffffffu, slot, 0);
      // The request's record: from the host's staging into the device table,
      // one 16-byte word per lane, stamped with the admission time.
      uint4 w = make_uint4(0u, 0u, 0u, 0u);
      if (lane < kRecWords) {
        w = ld_volatile_v4(reinterpret_cast<const uint4*>(sv.stage + slot) + lane);
        if (lane == 9) {
          const unsigned long long t = (unsigned long long)now_ns();
          w.z = (uint32_t)t;
          w.w = (uint32_t)(t >> 32);
        }
        __stcg(reinterpret_cast<uint4*>(sv.slots + slot) + lane, w);
      }
      const unsigned long long src = ((unsigned long long)__shfl_sync(0xffffffffu, w.y, 5) << 32) |
                                     __shfl_sync(0xffffffffu, w.x, 5);
      const unsigned long long n = ((unsigned long long)__shfl_sync(0xffffffffu, w.w, 6) << 32) |
                                   __shfl_sync(0xffffffffu, w.z, 6);
      const uint32_t rcw = __shfl_sync(0xffffffffu, w.z, 8);
      const uint32_t rexp = __shfl_sync(0xffffffffu, w.w, 8);
      const uint32_t chk = __shfl_sync(0xffffffffu, w.x, 9);
      uint32_t bad = 0;
      if (chk) {
        const int32_t* s_ptr = reinterpret_cast<const int32_t*>(__shfl_sync(0xffffffffu, src, 0));
        for (uint32_t i = (uint32_t)lane; i < chk; i += 32) bad |= (uint32_t)__ldcg(s_ptr + i) >= (uint32_t)sv.nv;
        bad = __any_sync(0xffffffffu, bad != 0u) ? 1u : 0u;
      }
      if (lane == 0) {
        if (bad) {
          sv.slots[slot].t_first = sv.slots[slot].t_done = (unsigned long long)now_ns();
          __threadfence_system();
          sv.done[slot] = ((disp_next + 1) << 8) | (unsigned long long)(-kErrInvalid);
        } else if (n > 0) {
          act->k[n_act] = disp_next;
          act->pos[n_act] = 0;
          act->n[n_act] = n;
          act->cw[n_act] = rcw;
          act->w[n_act] = rexp;
          ++n_act;
        }
        ++disp_next;
      }
    }
    // Chunks go out in bursts of up to 128 consecutive chunks of one request,
    // up to four per lane.
    const unsigned long long consumed = lane == 0 ? ld_acquire_gpu(&st->q_consumed) : 0ull;
    int pushed = 0;
    for (;;) {
      int burst = 0;
      unsigned long long bk = 0, bpos = 0, bn = 0, bcw = 0;
      if (lane == 0 && n_act > 0 && tail - consumed < sv.depth && pushed < 4096) {
        // shortest remaining work first: walks not yet queued x expected moves
        rr = 0;
        unsigned long long best = ~0ull;
        for (int i = 0; i < n_act; ++i) {
          const unsigned long long work = (act->n[i] - act->pos[i]) * act->w[i];
          if (work < best) {
            best = work;
            rr = i;
          }
        }
        bk = act->k[rr];
        bpos = act->pos[rr];
        bn = act->n[rr];
        bcw = act->cw[rr];
        const unsigned long long left = (bn - bpos + bcw - 1) / bcw;
        const unsigned long long room = sv.depth - (tail - consumed);
        burst = (int)(left < 128 ? left : 128);
        if ((unsigned long long)burst > room) burst = (int)room;
      }
      burst = __shfl_sync(0xffffffffu, burst, 0);
      if (burst == 0) break;
      bk = __shfl_sync(0xffffffffu, bk, 0);
      bpos = __shfl_sync(0xffffffffu, bpos, 0);
      bn = __shfl_sync(0xffffffffu, bn, 0);
      bcw = __shfl_sync(0xffffffffu, bcw, 0);
      const unsigned long long t0 = __shfl_sync(0xffffffffu, tail, 0);
      for (int i = lane; i < burst; i += 32) {  // up to four entries per lane
        const unsigned long long b = bpos + (unsigned long long)i * bcw;
        const unsigned long long e = b + bcw < bn ? b + bcw : bn;
        Chunk* c = &sv.queue[(t0 + i) % kQueueCap];
        __stcg(&c->k, bk);
        __stcg(reinterpret_cast<uint2*>(&c->begin), make_uint2((uint32_t)b, (uint32_t)e));
        __stcg(&c->seq, t0 + i);
      }
      if (lane == 0) {
        tail = t0 + burst;
        pushed += burst;
        const unsigned long long npos = bpos + (unsigned long long)burst * bcw;
        if (npos >= bn) {  // fully queued: leaves the active set
          --n_act;
          act->k[rr] = act->k[n_act];
          act->pos[rr] = act->pos[n_act];
          act->n[rr] = act->n[n_act];
          act->cw[rr] = act->cw[n_act];
          act->w[rr] = act->w[n_act];
        } else {
          act->pos[rr] = npos;
        }
      }
    }
    pushed = __shfl_sync(0xffffffffu, pushed, 0);
    if (pushed) {
      __threadfence();  // every lane's chunk entries before the tail
      __syncwarp();
    }
    if (lane == 0) {
      if (pushed) {
        st_release_gpu(&st->q_tail, tail);
        idle_since = now_ns();
      } else {
        const long long t = now_ns();
        const bool nothing_left = n_act == 0 && disp_next >= P;
        if (sv.host->stop) go = 0;
        else if (t - idle_since > sv.idle_ns && nothing_left && ld_acquire_gpu(&st->q_consumed) == tail) go = 0;
        else __nanosleep(1000);
      }
      if (!go) {
        // save the dispatcher's state for the next launch, then end this one
        st->disp_next = disp_next;
        st->n_act = n_act;
        st->rr = rr;
        for (int i = 0; i < n_act; ++i) {
          st->act_k[i] = act->k[i];
          st->act_pos[i] = act->pos[i];
          st->act_n[i] = act->n[i];
          st->act_cw[i] = act->cw[i];
          st->act_w[i] = act->w[i];
        }
        __threadfence();
        atomicExch(&st->exit_now, 1);
      }
    }
    go = __shfl_sync(0xffffffffu, go, 0);
    if (!go) return;
  }
}

// 4- or 8-byte load past L1 (the slot table is rewritten between requests),
// returned as T through a byte copy.
template <typename T>
__device__ __forceinline__ T ldcg_as(const T* p) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4 or 8 bytes");
  T r;
  if constexpr (sizeof(T) == 8) {
    unsigned long long v;
    asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    memcpy(&r, &v, 8);
  } else {
    unsigned int v;
    asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    memcpy(&r, &v, 4);
  }
  return r;
}

// The warp copies a slot's descriptor into shared memory: one 8-byte word per
// lane, loaded past L1 (the slot table is rewritten between requests), so the
// copy costs one round trip to L2.  Every lane calls it; the copy is complete
// for every lane when it returns.
__device__ __forceinline__ void load_spec(const WalkSpec* src, WalkSpec* dst) {
  static_assert(sizeof(WalkSpec) % 8 == 0 && sizeof(WalkSpec) / 8 <= 32, "one 8-byte word per lane");
  const int lane = threadIdx.x & 31;
  if (lane < (int)(sizeof(WalkSpec) / 8)) {
    const unsigned long long v = __ldcg(reinterpret_cast<const unsigned long long*>(src) + lane);
    const unsigned sh = (unsigned)__cvta_generic_to_shared(reinterpret_cast<unsigned long long*>(dst) + lane);
    asm volatile("st.shared.u64 [%0], %1;" ::"r"(sh), "l"(v) : "memory");
  }
  __syncwarp();
}

// Usable descriptor for chunk [cb, ce) of request ck?  0 if so, else the
// number of the failed check.
__device__ __forceinline__ int spec_check(const WalkSpec& sp, unsigned long long ck, uint32_t cb, uint32_t ce,
                                          unsigned long long published) {
  if (ck >= published) return 1;
  if (!(cb < ce) || (int64_t)ce > sp.nwalks) return 2;
  if (sp.algo < 0 || sp.algo > N2V_W || sp.algo == MIXED || sp.wps < 1 || sp.max_len < 0 ||
      (sp.algo == METAPATH && sp.schema_len < 1) || (sp.algo == DW_OREJ && sp.T_stop == 0))
    return 3;
  const uintptr_t ptrs = reinterpret_cast<uintptr_t>(sp.sources) | reinterpret_cast<uintptr_t>(sp.out_paths) |
                         reinterpret_cast<uintptr_t>(sp.out_lengths);
  if (!sp.sources || !sp.out_paths || !sp.out_lengths || (ptrs & 3)) return 4;
  return 0;
}

__device__ __forceinline__ void record_bad(const ServeDev& sv, int bad, unsigned long long a, unsigned long long b,
                                           unsigned long long c, unsigned long long d) {
  if (atomicCAS(&sv.state->err, 0, bad) == 0) {
    sv.state->bad[0] = a;
    sv.state->bad[1] = b;
    sv.state->bad[2] = c;
    sv.state->bad[3] = d;
  }
}

// Status of a completed request from the error bits of its completion word
// (a request that met several kinds of error reports the internal one).
__device__ __forceinline__ unsigned long long status_byte(unsigned long long word) {
  if ((word >> kErrBitInternal) & 1ull) return (unsigned long long)(-kErrInternal);
  if ((word >> kErrBitRejectCap) & 1ull) return (unsigned long long)(-kErrRejectCap);
  return 0ull;
}

// Adds a warp's finished walks of slot e to the request's count and, when
// they were the request's last, publishes the request's status and done flag
// in one host-mapped word.  Every lane calls it: each lane's fence orders the
// outputs of its walks (all of them, this iteration's and earlier ones)
// before the count.
__device__ __forceinline__ void flush_finished(const ServeDev& sv, int e, const WalkSpec* spec,
                                               const unsigned long long* key, WarpState* wsp) {
  __threadfence();
  __syncwarp();
  if ((threadIdx.x & 31) == 0) {
    const unsigned long long cnt = wsp->fin[e];
    wsp->fin[e] = 0;
    const unsigned long long k = key[e];
    const int slot = (int)(k % (unsigned long long)sv.R);
    const unsigned long long old = atomicAdd(&sv.slots[slot].finished, cnt);
    if ((old & kCountMask) + cnt == (unsigned long long)spec[e].nwalks) {
      sv.slots[slot].t_done = (unsigned long long)now_ns();
      __threadfence_system();
      sv.done[slot] = ((k + 1) << 8) | status_byte(old);
    }
  }
  __syncwarp();
}

// Worker warps hold up to two requests in two descriptor slots: the current
// slot, which new walks come from, and the other, whose walks may still be
// running.  Idle lanes therefore start walks of a new request at once; a chunk
// of a third request waits until the other slot has drained.  A slot takes a
// new request only when none of its lanes is running and its finished walks
// have been counted.
//
// The step itself is the batch kernels' (the descriptor comes from shared
// memory instead of a kernel argument).  Finished walks are counted per warp
// and slot, and added to the request's count only when the warp holds no more
// walks of that request: one atomic per warp and request instead of one per
// finishing iteration, which for a large request would all land on the same
// address.
// COOP compiles in the warp-cooperative MetaPath scan and Node2Vec search
// (needed only when a graph without the label index or neighbour hash is
// tuned to use them); without it the kernel fits four blocks per SM.
template <bool COOP>
__global__ void __launch_bounds__(kServeThreads, COOP ? 3 : 4) serve_kernel(DevGraph g, ServeDev sv) {
  // Static shared memory (the block size is fixed): the compiler addresses it
  // directly, with no generic pointers held in registers.
  __shared__ WalkSpec s_spec[kServeWarps][2];          // the warp's two descriptor slots
  __shared__ unsigned long long s_key[kServeWarps][2];  // their request numbers
  __shared__ __align__(16) int32_t s_stage[kServeThreads * 8];
  __shared__ ActiveSet s_act;                            // the dispatcher's (block 0)
  __shared__ __align__(16) WarpState s_ws[kServeWarps];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  WalkSpec* spec = s_spec[wid];
  unsigned long long* key = s_key[wid];
  int32_t* stage_mem = s_stage;
  ActiveSet* act = &s_act;
  WarpState* wsp = &s_ws[wid];

  if (blockIdx.x == 0 && wid == 0) {
    dispatcher(sv, act);
    return;
  }
  if (lane < 2) key[lane] = ~0ull;
  if (lane == 0) {
    atomicAdd(&sv.state->live_workers, 1);
    WarpState w0;
    w0.ticket = 0;
    w0.pk = 0;
    w0.fin[0] = w0.fin[1] = 0;
    w0.idle_since = -1;
    w0.wlo = w0.whi = w0.pb = w0.pe = 0;
    w0.cur = 0;
    w0.pend = 0;
    w0.has_ticket = 0;
    w0.empty_polls = 0;
    w0.pad[0] = w0.pad[1] = 0;
    *wsp = w0;
  }
  __syncwarp();

  const unsigned lt_mask = (1u << lane) - 1u;
  step::Stage st;
  st.buf = stage_mem + threadIdx.x * 8;
  st.gpos = 0;
  st.lo = 0;
  step::Walker W;
  step::walker_init(W, 0u, 0);
  bool active = false;
  uint32_t walk = 0;                  // this lane's walk within its request (walk ids are 32-bit)
  int ent = 0;                        // this lane's slot
  unsigned long long moves_acc = 0;
  unsigned act_mask = 0;              // lanes with a walk (warp-uniform)
  // After an empty poll of the queue while some lanes still walk, the warp
  // skips its next polls for a few refills (warp-uniform): a poll is a round
  // trip to L2 that would otherwise precede every step of the warp's
  // remaining walks.
  int poll_wait = 0;

  for (;;) {
    if (act_mask != 0xffffffffu) {
    unsigned idle = ~act_mask;
    int cur = wsp->cur;
    uint32_t wlo = wsp->wlo, whi = wsp->whi;
    if (wlo < whi) {
      // Fast path: idle lanes take walks left in the current chunk.
      const int take = (int)min((uint32_t)__popc(idle), whi - wlo);
      const int rank = __popc(idle & lt_mask);
      if (((idle >> lane) & 1u) && rank < take) {
        const WalkSpec& sp = spec[cur];
        ent = cur;
        walk = wlo + (uint32_t)rank;
        const int32_t src = __ldcg(sp.sources + walk / sp.wps);
        step::walker_init(W, sp.walk_offset + walk, src);
        if (!sp.endpoints) {
          st.gpos = (int64_t)walk * ((int64_t)sp.max_len + 1);
          st.lo = (int)(st.gpos & 7);
          step::stage_put(st, sp.out_paths, src, (reinterpret_cast<uintptr_t>(sp.out_paths) & 31) == 0);
        }
        active = true;
      }
      wlo += (uint32_t)take;
      idle = __ballot_sync(0xffffffffu, !active);
      act_mask = ~idle;
      __syncwarp();
      if (lane == 0) wsp->wlo = wlo;
      __syncwarp();
    }
    // A partly busy warp that is waiting out its poll backoff only counts down.
    const bool skip_poll = idle != 0u && idle != 0xffffffffu && poll_wait > 0 && wsp->pend == 0;
    if (skip_poll) --poll_wait;
    if (idle != 0u && !skip_poll) {
    // the rest of the warp's bookkeeping, loaded for this refill and stored back below
    bool pend = wsp->pend != 0;
    bool has_ticket = wsp->has_ticket != 0;   // lane 0's
    unsigned long long ticket = wsp->ticket;
    unsigned long long pk = wsp->pk;
    uint32_t pb = wsp->pb, pe = wsp->pe;
    poll_wait = 0;
    int empty_polls = wsp->empty_polls;
    const unsigned was_active = act_mask;
    while (idle != 0u) {
      if (wlo >= whi) {
        if (!pend) {
          unsigned long long ck = 0;
          uint32_t cb = 0, ce = 0;
          int got = 0;
          if (lane == 0) {
            // A ticket (fetch-and-add on the queue head, which always succeeds)
            // names the next entry this warp reads once the tail passes it.
            // A warp with lanes still walking takes one only for an entry that
            // is already there and unclaimed: a ticket binds its entry to this
            // warp, and a warp that polls now and then would hold the entry up
            // while idle warps wait.
            ServeState* s = sv.state;
            const unsigned long long tl = ld_relaxed_gpu(&s->q_tail);
            if (!has_ticket && (idle == 0xffffffffu || *(volatile unsigned long long*)&s->q_head < tl)) {
              ticket = atomicAdd(&s->q_head, 1ull);
              has_ticket = true;
            }
            if (has_ticket && ticket < tl) {
              fence_acquire_gpu();  // the entry after the tail that covers it
              const Chunk* c = &sv.queue[ticket % kQueueCap];
              ck = ldcg_as(&c->k);
              cb = ldcg_as(&c->begin);
              ce = ldcg_as(&c->end);
              const unsigned long long seq = ldcg_as(&c->seq);
              __threadfence();
              atomicAdd(&s->q_consumed, 1ull);
              has_ticket = false;
              got = 1;
              if (seq != ticket) {  // overwritten before it was read: record, skip
                record_bad(sv, 7, ticket, seq, ck, 0);
                got = 0;
              }
            }
          }
          got = __shfl_sync(0xffffffffu, got, 0);
          if (!got) {
            // Lanes still walk and no entry is bound to this warp: back off
            // before the next poll.  A warp holding a ticket polls every refill.
            if (idle != 0xffffffffu && !__shfl_sync(0xffffffffu, has_ticket ? 1 : 0, 0)) {
              poll_wait = min(kPollSkip << min(empty_polls, 3), kPollSkipMax);
              ++empty_polls;
            }
            break;
          }
          empty_polls = 0;
          ck = __shfl_sync(0xffffffffu, ck, 0);
          cb = __shfl_sync(0xffffffffu, cb, 0);
          ce = __shfl_sync(0xffffffffu, ce, 0);
          if (ck == key[cur]) {  // more walks of the current request
            wlo = cb;
            whi = ce;
            continue;
          }
          pend = true;
          pk = ck;
          pb = cb;
          pe = ce;
        }
        const int other = 1 - cur;
        if (key[other] == pk) {  // the other slot already holds the request
          cur = other;
          wlo = pb;
          whi = pe;
          pend = false;
          continue;
        }
        // a slot takes a new request only once none of its lanes is running
        const bool other_busy = (act_mask & __ballot_sync(0xffffffffu, ent == other)) != 0u;
        const bool cur_busy = (act_mask & __ballot_sync(0xffffffffu, ent == cur)) != 0u;
        const int tgt = !other_busy ? other : (!cur_busy ? cur : -1);
        if (tgt < 0) break;
        if (wsp->fin[tgt] != 0) flush_finished(sv, tgt, spec, key, wsp);  // counted before it changes hands
        int bad = 0;
        // the published count for the self-check, in flight with the descriptor
        const unsigned long long pub_now = lane == 0 ? ld_relaxed_gpu(&sv.state->published) : 0ull;
        load_spec(&sv.slots[(int)(pk % (unsigned long long)sv.R)].spec, &spec[tgt]);
        if (lane == 0) {
          atomicCAS(&sv.slots[(int)(pk % (unsigned long long)sv.R)].t_first, 0ull, (unsigned long long)now_ns());
          bad = spec_check(spec[tgt], pk, pb, pe, pub_now);
          if (bad) record_bad(sv, bad, pk, ((unsigned long long)pb << 32) | pe, (unsigned long long)spec[tgt].nwalks,
                              reinterpret_cast<uintptr_t>(spec[tgt].out_paths));
          key[tgt] = bad ? ~0ull : pk;
        }
        bad = __shfl_sync(0xffffffffu, bad, 0);
        __syncwarp();
        pend = false;
        if (bad) continue;
        cur = tgt;
        wlo = pb;
        whi = pe;
        continue;
      }
      const int take = (int)min((uint32_t)__popc(idle), whi - wlo);
      const int rank = __popc(idle & lt_mask);
      if (((idle >> lane) & 1u) && rank < take) {
        const WalkSpec& sp = spec[cur];
        ent = cur;
        walk = wlo + (uint32_t)rank;
        const int32_t src = __ldcg(sp.sources + walk / sp.wps);
        step::walker_init(W, sp.walk_offset + walk, src);
        if (!sp.endpoints) {
          st.gpos = (int64_t)walk * ((int64_t)sp.max_len + 1);
          st.lo = (int)(st.gpos & 7);
          step::stage_put(st, sp.out_paths, src, (reinterpret_cast<uintptr_t>(sp.out_paths) & 31) == 0);
        }
        active = true;
      }
      wlo += (uint32_t)take;
      idle = __ballot_sync(0xffffffffu, !active);
      act_mask = ~idle;
    }
    __syncwarp();
    if (lane == 0) {
      if (act_mask != was_active) wsp->idle_since = -1;  // walks started: the warp is not idle
      wsp->empty_polls = empty_polls;
      wsp->cur = cur;
      wsp->wlo = wlo;
      wsp->whi = whi;
      wsp->pend = pend ? 1 : 0;
      wsp->has_ticket = has_ticket ? 1 : 0;
      wsp->ticket = ticket;
      wsp->pk = pk;
      wsp->pb = pb;
      wsp->pe = pe;
    }
    __syncwarp();
    }
    }

    if (act_mask == 0u) {
      // Idle: lane 0 waits until the queue holds the entry of this warp's
      // ticket (then the warp refills), the dispatcher ends the launch and no
      // entry waits for this warp, or an absolute bound of 1000 idle timeouts
      // passes should the dispatcher never end it.  The other lanes wait at the
      // shuffle: an idle warp takes few issue slots from the warps that walk.
      int go = 1;
      if (lane == 0) {
        if (wsp->idle_since < 0) wsp->idle_since = now_ns();
        const long long idle_since = wsp->idle_since;
        const bool has_ticket = wsp->has_ticket != 0;
        const unsigned long long ticket = wsp->ticket;
        for (;;) {
          const unsigned long long tl = ld_relaxed_gpu(&sv.state->q_tail);
          if (!has_ticket || ticket < tl) break;  // refill: take a ticket, or read the entry
          if (*(volatile int*)&sv.state->exit_now) {
            go = 0;
            break;
          }
          if (now_ns() - idle_since > 1000 * sv.idle_ns) {
            go = 0;
            break;
          }
          // warps whose ticket is near the tail poll often, the rest back off
          const unsigned long long dist = ticket - tl;
          __nanosleep(dist < 64 ? 256u : dist < 512 ? 2000u : 8000u);
        }
      }
      if (!__shfl_sync(0xffffffffu, go, 0)) break;
      continue;
    }

    // ---- one unit of work per active lane (the batch kernels' step)
    bool finishing = false;
    const WalkSpec& sp = spec[ent];
    int r = step::kIdle;
    int32_t next = -1;
    step::Pend pend_work;
    pend_work.kind = 0;
    pend_work.res = 0;
    if constexpr (COOP) {
      if (active) r = step::step_begin_dispatch<MIXED>(g, sp, W, next, pend_work, sv.coop);
      if (__any_sync(0xffffffffu, r == step::kDefer)) {
        step::warp_resolve(g, r, W, pend_work);
        if (r == step::kDefer) r = step::step_finish(g, sp, W, pend_work, next);
      }
    } else {
      // The warp's walking lanes share one algorithm when they all run walks
      // of one slot, or both slots hold requests of the same algorithm; the
      // warp then runs that algorithm's step (the batch kernel's), else each
      // lane's request picks it.
      const unsigned in1 = __ballot_sync(0xffffffffu, ent == 1);
      const int a0 = spec[0].algo, a1 = spec[1].algo;
      const int walgo = (act_mask & in1) == 0u ? a0 : (act_mask & ~in1) == 0u ? a1 : a0 == a1 ? a0 : -1;
      const step::Coop none{0x7fffffff, 0x7fffffff};
      if (active) {
        switch (walgo) {
          case DEEPWALK: r = step::step_begin<DEEPWALK>(g, sp, W, next, pend_work, none); break;
          case DEEPWALK_WEIGHTED: r = step::step_begin<DEEPWALK_WEIGHTED>(g, sp, W, next, pend_work, none); break;
          case PPR: r = step::step_begin<PPR>(g, sp, W, next, pend_work, none); break;
          case NODE2VEC: r = step::step_begin<NODE2VEC>(g, sp, W, next, pend_work, none); break;
          default: r = step::step_begin_dispatch<MIXED>(g, sp, W, next, pend_work, none); break;
        }
      }
    }
    if (active) {
      const bool aligned = (reinterpret_cast<uintptr_t>(sp.out_paths) & 31) == 0;
      if (r == step::kMoved) {
        step::advance(W, next);
        if (!sp.endpoints) step::stage_put(st, sp.out_paths, next, aligned);
      } else if (r == step::kRetry) {
        W.att += 1;
      } else {
        if (r == step::kFail || r == step::kBroken) {
          const int slot = (int)(key[ent] % (unsigned long long)sv.R);
          atomicOr(&sv.slots[slot].finished, 1ull << (r == step::kFail ? kErrBitRejectCap : kErrBitInternal));
        }
        if (sp.endpoints) __stcs(sp.out_paths + walk, W.cur);
        else step::stage_finish(st, sp.out_paths, aligned);
        __stcs(sp.out_lengths + walk, W.s + 1);
        moves_acc += (unsigned long long)W.s;
        finishing = true;
        active = false;
      }
    }
    const unsigned fin = __ballot_sync(0xffffffffu, finishing);
    if (fin) {
      // Count the finished walks per slot; hand a slot's count to its request
      // once the warp holds no more of its walks (none running, none left in
      // the current chunk).
      act_mask &= ~fin;
      const unsigned in1 = __ballot_sync(0xffffffffu, ent == 1);
      const int cur = wsp->cur;
      const bool left = wsp->wlo < wsp->whi;
      for (int e = 0; e < 2; ++e) {
        const unsigned fe = fin & (e ? in1 : ~in1);
        if (!fe) continue;
        if (lane == 0) wsp->fin[e] += (unsigned long long)__popc(fe);
        __syncwarp();
        const unsigned re = act_mask & (e ? in1 : ~in1);
        if (re == 0u && !(cur == e && left)) flush_finished(sv, e, spec, key, wsp);
      }
    }
  }
  // Nothing is left to count at exit (a warp leaves only when idle, after its
  // last walks' counts were handed over); flushing again is harmless.
  for (int e = 0; e < 2; ++e)
    if (wsp->fin[e] != 0) flush_finished(sv, e, spec, key, wsp);
  const unsigned long long mv = step::warp_sum(moves_acc);
  if (lane == 0) {
    if (mv) atomicAdd(&sv.state->moves, mv);
    __threadfence();
    atomicSub(&sv.state->live_workers, 1);
  }
}

}  // namespace

// -------------------------------------------------------------------- host

struct trw_server {
  trw_graph* g = nullptr;
  trw_serve_config cfg{};
  int R = 0;
  cudaStream_t stream = nullptr;       // the resident kernel
  cudaStream_t copy_stream = nullptr;  // descriptor uploads
  cudaEvent_t ev_after = nullptr;      // trw_serve_order_after: the caller's stream, recorded
  bool after_pending = false;          // ev_after recorded and not yet known to be complete
  bool cs_gated = false;               // the copy stream waits for an earlier ordering event: the next
                                       // request is published behind it
  cudaEvent_t ev_pub = nullptr;        // after the last copy-engine publication
  bool ce_pub_pending = false;         // ev_pub recorded and not yet known to be complete
  ServeState* state = nullptr;
  Chunk* queue = nullptr;
  SlotRec* slots = nullptr;
  int32_t* src_pool = nullptr;         // device copies of request sources (ring allocator)
  int64_t src_cap = 0;
  ServeHost* host = nullptr;           // mapped
  unsigned long long* done = nullptr;  // mapped [R]
  ServeHost* host_dev = nullptr;
  unsigned long long* done_dev = nullptr;
  SlotRec* slot_stage = nullptr;       // mapped [R]: the records the dispatcher copies in at admission
  SlotRec* slot_stage_dev = nullptr;
  unsigned long long* pub_stage = nullptr;  // pinned [R]: the count that publishes request k is pub_stage[k % R]
  int32_t* check_buf = nullptr;        // pinned: host copy of device sources for the range check
  int64_t check_cap = 0;
  // host bookkeeping, ring order
  unsigned long long next_k = 0;       // next request number
  unsigned long long oldest = 0;       // oldest request not yet collected
  std::vector<int64_t> req_walks, req_bytes, req_src_pos, req_src_n;
  std::vector<char> collected;
  int64_t inflight_walks = 0, inflight_bytes = 0;
  int64_t src_head = 0;                // ring allocator: next free position
  int block_threads = 256;
  int grid_blocks = 0;                 // the variant without warp cooperation
  int grid_blocks_coop = 0;            // the variant with it
  size_t smem = 0;
  uint64_t polls = 0;
  std::mutex mu;
};

extern "C" void trw_serve_config_default(trw_serve_config* c) {
  if (!c) return;
  c->max_inflight_walks = 1ll << 26;
  c->max_inflight_bytes = 16ll << 30;
  c->max_requests = 1024;
  c->idle_timeout_us = 2000;
}

static void server_release(trw_server* s) {
  if (!s) return;
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  if (s->ev_after) cudaEventDestroy(s->ev_after);
  if (s->ev_pub) cudaEventDestroy(s->ev_pub);
  cudaFree(s->state);
  cudaFree(s->queue);
  cudaFree(s->slots);
  cudaFree(s->src_pool);
  if (s->host) cudaFreeHost(s->host);
  if (s->done) cudaFreeHost(s->done);
  if (s->slot_stage) cudaFreeHost(s->slot_stage);
  if (s->pub_stage) cudaFreeHost(s->pub_stage);
  if (s->check_buf) cudaFreeHost(s->check_buf);
  delete s;
}

#define SV_TRY(call, what)                 \
  do {                                     \
    cudaError_t e_ = (call);               \
    if (e_ != cudaSuccess) {               \
      server_release(s);                   \
      return trw_cuda_fail(e_, what);      \
    }                                      \
  } while (0)

extern "C" trw_status trw_serve_create(trw_graph* g, const trw_serve_config* cfg_in, trw_server** out) {
  if (!g || !out) return trw_fail(TRW_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (trw_status dc = trw_check_device(g); dc != TRW_OK) return dc;
  trw_serve_config cfg;
  if (cfg_in) cfg = *cfg_in;
  else trw_serve_config_default(&cfg);
  if (cfg.max_requests < 1 || cfg.max_requests > 4096) return trw_fail(TRW_ERR_INVALID, "max_requests in [1, 4096]");
  if (cfg.max_inflight_walks < 1 || cfg.max_inflight_walks > (1ll << 31))
    return trw_fail(TRW_ERR_INVALID, "max_inflight_walks in [1, 2^31]");
  if (cfg.max_inflight_bytes < 1) return trw_fail(TRW_ERR_INVALID, "max_inflight_bytes >= 1");
  if (cfg.idle_timeout_us < 1 || cfg.idle_timeout_us > 10000000) return trw_fail(TRW_ERR_INVALID, "idle_timeout_us in [1, 1e7]");
  trw_server* s = new trw_server();
  s->g = g;
  s->cfg = cfg;
  s->R = cfg.max_requests;
  s->src_cap = cfg.max_inflight_walks;
  const int R = s->R;
  SV_TRY(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking), "stream");
  SV_TRY(cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking), "stream");
  SV_TRY(cudaEventCreateWithFlags(&s->ev_after, cudaEventDisableTiming), "event");
  SV_TRY(cudaEventCreateWithFlags(&s->ev_pub, cudaEventDisableTiming), "event");
  SV_TRY(trw_dev_malloc((void**)&s->state, sizeof(ServeState)), "serve state");
  SV_TRY(cudaMemset(s->state, 0, sizeof(ServeState)), "serve state");
  SV_TRY(trw_dev_malloc((void**)&s->queue, sizeof(Chunk) * kQueueCap), "chunk queue");
  SV_TRY(trw_dev_malloc((void**)&s->slots, sizeof(SlotRec) * R), "slot table");
  SV_TRY(cudaMemset(s->slots, 0, sizeof(SlotRec) * R), "slot table");
  SV_TRY(trw_dev_malloc((void**)&s->src_pool, sizeof(int32_t) * (size_t)s->src_cap), "source pool");
  SV_TRY(trw_host_alloc((void**)&s->host, sizeof(ServeHost), cudaHostAllocMapped), "mapped control");
  SV_TRY(trw_host_alloc((void**)&s->done, sizeof(unsigned long long) * R, cudaHostAllocMapped), "mapped flags");
  SV_TRY(trw_host_alloc((void**)&s->slot_stage, sizeof(SlotRec) * R, cudaHostAllocMapped), "mapped records");
  SV_TRY(trw_host_alloc((void**)&s->pub_stage, sizeof(unsigned long long) * R, cudaHostAllocDefault), "pinned staging");
  std::memset((void*)s->host, 0, sizeof(ServeHost));
  std::memset((void*)s->done, 0, sizeof(unsigned long long) * R);
  SV_TRY(cudaHostGetDevicePointer((void**)&s->host_dev, (void*)s->host, 0), "mapped pointer");
  SV_TRY(cudaHostGetDevicePointer((void**)&s->done_dev, (void*)s->done, 0), "mapped pointer");
  SV_TRY(cudaHostGetDevicePointer((void**)&s->slot_stage_dev, (void*)s->slot_stage, 0), "mapped pointer");
  s->req_walks.assign(R, 0);
  s->req_bytes.assign(R, 0);
  s->req_src_pos.assign(R, 0);
  s->req_src_n.assign(R, 0);
  s->collected.assign(R, 1);
  s->block_threads = kServeThreads;
  s->smem = 0;  // the kernel's shared memory is static
  int bps = 0, bps_coop = 0;
  SV_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, serve_kernel<false>, s->block_threads, s->smem),
         "occupancy");
  SV_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps_coop, serve_kernel<true>, s->block_threads, s->smem),
         "occupancy");
  if (bps < 1) bps = 1;
  if (bps_coop < 1) bps_coop = 1;
  s->grid_blocks = g->num_sms * bps;
  s->grid_blocks_coop = g->num_sms * bps_coop;
  *out = s;
  return TRW_OK;
}

static cudaError_t launch_if_idle(trw_server* s) {
  if (s->oldest == s->next_k) return cudaSuccess;  // nothing in flight
  cudaError_t q = cudaStreamQuery(s->stream);
  if (q == cudaErrorNotReady) return cudaSuccess;  // running
  if (q != cudaSuccess) return q;
  ServeDev sv;
  sv.state = s->state;
  sv.queue = s->queue;
  sv.slots = s->slots;
  sv.stage = s->slot_stage_dev;
  sv.host = s->host_dev;
  sv.done = s->done_dev;
  sv.R = s->R;
  sv.coop = step::Coop{s->g->tuning.coop_degree, s->g->tuning.search_degree};
  sv.idle_ns = (long long)s->cfg.idle_timeout_us * 1000;
  sv.nv = (int32_t)s->g->nv;
  {
    // enough queued chunks to cover the workers' claims between dispatcher rounds
    const unsigned long long workers = (unsigned long long)s->grid_blocks * (s->block_threads / 32);
    unsigned long long depth = workers / 4;
    if (depth < 64) depth = 64;
    if (depth > 4096) depth = 4096;
    sv.depth = depth;
  }
  cudaError_t e = cudaMemsetAsync(&s->state->exit_now, 0, sizeof(int), s->stream);
  // Tickets taken past the tail by the last launch are void: restart the
  // head at the tail (that launch ended with every pushed entry read).
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&s->state->q_head, &s->state->q_tail, sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                        s->stream);
  if (e != cudaSuccess) return e;
  // the cooperative variant only when the tuning asks for a warp path that no
  // prepared table replaces
  const trw_graph* g = s->g;
  const bool coop = (g->labels && !g->lerec && g->tuning.coop_degree < 0x7fffffff) ||
                    (!g->nh_slots && g->tuning.search_degree < 0x7fffffff);
  if (coop)
    serve_kernel<true><<<s->grid_blocks_coop, s->block_threads, s->smem, s->stream>>>(trw_dev_graph(g), sv);
  else
    serve_kernel<false><<<s->grid_blocks, s->block_threads, s->smem, s->stream>>>(trw_dev_graph(g), sv);
  return cudaGetLastError();
}

// Collect finished requests at the front of the ring (frees their slots and source ranges).
static void retire_front(trw_server* s) {
  while (s->oldest < s->next_k && s->collected[s->oldest % s->R]) ++s->oldest;
}

extern "C" trw_status trw_serve_order_after(trw_server* s, void* stream) {
  if (!s || !stream) return trw_fail(TRW_ERR_INVALID, "NULL server or stream");
  if (trw_status dc = trw_check_device(s->g); dc != TRW_OK) return dc;
  std::lock_guard<std::mutex> lk(s->mu);
  // A stream with nothing left to run orders nothing.  Otherwise the next
  // submit publishes through the copy stream, behind an event recorded here,
  // unless the event has completed by then.
  const cudaError_t q = cudaStreamQuery((cudaStream_t)stream);
  if (q == cudaSuccess) return TRW_OK;
  if (q != cudaErrorNotReady) return trw_cuda_fail(q, "serve order after");
  cudaError_t e = cudaSuccess;
  if (s->after_pending) {
    // an earlier call's event that no submit has consumed: the copy stream
    // takes it over before the event is recorded again
    e = cudaStreamWaitEvent(s->copy_stream, s->ev_after, 0);
    if (e != cudaSuccess) return trw_cuda_fail(e, "serve order after");
    s->cs_gated = true;
  }
  e = cudaEventRecord(s->ev_after, (cudaStream_t)stream);
  if (e != cudaSuccess) return trw_cuda_fail(e, "serve order after");
  s->after_pending = true;
  return TRW_OK;
}

extern "C" trw_status trw_serve_submit(trw_server* s, trw_algo algo, const trw_params* params, const int32_t* sources,
                                       int64_t n_sources, int32_t max_len, uint64_t seed, int32_t* out_paths,
                                       int32_t* out_lengths, uint64_t* req_id) {
  if (!s || !req_id) return trw_fail(TRW_ERR_INVALID, "NULL argument");
  if (trw_status dc = trw_check_device(s->g); dc != TRW_OK) return dc;
  WalkSpec sp;
  trw_status stt = trw_make_spec(s->g, algo, params, n_sources, max_len, seed, &sp);
  if (stt != TRW_OK) return stt;
  if (sp.nwalks > 0 && (!sources || !out_paths || !out_lengths)) return trw_fail(TRW_ERR_INVALID, "NULL buffer");
  if (sp.nwalks > 0 && (!trw_is_device_ptr(out_paths) || !trw_is_device_ptr(out_lengths)))
    return trw_fail(TRW_ERR_INVALID, "serve outputs must be device buffers");
  const bool src_dev = trw_is_device_ptr(sources);
  if (!src_dev && !trw_sources_in_range(sources, n_sources, s->g->nv))
    return trw_fail(TRW_ERR_INVALID, "a source vertex is outside [0, nv)");
  const int64_t out_bytes =
      (int64_t)sizeof(int32_t) * (sp.endpoints ? sp.nwalks : sp.nwalks * ((int64_t)max_len + 1)) + 4 * sp.nwalks;
  // Host sources are copied into the server's source pool; device sources
  // are read in place (they stay valid until the request is reported).
  const int64_t pool_n = src_dev ? 0 : n_sources;
  std::lock_guard<std::mutex> lk(s->mu);
  retire_front(s);
  if (s->next_k - s->oldest >= (unsigned long long)s->R) return trw_fail(TRW_ERR_BUSY, "all %d request slots in use", s->R);
  if (pool_n > s->src_cap || s->inflight_walks + sp.nwalks > s->cfg.max_inflight_walks)
    return trw_fail(TRW_ERR_BUSY, "walk admission limit %lld reached", (long long)s->cfg.max_inflight_walks);
  if (s->inflight_bytes + out_bytes > s->cfg.max_inflight_bytes)
    return trw_fail(TRW_ERR_BUSY, "output byte admission limit reached");
  // Ring allocation of the source copy, in request order: live ranges run
  // circularly from the oldest live request's range up to src_head.
  int64_t pos = -1;
  if (s->oldest == s->next_k) {
    s->src_head = 0;
    if (pool_n <= s->src_cap) pos = 0;
  } else {
    const int64_t lo_live = s->req_src_pos[s->oldest % s->R];
    if (lo_live < s->src_head) {  // free: [src_head, cap) and [0, lo_live)
      if (s->src_head + pool_n <= s->src_cap) pos = s->src_head;
      else if (pool_n <= lo_live) pos = 0;
    } else if (lo_live > s->src_head) {  // free: [src_head, lo_live)
      if (s->src_head + pool_n <= lo_live) pos = s->src_head;
    } else if (pool_n == 0) {
      pos = s->src_head;
    }
  }
  if (pos < 0) return trw_fail(TRW_ERR_BUSY, "source pool full");
  // Device sources of a small request are range-checked by the dispatcher
  // when it admits the request; larger ones here, through pinned memory.
  const bool dev_check = src_dev && n_sources > 0 && n_sources <= kDeviceCheckMax;
  if (src_dev && n_sources > 0 && !dev_check) {
    // device sources: one copy to pinned memory and a host range check
    // before anything is queued
    if (n_sources > s->check_cap) {
      if (s->check_buf) cudaFreeHost(s->check_buf);
      s->check_buf = nullptr;
      s->check_cap = 0;
      const cudaError_t ea = trw_host_alloc((void**)&s->check_buf, sizeof(int32_t) * (size_t)n_sources, cudaHostAllocDefault);
      if (ea != cudaSuccess) return trw_cuda_fail(ea, "serve source check buffer");
      s->check_cap = n_sources;
    }
    cudaError_t ec = cudaSuccess;
    if (s->after_pending) {  // the caller's writes of the sources first
      ec = cudaStreamWaitEvent(s->copy_stream, s->ev_after, 0);
      if (ec == cudaSuccess) s->after_pending = false;
    }
    if (ec == cudaSuccess)
      ec = cudaMemcpyAsync(s->check_buf, sources, sizeof(int32_t) * (size_t)n_sources, cudaMemcpyDeviceToHost,
                           s->copy_stream);
    if (ec == cudaSuccess) ec = cudaStreamSynchronize(s->copy_stream);
    if (ec != cudaSuccess) return trw_cuda_fail(ec, "serve source check");
    s->cs_gated = false;  // every wait on the copy stream has completed
    if (!trw_sources_in_range(s->check_buf, n_sources, s->g->nv))
      return trw_fail(TRW_ERR_INVALID, "a source vertex is outside [0, nv)");
  }
  const unsigned long long k = s->next_k;
  const int slot = (int)(k % (unsigned long long)s->R);
  sp.sources = src_dev ? sources : s->src_pool + pos;
  sp.out_paths = out_paths;
  sp.out_lengths = out_lengths;
  // Walks per chunk: one walk per lane (32) while the request fits in the
  // resident lanes, so its latency is its longest walk; a larger request
  // takes about 20 expected moves per lane per chunk.  (Chunks sized to two
  // per worker warp made large requests slower: the tail imbalance cost more
  // than the dispatcher's work saved.)
  double exp_moves = (double)max_len;
  if (algo == TRW_PPR && params && params->ppr_stop > 0) exp_moves = std::min(exp_moves, 1.0 / params->ppr_stop);
  if (exp_moves < 1) exp_moves = 1;
  const int64_t lanes = (int64_t)s->grid_blocks * s->block_threads;
  const uint32_t cw = sp.nwalks <= lanes ? 32u : (uint32_t)std::max(32.0, std::min(2048.0, 640.0 / exp_moves));
  SlotRec& rec = s->slot_stage[slot];
  rec.spec = sp;
  rec.finished = 0;
  rec.cw = cw;
  rec.exp_moves = (uint32_t)std::max(1.0, std::ceil(exp_moves));
  rec.check_n = dev_check ? (uint32_t)n_sources : 0u;
  rec.pad = 0;
  rec.t_admit = rec.t_first = rec.t_done = 0;
  // Publication waits for nothing.  The record stays in mapped host memory,
  // where the dispatcher copies it into the device table when it admits the
  // request; the request count goes either straight into mapped memory or,
  // while an ordering event or an earlier copy-engine publication is still
  // pending, or host sources must go up first, through the copy stream in
  // submission order.  The record is not rewritten before the request is
  // collected, long after its admission.
  cudaStream_t cs = s->copy_stream;
  s->done[slot] = 0;
  cudaError_t e = cudaSuccess;
  bool direct = pool_n == 0 && !s->cs_gated;
  if (direct && s->after_pending) {
    const cudaError_t q = cudaEventQuery(s->ev_after);
    if (q == cudaSuccess) s->after_pending = false;
    else if (q == cudaErrorNotReady) direct = false;
    else return trw_cuda_fail(q, "serve order after");
  }
  if (direct && s->ce_pub_pending) {
    const cudaError_t q = cudaEventQuery(s->ev_pub);
    if (q == cudaSuccess) s->ce_pub_pending = false;
    else if (q == cudaErrorNotReady) direct = false;
    else return trw_cuda_fail(q, "serve publication");
  }
  if (direct) {
    __atomic_store_n(&s->host->published, k + 1, __ATOMIC_RELEASE);  // after the record's stores
  } else {
    if (s->after_pending) {
      e = cudaStreamWaitEvent(cs, s->ev_after, 0);
      if (e == cudaSuccess) s->after_pending = false;
    }
    if (e == cudaSuccess && pool_n > 0)
      e = cudaMemcpyAsync(s->src_pool + pos, sources, sizeof(int32_t) * (size_t)pool_n, cudaMemcpyHostToDevice, cs);
    s->pub_stage[slot] = k + 1;
    std::atomic_thread_fence(std::memory_order_seq_cst);  // the record before the count
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&s->state->published, &s->pub_stage[slot], sizeof(unsigned long long), cudaMemcpyHostToDevice,
                          cs);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev_pub, cs);
    if (e == cudaSuccess) {
      s->ce_pub_pending = true;
      s->cs_gated = false;  // this publication follows every wait on the copy stream
    }
    if (e != cudaSuccess) return trw_cuda_fail(e, "serve submit upload");
  }
  s->req_walks[slot] = sp.nwalks;
  s->req_bytes[slot] = out_bytes;
  s->req_src_pos[slot] = pos;
  s->req_src_n[slot] = pool_n;
  s->collected[slot] = 0;
  s->inflight_walks += sp.nwalks;
  s->inflight_bytes += out_bytes;
  s->src_head = pos + pool_n;
  s->next_k = k + 1;
  if (sp.nwalks == 0) {
    s->done[slot] = (k + 1) << 8;  // nothing to run
  }
  std::atomic_thread_fence(std::memory_order_seq_cst);
  e = launch_if_idle(s);
  if (e != cudaSuccess) return trw_cuda_fail(e, "serve kernel launch");
  *req_id = k;
  return TRW_OK;
}

// A failed device self-check, reported as TRW_ERR_INTERNAL with what it saw.
static trw_status check_state(trw_server* s) {
  ServeState st;
  cudaError_t e = cudaMemcpyAsync(&st, s->state, sizeof(ServeState), cudaMemcpyDeviceToHost, s->copy_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
  if (e != cudaSuccess) return trw_cuda_fail(e, "serve state");
  if (st.err != 0)
    return trw_fail(TRW_ERR_INTERNAL, "serve self-check %d failed: request %llu range %llx nwalks %llu out %llx", st.err,
                    st.bad[0], st.bad[1], st.bad[2], st.bad[3]);
  return TRW_OK;
}

static trw_status poll_locked(trw_server* s, uint64_t k) {
  if (k >= s->next_k || k + (unsigned long long)s->R < s->next_k) return trw_fail(TRW_ERR_NOT_FOUND, "unknown request %llu", (unsigned long long)k);
  const int slot = (int)(k % (unsigned long long)s->R);
  if (s->collected[slot]) return trw_fail(TRW_ERR_NOT_FOUND, "request %llu already collected", (unsigned long long)k);
  const unsigned long long d = reinterpret_cast<volatile unsigned long long*>(s->done)[slot];
  if ((d >> 8) != k + 1) {
    cudaError_t e = launch_if_idle(s);
    if (e != cudaSuccess) return trw_cuda_fail(e, "serve kernel relaunch");
    if ((++s->polls & 63) == 0) {
      trw_status cs = check_state(s);
      if (cs != TRW_OK) return cs;
    }
    return TRW_PENDING;
  }
  std::atomic_thread_fence(std::memory_order_acquire);
  const int err = -(int)(d & 0xffu);
  s->collected[slot] = 1;
  s->inflight_walks -= s->req_walks[slot];
  s->inflight_bytes -= s->req_bytes[slot];
  retire_front(s);
  if (err == kErrRejectCap) return trw_fail(TRW_ERR_REJECT_CAP, "request %llu: a rejection step hit the cap", (unsigned long long)k);
  if (err == kErrInvalid) return trw_fail(TRW_ERR_INVALID, "request %llu: a source vertex is outside [0, nv)", (unsigned long long)k);
  if (err != 0) return trw_fail(TRW_ERR_INTERNAL, "request %llu: device status %d", (unsigned long long)k, err);
  return TRW_OK;
}

extern "C" trw_status trw_serve_poll(trw_server* s, uint64_t req_id) {
  if (!s) return trw_fail(TRW_ERR_INVALID, "NULL server");
  if (trw_status dc = trw_check_device(s->g); dc != TRW_OK) return dc;
  std::lock_guard<std::mutex> lk(s->mu);
  return poll_locked(s, req_id);
}

extern "C" trw_status trw_serve_reap(trw_server* s, uint64_t* ids, int32_t* statuses, int32_t max, int32_t* n_out) {
  if (!s || !n_out || max < 0 || (max > 0 && (!ids || !statuses))) return trw_fail(TRW_ERR_INVALID, "bad arguments");
  if (trw_status dc = trw_check_device(s->g); dc != TRW_OK) return dc;
  *n_out = 0;
  std::lock_guard<std::mutex> lk(s->mu);
  int32_t n = 0;
  bool pending = false;
  for (unsigned long long k = s->oldest; k < s->next_k && n < max; ++k) {
    const int slot = (int)(k % (unsigned long long)s->R);
    if (s->collected[slot]) continue;
    const unsigned long long d = reinterpret_cast<volatile unsigned long long*>(s->done)[slot];
    if ((d >> 8) != k + 1) {
      pending = true;
      continue;
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    const int err = -(int)(d & 0xffu);
    s->collected[slot] = 1;
    s->inflight_walks -= s->req_walks[slot];
    s->inflight_bytes -= s->req_bytes[slot];
    ids[n] = k;
    statuses[n] = err == 0 ? TRW_OK
                  : err == kErrRejectCap ? TRW_ERR_REJECT_CAP
                  : err == kErrInvalid ? TRW_ERR_INVALID
                                       : TRW_ERR_INTERNAL;
    ++n;
  }
  retire_front(s);
  *n_out = n;
  if (pending && n == 0) {
    cudaError_t e = launch_if_idle(s);
    if (e != cudaSuccess) return trw_cuda_fail(e, "serve kernel relaunch");
    if ((++s->polls & 63) == 0) return check_state(s);
  }
  return TRW_OK;
}

extern "C" trw_status trw_serve_trace(trw_server* s, uint64_t req_id, uint64_t* t_ns) {
  if (!s || !t_ns) return trw_fail(TRW_ERR_INVALID, "NULL argument");
  if (trw_status dc = trw_check_device(s->g); dc != TRW_OK) return dc;
  std::lock_guard<std::mutex> lk(s->mu);
  if (req_id >= s->next_k || req_id + (unsigned long long)s->R < s->next_k)
    return trw_fail(TRW_ERR_NOT_FOUND, "request %llu is not in the slot table", (unsigned long long)req_id);
  const int slot = (int)(req_id % (unsigned long long)s->R);
  unsigned long long t[3];
  cudaError_t e = cudaMemcpyAsync(t, &s->slots[slot].t_admit, sizeof(t), cudaMemcpyDeviceToHost, s->copy_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
  if (e != cudaSuccess) return trw_cuda_fail(e, "serve trace");
  for (int i = 0; i < 3; ++i) t_ns[i] = t[i];
  return TRW_OK;
}

extern "C" trw_status trw_serve_drain(trw_server* s, int32_t timeout_ms) {
  if (!s) return trw_fail(TRW_ERR_INVALID, "NULL server");
  if (trw_status dc = trw_check_device(s->g); dc != TRW_OK) return dc;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      bool pending = false;
      for (unsigned long long k = s->oldest; k < s->next_k; ++k) {
        const int slot = (int)(k % (unsigned long long)s->R);
        if (s->collected[slot]) continue;
        const unsigned long long d = reinterpret_cast<volatile unsigned long long*>(s->done)[slot];
        if ((d >> 8) != k + 1) pending = true;
      }
      if (!pending) return check_state(s);
      cudaError_t e = launch_if_idle(s);
      if (e != cudaSuccess) return trw_cuda_fail(e, "serve kernel relaunch");
      trw_status cs = check_state(s);
      if (cs != TRW_OK) return cs;
    }
    if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms))
      return trw_fail(TRW_ERR_TIMEOUT, "requests still running after %d ms", timeout_ms);
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

extern "C" void trw_serve_destroy(trw_server* s) {
  if (!s) return;
  reinterpret_cast<volatile unsigned int*>(&s->host->stop)[0] = 1u;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  cudaStreamSynchronize(s->stream);
  server_release(s);
}
