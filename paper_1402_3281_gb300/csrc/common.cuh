// common.cuh -- shared definitions of the sm_103a SCLaP library: the
// counter-based hash, the segmented ("batched") level description, launch
// helpers and small warp/block primitives.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/sclap.h"

namespace sclap {

// ---------------------------------------------------------------------------
// Errors.  Host code throws sclap::Error; the C ABI converts it to a code.
// ---------------------------------------------------------------------------
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define SCLAP_CUDA(call)                                                                   \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw ::sclap::Error(e_ == cudaErrorMemoryAllocation ? SCLAP_ENOMEM : SCLAP_ECUDA,   \
                           std::string(#call) + ": " + cudaGetErrorString(e_));            \
  } while (0)

#define SCLAP_LAUNCH_CHECK() SCLAP_CUDA(cudaGetLastError())

// Process-wide instrumentation (see sclap_profile in sclap.h).
struct ProfileState {
  std::atomic<int64_t> launches{0};
  std::atomic<bool> enabled{false};
  std::atomic<bool> timeline{false};
  std::mutex mu;
  double ms[4] = {};
  int64_t nlaunch[4] = {}, nodes[4] = {}, arcs[4] = {};
  int64_t arcs_unit = 0;     // arcs of propose launches on levels without edge weights
  double sweep_ms = 0;       // propose phases, fork to join (concurrent launches)
  int64_t sweeps = 0;
  // per sub-round: run kind, round, colour class, nodes, arcs, propose ms,
  // admission ms (7 values each)
  std::vector<double> phases;
  // timeline mode: an event after every launch; the time from the previous
  // event of the same call to this one is charged to the kernel (device time
  // plus any idle gap before it)
  std::vector<std::pair<const char*, cudaEvent_t>> marks;
};
ProfileState& profile();
void timeline_mark(const char* name, cudaStream_t s);
std::string timeline_dump();
// cudaStreamSynchronize that also marks the timeline ("host": the copy and
// round trip that preceded the wait).
inline void stream_sync(cudaStream_t s) {
  SCLAP_CUDA(cudaStreamSynchronize(s));
  if (profile().timeline.load(std::memory_order_relaxed)) timeline_mark("host", s);
}
cudaEvent_t event_from_pool();
cudaStream_t side_stream(int i);

// Launch choices of the LP sweep that change scheduling, never results
// (sclap_tuning in sclap.h): rows of degree <= small_max_deg (8 or 16) get
// one thread per node, longer rows up to 128 one warp; grid caps in CTAs per
// SM; concurrent propose launches per colour class.
struct Tuning {
  int32_t small_max_deg = 16;
  int32_t small_ctas_per_sm = 8;
  int32_t warp_ctas_per_sm = 8;
  int32_t admit_ctas_per_sm = 16;
  int32_t concurrent = 1;
  int32_t pdl = 1;
  int32_t fused_admission = 0;   // 1: admission as one cooperative launch
  int32_t contract_table_slots = 0;   // slots per contraction pass (0: automatic)
  int32_t ip_trial_group = 0;         // trials replicated at once (0: automatic)
  int32_t contract_merge = 0;         // 1: contraction by member lists and merges
};
// Device memory still obtainable: free memory plus what the allocator pool
// holds unused.
int64_t obtainable_device_bytes();
// Slots of the contraction table one pass may use: the tuning value, or
// (automatic) half of the obtainable memory at 12 bytes per slot.
int64_t table_pass_slots();
Tuning tuning_get();
void tuning_set(const Tuning& t);
void event_to_pool(cudaEvent_t e);
#define SCLAP_NOTE_LAUNCH(name)                                               \
  do {                                                                        \
    ::sclap::profile().launches.fetch_add(1, std::memory_order_relaxed);      \
    if (::sclap::profile().timeline.load(std::memory_order_relaxed))          \
      ::sclap::timeline_mark(name, s);                                        \
  } while (0)

// Programmatic dependent launch.  A kernel launched with pdl = true may be
// scheduled while the previous kernel of its stream drains (on this GPU a
// dependent launch boundary measured 4.1 us per kernel without, 1.4-2.1 us
// with); its first statement is griddep_wait(), which returns once that
// kernel has completed and its writes are visible (and at once for a normal
// launch).  Only for a kernel whose preceding operation in the stream is a
// kernel launch (under stream capture it becomes a programmatic edge).
__device__ __forceinline__ void griddep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
template <typename... KArgs, typename... Args>
inline void launch_k(bool pdl, void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem,
                     cudaStream_t st, Args... args) {
  if (!pdl) {
    k<<<grid, block, smem, st>>>(args...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  SCLAP_CUDA(cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...));
}

// Device error word bits (set by kernels, read by the host after a phase).
enum : int32_t {
  DERR_HASH_FULL = 1,     // open-addressing table ran out of slots
  DERR_W_OVERFLOW = 2,    // coarse edge weight above INT32_MAX
  DERR_BAD_CSR = 4,       // validation
  DERR_INTERNAL = 8,
  DERR_TIMEOUT = 16,      // a bounded device-side wait ran out of iterations
  DERR_BOUNDS = 32,       // SCLAP_CHECK builds: a checked index was out of range
};

// Bounds checks of the SCLAP_CHECK build (compiled with -DSCLAP_CHECK=1):
// data-dependent indices (a neighbour, a label, a coarse id, a table slot)
// are checked against their array's length before the access; an index out
// of range sets DERR_BOUNDS in the kernel's error word and the access is
// skipped (a load yields zero), so the kernel never touches memory outside
// its arrays and the call ends with SCLAP_EINTERNAL.  In the normal build
// both macros are the plain access / `true`.
#if defined(SCLAP_CHECK) && SCLAP_CHECK
__device__ __forceinline__ bool sclap_chk(int64_t i, int64_t n, int32_t* err) {
  if (i >= 0 && i < n) return true;
  atomicOr(err, DERR_BOUNDS);
  return false;
}
template <class T>
__device__ __forceinline__ T sclap_chk_ld(const T* p, int64_t i, int64_t n, int32_t* err) {
  return sclap_chk(i, n, err) ? p[i] : T();
}
#define SCLAP_OK(i, n, err) sclap_chk((int64_t)(i), (int64_t)(n), (err))
#define SCLAP_LD(p, i, n, err) sclap_chk_ld((p), (int64_t)(i), (int64_t)(n), (err))
#else
#define SCLAP_OK(i, n, err) true
#define SCLAP_LD(p, i, n, err) ((p)[i])
#endif

// ---------------------------------------------------------------------------
// Grid-wide barrier of a cooperative launch (every CTA resident at once),
// with a bounded wait.  Thread 0 of each CTA reads the generation, arrives
// on the counter (release), and the last arriver resets the counter and
// advances the generation; the others poll the generation (acquire) at most
// `limit` times, ~0.5 us apart.  A wait that runs out sets DERR_TIMEOUT in
// the error word and the CTA is told to leave (returns false); the
// remaining CTAs then run out at their next barrier, so no CTA waits
// forever.  The state (two words, zeroed once) is left ready for the next
// barrier after every completed one.
// ---------------------------------------------------------------------------
struct GridSync {
  unsigned int arrive;
  unsigned int gen;
};
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Barrier of the `nblocks` CTAs that share `gs` (a group of CTAs of a
// cooperative launch, or the whole grid: grid_sync).
__device__ __forceinline__ bool group_sync(GridSync* gs, unsigned int nblocks, int32_t* err,
                                           uint32_t limit) {
  __shared__ int sh_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int g = ld_acquire_gpu(&gs->gen);
    __threadfence();
    const unsigned int prev = atomicAdd(&gs->arrive, 1u);
    if (prev == nblocks - 1) {
      gs->arrive = 0;
      __threadfence();
      atomicAdd(&gs->gen, 1u);
    } else {
      uint32_t it = 0;
      while (ld_acquire_gpu(&gs->gen) == g) {
        if (++it > limit) {
          atomicOr(err, DERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    sh_ok = ok;
  }
  __syncthreads();
  return sh_ok != 0;
}
__device__ __forceinline__ bool grid_sync(GridSync* gs, int32_t* err, uint32_t limit) {
  return group_sync(gs, gridDim.x, err, limit);
}

// Iteration limit of every bounded device-side wait (about 2 s at the
// default); a host-side fault-injection setting (sclap_debug_inject) may
// lower it to make waits run out on purpose.
uint32_t wait_limit();
// Probe limit of the open-addressing tables of the LP sweep (default: the
// table size, i.e. no limit); lowered only by sclap_debug_inject.
uint32_t probe_limit();
// Sets the three fault-injection values (see sclap_debug_inject).
void debug_inject(uint32_t wait, uint32_t probe, int32_t fail_allocs);
// Called by every device allocation: true for the allocation chosen to fail
// by sclap_debug_inject (the fail_allocs-th from the call on).
bool take_injected_alloc_failure();

// Cooperative launch (all CTAs co-resident; required by grid_sync).
template <typename... KArgs, typename... Args>
inline void launch_coop(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem,
                        cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  SCLAP_CUDA(cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...));
}

// ---------------------------------------------------------------------------
// SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014) and the keyed
// chain used for every random choice.  All hashes take graph-local ids so a
// graph's result does not depend on its position in a batch.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t hkey(uint64_t seed, uint64_t phase, uint64_t level,
                                                  uint64_t round) {
  return mix64(mix64(mix64(mix64(seed) ^ phase) ^ level) ^ round);
}

enum Phase : int32_t {
  PH_CLUSTER = 1, PH_REFINE = 2, PH_TRIAL = 3, PH_GGG = 4, PH_IPREF = 5, PH_REPAIR = 6,
  PH_ENSEMBLE = 7, PH_VCYCLE = 8
};
enum Mode : int32_t { MODE_CLUSTER = 0, MODE_REFINE = 1, MODE_REPAIR = 2 };

// Degree buckets of the LP sweep.  0..2 (degree <= 4 / 8 / 16): one thread
// per node, the row sorted in registers; 3..4 (<= 32 / 128, and overloaded
// nodes up to 128): one warp per node with a 256-slot shared table; 5..7
// (<= 512 / 2048 / 8192): one CTA of 128/256/512 threads per node with a
// shared table of 1024/4096/16384 slots; 8: one CTA per node, table in
// global scratch (hubs).  Nodes of overloaded blocks skip buckets 0..3.
constexpr int NB = 9;
constexpr int B4_MAXDEG = 128, B4_SLOTS = 256;
constexpr int B5_MAXDEG = 512, B5_SLOTS = 1024;
constexpr int B6_MAXDEG = 2048, B6_SLOTS = 4096;
constexpr int B7_MAXDEG = 8192, B7_SLOTS = 16384;

// Slots of the global-memory table of a hub of degree d: at most half full.
__host__ __device__ __forceinline__ int64_t hub_table_slots(int64_t d) {
  int64_t c = 32;
  while (c < 2 * d) c <<= 1;
  return c;
}

__host__ __device__ __forceinline__ int bucket_of(int64_t deg, bool overloaded) {
  if (!overloaded) {
    if (deg <= 4) return 0;
    if (deg <= 8) return 1;
    if (deg <= 16) return 2;
    if (deg <= 32) return 3;
  }
  if (deg <= B4_MAXDEG) return 4;
  if (deg <= B5_MAXDEG) return 5;
  if (deg <= B6_MAXDEG) return 6;
  if (deg <= B7_MAXDEG) return 7;
  return 8;
}

// Node and edge weight arrays of a level may be NULL: every weight is then 1
// (the input level of unit-weight graphs keeps no array of ones).  The slot
// array may be NULL when a level holds one graph (every node in slot 0).
__device__ __forceinline__ int32_t wat(const int32_t* __restrict__ w, int64_t i) {
  return w ? w[i] : 1;
}
__device__ __forceinline__ int32_t slot_at(const int32_t* __restrict__ gid, int64_t v) {
  return gid ? gid[v] : 0;
}

// Weight of a cluster or block.  Node weights are validated to sum below
// 2^31, so every label weight fits in 32 bits; sums with a node weight are
// formed in 64 bits.
using wgt_t = int32_t;

// ---------------------------------------------------------------------------
// A level: one CSR holding the graphs of all slots back to back (node ids are
// global, node range of slot s = [noff[s], noff[s+1])).
// ---------------------------------------------------------------------------
struct LevelView {
  int64_t N = 0, M = 0;
  const int64_t* row_ptr = nullptr;
  const int32_t* col = nullptr;
  const int32_t* ew = nullptr;    // NULL: unit edge weights
  const int32_t* nw = nullptr;    // NULL: unit node weights
  const int32_t* gid = nullptr;   // slot of each node (NULL: one slot)
  // every sum of arc weights over a row (so every connection) is below 2^32:
  // the propose tables may accumulate with 32-bit atomics
  bool narrow = false;
  // every graph's total arc weight is at most INT32_MAX, so no sum of arc
  // weights (a coarse arc's weight in particular) can overflow int32
  bool sums31 = false;
};

// Per-slot parameters of an LP run (device arrays of `nslots` entries).
struct SlotParams {
  int32_t nslots = 0;
  const int64_t* noff = nullptr;    // [nslots+1]
  const int64_t* loff = nullptr;    // label offset: local label = label - loff
  const int64_t* bound = nullptr;   // U (clustering) or Lmax (local search)
  const uint64_t* seed = nullptr;   // seed key fed to hkey
  const int32_t* level = nullptr;   // level id fed to hkey
  const int32_t* nlab = nullptr;    // labels of the slot (k in local search)
  int32_t* done = nullptr;          // 1: slot takes no part in further rounds
  int64_t* moved = nullptr;         // moves of the current round
  uint64_t* rkey = nullptr;         // key of the current round
  int32_t* rounds = nullptr;        // rounds run
};

// ---------------------------------------------------------------------------
// Small helpers.
// ---------------------------------------------------------------------------
inline int num_sms() {
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }();
  return sms;
}

inline unsigned grid_for(int64_t items, int per_block, int64_t cap) {
  int64_t g = (items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

__device__ __forceinline__ unsigned long long* ull(int64_t* p) {
  return reinterpret_cast<unsigned long long*>(p);
}

// Candidate order of the move rule: stronger connection first, then smaller
// tie hash, then smaller local label.  conn < 0 marks "no candidate".
struct Cand {
  int64_t conn;
  uint64_t h;
  int32_t C;  // local label
};
// Evaluated with bitwise logic on predicates (no short-circuit), so it
// compiles to compares and selects rather than branches.
__device__ __forceinline__ bool cand_better(const Cand& a, const Cand& b) {
  const bool gt = a.conn > b.conn, eq = a.conn == b.conn;
  return gt | (eq & ((a.h < b.h) | ((a.h == b.h) & (a.C < b.C))));
}
__device__ __forceinline__ Cand cand_pick(bool take, const Cand& x, const Cand& c) {
  Cand r;
  r.conn = take ? x.conn : c.conn;
  r.h = take ? x.h : c.h;
  r.C = take ? x.C : c.C;
  return r;
}
__device__ __forceinline__ Cand shfl_xor_cand(const Cand& c, int off, int width = 32) {
  Cand o;
  o.conn = __shfl_xor_sync(0xffffffffu, (long long)c.conn, off, width);
  o.h = __shfl_xor_sync(0xffffffffu, (unsigned long long)c.h, off, width);
  o.C = __shfl_xor_sync(0xffffffffu, c.C, off, width);
  return o;
}
__device__ __forceinline__ Cand warp_best(Cand c, int width = 32) {
#pragma unroll
  for (int off = width / 2; off > 0; off >>= 1) {
    const Cand o = shfl_xor_cand(c, off, width);
    c = cand_pick(cand_better(o, c), o, c);
  }
  return c;
}
__device__ __forceinline__ long long warp_max_ll(long long x, int width = 32) {
#pragma unroll
  for (int off = width / 2; off > 0; off >>= 1) {
    long long o = __shfl_xor_sync(0xffffffffu, x, off, width);
    x = o > x ? o : x;
  }
  return x;
}
__device__ __forceinline__ long long warp_sum_ll(long long x) {
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
}

// Sum of positive int32 values over the lanes of `mask` as a 64-bit number,
// from two 32-bit warp reductions of the 16-bit halves.
__device__ __forceinline__ int64_t match_sum(unsigned mask, int32_t w) {
  unsigned lo = __reduce_add_sync(mask, (unsigned)w & 0xffffu);
  unsigned hi = __reduce_add_sync(mask, (unsigned)w >> 16);
  return ((int64_t)hi << 16) + (int64_t)lo;
}

// Admission key: smaller key = admitted first.  High half: larger gain first
// (gain clamped to int32); low half: smaller priority hash first.
__device__ __forceinline__ uint64_t admission_key(int64_t gain, uint32_t prio) {
  int64_t g = gain > INT32_MAX ? INT32_MAX : (gain < INT32_MIN ? INT32_MIN : gain);
  uint32_t hi = (uint32_t)((int64_t)INT32_MAX - g);
  return ((uint64_t)hi << 32) | prio;
}

__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }
__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

__host__ __device__ __forceinline__ int ceil_log2(int64_t x) {
  int l = 0;
  while (((int64_t)1 << l) < x) ++l;
  return l;
}

// Open-addressing table slot for key C (multiplicative hashing).
__device__ __forceinline__ uint32_t table_slot(int32_t C, int logcap) {
  return logcap == 0 ? 0u : (((uint32_t)C * 0x9E3779B1u) >> (32 - logcap));
}

// Message of a failed device allocation: the request, the device's free and
// total memory, and what the allocator pool holds and uses.
std::string alloc_failure_message(size_t bytes, cudaError_t e);

// ---------------------------------------------------------------------------
// Device buffers from the stream-ordered allocator.
// ---------------------------------------------------------------------------
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(size_t count, cudaStream_t st) { alloc(count, st); }
  void alloc(size_t count, cudaStream_t st) {
    release();
    s = st;
    if (count && take_injected_alloc_failure())
      throw Error(SCLAP_ENOMEM, "device allocation failed (injected)");
    n = count;
    if (count) {
      const cudaError_t e = cudaMallocAsync((void**)&p, count * sizeof(T), st);
      if (e != cudaSuccess) {
        p = nullptr;
        n = 0;
        cudaGetLastError();
        throw Error(e == cudaErrorMemoryAllocation ? SCLAP_ENOMEM : SCLAP_ECUDA,
                    alloc_failure_message(count * sizeof(T), e));
      }
    }
  }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    n = 0;
  }
  void zero() {
    if (n) SCLAP_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
  }
  void fill_bytes(int v) {
    if (n) SCLAP_CUDA(cudaMemsetAsync(p, v, n * sizeof(T), s));
  }
  void upload(const T* h, size_t count) {
    if (count) SCLAP_CUDA(cudaMemcpyAsync(p, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
  }
  void upload(const std::vector<T>& v) { upload(v.data(), v.size()); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept { *this = std::move(o); }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; n = o.n; s = o.s;
      o.p = nullptr; o.n = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
};

// ---------------------------------------------------------------------------
// Entry points of the kernel files (host side).
// ---------------------------------------------------------------------------
// scan.cu: out[0..n] = exclusive prefix sums of in[0..n) (out[n] = total).
void scan_excl_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);
void scan_excl_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
void scan_excl_u8_to_i64(const uint8_t* in, int64_t* out, int64_t n, cudaStream_t s);
// out[i] = number of keys[0..i) that are >= 0 (occupied hash slots).
void scan_excl_occupied(const int32_t* keys, int64_t* out, int64_t n, cudaStream_t s);
// largest row length (atomicMax into *out, which the caller zeroes)
// out[0] = largest degree of the level, out[1] = nodes with degree > thr,
// out[2] = the table slots of those nodes together (out zeroed by the caller).
void level_degree_stats(const int64_t* row_ptr, int64_t N, int64_t thr, int64_t* out,
                        cudaStream_t s);
// slot id of every node from node offsets
void fill_gid(const int64_t* noff, int32_t nslots, int32_t* gid, int64_t N, cudaStream_t s);

// lp.cu
struct LPBuffers;
struct LPRun {
  int mode = MODE_CLUSTER;
  int phase = PH_CLUSTER;
  int rounds = 10;
  int sub_rounds = 8;
  bool stop_rule = true;       // 5% rule (not in repair)
  bool use_active = false;     // local search: active nodes
  bool raw_key = false;        // slot seed is used as the round key itself
  bool graph = false;          // run the rounds as one CUDA graph (WHILE node)
  const int32_t* rblk = nullptr;  // clustering: respect this partition (V-cycles)
};
// Runs `run.rounds` synchronous LP rounds on `lv` for every slot not marked
// done; label/W are updated in place.  Returns the number of arcs scanned.
int64_t lp_run(const LevelView& lv, const SlotParams& sp, int32_t* label, wgt_t* W,
               int64_t Wsize, const LPRun& run, int32_t* d_err, cudaStream_t s,
               const uint8_t* active_init = nullptr, uint8_t* active_next_out = nullptr);
void lp_round_begin_host_keys(const SlotParams& sp, int phase, int r, int mode,
                              const wgt_t* W, cudaStream_t s);

// contract.cu -- cluster contraction (Sec. 3.1) of every slot of a level.
struct ContractWork {
  DevBuf<int32_t> flag;        // [N] label used
  DevBuf<int64_t> cid;         // [N+1] exclusive scan of flag: rank of a label
  std::vector<int64_t> cid_at; // cid at each slot's first node [nslots+1]
};
struct CoarseLevel {
  int64_t N = 0, M = 0;
  DevBuf<int64_t> row_ptr;
  DevBuf<int32_t> col, ew, nw, gid;
  DevBuf<int64_t> noff_d;
  std::vector<int64_t> noff;   // [nslots+1]
  std::vector<int64_t> aoff;   // arc offset of each slot [nslots+1]
  LevelView view() const {
    LevelView v;
    v.N = N; v.M = M; v.row_ptr = row_ptr.p; v.col = col.p; v.ew = ew.p; v.nw = nw.p;
    v.gid = gid.p;
    return v;
  }
};
// Step 1: ranks the used labels; nc_slot[s] = coarse nodes of slot s.
// Overlay of two clusterings of a batched level (ensemble clusterings): for
// every node of a slot with part[slot] != 0, O[v] becomes the smallest node
// id sharing both its O and its C label; other slots keep O.  Errors (table
// overflow) are or-ed into err.
void overlay_labels(const LevelView& lv, const int32_t* part, int32_t* O, const int32_t* C,
                    int32_t* err, cudaStream_t s);

void contract_rank(const LevelView& lv, const std::vector<int64_t>& noff, const int32_t* label,
                   ContractWork& w, std::vector<int64_t>& nc_slot, cudaStream_t s);
// Step 2: builds the coarse graph of the slots with keep[s] != 0 (the other
// slots get no coarse nodes and cmap = -1).  cmap: [N] fine -> coarse id.
void contract_build(const LevelView& lv, const std::vector<int64_t>& noff, const int32_t* label,
                    const ContractWork& w, const std::vector<uint8_t>& keep, int32_t* cmap,
                    CoarseLevel& out, int32_t* d_err, cudaStream_t s);

// ip.cu -- initial partitioning of the coarsest graphs (all trials of all
// graphs in one batch), cut, projection.
struct CopyTask {              // copy one graph segment (NULL weights -> unit)
  const int64_t* row_ptr;
  const int32_t* col;
  const int32_t* ew;
  const int32_t* nw;
  int64_t src_n0, src_a0, n, m, dst_n0, dst_a0;
  // optional renumbering: rank[v] - rbase is the new id of a node with
  // neighbours (rank = exclusive scan of "has neighbours"); isolated nodes
  // are dropped.  NULL: plain copy.
  const int64_t* rank;
  int64_t rbase;
  int64_t nd;                  // nodes written (renumbered tasks; 0: n)
};
// Copies graph segments; row_ptr[N_total] = M_total.  Tasks with the same
// source segment (the trials of one graph) are copied once from the source
// and then from that first copy, with the node and arc offsets shifted (a
// streaming copy instead of one renumbering gather per arc).  N_total_override < 0:
// the end of the last plain task.  ew / nw may be NULL: the destination
// level keeps no weight array (unit weights).
void ip_replicate(const std::vector<CopyTask>& tasks, int64_t* row_ptr, int32_t* col,
                  int32_t* ew, int32_t* nw, int64_t M_total, cudaStream_t s,
                  int64_t N_total_override = -1);
struct GGGArgs {
  const int64_t* row_ptr;
  const int32_t* col;
  const int32_t* ew;
  const int32_t* nw;
  const int64_t* noff;     // trial slot node offsets
  const int64_t* boff;     // trial slot block offsets
  const int32_t* nlab;     // k per trial slot
  const int64_t* avg;      // ceil(c(V)/k) per trial slot
  const uint64_t* tkey;    // trial key per slot
  const int32_t* level;    // coarsest level index per slot
  int32_t* label;          // out: global block ids
  wgt_t* W;                // out: block weights
  int64_t* conn;           // scratch [N]
  int32_t* step;           // scratch [N]
  int32_t* front;          // scratch [N]: newly reached nodes (step alternates with it)
  int32_t* heavy;          // scratch [N]: a step's long rows (grouped growing)
  int64_t N;               // nodes of all trial slots (array lengths for bounds checks)
  uint32_t* asg;           // scratch [N / 32 + 1]: assigned-node bitmap (grouped growing)
  int64_t* wfA;            // scratch [sum k]
  int32_t* wforder;        // scratch [sum k]
  int32_t nslots;
  const int32_t* order;    // trial slots in the order they are taken (set by ggg_trials)
  int32_t* next;           // queue position (set by ggg_trials)
  int32_t* err;            // device error word (bounded waits, bounds-check builds)
};
// noff: host copy of the trial slot node offsets [nslots + 1]; nlab: host
// copy of k per trial slot.
void ggg_trials(const GGGArgs& a, const std::vector<int64_t>& noff,
                const std::vector<int32_t>& nlab, cudaStream_t s);
// cut2[slot] += twice the cut of each slot (arcs counted from both ends).
void slot_cut(const LevelView& lv, const int32_t* label, int64_t* cut2, cudaStream_t s);
struct SelectTask {            // choose the best trial of one graph, copy it out
  int32_t* dst_blk;            // level array of the graph's coarsest level
  int64_t dst_n0, n;
  int64_t slot0;               // first trial slot of the graph
  int32_t trials, k;
  int32_t trial0;              // index of the first of these trials among all
  int64_t Lmax, g_boff;        // graph's block offset in the refinement block space
  int32_t g;
  const int64_t* rank;         // renumbering of the trial graphs (see CopyTask)
  int64_t rbase;
};
// Water-filling of the isolated nodes (dst_blk < 0) of one graph into its
// lightest blocks, in node order; iso_prefix is the exclusive scan of the
// isolated nodes' weights over the level.
struct FillTask {
  int32_t* blk;
  const int32_t* nw;
  const int64_t* iso_prefix;
  int64_t n0, n, g_boff;
  int32_t k;
};
void waterfill_isolated(const std::vector<FillTask>& tasks, wgt_t* Wg, int64_t Ktot,
                        cudaStream_t s);
// flags[v] = 1 if v has neighbours; iso_w[v] = nw[v] if it has none, else 0.
void isolated_flags(const int64_t* row_ptr, const int32_t* nw, int64_t N, uint8_t* flags,
                    int32_t* iso_w, cudaStream_t s);
// best[g], ipcut[g] on the device; block weights copied to Wg[g_boff..].
// Trials may come in groups (one call per group, in increasing trial
// order): best[g] < 0 means no trial yet; a group's best trial replaces the
// kept one only if strictly better by (overload, cut), so the earliest of
// equal trials wins, as with all trials at once.  rb_ov: overload of the
// kept trial per graph.
void ip_select_copy(const std::vector<SelectTask>& tasks, const int64_t* cut2,
                    const wgt_t* ip_W, const int64_t* ip_noff, const int64_t* ip_boff,
                    const int32_t* ip_label, wgt_t* Wg, int32_t* best, int64_t* ipcut,
                    int64_t* rb_ov, cudaStream_t s);
// fine_blk[v] = coarse_blk[cmap[v]] where cmap[v] >= 0.
// V-cycles: coarse_blk[cmap[v]] = fine_blk[v] for every fine node with
// cmap[v] >= 0 (all members of a coarse node share one block).
void lift_blocks(const int32_t* cmap, const int32_t* fine_blk, int32_t* coarse_blk, int64_t N,
                 cudaStream_t s);
void project(const int32_t* cmap, const int32_t* coarse_blk, int32_t* fine_blk, int64_t N,
             cudaStream_t s);
// Block weights of every slot from scratch: W[label[v]] += nw[v].
void block_weights(const int32_t* label, const int32_t* nw, int64_t N, wgt_t* W, cudaStream_t s);

}  // namespace sclap
