// driver.cu -- the multilevel scheme (Sec. 1 Fig. 1, Sec. 3) over a batch of
// graphs, and the C ABI declared in include/sclap.h.
//
// All graphs of a call live in one segmented level (slot g = graph g), so
// every kernel launch of a level covers every graph still at that level.
// Coarsening: SCLaP clustering (bound U) + contraction while a graph has more
// than max(coarse_min_nodes, 60k) nodes and a contraction removes >= 5% of
// them.  Initial partitioning: all trials of all graphs in one batch.
// Uncoarsening: projection + LP local search (bound Lmax, active nodes) level
// by level; a final repair pass on the input level if a block is still
// above Lmax.  The host only reads level sizes back between levels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <chrono>
#include <memory>
#include <thread>

#include "common.cuh"

namespace sclap {
namespace {

thread_local std::string g_last_error;

void init_pool() {
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  });
}

// Clusterings per ensemble (Sec. 5): 18 for k < 16, 7 for k = 16..32, 3 above.
int32_t ensemble_size_for(int32_t k, const sclap_config& c) {
  if (c.ensemble_size > 0) return c.ensemble_size;
  return k < 16 ? 18 : (k <= 32 ? 7 : 3);
}

sclap_config resolve_cfg(const sclap_config* c) {
  sclap_config r;
  sclap_default_config(&r);
  if (c) r = *c;
  if (r.lp_rounds_coarse < 0 || r.lp_rounds_refine < 0 || r.f < 1 || r.coarse_min_nodes < 1 ||
      r.ip_trials < 1 || r.sub_rounds < 1 || r.sub_rounds > 64 || r.repair_rounds < 0 ||
      r.max_levels < 1 || r.cluster_active < 0 || r.cluster_active > 1 || r.graph_rounds < 0 ||
      r.graph_rounds > 1 || r.ensemble < 0 || r.ensemble > 1 || r.ensemble_size < 0 ||
      r.vcycles < 0)
    throw Error(SCLAP_EINVAL, "invalid sclap_config");
  return r;
}

// ------------------------------------------------------------- validation
// Checks a batched level as built from the inputs (one warp per 32 nodes,
// arcs flattened across lanes): row offsets non-decreasing and inside the
// slot's arc range, neighbours inside the slot, no self-loops, positive
// weights.  Per-slot error flags, c(V) and max c(v).  Arcs are read only
// inside ranges already checked, so malformed input cannot send a read out
// of the level's arrays.
__global__ void __launch_bounds__(256) k_validate_level(
    const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
    const int32_t* __restrict__ ew, const int32_t* __restrict__ nw,
    const int64_t* __restrict__ noff, const int64_t* __restrict__ aoff, int32_t nslots,
    int64_t N, int32_t* gerr, unsigned long long* cV, int32_t* maxc,
    unsigned long long* arcw) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = w0 * 32; base < N; base += nwarps * 32) {
    const int64_t v = base + lane;
    int32_t s = -1;
    int64_t rs = 0, d = 0;
    bool bad = false;
    int32_t w = 0;
    if (v < N) {
      int32_t lo = 0, hi = nslots - 1;
      while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (noff[mid] <= v) lo = mid; else hi = mid - 1;
      }
      s = lo;
      rs = row_ptr[v];
      const int64_t re = row_ptr[v + 1];
      if (rs > re || rs < aoff[s] || re > aoff[s + 1]) bad = true;
      if (v == noff[s] && rs != aoff[s]) bad = true;
      if (v == noff[s + 1] - 1 && re != aoff[s + 1]) bad = true;
      w = wat(nw, v);
      if (w <= 0) bad = true;
      d = bad ? 0 : re - rs;
    }
    // per-slot sums of node weights (lanes of one slot merged)
    const unsigned mm = __match_any_sync(0xffffffffu, s);
    const int64_t wsum = match_sum(mm, w > 0 ? w : 0);
    const int wmax = __reduce_max_sync(mm, w > 0 ? w : 0);
    if (s >= 0 && lane == __ffs(mm) - 1) {
      atomicAdd(&cV[s], (unsigned long long)wsum);
      atomicMax(&maxc[s], wmax);
    }
    long long incl = d;
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const long long excl = incl - d;
    const long long total = __shfl_sync(0xffffffffu, incl, 31);
    // total arc weight per slot: summed in registers when the warp's nodes
    // all lie in one slot, else one atomic per arc
    const int32_t s0 = __shfl_sync(0xffffffffu, s, 0);
    const bool uni = __all_sync(0xffffffffu, s < 0 || s == s0);
    unsigned long long acc = 0;
    for (long long x0 = 0; x0 < total; x0 += 32) {
      const long long x = x0 + lane;
      int L = 0;
      for (int step = 16; step > 0; step >>= 1) {
        long long y = __shfl_sync(0xffffffffu, incl, L + step - 1);
        if (y <= x) L += step;
      }
      const long long rsL = __shfl_sync(0xffffffffu, (long long)rs, L);
      const long long exL = __shfl_sync(0xffffffffu, excl, L);
      const int32_t sL = __shfl_sync(0xffffffffu, s, L);
      if (x < total) {
        const int64_t e = rsL + (x - exL);
        const int64_t src = base + L;
        const int32_t c = col[e];
        const int32_t we = wat(ew, e);
        if (c < noff[sL] || c >= noff[sL + 1] || c == src || we <= 0) atomicOr(&gerr[sL], 1);
        const unsigned long long wp = we > 0 ? (unsigned long long)we : 0ull;
        if (uni) acc += wp;
        else if (wp) atomicAdd(&arcw[sL], wp);
      }
    }
    if (uni) {
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0 && acc) atomicAdd(&arcw[s0], acc);
    }
    if (bad && s >= 0) atomicOr(&gerr[s], 1);
  }
}

__global__ void k_iota(int32_t* label, int64_t N) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x)
    label[v] = (int32_t)v;
}

// comm[v] <- cmap[comm[v]]: one more contraction composed into the
// input-node-to-coarse-node map.
__global__ void k_compose(int32_t* __restrict__ comm, const int32_t* __restrict__ cmap,
                          int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    comm[v] = cmap[comm[v]];
}

__global__ void k_w_from_nw(const int32_t* nw, int64_t N, wgt_t* W) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x)
    W[v] = wat(nw, v);
}

#if defined(SCLAP_CHECK) && SCLAP_CHECK
// Bounds-check self test: index n - 1 of buf is read; index n is checked
// and refused (never read).  err[0] / err[1]: the error word of each.
__global__ void k_check_selftest(const int32_t* buf, int64_t n, int32_t* out, int32_t* err) {
  out[0] = SCLAP_LD(buf, n - 1, n, &err[0]);
  out[1] = SCLAP_LD(buf, n, n, &err[1]);
}
#endif

__global__ void k_check_range(const int32_t* __restrict__ a, int64_t n, int64_t lo, int64_t hi,
                              int32_t* err) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    if (a[v] < lo || a[v] >= hi) atomicOr(err, DERR_BAD_CSR);
}

__global__ void k_gather_at(const int64_t* __restrict__ src, const int64_t* __restrict__ idx, int n,
                            int64_t* __restrict__ dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

__global__ void k_narrow(const int64_t* __restrict__ in, int64_t n, wgt_t* __restrict__ out,
                         int32_t* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = in[i];
    if (x < INT32_MIN || x > INT32_MAX) atomicOr(err, DERR_BAD_CSR);
    out[i] = (wgt_t)x;
  }
}
__global__ void k_widen(const wgt_t* __restrict__ in, int64_t n, int64_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

struct OutTask {
  int32_t* out;
  int64_t n0, n, boff;
};
__global__ void k_write_out(const OutTask* __restrict__ t, const int32_t* __restrict__ blk) {
  const OutTask o = t[blockIdx.y];
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < o.n;
       v += (int64_t)gridDim.x * blockDim.x)
    o.out[v] = (int32_t)(blk[o.n0 + v] - o.boff);
}

// ------------------------------------------------------------- slot arrays
struct Slots {
  DevBuf<int64_t> loff, bound, moved;
  DevBuf<uint64_t> seed, rkey;
  DevBuf<int32_t> level, nlab, done, rounds;
  SlotParams sp;
  Slots(cudaStream_t s, int n, const int64_t* noff_d, const std::vector<int64_t>& h_loff,
        const std::vector<int64_t>& h_bound, const std::vector<uint64_t>& h_seed,
        const std::vector<int32_t>& h_level, const std::vector<int32_t>& h_nlab,
        const std::vector<int32_t>& h_done)
      : loff(n, s), bound(n, s), moved(n, s), seed(n, s), rkey(n, s), level(n, s), nlab(n, s),
        done(n, s), rounds(n, s) {
    loff.upload(h_loff); bound.upload(h_bound); seed.upload(h_seed); level.upload(h_level);
    nlab.upload(h_nlab); done.upload(h_done); rounds.zero(); moved.zero();
    sp.nslots = n; sp.noff = noff_d; sp.loff = loff.p; sp.bound = bound.p; sp.seed = seed.p;
    sp.level = level.p; sp.nlab = nlab.p; sp.done = done.p; sp.moved = moved.p; sp.rkey = rkey.p;
    sp.rounds = rounds.p;
  }
  std::vector<int32_t> host_rounds(cudaStream_t s) {
    std::vector<int32_t> r(sp.nslots);
    SCLAP_CUDA(cudaMemcpyAsync(r.data(), rounds.p, r.size() * sizeof(int32_t),
                               cudaMemcpyDeviceToHost, s));
    stream_sync(s);
    return r;
  }
};

// A batched level.  Its graph arrays are owned, or (the input level of a
// single device-resident graph) borrowed from the caller, read in place and
// never written.  Weight arrays are NULL for unit weights, the slot array
// NULL for a level holding one graph.
struct Level {
  int64_t N = 0, M = 0;
  DevBuf<int64_t> row_ptr, noff_d;
  DevBuf<int32_t> col, ew, nw, gid, cmap, blk;
  const int64_t* rp_in = nullptr;          // borrowed arrays (input level)
  const int32_t* col_in = nullptr;
  const int32_t* ew_in = nullptr;
  const int32_t* nw_in = nullptr;
  bool borrowed = false;
  std::vector<int64_t> noff, aoff;
  // every sum of arc weights over a row of this level fits in 32 bits: true
  // when every graph's total arc weight does (which then holds on every
  // level of its hierarchy: contraction only merges or drops arcs), and on
  // an input level of unit weights (a row's sum is its degree, < 2^31)
  bool narrow = false;
  bool narrow_total = false;   // the total-weight rule alone (inherited by coarse levels)
  bool sums31 = false;         // every graph's total arc weight <= INT32_MAX (inherited)
  const int64_t* rp() const { return borrowed ? rp_in : row_ptr.p; }
  const int32_t* colp() const { return borrowed ? col_in : col.p; }
  const int32_t* ewp() const { return borrowed ? ew_in : ew.p; }
  const int32_t* nwp() const { return borrowed ? nw_in : nw.p; }
  LevelView view() const {
    LevelView v;
    v.N = N; v.M = M; v.row_ptr = rp(); v.col = colp(); v.ew = ewp(); v.nw = nwp();
    v.gid = gid.p;
    v.narrow = narrow;
    v.sums31 = sums31;
    return v;
  }
};

// One input graph, arrays already in device memory.
struct GIn {
  int64_t n = 0, m = 0;
  const int64_t* row_ptr = nullptr;
  const int32_t* col = nullptr;
  const int32_t* nw = nullptr;
  const int32_t* ew = nullptr;
  int32_t k = 2;
  double eps = 0.03;
  uint64_t seed = 0;
};

struct GOut {
  int32_t status = SCLAP_OK;
  int64_t cut = 0, maxbw = 0;
  sclap_stats st{};
};

// Lmax = floor((1+eps) * ceil(cV/k)); U = max(max c(v), floor(Lmax/f)).
void bounds(int64_t cV, int64_t maxc, int32_t k, double eps, int32_t f, int64_t* Lmax,
            int64_t* U) {
  const int64_t avg = (cV + k - 1) / k;
  const int64_t L = (int64_t)std::floor((1.0 + eps) * (double)avg);
  *Lmax = L;
  *U = std::max<int64_t>(maxc, L / f);
}

void check_err(int32_t* d_err, cudaStream_t s) {
  int32_t e = 0;
  SCLAP_CUDA(cudaMemcpyAsync(&e, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  stream_sync(s);
  if (e & DERR_TIMEOUT) throw Error(SCLAP_ETIMEOUT, "a bounded device-side wait ran out");
  if (e & DERR_W_OVERFLOW) throw Error(SCLAP_EOVERFLOW, "coarse edge weight above INT32_MAX");
  if (e & DERR_HASH_FULL) throw Error(SCLAP_EINTERNAL, "hash table full");
  if (e & DERR_BAD_CSR) throw Error(SCLAP_ECSR, "malformed CSR");
  if (e & DERR_BOUNDS) throw Error(SCLAP_EINTERNAL, "bounds check failed (SCLAP_CHECK build)");
  if (e) throw Error(SCLAP_EINTERNAL, "device error word set");
}

// Raises SCLAP_EINVAL unless every a[v] lies in [lo, hi).
void check_range(const int32_t* a, int64_t n, int64_t lo, int64_t hi, cudaStream_t s,
                 const char* what) {
  DevBuf<int32_t> err(1, s);
  err.zero();
  k_check_range<<<grid_for(n, 256, (int64_t)num_sms() * 8), 256, 0, s>>>(a, n, lo, hi, err.p); SCLAP_NOTE_LAUNCH("k_check_range");
  SCLAP_LAUNCH_CHECK();
  int32_t e = 0;
  SCLAP_CUDA(cudaMemcpyAsync(&e, err.p, 4, cudaMemcpyDeviceToHost, s));
  stream_sync(s);
  if (e) throw Error(SCLAP_EINVAL, std::string(what) + " out of range");
}

void build_level0(const std::vector<GIn>& gs, struct Level& L, cudaStream_t s);

// Validates the batched level L (built by build_level0 from `B` inputs):
// per-graph status (SCLAP_OK, SCLAP_ECSR or SCLAP_EOVERFLOW), c(V), max c(v)
// and whether the graph's total arc weight fits in 32 bits (every sum of arc
// weights met later, at any level of its hierarchy, is at most that total:
// contraction only merges or drops arcs).
void validate_level(const Level& L, int B, std::vector<int32_t>& status,
                    std::vector<int64_t>& cV, std::vector<int64_t>& maxc,
                    std::vector<char>& narrow, cudaStream_t s,
                    std::vector<char>* sums31 = nullptr) {
  DevBuf<int32_t> err(B, s), mx(B, s);
  DevBuf<unsigned long long> sum(B, s), arcw(B, s);
  DevBuf<int64_t> d_aoff(B + 1, s);
  err.zero(); mx.zero(); sum.zero(); arcw.zero();
  d_aoff.upload(L.aoff);
  if (L.N > 0) {
    k_validate_level<<<grid_for(L.N, 256, (int64_t)num_sms() * 16), 256, 0, s>>>(
        L.rp(), L.colp(), L.ewp(), L.nwp(), L.noff_d.p, d_aoff.p, B, L.N, err.p, sum.p, mx.p,
        arcw.p); SCLAP_NOTE_LAUNCH("k_validate_level");
    SCLAP_LAUNCH_CHECK();
  }
  std::vector<int32_t> e(B), m(B);
  std::vector<unsigned long long> w(B), aw(B);
  SCLAP_CUDA(cudaMemcpyAsync(e.data(), err.p, B * 4, cudaMemcpyDeviceToHost, s));
  SCLAP_CUDA(cudaMemcpyAsync(m.data(), mx.p, B * 4, cudaMemcpyDeviceToHost, s));
  SCLAP_CUDA(cudaMemcpyAsync(w.data(), sum.p, B * 8, cudaMemcpyDeviceToHost, s));
  SCLAP_CUDA(cudaMemcpyAsync(aw.data(), arcw.p, B * 8, cudaMemcpyDeviceToHost, s));
  stream_sync(s);
  status.assign(B, SCLAP_OK);
  cV.assign(B, 0);
  maxc.assign(B, 0);
  narrow.assign(B, 0);
  if (sums31) sums31->assign(B, 0);
  for (int g = 0; g < B; ++g) {
    if (e[g]) status[g] = SCLAP_ECSR;
    else if (w[g] >= (1ull << 31)) status[g] = SCLAP_EOVERFLOW;
    cV[g] = (int64_t)w[g];
    maxc[g] = m[g];
    narrow[g] = aw[g] <= 0xffffffffull ? 1 : 0;
    if (sums31) (*sums31)[g] = aw[g] <= (unsigned long long)INT32_MAX ? 1 : 0;
  }
}

// Validates one device-resident graph (step entry points); returns c(V) and
// max c(v) or throws.
void validate(const GIn& g, cudaStream_t s, int64_t* cV, int64_t* maxc, bool* narrow = nullptr) {
  Level L;
  build_level0({g}, L, s);
  std::vector<int32_t> st;
  std::vector<int64_t> a, b;
  std::vector<char> nar;
  validate_level(L, 1, st, a, b, nar, s);
  if (st[0] == SCLAP_ECSR)
    throw Error(SCLAP_ECSR, "malformed CSR (row_ptr, column range, self-loop or weight)");
  if (st[0] == SCLAP_EOVERFLOW) throw Error(SCLAP_EOVERFLOW, "sum of node weights must be < 2^31");
  *cV = a[0];
  *maxc = b[0];
  if (narrow) *narrow = nar[0] != 0;
}

// Builds the level holding the graphs `gs` back to back.  One graph is used
// in place (its device arrays are only read; no copy, no slot array); a
// batch is copied into one segmented CSR.  Weight arrays are kept only when
// some graph has weights: a batch of unit-weight graphs keeps none.
void build_level0(const std::vector<GIn>& gs, Level& L, cudaStream_t s) {
  const int B = (int)gs.size();
  L.noff.assign(B + 1, 0);
  L.aoff.assign(B + 1, 0);
  for (int i = 0; i < B; ++i) {
    L.noff[i + 1] = L.noff[i] + gs[i].n;
    L.aoff[i + 1] = L.aoff[i] + gs[i].m;
  }
  L.N = L.noff[B];
  L.M = L.aoff[B];
  if (L.N >= ((int64_t)1 << 31)) throw Error(SCLAP_EINVAL, "total node count must be < 2^31");
  L.noff_d.alloc(B + 1, s);
  L.noff_d.upload(L.noff);
  if (B == 1) {
    L.borrowed = true;
    L.rp_in = gs[0].row_ptr;
    L.col_in = gs[0].col;
    L.ew_in = gs[0].ew;
    L.nw_in = gs[0].nw;
    return;
  }
  bool any_ew = false, any_nw = false;
  for (const GIn& g : gs) {
    any_ew = any_ew || g.ew != nullptr;
    any_nw = any_nw || g.nw != nullptr;
  }
  L.row_ptr.alloc(L.N + 1, s);
  L.col.alloc(std::max<int64_t>(L.M, 1), s);
  if (any_ew) L.ew.alloc(std::max<int64_t>(L.M, 1), s);
  if (any_nw) L.nw.alloc(std::max<int64_t>(L.N, 1), s);
  std::vector<CopyTask> tasks(B);
  for (int i = 0; i < B; ++i)
    tasks[i] = CopyTask{gs[i].row_ptr, gs[i].col, gs[i].ew, gs[i].nw, 0, 0, gs[i].n, gs[i].m,
                        L.noff[i], L.aoff[i], nullptr, 0, gs[i].n};
  ip_replicate(tasks, L.row_ptr.p, L.col.p, L.ew.p, L.nw.p, L.M, s);
  L.gid.alloc(std::max<int64_t>(L.N, 1), s);
  fill_gid(L.noff_d.p, B, L.gid.p, L.N, s);
}

struct GState {
  int32_t k;
  uint64_t seed;
  int64_t cV, Lmax, U, avg, T;
  int32_t q = 0;
  int64_t boff = 0;
  std::vector<int64_t> n_at, m_at;
  std::vector<int32_t> crounds, rrounds;
};



// ---------------------------------------------------------------------------
// Initial partitioning of a set of coarsest graphs: every graph gets
// cfg.ip_trials trials (greedy growing + water-filling + LP local search),
// all in one trial batch; the best trial of each graph is copied into its
// level's block array and its block weights into Wg.
// ---------------------------------------------------------------------------
struct IPIn {
  const Level* Q;      // level holding the graph
  int g;               // slot of the graph in Q
  int32_t k;
  int64_t Lmax, avg;
  uint64_t seed;
  int32_t q;           // level index (hash input)
  int64_t boff;        // graph's offset in the block space of Wg
  int32_t* dst_blk;    // block array of Q
};

void run_ip(const std::vector<IPIn>& in, const sclap_config& cfg, wgt_t* Wg,
            std::vector<int32_t>& best, std::vector<int64_t>& ipcut, int64_t* lp_arcs,
            int32_t* d_err, cudaStream_t s) {
  const int B = (int)in.size();
  const int T = cfg.ip_trials;
  // Trials run on the nodes that have neighbours: per level holding coarsest
  // graphs, rank them (scan of "has neighbours") and keep the isolated
  // nodes' weight prefix for the water-filling afterwards.
  struct LevelAux {
    DevBuf<int64_t> rank, iso_prefix;
    std::vector<int64_t> rank_at;
  };
  std::vector<std::pair<const Level*, std::unique_ptr<LevelAux>>> aux;
  auto aux_of = [&](const Level* Q) -> LevelAux& {
    for (auto& p : aux)
      if (p.first == Q) return *p.second;
    std::unique_ptr<LevelAux> x(new LevelAux());
    const int ns = (int)Q->noff.size() - 1;
    DevBuf<uint8_t> flags(std::max<int64_t>(Q->N, 1), s);
    DevBuf<int32_t> iso(std::max<int64_t>(Q->N, 1), s);
    isolated_flags(Q->rp(), Q->nwp(), Q->N, flags.p, iso.p, s);
    x->rank.alloc(Q->N + 1, s);
    x->iso_prefix.alloc(Q->N + 1, s);
    scan_excl_u8_to_i64(flags.p, x->rank.p, Q->N, s);
    scan_excl_i32_to_i64(iso.p, x->iso_prefix.p, Q->N, s);
    x->rank_at.assign(ns + 1, 0);
    DevBuf<int64_t> got(ns + 1, s);
    k_gather_at<<<grid_for(ns + 1, 128, 64), 128, 0, s>>>(x->rank.p, Q->noff_d.p, ns + 1, got.p); SCLAP_NOTE_LAUNCH("k_gather_at");
    SCLAP_LAUNCH_CHECK();
    SCLAP_CUDA(cudaMemcpyAsync(x->rank_at.data(), got.p, (ns + 1) * sizeof(int64_t),
                               cudaMemcpyDeviceToHost, s));
    stream_sync(s);
    aux.emplace_back(Q, std::move(x));
    return *aux.back().second;
  };
  // Trials run in groups whose replicated graphs fit in memory (all of them
  // at once unless the coarsest graphs are very large): about 204 bytes per
  // node and 8 per arc of each trial copy (graph, growing and LP state),
  // against half of the device memory still obtainable, or the tuning's
  // group size.  Results do not depend on the grouping: a trial's
  // arithmetic is independent of the others, and the best trial is kept
  // across groups in trial order.
  int64_t per_trial = 0;
  for (int g = 0; g < B; ++g) {
    const Level& Q = *in[g].Q;
    LevelAux& X = aux_of(&Q);
    const int x = in[g].g;
    per_trial += 204 * (X.rank_at[x + 1] - X.rank_at[x]) + 8 * (Q.aoff[x + 1] - Q.aoff[x]) + 64;
  }
  const Tuning tu = tuning_get();
  const int64_t fit = tu.ip_trial_group > 0
                          ? tu.ip_trial_group
                          : obtainable_device_bytes() / 2 / std::max<int64_t>(per_trial, 1);
  const int TG = (int)std::max<int64_t>(1, std::min<int64_t>(T, fit));
  DevBuf<int32_t> d_best(B, s);
  DevBuf<int64_t> d_cut(B, s), d_ov(B, s);
  d_best.fill_bytes(0xff);
  for (int t0 = 0; t0 < T; t0 += TG) {
  const int T = std::min(TG, cfg.ip_trials - t0);   // trials of this group
  const int S = B * T;
  std::vector<int64_t> noff(S + 1, 0), aoff(S + 1, 0), boff(S + 1, 0);
  std::vector<CopyTask> tasks;
  tasks.reserve(S);
  for (int g = 0; g < B; ++g) {
    const Level& Q = *in[g].Q;
    LevelAux& X = aux_of(&Q);
    const int x = in[g].g;
    const int64_t n = Q.noff[x + 1] - Q.noff[x], m = Q.aoff[x + 1] - Q.aoff[x];
    const int64_t nA = X.rank_at[x + 1] - X.rank_at[x];
    for (int t = 0; t < T; ++t) {
      const int i = g * T + t;
      noff[i + 1] = noff[i] + nA;
      aoff[i + 1] = aoff[i] + m;
      boff[i + 1] = boff[i] + in[g].k;
      tasks.push_back(CopyTask{Q.rp(), Q.colp(), Q.ewp(), Q.nwp(), Q.noff[x], Q.aoff[x], n, m,
                               noff[i], aoff[i], X.rank.p, X.rank_at[x], nA});
    }
  }
  Level ip;
  ip.narrow = true;
  for (const IPIn& x : in) ip.narrow = ip.narrow && x.Q->narrow;
  ip.N = noff[S];
  ip.M = aoff[S];
  if (ip.N >= ((int64_t)1 << 31)) throw Error(SCLAP_EINVAL, "trial batch too large");
  ip.row_ptr.alloc(ip.N + 1, s);
  ip.col.alloc(std::max<int64_t>(ip.M, 1), s);
  ip.ew.alloc(std::max<int64_t>(ip.M, 1), s);
  ip.nw.alloc(std::max<int64_t>(ip.N, 1), s);
  ip_replicate(tasks, ip.row_ptr.p, ip.col.p, ip.ew.p, ip.nw.p, ip.M, s, ip.N);
  ip.noff = noff;
  ip.aoff = aoff;
  ip.noff_d.alloc(S + 1, s);
  ip.noff_d.upload(noff);
  ip.gid.alloc(std::max<int64_t>(ip.N, 1), s);
  fill_gid(ip.noff_d.p, S, ip.gid.p, ip.N, s);

  const int64_t K = boff[S];
  DevBuf<int32_t> label(std::max<int64_t>(ip.N, 1), s), step(std::max<int64_t>(ip.N, 1), s),
      front(std::max<int64_t>(ip.N, 1), s), heavy(std::max<int64_t>(ip.N, 1), s);
  DevBuf<wgt_t> W(std::max<int64_t>(K, 1), s);
  DevBuf<int64_t> conn(std::max<int64_t>(ip.N, 1), s);
  DevBuf<int64_t> wfA(std::max<int64_t>(K, 1), s), d_boff(S + 1, s), d_avg(S, s);
  DevBuf<int32_t> wforder(std::max<int64_t>(K, 1), s);
  std::vector<int64_t> h_avg(S), h_bound(S);
  std::vector<uint64_t> h_tkey(S);
  std::vector<int32_t> h_level(S), h_nlab(S), h_done(S, 0);
  for (int g = 0; g < B; ++g)
    for (int t = 0; t < T; ++t) {
      const int i = g * T + t;
      h_avg[i] = in[g].avg;
      h_bound[i] = in[g].Lmax;
      h_tkey[i] = hkey(in[g].seed, PH_TRIAL, (uint64_t)in[g].q, (uint64_t)(t0 + t));
      h_level[i] = in[g].q;
      h_nlab[i] = in[g].k;
    }
  d_boff.upload(boff);
  d_avg.upload(h_avg);
  std::vector<int64_t> h_loff(boff.begin(), boff.end() - 1);
  Slots sl(s, S, ip.noff_d.p, h_loff, h_bound, h_tkey, h_level, h_nlab, h_done);

  GGGArgs ga{};
  ga.row_ptr = ip.row_ptr.p; ga.col = ip.col.p; ga.ew = ip.ew.p; ga.nw = ip.nw.p;
  ga.noff = ip.noff_d.p; ga.boff = d_boff.p; ga.nlab = sl.nlab.p; ga.avg = d_avg.p;
  ga.tkey = sl.seed.p; ga.level = sl.level.p; ga.label = label.p; ga.W = W.p;
  ga.conn = conn.p; ga.step = step.p; ga.front = front.p; ga.heavy = heavy.p;
  ga.wfA = wfA.p; ga.wforder = wforder.p;
  ga.nslots = S;
  ga.N = ip.N;
  ga.err = d_err;
  ggg_trials(ga, noff, h_nlab, s);

  LPRun run;
  run.mode = MODE_REFINE;
  run.phase = PH_IPREF;
  run.rounds = cfg.lp_rounds_refine;
  run.sub_rounds = cfg.sub_rounds;
  run.graph = cfg.graph_rounds != 0;
  run.use_active = true;
  *lp_arcs += lp_run(ip.view(), sl.sp, label.p, W.p, K, run, d_err, s);

  DevBuf<int64_t> cut2(S, s);
  cut2.zero();
  slot_cut(ip.view(), label.p, cut2.p, s);
  std::vector<SelectTask> sel(B);
  for (int g = 0; g < B; ++g) {
    const Level& Q = *in[g].Q;
    const int x = in[g].g;
    LevelAux& X = aux_of(&Q);
    sel[g] = SelectTask{in[g].dst_blk, Q.noff[x], Q.noff[x + 1] - Q.noff[x], (int64_t)g * T, T,
                        in[g].k, t0, in[g].Lmax, in[g].boff, g, X.rank.p, X.rank_at[x]};
  }
  ip_select_copy(sel, cut2.p, W.p, ip.noff_d.p, d_boff.p, label.p, Wg, d_best.p, d_cut.p,
                 d_ov.p, s);
  }
  std::vector<FillTask> fill(B);
  int64_t Kmax = 0;
  for (int g = 0; g < B; ++g) {
    const Level& Q = *in[g].Q;
    LevelAux& X = aux_of(&Q);
    const int x = in[g].g;
    fill[g] = FillTask{in[g].dst_blk, Q.nwp(), X.iso_prefix.p, Q.noff[x], Q.noff[x + 1] - Q.noff[x],
                       in[g].boff, in[g].k};
    Kmax = std::max(Kmax, in[g].boff + in[g].k);
  }
  waterfill_isolated(fill, Wg, Kmax, s);
  best.assign(B, 0);
  ipcut.assign(B, 0);
  SCLAP_CUDA(cudaMemcpyAsync(best.data(), d_best.p, B * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SCLAP_CUDA(cudaMemcpyAsync(ipcut.data(), d_cut.p, B * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  stream_sync(s);
}

// ---------------------------------------------------------------------------
// The multilevel partitioner over a batch of validated graphs.
// ---------------------------------------------------------------------------
void run_valid_batch(const std::vector<GIn>& gs, const std::vector<int64_t>& cV,
                     const std::vector<int64_t>& maxc, const sclap_config& cfg,
                     const std::vector<int32_t*>& outs, std::vector<GOut>& res,
                     std::unique_ptr<Level> level0, cudaStream_t s);

// Validates the inputs on the device and partitions the valid ones together;
// invalid graphs get their error in res[g].status.
void run_batch(const std::vector<GIn>& gs_in, const sclap_config& cfg,
               const std::vector<int32_t*>& outs_in, std::vector<GOut>& res, cudaStream_t s) {
  const int B = (int)gs_in.size();
  res.assign(B, GOut{});
  if (profile().timeline.load()) timeline_mark("<call>", s);
  std::unique_ptr<Level> L0(new Level());
  build_level0(gs_in, *L0, s);
  std::vector<int32_t> status;
  std::vector<int64_t> cV, maxc;
  std::vector<char> narrow, small;
  validate_level(*L0, B, status, cV, maxc, narrow, s, &small);
  std::vector<int> ok;
  bool all_narrow = true, all_small = true;
  for (int g = 0; g < B; ++g) {
    if (status[g] == SCLAP_OK) {
      ok.push_back(g);
      all_narrow = all_narrow && narrow[g];
      all_small = all_small && small[g];
    } else {
      res[g].status = status[g];
    }
  }
  if ((int)ok.size() == B) {
    L0->narrow_total = all_narrow;
    L0->narrow = all_narrow || L0->ewp() == nullptr;
    L0->sums31 = all_small;
    run_valid_batch(gs_in, cV, maxc, cfg, outs_in, res, std::move(L0), s);
    return;
  }
  if (ok.empty()) return;
  std::vector<GIn> gs;
  std::vector<int64_t> c2, m2;
  std::vector<int32_t*> outs;
  for (int g : ok) {
    gs.push_back(gs_in[g]);
    c2.push_back(cV[g]);
    m2.push_back(maxc[g]);
    outs.push_back(outs_in[g]);
  }
  L0.reset(new Level());
  build_level0(gs, *L0, s);
  L0->narrow_total = all_narrow;
  L0->narrow = all_narrow || L0->ewp() == nullptr;
  L0->sums31 = all_small;
  std::vector<GOut> r2;
  run_valid_batch(gs, c2, m2, cfg, outs, r2, std::move(L0), s);
  for (size_t j = 0; j < ok.size(); ++j) res[ok[j]] = r2[j];
}

void run_valid_batch(const std::vector<GIn>& gs, const std::vector<int64_t>& cV,
                     const std::vector<int64_t>& maxc, const sclap_config& cfg,
                     const std::vector<int32_t*>& outs, std::vector<GOut>& res,
                     std::unique_ptr<Level> level0, cudaStream_t s) {
  const int B = (int)gs.size();
  res.assign(B, GOut{});
  std::vector<GState> st(B);
  int64_t Ktot = 0;
  for (int g = 0; g < B; ++g) {
    GState& x = st[g];
    x.k = gs[g].k;
    x.seed = gs[g].seed;
    x.cV = cV[g];
    bounds(cV[g], maxc[g], x.k, gs[g].eps, cfg.f, &x.Lmax, &x.U);
    x.avg = (cV[g] + x.k - 1) / x.k;
    x.T = std::max<int64_t>(cfg.coarse_min_nodes, 60 * (int64_t)x.k);
    x.boff = Ktot;
    Ktot += x.k;
    x.n_at.push_back(gs[g].n);
    x.m_at.push_back(gs[g].m);
  }
  DevBuf<int32_t> d_err(1, s);
  d_err.zero();
  int64_t lp_arcs = 0;
  const int sms = num_sms();

  std::vector<std::unique_ptr<Level>> lv;
  lv.push_back(std::move(level0));

  // ---------------- coarsening (as a stage: later V-cycles run it again)
  // Builds the hierarchy above lv[0] (the only level when called).  seeds:
  // per-slot keys of the clusterings; respect: clusterings stay inside the
  // blocks of lv[L]->blk (V-cycles), coarse levels get the projected blocks;
  // record: fill the statistics.  q[g] receives slot g's coarsest level.
  auto coarsen = [&](const std::vector<uint64_t>& seeds, bool respect, bool record,
                     std::vector<int32_t>& q) {
    q.assign(B, 0);
    std::vector<char> coarsening(B, 0);
    for (int g = 0; g < B; ++g)
      coarsening[g] = (gs[g].n > st[g].T && 1 < cfg.max_levels) ? 1 : 0;
    for (int L = 0;; ++L) {
      bool any = false;
      for (int g = 0; g < B; ++g) any = any || coarsening[g];
      if (!any) break;
      Level& cur = *lv[L];
      const LevelView v = cur.view();
      std::vector<int64_t> h_bound(B);
      std::vector<int32_t> h_level(B, L), h_nlab(B, 0), h_done(B);
      for (int g = 0; g < B; ++g) {
        h_bound[g] = st[g].U;
        h_done[g] = coarsening[g] ? 0 : 1;
      }
      std::vector<int64_t> h_loff(cur.noff.begin(), cur.noff.end() - 1);
      Slots sl(s, B, cur.noff_d.p, h_loff, h_bound, seeds, h_level, h_nlab, h_done);
      DevBuf<int32_t> label(std::max<int64_t>(v.N, 1), s);
      DevBuf<wgt_t> W(std::max<int64_t>(v.N, 1), s);
      k_iota<<<grid_for(v.N, 256, (int64_t)sms * 16), 256, 0, s>>>(label.p, v.N); SCLAP_NOTE_LAUNCH("k_iota");
      k_w_from_nw<<<grid_for(v.N, 256, (int64_t)sms * 16), 256, 0, s>>>(v.nw, v.N, W.p); SCLAP_NOTE_LAUNCH("k_w_from_nw");
      SCLAP_LAUNCH_CHECK();
      LPRun run;
      run.mode = MODE_CLUSTER;
      run.phase = PH_CLUSTER;
      run.rounds = cfg.lp_rounds_coarse;
      run.sub_rounds = cfg.sub_rounds;
      run.graph = cfg.graph_rounds != 0;
      run.use_active = cfg.cluster_active != 0;
      run.rblk = respect ? cur.blk.p : nullptr;
      lp_arcs += lp_run(v, sl.sp, label.p, W.p, v.N, run, d_err.p, s);
      const std::vector<int32_t> rr = sl.host_rounds(s);
      if (record)
        for (int g = 0; g < B; ++g)
          if (coarsening[g]) st[g].crounds.push_back(rr[g]);
      if (cfg.ensemble) {
        // ensemble clusterings: clustering j >= 1 of every slot whose ensemble
        // is that large, overlaid onto the labels so far
        std::vector<int32_t> ell(B, 1);
        int32_t ell_max = 1;
        for (int g = 0; g < B; ++g)
          if (coarsening[g]) {
            ell[g] = ensemble_size_for(st[g].k, cfg);
            ell_max = std::max(ell_max, ell[g]);
          }
        if (ell_max > 1) {
          DevBuf<int32_t> C(std::max<int64_t>(v.N, 1), s), part(B, s);
          for (int32_t j = 1; j < ell_max; ++j) {
            std::vector<uint64_t> sj(B);
            std::vector<int32_t> dj(B), pj(B);
            for (int g = 0; g < B; ++g) {
              pj[g] = coarsening[g] && j < ell[g] ? 1 : 0;
              dj[g] = pj[g] ? 0 : 1;
              sj[g] = hkey(seeds[g], PH_ENSEMBLE, (uint64_t)L, (uint64_t)j);
            }
            Slots slj(s, B, cur.noff_d.p, h_loff, h_bound, sj, h_level, h_nlab, dj);
            k_iota<<<grid_for(v.N, 256, (int64_t)sms * 16), 256, 0, s>>>(C.p, v.N); SCLAP_NOTE_LAUNCH("k_iota");
            k_w_from_nw<<<grid_for(v.N, 256, (int64_t)sms * 16), 256, 0, s>>>(v.nw, v.N, W.p); SCLAP_NOTE_LAUNCH("k_w_from_nw");
            lp_arcs += lp_run(v, slj.sp, C.p, W.p, v.N, run, d_err.p, s);
            part.upload(pj);
            overlay_labels(v, part.p, label.p, C.p, d_err.p, s);
          }
        }
      }
      ContractWork cw;
      std::vector<int64_t> nc;
      contract_rank(v, cur.noff, label.p, cw, nc, s);
      std::vector<uint8_t> keep(B, 0);
      bool anykeep = false;
      for (int g = 0; g < B; ++g) {
        if (!coarsening[g]) continue;
        const int64_t n = cur.noff[g + 1] - cur.noff[g];
        if (20 * (n - nc[g]) < n) {
          coarsening[g] = 0;   // shrink below 5%: this level stays the coarsest
        } else {
          keep[g] = 1;
          anykeep = true;
        }
      }
      if (!anykeep) break;
      cur.cmap.alloc(std::max<int64_t>(v.N, 1), s);
      CoarseLevel co;
      contract_build(v, cur.noff, label.p, cw, keep, cur.cmap.p, co, d_err.p, s);
      std::unique_ptr<Level> nx(new Level());
      nx->narrow = cur.narrow_total;
      nx->narrow_total = cur.narrow_total;
      nx->sums31 = cur.sums31;
      nx->N = co.N;
      nx->M = co.M;
      nx->row_ptr = std::move(co.row_ptr);
      nx->col = std::move(co.col);
      nx->ew = std::move(co.ew);
      nx->nw = std::move(co.nw);
      nx->gid = std::move(co.gid);
      nx->noff_d = std::move(co.noff_d);
      nx->noff = co.noff;
      nx->aoff = co.aoff;
      if (respect) {
        // the partition moves up with the clusters (all members share a block)
        nx->blk.alloc(std::max<int64_t>(nx->N, 1), s);
        lift_blocks(cur.cmap.p, cur.blk.p, nx->blk.p, v.N, s);
      }
      for (int g = 0; g < B; ++g) {
        if (!keep[g]) continue;
        q[g] = L + 1;
        const int64_t n = nx->noff[g + 1] - nx->noff[g];
        if (record) {
          st[g].n_at.push_back(n);
          st[g].m_at.push_back(nx->aoff[g + 1] - nx->aoff[g]);
        }
        coarsening[g] = (n > st[g].T && L + 2 < cfg.max_levels) ? 1 : 0;
      }
      lv.push_back(std::move(nx));
    }
    check_err(d_err.p, s);
  };

  std::vector<uint64_t> seed0(B);
  for (int g = 0; g < B; ++g) seed0[g] = st[g].seed;
  {
    std::vector<int32_t> q;
    coarsen(seed0, false, true, q);
    for (int g = 0; g < B; ++g) st[g].q = q[g];
  }
  const int nlev = (int)lv.size();
  for (int L = 0; L < nlev; ++L) lv[L]->blk.alloc(std::max<int64_t>(lv[L]->N, 1), s);

  // ---------------- initial partitioning
  DevBuf<wgt_t> Wg(std::max<int64_t>(Ktot, 1), s);
  {
    std::vector<IPIn> in(B);
    for (int g = 0; g < B; ++g) {
      const Level* Q = lv[st[g].q].get();
      in[g] = IPIn{Q, g, st[g].k, st[g].Lmax, st[g].avg, st[g].seed, st[g].q, st[g].boff,
                   Q->blk.p};
    }
    std::vector<int32_t> best;
    std::vector<int64_t> ipcut;
    run_ip(in, cfg, Wg.p, best, ipcut, &lp_arcs, d_err.p, s);
    for (int g = 0; g < B; ++g) {
      res[g].st.ip_best_trial = best[g];
      res[g].st.ip_cut = ipcut[g];
    }
  }

  // ---------------- uncoarsening: project, then LP local search (a stage)
  std::vector<int64_t> h_Lmax(B), h_boff(B);
  std::vector<int32_t> h_k(B);
  for (int g = 0; g < B; ++g) {
    h_Lmax[g] = st[g].Lmax;
    h_boff[g] = st[g].boff;
    h_k[g] = st[g].k;
    st[g].rrounds.assign(st[g].q + 1, 0);
  }
  // From the top of lv down to the input level: project, then refine every
  // slot whose hierarchy reaches that level (below its coarsest level, and
  // at it too when refine_top: the partition there was projected up, not
  // computed by initial partitioning).
  auto uncoarsen = [&](const std::vector<uint64_t>& seeds, const std::vector<int32_t>& q,
                       bool refine_top, bool record) {
    const int top = (int)lv.size() - 1;
    for (int L = refine_top ? top : top - 1; L >= 0; --L) {
      Level& F = *lv[L];
      if (L < top) {
        project(F.cmap.p, lv[L + 1]->blk.p, F.blk.p, F.N, s);
        lv[L + 1].reset();
      }
      std::vector<int32_t> h_level(B, L), h_done(B);
      bool any = false;
      for (int g = 0; g < B; ++g) {
        h_done[g] = (refine_top ? q[g] >= L : q[g] > L) ? 0 : 1;
        any = any || !h_done[g];
      }
      if (!any) continue;
      Slots sl(s, B, F.noff_d.p, h_boff, h_Lmax, seeds, h_level, h_k, h_done);
      LPRun run;
      run.mode = MODE_REFINE;
      run.phase = PH_REFINE;
      run.rounds = cfg.lp_rounds_refine;
      run.sub_rounds = cfg.sub_rounds;
      run.graph = cfg.graph_rounds != 0;
      run.use_active = true;
      lp_arcs += lp_run(F.view(), sl.sp, F.blk.p, Wg.p, Ktot, run, d_err.p, s);
      if (record) {
        const std::vector<int32_t> rr = sl.host_rounds(s);
        for (int g = 0; g < B; ++g)
          if (q[g] > L) st[g].rrounds[L] = rr[g];
      }
    }
    lv.resize(1);
  };
  // ---------------- balance repair on the input level (a stage)
  auto repair = [&](const std::vector<uint64_t>& seeds) {
    Level& F0 = *lv[0];
    if (cfg.repair_rounds <= 0) return;
    std::vector<int32_t> h_level(B, 0), h_done(B, 0);
    Slots sl(s, B, F0.noff_d.p, h_boff, h_Lmax, seeds, h_level, h_k, h_done);
    LPRun run;
    run.mode = MODE_REPAIR;
    run.phase = PH_REPAIR;
    run.rounds = cfg.repair_rounds;
    run.sub_rounds = cfg.sub_rounds;
    run.graph = cfg.graph_rounds != 0;
    run.stop_rule = false;
    lp_arcs += lp_run(F0.view(), sl.sp, F0.blk.p, Wg.p, Ktot, run, d_err.p, s);
  };
  {
    std::vector<int32_t> q(B);
    for (int g = 0; g < B; ++g) q[g] = st[g].q;
    uncoarsen(seed0, q, false, true);
  }
  repair(seed0);
  check_err(d_err.p, s);

  // ---------------- iterated V-cycles (Sec. 4 "Iterated Multilevel
  // Algorithms", App. A): coarsen again with clusterings inside the blocks
  // of the current partition (cut edges are never contracted), start from
  // that partition on the coarsest level, refine every level on the way back,
  // repair.  Cycle c uses hkey(seed, VCYCLE, c, 0) in place of the seed.
  for (int32_t cyc = 1; cyc < std::max(1, cfg.vcycles); ++cyc) {
    std::vector<uint64_t> sc(B);
    for (int g = 0; g < B; ++g) sc[g] = hkey(st[g].seed, PH_VCYCLE, (uint64_t)cyc, 0);
    std::vector<int32_t> q;
    coarsen(sc, true, false, q);
    uncoarsen(sc, q, true, false);
    repair(sc);
    check_err(d_err.p, s);
  }
  Level& F0 = *lv[0];

  // ---------------- cut, outputs
  DevBuf<int64_t> cut2(B, s);
  cut2.zero();
  slot_cut(F0.view(), F0.blk.p, cut2.p, s);
  std::vector<OutTask> ot(B);
  int64_t mx = 1;
  for (int g = 0; g < B; ++g) {
    ot[g] = OutTask{outs[g], F0.noff[g], gs[g].n, st[g].boff};
    mx = std::max(mx, gs[g].n);
  }
  DevBuf<OutTask> d_ot(B, s);
  d_ot.upload(ot);
  for (int b0 = 0; b0 < B; b0 += 65535) {
    dim3 grid(grid_for(mx, 256, 256), (unsigned)std::min(65535, B - b0));
    k_write_out<<<grid, 256, 0, s>>>(d_ot.p + b0, F0.blk.p); SCLAP_NOTE_LAUNCH("k_write_out");
  }
  SCLAP_LAUNCH_CHECK();
  std::vector<int64_t> h_cut2(B);
  std::vector<wgt_t> h_W(Ktot);
  SCLAP_CUDA(cudaMemcpyAsync(h_cut2.data(), cut2.p, B * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SCLAP_CUDA(cudaMemcpyAsync(h_W.data(), Wg.p, Ktot * sizeof(wgt_t), cudaMemcpyDeviceToHost, s));
  stream_sync(s);
  for (int g = 0; g < B; ++g) {
    GOut& o = res[g];
    o.cut = h_cut2[g] / 2;
    int64_t m = 0;
    for (int b = 0; b < st[g].k; ++b) m = std::max<int64_t>(m, h_W[st[g].boff + b]);
    o.maxbw = m;
    o.status = m <= st[g].Lmax ? SCLAP_OK : SCLAP_EINFEASIBLE;
    sclap_stats& x = o.st;
    x.levels = st[g].q + 1;
    for (int l = 0; l <= st[g].q && l < 64; ++l) {
      x.level_n[l] = st[g].n_at[l];
      x.level_m[l] = st[g].m_at[l];
      x.refine_rounds[l] = l < (int)st[g].rrounds.size() ? st[g].rrounds[l] : 0;
    }
    for (size_t l = 0; l < st[g].crounds.size() && l < 64; ++l) x.cluster_rounds[l] = st[g].crounds[l];
    x.Lmax = st[g].Lmax;
    x.U = st[g].U;
    x.lp_arcs = lp_arcs;
  }
}

// ---------------------------------------------------------------------------
// Helpers for the C ABI.
// ---------------------------------------------------------------------------
template <class F>
int guarded(F&& f) {
  try {
    init_pool();
    f();
    g_last_error.clear();
    return SCLAP_OK;
  } catch (const Error& e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return SCLAP_EINTERNAL;
  } catch (...) {
    g_last_error = "unknown exception";
    return SCLAP_EINTERNAL;
  }
}

void check_args(int64_t n, const void* row_ptr, const void* col, int32_t k, double eps,
                const void* out) {
  if (n < 1 || n >= ((int64_t)1 << 31)) throw Error(SCLAP_EINVAL, "n must be in [1, 2^31)");
  if (!row_ptr || !out) throw Error(SCLAP_EINVAL, "NULL array");
  (void)col;   // may be NULL when the graph has no arcs (checked once m is known)
  if (k < 1 || (int64_t)k > n) throw Error(SCLAP_EINVAL, "k must be in [1, n]");
  if (!(eps >= 0.0) || !std::isfinite(eps)) throw Error(SCLAP_EINVAL, "eps must be >= 0");
}

int64_t device_arcs(const int64_t* row_ptr, int64_t n, cudaStream_t s) {
  int64_t m = 0;
  SCLAP_CUDA(cudaMemcpyAsync(&m, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  stream_sync(s);
  if (m < 0 || m >= ((int64_t)1 << 40)) throw Error(SCLAP_ECSR, "row_ptr[n] out of range");
  return m;
}

__global__ void k_read_ends(const int64_t* const* __restrict__ ends, int n, int64_t* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = *ends[i];
}

// row_ptr[n] of many device graphs with one launch and one copy.
std::vector<int64_t> device_arcs_many(const std::vector<const int64_t*>& ends, cudaStream_t s) {
  const int n = (int)ends.size();
  std::vector<int64_t> m(n, 0);
  if (n == 0) return m;
  DevBuf<const int64_t*> d(n, s);
  d.upload(ends);
  DevBuf<int64_t> out(n, s);
  k_read_ends<<<grid_for(n, 128, 64), 128, 0, s>>>(d.p, n, out.p); SCLAP_NOTE_LAUNCH("k_read_ends");
  SCLAP_LAUNCH_CHECK();
  SCLAP_CUDA(cudaMemcpyAsync(m.data(), out.p, n * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  stream_sync(s);
  for (int64_t x : m)
    if (x < 0 || x >= ((int64_t)1 << 40)) throw Error(SCLAP_ECSR, "row_ptr[n] out of range");
  return m;
}

void check_col(const void* col, int64_t m) {
  if (m > 0 && !col) throw Error(SCLAP_EINVAL, "NULL col with arcs present");
}

// Owned device copy of a host graph.
struct HostUpload {
  DevBuf<int64_t> rp;
  DevBuf<int32_t> col, nw, ew;
  GIn g;
  HostUpload(int64_t n, const int64_t* row_ptr, const int32_t* c, const int32_t* node_w,
             const int32_t* edge_w, cudaStream_t s) {
    const int64_t m = row_ptr[n];
    if (m < 0) throw Error(SCLAP_ECSR, "row_ptr[n] < 0");
    check_col(c, m);
    rp.alloc(n + 1, s);
    rp.upload(row_ptr, n + 1);
    col.alloc(std::max<int64_t>(m, 1), s);
    col.upload(c, m);
    if (node_w) { nw.alloc(n, s); nw.upload(node_w, n); }
    if (edge_w) { ew.alloc(std::max<int64_t>(m, 1), s); ew.upload(edge_w, m); }
    g.n = n; g.m = m; g.row_ptr = rp.p; g.col = col.p;
    g.nw = node_w ? nw.p : nullptr;
    g.ew = edge_w ? ew.p : nullptr;
  }
};

// Host arrays of a batch go through one pinned staging buffer per calling
// thread, kept and grown across calls: host threads pack every graph's
// arrays into it, one copy moves them to one device buffer, and the block
// arrays come back the same way.  (One pageable copy per array costs a
// driver-staged transfer each: about a thousand per 512-graph batch.)
struct PinnedStage {
  void* p = nullptr;
  size_t cap = 0;
  PinnedStage() = default;
  PinnedStage(const PinnedStage&) = delete;
  PinnedStage& operator=(const PinnedStage&) = delete;
  ~PinnedStage() {
    if (p) cudaFreeHost(p);
  }
  // NULL when pinned memory cannot be had (the caller copies array by array)
  char* get(size_t bytes) {
    if (bytes > cap) {
      if (p) cudaFreeHost(p);
      p = nullptr;
      cap = 0;
      const size_t want = std::max<size_t>(bytes + bytes / 4, (size_t)1 << 20);
      if (cudaHostAlloc(&p, want, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        return nullptr;
      }
      cap = want;
    }
    return static_cast<char*>(p);
  }
};
thread_local PinnedStage t_stage;

struct Piece {
  void* dst;
  const void* src;
  size_t bytes;
};
// The pieces' memcpys on up to 8 host threads, split into runs of about
// equal bytes.
void parallel_copy(const std::vector<Piece>& pieces) {
  size_t total = 0;
  for (const Piece& x : pieces) total += x.bytes;
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int nt = (int)std::min<size_t>(std::min(8u, hw), std::max<size_t>(1, total >> 24));
  if (nt <= 1) {
    for (const Piece& x : pieces) std::memcpy(x.dst, x.src, x.bytes);
    return;
  }
  // cut the byte stream into nt ranges; a piece may be split between threads
  auto run = [&](size_t lo, size_t hi) {
    size_t at = 0;
    for (const Piece& x : pieces) {
      const size_t a = std::max(lo, at), b = std::min(hi, at + x.bytes);
      if (a < b)
        std::memcpy(static_cast<char*>(x.dst) + (a - at),
                    static_cast<const char*>(x.src) + (a - at), b - a);
      at += x.bytes;
      if (at >= hi) break;
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(run, total * t / nt, total * (t + 1) / nt);
  run(0, total / nt);
  for (auto& x : th) x.join();
}

// A one-slot level holding a copy of a device graph (step entry points).
void single_level(const GIn& g, Level& L, cudaStream_t s) {
  std::vector<GIn> v{g};
  build_level0(v, L, s);
}

void fill_stats(sclap_stats* dst, const GOut& o) {
  if (dst) *dst = o.st;
}

}  // namespace
}  // namespace sclap

using namespace sclap;

// Message returned by sclap_last_error() for entry points defined in other
// translation units.
namespace sclap {
void record_last_error(const char* msg) { g_last_error = msg ? msg : ""; }
}  // namespace sclap

extern "C" {

void sclap_default_config(sclap_config* c) {
  if (!c) return;
  c->lp_rounds_coarse = 10;
  c->lp_rounds_refine = 10;
  c->f = 18;
  c->coarse_min_nodes = 1000;
  c->ip_trials = 16;
  c->sub_rounds = 8;
  c->repair_rounds = 64;
  c->max_levels = 64;
  c->cluster_active = 0;
  c->graph_rounds = 0;
  c->ensemble = 0;
  c->ensemble_size = 0;
  c->vcycles = 1;
}

const char* sclap_error_string(int code) {
  switch (code) {
    case SCLAP_OK: return "ok";
    case SCLAP_EINVAL: return "invalid argument";
    case SCLAP_ECSR: return "malformed CSR input";
    case SCLAP_ENOMEM: return "device out of memory";
    case SCLAP_ECUDA: return "CUDA error";
    case SCLAP_EOVERFLOW: return "integer weight overflow";
    case SCLAP_EINFEASIBLE: return "balance constraint could not be met";
    case SCLAP_ETIMEOUT: return "bounded device wait timed out";
    case SCLAP_EINTERNAL: return "internal error";
    case SCLAP_PENDING: return "request pending";
    default: return "unknown error code";
  }
}

const char* sclap_last_error(void) { return g_last_error.c_str(); }

int sclap_partition(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* node_w,
                    const int32_t* edge_w, int32_t k, double eps, uint64_t seed,
                    const sclap_config* cfg, int32_t* block_out, int64_t* cut_out,
                    int64_t* max_block_weight_out, sclap_stats* stats) {
  int status = SCLAP_OK;
  int rc = guarded([&] {
    check_args(n, row_ptr, col, k, eps, block_out);
    const sclap_config c = resolve_cfg(cfg);
    cudaStream_t s = 0;
    HostUpload up(n, row_ptr, col, node_w, edge_w, s);
    up.g.k = k; up.g.eps = eps; up.g.seed = seed;
    DevBuf<int32_t> out(n, s);
    std::vector<GOut> res;
    run_batch({up.g}, c, {out.p}, res, s);
    if (res[0].status != SCLAP_OK && res[0].status != SCLAP_EINFEASIBLE)
      throw Error(res[0].status, "invalid input graph");
    SCLAP_CUDA(cudaMemcpyAsync(block_out, out.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    stream_sync(s);
    if (cut_out) *cut_out = res[0].cut;
    if (max_block_weight_out) *max_block_weight_out = res[0].maxbw;
    fill_stats(stats, res[0]);
    status = res[0].status;
  });
  return rc != SCLAP_OK ? rc : status;
}

int sclap_partition_device(int64_t n, const int64_t* row_ptr, const int32_t* col,
                           const int32_t* node_w, const int32_t* edge_w, int32_t k, double eps,
                           uint64_t seed, const sclap_config* cfg, int32_t* block_out,
                           int64_t* cut_out, int64_t* max_block_weight_out, sclap_stats* stats,
                           void* stream) {
  int status = SCLAP_OK;
  int rc = guarded([&] {
    check_args(n, row_ptr, col, k, eps, block_out);
    const sclap_config c = resolve_cfg(cfg);
    cudaStream_t s = (cudaStream_t)stream;
    GIn g;
    g.n = n; g.m = device_arcs(row_ptr, n, s); g.row_ptr = row_ptr; g.col = col;
    g.nw = node_w; g.ew = edge_w; g.k = k; g.eps = eps; g.seed = seed;
    check_col(g.col, g.m);
    std::vector<GOut> res;
    run_batch({g}, c, {block_out}, res, s);
    if (res[0].status != SCLAP_OK && res[0].status != SCLAP_EINFEASIBLE)
      throw Error(res[0].status, "invalid input graph");
    stream_sync(s);
    if (cut_out) *cut_out = res[0].cut;
    if (max_block_weight_out) *max_block_weight_out = res[0].maxbw;
    fill_stats(stats, res[0]);
    status = res[0].status;
  });
  return rc != SCLAP_OK ? rc : status;
}

int sclap_partition_batch(int32_t count, sclap_graph* graphs, const sclap_config* cfg,
                          int32_t device_ptrs, void* stream) {
  int first_err = SCLAP_OK;
  int rc = guarded([&] {
    if (count < 0 || (count > 0 && !graphs)) throw Error(SCLAP_EINVAL, "bad batch");
    const sclap_config c = resolve_cfg(cfg);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<std::unique_ptr<HostUpload>> ups;
    std::vector<GIn> gs;
    std::vector<int64_t> cV, maxc;
    std::vector<int> idx;
    std::vector<std::unique_ptr<DevBuf<int32_t>>> outbufs;
    std::vector<int32_t*> outs;
    std::vector<int64_t> dev_m(count, 0);
    if (device_ptrs) {
      std::vector<const int64_t*> ends;
      std::vector<int> who;
      for (int i = 0; i < count; ++i) {
        const sclap_graph& G = graphs[i];
        if (G.row_ptr && G.n >= 1 && G.n < ((int64_t)1 << 31)) {
          ends.push_back(G.row_ptr + G.n);
          who.push_back(i);
        }
      }
      const std::vector<int64_t> m = device_arcs_many(ends, s);
      for (size_t j = 0; j < who.size(); ++j) dev_m[who[j]] = m[j];
    }
    // host arrays: sizes and packed offsets (16-byte aligned) of every valid
    // graph, so that one pinned buffer and one copy carry them all
    struct Pack { int64_t m; size_t rp, col, nw, ew; };
    std::vector<Pack> pk(count);
    size_t in_bytes = 0, out_bytes = 0;
    auto take = [&](size_t bytes) {
      const size_t at = in_bytes;
      in_bytes += (bytes + 15) & ~(size_t)15;
      return at;
    };
    char* stage = nullptr;
    DevBuf<char> din;
    DevBuf<int32_t> dout;
    if (!device_ptrs) {
      for (int i = 0; i < count; ++i) {
        const sclap_graph& G = graphs[i];
        pk[i].m = -1;
        if (G.row_ptr && G.n >= 1 && G.n < ((int64_t)1 << 31)) {
          const int64_t m = G.row_ptr[G.n];
          if (m < 0) continue;
          pk[i].m = m;
          pk[i].rp = take((G.n + 1) * sizeof(int64_t));
          pk[i].col = take(m * sizeof(int32_t));
          pk[i].nw = G.node_w ? take(G.n * sizeof(int32_t)) : 0;
          pk[i].ew = G.edge_w ? take(m * sizeof(int32_t)) : 0;
          out_bytes += G.n * sizeof(int32_t);
        }
      }
      if (in_bytes > 0) stage = t_stage.get(std::max(in_bytes, out_bytes));
      if (stage) {
        std::vector<Piece> pieces;
        for (int i = 0; i < count; ++i) {
          const sclap_graph& G = graphs[i];
          if (pk[i].m < 0 || (pk[i].m > 0 && !G.col)) continue;
          pieces.push_back({stage + pk[i].rp, G.row_ptr, (G.n + 1) * sizeof(int64_t)});
          pieces.push_back({stage + pk[i].col, G.col, pk[i].m * sizeof(int32_t)});
          if (G.node_w) pieces.push_back({stage + pk[i].nw, G.node_w, G.n * sizeof(int32_t)});
          if (G.edge_w) pieces.push_back({stage + pk[i].ew, G.edge_w, pk[i].m * sizeof(int32_t)});
        }
        parallel_copy(pieces);
        din.alloc(in_bytes, s);
        SCLAP_CUDA(cudaMemcpyAsync(din.p, stage, in_bytes, cudaMemcpyHostToDevice, s));
        dout.alloc(std::max<size_t>(out_bytes / sizeof(int32_t), 1), s);
        stream_sync(s);   // the stage is free again (it carries the blocks back)
      }
    }
    int64_t out_at = 0;
    for (int i = 0; i < count; ++i) {
      sclap_graph& G = graphs[i];
      G.status = guarded([&] {
        check_args(G.n, G.row_ptr, G.col, G.k, G.eps, G.block_out);
        GIn g;
        if (device_ptrs) {
          g.n = G.n; g.m = dev_m[i]; g.row_ptr = G.row_ptr;
          g.col = G.col; g.nw = G.node_w; g.ew = G.edge_w;
        } else if (stage) {
          if (pk[i].m < 0) throw Error(SCLAP_ECSR, "row_ptr[n] < 0");
          g.n = G.n;
          g.m = pk[i].m;
          g.row_ptr = reinterpret_cast<const int64_t*>(din.p + pk[i].rp);
          g.col = reinterpret_cast<const int32_t*>(din.p + pk[i].col);
          g.nw = G.node_w ? reinterpret_cast<const int32_t*>(din.p + pk[i].nw) : nullptr;
          g.ew = G.edge_w ? reinterpret_cast<const int32_t*>(din.p + pk[i].ew) : nullptr;
          check_col(G.col, g.m);
        } else {
          ups.emplace_back(new HostUpload(G.n, G.row_ptr, G.col, G.node_w, G.edge_w, s));
          g = ups.back()->g;
        }
        g.k = G.k; g.eps = G.eps; g.seed = G.seed;
        check_col(g.col, g.m);
        gs.push_back(g);
        idx.push_back(i);
        if (device_ptrs) {
          outs.push_back(G.block_out);
        } else if (stage) {
          outs.push_back(dout.p + out_at);
          out_at += G.n;
        } else {
          outbufs.emplace_back(new DevBuf<int32_t>(G.n, s));
          outs.push_back(outbufs.back()->p);
        }
      });
      if (G.status != SCLAP_OK && first_err == SCLAP_OK) first_err = G.status;
    }
    if (gs.empty()) return;
    std::vector<GOut> res;
    run_batch(gs, c, outs, res, s);
    if (!device_ptrs && stage) {
      // every block array back in one copy, then out to the callers' arrays
      SCLAP_CUDA(cudaMemcpyAsync(stage, dout.p, out_at * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                 s));
      stream_sync(s);
      std::vector<Piece> pieces;
      for (size_t j = 0; j < gs.size(); ++j) {
        const sclap_graph& G = graphs[idx[j]];
        pieces.push_back({G.block_out, stage + (outs[j] - dout.p) * sizeof(int32_t),
                          G.n * sizeof(int32_t)});
      }
      parallel_copy(pieces);
    }
    for (size_t j = 0; j < gs.size(); ++j) {
      sclap_graph& G = graphs[idx[j]];
      if (!device_ptrs && !stage)
        SCLAP_CUDA(cudaMemcpyAsync(G.block_out, outs[j], G.n * sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, s));
      G.cut = res[j].cut;
      G.max_block_weight = res[j].maxbw;
      G.status = res[j].status;
      if (G.status != SCLAP_OK && G.status != SCLAP_EINFEASIBLE) continue;
      if (G.status != SCLAP_OK && first_err == SCLAP_OK) first_err = G.status;
    }
    stream_sync(s);
  });
  return rc != SCLAP_OK ? rc : first_err;
}

int sclap_lp_round(int32_t mode, int64_t n, const int64_t* row_ptr, const int32_t* col,
                   const int32_t* node_w, const int32_t* edge_w, int32_t* label, int64_t* W,
                   int64_t nlabels, int64_t bound, uint64_t rkey, int32_t sub_rounds,
                   const uint8_t* active_cur, uint8_t* active_next, int64_t* moved_out,
                   void* stream) {
  return guarded([&] {
    if (mode != 0 && mode != 1) throw Error(SCLAP_EINVAL, "mode must be 0 or 1");
    if (n < 1 || !row_ptr || !col || !label || !W || nlabels < 1 || sub_rounds < 1 ||
        sub_rounds > 64)
      throw Error(SCLAP_EINVAL, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    GIn g;
    g.n = n; g.m = device_arcs(row_ptr, n, s); g.row_ptr = row_ptr; g.col = col; g.nw = node_w;
    g.ew = edge_w;
    check_col(g.col, g.m);
    int64_t cV, maxc;
    bool nar = false;
    validate(g, s, &cV, &maxc, &nar);
    if (mode == 0 && nlabels < n) throw Error(SCLAP_EINVAL, "clustering needs nlabels >= n");
    check_range(label, n, 0, nlabels, s, "label");
    Level L;
    single_level(g, L, s);
    L.narrow = nar;
    Slots sl(s, 1, L.noff_d.p, {0}, {bound}, {rkey}, {0}, {(int32_t)nlabels}, {0});
    LPRun run;
    run.mode = mode == 0 ? MODE_CLUSTER : MODE_REFINE;
    run.rounds = 1;
    run.sub_rounds = sub_rounds;
    run.stop_rule = false;
    run.raw_key = true;
    DevBuf<int32_t> d_err(1, s);
    d_err.zero();
    DevBuf<wgt_t> W32(nlabels, s);
    k_narrow<<<grid_for(nlabels, 256, 1024), 256, 0, s>>>(W, nlabels, W32.p, d_err.p); SCLAP_NOTE_LAUNCH("k_narrow");
    check_err(d_err.p, s);
    lp_run(L.view(), sl.sp, label, W32.p, nlabels, run, d_err.p, s, active_cur, active_next);
    k_widen<<<grid_for(nlabels, 256, 1024), 256, 0, s>>>(W32.p, nlabels, W); SCLAP_NOTE_LAUNCH("k_widen");
    check_err(d_err.p, s);
    int64_t mv = 0;
    SCLAP_CUDA(cudaMemcpyAsync(&mv, sl.moved.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    stream_sync(s);
    if (moved_out) *moved_out = mv;
  });
}

int sclap_cluster(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* node_w,
                  const int32_t* edge_w, int64_t U, uint64_t seed, int32_t level,
                  const sclap_config* cfg, int32_t* label_out, int32_t* rounds_out,
                  void* stream) {
  return guarded([&] {
    if (n < 1 || !row_ptr || !col || !label_out) throw Error(SCLAP_EINVAL, "bad argument");
    const sclap_config c = resolve_cfg(cfg);
    cudaStream_t s = (cudaStream_t)stream;
    GIn g;
    g.n = n; g.m = device_arcs(row_ptr, n, s); g.row_ptr = row_ptr; g.col = col; g.nw = node_w;
    g.ew = edge_w;
    check_col(g.col, g.m);
    int64_t cV, maxc;
    bool nar = false;
    validate(g, s, &cV, &maxc, &nar);
    Level L;
    single_level(g, L, s);
    L.narrow = nar;
    Slots sl(s, 1, L.noff_d.p, {0}, {U}, {seed}, {level}, {0}, {0});
    DevBuf<wgt_t> W(n, s);
    k_iota<<<grid_for(n, 256, (int64_t)num_sms() * 16), 256, 0, s>>>(label_out, n); SCLAP_NOTE_LAUNCH("k_iota");
    k_w_from_nw<<<grid_for(n, 256, (int64_t)num_sms() * 16), 256, 0, s>>>(L.nwp(), n, W.p); SCLAP_NOTE_LAUNCH("k_w_from_nw");
    LPRun run;
    run.mode = MODE_CLUSTER;
    run.phase = PH_CLUSTER;
    run.rounds = c.lp_rounds_coarse;
    run.sub_rounds = c.sub_rounds;
    run.graph = c.graph_rounds != 0;
    run.use_active = c.cluster_active != 0;
    DevBuf<int32_t> d_err(1, s);
    d_err.zero();
    lp_run(L.view(), sl.sp, label_out, W.p, n, run, d_err.p, s);
    check_err(d_err.p, s);
    if (rounds_out) *rounds_out = sl.host_rounds(s)[0];
  });
}

int sclap_cluster_hierarchy(int64_t n, const int64_t* row_ptr, const int32_t* col,
                            const int32_t* node_w, const int32_t* edge_w, int64_t U,
                            int64_t stop_nodes, uint64_t seed, const sclap_config* cfg,
                            int32_t* comm_out, int32_t* levels_out, int64_t* level_n_out,
                            int32_t cap, void* stream) {
  return guarded([&] {
    if (n < 1 || n >= ((int64_t)1 << 31) || !row_ptr || !comm_out || U < 1)
      throw Error(SCLAP_EINVAL, "bad argument");
    const sclap_config c = resolve_cfg(cfg);
    cudaStream_t s = (cudaStream_t)stream;
    GIn g;
    g.n = n; g.m = device_arcs(row_ptr, n, s); g.row_ptr = row_ptr; g.col = col; g.nw = node_w;
    g.ew = edge_w;
    check_col(g.col, g.m);
    int64_t cV, maxc;
    bool nar = false;
    validate(g, s, &cV, &maxc, &nar);
    const int sms = num_sms();
    std::unique_ptr<Level> cur(new Level());
    single_level(g, *cur, s);
    cur->narrow = nar;
    k_iota<<<grid_for(n, 256, (int64_t)sms * 16), 256, 0, s>>>(comm_out, n); SCLAP_NOTE_LAUNCH("k_iota");
    int32_t levels = 0;
    if (level_n_out && cap > 0) level_n_out[0] = n;
    DevBuf<int32_t> d_err(1, s);
    d_err.zero();
    while (cur->N > stop_nodes && levels + 1 < c.max_levels) {
      const LevelView v = cur->view();
      Slots sl(s, 1, cur->noff_d.p, {0}, {U}, {seed}, {levels}, {0}, {0});
      DevBuf<int32_t> label(v.N, s);
      DevBuf<wgt_t> W(v.N, s);
      k_iota<<<grid_for(v.N, 256, (int64_t)sms * 16), 256, 0, s>>>(label.p, v.N); SCLAP_NOTE_LAUNCH("k_iota");
      k_w_from_nw<<<grid_for(v.N, 256, (int64_t)sms * 16), 256, 0, s>>>(v.nw, v.N, W.p); SCLAP_NOTE_LAUNCH("k_w_from_nw");
      LPRun run;
      run.mode = MODE_CLUSTER;
      run.phase = PH_CLUSTER;
      run.rounds = c.lp_rounds_coarse;
      run.sub_rounds = c.sub_rounds;
      run.graph = c.graph_rounds != 0;
      run.use_active = c.cluster_active != 0;
      lp_run(v, sl.sp, label.p, W.p, v.N, run, d_err.p, s);
      ContractWork cw;
      std::vector<int64_t> nc;
      contract_rank(v, cur->noff, label.p, cw, nc, s);
      if (20 * (v.N - nc[0]) < v.N) break;          // shrink below 5%: discarded
      cur->cmap.alloc(v.N, s);
      CoarseLevel co;
      contract_build(v, cur->noff, label.p, cw, {1}, cur->cmap.p, co, d_err.p, s);
      k_compose<<<grid_for(n, 256, (int64_t)sms * 16), 256, 0, s>>>(comm_out, cur->cmap.p, n); SCLAP_NOTE_LAUNCH("k_compose");
      std::unique_ptr<Level> nx(new Level());
      nx->narrow = cur->narrow;
      nx->N = co.N;
      nx->M = co.M;
      nx->row_ptr = std::move(co.row_ptr);
      nx->col = std::move(co.col);
      nx->ew = std::move(co.ew);
      nx->nw = std::move(co.nw);
      nx->gid = std::move(co.gid);
      nx->noff_d = std::move(co.noff_d);
      nx->noff = co.noff;
      nx->aoff = co.aoff;
      cur = std::move(nx);
      ++levels;
      if (level_n_out && levels < cap) level_n_out[levels] = cur->N;
    }
    check_err(d_err.p, s);
    stream_sync(s);
    if (levels_out) *levels_out = levels;
  });
}

int sclap_contract(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* node_w,
                   const int32_t* edge_w, const int32_t* label, int32_t* cmap, int64_t* nc_out,
                   int32_t* cnode_w, int64_t* crow_ptr, int32_t* ccol, int32_t* cedge_w,
                   int64_t* mc_out, void* stream) {
  return guarded([&] {
    if (n < 1 || !row_ptr || !col || !label || !cmap || !cnode_w || !crow_ptr || !ccol ||
        !cedge_w)
      throw Error(SCLAP_EINVAL, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    GIn g;
    g.n = n; g.m = device_arcs(row_ptr, n, s); g.row_ptr = row_ptr; g.col = col; g.nw = node_w;
    g.ew = edge_w;
    check_col(g.col, g.m);
    int64_t cV, maxc;
    bool nar = false;
    validate(g, s, &cV, &maxc, &nar);
    check_range(label, n, 0, n, s, "label");
    Level L;
    single_level(g, L, s);
    L.narrow = nar;
    ContractWork w;
    std::vector<int64_t> nc;
    contract_rank(L.view(), L.noff, label, w, nc, s);
    CoarseLevel co;
    DevBuf<int32_t> d_err(1, s);
    d_err.zero();
    contract_build(L.view(), L.noff, label, w, {1}, cmap, co, d_err.p, s);
    check_err(d_err.p, s);
    SCLAP_CUDA(cudaMemcpyAsync(cnode_w, co.nw.p, co.N * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    SCLAP_CUDA(cudaMemcpyAsync(crow_ptr, co.row_ptr.p, (co.N + 1) * sizeof(int64_t),
                               cudaMemcpyDeviceToDevice, s));
    if (co.M > 0) {
      SCLAP_CUDA(cudaMemcpyAsync(ccol, co.col.p, co.M * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
      SCLAP_CUDA(cudaMemcpyAsync(cedge_w, co.ew.p, co.M * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
    stream_sync(s);
    if (nc_out) *nc_out = co.N;
    if (mc_out) *mc_out = co.M;
  });
}

int sclap_initial_partition(int64_t n, const int64_t* row_ptr, const int32_t* col,
                            const int32_t* node_w, const int32_t* edge_w, int32_t k,
                            int64_t Lmax, int64_t avg, uint64_t seed, int32_t level,
                            const sclap_config* cfg, int32_t* block_out, int64_t* cut_out,
                            int32_t* best_trial_out, void* stream) {
  return guarded([&] {
    if (n < 1 || !row_ptr || !col || !block_out || k < 1 || k > n)
      throw Error(SCLAP_EINVAL, "bad argument");
    const sclap_config c = resolve_cfg(cfg);
    cudaStream_t s = (cudaStream_t)stream;
    GIn g;
    g.n = n; g.m = device_arcs(row_ptr, n, s); g.row_ptr = row_ptr; g.col = col; g.nw = node_w;
    g.ew = edge_w;
    check_col(g.col, g.m);
    int64_t cV, maxc;
    bool nar = false;
    validate(g, s, &cV, &maxc, &nar);
    Level L;
    single_level(g, L, s);
    L.narrow = nar;
    DevBuf<wgt_t> Wg(k, s);
    DevBuf<int32_t> d_err(1, s);
    d_err.zero();
    std::vector<IPIn> in{IPIn{&L, 0, k, Lmax, avg, seed, level, 0, block_out}};
    std::vector<int32_t> best;
    std::vector<int64_t> ipcut;
    int64_t arcs = 0;
    run_ip(in, c, Wg.p, best, ipcut, &arcs, d_err.p, s);
    check_err(d_err.p, s);
    if (cut_out) *cut_out = ipcut[0];
    if (best_trial_out) *best_trial_out = best[0];
  });
}

int sclap_refine(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* node_w,
                 const int32_t* edge_w, int32_t k, int64_t Lmax, uint64_t seed, int32_t phase,
                 int32_t level, const sclap_config* cfg, int32_t* block, int32_t* rounds_out,
                 void* stream) {
  return guarded([&] {
    if (n < 1 || !row_ptr || !col || !block || k < 1) throw Error(SCLAP_EINVAL, "bad argument");
    const sclap_config c = resolve_cfg(cfg);
    cudaStream_t s = (cudaStream_t)stream;
    GIn g;
    g.n = n; g.m = device_arcs(row_ptr, n, s); g.row_ptr = row_ptr; g.col = col; g.nw = node_w;
    g.ew = edge_w;
    check_col(g.col, g.m);
    int64_t cV, maxc;
    bool nar = false;
    validate(g, s, &cV, &maxc, &nar);
    check_range(block, n, 0, k, s, "block");
    Level L;
    single_level(g, L, s);
    L.narrow = nar;
    DevBuf<wgt_t> W(k, s);
    W.zero();
    block_weights(block, L.nwp(), n, W.p, s);
    Slots sl(s, 1, L.noff_d.p, {0}, {Lmax}, {seed}, {level}, {k}, {0});
    LPRun run;
    run.mode = MODE_REFINE;
    run.phase = phase;
    run.rounds = c.lp_rounds_refine;
    run.sub_rounds = c.sub_rounds;
    run.graph = c.graph_rounds != 0;
    run.use_active = true;
    DevBuf<int32_t> d_err(1, s);
    d_err.zero();
    lp_run(L.view(), sl.sp, block, W.p, k, run, d_err.p, s);
    check_err(d_err.p, s);
    if (rounds_out) *rounds_out = sl.host_rounds(s)[0];
  });
}

int sclap_cut(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* edge_w,
              const int32_t* block, int64_t* cut_out, void* stream) {
  return guarded([&] {
    if (n < 1 || !row_ptr || !col || !block) throw Error(SCLAP_EINVAL, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    GIn g;
    g.n = n; g.m = device_arcs(row_ptr, n, s); g.row_ptr = row_ptr; g.col = col; g.ew = edge_w;
    check_col(g.col, g.m);
    int64_t cV, maxc;
    bool nar = false;
    validate(g, s, &cV, &maxc, &nar);
    Level L;
    single_level(g, L, s);
    L.narrow = nar;
    DevBuf<int64_t> cut2(1, s);
    cut2.zero();
    slot_cut(L.view(), block, cut2.p, s);
    int64_t c2 = 0;
    SCLAP_CUDA(cudaMemcpyAsync(&c2, cut2.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    stream_sync(s);
    if (cut_out) *cut_out = c2 / 2;
  });
}

int sclap_check_build(void) {
#if defined(SCLAP_CHECK) && SCLAP_CHECK
  return 1;
#else
  return 0;
#endif
}

int sclap_check_selftest(void* stream) {
  return guarded([&] {
#if defined(SCLAP_CHECK) && SCLAP_CHECK
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevBuf<int32_t> buf(4, s), out(2, s), err(2, s);
    const std::vector<int32_t> init{10, 11, 12, 13};
    buf.upload(init);
    err.zero();
    k_check_selftest<<<1, 1, 0, s>>>(buf.p, 4, out.p, err.p); SCLAP_NOTE_LAUNCH("k_check_selftest");
    SCLAP_LAUNCH_CHECK();
    int32_t h[4] = {0, 0, 0, 0};
    SCLAP_CUDA(cudaMemcpyAsync(h, out.p, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SCLAP_CUDA(cudaMemcpyAsync(h + 2, err.p, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    stream_sync(s);
    if (h[0] != 13 || h[1] != 0 || h[2] != 0 || h[3] != DERR_BOUNDS)
      throw Error(SCLAP_EINTERNAL, "bounds-check self test failed");
#else
    (void)stream;
    throw Error(SCLAP_EINVAL, "not a bounds-check build");
#endif
  });
}

int sclap_debug_inject(int64_t wait, int64_t probe, int32_t fail_allocs) {
  return guarded([&] {
    if (wait < 0 || probe < 0 || fail_allocs < 0 || wait > 0xffffffffll || probe > 0xffffffffll)
      throw Error(SCLAP_EINVAL, "fault-injection value out of range");
    debug_inject(wait == 0 ? (1u << 22) : (uint32_t)wait,
                 probe == 0 ? 0xffffffffu : (uint32_t)probe, fail_allocs);
  });
}

void sclap_get_tuning(sclap_tuning* out) {
  if (!out) return;
  const Tuning t = tuning_get();
  out->small_max_deg = t.small_max_deg;
  out->small_ctas_per_sm = t.small_ctas_per_sm;
  out->warp_ctas_per_sm = t.warp_ctas_per_sm;
  out->admit_ctas_per_sm = t.admit_ctas_per_sm;
  out->concurrent = t.concurrent;
  out->pdl = t.pdl;
  out->fused_admission = t.fused_admission;
  out->contract_table_slots = t.contract_table_slots;
  out->ip_trial_group = t.ip_trial_group;
  out->contract_merge = t.contract_merge;
}

int sclap_set_tuning(const sclap_tuning* in) {
  return guarded([&] {
    if (!in) throw Error(SCLAP_EINVAL, "NULL tuning");
    if ((in->small_max_deg != 8 && in->small_max_deg != 16) || in->small_ctas_per_sm < 1 ||
        in->small_ctas_per_sm > 32 || in->warp_ctas_per_sm < 1 || in->warp_ctas_per_sm > 32 ||
        in->admit_ctas_per_sm < 1 || in->admit_ctas_per_sm > 64 || in->concurrent < 0 ||
        in->concurrent > 1 || in->pdl < 0 || in->pdl > 1 || in->fused_admission < 0 ||
        in->fused_admission > 1 || in->contract_table_slots < 0 || in->ip_trial_group < 0 ||
        in->contract_merge < 0 || in->contract_merge > 1)
      throw Error(SCLAP_EINVAL, "tuning value out of range");
    Tuning t;
    t.small_max_deg = in->small_max_deg;
    t.small_ctas_per_sm = in->small_ctas_per_sm;
    t.warp_ctas_per_sm = in->warp_ctas_per_sm;
    t.admit_ctas_per_sm = in->admit_ctas_per_sm;
    t.concurrent = in->concurrent;
    t.pdl = in->pdl;
    t.fused_admission = in->fused_admission;
    t.contract_table_slots = in->contract_table_slots;
    t.ip_trial_group = in->ip_trial_group;
    t.contract_merge = in->contract_merge;
    tuning_set(t);
  });
}

int sclap_autotune(int32_t count, sclap_graph* graphs, const sclap_config* cfg,
                   int32_t device_ptrs, int32_t reps, sclap_tuning* out, void* stream) {
  return guarded([&] {
    if (count < 1 || !graphs || reps < 1) throw Error(SCLAP_EINVAL, "bad argument");
    const sclap_config c = resolve_cfg(cfg);
    std::vector<int64_t> ref(count);
    auto run_once = [&](const Tuning& t, bool record) -> double {
      tuning_set(t);
      const auto t0 = std::chrono::steady_clock::now();
      const int rc = sclap_partition_batch(count, graphs, &c, device_ptrs, stream);
      const double ms =
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (rc != SCLAP_OK && rc != SCLAP_EINFEASIBLE) throw Error(rc, "autotune: a run failed");
      for (int32_t i = 0; i < count; ++i) {
        if (record) ref[i] = graphs[i].cut;
        else if (graphs[i].cut != ref[i])
          throw Error(SCLAP_EINTERNAL, "autotune: a setting changed a result");
      }
      return ms;
    };
    auto measure = [&](const Tuning& t) {
      std::vector<double> ms;
      for (int32_t r = 0; r < reps; ++r) ms.push_back(run_once(t, false));
      std::sort(ms.begin(), ms.end());
      return ms[ms.size() / 2];
    };
    const Tuning start = tuning_get();
    Tuning best = start;
    try {
      run_once(best, true);                       // warm-up, reference results
      double best_ms = measure(best);
      struct Param { int32_t Tuning::*f; std::vector<int32_t> vals; };
      const Param params[] = {
          {&Tuning::small_max_deg, {16, 8}},
          {&Tuning::small_ctas_per_sm, {4, 8, 16}},
          {&Tuning::warp_ctas_per_sm, {4, 8, 16}},
          {&Tuning::admit_ctas_per_sm, {8, 16, 32}},
          {&Tuning::concurrent, {1, 0}},
          {&Tuning::pdl, {1, 0}},
          {&Tuning::fused_admission, {0, 1}},
          {&Tuning::contract_merge, {0, 1}},
      };
      for (const Param& p : params) {
        for (int32_t v : p.vals) {
          if (best.*(p.f) == v) continue;
          Tuning t = best;
          t.*(p.f) = v;
          const double ms = measure(t);
          if (ms < 0.98 * best_ms) {
            best = t;
            best_ms = ms;
          }
        }
      }
    } catch (...) {
      tuning_set(start);
      throw;
    }
    tuning_set(best);
    if (out) sclap_get_tuning(out);
  });
}

void sclap_profile_enable(int on) { profile().enabled.store(on != 0); }

void sclap_profile_timeline(int on) { profile().timeline.store(on != 0); }

int64_t sclap_profile_dump(char* buf, int64_t cap) {
  const std::string t = timeline_dump();
  if (buf && cap > 0) {
    const int64_t n = std::min<int64_t>(cap - 1, (int64_t)t.size());
    std::memcpy(buf, t.data(), (size_t)n);
    buf[n] = 0;
  }
  return (int64_t)t.size() + 1;
}

void sclap_profile_reset(void) {
  ProfileState& P = profile();
  std::lock_guard<std::mutex> lk(P.mu);
  P.launches.store(0);
  for (int b = 0; b < 4; ++b) { P.ms[b] = 0; P.nlaunch[b] = 0; P.nodes[b] = 0; P.arcs[b] = 0; }
  P.arcs_unit = 0;
  P.sweep_ms = 0;
  P.sweeps = 0;
  P.phases.clear();
}

int64_t sclap_profile_phases(double* out, int64_t cap) {
  ProfileState& P = profile();
  std::lock_guard<std::mutex> lk(P.mu);
  const int64_t n = (int64_t)P.phases.size() / 7;
  if (out && cap > 0) {
    const int64_t m = std::min(n, cap);
    std::memcpy(out, P.phases.data(), (size_t)(m * 7) * sizeof(double));
  }
  return n;
}

void sclap_profile_read(sclap_profile* out) {
  if (!out) return;
  ProfileState& P = profile();
  std::lock_guard<std::mutex> lk(P.mu);
  out->kernel_launches = P.launches.load();
  for (int b = 0; b < 4; ++b) {
    out->propose_launches[b] = P.nlaunch[b];
    out->propose_ms[b] = P.ms[b];
    out->propose_nodes[b] = P.nodes[b];
    out->propose_arcs[b] = P.arcs[b];
  }
  out->sweep_ms = P.sweep_ms;
  out->sweeps = P.sweeps;
  out->propose_arcs_unit = P.arcs_unit;
}

}  // extern "C"
