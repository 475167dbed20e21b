// contract.cu -- cluster contraction (Sec. 3.1) for every slot of a level.
//
// Each cluster becomes one coarse node (id = rank of its label, contiguous
// per slot); its weight is the sum of its members; two coarse nodes are
// adjacent iff their clusters are, with the summed weight of the fine edges
// between them.  GPU plan: rank the labels by a scan; stream the fine arcs in
// node order (warp per 32 nodes, arcs flattened across lanes) once to count
// each coarse node's inter-cluster arcs, size one open-addressing region per
// coarse node from that count (next_pow2 of it: the distinct coarse
// neighbours never outnumber the arcs, and are usually far fewer), stream the arcs again inserting (coarse
// neighbour, weight) with one 64-bit CAS or atomic add each (a claim also
// records the slot's owner and counts its degree), scan the degrees into row
// offsets, and place every occupied slot in its owner's row.  The order of a
// row's arcs is not fixed, which no later step depends on; all sums are
// integer, hence deterministic.  An alternative path (tuning contract_merge)
// replaces the global table by member lists and per-coarse-node merges in
// shared memory (the contraction by segments below) wherever its regions
// fit in memory; it measured slower than the hash tables.
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace sclap {
namespace {

__global__ void k_mark(const int32_t* __restrict__ label, int64_t N, int32_t* __restrict__ flag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x)
    flag[label[v]] = 1;
}

__global__ void k_gather(const int64_t* __restrict__ src, const int64_t* __restrict__ idx, int n,
                         int64_t* __restrict__ dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

struct CArgs {
  const int64_t* row_ptr;
  const int32_t* col;
  const int32_t* ew;
  const int32_t* nw;
  const int32_t* gid;
  const int32_t* label;
  const int64_t* cid;
  const int64_t* delta;
  const uint8_t* keep;
  int32_t* cmap;
  int32_t* cnw;
  int32_t* inter;          // inter-cluster arcs per coarse node
  const int64_t* tbase;    // table region of each coarse node
  unsigned long long* tslot;   // (coarse neighbour << 32) | summed weight; ~0 = empty
  int32_t* cdeg;           // distinct coarse neighbours per coarse node (slots claimed)
  int32_t* towner;         // coarse node owning each claimed slot
  int32_t* err;
  // pass of the table build: only sources with coarse id in [c_lo, c_hi)
  // insert, into the table regions of that range, which start at toff
  int32_t c_lo, c_hi;
  int64_t toff;
  // no coarse arc weight can exceed INT32_MAX (level's total arc weight
  // bounds it): adds need no overflow check, so they do not wait for the
  // old value
  bool sums31;
  // rows longer than `heavy` arcs are left to the heavy-row kernels (split
  // into chunks over many CTAs); 0: no split
  int64_t heavy;
  int64_t N, Nc;     // fine and coarse nodes (array lengths for bounds checks)
};

__global__ void k_map(CArgs a, int64_t N) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = slot_at(a.gid, v);
    if (!a.keep[s]) { a.cmap[v] = -1; continue; }
    const int32_t c = (int32_t)(SCLAP_LD(a.cid, a.label[v], a.N + 1, a.err) + a.delta[s]);
    a.cmap[v] = c;
    if (SCLAP_OK(c, a.Nc, a.err)) atomicAdd(&a.cnw[c], wat(a.nw, v));
  }
}

// Visits every arc (v, u) of the level with cmap[v] >= 0, 32 source nodes per
// warp, the arcs of those nodes spread over the lanes; calls f(cv, cu, w) on
// every lane (cu = -1 on lanes without an inter-cluster arc) so the warp can
// cooperate.
template <class F>
__device__ __forceinline__ void for_inter_arcs(const CArgs& a, int64_t N, F f) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = w0 * 32; base < N; base += nwarps * 32) {
    const int64_t v = base + lane;
    int64_t rs = 0, d = 0;
    int32_t cv = -1;
    if (v < N) {
      cv = a.cmap[v];
      if (cv >= a.c_lo && cv < a.c_hi) {
        rs = a.row_ptr[v];
        d = a.row_ptr[v + 1] - rs;
        if (a.heavy > 0 && d > a.heavy) d = 0;     // a heavy row: chunked elsewhere
      }
    }
    long long incl = d;
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const long long excl = incl - d;
    const long long total = __shfl_sync(0xffffffffu, incl, 31);
    for (long long x0 = 0; x0 < total; x0 += 32) {
      const long long x = x0 + lane;
      int L = 0;
      for (int step = 16; step > 0; step >>= 1) {
        long long y = __shfl_sync(0xffffffffu, incl, L + step - 1);
        if (y <= x) L += step;
      }
      const long long rsL = __shfl_sync(0xffffffffu, (long long)rs, L);
      const long long exL = __shfl_sync(0xffffffffu, excl, L);
      const int32_t cvL = __shfl_sync(0xffffffffu, cv, L);
      int32_t cu = -1, w = 0;
      if (x < total) {
        const int64_t e = rsL + (x - exL);
        cu = SCLAP_LD(a.cmap, a.col[e], a.N, a.err);
        if (cu == cvL) cu = -1;
        else w = wat(a.ew, e);
      }
      f(cvL, cu, w);
    }
  }
}

// Inter-cluster arcs per coarse node.  The lanes' arcs are in source order,
// so lanes with the same coarse source form runs of consecutive lanes; two
// ballots give each run's count and its last lane adds it (runs with equal
// sources that are not adjacent simply add separately).
__global__ void __launch_bounds__(256) k_count_inter(CArgs a, int64_t N) {
  const int lane = threadIdx.x & 31;
  for_inter_arcs(a, N, [&](int32_t cv, int32_t cu, int32_t) {
    const unsigned inter = __ballot_sync(0xffffffffu, cu >= 0);
    const int32_t prev = __shfl_up_sync(0xffffffffu, cv, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != cv);
    const bool last = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (last) {
      const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);   // lanes 0..lane
      const int first = 31 - __clz(heads & upto);                               // run start
      const int c = __popc(inter & upto & ~((1u << first) - 1u));
      if (c && SCLAP_OK(cv, a.Nc, a.err)) atomicAdd(&a.inter[cv], c);
    }
  });
}

__global__ void k_table_caps(const int32_t* __restrict__ inter, int64_t Nc, int64_t* __restrict__ cap) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < Nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = inter[c];
    cap[c] = x > 0 ? ((int64_t)1 << ceil_log2((int64_t)x)) : 0;
  }
}

// A slot packs (coarse neighbour, summed weight) in one 64-bit word: the
// first arc claims an empty slot with one CAS carrying its weight, later arcs
// add to the low half with one atomicAdd.  A coarse edge weight must fit in
// int32, so a sum reaching 2^31 is reported (and cannot carry into the key).
__device__ __forceinline__ void insert_arc(const CArgs& a, int32_t cv, int32_t cu, int32_t w) {
  if (!SCLAP_OK(cv, a.Nc, a.err) || !SCLAP_OK(cu, a.Nc, a.err)) return;
  const int64_t sum = w;
  const int64_t base = a.tbase[cv] - a.toff;
  const int logcap = ceil_log2(a.tbase[cv + 1] - a.tbase[cv]);
  const uint32_t mask = (1u << logcap) - 1;
  uint32_t sl = table_slot(cu, logcap);
  const unsigned long long mine = ((unsigned long long)(uint32_t)cu << 32) | (uint64_t)sum;
  for (uint32_t p = 0; p <= mask; ++p) {
    unsigned long long* slot = &a.tslot[base + sl];
    unsigned long long cur = *slot;
    if (cur == ~0ull) {
      cur = atomicCAS(slot, ~0ull, mine);
      if (cur == ~0ull) {            // claimed: one more coarse arc of cv
        a.towner[base + sl] = cv;
        atomicAdd(&a.cdeg[cv], 1);
        return;
      }
    }
    if ((uint32_t)(cur >> 32) == (uint32_t)cu) {
      if (a.sums31) {
        atomicAdd(slot, (unsigned long long)sum);
        return;
      }
      const unsigned long long old = atomicAdd(slot, (unsigned long long)sum);
      if ((old & 0xffffffffull) + (unsigned long long)sum > (unsigned long long)INT32_MAX)
        atomicOr(a.err, DERR_W_OVERFLOW);
      return;
    }
    sl = (sl + 1) & mask;
  }
  atomicOr(a.err, DERR_HASH_FULL);
}

__global__ void __launch_bounds__(256) k_insert(CArgs a, int64_t N) {
  for_inter_arcs(a, N, [&](int32_t cv, int32_t cu, int32_t w) {
    if (cu >= 0) insert_arc(a, cv, cu, w);
  });
}

// Heavy rows (more than `heavy` arcs, cmap >= 0): listed once per level,
// then cut into chunks of HV_CH arcs (hoff: exclusive scan of the chunks
// per listed row) that CTAs take in turn, so that a hub's row is spread
// over the whole grid instead of being one warp's serial job.
constexpr int HV_CH = 2048;

__global__ void k_heavy_list(CArgs a, int64_t N, int32_t* __restrict__ list, int32_t* cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x; v0 < N; v0 += stride) {
    const int64_t v = v0 + threadIdx.x;
    const bool h = v < N && a.cmap[v] >= 0 && a.row_ptr[v + 1] - a.row_ptr[v] > a.heavy;
    const unsigned m = __ballot_sync(0xffffffffu, h);
    if (!m) continue;
    int q0 = 0;
    if (lane == 0) q0 = atomicAdd(cnt, __popc(m));
    q0 = __shfl_sync(0xffffffffu, q0, 0);
    if (h) list[q0 + __popc(m & ((1u << lane) - 1))] = (int32_t)v;
  }
}
__global__ void k_heavy_chunks(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ list,
                               int32_t nh, int32_t* __restrict__ nch) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nh; i += gridDim.x * blockDim.x) {
    const int32_t v = list[i];
    nch[i] = (int32_t)((row_ptr[v + 1] - row_ptr[v] + HV_CH - 1) / HV_CH);
  }
}

// Calls f(cv, cu, w) for every arc of every chunk this CTA takes (cu = -1
// for an arc inside the cluster); all threads of the CTA loop alike.
template <class F>
__device__ __forceinline__ void for_heavy_arcs(const CArgs& a, const int32_t* __restrict__ list,
                                               const int64_t* __restrict__ hoff, int32_t nh, F f) {
  const int64_t total = hoff[nh];
  for (int64_t q = blockIdx.x; q < total; q += gridDim.x) {
    int32_t lo = 0, hi = nh - 1;           // last list position i with hoff[i] <= q
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (hoff[mid] <= q) lo = mid;
      else hi = mid - 1;
    }
    const int32_t v = list[lo];
    const int32_t cv = a.cmap[v];
    if (cv < a.c_lo || cv >= a.c_hi) continue;
    const int64_t e0 = a.row_ptr[v] + (q - hoff[lo]) * HV_CH;
    const int64_t e1 = min(e0 + HV_CH, a.row_ptr[v + 1]);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      int32_t cu = SCLAP_LD(a.cmap, a.col[e], a.N, a.err);
      int32_t w = 0;
      if (cu == cv) cu = -1;
      else w = wat(a.ew, e);
      f(cv, cu, w);
    }
  }
}

__global__ void __launch_bounds__(256) k_count_heavy(CArgs a, const int32_t* __restrict__ list,
                                                     const int64_t* __restrict__ hoff, int32_t nh) {
  // a chunk belongs to one row, so one coarse source: count per thread,
  // reduce per warp, one atomic per warp and chunk
  const int lane = threadIdx.x & 31;
  const int64_t total = hoff[nh];
  for (int64_t q = blockIdx.x; q < total; q += gridDim.x) {
    int32_t lo = 0, hi = nh - 1;
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (hoff[mid] <= q) lo = mid;
      else hi = mid - 1;
    }
    const int32_t v = list[lo];
    const int32_t cv = a.cmap[v];
    const int64_t e0 = a.row_ptr[v] + (q - hoff[lo]) * HV_CH;
    const int64_t e1 = min(e0 + HV_CH, a.row_ptr[v + 1]);
    int c = 0;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x)
      c += SCLAP_LD(a.cmap, a.col[e], a.N, a.err) != cv;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0 && c && SCLAP_OK(cv, a.Nc, a.err)) atomicAdd(&a.inter[cv], c);
  }
}

__global__ void __launch_bounds__(256) k_insert_heavy(CArgs a, const int32_t* __restrict__ list,
                                                      const int64_t* __restrict__ hoff, int32_t nh) {
  for_heavy_arcs(a, list, hoff, nh, [&](int32_t cv, int32_t cu, int32_t w) {
    if (cu >= 0) insert_arc(a, cv, cu, w);
  });
}

// Coarse rows: one thread per table slot; an occupied slot goes to its
// owner's row (offsets from a scan of the claimed-slot counts) at a position
// taken from a per-row counter.  The order of a row's arcs is therefore not
// fixed, as the slot order already was not (concurrent claims in one region
// race); nothing computed from a coarse graph depends on that order.
__global__ void k_emit(const unsigned long long* __restrict__ tslot,
                       const int32_t* __restrict__ towner, const int64_t* __restrict__ crow,
                       int32_t* __restrict__ fill, int64_t T, int32_t* __restrict__ ccol,
                       int32_t* __restrict__ cew) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < T;
       j += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long x = tslot[j];
    if (x == ~0ull) continue;
    const int32_t c = towner[j];
    const int64_t p = crow[c] + atomicAdd(&fill[c], 1);
    ccol[p] = (int32_t)(x >> 32);
    cew[p] = (int32_t)(x & 0xffffffffull);
  }
}

// ------------------------------------------------------------------------
// Contraction by segments: the fine nodes are counting-sorted by coarse id
// (member lists), and the inter-cluster arcs of each coarse node's members
// are merged into (coarse neighbour, summed weight) pairs.  Three classes,
// by the node's inter-cluster arcs x and its members' arcs t (the work):
//   warp   x <= MW_MAX, t <= MW_ARCS: one warp, table in shared memory;
//   CTA    x <= MB_MAX, t <= MB_ARCS: one CTA, table in shared memory;
//   large  the rest: the members' arcs of all large nodes are spread evenly
//          over the grid and inserted into per-node regions of a global
//          table (next_pow2(x) slots), which one CTA per node then reads.
// Each node writes its distinct pairs into a region of its own (offsets: the
// scan of x) and its distinct count; the scan of the counts gives the coarse
// row offsets and one pass moves the pairs into the rows.  Global atomics
// remain only for the large class.
constexpr int MW_MAX = 64, MW_CAP = 128, MW_LOG = 7, MW_ARCS = 2048;
constexpr int MB_NT = 256, MB_MAX = 2048, MB_CAP = 4096, MB_LOG = 12, MB_ARCS = 32768;
constexpr size_t merge_cta_smem() {
  return (size_t)MB_CAP * 2 * sizeof(int32_t) + (size_t)MB_MAX * sizeof(int32_t);
}

struct MArgs {
  const int64_t* row_ptr;
  const int32_t* col;
  const int32_t* ew;
  const int32_t* cmap;
  const int32_t* members;     // fine nodes by coarse id
  const int64_t* moff;        // [Nc + 1]
  const int32_t* inter;       // x: inter-cluster arcs per coarse node
  const int64_t* marcs;       // t: arcs of the members per coarse node
  const int64_t* soff;        // [Nc + 1] region offsets (scan of x)
  const int64_t* tbase;       // [Nc + 1] global table regions (large nodes only)
  unsigned long long* tslot;  // global table slots (~0 = empty)
  int32_t* rcol;              // regions: coarse neighbour
  int32_t* rew;               //          summed weight
  int32_t* cdeg;              // distinct coarse neighbours per coarse node
  const int32_t* list;        // coarse nodes of the launch's class
  const int32_t* nlist;       // their number
  int32_t* err;
  int64_t Nc;
};

__device__ __forceinline__ bool warp_class(int32_t x, int64_t t) {
  return x > 0 && x <= MW_MAX && t <= MW_ARCS;
}

__global__ void k_member_count(const int32_t* __restrict__ cmap, const int64_t* __restrict__ row_ptr,
                               int64_t N, int32_t* mcnt, unsigned long long* marcs) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cmap[v];
    if (c < 0) continue;
    atomicAdd(&mcnt[c], 1);
    const int64_t d = row_ptr[v + 1] - row_ptr[v];
    if (d) atomicAdd(&marcs[c], (unsigned long long)d);
  }
}
__global__ void k_member_fill(const int32_t* __restrict__ cmap, int64_t N,
                              const int64_t* __restrict__ moff, int32_t* mfill,
                              int32_t* __restrict__ members) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cmap[v];
    if (c >= 0) members[moff[c] + atomicAdd(&mfill[c], 1)] = (int32_t)v;
  }
}

// Lists the CTA-class nodes at lists[0..cnt[0]) and the large ones at
// lists[Nc..Nc + cnt[1]); cap[c] = table slots of node c (large only).
__global__ void k_merge_classes(const int32_t* __restrict__ inter,
                                const int64_t* __restrict__ marcs, int64_t Nc,
                                int32_t* __restrict__ lists, int32_t* cnt,
                                int64_t* __restrict__ cap) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c0 = (int64_t)blockIdx.x * blockDim.x; c0 < Nc; c0 += stride) {
    const int64_t c = c0 + threadIdx.x;
    int cls = -1;
    int32_t x = 0;
    if (c < Nc) {
      x = inter[c];
      const int64_t t = marcs[c];
      cls = (x == 0 || warp_class(x, t)) ? -1 : (x <= MB_MAX && t <= MB_ARCS) ? 0 : 1;
      cap[c] = cls == 1 ? ((int64_t)1 << ceil_log2((int64_t)x)) : 0;
    }
    for (int k = 0; k < 2; ++k) {
      const bool mine = cls == k;
      const unsigned m = __ballot_sync(0xffffffffu, mine);
      if (!m) continue;
      int q0 = 0;
      if (lane == 0) q0 = atomicAdd(&cnt[k], __popc(m));
      q0 = __shfl_sync(0xffffffffu, q0, 0);
      if (mine) lists[(int64_t)k * Nc + q0 + __popc(m & ((1u << lane) - 1))] = (int32_t)c;
    }
  }
}

// The warp's 32 lanes hold one fine node each (rs, d: row start and degree,
// d = 0 for none) with the coarse id cv.  Calls f(cv, cu, w) twice per
// pass over the lanes' arcs, flattened across the warp, two arcs per lane
// and pass so that two gathers are in flight (cu = -1 on lanes without an
// inter-cluster arc).  All lanes call f the same number of times.
template <class F>
__device__ __forceinline__ void flat_arcs(const MArgs& a, int64_t rs, int64_t d, int32_t cv, F f) {
  const int lane = threadIdx.x & 31;
  long long incl = d;
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const long long excl = incl - d;
  const long long total = __shfl_sync(0xffffffffu, incl, 31);
  for (long long x0 = 0; x0 < total; x0 += 64) {
    int64_t e[2];
    int32_t cvs[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long x = x0 + 32 * h + lane;
      int L = 0;
      for (int step = 16; step > 0; step >>= 1) {
        const long long y = __shfl_sync(0xffffffffu, incl, L + step - 1);
        if (y <= x) L += step;
      }
      const long long rsL = __shfl_sync(0xffffffffu, (long long)rs, L);
      const long long exL = __shfl_sync(0xffffffffu, excl, L);
      cvs[h] = __shfl_sync(0xffffffffu, cv, L);
      e[h] = x < total ? rsL + (x - exL) : -1;
    }
    int32_t u[2], cu[2], w[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) u[h] = e[h] >= 0 ? a.col[e[h]] : 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      cu[h] = e[h] >= 0 ? a.cmap[u[h]] : -1;
      if (cu[h] == cvs[h]) cu[h] = -1;
      w[h] = cu[h] >= 0 ? wat(a.ew, e[h]) : 0;
    }
    f(cvs[0], cu[0], w[0]);
    f(cvs[1], cu[1], w[1]);
  }
}

// Calls f(cu, w) (as flat_arcs) for the arcs of the members [m0, m1) of
// coarse node c, 32 members per pass, the warp's next members mstride on.
template <class F>
__device__ __forceinline__ void member_arcs_warp(const MArgs& a, int32_t c, int64_t m0, int64_t m1,
                                                 int64_t mstride, F f) {
  const int lane = threadIdx.x & 31;
  for (int64_t mb = m0; mb < m1; mb += mstride) {
    const int64_t mi = mb + lane;
    int64_t rs = 0, d = 0;
    if (mi < m1) {
      const int32_t v = a.members[mi];
      rs = a.row_ptr[v];
      d = a.row_ptr[v + 1] - rs;
    }
    flat_arcs(a, rs, d, c, [&](int32_t, int32_t cu, int32_t w) { f(cu, w); });
  }
}

// Adds (cu, w) to a shared open-addressing table of (key, weight) pairs;
// returns the slot when this call created the key, else -1.
__device__ __forceinline__ int32_t merge_add(int32_t* keys, int32_t* vals, int logcap, int32_t cu,
                                             int32_t w, int32_t* err) {
  const uint32_t mask = (1u << logcap) - 1;
  uint32_t sl = table_slot(cu, logcap);
  for (uint32_t p = 0; p <= mask; ++p) {
    const int32_t prev = atomicCAS(&keys[sl], -1, cu);
    if (prev == -1 || prev == cu) {
      const int32_t old = atomicAdd(&vals[sl], w);
      if ((int64_t)old + w > INT32_MAX) atomicOr(err, DERR_W_OVERFLOW);
      return prev == -1 ? (int32_t)sl : -1;
    }
    sl = (sl + 1) & mask;
  }
  atomicOr(err, DERR_HASH_FULL);
  return -1;
}

// Warp class: one warp per coarse node.
__global__ void __launch_bounds__(256) k_merge_warp(MArgs a) {
  __shared__ int32_t sk[8][MW_CAP], sv[8][MW_CAP];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* keys = sk[wib];
  int32_t* vals = sv[wib];
  for (int j = lane; j < MW_CAP; j += 32) { keys[j] = -1; vals[j] = 0; }
  __syncwarp();
  const int64_t nwarps = (int64_t)gridDim.x * 8;
  for (int64_t c = (int64_t)blockIdx.x * 8 + wib; c < a.Nc; c += nwarps) {
    if (!warp_class(a.inter[c], a.marcs[c])) continue;
    member_arcs_warp(a, (int32_t)c, a.moff[c], a.moff[c + 1], 32, [&](int32_t cu, int32_t w) {
      if (cu >= 0) merge_add(keys, vals, MW_LOG, cu, w, a.err);
    });
    __syncwarp();
    const int64_t base = a.soff[c];
    int32_t n = 0;
    for (int j0 = 0; j0 < MW_CAP; j0 += 32) {
      const int j = j0 + lane;
      const bool occ = keys[j] >= 0;
      const unsigned m = __ballot_sync(0xffffffffu, occ);
      if (occ) {
        const int q = n + __popc(m & ((1u << lane) - 1));
        a.rcol[base + q] = keys[j];
        a.rew[base + q] = vals[j];
        keys[j] = -1;
        vals[j] = 0;
      }
      n += __popc(m);
    }
    if (lane == 0) a.cdeg[c] = n;
    __syncwarp();
  }
}

// CTA class: one CTA per listed node; a list of the created slots makes the
// read-out and the reset of the table proportional to the distinct count.
__global__ void __launch_bounds__(MB_NT) k_merge_cta(MArgs a) {
  extern __shared__ int32_t msm[];
  __shared__ int32_t sh_n;
  int32_t* keys = msm;
  int32_t* vals = msm + MB_CAP;
  int32_t* made = msm + 2 * MB_CAP;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int j = tid; j < MB_CAP; j += MB_NT) { keys[j] = -1; vals[j] = 0; }
  if (tid == 0) sh_n = 0;
  __syncthreads();
  const int32_t nl = *a.nlist;
  for (int32_t i = blockIdx.x; i < nl; i += gridDim.x) {
    const int32_t c = a.list[i];
    member_arcs_warp(a, c, a.moff[c] + (int64_t)wid * 32, a.moff[c + 1], (int64_t)MB_NT,
                     [&](int32_t cu, int32_t w) {
      const int32_t sl = cu >= 0 ? merge_add(keys, vals, MB_LOG, cu, w, a.err) : -1;
      const unsigned m = __ballot_sync(0xffffffffu, sl >= 0);
      if (m) {
        int q0 = 0;
        const int first = __ffs(m) - 1;
        if (lane == first) q0 = atomicAdd(&sh_n, __popc(m));
        q0 = __shfl_sync(0xffffffffu, q0, first);
        if (sl >= 0) made[q0 + __popc(m & ((1u << lane) - 1))] = sl;
      }
    });
    __syncthreads();
    const int n = sh_n;
    const int64_t base = a.soff[c];
    for (int j = tid; j < n; j += MB_NT) {
      const int32_t sl = made[j];
      a.rcol[base + j] = keys[sl];
      a.rew[base + j] = vals[sl];
      keys[sl] = -1;
      vals[sl] = 0;
    }
    __syncthreads();
    if (tid == 0) {
      a.cdeg[c] = n;
      sh_n = 0;
    }
    __syncthreads();
  }
}

// Large class.  Work comes in chunks so that no node is one CTA's serial
// job: insertion chunks of LM_CH members, read-out chunks of LE_CH table
// slots; per large node (list position i) ich[i] and ech[i] chunks, whose
// exclusive scans ioff / eoff number them.
constexpr int LM_CH = 256, LE_CH = 4096;
constexpr int LT_CAP = 8192, LT_LOG = 13, LT_FILL = 6144;
constexpr size_t merge_large_smem() { return (size_t)LT_CAP * 2 * sizeof(int32_t); }

__global__ void k_large_chunks(const int32_t* __restrict__ list, int32_t nl,
                               const int64_t* __restrict__ moff, const int64_t* __restrict__ tbase,
                               int32_t* __restrict__ ich, int32_t* __restrict__ ech) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nl; i += gridDim.x * blockDim.x) {
    const int32_t c = list[i];
    ich[i] = (int32_t)((moff[c + 1] - moff[c] + LM_CH - 1) / LM_CH);
    ech[i] = (int32_t)((tbase[c + 1] - tbase[c] + LE_CH - 1) / LE_CH);
  }
}

// Last list position i with off[i] <= q (off nondecreasing, off[0] = 0).
__device__ __forceinline__ int32_t chunk_owner(const int64_t* __restrict__ off, int32_t nl, int64_t q) {
  int32_t lo = 0, hi = nl - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= q) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Adds (cu, w) to the region [tb, tb + 2^logcap) of the global table, a slot
// packing (coarse neighbour << 32 | summed weight).
__device__ __forceinline__ void global_add(const MArgs& a, int64_t tb, int logcap, int32_t cu,
                                           int32_t w) {
  const uint32_t mask = (1u << logcap) - 1;
  uint32_t sl = table_slot(cu, logcap);
  const unsigned long long mine = ((unsigned long long)(uint32_t)cu << 32) | (uint32_t)w;
  for (uint32_t q = 0; q <= mask; ++q) {
    unsigned long long* slot = &a.tslot[tb + sl];
    unsigned long long cur = *slot;
    if (cur == ~0ull) {
      cur = atomicCAS(slot, ~0ull, mine);
      if (cur == ~0ull) return;
    }
    if ((uint32_t)(cur >> 32) == (uint32_t)cu) {
      const unsigned long long old = atomicAdd(slot, (unsigned long long)w);
      if ((old & 0xffffffffull) + (unsigned long long)w > (unsigned long long)INT32_MAX)
        atomicOr(a.err, DERR_W_OVERFLOW);
      return;
    }
    sl = (sl + 1) & mask;
  }
  atomicOr(a.err, DERR_HASH_FULL);
}

// Adds (cu, w) to the CTA's shared table unless that would create a key
// beyond LT_FILL of them (then returns false and the caller adds to the
// global table directly).  At most LT_FILL + (threads - 1) keys exist, so
// the table never fills.
__device__ __forceinline__ bool shared_add(int32_t* keys, int32_t* vals, int32_t* made,
                                           int32_t cu, int32_t w, int32_t* err) {
  volatile int32_t* vk = keys;
  uint32_t sl = table_slot(cu, LT_LOG);
  for (int p = 0; p < LT_CAP; ++p) {
    int32_t k = vk[sl];
    if (k == -1) {
      if (*(volatile int32_t*)made >= LT_FILL) return false;
      k = atomicCAS(&keys[sl], -1, cu);
      if (k == -1) atomicAdd(made, 1);
    }
    if (k == -1 || k == cu) {
      const int32_t old = atomicAdd(&vals[sl], w);
      if ((int64_t)old + w > INT32_MAX) atomicOr(err, DERR_W_OVERFLOW);
      return true;
    }
    sl = (sl + 1) & (LT_CAP - 1);
  }
  return false;
}

// Large class, insertion: one CTA per chunk of LM_CH members of one node
// combines the chunk's arcs in shared memory, then adds each distinct
// (neighbour, partial sum) to the node's global region once.
__global__ void __launch_bounds__(MB_NT, 3) k_merge_large(MArgs a, const int64_t* __restrict__ ioff,
                                                       int32_t nl) {
  extern __shared__ int32_t lsm[];
  __shared__ int32_t sh_made;
  int32_t* keys = lsm;
  int32_t* vals = lsm + LT_CAP;
  const int tid = threadIdx.x, wid = tid >> 5;
  for (int j = tid; j < LT_CAP; j += MB_NT) { keys[j] = -1; vals[j] = 0; }
  if (tid == 0) sh_made = 0;
  __syncthreads();
  const int64_t total = ioff[nl];
  for (int64_t q = blockIdx.x; q < total; q += gridDim.x) {
    const int32_t i = chunk_owner(ioff, nl, q);
    const int32_t c = a.list[i];
    const int64_t m0 = a.moff[c] + (q - ioff[i]) * LM_CH;
    const int64_t m1 = min(m0 + LM_CH, a.moff[c + 1]);
    const int64_t tb = a.tbase[c];
    const int logcap = ceil_log2(a.tbase[c + 1] - tb);
    member_arcs_warp(a, c, m0 + (int64_t)wid * 32, m1, (int64_t)MB_NT, [&](int32_t cu, int32_t w) {
      if (cu < 0) return;
      if (!shared_add(keys, vals, &sh_made, cu, w, a.err)) global_add(a, tb, logcap, cu, w);
    });
    __syncthreads();
    if (sh_made > 0) {
      for (int j = tid; j < LT_CAP; j += MB_NT) {
        const int32_t k = keys[j];
        if (k >= 0) {
          global_add(a, tb, logcap, k, vals[j]);
          keys[j] = -1;
          vals[j] = 0;
        }
      }
    }
    __syncthreads();
    if (tid == 0) sh_made = 0;
    __syncthreads();
  }
}

// Large class, read-out: one CTA per chunk of LE_CH slots of one node's
// region compacts the occupied slots in shared memory, takes its place in
// the node's pairs with one atomic add on the node's distinct count, and
// writes them (the order of a node's pairs is not fixed).
__global__ void __launch_bounds__(MB_NT) k_merge_emit_large(MArgs a, const int64_t* __restrict__ eoff,
                                                            int32_t nl) {
  __shared__ int32_t sk[LE_CH], sv[LE_CH];
  __shared__ int32_t sh_n, sh_base;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) sh_n = 0;
  __syncthreads();
  const int64_t total = eoff[nl];
  for (int64_t q = blockIdx.x; q < total; q += gridDim.x) {
    const int32_t i = chunk_owner(eoff, nl, q);
    const int32_t c = a.list[i];
    const int64_t s0 = a.tbase[c] + (q - eoff[i]) * LE_CH;
    const int64_t s1 = min(s0 + LE_CH, a.tbase[c + 1]);
    for (int64_t j0 = s0; j0 < s1; j0 += MB_NT) {
      const int64_t j = j0 + tid;
      const unsigned long long v = j < s1 ? a.tslot[j] : ~0ull;
      const bool occ = v != ~0ull;
      const unsigned m = __ballot_sync(0xffffffffu, occ);
      int q0 = 0;
      if (lane == 0 && m) q0 = atomicAdd(&sh_n, __popc(m));
      q0 = __shfl_sync(0xffffffffu, q0, 0);
      if (occ) {
        const int r = q0 + __popc(m & ((1u << lane) - 1));
        sk[r] = (int32_t)(v >> 32);
        sv[r] = (int32_t)(v & 0xffffffffull);
      }
    }
    __syncthreads();
    const int n = sh_n;
    if (tid == 0 && n > 0) sh_base = atomicAdd(&a.cdeg[c], n);
    __syncthreads();
    if (n > 0) {
      const int64_t base = a.soff[c] + sh_base;
      for (int r = tid; r < n; r += MB_NT) {
        a.rcol[base + r] = sk[r];
        a.rew[base + r] = sv[r];
      }
    }
    __syncthreads();
    if (tid == 0) sh_n = 0;
    __syncthreads();
  }
}

// Coarse rows from the regions: one warp per coarse node copies its pairs.
__global__ void k_rows_from_regions(const int64_t* __restrict__ soff,
                                    const int32_t* __restrict__ cdeg,
                                    const int64_t* __restrict__ crow,
                                    const int32_t* __restrict__ rcol,
                                    const int32_t* __restrict__ rew, int64_t Nc,
                                    int32_t* __restrict__ ccol, int32_t* __restrict__ cew) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < Nc; c += nwarps) {
    const int64_t s0 = soff[c], d0 = crow[c];
    const int32_t n = cdeg[c];
    for (int j = lane; j < n; j += 32) {
      ccol[d0 + j] = rcol[s0 + j];
      cew[d0 + j] = rew[s0 + j];
    }
  }
}

// Overlay (ensemble clusterings): the pair (O[v], C[v]) keys an open-
// addressing table whose entry keeps the smallest node id with that pair.
// Labels are node ids < 2^31, so a key never equals the empty marker ~0.
__device__ __forceinline__ uint64_t pair_key(int32_t o, int32_t c) {
  return ((uint64_t)(uint32_t)o << 32) | (uint32_t)c;
}

__global__ void k_overlay_insert(const int32_t* __restrict__ gid, const int32_t* __restrict__ part,
                                 const int32_t* __restrict__ O, const int32_t* __restrict__ C,
                                 int64_t N, unsigned long long* keys, int32_t* rep, int logcap,
                                 int32_t* err) {
  const uint64_t mask = ((uint64_t)1 << logcap) - 1;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (!part[slot_at(gid, v)]) continue;
    const unsigned long long key = pair_key(O[v], C[v]);
    uint64_t s = mix64(key) & mask;
    bool placed = false;
    for (uint64_t p = 0; p <= mask; ++p) {
      unsigned long long cur = keys[s];
      if (cur == ~0ull) cur = atomicCAS(&keys[s], ~0ull, key);
      if (cur == ~0ull || cur == key) {
        atomicMin(&rep[s], (int32_t)v);
        placed = true;
        break;
      }
      s = (s + 1) & mask;
    }
    if (!placed) atomicOr(err, DERR_HASH_FULL);
  }
}

__global__ void k_overlay_apply(const int32_t* __restrict__ gid, const int32_t* __restrict__ part,
                                int32_t* O, const int32_t* __restrict__ C, int64_t N,
                                const unsigned long long* __restrict__ keys,
                                const int32_t* __restrict__ rep, int logcap) {
  const uint64_t mask = ((uint64_t)1 << logcap) - 1;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (!part[slot_at(gid, v)]) continue;
    const unsigned long long key = pair_key(O[v], C[v]);
    uint64_t s = mix64(key) & mask;
    for (uint64_t p = 0; p <= mask; ++p) {
      const unsigned long long cur = keys[s];
      if (cur == key) { O[v] = rep[s]; break; }
      if (cur == ~0ull) break;          // cannot happen after the insert pass
      s = (s + 1) & mask;
    }
  }
}

// Node ids per slot and the arc offsets of the slots of a built level.
void finish_level(CoarseLevel& out, int ns, cudaStream_t s) {
  const int64_t Nc = out.N;
  out.gid.alloc(std::max<int64_t>(Nc, 1), s);
  fill_gid(out.noff_d.p, ns, out.gid.p, Nc, s);
  DevBuf<int64_t> ga(ns + 1, s);
  k_gather<<<grid_for(ns + 1, 128, 64), 128, 0, s>>>(out.row_ptr.p, out.noff_d.p, ns + 1, ga.p); SCLAP_NOTE_LAUNCH("k_gather");
  SCLAP_LAUNCH_CHECK();
  out.aoff.assign(ns + 1, 0);
  SCLAP_CUDA(cudaMemcpyAsync(out.aoff.data(), ga.p, (ns + 1) * sizeof(int64_t),
                             cudaMemcpyDeviceToHost, s));
  stream_sync(s);
}

// The coarse arcs by segments (member lists and per-node merges, see the
// kernels above).  Returns false, having built nothing, when the regions,
// member lists and the table of the large nodes would take more than the
// memory of Tcap slots of the hash table path (12 bytes each).
bool contract_merge(const LevelView& lv, int64_t N, int64_t Nc, DevBuf<int32_t>& inter,
                    DevBuf<int64_t>& cap, DevBuf<int64_t>& tbase, const CArgs& ca, int64_t Tcap,
                    CoarseLevel& out, int32_t* d_err, cudaStream_t s) {
  const int sms = num_sms();
  DevBuf<int64_t> soff(Nc + 1, s);
  DevBuf<int32_t> mcnt(Nc, s), lists(2 * Nc, s), cnt(2, s);
  DevBuf<unsigned long long> marcs(Nc, s);
  scan_excl_i32_to_i64(inter.p, soff.p, Nc, s);
  mcnt.zero();
  marcs.zero();
  cnt.zero();
  const unsigned ng = grid_for(N, 256, (int64_t)sms * 16);
  const unsigned cg = grid_for(Nc, 256, (int64_t)sms * 16);
  k_member_count<<<ng, 256, 0, s>>>(ca.cmap, lv.row_ptr, N, mcnt.p, marcs.p); SCLAP_NOTE_LAUNCH("k_member_count");
  const int64_t* marcs_i = reinterpret_cast<const int64_t*>(marcs.p);
  k_merge_classes<<<cg, 256, 0, s>>>(inter.p, marcs_i, Nc, lists.p, cnt.p, cap.p); SCLAP_NOTE_LAUNCH("k_merge_classes");
  scan_excl_i64(cap.p, tbase.p, Nc, s);
  int64_t h[3] = {0, 0, 0};
  int32_t hc[2] = {0, 0};
  SCLAP_CUDA(cudaMemcpyAsync(&h[0], soff.p + Nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SCLAP_CUDA(cudaMemcpyAsync(&h[1], tbase.p + Nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SCLAP_CUDA(cudaMemcpyAsync(hc, cnt.p, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  stream_sync(s);
  const int64_t Mi = h[0], T = h[1];
  const int32_t nb = hc[0], nl = hc[1];
  if (8 * Mi + 8 * T + 4 * N + 8 * Nc + 12 * (int64_t)nl > 12 * Tcap) return false;

  // member lists: fine nodes counting-sorted by coarse id
  DevBuf<int32_t> members(N, s), cdeg(Nc, s);
  DevBuf<int64_t> moff(Nc + 1, s);
  cdeg.zero();
  scan_excl_i32_to_i64(mcnt.p, moff.p, Nc, s);
  mcnt.zero();
  k_member_fill<<<ng, 256, 0, s>>>(ca.cmap, N, moff.p, mcnt.p, members.p); SCLAP_NOTE_LAUNCH("k_member_fill");

  DevBuf<int32_t> rcol(std::max<int64_t>(Mi, 1), s), rew(std::max<int64_t>(Mi, 1), s);
  MArgs m{};
  m.row_ptr = lv.row_ptr; m.col = lv.col; m.ew = lv.ew; m.cmap = ca.cmap;
  m.members = members.p; m.moff = moff.p; m.inter = inter.p; m.marcs = marcs_i; m.soff = soff.p;
  m.tbase = tbase.p; m.rcol = rcol.p; m.rew = rew.p; m.cdeg = cdeg.p;
  m.err = d_err; m.Nc = Nc;
  k_merge_warp<<<grid_for(Nc * 32, 256, (int64_t)sms * 8), 256, 0, s>>>(m); SCLAP_NOTE_LAUNCH("k_merge_warp");
  if (nb > 0) {
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
      SCLAP_CUDA(cudaFuncSetAttribute(k_merge_cta, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)merge_cta_smem()));
    });
    m.list = lists.p;
    m.nlist = cnt.p;
    k_merge_cta<<<(unsigned)std::min<int64_t>(nb, (int64_t)sms * 5), MB_NT, merge_cta_smem(), s>>>(m); SCLAP_NOTE_LAUNCH("k_merge_cta");
  }
  DevBuf<unsigned long long> tslot(std::max<int64_t>(T, 1), s);
  if (nl > 0) {
    DevBuf<int32_t> ich(nl, s), ech(nl, s);
    DevBuf<int64_t> ioff(nl + 1, s), eoff(nl + 1, s);
    tslot.fill_bytes(0xff);
    m.tslot = tslot.p;
    m.list = lists.p + Nc;
    m.nlist = cnt.p + 1;
    k_large_chunks<<<grid_for(nl, 256, (int64_t)sms * 4), 256, 0, s>>>(m.list, nl, moff.p, tbase.p, ich.p, ech.p); SCLAP_NOTE_LAUNCH("k_large_chunks");
    scan_excl_i32_to_i64(ich.p, ioff.p, nl, s);
    scan_excl_i32_to_i64(ech.p, eoff.p, nl, s);
    static std::once_flag large_once;
    std::call_once(large_once, [] {
      SCLAP_CUDA(cudaFuncSetAttribute(k_merge_large, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)merge_large_smem()));
    });
    // chunk counts stay on the device: the grids are resident-sized and
    // stride over them
    k_merge_large<<<(unsigned)sms * 3, MB_NT, merge_large_smem(), s>>>(m, ioff.p, nl); SCLAP_NOTE_LAUNCH("k_merge_large");
    k_merge_emit_large<<<(unsigned)sms * 6, MB_NT, 0, s>>>(m, eoff.p, nl); SCLAP_NOTE_LAUNCH("k_merge_emit_large");
  }
  SCLAP_LAUNCH_CHECK();

  out.row_ptr.alloc(Nc + 1, s);
  scan_excl_i32_to_i64(cdeg.p, out.row_ptr.p, Nc, s);
  int64_t Mc = 0;
  SCLAP_CUDA(cudaMemcpyAsync(&Mc, out.row_ptr.p + Nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  stream_sync(s);
  out.M = Mc;
  out.col.alloc(std::max<int64_t>(Mc, 1), s);
  out.ew.alloc(std::max<int64_t>(Mc, 1), s);
  k_rows_from_regions<<<grid_for(Nc * 32, 256, (int64_t)sms * 16), 256, 0, s>>>(
      soff.p, cdeg.p, out.row_ptr.p, rcol.p, rew.p, Nc, out.col.p, out.ew.p); SCLAP_NOTE_LAUNCH("k_rows_from_regions");
  SCLAP_LAUNCH_CHECK();
  return true;
}

}  // namespace

void contract_rank(const LevelView& lv, const std::vector<int64_t>& noff, const int32_t* label,
                   ContractWork& w, std::vector<int64_t>& nc_slot, cudaStream_t s) {
  const int64_t N = lv.N;
  const int ns = (int)noff.size() - 1;
  w.flag.alloc(N, s);
  w.flag.zero();
  w.cid.alloc(N + 1, s);
  const int sms = num_sms();
  if (N > 0) { k_mark<<<grid_for(N, 256, (int64_t)sms * 16), 256, 0, s>>>(label, N, w.flag.p); SCLAP_NOTE_LAUNCH("k_mark"); }
  scan_excl_i32_to_i64(w.flag.p, w.cid.p, N, s);
  DevBuf<int64_t> idx(ns + 1, s), got(ns + 1, s);
  idx.upload(noff);
  k_gather<<<grid_for(ns + 1, 128, 64), 128, 0, s>>>(w.cid.p, idx.p, ns + 1, got.p); SCLAP_NOTE_LAUNCH("k_gather");
  SCLAP_LAUNCH_CHECK();
  w.cid_at.assign(ns + 1, 0);
  SCLAP_CUDA(cudaMemcpyAsync(w.cid_at.data(), got.p, (ns + 1) * sizeof(int64_t),
                             cudaMemcpyDeviceToHost, s));
  stream_sync(s);
  nc_slot.assign(ns, 0);
  for (int i = 0; i < ns; ++i) nc_slot[i] = w.cid_at[i + 1] - w.cid_at[i];
}

void contract_build(const LevelView& lv, const std::vector<int64_t>& noff, const int32_t* label,
                    const ContractWork& w, const std::vector<uint8_t>& keep, int32_t* cmap,
                    CoarseLevel& out, int32_t* d_err, cudaStream_t s) {
  const int64_t N = lv.N;
  const int ns = (int)noff.size() - 1;
  const int sms = num_sms();
  std::vector<int64_t> cno(ns + 1, 0), delta(ns, 0);
  for (int i = 0; i < ns; ++i) {
    const int64_t nc = keep[i] ? w.cid_at[i + 1] - w.cid_at[i] : 0;
    cno[i + 1] = cno[i] + nc;
    delta[i] = cno[i] - w.cid_at[i];
  }
  const int64_t Nc = cno[ns];
  DevBuf<int64_t> d_delta(ns, s);
  d_delta.upload(delta);
  DevBuf<uint8_t> d_keep(ns, s);
  d_keep.upload(keep);

  out.N = Nc;
  out.noff = cno;
  out.noff_d.alloc(ns + 1, s);
  out.noff_d.upload(cno);
  out.nw.alloc(std::max<int64_t>(Nc, 1), s);
  out.nw.zero();
  DevBuf<int32_t> inter(std::max<int64_t>(Nc, 1), s);
  DevBuf<int64_t> cap(std::max<int64_t>(Nc, 1), s), tbase(Nc + 1, s);
  inter.zero();

  CArgs a{};
  a.row_ptr = lv.row_ptr; a.col = lv.col; a.ew = lv.ew; a.nw = lv.nw; a.gid = lv.gid;
  a.label = label; a.cid = w.cid.p; a.delta = d_delta.p; a.keep = d_keep.p; a.cmap = cmap;
  a.cnw = out.nw.p; a.inter = inter.p; a.tbase = tbase.p; a.err = d_err;
  a.c_lo = 0; a.c_hi = INT32_MAX; a.toff = 0; a.sums31 = lv.sums31;
  a.N = N; a.Nc = Nc;

  const unsigned ng = grid_for(N, 256, (int64_t)sms * 16);
  const unsigned wg = grid_for(N, 256, (int64_t)sms * 16);   // 8 warps x 32 nodes per block
  const unsigned hg = (unsigned)sms * 8;                      // heavy-row chunks, grid-stride
  // rows above HEAVY_ROW arcs: listed, cut into chunks, spread over the grid
  constexpr int64_t HEAVY_ROW = 2048;
  DevBuf<int32_t> hlist(std::max<int64_t>(1, std::min<int64_t>(N, lv.M / (HEAVY_ROW + 1) + 1)), s);
  DevBuf<int64_t> hoff;
  int32_t nh = 0;
  if (N > 0) {
    k_map<<<ng, 256, 0, s>>>(a, N); SCLAP_NOTE_LAUNCH("k_map");
    a.heavy = HEAVY_ROW;
    DevBuf<int32_t> hcnt(1, s);
    hcnt.zero();
    k_heavy_list<<<ng, 256, 0, s>>>(a, N, hlist.p, hcnt.p); SCLAP_NOTE_LAUNCH("k_heavy_list");
    SCLAP_CUDA(cudaMemcpyAsync(&nh, hcnt.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    stream_sync(s);
    if (nh > 0) {
      DevBuf<int32_t> nch(nh, s);
      hoff.alloc(nh + 1, s);
      k_heavy_chunks<<<grid_for(nh, 256, (int64_t)sms * 4), 256, 0, s>>>(lv.row_ptr, hlist.p, nh, nch.p); SCLAP_NOTE_LAUNCH("k_heavy_chunks");
      scan_excl_i32_to_i64(nch.p, hoff.p, nh, s);
    }
    k_count_inter<<<wg, 256, 0, s>>>(a, N); SCLAP_NOTE_LAUNCH("k_count_inter");
    if (nh > 0) { k_count_heavy<<<hg, 256, 0, s>>>(a, hlist.p, hoff.p, nh); SCLAP_NOTE_LAUNCH("k_count_heavy"); }
  }
  auto insert = [&] {
    k_insert<<<wg, 256, 0, s>>>(a, N); SCLAP_NOTE_LAUNCH("k_insert");
    if (nh > 0) { k_insert_heavy<<<hg, 256, 0, s>>>(a, hlist.p, hoff.p, nh); SCLAP_NOTE_LAUNCH("k_insert_heavy"); }
  };
  const int64_t Tcap = table_pass_slots();
  if (tuning_get().contract_merge && N > 0 && Nc > 0 &&
      contract_merge(lv, N, Nc, inter, cap, tbase, a, Tcap, out, d_err, s)) {
    finish_level(out, ns, s);
    return;
  }
  if (Nc > 0) {
    k_table_caps<<<grid_for(Nc, 256, (int64_t)sms * 16), 256, 0, s>>>(inter.p, Nc, cap.p); SCLAP_NOTE_LAUNCH("k_table_caps");
  }
  scan_excl_i64(cap.p, tbase.p, Nc, s);
  int64_t T = 0;
  SCLAP_CUDA(cudaMemcpyAsync(&T, tbase.p + Nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  stream_sync(s);
  // the inter-arc counts have served (table sizes); the array now counts
  // claimed slots, i.e. the coarse degrees
  a.cdeg = inter.p;
  SCLAP_CUDA(cudaMemsetAsync(inter.p, 0, (size_t)std::max<int64_t>(Nc, 1) * sizeof(int32_t), s));
  out.row_ptr.alloc(Nc + 1, s);
  if (T <= Tcap) {
    // one pass: the whole table at once
    DevBuf<unsigned long long> tslot(std::max<int64_t>(T, 1), s);
    DevBuf<int32_t> towner(std::max<int64_t>(T, 1), s);
    tslot.fill_bytes(0xff);
    a.tslot = tslot.p;
    a.towner = towner.p;
    if (N > 0 && T > 0) insert();
    scan_excl_i32_to_i64(inter.p, out.row_ptr.p, Nc, s);
    int64_t Mc = 0;
    SCLAP_CUDA(cudaMemcpyAsync(&Mc, out.row_ptr.p + Nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    stream_sync(s);
    out.M = Mc;
    out.col.alloc(std::max<int64_t>(Mc, 1), s);
    out.ew.alloc(std::max<int64_t>(Mc, 1), s);
    if (Nc > 0 && T > 0) {
      SCLAP_CUDA(cudaMemsetAsync(inter.p, 0, (size_t)Nc * sizeof(int32_t), s));   // row fill
      k_emit<<<grid_for(T, 256, (int64_t)sms * 32), 256, 0, s>>>(tslot.p, towner.p, out.row_ptr.p,
                                                                 inter.p, T, out.col.p, out.ew.p); SCLAP_NOTE_LAUNCH("k_emit");
    }
  } else {
    // Passes over ranges of coarse nodes whose table regions fit in Tcap
    // slots (a region larger than that gets a pass of its own).  Each pass
    // streams every fine node but inserts only the arcs of sources in its
    // range.  Sweep 1 counts the coarse degrees, which give the row offsets
    // and the exact size of the coarse arrays; sweep 2 inserts again and
    // emits every pass's rows in place.  Identical result to one pass.
    std::vector<int64_t> htb(Nc + 1);
    SCLAP_CUDA(cudaMemcpyAsync(htb.data(), tbase.p, (Nc + 1) * sizeof(int64_t),
                               cudaMemcpyDeviceToHost, s));
    stream_sync(s);
    std::vector<int32_t> cut_at{0};
    while (cut_at.back() < Nc) {
      const int64_t lo = cut_at.back();
      int64_t hi = std::upper_bound(htb.begin() + lo + 1, htb.end(), htb[lo] + Tcap) -
                   htb.begin() - 1;
      if (hi <= lo) hi = lo + 1;
      cut_at.push_back((int32_t)hi);
    }
    int64_t Tmax = 1;
    for (size_t q = 0; q + 1 < cut_at.size(); ++q)
      Tmax = std::max<int64_t>(Tmax, htb[cut_at[q + 1]] - htb[cut_at[q]]);
    DevBuf<unsigned long long> tslot(Tmax, s);
    DevBuf<int32_t> towner(Tmax, s), claims(std::max<int64_t>(Nc, 1), s);
    a.tslot = tslot.p;
    a.towner = towner.p;
    auto pass = [&](size_t q) {
      a.c_lo = cut_at[q];
      a.c_hi = cut_at[q + 1];
      a.toff = htb[a.c_lo];
      SCLAP_CUDA(cudaMemsetAsync(tslot.p, 0xff, (size_t)(htb[a.c_hi] - a.toff) * 8, s));
      if (N > 0) insert();
      return htb[a.c_hi] - a.toff;
    };
    for (size_t q = 0; q + 1 < cut_at.size(); ++q) pass(q);            // sweep 1: degrees
    scan_excl_i32_to_i64(inter.p, out.row_ptr.p, Nc, s);
    int64_t Mc = 0;
    SCLAP_CUDA(cudaMemcpyAsync(&Mc, out.row_ptr.p + Nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    stream_sync(s);
    out.M = Mc;
    out.col.alloc(std::max<int64_t>(Mc, 1), s);
    out.ew.alloc(std::max<int64_t>(Mc, 1), s);
    a.cdeg = claims.p;                   // sweep 2 counts claims apart from the row fill
    SCLAP_CUDA(cudaMemsetAsync(inter.p, 0, (size_t)Nc * sizeof(int32_t), s));   // row fill
    for (size_t q = 0; q + 1 < cut_at.size(); ++q) {                    // sweep 2: emit
      const int64_t Tp = pass(q);
      k_emit<<<grid_for(Tp, 256, (int64_t)sms * 32), 256, 0, s>>>(tslot.p, towner.p,
                                                                  out.row_ptr.p, inter.p, Tp,
                                                                  out.col.p, out.ew.p); SCLAP_NOTE_LAUNCH("k_emit");
    }
  }
  SCLAP_LAUNCH_CHECK();
  finish_level(out, ns, s);
}

void overlay_labels(const LevelView& lv, const int32_t* part, int32_t* O, const int32_t* C,
                    int32_t* err, cudaStream_t s) {
  if (lv.N == 0) return;
  const int logcap = ceil_log2(std::max<int64_t>(2 * lv.N, 64));
  const int64_t cap = (int64_t)1 << logcap;
  DevBuf<unsigned long long> keys(cap, s);
  DevBuf<int32_t> rep(cap, s);
  keys.fill_bytes(0xff);
  rep.fill_bytes(0x7f);                    // 0x7f7f7f7f: above every node id
  const unsigned g = grid_for(lv.N, 256, (int64_t)num_sms() * 16);
  k_overlay_insert<<<g, 256, 0, s>>>(lv.gid, part, O, C, lv.N, keys.p, rep.p, logcap, err); SCLAP_NOTE_LAUNCH("k_overlay_insert");
  k_overlay_apply<<<g, 256, 0, s>>>(lv.gid, part, O, C, lv.N, keys.p, rep.p, logcap); SCLAP_NOTE_LAUNCH("k_overlay_apply");
  SCLAP_LAUNCH_CHECK();
}

}  // namespace sclap
