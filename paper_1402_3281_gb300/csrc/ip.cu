// ip.cu -- initial partitioning of the coarsest graphs, cut, projection.
//
// The paper partitions the coarsest graph with KaHIP's recursive bisection,
// which it does not specify.  Here every graph gets `trials` independent
// trials, all graphs' trials forming one batch: greedy graph growing (one CTA
// per trial: block j starts at a hashed seed and absorbs the unassigned
// nodes connected to it, in node-id order, while it stays <= ceil(c(V)/k)),
// water-filling of the leftovers, then LP local search (the lp.cu kernels on
// the whole trial batch).  The best trial by (overload, cut, trial) is kept.
#include <algorithm>

#include <map>
#include <tuple>

#include "common.cuh"

namespace sclap {
namespace {

// CTA sizes of the greedy-growing kernel: 128 threads when a batch has many
// trials (more trials in flight), 512 when it has few (wider steps).
constexpr int GNT_MANY = 128, GNT_FEW = 1024;
constexpr int GPER = 8;   // consecutive nodes per thread in the greedy-growing scans
// arcs per thread per pass in the greedy-growing accumulation (more in the
// wide CTAs, which have the registers and run on few trials)
template <int GNT> struct Garc { static constexpr int value = GNT >= 512 ? 8 : 4; };

__global__ void k_replicate(const CopyTask* __restrict__ tasks, int64_t* __restrict__ row_ptr,
                            int32_t* __restrict__ col, int32_t* __restrict__ ew,
                            int32_t* __restrict__ nw) {
  const CopyTask t = tasks[blockIdx.y];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < t.n; v += stride) {
    int64_t d = v;
    if (t.rank) {
      const int64_t r0 = t.rank[t.src_n0 + v];
      if (t.rank[t.src_n0 + v + 1] == r0) continue;   // isolated: dropped
      d = r0 - t.rbase;
    }
    row_ptr[t.dst_n0 + d] = t.dst_a0 + (t.row_ptr[t.src_n0 + v] - t.src_a0);
    if (nw) nw[t.dst_n0 + d] = wat(t.nw, t.src_n0 + v);
  }
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < t.m; e += stride) {
    const int64_t u = t.col[t.src_a0 + e];
    const int64_t du = t.rank ? t.rank[u] - t.rbase : u - t.src_n0;
    col[t.dst_a0 + e] = (int32_t)(du + t.dst_n0);
    if (ew) ew[t.dst_a0 + e] = wat(t.ew, t.src_a0 + e);
  }
}

// A later copy of an already copied segment: nodes [0, nd) and arcs
// [0, m) of the first copy (at tn0 / ta0) to dn0 / da0, row offsets shifted
// by the arc offset difference and neighbour ids by the node offset
// difference.
struct CopyFrom {
  int64_t dn0, da0, tn0, ta0, nd, m;
};
__global__ void k_replicate_from(const CopyFrom* __restrict__ tasks, int64_t* __restrict__ row_ptr,
                                 int32_t* __restrict__ col, int32_t* __restrict__ ew,
                                 int32_t* __restrict__ nw) {
  const CopyFrom t = tasks[blockIdx.y];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t da = t.da0 - t.ta0;
  const int32_t dn = (int32_t)(t.dn0 - t.tn0);
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < t.nd; v += stride) {
    row_ptr[t.dn0 + v] = row_ptr[t.tn0 + v] + da;
    if (nw) nw[t.dn0 + v] = nw[t.tn0 + v];
  }
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < t.m; e += stride) {
    col[t.da0 + e] = col[t.ta0 + e] + dn;
    if (ew) ew[t.da0 + e] = ew[t.ta0 + e];
  }
}

// Block-wide inclusive scan of an int64 (all GNT threads call it).
template <int GNT>
__device__ int64_t block_incl_scan(int64_t x, int64_t* sh, int64_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, (long long)x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t v = lane < GNT / 32 ? sh[lane] : 0;
    int64_t vi = v;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, (long long)vi, o);
      if (lane >= o) vi += y;
    }
    if (lane < GNT / 32) sh[lane] = vi - v;
    if (lane == 31) sh[32] = vi;
  }
  __syncthreads();
  x += sh[wid];
  *total = sh[32];
  __syncthreads();
  return x;
}

template <int GNT>
__device__ int64_t block_sum(int64_t x, int64_t* sh) {
  int64_t tot;
  block_incl_scan<GNT>(x, sh, &tot);
  return tot;
}

template <int GNT>
__global__ void __launch_bounds__(GNT) k_ggg(GGGArgs a) {
  constexpr int GARC = Garc<GNT>::value;
  __shared__ int64_t sh[33];
  __shared__ uint64_t shh[GNT / 32];
  __shared__ int32_t shv[GNT / 32];
  __shared__ int64_t Wj_sh, accw_sh;
  __shared__ int32_t nstep_sh, seed_sh, nfront_sh;
  // a chunk of step nodes: row start, first and one-past-last arc offset
  __shared__ int64_t st_rs[GNT], st_ex[GNT], st_in[GNT];
  __shared__ int32_t next_sh;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // trials are taken from a queue ordered by size, largest first, so the
  // long trials of the batch start first and on different CTAs
  for (;;) {
    if (tid == 0) next_sh = atomicAdd(a.next, 1);
    __syncthreads();
    const int32_t qi = next_sh;
    __syncthreads();
    if (qi >= a.nslots) break;
    const int32_t s = a.order[qi];
    const int64_t base = a.noff[s], n = a.noff[s + 1] - base;
    const int32_t k = a.nlab[s];
    const int64_t bo = a.boff[s], avg = a.avg[s];
    const uint64_t tkey = a.tkey[s];
    const int32_t lvl = a.level[s];
    for (int64_t v = tid; v < n; v += GNT) a.label[base + v] = -1;
    for (int32_t b = tid; b < k; b += GNT) a.W[bo + b] = 0;
    __syncthreads();
    for (int32_t j = 0; j < k; ++j) {
      // seed: unassigned non-isolated node with the smallest hash
      const uint64_t skey = hkey(tkey, PH_GGG, (uint64_t)lvl, (uint64_t)j);
      uint64_t bh = ~0ull;
      int32_t bv = -1;
      // (the same pass clears the connections left by the previous block)
      for (int64_t v0 = (int64_t)tid * GPER; v0 < n; v0 += (int64_t)GNT * GPER) {
#pragma unroll
        for (int i = 0; i < GPER; ++i) {
          const int64_t v = v0 + i;
          if (v >= n) break;
          const int64_t gv = base + v;
          a.conn[gv] = 0;
          if (a.label[gv] >= 0 || a.row_ptr[gv + 1] == a.row_ptr[gv]) continue;
          const uint64_t h = mix64(skey ^ (uint64_t)v);
          if (bv < 0 || h < bh) { bh = h; bv = (int32_t)v; }
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        uint64_t oh = __shfl_xor_sync(0xffffffffu, (unsigned long long)bh, o);
        int32_t ov = __shfl_xor_sync(0xffffffffu, bv, o);
        if (ov >= 0 && (bv < 0 || oh < bh || (oh == bh && ov < bv))) { bh = oh; bv = ov; }
      }
      if (lane == 0) { shh[wid] = bh; shv[wid] = bv; }
      __syncthreads();
      if (tid == 0) {
        uint64_t h = ~0ull;
        int32_t v = -1;
        for (int w = 0; w < GNT / 32; ++w)
          if (shv[w] >= 0 && (v < 0 || shh[w] < h || (shh[w] == h && shv[w] < v))) {
            h = shh[w]; v = shv[w];
          }
        seed_sh = v;
      }
      __syncthreads();
      const int32_t seed = seed_sh;
      if (seed < 0) break;
      // step nodes and newly reached nodes: two scratch lists that swap roles
      int32_t* stp = a.step + base;
      int32_t* frt = a.front + base;
      // while every step has absorbed all its candidates, the candidates of
      // the next step are exactly the nodes first reached by this one, listed
      // as they are reached; the first step whose candidates do not all fit
      // switches the block to the ordered scan over all nodes
      bool ordered = false;
      __syncthreads();
      if (tid == 0) {
        a.label[base + seed] = (int32_t)(bo + j);
        stp[0] = (int32_t)(base + seed);
        nstep_sh = 1;
        nfront_sh = 0;
        Wj_sh = a.nw[base + seed];
      }
      __syncthreads();
      while (true) {
        // connections of unassigned nodes to the block grow with each step;
        // the arcs of up to GNT step nodes at a time are spread over all
        // threads (a hub in the step does not hold back one warp)
        const int32_t nstep = nstep_sh;
        int64_t fw = 0;   // weight of the nodes this thread listed
        for (int32_t q0 = 0; q0 < nstep; q0 += GNT) {
          const int32_t q = q0 + tid;
          int64_t rs = 0, d = 0;
          if (q < nstep) {
            const int32_t u = stp[q];
            rs = a.row_ptr[u];
            d = a.row_ptr[u + 1] - rs;
          }
          int64_t tot;
          const int64_t incl = block_incl_scan<GNT>(d, sh, &tot);
          st_rs[tid] = rs;
          st_ex[tid] = incl - d;
          st_in[tid] = incl;
          __syncthreads();
          const int cnt = min(GNT, nstep - q0);
          // GARC arcs per thread per pass, their chains (owner search, arc,
          // label, connection add) interleaved so the loads overlap
          for (int64_t x0 = tid; x0 < tot; x0 += (int64_t)GNT * GARC) {
            int32_t y[GARC], w[GARC], lab[GARC];
#pragma unroll
            for (int u = 0; u < GARC; ++u) {
              const int64_t x = x0 + (int64_t)u * GNT;
              y[u] = -1;
              w[u] = 0;
              if (x >= tot) continue;
              // owner: the first step node whose arcs end after x (skips
              // step nodes without arcs)
              int lo = 0, hi = cnt - 1;
              while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (st_in[mid] > x) hi = mid; else lo = mid + 1;
              }
              const int64_t e = st_rs[lo] + (x - st_ex[lo]);
              y[u] = a.col[e];
              w[u] = a.ew[e];
              if (!SCLAP_OK(y[u], a.N, a.err)) y[u] = -1;
            }
#pragma unroll
            for (int u = 0; u < GARC; ++u) lab[u] = y[u] >= 0 ? a.label[y[u]] : 0;
            unsigned long long old[GARC];
#pragma unroll
            for (int u = 0; u < GARC; ++u)
              old[u] = (y[u] >= 0 && lab[u] < 0)
                           ? atomicAdd(ull(&a.conn[y[u]]), (unsigned long long)w[u])
                           : 1ull;
#pragma unroll
            for (int u = 0; u < GARC; ++u) {
              if (!ordered && old[u] == 0) {       // first arc into y (weights > 0)
                frt[atomicAdd(&nfront_sh, 1)] = y[u];
                fw += a.nw[y[u]];
              }
            }
          }
          __syncthreads();
        }
        const int64_t Wj = Wj_sh;
        if (Wj >= avg) break;
        if (!ordered) {
          const int64_t fsum = block_sum<GNT>(fw, sh);
          const int32_t nf = nfront_sh;
          if (Wj + fsum <= avg) {
            // all of them fit: they are the next step, in any order
            for (int32_t q = tid; q < nf; q += GNT) a.label[frt[q]] = (int32_t)(bo + j);
            int32_t* t = stp; stp = frt; frt = t;
            __syncthreads();
            if (tid == 0) {
              nstep_sh = nf;
              nfront_sh = 0;
              Wj_sh = Wj + fsum;
            }
            __syncthreads();
            if (nf == 0) break;
            continue;
          }
          ordered = true;
        }
        if (tid == 0) accw_sh = 0;
        // connected unassigned nodes in id order, longest prefix that fits;
        // each thread takes GPER consecutive nodes per pass (its prefix is
        // serial, the block scans give its offsets), so one pair of block
        // scans covers GPER * GNT nodes
        int64_t cw_all = 0;
        for (int64_t v0 = (int64_t)tid * GPER; v0 < n; v0 += (int64_t)GNT * GPER) {
#pragma unroll
          for (int i = 0; i < GPER; ++i) {
            const int64_t v = v0 + i;
            if (v < n && a.label[base + v] < 0 && a.conn[base + v] > 0) cw_all += a.nw[base + v];
          }
        }
        const bool all_fit = Wj + block_sum<GNT>(cw_all, sh) <= avg;
        int64_t carry_w = 0;
        int32_t carry_c = 0;
        int64_t acc_w = 0;
        for (int64_t c0 = 0; c0 < n; c0 += (int64_t)GNT * GPER) {
          const int64_t vb = c0 + (int64_t)tid * GPER;
          int32_t wt[GPER];                        // node weight, -1: not a candidate
          int64_t tsum = 0;
#pragma unroll
          for (int i = 0; i < GPER; ++i) {
            const int64_t v = vb + i;
            const bool cand = v < n && a.label[base + v] < 0 && a.conn[base + v] > 0;
            wt[i] = cand ? a.nw[base + v] : -1;
            tsum += cand ? wt[i] : 0;
          }
          int64_t tw = 0, pre = 0;
          if (!all_fit) pre = block_incl_scan<GNT>(tsum, sh, &tw) - tsum;
          int64_t run = pre, na = 0;
          uint32_t adm = 0;
#pragma unroll
          for (int i = 0; i < GPER; ++i) {
            if (wt[i] < 0) continue;
            run += wt[i];
            if (all_fit || Wj + carry_w + run <= avg) {
              adm |= 1u << i;
              ++na;
            }
          }
          int64_t tc;
          int64_t pos = block_incl_scan<GNT>(na, sh, &tc) - na + carry_c;
#pragma unroll
          for (int i = 0; i < GPER; ++i) {
            if (!((adm >> i) & 1u)) continue;
            stp[pos++] = (int32_t)(base + vb + i);
            acc_w += wt[i];
          }
          carry_w += tw;
          carry_c += (int32_t)tc;
          if (!all_fit && Wj + carry_w > avg) break;   // no later candidate can fit
        }
        if (acc_w) atomicAdd(ull(&accw_sh), (unsigned long long)acc_w);
        __syncthreads();
        if (tid == 0) {
          nstep_sh = carry_c;
          Wj_sh = Wj + accw_sh;
        }
        __syncthreads();
        const int32_t ns2 = nstep_sh;
        if (ns2 == 0) break;
        for (int32_t q = tid; q < ns2; q += GNT) a.label[stp[q]] = (int32_t)(bo + j);
        __syncthreads();
      }
      if (tid == 0) a.W[bo + j] = (wgt_t)Wj_sh;
      __syncthreads();
    }
    // water-filling of the nodes left unassigned
    int64_t r = 0;
    for (int64_t v = tid; v < n; v += GNT)
      if (a.label[base + v] < 0) r += a.nw[base + v];
    const int64_t R = block_sum<GNT>(r, sh);
    if (R > 0) {
      if (tid == 0) {
        int64_t lo = a.W[bo], hi = a.W[bo];
        for (int32_t b = 1; b < k; ++b) {
          lo = min64(lo, (int64_t)a.W[bo + b]);
          hi = max64(hi, (int64_t)a.W[bo + b]);
        }
        hi += R;
        while (lo < hi) {
          const int64_t mid = lo + (hi - lo) / 2;
          int64_t f = 0;
          for (int32_t b = 0; b < k; ++b) f += max64(0, mid - (int64_t)a.W[bo + b]);
          if (f >= R) hi = mid; else lo = mid + 1;
        }
        const int64_t L = lo;
        for (int32_t j = 0; j < k; ++j) {       // insertion sort by (W, id)
          int32_t b = j;
          int32_t p = j;
          while (p > 0) {
            const int32_t q = a.wforder[bo + p - 1];
            if (a.W[bo + q] > a.W[bo + b] || (a.W[bo + q] == a.W[bo + b] && q > b)) {
              a.wforder[bo + p] = q;
              --p;
            } else {
              break;
            }
          }
          a.wforder[bo + p] = b;
        }
        int64_t acc = 0;
        for (int32_t j = 0; j < k; ++j) {
          a.wfA[bo + j] = acc;
          acc += max64(0, L - (int64_t)a.W[bo + a.wforder[bo + j]]);
        }
      }
      __syncthreads();
      int64_t carry = 0;
      for (int64_t v0 = 0; v0 < n; v0 += GNT) {
        const int64_t v = v0 + tid;
        const bool left = v < n && a.label[base + v] < 0;
        const int64_t wt = left ? a.nw[base + v] : 0;
        int64_t tw;
        const int64_t iw = block_incl_scan<GNT>(wt, sh, &tw);
        if (left) {
          const int64_t p = carry + iw - wt;
          int32_t lo = 0, hi = k - 1;               // last j with A[j] <= p
          while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (a.wfA[bo + mid] <= p) lo = mid; else hi = mid - 1;
          }
          const int32_t b = a.wforder[bo + lo];
          a.label[base + v] = (int32_t)(bo + b);
          atomicAdd(&a.W[bo + b], (wgt_t)wt);
        }
        carry += tw;
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------------
// Greedy growing of few, large trials: each trial is grown by a group of cpt
// CTAs of one cooperative launch (CTAs g * cpt .. g * cpt + cpt - 1 grow
// trial slot g), with the same rules as k_ggg.  The group shares the
// trial's step and front lists and a few counters in global memory and
// meets at a barrier of its own (bounded wait: a wait that runs out sets
// DERR_TIMEOUT and the group leaves).  Each CTA owns a contiguous range of
// the trial's nodes for the scans (seed search, ordered candidates,
// water-filling); id-ordered prefixes over the whole trial are the CTAs'
// partial sums in rank order plus the CTA's own scan.  The step nodes'
// arcs are shared out by step node in chunks of GG_NT per CTA; a step node
// with more than GG_HEAVY arcs (known in advance: the step that builds the
// next step records whether it took one) is listed instead, and after a
// group barrier the listed rows are read by all CTAs of the group together.
// Every decision is a set or an id-ordered prefix, so the result equals
// k_ggg's.
struct GroupState {
  GridSync bar;
  int32_t nstep, nfront, nnext, seed;
  int64_t Wj, fsum, accw;
  // heavy step nodes (more than GG_HEAVY arcs): whether the current step
  // has any, whether the frontier / the ordered selection being built took
  // one, and the current step's list length
  int32_t step_heavy, front_heavy, next_heavy, nheavy;
};
constexpr int GG_NT = 512;
constexpr int64_t GG_HEAVY = 8 * GG_NT;

// Assigned-node bitmap of the grouped growing (one bit per node of the
// trial level, set when a growth step assigns the node): the arc passes ask
// it whether a head is still free, a read that stays in L2 where the label
// array (32 bits per node, one trial copy per slot) does not.
__device__ __forceinline__ bool is_assigned(const uint32_t* asg, int64_t y) {
  return (asg[y >> 5] >> (y & 31)) & 1u;
}
__device__ __forceinline__ void mark_assigned(uint32_t* asg, int64_t y) {
  atomicOr(&asg[y >> 5], 1u << (y & 31));
}

__global__ void __launch_bounds__(GG_NT) k_ggg_group(GGGArgs a, int32_t cpt, GroupState* gst,
                                                     uint64_t* ph, int32_t* pv, int64_t* pw,
                                                     uint32_t lim) {
  __shared__ int64_t sh[33];
  __shared__ uint64_t shh[GG_NT / 32];
  __shared__ int32_t shv[GG_NT / 32];
  __shared__ int64_t st_rs[GG_NT], st_ex[GG_NT], st_in[GG_NT];
  __shared__ int64_t pre_sh, tot_sh;
  __shared__ int32_t seed_sh;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int32_t s = (int32_t)(blockIdx.x / cpt);
  const int r = (int)(blockIdx.x % cpt);
  GroupState* st = gst + s;
  uint64_t* gph = ph + (int64_t)s * cpt;
  int32_t* gpv = pv + (int64_t)s * cpt;
  int64_t* gpw = pw + (int64_t)s * cpt;
  const int64_t base = a.noff[s], n = a.noff[s + 1] - base;
  const int32_t k = a.nlab[s];
  const int64_t bo = a.boff[s], avg = a.avg[s];
  const uint64_t tkey = a.tkey[s];
  const int32_t lvl = a.level[s];
  const int64_t r0 = n * r / cpt, r1 = n * (r + 1) / cpt;   // this CTA's node range
  const int64_t qstride = (int64_t)GG_NT * cpt;            // step-list share-out
  auto sync = [&]() { return group_sync(&st->bar, (unsigned)cpt, a.err, lim); };
  // exclusive prefix and total over the CTAs of the group of the values
  // they left in gpw (after a barrier)
  auto group_prefix = [&]() {
    if (tid == 0) {
      int64_t p = 0, t = 0;
      for (int q = 0; q < cpt; ++q) {
        const int64_t x = *(volatile int64_t*)&gpw[q];
        if (q < r) p += x;
        t += x;
      }
      pre_sh = p;
      tot_sh = t;
    }
    __syncthreads();
  };
  for (int64_t v = r0 + tid; v < r1; v += GG_NT) a.label[base + v] = -1;
  if (r == 0)
    for (int32_t b = tid; b < k; b += GG_NT) a.W[bo + b] = 0;
  if (!sync()) return;
  int32_t* stp = a.step + base;
  int32_t* frt = a.front + base;
  int32_t* hvl = a.heavy + base;
  for (int32_t j = 0; j < k; ++j) {
    // seed: unassigned non-isolated node with the smallest hash (the same
    // pass clears the connections of the previous block)
    const uint64_t skey = hkey(tkey, PH_GGG, (uint64_t)lvl, (uint64_t)j);
    uint64_t bh = ~0ull;
    int32_t bv = -1;
    for (int64_t v = r0 + tid; v < r1; v += GG_NT) {
      const int64_t gv = base + v;
      a.conn[gv] = 0;
      if (a.label[gv] >= 0 || a.row_ptr[gv + 1] == a.row_ptr[gv]) continue;
      const uint64_t h = mix64(skey ^ (uint64_t)v);
      if (bv < 0 || h < bh) { bh = h; bv = (int32_t)v; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t oh = __shfl_xor_sync(0xffffffffu, (unsigned long long)bh, o);
      const int32_t ov = __shfl_xor_sync(0xffffffffu, bv, o);
      if (ov >= 0 && (bv < 0 || oh < bh || (oh == bh && ov < bv))) { bh = oh; bv = ov; }
    }
    if (lane == 0) { shh[wid] = bh; shv[wid] = bv; }
    __syncthreads();
    if (tid == 0) {
      uint64_t h = ~0ull;
      int32_t v = -1;
      for (int w = 0; w < GG_NT / 32; ++w)
        if (shv[w] >= 0 && (v < 0 || shh[w] < h || (shh[w] == h && shv[w] < v))) {
          h = shh[w]; v = shv[w];
        }
      gph[r] = h;
      gpv[r] = v;
    }
    if (!sync()) return;
    if (tid == 0) {
      uint64_t h = ~0ull;
      int32_t v = -1;
      for (int q = 0; q < cpt; ++q) {
        const uint64_t qh = *(volatile uint64_t*)&gph[q];
        const int32_t qv = *(volatile int32_t*)&gpv[q];
        if (qv >= 0 && (v < 0 || qh < h || (qh == h && qv < v))) { h = qh; v = qv; }
      }
      seed_sh = v;
    }
    __syncthreads();
    const int32_t seed = seed_sh;
    if (seed < 0) break;
    if (r == 0 && tid == 0) {
      a.label[base + seed] = (int32_t)(bo + j);
      mark_assigned(a.asg, base + seed);
      stp[0] = (int32_t)(base + seed);
      st->nstep = 1;
      st->nfront = 0;
      st->nnext = 0;
      st->fsum = 0;
      st->accw = 0;
      st->Wj = a.nw[base + seed];
      st->step_heavy = a.row_ptr[base + seed + 1] - a.row_ptr[base + seed] > GG_HEAVY;
      st->front_heavy = 0;
      st->next_heavy = 0;
      st->nheavy = 0;
    }
    bool ordered = false;
    if (!sync()) return;
    while (true) {
      const int32_t nstep = *(volatile int32_t*)&st->nstep;
      const bool hv_step = *(volatile int32_t*)&st->step_heavy != 0;
      int64_t fw = 0;
      // an arc out of the step: connection of an unassigned head; its first
      // arc lists it as reached (weights > 0)
      auto visit = [&](int64_t e) {
        const int32_t y = a.col[e];
        if (!SCLAP_OK(y, a.N, a.err) || is_assigned(a.asg, y)) return;
        const unsigned long long old = atomicAdd(ull(&a.conn[y]), (unsigned long long)a.ew[e]);
        if (!ordered && old == 0) {
          frt[atomicAdd(&st->nfront, 1)] = y;
          fw += a.nw[y];
          if (a.row_ptr[y + 1] - a.row_ptr[y] > GG_HEAVY)
            *(volatile int32_t*)&st->front_heavy = 1;
        }
      };
      for (int64_t q0 = (int64_t)r * GG_NT; q0 < nstep; q0 += qstride) {
        const int64_t q = q0 + tid;
        int64_t rs = 0, d = 0;
        if (q < nstep) {
          const int32_t u = stp[q];
          rs = a.row_ptr[u];
          d = a.row_ptr[u + 1] - rs;
          if (hv_step && d > GG_HEAVY) {          // read by the whole group below
            hvl[atomicAdd(&st->nheavy, 1)] = u;
            d = 0;
          }
        }
        int64_t tot;
        const int64_t incl = block_incl_scan<GG_NT>(d, sh, &tot);
        st_rs[tid] = rs;
        st_ex[tid] = incl - d;
        st_in[tid] = incl;
        __syncthreads();
        const int cnt = (int)min64(GG_NT, nstep - q0);
        for (int64_t x = tid; x < tot; x += GG_NT) {
          int lo = 0, hi = cnt - 1;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (st_in[mid] > x) hi = mid; else lo = mid + 1;
          }
          visit(st_rs[lo] + (x - st_ex[lo]));
        }
        __syncthreads();
      }
      if (hv_step) {
        if (!sync()) return;                     // the heavy list is complete
        const int32_t nh = *(volatile int32_t*)&st->nheavy;
        for (int32_t hq = 0; hq < nh; ++hq) {
          const int32_t u = hvl[hq];
          const int64_t re = a.row_ptr[u + 1];
          for (int64_t e = a.row_ptr[u] + (int64_t)r * GG_NT + tid; e < re; e += qstride)
            visit(e);
        }
      }
      const int64_t fwb = block_sum<GG_NT>(fw, sh);
      if (tid == 0 && fwb) atomicAdd(ull(&st->fsum), (unsigned long long)fwb);
      if (!sync()) return;
      const int64_t Wj = *(volatile int64_t*)&st->Wj;
      if (Wj >= avg) break;
      if (!ordered) {
        const int64_t fsum = *(volatile int64_t*)&st->fsum;
        const int32_t nf = *(volatile int32_t*)&st->nfront;
        if (Wj + fsum <= avg) {
          // all of them fit: they are the next step, in any order
          for (int64_t q = (int64_t)r * GG_NT + tid; q < nf; q += qstride) {
            a.label[frt[q]] = (int32_t)(bo + j);
            mark_assigned(a.asg, frt[q]);
          }
          int32_t* t = stp; stp = frt; frt = t;
          if (!sync()) return;
          if (r == 0 && tid == 0) {
            st->nstep = nf;
            st->nfront = 0;
            st->fsum = 0;
            st->Wj = Wj + fsum;
            st->step_heavy = st->front_heavy;
            st->front_heavy = 0;
            st->nheavy = 0;
          }
          if (!sync()) return;
          if (nf == 0) break;
          continue;
        }
        ordered = true;
      }
      // connected unassigned nodes in id order, longest prefix that fits:
      // this CTA's range starts after the candidate weight of the ranks below
      int64_t cw = 0;
      for (int64_t v = r0 + tid; v < r1; v += GG_NT)
        if (a.label[base + v] < 0 && a.conn[base + v] > 0) cw += a.nw[base + v];
      const int64_t cwb = block_sum<GG_NT>(cw, sh);
      if (tid == 0) gpw[r] = cwb;
      if (!sync()) return;
      group_prefix();
      const bool all_fit = Wj + tot_sh <= avg;
      int64_t carry_w = pre_sh, acc_w = 0;
      for (int64_t c0 = r0; c0 < r1; c0 += GG_NT) {
        if (!all_fit && Wj + carry_w > avg) break;          // no later candidate fits
        const int64_t v = c0 + tid;
        const bool cand = v < r1 && a.label[base + v] < 0 && a.conn[base + v] > 0;
        const int64_t wt = cand ? a.nw[base + v] : 0;
        int64_t tw;
        const int64_t iw = block_incl_scan<GG_NT>(wt, sh, &tw);
        if (cand && (all_fit || Wj + carry_w + iw <= avg)) {
          stp[atomicAdd(&st->nnext, 1)] = (int32_t)(base + v);
          acc_w += wt;
          if (a.row_ptr[base + v + 1] - a.row_ptr[base + v] > GG_HEAVY)
            *(volatile int32_t*)&st->next_heavy = 1;
        }
        carry_w += tw;
      }
      const int64_t accb = block_sum<GG_NT>(acc_w, sh);
      if (tid == 0 && accb) atomicAdd(ull(&st->accw), (unsigned long long)accb);
      if (!sync()) return;
      const int32_t ns2 = *(volatile int32_t*)&st->nnext;
      const int64_t newW = Wj + *(volatile int64_t*)&st->accw;
      for (int64_t q = (int64_t)r * GG_NT + tid; q < ns2; q += qstride) {
        a.label[stp[q]] = (int32_t)(bo + j);
        mark_assigned(a.asg, stp[q]);
      }
      if (!sync()) return;
      if (r == 0 && tid == 0) {
        st->nstep = ns2;
        st->Wj = newW;
        st->nnext = 0;
        st->accw = 0;
        st->step_heavy = st->next_heavy;
        st->next_heavy = 0;
        st->front_heavy = 0;
        st->nheavy = 0;
      }
      if (!sync()) return;
      if (ns2 == 0) break;
    }
    if (r == 0 && tid == 0) a.W[bo + j] = (wgt_t)*(volatile int64_t*)&st->Wj;
    if (!sync()) return;
  }
  // water-filling of the nodes left unassigned, in id order over the trial
  int64_t rw = 0;
  for (int64_t v = r0 + tid; v < r1; v += GG_NT)
    if (a.label[base + v] < 0) rw += a.nw[base + v];
  const int64_t rwb = block_sum<GG_NT>(rw, sh);
  if (tid == 0) gpw[r] = rwb;
  if (!sync()) return;
  group_prefix();
  const int64_t R = tot_sh;
  if (R == 0) return;
  if (r == 0 && tid == 0) {
    int64_t lo = a.W[bo], hi = a.W[bo];
    for (int32_t b = 1; b < k; ++b) {
      lo = min64(lo, (int64_t)a.W[bo + b]);
      hi = max64(hi, (int64_t)a.W[bo + b]);
    }
    hi += R;
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      int64_t f = 0;
      for (int32_t b = 0; b < k; ++b) f += max64(0, mid - (int64_t)a.W[bo + b]);
      if (f >= R) hi = mid; else lo = mid + 1;
    }
    const int64_t L = lo;
    for (int32_t jj = 0; jj < k; ++jj) {       // insertion sort by (W, id)
      int32_t p = jj;
      while (p > 0) {
        const int32_t q = a.wforder[bo + p - 1];
        if (a.W[bo + q] > a.W[bo + jj] || (a.W[bo + q] == a.W[bo + jj] && q > jj)) {
          a.wforder[bo + p] = q;
          --p;
        } else {
          break;
        }
      }
      a.wforder[bo + p] = jj;
    }
    int64_t acc = 0;
    for (int32_t jj = 0; jj < k; ++jj) {
      a.wfA[bo + jj] = acc;
      acc += max64(0, L - (int64_t)a.W[bo + a.wforder[bo + jj]]);
    }
  }
  if (!sync()) return;
  int64_t carry = pre_sh;
  for (int64_t v0 = r0; v0 < r1; v0 += GG_NT) {
    const int64_t v = v0 + tid;
    const bool left = v < r1 && a.label[base + v] < 0;
    const int64_t wt = left ? a.nw[base + v] : 0;
    int64_t tw;
    const int64_t iw = block_incl_scan<GG_NT>(wt, sh, &tw);
    if (left) {
      const int64_t p = carry + iw - wt;
      int32_t lo = 0, hi = k - 1;               // last j with A[j] <= p
      while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (a.wfA[bo + mid] <= p) lo = mid; else hi = mid - 1;
      }
      const int32_t b = a.wforder[bo + lo];
      a.label[base + v] = (int32_t)(bo + b);
      atomicAdd(&a.W[bo + b], (wgt_t)wt);
    }
    carry += tw;
  }
}

// Twice the cut of every slot: 32 nodes per warp, their arcs spread over
// the lanes.  When the warp's 32 nodes lie in one slot (all but the groups
// that straddle a slot boundary) each lane sums in a register and the warp
// merges once per group; otherwise every cut arc is added on its own.  Rows
// longer than CUT_CH arcs are queued in chunks of CUT_CH arcs for
// k_slot_cut_long instead (at most 2 * arcs / CUT_CH chunks).
constexpr int64_t CUT_CH = 4096;
struct CutChunk {
  int64_t lo, hi;
  int32_t v, pad;
};
__global__ void __launch_bounds__(256) k_slot_cut(const int64_t* __restrict__ row_ptr,
                                                  const int32_t* __restrict__ col,
                                                  const int32_t* __restrict__ ew,
                                                  const int32_t* __restrict__ gid,
                                                  const int32_t* __restrict__ label, int64_t N,
                                                  int64_t* __restrict__ cut2,
                                                  CutChunk* __restrict__ q, int32_t* qn) {
  __shared__ int sh_slot;
  __shared__ unsigned long long sh_sum;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (threadIdx.x == 0) {
    const int64_t v0 = (int64_t)blockIdx.x * blockDim.x;
    sh_slot = v0 < N ? slot_at(gid, v0) : -1;
    sh_sum = 0;
  }
  __syncthreads();
  for (int64_t base = w0 * 32; base < N; base += nwarps * 32) {
    const int64_t v = base + lane;
    int64_t rs = 0, d = 0;
    int32_t lv = 0, s = -1;
    if (v < N) {
      rs = row_ptr[v];
      d = row_ptr[v + 1] - rs;
      lv = label[v];
      s = slot_at(gid, v);
      if (d > CUT_CH) {
        const int32_t nch = (int32_t)((d + CUT_CH - 1) / CUT_CH);
        const int32_t q0 = atomicAdd(qn, nch);
        for (int32_t c = 0; c < nch; ++c)
          q[q0 + c] = CutChunk{rs + c * CUT_CH, min64(rs + (c + 1) * CUT_CH, rs + d), (int32_t)v, 0};
        d = 0;
      }
    }
    long long incl = d;
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const long long excl = incl - d;
    const long long total = __shfl_sync(0xffffffffu, incl, 31);
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
      const int32_t lvL = __shfl_sync(0xffffffffu, lv, L);
      const int32_t sL = __shfl_sync(0xffffffffu, s, L);
      if (x < total) {
        const int64_t e = rsL + (x - exL);
        if (label[col[e]] != lvL) {
          const int32_t w = wat(ew, e);
          if (uni) acc += (unsigned long long)w;
          else if (sL == sh_slot) atomicAdd(&sh_sum, (unsigned long long)w);
          else atomicAdd(ull(&cut2[sL]), (unsigned long long)w);
        }
      }
    }
    if (uni) {
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0 && acc) {
        if (s0 == sh_slot) atomicAdd(&sh_sum, acc);
        else atomicAdd(ull(&cut2[s0]), acc);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && sh_sum) atomicAdd(ull(&cut2[sh_slot]), sh_sum);
}

// The queued chunks of long rows: one CTA per chunk, one atomic per chunk.
__global__ void __launch_bounds__(256) k_slot_cut_long(const int32_t* __restrict__ col,
                                                       const int32_t* __restrict__ ew,
                                                       const int32_t* __restrict__ gid,
                                                       const int32_t* __restrict__ label,
                                                       const CutChunk* __restrict__ q,
                                                       const int32_t* qn,
                                                       int64_t* __restrict__ cut2) {
  __shared__ unsigned long long sh[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int32_t n = *qn;
  for (int32_t i = blockIdx.x; i < n; i += gridDim.x) {
    const CutChunk c = q[i];
    const int32_t lv = label[c.v];
    unsigned long long acc = 0;
    for (int64_t e = c.lo + threadIdx.x; e < c.hi; e += blockDim.x)
      if (label[col[e]] != lv) acc += (unsigned long long)wat(ew, e);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sh[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < 8; ++w) t += sh[w];
      if (t) atomicAdd(ull(&cut2[slot_at(gid, c.v)]), t);
    }
    __syncthreads();
  }
}

// Best trial of each task (a graph's trials of one group): least overload,
// then least cut; it replaces the graph's best so far only if better (the
// groups run in trial order, so the first best trial wins ties).  take[i] =
// the task's trial to copy out, or -1.
__global__ void k_select_best(const SelectTask* __restrict__ tasks, int32_t ntasks,
                              const int64_t* __restrict__ cut2, const wgt_t* __restrict__ ip_W,
                              const int64_t* __restrict__ ip_boff, int32_t* __restrict__ best,
                              int64_t* __restrict__ ipcut, int64_t* __restrict__ rb_ov,
                              int32_t* __restrict__ take) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntasks) return;
  const SelectTask t = tasks[i];
  int64_t bo = -1, bc = -1;
  int32_t bt = -1;
  for (int32_t tr = 0; tr < t.trials; ++tr) {
    const int64_t slot = t.slot0 + tr;
    int64_t mx = 0;
    for (int32_t b = 0; b < t.k; ++b) mx = max64(mx, (int64_t)ip_W[ip_boff[slot] + b]);
    const int64_t ov = max64(0, mx - t.Lmax);
    const int64_t c = cut2[slot] / 2;
    if (bt < 0 || ov < bo || (ov == bo && c < bc)) { bo = ov; bc = c; bt = tr; }
  }
  const bool tk = best[t.g] < 0 || bo < rb_ov[t.g] || (bo == rb_ov[t.g] && bc < ipcut[t.g]);
  if (tk) {
    best[t.g] = t.trial0 + bt;
    ipcut[t.g] = bc;
    rb_ov[t.g] = bo;
  }
  take[i] = tk ? bt : -1;
}

// Copies the taken trial's blocks out: tasks along y, chunks of SC_CH nodes
// along x.
constexpr int64_t SC_CH = 65536;
__global__ void k_copy_best(const SelectTask* __restrict__ tasks, const int32_t* __restrict__ take,
                            const int64_t* __restrict__ ip_noff, const int64_t* __restrict__ ip_boff,
                            const int32_t* __restrict__ ip_label, const wgt_t* __restrict__ ip_W,
                            wgt_t* __restrict__ Wg) {
  const int32_t bt = take[blockIdx.y];
  if (bt < 0) return;
  const SelectTask t = tasks[blockIdx.y];
  const int64_t slot = t.slot0 + bt;
  const int64_t src = ip_noff[slot], sbo = ip_boff[slot];
  const int64_t v1 = min64(((int64_t)blockIdx.x + 1) * SC_CH, t.n);
  for (int64_t v = (int64_t)blockIdx.x * SC_CH + threadIdx.x; v < v1; v += blockDim.x) {
    int64_t d = v;
    if (t.rank) {
      const int64_t r0 = t.rank[t.dst_n0 + v];
      if (t.rank[t.dst_n0 + v + 1] == r0) { t.dst_blk[t.dst_n0 + v] = -1; continue; }
      d = r0 - t.rbase;
    }
    t.dst_blk[t.dst_n0 + v] = (int32_t)(t.g_boff + (ip_label[src + d] - sbo));
  }
  if (blockIdx.x == 0)
    for (int32_t b = threadIdx.x; b < t.k; b += blockDim.x) Wg[t.g_boff + b] = ip_W[sbo + b];
}

__global__ void k_project(const int32_t* __restrict__ cmap, const int32_t* __restrict__ cblk,
                          int32_t* __restrict__ fblk, int64_t N) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cmap[v];
    if (c >= 0) fblk[v] = cblk[c];
  }
}

__global__ void k_lift_blocks(const int32_t* __restrict__ cmap, const int32_t* __restrict__ fblk,
                              int32_t* __restrict__ cblk, int64_t N) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cmap[v];
    if (c >= 0) cblk[c] = fblk[v];
  }
}

__global__ void k_block_weights(const int32_t* __restrict__ label, const int32_t* __restrict__ nw,
                                int64_t N, wgt_t* __restrict__ W) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&W[label[v]], (wgt_t)wat(nw, v));
}

__global__ void k_isolated(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ nw,
                           int64_t N, uint8_t* __restrict__ flags, int32_t* __restrict__ iso_w) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    const bool has = row_ptr[v + 1] > row_ptr[v];
    flags[v] = has ? 1 : 0;
    iso_w[v] = has ? 0 : wat(nw, v);
  }
}

// One thread per graph: fill level L (smallest L with sum_b max(0, L - W_b)
// >= R), blocks ordered by (weight, id), and the start of each block's
// stretch of free capacity below L.
__global__ void k_wf_setup(const FillTask* __restrict__ tasks, int ntasks, const wgt_t* Wg,
                           int32_t* order, int64_t* A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntasks) return;
  const FillTask t = tasks[i];
  const int64_t R = t.iso_prefix[t.n0 + t.n] - t.iso_prefix[t.n0];
  if (R == 0) return;
  const wgt_t* W = Wg + t.g_boff;
  int64_t lo = W[0], hi = W[0];
  for (int32_t b = 1; b < t.k; ++b) { lo = min64(lo, (int64_t)W[b]); hi = max64(hi, (int64_t)W[b]); }
  hi += R;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    int64_t f = 0;
    for (int32_t b = 0; b < t.k; ++b) f += max64(0, mid - (int64_t)W[b]);
    if (f >= R) hi = mid; else lo = mid + 1;
  }
  int32_t* ord = order + t.g_boff;
  for (int32_t j = 0; j < t.k; ++j) {
    int32_t p = j;
    while (p > 0) {
      const int32_t q = ord[p - 1];
      if (W[q] > W[j] || (W[q] == W[j] && q > j)) { ord[p] = q; --p; } else break;
    }
    ord[p] = j;
  }
  int64_t acc = 0;
  for (int32_t j = 0; j < t.k; ++j) {
    A[t.g_boff + j] = acc;
    acc += max64(0, lo - (int64_t)W[ord[j]]);
  }
}

__global__ void k_wf_assign(const FillTask* __restrict__ tasks, wgt_t* Wg,
                            const int32_t* __restrict__ order, const int64_t* __restrict__ A) {
  const FillTask t = tasks[blockIdx.y];
  const int64_t base = t.iso_prefix[t.n0];
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < t.n;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (t.blk[t.n0 + v] >= 0) continue;
    const int64_t p = t.iso_prefix[t.n0 + v] - base;
    int32_t lo = 0, hi = t.k - 1;   // last j with A[j] <= p
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (A[t.g_boff + mid] <= p) lo = mid; else hi = mid - 1;
    }
    const int32_t b = order[t.g_boff + lo];
    t.blk[t.n0 + v] = (int32_t)(t.g_boff + b);
    atomicAdd(&Wg[t.g_boff + b], (wgt_t)wat(t.nw, t.n0 + v));
  }
}

}  // namespace

void isolated_flags(const int64_t* row_ptr, const int32_t* nw, int64_t N, uint8_t* flags,
                    int32_t* iso_w, cudaStream_t s) {
  if (N <= 0) return;
  k_isolated<<<grid_for(N, 256, (int64_t)num_sms() * 16), 256, 0, s>>>(row_ptr, nw, N, flags, iso_w); SCLAP_NOTE_LAUNCH("k_isolated");
  SCLAP_LAUNCH_CHECK();
}

void waterfill_isolated(const std::vector<FillTask>& tasks, wgt_t* Wg, int64_t Ktot,
                        cudaStream_t s) {
  if (tasks.empty()) return;
  DevBuf<FillTask> d(tasks.size(), s);
  d.upload(tasks);
  DevBuf<int32_t> order(std::max<int64_t>(Ktot, 1), s);
  DevBuf<int64_t> A(std::max<int64_t>(Ktot, 1), s);
  const int nt = (int)tasks.size();
  k_wf_setup<<<(nt + 127) / 128, 128, 0, s>>>(d.p, nt, Wg, order.p, A.p); SCLAP_NOTE_LAUNCH("k_wf_setup");
  int64_t mx = 1;
  for (const auto& t : tasks) mx = std::max(mx, t.n);
  const int64_t per_task = std::max<int64_t>(64, (int64_t)num_sms() * 8 / nt);
  for (int t0 = 0; t0 < nt; t0 += 65535) {
    dim3 grid(grid_for(mx, 256, per_task), (unsigned)std::min(65535, nt - t0));
    k_wf_assign<<<grid, 256, 0, s>>>(d.p + t0, Wg, order.p, A.p); SCLAP_NOTE_LAUNCH("k_wf_assign");
  }
  SCLAP_LAUNCH_CHECK();
  stream_sync(s);   // task array freed on return
}

void ip_replicate(const std::vector<CopyTask>& tasks, int64_t* row_ptr, int32_t* col,
                  int32_t* ew, int32_t* nw, int64_t M_total, cudaStream_t s,
                  int64_t N_total_override) {
  if (tasks.empty()) return;
  // the first task of each source segment copies from the source, the
  // others from that copy
  std::vector<CopyTask> first;
  std::vector<CopyFrom> later;
  std::map<std::tuple<const void*, int64_t, int64_t, int64_t, const void*, int64_t>, size_t> seen;
  for (const auto& t : tasks) {
    const auto key = std::make_tuple((const void*)t.col, t.src_n0, t.src_a0, t.m,
                                     (const void*)t.rank, t.rbase);
    const auto it = seen.find(key);
    if (it == seen.end()) {
      seen.emplace(key, first.size());
      first.push_back(t);
    } else {
      const CopyTask& f = first[it->second];
      later.push_back(CopyFrom{t.dst_n0, t.dst_a0, f.dst_n0, f.dst_a0, t.nd ? t.nd : t.n, t.m});
    }
  }
  DevBuf<CopyTask> d(first.size(), s);
  d.upload(first);
  int64_t mx = 1;
  for (const auto& t : first) mx = std::max(mx, std::max(t.n, t.m));
  // at least 64 CTAs per task, more when few tasks would leave SMs idle
  const int64_t per_task = std::max<int64_t>(64, (int64_t)num_sms() * 8 / (int64_t)first.size());
  for (size_t t0 = 0; t0 < first.size(); t0 += 65535) {
    const unsigned ny = (unsigned)std::min<size_t>(65535, first.size() - t0);
    dim3 grid(grid_for(mx, 256, per_task), ny);
    k_replicate<<<grid, 256, 0, s>>>(d.p + t0, row_ptr, col, ew, nw); SCLAP_NOTE_LAUNCH("k_replicate");
  }
  DevBuf<CopyFrom> dl(std::max<size_t>(later.size(), 1), s);
  if (!later.empty()) {
    dl.upload(later);
    int64_t ml = 1;
    for (const auto& t : later) ml = std::max(ml, std::max(t.nd, t.m));
    const int64_t per_l = std::max<int64_t>(64, (int64_t)num_sms() * 8 / (int64_t)later.size());
    for (size_t t0 = 0; t0 < later.size(); t0 += 65535) {
      const unsigned ny = (unsigned)std::min<size_t>(65535, later.size() - t0);
      dim3 grid(grid_for(ml, 256, per_l), ny);
      k_replicate_from<<<grid, 256, 0, s>>>(dl.p + t0, row_ptr, col, ew, nw); SCLAP_NOTE_LAUNCH("k_replicate_from");
    }
  }
  int64_t endv = M_total;
  int64_t Ntot = 0;
  for (const auto& t : tasks) {
    const int64_t nd = t.rank ? 0 : t.n;   // renumbered tasks: caller passes dst end below
    Ntot = std::max(Ntot, t.dst_n0 + nd);
  }
  if (N_total_override >= 0) Ntot = N_total_override;
  SCLAP_CUDA(cudaMemcpyAsync(row_ptr + Ntot, &endv, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  stream_sync(s);   // endv lives on the host stack
  SCLAP_LAUNCH_CHECK();
}

void ggg_trials(const GGGArgs& a_in, const std::vector<int64_t>& noff,
                const std::vector<int32_t>& nlab, cudaStream_t s) {
  if (a_in.nslots <= 0) return;
  const int32_t S = a_in.nslots;
  // longest processing time first: trial slots by node count, descending
  std::vector<int32_t> order(S);
  for (int32_t i = 0; i < S; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
    return noff[x + 1] - noff[x] > noff[y + 1] - noff[y];
  });
  DevBuf<int32_t> d_order(S, s), d_next(1, s);
  d_order.upload(order);
  d_next.zero();
  GGGArgs a = a_in;
  a.order = d_order.p;
  a.next = d_next.p;
  // a trial is a chain of small steps, so the kernel is bound by how many
  // trials are in flight: small CTAs when the trials outnumber the resident
  // 512-thread CTAs
  int few_per_sm = 0, many_per_sm = 0;
  SCLAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&few_per_sm, k_ggg<GNT_FEW>, GNT_FEW, 0));
  SCLAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&many_per_sm, k_ggg<GNT_MANY>, GNT_MANY, 0));
  const int64_t few_resident = (int64_t)num_sms() * std::max(few_per_sm, 1);
  const int64_t many_resident = (int64_t)num_sms() * std::max(many_per_sm, 1);
  // few trials of large blocks: a group of CTAs per trial (the resident
  // CTAs shared out, at most 256 per trial, and only when every trial gets
  // at least 4).  A growth step
  // costs the group a few barriers, so the groups pay off only when the
  // blocks are large: measured faster on R-MAT scale 22 at k = 2 and 8 and
  // on scale 25 at k = 16 (1149 -> 369 ms), slower on scale 22 at k = 32
  // and 64, and the same gate cannot separate them at 2^16 or 2^17 nodes per
  // block (scale 22, k = 8 fell below 2^15 as well); the gate is 2^14
  // nodes per block on average in some trial.
  int group_per_sm = 0;
  SCLAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&group_per_sm, k_ggg_group, GG_NT, 0));
  const int64_t group_resident = (int64_t)num_sms() * std::max(group_per_sm, 1);
  const int64_t cpt = std::min<int64_t>(256, group_resident / S);
  int64_t per_block = 0;
  for (int32_t i = 0; i < S; ++i)
    per_block = std::max(per_block, (noff[i + 1] - noff[i]) / std::max<int32_t>(1, nlab[i]));
  if (cpt >= 4 && per_block >= ((int64_t)1 << 14)) {
    DevBuf<GroupState> gs(S, s);
    DevBuf<uint32_t> asg((size_t)((a.N + 31) / 32 + 1), s);
    asg.zero();
    a.asg = asg.p;
    DevBuf<uint64_t> ph(S * cpt, s);
    DevBuf<int32_t> pv(S * cpt, s);
    DevBuf<int64_t> pw(S * cpt, s);
    gs.zero();
    launch_coop(k_ggg_group, (unsigned)(S * cpt), GG_NT, 0, s, a, (int32_t)cpt, gs.p, ph.p, pv.p,
                pw.p, wait_limit()); SCLAP_NOTE_LAUNCH("k_ggg_group");
    SCLAP_LAUNCH_CHECK();
    return;
  }
  if (S > few_resident) {
    k_ggg<GNT_MANY><<<(unsigned)std::min<int64_t>(S, many_resident), GNT_MANY, 0, s>>>(a); SCLAP_NOTE_LAUNCH("k_ggg");
  } else {
    k_ggg<GNT_FEW><<<(unsigned)std::min<int64_t>(S, few_resident), GNT_FEW, 0, s>>>(a); SCLAP_NOTE_LAUNCH("k_ggg");
  }
  SCLAP_LAUNCH_CHECK();
}

void slot_cut(const LevelView& lv, const int32_t* label, int64_t* cut2, cudaStream_t s) {
  if (lv.N <= 0) return;
  DevBuf<CutChunk> q((size_t)(2 * (lv.M / CUT_CH) + 2), s);
  DevBuf<int32_t> qn(1, s);
  qn.zero();
  k_slot_cut<<<grid_for(lv.N, 256, (int64_t)num_sms() * 16), 256, 0, s>>>(
      lv.row_ptr, lv.col, lv.ew, lv.gid, label, lv.N, cut2, q.p, qn.p); SCLAP_NOTE_LAUNCH("k_slot_cut");
  k_slot_cut_long<<<(unsigned)num_sms() * 8, 256, 0, s>>>(lv.col, lv.ew, lv.gid, label, q.p, qn.p,
                                                          cut2); SCLAP_NOTE_LAUNCH("k_slot_cut_long");
  SCLAP_LAUNCH_CHECK();
}

void ip_select_copy(const std::vector<SelectTask>& tasks, const int64_t* cut2,
                    const wgt_t* ip_W, const int64_t* ip_noff, const int64_t* ip_boff,
                    const int32_t* ip_label, wgt_t* Wg, int32_t* best, int64_t* ipcut,
                    int64_t* rb_ov, cudaStream_t s) {
  if (tasks.empty()) return;
  const int32_t nt = (int32_t)tasks.size();
  DevBuf<SelectTask> d(nt, s);
  DevBuf<int32_t> take(nt, s);
  d.upload(tasks);
  k_select_best<<<(nt + 127) / 128, 128, 0, s>>>(d.p, nt, cut2, ip_W, ip_boff, best, ipcut, rb_ov,
                                                 take.p); SCLAP_NOTE_LAUNCH("k_select_best");
  int64_t mx = 1;
  for (const auto& t : tasks) mx = std::max(mx, t.n);
  for (int32_t t0 = 0; t0 < nt; t0 += 65535) {
    dim3 grid((unsigned)((mx + SC_CH - 1) / SC_CH), (unsigned)std::min(65535, nt - t0));
    k_copy_best<<<grid, 256, 0, s>>>(d.p + t0, take.p + t0, ip_noff, ip_boff, ip_label, ip_W, Wg); SCLAP_NOTE_LAUNCH("k_copy_best");
  }
  SCLAP_LAUNCH_CHECK();
  stream_sync(s);   // the task array is freed on return
}

void project(const int32_t* cmap, const int32_t* coarse_blk, int32_t* fine_blk, int64_t N,
             cudaStream_t s) {
  if (N <= 0) return;
  k_project<<<grid_for(N, 256, (int64_t)num_sms() * 16), 256, 0, s>>>(cmap, coarse_blk,
                                                                      fine_blk, N); SCLAP_NOTE_LAUNCH("k_project");
  SCLAP_LAUNCH_CHECK();
}

void lift_blocks(const int32_t* cmap, const int32_t* fine_blk, int32_t* coarse_blk, int64_t N,
                 cudaStream_t s) {
  if (N <= 0) return;
  k_lift_blocks<<<grid_for(N, 256, (int64_t)num_sms() * 16), 256, 0, s>>>(cmap, fine_blk,
                                                                          coarse_blk, N); SCLAP_NOTE_LAUNCH("k_lift_blocks");
  SCLAP_LAUNCH_CHECK();
}

void block_weights(const int32_t* label, const int32_t* nw, int64_t N, wgt_t* W,
                   cudaStream_t s) {
  if (N <= 0) return;
  k_block_weights<<<grid_for(N, 256, (int64_t)num_sms() * 16), 256, 0, s>>>(label, nw, N, W); SCLAP_NOTE_LAUNCH("k_block_weights");
  SCLAP_LAUNCH_CHECK();
}

}  // namespace sclap
