// contract.cu -- cluster contraction (Sec. 3.1) for every slot of a level.
//
// Each cluster becomes one coarse node (id = rank of its label, contiguous
// per slot); its weight is the sum of its members; two coarse nodes are
// adjacent iff their clusters are, with the summed weight of the fine edges
// between them.  GPU plan: rank labels by a scan, group the members of every
// coarse node (counting sort), then give each coarse node a warp or a CTA
// that streams its members' arcs (flattened across members so lanes stay
// busy), maps each neighbour to its coarse id and sums weights per coarse
// neighbour in an open-addressing table (shared memory; global scratch for
// hub clusters).  Rows come out in table order, which no later step depends
// on.
#include "common.cuh"

namespace sclap {
namespace {

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
  int32_t* ccnt;
  int64_t* carcs;
  const int64_t* moff;
  int32_t* mfill;
  int32_t* members;
  const int64_t* toff;
  int32_t* tcol;
  int32_t* tw;
  int32_t* cdeg;
  int32_t* bcnt;
  int32_t* bfill;
  int64_t* boff;
  int32_t* blist;
  int64_t* maxarcs;
  int32_t* err;
};

constexpr int CB_WARP_MAX = 512;    // member arcs handled by one warp (1024-slot table)
constexpr int CB_CTA_MAX = 4096;    // by one CTA with a shared table (8192 slots)

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

__global__ void k_map(CArgs a, int64_t N) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = a.gid[v];
    if (!a.keep[s]) { a.cmap[v] = -1; continue; }
    const int32_t c = (int32_t)(a.cid[a.label[v]] + a.delta[s]);
    a.cmap[v] = c;
    atomicAdd(&a.cnw[c], a.nw[v]);
    atomicAdd(&a.ccnt[c], 1);
    atomicAdd(ull(&a.carcs[c]), (unsigned long long)(a.row_ptr[v + 1] - a.row_ptr[v]));
  }
}

__global__ void k_members(CArgs a, int64_t N) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = a.cmap[v];
    if (c < 0) continue;
    a.members[a.moff[c] + atomicAdd(&a.mfill[c], 1)] = (int32_t)v;
  }
}

__device__ __forceinline__ int cbucket(int64_t arcs) {
  return arcs <= CB_WARP_MAX ? 0 : (arcs <= CB_CTA_MAX ? 1 : 2);
}

template <int PASS>
__global__ void __launch_bounds__(256) k_cbucket(CArgs a, int64_t Nc) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = w0 * 32; base < Nc; base += nw * 32) {
    const int64_t c = base + lane;
    int key = -1;
    int64_t arcs = 0;
    if (c < Nc) {
      arcs = a.carcs[c];
      key = cbucket(arcs);
    }
    const unsigned mm = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(mm) - 1;
    if (PASS == 0) {
      if (key >= 0 && lane == leader) atomicAdd(&a.bcnt[key], __popc(mm));
      long long m = warp_max_ll(arcs);
      if (lane == 0 && m > 0) atomicMax(ull(a.maxarcs), (unsigned long long)m);
    } else {
      int bp = 0;
      if (key >= 0 && lane == leader) bp = atomicAdd(&a.bfill[key], __popc(mm));
      bp = __shfl_sync(0xffffffffu, bp, leader);
      if (key >= 0) a.blist[a.boff[key] + bp + __popc(mm & ((1u << lane) - 1))] = (int32_t)c;
    }
  }
}

__device__ __forceinline__ void ctable_add(int32_t* keys, unsigned long long* vals, int logcap,
                                           int32_t K, int64_t w, int32_t* err) {
  const uint32_t mask = (1u << logcap) - 1;
  uint32_t s = table_slot(K, logcap);
  for (uint32_t p = 0; p <= mask; ++p) {
    const int32_t k = atomicCAS(&keys[s], -1, K);
    if (k == -1 || k == K) {
      atomicAdd(&vals[s], (unsigned long long)w);
      return;
    }
    s = (s + 1) & mask;
  }
  atomicOr(err, DERR_HASH_FULL);
}

// The arcs of coarse node c's members, flattened: each warp takes 32 members
// at a time, scans their degrees, and its lanes walk the concatenated arc
// range; lane x finds its member by binary lifting over the scanned degrees.
__device__ void accumulate_members(const CArgs& a, int32_t c, int wrank, int nwarps,
                                   int32_t* keys, unsigned long long* vals, int logcap) {
  const int lane = threadIdx.x & 31;
  const int64_t mb = a.moff[c], me = a.moff[c + 1];
  for (int64_t j0 = mb + (int64_t)wrank * 32; j0 < me; j0 += (int64_t)nwarps * 32) {
    const int64_t j = j0 + lane;
    int64_t rs = 0, d = 0;
    if (j < me) {
      const int32_t m = a.members[j];
      rs = a.row_ptr[m];
      d = a.row_ptr[m + 1] - rs;
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
        long long v = __shfl_sync(0xffffffffu, incl, L + step - 1);
        if (v <= x) L += step;
      }
      const long long rsL = __shfl_sync(0xffffffffu, (long long)rs, L);
      const long long exL = __shfl_sync(0xffffffffu, excl, L);
      int32_t cu = -1, w = 0;
      if (x < total) {
        const int64_t e = rsL + (x - exL);
        cu = a.cmap[a.col[e]];
        w = a.ew[e];
        if (cu == c) { cu = -1; w = 0; }
      }
      const unsigned mm = __match_any_sync(0xffffffffu, cu);
      const int64_t sum = match_sum(mm, w);
      if (cu >= 0 && lane == __ffs(mm) - 1) ctable_add(keys, vals, logcap, cu, sum, a.err);
    }
  }
}

// One warp per coarse node with <= 512 member arcs.
__global__ void __launch_bounds__(256) k_caccum_warp(CArgs a, int64_t lbeg, int64_t cnt) {
  extern __shared__ unsigned long long smem_u64[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  unsigned long long* vals = smem_u64 + wib * WARP_HASH_SLOTS;
  int32_t* keys = reinterpret_cast<int32_t*>(smem_u64 + 8 * WARP_HASH_SLOTS) + wib * WARP_HASH_SLOTS;
  for (int j = lane; j < WARP_HASH_SLOTS; j += 32) { keys[j] = -1; vals[j] = 0; }
  __syncwarp();
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t li = warp; li < cnt; li += nwarps) {
    const int32_t c = a.blist[lbeg + li];
    const int logcap = ceil_log2(max64(2 * a.carcs[c], 32));
    const int cap = 1 << logcap;
    accumulate_members(a, c, 0, 1, keys, vals, logcap);
    __syncwarp();
    const int64_t base = a.toff[c];
    int n = 0;
    for (int j0 = 0; j0 < cap; j0 += 32) {
      const int j = j0 + lane;
      const int32_t K = keys[j];
      const bool occ = K != -1;
      const unsigned bal = __ballot_sync(0xffffffffu, occ);
      if (occ) {
        const unsigned long long val = vals[j];
        if (val > (unsigned long long)INT32_MAX) atomicOr(a.err, DERR_W_OVERFLOW);
        const int pos = n + __popc(bal & ((1u << lane) - 1));
        a.tcol[base + pos] = K;
        a.tw[base + pos] = (int32_t)min(val, (unsigned long long)INT32_MAX);
        keys[j] = -1;
        vals[j] = 0;
      }
      n += __popc(bal);
    }
    if (lane == 0) a.cdeg[c] = n;
    __syncwarp();
  }
}

// One CTA per larger coarse node; table in shared memory or global scratch.
template <bool GLOBAL>
__global__ void __launch_bounds__(512) k_caccum_cta(CArgs a, int64_t lbeg, int64_t cnt,
                                                    int32_t* gkeys, unsigned long long* gvals,
                                                    int64_t gcap) {
  constexpr int NT = 512;
  extern __shared__ unsigned long long smem_u64[];
  __shared__ int sh_n;
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  unsigned long long* vals;
  int32_t* keys;
  if (GLOBAL) {
    vals = gvals + (int64_t)blockIdx.x * gcap;
    keys = gkeys + (int64_t)blockIdx.x * gcap;
  } else {
    vals = smem_u64;
    keys = reinterpret_cast<int32_t*>(smem_u64 + CTA_HASH_SLOTS);
    for (int j = tid; j < CTA_HASH_SLOTS; j += NT) { keys[j] = -1; vals[j] = 0; }
  }
  __syncthreads();
  for (int64_t li = blockIdx.x; li < cnt; li += gridDim.x) {
    const int32_t c = a.blist[lbeg + li];
    const int logcap = ceil_log2(max64(2 * a.carcs[c], 32));
    const int64_t cap = (int64_t)1 << logcap;
    if (tid == 0) sh_n = 0;
    accumulate_members(a, c, wib, NT / 32, keys, vals, logcap);
    __syncthreads();
    const int64_t base = a.toff[c];
    for (int64_t j0 = 0; j0 < cap; j0 += NT) {
      const int64_t j = j0 + tid;
      const int32_t K = j < cap ? keys[j] : -1;
      const bool occ = K != -1;
      const unsigned bal = __ballot_sync(0xffffffffu, occ);
      int wbase = 0;
      if (lane == 0 && bal) wbase = atomicAdd(&sh_n, __popc(bal));
      wbase = __shfl_sync(0xffffffffu, wbase, 0);
      if (occ) {
        const unsigned long long val = vals[j];
        if (val > (unsigned long long)INT32_MAX) atomicOr(a.err, DERR_W_OVERFLOW);
        const int pos = wbase + __popc(bal & ((1u << lane) - 1));
        a.tcol[base + pos] = K;
        a.tw[base + pos] = (int32_t)min(val, (unsigned long long)INT32_MAX);
        keys[j] = -1;
        vals[j] = 0;
      }
    }
    __syncthreads();
    if (tid == 0) a.cdeg[c] = sh_n;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_compact(const int64_t* __restrict__ toff,
                                                 const int32_t* __restrict__ cdeg,
                                                 const int64_t* __restrict__ crow,
                                                 const int32_t* __restrict__ tcol,
                                                 const int32_t* __restrict__ tw, int64_t Nc,
                                                 int32_t* __restrict__ ccol,
                                                 int32_t* __restrict__ cew) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < Nc; c += nwarps) {
    const int64_t src = toff[c], dst = crow[c];
    const int n = cdeg[c];
    for (int j = lane; j < n; j += 32) {
      ccol[dst + j] = tcol[src + j];
      cew[dst + j] = tw[src + j];
    }
  }
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
  if (N > 0) { k_mark<<<grid_for(N, 256, (int64_t)sms * 16), 256, 0, s>>>(label, N, w.flag.p); SCLAP_NOTE_LAUNCH(); }
  scan_excl_i32_to_i64(w.flag.p, w.cid.p, N, s);
  DevBuf<int64_t> idx(ns + 1, s), got(ns + 1, s);
  idx.upload(noff);
  k_gather<<<grid_for(ns + 1, 128, 64), 128, 0, s>>>(w.cid.p, idx.p, ns + 1, got.p); SCLAP_NOTE_LAUNCH();
  SCLAP_LAUNCH_CHECK();
  w.cid_at.assign(ns + 1, 0);
  SCLAP_CUDA(cudaMemcpyAsync(w.cid_at.data(), got.p, (ns + 1) * sizeof(int64_t),
                             cudaMemcpyDeviceToHost, s));
  SCLAP_CUDA(cudaStreamSynchronize(s));
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
  out.nw.alloc(Nc, s);
  out.nw.zero();
  DevBuf<int32_t> ccnt(Nc, s), mfill(Nc, s), cdeg(Nc, s);
  DevBuf<int64_t> carcs(Nc, s), moff(Nc + 1, s), toff(Nc + 1, s);
  ccnt.zero(); mfill.zero(); carcs.zero();

  CArgs a{};
  a.row_ptr = lv.row_ptr; a.col = lv.col; a.ew = lv.ew; a.nw = lv.nw; a.gid = lv.gid;
  a.label = label; a.cid = w.cid.p; a.delta = d_delta.p; a.keep = d_keep.p; a.cmap = cmap;
  a.cnw = out.nw.p; a.ccnt = ccnt.p; a.carcs = carcs.p; a.moff = moff.p; a.mfill = mfill.p;
  a.toff = toff.p; a.cdeg = cdeg.p; a.err = d_err;

  const unsigned ng = grid_for(N, 256, (int64_t)sms * 16);
  if (N > 0) { k_map<<<ng, 256, 0, s>>>(a, N); SCLAP_NOTE_LAUNCH(); }
  scan_excl_i32_to_i64(ccnt.p, moff.p, Nc, s);
  scan_excl_i64(carcs.p, toff.p, Nc, s);
  DevBuf<int32_t> members(std::max<int64_t>(N, 1), s);
  a.members = members.p;
  if (N > 0) { k_members<<<ng, 256, 0, s>>>(a, N); SCLAP_NOTE_LAUNCH(); }

  DevBuf<int32_t> bcnt(3, s), bfill(3, s), blist(std::max<int64_t>(Nc, 1), s);
  DevBuf<int64_t> boff(4, s), maxarcs(1, s);
  bcnt.zero(); bfill.zero(); maxarcs.zero();
  a.bcnt = bcnt.p; a.bfill = bfill.p; a.boff = boff.p; a.blist = blist.p; a.maxarcs = maxarcs.p;
  const unsigned cg = grid_for(Nc, 256, (int64_t)sms * 16);
  if (Nc > 0) { k_cbucket<0><<<cg, 256, 0, s>>>(a, Nc); SCLAP_NOTE_LAUNCH(); }
  std::vector<int32_t> hc(3);
  int64_t hmax = 0, tot = 0;
  SCLAP_CUDA(cudaMemcpyAsync(hc.data(), bcnt.p, 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SCLAP_CUDA(cudaMemcpyAsync(&hmax, maxarcs.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SCLAP_CUDA(cudaMemcpyAsync(&tot, toff.p + Nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SCLAP_CUDA(cudaStreamSynchronize(s));
  std::vector<int64_t> hb = {0, hc[0], (int64_t)hc[0] + hc[1], (int64_t)hc[0] + hc[1] + hc[2]};
  boff.upload(hb);
  if (Nc > 0) { k_cbucket<1><<<cg, 256, 0, s>>>(a, Nc); SCLAP_NOTE_LAUNCH(); }

  DevBuf<int32_t> tcol(std::max<int64_t>(tot, 1), s), tw(std::max<int64_t>(tot, 1), s);
  a.tcol = tcol.p; a.tw = tw.p;
  const size_t warp_smem = 8 * WARP_HASH_SLOTS * (sizeof(unsigned long long) + sizeof(int32_t));
  const size_t cta_smem = CTA_HASH_SLOTS * (sizeof(unsigned long long) + sizeof(int32_t));
  static bool attrs = false;
  if (!attrs) {
    SCLAP_CUDA(cudaFuncSetAttribute(k_caccum_warp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)warp_smem));
    SCLAP_CUDA(cudaFuncSetAttribute(k_caccum_cta<false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cta_smem));
    attrs = true;
  }
  if (hc[0] > 0) {
    k_caccum_warp<<<grid_for(hc[0], 8, (int64_t)sms * 2), 256, warp_smem, s>>>(a, hb[0], hc[0]); SCLAP_NOTE_LAUNCH();
  }
  if (hc[1] > 0) {
    k_caccum_cta<false><<<grid_for(hc[1], 1, (int64_t)sms * 2), 512, cta_smem, s>>>(
        a, hb[1], hc[1], nullptr, nullptr, 0); SCLAP_NOTE_LAUNCH();
  }
  DevBuf<int32_t> gkeys;
  DevBuf<unsigned long long> gvals;
  if (hc[2] > 0) {
    const int64_t gcap = (int64_t)1 << ceil_log2(std::max<int64_t>(2 * hmax, 32));
    const int gb = (int)std::min<int64_t>(hc[2], sms);
    gkeys.alloc((size_t)gb * gcap, s);
    gvals.alloc((size_t)gb * gcap, s);
    gkeys.fill_bytes(0xff);
    gvals.zero();
    k_caccum_cta<true><<<gb, 512, 0, s>>>(a, hb[2], hc[2], gkeys.p, gvals.p, gcap); SCLAP_NOTE_LAUNCH();
  }
  SCLAP_LAUNCH_CHECK();

  out.row_ptr.alloc(Nc + 1, s);
  scan_excl_i32_to_i64(cdeg.p, out.row_ptr.p, Nc, s);
  int64_t Mc = 0;
  SCLAP_CUDA(cudaMemcpyAsync(&Mc, out.row_ptr.p + Nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SCLAP_CUDA(cudaStreamSynchronize(s));
  out.M = Mc;
  out.col.alloc(std::max<int64_t>(Mc, 1), s);
  out.ew.alloc(std::max<int64_t>(Mc, 1), s);
  if (Nc > 0) {
    k_compact<<<grid_for(Nc, 8, (int64_t)sms * 16), 256, 0, s>>>(toff.p, cdeg.p, out.row_ptr.p,
                                                                 tcol.p, tw.p, Nc, out.col.p,
                                                                 out.ew.p); SCLAP_NOTE_LAUNCH();
  }
  out.gid.alloc(std::max<int64_t>(Nc, 1), s);
  fill_gid(out.noff_d.p, ns, out.gid.p, Nc, s);
  DevBuf<int64_t> ga(ns + 1, s);
  k_gather<<<grid_for(ns + 1, 128, 64), 128, 0, s>>>(out.row_ptr.p, out.noff_d.p, ns + 1, ga.p); SCLAP_NOTE_LAUNCH();
  SCLAP_LAUNCH_CHECK();
  out.aoff.assign(ns + 1, 0);
  SCLAP_CUDA(cudaMemcpyAsync(out.aoff.data(), ga.p, (ns + 1) * sizeof(int64_t),
                             cudaMemcpyDeviceToHost, s));
  SCLAP_CUDA(cudaStreamSynchronize(s));
}

}  // namespace sclap
