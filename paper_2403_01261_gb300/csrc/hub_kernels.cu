// hub_kernels.cu -- the sweep for hub vertices (class 9).
//
// One block per hub would leave the largest rows (a million entries and
// more on R-MAT scale 25) to a single SM at the end of the launch.  Two
// designs share the plan and final kernels:
//   1. hub_plan_kernel (one block): lists the frontier's hubs up to the
//      cluster bound for the cluster kernel (the longest first), numbers the
//      pieces of the others (prefix sums), and places every hub's global
//      table region (2 d slots) and used-slot list (d entries);
//   2a. hub_cluster_kernel (default, every hub): one 8-CTA thread-block
//      cluster per row, the row's label table spread over the CTAs' shared
//      memories and filled with distributed-shared-memory atomics; each CTA
//      then scans its own table for the largest packed key (see the kernel);
//   2b. hub_piece_kernel: a block aggregates one 8192-entry piece in a
//      shared-memory table (a piece has at most HUB_PIECE < 3/4 of the
//      table's slots distinct labels, so it never overflows), then adds each
//      of its (label, sum) pairs to the hub's global table.  Every add
//      returns the label's new total, so the largest packed key
//      (sum << 32 | ~label) over all adds of all pieces is the hub's argmax
//      with smallest-label ties -- the same argument as within one block; it
//      is combined with one atomicMax per piece.  Entries carrying the hub's
//      own label are counted separately and added once per piece;
//   3. hub_final_kernel: per hub, the own-label key is compared with the
//      best key, the label written and counted, the table slots the pieces
//      (or an overflowed cluster) claimed are reset (the tables stay empty
//      between sweeps), and the neighbours of a changed hub are marked.
#include <cooperative_groups.h>

#include "sweep_device.cuh"

namespace cg = cooperative_groups;

namespace gsl {

namespace {

constexpr int HUB_PIECE = 8192;   // entries per piece (distinct labels <= 8192 < 3/4 of 12288 slots)
constexpr unsigned HUB_CLUSTER = 8;   // CTAs per cluster of the cluster kernel (the portable maximum)
constexpr long long HUB_CLU_BIG = 65536;   // cluster rows longer than this are listed first
constexpr int HUB_DSM_PROBES = 128;        // probe bound of the distributed table (overflow past it)

// Global-table insert that records every slot it claims in `used`.
__device__ __forceinline__ unsigned hub_slot_add(unsigned long long* tab, unsigned cap, unsigned lbl, unsigned c,
                                                 unsigned* used, unsigned* used_cnt, long long tab_base, int* err,
                                                 int probe_cap) {
  unsigned h = __umulhi(hash32(lbl), cap);
  const unsigned long long mine = ((unsigned long long)lbl << 32) | c;
  for (int p = 0; p < probe_cap; ++p) {
    unsigned long long x = __ldcg(tab + h);
    if (x == EMPTY64) {
      x = atomicCAS(tab + h, EMPTY64, mine);
      if (x == EMPTY64) {
        used[atomicAdd(used_cnt, 1u)] = (unsigned)(tab_base + h);
        return c;
      }
    }
    if ((unsigned)(x >> 32) == lbl) {
      const unsigned long long old = atomicAdd(tab + h, (unsigned long long)c);
      return (unsigned)old + c;
    }
    if (++h == cap) h = 0;
  }
  raise_err(err, ERRBIT_TIMEOUT);
  return 0;
}

// Insert into the cluster's distributed table (see cluster_row): one
// compare-and-swap per probe claims the slot or finds the label there, and
// the count is added without waiting for the result (the argmax is read
// from the tables once every insert has landed).  Returns false when
// HUB_DSM_PROBES probes found neither: the table is too full.
__device__ __forceinline__ bool dsm_slot_add(cg::cluster_group& cl, SlotTable t, unsigned cap, unsigned lbl,
                                             unsigned c) {
  const unsigned x = hash32(lbl);
  const unsigned owner = __umulhi(x, HUB_CLUSTER);
  unsigned* keys = cl.map_shared_rank(t.keys, owner);
  unsigned* sums = cl.map_shared_rank(t.sums, owner);
  unsigned h = __umulhi(x * (unsigned)HUB_CLUSTER, cap);
  for (int p = 0; p < HUB_DSM_PROBES; ++p) {
    const unsigned k = atomicCAS(keys + h, EMPTY32, lbl);
    if (k == EMPTY32 || k == lbl) {
      atomicAdd(sums + h, c);
      return true;
    }
    if (++h == cap) h = 0;
  }
  return false;
}

__device__ __forceinline__ int piece_hub(const int* piece_start, int cnt, int p) {
  int lo = 0, hi = cnt;   // piece_start[lo] <= p < piece_start[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (piece_start[mid] <= p) lo = mid;
    else hi = mid;
  }
  return lo;
}

}  // namespace

// Hubs of degree <= cmax go to the cluster kernel (listed in hp.clu) and
// get no pieces; every hub keeps its global table region and used list.
__global__ void __launch_bounds__(1024) hub_plan_kernel(SweepArgs a, HubPlan hp, long long cmax) {
  const unsigned cnt = a.ctr->cls_count[CLS_HUB];
  const int* __restrict__ work = a.work + a.ctr->cls_start[CLS_HUB];
  __shared__ long long s_pieces[1024], s_entries[1024];
  __shared__ int s_clu[1024];
  __shared__ long long base_p, base_e;
  __shared__ int base_c;
  if (threadIdx.x == 0) {
    base_p = 0;
    base_e = 0;
    base_c = 0;
  }
  __syncthreads();
  for (unsigned i0 = 0; i0 < cnt; i0 += blockDim.x) {
    const unsigned i = i0 + threadIdx.x;
    long long d = 0;
    if (i < cnt) {
      const int v = work[i];
      d = a.off[v + 1] - a.off[v];
      hp.best[i] = 0;
      hp.own[i] = 0;
      hp.wsum[i] = 0;
      hp.used_cnt[i] = 0;
    }
    s_pieces[threadIdx.x] = d <= cmax ? 0 : (d + HUB_PIECE - 1) / HUB_PIECE;
    s_entries[threadIdx.x] = d;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {   // inclusive scans
      const long long xp = threadIdx.x >= (unsigned)o ? s_pieces[threadIdx.x - o] : 0;
      const long long xe = threadIdx.x >= (unsigned)o ? s_entries[threadIdx.x - o] : 0;
      __syncthreads();
      s_pieces[threadIdx.x] += xp;
      s_entries[threadIdx.x] += xe;
      __syncthreads();
    }
    if (i < cnt) {
      hp.piece_start[i + 1] = (int)(base_p + s_pieces[threadIdx.x]);
      hp.ustart[i + 1] = base_e + s_entries[threadIdx.x];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      base_p += s_pieces[blockDim.x - 1];
      base_e += s_entries[blockDim.x - 1];
    }
    __syncthreads();
  }
  // the cluster list, rows above HUB_CLU_BIG first (they are taken first,
  // which shortens the kernel's tail)
  for (int pass = 0; pass < 2; ++pass) {
    for (unsigned i0 = 0; i0 < cnt; i0 += blockDim.x) {
      const unsigned i = i0 + threadIdx.x;
      bool clu = false;
      if (i < cnt) {
        const int v = work[i];
        const long long d = a.off[v + 1] - a.off[v];
        clu = d <= cmax && (d > HUB_CLU_BIG) == (pass == 0);
      }
      s_clu[threadIdx.x] = clu ? 1 : 0;
      __syncthreads();
      for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const int xc = threadIdx.x >= (unsigned)o ? s_clu[threadIdx.x - o] : 0;
        __syncthreads();
        s_clu[threadIdx.x] += xc;
        __syncthreads();
      }
      if (clu) hp.clu[base_c + s_clu[threadIdx.x] - 1] = (int)i;
      __syncthreads();
      if (threadIdx.x == 0) base_c += s_clu[blockDim.x - 1];
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    hp.piece_start[0] = 0;
    hp.ustart[0] = 0;
    a.ctr->hub_pieces = (unsigned)base_p;
    a.ctr->hub_clusters = (unsigned)base_c;
    a.ctr->hub_clu_next = 0;
  }
}

// One CTA's share of hub row v in the cluster kernel.  Virtual thread tid
// of nthr (all threads of the cluster) takes 32-entry chunks as block_row
// does, so the whole cluster sweeps the row in rounds of nthr * 4 entries.
// DSMEM (GLOBAL false): each distinct label of a warp's chunk is added to
// the cluster's distributed table: the top bits of its hash pick the owning
// CTA, the rest the first slot of a linear probe in that CTA's table (cap
// slots).  A probe that finds no slot in HUB_DSM_PROBES steps raises the
// overflow flag of every CTA in the cluster, and warps stop at their next
// chunk.  The pass publishes own / wsum in sh[par]; the best key is read
// from the tables afterwards.  GLOBAL: the row goes to the hub's global
// table instead (after an overflow), and the best key over the returned
// totals is published too.  Block-uniform end.
template <bool WEIGHTED, bool ASYNC, bool GLOBAL>
__device__ __forceinline__ void cluster_row(const SweepArgs& a, int v, int own, const int* cp, const int* wp,
                                            const int* lp, int d, int tid, int nthr, SlotTable tab, unsigned cap,
                                            unsigned long long* gtab, unsigned gcap, unsigned* gused,
                                            unsigned* gused_cnt, long long gbase, const Pol& pol,
                                            BlockRowShared& sh, int par, cg::cluster_group& cl) {
  const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
  const int step = nw * 128;
  const int cb = wid * 32 + lane;
  const int cu = nw * 32;
  unsigned long long best = 0, wsum = 0;
  unsigned own_sum = 0;
  int jn[4], wn[4], ln[4], lw[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) load_entry<WEIGHTED>(a, cp, wp, d, cb + u * cu, pol, jn[u], wn[u]);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (jn[u] >= 0) wsum += (unsigned long long)wn[u];
    ln[u] = entry_label<ASYNC>(a, lp, cb + u * cu, jn[u], v, pol);
    lw[u] = wn[u];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) load_entry<WEIGHTED>(a, cp, wp, d, step + cb + u * cu, pol, jn[u], wn[u]);
  if (threadIdx.x == 0) {
    sh.best[par] = 0;
    sh.wsum[par] = 0;
    sh.own[par] = 0;
  }
  __syncthreads();
  for (int r0 = 0; r0 < d; r0 += step) {
    int l[4], w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      l[u] = ln[u];
      w[u] = lw[u];
    }
    if (r0 + step < d) {   // cluster-uniform
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (jn[u] >= 0) wsum += (unsigned long long)wn[u];
        ln[u] = entry_label<ASYNC>(a, lp, r0 + step + cb + u * cu, jn[u], v, pol);
        lw[u] = wn[u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) load_entry<WEIGHTED>(a, cp, wp, d, r0 + 2 * step + cb + u * cu, pol, jn[u], wn[u]);
    }
    bool stop = false;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (!stop && r0 + (u * nw + wid) * 32 < d) {   // warp-uniform
        if (!GLOBAL && __shfl_sync(FULL, lane == 0 ? *(volatile int*)&sh.ovf[par] : 0, 0)) {
          stop = true;
        } else {
          const bool mine = l[u] == own;
          own_sum += WEIGHTED ? __reduce_add_sync(FULL, mine ? (unsigned)w[u] : 0u)
                              : (unsigned)__popc(__ballot_sync(FULL, mine));
          if (mine) l[u] = -1;
          if (__ballot_sync(FULL, l[u] >= 0) == 0) continue;
          const unsigned m = label_group(l[u], a.spread);
          const unsigned c = WEIGHTED ? __reduce_add_sync(m, (unsigned)w[u]) : (unsigned)__popc(m);
          const bool leader = l[u] >= 0 && (m & lanemask_lt()) == 0;
          if (GLOBAL) {
            if (leader) {
              const unsigned sum = hub_slot_add(gtab, gcap, (unsigned)l[u], c, gused, gused_cnt, gbase, &a.ctr->err,
                                                         a.probe_cap);
              const unsigned long long k = pack_key(sum, l[u]);
              best = k > best ? k : best;
            }
          } else {
            const bool full = leader && !dsm_slot_add(cl, tab, cap, (unsigned)l[u], c);
            if (__any_sync(FULL, full) && lane == 0) {
              for (unsigned r = 0; r < HUB_CLUSTER; ++r) *(volatile int*)cl.map_shared_rank(&sh.ovf[par], r) = 1;
            }
          }
        }
      }
    }
    if (stop) break;
  }
  block_publish<WEIGHTED>(a, sh, par, best, wsum, own_sum);
  __syncthreads();
}

// The cluster's own-label pass over a hub row (own_weight_pass over the
// cluster's virtual threads).  Each warp adds its round's own-label weight
// to rank 0's counter `cnt` and stops once the returned total is more than
// half of `bound` (the row's d entries, or its weighted degree from sweep
// 1): the own label then holds a strict majority whatever the rest carries.
template <bool WEIGHTED, bool ASYNC>
__device__ __forceinline__ void cluster_own_pass(const SweepArgs& a, int v, int own, const int* cp, const int* wp,
                                                 const int* lp, int d, int tid, int nthr, const Pol& pol,
                                                 unsigned& own_w, unsigned& tot_w, unsigned* cnt,
                                                 unsigned long long bound) {
  const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
  const int step = nw * 128;
  const int cb = wid * 32 + lane, cu = nw * 32;
  int jn[4], wn[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) load_entry<WEIGHTED>(a, cp, wp, d, cb + u * cu, pol, jn[u], wn[u]);
  for (int r0 = 0; r0 < d; r0 += step) {
    int l[4], w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      l[u] = entry_label<ASYNC>(a, lp, r0 + cb + u * cu, jn[u], v, pol);
      w[u] = wn[u];
    }
    const bool more = r0 + step < d;   // cluster-uniform
    if (more) {
#pragma unroll
      for (int u = 0; u < 4; ++u) load_entry<WEIGHTED>(a, cp, wp, d, r0 + step + cb + u * cu, pol, jn[u], wn[u]);
    }
    unsigned o = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (l[u] >= 0) {
        tot_w += (unsigned)w[u];
        if (l[u] == own) {
          own_w += (unsigned)w[u];
          o += (unsigned)w[u];
        }
      }
    }
    if (more && bound != ~0ull) {
      o = __reduce_add_sync(FULL, o);
      unsigned total = 0;
      if (lane == 0 && o) total = atomicAdd(cnt, o) + o;
      if (2ull * __shfl_sync(FULL, total, 0) > bound) return;
    }
  }
}

// Hubs of degree <= cmax (listed by the plan kernel), one thread-block
// cluster at a time: rank 0 takes the next hub from a counter, the row is
// aggregated in the CTAs' shared tables (cluster_row), each CTA scans its
// own table for the largest packed key (every label sits in one slot of one
// table, with its final total) and adds that key, its own-label count and
// weight to hp.best / hp.own / hp.wsum, which hub_final_kernel reads as it
// reads the pieces'.  After an overflow
// (flags read from all CTAs after the second barrier, so the decision is
// the same in every CTA) the CTAs redo the row in the hub's global table.
// Two cluster barriers per hub: A after the tables are cleared (no insert
// can reach a table before it is empty), B after every insert (all flags
// final).  Per-hub shared values alternate between two copies (par), so a
// CTA clears one copy while others may still read the previous hub's.
// With `maj` (sweeps whose rows mostly keep their label) the cluster first
// weighs the row's own label (own_weight_pass, barrier C, totals read from
// all CTAs): a strict majority is Eq. 2's argmax, the label stays and the
// table pass is skipped.
// Every branch around a barrier depends only on values all CTAs of the
// cluster read alike (the hub index from rank 0, the OR of the flags, the
// majority totals).
template <bool WEIGHTED, bool ASYNC>
__global__ void __launch_bounds__(512, 2) hub_cluster_kernel(SweepArgs a, HubPlan hp, unsigned tb, int maj) {
  extern __shared__ unsigned long long smem_c64[];
  __shared__ BlockRowShared sh;
  __shared__ int s_hub[2], s_ovf[2];
  __shared__ unsigned long long s_mown[2], s_mtot[2];
  __shared__ unsigned s_mcnt[2];   // rank 0's: own-label entries counted so far (unit weights)
  __shared__ int s_skip[2];
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank();
  const int nclu = (int)a.ctr->hub_clusters;
  const int* __restrict__ work = a.work + a.ctr->cls_start[CLS_HUB];
  const Pol pol = make_pol();
  const SlotTable st = make_table(smem_c64, tb);
  const int tid = (int)(rank * blockDim.x + threadIdx.x), nthr = HUB_CLUSTER * (int)blockDim.x;
  for (int par = 0;; par ^= 1) {
    for (unsigned k = threadIdx.x; k < tb; k += blockDim.x) {
      st.keys[k] = EMPTY32;
      st.sums[k] = 0;
    }
    if (threadIdx.x == 0) {
      sh.ovf[par] = 0;
      s_mown[par] = 0;
      s_mtot[par] = 0;
      s_mcnt[par] = 0;
      if (rank == 0) s_hub[par] = (int)atomicAdd(&a.ctr->hub_clu_next, 1u);
    }
    cl.sync();   // A
    const int q = *(volatile int*)cl.map_shared_rank(&s_hub[par], 0);
    if (q >= nclu) break;
    const int i = hp.clu[q];
    const int v = work[i];
    const long long s = a.off[v];
    const int d = (int)(a.off[v + 1] - s);
    const int own = own_label<ASYNC>(a, v);
    const int* cp = a.col + s;
    const int* wp = a.w + s;
    const int* lp = a.lg ? a.lg + s : nullptr;
    if (maj) {
      unsigned own_w = 0, tot_w = 0;
      const unsigned long long bound =
          !WEIGHTED ? (unsigned long long)d : (a.kw ? (unsigned long long)a.kw[v] : ~0ull);
      cluster_own_pass<WEIGHTED, ASYNC>(a, v, own, cp, wp, lp, d, tid, nthr, pol, own_w, tot_w,
                                        cl.map_shared_rank(&s_mcnt[par], 0), bound);
      const unsigned long long ow = warp_sum_u64(own_w), tw = warp_sum_u64(tot_w);
      if ((threadIdx.x & 31) == 0) {
        if (ow) atomicAdd(&s_mown[par], ow);
        if (tw) atomicAdd(&s_mtot[par], tw);
      }
      cl.sync();   // C
      if (threadIdx.x < 32) {
        unsigned long long o = 0, t = 0;
        if (threadIdx.x < HUB_CLUSTER) {
          o = *(volatile unsigned long long*)cl.map_shared_rank(&s_mown[par], threadIdx.x);
          t = *(volatile unsigned long long*)cl.map_shared_rank(&s_mtot[par], threadIdx.x);
        }
        o = warp_sum_u64(o);
        t = warp_sum_u64(t);
        // a strict majority of the row, or (the pass stopped early) more
        // than half of its total
        if (threadIdx.x == 0) s_skip[par] = 2 * o > t || 2 * o > bound;
      }
      __syncthreads();
      if (s_skip[par]) continue;   // the label stays (hp.best 0, hp.own 0)
    }
    cluster_row<WEIGHTED, ASYNC, false>(a, v, own, cp, wp, lp, d, tid, nthr, st, tb, nullptr, 0, nullptr, nullptr, 0,
                                        pol, sh, par, cl);
    cl.sync();   // B
    if (threadIdx.x < 32) {
      const int f = threadIdx.x < HUB_CLUSTER ? *(volatile int*)cl.map_shared_rank(&sh.ovf[par], threadIdx.x) : 0;
      const int any = __any_sync(FULL, f);
      if (threadIdx.x == 0) s_ovf[par] = any;
    }
    __syncthreads();
    if (!s_ovf[par]) {
      unsigned long long b = 0;
      for (unsigned k = threadIdx.x; k < tb; k += blockDim.x) {
        const unsigned key = st.keys[k];
        if (key != EMPTY32) {
          const unsigned long long x = pack_key(st.sums[k], (int)key);
          b = x > b ? x : b;
        }
      }
      b = warp_max_u64(b);
      if ((threadIdx.x & 31) == 0 && b) atomicMax(&sh.best[par], b);
      __syncthreads();
    } else {
      cluster_row<WEIGHTED, ASYNC, true>(a, v, own, cp, wp, lp, d, tid, nthr, st, tb, hp.tab + 2 * hp.ustart[i],
                                         (unsigned)(2 * d), hp.used + hp.ustart[i], hp.used_cnt + i,
                                         2 * hp.ustart[i], pol, sh, par, cl);
    }
    if (threadIdx.x == 0) {
      if (sh.best[par]) atomicMax(hp.best + i, sh.best[par]);
      if (sh.own[par]) atomicAdd(hp.own + i, sh.own[par]);
      if (WEIGHTED && a.check && sh.wsum[par]) atomicAdd(hp.wsum + i, sh.wsum[par]);
    }
  }
  cl.sync();   // rank 0's s_hub stays readable until every CTA has read it
}

template <bool WEIGHTED, bool ASYNC>
__global__ void __launch_bounds__(512, 2) hub_piece_kernel(SweepArgs a, HubPlan hp, unsigned tb) {
  extern __shared__ unsigned long long smem_h64[];
  __shared__ BlockRowShared sh;
  const unsigned cnt = a.ctr->cls_count[CLS_HUB];
  const unsigned pieces = a.ctr->hub_pieces;
  const int* __restrict__ work = a.work + a.ctr->cls_start[CLS_HUB];
  const Pol pol = make_pol();
  int par = 0;
  for (unsigned p = blockIdx.x; p < pieces; p += gridDim.x, par ^= 1) {
    const int i = piece_hub(hp.piece_start, (int)cnt, (int)p);
    const int v = work[i];
    const long long s = a.off[v];
    const long long d = a.off[v + 1] - s;
    const long long e0 = (long long)(p - (unsigned)hp.piece_start[i]) * HUB_PIECE;
    const int len = (int)(d - e0 < HUB_PIECE ? d - e0 : HUB_PIECE);
    const int own = own_label<ASYNC>(a, v);
    const int* cp = a.col + s + e0;
    const int* wp = a.w + s + e0;
    const int* lp = a.lg ? a.lg + s + e0 : nullptr;
    const unsigned want = 2u * (unsigned)len;
    const unsigned cap = want < tb ? want : tb;
    const SlotTable st = make_table(smem_h64, tb);
    block_row<WEIGHTED, ASYNC, false>(a, v, own, cp, wp, lp, len, st, cap, 0xFFFFFFFFu, pol, sh, par);
    // the piece's (label, sum) pairs into the hub's global table
    unsigned long long* tab = hp.tab + 2 * hp.ustart[i];
    const unsigned gcap = (unsigned)(2 * d);
    unsigned long long best = 0;
    for (unsigned k = threadIdx.x; k < cap; k += blockDim.x) {
      const unsigned lbl = st.keys[k];
      if (lbl == EMPTY32) continue;
      const unsigned sum = hub_slot_add(tab, gcap, lbl, st.sums[k], hp.used + hp.ustart[i], hp.used_cnt + i,
                                        2 * hp.ustart[i], &a.ctr->err, a.probe_cap);
      const unsigned long long key = pack_key(sum, (int)lbl);
      best = key > best ? key : best;
    }
    best = warp_max_u64(best);
    if ((threadIdx.x & 31) == 0 && best) atomicMax(hp.best + i, best);
    if (threadIdx.x == 0) {
      if (sh.own[par]) atomicAdd(hp.own + i, sh.own[par]);
      if (WEIGHTED && a.check && sh.wsum[par]) atomicAdd(hp.wsum + i, sh.wsum[par]);
    }
    __syncthreads();   // the table is cleared for the next piece
  }
}

template <bool ASYNC>
__global__ void __launch_bounds__(256) hub_final_kernel(SweepArgs a, HubPlan hp, int weighted) {
  const unsigned cnt = a.ctr->cls_count[CLS_HUB];
  const int* __restrict__ work = a.work + a.ctr->cls_start[CLS_HUB];
  const Pol pol = make_pol();
  unsigned long long my_dn = 0, my_scan = 0;
  for (unsigned i = blockIdx.x; i < cnt; i += gridDim.x) {
    const int v = work[i];
    const long long s = a.off[v];
    const int d = (int)(a.off[v + 1] - s);
    const int old = own_label<ASYNC>(a, v);
    unsigned long long b = hp.best[i];
    const unsigned own_sum = hp.own[i];
    if (own_sum) {
      const unsigned long long k = pack_key(own_sum, old);
      b = k > b ? k : b;
    }
    const int nl = b ? (int)~(unsigned)b : old;
    const bool changed = nl != old;
    if (threadIdx.x == 0) {
      if (weighted && a.check && hp.wsum[i] >= (1ull << 31)) raise_err(&a.ctr->err, ERRBIT_OVERFLOW);
      if (weighted && a.check && a.kw) a.kw[v] = hp.wsum[i] < (1ull << 32) ? (unsigned)hp.wsum[i] : ~0u;
      store_label<ASYNC>(a, v, nl, changed);
      if (changed) count_graph_change(a, v);
      my_scan += (unsigned long long)d;
      my_dn += changed ? 1ull : 0ull;
    }
    // reset the slots this hub's pieces claimed
    const unsigned used = hp.used_cnt[i];
    const unsigned* ul = hp.used + hp.ustart[i];
    for (unsigned k = threadIdx.x; k < used; k += blockDim.x) hp.tab[ul[k]] = EMPTY64;
    if (changed && a.mark) {
      const int* cp = a.col + s;
      for (int x = threadIdx.x; x < d; x += blockDim.x) {
        const int j = ld_stream(cp + x, pol.stream);
        if ((unsigned)j < (unsigned)a.n) a.fnext[j] = 1;
      }
      if (!ASYNC && threadIdx.x == 0) a.fnext[v] = 1;
    }
  }
  flush_counters(a.ctr, CLS_HUB, my_dn, my_scan);
}

namespace {
// Clusters of the cluster kernel resident at once for the given table size
// (0: such clusters cannot run); cached per size.
template <bool W, bool A>
int cluster_slots(size_t smem) {
  thread_local size_t cached_smem = 0;   // per host thread (see block_grid_size)
  thread_local int cached = 0;
  if (cached_smem == smem) return cached;
  cached_smem = smem;
  cached = 0;
  if (raise_smem_limit((const void*)hub_cluster_kernel<W, A>, smem) != cudaSuccess ||
      (HUB_CLUSTER > 8 &&
       cudaFuncSetAttribute(hub_cluster_kernel<W, A>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
           cudaSuccess)) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = HUB_CLUSTER;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(HUB_CLUSTER, 1, 1);
  cfg.blockDim = dim3(512, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, hub_cluster_kernel<W, A>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  cached = n;
  return cached;
}

template <bool W, bool A>
cudaError_t launch_hub_t(const SweepArgs& a, const HubPlan& hp, bool maj, const Tuning& t, const DeviceInfo& di,
                         cudaStream_t s, int* kernels) {
  const size_t smem = (size_t)t.blk_slots * sizeof(unsigned long long);
  raise_smem_limit((const void*)hub_piece_kernel<W, A>, smem);
  const int nclusters = t.hub_cluster_max > 0 ? cluster_slots<W, A>(smem) : 0;
  hub_plan_kernel<<<1, 1024, 0, s>>>(a, hp, nclusters > 0 ? (long long)t.hub_cluster_max : 0ll);
  int launches = 3;
  if (nclusters > 0) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = HUB_CLUSTER;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(HUB_CLUSTER * (unsigned)nclusters, 1, 1);
    cfg.blockDim = dim3(512, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, hub_cluster_kernel<W, A>, a, hp, (unsigned)t.blk_slots, maj ? 1 : 0);
    if (e != cudaSuccess) return e;
    ++launches;
  }
  hub_piece_kernel<W, A><<<(int)block_grid_size(t, di), t.blk_block, smem, s>>>(a, hp, (unsigned)t.blk_slots);
  hub_final_kernel<A><<<2 * di.sm_count, 256, 0, s>>>(a, hp, W ? 1 : 0);
  count_launches(launches);
  *kernels = launches;
  return cudaGetLastError();
}
}  // namespace

bool hub_pieces_fit(const Tuning& t) { return HUB_PIECE * 4 <= t.blk_slots * 3 - 4 * 512; }

cudaError_t launch_hub_pieces(const SweepArgs& a, const HubPlan& hp, bool weighted, bool async_mode, bool majority,
                              const Tuning& t, const DeviceInfo& di, cudaStream_t s, int* kernels) {
  if (weighted)
    return async_mode ? launch_hub_t<true, true>(a, hp, majority, t, di, s, kernels)
                      : launch_hub_t<true, false>(a, hp, majority, t, di, s, kernels);
  return async_mode ? launch_hub_t<false, true>(a, hp, majority, t, di, s, kernels)
                    : launch_hub_t<false, false>(a, hp, majority, t, di, s, kernels);
}

}  // namespace gsl
