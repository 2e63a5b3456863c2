// sweep_device.cuh -- device helpers shared by the sweep kernels (the
// degree-class kernels and the hub-piece kernels): entry loads, label
// reads and writes, the packed argmax key and the shared/global hash-table
// insert.  Included by one translation unit each; everything is inline.
#pragma once

#include "kernels.h"

namespace gsl {
namespace {

constexpr unsigned long long EMPTY64 = ~0ull;

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ unsigned long long pack_key(unsigned sum, int lbl) {
  return ((unsigned long long)sum << 32) | (unsigned long long)(~(unsigned)lbl);
}

// Adds the per-thread sweep statistics of the whole block to the counters.
__device__ __forceinline__ void flush_counters(Counters* ctr, int cls, unsigned long long dn,
                                               unsigned long long scanned) {
  __shared__ unsigned long long acc[2];
  if (threadIdx.x == 0) { acc[0] = 0; acc[1] = 0; }
  __syncthreads();
  dn = warp_sum_u64(dn);
  scanned = warp_sum_u64(scanned);
  if ((threadIdx.x & 31) == 0) {
    if (dn) atomicAdd(&acc[0], dn);
    if (scanned) atomicAdd(&acc[1], scanned);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (acc[0]) atomicAdd(&ctr->dn, acc[0]);
    if (acc[1]) {
      atomicAdd(&ctr->scanned, acc[1]);
      atomicAdd(&ctr->cls_scanned[cls], acc[1]);
    }
  }
}

// Cache policies, created once per thread: columns and weights are streamed
// (evict first), labels are gathered repeatedly (evict last).
struct Pol {
  unsigned long long stream, label;
};
__device__ __forceinline__ Pol make_pol() { return {policy_evict_first(), policy_evict_last()}; }

// Entry e of the row starting at cp / wp: neighbour j (-1 past the row end
// or when out of range) and its weight.
template <bool WEIGHTED>
__device__ __forceinline__ void load_entry(const SweepArgs& a, const int* cp, const int* wp, int d, int e,
                                           const Pol& pol, int& j, int& wt) {
  j = -1;
  wt = 0;
  if (e < d) {
    j = ld_stream(cp + e, pol.stream);
    wt = WEIGHTED ? ld_stream(wp + e, pol.stream) : 1;
    if ((unsigned)j >= (unsigned)a.n || (WEIGHTED && a.check && wt <= 0)) {
      raise_err(&a.ctr->err, ERRBIT_INVALID);
      j = -1;
    }
  }
}

// Batched mode, first sweep: every column of a row must lie in the row's
// own graph (a packed batch has no edges between graphs).
__device__ __forceinline__ void check_same_graph(const SweepArgs& a, int v, int j) {
  if (a.gid && a.check && j >= 0 && __ldg(a.gid + j) != __ldg(a.gid + v)) raise_err(&a.ctr->err, ERRBIT_INVALID);
}

// Batched mode: per-graph change count.
__device__ __forceinline__ void count_graph_change(const SweepArgs& a, int v) {
  if (a.dn_graph) atomicAdd(a.dn_graph + a.gid[v], 1u);
}

__device__ __forceinline__ bool stopped(const SweepArgs& a) { return a.stop && *(volatile const int*)a.stop; }

template <bool ASYNC>
__device__ __forceinline__ int gather_label(const SweepArgs& a, int j, const Pol& pol) {
  if (a.ident) return j;
  return ASYNC ? ld_label_rw(a.prev + j) : ld_label_ro(a.prev + j, pol.label);
}

// Label of entry e of a row whose neighbour is j: -1 for no neighbour (past
// the row end, out of range) and for the vertex itself (Eq. 2 skips j = i).
// With pre-gathered labels (lp = the row's part of a.lg) the label is a
// coalesced read of lp[e] instead of a gather.
template <bool ASYNC>
__device__ __forceinline__ int entry_label(const SweepArgs& a, const int* lp, int e, int j, int v, const Pol& pol) {
  if (j < 0 || j == v) return -1;
  if (!ASYNC && lp) return ld_stream(lp + e, pol.stream);
  return gather_label<ASYNC>(a, j, pol);
}

template <bool ASYNC>
__device__ __forceinline__ int own_label(const SweepArgs& a, int v) {
  if (a.ident) return v;
  return ASYNC ? ld_label_rw(a.prev + v) : a.prev[v];
}

template <bool ASYNC>
__device__ __forceinline__ void store_label(const SweepArgs& a, int v, int nl, bool changed) {
  if (!ASYNC) a.next[v] = nl;             // Jacobi: C^t is written for every processed vertex
  else if (changed) __stcg(a.next + v, nl);
}

// Hash tables of the d > 32 kernels: two 32-bit arrays, keys (the label,
// EMPTY32 when free) and sums.  A new label claims a key with atomicCAS;
// every entry group then adds its count to the sum with a 32-bit atomicAdd,
// which returns the label's new total (32-bit shared atomics are several
// times faster than 64-bit ones).  A table of `region` slots lives in
// `region` 64-bit words: keys first, sums after.  Linear probing from
// __umulhi(hash, cap), so any capacity works.
constexpr unsigned EMPTY32 = 0xFFFFFFFFu;

struct SlotTable {
  unsigned* keys;
  unsigned* sums;
};

__device__ __forceinline__ SlotTable make_table(unsigned long long* base, long long region) {
  unsigned* k = reinterpret_cast<unsigned*>(base);
  return {k, k + region};
}

template <bool GLOBAL>
__device__ __forceinline__ unsigned slot_add(SlotTable t, unsigned cap, unsigned lbl, unsigned c, bool& created,
                                             int* err, int probe_cap) {
  unsigned h = __umulhi(hash32(lbl), cap);
  for (int p = 0; p < probe_cap; ++p) {
    unsigned k = GLOBAL ? __ldcg(t.keys + h) : *(volatile unsigned*)(t.keys + h);
    if (k == EMPTY32) {
      k = atomicCAS(t.keys + h, EMPTY32, lbl);
      if (k == EMPTY32) {
        created = true;
        return atomicAdd(t.sums + h, c) + c;
      }
    }
    if (k == lbl) return atomicAdd(t.sums + h, c) + c;
    if (++h == cap) h = 0;
  }
  raise_err(err, ERRBIT_TIMEOUT);
  return 0;
}

// Shared-table insert that probes by compare-and-swap: one atomic per probe
// tells claimed (EMPTY), found (the label) or taken (probe on).
__device__ __forceinline__ unsigned slot_add_cas(SlotTable t, unsigned cap, unsigned lbl, unsigned c, bool& created,
                                                 int* err, int probe_cap) {
  unsigned h = __umulhi(hash32(lbl), cap);
  for (int p = 0; p < probe_cap; ++p) {
    const unsigned k = atomicCAS(t.keys + h, EMPTY32, lbl);
    if (k == EMPTY32 || k == lbl) {
      created = k == EMPTY32;
      return atomicAdd(t.sums + h, c) + c;
    }
    if (++h == cap) h = 0;
  }
  raise_err(err, ERRBIT_TIMEOUT);
  return 0;
}

// Sweep 2's entry load and label: columns were range-checked in sweep 1 (a
// bad one failed the call there), so an out-of-range column is only
// clamped away (memory safety for the batched loop, which reads errors at
// the end); no pre-gathered labels or identity labelling in sweep 2.
__device__ __forceinline__ int spread_col(const SweepArgs& a, const int* cp, int d, int e, const Pol& pol) {
  const int j = e < d ? ld_stream(cp + e, pol.stream) : -1;
  return (unsigned)j < (unsigned)a.n ? j : -1;
}
__device__ __forceinline__ int spread_label(const SweepArgs& a, int j, int v, const Pol& pol) {
  return (j < 0 || j == v) ? -1 : ld_label_ro(a.prev + j, pol.label);
}

// Lanes of a warp's chunk holding label l, merged so that one insert per
// distinct label reaches the table.  When the labels read are nearly all
// distinct (a.spread) the match costs more than it merges: every lane is
// its own group.
__device__ __forceinline__ unsigned label_group(int l, int spread) {
  if (spread) return 1u << (threadIdx.x & 31);
  return __match_any_sync(FULL, l);
}

// Row loops specialised for sweep 2 from the identity labelling (SPREAD):
// the labels of sweep 1 are nearly all distinct and the vertex's own label
// is rarely among them, so every lane inserts its own entry (no label
// match) and the own label goes into the table like any other label (no
// per-chunk own-label count); the running maximum then covers it, so the
// result is the same.

}  // namespace

// Per-row values shared by a block.  Rows alternate between two copies, so
// a row's copy can be reset while slower threads still read the previous
// row's: the one before that is provably no longer read.
struct BlockRowShared {
  unsigned long long best[2], wsum[2];
  unsigned used[2], own[2];
  int ovf[2];
};

// Own-label majority pass: one lean pass over the row sums, per thread, the
// weight of the entries that carry the vertex's own label and the weight of
// all entries (the vertex itself excluded).  When the own label holds more
// than half of the total it is Eq. 2's strict argmax and the row needs no
// table.  Thread tid of nthreads takes 32-entry chunks as block_row does,
// with the columns of the next round requested before this round's labels
// are compared.
template <bool WEIGHTED, bool ASYNC>
__device__ __forceinline__ void own_weight_pass(const SweepArgs& a, int v, int own, const int* cp, const int* wp,
                                                const int* lp, int d, int tid, int nthreads, const Pol& pol,
                                                unsigned& own_w, unsigned& tot_w) {
  const int lane = tid & 31, wid = tid >> 5, nw = nthreads >> 5;
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
    if (r0 + step < d) {
#pragma unroll
      for (int u = 0; u < 4; ++u) load_entry<WEIGHTED>(a, cp, wp, d, r0 + step + cb + u * cu, pol, jn[u], wn[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (l[u] >= 0) {
        tot_w += (unsigned)w[u];
        if (l[u] == own) own_w += (unsigned)w[u];
      }
    }
  }
}

// Reduces the block's per-thread partial results into sh[par]; the caller
// synchronises before reading them.
template <bool WEIGHTED>
__device__ __forceinline__ void block_publish(const SweepArgs& a, BlockRowShared& sh, int par,
                                              unsigned long long best, unsigned long long wsum, unsigned own_sum) {
  const int lane = threadIdx.x & 31;
  best = warp_max_u64(best);
  if (lane == 0 && best) atomicMax(&sh.best[par], best);
  if (lane == 0 && own_sum) atomicAdd(&sh.own[par], own_sum);   // own_sum is warp-uniform
  if (WEIGHTED && a.check) {
    wsum = warp_sum_u64(wsum);
    if (lane == 0 && wsum) atomicAdd(&sh.wsum[par], wsum);
  }
}

// One block aggregates the row of v into `tab` and publishes the result in
// sh[par].  A round covers blockDim.x * 4 entries; chunk u of warp w in the
// round starting at r0 holds entries r0 + (u * warps + w) * 32 + lane, so a
// row shorter than a round still spreads over every warp.  With a finite
// `limit` (shared table), a warp checks the overflow flag before each round
// and adds its new slots (at most 128) to the block's count after it; past
// `limit` the flag is raised and the row is abandoned.  Returns the flag (block-uniform
// after the closing barrier).  The global-table pass (limit infinite) leaves
// the flag alone, so every thread still reads the value that sent it there.
template <bool WEIGHTED, bool ASYNC, bool GLOBAL, bool SPREAD = false>
__device__ __forceinline__ int block_row(const SweepArgs& a, int v, int own, const int* cp, const int* wp,
                                         const int* lp, int d,
                                         SlotTable tab, unsigned cap, unsigned limit, const Pol& pol,
                                         BlockRowShared& sh, int par) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int step = nw * 128;
  const int cb = wid * 32 + lane;   // offset of chunk 0 within a round
  const int cu = nw * 32;           // distance between the chunks of a warp
  unsigned long long best = 0, wsum = 0;
  unsigned own_sum = 0;
  int jn[4], wn[4], ln[4], lw[4];
  constexpr bool LEAN = SPREAD && !WEIGHTED;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (LEAN) { jn[u] = spread_col(a, cp, d, cb + u * cu, pol); wn[u] = 1; }
    else load_entry<WEIGHTED>(a, cp, wp, d, cb + u * cu, pol, jn[u], wn[u]);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (!LEAN) check_same_graph(a, v, jn[u]);
    if (jn[u] >= 0) wsum += (unsigned long long)wn[u];
    ln[u] = LEAN ? spread_label(a, jn[u], v, pol) : entry_label<ASYNC>(a, lp, cb + u * cu, jn[u], v, pol);
    lw[u] = wn[u];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (LEAN) { jn[u] = spread_col(a, cp, d, step + cb + u * cu, pol); wn[u] = 1; }
    else load_entry<WEIGHTED>(a, cp, wp, d, step + cb + u * cu, pol, jn[u], wn[u]);
  }
  for (unsigned k = threadIdx.x; k < cap; k += blockDim.x) {
    tab.keys[k] = EMPTY32;
    tab.sums[k] = 0;
  }
  if (threadIdx.x == 0) {
    sh.best[par] = 0;
    sh.wsum[par] = 0;
    sh.own[par] = 0;
    if (!GLOBAL) {
      sh.used[par] = 0;
      sh.ovf[par] = 0;
    }
  }
  __syncthreads();
  for (int r0 = 0; r0 < d; r0 += step) {
    int l[4], w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      l[u] = ln[u];
      w[u] = lw[u];
    }
    if (r0 + step < d) {   // block-uniform
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (!LEAN) check_same_graph(a, v, jn[u]);
        if (jn[u] >= 0) wsum += (unsigned long long)wn[u];
        ln[u] = LEAN ? spread_label(a, jn[u], v, pol) : entry_label<ASYNC>(a, lp, r0 + step + cb + u * cu, jn[u], v, pol);
        lw[u] = wn[u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (LEAN) { jn[u] = spread_col(a, cp, d, r0 + 2 * step + cb + u * cu, pol); wn[u] = 1; }
        else load_entry<WEIGHTED>(a, cp, wp, d, r0 + 2 * step + cb + u * cu, pol, jn[u], wn[u]);
      }
    }
    const bool counted = !GLOBAL && limit != 0xFFFFFFFFu;
    if (counted && __shfl_sync(FULL, lane == 0 ? *(volatile int*)&sh.ovf[par] : 0, 0)) break;   // warp-uniform
    unsigned created_round = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (r0 + (u * nw + wid) * 32 < d) {   // warp-uniform
        if (!SPREAD) {
          const bool mine = l[u] == own;
          own_sum += WEIGHTED ? __reduce_add_sync(FULL, mine ? (unsigned)w[u] : 0u)
                              : (unsigned)__popc(__ballot_sync(FULL, mine));
          if (mine) l[u] = -1;
        }
        if (__ballot_sync(FULL, l[u] >= 0) == 0) continue;
        const unsigned m = SPREAD ? 1u << lane : label_group(l[u], a.spread);
        const unsigned c = SPREAD ? (WEIGHTED ? (unsigned)w[u] : 1u)
                                  : (WEIGHTED ? __reduce_add_sync(m, (unsigned)w[u]) : (unsigned)__popc(m));
        bool created = false;
        if (l[u] >= 0 && (SPREAD || (m & lanemask_lt()) == 0)) {
          const unsigned sum = (LEAN && !GLOBAL)
                                   ? slot_add_cas(tab, cap, (unsigned)l[u], c, created, &a.ctr->err, a.probe_cap)
                                   : slot_add<GLOBAL>(tab, cap, (unsigned)l[u], c, created, &a.ctr->err, a.probe_cap);
          const unsigned long long k = pack_key(sum, l[u]);
          best = k > best ? k : best;
        }
        if (counted) created_round += __popc(__ballot_sync(FULL, created));
      }
    }
    if (counted && lane == 0 && created_round && atomicAdd(&sh.used[par], created_round) + created_round > limit)
      *(volatile int*)&sh.ovf[par] = 1;
  }
  block_publish<WEIGHTED>(a, sh, par, best, wsum, own_sum);
  __syncthreads();
  return GLOBAL ? 0 : *(volatile int*)&sh.ovf[par];
}

}  // namespace gsl
