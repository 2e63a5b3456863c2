// lpa_kernels.cu -- the label-propagation sweep of GSL-LPA on sm_103a.
//
// One sweep applies Eq. 2 (C_i = argmax_c sum_{j in J_i, C_j = c} w_ij,
// scanCommunities() of Algorithm 3 skipping j == i) to every vertex of the
// frontier, with ties going to the smallest label.  Integer weights make the
// per-label sums exact and the argmax a max over the packed 64-bit key
// (sum << 32 | ~label), so the result does not depend on the order in which
// threads add: the synchronous sweep is deterministic.
//
// Work is split by degree class (binning pass below):
//   d <= 32          lane groups of G = 1..32 lanes, one vertex per group;
//                    equal labels are found with __match_any_sync and summed
//                    with __popc / __reduce_add_sync; the argmax is two
//                    __reduce_max_sync.  No shared memory.
//   d <= warp_small  one warp per vertex, 4 KB shared table (never overflows).
//   d <= warp_max    one warp per vertex, 8 KB shared table, global spill.
//   d <= blk_max     one block per vertex, 96 KB shared table, global spill.
//   larger           one block per vertex, straight to global tables when
//                    labels are known to be mostly distinct.
// The hash kernels never scan their table: every insert returns the new sum
// of its label, each thread keeps the largest packed key it has produced,
// and the final sum of every label is produced by the thread that added
// last, so the maximum of those keys is the argmax.
//
// Pruning (lpaMove(): a processed vertex is re-marked when a neighbour
// changes): a vertex whose label changes sets the next-frontier flag of each
// neighbour and, in synchronous mode, of itself (the double buffer then
// stays consistent for unprocessed vertices).  Eq. 2 depends on neighbour
// labels only, so skipping the other vertices gives the same labels as a
// full sweep.
#include <atomic>
#include <mutex>
#include <unordered_map>

#include "sweep_device.cuh"

namespace gsl {


// ---------------------------------------------------------------------------
// Static classification of all vertices: class totals, region starts, max
// degree; validates the offsets array.
__global__ void class_histogram_kernel(const long long* __restrict__ off, long long n, long long nnz, ClassBounds cb,
                                       Counters* ctr) {
  __shared__ unsigned long long hist[NCLASS];
  __shared__ unsigned long long hub_e;
  __shared__ long long maxd;
  __shared__ int bad;
  if (threadIdx.x < NCLASS) hist[threadIdx.x] = 0;
  if (threadIdx.x == 0) { maxd = 0; bad = 0; hub_e = 0; }
  __syncthreads();
  long long lmax = 0;
  int lbad = 0;
  // whole warps step together (the bound is warp-uniform), so that equal
  // classes are counted with one shared atomic per warp
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long v0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
  for (long long w = v0; w < n; w += stride) {
    const long long v = w + (threadIdx.x & 31);
    int c = -1;
    if (v < n) {
      const long long s = off[v], e = off[v + 1];
      if (s < 0 || e < s || e > nnz) {
        lbad |= ERRBIT_INVALID;
      } else if (e - s >= (1ll << 31)) {
        lbad |= ERRBIT_OVERFLOW;
      } else {
        const long long d = e - s;
        lmax = d > lmax ? d : lmax;
        c = degree_class(d, cb.warp_small, cb.warp_max, cb.blk_max);
        if (c == CLS_HUB) atomicAdd(&hub_e, (unsigned long long)d);
      }
      if (v == 0 && s != 0) lbad |= ERRBIT_INVALID;
      if (v == n - 1 && e != nnz) lbad |= ERRBIT_INVALID;
    }
    const unsigned m = __match_any_sync(FULL, c);
    if (c >= 0 && (m & lanemask_lt()) == 0) atomicAdd(&hist[c], (unsigned long long)__popc(m));
  }
  if (lmax) atomicMax(&maxd, lmax);
  if (lbad) atomicOr(&bad, lbad);
  __syncthreads();
  if (threadIdx.x < NCLASS && hist[threadIdx.x]) atomicAdd(&ctr->cls_total[threadIdx.x], hist[threadIdx.x]);
  if (threadIdx.x == 0) {
    if (maxd) atomicMax(&ctr->max_degree, maxd);
    if (hub_e) atomicAdd(&ctr->hub_entries, hub_e);
    if (bad) atomicOr(&ctr->err, bad);
  }
}

__global__ void class_starts_kernel(Counters* ctr) {
  unsigned long long run = 0;
  for (int c = 0; c < NCLASS; ++c) {
    ctr->cls_start[c] = run;
    run += ctr->cls_total[c];
  }
}

// ---------------------------------------------------------------------------
// Phase of vertex v in the asynchronous sweep with seed `seed` (the sweep
// number): the top bit of a mixed hash, so that two neighbours fall in the
// same phase of a sweep with probability 1/2, independently from sweep to
// sweep.
__device__ __forceinline__ int sweep_phase(long long v, unsigned seed) {
  unsigned h = (unsigned)v * 0x9E3779B1u + seed * 0x85EBCA6Bu;
  h ^= h >> 16;
  h *= 0x7FEB352Du;
  h ^= h >> 15;
  h *= 0x846CA68Bu;
  h ^= h >> 16;
  return (int)(h >> 31);
}

// Frontier binning: every vertex with its flag set (or every vertex when
// all_active) is appended to its class region; the flag is cleared, which
// leaves the flag array zeroed for reuse as the frontier after next.  With
// phase >= 0 only the vertices of that phase (sweep_phase) are taken; the
// flags of the others stay set for the binning of the other phase.
// PHASED is a template flag so that the one-phase binning of synchronous
// sweeps carries no phase test.
constexpr int BIN_ITEMS = 8;
constexpr int BIN_BLOCKS = 6;   // resident 256-thread blocks per SM (40 registers); the grid is no larger

template <bool PHASED>
__global__ void __launch_bounds__(256, BIN_BLOCKS) bin_kernel(const long long* __restrict__ off, long long n,
                                                   unsigned char* __restrict__ fcur, int all_active, ClassBounds cb,
                                                   int* __restrict__ work, Counters* ctr, const int* __restrict__ gid,
                                                   const unsigned char* __restrict__ done, const int* stop, int phase,
                                                   unsigned seed) {
  if (stop && *(volatile const int*)stop) return;
  __shared__ unsigned cnt[NCLASS];
  __shared__ unsigned base[NCLASS];
  const long long tile = (long long)blockDim.x * BIN_ITEMS;
  for (long long t0 = (long long)blockIdx.x * tile; t0 < n; t0 += (long long)gridDim.x * tile) {
    if (threadIdx.x < NCLASS) cnt[threadIdx.x] = 0;
    __syncthreads();
    int cls[BIN_ITEMS];
    unsigned pos[BIN_ITEMS];
#pragma unroll
    for (int k = 0; k < BIN_ITEMS; ++k) {
      const long long v = t0 + (long long)k * blockDim.x + threadIdx.x;
      cls[k] = -1;
      if (v < n) {
        bool act = all_active != 0;
        if (!PHASED) {
          if (!act && fcur[v]) {
            act = true;
            fcur[v] = 0;
          }
        } else if (act) {
          if (sweep_phase(v, seed) != phase) act = false;
        } else if (fcur[v] && sweep_phase(v, seed) == phase) {
          act = true;
          fcur[v] = 0;
        }
        if (act && gid && done[gid[v]]) act = false;   // batched: this vertex's graph has stopped
        if (act) cls[k] = degree_class(off[v + 1] - off[v], cb.warp_small, cb.warp_max, cb.blk_max);
      }
    }
    // every item's class is known before any is counted, so that the
    // tile's offset loads are all in flight together
#pragma unroll
    for (int k = 0; k < BIN_ITEMS; ++k) {
      // one shared-memory add per class present in the warp
      const unsigned m = __match_any_sync(FULL, cls[k]);
      const int leader = __ffs(m) - 1;
      unsigned b = 0;
      if ((int)(threadIdx.x & 31) == leader && cls[k] >= 0) b = atomicAdd(&cnt[cls[k]], (unsigned)__popc(m));
      pos[k] = __shfl_sync(FULL, b, leader) + (unsigned)__popc(m & lanemask_lt());
    }
    __syncthreads();
    if (threadIdx.x < NCLASS) base[threadIdx.x] = cnt[threadIdx.x] ? atomicAdd(&ctr->cls_count[threadIdx.x], cnt[threadIdx.x]) : 0u;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BIN_ITEMS; ++k) {
      if (cls[k] >= 0) {
        const long long v = t0 + (long long)k * blockDim.x + threadIdx.x;
        work[ctr->cls_start[cls[k]] + base[cls[k]] + pos[k]] = (int)v;
      }
    }
    __syncthreads();
  }
}

__global__ void init_labels_kernel(const int* __restrict__ init, int* __restrict__ a, int* __restrict__ b, long long n,
                                   Counters* ctr) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    int x = (int)v;
    if (init) {
      x = init[v];
      if (x < 0 || x >= n) {
        raise_err(&ctr->err, ERRBIT_INVALID);
        x = (int)v;
      }
    }
    a[v] = x;
    if (b) b[v] = x;
  }
}

// ---------------------------------------------------------------------------
// Classes 0..5: G lanes per vertex, 32/G vertices per warp per step.  A row
// costs a chain of dependent loads (worklist entry, offsets, column, label),
// so the rows of later steps are fetched ahead: the worklist entry two steps
// ahead, the offsets one step ahead.  Eight 256-thread blocks per SM (32
// registers): the kernel waits on its label gathers, and full occupancy
// hides them better than fewer blocks with the column fetched ahead too.
constexpr int GROUP_MIN_BLOCKS = 8;   // 256-thread blocks per SM

template <int G, bool WEIGHTED, bool ASYNC>
__global__ void __launch_bounds__(256, GROUP_MIN_BLOCKS) sweep_group_kernel(SweepArgs a, int cls) {
  if (stopped(a)) return;
  const unsigned cnt = a.ctr->cls_count[cls];
  const int* __restrict__ work = a.work + a.ctr->cls_start[cls];
  const Pol pol = make_pol();
  const int lane = threadIdx.x & 31;
  const int gl = lane & (G - 1);
  const int gbase = lane & ~(G - 1);
  const unsigned gmask = (G == 32) ? FULL : (((1u << G) - 1u) << gbase);
  constexpr int PER_WARP = 32 / G;
  const long long warp_id = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long stride = nwarps * PER_WARP;
  // this lane group's row in the step whose first item is `it`: its vertex,
  // or -1 past the worklist (then nothing of the row is read)
  auto vertex_at = [&](long long it) -> int { return it < (long long)cnt ? work[it] : -1; };
  auto row_of = [&](int u, long long& rs, int& rd) {
    rs = 0;
    rd = 0;
    if (u >= 0) {
      rs = a.off[u];
      rd = (int)(a.off[u + 1] - rs);
    }
  };
  const long long item0 = warp_id * PER_WARP + lane / G;
  int v = vertex_at(item0), vn = vertex_at(item0 + stride);
  long long s;
  int d;
  row_of(v, s, d);
  unsigned long long my_dn = 0, my_scan = 0;
  for (long long wb = warp_id * PER_WARP; wb < (long long)cnt; wb += stride) {
    const long long item = wb + lane / G;
    // fetch ahead: the worklist entry two steps on, the offsets of the next step
    const int vf = vertex_at(item + 2 * stride);
    long long sf;
    int df;
    row_of(vn, sf, df);
    int j, wt;
    load_entry<WEIGHTED>(a, a.col + s, a.w + s, d, gl, pol, j, wt);
    const bool has = v >= 0;
    const int vv = has ? v : 0;
    check_same_graph(a, vv, j);
    const bool nb = j >= 0;
    const bool valid = nb && j != vv;       // scanCommunities skips j == i
    const int lbl = entry_label<ASYNC>(a, a.lg ? a.lg + s : nullptr, gl, j, vv, pol);
    const int old = (has && gl == 0) ? own_label<ASYNC>(a, vv) : 0;
    if (WEIGHTED && a.check) {
      unsigned long long ws = nb ? (unsigned long long)wt : 0ull;
#pragma unroll
      for (int o = G / 2; o >= 1; o >>= 1) ws += __shfl_xor_sync(FULL, ws, o);
      if (gl == 0 && has && ws >= (1ull << 31)) raise_err(&a.ctr->err, ERRBIT_OVERFLOW);
    }
    const unsigned m = __match_any_sync(FULL, lbl) & gmask;
    const unsigned c = WEIGHTED ? __reduce_add_sync(m, (unsigned)wt) : (unsigned)__popc(m);
    const unsigned cc = valid ? c : 0u;
    const unsigned mc = __reduce_max_sync(gmask, cc);
    const unsigned cand = (valid && cc == mc) ? ~(unsigned)lbl : 0u;
    const unsigned binv = __reduce_max_sync(gmask, cand);
    bool changed = false;
    if (has && gl == 0) {
      const int nl = mc ? (int)~binv : old;
      changed = nl != old;
      store_label<ASYNC>(a, vv, nl, changed);
      if (changed) count_graph_change(a, vv);
      my_scan += (unsigned long long)d;
      my_dn += changed ? 1ull : 0ull;
    }
    if (a.mark) {
      const unsigned chm = __ballot_sync(FULL, changed);
      if ((chm >> gbase) & 1u) {
        if (nb) a.fnext[j] = 1;
        if (!ASYNC && gl == 0) a.fnext[vv] = 1;
      }
    }
    v = vn;
    s = sf;
    d = df;
    vn = vf;
  }
  flush_counters(a.ctr, cls, my_dn, my_scan);
}

// ---------------------------------------------------------------------------
// Sweep 1 from the identity labelling on a row whose columns are strictly
// increasing: every neighbour id is its own label and occurs once, so the
// sum of label j is w_ij and the argmax is the max of (w_ij, ~j).  Returns
// false if the row is not strictly increasing (the caller then hashes).
// `best` is the per-thread partial key; `wsum` the per-thread weight sum.
template <bool WEIGHTED>
__device__ __forceinline__ bool ident_sorted_pass(const SweepArgs& a, int v, long long s, int d, int tid, int nthreads,
                                                  const Pol& pol, unsigned long long& best, unsigned long long& wsum) {
  bool sorted = true;
  const int* cp = a.col + s;
  const int* wp = a.w + s;
  const int lane = tid & 31, wid = tid >> 5, nw = nthreads >> 5;
  // each warp takes 128-entry rounds: four chunks in flight per lane
  for (int e0 = wid * 128; e0 < d; e0 += nw * 128) {
    int j[4], w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) load_entry<WEIGHTED>(a, cp, wp, d, e0 + 32 * u + lane, pol, j[u], w[u]);
    const int tail = (lane == 31 && e0 + 128 < d) ? ld_stream(cp + e0 + 128, pol.stream) : 0x7FFFFFFF;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + 32 * u + lane;
      int nxt = __shfl_down_sync(FULL, j[u], 1);
      const int head = u < 3 ? __shfl_sync(FULL, j[u < 3 ? u + 1 : u], 0) : tail;
      if (lane == 31) nxt = head;
      check_same_graph(a, v, j[u]);
      if (j[u] >= 0 && e + 1 < d && !(j[u] < nxt)) sorted = false;
      if (j[u] < 0 && e < d) sorted = false;      // invalid entry: let the hash path handle it
      if (j[u] >= 0) {
        wsum += (unsigned long long)w[u];
        if (j[u] != v) {
          const unsigned long long k = pack_key((unsigned)w[u], j[u]);
          best = k > best ? k : best;
        }
      }
    }
  }
  return sorted;
}

// ---------------------------------------------------------------------------

// Rows of 33..SORT_MAX entries, unit weights: one warp sorts the row's
// labels in registers instead of hashing them.  Lane l holds entries
// r * 32 + l (r < SORT_K); a bitonic network (shuffles for partners in other
// lanes, in-register steps for partners r ^ (j / 32)) sorts the keys
// ascending, with absent entries (past the row end, out of range, the vertex
// itself) as 0xFFFFFFFF at the end.  Equal labels then form runs: a run's
// length is the label's count, and the largest packed key (count, ~label)
// over the run starts is Eq. 2's argmax with ties to the smallest label, the
// same as the table's.  No shared memory, no atomics.  Returns the lane's
// partial key (0: none).
constexpr int SORT_K = 2;
constexpr int SORT_MAX = 32 * SORT_K;

template <bool ASYNC>
__device__ __forceinline__ unsigned long long warp_sort_row(const SweepArgs& a, int v, const int* cp, const int* lp,
                                                            int d, const Pol& pol) {
  constexpr int N = 32 * SORT_K;
  const int lane = threadIdx.x & 31;
  unsigned x[SORT_K];
#pragma unroll
  for (int r = 0; r < SORT_K; ++r) {
    int j, wt;
    load_entry<false>(a, cp, nullptr, d, r * 32 + lane, pol, j, wt);
    check_same_graph(a, v, j);
    const int l = entry_label<ASYNC>(a, lp, r * 32 + lane, j, v, pol);
    x[r] = l >= 0 ? (unsigned)l : 0xFFFFFFFFu;
  }
#pragma unroll
  for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= 32) {   // partner r ^ (j / 32): the same lane's other keys
#pragma unroll
        for (int r = 0; r < SORT_K; ++r) {
          const int h = r ^ (j >> 5);
          if (r < h) {
            const bool ascending = (((r * 32 + lane) & k) == 0);
            const unsigned lo = min(x[r], x[h]), hi = max(x[r], x[h]);
            x[r] = ascending ? lo : hi;
            x[h] = ascending ? hi : lo;
          }
        }
      } else {
#pragma unroll
        for (int r = 0; r < SORT_K; ++r) {
          const unsigned y = __shfl_xor_sync(FULL, x[r], j);
          const bool ascending = (((r * 32 + lane) & k) == 0);
          const bool keep_min = ((lane & j) == 0) == ascending;
          x[r] = keep_min ? min(x[r], y) : max(x[r], y);
        }
      }
    }
  }
  // run starts: key i differs from key i - 1
  unsigned w[SORT_K];
  bool st[SORT_K];
#pragma unroll
  for (int r = 0; r < SORT_K; ++r) {
    unsigned p = __shfl_up_sync(FULL, x[r], 1);
    const unsigned last = __shfl_sync(FULL, x[r > 0 ? r - 1 : 0], 31);
    if (lane == 0 && r > 0) p = last;
    st[r] = (lane == 0 && r == 0) || x[r] != p;
    w[r] = __ballot_sync(FULL, st[r]);
  }
  unsigned long long best = 0;
#pragma unroll
  for (int r = 0; r < SORT_K; ++r) {
    if (st[r] && x[r] != 0xFFFFFFFFu) {
      const unsigned above = lane < 31 ? w[r] & ~((2u << lane) - 1u) : 0u;
      int next = N;
      if (above) {
        next = r * 32 + __ffs((int)above) - 1;
      } else {
#pragma unroll
        for (int q = SORT_K - 1; q > r; --q)
          if (w[q]) next = q * 32 + __ffs((int)w[q]) - 1;
      }
      const unsigned long long key = pack_key((unsigned)(next - (r * 32 + lane)), (int)x[r]);
      best = key > best ? key : best;
    }
  }
  return best;
}

// One warp aggregates the row (cp, wp, d) of vertex v into `tab` (cap
// slots).  Four 32-entry chunks are loaded (columns, then labels) before any
// is hashed, so each lane keeps eight loads in flight.  Within a chunk equal
// labels are merged with __match_any_sync (label_group) and only the lowest
// lane of each group inserts.  Returns true (warp-uniform) once more than `limit`
// distinct labels have been inserted: the table is then abandoned.
template <bool WEIGHTED, bool ASYNC, bool GLOBAL, bool SPREAD = false, bool LEAN_OK = false>
__device__ __forceinline__ bool warp_row(const SweepArgs& a, int v, int own, const int* cp, const int* wp,
                                         const int* lp, int d,
                                         SlotTable tab, unsigned cap, unsigned limit, const Pol& pol,
                                         unsigned long long& best, unsigned long long& wsum, unsigned& own_sum) {
  const int lane = threadIdx.x & 31;
  // three rounds in flight: labels of round r+1 and columns of round r+2
  // are requested before round r is hashed
  int jn[4], wn[4], ln[4], lw[4];
  // sweep 2's lean loads (sweep_device.cuh) in classes 6 and 7 (class 6:
  // 9.1 -> 8.5 ms per step on R-MAT 25); the compare-and-swap-first insert
  // in class 7 only (on class 6's short rows it measured 9.2 -> 9.5 ms)
  constexpr bool LEAN = SPREAD && !WEIGHTED;
  constexpr bool LEAN_CAS = LEAN && LEAN_OK;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (LEAN) {
      jn[u] = spread_col(a, cp, d, 32 * u + lane, pol);
      wn[u] = 1;
    } else {
      load_entry<WEIGHTED>(a, cp, wp, d, 32 * u + lane, pol, jn[u], wn[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (!LEAN) check_same_graph(a, v, jn[u]);
    if (jn[u] >= 0) wsum += (unsigned long long)wn[u];
    ln[u] = LEAN ? spread_label(a, jn[u], v, pol) : entry_label<ASYNC>(a, lp, 32 * u + lane, jn[u], v, pol);
    lw[u] = wn[u];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (LEAN) {
      jn[u] = spread_col(a, cp, d, 128 + 32 * u + lane, pol);
      wn[u] = 1;
    } else {
      load_entry<WEIGHTED>(a, cp, wp, d, 128 + 32 * u + lane, pol, jn[u], wn[u]);
    }
  }
  for (unsigned k = lane; k < cap; k += 32) {
    tab.keys[k] = EMPTY32;
    tab.sums[k] = 0;
  }
  __syncwarp();
  unsigned used = 0;
  for (int e0 = 0; e0 < d; e0 += 128) {
    int l[4], w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      l[u] = ln[u];
      w[u] = lw[u];
    }
    if (e0 + 128 < d) {   // warp-uniform
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (!LEAN) check_same_graph(a, v, jn[u]);
        if (jn[u] >= 0) wsum += (unsigned long long)wn[u];
        ln[u] = LEAN ? spread_label(a, jn[u], v, pol)
                     : entry_label<ASYNC>(a, lp, e0 + 128 + 32 * u + lane, jn[u], v, pol);
        lw[u] = wn[u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (LEAN) {
          jn[u] = spread_col(a, cp, d, e0 + 256 + 32 * u + lane, pol);
          wn[u] = 1;
        } else {
          load_entry<WEIGHTED>(a, cp, wp, d, e0 + 256 + 32 * u + lane, pol, jn[u], wn[u]);
        }
      }
    }
    if (!WEIGHTED && !SPREAD) {
      // entries carrying the vertex's own label are counted in registers,
      // the round's four chunks first: once they are more than half of the
      // row's d entries no other label can reach their count, and the rest
      // of the row is not needed (after sweep 1, which reads every entry)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (e0 + 32 * u < d) {   // warp-uniform: skip empty chunks of short rows
          const bool mine = l[u] == own;
          own_sum += (unsigned)__popc(__ballot_sync(FULL, mine));
          if (mine) l[u] = -1;
        }
      }
      if (!a.check && 2u * own_sum > (unsigned)d) return false;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (e0 + 32 * u < d) {   // warp-uniform: skip empty chunks of short rows
        if (WEIGHTED && !SPREAD) {   // own-label weights summed in registers
          const bool mine = l[u] == own;
          own_sum += __reduce_add_sync(FULL, mine ? (unsigned)w[u] : 0u);
          if (mine) l[u] = -1;
        }
        if (__ballot_sync(FULL, l[u] >= 0) == 0) continue;
        const unsigned m = SPREAD ? 1u << lane : label_group(l[u], a.spread);
        const unsigned c = SPREAD ? (WEIGHTED ? (unsigned)w[u] : 1u)
                                  : (WEIGHTED ? __reduce_add_sync(m, (unsigned)w[u]) : (unsigned)__popc(m));
        bool created = false;
        if (l[u] >= 0 && (SPREAD || (m & lanemask_lt()) == 0)) {
          const unsigned sum = (LEAN_CAS && !GLOBAL)
                                   ? slot_add_cas(tab, cap, (unsigned)l[u], c, created, &a.ctr->err, a.probe_cap)
                                   : slot_add<GLOBAL>(tab, cap, (unsigned)l[u], c, created, &a.ctr->err, a.probe_cap);
          const unsigned long long k = pack_key(sum, l[u]);
          best = k > best ? k : best;
        }
        if (limit != 0xFFFFFFFFu) used += __popc(__ballot_sync(FULL, created));
      }
    }
    if (used > limit) return true;   // at most 128 slots past the limit
  }
  return false;
}

// Classes 6 and 7: one warp per vertex, TW slots of shared memory per warp
// (class 6: four 256-thread blocks per SM, registers capped to fit; class
// 7's 8 KB tables allow three).
// With SPILL, a vertex whose labels overflow the shared table is redone in
// the warp's region of the global fallback tables (2 * warp_max slots);
// without it the class bound guarantees 2 d <= TW.  The worklist entry of
// the row after next and the offsets of the next row are loaded while the
// current one is processed.
template <bool WEIGHTED, bool ASYNC, int TW, bool SPILL, bool SPREAD = false>
__global__ void __launch_bounds__(256, TW <= 512 ? 4 : 3) sweep_warp_kernel(SweepArgs a, int cls) {
  if (stopped(a)) return;
  extern __shared__ unsigned long long smem_w64[];
  const int lane = threadIdx.x & 31;
  const SlotTable tab = make_table(smem_w64 + (size_t)(threadIdx.x >> 5) * TW, TW);
  const long long warp_id = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const SlotTable gtab = SPILL ? make_table(a.wtab + warp_id * a.wtab_region, a.wtab_region) : SlotTable{nullptr, nullptr};
  const unsigned cnt = a.ctr->cls_count[cls];
  const int* __restrict__ work = a.work + a.ctr->cls_start[cls];
  const Pol pol = make_pol();
  unsigned long long my_dn = 0, my_scan = 0;
  long long item = warp_id;
  int vn = 0, vnn = 0;
  long long sn = 0, en = 0;
  if (item < (long long)cnt) {
    vn = work[item];
    sn = a.off[vn];
    en = a.off[vn + 1];
  }
  if (item + nwarps < (long long)cnt) vnn = work[item + nwarps];
  while (item < (long long)cnt) {
    const int v = vn;
    const long long s = sn;
    const int d = (int)(en - sn);
    const long long next_item = item + nwarps;
    if (next_item < (long long)cnt) {   // its worklist entry came one row earlier
      vn = vnn;
      sn = a.off[vn];
      en = a.off[vn + 1];
    }
    if (next_item + nwarps < (long long)cnt) vnn = work[next_item + nwarps];
    const int old = own_label<ASYNC>(a, v);
    const int* cp = a.col + s;
    const int* wp = a.w + s;
    unsigned long long best = 0, wsum = 0;
    bool done = false;
    if (a.ident && !ASYNC) done = __all_sync(FULL, ident_sorted_pass<WEIGHTED>(a, v, s, d, lane, 32, pol, best, wsum));
    if (!done && !WEIGHTED && d <= SORT_MAX) {   // warp-uniform
      best = warp_sort_row<ASYNC>(a, v, cp, a.lg ? a.lg + s : nullptr, d, pol);
      done = true;
    }
    if (!done) {
      best = 0;
      wsum = 0;
      const unsigned want = 2u * (unsigned)d;
      const unsigned cap = want < (unsigned)TW ? want : (unsigned)TW;
      const unsigned limit = (!SPILL || cap >= want) ? 0xFFFFFFFFu : cap / 4 * 3 - 128;
      unsigned own_sum = 0;
      const int* lp = a.lg ? a.lg + s : nullptr;
      if (warp_row<WEIGHTED, ASYNC, false, SPREAD, SPILL>(a, v, old, cp, wp, lp, d, tab, cap, limit, pol, best, wsum,
                                                          own_sum) &&
          SPILL) {
        best = 0;
        wsum = 0;
        own_sum = 0;
        warp_row<WEIGHTED, ASYNC, true, SPREAD, SPILL>(a, v, old, cp, wp, lp, d, gtab, want, 0xFFFFFFFFu, pol, best,
                                                       wsum, own_sum);
      }
      __syncwarp();
      if (own_sum) {   // own_sum is warp-uniform
        const unsigned long long k = pack_key(own_sum, old);
        best = k > best ? k : best;
      }
    }
    best = warp_max_u64(best);
    if (WEIGHTED && a.check) {
      wsum = warp_sum_u64(wsum);
      if (lane == 0 && wsum >= (1ull << 31)) raise_err(&a.ctr->err, ERRBIT_OVERFLOW);
      if (lane == 0 && a.kw) a.kw[v] = wsum < (1ull << 32) ? (unsigned)wsum : ~0u;
    }
    const int nl = best ? (int)~(unsigned)best : old;
    const bool changed = nl != old;
    if (lane == 0) {
      store_label<ASYNC>(a, v, nl, changed);
      if (changed) count_graph_change(a, v);
      my_scan += (unsigned long long)d;
      my_dn += changed ? 1ull : 0ull;
    }
    if (changed && a.mark) {
      for (int e = lane; e < d; e += 32) {
        const int j = ld_stream(cp + e, pol.stream);
        if ((unsigned)j < (unsigned)a.n) a.fnext[j] = 1;
      }
      if (!ASYNC && lane == 0) a.fnext[v] = 1;
    }
    item = next_item;
  }
  flush_counters(a.ctr, cls, my_dn, my_scan);
}

// Classes 8 and 9: one block per vertex, `tb` slots of shared memory; a
// vertex whose labels overflow it (or, when gthresh > 0, whose degree
// exceeds gthresh) is aggregated in the block's region of the global
// fallback tables instead (a.btab_region slots).  Two barriers per row: one
// after the table is cleared, one after the partial results are published.
// The worklist entry of the row after next and the offsets and own label
// of the next row are loaded while the current row is processed.
template <bool WEIGHTED, bool ASYNC, bool SPREAD = false>
__global__ void __launch_bounds__(512, 2) sweep_block_kernel(SweepArgs a, int cls, unsigned tb, int gthresh) {
  if (stopped(a)) return;
  extern __shared__ unsigned long long smem_b64[];
  __shared__ BlockRowShared sh;
  const SlotTable gtab = make_table(a.btab + (long long)blockIdx.x * a.btab_region, a.btab_region);
  const SlotTable stab = make_table(smem_b64, tb);
  const unsigned cnt = a.ctr->cls_count[cls];
  const int* __restrict__ work = a.work + a.ctr->cls_start[cls];
  const Pol pol = make_pol();
  const long long G = gridDim.x;
  unsigned long long my_dn = 0, my_scan = 0;
  long long item = blockIdx.x;
  int v = 0, old = 0, v1 = 0;
  long long s = 0, e = 0;
  if (item < (long long)cnt) {
    v = work[item];
    s = a.off[v];
    e = a.off[v + 1];
    old = own_label<ASYNC>(a, v);
  }
  if (item + G < (long long)cnt) v1 = work[item + G];
  for (int par = 0; item < (long long)cnt; item += G, par ^= 1) {
    long long s1 = 0, e1 = 0;
    int old1 = 0, v2 = 0;
    if (item + G < (long long)cnt) {
      s1 = a.off[v1];
      e1 = a.off[v1 + 1];
      old1 = own_label<ASYNC>(a, v1);
    }
    if (item + 2 * G < (long long)cnt) v2 = work[item + 2 * G];
    const int d = (int)(e - s);
    const int* cp = a.col + s;
    const int* wp = a.w + s;
    const int* lp = a.lg ? a.lg + s : nullptr;
    int sorted = 0;
    if (a.ident && !ASYNC) {
      unsigned long long best = 0, wsum = 0;
      if (threadIdx.x == 0) {
        sh.best[par] = 0;
        sh.wsum[par] = 0;
        sh.own[par] = 0;
      }
      sorted = __syncthreads_and(ident_sorted_pass<WEIGHTED>(a, v, s, d, threadIdx.x, blockDim.x, pol, best, wsum));
      if (sorted) {
        block_publish<WEIGHTED>(a, sh, par, best, wsum, 0u);
        __syncthreads();
      }
    }
    if (!sorted) {
      const unsigned want = 2u * (unsigned)d;
      int ovf = 1;
      if (!(gthresh > 0 && d > gthresh)) {
        const unsigned cap = want < tb ? want : tb;
        // each warp may add up to 128 new slots (one round) after the flag is
        // raised: at most 4 * threads, within the last quarter of a table of
        // at least 16 * threads slots
        const unsigned limit = cap >= want ? 0xFFFFFFFFu : cap / 4 * 3;
        ovf = block_row<WEIGHTED, ASYNC, false, SPREAD>(a, v, old, cp, wp, lp, d, stab, cap, limit, pol, sh, par);
      }
      if (ovf)
        block_row<WEIGHTED, ASYNC, true, SPREAD>(a, v, old, cp, wp, lp, d, gtab, want, 0xFFFFFFFFu, pol, sh, par);
    }
    unsigned long long b = sh.best[par];
    const unsigned own_sum = sh.own[par];
    if (own_sum) {
      const unsigned long long k = pack_key(own_sum, old);
      b = k > b ? k : b;
    }
    const int nl = b ? (int)~(unsigned)b : old;
    const bool changed = nl != old;
    if (threadIdx.x == 0) {
      if (WEIGHTED && a.check && sh.wsum[par] >= (1ull << 31)) raise_err(&a.ctr->err, ERRBIT_OVERFLOW);
      if (WEIGHTED && a.check && a.kw) a.kw[v] = sh.wsum[par] < (1ull << 32) ? (unsigned)sh.wsum[par] : ~0u;
      store_label<ASYNC>(a, v, nl, changed);
      if (changed) count_graph_change(a, v);
      my_scan += (unsigned long long)d;
      my_dn += changed ? 1ull : 0ull;
    }
    if (changed && a.mark) {   // block-uniform
      for (int x = threadIdx.x; x < d; x += blockDim.x) {
        const int j = ld_stream(cp + x, pol.stream);
        if ((unsigned)j < (unsigned)a.n) a.fnext[j] = 1;
      }
      if (!ASYNC && threadIdx.x == 0) a.fnext[v] = 1;
    }
    v = v1;
    s = s1;
    e = e1;
    old = old1;
    v1 = v2;
  }
  flush_counters(a.ctr, cls, my_dn, my_scan);
}

// ---------------------------------------------------------------------------
// The filter's pass over one row, one warp (own_weight_pass with 32
// threads): it stops as soon as the own label holds more than half of the
// row's total (d entries, or the weighted degree from sweep 1), since it
// then holds a strict majority of the whole row whatever the rest carries
// (`early`).  Returns the entries read.
template <bool WEIGHTED, bool ASYNC>
__device__ __forceinline__ int filter_row(const SweepArgs& a, int v, int own, const int* cp, const int* wp,
                                          const int* lp, int d, const Pol& pol, unsigned& own_w, unsigned& tot_w,
                                          bool& early) {
  const int lane = threadIdx.x & 31;
  const unsigned long long bound = !WEIGHTED ? (unsigned long long)d : (a.kw ? (unsigned long long)a.kw[v] : ~0ull);
  int jn[4], wn[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) load_entry<WEIGHTED>(a, cp, wp, d, lane + 32 * u, pol, jn[u], wn[u]);
  for (int r0 = 0; r0 < d; r0 += 128) {
    int l[4], w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      l[u] = entry_label<ASYNC>(a, lp, r0 + lane + 32 * u, jn[u], v, pol);
      w[u] = wn[u];
    }
    const bool more = r0 + 128 < d;   // warp-uniform
    if (more) {
#pragma unroll
      for (int u = 0; u < 4; ++u) load_entry<WEIGHTED>(a, cp, wp, d, r0 + 128 + lane + 32 * u, pol, jn[u], wn[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (l[u] >= 0) {
        tot_w += (unsigned)w[u];
        if (l[u] == own) own_w += (unsigned)w[u];
      }
    }
    if (more && 2ull * __reduce_add_sync(FULL, own_w) > bound) {
      early = true;
      return r0 + 128;
    }
  }
  return d;
}

// Own-label majority filter for classes 7 and 8 (rows of 257..blk_max
// entries by default: long enough that one extra lean pass costs less than
// a table), run before their table kernels once labels have started to
// settle.  One warp per row, no shared memory and registers capped for six
// 256-thread blocks per SM (many rows in flight): the weight of the row's entries carrying the vertex's
// own label is compared with the row's total (the vertex itself excluded).
// A strict majority is Eq. 2's argmax: the label stays and the row is done.
// Other rows are appended to `out` at their class's region and counted in
// Counters::uns_count; filter_counts_kernel then makes those the class
// counts for the table kernels.
template <bool WEIGHTED, bool ASYNC>
__global__ void __launch_bounds__(256, 6) majority_filter_kernel(SweepArgs a, int* __restrict__ out, int first_cls) {
  if (stopped(a)) return;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const Pol pol = make_pol();
  const long long c6 = first_cls <= CLS_WARP_S ? a.ctr->cls_count[CLS_WARP_S] : 0;
  const long long c67 = c6 + a.ctr->cls_count[CLS_WARP_L];
  const long long total = c67 + a.ctr->cls_count[CLS_BLOCK];
  unsigned long long my_scan = 0, my_settled = 0;
  for (long long i = warp; i < total; i += nwarps) {
    const int cls = i < c6 ? CLS_WARP_S : (i < c67 ? CLS_WARP_L : CLS_BLOCK);
    const long long start = a.ctr->cls_start[cls];
    const int v = a.work[start + (i - (i < c6 ? 0 : (i < c67 ? c6 : c67)))];
    const long long s = a.off[v];
    const int d = (int)(a.off[v + 1] - s);
    const int old = own_label<ASYNC>(a, v);
    unsigned ow = 0, tw = 0;
    bool early = false;
    const int read = filter_row<WEIGHTED, ASYNC>(a, v, old, a.col + s, a.w + s, a.lg ? a.lg + s : nullptr, d, pol, ow,
                                                 tw, early);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      ow += __shfl_xor_sync(FULL, ow, o);
      tw += __shfl_xor_sync(FULL, tw, o);
    }
    if (lane == 0) {
      if (early || 2ull * ow > (unsigned long long)tw) {
        store_label<ASYNC>(a, v, old, false);
        my_scan += (unsigned long long)read;
        my_settled += 1;
      } else {
        out[start + atomicAdd(&a.ctr->uns_count[cls], 1u)] = v;
      }
    }
  }
  my_scan = warp_sum_u64(my_scan);
  my_settled = warp_sum_u64(my_settled);
  if (lane == 0) {
    if (my_scan) atomicAdd(&a.ctr->scanned, my_scan);
    if (my_settled) atomicAdd(&a.ctr->fast_active, my_settled);
  }
}

__global__ void filter_counts_kernel(Counters* ctr, const int* stop, int first_cls) {
  if (stop && *(volatile const int*)stop) return;
  for (int k = first_cls; k <= CLS_BLOCK; ++k) ctr->cls_count[k] = ctr->uns_count[k];
}

cudaError_t launch_filter_counts(Counters* ctr, const int* stop, cudaStream_t s, int first_cls) {
  filter_counts_kernel<<<1, 1, 0, s>>>(ctr, stop, first_cls);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_majority_filter(const SweepArgs& a, int* out, bool weighted, bool async_mode,
                                   const DeviceInfo& di, cudaStream_t s, int first_cls) {
  const int grid = 16 * di.sm_count;
  if (weighted) {
    if (async_mode) majority_filter_kernel<true, true><<<grid, 256, 0, s>>>(a, out, first_cls);
    else majority_filter_kernel<true, false><<<grid, 256, 0, s>>>(a, out, first_cls);
  } else {
    if (async_mode) majority_filter_kernel<false, true><<<grid, 256, 0, s>>>(a, out, first_cls);
    else majority_filter_kernel<false, false><<<grid, 256, 0, s>>>(a, out, first_cls);
  }
  filter_counts_kernel<<<1, 1, 0, s>>>(a.ctr, a.stop, first_cls);
  count_launches(2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Edge-parallel gather of a synchronous sweep's neighbour labels.  The class
// kernels hold hash tables in shared memory, which caps their occupancy,
// and they interleave dependent loads with hashing; this pass has neither:
// every thread keeps four independent gathers in flight at full occupancy,
// and the class kernels then read the labels as a coalesced stream.
__global__ void __launch_bounds__(256) pregather_kernel(const int* __restrict__ col, long long nnz,
                                                        const int* __restrict__ prev, long long n,
                                                        int* __restrict__ lg) {
  const unsigned long long ps = policy_evict_first(), pl = policy_evict_last();
  const long long st = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * st < nnz; i += 4 * st) {
    int j[4], l[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) j[u] = ld_stream(col + i + u * st, ps);
#pragma unroll
    for (int u = 0; u < 4; ++u) l[u] = (unsigned)j[u] < (unsigned)n ? ld_label_ro(prev + j[u], pl) : -1;
#pragma unroll
    for (int u = 0; u < 4; ++u) __stcs(lg + i + u * st, l[u]);
  }
  for (; i < nnz; i += st) {
    const int j = ld_stream(col + i, ps);
    __stcs(lg + i, (unsigned)j < (unsigned)n ? ld_label_ro(prev + j, pl) : -1);
  }
}

cudaError_t launch_pregather(const int* col, long long nnz, const int* prev, long long n, int* lg,
                             const DeviceInfo& di, cudaStream_t s) {
  if (nnz <= 0) return cudaSuccess;
  long long blocks = (nnz + 255) / 256;
  const long long cap = 16ll * di.sm_count;
  pregather_kernel<<<(int)(blocks < cap ? blocks : cap), 256, 0, s>>>(col, nnz, prev, n, lg);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Sweep 1 from the identity labelling with unit weights, as three streaming
// passes instead of per-vertex row scans.  When a row is strictly
// increasing every neighbour label (its id) occurs once with weight 1, so
// Eq. 2's argmax with smallest-label ties is the smallest neighbour other
// than the vertex itself: the first entry of the row, or the second when
// the first is a self-loop.
//   1. rowstart_kernel: bit off[v] set for every non-empty row;
//   2. sorted_check_kernel: edge-parallel, flags every row that is not
//      strictly increasing and checks every column's range;
//   3. ident_first_kernel: writes the label of every unflagged row.
// Flagged rows keep their flag and are swept by the hash kernels.
__global__ void rowstart_kernel(const long long* __restrict__ off, long long n, unsigned* __restrict__ bits) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    const long long st = off[v];
    if (off[v + 1] > st) atomicOr(bits + (st >> 5), 1u << (st & 31));
  }
}

__device__ __forceinline__ long long row_of(const long long* off, long long n, long long e) {
  long long lo = 0, hi = n;   // largest r with off[r] <= e
  while (hi - lo > 1) {
    const long long mid = (lo + hi) >> 1;
    if (off[mid] <= e) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Entry e (column je) against entry e + 1 (column jn): the row is not
// strictly increasing if e + 1 continues e's row and jn <= je.  `end` is
// the end of the checked range, a row boundary (or nnz).  A flagged row
// also raises *any_bad when it is given.
__device__ __forceinline__ void check_order(const long long* off, long long n, long long end, const unsigned* bits,
                                            unsigned char* bad, unsigned* any_bad, long long e, int je, int jn) {
  const long long f = e + 1;
  if (f < end && ((__ldg(bits + (f >> 5)) >> (f & 31)) & 1u) == 0 && !(je < jn)) {
    bad[row_of(off, n, e)] = 1;
    if (any_bad && __ldcg(any_bad) == 0) atomicOr(any_bad, 1u);
  }
}

__device__ __forceinline__ void check_pair(const long long* off, long long n, long long end, const unsigned* bits,
                                           unsigned char* bad, unsigned* any_bad, Counters* ctr, long long e, int je,
                                           int jn) {
  if ((unsigned)je >= (unsigned)n) raise_err(&ctr->err, ERRBIT_INVALID);
  check_order(off, n, end, bits, bad, any_bad, e, je, jn);
}

// The entries [e0, e1) of a range that ends at a row boundary (the whole
// array: e0 = 0, e1 = nnz).  Sixteen entries per thread per round, as four
// 16-byte loads issued together; the few entries before the first 16-byte
// boundary and after the last whole quad are checked by one thread.  The
// entry after a thread's quad comes from the next lane (or the next quad
// row of the warp).  Entry indices (bits, rows, the quads' positions) are
// absolute.
__global__ void __launch_bounds__(256) sorted_check_kernel(const long long* __restrict__ off, long long n,
                                                            const int* __restrict__ col, long long e0, long long e1,
                                                            const unsigned* __restrict__ bits,
                                                            unsigned char* __restrict__ bad, unsigned* any_bad,
                                                            Counters* ctr) {
  const unsigned long long pol = policy_evict_first();
  const int lane = threadIdx.x & 31;
  const long long nnz = e1;   // the checked range ends here (a row boundary)
  long long head = e0 + ((long long)((16 - ((unsigned long long)(col + e0) & 15)) & 15) >> 2);   // 4-byte aligned
  if (head > nnz) head = nnz;
  const long long nq = (nnz - head) >> 2;
  const long long tail0 = head + 4 * nq;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid == 0) {
    for (long long e = e0; e < head; ++e)
      check_pair(off, n, nnz, bits, bad, any_bad, ctr, e, col[e], e + 1 < nnz ? col[e + 1] : 0);
    for (long long e = tail0; e < nnz; ++e)
      check_pair(off, n, nnz, bits, bad, any_bad, ctr, e, col[e], e + 1 < nnz ? col[e + 1] : 0);
  }
  const int4* cq = reinterpret_cast<const int4*>(col + head);
  const long long warp = tid >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long qb = warp * 128; qb < nq; qb += nwarps * 128) {   // warp-uniform; 128 quads per round
    int4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long q = qb + u * 32 + lane;
      v[u] = q < nq ? ld_stream4(cq + q, pol) : make_int4(0, 0, 0, 0);
    }
    const long long elast = head + 4 * (qb + 128);   // the entry after the round's last quad
    const int tailx = (lane == 31 && qb + 128 <= nq && elast < nnz) ? ld_stream(col + elast, pol) : 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int nx = __shfl_down_sync(FULL, v[u].x, 1);
      const int hx = u < 3 ? __shfl_sync(FULL, v[u < 3 ? u + 1 : u].x, 0) : tailx;
      if (lane == 31) nx = hx;
      const long long q = qb + u * 32 + lane;
      if (q < nq) {
        const long long e = head + 4 * q;
        if (q + 1 >= nq) nx = e + 4 < nnz ? col[e + 4] : 0;   // the next entry lies in the scalar tail
        const unsigned mx = max(max((unsigned)v[u].x, (unsigned)v[u].y), max((unsigned)v[u].z, (unsigned)v[u].w));
        if (mx >= (unsigned)n) raise_err(&ctr->err, ERRBIT_INVALID);
        // four increasing pairs need no row bounds: only a quad with a
        // descent (a row start, or a row out of order) is checked pair by pair
        if (!(v[u].x < v[u].y && v[u].y < v[u].z && v[u].z < v[u].w && (v[u].w < nx || e + 4 >= nnz))) {
          check_order(off, n, nnz, bits, bad, any_bad, e, v[u].x, v[u].y);
          check_order(off, n, nnz, bits, bad, any_bad, e + 1, v[u].y, v[u].z);
          check_order(off, n, nnz, bits, bad, any_bad, e + 2, v[u].z, v[u].w);
          check_order(off, n, nnz, bits, bad, any_bad, e + 3, v[u].w, nx);
        }
      }
    }
  }
}

__global__ void ident_first_kernel(const long long* __restrict__ off, long long n, const int* __restrict__ col,
                                   const unsigned char* __restrict__ bad, int* __restrict__ next, Counters* ctr) {
  unsigned long long my_dn = 0, my_scan = 0, my_act = 0;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    const long long st = off[v], d = off[v + 1] - st;
    if (d == 0 || bad[v]) continue;   // an empty row keeps its label, already in `next`
    my_act += 1;
    int nl = col[st];
    if (nl == (int)v) nl = d > 1 ? col[st + 1] : (int)v;
    if ((unsigned)nl >= (unsigned)n) nl = (int)v;   // out of range: reported by the check pass
    next[v] = nl;
    my_dn += nl != (int)v ? 1ull : 0ull;
    my_scan += (unsigned long long)d;
  }
  my_dn = warp_sum_u64(my_dn);
  my_scan = warp_sum_u64(my_scan);
  my_act = warp_sum_u64(my_act);
  if ((threadIdx.x & 31) == 0) {
    if (my_dn) atomicAdd(&ctr->dn, my_dn);
    if (my_scan) atomicAdd(&ctr->scanned, my_scan);
    if (my_act) atomicAdd(&ctr->fast_active, my_act);
  }
}

namespace {
// One wave of 256-thread blocks of `kernel`: as many as are resident at once
// (the streaming passes of sweep 1 use more registers than eight blocks per
// SM allow, and a second wave would run at part of the bandwidth).
template <typename K>
int one_wave_grid(K kernel, const DeviceInfo& di) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 0;
  }
  return (per_sm < 1 ? 1 : per_sm) * di.sm_count;
}
}  // namespace

cudaError_t launch_row_check(const long long* off, long long n, const int* col, long long nnz, unsigned* bits,
                             unsigned char* bad, Counters* ctr, const DeviceInfo& di, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int g = 8 * di.sm_count;
  thread_local int gc = 0;
  if (!gc) gc = one_wave_grid(sorted_check_kernel, di);
  cudaMemsetAsync(bits, 0, sizeof(unsigned) * (size_t)((nnz >> 5) + 1), s);
  rowstart_kernel<<<g, 256, 0, s>>>(off, n, bits);
  if (nnz > 0) sorted_check_kernel<<<gc, 256, 0, s>>>(off, n, col, 0, nnz, bits, bad, nullptr, ctr);
  count_launches(nnz > 0 ? 2 : 1);
  return cudaGetLastError();
}

cudaError_t launch_ident_stream(const long long* off, long long n, const int* col, long long nnz, unsigned* bits,
                                unsigned char* bad, int* next, Counters* ctr, const DeviceInfo& di, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (cudaError_t e = launch_row_check(off, n, col, nnz, bits, bad, ctr, di, s)) return e;
  thread_local int gi = 0;
  if (!gi) gi = one_wave_grid(ident_first_kernel, di);
  ident_first_kernel<<<gi, 256, 0, s>>>(off, n, col, bad, next, ctr);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pieces of the first two sweeps while the columns are still arriving
// (gsl_gsllpa_host): the rows are cut into chunks at row boundaries, and a
// chunk's columns are checked and its rows swept as soon as it has landed.

// All-active binning of the rows [v0, v1) (sweep 2 runs on every vertex):
// appended to their class regions as bin_kernel does.
__global__ void __launch_bounds__(256) bin_range_kernel(const long long* __restrict__ off, long long v0, long long v1,
                                                         ClassBounds cb, int* __restrict__ work, Counters* ctr) {
  __shared__ unsigned cnt[NCLASS];
  __shared__ unsigned base[NCLASS];
  const long long tile = (long long)blockDim.x * BIN_ITEMS;
  for (long long t0 = v0 + (long long)blockIdx.x * tile; t0 < v1; t0 += (long long)gridDim.x * tile) {
    if (threadIdx.x < NCLASS) cnt[threadIdx.x] = 0;
    __syncthreads();
    int cls[BIN_ITEMS];
    unsigned pos[BIN_ITEMS];
#pragma unroll
    for (int k = 0; k < BIN_ITEMS; ++k) {
      const long long v = t0 + (long long)k * blockDim.x + threadIdx.x;
      cls[k] = v < v1 ? degree_class(off[v + 1] - off[v], cb.warp_small, cb.warp_max, cb.blk_max) : -1;
      const unsigned m = __match_any_sync(FULL, cls[k]);
      const int leader = __ffs(m) - 1;
      unsigned b = 0;
      if ((int)(threadIdx.x & 31) == leader && cls[k] >= 0) b = atomicAdd(&cnt[cls[k]], (unsigned)__popc(m));
      pos[k] = __shfl_sync(FULL, b, leader) + (unsigned)__popc(m & lanemask_lt());
    }
    __syncthreads();
    if (threadIdx.x < NCLASS) base[threadIdx.x] = cnt[threadIdx.x] ? atomicAdd(&ctr->cls_count[threadIdx.x], cnt[threadIdx.x]) : 0u;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BIN_ITEMS; ++k) {
      if (cls[k] >= 0) {
        const long long v = t0 + (long long)k * blockDim.x + threadIdx.x;
        work[ctr->cls_start[cls[k]] + base[cls[k]] + pos[k]] = (int)v;
      }
    }
    __syncthreads();
  }
}

// Sweep 1 from the identity labelling on rows assumed strictly increasing,
// reading only each row's first entries, from `col` (which may be host
// memory the device can read): the labels and counts ident_first_kernel
// gives when no row is flagged.
cudaError_t launch_ident_first(const long long* off, long long n, const int* col, const unsigned char* zero_flags,
                               int* next, Counters* ctr, const DeviceInfo& di, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ident_first_kernel<<<16 * di.sm_count, 256, 0, s>>>(off, n, col, zero_flags, next, ctr);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_rowstart(const long long* off, long long n, unsigned* bits, long long nbits_words,
                            const DeviceInfo& di, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(unsigned) * (size_t)nbits_words, s)) return e;
  rowstart_kernel<<<8 * di.sm_count, 256, 0, s>>>(off, n, bits);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_chunk_check(const long long* off, long long n, const int* col, long long nnz, long long e0,
                               long long e1, const unsigned* bits, unsigned char* bad, unsigned* any_bad,
                               Counters* ctr, const DeviceInfo& di, cudaStream_t s) {
  (void)nnz;
  if (e1 <= e0) return cudaSuccess;
  thread_local int gc = 0;
  if (!gc) gc = one_wave_grid(sorted_check_kernel, di);
  sorted_check_kernel<<<gc, 256, 0, s>>>(off, n, col, e0, e1, bits, bad, any_bad, ctr);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_bin_range(const long long* off, long long v0, long long v1, const Tuning& t, int* work,
                             Counters* ctr, const DeviceInfo& di, cudaStream_t s) {
  if (v1 <= v0) return cudaSuccess;
  const long long tile = 256ll * BIN_ITEMS;
  long long blocks = (v1 - v0 + tile - 1) / tile;
  const long long cap = 8ll * di.sm_count;
  bin_range_kernel<<<(int)(blocks < cap ? blocks : cap), 256, 0, s>>>(off, v0, v1, class_bounds(t), work, ctr);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// launchers
namespace {
std::atomic<long long> g_launches{0};

template <typename K>
int occupancy_grid(K kernel, int block, size_t smem, const DeviceInfo& di) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
  cudaGetLastError();
  if (per_sm < 1) per_sm = 1;
  return per_sm * di.sm_count;
}

constexpr int TW_SMALL = 512;    // slots per warp, class 6 (2 d <= 512)
constexpr int TW_LARGE = 1024;   // slots per warp, class 7

// One warp per row (classes 6 and 7); the grid is sized once per host
// thread and instantiation from the kernel's occupancy.  With SPILL every
// warp owns one region of the global fallback tables, which are sized for
// warp_grid_warps warps: the grid never exceeds that.
template <bool W, bool A, int TW, bool SPILL, bool SPREAD>
void launch_warp_class(const SweepArgs& a, int cls, const Tuning& t, const DeviceInfo& di, cudaStream_t s) {
  const size_t smem = (size_t)(t.warp_block / 32) * TW * sizeof(unsigned long long);
  thread_local int grid = 0;
  if (!grid) {
    raise_smem_limit((const void*)sweep_warp_kernel<W, A, TW, SPILL, SPREAD>, smem);
    grid = occupancy_grid(sweep_warp_kernel<W, A, TW, SPILL, SPREAD>, t.warp_block, smem, di);
    if (SPILL) {
      const long long cap = warp_grid_warps(t, di) / (t.warp_block / 32);
      if (grid > cap) grid = (int)(cap > 0 ? cap : 1);
    }
  }
  sweep_warp_kernel<W, A, TW, SPILL, SPREAD><<<grid, t.warp_block, smem, s>>>(a, cls);
}

template <bool W, bool A>
cudaError_t launch_sweep_t(const SweepArgs& a, int cls, const Tuning& t, const DeviceInfo& di, cudaStream_t s) {
  switch (cls) {
#define GSL_LAUNCH_GROUP(G, CLS)                                                                 \
  case CLS: {                                                                                    \
    thread_local int grid = 0;                                                                   \
    if (!grid) grid = occupancy_grid(sweep_group_kernel<G, W, A>, t.group_block, 0, di);         \
    sweep_group_kernel<G, W, A><<<grid, t.group_block, 0, s>>>(a, CLS);                          \
    break;                                                                                       \
  }
    GSL_LAUNCH_GROUP(1, 0)
    GSL_LAUNCH_GROUP(2, 1)
    GSL_LAUNCH_GROUP(4, 2)
    GSL_LAUNCH_GROUP(8, 3)
    GSL_LAUNCH_GROUP(16, 4)
    GSL_LAUNCH_GROUP(32, 5)
#undef GSL_LAUNCH_GROUP
    case CLS_WARP_S:
      if (!A && a.spread && !a.lg) launch_warp_class<W, A, TW_SMALL, false, true>(a, CLS_WARP_S, t, di, s);
      else launch_warp_class<W, A, TW_SMALL, false, false>(a, CLS_WARP_S, t, di, s);
      break;
    case CLS_WARP_L:
      if (!A && a.spread && !a.lg) launch_warp_class<W, A, TW_LARGE, true, true>(a, CLS_WARP_L, t, di, s);
      else launch_warp_class<W, A, TW_LARGE, true, false>(a, CLS_WARP_L, t, di, s);
      break;
    case CLS_BLOCK:
    case CLS_HUB: {
      const size_t smem = (size_t)t.blk_slots * sizeof(unsigned long long);
      const int grid = (int)block_grid_size(t, di);
      const int gth = cls == CLS_HUB ? a.gthresh : 0;
      if (!A && a.spread && !a.lg) {
        raise_smem_limit((const void*)sweep_block_kernel<W, A, true>, smem);
        sweep_block_kernel<W, A, true><<<grid, t.blk_block, smem, s>>>(a, cls, (unsigned)t.blk_slots, gth);
      } else {
        raise_smem_limit((const void*)sweep_block_kernel<W, A, false>, smem);
        sweep_block_kernel<W, A, false><<<grid, t.blk_block, smem, s>>>(a, cls, (unsigned)t.blk_slots, gth);
      }
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  count_launches(1);
  return cudaGetLastError();
}
}  // namespace

void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

cudaError_t raise_smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> limits;
  std::lock_guard<std::mutex> g(mu);
  size_t& cur = limits[fn];
  if (bytes <= cur) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

long long block_grid_size(const Tuning& t, const DeviceInfo& di) {
  // per host thread: contexts with different block shapes may run on several threads at once
  thread_local long long cached = 0;
  thread_local int cached_slots = 0, cached_block = 0;
  if (cached && cached_slots == t.blk_slots && cached_block == t.blk_block) return cached;
  int per_sm = 0;
  const size_t smem = (size_t)t.blk_slots * sizeof(unsigned long long);
  raise_smem_limit((const void*)sweep_block_kernel<false, false>, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_block_kernel<false, false>, t.blk_block, smem);
  cudaGetLastError();
  if (per_sm < 1) per_sm = 1;
  cached = (long long)per_sm * di.sm_count;
  cached_slots = t.blk_slots;
  cached_block = t.blk_block;
  return cached;
}

long long warp_grid_warps(const Tuning& t, const DeviceInfo& di) {
  int per_sm = 0;
  const size_t smem = (size_t)(t.warp_block / 32) * TW_LARGE * sizeof(unsigned long long);
  raise_smem_limit((const void*)sweep_warp_kernel<false, false, TW_LARGE, true>, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_warp_kernel<false, false, TW_LARGE, true>,
                                                t.warp_block, smem);
  cudaGetLastError();
  if (per_sm < 1) per_sm = 1;
  return (long long)per_sm * di.sm_count * (t.warp_block / 32);
}

ClassBounds class_bounds(const Tuning& t) {
  ClassBounds cb;
  cb.warp_max = t.warp_max;
  cb.warp_small = TW_SMALL / 2 < t.warp_max ? TW_SMALL / 2 : t.warp_max;
  cb.blk_max = t.blk_max;
  return cb;
}

cudaError_t launch_class_histogram(const long long* off, long long n, long long nnz, const Tuning& t, Counters* ctr,
                                   const DeviceInfo& di, cudaStream_t s) {
  if (n > 0) {
    long long blocks = (n + 255) / 256;
    const long long cap = 8ll * di.sm_count;
    class_histogram_kernel<<<(int)(blocks < cap ? blocks : cap), 256, 0, s>>>(off, n, nnz, class_bounds(t), ctr);
  }
  class_starts_kernel<<<1, 1, 0, s>>>(ctr);
  count_launches(n > 0 ? 2 : 1);
  return cudaGetLastError();
}

cudaError_t launch_bin(const long long* off, long long n, unsigned char* fcur, int all_active, const Tuning& t,
                       int* work, Counters* ctr, const DeviceInfo& di, cudaStream_t s, const int* gid,
                       const unsigned char* done, const int* stop, int phase, unsigned seed) {
  if (n <= 0) return cudaSuccess;
  const long long tile = 256ll * BIN_ITEMS;
  long long blocks = (n + tile - 1) / tile;
  const long long cap = (long long)BIN_BLOCKS * di.sm_count;
  const int grid = (int)(blocks < cap ? blocks : cap);
  if (phase >= 0)
    bin_kernel<true><<<grid, 256, 0, s>>>(off, n, fcur, all_active, class_bounds(t), work, ctr, gid, done, stop, phase,
                                          seed);
  else
    bin_kernel<false><<<grid, 256, 0, s>>>(off, n, fcur, all_active, class_bounds(t), work, ctr, gid, done, stop, -1,
                                           0u);
  count_launches(1);
  return cudaGetLastError();
}

// Between the two phases of an asynchronous sweep: the first phase's class
// counts move to phase_cls and the per-phase worklist counters restart.
__global__ void phase_reset_kernel(Counters* ctr, const int* stop) {
  if (stop && *(volatile const int*)stop) return;
  for (int k = 0; k < NCLASS; ++k) {
    ctr->phase_cls[k] += ctr->cls_count[k];
    ctr->cls_count[k] = 0;
    ctr->uns_count[k] = 0;
  }
  ctr->hub_pieces = 0;
  ctr->hub_clusters = 0;
  ctr->hub_clu_next = 0;
}

cudaError_t launch_phase_reset(Counters* ctr, const int* stop, cudaStream_t s) {
  phase_reset_kernel<<<1, 1, 0, s>>>(ctr, stop);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_init_labels(const int* init, int* a, int* b, long long n, Counters* ctr, const DeviceInfo& di,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  const long long cap = 8ll * di.sm_count;
  init_labels_kernel<<<(int)(blocks < cap ? blocks : cap), 256, 0, s>>>(init, a, b, n, ctr);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_sweep_class(const SweepArgs& a, int cls, bool weighted, bool async_mode, const Tuning& t,
                               const DeviceInfo& di, cudaStream_t s) {
  if (weighted)
    return async_mode ? launch_sweep_t<true, true>(a, cls, t, di, s) : launch_sweep_t<true, false>(a, cls, t, di, s);
  return async_mode ? launch_sweep_t<false, true>(a, cls, t, di, s) : launch_sweep_t<false, false>(a, cls, t, di, s);
}

cudaError_t launch_sweep(const SweepArgs& a, bool weighted, bool async_mode, const Tuning& t, const DeviceInfo& di,
                         cudaStream_t s) {
  for (int c = 0; c < NCLASS; ++c)
    if (cudaError_t e = launch_sweep_class(a, c, weighted, async_mode, t, di, s)) return e;
  return cudaSuccess;
}

}  // namespace gsl
