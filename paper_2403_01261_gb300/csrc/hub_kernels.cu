// hub_kernels.cu -- the sweep for hub vertices (class 9), split into pieces.
//
// One block per hub would leave the largest rows (a million entries and
// more on R-MAT scale 25) to a single SM at the end of the launch.  Here a
// hub's row is cut into pieces of HUB_PIECE entries, and any block may take
// any piece:
//   1. hub_plan_kernel (one block): numbers the pieces of the frontier's
//      hubs (prefix sums) and places every hub's global table region
//      (2 d slots) and used-slot list (d entries);
//   2. hub_piece_kernel: a block aggregates one piece in a shared-memory
//      table (a piece has at most HUB_PIECE < 3/4 of the table's slots
//      distinct labels, so it never overflows), then adds each of its
//      (label, sum) pairs to the hub's global table.  Every add returns the
//      label's new total, so the largest packed key (sum << 32 | ~label)
//      over all adds of all pieces is the hub's argmax with smallest-label
//      ties -- the same argument as within one block; it is combined with
//      one atomicMax per piece.  Entries carrying the hub's own label are
//      counted separately and added once per piece;
//   3. hub_final_kernel: per hub, the own-label key is compared with the
//      best key, the label written and counted, the table slots the pieces
//      claimed are reset (the tables stay empty between sweeps), and the
//      neighbours of a changed hub are marked.
#include "sweep_device.cuh"

namespace gsl {

namespace {

constexpr int HUB_PIECE = 8192;   // entries per piece (distinct labels <= 8192 < 3/4 of 12288 slots)

// Global-table insert that records every slot it claims in `used`.
__device__ __forceinline__ unsigned hub_slot_add(unsigned long long* tab, unsigned cap, unsigned lbl, unsigned c,
                                                 unsigned* used, unsigned* used_cnt, long long tab_base, int* err) {
  unsigned h = __umulhi(hash32(lbl), cap);
  const unsigned long long mine = ((unsigned long long)lbl << 32) | c;
  for (int p = 0; p < PROBE_CAP; ++p) {
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

__global__ void __launch_bounds__(1024) hub_plan_kernel(SweepArgs a, HubPlan hp) {
  const unsigned cnt = a.ctr->cls_count[CLS_HUB];
  const int* __restrict__ work = a.work + a.ctr->cls_start[CLS_HUB];
  __shared__ long long s_pieces[1024], s_entries[1024];
  __shared__ long long base_p, base_e;
  if (threadIdx.x == 0) {
    base_p = 0;
    base_e = 0;
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
    s_pieces[threadIdx.x] = (d + HUB_PIECE - 1) / HUB_PIECE;
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
  if (threadIdx.x == 0) {
    hp.piece_start[0] = 0;
    hp.ustart[0] = 0;
    a.ctr->hub_pieces = (unsigned)base_p;
  }
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
                                        2 * hp.ustart[i], &a.ctr->err);
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
template <bool W, bool A>
cudaError_t launch_hub_t(const SweepArgs& a, const HubPlan& hp, const Tuning& t, const DeviceInfo& di,
                         cudaStream_t s) {
  const size_t smem = (size_t)t.blk_slots * sizeof(unsigned long long);
  static size_t attr_smem = 0;
  if (attr_smem != smem) {
    cudaFuncSetAttribute(hub_piece_kernel<W, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_smem = smem;
  }
  hub_plan_kernel<<<1, 1024, 0, s>>>(a, hp);
  hub_piece_kernel<W, A><<<(int)block_grid_size(t, di), t.blk_block, smem, s>>>(a, hp, (unsigned)t.blk_slots);
  hub_final_kernel<A><<<2 * di.sm_count, 256, 0, s>>>(a, hp, W ? 1 : 0);
  count_launches(3);
  return cudaGetLastError();
}
}  // namespace

bool hub_pieces_fit(const Tuning& t) { return HUB_PIECE * 4 <= t.blk_slots * 3 - 4 * 512; }

cudaError_t launch_hub_pieces(const SweepArgs& a, const HubPlan& hp, bool weighted, bool async_mode, const Tuning& t,
                              const DeviceInfo& di, cudaStream_t s) {
  if (weighted)
    return async_mode ? launch_hub_t<true, true>(a, hp, t, di, s) : launch_hub_t<true, false>(a, hp, t, di, s);
  return async_mode ? launch_hub_t<false, true>(a, hp, t, di, s) : launch_hub_t<false, false>(a, hp, t, di, s);
}

}  // namespace gsl
