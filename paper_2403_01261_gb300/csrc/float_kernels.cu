// float_kernels.cu -- LPA sweeps and modularity at the paper's precision:
// float32 edge weights, float64 label sums (Section 4.1).
//
// Eq. 2 picks the label with the largest float64 sum, ties to the smallest
// label.  Unlike the int32 path, sums of non-integer weights depend on the
// order of the additions, so labels can differ from a sequential evaluation
// where two sums agree to rounding; when every partial sum is exact in
// float64 (small integers, dyadic fractions) the result is exact.
//   d <= 32   lane groups: equal labels found with __match_any_sync; each
//             lane sums its group's weights in lane order (row order); the
//             argmax is a shuffle reduction over (sum, label);
//   d > 32    one block per row: a table of (label, float64 sum) slots in
//             shared memory (global memory when 2 d exceeds it); labels are
//             merged per 32-entry chunk first; after all adds the table is
//             scanned for the argmax.
#include <cfloat>

#include "sweep_device.cuh"

namespace gsl {

namespace {

constexpr int F_BLOCK = 256;            // threads per block of the table kernel
constexpr unsigned F_TABLE_SLOTS = 8192;  // shared-memory slots per block (12 bytes each)
constexpr int F_BLOCKS_PER_SM = 2;

// (s1, l1) beats (s2, l2): larger sum, then smaller label; label -1 = none.
__device__ __forceinline__ bool fbetter(double s1, int l1, double s2, int l2) {
  if (l1 < 0) return false;
  if (l2 < 0) return true;
  return s1 > s2 || (s1 == s2 && l1 < l2);
}

template <int WIDTH>
__device__ __forceinline__ void fbest_reduce(double& s, int& l) {
#pragma unroll
  for (int o = WIDTH / 2; o >= 1; o >>= 1) {
    const double s2 = __shfl_xor_sync(FULL, s, o, WIDTH);
    const int l2 = __shfl_xor_sync(FULL, l, o, WIDTH);
    if (fbetter(s2, l2, s, l)) {
      s = s2;
      l = l2;
    }
  }
}

// Entry e of a row: neighbour j (-1 past the end or out of range) and its
// float weight; with `check`, a weight that is not finite and positive is
// reported.
__device__ __forceinline__ void load_entry_f(const SweepArgs& a, const int* cp, const float* wp, int d, int e,
                                             const Pol& pol, int& j, float& w) {
  j = -1;
  w = 0.f;
  if (e < d) {
    j = ld_stream(cp + e, pol.stream);
    w = __ldg(wp + e);
    if ((unsigned)j >= (unsigned)a.n || (a.check && !(w > 0.f && w <= FLT_MAX))) {
      raise_err(&a.ctr->err, ERRBIT_INVALID);
      j = -1;
    }
  }
}

// Sum of w over the lanes of mask m in ascending lane order (row order),
// for every lane at once: the loop runs as often as the largest mask has
// bits, one shuffle per step.
__device__ __forceinline__ double group_sum(unsigned m, float w) {
  const int lane = threadIdx.x & 31;
  const int steps = __reduce_max_sync(FULL, (unsigned)__popc(m));
  double sum = 0.0;
  unsigned mm = m;
  for (int t = 0; t < steps; ++t) {
    const int src = mm ? __ffs(mm) - 1 : lane;
    const double x = (double)__shfl_sync(FULL, w, src);
    if (mm) {
      sum += x;
      mm &= mm - 1;
    }
  }
  return sum;
}

// Adds c to label lbl's sum in an open-addressing table of cap slots.
template <bool GLOBAL>
__device__ __forceinline__ void fslot_add(unsigned* keys, double* vals, unsigned cap, unsigned lbl, double c,
                                          int* err, int probe_cap) {
  unsigned h = __umulhi(hash32(lbl), cap);
  for (int p = 0; p < probe_cap; ++p) {
    unsigned k = GLOBAL ? __ldcg(keys + h) : *(volatile unsigned*)(keys + h);
    if (k == EMPTY32) k = atomicCAS(keys + h, EMPTY32, lbl);
    if (k == EMPTY32 || k == lbl) {
      atomicAdd(vals + h, c);
      return;
    }
    if (++h == cap) h = 0;
  }
  raise_err(err, ERRBIT_TIMEOUT);
}

}  // namespace

template <int G, bool ASYNC>
__global__ void __launch_bounds__(256) sweep_f_group_kernel(SweepArgs a, const float* __restrict__ wf, int cls) {
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
  unsigned long long my_dn = 0, my_scan = 0;
  for (long long wb = warp_id * PER_WARP; wb < (long long)cnt; wb += nwarps * PER_WARP) {
    const long long item = wb + lane / G;
    const bool has = item < (long long)cnt;
    int v = 0, d = 0;
    long long s = 0;
    if (has) {
      v = work[item];
      s = a.off[v];
      d = (int)(a.off[v + 1] - s);
    }
    int j;
    float w;
    load_entry_f(a, a.col + s, wf + s, d, gl, pol, j, w);
    const int lbl = entry_label<ASYNC>(a, nullptr, gl, j, v, pol);
    const unsigned m = __match_any_sync(FULL, lbl) & gmask;
    const double sum = group_sum(m, w);   // this lane's label: its group's weights in lane order
    double bs = sum;
    int bl = lbl;
    fbest_reduce<G>(bs, bl);
    bool changed = false;
    if (has && gl == 0) {
      const int old = own_label<ASYNC>(a, v);
      const int nl = bl >= 0 ? bl : old;
      changed = nl != old;
      store_label<ASYNC>(a, v, nl, changed);
      if (changed) count_graph_change(a, v);
      my_scan += (unsigned long long)d;
      my_dn += changed ? 1ull : 0ull;
    }
    if (a.mark) {
      const unsigned chm = __ballot_sync(FULL, changed);
      if ((chm >> gbase) & 1u) {
        if (j >= 0) a.fnext[j] = 1;
        if (!ASYNC && gl == 0) a.fnext[v] = 1;
      }
    }
  }
  flush_counters(a.ctr, cls, my_dn, my_scan);
}

// One block per row of classes 6..9; `tb` table slots in shared memory,
// global regions of 2 * (largest degree) slots per block otherwise.
template <bool ASYNC>
__global__ void __launch_bounds__(F_BLOCK) sweep_f_block_kernel(SweepArgs a, const float* __restrict__ wf, int cls,
                                                               unsigned tb, unsigned* gkeys, double* gvals,
                                                               long long region) {
  extern __shared__ unsigned char smem_f[];
  double* svals = reinterpret_cast<double*>(smem_f);
  unsigned* skeys = reinterpret_cast<unsigned*>(smem_f + sizeof(double) * tb);
  __shared__ double s_bs[F_BLOCK / 32];
  __shared__ int s_bl[F_BLOCK / 32];
  __shared__ int s_changed;
  __shared__ double s_own;
  const unsigned cnt = a.ctr->cls_count[cls];
  const int* __restrict__ work = a.work + a.ctr->cls_start[cls];
  const Pol pol = make_pol();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long my_dn = 0, my_scan = 0;
  for (long long item = blockIdx.x; item < (long long)cnt; item += gridDim.x) {
    const int v = work[item];
    const long long s = a.off[v];
    const int d = (int)(a.off[v + 1] - s);
    const bool global = 2u * (unsigned)d > tb;
    const unsigned cap = 2u * (unsigned)d;
    unsigned* keys = global ? gkeys + (long long)blockIdx.x * region : skeys;
    double* vals = global ? gvals + (long long)blockIdx.x * region : svals;
    for (unsigned k = threadIdx.x; k < cap; k += blockDim.x) {
      keys[k] = EMPTY32;
      vals[k] = 0.0;
    }
    if (threadIdx.x == 0) s_own = 0.0;
    const int old = own_label<ASYNC>(a, v);
    __syncthreads();
    const int* cp = a.col + s;
    const float* wp = wf + s;
    double own_acc = 0.0;   // entries carrying the vertex's own label stay out of the table
    for (int e0 = wid * 32; e0 < d; e0 += blockDim.x) {   // warp-uniform 32-entry chunks
      int j;
      float w;
      load_entry_f(a, cp, wp, d, e0 + lane, pol, j, w);
      int lbl = entry_label<ASYNC>(a, nullptr, e0 + lane, j, v, pol);
      if (lbl == old) {
        own_acc += (double)w;
        lbl = -1;
      }
      if (__ballot_sync(FULL, lbl >= 0) == 0) continue;
      const unsigned m = __match_any_sync(FULL, lbl);
      const double sum = group_sum(m, w);
      if (lbl >= 0 && (m & lanemask_lt()) == 0) {
        if (global) fslot_add<true>(keys, vals, cap, (unsigned)lbl, sum, &a.ctr->err, a.probe_cap);
        else fslot_add<false>(keys, vals, cap, (unsigned)lbl, sum, &a.ctr->err, a.probe_cap);
      }
    }
    for (int o = 16; o; o >>= 1) own_acc += __shfl_xor_sync(FULL, own_acc, o);
    if (lane == 0 && own_acc != 0.0) atomicAdd(&s_own, own_acc);
    if (global) __threadfence_block();
    __syncthreads();
    double bs = -1.0;
    int bl = -1;
    for (unsigned k = threadIdx.x; k < cap; k += blockDim.x) {
      const unsigned key = global ? __ldcg(keys + k) : keys[k];
      if (key == EMPTY32) continue;
      const double val = global ? __ldcg(vals + k) : vals[k];
      if (fbetter(val, (int)key, bs, bl)) {
        bs = val;
        bl = (int)key;
      }
    }
    fbest_reduce<32>(bs, bl);
    if (lane == 0) {
      s_bs[wid] = bs;
      s_bl[wid] = bl;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
        if (fbetter(s_bs[k], s_bl[k], bs, bl)) {
          bs = s_bs[k];
          bl = s_bl[k];
        }
      if (s_own > 0.0 && fbetter(s_own, old, bs, bl)) {
        bs = s_own;
        bl = old;
      }
      const int nl = bl >= 0 ? bl : old;
      const bool changed = nl != old;
      store_label<ASYNC>(a, v, nl, changed);
      if (changed) count_graph_change(a, v);
      my_scan += (unsigned long long)d;
      my_dn += changed ? 1ull : 0ull;
      s_changed = changed;
    }
    __syncthreads();
    if (s_changed && a.mark) {
      for (int e = threadIdx.x; e < d; e += blockDim.x) {
        const int jj = ld_stream(cp + e, pol.stream);
        if ((unsigned)jj < (unsigned)a.n) a.fnext[jj] = 1;
      }
      if (!ASYNC && threadIdx.x == 0) a.fnext[v] = 1;
    }
    __syncthreads();
  }
  flush_counters(a.ctr, cls, my_dn, my_scan);
}

// ------------------------------------------------------- sweep 1, streamed
// From the identity labels a strictly increasing row holds every label once
// (its neighbour's id) with that entry's weight, so Eq. 2 picks the
// neighbour of largest weight, the smallest id among equal weights.  Rows
// the check pass flagged are left for the table kernels.
__device__ __forceinline__ void f_stream_entry(const int* col, const float* wf, long long e, long long v, long long n,
                                               Counters* ctr, double& bw, int& bj) {
  const int j = col[e];
  const float w = wf[e];
  if (!(w > 0.f && w <= FLT_MAX)) raise_err(&ctr->err, ERRBIT_INVALID);
  if (j == (int)v || (unsigned)j >= (unsigned)n) return;
  if (fbetter((double)w, j, bw, bj)) {
    bw = (double)w;
    bj = j;
  }
}

// A warp takes 32 consecutive vertices: each lane scans its own row when it
// has at most 32 entries, then the warp scans the longer rows together.
__global__ void __launch_bounds__(256) ident_max_f_kernel(const long long* __restrict__ off, long long n,
                                                          const int* __restrict__ col, const float* __restrict__ wf,
                                                          const unsigned char* __restrict__ bad,
                                                          int* __restrict__ next, Counters* ctr) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long my_dn = 0, my_scan = 0, my_act = 0;
  for (long long base = warp * 32; base < n; base += nwarps * 32) {   // warp-uniform
    const long long v = base + lane;
    long long st = 0;
    int d = 0;
    bool mine = false;
    if (v < n) {
      st = off[v];
      d = (int)(off[v + 1] - st);
      mine = d > 0 && !bad[v];
    }
    if (mine && d <= 32) {
      double bw = -1.0;
      int bj = -1;
      for (int x = 0; x < d; ++x) f_stream_entry(col, wf, st + x, v, n, ctr, bw, bj);
      const int nl = bj >= 0 ? bj : (int)v;
      next[v] = nl;
      my_dn += nl != (int)v ? 1ull : 0ull;
      my_scan += (unsigned long long)d;
      my_act += 1;
    }
    unsigned longm = __ballot_sync(FULL, mine && d > 32);
    while (longm) {
      const int src = __ffs(longm) - 1;
      longm &= longm - 1;
      const long long vv = __shfl_sync(FULL, v, src);
      const long long sst = __shfl_sync(FULL, st, src);
      const int dd = __shfl_sync(FULL, d, src);
      double bw = -1.0;
      int bj = -1;
      for (int x = lane; x < dd; x += 32) f_stream_entry(col, wf, sst + x, vv, n, ctr, bw, bj);
      fbest_reduce<32>(bw, bj);
      if (lane == src) {
        const int nl = bj >= 0 ? bj : (int)vv;
        next[vv] = nl;
        my_dn += nl != (int)vv ? 1ull : 0ull;
        my_scan += (unsigned long long)dd;
        my_act += 1;
      }
    }
  }
  my_dn = warp_sum_u64(my_dn);
  my_scan = warp_sum_u64(my_scan);
  my_act = warp_sum_u64(my_act);
  if (lane == 0) {
    if (my_dn) atomicAdd(&ctr->dn, my_dn);
    if (my_scan) atomicAdd(&ctr->scanned, my_scan);
    if (my_act) atomicAdd(&ctr->fast_active, my_act);
  }
}

cudaError_t launch_ident_stream_f32(const long long* off, long long n, const int* col, const float* wf,
                                    long long nnz, unsigned* bits, unsigned char* bad, int* next, Counters* ctr,
                                    const DeviceInfo& di, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (cudaError_t e = launch_row_check(off, n, col, nnz, bits, bad, ctr, di, s)) return e;
  ident_max_f_kernel<<<16 * di.sm_count, 256, 0, s>>>(off, n, col, wf, bad, next, ctr);
  count_launches(1);
  return cudaGetLastError();
}

// Class 6 (33..256 entries): one warp per row with its own shared table of
// F_WARP_SLOTS (label, float64 sum) slots; own-label entries are summed
// outside the table; the warp scans its table for the argmax.
constexpr int F_WARP_SLOTS = 512;   // 2 * 256
constexpr int F_WARP_BLOCK = 128;   // 4 warps, 4 * 512 * 12 bytes = 24 KB

template <bool ASYNC>
__global__ void __launch_bounds__(F_WARP_BLOCK) sweep_f_warp_kernel(SweepArgs a, const float* __restrict__ wf,
                                                                   int cls) {
  __shared__ double svals_all[(F_WARP_BLOCK / 32) * F_WARP_SLOTS];
  __shared__ unsigned skeys_all[(F_WARP_BLOCK / 32) * F_WARP_SLOTS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double* vals = svals_all + wid * F_WARP_SLOTS;
  unsigned* keys = skeys_all + wid * F_WARP_SLOTS;
  const unsigned cnt = a.ctr->cls_count[cls];
  const int* __restrict__ work = a.work + a.ctr->cls_start[cls];
  const Pol pol = make_pol();
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long my_dn = 0, my_scan = 0;
  for (long long item = warp; item < (long long)cnt; item += nwarps) {
    const int v = work[item];
    const long long s = a.off[v];
    const int d = (int)(a.off[v + 1] - s);
    const unsigned cap = 2u * (unsigned)d;   // <= F_WARP_SLOTS for this class
    for (unsigned k = lane; k < cap; k += 32) {
      keys[k] = EMPTY32;
      vals[k] = 0.0;
    }
    __syncwarp();
    const int old = own_label<ASYNC>(a, v);
    double own_acc = 0.0;
    for (int e0 = 0; e0 < d; e0 += 32) {
      int j;
      float w;
      load_entry_f(a, a.col + s, wf + s, d, e0 + lane, pol, j, w);
      int lbl = entry_label<ASYNC>(a, nullptr, e0 + lane, j, v, pol);
      if (lbl == old) {
        own_acc += (double)w;
        lbl = -1;
      }
      if (__ballot_sync(FULL, lbl >= 0) == 0) continue;
      const unsigned m = __match_any_sync(FULL, lbl);
      const double sum = group_sum(m, w);
      if (lbl >= 0 && (m & lanemask_lt()) == 0) fslot_add<false>(keys, vals, cap, (unsigned)lbl, sum, &a.ctr->err, a.probe_cap);
    }
    __syncwarp();
    double bs = -1.0;
    int bl = -1;
    for (unsigned k = lane; k < cap; k += 32) {
      const unsigned key = keys[k];
      if (key != EMPTY32 && fbetter(vals[k], (int)key, bs, bl)) {
        bs = vals[k];
        bl = (int)key;
      }
    }
    for (int o = 16; o; o >>= 1) own_acc += __shfl_xor_sync(FULL, own_acc, o);
    if (own_acc > 0.0 && fbetter(own_acc, old, bs, bl)) {   // the same on every lane
      bs = own_acc;
      bl = old;
    }
    fbest_reduce<32>(bs, bl);
    const int nl = bl >= 0 ? bl : old;
    const bool changed = nl != old;
    if (lane == 0) {
      store_label<ASYNC>(a, v, nl, changed);
      if (changed) count_graph_change(a, v);
      my_scan += (unsigned long long)d;
      my_dn += changed ? 1ull : 0ull;
    }
    if (changed && a.mark) {
      for (int x = lane; x < d; x += 32) {
        const int jj = ld_stream(a.col + s + x, pol.stream);
        if ((unsigned)jj < (unsigned)a.n) a.fnext[jj] = 1;
      }
      if (!ASYNC && lane == 0) a.fnext[v] = 1;
    }
    __syncwarp();
  }
  flush_counters(a.ctr, cls, my_dn, my_scan);
}

// ------------------------------------------------------------- Eq. 1, f64
// Per vertex K_i (float64 sum of its row), S1 += weights of its entries in
// its own community, Sigma[C_i] += K_i; then S2 = sum Sigma_c^2.
__global__ void __launch_bounds__(256) mod_f_rows_kernel(const long long* __restrict__ off, const int* __restrict__ col,
                                                         const float* __restrict__ wf, const int* __restrict__ labels,
                                                         long long n, double* __restrict__ sigma, double* sums,
                                                         Counters* ctr) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  double tk = 0.0, ts1 = 0.0;
  for (long long u = warp; u < n; u += nwarps) {
    const int cu = labels[u];
    if ((unsigned)cu >= (unsigned)n) {
      if (lane == 0) raise_err(&ctr->err, ERRBIT_INVALID);
      continue;
    }
    double k = 0.0;
    for (long long x = off[u] + lane; x < off[u + 1]; x += 32) {
      const int j = col[x];
      const float w = wf[x];
      if ((unsigned)j >= (unsigned)n || !(w > 0.f && w <= FLT_MAX)) {
        raise_err(&ctr->err, ERRBIT_INVALID);
        continue;
      }
      k += (double)w;
      if (labels[j] == cu) ts1 += (double)w;
    }
    for (int o = 16; o; o >>= 1) k += __shfl_xor_sync(FULL, k, o);
    if (lane == 0 && k != 0.0) atomicAdd(sigma + cu, k);
    tk += lane == 0 ? k : 0.0;
  }
  for (int o = 16; o; o >>= 1) {
    tk += __shfl_xor_sync(FULL, tk, o);
    ts1 += __shfl_xor_sync(FULL, ts1, o);
  }
  if (lane == 0) {
    if (tk != 0.0) atomicAdd(sums, tk);
    if (ts1 != 0.0) atomicAdd(sums + 1, ts1);
  }
}

__global__ void __launch_bounds__(256) mod_f_square_kernel(const double* __restrict__ sigma, long long n, double* sums) {
  double acc = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
    acc += sigma[c] * sigma[c];
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(sums + 2, acc);
}

// Own-label majority filter with float weights for classes 7 and 8, as the
// integer filter (lpa_kernels.cu): one warp per row sums, in float64, the
// weights of the entries carrying the vertex's own label and of all entries
// (the vertex itself excluded); a strict majority keeps the label (Eq. 2's
// argmax), other rows go to `out` for the table kernel.  Four 32-entry
// chunks are loaded before they are summed.
template <bool ASYNC>
__global__ void __launch_bounds__(256) majority_filter_f_kernel(SweepArgs a, const float* __restrict__ wf,
                                                                int* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const Pol pol = make_pol();
  const long long c7 = a.ctr->cls_count[CLS_WARP_L];
  const long long total = c7 + a.ctr->cls_count[CLS_BLOCK];
  unsigned long long my_scan = 0, my_settled = 0;
  for (long long i = warp; i < total; i += nwarps) {
    const int cls = i < c7 ? CLS_WARP_L : CLS_BLOCK;
    const long long start = a.ctr->cls_start[cls];
    const int v = a.work[start + (i < c7 ? i : i - c7)];
    const long long s = a.off[v];
    const int d = (int)(a.off[v + 1] - s);
    const int old = own_label<ASYNC>(a, v);
    double ow = 0.0, tw = 0.0;
    for (int e0 = 0; e0 < d; e0 += 128) {
      int j[4];
      float w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) load_entry_f(a, a.col + s, wf + s, d, e0 + 32 * u + lane, pol, j[u], w[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int l = entry_label<ASYNC>(a, nullptr, e0 + 32 * u + lane, j[u], v, pol);
        if (l >= 0) {
          tw += (double)w[u];
          if (l == old) ow += (double)w[u];
        }
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      ow += __shfl_xor_sync(FULL, ow, o);
      tw += __shfl_xor_sync(FULL, tw, o);
    }
    if (lane == 0) {
      if (2.0 * ow > tw) {
        store_label<ASYNC>(a, v, old, false);
        my_scan += (unsigned long long)d;
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

// ---------------------------------------------------------------- launchers
namespace {
template <bool A>
cudaError_t launch_f_t(const SweepArgs& a, const float* wf, int cls, unsigned* gkeys, double* gvals,
                       long long region, const DeviceInfo& di, cudaStream_t s) {
  const int grid = 8 * di.sm_count;
  switch (cls) {
    case 0: sweep_f_group_kernel<1, A><<<grid, 256, 0, s>>>(a, wf, cls); break;
    case 1: sweep_f_group_kernel<2, A><<<grid, 256, 0, s>>>(a, wf, cls); break;
    case 2: sweep_f_group_kernel<4, A><<<grid, 256, 0, s>>>(a, wf, cls); break;
    case 3: sweep_f_group_kernel<8, A><<<grid, 256, 0, s>>>(a, wf, cls); break;
    case 4: sweep_f_group_kernel<16, A><<<grid, 256, 0, s>>>(a, wf, cls); break;
    case 5: sweep_f_group_kernel<32, A><<<grid, 256, 0, s>>>(a, wf, cls); break;
    case 6:   // d <= warp_small <= 256: 2 d slots always fit a warp's table
      sweep_f_warp_kernel<A><<<4 * grid, F_WARP_BLOCK, 0, s>>>(a, wf, cls);
      break;
    default: {
      const unsigned tb = F_TABLE_SLOTS;
      const size_t smem = (size_t)tb * (sizeof(double) + sizeof(unsigned));
      raise_smem_limit((const void*)sweep_f_block_kernel<A>, smem);
      sweep_f_block_kernel<A><<<F_BLOCKS_PER_SM * di.sm_count, F_BLOCK, smem, s>>>(a, wf, cls, tb, gkeys, gvals,
                                                                                   region);
    }
  }
  count_launches(1);
  return cudaGetLastError();
}
}  // namespace

long long float_table_blocks(const DeviceInfo& di) { return (long long)F_BLOCKS_PER_SM * di.sm_count; }

cudaError_t launch_majority_filter_f32(const SweepArgs& a, const float* wf, int* out, bool async_mode,
                                       const DeviceInfo& di, cudaStream_t s) {
  const int grid = 16 * di.sm_count;
  if (async_mode) majority_filter_f_kernel<true><<<grid, 256, 0, s>>>(a, wf, out);
  else majority_filter_f_kernel<false><<<grid, 256, 0, s>>>(a, wf, out);
  count_launches(1);
  if (cudaError_t e = cudaGetLastError()) return e;
  return launch_filter_counts(a.ctr, a.stop, s);
}

cudaError_t launch_sweep_f32(const SweepArgs& a, const float* wf, int cls, bool async_mode, unsigned* gkeys,
                             double* gvals, long long region, const DeviceInfo& di, cudaStream_t s) {
  return async_mode ? launch_f_t<true>(a, wf, cls, gkeys, gvals, region, di, s)
                    : launch_f_t<false>(a, wf, cls, gkeys, gvals, region, di, s);
}

cudaError_t launch_modularity_f32(const long long* off, const int* col, const float* wf, const int* labels,
                                  long long n, double* sigma, double* sums, Counters* ctr, const DeviceInfo& di,
                                  cudaStream_t s) {
  cudaMemsetAsync(sigma, 0, sizeof(double) * (size_t)n, s);
  cudaMemsetAsync(sums, 0, sizeof(double) * 3, s);
  mod_f_rows_kernel<<<16 * di.sm_count, 256, 0, s>>>(off, col, wf, labels, n, sigma, sums, ctr);
  mod_f_square_kernel<<<8 * di.sm_count, 256, 0, s>>>(sigma, n, sums);
  count_launches(2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exact fixed-point form of float32 weights.  A finite positive float32 is
// m * 2^q with an integer m < 2^24; if every weight of the graph is a
// multiple of 2^-S (S = -min q) and every row's total times 2^S stays below
// 2^31, then w * 2^S are int32 values whose integer row sums are exact, and
// so are the float64 sums of the float path (every partial sum is a
// multiple of 2^-S below 2^31-S, well inside float64's 53 bits).  Both
// paths then compare the same numbers scaled by 2^S, so the integer sweeps
// give the float path's labels.
//
// out[0] = 1024 + min over weights of q (exponent of the lowest set bit),
// out[1] = 1024 + max over weights of the exponent of the highest set bit,
// out[2] = 1 if a weight is not finite and positive or is subnormal.
__global__ void __launch_bounds__(256) f32_exact_scan_kernel(const float* __restrict__ w, long long nnz,
                                                             int* __restrict__ out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  int lo = 1 << 30, hi = -(1 << 30), bad = 0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
    const unsigned b = __float_as_uint(__ldcs(w + e));
    const unsigned ex = (b >> 23) & 0xFFu;
    if ((b >> 31) || ex == 0 || ex == 0xFFu) {   // negative, zero, subnormal, inf or nan
      bad = 1;
      continue;
    }
    const unsigned m = (b & 0x7FFFFFu) | 0x800000u;
    const int q = (int)ex - 150 + (__ffs(m) - 1);
    lo = q < lo ? q : lo;
    hi = (int)ex - 127 > hi ? (int)ex - 127 : hi;
  }
  lo = __reduce_min_sync(FULL, lo);
  hi = __reduce_max_sync(FULL, hi);
  bad = __reduce_or_sync(FULL, (unsigned)bad);
  if ((threadIdx.x & 31) == 0) {
    if (lo != (1 << 30)) atomicMin(out, 1024 + lo);
    if (hi != -(1 << 30)) atomicMax(out + 1, 1024 + hi);
    if (bad) atomicOr(out + 2, 1);
  }
}

__global__ void __launch_bounds__(256) f32_to_fixed_kernel(const float* __restrict__ w, long long nnz, int shift,
                                                           int* __restrict__ wi) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const float scale = __int_as_float((127 + shift) << 23);   // 2^shift: the products are exact
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride)
    __stcs(wi + e, (int)(__ldcs(w + e) * scale));
}

cudaError_t launch_f32_exact_scan(const float* w, long long nnz, int* out, const DeviceInfo& di, cudaStream_t s) {
  cudaMemsetAsync(out, 0x7F, sizeof(int), s);           // a large minimum to start from
  cudaMemsetAsync(out + 1, 0, 2 * sizeof(int), s);
  f32_exact_scan_kernel<<<8 * di.sm_count, 256, 0, s>>>(w, nnz, out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_f32_to_fixed(const float* w, long long nnz, int shift, int* wi, const DeviceInfo& di,
                                cudaStream_t s) {
  f32_to_fixed_kernel<<<8 * di.sm_count, 256, 0, s>>>(w, nnz, shift, wi);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace gsl
