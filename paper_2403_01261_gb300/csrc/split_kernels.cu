// split_kernels.cu -- split last (Algorithm 2) and label renumbering on sm_103a.
//
// Algorithm 2 labels every connected piece of every community with the
// vertex its BFS started from; scanning start vertices in ascending order
// makes that the smallest vertex of the piece.  Here the pieces are found
// as the connected components of the subgraph of edges (u, j) with
// C[u] == C[j], by lock-free union-find instead of one BFS per piece:
//   - parent[v] <= v at all times; a union links the larger of two roots
//     below the smaller with atomicCAS, so the root of every tree is the
//     smallest vertex of its component -- Algorithm 2's label;
//   - find follows parents with path halving (benign racy stores: every
//     value written is an ancestor of the vertex);
//   - edges are offered in two phases (neighbour sampling after Sutton,
//     Ben-Nun and Bar-Noy, "Optimizing Parallel Graph Connectivity
//     Computation via Subgraph Sampling", IPDPS 2018): first every vertex
//     links with its first SPLIT_SAMPLE row entries of its own community;
//     after flattening, every community names one of its pieces (the root
//     one of its vertices holds, the last write winning; the community of
//     the most frequent root among sampled vertices names that root), and
//     only vertices outside their community's named piece offer their
//     remaining entries.  An edge inside a named piece is redundant, and an
//     edge between a named piece and another piece of the same community is
//     offered from the other end, so the components are the same as
//     offering every edge.  Communities are mapped to a table of n slots
//     (label c in [0, n) to slot c, others by a hash); a slot shared by two
//     communities names a piece of one of them, and the other's vertices
//     then all offer their entries, which is slower but still exact.
// All loops are bounded (parents strictly decrease along a path and a
// failed CAS strictly lowers the root being linked); the bound is a safety
// net that raises ERRBIT_TIMEOUT.
#include "kernels.h"

namespace gsl {

namespace {

// Bound of the union-find loops.  The default is a compile-time constant
// (the loops are measurably faster that way); kernels instantiated with
// UfCap<0> take a bound lowered at run time (gsl_ctx_set_retry_bounds).
constexpr int UF_CAP = 1 << 26;
template <int FIXED>
struct UfCap {
  int runtime;
  __device__ __forceinline__ int get() const { return FIXED > 0 ? FIXED : runtime; }
};

template <int F>
__device__ __forceinline__ int uf_find(int* p, int x, int* err, UfCap<F> cap) {
  const int bound = cap.get();
  for (int it = 0; it < bound; ++it) {
    const int px = __ldcg(p + x);
    if (px == x) return x;
    const int ppx = __ldcg(p + px);
    if (ppx != px) __stcg(p + x, ppx);
    x = ppx;
  }
  raise_err(err, ERRBIT_TIMEOUT);
  return x;
}

template <int F>
__device__ __forceinline__ void uf_unite(int* p, int a, int b, int* err, UfCap<F> cap) {
  const int bound = cap.get();
  for (int it = 0; it < bound; ++it) {
    a = uf_find(p, a, err, cap);
    b = uf_find(p, b, err, cap);
    if (a == b) return;
    const int hi = a > b ? a : b, lo = a > b ? b : a;
    const int old = atomicCAS(p + hi, hi, lo);
    if (old == hi) return;
    a = old;   // hi got a parent meanwhile: continue from it
    b = lo;
  }
  raise_err(err, ERRBIT_TIMEOUT);
}

// Slot of community label c in a table of n entries.
__device__ __forceinline__ long long comm_slot(int c, long long n) {
  if (c >= 0 && (long long)c < n) return c;
  unsigned x = (unsigned)c;
  x ^= x >> 16;
  x *= 0x7FEB352Du;
  x ^= x >> 15;
  x *= 0x846CA68Bu;
  x ^= x >> 16;
  return (long long)(((unsigned long long)x * (unsigned long long)n) >> 32);
}

constexpr int SPLIT_SAMPLE = 2;   // same-community links per vertex before the named pieces are known
constexpr int SPLIT_SCAN = 8;     // row entries the sampling pass looks at for them

// Offers entry e of u's row to the union-find if it is an intra-community
// edge; returns whether it was one.
template <int F>
__device__ __forceinline__ bool hook_entry(const int* col, const int* labels, int* p, long long n, int u, int cu,
                                           long long e, int* err, UfCap<F> cap) {
  const int j = ld_stream(col + e);
  if ((unsigned)j >= (unsigned)n) {
    raise_err(err, ERRBIT_INVALID);
    return false;
  }
  if (j == u || ld_label_ro(labels + j) != cu) return false;
  uf_unite(p, u, j, err, cap);
  return true;
}

// The same after flattening, with ru = u's parent read once per row: when
// j's parent is ru, u and j already share a tree (trees only merge), so the
// union is skipped without walking either path.
template <int F>
__device__ __forceinline__ void hook_entry_flat(const int* col, const int* labels, int* p, long long n, int u,
                                                int cu, int ru, long long e, int* err, UfCap<F> cap) {
  const int j = ld_stream(col + e);
  if ((unsigned)j >= (unsigned)n) {
    raise_err(err, ERRBIT_INVALID);
    return;
  }
  if (j == u || ld_label_ro(labels + j) != cu) return;
  if (__ldcg(p + j) == ru) return;
  uf_unite(p, u, j, err, cap);
}

}  // namespace

__global__ void init_parent_kernel(int* __restrict__ p, long long n) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
    p[v] = (int)v;
}

// Phase 1: every vertex links with the first SPLIT_SAMPLE same-community
// neighbours among its first SPLIT_SCAN row entries.
// The first two entries' columns and labels are requested together; the
// rest of the scan (when they are not both links) goes one entry at a time.
template <int F>
__global__ void sample_link_kernel(const long long* __restrict__ off, const int* __restrict__ col,
                                   const int* __restrict__ labels, int* p, long long n, Counters* ctr, UfCap<F> cap) {
  static_assert(SPLIT_SAMPLE == 2, "the first two entries are loaded together");
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
    const long long s = off[u], e = off[u + 1];
    if (s >= e) continue;
    const int cu = labels[u];
    const int j0 = ld_stream(col + s), j1 = s + 1 < e ? ld_stream(col + s + 1) : -1;
    const bool v0 = (unsigned)j0 < (unsigned)n, v1 = (unsigned)j1 < (unsigned)n;
    if (!v0 || (s + 1 < e && !v1)) raise_err(&ctr->err, ERRBIT_INVALID);
    const int l0 = v0 && j0 != (int)u ? ld_label_ro(labels + j0) : ~cu;
    const int l1 = v1 && j1 != (int)u ? ld_label_ro(labels + j1) : ~cu;
    int linked = 0;
    if (l0 == cu) {
      uf_unite(p, (int)u, j0, &ctr->err, cap);
      ++linked;
    }
    if (l1 == cu) {
      uf_unite(p, (int)u, j1, &ctr->err, cap);
      ++linked;
    }
    for (int k = 2; k < SPLIT_SCAN && linked < SPLIT_SAMPLE && s + k < e; ++k)
      linked += hook_entry(col, labels, p, n, (int)u, cu, s + k, &ctr->err, cap) ? 1 : 0;
  }
}

// Phases 2 and 5: every parent becomes the root.
template <int F>
__global__ void flatten_kernel(int* p, int* out, long long n, Counters* ctr, UfCap<F> cap) {   // out may equal p
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
    out[v] = uf_find(p, (int)v, &ctr->err, cap);
}

// Phase 3: the most frequent root among 1024 sampled vertices (one block
// of 1024 threads: sample, bitonic sort in shared memory, longest run).
__global__ void __launch_bounds__(1024) giant_kernel(const int* p, long long n, Counters* ctr) {
  __shared__ int a[1024];
  const unsigned t = threadIdx.x;
  const unsigned long long x = ((unsigned long long)hash32(t * 2654435761u + 0x9E37u) * (unsigned long long)n) >> 32;
  a[t] = __ldcg(p + x);
  __syncthreads();
  for (unsigned k = 2; k <= 1024; k <<= 1) {
    for (unsigned j = k >> 1; j > 0; j >>= 1) {
      const unsigned q = t ^ j;
      if (q > t) {
        const bool up = (t & k) == 0;
        const int x0 = a[t], x1 = a[q];
        if ((x0 > x1) == up) {
          a[t] = x1;
          a[q] = x0;
        }
      }
      __syncthreads();
    }
  }
  if (t == 0) {
    int best = a[0], best_run = 0, run = 0;
    for (int i = 0; i < 1024; ++i) {
      run = (i > 0 && a[i] == a[i - 1]) ? run + 1 : 1;
      if (run > best_run) {
        best_run = run;
        best = a[i];
      }
    }
    ctr->giant = best;
  }
}

// Phase 3b: every community names a piece: the root its vertices hold
// after flattening, the last write winning; then the community of the most
// frequent sampled root (giant_kernel) names that root.  Every slot read
// later was written by the vertex reading it, so no initial value is needed.
__global__ void name_pieces_kernel(const int* __restrict__ p, const int* __restrict__ labels, long long n,
                                   int* __restrict__ named) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
    named[comm_slot(labels[v], n)] = p[v];
}

__global__ void name_giant_kernel(const int* __restrict__ labels, long long n, int* __restrict__ named,
                                  const Counters* ctr) {
  const int g = ctr->giant;
  if (g >= 0 && (long long)g < n) named[comm_slot(labels[g], n)] = g;
}

// Phase 4, classes 0..7: G lanes per vertex; vertices in their community's
// named piece are skipped, the others offer entries SPLIT_SAMPLE.. of their
// row (both directions: the other end may be skipped).
template <int G, int F>
__global__ void __launch_bounds__(256) hook_group_kernel(const long long* __restrict__ off, const int* __restrict__ col,
                                                          const int* __restrict__ labels, int* p, long long n,
                                                          const int* __restrict__ work, Counters* ctr, int cls,
                                                          UfCap<F> cap, const int* __restrict__ named) {
  const unsigned cnt = (unsigned)ctr->cls_total[cls];
  const int* w = work + ctr->cls_start[cls];
  const int gl = threadIdx.x & (G - 1);
  const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const long long ng = ((long long)gridDim.x * blockDim.x) / G;
  for (long long item = gid; item < (long long)cnt; item += ng) {
    const int u = w[item];
    const long long s = off[u], e = off[u + 1];
    if (e - s <= SPLIT_SAMPLE) continue;
    const int ru = __ldcg(p + u);
    const int cu = labels[u];
    if (ru == named[comm_slot(cu, n)]) continue;
    for (long long k = s + SPLIT_SAMPLE + gl; k < e; k += G) hook_entry_flat(col, labels, p, n, u, cu, ru, k, &ctr->err, cap);
  }
}

// Phase 4, classes 8..9: one block per vertex.
template <int F>
__global__ void __launch_bounds__(512) hook_block_kernel(const long long* __restrict__ off, const int* __restrict__ col,
                                                          const int* __restrict__ labels, int* p, long long n,
                                                          const int* __restrict__ work, Counters* ctr, int cls,
                                                          UfCap<F> cap, const int* __restrict__ named) {
  const unsigned cnt = (unsigned)ctr->cls_total[cls];
  const int* w = work + ctr->cls_start[cls];
  __shared__ int s_root;
  for (long long item = blockIdx.x; item < (long long)cnt; item += gridDim.x) {
    const int u = w[item];
    const long long s = off[u], e = off[u + 1];
    if (threadIdx.x == 0) s_root = __ldcg(p + u);
    __syncthreads();
    const int ru = s_root;
    __syncthreads();
    const int cu = labels[u];
    if (ru == named[comm_slot(cu, n)]) continue;
    for (long long k = s + SPLIT_SAMPLE + threadIdx.x; k < e; k += blockDim.x)
      hook_entry_flat(col, labels, p, n, u, cu, ru, k, &ctr->err, cap);
  }
}

// ---------------------------------------------------------------- renumber
// rank of every representative (out[v] == v) among all representatives,
// then out[v] = rank[out[v]]: pieces numbered 0..k-1 by smallest vertex.
constexpr int RN_THREADS = 256;
constexpr int RN_ITEMS = 8;
constexpr long long RN_TILE = (long long)RN_THREADS * RN_ITEMS;

// Representatives per tile of RN_TILE vertices (thread t of the block takes
// vertices t * RN_ITEMS .. + RN_ITEMS - 1 of the tile, as rn_rank_kernel
// does).  A thread's eight labels are read as two 16-byte loads where the
// array is 16-byte aligned and the eight lie inside it.
__global__ void __launch_bounds__(RN_THREADS) rn_count_kernel(const int* __restrict__ rep, long long n,
                                                               unsigned long long* __restrict__ block_sums) {
  static_assert(RN_ITEMS == 8, "two 16-byte loads per thread");
  __shared__ unsigned acc;
  if (threadIdx.x == 0) acc = 0;
  __syncthreads();
  const long long v0 = (long long)blockIdx.x * RN_TILE + (long long)threadIdx.x * RN_ITEMS;
  unsigned c = 0;
  if ((reinterpret_cast<uintptr_t>(rep) & 15) == 0 && v0 + RN_ITEMS <= n) {
    const int4 x = __ldg(reinterpret_cast<const int4*>(rep + v0));
    const int4 y = __ldg(reinterpret_cast<const int4*>(rep + v0 + 4));
    const int v = (int)v0;
    c = (x.x == v) + (x.y == v + 1) + (x.z == v + 2) + (x.w == v + 3) + (y.x == v + 4) + (y.y == v + 5) +
        (y.z == v + 6) + (y.w == v + 7);
  } else {
    for (int k = 0; k < RN_ITEMS; ++k) {
      const long long v = v0 + k;
      if (v < n && rep[v] == (int)v) ++c;
    }
  }
  c = __reduce_add_sync(FULL, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&acc, c);
  __syncthreads();
  if (threadIdx.x == 0) block_sums[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(1024) rn_scan_kernel(unsigned long long* block_sums, long long nb,
                                                        unsigned long long* total) {
  __shared__ unsigned long long buf[1024];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (long long b0 = 0; b0 < nb; b0 += 1024) {
    const long long b = b0 + threadIdx.x;
    const unsigned long long x = b < nb ? block_sums[b] : 0ull;
    buf[threadIdx.x] = x;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {   // Hillis-Steele inclusive scan
      const unsigned long long y = threadIdx.x >= (unsigned)o ? buf[threadIdx.x - o] : 0ull;
      __syncthreads();
      buf[threadIdx.x] += y;
      __syncthreads();
    }
    if (b < nb) block_sums[b] = carry + buf[threadIdx.x] - x;   // exclusive
    __syncthreads();
    if (threadIdx.x == 0) carry += buf[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(RN_THREADS) rn_rank_kernel(const int* __restrict__ rep, long long n,
                                                              const unsigned long long* __restrict__ block_sums,
                                                              int* __restrict__ rank) {
  __shared__ unsigned warp_tot[RN_THREADS / 32];
  const long long t0 = (long long)blockIdx.x * RN_TILE;
  unsigned flags = 0, c = 0;
  for (int k = 0; k < RN_ITEMS; ++k) {
    const long long v = t0 + (long long)threadIdx.x * RN_ITEMS + k;
    if (v < n && rep[v] == (int)v) { flags |= 1u << k; ++c; }
  }
  // exclusive scan of c over the block
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned incl = c;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  unsigned wbase = 0;
  for (int w = 0; w < wid; ++w) wbase += warp_tot[w];
  unsigned long long r = block_sums[blockIdx.x] + wbase + incl - c;
  for (int k = 0; k < RN_ITEMS; ++k) {
    if (flags >> k & 1u) {
      const long long v = t0 + (long long)threadIdx.x * RN_ITEMS + k;
      rank[v] = (int)r++;
    }
  }
}

__global__ void rn_apply_kernel(const int* __restrict__ rep, int* __restrict__ out, const int* __restrict__ rank,
                                long long n) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
    out[v] = rank[rep[v]];
}

// ------------------------------------------------------------ Algorithm 4
// A community is disconnected when it holds more than one piece.  With the
// pieces from the union-find (every piece labelled by its smallest vertex),
// each piece representative adds one to its community's count; flags are
// the communities with a count of two or more.
__global__ void disc_count_kernel(const int* __restrict__ rep, const int* __restrict__ labels, long long n,
                                  int* __restrict__ cnt, Counters* ctr) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    const int c = labels[v];
    if ((unsigned)c >= (unsigned)n) {
      raise_err(&ctr->err, ERRBIT_INVALID);
      continue;
    }
    if (rep[v] == (int)v) atomicAdd(cnt + c, 1);
  }
}

__global__ void disc_flag_kernel(const int* __restrict__ cnt, long long n, unsigned char* __restrict__ flags,
                                 unsigned long long* total) {
  unsigned long long mine = 0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const bool f = cnt[c] >= 2;
    if (flags) flags[c] = f ? 1 : 0;
    mine += f ? 1ull : 0ull;
  }
  mine = warp_sum_u64(mine);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(total, mine);
}

// ------------------------------------------------------------ Algorithm 1
// One sweep of SL-LP / SL-LPP: every vertex (with pruning: every vertex of
// the current frontier) takes the smallest piece label over itself and its
// neighbours of the same community, in place.  A warp handles a vertex;
// labels only decrease, so concurrent updates converge to the same fixed
// point as the sequential sweep: the smallest vertex id of every piece.
// With pruning, a vertex that changed puts its same-community neighbours in
// the next frontier.
__global__ void __launch_bounds__(256) split_lp_kernel(const long long* __restrict__ off, const int* __restrict__ col,
                                                       const int* __restrict__ labels, long long n, int* cp,
                                                       unsigned char* __restrict__ fcur,
                                                       unsigned char* __restrict__ fnext, int prune, Counters* ctr) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long my_dn = 0;
  for (long long v = warp; v < n; v += nwarps) {
    if (prune) {
      if (!fcur[v]) continue;   // warp-uniform
      __syncwarp();
      if (lane == 0) fcur[v] = 0;
    }
    const long long s = off[v], e = off[v + 1];
    const int c = labels[v];
    const int cur = __ldcg(cp + v);
    int m = cur;
    for (long long x = s + lane; x < e; x += 32) {
      const int j = ld_stream(col + x);
      if ((unsigned)j >= (unsigned)n) {
        raise_err(&ctr->err, ERRBIT_INVALID);
        continue;
      }
      if (ld_label_ro(labels + j) == c) {
        const int pj = __ldcg(cp + j);
        m = pj < m ? pj : m;
      }
    }
    m = __reduce_min_sync(FULL, m);
    if (m < cur) {   // warp-uniform
      if (lane == 0) __stcg(cp + v, m);
      my_dn += lane == 0 ? 1ull : 0ull;
      if (prune) {
        for (long long x = s + lane; x < e; x += 32) {
          const int j = ld_stream(col + x);
          if ((unsigned)j < (unsigned)n && ld_label_ro(labels + j) == c) fnext[j] = 1;
        }
      }
    }
  }
  my_dn = warp_sum_u64(my_dn);
  if (lane == 0 && my_dn) atomicAdd(&ctr->dn, my_dn);
}

__global__ void iota_kernel(int* __restrict__ p, unsigned char* __restrict__ f, long long n) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    p[v] = (int)v;
    if (f) f[v] = 1;
  }
}

// ---------------------------------------------------------------- launchers
namespace {
int grid_for(long long items, int block, const DeviceInfo& di, int per_sm = 8) {
  long long b = (items + block - 1) / block;
  const long long cap = (long long)per_sm * di.sm_count;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}
}  // namespace

template <int F>
void launch_split_t(const long long* off, const int* col, long long n, const int* labels, const int* work,
                    Counters* ctr, int* parent, int* named, int* out, UfCap<F> cap, const DeviceInfo& di,
                    cudaStream_t s) {
  init_parent_kernel<<<grid_for(n, 256, di), 256, 0, s>>>(parent, n);
  sample_link_kernel<F><<<grid_for(n, 256, di), 256, 0, s>>>(off, col, labels, parent, n, ctr, cap);
  flatten_kernel<F><<<grid_for(n, 256, di), 256, 0, s>>>(parent, parent, n, ctr, cap);
  giant_kernel<<<1, 1024, 0, s>>>(parent, n, ctr);
  name_pieces_kernel<<<grid_for(n, 256, di), 256, 0, s>>>(parent, labels, n, named);
  name_giant_kernel<<<1, 1, 0, s>>>(labels, n, named, ctr);
  const int g = 8 * di.sm_count;
  hook_group_kernel<1, F><<<g, 256, 0, s>>>(off, col, labels, parent, n, work, ctr, 0, cap, named);
  hook_group_kernel<2, F><<<g, 256, 0, s>>>(off, col, labels, parent, n, work, ctr, 1, cap, named);
  hook_group_kernel<4, F><<<g, 256, 0, s>>>(off, col, labels, parent, n, work, ctr, 2, cap, named);
  hook_group_kernel<8, F><<<g, 256, 0, s>>>(off, col, labels, parent, n, work, ctr, 3, cap, named);
  hook_group_kernel<16, F><<<g, 256, 0, s>>>(off, col, labels, parent, n, work, ctr, 4, cap, named);
  hook_group_kernel<32, F><<<g, 256, 0, s>>>(off, col, labels, parent, n, work, ctr, 5, cap, named);
  hook_group_kernel<32, F><<<g, 256, 0, s>>>(off, col, labels, parent, n, work, ctr, CLS_WARP_S, cap, named);
  hook_group_kernel<32, F><<<g, 256, 0, s>>>(off, col, labels, parent, n, work, ctr, CLS_WARP_L, cap, named);
  hook_block_kernel<F><<<4 * di.sm_count, 512, 0, s>>>(off, col, labels, parent, n, work, ctr, CLS_BLOCK, cap, named);
  hook_block_kernel<F><<<4 * di.sm_count, 512, 0, s>>>(off, col, labels, parent, n, work, ctr, CLS_HUB, cap, named);
  flatten_kernel<F><<<grid_for(n, 256, di), 256, 0, s>>>(parent, out, n, ctr, cap);
  count_launches(17);
}

cudaError_t launch_split(const long long* off, const int* col, long long n, const int* labels, const int* work,
                         Counters* ctr, int* parent, int* named, int* out, const Tuning& t, const DeviceInfo& di,
                         cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (t.uf_cap == UF_CAP)
    launch_split_t(off, col, n, labels, work, ctr, parent, named, out, UfCap<UF_CAP>{0}, di, s);
  else
    launch_split_t(off, col, n, labels, work, ctr, parent, named, out, UfCap<0>{t.uf_cap}, di, s);
  return cudaGetLastError();
}

cudaError_t launch_disconnected(const int* rep, const int* labels, long long n, int* cnt, unsigned char* flags,
                                unsigned long long* total, Counters* ctr, const DeviceInfo& di, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)n, s);
  cudaMemsetAsync(total, 0, sizeof(unsigned long long), s);
  disc_count_kernel<<<grid_for(n, 256, di), 256, 0, s>>>(rep, labels, n, cnt, ctr);
  disc_flag_kernel<<<grid_for(n, 256, di), 256, 0, s>>>(cnt, n, flags, total);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_split_lp_init(int* cp, unsigned char* f, long long n, const DeviceInfo& di, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  iota_kernel<<<grid_for(n, 256, di), 256, 0, s>>>(cp, f, n);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_split_lp_sweep(const long long* off, const int* col, const int* labels, long long n, int* cp,
                                  unsigned char* fcur, unsigned char* fnext, int prune, Counters* ctr,
                                  const DeviceInfo& di, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  split_lp_kernel<<<16 * di.sm_count, 256, 0, s>>>(off, col, labels, n, cp, fcur, fnext, prune, ctr);
  count_launches(1);
  return cudaGetLastError();
}

long long renumber_blocks(long long n) { return (n + RN_TILE - 1) / RN_TILE; }

cudaError_t launch_renumber(const int* rep, int* out, long long n, int* rank, unsigned long long* block_sums,
                            long long nblocks_cap, unsigned long long* k_dev, const DeviceInfo& di, cudaStream_t s) {
  const long long nb = renumber_blocks(n);
  if (nb > nblocks_cap) return cudaErrorInvalidValue;
  if (n <= 0) {
    cudaMemsetAsync(k_dev, 0, sizeof(unsigned long long), s);
    return cudaGetLastError();
  }
  rn_count_kernel<<<(int)nb, RN_THREADS, 0, s>>>(rep, n, block_sums);
  rn_scan_kernel<<<1, 1024, 0, s>>>(block_sums, nb, k_dev);
  count_launches(2);
  if (!out) return cudaGetLastError();   // count only
  rn_rank_kernel<<<(int)nb, RN_THREADS, 0, s>>>(rep, n, block_sums, rank);
  rn_apply_kernel<<<grid_for(n, 256, di), 256, 0, s>>>(rep, out, rank, n);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace gsl
