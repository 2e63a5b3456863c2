// modularity_kernels.cu -- Eq. 1 on sm_103a with exact integer sums.
//
// Q = sum_c [ sigma_c / 2m - (Sigma_c / 2m)^2 ].  Over a symmetric CSR:
//   2m            = sum of all entry weights (weighted degrees K_i summed),
//   S1            = sum_c sigma_c = weights of entries (i, j) with C_i == C_j,
//   Sigma_c       = sum of K_i over the vertices of c,
//   S2            = sum_c Sigma_c^2 (128-bit).
// Pass 1 (per vertex, by degree class) accumulates K_i into Sigma[C_i] and
// the block sums of 2m and S1; pass 2 squares and sums Sigma in 128 bits;
// the host forms Q once in double.  All sums are integers, so the result is
// independent of summation order.
#include "kernels.h"

namespace gsl {

namespace {

struct U128 {
  unsigned long long lo, hi;
};
__device__ __forceinline__ U128 add128(U128 a, U128 b) {
  U128 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
  return r;
}
__device__ __forceinline__ U128 sq64(unsigned long long x) {
  U128 r;
  r.lo = x * x;
  r.hi = __umul64hi(x, x);
  return r;
}

__device__ __forceinline__ void flush_sums(ModSums* out, unsigned long long k, unsigned long long s1) {
  __shared__ unsigned long long acc[2];
  if (threadIdx.x == 0) { acc[0] = 0; acc[1] = 0; }
  __syncthreads();
  for (int o = 16; o; o >>= 1) {
    k += __shfl_xor_sync(FULL, k, o);
    s1 += __shfl_xor_sync(FULL, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[0], k);
    atomicAdd(&acc[1], s1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (acc[0]) atomicAdd(&out->two_m, acc[0]);
    if (acc[1]) atomicAdd(&out->s1, acc[1]);
  }
}

// One row slice: returns (sum of weights, sum of weights inside C_u).
template <bool WEIGHTED>
__device__ __forceinline__ void mod_entry(const int* col, const int* w, const int* labels, long long n, int cu,
                                          long long e, unsigned long long& k, unsigned long long& s1, int* err) {
  const int j = ld_stream(col + e);
  const unsigned long long we = WEIGHTED ? (unsigned long long)(unsigned)ld_stream(w + e) : 1ull;
  if ((unsigned)j >= (unsigned)n) {
    raise_err(err, ERRBIT_INVALID);
    return;
  }
  k += we;
  if (ld_label_ro(labels + j) == cu) s1 += we;
}

}  // namespace

template <int G, bool WEIGHTED>
__global__ void __launch_bounds__(256) mod_group_kernel(const long long* __restrict__ off, const int* __restrict__ col,
                                                         const int* __restrict__ w, const int* __restrict__ labels,
                                                         long long n, const int* __restrict__ work, Counters* ctr,
                                                         int cls, unsigned long long* sigma, ModSums* out) {
  const unsigned cnt = (unsigned)ctr->cls_total[cls];
  const int* wl = work + ctr->cls_start[cls];
  const int gl = threadIdx.x & (G - 1);
  const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const long long ng = ((long long)gridDim.x * blockDim.x) / G;
  unsigned long long tk = 0, ts1 = 0;
  // the loop trip count differs between groups: no warp collectives inside
  for (long long item = gid; item < (long long)cnt; item += ng) {
    const int u = wl[item];
    const long long s = off[u], e = off[u + 1];
    const int cu = labels[u];
    if ((unsigned)cu >= (unsigned)n) {
      raise_err(&ctr->err, ERRBIT_INVALID);
      continue;
    }
    unsigned long long k = 0;
    for (long long x = s + gl; x < e; x += G) mod_entry<WEIGHTED>(col, w, labels, n, cu, x, k, ts1, &ctr->err);
    tk += k;
    if (k) atomicAdd(sigma + cu, k);
  }
  flush_sums(out, tk, ts1);
}

template <bool WEIGHTED>
__global__ void __launch_bounds__(512) mod_block_kernel(const long long* __restrict__ off, const int* __restrict__ col,
                                                         const int* __restrict__ w, const int* __restrict__ labels,
                                                         long long n, const int* __restrict__ work, Counters* ctr,
                                                         int cls, unsigned long long* sigma, ModSums* out) {
  const unsigned cnt = (unsigned)ctr->cls_total[cls];
  const int* wl = work + ctr->cls_start[cls];
  unsigned long long tk = 0, ts1 = 0;
  for (long long item = blockIdx.x; item < (long long)cnt; item += gridDim.x) {
    const int u = wl[item];
    const long long s = off[u], e = off[u + 1];
    const int cu = labels[u];
    if ((unsigned)cu >= (unsigned)n) {
      if (threadIdx.x == 0) raise_err(&ctr->err, ERRBIT_INVALID);
      continue;
    }
    unsigned long long k = 0;
    for (long long x = s + threadIdx.x; x < e; x += blockDim.x) mod_entry<WEIGHTED>(col, w, labels, n, cu, x, k, ts1, &ctr->err);
    tk += k;
    if (k) atomicAdd(sigma + cu, k);
  }
  flush_sums(out, tk, ts1);
}

// Isolated vertices (degree 0) contribute nothing to 2m, S1 or Sigma; their
// labels still have to be in range.
__global__ void mod_check_labels_kernel(const int* __restrict__ labels, long long n, Counters* ctr) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
    if ((unsigned)labels[v] >= (unsigned)n) raise_err(&ctr->err, ERRBIT_INVALID);
}

__global__ void __launch_bounds__(256) mod_square_kernel(const unsigned long long* __restrict__ sigma, long long n,
                                                          unsigned long long* partials) {
  U128 acc{0, 0};
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
    acc = add128(acc, sq64(sigma[c]));
  __shared__ unsigned long long lo[256], hi[256];
  lo[threadIdx.x] = acc.lo;
  hi[threadIdx.x] = acc.hi;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < (unsigned)o) {
      U128 a{lo[threadIdx.x], hi[threadIdx.x]}, b{lo[threadIdx.x + o], hi[threadIdx.x + o]};
      const U128 r = add128(a, b);
      lo[threadIdx.x] = r.lo;
      hi[threadIdx.x] = r.hi;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = lo[0];
    partials[2 * blockIdx.x + 1] = hi[0];
  }
}

__global__ void mod_final_kernel(const unsigned long long* partials, long long nparts, ModSums* out) {
  if (threadIdx.x != 0) return;
  U128 acc{0, 0};
  for (long long b = 0; b < nparts; ++b) acc = add128(acc, U128{partials[2 * b], partials[2 * b + 1]});
  out->s2_lo = acc.lo;
  out->s2_hi = acc.hi;
}

long long modularity_partials(const DeviceInfo& di) { return 4ll * di.sm_count; }

cudaError_t launch_modularity(const long long* off, const int* col, const int* w, long long n, const int* labels,
                              const int* work, Counters* ctr, unsigned long long* sigma, unsigned long long* partials,
                              long long nparts, ModSums* out, const Tuning& t, const DeviceInfo& di, cudaStream_t s) {
  (void)t;
  if (n <= 0) return cudaSuccess;
  const int g = 8 * di.sm_count;
  mod_check_labels_kernel<<<g, 256, 0, s>>>(labels, n, ctr);
  if (w) {
    mod_group_kernel<1, true><<<g, 256, 0, s>>>(off, col, w, labels, n, work, ctr, 0, sigma, out);
    mod_group_kernel<2, true><<<g, 256, 0, s>>>(off, col, w, labels, n, work, ctr, 1, sigma, out);
    mod_group_kernel<4, true><<<g, 256, 0, s>>>(off, col, w, labels, n, work, ctr, 2, sigma, out);
    mod_group_kernel<8, true><<<g, 256, 0, s>>>(off, col, w, labels, n, work, ctr, 3, sigma, out);
    mod_group_kernel<16, true><<<g, 256, 0, s>>>(off, col, w, labels, n, work, ctr, 4, sigma, out);
    mod_group_kernel<32, true><<<g, 256, 0, s>>>(off, col, w, labels, n, work, ctr, 5, sigma, out);
    mod_group_kernel<32, true><<<g, 256, 0, s>>>(off, col, w, labels, n, work, ctr, CLS_WARP_S, sigma, out);
    mod_group_kernel<32, true><<<g, 256, 0, s>>>(off, col, w, labels, n, work, ctr, CLS_WARP_L, sigma, out);
    mod_block_kernel<true><<<4 * di.sm_count, 512, 0, s>>>(off, col, w, labels, n, work, ctr, CLS_BLOCK, sigma, out);
    mod_block_kernel<true><<<4 * di.sm_count, 512, 0, s>>>(off, col, w, labels, n, work, ctr, CLS_HUB, sigma, out);
  } else {
    mod_group_kernel<1, false><<<g, 256, 0, s>>>(off, col, w, labels, n, work, ctr, 0, sigma, out);
    mod_group_kernel<2, false><<<g, 256, 0, s>>>(off, col, w, labels, n, work, ctr, 1, sigma, out);
    mod_group_kernel<4, false><<<g, 256, 0, s>>>(off, col, w, labels, n, work, ctr, 2, sigma, out);
    mod_group_kernel<8, false><<<g, 256, 0, s>>>(off, col, w, labels, n, work, ctr, 3, sigma, out);
    mod_group_kernel<16, false><<<g, 256, 0, s>>>(off, col, w, labels, n, work, ctr, 4, sigma, out);
    mod_group_kernel<32, false><<<g, 256, 0, s>>>(off, col, w, labels, n, work, ctr, 5, sigma, out);
    mod_group_kernel<32, false><<<g, 256, 0, s>>>(off, col, w, labels, n, work, ctr, CLS_WARP_S, sigma, out);
    mod_group_kernel<32, false><<<g, 256, 0, s>>>(off, col, w, labels, n, work, ctr, CLS_WARP_L, sigma, out);
    mod_block_kernel<false><<<4 * di.sm_count, 512, 0, s>>>(off, col, w, labels, n, work, ctr, CLS_BLOCK, sigma, out);
    mod_block_kernel<false><<<4 * di.sm_count, 512, 0, s>>>(off, col, w, labels, n, work, ctr, CLS_HUB, sigma, out);
  }
  const long long np = nparts < modularity_partials(di) ? nparts : modularity_partials(di);
  mod_square_kernel<<<(int)np, 256, 0, s>>>(sigma, n, partials);
  mod_final_kernel<<<1, 32, 0, s>>>(partials, np, out);
  count_launches(13);
  return cudaGetLastError();
}

}  // namespace gsl
