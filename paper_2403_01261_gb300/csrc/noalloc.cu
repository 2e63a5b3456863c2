// noalloc.cu -- modularity (Eq. 1) for callers that cannot allocate memory.
//
// gsl_modularity needs a context, and a context allocates its scratch with
// cudaMalloc.  Some callers cannot do that: a request loop that must not
// pay the device-wide synchronisation cudaMalloc / cudaFree can cause, or a
// process whose GPU memory is already reserved in full by another
// allocator.  gsl_modularity_noalloc computes the same value with all of its
// scratch (per-community degree sums, partial sums, error word) in one
// fixed, file-scope device array, so it allocates nothing.  The array holds
// GSL_NOALLOC_MAX_N community sums: every GPU that loads the library keeps
// about 32 MB reserved for it until the process exits.
#include <cstddef>
#include <cstdint>
#include <mutex>

#include "../../include/gsllpa.h"
#include "common.cuh"

namespace {

constexpr int NA_PARTIALS = 512;   // blocks of the squaring pass

struct NaHeader {
  unsigned long long two_m;
  unsigned long long s1;
  unsigned long long s2_lo, s2_hi;
  int err;
  int pad;
  unsigned long long partials[2 * NA_PARTIALS];
};
constexpr size_t NA_SIGMA_OFFSET = (sizeof(NaHeader) + 255) / 256 * 256;
constexpr size_t NA_BYTES = NA_SIGMA_OFFSET + sizeof(unsigned long long) * (size_t)GSL_NOALLOC_MAX_N;

// The scratch.  Host code must not use this name as an address: it resolves
// the device address with cudaGetSymbolAddress once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
void* g_na_addr[NA_MAX_DEVICES] = {};

// Device address of the scratch on the current device (set up on first use).
int na_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    cudaGetLastError();
    return GSL_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return GSL_ERR_CUDA;
    }
    g_na_addr[dev] = p;
  }
  *out = g_na_addr[dev];
  return GSL_OK;
}

__global__ void na_clear_kernel(unsigned char* scratch, long long n) {
  NaHeader* h = reinterpret_cast<NaHeader*>(scratch);
  unsigned long long* sigma = reinterpret_cast<unsigned long long*>(scratch + NA_SIGMA_OFFSET);
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid == 0) {
    h->two_m = 0;
    h->s1 = 0;
    h->s2_lo = 0;
    h->s2_hi = 0;
    h->err = 0;
  }
  for (long long c = tid; c < n; c += (long long)gridDim.x * blockDim.x) sigma[c] = 0;
}

// One warp per vertex: K_u = sum of its weights into Sigma[C_u]; weights of
// entries inside C_u into S1; K_u into 2m.  Offsets, columns, weights and
// labels are range checked (an out-of-range value sets err and is skipped).
template <bool WEIGHTED>
__global__ void __launch_bounds__(256) na_rows_kernel(const long long* __restrict__ off, const int* __restrict__ col,
                                                       const int* __restrict__ w, const int* __restrict__ labels,
                                                       long long n, long long nnz, unsigned char* scratch) {
  NaHeader* h = reinterpret_cast<NaHeader*>(scratch);
  unsigned long long* sigma = reinterpret_cast<unsigned long long*>(scratch + NA_SIGMA_OFFSET);
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long tk = 0, ts1 = 0;
  int bad = 0;
  for (long long u = warp; u < n; u += nwarps) {
    const long long s = off[u], e = off[u + 1];
    const int cu = labels[u];
    if (s < 0 || e < s || e > nnz || (u == 0 && s != 0) || (u == n - 1 && e != nnz) || cu < 0 || cu >= n) {
      bad = 1;
      continue;
    }
    unsigned long long k = 0;
    for (long long x = s + lane; x < e; x += 32) {
      const int j = col[x];
      const long long we = WEIGHTED ? (long long)w[x] : 1;
      if (j < 0 || j >= n || we <= 0) {
        bad = 1;
        continue;
      }
      k += (unsigned long long)we;
      if (labels[j] == cu) ts1 += (unsigned long long)we;
    }
    for (int o = 16; o; o >>= 1) k += __shfl_xor_sync(gsl::FULL, k, o);
    if (lane == 0 && k) atomicAdd(sigma + cu, k);
    tk += lane == 0 ? k : 0ull;
  }
  for (int o = 16; o; o >>= 1) {
    tk += __shfl_xor_sync(gsl::FULL, tk, o);
    ts1 += __shfl_xor_sync(gsl::FULL, ts1, o);
  }
  bad = __any_sync(gsl::FULL, bad);
  if (lane == 0) {
    if (tk) atomicAdd(&h->two_m, tk);
    if (ts1) atomicAdd(&h->s1, ts1);
    if (bad) atomicOr(&h->err, 1);
  }
}

// S2 = sum_c Sigma_c^2 in 128 bits: per-block partials, then one block adds them.
__global__ void __launch_bounds__(256) na_square_kernel(long long n, unsigned char* scratch) {
  NaHeader* h = reinterpret_cast<NaHeader*>(scratch);
  const unsigned long long* sigma = reinterpret_cast<const unsigned long long*>(scratch + NA_SIGMA_OFFSET);
  unsigned long long lo = 0, hi = 0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const unsigned long long x = sigma[c];
    const unsigned long long plo = x * x, phi = __umul64hi(x, x);
    lo += plo;
    hi += phi + (lo < plo ? 1ull : 0ull);
  }
  __shared__ unsigned long long slo[256], shi[256];
  slo[threadIdx.x] = lo;
  shi[threadIdx.x] = hi;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < (unsigned)o) {
      const unsigned long long a = slo[threadIdx.x], b = slo[threadIdx.x + o];
      slo[threadIdx.x] = a + b;
      shi[threadIdx.x] += shi[threadIdx.x + o] + (a + b < a ? 1ull : 0ull);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    h->partials[2 * blockIdx.x] = slo[0];
    h->partials[2 * blockIdx.x + 1] = shi[0];
  }
}

__global__ void na_final_kernel(unsigned char* scratch, int nparts) {
  NaHeader* h = reinterpret_cast<NaHeader*>(scratch);
  if (threadIdx.x != 0) return;
  unsigned long long lo = 0, hi = 0;
  for (int b = 0; b < nparts; ++b) {
    const unsigned long long plo = h->partials[2 * b];
    lo += plo;
    hi += h->partials[2 * b + 1] + (lo < plo ? 1ull : 0ull);
  }
  h->s2_lo = lo;
  h->s2_hi = hi;
}

}  // namespace

extern "C" int gsl_modularity_noalloc(const gsl_csr* g, const int32_t* weights, const int32_t* labels,
                                      double* q_out, void* stream) {
  if (!g || !q_out) return GSL_ERR_INVALID;
  if (g->n < 0 || g->nnz < 0 || !g->offsets || (g->nnz > 0 && !g->cols) || (g->n > 0 && !labels))
    return GSL_ERR_INVALID;
  if (g->n > GSL_NOALLOC_MAX_N) return GSL_ERR_INVALID;   // beyond the fixed scratch
  *q_out = 0.0;
  if (g->n == 0) return GSL_OK;
  void* p = nullptr;
  if (int r = na_scratch(&p)) return r;
  unsigned char* scratch = static_cast<unsigned char*>(p);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long n = g->n;
  const long long* off = reinterpret_cast<const long long*>(g->offsets);
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = 8 * (sms > 0 ? sms : 1);
  // A launch error left pending by earlier, unrelated work on this thread is
  // cleared here, so that the check after the launches sees only this call's.
  cudaGetLastError();
  na_clear_kernel<<<grid, 256, 0, s>>>(scratch, n);
  if (weights)
    na_rows_kernel<true><<<grid, 256, 0, s>>>(off, g->cols, weights, labels, n, g->nnz, scratch);
  else
    na_rows_kernel<false><<<grid, 256, 0, s>>>(off, g->cols, weights, labels, n, g->nnz, scratch);
  na_square_kernel<<<NA_PARTIALS, 256, 0, s>>>(n, scratch);
  na_final_kernel<<<1, 32, 0, s>>>(scratch, NA_PARTIALS);
  if (cudaGetLastError() != cudaSuccess) return GSL_ERR_CUDA;
  NaHeader res;
  if (cudaMemcpyAsync(&res, scratch, offsetof(NaHeader, partials), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return GSL_ERR_CUDA;
  }
  if (res.err) return GSL_ERR_INVALID;
  if (res.two_m == 0) return GSL_OK;
  const unsigned __int128 s2 = ((unsigned __int128)res.s2_hi << 64) | res.s2_lo;
  const double dm = (double)res.two_m;
  *q_out = (double)res.s1 / dm - (double)s2 / (dm * dm);
  return GSL_OK;
}
