// batch_kernels.cu -- per-graph bookkeeping of batched GSL-LPA.
//
// A batch is many independent graphs packed into one CSR: graph g owns the
// vertices [vptr[g], vptr[g+1]) and its rows hold only those vertices.  Every
// graph keeps the semantics of a solo run: its own change count dN_g, its
// own stop test dN_g / N_g <= tolerance (Algorithm 3), its own sweep count.
// Because a graph's labels are vertex ids shifted by vptr[g], the
// smallest-label tie-break and the smallest-vertex split labels are the solo
// results shifted by vptr[g], and are shifted back at the end.
#include "kernels.h"

namespace gsl {

namespace {
__device__ __forceinline__ int graph_of(const long long* vptr, int num_graphs, long long v) {
  int lo = 0, hi = num_graphs;   // vptr[lo] <= v < vptr[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (vptr[mid] <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}

int grid_for(long long items, const DeviceInfo& di) {
  long long b = (items + 255) / 256;
  const long long cap = 8ll * di.sm_count;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}
}  // namespace

__global__ void fill_gid_kernel(const long long* __restrict__ vptr, int num_graphs, long long n, int* __restrict__ gid) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
    gid[v] = graph_of(vptr, num_graphs, v);
}

// After sweep t: every graph still running records t, and stops if its
// change fraction is within the tolerance or t reached max_iters.  The last
// graph to stop raises `stop`, which makes the remaining captured sweeps
// return at once.
__global__ void graph_update_kernel(int t, double tol, int max_iters, const long long* __restrict__ vptr,
                                    int num_graphs, const unsigned* __restrict__ dn_graph, int* __restrict__ iters,
                                    unsigned char* __restrict__ done, int* stop) {
  __shared__ int running;
  if (threadIdx.x == 0) running = 0;
  __syncthreads();
  int mine = 0;
  for (int g = threadIdx.x; g < num_graphs; g += blockDim.x) {
    if (done[g]) continue;
    const long long ng = vptr[g + 1] - vptr[g];
    if (t == 0) {   // before the first sweep: empty graphs and max_iters = 0 stop at once
      iters[g] = 0;
      if (ng == 0 || max_iters <= 0) done[g] = 1;
      else mine = 1;
      continue;
    }
    iters[g] = t;
    if ((double)dn_graph[g] / (double)ng <= tol || t >= max_iters) done[g] = 1;
    else mine = 1;
  }
  if (mine) atomicOr(&running, 1);
  __syncthreads();
  if (threadIdx.x == 0 && !running) *stop = 1;
}

// Final labels: graph g's labels are in the buffer its last sweep wrote.
__global__ void batch_final_kernel(const int* __restrict__ b0, const int* __restrict__ b1, const int* __restrict__ iters,
                                   const int* __restrict__ gid, long long n, int async_mode, int* __restrict__ out) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
    out[v] = (async_mode || (iters[gid[v]] & 1) == 0) ? b0[v] : b1[v];
}

__global__ void localize_kernel(const long long* __restrict__ vptr, const int* __restrict__ gid, long long n,
                                int* __restrict__ labels) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
    labels[v] = (int)(labels[v] - vptr[gid[v]]);
}

cudaError_t launch_fill_gid(const long long* vptr, int num_graphs, long long n, int* gid, const DeviceInfo& di,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  fill_gid_kernel<<<grid_for(n, di), 256, 0, s>>>(vptr, num_graphs, n, gid);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_graph_update(int t, double tol, int max_iters, const long long* vptr, int num_graphs,
                                const unsigned* dn_graph, int* iters, unsigned char* done, int* stop,
                                cudaStream_t s) {
  graph_update_kernel<<<1, 1024, 0, s>>>(t, tol, max_iters, vptr, num_graphs, dn_graph, iters, done, stop);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_batch_final(const int* const* bufs, const int* iters, const int* gid, long long n, int async_mode,
                               int* out, const DeviceInfo& di, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  batch_final_kernel<<<grid_for(n, di), 256, 0, s>>>(bufs[0], bufs[1], iters, gid, n, async_mode, out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_localize(const long long* vptr, const int* gid, long long n, int* labels, const DeviceInfo& di,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  localize_kernel<<<grid_for(n, di), 256, 0, s>>>(vptr, gid, n, labels);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace gsl
