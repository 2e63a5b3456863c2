// common.cuh -- device-side helpers shared by the GSL-LPA kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gsl {

constexpr unsigned FULL = 0xFFFFFFFFu;

// Error bits raised by kernels into Counters::err (host maps them to GSL_ERR_*).
constexpr int ERRBIT_INVALID = 1;   // column / label / weight out of range
constexpr int ERRBIT_OVERFLOW = 2;  // weighted degree >= 2^31
constexpr int ERRBIT_TIMEOUT = 4;   // a bounded retry loop ran out

// Degree classes of the sweep.  A vertex of degree d goes to
//   class 0..5 : d in [1,1], [2,2], [3,4], [5,8], [9,16], [17,32]  (lane groups of 1..32)
//   class 6    : 32 < d <= warp_small   (one warp, small shared-memory table)
//   class 7    : warp_small < d <= warp_max (one warp, large shared-memory table)
//   class 8    : warp_max < d <= blk_max   (one block, shared-memory table)
//   class 9    : d > blk_max               (one block, may use global tables)
// Degree-0 vertices never change label and are not binned.
constexpr int NCLASS = 10;
constexpr int CLS_WARP_S = 6;
constexpr int CLS_WARP_L = 7;
constexpr int CLS_BLOCK = 8;
constexpr int CLS_HUB = 9;

// Device-resident counters.  The per-sweep fields come first so that one
// memset of [0, offsetof(err)) resets them between sweeps.
struct Counters {
  unsigned long long dn;        // vertices whose label changed
  unsigned long long scanned;   // CSR entries read by the sweep
  unsigned int cls_count[NCLASS];          // frontier vertices per class this sweep
  unsigned int pad0;
  unsigned long long cls_scanned[NCLASS];  // CSR entries read per class this sweep
  unsigned long long fast_active;          // vertices settled by the streaming identity sweep
  unsigned int hub_pieces;                 // pieces of this sweep's class-9 rows
  unsigned int hub_clusters;               // class-9 rows taken by thread-block clusters
  unsigned int hub_clu_next;               // the next of those rows to be taken
  unsigned int pad3;
  unsigned int uns_count[NCLASS];          // majority filter: rows left for the table kernels
  unsigned int phase_cls[NCLASS];          // asynchronous sweeps: cls_count of the sweep's first phase
  int err;                      // ERRBIT_* (sticky for the call)
  unsigned any_bad;             // host-buffer overlap: a landed row is not strictly increasing (sticky)
  int pad1;
  // per-graph data filled by the class histogram
  unsigned long long cls_total[NCLASS];  // all vertices per class
  unsigned long long cls_start[NCLASS];  // start of each class's region in the worklist
  long long max_degree;
  unsigned long long hub_entries;        // entries of all class-9 rows
  int giant;                    // split: root of the most frequent sampled piece
  int pad2;
};

__device__ __forceinline__ void raise_err(int* err, int bit) {
  if ((__ldcg(err) & bit) == 0) atomicOr(err, bit);
}

__device__ __forceinline__ int degree_class(long long d, int warp_small, int warp_max, int blk_max) {
  if (d <= 0) return -1;
  if (d <= 32) return 32 - __clz((int)(d - 1));  // 1->0, 2->1, 3..4->2, 5..8->3, 9..16->4, 17..32->5
  if (d <= warp_small) return CLS_WARP_S;
  if (d <= warp_max) return CLS_WARP_L;
  if (d <= blk_max) return CLS_BLOCK;
  return CLS_HUB;
}

// Streaming load for data read exactly once (CSR columns / weights): no L1
// allocation and an L2 evict-first policy, so the stream does not push the
// label array out of L2.  Kernels create the policies once and pass them.
__device__ __forceinline__ unsigned long long policy_evict_first() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long policy_evict_last() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ int ld_stream(const int* p, unsigned long long pol) {
  int v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ int ld_stream(const int* p) { return ld_stream(p, policy_evict_first()); }
// 16-byte streaming load (p must be 16-byte aligned).
__device__ __forceinline__ int4 ld_stream4(const int4* p, unsigned long long pol) {
  int4 v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p), "l"(pol));
  return v;
}
// Gather of a label that stays constant for the whole kernel (Jacobi sweep):
// read-only path, L2 evict-last policy.
__device__ __forceinline__ int ld_label_ro(const int* p, unsigned long long pol) {
  int v;
  asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ int ld_label_ro(const int* p) { return ld_label_ro(p, policy_evict_last()); }
// Gather of a label that other threads may be writing (in-place sweep):
// coherent at L2.
__device__ __forceinline__ int ld_label_rw(const int* p) { return __ldcg(p); }

__device__ __forceinline__ uint32_t hash32(uint32_t x) { return x * 0x9E3779B1u; }

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    unsigned long long y = __shfl_xor_sync(FULL, x, o);
    x = y > x ? y : x;
  }
  return x;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}


__host__ __device__ __forceinline__ unsigned next_pow2(unsigned x) {
  unsigned p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace gsl
