// kernels.h -- host-side launchers of the GSL-LPA kernels (internal header).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "common.cuh"

namespace gsl {

// Arguments of one label-propagation sweep.
struct SweepArgs {
  const long long* off;      // CSR offsets [n+1]
  const int* col;            // CSR columns [nnz]
  const int* w;              // weights [nnz] or nullptr (unit)
  const int* prev;           // labels read (C^{t-1}); == next in async mode
  int* next;                 // labels written (C^t)
  unsigned char* fnext;      // frontier flags of the next sweep (set, never cleared here)
  const int* work;           // worklist (class regions at Counters::cls_start)
  Counters* ctr;
  unsigned long long* wtab;  // global fallback tables of the warp kernel, one region per warp
  long long wtab_region;     // slots per warp region (2 * warp_max)
  unsigned long long* btab;  // global fallback tables of the block kernel, one region per block
  long long btab_region;     // slots per block region (2 * largest degree of classes 7-8)
  long long n;
  int gthresh;               // hub degree above which the block kernel goes straight to global tables (0: never)
  // batched mode (many graphs packed in one CSR); all null for one graph
  const int* gid;            // graph of every vertex
  const long long* vptr;     // vertex range of every graph [vptr[g], vptr[g+1])
  unsigned* dn_graph;        // per-graph change count of this sweep
  const int* stop;           // nonzero: every graph is done, kernels return at once
  int ident;                 // prev is the identity labelling (not read)
  int check;                 // validate weights and weighted degrees
  int mark;                  // mark neighbours of changed vertices in fnext
  const int* lg;             // sync mode: labels gathered per entry, lg[e] = prev[col[e]] (null: gather)
  int spread;                // labels read are nearly all distinct (sweep 2 from the identity labelling)
  unsigned* kw;              // weighted degree per vertex of classes 6-9: written in sweep 1 (check), then read by
                             // the early stops of the majority filter and the hub clusters (null: none)
  int probe_cap;             // bound on the probes of one hash-table insert (past it: ERRBIT_TIMEOUT)
};

struct Tuning {
  int warp_max = 1024;       // class 6 upper degree bound (one warp per vertex)
  int blk_max = 32768;       // class 7 upper degree bound (one block per vertex; above: class 8)
  int warp_slots = 1024;     // shared-memory table slots per warp of class 7 (8 bytes each)
  int blk_slots = 12288;     // shared-memory table slots per block
  int group_block = 256;     // threads per block of the lane-group kernels
  int warp_block = 256;      // threads per block of the warp kernel
  int blk_block = 512;       // threads per block of the block kernel
  int pregather = 0;         // two-phase sweeps: 0 never, 1 when the frontier is large, 2 always
  int majority = 1;          // own-label majority pass: 0 never, 1 once labels settle, 2 always
  int hub_cluster_max = 1 << 30;  // hubs up to this degree go to one thread-block cluster each (0: never)
  int probe_cap = 1 << 24;   // bound on the probes of one hash-table insert
  int uf_cap = 1 << 26;      // bound on the steps of one union-find find or union (split_kernels.cu UF_CAP)
};

// Degree bounds of the classes (see common.cuh).
struct ClassBounds {
  int warp_small;
  int warp_max;
  int blk_max;
};

struct DeviceInfo {
  int sm_count = 0;
  int max_smem_optin = 0;
};

// lpa_kernels.cu
cudaError_t launch_class_histogram(const long long* off, long long n, long long nnz, const Tuning& t,
                                   Counters* ctr, const DeviceInfo& di, cudaStream_t s);
// phase >= 0: only the frontier vertices of that phase of an asynchronous
// sweep (a hash of the vertex id and `seed`); the others keep their flags.
cudaError_t launch_bin(const long long* off, long long n, unsigned char* fcur, int all_active,
                       const Tuning& t, int* work, Counters* ctr, const DeviceInfo& di, cudaStream_t s,
                       const int* gid = nullptr, const unsigned char* done = nullptr, const int* stop = nullptr,
                       int phase = -1, unsigned seed = 0);
// Between the two phases of an asynchronous sweep (see Counters::phase_cls).
cudaError_t launch_phase_reset(Counters* ctr, const int* stop, cudaStream_t s);
cudaError_t launch_sweep(const SweepArgs& a, bool weighted, bool async_mode, const Tuning& t,
                         const DeviceInfo& di, cudaStream_t s);
cudaError_t launch_sweep_class(const SweepArgs& a, int cls, bool weighted, bool async_mode, const Tuning& t,
                               const DeviceInfo& di, cudaStream_t s);
void count_launches(long long k);   // process-wide tally of kernels this library launched
// Raises kernel fn's dynamic shared-memory limit to at least `bytes` (never
// lowers it, so launches of other host threads with smaller tables stay
// valid); thread-safe.
cudaError_t raise_smem_limit(const void* fn, size_t bytes);
long long launches_total();
// Own-label majority filter over classes first_cls..8 (first_cls 6 or 7):
// settled rows keep their label; the others go to `out` (n ints, class
// regions as in the worklist) and become the class counts of the warp and
// block kernels, which must then read `out` as their worklist.
// The class counts of classes first_cls..8 become the rows a filter passed on.
cudaError_t launch_filter_counts(Counters* ctr, const int* stop, cudaStream_t s, int first_cls = CLS_WARP_L);
cudaError_t launch_majority_filter(const SweepArgs& a, int* out, bool weighted, bool async_mode,
                                   const DeviceInfo& di, cudaStream_t s, int first_cls = CLS_WARP_L);
// Edge-parallel label gather for a synchronous sweep: lg[e] = prev[col[e]]
// for every CSR entry (-1 for an out-of-range column).
cudaError_t launch_pregather(const int* col, long long nnz, const int* prev, long long n, int* lg,
                             const DeviceInfo& di, cudaStream_t s);
// Streaming sweep 1 (identity labels, unit weights): bits holds nnz/32+1
// words of scratch; rows that are not strictly increasing are flagged in
// `bad` (n bytes, zero on entry) and left for the hash kernels.
cudaError_t launch_ident_stream(const long long* off, long long n, const int* col, long long nnz, unsigned* bits,
                                unsigned char* bad, int* next, Counters* ctr, const DeviceInfo& di, cudaStream_t s);
// The first two of those passes (row starts, strict-increase check).
cudaError_t launch_row_check(const long long* off, long long n, const int* col, long long nnz, unsigned* bits,
                             unsigned char* bad, Counters* ctr, const DeviceInfo& di, cudaStream_t s);
// Sweeps 1 and 2 while the columns arrive in row-aligned chunks
// (gsl_gsllpa_host): the row-start bitmap (offsets only, bits zeroed
// first), sweep 1 from each row's first entries assuming every row is
// strictly increasing (col may be host memory the device reads), the
// verification of a landed chunk [e0, e1) (flags rows that are not strictly
// increasing in `bad` and raises *any_bad), and the all-active binning of
// the chunk's rows [v0, v1).
cudaError_t launch_rowstart(const long long* off, long long n, unsigned* bits, long long nbits_words,
                            const DeviceInfo& di, cudaStream_t s);
cudaError_t launch_ident_first(const long long* off, long long n, const int* col, const unsigned char* zero_flags,
                               int* next, Counters* ctr, const DeviceInfo& di, cudaStream_t s);
cudaError_t launch_chunk_check(const long long* off, long long n, const int* col, long long nnz, long long e0,
                               long long e1, const unsigned* bits, unsigned char* bad, unsigned* any_bad,
                               Counters* ctr, const DeviceInfo& di, cudaStream_t s);
cudaError_t launch_bin_range(const long long* off, long long v0, long long v1, const Tuning& t, int* work,
                             Counters* ctr, const DeviceInfo& di, cudaStream_t s);
// Streaming sweep 1 with float weights: for strictly increasing rows the
// label is the neighbour of largest weight (smallest id among equals).
cudaError_t launch_ident_stream_f32(const long long* off, long long n, const int* col, const float* wf,
                                    long long nnz, unsigned* bits, unsigned char* bad, int* next, Counters* ctr,
                                    const DeviceInfo& di, cudaStream_t s);
cudaError_t launch_init_labels(const int* init, int* a, int* b, long long n, Counters* ctr,
                               const DeviceInfo& di, cudaStream_t s);
long long block_grid_size(const Tuning& t, const DeviceInfo& di);   // blocks of the class 8/9 kernel
long long warp_grid_warps(const Tuning& t, const DeviceInfo& di);   // warps of the class 7 kernel
ClassBounds class_bounds(const Tuning& t);

// batch_kernels.cu
cudaError_t launch_fill_gid(const long long* vptr, int num_graphs, long long n, int* gid, const DeviceInfo& di,
                            cudaStream_t s);
cudaError_t launch_graph_update(int t, double tol, int max_iters, const long long* vptr, int num_graphs,
                                const unsigned* dn_graph, int* iters, unsigned char* done, int* stop,
                                cudaStream_t s);
cudaError_t launch_batch_final(const int* const* bufs, const int* iters, const int* gid, long long n, int async_mode,
                               int* out, const DeviceInfo& di, cudaStream_t s);
cudaError_t launch_localize(const long long* vptr, const int* gid, long long n, int* labels, const DeviceInfo& di,
                            cudaStream_t s);

// hub_kernels.cu: class 9 in pieces.  Arrays sized by the class's vertex
// total (best, own, wsum, used_cnt: one per hub; piece_start, ustart: one
// more) and its entry total E (used: E slot indices; tab: 2 E slots, all
// EMPTY between sweeps; slot indices must stay below 2^32).
struct HubPlan {
  int* piece_start;             // first piece of frontier hub i (prefix sums)
  long long* ustart;            // first entry of hub i's regions (prefix sums of degrees)
  unsigned long long* best;     // largest packed key over hub i's pieces
  unsigned* own;                // entries of hub i carrying its own label
  unsigned long long* wsum;     // weighted degree of hub i (checked when weighted)
  unsigned* used_cnt;           // table slots claimed for hub i
  unsigned* used;               // their indices: hub i at used[ustart[i]..]
  unsigned long long* tab;      // hub i's table at tab[2 ustart[i] .. 2 ustart[i+1])
  int* clu;                     // frontier hubs taken by clusters (indices i), hub_clusters of them
};
// True when a piece always fits the block kernel's shared table.
bool hub_pieces_fit(const Tuning& t);
// Class 9: plan, cluster kernel (hubs up to t.hub_cluster_max; with
// `majority`, rows whose own label holds a strict majority keep it without
// a table), pieces, final pass.  *kernels = launches made.
cudaError_t launch_hub_pieces(const SweepArgs& a, const HubPlan& hp, bool weighted, bool async_mode, bool majority,
                              const Tuning& t, const DeviceInfo& di, cudaStream_t s, int* kernels);

// float_kernels.cu: sweeps with float32 weights and float64 sums.  Classes
// 6..9 use one block per row; rows whose 2 d slots exceed shared memory use
// the block's region (`region` slots, >= 2 * largest degree) of gkeys/gvals,
// float_table_blocks(di) regions in all.
long long float_table_blocks(const DeviceInfo& di);
cudaError_t launch_sweep_f32(const SweepArgs& a, const float* wf, int cls, bool async_mode, unsigned* gkeys,
                             double* gvals, long long region, const DeviceInfo& di, cudaStream_t s);
// Own-label majority filter for float weights (classes 7-8, float64 sums),
// as launch_majority_filter.
cudaError_t launch_majority_filter_f32(const SweepArgs& a, const float* wf, int* out, bool async_mode,
                                       const DeviceInfo& di, cudaStream_t s);
// Exact fixed-point form of float weights (float_kernels.cu): out[0..2] =
// 1024 + lowest set-bit exponent, 1024 + highest set-bit exponent, invalid
// flag; then wi[e] = w[e] * 2^shift.
cudaError_t launch_f32_exact_scan(const float* w, long long nnz, int* out, const DeviceInfo& di, cudaStream_t s);
cudaError_t launch_f32_to_fixed(const float* w, long long nnz, int shift, int* wi, const DeviceInfo& di,
                                cudaStream_t s);
// Eq. 1 with float weights: sums[0] = 2m, sums[1] = S1, sums[2] = S2 (sigma: n doubles).
cudaError_t launch_modularity_f32(const long long* off, const int* col, const float* wf, const int* labels,
                                  long long n, double* sigma, double* sums, Counters* ctr, const DeviceInfo& di,
                                  cudaStream_t s);

// split_kernels.cu.  parent and named: n ints of scratch each.
cudaError_t launch_split(const long long* off, const int* col, long long n, const int* labels,
                         const int* work, Counters* ctr, int* parent, int* named, int* out, const Tuning& t,
                         const DeviceInfo& di, cudaStream_t s);
cudaError_t launch_renumber(const int* rep, int* out, long long n, int* rank, unsigned long long* block_sums,
                            long long nblocks_cap, unsigned long long* k_dev, const DeviceInfo& di,
                            cudaStream_t s);
long long renumber_blocks(long long n);
// Algorithm 4 from split representatives: cnt (n ints) receives the pieces
// per community, flags (nullable, n bytes) the disconnected communities,
// *total their number.
cudaError_t launch_disconnected(const int* rep, const int* labels, long long n, int* cnt, unsigned char* flags,
                                unsigned long long* total, Counters* ctr, const DeviceInfo& di, cudaStream_t s);
// Algorithm 1: cp = identity (and every frontier flag set), then sweeps
// until Counters::dn stays zero.
cudaError_t launch_split_lp_init(int* cp, unsigned char* f, long long n, const DeviceInfo& di, cudaStream_t s);
cudaError_t launch_split_lp_sweep(const long long* off, const int* col, const int* labels, long long n, int* cp,
                                  unsigned char* fcur, unsigned char* fnext, int prune, Counters* ctr,
                                  const DeviceInfo& di, cudaStream_t s);

// modularity_kernels.cu
struct ModSums {
  unsigned long long two_m;
  unsigned long long s1;
  unsigned long long s2_lo, s2_hi;
};
cudaError_t launch_modularity(const long long* off, const int* col, const int* w, long long n,
                              const int* labels, const int* work, Counters* ctr,
                              unsigned long long* sigma, unsigned long long* partials, long long nparts,
                              ModSums* out, const Tuning& t, const DeviceInfo& di, cudaStream_t s);
long long modularity_partials(const DeviceInfo& di);

}  // namespace gsl
