// gsllpa.cu -- host orchestration and C ABI of the GSL-LPA library.
//
// lpa() of Algorithm 3 runs as a host loop of sweeps: bin the frontier by
// degree class, launch the class kernels, read the change count back, stop
// when dN/N <= tolerance or after max_iters sweeps.  The split of Algorithm
// 2 and the modularity of Eq. 1 follow as separate kernel sequences.  The
// context owns all scratch memory and grows it on demand.
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <algorithm>
#include <vector>

#include "../../include/gsllpa.h"
#include "kernels.h"

using namespace gsl;

struct gsl_ctx {
  int device = 0;
  DeviceInfo di;
  Tuning tune;
  std::string last_error;

  long long cap_n = 0;             // vertex capacity of the per-vertex scratch
  int* lab[2] = {nullptr, nullptr};
  unsigned char* flag[2] = {nullptr, nullptr};
  int* work = nullptr;
  int* parent = nullptr;
  int* rank = nullptr;
  unsigned long long* sigma = nullptr;
  long long cap_sigma = 0;
  unsigned long long* block_sums = nullptr;
  long long cap_blocks = 0;
  unsigned long long* partials = nullptr;
  long long cap_partials = 0;

  unsigned* rowbits = nullptr;          // row-start bitmap of the streaming identity sweep
  long long cap_rowbits = 0;
  unsigned* fkeys = nullptr;            // float-weight sweep: global table regions (keys, sums)
  double* fvals = nullptr;
  long long cap_fkeys = 0, cap_fvals = 0;
  int* work2 = nullptr;                 // worklist of the rows the majority filter leaves
  long long cap_work2 = 0;
  int* lg = nullptr;                    // labels gathered per CSR entry (two-phase sweeps)
  long long cap_lg = 0;
  unsigned long long* wtab = nullptr;   // warp-kernel fallback tables
  long long cap_wtab = 0;
  unsigned long long* btab = nullptr;   // block-kernel fallback tables
  long long cap_btab = 0;
  // class 9 in pieces (hub_kernels.cu)
  int* hub_piece_start = nullptr;
  long long* hub_ustart = nullptr;
  unsigned long long* hub_best = nullptr;
  unsigned* hub_own = nullptr;
  unsigned long long* hub_wsum = nullptr;
  unsigned* hub_used_cnt = nullptr;
  int* hub_clu = nullptr;
  long long cap_hub_v = 0;              // entries of each of the seven per-hub arrays
  unsigned* hub_used = nullptr;
  long long cap_hub_used = 0;
  unsigned long long* hub_tab = nullptr;
  long long cap_hub_tab = 0;
  bool hub_ready = false;               // pieces usable for the prepared graph
  bool hub_dirty = true;                // hub_tab may hold non-empty slots

  Counters* ctr = nullptr;         // device
  Counters* ctr_h = nullptr;       // pinned host mirror
  ModSums* sums = nullptr;         // device
  ModSums* sums_h = nullptr;       // pinned
  unsigned long long* k_dev = nullptr;
  unsigned long long* k_h = nullptr;

  // staging of the host-buffer entry point
  long long* st_off = nullptr;
  long long cap_st_off = 0;
  int* st_col = nullptr;
  long long cap_st_col = 0;
  int* st_w = nullptr;
  long long cap_st_w = 0;
  int* st_lab = nullptr;
  long long cap_st_lab = 0;
  unsigned* kw = nullptr;               // weighted degrees (integer-weight sweeps)
  long long cap_kw = 0;
  // float weights in exact fixed point (run on the integer sweeps)
  int f32_fixed = 1;                    // 0: always float64 sums; 1: fixed point when exact
  int* fix_w = nullptr;
  long long cap_fix_w = 0;
  int* fix_dev = nullptr;               // 3 ints
  int* fix_h = nullptr;                 // pinned mirror

  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};

  // host-buffer path: column chunks copied on their own stream
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> chunk_ev;
  long long host_overlap_min = 1ll << 24;   // entries from which gsl_gsllpa_host overlaps copies and sweeps

  // batched mode
  int* gid = nullptr;
  long long cap_gid = 0;
  long long* vptr = nullptr;
  long long cap_vptr = 0;
  unsigned* dn_graph = nullptr;
  long long cap_dng = 0;
  int* iters = nullptr;
  long long cap_iters = 0;
  unsigned char* done = nullptr;
  long long cap_done = 0;
  int* stop = nullptr;
  long long cap_stop = 0;
  int* lab_tmp = nullptr;
  long long cap_lab_tmp = 0;
  cudaStream_t cap_stream = nullptr;   // captures and replays the batched sweep loop
  cudaGraphExec_t batch_exec = nullptr;
  bool batch_direct = false;           // launch the batched loop directly instead of as a CUDA graph
  std::vector<long long> batch_key;    // arguments the captured graph was built for

  // profiling (gsl_ctx_set_profiling): CUDA-event time per launch sequence
  bool prof = false;
  gsl_profile profile{};
  std::vector<cudaEvent_t> evpool;
  struct Pending {
    int slot, e0, e1;
  };
  std::vector<Pending> pending;
  int ev_used = 0;
};

namespace {

// int64_t is `long` on LP64 Linux; the kernels take `long long`.
inline const long long* OFF(const gsl_csr* g) { return reinterpret_cast<const long long*>(g->offsets); }

// Single-graph sweeps: from this sweep on, the own-label majority filter
// takes the rows of class 6 too, once most of them keep their label (R-MAT
// 25, ms per step: from sweep 4 51.3 -> 50.6; from sweep 3 no gain, as
// sweep 3's class-6 rows mostly change and the filter's pass over them is
// then repeated by the warp kernel).  The batched loop's planted-partition
// graphs settle later (4096-graph batch, ms per step: none 459.8, from
// sweep 4 500.5, from sweep 6 454.1).
constexpr int FILTER6_FROM = 4;
constexpr int BATCH_FILTER6_FROM = 6;

int fail(gsl_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->last_error = buf;
  }
  return code;
}

#define CK(call)                                                                                     \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) {                                                                         \
      cudaGetLastError();                                                                            \
      return fail(c, e_ == cudaErrorMemoryAllocation ? GSL_ERR_NOMEM : GSL_ERR_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                                \
    }                                                                                                \
  } while (0)

template <typename T>
int grow(gsl_ctx* c, T*& ptr, long long& cap, long long need) {
  if (need <= cap && ptr) return GSL_OK;
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  cap = 0;
  long long alloc = need > 0 ? need : 1;
  cudaError_t e = cudaMalloc(&ptr, sizeof(T) * (size_t)alloc);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
    return fail(c, GSL_ERR_NOMEM, "cudaMalloc of %lld bytes failed: %s", (long long)(sizeof(T) * alloc),
                cudaGetErrorString(e));
  }
  cap = alloc;
  return GSL_OK;
}

int ensure_vertex_scratch(gsl_ctx* c, long long n) {
  if (n <= c->cap_n && c->lab[0]) return GSL_OK;
  long long dummy;
  for (int i = 0; i < 2; ++i) {
    dummy = 0;
    if (c->lab[i]) cudaFree(c->lab[i]);
    c->lab[i] = nullptr;
    if (int r = grow(c, c->lab[i], dummy, n)) return r;
    dummy = 0;
    if (c->flag[i]) cudaFree(c->flag[i]);
    c->flag[i] = nullptr;
    if (int r = grow(c, c->flag[i], dummy, n)) return r;
  }
  dummy = 0;
  if (c->work) cudaFree(c->work);
  c->work = nullptr;
  if (int r = grow(c, c->work, dummy, n)) return r;
  dummy = 0;
  if (c->parent) cudaFree(c->parent);
  c->parent = nullptr;
  if (int r = grow(c, c->parent, dummy, n)) return r;
  dummy = 0;
  if (c->rank) cudaFree(c->rank);
  c->rank = nullptr;
  if (int r = grow(c, c->rank, dummy, n)) return r;
  c->cap_n = n;
  return GSL_OK;
}

int check_csr(gsl_ctx* c, const gsl_csr* g) {
  if (!g) return fail(c, GSL_ERR_INVALID, "graph is NULL");
  if (g->n < 0 || g->n >= (1ll << 31)) return fail(c, GSL_ERR_INVALID, "n = %lld outside [0, 2^31)", (long long)g->n);
  if (g->nnz < 0) return fail(c, GSL_ERR_INVALID, "nnz = %lld < 0", (long long)g->nnz);
  if (!g->offsets) return fail(c, GSL_ERR_INVALID, "offsets is NULL");
  if (g->nnz > 0 && !g->cols) return fail(c, GSL_ERR_INVALID, "cols is NULL");
  return GSL_OK;
}

int map_err(gsl_ctx* c, int bits, const char* where) {
  if (bits & ERRBIT_INVALID) return fail(c, GSL_ERR_INVALID, "%s: malformed graph or labels (offsets, column, weight or label out of range)", where);
  if (bits & ERRBIT_OVERFLOW) return fail(c, GSL_ERR_OVERFLOW, "%s: a weighted degree is >= 2^31", where);
  if (bits & ERRBIT_TIMEOUT) return fail(c, GSL_ERR_TIMEOUT, "%s: a device retry loop hit its bound", where);
  return GSL_OK;
}

// ------------------------------------------------------------- profiling
enum Slot {
  SL_CLASSIFY = 0, SL_INIT, SL_BIN, SL_SWEEP0, SL_SPLIT = SL_SWEEP0 + NCLASS, SL_COUNT, SL_MOD, SL_IDENT, SL_PRE,
  SL_FILTER, SL_N
};
const char* slot_name(int k) {
  static const char* names[SL_N] = {"classify", "init_labels", "bin_frontier", "sweep_deg1", "sweep_deg2",
                                    "sweep_deg3_4", "sweep_deg5_8", "sweep_deg9_16", "sweep_deg17_32",
                                    "sweep_warp_small", "sweep_warp_large", "sweep_block", "sweep_hub",
                                    "split_unionfind", "split_count_renumber", "modularity", "sweep1_stream", "pregather", "majority_filter"};
  return names[k];
}

int prof_begin(gsl_ctx* c, cudaStream_t s) {
  if (!c->prof) return -1;
  while ((int)c->evpool.size() < c->ev_used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    c->evpool.push_back(e);
  }
  const int e0 = c->ev_used;
  c->ev_used += 2;
  cudaEventRecord(c->evpool[e0], s);
  return e0;
}

void prof_end(gsl_ctx* c, int e0, int slot, cudaStream_t s, long long kernels) {
  if (e0 < 0) return;
  cudaEventRecord(c->evpool[e0 + 1], s);
  c->pending.push_back({slot, e0, e0 + 1});
  c->profile.slot[slot].launches += 1;
  c->profile.slot[slot].kernels += kernels;
}

// Call after the stream has been synchronised.
void prof_resolve(gsl_ctx* c) {
  for (const auto& p : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->evpool[p.e0], c->evpool[p.e1]) == cudaSuccess) c->profile.slot[p.slot].ms += ms;
    else cudaGetLastError();
  }
  c->pending.clear();
  c->ev_used = 0;
}

// Resets all counters, classifies every vertex by degree (validating the
// offsets) and sizes the hub tables.  Synchronises the stream.
int prepare_graph(gsl_ctx* c, const gsl_csr* g, cudaStream_t s) {
  CK(cudaMemsetAsync(c->ctr, 0, sizeof(Counters), s));
  const int pe = prof_begin(c, s);
  CK(launch_class_histogram(OFF(g), g->n, g->nnz, c->tune, c->ctr, c->di, s));
  prof_end(c, pe, SL_CLASSIFY, s, 2);
  c->profile.slot[SL_CLASSIFY].vertices += g->n;
  c->profile.slot[SL_CLASSIFY].bytes += 8.0 * (double)(g->n + 1);
  CK(cudaMemcpyAsync(c->ctr_h, c->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  prof_resolve(c);
  if (int r = map_err(c, c->ctr_h->err, "offsets")) return r;
  const long long maxd = c->ctr_h->max_degree;
  if (maxd > c->tune.warp_slots / 2 && maxd > 32) {
    // a class-6 vertex may overflow its shared table: 2 * warp_max slots per warp
    const long long need = warp_grid_warps(c->tune, c->di) * 2ll * c->tune.warp_max;
    if (int r = grow(c, c->wtab, c->cap_wtab, need)) return r;
  }
  if (maxd > c->tune.warp_max) {
    const long long need = block_grid_size(c->tune, c->di) * 2ll * maxd;
    if (int r = grow(c, c->btab, c->cap_btab, need)) return r;
  }
  // class 9 (hubs) in pieces: per-hub plan arrays and table regions
  const long long hubs = (long long)c->ctr_h->cls_total[CLS_HUB];
  const long long hub_e = (long long)c->ctr_h->hub_entries;
  c->hub_ready = hubs > 0 && hub_pieces_fit(c->tune) && 2 * hub_e < (1ll << 32);
  if (c->hub_ready) {
    const long long old_tab = c->cap_hub_tab;
    const unsigned long long* old_ptr = c->hub_tab;
    if (c->cap_hub_v < hubs + 1) {   // the seven per-hub arrays share one capacity
      long long k0 = 0, k1 = 0, k2 = 0, k3 = 0, k4 = 0, k5 = 0, k6 = 0;
      c->cap_hub_v = 0;
      if (int r = grow(c, c->hub_piece_start, k0, hubs + 1)) return r;
      if (int r = grow(c, c->hub_ustart, k1, hubs + 1)) return r;
      if (int r = grow(c, c->hub_best, k2, hubs + 1)) return r;
      if (int r = grow(c, c->hub_own, k3, hubs + 1)) return r;
      if (int r = grow(c, c->hub_wsum, k4, hubs + 1)) return r;
      if (int r = grow(c, c->hub_used_cnt, k5, hubs + 1)) return r;
      if (int r = grow(c, c->hub_clu, k6, hubs + 1)) return r;
      c->cap_hub_v = hubs + 1;
    }
    if (int r = grow(c, c->hub_used, c->cap_hub_used, hub_e)) return r;
    if (int r = grow(c, c->hub_tab, c->cap_hub_tab, 2 * hub_e)) return r;
    if (c->hub_dirty || c->cap_hub_tab != old_tab || c->hub_tab != old_ptr) {
      CK(cudaMemsetAsync(c->hub_tab, 0xFF, sizeof(unsigned long long) * (size_t)c->cap_hub_tab, s));
      c->hub_dirty = false;
    }
  }
  return GSL_OK;
}


int reset_sweep_counters(gsl_ctx* c, cudaStream_t s) {
  CK(cudaMemsetAsync(c->ctr, 0, offsetof(Counters, err), s));
  return GSL_OK;
}

// State of a synchronous sweep loop whose first `done` sweeps ran elsewhere
// (the host-buffer path runs sweeps 1 and 2 while the columns arrive): the
// labels of sweep `done` are in lab[done & 1], the frontier flags are as
// that sweep left them, and the per-sweep statistics up to it are filled.
struct LpaResume {
  int done;              // sweeps already run
  bool converged;        // the stop test already held after sweep `done`
  bool marked_prev;      // sweep `done` marked the neighbours of changed vertices
  long long dn_prev;     // its change count
  long long scanned;     // entries read by those sweeps
};

// The sweep loop.  On success *final points at the scratch buffer holding
// the labels.  prepare_graph must have run.
int run_lpa(gsl_ctx* c, const gsl_csr* g, const int32_t* weights, const int32_t* labels_init, double tol,
            int32_t max_iters, int32_t mode, gsl_stats* st, cudaStream_t s, int** final,
            const LpaResume* resume = nullptr) {
  const long long n = g->n;
  const bool async_mode = mode == GSL_MODE_ASYNC;
  if (!resume) {
    CK(cudaMemsetAsync(c->flag[0], 0, (size_t)n, s));
    CK(cudaMemsetAsync(c->flag[1], 0, (size_t)n, s));
    const int pe = prof_begin(c, s);
    CK(launch_init_labels(labels_init, c->lab[0], async_mode ? nullptr : c->lab[1], n, c->ctr, c->di, s));
    prof_end(c, pe, SL_INIT, s, 1);
    c->profile.slot[SL_INIT].vertices += n;
    c->profile.slot[SL_INIT].bytes += (double)n * ((labels_init ? 4.0 : 0.0) + (async_mode ? 4.0 : 8.0));
  }
  SweepArgs a{};
  a.off = OFF(g);
  a.col = g->cols;
  a.w = weights;
  a.ctr = c->ctr;
  a.probe_cap = c->tune.probe_cap;
  a.work = c->work;
  a.wtab = c->wtab;
  a.wtab_region = 2ll * c->tune.warp_max;
  a.btab = c->btab;
  a.btab_region = 2ll * c->ctr_h->max_degree;
  a.n = n;
  if (weights) {   // weighted degrees, written by sweep 1 for the early stops of later sweeps
    if (int r = grow(c, c->kw, c->cap_kw, n)) return r;
    a.kw = c->kw;
  }
  int t = resume ? resume->done : 0;
  bool converged = resume ? resume->converged : false, marked_prev = resume ? resume->marked_prev : false;
  long long dn_prev = resume ? resume->dn_prev : n;
  long long scanned = resume ? resume->scanned : 0;
  while (t < max_iters && !converged) {
    ++t;
    if (int r = reset_sweep_counters(c, s)) return r;
    bool all_active = t == 1 || !marked_prev;
    // Sweep 1 from the identity labels with unit weights streams the rows;
    // only rows that are not strictly increasing (flagged in flag[1]) go
    // through the binned hash kernels below.
    const bool stream1 = t == 1 && !async_mode && !labels_init && !weights;
    if (stream1) {
      if (int r = grow(c, c->rowbits, c->cap_rowbits, (g->nnz >> 5) + 1)) return r;
      const int pe = prof_begin(c, s);
      CK(launch_ident_stream(OFF(g), n, g->cols, g->nnz, c->rowbits, c->flag[1], c->lab[1], c->ctr, c->di, s));
      prof_end(c, pe, SL_IDENT, s, 3);
      c->profile.slot[SL_IDENT].vertices += n;
      c->profile.slot[SL_IDENT].entries += g->nnz;
      c->profile.slot[SL_IDENT].bytes += 4.0 * (double)g->nnz + 16.0 * (double)n;
      all_active = false;   // the bin pass below picks up the flagged rows only
    }
    if (async_mode) {
      a.prev = c->lab[0];
      a.next = c->lab[0];
    } else {
      a.prev = c->lab[(t - 1) & 1];
      a.next = c->lab[t & 1];
    }
    a.fnext = c->flag[(t + 1) & 1];
    // (rows left over by the streaming pass are not strictly increasing, so
    // the sorted-row shortcut of the hash kernels would fail on them)
    a.ident = (!async_mode && !labels_init && t == 1 && !stream1) ? 1 : 0;
    // Two-phase sweep: gather every entry's label at full occupancy first,
    // then the class kernels read them as a stream.  Worth it when the
    // frontier holds most rows.
    a.lg = nullptr;
    if (!async_mode && !a.ident && !stream1 && g->nnz > 0 &&
        (c->tune.pregather == 2 || (c->tune.pregather == 1 && g->nnz >= (1ll << 22) && (all_active || 4 * dn_prev > n)))) {
      if (int r = grow(c, c->lg, c->cap_lg, g->nnz)) return r;
      const int pe = prof_begin(c, s);
      CK(launch_pregather(g->cols, g->nnz, a.prev, n, c->lg, c->di, s));
      prof_end(c, pe, SL_PRE, s, 1);
      c->profile.slot[SL_PRE].entries += g->nnz;
      c->profile.slot[SL_PRE].bytes += 12.0 * (double)g->nnz;
      a.lg = c->lg;
    }
    a.check = t == 1 ? 1 : 0;
    // the first sweep that gathers labels after the identity sweep sees
    // almost as many distinct labels as neighbours (about 0.3 d on R-MAT
    // hubs): hubs beyond three shared tables' worth go to global tables
    a.gthresh = (t == 2 && !async_mode && !labels_init) ? 3 * c->tune.blk_slots : 0;
    a.spread = (t == 2 && !async_mode && !labels_init) ? 1 : 0;
    // Sweep 1 changes every vertex that has a neighbour, and a sweep after
    // one that changed more than half of the vertices is run on all
    // vertices: marking would select nearly everything anyway.
    a.mark = (t > 1 && 2 * dn_prev <= n) ? 1 : 0;
    // from sweep 3 on, most long rows keep a majority of their own label
    // (sweep 2 reads the labels of sweep 1, which are nearly all distinct):
    // filter those out before the tables
    const bool filter = !a.ident && !a.check && (c->tune.majority == 2 || (c->tune.majority == 1 && t >= 3));
    if (filter)
      if (int r = grow(c, c->work2, c->cap_work2, n)) return r;
    // from FILTER6_FROM on the filter takes class 6 (rows of 33..warp_small
    // entries) as well
    const int filter_from = (filter && t >= FILTER6_FROM) ? CLS_WARP_S : CLS_WARP_L;
    // An asynchronous sweep runs its frontier in two phases chosen by a hash
    // of the vertex id and the sweep number, the second reading the labels
    // the first wrote: neighbours that would update at the same moment every
    // sweep (and swap labels forever) fall in different phases half of the
    // time.  A synchronous sweep is one phase.
    const int phases = async_mode ? 2 : 1;
    for (int ph = 0; ph < phases; ++ph) {
      if (ph == 1) CK(launch_phase_reset(c->ctr, nullptr, s));
      {
        const int pe = prof_begin(c, s);
        CK(launch_bin(OFF(g), n, c->flag[t & 1], all_active ? 1 : 0, c->tune, c->work, c->ctr, c->di, s, nullptr,
                      nullptr, nullptr, async_mode ? ph : -1, (unsigned)t));
        prof_end(c, pe, SL_BIN, s, 1);
      }
      SweepArgs af = a;   // the filtered classes read the filter's worklist
      if (filter) {
        const int pe = prof_begin(c, s);
        CK(launch_majority_filter(a, c->work2, weights != nullptr, async_mode, c->di, s, filter_from));
        prof_end(c, pe, SL_FILTER, s, 2);
        af.work = c->work2;
      }
      for (int k = NCLASS - 1; k >= 0; --k) {   // the longest rows first
        const int pe = prof_begin(c, s);
        if (k == CLS_WARP_L || k == CLS_BLOCK || (k == CLS_WARP_S && filter_from == CLS_WARP_S)) {
          CK(launch_sweep_class(af, k, weights != nullptr, async_mode, c->tune, c->di, s));
          prof_end(c, pe, SL_SWEEP0 + k, s, 1);
        } else if (k == CLS_HUB && c->hub_ready) {
          HubPlan hp{c->hub_piece_start, c->hub_ustart, c->hub_best, c->hub_own,
                     c->hub_wsum,        c->hub_used_cnt, c->hub_used, c->hub_tab, c->hub_clu};
          c->hub_dirty = true;   // until this sweep is known to have finished cleanly
          int kernels = 0;
          CK(launch_hub_pieces(a, hp, weights != nullptr, async_mode, filter, c->tune, c->di, s, &kernels));
          prof_end(c, pe, SL_SWEEP0 + k, s, kernels);
        } else {
          CK(launch_sweep_class(a, k, weights != nullptr, async_mode, c->tune, c->di, s));
          prof_end(c, pe, SL_SWEEP0 + k, s, 1);
        }
      }
    }
    CK(cudaMemcpyAsync(c->ctr_h, c->ctr, offsetof(Counters, pad1), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (c->prof) {
      prof_resolve(c);
      // algorithmic bytes: per processed vertex its two offsets (8 B, shared
      // with the next row), worklist entry, own label (not read from the
      // identity labelling) and label write; per entry the column, the
      // neighbour's label (not read from the identity labelling) and weight
      const double per_v = 8.0 + 4.0 + (a.ident ? 0.0 : 4.0) + 4.0;
      const double per_e = 4.0 + (a.ident ? 0.0 : 4.0) + (weights ? 4.0 : 0.0);
      long long act_all = 0;
      for (int k = 0; k < NCLASS; ++k) {
        auto& sl = c->profile.slot[SL_SWEEP0 + k];
        const long long v = (long long)(c->ctr_h->cls_count[k] + c->ctr_h->phase_cls[k]);
        const long long e = (long long)c->ctr_h->cls_scanned[k];
        sl.vertices += v;
        sl.entries += e;
        sl.bytes += per_v * (double)v + per_e * (double)e;
        act_all += v;
      }
      if (filter) {
        // the filter read every row of classes 7 and 8: the settled ones (their
        // entries are in `scanned` but in no class) and those it passed on
        long long cls_e = 0, rows = (long long)c->ctr_h->fast_active;
        for (int k = 0; k < NCLASS; ++k) cls_e += (long long)c->ctr_h->cls_scanned[k];
        long long fe = (long long)c->ctr_h->scanned - cls_e;
        for (int k = CLS_WARP_L; k <= CLS_BLOCK; ++k) {
          fe += (long long)c->ctr_h->cls_scanned[k];
          rows += (long long)(c->ctr_h->cls_count[k] + c->ctr_h->phase_cls[k]);
        }
        auto& sf = c->profile.slot[SL_FILTER];
        sf.vertices += rows;
        sf.entries += fe;
        sf.bytes += per_v * (double)rows + per_e * (double)fe;
      }
      auto& sb = c->profile.slot[SL_BIN];
      sb.vertices += all_active ? n : act_all;
      sb.bytes += (all_active ? 0.0 : (double)n) + (all_active ? 16.0 * (double)n : 16.0 * (double)act_all) +
                  4.0 * (double)act_all;
    }
    if (int r = map_err(c, c->ctr_h->err, "lpa")) return r;
    c->hub_dirty = false;   // every hub's final pass reset the slots its pieces claimed
    const long long dn = (long long)c->ctr_h->dn;
    long long act = (long long)c->ctr_h->fast_active;
    for (int k = 0; k < NCLASS; ++k) act += (long long)(c->ctr_h->cls_count[k] + c->ctr_h->phase_cls[k]);
    scanned += (long long)c->ctr_h->scanned;
    if (st && t <= GSL_STATS_SWEEPS) {
      st->changed[t - 1] = dn;
      st->active[t - 1] = act;
    }
    marked_prev = a.mark != 0;
    dn_prev = dn;
    if ((double)dn / (double)n <= tol) {
      converged = true;
      break;
    }
  }
  if (st) {
    st->iterations = t;
    st->converged = converged ? 1 : 0;
    st->edges_scanned = scanned;
  }
  *final = async_mode ? c->lab[0] : c->lab[t & 1];
  return GSL_OK;
}

// The sweep loop with float32 weights and float64 sums (float_kernels.cu):
// the same frontier, stop test and statistics as run_lpa, without the
// integer-only devices (streaming first sweep, two-phase gathers, majority
// filter, hub pieces).
int run_lpa_f32(gsl_ctx* c, const gsl_csr* g, const float* wf, const int32_t* labels_init, double tol,
                int32_t max_iters, int32_t mode, gsl_stats* st, cudaStream_t s, int** final) {
  const long long n = g->n;
  const bool async_mode = mode == GSL_MODE_ASYNC;
  const long long maxd = c->ctr_h->max_degree;
  const long long region = 2 * (maxd > 0 ? maxd : 1);
  if (2 * maxd > 8192) {   // rows whose table does not fit shared memory
    const long long need = float_table_blocks(c->di) * region;
    if (int r = grow(c, c->fkeys, c->cap_fkeys, need)) return r;
    if (int r = grow(c, c->fvals, c->cap_fvals, need)) return r;
  }
  CK(cudaMemsetAsync(c->flag[0], 0, (size_t)n, s));
  CK(cudaMemsetAsync(c->flag[1], 0, (size_t)n, s));
  CK(launch_init_labels(labels_init, c->lab[0], async_mode ? nullptr : c->lab[1], n, c->ctr, c->di, s));
  SweepArgs a{};
  a.off = OFF(g);
  a.col = g->cols;
  a.ctr = c->ctr;
  a.probe_cap = c->tune.probe_cap;
  a.work = c->work;
  a.n = n;
  int t = 0;
  bool converged = false, marked_prev = false;
  long long dn_prev = n, scanned = 0;
  while (t < max_iters) {
    ++t;
    if (int r = reset_sweep_counters(c, s)) return r;
    bool all_active = t == 1 || !marked_prev;
    if (t == 1 && !async_mode && !labels_init) {
      // sweep 1 from the identity labels streams the strictly increasing
      // rows; the others (flagged in flag[1]) go through the table kernels
      if (int r = grow(c, c->rowbits, c->cap_rowbits, (g->nnz >> 5) + 1)) return r;
      const int pe = prof_begin(c, s);
      CK(launch_ident_stream_f32(OFF(g), n, g->cols, wf, g->nnz, c->rowbits, c->flag[1], c->lab[1], c->ctr, c->di,
                                 s));
      prof_end(c, pe, SL_IDENT, s, 3);
      c->profile.slot[SL_IDENT].vertices += n;
      c->profile.slot[SL_IDENT].entries += g->nnz;
      c->profile.slot[SL_IDENT].bytes += 8.0 * (double)g->nnz + 16.0 * (double)n;   // columns, weights
      all_active = false;
    }
    a.prev = async_mode ? c->lab[0] : c->lab[(t - 1) & 1];
    a.next = async_mode ? c->lab[0] : c->lab[t & 1];
    a.fnext = c->flag[(t + 1) & 1];
    a.check = t == 1 ? 1 : 0;
    a.mark = (t > 1 && 2 * dn_prev <= n) ? 1 : 0;
    // the own-label majority filter for classes 7 and 8, as in run_lpa
    const bool filter = !a.check && (c->tune.majority == 2 || (c->tune.majority == 1 && t >= 3));
    if (filter)
      if (int r = grow(c, c->work2, c->cap_work2, n)) return r;
    const int phases = async_mode ? 2 : 1;   // asynchronous sweeps in two phases, as in run_lpa
    for (int ph = 0; ph < phases; ++ph) {
      if (ph == 1) CK(launch_phase_reset(c->ctr, nullptr, s));
      {
        const int pe = prof_begin(c, s);
        CK(launch_bin(OFF(g), n, c->flag[t & 1], all_active ? 1 : 0, c->tune, c->work, c->ctr, c->di, s, nullptr,
                      nullptr, nullptr, async_mode ? ph : -1, (unsigned)t));
        prof_end(c, pe, SL_BIN, s, 1);
      }
      SweepArgs af = a;
      if (filter) {
        const int pe = prof_begin(c, s);
        CK(launch_majority_filter_f32(a, wf, c->work2, async_mode, c->di, s));
        prof_end(c, pe, SL_FILTER, s, 2);
        af.work = c->work2;
      }
      for (int k = 0; k < NCLASS; ++k) {
        const int pe = prof_begin(c, s);
        CK(launch_sweep_f32(k == CLS_WARP_L || k == CLS_BLOCK ? af : a, wf, k, async_mode, c->fkeys, c->fvals,
                            region, c->di, s));
        prof_end(c, pe, SL_SWEEP0 + k, s, 1);
      }
    }
    CK(cudaMemcpyAsync(c->ctr_h, c->ctr, offsetof(Counters, pad1), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (c->prof) {
      prof_resolve(c);
      // algorithmic bytes as in run_lpa: per processed vertex offsets,
      // worklist entry, own label and label write; per entry the column, the
      // neighbour's label and the float weight
      long long act_all = 0;
      for (int k = 0; k < NCLASS; ++k) {
        auto& sl = c->profile.slot[SL_SWEEP0 + k];
        const long long v = (long long)(c->ctr_h->cls_count[k] + c->ctr_h->phase_cls[k]);
        const long long e = (long long)c->ctr_h->cls_scanned[k];
        sl.vertices += v;
        sl.entries += e;
        sl.bytes += 20.0 * (double)v + 12.0 * (double)e;
        act_all += v;
      }
      if (filter) {   // the filter read every row of classes 7 and 8 (as in run_lpa)
        long long cls_e = 0, rows = (long long)c->ctr_h->fast_active;
        for (int k = 0; k < NCLASS; ++k) cls_e += (long long)c->ctr_h->cls_scanned[k];
        long long fe = (long long)c->ctr_h->scanned - cls_e;
        for (int k = CLS_WARP_L; k <= CLS_BLOCK; ++k) {
          fe += (long long)c->ctr_h->cls_scanned[k];
          rows += (long long)(c->ctr_h->cls_count[k] + c->ctr_h->phase_cls[k]);
        }
        auto& sf = c->profile.slot[SL_FILTER];
        sf.vertices += rows;
        sf.entries += fe;
        sf.bytes += 20.0 * (double)rows + 12.0 * (double)fe;
      }
      auto& sb = c->profile.slot[SL_BIN];
      sb.vertices += all_active ? n : act_all;
      sb.bytes += (all_active ? 0.0 : (double)n) + 16.0 * (double)(all_active ? n : act_all) + 4.0 * (double)act_all;
    }
    if (int r = map_err(c, c->ctr_h->err, "lpa_f32")) return r;
    const long long dn = (long long)c->ctr_h->dn;
    long long act = (long long)c->ctr_h->fast_active;
    for (int k = 0; k < NCLASS; ++k) act += (long long)(c->ctr_h->cls_count[k] + c->ctr_h->phase_cls[k]);
    scanned += (long long)c->ctr_h->scanned;
    if (st && t <= GSL_STATS_SWEEPS) {
      st->changed[t - 1] = dn;
      st->active[t - 1] = act;
    }
    marked_prev = a.mark != 0;
    dn_prev = dn;
    if ((double)dn / (double)n <= tol) {
      converged = true;
      break;
    }
  }
  if (st) {
    st->iterations = t;
    st->converged = converged ? 1 : 0;
    st->edges_scanned = scanned;
  }
  *final = async_mode ? c->lab[0] : c->lab[t & 1];
  return GSL_OK;
}

// Float weights that are all multiples of 2^-S with every row total below
// 2^(31-S) (checked through the largest weight and the largest degree) are
// converted to int32 w * 2^S (float_kernels.cu): the integer sweeps then
// compare the float path's exact float64 sums scaled by 2^S, so they give
// its labels.  Sets *wi to the converted weights, or leaves it NULL (float
// path) when the weights do not qualify or the context's mode is 0; invalid
// weights are left to the float path, which reports them.  After
// prepare_graph(g).
int f32_fixed_point(gsl_ctx* c, const gsl_csr* g, const float* w, cudaStream_t s, int** wi) {
  *wi = nullptr;
  if (c->f32_fixed == 0 || g->nnz == 0) return GSL_OK;
  CK(launch_f32_exact_scan(w, g->nnz, c->fix_dev, c->di, s));
  CK(cudaMemcpyAsync(c->fix_h, c->fix_dev, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (c->fix_h[2]) return GSL_OK;
  const int lo = c->fix_h[0] - 1024, hi = c->fix_h[1] - 1024;
  const int shift = lo < 0 ? -lo : 0;
  int dbits = 0;   // ceil(log2(largest degree))
  while ((1ll << dbits) < c->ctr_h->max_degree) ++dbits;
  // a weight is below 2^(hi+1), so a row total times 2^shift is below 2^(hi+1+shift+dbits)
  if (shift > 30 || hi + 1 + shift + dbits > 31) return GSL_OK;
  if (int r = grow(c, c->fix_w, c->cap_fix_w, g->nnz)) return r;
  CK(launch_f32_to_fixed(w, g->nnz, shift, c->fix_w, c->di, s));
  *wi = c->fix_w;
  return GSL_OK;
}

int run_split(gsl_ctx* c, const gsl_csr* g, const int32_t* labels_in, int32_t* labels_out, int32_t renumber,
              long long* k, cudaStream_t s) {
  const long long n = g->n;
  if (int r = reset_sweep_counters(c, s)) return r;
  int pe = prof_begin(c, s);
  CK(launch_bin(OFF(g), n, nullptr, 1, c->tune, c->work, c->ctr, c->di, s));
  prof_end(c, pe, SL_BIN, s, 1);
  c->profile.slot[SL_BIN].vertices += n;
  c->profile.slot[SL_BIN].bytes += 20.0 * (double)n;
  pe = prof_begin(c, s);
  // c->rank is free until the renumbering below: it holds the named pieces
  CK(launch_split(OFF(g), g->cols, n, labels_in, c->work, c->ctr, c->parent, c->rank, labels_out, c->tune, c->di,
                  s));
  prof_end(c, pe, SL_SPLIT, s, 17);
  // per vertex: parent init, own label, offsets, compress read and label
  // write; per entry: the column and, for the half with j < u, the label
  c->profile.slot[SL_SPLIT].vertices += n;
  c->profile.slot[SL_SPLIT].entries += g->nnz;
  c->profile.slot[SL_SPLIT].bytes += (4.0 + 4.0 + 8.0 + 4.0 + 4.0) * (double)n + 6.0 * (double)g->nnz;
  const long long nb = renumber_blocks(n);
  if (int r = grow(c, c->block_sums, c->cap_blocks, nb > 0 ? nb : 1)) return r;
  pe = prof_begin(c, s);
  if (renumber) {
    CK(launch_renumber(labels_out, labels_out, n, c->rank, c->block_sums, c->cap_blocks, c->k_dev, c->di, s));
  } else {
    // count the pieces (representatives) without renumbering
    CK(launch_renumber(labels_out, nullptr, n, c->rank, c->block_sums, c->cap_blocks, c->k_dev, c->di, s));
  }
  prof_end(c, pe, SL_COUNT, s, renumber ? 4 : 2);
  c->profile.slot[SL_COUNT].vertices += n;
  c->profile.slot[SL_COUNT].bytes += (renumber ? 4.0 * 4.0 : 4.0) * (double)n;
  CK(cudaMemcpyAsync(c->k_h, c->k_dev, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(c->ctr_h, c->ctr, offsetof(Counters, pad1), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  prof_resolve(c);
  if (int r = map_err(c, c->ctr_h->err, "split")) return r;
  *k = (long long)*c->k_h;
  return GSL_OK;
}

int run_modularity(gsl_ctx* c, const gsl_csr* g, const int32_t* weights, const int32_t* labels, double* q,
                   cudaStream_t s) {
  const long long n = g->n;
  if (int r = grow(c, c->sigma, c->cap_sigma, n)) return r;
  const long long np = modularity_partials(c->di);
  if (int r = grow(c, c->partials, c->cap_partials, 2 * np)) return r;
  CK(cudaMemsetAsync(c->sigma, 0, sizeof(unsigned long long) * (size_t)n, s));
  CK(cudaMemsetAsync(c->sums, 0, sizeof(ModSums), s));
  if (int r = reset_sweep_counters(c, s)) return r;
  CK(launch_bin(OFF(g), n, nullptr, 1, c->tune, c->work, c->ctr, c->di, s));
  const int pe = prof_begin(c, s);
  CK(launch_modularity(OFF(g), g->cols, weights, n, labels, c->work, c->ctr, c->sigma, c->partials, np, c->sums,
                       c->tune, c->di, s));
  prof_end(c, pe, SL_MOD, s, 13);
  // per vertex: offsets, label, Sigma update (read+write) and square pass;
  // per entry: column, neighbour label and weight
  c->profile.slot[SL_MOD].vertices += n;
  c->profile.slot[SL_MOD].entries += g->nnz;
  c->profile.slot[SL_MOD].bytes += (8.0 + 4.0 + 16.0 + 8.0) * (double)n + (8.0 + (weights ? 4.0 : 0.0)) * (double)g->nnz;
  CK(cudaMemcpyAsync(c->sums_h, c->sums, sizeof(ModSums), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(c->ctr_h, c->ctr, offsetof(Counters, pad1), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  prof_resolve(c);
  if (int r = map_err(c, c->ctr_h->err, "modularity")) return r;
  const ModSums& m = *c->sums_h;
  if (m.two_m == 0) {
    *q = 0.0;
    return GSL_OK;
  }
  const unsigned __int128 s2 = ((unsigned __int128)m.s2_hi << 64) | m.s2_lo;
  const double dm = (double)m.two_m;
  *q = (double)m.s1 / dm - (double)s2 / (dm * dm);
  return GSL_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

int check_lpa_args(gsl_ctx* c, const gsl_csr* g, double tol, int32_t max_iters, int32_t mode, const void* out) {
  if (int r = check_csr(c, g)) return r;
  if (!(tol >= 0.0)) return fail(c, GSL_ERR_INVALID, "tolerance must be >= 0");
  if (max_iters < 0) return fail(c, GSL_ERR_INVALID, "max_iters must be >= 0");
  if (mode != GSL_MODE_SYNC && mode != GSL_MODE_ASYNC) return fail(c, GSL_ERR_INVALID, "unknown mode %d", mode);
  if (g->n > 0 && !out) return fail(c, GSL_ERR_INVALID, "labels_out is NULL");
  return GSL_OK;
}

// Enqueues the batched sweep loop (max_iters sweeps, unrolled, each
// returning at once after every graph has stopped) and the final label
// gather on stream cs, without synchronising: used under stream capture and
// for direct launches.  prepare_graph, the vptr/gid upload and the per-graph
// state reset must have been enqueued before.
cudaError_t enqueue_batch_sweeps(gsl_ctx* c, const gsl_csr* g, int num_graphs, const int32_t* weights, double tol,
                                 int max_iters, bool async_mode, cudaStream_t cs) {
  const long long n = g->n;
  cudaError_t cerr = cudaSuccess;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && cerr == cudaSuccess) cerr = e;
  };
  ck(cudaMemsetAsync(c->flag[0], 0, (size_t)n, cs));
  ck(cudaMemsetAsync(c->flag[1], 0, (size_t)n, cs));
  ck(launch_init_labels(nullptr, c->lab[0], async_mode ? nullptr : c->lab[1], n, c->ctr, c->di, cs));
  SweepArgs a{};
  a.off = OFF(g);
  a.col = g->cols;
  a.w = weights;
  a.ctr = c->ctr;
  a.probe_cap = c->tune.probe_cap;
  a.work = c->work;
  a.wtab = c->wtab;
  a.wtab_region = 2ll * c->tune.warp_max;
  a.btab = c->btab;
  a.btab_region = 2ll * c->ctr_h->max_degree;
  a.n = n;
  a.gid = c->gid;
  a.vptr = c->vptr;
  a.dn_graph = c->dn_graph;
  a.stop = c->stop;
  for (int t = 1; t <= max_iters; ++t) {
    ck(cudaMemsetAsync(c->ctr, 0, offsetof(Counters, err), cs));
    ck(cudaMemsetAsync(c->dn_graph, 0, sizeof(unsigned) * (size_t)num_graphs, cs));
    // per-slot profiling only when launching directly (not inside a capture)
    const bool prof = c->prof && c->batch_direct;
    int pe = -1;
    a.prev = async_mode ? c->lab[0] : c->lab[(t - 1) & 1];
    a.next = async_mode ? c->lab[0] : c->lab[t & 1];
    a.fnext = c->flag[(t + 1) & 1];
    a.ident = (!async_mode && t == 1) ? 1 : 0;
    a.check = t == 1 ? 1 : 0;
    a.mark = t >= 2 ? 1 : 0;   // sweep 2 runs on all vertices, later ones on the marked frontier
    const bool filter = !a.ident && !a.check && (c->tune.majority == 2 || (c->tune.majority == 1 && t >= 3));
    const int filter_from = (filter && t >= BATCH_FILTER6_FROM) ? CLS_WARP_S : CLS_WARP_L;
    a.gthresh = (t == 2 && !async_mode) ? 3 * c->tune.blk_slots : 0;
    a.spread = (t == 2 && !async_mode) ? 1 : 0;
    const int phases = async_mode ? 2 : 1;   // asynchronous sweeps in two phases, as in run_lpa
    for (int ph = 0; ph < phases; ++ph) {
      if (ph == 1) ck(launch_phase_reset(c->ctr, c->stop, cs));
      pe = prof ? prof_begin(c, cs) : -1;
      ck(launch_bin(OFF(g), n, c->flag[t & 1], t <= 2 ? 1 : 0, c->tune, c->work, c->ctr, c->di, cs, c->gid, c->done,
                    c->stop, async_mode ? ph : -1, (unsigned)t));
      if (prof) prof_end(c, pe, SL_BIN, cs, 1);
      SweepArgs af = a;
      if (filter) {
        pe = prof ? prof_begin(c, cs) : -1;
        ck(launch_majority_filter(a, c->work2, weights != nullptr, async_mode, c->di, cs, filter_from));
        if (prof) prof_end(c, pe, SL_FILTER, cs, 2);
        af.work = c->work2;
      }
      for (int k = 0; k < NCLASS; ++k) {
        pe = prof ? prof_begin(c, cs) : -1;
        const bool filtered = k == CLS_WARP_L || k == CLS_BLOCK || (k == CLS_WARP_S && filter_from == CLS_WARP_S);
        ck(launch_sweep_class(filtered ? af : a, k, weights != nullptr, async_mode, c->tune, c->di, cs));
        if (prof) prof_end(c, pe, SL_SWEEP0 + k, cs, 1);
      }
    }
    ck(launch_graph_update(t, tol, max_iters, c->vptr, num_graphs, c->dn_graph, c->iters, c->done, c->stop, cs));
  }
  const int* bufs[2] = {c->lab[0], c->lab[1]};
  ck(launch_batch_final(bufs, c->iters, c->gid, n, async_mode ? 1 : 0, c->lab_tmp, c->di, cs));
  return cerr;
}

}  // namespace

extern "C" {

int gsl_version(void) { return 100; }

const char* gsl_strerror(int code) {
  switch (code) {
    case GSL_OK: return "ok";
    case GSL_ERR_INVALID: return "invalid argument or malformed input";
    case GSL_ERR_OVERFLOW: return "weighted degree overflows int32";
    case GSL_ERR_NOMEM: return "out of memory";
    case GSL_ERR_CUDA: return "CUDA error";
    case GSL_ERR_TIMEOUT: return "device retry bound reached";
    default: return "unknown error";
  }
}

const char* gsl_ctx_last_error(gsl_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

int gsl_ctx_create(gsl_ctx** out, int device) {
  if (!out) return GSL_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return GSL_ERR_CUDA;
  }
  gsl_ctx* c = new gsl_ctx();
  c->device = device;
  DeviceGuard dg(device);
  cudaDeviceGetAttribute(&c->di.sm_count, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&c->di.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  bool ok = cudaMalloc(&c->ctr, sizeof(Counters)) == cudaSuccess &&
            cudaMallocHost(&c->ctr_h, sizeof(Counters)) == cudaSuccess &&
            cudaMalloc(&c->sums, sizeof(ModSums)) == cudaSuccess &&
            cudaMallocHost(&c->sums_h, sizeof(ModSums)) == cudaSuccess &&
            cudaMalloc(&c->k_dev, sizeof(unsigned long long)) == cudaSuccess &&
            cudaMallocHost(&c->k_h, sizeof(unsigned long long)) == cudaSuccess &&
            cudaMalloc(&c->fix_dev, 3 * sizeof(int)) == cudaSuccess &&
            cudaMallocHost(&c->fix_h, 3 * sizeof(int)) == cudaSuccess;
  for (int i = 0; ok && i < 4; ++i) ok = cudaEventCreate(&c->ev[i]) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    gsl_ctx_destroy(c);
    return GSL_ERR_NOMEM;
  }
  memset(c->ctr_h, 0, sizeof(Counters));
  *out = c;
  return GSL_OK;
}

int gsl_ctx_destroy(gsl_ctx* c) {
  if (!c) return GSL_OK;
  DeviceGuard dg(c->device);
  void* dptrs[] = {c->lab[0], c->lab[1], c->flag[0], c->flag[1], c->work, c->parent, c->rank, c->sigma,
                   c->block_sums, c->partials, c->wtab, c->btab, c->rowbits, c->lg, c->work2, c->fkeys, c->fvals, c->hub_piece_start,
                   c->hub_ustart, c->hub_best, c->hub_own, c->hub_wsum, c->hub_used_cnt, c->hub_clu, c->hub_used, c->hub_tab,
                   c->ctr, c->sums, c->k_dev,
                   c->st_off, c->st_col, c->st_w, c->st_lab, c->fix_w, c->fix_dev, c->kw};
  for (void* p : dptrs)
    if (p) cudaFree(p);
  if (c->ctr_h) cudaFreeHost(c->ctr_h);
  if (c->sums_h) cudaFreeHost(c->sums_h);
  if (c->k_h) cudaFreeHost(c->k_h);
  if (c->fix_h) cudaFreeHost(c->fix_h);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->evpool) cudaEventDestroy(e);
  for (auto& e : c->chunk_ev) cudaEventDestroy(e);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  void* bptrs[] = {c->gid, c->vptr, c->dn_graph, c->iters, c->done, c->stop, c->lab_tmp};
  for (void* p : bptrs)
    if (p) cudaFree(p);
  delete c;
  return GSL_OK;
}

int gsl_ctx_set_tuning(gsl_ctx* c, int32_t warp_max, int32_t blk_max) {
  if (!c) return GSL_ERR_INVALID;
  if (warp_max < 32 || warp_max > (1 << 20) || blk_max < warp_max)
    return fail(c, GSL_ERR_INVALID, "need 32 <= warp_max <= 2^20 and blk_max >= warp_max");
  c->tune.warp_max = warp_max;
  c->tune.blk_max = blk_max;
  return GSL_OK;
}

}  // extern "C"

// Candidate settings of the autotuners, for a graph with the given sorted
// degrees.  Two settings are the same run when they bin every vertex alike
// and agree on every knob that acts on the classes the graph populates:
// the block shape only matters with rows above warp_max, the majority
// filter only with rows in classes 7-8 (warp_small+1 .. blk_max).
namespace {
struct TuneSpace {
  bool pregather;   // also try two-phase sweeps
};

long long count_le(const std::vector<long long>& deg_sorted, long long x) {
  return (long long)(std::upper_bound(deg_sorted.begin(), deg_sorted.end(), x) - deg_sorted.begin());
}

bool same_run(const std::vector<long long>& deg_sorted, const gsl::Tuning& a, const gsl::Tuning& b) {
  const gsl::ClassBounds ca = gsl::class_bounds(a), cb = gsl::class_bounds(b);
  const long long n = (long long)deg_sorted.size();
  if (count_le(deg_sorted, ca.warp_small) != count_le(deg_sorted, cb.warp_small) ||
      count_le(deg_sorted, ca.warp_max) != count_le(deg_sorted, cb.warp_max) ||
      count_le(deg_sorted, ca.blk_max) != count_le(deg_sorted, cb.blk_max))
    return false;
  if (a.pregather != b.pregather) return false;
  const bool block_rows = count_le(deg_sorted, ca.warp_max) < n;
  if (block_rows && (a.blk_block != b.blk_block || a.blk_slots != b.blk_slots)) return false;
  const bool filter_rows = count_le(deg_sorted, ca.blk_max) > count_le(deg_sorted, ca.warp_small);
  if (filter_rows && a.majority != b.majority) return false;
  return true;
}

std::vector<gsl::Tuning> tune_candidates(const std::vector<long long>& deg_sorted, const gsl::Tuning& entry,
                                         const TuneSpace& sp, int max_smem) {
  std::vector<gsl::Tuning> cand{entry};
  const int shapes[2][2] = {{512, 12288}, {256, 6144}};
  for (int pg : {0, 1}) {
    if (pg && !sp.pregather) continue;
    for (int maj : {1, 0, 2})
      for (const auto& sh : shapes) {
        if ((long long)sh[1] * 8 + 1024 > max_smem) continue;
        for (int wm : {128, 256, 512, 1024})
          for (int bm : {4096, 12288, 32768, 131072}) {
            if (bm < wm) continue;
            gsl::Tuning t = entry;
            t.warp_max = wm;
            t.blk_max = bm;
            t.pregather = pg;
            t.majority = maj;
            t.blk_block = sh[0];
            t.blk_slots = sh[1];
            bool dup = false;
            for (const gsl::Tuning& u : cand) dup = dup || same_run(deg_sorted, t, u);
            if (!dup) cand.push_back(t);
          }
      }
  }
  return cand;
}

// Sorted degrees of a device CSR (host copy of the offsets).
int sorted_degrees(gsl_ctx* c, const gsl_csr* g, cudaStream_t s, std::vector<long long>* deg) {
  std::vector<long long> offs((size_t)g->n + 1);
  CK(cudaMemcpyAsync(offs.data(), g->offsets, sizeof(int64_t) * offs.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  deg->resize((size_t)g->n);
  for (long long v = 0; v < g->n; ++v) (*deg)[(size_t)v] = offs[(size_t)v + 1] - offs[(size_t)v];
  std::sort(deg->begin(), deg->end());
  return GSL_OK;
}

void fill_result(const gsl::Tuning& t, gsl_tune_result* out) {
  out->warp_max = t.warp_max;
  out->blk_max = t.blk_max;
  out->pregather = t.pregather;
  out->majority = t.majority;
  out->blk_threads = t.blk_block;
  out->blk_slots = t.blk_slots;
}

// Times every candidate with time_one (an untimed warm-up run of the entry
// setting first) and leaves the fastest on the context; on error the entry
// setting is restored.
template <typename F>
int tune_loop(gsl_ctx* c, const std::vector<gsl::Tuning>& cand, gsl_tune_result* out, F&& time_one) {
  const gsl::Tuning entry = c->tune;
  float ms = 0.f, best_ms = 0.f;
  int best = 0;
  for (size_t k = 0; k < cand.size(); ++k) {
    if (k == 0) {
      if (int r = time_one(cand[0], &ms)) {
        c->tune = entry;
        return r;
      }
    }
    if (int r = time_one(cand[k], &ms)) {
      c->tune = entry;
      return r;
    }
    if (k == 0) out->entry_ms = ms;
    if (k == 0 || ms < best_ms) {
      best_ms = ms;
      best = (int)k;
    }
  }
  c->tune = cand[(size_t)best];
  c->batch_key.clear();
  fill_result(c->tune, out);
  out->candidates = (int32_t)cand.size();
  out->best_ms = best_ms;
  return GSL_OK;
}
}  // namespace

extern "C" {

int gsl_autotune(gsl_ctx* c, const gsl_csr* g, const int32_t* weights, int32_t mode, int32_t sweeps,
                 gsl_tune_result* out, void* stream) {
  if (!c) return GSL_ERR_INVALID;
  c->last_error.clear();
  if (!out) return fail(c, GSL_ERR_INVALID, "out is NULL");
  if (sweeps < 1 || sweeps > GSL_STATS_SWEEPS) return fail(c, GSL_ERR_INVALID, "need 1 <= sweeps <= 64");
  if (int r = check_csr(c, g)) return r;
  if (mode != GSL_MODE_SYNC && mode != GSL_MODE_ASYNC) return fail(c, GSL_ERR_INVALID, "unknown mode");
  memset(out, 0, sizeof(*out));
  fill_result(c->tune, out);
  out->sweeps = sweeps;
  if (g->n == 0) return GSL_OK;
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (int r = ensure_vertex_scratch(c, g->n)) return r;
  std::vector<long long> deg;
  if (int r = sorted_degrees(c, g, s, &deg)) return r;
  const std::vector<Tuning> cand = tune_candidates(deg, c->tune, TuneSpace{true}, c->di.max_smem_optin);
  return tune_loop(c, cand, out, [&](const Tuning& t, float* ms) -> int {
    c->tune = t;
    if (int r = prepare_graph(c, g, s)) return r;
    int* fin = nullptr;
    CK(cudaEventRecord(c->ev[0], s));
    if (int r = run_lpa(c, g, weights, nullptr, 0.0, sweeps, mode, nullptr, s, &fin)) return r;
    CK(cudaEventRecord(c->ev[1], s));
    CK(cudaEventSynchronize(c->ev[1]));
    CK(cudaEventElapsedTime(ms, c->ev[0], c->ev[1]));
    return GSL_OK;
  });
}

int gsl_autotune_batch(gsl_ctx* c, const gsl_csr* g, int32_t num_graphs, const int64_t* vptr_host,
                       const int32_t* weights, double tol, int32_t max_iters, int32_t mode, int32_t* labels_out,
                       gsl_tune_result* out, void* stream) {
  if (!c) return GSL_ERR_INVALID;
  c->last_error.clear();
  if (!out) return fail(c, GSL_ERR_INVALID, "out is NULL");
  if (int r = check_lpa_args(c, g, tol, max_iters, mode, labels_out)) return r;
  if (num_graphs < 1 || !vptr_host) return fail(c, GSL_ERR_INVALID, "need num_graphs >= 1 and vptr");
  memset(out, 0, sizeof(*out));
  fill_result(c->tune, out);
  out->sweeps = max_iters;
  if (g->n == 0) return GSL_OK;
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<long long> deg;
  if (int r = sorted_degrees(c, g, s, &deg)) return r;
  // the batched loop has no two-phase mode
  const std::vector<Tuning> cand = tune_candidates(deg, c->tune, TuneSpace{false}, c->di.max_smem_optin);
  return tune_loop(c, cand, out, [&](const Tuning& t, float* ms) -> int {
    c->tune = t;
    c->batch_key.clear();
    // first call captures the sweep loop for this setting; the second, timed, replays it
    for (int rep = 0; rep < 2; ++rep) {
      gsl_batch_stats st{};
      if (int r = gsl_gsllpa_batch(c, g, num_graphs, vptr_host, weights, tol, max_iters, mode, labels_out, nullptr,
                                   &st, stream))
        return r;
      *ms = st.ms;
    }
    return GSL_OK;
  });
}

int gsl_ctx_set_block_config(gsl_ctx* c, int32_t threads, int32_t table_slots) {
  if (!c) return GSL_ERR_INVALID;
  if (threads != 128 && threads != 256 && threads != 512)
    return fail(c, GSL_ERR_INVALID, "block threads must be 128, 256 or 512");
  const long long bytes = (long long)table_slots * 8 + 1024;   // + the kernel's static shared memory
  if (table_slots < 16 * threads || bytes > c->di.max_smem_optin)
    return fail(c, GSL_ERR_INVALID, "table_slots must be >= 16 * threads and fit the shared memory of one block");
  c->tune.blk_block = threads;
  c->tune.blk_slots = table_slots;
  c->batch_key.clear();   // the captured batched loop used the old shape
  return GSL_OK;
}

int gsl_ctx_set_majority(gsl_ctx* c, int32_t mode) {
  if (!c) return GSL_ERR_INVALID;
  if (mode < 0 || mode > 2) return fail(c, GSL_ERR_INVALID, "majority mode must be 0, 1 or 2");
  c->tune.majority = mode;
  c->batch_key.clear();
  return GSL_OK;
}

int gsl_ctx_set_f32_fixed(gsl_ctx* c, int32_t mode) {
  if (!c) return GSL_ERR_INVALID;
  if (mode < 0 || mode > 1) return fail(c, GSL_ERR_INVALID, "f32 fixed-point mode must be 0 or 1");
  c->f32_fixed = mode;
  return GSL_OK;
}

int gsl_ctx_set_hub_cluster(gsl_ctx* c, int64_t max_degree) {
  if (!c) return GSL_ERR_INVALID;
  if (max_degree < 0) return fail(c, GSL_ERR_INVALID, "hub cluster degree must be >= 0");
  c->tune.hub_cluster_max = max_degree > (1ll << 30) ? (1 << 30) : (int)max_degree;
  return GSL_OK;
}

int gsl_ctx_set_retry_bounds(gsl_ctx* c, int32_t probe_bound, int32_t unionfind_bound) {
  if (!c) return GSL_ERR_INVALID;
  if (probe_bound < 0 || unionfind_bound < 0) return fail(c, GSL_ERR_INVALID, "retry bounds must be >= 0");
  const Tuning d;
  c->tune.probe_cap = probe_bound ? probe_bound : d.probe_cap;
  c->tune.uf_cap = unionfind_bound ? unionfind_bound : d.uf_cap;
  c->batch_key.clear();   // the captured batched loop holds the old bound
  return GSL_OK;
}

int gsl_ctx_set_pregather(gsl_ctx* c, int32_t mode) {
  if (!c) return GSL_ERR_INVALID;
  if (mode < 0 || mode > 2) return fail(c, GSL_ERR_INVALID, "pregather mode must be 0, 1 or 2");
  c->tune.pregather = mode;
  return GSL_OK;
}

int gsl_ctx_set_batch_mode(gsl_ctx* c, int32_t use_cuda_graph) {
  if (!c) return GSL_ERR_INVALID;
  c->batch_direct = use_cuda_graph == 0;
  return GSL_OK;
}

int gsl_ctx_set_profiling(gsl_ctx* c, int32_t enable) {
  if (!c) return GSL_ERR_INVALID;
  c->prof = enable != 0;
  memset(&c->profile, 0, sizeof(c->profile));
  c->pending.clear();
  c->ev_used = 0;
  return GSL_OK;
}

int gsl_ctx_get_profile(gsl_ctx* c, gsl_profile* out) {
  if (!c || !out) return GSL_ERR_INVALID;
  *out = c->profile;
  out->nslots = SL_N;
  for (int k = 0; k < SL_N; ++k) {
    strncpy(out->slot[k].name, slot_name(k), sizeof(out->slot[k].name) - 1);
    out->slot[k].name[sizeof(out->slot[k].name) - 1] = 0;
  }
  return GSL_OK;
}

int64_t gsl_kernel_launches(void) { return launches_total(); }

int gsl_lpa(gsl_ctx* c, const gsl_csr* g, const int32_t* weights, const int32_t* labels_init, double tol,
            int32_t max_iters, int32_t mode, int32_t* labels_out, gsl_stats* st, void* stream) {
  if (!c) return GSL_ERR_INVALID;
  c->last_error.clear();
  if (int r = check_lpa_args(c, g, tol, max_iters, mode, labels_out)) return r;
  if (st) memset(st, 0, sizeof(*st));
  if (g->n == 0) return GSL_OK;
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (int r = ensure_vertex_scratch(c, g->n)) return r;
  CK(cudaEventRecord(c->ev[0], s));
  if (int r = prepare_graph(c, g, s)) return r;
  int* fin = nullptr;
  if (int r = run_lpa(c, g, weights, labels_init, tol, max_iters, mode, st, s, &fin)) return r;
  CK(cudaMemcpyAsync(labels_out, fin, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToDevice, s));
  CK(cudaEventRecord(c->ev[1], s));
  CK(cudaEventSynchronize(c->ev[1]));
  if (st) cudaEventElapsedTime(&st->ms_lpa, c->ev[0], c->ev[1]);
  return GSL_OK;
}

int gsl_lpa_f32(gsl_ctx* c, const gsl_csr* g, const float* weights, const int32_t* labels_init, double tol,
                int32_t max_iters, int32_t mode, int32_t* labels_out, gsl_stats* st, void* stream) {
  if (!c) return GSL_ERR_INVALID;
  c->last_error.clear();
  if (int r = check_lpa_args(c, g, tol, max_iters, mode, labels_out)) return r;
  if (g->nnz > 0 && !weights) return fail(c, GSL_ERR_INVALID, "weights is NULL");
  if (st) memset(st, 0, sizeof(*st));
  if (g->n == 0) return GSL_OK;
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (int r = ensure_vertex_scratch(c, g->n)) return r;
  CK(cudaEventRecord(c->ev[0], s));
  if (int r = prepare_graph(c, g, s)) return r;
  int* wi = nullptr;
  if (int r = f32_fixed_point(c, g, weights, s, &wi)) return r;
  int* fin = nullptr;
  if (wi) {
    if (int r = run_lpa(c, g, wi, labels_init, tol, max_iters, mode, st, s, &fin)) return r;
  } else {
    if (int r = run_lpa_f32(c, g, weights, labels_init, tol, max_iters, mode, st, s, &fin)) return r;
  }
  CK(cudaMemcpyAsync(labels_out, fin, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToDevice, s));
  CK(cudaEventRecord(c->ev[1], s));
  CK(cudaEventSynchronize(c->ev[1]));
  if (st) cudaEventElapsedTime(&st->ms_lpa, c->ev[0], c->ev[1]);
  return GSL_OK;
}

int gsl_gsllpa_f32(gsl_ctx* c, const gsl_csr* g, const float* weights, double tol, int32_t max_iters, int32_t mode,
                   int32_t* labels_out, gsl_stats* st, void* stream) {
  if (!c) return GSL_ERR_INVALID;
  c->last_error.clear();
  if (int r = check_lpa_args(c, g, tol, max_iters, mode, labels_out)) return r;
  if (g->nnz > 0 && !weights) return fail(c, GSL_ERR_INVALID, "weights is NULL");
  if (st) memset(st, 0, sizeof(*st));
  if (g->n == 0) return GSL_OK;
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (int r = ensure_vertex_scratch(c, g->n)) return r;
  CK(cudaEventRecord(c->ev[0], s));
  if (int r = prepare_graph(c, g, s)) return r;
  int* wi = nullptr;
  if (int r = f32_fixed_point(c, g, weights, s, &wi)) return r;
  int* fin = nullptr;
  if (wi) {
    if (int r = run_lpa(c, g, wi, nullptr, tol, max_iters, mode, st, s, &fin)) return r;
  } else {
    if (int r = run_lpa_f32(c, g, weights, nullptr, tol, max_iters, mode, st, s, &fin)) return r;
  }
  CK(cudaEventRecord(c->ev[1], s));
  long long k = 0;
  if (int r = run_split(c, g, fin, labels_out, 0, &k, s)) return r;
  CK(cudaEventRecord(c->ev[2], s));
  CK(cudaEventSynchronize(c->ev[2]));
  if (st) {
    cudaEventElapsedTime(&st->ms_lpa, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&st->ms_split, c->ev[1], c->ev[2]);
    st->communities = k;
  }
  return GSL_OK;
}

int gsl_modularity_f32(gsl_ctx* c, const gsl_csr* g, const float* weights, const int32_t* labels, double* q_out,
                       void* stream) {
  if (!c) return GSL_ERR_INVALID;
  c->last_error.clear();
  if (int r = check_csr(c, g)) return r;
  if (!q_out) return fail(c, GSL_ERR_INVALID, "q_out is NULL");
  if (g->n > 0 && !labels) return fail(c, GSL_ERR_INVALID, "labels is NULL");
  if (g->nnz > 0 && !weights) return fail(c, GSL_ERR_INVALID, "weights is NULL");
  *q_out = 0.0;
  if (g->n == 0) return GSL_OK;
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (int r = ensure_vertex_scratch(c, g->n)) return r;
  if (int r = prepare_graph(c, g, s)) return r;
  if (int r = grow(c, c->sigma, c->cap_sigma, g->n)) return r;   // n doubles (8 bytes, as the u64 sums)
  double* sums = reinterpret_cast<double*>(c->sums);
  CK(launch_modularity_f32(OFF(g), g->cols, weights, labels, g->n, reinterpret_cast<double*>(c->sigma), sums, c->ctr,
                           c->di, s));
  double h[3];
  CK(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(c->ctr_h, c->ctr, offsetof(Counters, pad1), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (int r = map_err(c, c->ctr_h->err, "modularity_f32")) return r;
  *q_out = h[0] == 0.0 ? 0.0 : h[1] / h[0] - h[2] / (h[0] * h[0]);
  return GSL_OK;
}

int gsl_split(gsl_ctx* c, const gsl_csr* g, const int32_t* labels_in, int32_t* labels_out, int32_t renumber,
              int64_t* k_out, void* stream) {
  if (!c) return GSL_ERR_INVALID;
  c->last_error.clear();
  if (int r = check_csr(c, g)) return r;
  if (g->n > 0 && (!labels_in || !labels_out)) return fail(c, GSL_ERR_INVALID, "labels pointer is NULL");
  if (renumber != 0 && renumber != 1) return fail(c, GSL_ERR_INVALID, "renumber must be 0 or 1");
  if (g->n == 0) {
    if (k_out) *k_out = 0;
    return GSL_OK;
  }
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (int r = ensure_vertex_scratch(c, g->n)) return r;
  if (int r = prepare_graph(c, g, s)) return r;
  long long k = 0;
  if (int r = run_split(c, g, labels_in, labels_out, renumber, &k, s)) return r;
  if (k_out) *k_out = k;
  return GSL_OK;
}

int gsl_split_lp(gsl_ctx* c, const gsl_csr* g, const int32_t* labels_in, int32_t* labels_out, int32_t pruning,
                 int32_t* sweeps_out, void* stream) {
  if (!c) return GSL_ERR_INVALID;
  c->last_error.clear();
  if (int r = check_csr(c, g)) return r;
  if (g->n > 0 && (!labels_in || !labels_out)) return fail(c, GSL_ERR_INVALID, "labels pointer is NULL");
  if (g->n > 0 && labels_in == labels_out) return fail(c, GSL_ERR_INVALID, "labels_out must not overlap labels_in");
  if (pruning != 0 && pruning != 1) return fail(c, GSL_ERR_INVALID, "pruning must be 0 or 1");
  if (sweeps_out) *sweeps_out = 0;
  if (g->n == 0) return GSL_OK;
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = g->n;
  if (int r = ensure_vertex_scratch(c, n)) return r;
  if (int r = prepare_graph(c, g, s)) return r;   // validates the offsets
  CK(launch_split_lp_init(labels_out, pruning ? c->flag[0] : nullptr, n, c->di, s));
  if (pruning) CK(cudaMemsetAsync(c->flag[1], 0, (size_t)n, s));
  int t = 0;
  for (;;) {
    if (t > n) return fail(c, GSL_ERR_TIMEOUT, "split_lp: no fixed point after n + 1 sweeps");
    ++t;
    if (int r = reset_sweep_counters(c, s)) return r;
    const int pe = prof_begin(c, s);
    CK(launch_split_lp_sweep(OFF(g), g->cols, labels_in, n, labels_out, c->flag[(t - 1) & 1], c->flag[t & 1],
                             pruning, c->ctr, c->di, s));
    prof_end(c, pe, SL_SPLIT, s, 1);
    CK(cudaMemcpyAsync(c->ctr_h, c->ctr, offsetof(Counters, pad1), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    prof_resolve(c);
    if (int r = map_err(c, c->ctr_h->err, "split_lp")) return r;
    if (c->ctr_h->dn == 0) break;
  }
  if (sweeps_out) *sweeps_out = t;
  return GSL_OK;
}

int gsl_disconnected(gsl_ctx* c, const gsl_csr* g, const int32_t* labels, uint8_t* flags_out, int64_t* count_out,
                     void* stream) {
  if (!c) return GSL_ERR_INVALID;
  c->last_error.clear();
  if (int r = check_csr(c, g)) return r;
  if (!count_out) return fail(c, GSL_ERR_INVALID, "count_out is NULL");
  if (g->n > 0 && !labels) return fail(c, GSL_ERR_INVALID, "labels is NULL");
  *count_out = 0;
  if (g->n == 0) return GSL_OK;
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = g->n;
  if (int r = ensure_vertex_scratch(c, n)) return r;
  if (int r = prepare_graph(c, g, s)) return r;
  long long k = 0;
  if (int r = run_split(c, g, labels, c->lab[0], 0, &k, s)) return r;
  CK(launch_disconnected(c->lab[0], labels, n, c->lab[1], flags_out, c->k_dev, c->ctr, c->di, s));
  CK(cudaMemcpyAsync(c->k_h, c->k_dev, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(c->ctr_h, c->ctr, offsetof(Counters, pad1), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (int r = map_err(c, c->ctr_h->err, "disconnected")) return r;
  *count_out = (int64_t)*c->k_h;
  return GSL_OK;
}

int gsl_modularity(gsl_ctx* c, const gsl_csr* g, const int32_t* weights, const int32_t* labels, double* q_out,
                   void* stream) {
  if (!c) return GSL_ERR_INVALID;
  c->last_error.clear();
  if (int r = check_csr(c, g)) return r;
  if (!q_out) return fail(c, GSL_ERR_INVALID, "q_out is NULL");
  if (g->n > 0 && !labels) return fail(c, GSL_ERR_INVALID, "labels is NULL");
  *q_out = 0.0;
  if (g->n == 0) return GSL_OK;
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (int r = ensure_vertex_scratch(c, g->n)) return r;
  if (int r = prepare_graph(c, g, s)) return r;
  return run_modularity(c, g, weights, labels, q_out, s);
}

int gsl_gsllpa(gsl_ctx* c, const gsl_csr* g, const int32_t* weights, double tol, int32_t max_iters, int32_t mode,
               int32_t* labels_out, gsl_stats* st, void* stream) {
  if (!c) return GSL_ERR_INVALID;
  c->last_error.clear();
  if (int r = check_lpa_args(c, g, tol, max_iters, mode, labels_out)) return r;
  if (st) memset(st, 0, sizeof(*st));
  if (g->n == 0) return GSL_OK;
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (int r = ensure_vertex_scratch(c, g->n)) return r;
  CK(cudaEventRecord(c->ev[0], s));
  if (int r = prepare_graph(c, g, s)) return r;
  int* fin = nullptr;
  if (int r = run_lpa(c, g, weights, nullptr, tol, max_iters, mode, st, s, &fin)) return r;
  CK(cudaEventRecord(c->ev[1], s));
  long long k = 0;
  if (int r = run_split(c, g, fin, labels_out, 0, &k, s)) return r;
  CK(cudaEventRecord(c->ev[2], s));
  CK(cudaEventSynchronize(c->ev[2]));
  if (st) {
    cudaEventElapsedTime(&st->ms_lpa, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&st->ms_split, c->ev[1], c->ev[2]);
    st->communities = k;
  }
  return GSL_OK;
}

int gsl_gsllpa_batch(gsl_ctx* c, const gsl_csr* g, int32_t num_graphs, const int64_t* vptr_host,
                     const int32_t* weights, double tol, int32_t max_iters, int32_t mode, int32_t* labels_out,
                     int32_t* iterations_out, gsl_batch_stats* st, void* stream) {
  if (!c) return GSL_ERR_INVALID;
  c->last_error.clear();
  if (int r = check_lpa_args(c, g, tol, max_iters, mode, labels_out)) return r;
  if (num_graphs < 1 || !vptr_host) return fail(c, GSL_ERR_INVALID, "need num_graphs >= 1 and vptr");
  if (vptr_host[0] != 0 || vptr_host[num_graphs] != g->n)
    return fail(c, GSL_ERR_INVALID, "vptr must start at 0 and end at n");
  for (int k = 0; k < num_graphs; ++k)
    if (vptr_host[k + 1] < vptr_host[k]) return fail(c, GSL_ERR_INVALID, "vptr must be nondecreasing");
  if (st) memset(st, 0, sizeof(*st));
  const long long n = g->n;
  const bool async_mode = mode == GSL_MODE_ASYNC;
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  if (int r = ensure_vertex_scratch(c, n > 0 ? n : 1)) return r;
  if (int r = grow(c, c->gid, c->cap_gid, n)) return r;
  if (int r = grow(c, c->lab_tmp, c->cap_lab_tmp, n)) return r;
  if (int r = grow(c, c->work2, c->cap_work2, n > 0 ? n : 1)) return r;
  if (int r = grow(c, c->vptr, c->cap_vptr, (long long)num_graphs + 1)) return r;
  if (int r = grow(c, c->dn_graph, c->cap_dng, num_graphs)) return r;
  if (int r = grow(c, c->iters, c->cap_iters, num_graphs)) return r;
  if (int r = grow(c, c->done, c->cap_done, num_graphs)) return r;
  if (int r = grow(c, c->stop, c->cap_stop, 1)) return r;
  CK(cudaEventRecord(c->ev[0], s));
  CK(cudaMemcpyAsync(c->vptr, vptr_host, sizeof(int64_t) * (size_t)(num_graphs + 1), cudaMemcpyHostToDevice, s));
  CK(launch_fill_gid(c->vptr, num_graphs, n, c->gid, c->di, s));
  if (n > 0)
    if (int r = prepare_graph(c, g, s)) return r;
  CK(cudaMemsetAsync(c->done, 0, (size_t)num_graphs, s));
  CK(cudaMemsetAsync(c->iters, 0, sizeof(int) * (size_t)num_graphs, s));
  CK(cudaMemsetAsync(c->stop, 0, sizeof(int), s));
  CK(launch_graph_update(0, tol, max_iters, c->vptr, num_graphs, c->dn_graph, c->iters, c->done, c->stop, s));
  // The sweep loop, unrolled over max_iters and captured once as a CUDA
  // graph; sweeps after the last graph stops return at once.
  const std::vector<long long> key = {(long long)OFF(g), (long long)g->cols, (long long)weights, n, g->nnz,
                                      num_graphs, max_iters, mode, (long long)(tol * 1e12), c->ctr_h->max_degree,
                                      (long long)c->lab[0], (long long)c->wtab, (long long)c->btab,
                                      c->tune.warp_max, c->tune.blk_max, (long long)c->work2,
                                      c->tune.majority, c->tune.blk_block, c->tune.blk_slots, c->tune.probe_cap,
                                      c->tune.uf_cap};
  long long graph_launches = 0;
  if (n > 0) {
    if (c->batch_direct) {
      const cudaError_t e = enqueue_batch_sweeps(c, g, num_graphs, weights, tol, max_iters, async_mode, s);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, GSL_ERR_CUDA, "batched sweep loop: %s", cudaGetErrorString(e));
      }
    } else if (!c->batch_exec || c->batch_key != key) {
      if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
      c->batch_exec = nullptr;
      cudaStream_t cs = c->cap_stream;
      CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      const cudaError_t cerr = enqueue_batch_sweeps(c, g, num_graphs, weights, tol, max_iters, async_mode, cs);
      cudaGraph_t graph = nullptr;
      const cudaError_t e_end = cudaStreamEndCapture(cs, &graph);
      if (cerr != cudaSuccess || e_end != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(c, GSL_ERR_CUDA, "capturing the batched sweep loop failed: %s",
                    cudaGetErrorString(cerr != cudaSuccess ? cerr : e_end));
      }
      const cudaError_t e_inst = cudaGraphInstantiate(&c->batch_exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e_inst != cudaSuccess) {
        cudaGetLastError();
        c->batch_exec = nullptr;
        return fail(c, GSL_ERR_CUDA, "instantiating the batched sweep loop failed: %s", cudaGetErrorString(e_inst));
      }
      c->batch_key = key;
    }
    if (!c->batch_direct) {
      CK(cudaEventRecord(c->ev[3], s));
      CK(cudaStreamWaitEvent(c->cap_stream, c->ev[3], 0));
      CK(cudaGraphLaunch(c->batch_exec, c->cap_stream));
      graph_launches = 1;
      CK(cudaEventRecord(c->ev[3], c->cap_stream));
      CK(cudaStreamWaitEvent(s, c->ev[3], 0));
    }
    CK(cudaEventRecord(c->ev[1], s));
    long long k = 0;
    if (int r = run_split(c, g, c->lab_tmp, labels_out, 0, &k, s)) return r;
    CK(launch_localize(c->vptr, c->gid, n, labels_out, c->di, s));
  }
  if (iterations_out)
    CK(cudaMemcpyAsync(iterations_out, c->iters, sizeof(int32_t) * (size_t)num_graphs, cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(c->ev[2], s));
  CK(cudaEventSynchronize(c->ev[2]));
  if (int r = map_err(c, c->ctr_h->err, "batch")) return r;
  if (st) {
    cudaEventElapsedTime(&st->ms, c->ev[0], c->ev[2]);
    st->graph_launches = graph_launches;
    st->num_graphs = num_graphs;
  }
  return GSL_OK;
}

}  // extern "C"

namespace {

constexpr int HOST_CHUNKS = 5;    // row-aligned column chunks of the overlapped host-buffer path
// Each chunk holds this fraction of the previous one's entries.  Sweep 2 of
// the last chunk runs after the copy has ended, so a smaller last chunk
// shortens the call; the ratio keeps every chunk's sweep-2 work within the
// time the next chunk takes to land (sweep 2 needs about 0.8 of the copy
// time on R-MAT 25).  R-MAT 25 end to end, median of 12 calls: 4 equal
// chunks 67.2 ms; 4 / 5 / 6 chunks at 0.8 / 0.8 / 0.75: 66.4 / 65.8 / 66.2.
constexpr double HOST_CHUNK_RATIO = 0.8;

// gsl_gsllpa on host buffers with the column copy overlapped by the first
// two sweeps (synchronous mode, unit weights, pinned columns the device can
// read).  The offsets are copied first.  The columns then travel to the
// device in HOST_CHUNKS row-aligned chunks on the context's copy stream.
// Meanwhile sweep 1 is evaluated from each row's first entries, read from
// host memory, on the premise that every row is strictly increasing (then
// the smallest neighbour other than the vertex wins, as in the streaming
// first sweep).  As each chunk lands, its entries are checked (range, and
// the premise) and its rows run sweep 2.  Once every chunk has landed, a
// row that broke the premise sends the call back to the plain path on the
// copied graph.  Otherwise sweeps 3.. and the split follow as usual, so the
// labels and statistics are those of gsl_gsllpa.  *handled stays false
// when the call does not qualify (the caller takes the plain path).
int gsllpa_host_overlapped(gsl_ctx* c, int64_t n, int64_t nnz, const int64_t* offsets_host, const int32_t* cols_host,
                           double tol, int32_t max_iters, int32_t* labels_out_host, gsl_stats* st, cudaStream_t s,
                           bool* handled) {
  *handled = false;
  if (c->host_overlap_min <= 0 || nnz < c->host_overlap_min || max_iters < 1 || c->prof) return GSL_OK;
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, cols_host) != cudaSuccess) {
    cudaGetLastError();
    return GSL_OK;
  }
  if (pa.type != cudaMemoryTypeHost || !pa.devicePointer) return GSL_OK;   // pageable: plain path
  const int* cols_dev_view = static_cast<const int*>(pa.devicePointer);
  // row-aligned chunks of geometrically shrinking size, from the host offsets;
  // their bounds must be in range before any copy is issued (the plain path
  // validates malformed offsets on the device and reports them)
  if (offsets_host[0] != 0 || offsets_host[n] != nnz) return GSL_OK;
  double wsum = 0.0;
  for (int k = 0; k < HOST_CHUNKS; ++k) wsum += std::pow(HOST_CHUNK_RATIO, (double)k);
  std::vector<long long> vb{0};
  double acc = 0.0;
  for (int k = 1; k < HOST_CHUNKS; ++k) {
    acc += std::pow(HOST_CHUNK_RATIO, (double)(k - 1));
    const long long target = (long long)((double)nnz * (acc / wsum));
    const long long v = (long long)(std::lower_bound(offsets_host, offsets_host + n + 1, (int64_t)target) - offsets_host);
    if (v > vb.back() && v < n) vb.push_back(v);
  }
  vb.push_back(n);
  const int K = (int)vb.size() - 1;
  for (int k = 0; k < K; ++k)
    if (offsets_host[vb[k]] < 0 || offsets_host[vb[k + 1]] < offsets_host[vb[k]] || offsets_host[vb[k + 1]] > nnz)
      return GSL_OK;
  *handled = true;
  {
    const gsl_csr gh{n, nnz, offsets_host, cols_host};
    if (int r = check_lpa_args(c, &gh, tol, max_iters, GSL_MODE_SYNC, labels_out_host)) return r;
  }
  if (int r = grow(c, c->st_off, c->cap_st_off, n + 1)) return r;
  if (int r = grow(c, c->st_col, c->cap_st_col, nnz)) return r;
  if (int r = grow(c, c->st_lab, c->cap_st_lab, n)) return r;
  if (int r = ensure_vertex_scratch(c, n)) return r;
  const long long words = (nnz >> 5) + 1;
  if (int r = grow(c, c->rowbits, c->cap_rowbits, words)) return r;
  if (!c->copy_stream) CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  while ((int)c->chunk_ev.size() < HOST_CHUNKS) {
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c->chunk_ev.push_back(e);
  }
  gsl_csr g{n, nnz, reinterpret_cast<const int64_t*>(c->st_off), c->st_col};
  CK(cudaEventRecord(c->ev[0], s));
  CK(cudaMemcpyAsync(c->st_off, offsets_host, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, s));
  // the copies: the copy stream waits for the previous work on s (st_col may
  // still be read there); every return below waits for the copies first, so
  // that none is still reading the caller's buffers
  CK(cudaEventRecord(c->ev[3], s));
  CK(cudaStreamWaitEvent(c->copy_stream, c->ev[3], 0));
  struct CopyWait {
    cudaStream_t cs;
    ~CopyWait() {
      if (cudaStreamSynchronize(cs) != cudaSuccess) cudaGetLastError();
    }
  } copy_wait{c->copy_stream};
  for (int k = 0; k < K; ++k) {
    const long long e0 = offsets_host[vb[k]], e1 = offsets_host[vb[k + 1]];
    if (e1 > e0)
      CK(cudaMemcpyAsync(c->st_col + e0, cols_host + e0, sizeof(int32_t) * (size_t)(e1 - e0), cudaMemcpyHostToDevice,
                         c->copy_stream));
    CK(cudaEventRecord(c->chunk_ev[(size_t)k], c->copy_stream));
  }
  // offsets: validated and classified (synchronises s; the copies go on)
  if (int r = prepare_graph(c, &g, s)) return r;
  CK(cudaMemsetAsync(c->flag[0], 0, (size_t)n, s));
  CK(cudaMemsetAsync(c->flag[1], 0, (size_t)n, s));
  CK(launch_init_labels(nullptr, c->lab[0], c->lab[1], n, c->ctr, c->di, s));
  CK(launch_rowstart(OFF(&g), n, c->rowbits, words, c->di, s));
  // sweep 1 from the first entries of the rows, read from host memory
  if (int r = reset_sweep_counters(c, s)) return r;
  CK(launch_ident_first(OFF(&g), n, cols_dev_view, c->flag[0], c->lab[1], c->ctr, c->di, s));
  CK(cudaMemcpyAsync(c->ctr_h, c->ctr, offsetof(Counters, pad1), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const long long dn1 = (long long)c->ctr_h->dn, act1 = (long long)c->ctr_h->fast_active;
  const long long scan1 = (long long)c->ctr_h->scanned;
  const bool stop1 = (double)dn1 / (double)n <= tol || max_iters == 1;
  // sweep 2 chunk by chunk as the columns land (every chunk is checked in any case)
  if (int r = reset_sweep_counters(c, s)) return r;
  SweepArgs a{};
  a.off = OFF(&g);
  a.col = g.cols;
  a.w = nullptr;
  a.ctr = c->ctr;
  a.probe_cap = c->tune.probe_cap;
  a.work = c->work;
  a.wtab = c->wtab;
  a.wtab_region = 2ll * c->tune.warp_max;
  a.btab = c->btab;
  a.btab_region = 2ll * c->ctr_h->max_degree;
  a.n = n;
  a.prev = c->lab[1];
  a.next = c->lab[0];
  a.fnext = c->flag[1];
  a.gthresh = 3 * c->tune.blk_slots;   // as run_lpa's sweep 2
  a.spread = 1;
  a.mark = 2 * dn1 <= n ? 1 : 0;
  const bool filter = c->tune.majority == 2;
  if (filter)
    if (int r = grow(c, c->work2, c->cap_work2, n)) return r;
  if (!stop1) c->hub_dirty = true;
  for (int k = 0; k < K; ++k) {
    CK(cudaStreamWaitEvent(s, c->chunk_ev[(size_t)k], 0));
    const long long e0 = offsets_host[vb[k]], e1 = offsets_host[vb[k + 1]];
    CK(launch_chunk_check(OFF(&g), n, g.cols, nnz, e0, e1, c->rowbits, c->flag[0], &c->ctr->any_bad, c->ctr, c->di,
                          s));
    if (stop1) continue;
    if (k > 0) CK(launch_phase_reset(c->ctr, nullptr, s));
    CK(launch_bin_range(OFF(&g), vb[k], vb[k + 1], c->tune, c->work, c->ctr, c->di, s));
    SweepArgs af = a;
    if (filter) {
      CK(launch_majority_filter(a, c->work2, false, false, c->di, s));
      af.work = c->work2;
    }
    for (int cls = NCLASS - 1; cls >= 0; --cls) {
      if (cls == CLS_WARP_L || cls == CLS_BLOCK) {
        CK(launch_sweep_class(af, cls, false, false, c->tune, c->di, s));
      } else if (cls == CLS_HUB && c->hub_ready) {
        HubPlan hp{c->hub_piece_start, c->hub_ustart, c->hub_best, c->hub_own,
                   c->hub_wsum,        c->hub_used_cnt, c->hub_used, c->hub_tab, c->hub_clu};
        int kernels = 0;
        CK(launch_hub_pieces(a, hp, false, false, filter, c->tune, c->di, s, &kernels));
      } else {
        CK(launch_sweep_class(a, cls, false, false, c->tune, c->di, s));
      }
    }
  }
  CK(cudaMemcpyAsync(c->ctr_h, c->ctr, offsetof(Counters, pad1), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (int r = map_err(c, c->ctr_h->err, "lpa")) return r;
  if (c->ctr_h->any_bad) {
    // a row is not strictly increasing: the first sweep's premise failed
    if (st) memset(st, 0, sizeof(*st));
    if (int r = gsl_gsllpa(c, &g, nullptr, tol, max_iters, GSL_MODE_SYNC, c->st_lab, st, s)) return r;
    CK(cudaMemcpyAsync(labels_out_host, c->st_lab, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return GSL_OK;
  }
  c->hub_dirty = false;
  LpaResume rs{};
  rs.done = 1;
  rs.converged = (double)dn1 / (double)n <= tol;
  rs.marked_prev = false;
  rs.dn_prev = dn1;
  rs.scanned = scan1;
  if (st) {
    st->changed[0] = dn1;
    st->active[0] = act1;
  }
  if (!stop1) {
    const long long dn2 = (long long)c->ctr_h->dn;
    long long act2 = (long long)c->ctr_h->fast_active;
    for (int k = 0; k < NCLASS; ++k) act2 += (long long)(c->ctr_h->cls_count[k] + c->ctr_h->phase_cls[k]);
    rs.done = 2;
    rs.converged = (double)dn2 / (double)n <= tol;
    rs.marked_prev = a.mark != 0;
    rs.dn_prev = dn2;
    rs.scanned += (long long)c->ctr_h->scanned;
    if (st && GSL_STATS_SWEEPS >= 2) {
      st->changed[1] = dn2;
      st->active[1] = act2;
    }
  }
  int* fin = nullptr;
  if (int r = run_lpa(c, &g, nullptr, nullptr, tol, max_iters, GSL_MODE_SYNC, st, s, &fin, &rs)) return r;
  CK(cudaEventRecord(c->ev[1], s));
  long long k = 0;
  if (int r = run_split(c, &g, fin, c->st_lab, 0, &k, s)) return r;
  CK(cudaEventRecord(c->ev[2], s));
  CK(cudaMemcpyAsync(labels_out_host, c->st_lab, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (st) {
    cudaEventElapsedTime(&st->ms_lpa, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&st->ms_split, c->ev[1], c->ev[2]);
    st->communities = k;
  }
  return GSL_OK;
}

}  // namespace

extern "C" {

int gsl_ctx_set_host_overlap(gsl_ctx* c, int64_t min_entries) {
  if (!c) return GSL_ERR_INVALID;
  if (min_entries < 0) return fail(c, GSL_ERR_INVALID, "min_entries must be >= 0");
  c->host_overlap_min = min_entries;
  return GSL_OK;
}

int gsl_gsllpa_host(gsl_ctx* c, int64_t n, int64_t nnz, const int64_t* offsets_host, const int32_t* cols_host,
                    const int32_t* weights_host, double tol, int32_t max_iters, int32_t mode,
                    int32_t* labels_out_host, gsl_stats* st, void* stream) {
  if (!c) return GSL_ERR_INVALID;
  c->last_error.clear();
  if (n < 0 || n >= (1ll << 31) || nnz < 0) return fail(c, GSL_ERR_INVALID, "bad sizes n=%lld nnz=%lld", (long long)n, (long long)nnz);
  if (!offsets_host || (nnz > 0 && !cols_host) || (n > 0 && !labels_out_host))
    return fail(c, GSL_ERR_INVALID, "host pointer is NULL");
  if (st) memset(st, 0, sizeof(*st));
  if (n == 0) return GSL_OK;
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (!weights_host && mode == GSL_MODE_SYNC) {
    bool handled = false;
    const int r = gsllpa_host_overlapped(c, n, nnz, offsets_host, cols_host, tol, max_iters, labels_out_host, st, s,
                                         &handled);
    if (handled) return r;
  }
  if (int r = grow(c, c->st_off, c->cap_st_off, n + 1)) return r;
  if (int r = grow(c, c->st_col, c->cap_st_col, nnz)) return r;
  if (weights_host)
    if (int r = grow(c, c->st_w, c->cap_st_w, nnz)) return r;
  if (int r = grow(c, c->st_lab, c->cap_st_lab, n)) return r;
  CK(cudaMemcpyAsync(c->st_off, offsets_host, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, s));
  if (nnz > 0) CK(cudaMemcpyAsync(c->st_col, cols_host, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, s));
  if (weights_host && nnz > 0)
    CK(cudaMemcpyAsync(c->st_w, weights_host, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, s));
  gsl_csr g{n, nnz, reinterpret_cast<const int64_t*>(c->st_off), c->st_col};
  if (int r = gsl_gsllpa(c, &g, weights_host ? c->st_w : nullptr, tol, max_iters, mode, c->st_lab, st, stream))
    return r;
  CK(cudaMemcpyAsync(labels_out_host, c->st_lab, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return GSL_OK;
}

}  // extern "C"
