// server.cu -- continuous-batching request loop for GSL-LPA (host runtime).
//
// Requests (one graph each, host CSR) are queued as they arrive.  The
// server owns `slots` workers; each worker has its own library context, its
// own CUDA stream and device buffers kept resident for the server's life,
// sized at creation from the free device memory.  A free worker takes the
// oldest waiting requests that fit its buffers (admission by memory), packs
// them into one batch CSR on the device, runs batched GSL-LPA on it (every
// graph keeps its solo result) and hands each request its labels.  Requests
// that arrive while batches are on the GPU are admitted by the next worker
// to free up, so batches of different requests overlap on the device.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/gsllpa.h"
#include "kernels.h"

namespace {

using clk = std::chrono::steady_clock;

// Shifts graph k's copied offsets by its first entry and its columns by its
// first vertex, turning the concatenated solo CSRs into one batch CSR.
__global__ void pack_shift_kernel(long long* __restrict__ off, int* __restrict__ col,
                                  const long long* __restrict__ vbase, const long long* __restrict__ ebase) {
  const int k = blockIdx.y;
  const long long v0 = vbase[k], v1 = vbase[k + 1], e0 = ebase[k], e1 = ebase[k + 1];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = v0 + 1 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= v1; i += stride) off[i] += e0;
  for (long long e = e0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; e < e1; e += stride)
    col[e] += (int)v0;
}

struct Request {
  int64_t id;
  int64_t n, nnz;
  const int64_t* offsets;
  const int32_t* cols;
  std::vector<int32_t> labels;
  int32_t sweeps = 0;
  int status = GSL_OK;
  bool done = false;
  clk::time_point t_submit, t_start, t_done;
  int64_t batch_graphs = 0;
  float h2d_ms = 0.f, compute_ms = 0.f, d2h_ms = 0.f;
};

struct Slot {
  gsl_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  long long* off = nullptr;      // batch CSR offsets (cap_v + 1)
  int* col = nullptr;            // batch CSR columns (cap_e)
  int* lab = nullptr;            // batch labels (cap_v)
  long long* bases = nullptr;    // vbase / ebase of the batch graphs (device)
  long long* bases_h = nullptr;  // pinned
  int* lab_h = nullptr;          // pinned labels
  std::vector<int64_t> vptr;
  std::vector<int32_t> iters;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};   // copies in, kernels, copy out
};

// Device time of a batch's phases from the slot's events (after its stream
// has been synchronised); zeros when an event query fails.
void phase_times(Slot& sl, float* h2d, float* comp, float* d2h) {
  *h2d = *comp = *d2h = 0.f;
  if (cudaEventElapsedTime(h2d, sl.ev[0], sl.ev[1]) != cudaSuccess ||
      cudaEventElapsedTime(comp, sl.ev[1], sl.ev[2]) != cudaSuccess ||
      cudaEventElapsedTime(d2h, sl.ev[2], sl.ev[3]) != cudaSuccess) {
    cudaGetLastError();
    *h2d = *comp = *d2h = 0.f;
  }
}

}  // namespace

struct gsl_server {
  gsl_server_config cfg{};
  int64_t cap_v = 0, cap_e = 0;
  std::vector<Slot> slots;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<int64_t, Request*> reqs;
  int64_t next_id = 1;
  bool stopping = false;
  std::atomic<int64_t> completed{0}, batches{0}, graphs_in_batches{0}, busy_workers{0}, max_busy{0};
};

namespace {

// A request of at least this many CSR entries keeps the GPU busy on its own
// and runs alone through the single-graph path (streaming first sweep, hub
// pieces, majority filter); smaller ones are packed into batches.
constexpr int64_t SOLO_ENTRIES = 1ll << 22;

void worker_loop(gsl_server* S, int w) {
  Slot& sl = S->slots[w];
  int dev = S->cfg.device;
  cudaSetDevice(dev);
  const int maxg = S->cfg.max_batch_graphs > 0 ? S->cfg.max_batch_graphs : 1024;
  for (;;) {
    std::vector<Request*> batch;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stopping || !S->queue.empty(); });
      if (S->stopping && S->queue.empty()) return;
      int64_t v = 0, e = 0;
      while (!S->queue.empty() && (int)batch.size() < maxg) {
        Request* r = S->queue.front();
        const bool solo = r->nnz >= SOLO_ENTRIES;
        if (solo && !batch.empty()) break;                              // a large request goes alone
        if (v + r->n > S->cap_v || e + r->nnz > S->cap_e) break;   // FIFO: the head waits for a free slot
        S->queue.pop_front();
        v += r->n;
        e += r->nnz;
        batch.push_back(r);
        if (solo) break;
      }
    }
    if (batch.empty()) continue;
    const int64_t busy = ++S->busy_workers;
    int64_t mb = S->max_busy.load();
    while (busy > mb && !S->max_busy.compare_exchange_weak(mb, busy)) {
    }
    const auto t_start = clk::now();
    const int G = (int)batch.size();
    sl.vptr.assign(G + 1, 0);
    std::vector<int64_t> eptr(G + 1, 0);
    for (int k = 0; k < G; ++k) {
      sl.vptr[k + 1] = sl.vptr[k] + batch[k]->n;
      eptr[k + 1] = eptr[k] + batch[k]->nnz;
    }
    int rc = GSL_OK;
    cudaStream_t s = sl.stream;
    if (G == 1 && batch[0]->nnz >= SOLO_ENTRIES) {
      Request* r = batch[0];
      gsl_stats st{};
      cudaEventRecord(sl.ev[0], s);
      if (cudaMemcpyAsync(sl.off, r->offsets, sizeof(int64_t) * (size_t)(r->n + 1), cudaMemcpyHostToDevice, s) !=
              cudaSuccess ||
          cudaMemcpyAsync(sl.col, r->cols, sizeof(int32_t) * (size_t)r->nnz, cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = GSL_ERR_CUDA;
      cudaEventRecord(sl.ev[1], s);
      gsl_csr csr{r->n, r->nnz, reinterpret_cast<const int64_t*>(sl.off), sl.col};
      if (rc == GSL_OK)
        rc = gsl_gsllpa(sl.ctx, &csr, nullptr, S->cfg.tolerance, S->cfg.max_iters, S->cfg.mode, sl.lab, &st, s);
      cudaEventRecord(sl.ev[2], s);
      if (rc == GSL_OK &&
          (cudaMemcpyAsync(sl.lab_h, sl.lab, sizeof(int32_t) * (size_t)r->n, cudaMemcpyDeviceToHost, s) !=
               cudaSuccess ||
           cudaEventRecord(sl.ev[3], s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess))
        rc = GSL_ERR_CUDA;
      if (rc != GSL_OK) cudaGetLastError();
      const auto t_done = clk::now();
      float h2d = 0.f, comp = 0.f, d2h = 0.f;
      if (rc == GSL_OK) phase_times(sl, &h2d, &comp, &d2h);
      {
        std::lock_guard<std::mutex> lk(S->mu);
        r->status = rc;
        if (rc == GSL_OK) {
          r->labels.assign(sl.lab_h, sl.lab_h + r->n);
          r->sweeps = st.iterations;
        }
        r->t_start = t_start;
        r->t_done = t_done;
        r->batch_graphs = 1;
        r->h2d_ms = h2d;
        r->compute_ms = comp;
        r->d2h_ms = d2h;
        r->done = true;
      }
      S->cv_done.notify_all();
      S->batches++;
      S->graphs_in_batches += 1;
      S->completed += 1;
      S->busy_workers--;
      continue;
    }
    // pack: copy every solo CSR to its place, then shift offsets and columns
    cudaEventRecord(sl.ev[0], s);
    for (int k = 0; k < G && rc == GSL_OK; ++k) {
      Request* r = batch[k];
      if (r->n > 0 &&
          cudaMemcpyAsync(sl.off + sl.vptr[k] + 1, r->offsets + 1, sizeof(int64_t) * (size_t)r->n,
                          cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = GSL_ERR_CUDA;
      if (r->nnz > 0 &&
          cudaMemcpyAsync(sl.col + eptr[k], r->cols, sizeof(int32_t) * (size_t)r->nnz, cudaMemcpyHostToDevice, s) !=
              cudaSuccess)
        rc = GSL_ERR_CUDA;
    }
    for (int k = 0; k <= G; ++k) {
      sl.bases_h[k] = sl.vptr[k];
      sl.bases_h[G + 1 + k] = eptr[k];
    }
    if (rc == GSL_OK &&
        (cudaMemsetAsync(sl.off, 0, sizeof(long long), s) != cudaSuccess ||
         cudaMemcpyAsync(sl.bases, sl.bases_h, sizeof(long long) * (size_t)(2 * (G + 1)), cudaMemcpyHostToDevice,
                         s) != cudaSuccess))
      rc = GSL_ERR_CUDA;
    if (rc == GSL_OK) {
      dim3 grid(64, (unsigned)G);
      pack_shift_kernel<<<grid, 256, 0, s>>>(sl.off, sl.col, sl.bases, sl.bases + G + 1);
      gsl::count_launches(1);
      if (cudaGetLastError() != cudaSuccess) rc = GSL_ERR_CUDA;
    }
    const int64_t n = sl.vptr[G], nnz = eptr[G];
    cudaEventRecord(sl.ev[1], s);
    if (rc == GSL_OK) {
      gsl_csr csr{n, nnz, reinterpret_cast<const int64_t*>(sl.off), sl.col};
      sl.iters.assign(G, 0);
      rc = gsl_gsllpa_batch(sl.ctx, &csr, G, sl.vptr.data(), nullptr, S->cfg.tolerance, S->cfg.max_iters,
                            S->cfg.mode, sl.lab, sl.iters.data(), nullptr, s);
    }
    cudaEventRecord(sl.ev[2], s);
    if (rc == GSL_OK && n > 0 &&
        (cudaMemcpyAsync(sl.lab_h, sl.lab, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         cudaEventRecord(sl.ev[3], s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess))
      rc = GSL_ERR_CUDA;
    if (rc != GSL_OK) cudaGetLastError();
    const auto t_done = clk::now();
    float h2d = 0.f, comp = 0.f, d2h = 0.f;
    if (rc == GSL_OK && n > 0) phase_times(sl, &h2d, &comp, &d2h);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (int k = 0; k < G; ++k) {
        Request* r = batch[k];
        r->status = rc;
        if (rc == GSL_OK) {
          r->labels.assign(sl.lab_h + sl.vptr[k], sl.lab_h + sl.vptr[k + 1]);
          r->sweeps = sl.iters[k];
        }
        r->t_start = t_start;
        r->t_done = t_done;
        r->batch_graphs = G;
        r->h2d_ms = h2d;
        r->compute_ms = comp;
        r->d2h_ms = d2h;
        r->done = true;
      }
    }
    S->cv_done.notify_all();
    S->batches++;
    S->graphs_in_batches += G;
    S->completed += G;
    S->busy_workers--;
  }
}

void free_slot(Slot& sl) {
  if (sl.ctx) gsl_ctx_destroy(sl.ctx);
  for (auto& e : sl.ev)
    if (e) cudaEventDestroy(e);
  void* d[] = {sl.off, sl.col, sl.lab, sl.bases};
  for (void* p : d)
    if (p) cudaFree(p);
  if (sl.bases_h) cudaFreeHost(sl.bases_h);
  if (sl.lab_h) cudaFreeHost(sl.lab_h);
  if (sl.stream) cudaStreamDestroy(sl.stream);
  sl = Slot();
}

}  // namespace

extern "C" {

int gsl_server_create(gsl_server** out, const gsl_server_config* cfg) {
  if (!out || !cfg || cfg->slots < 1 || cfg->slots > 64 || cfg->max_iters < 0 || !(cfg->tolerance >= 0.0) ||
      (cfg->mode != GSL_MODE_SYNC && cfg->mode != GSL_MODE_ASYNC) || cfg->max_batch_graphs < 0 ||
      cfg->max_batch_graphs > 65535)
    return GSL_ERR_INVALID;
  *out = nullptr;
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
    cudaGetLastError();
    return GSL_ERR_CUDA;
  }
  gsl_server* S = new gsl_server();
  S->cfg = *cfg;
  // admission capacity per slot: from the configuration, or a share of the
  // free device memory (columns 4 B per entry; about 64 B per vertex of
  // batch arrays and context scratch; the rest left for hub tables)
  S->cap_v = cfg->slot_vertices;
  S->cap_e = cfg->slot_entries;
  if (S->cap_v <= 0 || S->cap_e <= 0) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const double share = (cfg->memory_fraction > 0.0 && cfg->memory_fraction <= 0.95 ? cfg->memory_fraction : 0.5) *
                         (double)free_b / cfg->slots;
    if (S->cap_e <= 0) S->cap_e = (int64_t)(share * 0.6 / 4.0);
    if (S->cap_v <= 0) S->cap_v = (int64_t)(share * 0.25 / 64.0);
  }
  S->slots.resize(cfg->slots);
  bool ok = true;
  for (auto& sl : S->slots) {
    ok = ok && gsl_ctx_create(&sl.ctx, cfg->device) == GSL_OK;
    ok = ok && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaMalloc(&sl.off, sizeof(long long) * (size_t)(S->cap_v + 1)) == cudaSuccess;
    ok = ok && cudaMalloc(&sl.col, sizeof(int) * (size_t)std::max<int64_t>(S->cap_e, 1)) == cudaSuccess;
    ok = ok && cudaMalloc(&sl.lab, sizeof(int) * (size_t)std::max<int64_t>(S->cap_v, 1)) == cudaSuccess;
    const int maxg = cfg->max_batch_graphs > 0 ? cfg->max_batch_graphs : 1024;
    ok = ok && cudaMalloc(&sl.bases, sizeof(long long) * (size_t)(2 * (maxg + 1))) == cudaSuccess;
    ok = ok && cudaMallocHost(&sl.bases_h, sizeof(long long) * (size_t)(2 * (maxg + 1))) == cudaSuccess;
    ok = ok && cudaMallocHost(&sl.lab_h, sizeof(int) * (size_t)std::max<int64_t>(S->cap_v, 1)) == cudaSuccess;
    for (auto& e : sl.ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
    if (ok) gsl_ctx_set_batch_mode(sl.ctx, 0);   // batches change shape every time: launch directly
  }
  if (!ok) {
    cudaGetLastError();
    for (auto& sl : S->slots) free_slot(sl);
    delete S;
    return GSL_ERR_NOMEM;
  }
  for (int w = 0; w < cfg->slots; ++w) S->workers.emplace_back(worker_loop, S, w);
  *out = S;
  return GSL_OK;
}

int gsl_server_capacity(gsl_server* S, int64_t* max_vertices, int64_t* max_entries) {
  if (!S) return GSL_ERR_INVALID;
  if (max_vertices) *max_vertices = S->cap_v;
  if (max_entries) *max_entries = S->cap_e;
  return GSL_OK;
}

int gsl_server_submit(gsl_server* S, int64_t n, int64_t nnz, const int64_t* offsets, const int32_t* cols,
                      int64_t* request_id) {
  if (!S || !request_id || n < 0 || nnz < 0 || !offsets || (nnz > 0 && !cols)) return GSL_ERR_INVALID;
  if (n > S->cap_v || nnz > S->cap_e) return GSL_ERR_NOMEM;   // can never be admitted
  Request* r = new Request();
  r->n = n;
  r->nnz = nnz;
  r->offsets = offsets;
  r->cols = cols;
  r->t_submit = clk::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    S->reqs[r->id] = r;
    S->queue.push_back(r);
    *request_id = r->id;
  }
  S->cv_work.notify_one();
  return GSL_OK;
}

int gsl_server_wait(gsl_server* S, int64_t id, int32_t* labels_out, gsl_request_info* info) {
  if (!S) return GSL_ERR_INVALID;
  Request* r = nullptr;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return GSL_ERR_INVALID;
    r = it->second;
    S->cv_done.wait(lk, [&] { return r->done; });
    S->reqs.erase(it);
  }
  const int rc = r->status;
  if (rc == GSL_OK && labels_out && r->n > 0) memcpy(labels_out, r->labels.data(), sizeof(int32_t) * (size_t)r->n);
  if (info) {
    info->status = rc;
    info->sweeps = r->sweeps;
    info->batch_graphs = r->batch_graphs;
    info->queue_ms = std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count();
    info->service_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_start).count();
    info->latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    info->h2d_ms = r->h2d_ms;
    info->compute_ms = r->compute_ms;
    info->d2h_ms = r->d2h_ms;
  }
  delete r;
  return rc;
}

int gsl_server_get_stats(gsl_server* S, gsl_server_stats* out) {
  if (!S || !out) return GSL_ERR_INVALID;
  out->completed = S->completed.load();
  out->batches = S->batches.load();
  out->max_concurrent_batches = S->max_busy.load();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    out->queued = (int64_t)S->queue.size();
  }
  return GSL_OK;
}

int gsl_server_destroy(gsl_server* S) {
  if (!S) return GSL_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  cudaSetDevice(S->cfg.device);
  for (auto& sl : S->slots) free_slot(sl);
  for (auto& kv : S->reqs) delete kv.second;
  delete S;
  return GSL_OK;
}

}  // extern "C"
