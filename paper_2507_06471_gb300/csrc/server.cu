// Serving engine: community-detection requests (LPA or Louvain on one graph
// each) admitted continuously onto one GPU.
//
// A submitted request is copied and queued. W worker slots, each with its own
// CUDA stream, take work whenever the slot is free and the device-memory
// budget can hold it, so requests that arrive while others run are admitted
// as slots and memory free up, and their kernels overlap on the device. Small
// waiting requests of the same algorithm are packed block-diagonally and
// solved by one batched call (one launch per kernel for all of them); large
// ones run alone. Every request's result is the one a solo run gives (the
// batched calls guarantee that per graph).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "common.cuh"

namespace {

using clk = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  int kind = 0;  // CD_REQ_LPA or CD_REQ_LOUVAIN
  int64_t n = 0, nnz = 0;
  std::vector<int64_t> off;
  std::vector<int32_t> cols, w;  // w empty: unit weights
  int64_t bytes = 0;             // admission estimate
  clk::time_point t_submit, t_start, t_done;
  bool done = false;
  int status = CD_OK;
  std::vector<int32_t> labels;
  int32_t iters = 0;  // LPA rounds or Louvain levels
  double q = 0.0;
  int batched_with = 1;
};

}  // namespace

struct cd_server {
  cd_params params;
  int device = 0;
  int slots = 1;
  int64_t budget = 0, in_use = 0;
  int64_t small_n = 0;     // requests with n <= small_n may be packed together
  int64_t batch_arcs = 0;  // arcs per packed batch at most
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<int64_t, std::shared_ptr<Request>> all;
  int64_t next_id = 1;
  bool stopping = false;
  std::vector<std::thread> workers;
  int64_t admitted = 0, completed = 0, packed_calls = 0;
};

namespace {

int64_t estimate_bytes(int64_t n, int64_t nnz) {
  // CSR and weights, deg_w, run state, bins, aggregation keys/values (32 B per
  // arc), plus a fixed slack for pools and small arrays
  return 64 * nnz + 96 * n + (16ll << 20);
}

void solve_one(cd_server* s, cudaStream_t st, Request& r) {
  cd_graph* g = nullptr;
  int rc = cd_csr_upload(r.off.data(), 1, r.cols.data(), r.w.empty() ? nullptr : r.w.data(), r.n, r.nnz, 0, st, &g);
  r.labels.assign(r.n, 0);
  if (!rc) {
    if (r.kind == CD_REQ_LPA)
      rc = cd_lpa_run(g, &s->params, r.labels.data(), 0, &r.iters);
    else
      rc = cd_louvain_run(g, &s->params, r.labels.data(), 0, &r.iters, &r.q);
  }
  if (g) cd_graph_free(g);
  r.status = rc;
}

void solve_packed(cd_server* s, cudaStream_t st, std::vector<std::shared_ptr<Request>>& rs) {
  const int64_t B = (int64_t)rs.size();
  std::vector<int64_t> vstart(B + 1, 0), astart(B + 1, 0);
  bool weighted = false;
  for (int64_t b = 0; b < B; ++b) {
    vstart[b + 1] = vstart[b] + rs[b]->n;
    astart[b + 1] = astart[b] + rs[b]->nnz;
    weighted = weighted || !rs[b]->w.empty();
  }
  const int64_t n = vstart[B], nnz = astart[B];
  std::vector<int64_t> off(n + 1, 0);
  std::vector<int32_t> cols(nnz), w(weighted ? nnz : 0, 1);
  for (int64_t b = 0; b < B; ++b) {
    const Request& r = *rs[b];
    for (int64_t v = 0; v < r.n; ++v) off[vstart[b] + v + 1] = r.off[v + 1] + astart[b];
    for (int64_t e = 0; e < r.nnz; ++e) cols[astart[b] + e] = r.cols[e] + (int32_t)vstart[b];
    if (weighted && !r.w.empty()) std::copy(r.w.begin(), r.w.end(), w.begin() + astart[b]);
  }
  cd_graph* g = nullptr;
  int rc = cd_csr_upload(off.data(), 1, cols.data(), weighted ? w.data() : nullptr, n, nnz, 0, st, &g);
  if (!rc) rc = cd_graph_set_batches(g, vstart.data(), B, 0);
  std::vector<int32_t> lab(n, 0), iters(B, 0);
  std::vector<double> q(B, 0.0);
  if (!rc) {
    if (rs[0]->kind == CD_REQ_LPA)
      rc = cd_batch_lpa_run(g, &s->params, lab.data(), 0, iters.data());
    else
      rc = cd_batch_louvain_run(g, &s->params, lab.data(), 0, iters.data(), q.data());
  }
  if (g) cd_graph_free(g);
  if (rc) {  // a packed call failed: solve the members one by one
    for (auto& r : rs) solve_one(s, st, *r);
    return;
  }
  for (int64_t b = 0; b < B; ++b) {
    Request& r = *rs[b];
    r.labels.assign(lab.begin() + vstart[b], lab.begin() + vstart[b + 1]);
    r.iters = iters[b];
    r.q = q[b];
    r.status = CD_OK;
    r.batched_with = (int)B;
  }
}

// Next work for a free slot (called with the lock held). Admission is in
// arrival order with a reservation: when the oldest waiting request does not
// fit the memory left, later requests are admitted only within the budget
// minus its size, so it starts as soon as running work returns that much.
// A small request takes along the following small requests of the same
// algorithm that fit.
bool take_work(cd_server* s, std::vector<std::shared_ptr<Request>>& out, int64_t& bytes) {
  out.clear();
  bytes = 0;
  int64_t limit = s->budget;
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    const auto& r = *it;
    if (s->in_use + r->bytes > limit) {
      if (it == s->queue.begin()) limit -= r->bytes;  // reserve for the head
      continue;
    }
    out.push_back(r);
    bytes = r->bytes;
    s->queue.erase(it);
    break;
  }
  if (out.empty()) return false;
  if (out[0]->n <= s->small_n) {
    int64_t arcs = out[0]->nnz;
    for (auto it = s->queue.begin(); it != s->queue.end();) {
      const auto& r = *it;
      if (r->kind == out[0]->kind && r->n <= s->small_n && arcs + r->nnz <= s->batch_arcs &&
          s->in_use + bytes + r->bytes <= limit) {
        arcs += r->nnz;
        bytes += r->bytes;
        out.push_back(r);
        it = s->queue.erase(it);
      } else {
        ++it;
      }
    }
  }
  s->in_use += bytes;
  s->admitted += (int64_t)out.size();
  return true;
}

void worker_main(cd_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    std::vector<std::shared_ptr<Request>> work;
    int64_t bytes = 0;
    {
      // on shutdown the queue is drained first
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv_work.wait(lock, [&] { return take_work(s, work, bytes) || (s->stopping && s->queue.empty()); });
      if (work.empty()) break;
    }
    const auto t0 = clk::now();
    for (auto& r : work) r->t_start = t0;
    if (work.size() == 1)
      solve_one(s, st, *work[0]);
    else
      solve_packed(s, st, work);
    const auto t1 = clk::now();
    {
      std::lock_guard<std::mutex> lock(s->mu);
      for (auto& r : work) {
        r->t_done = t1;
        r->done = true;
        // keep the result, drop the input copy
        std::vector<int64_t>().swap(r->off);
        std::vector<int32_t>().swap(r->cols);
        std::vector<int32_t>().swap(r->w);
      }
      s->in_use -= bytes;
      s->completed += (int64_t)work.size();
      if (work.size() > 1) s->packed_calls += 1;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();  // memory came back: others may fit now
  }
  cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

int cd_server_create(const cd_params* p, int32_t slots, int64_t mem_budget_bytes, int64_t small_n,
                     int64_t batch_arcs, cd_server** out) {
  if (!p || !out || slots < 1 || slots > 64 || small_n < 0 || batch_arcs < 0) return CD_EINVAL;
  cd_server* s = new cd_server();
  s->params = *p;
  s->params.timing = 0;
  // device_loop 1 means "batched calls": the workers' packed calls keep the
  // host loop, since several workers capturing and instantiating round graphs
  // at once cost more than the round trips they save (2 still forces it)
  if (s->params.device_loop == 1) s->params.device_loop = 0;
  cudaGetDevice(&s->device);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    delete s;
    return cd::set_cuda_error(cudaGetLastError());
  }
  s->budget = mem_budget_bytes > 0 ? mem_budget_bytes : (int64_t)(0.8 * (double)free_b);
  s->slots = slots;
  s->small_n = small_n;
  s->batch_arcs = batch_arcs;
  for (int i = 0; i < slots; ++i) s->workers.emplace_back(worker_main, s);
  *out = s;
  return CD_OK;
}

int cd_server_submit(cd_server* s, int32_t kind, const void* offsets, int offsets_is_i64, const int32_t* cols,
                     const int32_t* w, int64_t n, int64_t nnz, int64_t* id_out) {
  if (!s || !id_out || (kind != CD_REQ_LPA && kind != CD_REQ_LOUVAIN) || n < 0 || nnz < 0 || !offsets ||
      (nnz > 0 && !cols))
    return CD_EINVAL;
  auto r = std::make_shared<Request>();
  r->kind = kind;
  r->n = n;
  r->nnz = nnz;
  r->bytes = estimate_bytes(n, nnz);
  if (r->bytes > s->budget) return CD_ENOMEM;  // can never be admitted
  r->off.resize(n + 1);
  if (offsets_is_i64)
    std::copy((const int64_t*)offsets, (const int64_t*)offsets + n + 1, r->off.begin());
  else
    std::copy((const int32_t*)offsets, (const int32_t*)offsets + n + 1, r->off.begin());
  r->cols.assign(cols, cols + nnz);
  if (w) r->w.assign(w, w + nnz);
  r->t_submit = clk::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stopping) return CD_EINVAL;
    r->id = s->next_id++;
    s->all[r->id] = r;
    s->queue.push_back(r);
  }
  s->cv_work.notify_one();
  *id_out = r->id;
  return CD_OK;
}

int cd_server_wait(cd_server* s, int64_t id, int64_t timeout_ms, cd_request_result* res, int32_t* labels_out) {
  if (!s) return CD_EINVAL;
  std::shared_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return CD_EINVAL;
    r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_ms < 0)
      s->cv_done.wait(lock, ready);
    else if (!s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), ready))
      return CD_ETIMEOUT;
    s->all.erase(id);
  }
  if (res) {
    res->status = r->status;
    res->n = r->n;
    res->iters = r->iters;
    res->q = r->q;
    res->batched_with = r->batched_with;
    res->queue_ms = std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count();
    res->latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  }
  if (labels_out && r->status == CD_OK) std::copy(r->labels.begin(), r->labels.end(), labels_out);
  return r->status;
}

int cd_server_stats(cd_server* s, int64_t* admitted, int64_t* completed, int64_t* packed_calls, int64_t* in_use) {
  if (!s) return CD_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if (admitted) *admitted = s->admitted;
  if (completed) *completed = s->completed;
  if (packed_calls) *packed_calls = s->packed_calls;
  if (in_use) *in_use = s->in_use;
  return CD_OK;
}

int cd_server_destroy(cd_server* s) {
  if (!s) return CD_OK;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
  return CD_OK;
}

}  // extern "C"
