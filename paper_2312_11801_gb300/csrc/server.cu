// Continuous-batching server and batched solve over the C ABI (host code only).
//
// Requests enter a FIFO queue.  A request is admitted when a solve slot is free and its
// device footprint (usbs_instance_bytes) fits the memory budget; finished instances stay
// resident in an LRU cache so that a later request naming one of them as its parent is
// warm-started from it with usbs_grow (the paper's warm start, Sec. 5.1).  Each slot is a
// host thread and each context owns its CUDA stream, so admitted solves overlap on the
// device.  In
// dry-run mode no CUDA call is made and a request occupies its slot for the service time
// the caller gives, which lets the scheduling be tested without a GPU.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  int64_t id = 0, parent = -1;
  double tol = 1e-3, fake_s = 0.0, t_arrival = 0.0, t_admit = 0.0;
  int64_t n = 0, m = 0, nnzA = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col, acon, ai, aj;
  std::vector<double> val, aval, b;
  std::vector<uint8_t> ineq;
  std::vector<float> psi;
  uint64_t bytes = 0;
  usbs_ctx* parent_ctx = nullptr;   // taken out of the cache for the grow
  uint64_t parent_bytes = 0;        // > 0 while the parent is held (also in dry-run mode)
  bool parent_held = false;         // the cache was searched for the parent
};

struct Cached {
  int64_t id;
  usbs_ctx* ctx;
  uint64_t bytes;
};

}  // namespace

struct usbs_server {
  usbs_server_params p{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::unique_ptr<Req>> pending;
  std::deque<std::unique_ptr<Req>> admitted;
  std::list<Cached> cache;                   // front = most recently finished
  std::vector<usbs_completion> done;
  uint64_t used = 0, peak_used = 0;
  int running = 0, peak_running = 0;
  int64_t finished = 0, rejected = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  Clock::time_point t0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

  void destroy_cached(Cached& c) {
    if (c.ctx) usbs_destroy(c.ctx);
    used -= c.bytes;
  }

  // Admit from the head of the queue while a slot and memory are free (FIFO; a request
  // that does not fit blocks those behind it).  Called with mu held.
  void admit() {
    while (!pending.empty() && running < p.max_slots) {
      Req& r = *pending.front();
      const uint64_t need = r.bytes;
      if (need > p.hbm_budget_bytes) {
        // can never fit: complete it with USBS_EBUSY
        usbs_completion c{};
        c.request_id = r.id;
        c.parent_id = r.parent;
        c.status = USBS_EBUSY;
        c.t_arrival = r.t_arrival;
        c.t_admit = c.t_finish = now();
        c.bytes = need;
        done.push_back(c);
        pending.pop_front();
        ++rejected;
        cv_done.notify_all();
        continue;
      }
      // take the parent out of the cache for this request's grow (it stays resident)
      if (r.parent >= 0 && !r.parent_held) {
        for (auto it = cache.begin(); it != cache.end(); ++it)
          if (it->id == r.parent) {
            r.parent_ctx = it->ctx;
            r.parent_bytes = it->bytes;
            r.parent_held = true;
            cache.erase(it);
            break;
          }
      }
      while (used + need > p.hbm_budget_bytes && !cache.empty()) {
        destroy_cached(cache.back());
        cache.pop_back();
      }
      if (used + need > p.hbm_budget_bytes) {
        if (running > 0) break;   // wait for a running solve to free its memory
        // nothing runs and nothing is cached: only the held parent is resident, and the
        // parent and the grown instance do not fit together, so the request starts cold
        if (r.parent_ctx) usbs_destroy(r.parent_ctx);
        used -= r.parent_bytes;
        r.parent_ctx = nullptr;
        r.parent_bytes = 0;
        continue;
      }
      used += need;
      peak_used = std::max(peak_used, used);
      ++running;
      peak_running = std::max(peak_running, running);
      r.t_admit = now();
      admitted.push_back(std::move(pending.front()));
      pending.pop_front();
      cv_work.notify_one();
    }
  }

  void worker(int slot) {
    if (!p.dry_run && p.solver.device >= 0) cudaSetDevice(p.solver.device);
    for (;;) {
      std::unique_ptr<Req> r;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || !admitted.empty(); });
        if (admitted.empty()) break;
        r = std::move(admitted.front());
        admitted.pop_front();
      }
      usbs_completion c{};
      c.request_id = r->id;
      c.parent_id = r->parent;
      c.slot = slot;
      c.t_arrival = r->t_arrival;
      c.t_admit = r->t_admit;
      c.bytes = r->bytes;
      usbs_ctx* ctx = nullptr;
      if (p.dry_run) {
        c.warm = r->parent_ctx != nullptr || r->parent_bytes > 0 ? 1 : 0;
        std::this_thread::sleep_for(std::chrono::duration<double>(r->fake_s));
        c.status = USBS_OK;
      } else {
        // every context owns its stream (created by usbs_create or usbs_grow, destroyed
        // with the context), so resident instances never outlive the stream they use and
        // solves of different requests overlap on the device
        usbs_params sp = p.solver;
        sp.stream = nullptr;
        int rc = USBS_OK;
        if (r->parent_ctx) {
          rc = usbs_grow(r->parent_ctx, &ctx, r->n, r->rowptr.data(), r->col.data(), r->val.data(),
                         r->m, r->nnzA, r->acon.data(), r->ai.data(), r->aj.data(), r->aval.data(),
                         r->b.data(), r->ineq.data(), r->psi.empty() ? nullptr : r->psi.data());
          c.warm = rc == USBS_OK ? 1 : 0;
        }
        if (!c.warm) {   // cold start, also when the problem does not extend the parent
          ctx = nullptr;
          rc = usbs_create(&ctx, r->n, r->rowptr.data(), r->col.data(), r->val.data(), r->m, r->nnzA,
                           r->acon.data(), r->ai.data(), r->aj.data(), r->aval.data(), r->b.data(),
                           r->ineq.data(), r->psi.empty() ? nullptr : r->psi.data(), &sp);
        }
        if (rc == USBS_OK) {
          usbs_result res{};
          rc = usbs_solve(ctx, c.warm, r->tol, &res);
          c.iters = res.iters;
          c.objective = res.last.objective;
          c.dual_bound = res.last.dual_bound;
          c.relgap = res.last.relgap;
          c.relinf = res.last.relinf;
        }
        c.status = rc;
        if (rc != USBS_OK && rc != USBS_ENOTCONV && ctx) {
          usbs_destroy(ctx);
          ctx = nullptr;
        }
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        c.t_finish = now();
        done.push_back(c);
        ++finished;
        --running;
        // the parent goes back to the cache (as most recent)
        if (r->parent_bytes > 0)
          cache.push_front({r->parent, r->parent_ctx, r->parent_bytes});
        const bool keep = p.cache_entries > 0 && (c.status == USBS_OK || c.status == USBS_ENOTCONV) &&
                          (p.dry_run || ctx);
        if (keep) {
          cache.push_front({r->id, ctx, r->bytes});
        } else {
          if (ctx) usbs_destroy(ctx);
          used -= r->bytes;
        }
        while ((int)cache.size() > p.cache_entries) {
          destroy_cached(cache.back());
          cache.pop_back();
        }
        admit();
      }
      cv_done.notify_all();
    }
  }
};

namespace usbs {

// device bytes of one context, following build_ctx's allocations
static uint64_t instance_bytes(int64_t n, int64_t nnz_off, int64_t m, int64_t nnzA, int r, int fp64,
                               bool offdiag_A) {
  const double es = fp64 ? 8.0 : 4.0;
  double b = 0.0;
  b += 4.0 * (n + 1) + nnz_off * (4.0 + 8.0 + es + (offdiag_A ? es : 0.0));  // pattern, values
  b += n * (8.0 + 2.0 * es);                                                    // diagonals
  b += 4.0 * (n + 1) + 12.0 * nnzA;                                             // diagonal lists
  b += 4.0 * (nnz_off + 1) + (offdiag_A ? 24.0 * nnzA : 0.0);                   // slot lists
  b += 4.0 * (m + 1) + nnzA * (8.0 + es) + 9.0 * m;                             // constraints, b
  b += 6.0 * 8.0 * m;                                                           // y, y~, AXbar, AX, nu, tmp
  b += es * 8.0 * n * (3 + 2 * NBMAX);                                          // V, V_new, W, Q, Q2
  b += 8.0 * n * r;                                                             // P, Psi
  b += 8.0 * ((double)parts_needed(n, m) * PART_STRIDE + RED_TOTAL) +
       2.0 * (sizeof(DevScalars) + sizeof(DevLanczos));
  return (uint64_t)(b * 1.02 + (1 << 20));                                      // + allocation slack
}

}  // namespace usbs

extern "C" {

uint64_t usbs_instance_bytes(int64_t n, int64_t nnzC, int64_t m, int64_t nnzA, int r,
                             int precision) {
  if (n < 1 || m < 1 || nnzA < 1 || nnzC < 0 || r < 0) return 0;
  // the merged pattern holds at most C's entries plus both orientations of A's
  return usbs::instance_bytes(n, nnzC + 2 * nnzA, m, nnzA, r, precision == USBS_PRECISION_FP64, true);
}

void usbs_server_params_default(usbs_server_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->hbm_budget_bytes = 0;
  p->max_slots = 8;
  p->cache_entries = 16;
  p->dry_run = 0;
  usbs_params_default(&p->solver);
}

int usbs_server_create(usbs_server** out, const usbs_server_params* p) {
  if (!out) return USBS_EINVAL;
  *out = nullptr;
  auto* s = new usbs_server();
  if (p) s->p = *p; else usbs_server_params_default(&s->p);
  if (s->p.max_slots < 1 || s->p.max_slots > 256 || s->p.cache_entries < 0) {
    delete s;
    return USBS_EINVAL;
  }
  if (s->p.hbm_budget_bytes == 0) {
    if (s->p.dry_run) {
      s->p.hbm_budget_bytes = (uint64_t)1 << 40;
    } else {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return USBS_ECUDA;
      }
      s->p.hbm_budget_bytes = (uint64_t)(0.8 * (double)fr);
    }
  }
  s->t0 = Clock::now();
  for (int i = 0; i < s->p.max_slots; ++i) s->workers.emplace_back([s, i] { s->worker(i); });
  *out = s;
  return USBS_OK;
}

int usbs_server_submit(usbs_server* s, int64_t request_id, int64_t parent_id, int64_t n,
                       const int64_t* C_rowptr, const int32_t* C_col, const double* C_val,
                       int64_t m, int64_t nnzA, const int32_t* A_con, const int32_t* A_i,
                       const int32_t* A_j, const double* A_val, const double* b,
                       const uint8_t* is_ineq, const float* Psi, double tol,
                       double fake_service_s) {
  if (!s || n < 1 || m < 1 || nnzA < 1 || !C_rowptr || !A_con || !A_i || !A_j || !A_val || !b ||
      !is_ineq || !(tol > 0.0))
    return USBS_EINVAL;
  auto r = std::make_unique<Req>();
  r->id = request_id;
  r->parent = parent_id;
  r->tol = tol;
  r->fake_s = fake_service_s;
  r->n = n;
  r->m = m;
  r->nnzA = nnzA;
  const int64_t nnzC = C_rowptr[n];
  if (nnzC < 0) return USBS_EINVAL;
  r->rowptr.assign(C_rowptr, C_rowptr + n + 1);
  if (nnzC > 0) {
    if (!C_col || !C_val) return USBS_EINVAL;
    r->col.assign(C_col, C_col + nnzC);
    r->val.assign(C_val, C_val + nnzC);
  }
  r->acon.assign(A_con, A_con + nnzA);
  r->ai.assign(A_i, A_i + nnzA);
  r->aj.assign(A_j, A_j + nnzA);
  r->aval.assign(A_val, A_val + nnzA);
  r->b.assign(b, b + m);
  r->ineq.assign(is_ineq, is_ineq + m);
  const int rk = s->p.solver.r;
  if (rk > 0) {
    if (!Psi) return USBS_EINVAL;
    r->psi.assign(Psi, Psi + n * rk);
  }
  r->bytes = usbs_instance_bytes(n, nnzC, m, nnzA, rk, s->p.solver.precision);
  std::lock_guard<std::mutex> lk(s->mu);
  r->t_arrival = s->now();
  s->pending.push_back(std::move(r));
  s->admit();
  return USBS_OK;
}

int usbs_server_poll(usbs_server* s, usbs_completion* out, int max, int wait_ms) {
  if (!s || !out || max < 1) return USBS_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
  const int k = std::min<int>(max, (int)s->done.size());
  for (int i = 0; i < k; ++i) out[i] = s->done[i];
  s->done.erase(s->done.begin(), s->done.begin() + k);
  return k;
}

int usbs_server_get_stats(usbs_server* s, usbs_server_stats* st) {
  if (!s || !st) return USBS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  st->used_bytes = s->used;
  st->peak_bytes = s->peak_used;
  st->budget_bytes = s->p.hbm_budget_bytes;
  st->pending = (int)s->pending.size();
  st->running = s->running;
  st->peak_running = s->peak_running;
  st->cached = (int)s->cache.size();
  st->finished = s->finished;
  st->rejected = s->rejected;
  return USBS_OK;
}

int usbs_server_destroy(usbs_server* s) {
  if (!s) return USBS_OK;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    // finish what is queued and running, then stop the workers
    s->cv_done.wait(lk, [&] { return s->pending.empty() && s->admitted.empty() && s->running == 0; });
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& c : s->cache)
    if (c.ctx) usbs_destroy(c.ctx);
  delete s;
  return USBS_OK;
}

int usbs_batch_solve(usbs_ctx** ctxs, int count, double tol, int max_concurrency,
                     usbs_result* results, int* status) {
  if (!ctxs || count < 0 || !results || !(tol > 0.0)) return USBS_EINVAL;
  if (count == 0) return USBS_OK;
  for (int i = 0; i < count; ++i)
    if (!ctxs[i]) return USBS_EINVAL;
  // contexts the persistent kernel can take, grouped by (precision, basis, size bucket);
  // one launch (a replayed CUDA graph) per group solves all of its instances
  std::vector<std::vector<usbs::Ctx*>> groups;
  std::vector<std::vector<int>> group_idx;
  std::vector<int> rest;
  for (int i = 0; i < count; ++i) {
    usbs::Ctx* c = reinterpret_cast<usbs::Ctx*>(ctxs[i]);
    if (!usbs::batch_eligible(c)) { rest.push_back(i); continue; }
    size_t g = 0;
    for (; g < groups.size(); ++g)
      if (groups[g][0]->fp64 == c->fp64 && groups[g][0]->J == c->J &&
          usbs::batch_bucket(groups[g][0]->n) == usbs::batch_bucket(c->n))
        break;
    if (g == groups.size()) { groups.emplace_back(); group_idx.emplace_back(); }
    groups[g].push_back(c);
    group_idx[g].push_back(i);
  }
  int worst = USBS_OK;
  for (size_t g = 0; g < groups.size(); ++g) {
    for (usbs::Ctx* c : groups[g])
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) return USBS_ECUDA;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return USBS_ECUDA;
    std::string err;
    const int rc = usbs::batch_run(groups[g], st, tol, err);
    cudaStreamDestroy(st);
    if (rc != USBS_OK) {
      for (usbs::Ctx* c : groups[g]) c->err = err;
      return rc;
    }
    for (size_t k = 0; k < groups[g].size(); ++k) {
      const int i = group_idx[g][k];
      const int r = usbs::batch_result(groups[g][k], &results[i]);
      if (status) status[i] = r;
      if (r != USBS_OK && r != USBS_ENOTCONV) worst = r;
    }
  }
  if (rest.empty()) return worst;
  const int nt = std::max(1, std::min((int)rest.size(), max_concurrency > 0 ? max_concurrency : 8));
  std::atomic<int> next{0};
  std::atomic<int> worst_t{USBS_OK};
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&] {
      for (;;) {
        const int k = next.fetch_add(1);
        if (k >= (int)rest.size()) break;
        const int i = rest[k];
        const int rc = usbs_solve(ctxs[i], 0, tol, &results[i]);
        if (status) status[i] = rc;
        if (rc != USBS_OK && rc != USBS_ENOTCONV) worst_t.store(rc);
      }
    });
  for (auto& t : th) t.join();
  return worst != USBS_OK ? worst : worst_t.load();
}

}  // extern "C"
