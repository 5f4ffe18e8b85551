// Serving runtime (include/fmpb.h, "Serving"): request queue, two worker
// threads with their own CUDA streams, an operator cache keyed by
// (mesh, lattice, k, form, n_t, precision) with LRU eviction, admission by
// HBM footprint and continuous batching of the right-hand sides of queued
// requests that share an operator.
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

#include "common.cuh"
#include "internal.cuh"

namespace fmpb {

fmpb_status plan_operator(const double* verts, int64_t nv, const int32_t* tris, int64_t ntri,
                          const fmpb_lattice* lattice, const fmpb_operator_opts* opts, int* form, int64_t* B,
                          int64_t* F, size_t* bytes);

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

uint64_t fnv1a(const void* data, size_t n, uint64_t h) {
  const unsigned char* p = (const unsigned char*)data;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

struct Request {
  uint64_t ticket = 0;
  std::vector<double> verts;
  std::vector<int32_t> tris;
  fmpb_lattice lattice;
  double k = 0;
  int form = FMPB_FORM_AUTO, n_t = 0, R = 1;
  std::vector<double> dirs;
  std::vector<fmpb_c64> amps;
  fmpb_c64* p_out = nullptr;
  uint64_t key = 0;
  int64_t N = 0;
  size_t op_bytes = 0, work_bytes = 0;
  // results
  fmpb_result res;
  bool done = false;
  Clock::time_point t_submit, t_start, t_end;
};

struct CacheEntry {
  uint64_t key;
  fmpb_operator* op;
  size_t bytes;
  bool busy;
  Clock::time_point last_used;
};

}  // namespace
}  // namespace fmpb

using namespace fmpb;

struct fmpb_server {
  fmpb_server_opts opts;
  int device = 0;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> tickets;
  std::vector<CacheEntry> cache;
  std::vector<uint64_t> building;   // keys being built by a worker
  size_t hbm_in_use = 0, hbm_high = 0;
  std::vector<std::thread> workers;
  bool stop = false;
  uint64_t next_ticket = 1;
  // stats
  int64_t submitted = 0, completed = 0, failed = 0, hits = 0, batches = 0;
  std::vector<double> latencies;
  bool have_first = false;
  Clock::time_point first_submit, last_done;

  bool key_busy(uint64_t key) {
    for (auto& c : cache)
      if (c.key == key && c.busy) return true;
    return std::find(building.begin(), building.end(), key) != building.end();
  }

  // Evicts idle operators (least recently used first) until `need` fits.
  bool make_room(size_t need) {
    while (hbm_in_use + need > budget) {
      int victim = -1;
      for (int i = 0; i < (int)cache.size(); ++i)
        if (!cache[i].busy && (victim < 0 || cache[i].last_used < cache[victim].last_used)) victim = i;
      if (victim < 0) return false;
      fmpb_operator_destroy(cache[victim].op);
      hbm_in_use -= cache[victim].bytes;
      cache.erase(cache.begin() + victim);
    }
    return true;
  }

  void worker_main() {
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
      std::vector<Request*> batch;
      fmpb_operator* cached = nullptr;
      bool build = false;
      size_t reserved = 0;
      {
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
          if (stop && queue.empty()) {
            if (st) cudaStreamDestroy(st);
            return;
          }
          // first queued request whose operator is not in use by the other worker
          auto it = std::find_if(queue.begin(), queue.end(), [&](Request* r) { return !key_busy(r->key); });
          if (it != queue.end()) {
            Request* head = *it;
            const uint64_t key = head->key;
            int rhs = 0;
            for (auto q = queue.begin(); q != queue.end();) {
              if ((*q)->key == key && (batch.empty() || rhs + (*q)->R <= opts.max_batch_rhs)) {
                rhs += (*q)->R;
                batch.push_back(*q);
                q = queue.erase(q);
              } else {
                ++q;
              }
            }
            break;
          }
          cv_work.wait(lk);
        }
        Request* head = batch[0];
        auto find_entry = [&]() -> CacheEntry* {
          for (auto& c : cache)
            if (c.key == head->key) return &c;
          return nullptr;
        };
        CacheEntry* entry = find_entry();
        size_t work = 0;
        for (Request* r : batch) work += r->work_bytes;
        const size_t need = work + (entry ? 0 : head->op_bytes);
        const auto now = Clock::now();
        for (Request* r : batch) r->t_start = now;
        if (entry) entry->busy = true;   // pin it before evicting anything
        const bool fits = make_room(need);
        entry = find_entry();             // eviction may have moved the entry
        if (!fits) {
          if (entry) entry->busy = false;
          for (Request* r : batch) {
            r->res.status = FMPB_ENOMEM;
            r->done = true;
            r->t_end = now;
            ++failed;
          }
          cv_done.notify_all();
          cv_work.notify_all();
          continue;
        }
        hbm_in_use += need;
        hbm_high = std::max(hbm_high, hbm_in_use);
        reserved = work;
        if (!entry) {
          build = true;
          building.push_back(head->key);
        } else {
          entry->last_used = now;
          cached = entry->op;
          ++hits;
        }
        ++batches;
      }
      run_batch(batch, cached, build, reserved, st);
    }
  }

  void run_batch(std::vector<Request*>& batch, fmpb_operator* cached, bool build, size_t reserved, cudaStream_t st) {
    Request* head = batch[0];
    fmpb_operator* op = cached;
    fmpb_status s = FMPB_OK;
    auto t0 = Clock::now();
    if (build) {
      fmpb_operator_opts oo{head->form, head->n_t, opts.precision};
      s = fmpb_operator_create(head->verts.data(), (int64_t)head->verts.size() / 3, head->tris.data(),
                               (int64_t)head->tris.size() / 3, &head->lattice, head->k, &oo, st, &op);
    }
    auto t1 = Clock::now();
    int R = 0;
    for (Request* r : batch) R += r->R;
    const int64_t N = head->N;
    std::vector<fmpb_solve_info> info(R);
    fmpb_c64 *b = nullptr, *p = nullptr;
    if (s == FMPB_OK) {
      if (cudaMalloc(&b, sizeof(fmpb_c64) * (size_t)R * N) != cudaSuccess ||
          cudaMalloc(&p, sizeof(fmpb_c64) * (size_t)R * N) != cudaSuccess) {
        cudaGetLastError();
        s = FMPB_ENOMEM;
      }
    }
    if (s == FMPB_OK) {
      std::vector<double> dirs;
      std::vector<fmpb_c64> amps;
      for (Request* r : batch) {
        dirs.insert(dirs.end(), r->dirs.begin(), r->dirs.end());
        amps.insert(amps.end(), r->amps.begin(), r->amps.end());
      }
      s = fmpb_rhs_plane_wave(op, R, dirs.data(), amps.data(), b, st);
      if (s == FMPB_OK) {
        fmpb_solve_opts so{opts.tol, opts.restart, opts.maxit, 0, 0.0};
        s = fmpb_solve(op, R, b, p, &so, info.data(), st);
      }
      if (s == FMPB_OK || s == FMPB_ENOCONV) {
        int64_t off = 0;
        for (Request* r : batch) {
          if (cudaMemcpyAsync(r->p_out, p + off * N, sizeof(fmpb_c64) * (size_t)r->R * N, cudaMemcpyDeviceToHost,
                              st) != cudaSuccess)
            s = FMPB_ECUDA;
          off += r->R;
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) s = FMPB_ECUDA;
      }
    }
    cudaFree(b);
    cudaFree(p);
    auto t2 = Clock::now();
    std::lock_guard<std::mutex> lk(mu);
    if (build) {
      building.erase(std::find(building.begin(), building.end(), head->key));
      if (op && s != FMPB_EINVAL) {
        cache.push_back(CacheEntry{head->key, op, head->op_bytes, false, t2});
        if ((int)cache.size() > opts.cache_entries) {
          // drop the least recently used idle entry beyond the cap
          int victim = -1;
          for (int i = 0; i < (int)cache.size(); ++i)
            if (!cache[i].busy && cache[i].key != head->key &&
                (victim < 0 || cache[i].last_used < cache[victim].last_used))
              victim = i;
          if (victim >= 0) {
            fmpb_operator_destroy(cache[victim].op);
            hbm_in_use -= cache[victim].bytes;
            cache.erase(cache.begin() + victim);
          }
        }
      } else {
        if (op) fmpb_operator_destroy(op);
        hbm_in_use -= head->op_bytes;
      }
    } else {
      for (auto& c : cache)
        if (c.key == head->key) {
          c.busy = false;
          c.last_used = t2;
        }
    }
    hbm_in_use -= reserved;
    int64_t off = 0;
    for (Request* r : batch) {
      r->t_end = t2;
      fmpb_status rs = s;
      if (s == FMPB_ENOCONV) {
        rs = FMPB_OK;
        for (int q = 0; q < r->R; ++q)
          if (!info[off + q].converged) rs = FMPB_ENOCONV;
      }
      r->res.status = rs;
      r->res.R = r->R;
      r->res.cache_hit = build ? 0 : 1;
      r->res.batched_with = (int)batch.size();
      r->res.build_ms = ms_since(t0, t1);
      r->res.solve_ms = ms_since(t1, t2);
      r->res.queue_ms = ms_since(r->t_submit, r->t_start);
      r->res.latency_ms = ms_since(r->t_submit, t2);
      int it = 0;
      double rr = 0.0;
      for (int q = 0; q < r->R; ++q) {
        it = std::max(it, info[off + q].iters);
        rr = std::max(rr, info[off + q].relres_true);
      }
      off += r->R;
      r->res.iters_max = it;
      r->res.relres_true_max = rr;
      r->done = true;
      if (rs == FMPB_OK) {
        ++completed;
        latencies.push_back(r->res.latency_ms);
        last_done = t2;
      } else {
        ++failed;
      }
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
};

extern "C" {

fmpb_status fmpb_server_create(const fmpb_server_opts* opts, fmpb_server** out) {
  if (!out) {
    set_error("server_create: out is NULL");
    return FMPB_EINVAL;
  }
  fmpb_server_opts o = opts ? *opts : fmpb_server_opts{0, 0, 0, FMPB_FP64, 0.0, 0, 0};
  if (o.max_batch_rhs <= 0) o.max_batch_rhs = 64;
  if (o.cache_entries <= 0) o.cache_entries = 8;
  if (o.restart <= 0) o.restart = 200;
  if (o.maxit <= 0) o.maxit = 3000;
  if (o.tol <= 0) o.tol = 1e-8;
  if (o.max_batch_rhs > 4096 || o.restart > 1000) {
    set_error("server_create: max_batch_rhs <= 4096 and restart <= 1000");
    return FMPB_EINVAL;
  }
  if (o.precision != FMPB_FP64 && o.precision != FMPB_FP32 && o.precision != FMPB_MIXED) {
    set_error("server_create: bad precision");
    return FMPB_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "server_create: cudaGetDevice");
  size_t freeb = 0, totalb = 0;
  e = cudaMemGetInfo(&freeb, &totalb);
  if (e != cudaSuccess) return cuda_status(e, "server_create: cudaMemGetInfo");
  fmpb_server* s = new (std::nothrow) fmpb_server();
  if (!s) {
    set_error("server_create: host allocation failed");
    return FMPB_ENOMEM;
  }
  s->opts = o;
  s->device = dev;
  s->budget = o.hbm_budget_bytes ? o.hbm_budget_bytes : (size_t)(0.8 * (double)freeb);
  for (int w = 0; w < 2; ++w) s->workers.emplace_back([s] { s->worker_main(); });
  *out = s;
  return FMPB_OK;
}

fmpb_status fmpb_server_submit(fmpb_server* srv, const fmpb_request* q, fmpb_c64* p_out, uint64_t* ticket) {
  if (!srv || !q || !p_out || !ticket || !q->verts || !q->tris || !q->dirs) {
    set_error("server_submit: NULL argument");
    return FMPB_EINVAL;
  }
  if (q->R < 1 || q->R > 64 || q->R > srv->opts.max_batch_rhs || !(q->k > 0.0)) {
    set_error("server_submit: need 1 <= R <= min(64, max_batch_rhs) and k > 0");
    return FMPB_EINVAL;
  }
  if (q->nv < 3 || q->ntri < 1 || q->ntri > (1 << 20)) {
    set_error("server_submit: bad mesh sizes");
    return FMPB_EINVAL;
  }
  fmpb_operator_opts oo{q->form, q->n_t, srv->opts.precision};
  int form = 0;
  int64_t B = 0, F = 0;
  size_t op_bytes = 0;
  FMPB_TRY(plan_operator(q->verts, q->nv, q->tris, q->ntri, &q->lattice, &oo, &form, &B, &F, &op_bytes));
  Request* r = new (std::nothrow) Request();
  if (!r) {
    set_error("server_submit: host allocation failed");
    return FMPB_ENOMEM;
  }
  r->verts.assign(q->verts, q->verts + 3 * q->nv);
  r->tris.assign(q->tris, q->tris + 3 * q->ntri);
  r->lattice = q->lattice;
  r->k = q->k;
  r->form = form;
  r->n_t = q->n_t;
  r->R = q->R;
  r->dirs.assign(q->dirs, q->dirs + 3 * q->R);
  r->amps.resize(q->R);
  for (int i = 0; i < q->R; ++i) r->amps[i] = q->amps ? q->amps[i] : fmpb_c64{1.0, 0.0};
  r->p_out = p_out;
  int64_t cells = (int64_t)q->lattice.counts[0] * q->lattice.counts[1] * q->lattice.counts[2];
  r->N = q->ntri * cells;
  r->op_bytes = op_bytes;
  const int m = srv->opts.restart;
  r->work_bytes = sizeof(fmpb_c64) * ((size_t)(m + 6) * q->R * r->N + 2 * (size_t)F * q->R * B + 2 * (size_t)cells * q->R * B);
  uint64_t h = 1469598103934665603ull;
  h = fnv1a(r->verts.data(), r->verts.size() * sizeof(double), h);
  h = fnv1a(r->tris.data(), r->tris.size() * sizeof(int32_t), h);
  h = fnv1a(&q->lattice, sizeof(fmpb_lattice), h);
  h = fnv1a(&q->k, sizeof(double), h);
  int tag[3] = {form, q->n_t, srv->opts.precision};
  h = fnv1a(tag, sizeof(tag), h);
  r->key = h;
  r->res = fmpb_result{};
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    r->ticket = srv->next_ticket++;
    r->t_submit = Clock::now();
    if (!srv->have_first) {
      srv->first_submit = r->t_submit;
      srv->have_first = true;
    }
    srv->tickets[r->ticket] = r;
    srv->queue.push_back(r);
    ++srv->submitted;
    *ticket = r->ticket;
  }
  srv->cv_work.notify_all();
  return FMPB_OK;
}

fmpb_status fmpb_server_wait(fmpb_server* srv, uint64_t ticket, int timeout_ms, fmpb_result* res) {
  if (!srv || !res) {
    set_error("server_wait: NULL argument");
    return FMPB_EINVAL;
  }
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->tickets.find(ticket);
  if (it == srv->tickets.end()) {
    set_error("server_wait: unknown ticket %llu", (unsigned long long)ticket);
    return FMPB_EINVAL;
  }
  Request* r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_ms > 0) {
    if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
      set_error("server_wait: ticket %llu still running after %d ms", (unsigned long long)ticket, timeout_ms);
      return FMPB_ETIMEOUT;
    }
  } else {
    srv->cv_done.wait(lk, ready);
  }
  *res = r->res;
  srv->tickets.erase(it);
  delete r;
  return FMPB_OK;
}

fmpb_status fmpb_server_get_stats(fmpb_server* srv, fmpb_server_stats* st) {
  if (!srv || !st) {
    set_error("server_get_stats: NULL argument");
    return FMPB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  st->submitted = srv->submitted;
  st->completed = srv->completed;
  st->failed = srv->failed;
  st->cache_hits = srv->hits;
  st->batches = srv->batches;
  std::vector<double> l = srv->latencies;
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) { return l.empty() ? 0.0 : l[std::min(l.size() - 1, (size_t)(q * (l.size() - 1) + 0.5))]; };
  st->p50_ms = pct(0.50);
  st->p99_ms = pct(0.99);
  double sum = 0.0;
  for (double v : l) sum += v;
  st->mean_ms = l.empty() ? 0.0 : sum / l.size();
  const double span = srv->completed ? ms_since(srv->first_submit, srv->last_done) : 0.0;
  st->solves_per_s = span > 0 ? srv->completed / (span / 1e3) : 0.0;
  st->hbm_in_use = srv->hbm_in_use;
  st->hbm_high_water = srv->hbm_high;
  return FMPB_OK;
}

void fmpb_server_destroy(fmpb_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->workers) t.join();
  for (auto& c : srv->cache) fmpb_operator_destroy(c.op);
  for (auto& kv : srv->tickets) delete kv.second;
  delete srv;
}

}  // extern "C"
