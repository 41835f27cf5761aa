// Serving loop: many solve requests with different operators and right-hand-side counts on
// one GPU, with factorisations cached in HBM and continuous batching.
//
// - Requests are queued on submit. A pool of worker threads, each with its own CUDA stream,
//   takes work: the oldest pending request and every other pending request with the same
//   operator (mesh, k, xi_prob, xi_prec, subdomains, coarse mesh, precision) and the same
//   solver settings are solved together as one batch of right-hand sides, in a block of
//   slots with room to spare (twice the starting right-hand sides rounded up to 8, at most 32).
// - Continuous batching: at every GMRES restart boundary of a running batch its worker
//   retires the requests whose right-hand sides have all finished (results returned at once)
//   and admits pending requests of the same operator and settings into free slots (a
//   contiguous run per request); their right-hand sides start from x = 0 in the same solve.
//   Each slot keeps its own arithmetic, so a request's result does not depend on the requests
//   it shares the batch with. Batches of different operators run concurrently on the workers'
//   streams.
// - Factorisations are cached by the preconditioner key (everything but xi_prob: the
//   preconditioner is built from A_{xi_prec} only, Sec. 6.2), so requests that differ in
//   xi_prob share factors; the operator A_{xi_prob} is set per batch.
// - Admission: a new factorisation is admitted only if its local factors (band storage,
//   planned before allocation) plus the Krylov workspace of the batch fit in the memory
//   budget after evicting unused cached factorisations (least recently used first) and in
//   the device's free memory; otherwise the batch waits for memory to free up. While a batch
//   waits, no other batch starts and running batches admit no new requests, so the batches
//   that hold memory finish within their own iteration limits and the waiting batch is not
//   starved by continuous batching. It fails (MX_ENOMEM) only after 30 s in which no other
//   batch held memory.
// - Latency is measured per request from submit to completion on the host clock.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>

#include "problem.cuh"

namespace mx {

bool allocator_hooked();  // common.cu: a device-allocation hook is installed

namespace {

using Clock = std::chrono::steady_clock;

// columns [c0, c0 + nr) of a solver block [n][cap] <-> a user block [nr][n]
__global__ void k_put_cols(int64_t n, int cap, int c0, int nr, const double2* user, double2* in) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * nr; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % nr);
    const int64_t i = t / nr;
    in[i * cap + c0 + r] = user[(int64_t)r * n + i];
  }
}
__global__ void k_get_cols(int64_t n, int cap, int c0, int nr, const double2* in, double2* user) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * nr; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % nr);
    const int64_t i = t / nr;
    user[(int64_t)r * n + i] = in[i * cap + c0 + r];
  }
}

struct Key {
  int n, core, overlap, coarse, precision, bc, prec;
  double k, xi_prec;
  bool operator<(const Key& o) const {
    return std::tie(n, core, overlap, coarse, precision, bc, prec, k, xi_prec) <
           std::tie(o.n, o.core, o.overlap, o.coarse, o.precision, o.bc, o.prec, o.k, o.xi_prec);
  }
  bool operator==(const Key& o) const { return !(*this < o) && !(o < *this); }
};

struct Req {
  int64_t id = 0;
  Key key{};
  double xi_prob = 0, tol = 1e-6, width = 0.1;
  int restart = 0, max_it = 200, nrhs = 1, nbumps = 1;
  std::vector<double> centres, pol;
  std::vector<double2> x;
  std::vector<mx_rhs_stats> stats;
  int rc = MX_OK;
  std::string err;
  bool done = false, taken = false;
  int slot0 = -1, left = 0;  // first slot in the running batch, right-hand sides not finished
  Clock::time_point t_submit, t_start, t_done;
};

struct Entry {
  std::unique_ptr<Problem> P;
  int64_t bytes = 0;
  bool busy = false;
  uint64_t last_used = 0;
};

}  // namespace

struct Server {
  int64_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int64_t> pending;
  std::map<int64_t, std::unique_ptr<Req>> reqs;
  std::map<Key, Entry> cache;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  bool stop = false;
  int64_t next_id = 1;
  uint64_t clock = 0;
  int64_t cached_bytes = 0;
  int device = 0;
  // statistics
  int64_t batches = 0, factorisations = 0, evictions = 0, completed = 0, joined = 0;
  int mem_waiters = 0;  // batches waiting for their factorisation to fit the budget

  static bool same_batch(const Req& a, const Req& b) {
    return a.key == b.key && a.xi_prob == b.xi_prob && a.tol == b.tol && a.restart == b.restart &&
           a.max_it == b.max_it;
  }

  static int64_t workspace_bytes(const Key& k, int64_t n_dof, int nrhs, int m) {
    const int64_t esz = k.precision == MX_MIXED ? 8 : 16;
    return n_dof * nrhs * ((int64_t)(m + 1) * 16 + (int64_t)m * esz + 6 * 16) + (64LL << 20);
  }

  // Evict unused entries (least recently used first) until `need` more bytes fit the budget.
  bool make_room(int64_t need) {
    while (cached_bytes + need > budget) {
      auto victim = cache.end();
      for (auto it = cache.begin(); it != cache.end(); ++it)
        if (!it->second.busy && (victim == cache.end() || it->second.last_used < victim->second.last_used))
          victim = it;
      if (victim == cache.end()) return false;
      cached_bytes -= victim->second.bytes;
      cache.erase(victim);
      ++evictions;
    }
    return true;
  }

  // Restart-boundary hook of a running batch: records finished right-hand sides, returns the
  // requests whose right-hand sides have all finished, and admits pending requests of the same
  // operator and settings into free runs of slots.
  struct BatchHook : SlotHook {
    Server& S;
    Problem& P;
    cudaStream_t s;
    int64_t n;
    int cap;
    const Req tmpl;  // the settings every request of the batch shares
    double2* tmp;    // [32][n] user-layout scratch
    std::vector<Req*>& live;
    std::vector<Req*> owner;  // per slot

    BatchHook(Server& S_, Problem& P_, cudaStream_t s_, int64_t n_, int cap_, const Req& t, double2* tmp_,
              std::vector<Req*>& live_)
        : S(S_), P(P_), s(s_), n(n_), cap(cap_), tmpl(copy_settings(t)), tmp(tmp_), live(live_), owner(cap_, nullptr) {}

    static Req copy_settings(const Req& r) {
      Req t;
      t.key = r.key;
      t.xi_prob = r.xi_prob;
      t.tol = r.tol;
      t.restart = r.restart;
      t.max_it = r.max_it;
      return t;
    }

    void own(Req* r, int c0) {
      r->slot0 = c0;
      r->left = r->nrhs;
      r->stats.assign(r->nrhs, mx_rhs_stats{});
      for (int c = c0; c < c0 + r->nrhs; ++c) owner[c] = r;
    }

    std::vector<int> at_restart(const double2* x_dev, double2* b_dev, const std::vector<int>& finished,
                                const std::vector<int32_t>& its, const std::vector<double>& rel,
                                const std::vector<double>& est) override {
      std::vector<Req*> complete;
      for (int c : finished) {
        Req* r = owner[c];
        if (!r) continue;  // a free slot
        mx_rhs_stats& st = r->stats[c - r->slot0];
        st.iterations = its[c];
        st.converged = rel[c] <= tmpl.tol ? 1 : 0;
        st.rel_residual = rel[c];
        st.rel_estimate = est[c];
        if (--r->left == 0) complete.push_back(r);
      }
      for (Req* r : complete) {  // results out, slots free
        MX_LAUNCH(k_get_cols<<<grid_for(n * r->nrhs, 256), 256, 0, s>>>(n, cap, r->slot0, r->nrhs, x_dev, tmp));
        MX_CHECK_LAUNCH();
        r->x.resize((size_t)n * r->nrhs);
        MX_CUDA(cudaMemcpyAsync(r->x.data(), tmp, sizeof(double2) * n * r->nrhs, cudaMemcpyDeviceToHost, s));
        MX_CUDA(cudaStreamSynchronize(s));
        for (int c = r->slot0; c < r->slot0 + r->nrhs; ++c) owner[c] = nullptr;
      }
      std::vector<Req*> adm;
      {
        std::lock_guard<std::mutex> g(S.mu);
        const auto now = Clock::now();
        for (Req* r : complete) {
          // the worker lets go of the request before it is marked done: a poll may free it
          live.erase(std::remove(live.begin(), live.end(), r), live.end());
          r->rc = std::all_of(r->stats.begin(), r->stats.end(), [](const mx_rhs_stats& x) { return x.converged != 0; })
                      ? MX_OK
                      : MX_ENOCONV;
          r->t_done = now;
          r->done = true;
          ++S.completed;
        }
        for (int64_t id : S.pending) {
          if (S.stop) break;  // the server is shutting down: pending requests are dropped
          if (S.mem_waiters > 0) break;  // another batch waits for the memory this one holds
          Req* q = S.reqs[id].get();
          if (q->taken || !same_batch(*q, tmpl)) continue;
          int run = 0, start = -1;
          for (int c = 0; c < cap && start < 0; ++c) {
            run = owner[c] ? 0 : run + 1;
            if (run == q->nrhs) start = c - q->nrhs + 1;
          }
          if (start < 0) continue;
          own(q, start);
          q->taken = true;
          q->t_start = now;
          ++S.joined;
          adm.push_back(q);
        }
        if (!adm.empty())
          S.pending.erase(std::remove_if(S.pending.begin(), S.pending.end(),
                                         [&](int64_t id) { return S.reqs[id]->taken; }),
                          S.pending.end());
      }
      if (!complete.empty()) S.cv_done.notify_all();
      std::vector<int> filled;
      for (Req* q : adm) {
        live.push_back(q);
        load_vector(P, q->nrhs, q->nbumps, q->centres.data(), q->pol.data(), q->width, tmp);
        MX_LAUNCH(k_put_cols<<<grid_for(n * q->nrhs, 256), 256, 0, s>>>(n, cap, q->slot0, q->nrhs, tmp, b_dev));
        MX_CHECK_LAUNCH();
        for (int c = q->slot0; c < q->slot0 + q->nrhs; ++c) filled.push_back(c);
      }
      return filled;
    }
  };

  void work(int wid) {
    cudaSetDevice(device);
    cudaStream_t s = streams[wid];
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      // find a batch whose operator is not busy
      std::vector<Req*> batch;
      Entry* entry = nullptr;
      bool create = false;
      while (!stop) {
        batch.clear();
        for (int64_t id : pending) {
          if (mem_waiters > 0) break;  // a batch waits for memory: it goes first
          Req* r = reqs[id].get();
          if (r->taken) continue;
          auto it = cache.find(r->key);
          if (it != cache.end() && it->second.busy) continue;
          // gather every pending request of the same operator and settings, up to 32 rhs
          int nr = 0;
          for (int64_t id2 : pending) {
            Req* q = reqs[id2].get();
            if (q->taken || !same_batch(*q, *r) || nr + q->nrhs > 32) continue;
            batch.push_back(q);
            nr += q->nrhs;
          }
          entry = it != cache.end() ? &it->second : nullptr;
          create = entry == nullptr;
          break;
        }
        if (!batch.empty()) break;
        cv_work.wait(lk);
      }
      if (stop) return;
      for (Req* r : batch) r->taken = true;
      ++batches;  // counted when it starts: its requests may complete before the batch returns
      pending.erase(std::remove_if(pending.begin(), pending.end(),
                                   [&](int64_t id) { return reqs[id]->taken; }),
                    pending.end());
      const Key key = batch[0]->key;
      if (create) {
        entry = &cache[key];
        entry->busy = true;
      } else {
        entry->busy = true;
      }
      lk.unlock();

      int rc = MX_OK;
      std::string err;
      int64_t charged = 0;  // bytes admitted into the budget for a new factorisation
      int nrhs = 0;
      for (Req* r : batch) nrhs += r->nrhs;
      // slots of the batch: room for as many right-hand sides again, rounded up to 8, at most 32
      const int cap = std::min(32, std::max(nrhs, ((2 * nrhs + 7) / 8) * 8));
      std::vector<Req*> live(batch.begin(), batch.end());  // grows with requests admitted on the way
      int64_t n_batch = 0;
      const auto t_start = Clock::now();
      for (Req* r : batch) r->t_start = t_start;
      try {
        if (create) {
          std::unique_ptr<Problem> P(create_problem(key.n, key.k, batch[0]->xi_prob, key.xi_prec, key.core,
                                                    key.overlap, key.coarse, key.precision, s, key.bc));
          P->prec_kind = key.prec;
          const int m = batch[0]->restart > 0 ? std::min(batch[0]->restart, batch[0]->max_it) : batch[0]->max_it;
          const int64_t need = local_factor_bytes(*P) + workspace_bytes(key, P->fine.n_dof, cap, m);
          // admission: memory budget (after evictions) and the device's free memory
          MX_REQUIRE(need <= budget, MX_ENOMEM,
                     "request needs " + std::to_string(need) + " bytes, more than the whole budget");
          bool admitted = false, waiting = false;
          for (int idle = 0; !admitted && idle < 600;) {  // idle: 50 ms waits with no other batch holding memory
            bool held = false;
            {
              std::lock_guard<std::mutex> g(mu);
              if (stop) break;
              admitted = make_room(need);
              if (admitted) {
                cached_bytes += need;
                entry->bytes = need;
              }
              for (const auto& e : cache) held = held || (e.second.busy && e.second.bytes > 0 && !(e.first == key));
              if (!admitted && !waiting) {
                waiting = true;
                ++mem_waiters;
              }
            }
            size_t fr = 0, tot = 0;
            // the device's free memory says something only when the library allocates from the
            // driver itself: a caching allocator keeps freed blocks, which it will hand out again
            if (admitted && !allocator_hooked() && cudaMemGetInfo(&fr, &tot) == cudaSuccess && (int64_t)fr < need) {
              std::lock_guard<std::mutex> g(mu);
              cached_bytes -= need;
              entry->bytes = 0;
              admitted = false;
              if (!waiting) {
                waiting = true;
                ++mem_waiters;
              }
            }
            if (!admitted) {
              idle = held ? 0 : idle + 1;
              std::this_thread::sleep_for(std::chrono::milliseconds(50));
            }
          }
          if (waiting) {
            {
              std::lock_guard<std::mutex> g(mu);
              --mem_waiters;
            }
            cv_work.notify_all();  // batches held back while this one waited may start
          }
          MX_REQUIRE(admitted, MX_ENOMEM, "request does not fit the memory budget");
          charged = need;
          factor_problem(*P);
          {
            std::lock_guard<std::mutex> g(mu);
            entry->P = std::move(P);
            entry->bytes = need;
            ++factorisations;
          }
        }
        Problem& P = *entry->P;
        P.stream = s;
        P.xi_prob = batch[0]->xi_prob;
        const int64_t n = P.fine.n_dof;
        n_batch = n;
        DevBuf<double2> f((size_t)n * cap), bi((size_t)n * cap), xi((size_t)n * cap), tmp((size_t)n * 32);
        MX_CUDA(cudaMemsetAsync(f.p, 0, f.bytes(), s));  // free slots: zero right-hand sides
        // load vectors of the starting requests, stacked as one block of right-hand sides
        BatchHook hook(*this, P, s, n, cap, *batch[0], tmp.p, live);
        int r0 = 0;
        for (Req* r : batch) {
          load_vector(P, r->nrhs, r->nbumps, r->centres.data(), r->pol.data(), r->width, f.p + (int64_t)r0 * n);
          hook.own(r, r0);
          r0 += r->nrhs;
        }
        transpose_to_internal(f.p, bi.p, n, cap, s);
        (void)gmres_solve(P, bi.p, xi.p, cap, batch[0]->tol, batch[0]->restart, batch[0]->max_it, nullptr, &hook);
      } catch (const Error& e) {
        rc = e.code;
        err = e.what();
      } catch (const std::exception& e) {
        rc = MX_ECUDA;
        err = e.what();
      }
      lk.lock();
      if (create && !entry->P) {  // failed before caching
        cached_bytes -= charged;
        cache.erase(key);
      } else {
        entry->busy = false;
        entry->last_used = ++clock;
      }
      const auto t_done = Clock::now();
      for (Req* r : live) {  // requests no restart boundary completed
        if (r->done) continue;
        if (rc == MX_OK) {  // only when every right-hand side of the batch was zero: x = 0
          r->x.assign((size_t)r->nrhs * n_batch, double2{0, 0});
          r->stats.assign(r->nrhs, mx_rhs_stats{0, 1, 0.0, 0.0});
        }
        r->rc = rc;
        r->err = err;
        r->t_done = t_done;
        r->done = true;
        ++completed;
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
  }
};

}  // namespace mx

using namespace mx;

extern "C" {

MX_API int mx_server_create(int64_t budget_bytes, int workers, mx_server* out) {
  try {
    MX_REQUIRE(out && budget_bytes > 0 && workers >= 1 && workers <= 16, MX_EINVAL, "bad server arguments");
    auto S = new Server();
    S->budget = budget_bytes;
    cudaGetDevice(&S->device);
    for (int w = 0; w < workers; ++w) {
      cudaStream_t st;
      MX_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      S->streams.push_back(st);
    }
    for (int w = 0; w < workers; ++w) S->workers.emplace_back([S, w] { S->work(w); });
    *out = reinterpret_cast<mx_server>(S);
    set_last_error("");
    return MX_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

MX_API int mx_server_submit(mx_server sv, const mx_request* q, int64_t* ticket) {
  try {
    MX_REQUIRE(sv && q && ticket, MX_EINVAL, "null argument");
    MX_REQUIRE(q->nrhs >= 1 && q->nrhs <= 32 && q->nbumps >= 1 && q->centres && q->pol && q->width > 0 && q->tol > 0 &&
                   q->max_it >= 1 && q->restart >= 0,
               MX_EINVAL, "bad request");
    MX_REQUIRE(q->n_cells >= 1 && q->core_cells >= 1 && q->k > 0 &&
                   (q->xi_prec != 0 || q->boundary == MX_BC_IMPEDANCE) &&
                   (q->boundary == MX_BC_PEC || q->boundary == MX_BC_IMPEDANCE) &&
                   (q->coarse_cells == 0 || q->n_cells % q->coarse_cells == 0),
               MX_EINVAL, "bad operator in request");
    MX_REQUIRE(q->prec_kind >= MX_PREC_AS && q->prec_kind <= MX_PREC_ADEF1 &&
                   (q->prec_kind == MX_PREC_AS || q->overlap_cells >= 1) &&
                   (q->prec_kind <= MX_PREC_RAS || q->coarse_cells > 0),
               MX_EINVAL, "bad preconditioner in request");
    auto S = reinterpret_cast<Server*>(sv);
    auto r = std::make_unique<Req>();
    r->key = Key{q->n_cells, q->core_cells, q->overlap_cells, q->coarse_cells, q->precision,
                 q->boundary, q->prec_kind, q->k, q->xi_prec};
    r->xi_prob = q->xi_prob;
    r->tol = q->tol;
    r->restart = q->restart;
    r->max_it = q->max_it;
    r->nrhs = q->nrhs;
    r->nbumps = q->nbumps;
    r->width = q->width;
    r->centres.assign(q->centres, q->centres + (size_t)q->nrhs * q->nbumps * 3);
    r->pol.assign(q->pol, q->pol + (size_t)q->nrhs * q->nbumps * 6);
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    *ticket = r->id;
    S->pending.push_back(r->id);
    S->reqs[r->id] = std::move(r);
    S->cv_work.notify_one();
    set_last_error("");
    return MX_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

MX_API int mx_server_poll(mx_server sv, int64_t ticket, int wait, void* x, mx_rhs_stats* stats,
                          mx_request_timing* timing) {
  try {
    MX_REQUIRE(sv, MX_EINVAL, "null server");
    auto S = reinterpret_cast<Server*>(sv);
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    MX_REQUIRE(it != S->reqs.end(), MX_EINVAL, "unknown ticket");
    Req* r = it->second.get();
    if (!r->done) {
      if (!wait) return 1;  // still running
      S->cv_done.wait(lk, [&] { return r->done; });
    }
    if (x) std::memcpy(x, r->x.data(), r->x.size() * sizeof(double2));
    if (stats) std::copy(r->stats.begin(), r->stats.end(), stats);
    if (timing) {
      timing->latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
      timing->queue_ms = std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count();
      timing->n_dof = (int64_t)(r->x.size() / std::max(1, r->nrhs));
    }
    const int rc = r->rc;
    const std::string err = r->err;
    S->reqs.erase(it);
    lk.unlock();
    set_last_error(err);
    return rc;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

MX_API int mx_server_stats(mx_server sv, mx_server_info* out) {
  if (!sv || !out) return MX_EINVAL;
  auto S = reinterpret_cast<Server*>(sv);
  std::lock_guard<std::mutex> lk(S->mu);
  out->batches = S->batches;
  out->factorisations = S->factorisations;
  out->evictions = S->evictions;
  out->completed = S->completed;
  out->cached_bytes = S->cached_bytes;
  out->cached_operators = (int32_t)S->cache.size();
  out->pending = (int32_t)S->pending.size();
  out->waiting_for_memory = S->mem_waiters;
  out->joined = S->joined;
  return MX_OK;
}

MX_API void mx_server_destroy(mx_server sv) {
  if (!sv) return;
  auto S = reinterpret_cast<Server*>(sv);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto st : S->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  delete S;
}

}  // extern "C"
