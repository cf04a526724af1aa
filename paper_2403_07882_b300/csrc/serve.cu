// Serving: continuous batching of solve requests from many cases (meshes)
// on one GPU, admitted by an HBM budget, with hierarchies kept resident.
//
// A case is a fixed LDU face addressing (Alg. 1's "first iteration"
// structure). Each request brings new coefficients and a right-hand side for
// one case (a later nonlinear iteration): the case's resident solver runs a
// values-only resetup and a solve. Worker threads ("slots") take requests in
// arrival order, skipping requests whose case is busy or does not fit yet; a
// case's requests are served one at a time in submission order, different
// cases run concurrently on their own CUDA streams, so their kernels overlap
// on the device. A case that is not resident is admitted when its estimated
// footprint fits in the budget after evicting least-recently-used idle cases;
// a case larger than the whole budget is rejected. Every solve is
// deterministic, so a case's results do not depend on what else is running.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <memory>
#include <cstdio>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket;
  int case_id;
  const double *diag, *upper, *lower, *b;
  double* x;
  int mem;  // BCS_MEM_HOST or BCS_MEM_DEVICE for all five arrays
  Clock::time_point submitted;
};

struct Done {
  bool done = false;
  bcs_result res{};
  double latency_ms = 0.0;
};

struct Case {
  int n = 0, C = 0, F = 0;
  std::vector<int32_t> owner, neighbour;
  bcs_solver* solver = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;  // a request's start / end on the stream
  bool busy = false;
  size_t bytes = 0;        // measured device footprint (0 until first admission)
  size_t estimate = 0;     // footprint estimate before the first admission
  uint64_t last_use = 0;
};

}  // namespace

struct bcs_server {
  std::mutex mu;
  std::condition_variable work_cv, done_cv;
  bcs_config cfg{};
  size_t budget = 0, resident = 0;
  bool stopping = false;
  std::vector<std::unique_ptr<Case>> cases;
  std::deque<Request> queue;
  std::unordered_map<int64_t, Done> done;
  int64_t next_ticket = 1;
  uint64_t clock = 0;
  long long submitted = 0, completed = 0, rejected = 0, evictions = 0, admissions = 0;
  long long batches = 0, batched = 0;
  int max_batch = 1;  // > 1: a worker solves up to this many resident cases' requests together
  std::vector<double> latencies;
  std::vector<std::pair<double, double>> spans;  // request intervals on the GPU timeline (ms from t0)
  cudaEvent_t t0 = nullptr;                       // reference of the timeline, recorded at create / reset
  cudaStream_t tstream = nullptr;
  std::vector<std::thread> workers;
  int device = 0;
  std::string last_error;  // message of the most recent failed request (guarded by mu)
};

namespace {

// Device footprint estimate of a case before its first admission, after
// the solver's allocations: FP64 fine matrix, its host-input staging and its
// cycle-precision copy, about half as much again for the coarser levels, the
// index arrays, the Krylov vectors and the cycle vectors. After the first
// admission the measured footprint replaces it.
size_t estimate_bytes(const Case& c, const bcs_config& cfg) {
  const double nn = (double)c.n * c.n, nnz = (double)c.C + 2.0 * c.F, N = (double)c.C * c.n;
  const double mat = nnz * nn * 8.0;
  const double cyc = cfg.precision == BCS_PREC_FP64 ? 0.0 : (cfg.precision == BCS_PREC_FP32 ? 0.5 : 0.25);
  const double levels = 1.5 * (mat * (1.0 + cyc) + (double)c.C * nn * 12.0) + mat;
  const double index = nnz * 28.0 + (double)c.C * 48.0;
  const double krylov = cfg.solver == BCS_BICGSTAB ? N * 8.0 * 12.0
                                                   : N * (8.0 * (cfg.restart + 1) + 4.0 * cfg.restart + 40.0);
  return (size_t)(levels + index + krylov + 1.5 * N * 16.0);
}

void drop_device_state(Case& c) {
  if (c.solver) bcs_destroy(c.solver);
  if (c.ev_a) cudaEventDestroy(c.ev_a);
  if (c.ev_b) cudaEventDestroy(c.ev_b);
  if (c.stream) cudaStreamDestroy(c.stream);
  c.solver = nullptr;
  c.stream = nullptr;
  c.ev_a = c.ev_b = nullptr;
}

void release_case(bcs_server* srv, Case& c) {
  drop_device_state(c);
  srv->resident -= c.bytes;
}

// Time covered by at least one / at least two of the intervals, and their
// summed length.
void coverage(std::vector<std::pair<double, double>> sp, double* lo, double* hi, double* one, double* two,
              double* sum) {
  *lo = *hi = *one = *two = *sum = 0.0;
  if (sp.empty()) return;
  std::vector<std::pair<double, int>> ev;
  ev.reserve(2 * sp.size());
  *lo = sp[0].first;
  *hi = sp[0].second;
  for (const auto& s : sp) {
    ev.push_back({s.first, +1});
    ev.push_back({s.second, -1});
    *lo = std::min(*lo, s.first);
    *hi = std::max(*hi, s.second);
    *sum += s.second - s.first;
  }
  std::sort(ev.begin(), ev.end());
  int depth = 0;
  double prev = ev[0].first;
  for (const auto& e : ev) {
    const double dt = e.first - prev;
    if (depth >= 1) *one += dt;
    if (depth >= 2) *two += dt;
    depth += e.second;
    prev = e.first;
  }
}

// Called with the lock held. Returns true when the case is (or can be made)
// resident; may evict idle cases. *reject is set when it can never fit.
bool admit(bcs_server* srv, Case& c, bool* reject) {
  *reject = false;
  if (c.solver) return true;
  const size_t need = c.bytes ? c.bytes : c.estimate;
  if (need > srv->budget) {
    *reject = true;
    return false;
  }
  while (srv->resident + need > srv->budget) {
    Case* lru = nullptr;
    for (auto& o : srv->cases)
      if (o->solver && !o->busy && (!lru || o->last_use < lru->last_use)) lru = o.get();
    if (!lru) return false;  // everything resident is busy: wait
    release_case(srv, *lru);
    srv->evictions++;
  }
  srv->resident += need;
  c.bytes = need;  // reserve; corrected after setup
  return true;
}

void finish(bcs_server* srv, const Request& r, const bcs_result& res) {
  Done& d = srv->done[r.ticket];
  d.done = true;
  d.res = res;
  d.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - r.submitted).count();
  srv->latencies.push_back(d.latency_ms);
  srv->completed++;
}

// A batch of requests of distinct resident cases: each case's values-only
// resetup on its own stream, then one batched solve (the results equal the
// cases' solves alone bit for bit); requests whose resetup fails are
// answered on their own, and a batch the batched solver refuses is solved
// case by case.
void serve_batch(bcs_server* srv, const std::vector<Request>& reqs) {
  const int k = (int)reqs.size();
  std::vector<bcs_status> st(k, BCS_OK);
  std::vector<bcs_result> res(k);
  std::vector<bool> timed(k, false);
  std::vector<bcs_solver*> solvers;
  std::vector<const double*> bs;
  std::vector<double*> xs;
  std::vector<int> idx;
  for (int i = 0; i < k; ++i) {
    Case& c = *srv->cases[reqs[i].case_id];
    timed[i] = cudaEventRecord(c.ev_a, c.stream) == cudaSuccess;
    st[i] = bcs_set_values(c.solver, reqs[i].diag, reqs[i].upper, reqs[i].lower, reqs[i].mem);
    if (st[i] == BCS_OK) {
      solvers.push_back(c.solver);
      bs.push_back(reqs[i].b);
      xs.push_back(reqs[i].x);
      idx.push_back(i);
    }
  }
  if (!solvers.empty()) {
    std::vector<bcs_result> br(solvers.size());
    const bcs_status bst = bcs_solve_batch(solvers.data(), (int)solvers.size(), bs.data(), xs.data(),
                                           reqs[idx[0]].mem, br.data());
    const bool refused = bst == BCS_EINVAL || bst == BCS_ESTATE || bst == BCS_ECUDA || bst == BCS_ENOMEM;
    for (size_t q = 0; q < idx.size(); ++q) {
      const int i = idx[q];
      Case& c = *srv->cases[reqs[i].case_id];
      if (refused) st[i] = bcs_solve(c.solver, reqs[i].b, reqs[i].x, reqs[i].mem, &res[i]);
      else {
        res[i] = br[q];
        st[i] = (bcs_status)br[q].status;
      }
    }
    if (!refused) {
      std::lock_guard<std::mutex> lk(srv->mu);
      srv->batches++;
      srv->batched += (long long)idx.size();
    }
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  for (int i = 0; i < k; ++i) {
    Case& c = *srv->cases[reqs[i].case_id];
    res[i].status = st[i];
    // the batch ran on the first solver's stream: its end closes every span
    cudaStream_t end_stream = solvers.empty() ? c.stream : srv->cases[reqs[idx[0]].case_id]->stream;
    if (timed[i] && st[i] != BCS_ECUDA && cudaEventRecord(c.ev_b, end_stream) == cudaSuccess &&
        cudaEventSynchronize(c.ev_b) == cudaSuccess) {
      float a = 0.f, b = 0.f;
      if (cudaEventElapsedTime(&a, srv->t0, c.ev_a) == cudaSuccess &&
          cudaEventElapsedTime(&b, srv->t0, c.ev_b) == cudaSuccess && b > 0.f)
        srv->spans.push_back({std::max(0.f, a), b});
      else
        (void)cudaGetLastError();
    }
    if (st[i] == BCS_ECUDA || st[i] == BCS_ENOMEM || st[i] == BCS_SINGULAR_BLOCK || st[i] == BCS_EINVAL) {
      srv->last_error = c.solver ? bcs_last_error(c.solver) : "solver creation failed";
      srv->resident -= c.bytes;
      c.bytes = 0;
      drop_device_state(c);
    }
    c.busy = false;
    finish(srv, reqs[i], res[i]);
  }
  srv->done_cv.notify_all();
  srv->work_cv.notify_all();
}

void worker(bcs_server* srv) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  for (;;) {
    // first queued request whose case is idle and admissible; requests of
    // cases that can never fit are answered with BCS_REJECTED
    auto it = srv->queue.end();
    bool changed = false;
    for (auto q = srv->queue.begin(); q != srv->queue.end(); ++q) {
      Case& c = *srv->cases[q->case_id];
      if (c.busy) continue;
      bool reject = false;
      if (admit(srv, c, &reject)) {
        it = q;
        break;
      }
      if (reject) {
        bcs_result res{};
        res.status = BCS_REJECTED;
        finish(srv, *q, res);
        srv->rejected++;
        srv->queue.erase(q);
        srv->done_cv.notify_all();
        changed = true;
        break;
      }
    }
    if (changed) continue;
    if (it == srv->queue.end()) {
      if (srv->stopping && srv->queue.empty()) return;
      srv->work_cv.wait(lk);
      continue;
    }
    Request r = *it;
    srv->queue.erase(it);
    Case& c = *srv->cases[r.case_id];
    c.busy = true;
    c.last_use = ++srv->clock;
    const bool fresh = c.solver == nullptr;
    // batching: the first queued request of other idle resident cases with
    // the same block size and memory kind join this one
    std::vector<Request> more;
    if (srv->max_batch > 1 && !fresh) {
      for (auto q = srv->queue.begin(); q != srv->queue.end() && (int)more.size() + 1 < srv->max_batch;) {
        Case& o = *srv->cases[q->case_id];
        if (!o.busy && o.solver && o.n == c.n && q->mem == r.mem) {
          o.busy = true;
          o.last_use = ++srv->clock;
          more.push_back(*q);
          q = srv->queue.erase(q);
        } else {
          ++q;
        }
      }
    }
    if (!more.empty()) {
      lk.unlock();
      more.insert(more.begin(), r);
      serve_batch(srv, more);
      lk.lock();
      continue;
    }
    lk.unlock();

    bcs_result res{};
    bcs_status st = BCS_OK;
    if (fresh) {
      st = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) == cudaSuccess ? BCS_OK : BCS_ECUDA;
      if (st == BCS_OK && (cudaEventCreate(&c.ev_a) != cudaSuccess || cudaEventCreate(&c.ev_b) != cudaSuccess))
        st = BCS_ECUDA;
      if (st == BCS_OK) st = bcs_create(&c.solver, c.n, &srv->cfg, c.stream);
      if (st == BCS_OK)
        st = bcs_set_structure(c.solver, c.C, c.F, c.owner.data(), c.neighbour.data(), BCS_MEM_HOST);
    }
    const bool timed = st == BCS_OK && cudaEventRecord(c.ev_a, c.stream) == cudaSuccess;
    if (st == BCS_OK) st = bcs_set_values(c.solver, r.diag, r.upper, r.lower, r.mem);
    if (st == BCS_OK) st = bcs_solve(c.solver, r.b, r.x, r.mem, &res);
    res.status = st;
    const bool span_ok = timed && st != BCS_ECUDA && cudaEventRecord(c.ev_b, c.stream) == cudaSuccess &&
                         cudaEventSynchronize(c.ev_b) == cudaSuccess;
    const size_t actual = c.solver ? bcs_device_bytes(c.solver) : 0;

    lk.lock();
    if (span_ok) {
      float a = 0.f, b = 0.f;
      if (cudaEventElapsedTime(&a, srv->t0, c.ev_a) == cudaSuccess &&
          cudaEventElapsedTime(&b, srv->t0, c.ev_b) == cudaSuccess && b > 0.f)
        srv->spans.push_back({std::max(0.f, a), b});
      else
        (void)cudaGetLastError();
    }
    if (st == BCS_ECUDA || st == BCS_ENOMEM || st == BCS_SINGULAR_BLOCK || st == BCS_EINVAL) {
      srv->last_error = c.solver ? bcs_last_error(c.solver) : "solver creation failed";
      // drop the case's device state; a later request rebuilds it
      srv->resident -= c.bytes;
      c.bytes = 0;
      drop_device_state(c);
    } else if (actual) {
      srv->resident = srv->resident - c.bytes + actual;
      c.bytes = actual;
      // the estimate may have been low: evict idle cases until within budget
      while (srv->resident > srv->budget) {
        Case* lru = nullptr;
        for (auto& o : srv->cases)
          if (o.get() != &c && o->solver && !o->busy && (!lru || o->last_use < lru->last_use)) lru = o.get();
        if (!lru) break;
        release_case(srv, *lru);
        srv->evictions++;
      }
    }
    if (fresh) srv->admissions++;
    c.busy = false;
    finish(srv, r, res);
    srv->done_cv.notify_all();
    srv->work_cv.notify_all();
  }
}

}  // namespace

extern "C" {

BCS_API bcs_status bcs_server_create(bcs_server** out, size_t budget_bytes, int slots, const bcs_config* cfg) {
  if (!out || slots < 1 || slots > 64) return BCS_EINVAL;
  *out = nullptr;
  bcs_config c;
  if (cfg) c = *cfg;
  else bcs_config_default(&c);
  bcs_server* srv = new (std::nothrow) bcs_server();
  if (!srv) return BCS_ENOMEM;
  srv->cfg = c;
  srv->cfg.profile = 0;
  if (cudaGetDevice(&srv->device) != cudaSuccess) {
    (void)cudaGetLastError();
    delete srv;
    return BCS_ECUDA;
  }
  if (budget_bytes == 0) {
    size_t freeb = 0, total = 0;
    if (cudaMemGetInfo(&freeb, &total) != cudaSuccess) {
      (void)cudaGetLastError();
      delete srv;
      return BCS_ECUDA;
    }
    budget_bytes = (size_t)(0.8 * (double)freeb);
  }
  srv->budget = budget_bytes;
  if (cudaStreamCreateWithFlags(&srv->tstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&srv->t0) != cudaSuccess || cudaEventRecord(srv->t0, srv->tstream) != cudaSuccess ||
      cudaEventSynchronize(srv->t0) != cudaSuccess) {
    (void)cudaGetLastError();
    if (srv->t0) cudaEventDestroy(srv->t0);
    if (srv->tstream) cudaStreamDestroy(srv->tstream);
    delete srv;
    return BCS_ECUDA;
  }
  for (int i = 0; i < slots; ++i) srv->workers.emplace_back(worker, srv);
  *out = srv;
  return BCS_OK;
}

BCS_API bcs_status bcs_server_destroy(bcs_server* srv) {
  if (!srv) return BCS_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stopping = true;
  }
  srv->work_cv.notify_all();
  for (auto& t : srv->workers) t.join();
  for (auto& c : srv->cases) release_case(srv, *c);
  cudaEventDestroy(srv->t0);
  cudaStreamDestroy(srv->tstream);
  delete srv;
  return BCS_OK;
}

BCS_API bcs_status bcs_server_register_case(bcs_server* srv, int n, int32_t n_cells, int32_t n_faces,
                                            const int32_t* owner, const int32_t* neighbour, int* case_id) {
  if (!srv || !case_id || n < 1 || n > 8 || n_cells < 1 || n_faces < 0 || (n_faces > 0 && (!owner || !neighbour)))
    return BCS_EINVAL;
  auto c = std::make_unique<Case>();
  c->n = n;
  c->C = n_cells;
  c->F = n_faces;
  c->owner.assign(owner, owner + n_faces);
  c->neighbour.assign(neighbour, neighbour + n_faces);
  std::lock_guard<std::mutex> lk(srv->mu);
  c->estimate = estimate_bytes(*c, srv->cfg);
  *case_id = (int)srv->cases.size();
  srv->cases.push_back(std::move(c));
  return BCS_OK;
}

BCS_API bcs_status bcs_server_submit(bcs_server* srv, int case_id, const double* diag, const double* upper,
                                    const double* lower, const double* b, double* x, int mem, int64_t* ticket) {
  if (!srv || !ticket || !diag || !b || !x) return BCS_EINVAL;
  if (mem != BCS_MEM_HOST && mem != BCS_MEM_DEVICE) return BCS_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (case_id < 0 || case_id >= (int)srv->cases.size()) return BCS_EINVAL;
  if (srv->cases[case_id]->F > 0 && (!upper || !lower)) return BCS_EINVAL;
  Request r{srv->next_ticket++, case_id, diag, upper, lower, b, x, mem, Clock::now()};
  srv->done[r.ticket] = Done{};
  srv->queue.push_back(r);
  srv->submitted++;
  *ticket = r.ticket;
  srv->work_cv.notify_one();
  return BCS_OK;
}

BCS_API bcs_status bcs_server_wait(bcs_server* srv, int64_t ticket, int timeout_ms, bcs_result* res,
                                  double* latency_ms) {
  if (!srv) return BCS_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->done.find(ticket);
  if (it == srv->done.end()) return BCS_EINVAL;
  const auto pred = [&] { return srv->done[ticket].done; };
  if (timeout_ms < 0) srv->done_cv.wait(lk, pred);
  else if (!srv->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return BCS_TIMEOUT;
  Done d = srv->done[ticket];
  srv->done.erase(ticket);
  if (res) *res = d.res;
  if (latency_ms) *latency_ms = d.latency_ms;
  return (bcs_status)d.res.status;
}

BCS_API bcs_status bcs_server_set_batch(bcs_server* srv, int max_batch) {
  if (!srv || max_batch < 1 || max_batch > BCS_BATCH_MAX) return BCS_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->max_batch = max_batch;
  return BCS_OK;
}

BCS_API bcs_status bcs_server_get_stats(bcs_server* srv, bcs_server_stats* st) {
  if (!srv || !st) return BCS_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = srv->submitted;
  st->completed = srv->completed;
  st->rejected = srv->rejected;
  st->evictions = srv->evictions;
  st->admissions = srv->admissions;
  st->queued = (long long)srv->queue.size();
  st->resident_bytes = srv->resident;
  st->budget_bytes = srv->budget;
  int res_cases = 0;
  for (auto& c : srv->cases) res_cases += c->solver != nullptr;
  st->resident_cases = res_cases;
  st->batches = srv->batches;
  st->batched_requests = srv->batched;
  if (!srv->latencies.empty()) {
    std::vector<double> l = srv->latencies;
    std::sort(l.begin(), l.end());
    const auto pct = [&](double p) {
      const size_t k = (size_t)std::min<double>(l.size() - 1, std::ceil(p * l.size()) - 1);
      return l[k];
    };
    st->p50_ms = pct(0.50);
    st->p99_ms = pct(0.99);
    double s = 0.0;
    for (double v : l) s += v;
    st->mean_ms = s / l.size();
  }
  double lo, hi, one, two, sum;
  coverage(srv->spans, &lo, &hi, &one, &two, &sum);
  st->window_ms = hi - lo;
  if (hi > lo) {
    st->busy_frac = one / (hi - lo);
    st->overlap_frac = two / (hi - lo);
    st->mean_in_flight = sum / (hi - lo);
  }
  return BCS_OK;
}

BCS_API bcs_status bcs_server_last_error(bcs_server* srv, char* buf, size_t len) {
  if (!srv || !buf || !len) return BCS_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  std::snprintf(buf, len, "%s", srv->last_error.c_str());
  return BCS_OK;
}

BCS_API bcs_status bcs_server_reset_stats(bcs_server* srv) {
  if (!srv) return BCS_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->latencies.clear();
  srv->spans.clear();
  srv->submitted = srv->completed = srv->rejected = srv->evictions = srv->admissions = 0;
  srv->batches = srv->batched = 0;
  if (cudaEventRecord(srv->t0, srv->tstream) != cudaSuccess || cudaEventSynchronize(srv->t0) != cudaSuccess)
    return BCS_ECUDA;
  return BCS_OK;
}

}  // extern "C"
