// ots_server.cu -- request loop with continuous batching (ots_server_* in include/ots.h).
//
// Threads of a server:
//   builders  take submitted requests, build the instance on the host (state graph, checks)
//             and upload it into the batch's device pool on their own stream.  A request that
//             does not fit in the free pool memory waits until a finished instance frees some
//             (admission by memory); builders never hold more prepared instances than there
//             are free slots.
//   driver    owns the batch: admits prepared instances into free slots between graph
//             launches, launches the tick graph while anything is resident, and retires
//             finished instances (flows and measures copied to the request, slot and memory
//             freed).  Requests that arrive while others run join the next launch, so their
//             work overlaps on the device.
//   large     solves, one at a time with the single-instance solver on its own stream,
//             the requests the batch kernel does not take (more than 256 commodities, or
//             per-commodity costs); its memory also comes from the pool.
// In plain mode (mode = 1) a single thread solves every request to completion, one after the
// other, with the single-instance solver: the one-instance-at-a-time baseline, same API.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "ots.h"
#include "ots_internal.h"

using namespace ots_host;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// A submitted request: owned copies of the descriptor's arrays, options, and the result.
struct Request {
  int64_t ticket = 0;
  ots_problem_desc d{};
  ots_solve_opts o{};
  std::vector<int32_t> esrc, edst, sc, ss, zc, zs, win_in, win_out, st_tail, st_head, st_hold;
  std::vector<double> ecost, ecap, wcost, wcap, ccost, cost_t, cap_t, ccap, sm, zm;
  int S = 0, T = 0;
  bool large = false;
  ots_problem *p = nullptr;                   // prepared batch member (between build and admit)
  int32_t batch_id = -1;
  ots_status status = OTS_PENDING;
  ots_solve_report rep{};
  std::vector<double> flows;                  // [T][S], t = 1..T
  std::string error;
  Clock::time_point t_submit, t_admit, t_done;
};

using ReqPtr = std::shared_ptr<Request>;

template <class T>
void copy_array(std::vector<T> &dst, const T *src, size_t n) {
  if (src && n) dst.assign(src, src + n);
  else dst.clear();
}

const double *ptr_or_null(const std::vector<double> &v) { return v.empty() ? nullptr : v.data(); }
const int32_t *ptr_or_null(const std::vector<int32_t> &v) { return v.empty() ? nullptr : v.data(); }

}  // namespace

struct ots_server {
  ots_server_desc desc{};
  ots_batch *batch = nullptr;
  int dev = 0;
  std::mutex mu;
  std::condition_variable cv_build, cv_drive, cv_large, cv_done;
  std::deque<ReqPtr> build_q, ready_q, large_q;
  std::map<int64_t, ReqPtr> all;              // every request not yet released
  std::map<int32_t, ReqPtr> resident;         // batch id -> request (driver thread)
  int64_t next_ticket = 1;
  int building = 0, large_running = 0;
  long long submitted = 0, completed = 0, failed = 0, batch_launches = 0;
  bool stop = false;
  std::vector<std::thread> threads;
};

namespace {

void finish(ots_server *s, const ReqPtr &r, ots_status st, const char *err) {
  // caller holds s->mu
  r->status = st;
  r->rep.status = st;
  r->t_done = Clock::now();
  r->rep.seconds = ms_between(r->t_submit, r->t_done) * 1e-3;
  if (err) r->error = err;
  if (st == OTS_OK) ++s->completed;
  else ++s->failed;
  s->cv_done.notify_all();
}

// Single-instance solve of one request (large lane and plain mode): create, solve, flows.
// With a batch, the instance's memory comes from the batch's pool: a request that does not
// fit waits until finished instances free enough of it.
void solve_single(ots_server *s, const ReqPtr &r, cudaStream_t stream) {
  ots_problem_desc d = r->d;
  d.device = s->dev;
  d.stream = stream;
  if (s->batch) {
    d.alloc = pool_alloc_cb;
    d.free_fn = pool_free_cb;
    d.alloc_ctx = batch_pool(s->batch);
  }
  ots_problem *p = nullptr;
  ots_status st = ots_create_problem(&d, &p);
  while (st == OTS_ERR_OOM && s->batch) {
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop || (s->resident.empty() && s->ready_q.empty() && s->building == 0)) break;
    s->cv_done.wait_for(lk, std::chrono::milliseconds(2));
    lk.unlock();
    st = ots_create_problem(&d, &p);
  }
  {
    std::unique_lock<std::mutex> lk(s->mu);
    r->t_admit = Clock::now();
  }
  ots_solve_report rep{};
  std::vector<double> flows;
  std::string err;
  if (st == OTS_OK) {
    st = ots_sinkhorn_solve(p, &r->o, &rep);
    if (st == OTS_OK || st == OTS_ERR_NOT_CONVERGED || st == OTS_ERR_TIMEOUT) {
      flows.resize((size_t)r->T * r->S);
      const ots_status fs = ots_get_flows(p, 1, r->T + 1, flows.data());
      if (fs != OTS_OK) { st = fs; flows.clear(); }
    }
  }
  if (st != OTS_OK) err = ots_last_error();
  ots_destroy_problem(p);
  std::unique_lock<std::mutex> lk(s->mu);
  r->rep = rep;
  r->flows.swap(flows);
  finish(s, r, st, err.empty() ? nullptr : err.c_str());
}

void builder_main(ots_server *s) {
  cudaSetDevice(s->dev);
  cudaStream_t stream = nullptr;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  for (;;) {
    ReqPtr r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // prepare no more instances than there are slots to put them in
      s->cv_build.wait(lk, [&] {
        return s->stop || (!s->build_q.empty() &&
                           (int)(s->resident.size() + s->ready_q.size()) + s->building < s->desc.batch.max_instances);
      });
      if (s->stop) break;
      r = s->build_q.front();
      s->build_q.pop_front();
      ++s->building;
    }
    ots_problem *p = nullptr;
    ots_status st = batch_prepare(s->batch, &r->d, stream, &p);
    if (st == OTS_OK && cudaStreamSynchronize(stream) != cudaSuccess) {
      st = fail(OTS_ERR_CUDA, "upload of a request failed");
      ots_destroy_problem(p);
      p = nullptr;
    }
    const std::string err = st == OTS_OK ? std::string() : std::string(ots_last_error());
    std::unique_lock<std::mutex> lk(s->mu);
    --s->building;
    if (st == OTS_ERR_OOM) {
      // not enough free pool memory now: wait for a finished instance (or fail if nothing
      // resident could ever free memory)
      if (s->resident.empty() && s->ready_q.empty() && s->building == 0) {
        finish(s, r, st, err.c_str());
      } else {
        s->build_q.push_front(r);
        s->cv_done.wait_for(lk, std::chrono::milliseconds(2));
      }
    } else if (st != OTS_OK) {
      finish(s, r, st, err.c_str());
    } else {
      r->p = p;
      s->ready_q.push_back(r);
      s->cv_drive.notify_one();
    }
    s->cv_build.notify_all();
  }
  if (stream) cudaStreamDestroy(stream);
}

void driver_main(ots_server *s) {
  cudaSetDevice(s->dev);
  std::vector<double> sf;
  for (;;) {
    // admit prepared instances
    std::vector<ReqPtr> admit;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_drive.wait(lk, [&] { return s->stop || !s->ready_q.empty() || !s->resident.empty(); });
      if (s->stop) break;
      while (!s->ready_q.empty() && (int)admit.size() < batch_free_slots(s->batch)) {
        admit.push_back(s->ready_q.front());
        s->ready_q.pop_front();
      }
    }
    for (auto &r : admit) {
      int32_t id = -1;
      ots_status st = batch_admit(s->batch, r->p, &r->o, &id);
      std::unique_lock<std::mutex> lk(s->mu);
      if (st != OTS_OK) {
        ots_destroy_problem(r->p);
        r->p = nullptr;
        finish(s, r, st, ots_last_error());
        continue;
      }
      r->p = nullptr;
      r->batch_id = id;
      r->t_admit = Clock::now();
      s->resident[id] = r;
    }
    if (s->resident.empty()) continue;
    int32_t running = 0;
    ots_status st = ots_batch_run(s->batch, 1, &running);
    std::vector<std::pair<int32_t, ReqPtr>> done;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      ++s->batch_launches;
      if (st != OTS_OK) {
        // a CUDA failure: every resident request fails with it
        for (auto &kv : s->resident) finish(s, kv.second, st, ots_last_error());
        s->resident.clear();
        continue;
      }
      for (auto &kv : s->resident) {
        ots_solve_report rep{};
        if (ots_batch_status(s->batch, kv.first, &rep) != OTS_PENDING) done.push_back(kv);
      }
    }
    for (auto &kv : done) {
      const ReqPtr &r = kv.second;
      ots_solve_report rep{};
      ots_status fs = ots_batch_status(s->batch, kv.first, &rep);
      std::vector<double> flows;
      if (fs == OTS_OK || fs == OTS_ERR_NOT_CONVERGED) {
        flows.resize((size_t)r->T * r->S);
        const ots_status gs = ots_batch_get_flows(s->batch, kv.first, 1, r->T + 1, flows.data());
        if (gs != OTS_OK) { fs = gs; flows.clear(); }
      }
      const std::string err = fs == OTS_OK ? std::string() : std::string(ots_last_error());
      ots_batch_remove(s->batch, kv.first);
      std::unique_lock<std::mutex> lk(s->mu);
      s->resident.erase(kv.first);
      r->rep = rep;
      r->flows.swap(flows);
      finish(s, r, fs, err.empty() ? nullptr : err.c_str());
      s->cv_build.notify_all();
    }
  }
}

void large_main(ots_server *s) {
  cudaSetDevice(s->dev);
  cudaStream_t stream = nullptr;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  for (;;) {
    ReqPtr r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_large.wait(lk, [&] { return s->stop || !s->large_q.empty(); });
      if (s->stop) break;
      r = s->large_q.front();
      s->large_q.pop_front();
      ++s->large_running;
    }
    solve_single(s, r, stream);
    std::unique_lock<std::mutex> lk(s->mu);
    --s->large_running;
  }
  if (stream) cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

ots_status ots_default_server_desc(ots_server_desc *d) {
  if (!d) return fail(OTS_ERR_INVALID_ARG, "desc is NULL");
  std::memset(d, 0, sizeof(*d));
  ots_default_batch_desc(&d->batch);
  d->batch.ticks_per_launch = 8;
  d->builder_threads = 2;
  d->mode = 0;
  return OTS_OK;
}

ots_status ots_server_create(const ots_server_desc *d, ots_server **out) {
  clear_error();
  if (!d || !out) return fail(OTS_ERR_INVALID_ARG, "desc or out is NULL");
  *out = nullptr;
  if (d->mode != 0 && d->mode != 1) return fail(OTS_ERR_INVALID_ARG, "mode must be 0 (batched) or 1 (plain)");
  if (d->builder_threads < 0 || d->max_queued < 0) return fail(OTS_ERR_INVALID_ARG, "bad server sizes");
  ots_server *s = new (std::nothrow) ots_server();
  if (!s) return fail(OTS_ERR_OOM, "host allocation failed");
  s->desc = *d;
  s->dev = d->batch.device;
  if (d->mode == 0) {
    ots_status st = ots_batch_create(&d->batch, &s->batch);
    if (st) { delete s; return st; }
    const int nb = d->builder_threads ? d->builder_threads : 2;
    for (int k = 0; k < nb; ++k) s->threads.emplace_back(builder_main, s);
    s->threads.emplace_back(driver_main, s);
  }
  s->threads.emplace_back(large_main, s);     // plain mode: the only solver thread
  *out = s;
  return OTS_OK;
}

ots_status ots_server_submit(ots_server *s, const ots_problem_desc *d, const ots_solve_opts *o, int64_t *ticket) {
  clear_error();
  if (!s || !d || !ticket) return fail(OTS_ERR_INVALID_ARG, "NULL argument");
  *ticket = 0;
  if (d->n_nodes < 1 || d->n_edges < 0 || d->T < 3 || d->L < 1 || d->n_sources < 0 || d->n_sinks < 0)
    return fail(OTS_ERR_INVALID_ARG, "bad sizes");
  auto r = std::make_shared<Request>();
  const size_t E = d->n_edges, V = d->n_nodes, S = E + (d->add_wait_loops ? V : 0);
  copy_array(r->esrc, d->edge_src, E);
  copy_array(r->edst, d->edge_dst, E);
  copy_array(r->ecost, d->edge_cost, E);
  copy_array(r->ecap, d->edge_capacity, E);
  copy_array(r->wcost, d->wait_cost, d->add_wait_loops ? V : 0);
  copy_array(r->wcap, d->wait_capacity, d->add_wait_loops ? V : 0);
  copy_array(r->ccost, d->commodity_cost, d->commodity_cost ? (size_t)d->L * S : 0);
  copy_array(r->cost_t, d->state_cost_t, d->state_cost_t ? (size_t)(d->T - 2) * S : 0);
  copy_array(r->cap_t, d->state_capacity_t, d->state_capacity_t ? (size_t)(d->T - 2) * S : 0);
  copy_array(r->win_in, d->commodity_t_in, d->commodity_t_in ? (size_t)d->L : 0);
  copy_array(r->ccap, d->commodity_capacity, d->commodity_capacity ? (size_t)d->L * S : 0);
  copy_array(r->win_out, d->commodity_t_out, d->commodity_t_out ? (size_t)d->L : 0);
  copy_array(r->st_tail, d->state_tail, d->state_tail ? S : 0);
  copy_array(r->st_head, d->state_head, d->state_head ? S : 0);
  copy_array(r->st_hold, d->state_hold, d->state_hold ? S : 0);
  copy_array(r->sc, d->src_commodity, d->n_sources);
  copy_array(r->ss, d->src_state, d->n_sources);
  copy_array(r->sm, d->src_mass, d->n_sources);
  copy_array(r->zc, d->snk_commodity, d->n_sinks);
  copy_array(r->zs, d->snk_state, d->n_sinks);
  copy_array(r->zm, d->snk_mass, d->n_sinks);
  r->d = *d;
  r->d.edge_src = ptr_or_null(r->esrc);
  r->d.edge_dst = ptr_or_null(r->edst);
  r->d.edge_cost = ptr_or_null(r->ecost);
  r->d.edge_capacity = ptr_or_null(r->ecap);
  r->d.wait_cost = ptr_or_null(r->wcost);
  r->d.wait_capacity = ptr_or_null(r->wcap);
  r->d.commodity_cost = ptr_or_null(r->ccost);
  r->d.state_cost_t = ptr_or_null(r->cost_t);
  r->d.state_capacity_t = ptr_or_null(r->cap_t);
  r->d.commodity_t_in = ptr_or_null(r->win_in);
  r->d.commodity_capacity = ptr_or_null(r->ccap);
  r->d.commodity_t_out = ptr_or_null(r->win_out);
  r->d.state_tail = ptr_or_null(r->st_tail);
  r->d.state_head = ptr_or_null(r->st_head);
  r->d.state_hold = ptr_or_null(r->st_hold);
  r->d.src_commodity = ptr_or_null(r->sc);
  r->d.src_state = ptr_or_null(r->ss);
  r->d.src_mass = ptr_or_null(r->sm);
  r->d.snk_commodity = ptr_or_null(r->zc);
  r->d.snk_state = ptr_or_null(r->zs);
  r->d.snk_mass = ptr_or_null(r->zm);
  r->d.stream = nullptr;
  r->d.alloc = nullptr;
  r->d.free_fn = nullptr;
  r->d.alloc_ctx = nullptr;
  ots_default_solve_opts(&r->o);
  if (o) r->o = *o;
  r->S = (int)S;
  r->T = d->T;
  r->large = s->desc.mode == 1 || d->L > 256 || d->commodity_cost != nullptr || d->commodity_capacity != nullptr ||
             d->commodity_t_in != nullptr || d->commodity_t_out != nullptr || d->state_tail != nullptr ||
             d->state_head != nullptr || d->state_hold != nullptr;
  r->t_submit = Clock::now();
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->desc.max_queued > 0) {
    const size_t open = s->build_q.size() + s->ready_q.size() + s->large_q.size() + s->resident.size() + s->building;
    if ((int)open >= s->desc.max_queued) return fail(OTS_ERR_OOM, "server queue full (%d requests)", s->desc.max_queued);
  }
  r->ticket = s->next_ticket++;
  s->all[r->ticket] = r;
  ++s->submitted;
  if (r->large) {
    s->large_q.push_back(r);
    s->cv_large.notify_one();
  } else {
    s->build_q.push_back(r);
    s->cv_build.notify_all();
  }
  *ticket = r->ticket;
  return OTS_OK;
}

ots_status ots_server_poll(ots_server *s, int64_t ticket, ots_solve_report *rep) {
  if (!s) return fail(OTS_ERR_INVALID_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(OTS_ERR_INVALID_ARG, "unknown ticket %lld", (long long)ticket);
  const Request &r = *it->second;
  if (rep) {
    *rep = r.rep;
    rep->status = r.status;
  }
  if (r.status != OTS_PENDING && r.status != OTS_OK && !r.error.empty()) fail(r.status, "%s", r.error.c_str());
  return r.status;
}

ots_status ots_server_wait(ots_server *s, int64_t ticket, double timeout_ms, ots_solve_report *rep) {
  if (!s) return fail(OTS_ERR_INVALID_ARG, "server is NULL");
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return fail(OTS_ERR_INVALID_ARG, "unknown ticket %lld", (long long)ticket);
    ReqPtr r = it->second;
    auto ready = [&] { return r->status != OTS_PENDING; };
    if (timeout_ms > 0) s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), ready);
    else s->cv_done.wait(lk, ready);
  }
  return ots_server_poll(s, ticket, rep);
}

ots_status ots_server_get_flows(ots_server *s, int64_t ticket, int32_t t_begin, int32_t t_end, double *out) {
  if (!s || !out) return fail(OTS_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(OTS_ERR_INVALID_ARG, "unknown ticket %lld", (long long)ticket);
  const Request &r = *it->second;
  if (r.status == OTS_PENDING) return OTS_PENDING;
  if (r.flows.empty()) return fail(r.status, "request finished without flows (%s)", ots_status_string(r.status));
  if (t_begin < 1 || t_end > r.T + 1 || t_begin >= t_end) return fail(OTS_ERR_INVALID_ARG, "bad t range");
  std::memcpy(out, r.flows.data() + (size_t)(t_begin - 1) * r.S, sizeof(double) * (size_t)(t_end - t_begin) * r.S);
  return OTS_OK;
}

ots_status ots_server_timing(ots_server *s, int64_t ticket, double *ms) {
  if (!s || !ms) return fail(OTS_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(OTS_ERR_INVALID_ARG, "unknown ticket %lld", (long long)ticket);
  const Request &r = *it->second;
  if (r.status == OTS_PENDING) return OTS_PENDING;
  const bool admitted = r.t_admit.time_since_epoch().count() != 0;
  ms[0] = admitted ? ms_between(r.t_submit, r.t_admit) : ms_between(r.t_submit, r.t_done);
  ms[1] = admitted ? ms_between(r.t_admit, r.t_done) : 0.0;
  ms[2] = ms_between(r.t_submit, r.t_done);
  return OTS_OK;
}

ots_status ots_server_release(ots_server *s, int64_t ticket) {
  if (!s) return fail(OTS_ERR_INVALID_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(OTS_ERR_INVALID_ARG, "unknown ticket %lld", (long long)ticket);
  if (it->second->status == OTS_PENDING) return fail(OTS_ERR_INVALID_ARG, "request %lld is still running", (long long)ticket);
  s->all.erase(it);
  return OTS_OK;
}

ots_status ots_server_info(ots_server *s, ots_server_stats *o) {
  if (!s || !o) return fail(OTS_ERR_INVALID_ARG, "NULL argument");
  std::memset(o, 0, sizeof(*o));
  std::unique_lock<std::mutex> lk(s->mu);
  o->submitted = s->submitted;
  o->completed = s->completed;
  o->failed = s->failed;
  o->queued = (int32_t)(s->build_q.size() + s->ready_q.size() + s->large_q.size());
  o->building = s->building;
  o->resident = (int32_t)s->resident.size();
  o->large_running = s->large_running;
  o->batch_launches = s->batch_launches;
  if (s->batch) {
    ots_batch_stats bs{};
    ots_batch_info(s->batch, &bs);
    o->pool_bytes = bs.pool_bytes;
    o->pool_used = bs.pool_used;
    o->batch_ticks = bs.ticks;
  }
  return OTS_OK;
}

void ots_server_destroy(ots_server *s) {
  if (!s) return;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_build.notify_all();
  s->cv_drive.notify_all();
  s->cv_large.notify_all();
  for (auto &t : s->threads) t.join();
  for (auto &kv : s->all)
    if (kv.second->p) ots_destroy_problem(kv.second->p);
  if (s->batch) ots_batch_destroy(s->batch);
  delete s;
}

}  // extern "C"
