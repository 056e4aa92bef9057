// Serving loop of the C ABI (declared in include/cosenu.h): a queue of
// independent runs executed by one batched solver under a device-memory budget.
//
// cosenu_submit() only queues a run and returns a ticket.  One worker thread
// owns the batch and repeats a round:
//   1. admission: queued runs, oldest first, join the batch while their
//      workspaces fit in the budget (and the member limit allows); the first
//      that does not fit stops admission (strict FIFO: no run is overtaken);
//   2. each admitted run gets its member grid, parameters and initial state;
//   3. the batch advances by the smallest number of steps any member still
//      needs, capped at the round length, so no run overshoots its step count
//      and new arrivals wait at most one round;
//   4. members that reached their step count, or whose error flag is set,
//      leave the batch: diagnostics, optional copy of the final state to the
//      caller's buffer, device memory released, result published.
// Results stay with the server until cosenu_poll / cosenu_wait collects them.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/cosenu.h"
#include "engine.cuh"

using namespace cosenu;

namespace {

thread_local std::string tl_serror;

enum Phase { kQueued, kRunning, kDone };

struct Job {
  uint64_t ticket = 0;
  cosenu_request req{};
  size_t bytes = 0;  // workspace bytes
  Phase phase = kQueued;
  bool cancel = false;
  cosenu_t member = nullptr;
  int64_t left = 0;  // steps still to take
  cosenu_result res{};
};

}  // namespace

struct cosenu_server_s {
  int device = 0;
  size_t budget = 0;
  int32_t max_running = 0;  // 0: no limit
  int32_t round_steps = 64;
  cosenu_batch_t batch = nullptr;
  std::chrono::steady_clock::time_point t0;

  std::mutex mu;
  std::condition_variable cv_work;  // worker: new runs, cancellation, stop
  std::condition_variable cv_done;  // waiters: results
  std::deque<Job*> queue;
  std::vector<Job*> running;  // worker-owned list (guarded by mu when read by stats)
  std::unordered_map<uint64_t, std::unique_ptr<Job>> jobs;
  uint64_t next_ticket = 1;
  size_t in_use = 0, peak = 0;
  int64_t submitted = 0, admitted = 0, finished = 0, rounds = 0, steps = 0;
  bool stop = false;
  std::thread worker;
  std::string error;
};

namespace {

int sfail(cosenu_server_t s, int code, const std::string& msg) {
  if (s) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->error = msg;
  } else {
    tl_serror = msg;
  }
  return code;
}

double now_s(const cosenu_server_t s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

// Publish a finished run (worker thread, mu held).
void finish(cosenu_server_t s, Job* j, int status) {
  j->res.status = status;
  j->res.t_done = now_s(s);
  j->phase = kDone;
  ++s->finished;
  s->cv_done.notify_all();
}

// Give the run its member grid and initial state (worker thread, mu not held).
int start_run(cosenu_server_t s, Job* j) {
  const cosenu_request& r = j->req;
  cosenu_t h = nullptr;
  int rc = cosenu_batch_add(s->batch, r.nz, r.nv, r.L, r.scheme, r.precision, &h);
  if (rc) return rc;
  j->member = h;
  rc = cosenu_set_params(h, &r.params);
  if (rc == COSENU_OK) {
    if (r.state)
      rc = cosenu_set_state(h, r.state, (size_t)8 * r.nz * r.nv);
    else
      rc = cosenu_set_state_collective(h, r.alpha, r.sigma_nu, r.sigma_nubar, r.eps0, r.seed);
  }
  return rc;
}

// Results of a member that leaves the batch (worker thread, mu not held).
int collect_run(Job* j, int status) {
  if (status != COSENU_OK) return status;
  int rc = cosenu_conserved(j->member, &j->res.conserved);
  if (rc == COSENU_OK && j->req.out_state)
    rc = cosenu_get_state(j->member, j->req.out_state, (size_t)8 * j->req.nz * j->req.nv);
  return rc;
}

void release(cosenu_server_t s, Job* j) {
  if (j->member) cosenu_batch_remove(s->batch, j->member);
  j->member = nullptr;
}

void worker_main(cosenu_server_t s) {
  cudaSetDevice(s->device);
  std::vector<uint32_t> flags;
  for (;;) {
    std::vector<Job*> admit;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty() || !s->running.empty(); });
      if (s->stop) break;
      // 1. admission, oldest first; cancelled queued runs finish here
      while (!s->queue.empty()) {
        Job* j = s->queue.front();
        if (j->cancel) {
          s->queue.pop_front();
          finish(s, j, COSENU_ECANCELLED);
          continue;
        }
        if (s->max_running > 0 &&
            (int32_t)(s->running.size() + admit.size()) >= s->max_running)
          break;
        if (s->in_use + j->bytes > s->budget) break;
        s->queue.pop_front();
        s->in_use += j->bytes;
        s->peak = std::max(s->peak, s->in_use);
        j->phase = kRunning;
        admit.push_back(j);
      }
    }
    // 2. members and initial states
    for (Job* j : admit) {
      const int rc = start_run(s, j);
      if (rc != COSENU_OK) release(s, j);
      std::lock_guard<std::mutex> lk(s->mu);
      if (rc != COSENU_OK) {
        s->in_use -= j->bytes;
        finish(s, j, rc);
        continue;
      }
      j->res.t_admit = now_s(s);
      j->left = j->req.nsteps;
      ++s->admitted;
      s->running.push_back(j);
    }
    // 3. one round of steps
    int64_t n = s->round_steps;
    bool any_cancel = false;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (Job* j : s->running) {
        n = std::min(n, j->left);
        any_cancel |= j->cancel;
      }
    }
    if (s->running.empty()) continue;
    int rc = COSENU_OK;
    if (n > 0 && !any_cancel) rc = cosenu_batch_step(s->batch, n);
    if (rc == COSENU_OK) rc = batch_member_flags(s->batch, &flags);
    std::unordered_map<cosenu_t, uint32_t> flag_of;  // error bits per member handle
    for (size_t i = 0; i < flags.size(); ++i)
      flag_of[cosenu_batch_member(s->batch, (int32_t)i)] = flags[i];
    if (rc == COSENU_OK && n > 0 && !any_cancel) {
      std::lock_guard<std::mutex> lk(s->mu);
      ++s->rounds;
      s->steps += n;
      for (Job* j : s->running) {
        j->left -= n;
        j->res.steps += n;
      }
    }
    // 4. members that leave the batch
    std::vector<std::pair<Job*, int>> leaving;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      std::vector<Job*> keep;
      for (Job* j : s->running) {
        int status = COSENU_OK;
        bool leave = j->left == 0;
        const uint32_t fl = flag_of.count(j->member) ? flag_of[j->member] : 0u;
        if (rc != COSENU_OK) {
          status = rc;
          leave = true;
        } else if (fl) {
          status = (fl & 2u) ? COSENU_ETIMEOUT : COSENU_ENONFINITE;
          leave = true;
        } else if (j->cancel) {
          status = COSENU_ECANCELLED;
          leave = true;
        }
        if (leave)
          leaving.push_back({j, status});
        else
          keep.push_back(j);
      }
      s->running = std::move(keep);
    }
    for (auto& jl : leaving) {
      const int status = collect_run(jl.first, jl.second);
      release(s, jl.first);
      std::lock_guard<std::mutex> lk(s->mu);
      s->in_use -= jl.first->bytes;
      finish(s, jl.first, status);
    }
  }
  // stopping: everything not finished is cancelled
  std::vector<Job*> rest;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    rest = s->running;
    s->running.clear();
    for (Job* j : s->queue) rest.push_back(j);
    s->queue.clear();
  }
  for (Job* j : rest) {
    release(s, j);
    std::lock_guard<std::mutex> lk(s->mu);
    if (j->phase == kRunning) s->in_use -= j->bytes;
    finish(s, j, COSENU_ECANCELLED);
  }
}

bool valid_request(const cosenu_request* r, std::string* why) {
  if (r->nsteps < 0) {
    *why = "nsteps must be >= 0";
    return false;
  }
  if (!r->state && (!(r->sigma_nu > 0.0) || !(r->sigma_nubar > 0.0))) {
    *why = "without a state, the collective initial state needs sigma_nu, sigma_nubar > 0";
    return false;
  }
  return true;
}

}  // namespace

extern "C" {

cosenu_server_t cosenu_server_create(size_t budget_bytes, int32_t max_running,
                                     int32_t round_steps) {
  if (budget_bytes == 0 || max_running < 0 || round_steps < 0) {
    sfail(nullptr, COSENU_EINVAL, "budget must be > 0; max_running, round_steps >= 0");
    return nullptr;
  }
  cosenu_server_t s = new (std::nothrow) cosenu_server_s;
  if (!s) {
    sfail(nullptr, COSENU_ENOMEM, "host allocation failed");
    return nullptr;
  }
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    sfail(nullptr, COSENU_ECUDA, "cudaGetDevice failed");
    delete s;
    return nullptr;
  }
  s->budget = budget_bytes;
  s->max_running = max_running;
  if (round_steps > 0) s->round_steps = round_steps;
  s->t0 = std::chrono::steady_clock::now();
  s->batch = cosenu_batch_create();
  if (!s->batch) {
    sfail(nullptr, COSENU_ECUDA, std::string("batch: ") + cosenu_batch_last_error(nullptr));
    delete s;
    return nullptr;
  }
  try {
    s->worker = std::thread(worker_main, s);
  } catch (...) {
    cosenu_batch_destroy(s->batch);
    delete s;
    sfail(nullptr, COSENU_ENOMEM, "could not start the worker thread");
    return nullptr;
  }
  return s;
}

void cosenu_server_destroy(cosenu_server_t s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cosenu_batch_destroy(s->batch);
  delete s;
}

int cosenu_submit(cosenu_server_t s, const cosenu_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket) return sfail(s, COSENU_EINVAL, "NULL argument");
  *ticket = 0;
  std::string why;
  if (!valid_request(r, &why)) return sfail(s, COSENU_EINVAL, why);
  const size_t bytes = cosenu_workspace_bytes(r->nz, r->nv, r->scheme, r->precision);
  if (bytes == 0) return sfail(s, COSENU_EINVAL, "invalid grid size, scheme or precision");
  if (bytes > s->budget)
    return sfail(s, COSENU_ENOMEM, "the run's workspace (" + std::to_string(bytes) +
                                       " bytes) exceeds the server's budget");
  auto j = std::make_unique<Job>();
  j->req = *r;
  j->bytes = bytes;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return COSENU_EINVAL;
    j->ticket = s->next_ticket++;
    j->res.status = COSENU_PENDING;
    j->res.t_submit = now_s(s);
    j->res.t_admit = -1.0;
    j->res.t_done = -1.0;
    *ticket = j->ticket;
    s->queue.push_back(j.get());
    s->jobs.emplace(j->ticket, std::move(j));
    ++s->submitted;
  }
  s->cv_work.notify_all();
  return COSENU_OK;
}

int cosenu_poll(cosenu_server_t s, uint64_t ticket, cosenu_result* out) {
  if (!s) return sfail(s, COSENU_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) {
    s->error = "unknown ticket";
    return COSENU_EINVAL;
  }
  Job* j = it->second.get();
  if (out) *out = j->res;
  if (j->phase != kDone) return COSENU_PENDING;
  s->jobs.erase(it);
  return COSENU_OK;
}

int cosenu_wait(cosenu_server_t s, uint64_t ticket, double timeout_s, cosenu_result* out) {
  if (!s) return sfail(s, COSENU_EINVAL, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto done = [&] {
    auto it = s->jobs.find(ticket);
    return it == s->jobs.end() || it->second->phase == kDone;
  };
  if (timeout_s < 0)
    s->cv_done.wait(lk, done);
  else
    s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) {
    s->error = "unknown ticket";
    return COSENU_EINVAL;
  }
  Job* j = it->second.get();
  if (out) *out = j->res;
  if (j->phase != kDone) return COSENU_PENDING;
  s->jobs.erase(it);
  return COSENU_OK;
}

int cosenu_cancel(cosenu_server_t s, uint64_t ticket) {
  if (!s) return sfail(s, COSENU_EINVAL, "NULL server");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) {
      s->error = "unknown ticket";
      return COSENU_EINVAL;
    }
    if (it->second->phase == kDone) return COSENU_OK;
    it->second->cancel = true;
  }
  s->cv_work.notify_all();
  return COSENU_OK;
}

int cosenu_server_get_stats(cosenu_server_t s, cosenu_server_stats* out) {
  if (!s || !out) return sfail(s, COSENU_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->admitted = s->admitted;
  out->finished = s->finished;
  out->rounds = s->rounds;
  out->steps = s->steps;
  out->queued = (int32_t)s->queue.size();
  out->running = (int32_t)s->running.size();
  out->bytes_in_use = s->in_use;
  out->peak_bytes = s->peak;
  out->budget = s->budget;
  return COSENU_OK;
}

const char* cosenu_server_last_error(cosenu_server_t s) {
  if (!s) return tl_serror.c_str();
  std::lock_guard<std::mutex> lk(s->mu);
  return s->error.c_str();
}

}  // extern "C"
