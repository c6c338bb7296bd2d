// Request loop over the solver: many systems, each resident with its preconditioner,
// solved concurrently by a pool of worker threads with one CUDA stream each.  Host code
// only; every solve runs through the public entry points (msp_setup, msp_update_values_host,
// msp_solve_host) on the worker's stream.
//
// Scheduling (one mutex, one condition variable):
//   * requests of one key run one at a time, in submit order (a handle is not thread-safe,
//     and the adaptive SETUP of Section 3.2 depends on the previous solve of the key);
//   * a request of a resident system needs only a free slot;
//   * a request that needs a new system is charged its estimated footprint against the
//     device-memory budget; idle resident systems (no request running or queued) are
//     released least recently used first to make room; if it still does not fit, it waits,
//     and so do the later requests that need a new system (they keep their order), while
//     later requests of resident systems, replacements included, may still start;
//   * once a system is set up its measured footprint replaces the estimate;
//   * a system grows once after its setup: its first update of values from the host
//     allocates the staging copy of the values (nnzb * b * b doubles, part of the
//     estimate).  That request is charged the copy before it runs and admitted like a new
//     system (idle systems released to make room, else it waits for a running request to
//     finish; with nothing running it starts anyway), so that the charged total does not
//     run past the budget after the fact.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "common.cuh"

namespace {

using SteadyClock = std::chrono::steady_clock;

double ms_between(SteadyClock::time_point a, SteadyClock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Job {
  int64_t ticket = 0;
  msp_request req{};
  msp_result res{};
  SteadyClock::time_point t_submit;
  bool done = false;
};

struct System {
  msp_handle h = nullptr;  // the CUDA executor's handle
  int64_t bytes = 0;       // charged against the budget (estimate until set up)
  bool busy = false;
  bool ready = false;      // set up (false while its first request runs)
  bool staged = false;     // holds the staging copy of host values (after its first update)
  int queued = 0;          // requests of this key waiting in the queue
  int queued_bare = 0;     // of those, requests without the pattern (they need it resident)
  uint64_t last_used = 0;
};

}  // namespace

struct msp_server_s {
  msp_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv;  // work available / job done / shutdown
  std::deque<Job*> queue;
  std::unordered_map<int64_t, Job*> jobs;  // every ticket not yet waited for
  std::unordered_map<int64_t, System> systems;
  std::vector<std::thread> workers;
  int64_t next_ticket = 1;
  uint64_t clock = 0;
  int64_t charged = 0;  // bytes of resident systems and of systems being set up
  msp_server_stats st{};
  bool stopping = false;
};

namespace {

// Work a worker takes: the job and the systems it must release before running it.
struct Pick {
  Job* job = nullptr;
  bool setup = false;
  std::vector<std::pair<int64_t, msp_handle>> evict;  // key, handle (CUDA executor)
};

// The staging copy of host values a system allocates at its first value update
int64_t staging_bytes(const msp_request& r) { return r.nnzb * (int64_t)r.b * r.b * 8; }

// Idle resident systems (not `key`, no request running), least recently used first, whose
// release raises `avail` to `need`; false if even all of them are not enough.  Only systems
// without queued requests, unless `queued_too`: then also those whose queued requests all
// carry the pattern (they set the system up again).
bool room_by_release(msp_server_s* S, int64_t key, int64_t avail, int64_t need,
                     std::vector<std::pair<uint64_t, int64_t>>& idle, bool queued_too = false) {
  idle.clear();
  if (avail >= need) return true;
  for (auto& kv : S->systems)
    if (kv.first != key && !kv.second.busy && kv.second.ready &&
        (kv.second.queued == 0 || (queued_too && kv.second.queued_bare == 0)))
      idle.push_back({kv.second.last_used, kv.first});
  std::sort(idle.begin(), idle.end());
  int64_t extra = 0;
  size_t k = 0;
  for (; k < idle.size() && avail + extra < need; ++k) extra += S->systems[idle[k].second].bytes;
  idle.resize(k);
  return avail + extra >= need;
}

void release_idle(msp_server_s* S, const std::vector<std::pair<uint64_t, int64_t>>& idle,
                  Pick& out) {
  for (auto& e : idle) {
    System& v = S->systems[e.second];
    out.evict.push_back({e.second, v.h});
    S->charged -= v.bytes;
    ++S->st.evictions;
    if (v.queued == 0) {
      S->systems.erase(e.second);
    } else {  // its queued requests set it up again
      v.h = nullptr;
      v.ready = false;
      v.staged = false;
      v.bytes = 0;
    }
  }
}

// Choose the next runnable job (server lock held).  Every queued key has an entry in
// S->systems (its queued count); `ready` marks the ones that are set up.
bool pick_job(msp_server_s* S, Pick& out) {
  std::unordered_set<int64_t> blocked_keys;
  bool memory_blocked = false;
  for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
    Job* j = *it;
    const int64_t key = j->req.key;
    if (blocked_keys.count(key)) continue;  // an earlier request of this key waits
    System& sy = S->systems[key];
    if (sy.busy) {
      blocked_keys.insert(key);
      continue;
    }
    const bool new_pattern = (j->req.flags & MSP_REQ_NEW_PATTERN) != 0;
    std::vector<std::pair<uint64_t, int64_t>> idle;  // last_used, key
    if (sy.ready && !new_pattern) {
      const int64_t grow = (!sy.staged && j->req.h_values) ? staging_bytes(j->req) : 0;
      if (!room_by_release(S, key, S->cfg.hbm_budget - S->charged, grow, idle)) {
        if (S->st.running > 0) {
          memory_blocked = true;  // later new systems wait behind it
          blocked_keys.insert(key);  // a running request will free or shrink its charge
          continue;
        }
        // nothing runs that could free memory: release idle systems whose queued requests
        // can set them up again; if even that is not enough, start anyway
        room_by_release(S, key, S->cfg.hbm_budget - S->charged, grow, idle, true);
      }
      release_idle(S, idle, out);
      System& me = S->systems[key];
      me.bytes += grow;
      if (j->req.h_values) me.staged = true;
      S->charged += grow;
      S->st.peak_charged_bytes = std::max(S->st.peak_charged_bytes, S->charged);
      out.job = j;
      out.setup = false;
      S->queue.erase(it);
      return true;
    }
    // needs memory for a new system (or for the replacement of its resident one).  Once a
    // request waits for memory, later new systems wait behind it; replacements of resident
    // systems may still go: a system with a queued request cannot be released to make room,
    // so holding its replacement back could leave both waiting for ever.
    if (memory_blocked && !sy.ready) {
      blocked_keys.insert(key);
      continue;
    }
    const int64_t need = msp_estimate_device_bytes(j->req.nb, j->req.b, j->req.nnzb, &S->cfg.cfg);
    const int64_t avail = S->cfg.hbm_budget - S->charged + (sy.ready ? sy.bytes : 0);
    if (!room_by_release(S, key, avail, need, idle)) {
      memory_blocked = true;
      blocked_keys.insert(key);
      continue;
    }
    // admitted.  The worker frees the systems it releases before it allocates anything for
    // the new one, so their bytes are uncharged at once.
    release_idle(S, idle, out);
    System& me = S->systems[key];
    if (me.ready) {
      out.evict.push_back({key, me.h});
      S->charged -= me.bytes;
      me.h = nullptr;
      me.ready = false;
    }
    me.bytes = need;
    S->charged += need;
    S->st.peak_charged_bytes = std::max(S->st.peak_charged_bytes, S->charged);
    out.job = j;
    out.setup = true;
    S->queue.erase(it);
    return true;
  }
  return false;
}

int release_system(msp_server_s* S, int64_t key, msp_handle h, int slot) {
  if (S->cfg.exec) {
    msp_request r{};
    r.key = key;
    int64_t b = 0;
    return S->cfg.exec(S->cfg.exec_user, MSP_EXEC_RELEASE, &r, slot, 0, &b);
  }
  return msp_free(h);
}

// The CUDA executor: set up (from the host pattern) or update values, then solve.
int cuda_run(msp_server_s* S, msp_handle* h, const msp_request& r, bool setup, cudaStream_t s,
             msp_solve_info* info, int64_t* bytes) {
  if (setup) {
    if (!r.h_row_ptr || !r.h_col_idx || !r.h_values) return MSP_ERR_ARG;
    msp::DevBuf<int> rp, ci;
    msp::DevBuf<double> v;
    const size_t nv = (size_t)r.nnzb * r.b * r.b;
    MSP_TRY(rp.alloc((size_t)r.nb + 1));
    MSP_TRY(ci.alloc((size_t)r.nnzb));
    MSP_TRY(v.alloc(nv));
    MSP_CUDA_TRY(cudaMemcpyAsync(rp.p, r.h_row_ptr, sizeof(int) * ((size_t)r.nb + 1),
                                 cudaMemcpyHostToDevice, s));
    MSP_CUDA_TRY(cudaMemcpyAsync(ci.p, r.h_col_idx, sizeof(int) * (size_t)r.nnzb,
                                 cudaMemcpyHostToDevice, s));
    MSP_CUDA_TRY(cudaMemcpyAsync(v.p, r.h_values, sizeof(double) * nv, cudaMemcpyHostToDevice, s));
    const int st = msp_setup(h, &S->cfg.cfg, r.nb, r.b, rp.p, ci.p, v.p, r.nnzb, s);
    MSP_CUDA_TRY(cudaStreamSynchronize(s));
    if (st != MSP_OK) return st;
  } else if (r.h_values) {
    MSP_TRY(msp_update_values_host(*h, r.h_values, s));
  }
  const int st = msp_solve_host(*h, r.h_rhs, r.h_x, r.rel_tol, info, s);
  msp_device_bytes(*h, bytes);
  return st;
}

void worker_main(msp_server_s* S, int slot) {
  cudaStream_t s = nullptr;
  if (!S->cfg.exec) {
    cudaSetDevice(S->cfg.device);
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  }
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    Pick p;
    while (!pick_job(S, p)) {
      if (S->stopping && S->queue.empty()) {
        lk.unlock();
        if (s) cudaStreamDestroy(s);
        return;
      }
      S->cv.wait(lk);
    }
    Job* j = p.job;
    const int64_t key = j->req.key;
    System& sys0 = S->systems[key];
    sys0.busy = true;
    --sys0.queued;
    if (!j->req.h_row_ptr || !j->req.h_col_idx) --sys0.queued_bare;
    msp_handle h = sys0.h;
    ++S->st.running;
    --S->st.queued;
    lk.unlock();

    for (size_t k = 0; k < p.evict.size(); ++k) release_system(S, p.evict[k].first, p.evict[k].second, slot);
    const auto t_start = SteadyClock::now();
    msp_result res{};
    res.ticket = j->ticket;
    res.key = key;
    res.slot = slot;
    res.setup = p.setup ? 1 : 0;
    int64_t bytes = 0;
    int st;
    if (S->cfg.exec) {
      st = S->cfg.exec(S->cfg.exec_user, MSP_EXEC_RUN, &j->req, slot, res.setup, &bytes);
      res.info.status = st;
    } else {
      if (p.setup) h = nullptr;
      st = cuda_run(S, &h, j->req, p.setup, s, &res.info, &bytes);
    }
    res.status = st;
    // with the CUDA executor a failed setup leaves no handle; a custom executor's system
    // counts as set up
    const bool have_system = S->cfg.exec != nullptr || h != nullptr;
    const bool release = (j->req.flags & MSP_REQ_RELEASE) != 0 || !have_system;
    if (release && have_system) release_system(S, key, h, slot);
    const auto t_end = SteadyClock::now();
    res.queue_ms = ms_between(j->t_submit, t_start);
    res.run_ms = ms_between(t_start, t_end);
    res.latency_ms = ms_between(j->t_submit, t_end);
    res.device_bytes = bytes;

    lk.lock();
    System& sys = S->systems[key];
    S->charged -= sys.bytes;
    sys.busy = false;
    if (release) {
      sys.h = nullptr;
      sys.ready = false;
      sys.bytes = 0;
      if (sys.queued == 0) S->systems.erase(key);  // later requests set it up again
    } else {
      sys.h = h;
      sys.bytes = bytes;
      sys.ready = true;
      sys.last_used = ++S->clock;
      S->charged += bytes;
    }
    // systems that only hold a queued count are not resident
    int64_t resident = 0, rb = 0;
    for (auto& kv : S->systems)
      if (kv.second.ready) {
        ++resident;
        rb += kv.second.bytes;
      }
    S->st.resident_systems = resident;
    S->st.resident_bytes = rb;
    S->st.peak_charged_bytes = std::max(S->st.peak_charged_bytes, S->charged);
    --S->st.running;
    ++S->st.completed;
    j->res = res;
    j->done = true;
    S->cv.notify_all();
  }
}

}  // namespace

extern "C" {

int64_t msp_estimate_device_bytes(int32_t nb, int32_t b, int64_t nnzb, const msp_config* cfg) {
  if (nb <= 0 || b <= 0 || nnzb <= 0) return 0;
  const int64_t bb = (int64_t)b * b, bn = (int64_t)(b - 1) * (b - 1);
  const int64_t n = (int64_t)nb * b;
  const int m = cfg ? cfg->restart : 30;
  const int64_t nc = std::min<int64_t>(cfg ? cfg->coarse_max : 10000, nb);  // coarsest level
  // level 0: values, BILU factors, stage-N blocks, staging for new values, column 0,
  // pattern and permutations; the pressure matrix and the AMG levels with their ELL
  // copies (at most about 3 nonzeros of pressure per block, both forms); Krylov bases V and
  // Z and work vectors; the coarsest dense inverse and its panel copy
  int64_t bytes = nnzb * (3 * bb * 8 + bn * 8 + b * 8 + 16) + (int64_t)nb * (bb * 8 + bn * 8 + 64);
  bytes += nnzb * 3 * (8 + 4) * 2;
  bytes += n * 8 * (2 * (int64_t)m + 16);
  bytes += nc * nc * 8 * 2;
  if (cfg && cfg->precision == MSP_PRECISION_FP32) bytes += nnzb * (2 * bb + bn) * 4;  // FP32 copies
  return bytes + (4ll << 20);
}

int msp_server_create(msp_server* out, const msp_server_config* cfg) {
  if (!out) return MSP_ERR_ARG;
  *out = nullptr;
  if (!cfg || cfg->slots < 1 || cfg->slots > 64 || cfg->hbm_budget <= 0) return MSP_ERR_ARG;
  msp_server_s* S = nullptr;
  try {
    S = new msp_server_s();
    S->cfg = *cfg;
    for (int k = 0; k < cfg->slots; ++k) S->workers.emplace_back(worker_main, S, k);
  } catch (...) {
    if (S) {
      {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
      }
      S->cv.notify_all();
      for (auto& t : S->workers) t.join();
      delete S;
    }
    return MSP_ERR_NOMEM;
  }
  *out = S;
  return MSP_OK;
}

int msp_server_submit(msp_server S, const msp_request* req, int64_t* ticket) {
  if (!S || !req || !ticket || req->nb <= 0 || req->b < 1 || req->b > 8 || req->nnzb < req->nb ||
      !req->h_rhs || !req->h_x || !(req->rel_tol > 0.0))
    return MSP_ERR_ARG;
  Job* j = new Job();
  j->req = *req;
  j->t_submit = SteadyClock::now();
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stopping) {
    delete j;
    return MSP_ERR_ARG;
  }
  j->ticket = S->next_ticket++;
  *ticket = j->ticket;
  S->jobs[j->ticket] = j;
  ++S->st.submitted;
  const int64_t need = msp_estimate_device_bytes(req->nb, req->b, req->nnzb, &S->cfg.cfg);
  if (need > S->cfg.hbm_budget) {
    j->res.ticket = j->ticket;
    j->res.key = req->key;
    j->res.status = MSP_ERR_NOMEM;
    j->res.slot = -1;
    j->done = true;
    ++S->st.rejected;
    ++S->st.completed;
    S->cv.notify_all();
    return MSP_OK;
  }
  System& sy = S->systems[req->key];
  sy.queued++;
  if (!req->h_row_ptr || !req->h_col_idx) sy.queued_bare++;
  S->queue.push_back(j);
  ++S->st.queued;
  S->cv.notify_all();
  return MSP_OK;
}

int msp_server_wait(msp_server S, int64_t ticket, double timeout_s, msp_result* res) {
  if (!S || !res) return MSP_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return MSP_ERR_ARG;
  Job* j = it->second;
  if (timeout_s < 0) {
    S->cv.wait(lk, [&] { return j->done; });
  } else if (!S->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return j->done; })) {
    return MSP_ERR_TIMEOUT;
  }
  *res = j->res;
  S->jobs.erase(ticket);
  delete j;
  return MSP_OK;
}

int msp_server_get_stats(msp_server S, msp_server_stats* st) {
  if (!S || !st) return MSP_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  *st = S->st;
  return MSP_OK;
}

int msp_server_free(msp_server S) {
  if (!S) return MSP_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
  }
  S->cv.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& kv : S->systems)
    if (kv.second.ready) release_system(S, kv.first, kv.second.h, 0);
  for (auto& kv : S->jobs) delete kv.second;
  delete S;
  return MSP_OK;
}

}  // extern "C"
