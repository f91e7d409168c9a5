// Serving loop: continuous batching of observe + suggest requests from many
// tuning sessions, admission by device memory.  See bo_server_* in
// include/bo_suggest.h for the contract.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <algorithm>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>

#include "bo_space_impl.h"

using namespace bo;
using namespace bo::host;

namespace {

struct Request {
  int64_t idx;
  double value;
  int32_t suggest;
  uint64_t tag;
  double t_submit;
};

// A registered session: its descriptor (with owned copies of the arrays), its
// space once admitted, and its pending requests.
struct Session {
  int64_t id = 0;
  bo_space_desc desc{};
  std::vector<int32_t> n_values;
  std::vector<std::vector<double>> values;
  std::vector<const double*> value_ptrs;
  std::vector<uint8_t> mask;
  size_t est_bytes = 0;
  bo_space* space = nullptr;
  bool closing = false;
  std::deque<Request> pending;
};

}  // namespace

struct bo_server {
  bo_server_config cfg{};
  int device = 0;
  int num_sms = 148;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::thread worker;
  int64_t next_id = 1;
  std::map<int64_t, Session> sessions;
  std::deque<int64_t> waiting;            // registered, not yet admitted, in order
  std::vector<int64_t> live;              // admitted, in the order of the current batch
  bo_batch* batch = nullptr;
  bool batch_stale = true;
  std::deque<bo_completion> done;
  bo_server_stats stats{};
  size_t bytes_in_use = 0;
};

namespace {

double now_s(const bo_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

// Admit waiting sessions in order while memory and slots allow (server lock held).
void admit(bo_server* S) {
  while (!S->waiting.empty()) {
    Session& ss = S->sessions[S->waiting.front()];
    if ((int)S->live.size() >= S->cfg.max_sessions ||
        S->bytes_in_use + ss.est_bytes > S->cfg.budget_bytes)
      break;
    bo_space_desc d = ss.desc;
    d.n_values = ss.n_values.data();
    d.values = ss.value_ptrs.data();
    d.invalid_mask = ss.mask.empty() ? nullptr : ss.mask.data();
    d.alloc = S->cfg.alloc;
    d.free = S->cfg.free;
    d.alloc_ctx = S->cfg.alloc_ctx;
    d.stream = S->cfg.stream;
    bo_space* sp = nullptr;
    // the descriptor passed its checks at open: what can fail here is the
    // device (memory, a launch); the requests carry that code
    if (const int rc = bo_space_create(&d, &sp); rc != BO_OK) {
      ++S->stats.rejected;
      for (auto& r : ss.pending) {
        bo_completion c{};
        c.tag = r.tag;
        c.session = ss.id;
        c.status = rc;
        c.idx = -1;
        c.t_submit = r.t_submit;
        c.t_done = now_s(S);
        S->done.push_back(c);
      }
      ss.pending.clear();
      S->waiting.pop_front();
      continue;
    }
    ss.space = sp;
    S->bytes_in_use += space_bytes(sp);
    S->live.push_back(ss.id);
    S->batch_stale = true;
    ++S->stats.admitted;
    S->waiting.pop_front();
  }
}

void retire_closed(bo_server* S) {
  for (size_t k = 0; k < S->live.size();) {
    Session& ss = S->sessions[S->live[k]];
    if (ss.closing && ss.pending.empty()) {
      if (S->batch) {                      // the batch refers to the space (and may own memory through it)
        bo_batch_destroy(S->batch);
        S->batch = nullptr;
      }
      S->bytes_in_use -= space_bytes(ss.space);
      bo_space_destroy(ss.space);
      ss.space = nullptr;
      ++S->stats.closed;
      S->sessions.erase(S->live[k]);
      S->live.erase(S->live.begin() + k);
      S->batch_stale = true;
    } else {
      ++k;
    }
  }
}

void serve(bo_server* S) {
  cudaSetDevice(S->device);
  std::vector<bo_space*> spaces;
  while (true) {
    std::vector<int> take;                 // positions in live with a request this iteration
    std::vector<Request> reqs;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // wake for requests, for a session to retire, or for a waiting session
      // that now fits (a waiting session that does not fit wakes nobody)
      S->cv_work.wait_for(lk, std::chrono::milliseconds(2), [&] {
        if (S->stop) return true;
        for (int64_t id : S->live) {
          const Session& ss = S->sessions[id];
          if (!ss.pending.empty() || ss.closing) return true;
        }
        if (S->waiting.empty()) return false;
        const Session& w = S->sessions[S->waiting.front()];
        return (int)S->live.size() < S->cfg.max_sessions && S->bytes_in_use + w.est_bytes <= S->cfg.budget_bytes;
      });
      if (S->stop) break;
      retire_closed(S);
      admit(S);
      bool work = false;
      for (int64_t id : S->live) work = work || !S->sessions[id].pending.empty();
      // the batch is rebuilt only when requests need it, so that a burst of
      // admissions costs one rebuild
      int batch_rc = BO_OK;
      if (work && S->batch_stale) {
        if (S->batch) bo_batch_destroy(S->batch);
        S->batch = nullptr;
        spaces.clear();
        for (int64_t id : S->live) spaces.push_back(S->sessions[id].space);
        if (!spaces.empty()) batch_rc = bo_batch_create(spaces.data(), (int32_t)spaces.size(), &S->batch);
        S->batch_stale = S->batch == nullptr;
      }
      for (size_t k = 0; k < S->live.size(); ++k) {
        Session& ss = S->sessions[S->live[k]];
        if (!ss.pending.empty()) {
          take.push_back((int)k);
          reqs.push_back(ss.pending.front());
          ss.pending.pop_front();
        }
      }
      if (!take.empty() && !S->batch) {    // no batch to run them on: each request fails
        for (size_t q = 0; q < take.size(); ++q) {
          bo_completion c{};
          c.tag = reqs[q].tag;
          c.session = S->live[take[q]];
          c.status = batch_rc != BO_OK ? batch_rc : BO_ERR_CUDA;
          c.idx = -1;
          c.t_submit = reqs[q].t_submit;
          c.t_done = now_s(S);
          ++S->stats.completed;
          S->done.push_back(c);
        }
        take.clear();
      }
      S->cv_done.notify_all();             // admissions / rejections may have produced completions
    }
    if (take.empty()) continue;
    const double t_start = now_s(S);
    const size_t n = spaces.size();
    std::vector<int64_t> idx(n, -1), out_idx(n, -1);
    std::vector<double> val(n, 0.0);
    std::vector<uint8_t> want(n, 0);
    std::vector<int32_t> st_obs(n, BO_OK), st_sug(n, BO_OK);
    std::vector<bo_suggest_info> info(n);
    for (size_t q = 0; q < take.size(); ++q) {
      idx[take[q]] = reqs[q].idx;
      val[take[q]] = reqs[q].value;
      want[take[q]] = reqs[q].suggest ? 1 : 0;
    }
    bo_batch_observe(S->batch, idx.data(), val.data(), st_obs.data());
    for (size_t q = 0; q < take.size(); ++q)      // a request whose observation failed gets no suggestion
      if (st_obs[take[q]] != BO_OK) want[take[q]] = 0;
    if (std::find(want.begin(), want.end(), 1) != want.end())
      bo_batch_suggest_some(S->batch, want.data(), out_idx.data(), st_sug.data(), info.data());
    const double t_done = now_s(S);
    std::lock_guard<std::mutex> lk(S->mu);
    ++S->stats.iterations;
    for (size_t q = 0; q < take.size(); ++q) {
      const int k = take[q];
      bo_completion c{};
      c.tag = reqs[q].tag;
      c.session = S->live[k];
      c.status = st_obs[k] != BO_OK ? st_obs[k] : st_sug[k];
      c.observed = reqs[q].idx >= 0 && st_obs[k] == BO_OK;
      c.idx = want[k] ? out_idx[k] : -1;
      if (want[k]) c.info = info[k];
      c.t_submit = reqs[q].t_submit;
      c.t_start = t_start;
      c.t_done = t_done;
      if (want[k]) S->stats.candidates_scored += info[k].n_scored;
      ++S->stats.completed;
      S->done.push_back(c);
    }
    S->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

int bo_server_create(const bo_server_config* cfg, bo_server** out) {
  if (!cfg || !out || cfg->max_sessions < 1) return fail(BO_ERR_ARG, "bad server configuration");
  bo_server* S = new (std::nothrow) bo_server();
  if (!S) return fail(BO_ERR_NOMEM, "host allocation failed");
  S->cfg = *cfg;
  cudaGetDevice(&S->device);
  cudaDeviceGetAttribute(&S->num_sms, cudaDevAttrMultiProcessorCount, S->device);
  S->t0 = std::chrono::steady_clock::now();
  S->worker = std::thread(serve, S);
  *out = S;
  return BO_OK;
}

int bo_server_open(bo_server* S, const bo_space_desc* desc, int64_t* session_out) {
  if (!S || !desc || !session_out) return fail(BO_ERR_ARG, "null argument");
  // the whole descriptor is checked here, as bo_space_create checks it, so that a
  // bad one is refused at once instead of failing its requests at admission
  int64_t total = 0;
  if (const int rc = check_space_desc(*desc, &total); rc != BO_OK) return rc;
  Session ss;
  ss.desc = *desc;
  for (int p = 0; p < desc->d; ++p) {
    ss.n_values.push_back(desc->n_values[p]);
    ss.values.emplace_back(desc->values[p], desc->values[p] + desc->n_values[p]);
  }
  for (auto& v : ss.values) ss.value_ptrs.push_back(v.data());
  int64_t n_valid = total;
  if (desc->invalid_mask) {
    ss.mask.assign(desc->invalid_mask, desc->invalid_mask + total);
    n_valid = 0;
    for (uint8_t m : ss.mask) n_valid += !m;
  }
  if (n_valid == 0) return fail(BO_ERR_ARG, "no valid configuration");
  if (desc->precision != BO_PREC_FP64 && n_valid >= (int64_t)0xFFFFFFFF)
    return fail(BO_ERR_ARG, "reduced precision holds fewer than 2^32 - 1 valid configurations");
  ss.est_bytes = space_device_bytes(desc->d, n_valid, desc->n_max, desc->precision, S->num_sms);
  std::lock_guard<std::mutex> lk(S->mu);
  if (ss.est_bytes > S->cfg.budget_bytes) {
    ++S->stats.rejected;
    return fail(BO_ERR_NOMEM, "session needs %zu bytes, above the budget of %zu", ss.est_bytes,
                S->cfg.budget_bytes);
  }
  ss.id = S->next_id++;
  *session_out = ss.id;
  S->waiting.push_back(ss.id);
  ++S->stats.queued;
  S->sessions.emplace(ss.id, std::move(ss));
  S->cv_work.notify_one();
  return BO_OK;
}

int bo_server_submit(bo_server* S, int64_t session, int64_t observe_idx, double observe_value, int32_t suggest,
                     uint64_t tag) {
  if (!S) return fail(BO_ERR_ARG, "null server");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->sessions.find(session);
  if (it == S->sessions.end() || it->second.closing) return fail(BO_ERR_ARG, "unknown or closed session");
  it->second.pending.push_back(Request{observe_idx, observe_value, suggest, tag, now_s(S)});
  ++S->stats.requests;
  S->cv_work.notify_one();
  return BO_OK;
}

int bo_server_poll(bo_server* S, bo_completion* out, int32_t max, int32_t* n_out, int32_t wait_ms) {
  if (!S || !n_out || (max > 0 && !out)) return fail(BO_ERR_ARG, "bad argument");
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->done.empty() && wait_ms > 0)
    S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !S->done.empty(); });
  int32_t n = 0;
  while (n < max && !S->done.empty()) {
    out[n++] = S->done.front();
    S->done.pop_front();
  }
  *n_out = n;
  return BO_OK;
}

int bo_server_close(bo_server* S, int64_t session) {
  if (!S) return fail(BO_ERR_ARG, "null server");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->sessions.find(session);
  if (it == S->sessions.end()) return fail(BO_ERR_ARG, "unknown session");
  if (!it->second.space) {                 // never admitted: drop it from the queue
    for (auto w = S->waiting.begin(); w != S->waiting.end(); ++w)
      if (*w == session) { S->waiting.erase(w); break; }
    S->sessions.erase(it);
    ++S->stats.closed;
  } else {
    it->second.closing = true;             // the worker releases it once its requests are served
  }
  S->cv_work.notify_one();
  return BO_OK;
}

int bo_server_stats_get(bo_server* S, bo_server_stats* out) {
  if (!S || !out) return fail(BO_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->stats;
  out->bytes_in_use = (int64_t)S->bytes_in_use;
  return BO_OK;
}

double bo_server_now(const bo_server* S) { return S ? now_s(S) : 0.0; }

int bo_server_destroy(bo_server* S) {
  if (!S) return fail(BO_ERR_ARG, "null server");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  cudaSetDevice(S->device);
  if (S->batch) bo_batch_destroy(S->batch);
  for (auto& kv : S->sessions)
    if (kv.second.space) bo_space_destroy(kv.second.space);
  delete S;
  return BO_OK;
}

}  // extern "C"
