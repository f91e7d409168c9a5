// Host-side state of a space, shared by the C ABI (bo_session.cpp) and the
// batched entry points (bo_batch.cpp).
#pragma once

#include <algorithm>
#include <deque>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "bo_internal.h"

namespace bo {
namespace host {

struct Pick {
  int64_t idx;
  std::vector<int> afs;
  double mu, sigma, score;
};

// Selection of acquisition functions (paper Sec. III-G, Table I).
//   single:   one AF, one pick per pass.
//   multi:    every active AF picks from one shared pass; each pair of AFs
//             with the same pick gains a duplicate each and becomes partners
//             (the pick is evaluated once, credited to both); at the start of
//             a round an AF whose count exceeds the threshold is pitted with
//             its partners and only the lowest dos among them stays.
//   advanced: an AF picks its best candidate not taken by an earlier AF in
//             the round; each round after the first, dos above mean*(1+rif)
//             counts 'over', below mean*(1-rif) counts 'under' (cumulative);
//             an 'under' count at the threshold promotes that AF to be the
//             only one, else an 'over' count at it skips the AF and resets
//             the others' counts.
// dos <- gamma * dos + o for every observation credited to an AF.
struct Selector {
  int mode = BO_AF_EI;
  std::vector<int> active;
  double dos[3] = {0, 0, 0};
  int dup[3] = {0, 0, 0};
  unsigned partners[3] = {0, 0, 0};
  int over[3] = {0, 0, 0}, under[3] = {0, 0, 0};
  int rounds = 0;
  int threshold = 5;
  double gamma = 0.65, rif = 0.1;

  void init(int m, int thr, double discount, double r) {
    mode = m;
    threshold = thr;
    rif = r;
    if (m == BO_AF_MULTI || m == BO_AF_ADV_MULTI) {
      active = {kEI, kPI, kLCB};
      gamma = discount > 0 ? discount : (m == BO_AF_MULTI ? 0.65 : 0.75);
    } else {
      active = {m};
    }
  }

  bool is_active(int a) const {
    return std::find(active.begin(), active.end(), a) != active.end();
  }

  void begin_round() {
    if (mode == BO_AF_MULTI && rounds > 0) {
      unsigned group = 0;
      for (int a : active)
        if (dup[a] > threshold) group |= (1u << a) | partners[a];
      if (group) {
        int keep = -1;
        for (int a = 0; a < 3; ++a)   // AF ids are in Table I order
          if ((group >> a & 1u) && is_active(a) && (keep < 0 || dos[a] < dos[keep])) keep = a;
        std::vector<int> next;
        for (int a : active)
          if (!(group >> a & 1u) || a == keep) next.push_back(a);
        active = next;
        for (int a = 0; a < 3; ++a) { dup[a] = 0; partners[a] = 0; }
      }
    } else if (mode == BO_AF_ADV_MULTI && rounds > 0 && active.size() >= 2) {
      double m = 0;
      for (int a : active) m += dos[a];
      m /= (double)active.size();
      for (int a : active) {
        if (dos[a] > m * (1.0 + rif)) ++over[a];
        else if (dos[a] < m * (1.0 - rif)) ++under[a];
      }
      int promote = -1, skip = -1;
      for (int a : active)
        if (promote < 0 && under[a] >= threshold) promote = a;
      for (int a : active)
        if (skip < 0 && over[a] >= threshold) skip = a;
      if (promote >= 0) {
        active = {promote};
      } else if (skip >= 0) {
        active.erase(std::find(active.begin(), active.end(), skip));
        for (int a : active) over[a] = under[a] = 0;
      }
    }
    ++rounds;
  }

  // picks of one round from the pass result, whose AF rows follow `active`
  std::vector<Pick> assign(const bo_pass_result& r) {
    std::vector<Pick> picks;
    for (size_t q = 0; q < active.size(); ++q) {
      const int a = active[q];
      if (mode == BO_AF_ADV_MULTI) {
        for (int k = 0; k < 3; ++k) {
          const int64_t i = r.top_idx[q][k];
          if (i < 0) break;
          bool taken = false;
          for (auto& p : picks) taken |= (p.idx == i);
          if (!taken) {
            picks.push_back({i, {a}, r.top_mu[q][k], r.top_sigma[q][k], r.top_score[q][k]});
            break;
          }
        }
        continue;
      }
      const int64_t i = r.top_idx[q][0];
      if (i < 0) continue;
      Pick* same = nullptr;
      for (auto& p : picks)
        if (p.idx == i) same = &p;
      if (same && mode == BO_AF_MULTI) {
        for (int b : same->afs) {
          ++dup[a];
          ++dup[b];
          partners[a] |= 1u << b;
          partners[b] |= 1u << a;
        }
        same->afs.push_back(a);
      } else if (!same) {
        picks.push_back({i, {a}, r.top_mu[q][0], r.top_sigma[q][0], r.top_score[q][0]});
      }
    }
    return picks;
  }

  void credit(const std::vector<int>& afs, double value) {
    if (mode != BO_AF_MULTI && mode != BO_AF_ADV_MULTI) return;
    for (int a : afs) dos[a] = gamma * dos[a] + value;
  }
};

}  // namespace host
}  // namespace bo

struct bo_space {
  bo_space_desc desc;
  int device = 0;
  cudaStream_t stream = nullptr;
  int d = 0;
  std::vector<int> sizes;
  std::vector<std::vector<double>> values;
  int64_t N = 0;
  std::vector<uint8_t> codes;        // [d][N] host copy
  std::vector<uint8_t> visited;      // [N]
  int64_t n_visited = 0;
  std::vector<int64_t> obs_idx;
  std::vector<double> obs_y;
  std::vector<double> fit_y;         // finite observations in fit order
  int n_fit = 0;
  int n_cap = 0;                     // desc.n_max
  bool cv_set = false;
  double mu_s = 0;
  uint64_t rng = 0;
  std::deque<int64_t> init_queue;    // initial design not yet suggested (LHS / maximin)
  bool init_built = false;
  bo::host::Selector sel;
  std::deque<bo::host::Pick> queue;
  std::map<int64_t, std::vector<int>> outstanding;
  bo::DevView v{};
  std::vector<std::pair<void*, size_t>> blocks;
  bo_pass_result* host_result = nullptr;   // pinned
  bo_pass_result last{};                   // result of the last prediction pass
  int64_t launches = 0;
  int replay_steps = 0;
  int poisoned = BO_OK;
  bool coop_update = true;           // one cooperative launch per observation update
  bool fused_acquire = false;        // tensor-core pass with the acquisition as its tail (one launch)
};

namespace bo {
namespace host {

int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
#define BO_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return bo::host::cuda_fail(e_, #call); \
  } while (0)

uint64_t splitmix64_next(uint64_t& state);
// The new observation idx as the update kernels read it (value y, the fit's
// mean and standard deviation after it).
void make_obs_new(const bo_space* s, int64_t idx, double y, double y_mean, double y_std, bo::ObsNew* o);
// The initial sample of bo_initial_design: `count` distinct valid-list indices
// into out, drawn from rng (advanced); valid_of maps a flat (row-major)
// configuration index to its valid-list index, or -1 when restricted.
int initial_design(const std::vector<std::vector<double>>& values, int64_t n_valid,
                   const std::function<int64_t(int64_t)>& valid_of, int count, int mode, int designs,
                   uint64_t& rng, int64_t* out);

int dalloc(bo_space* s, size_t bytes, void** out);
// Device bytes bo_space_create allocates for these sizes, and those a space holds.
size_t space_device_bytes(int d, int64_t N, int n_max, int precision, int num_sms);
// The device-free checks of a space descriptor (fields, value lists, size of
// the product, returned in *total_out): BO_OK or BO_ERR_ARG with the message set.
int check_space_desc(const bo_space_desc& D, int64_t* total_out);
size_t space_bytes(const bo_space* s);
void y_stats(const bo_space* s, double* mean, double* std_, double* ymin);
// Scalars of a prediction pass with the given active AFs (takes the
// contextual-variance baseline on the first pass).
int prepare_pass(bo_space* s, const std::vector<int>& afs, int slot, PassArgs* a);
// Host part of an observation: checks, bookkeeping, AF credit.  *fit is set
// when the value is finite (the device update then fits it as row *n_before).
int observe_host(bo_space* s, int64_t idx, double value, bool* fit, int* n_before, double* y_mean,
                 double* y_std);
// bo_suggest without its device pass: a random or queued pick (need_pass
// false), or the start of a new round (need_pass true).
int suggest_begin(bo_space* s, int64_t* idx_out, bo_suggest_info* info, bool* need_pass);
// Finish a round from the pass result r: picks, queue, the first pick.
int suggest_finish(bo_space* s, const bo_pass_result& r, int64_t* idx_out, bo_suggest_info* info);

// Time `launch` (a function enqueueing one prediction launch on `stream`,
// returning < 0 on failure) under each candidate TcShape; store and report the
// fastest under `key`.
template <typename Launch>
int autotune_shapes(cudaStream_t stream, int reps, int precision, double nu, int dmax, int n_pad, bool batched,
                    Launch launch, bo_tune_result* out);

}  // namespace host
}  // namespace bo

namespace bo {
namespace host {

template <typename Launch>
int autotune_shapes(cudaStream_t stream, int reps, int precision, double nu, int dmax, int n_pad, bool batched,
                    Launch launch, bo_tune_result* out) {
  reps = std::max(1, std::min(reps, 50));
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(BO_ERR_CUDA, "event creation failed");
  auto time_shape = [&](const TcShape& shape, double* ms) -> bool {
    tc_force_shape(&shape);
    bool ok = launch() >= 0;                      // warm (and function attributes)
    std::vector<float> t;
    for (int r = 0; ok && r < reps; ++r) {
      cudaEventRecord(e0, stream);
      ok = launch() >= 0;
      cudaEventRecord(e1, stream);
      float x = 0.0f;
      ok = ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&x, e0, e1) == cudaSuccess;
      t.push_back(x);
    }
    tc_force_shape(nullptr);
    if (!ok || t.empty()) return false;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return true;
  };
  TcShape best{};
  double best_ms = 0.0, default_ms = 0.0;
  int tried = 0;
  if (!time_shape(TcShape{}, &default_ms)) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return fail(BO_ERR_CUDA, "the default prediction launch failed");
  }
  best_ms = default_ms;
  ++tried;
  for (int sa : {2, 3, 4, 6, 8})
    for (int bs : {2, 3, 4, 6})
      for (int res : {0, -1}) {
        TcShape sh;
        sh.stages_a = sa;
        sh.b_slots = bs;
        sh.b_resident = res;
        double ms = 0.0;
        if (!time_shape(sh, &ms)) continue;   // does not fit shared memory
        ++tried;
        if (ms < best_ms) { best_ms = ms; best = sh; }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  tc_store_shape(precision, nu, dmax, n_pad, batched, best);
  if (out) {
    out->stages_a = best.stages_a;
    out->b_slots = best.b_slots;
    out->b_resident = best.b_resident;
    out->tried = tried;
    out->best_ms = best_ms;
    out->default_ms = default_ms;
  }
  return BO_OK;
}

}  // namespace host
}  // namespace bo
