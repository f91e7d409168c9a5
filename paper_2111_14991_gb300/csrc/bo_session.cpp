// Host side of the suggest library: the C ABI, the search-space build, the
// observation bookkeeping and the selection of acquisition functions.
//
// Device work per call:
//   bo_observe  -> observation update of L^-1, beta and alpha (FP64), or a visited bit
//   bo_suggest  -> prediction pass (K* tiles + contraction + row reduction),
//                  then acquisition + masked top-k, then one small copy back
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "bo_space_impl.h"

using namespace bo;
using namespace bo::host;

namespace {

thread_local std::string g_err;

}  // namespace

namespace bo {
namespace host {

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(BO_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// splitmix64 (Steele, Lea and Flood 2014), from its published definition.
uint64_t splitmix64_next(uint64_t& state) {
  state += 0x9E3779B97F4A7C15ull;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void make_obs_new(const bo_space* s, int64_t idx, double y, double y_mean, double y_std, ObsNew* o) {
  *o = ObsNew{};
  o->idx = (long long)idx;
  o->y_raw = y;
  o->y_mean = y_mean;
  o->inv_std = 1.0 / y_std;
  int off = 0;   // the squared-difference tables lie parameter after parameter, m_p^2 entries each
  for (int p = 0; p < s->d; ++p) {
    const int a = s->codes[(size_t)p * s->N + idx];
    o->a[p] = a;
    o->x[p] = s->values[p][a];
    o->off[p] = off;
    o->m[p] = s->sizes[p];
    off += s->sizes[p] * s->sizes[p];
  }
}

}  // namespace host
}  // namespace bo

namespace {
using bo::host::Pick;
}  // namespace

int bo::report_error(int code, const char* msg) {
  g_err = msg;
  return code;
}


namespace bo {
namespace host {

size_t space_device_bytes(int d, int64_t N, int n_max, int precision, int num_sms) {
  // the allocations of bo_space_create, each rounded up to 256 bytes
  auto r = [](size_t b) { return (std::max<size_t>(b, 256) + 255) / 256 * 256; };
  const int64_t N_pad = (N + kTileRows - 1) / kTileRows * kTileRows;
  const size_t n = (size_t)((n_max + 31) / 32 * 32);
  const size_t fsz = precision == BO_PREC_FP64 ? 8 : 4;
  size_t t = r(d * N_pad) + r(d * 256 * 8) + r(d * 256 * 4) + r((N_pad / 32 + 1) * 4);
  t += r(n * d * 8) + r(n * d) + r(kSqdMaxBytes) + r((2 * BO_MAX_PARAMS + 1) * 4);
  t += r(n * 8) + r(n * n * 8) + r(n * 8) + 2 * r(n * 8);
  if (precision != BO_PREC_FP64) {
    t += 2 * r(n * 8);
    t += r((size_t)(tc_dim_bucket(d) + 2) * n * 4);
    t += split_parts(precision) * r(lsplit_bytes((int)n, precision));
  }
  t += 2 * r(N_pad * fsz) + r((N_pad / 32 + num_sms) * 8) + 2 * r(n * 8) + r(8 * n * 8) + r(sizeof(DevStats));
  t += r((size_t)4 * num_sms * 9 * sizeof(TopEntry)) + r(1024 * sizeof(bo_pass_result));
  return t;
}

size_t space_bytes(const bo_space* s) {
  size_t t = 0;
  for (auto& b : s->blocks) t += b.second;
  return t;
}

int dalloc(bo_space* s, size_t bytes, void** out) {
  bytes = std::max<size_t>(bytes, 256);
  void* p = nullptr;
  if (s->desc.alloc) {
    p = s->desc.alloc(bytes, (void*)s->stream, s->desc.alloc_ctx);
    if (!p) return fail(BO_ERR_NOMEM, "device allocation of %zu bytes failed", bytes);
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
  }
  s->blocks.push_back({p, bytes});
  cudaError_t e = cudaMemsetAsync(p, 0, bytes, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  *out = p;
  return BO_OK;
}

template <typename T>
int dalloc_n(bo_space* s, size_t count, T** out) {
  return dalloc(s, count * sizeof(T), reinterpret_cast<void**>(out));
}

void release(bo_space* s) {
  if (s->stream || true) cudaStreamSynchronize(s->stream);
  for (auto& b : s->blocks) {
    if (s->desc.alloc) {
      if (s->desc.free) s->desc.free(b.first, b.second, (void*)s->stream, s->desc.alloc_ctx);
    } else {
      cudaFreeAsync(b.first, s->stream);
    }
  }
  s->blocks.clear();
  if (s->host_result) cudaFreeHost(s->host_result);
  s->host_result = nullptr;
  cudaStreamSynchronize(s->stream);
}

void y_stats(const bo_space* s, double* mean, double* std_, double* ymin) {
  double m = 0, mn = INFINITY;
  for (double y : s->fit_y) { m += y; mn = std::min(mn, y); }
  m /= (double)s->fit_y.size();
  double v = 0;
  for (double y : s->fit_y) v += (y - m) * (y - m);
  v = std::sqrt(v / (double)s->fit_y.size());
  if (s->desc.y_norm == BO_YNORM_NONE) { m = 0.0; v = 1.0; }
  if (v == 0.0) v = 1.0;
  *mean = m;
  *std_ = v;
  *ymin = mn;
}

double median(std::vector<double> a) {
  std::sort(a.begin(), a.end());
  const size_t n = a.size();
  return n % 2 ? a[n / 2] : 0.5 * (a[n / 2 - 1] + a[n / 2]);
}

int prepare_pass(bo_space* s, const std::vector<int>& afs, int slot, PassArgs* out) {
  PassArgs a{};
  a.n = s->n_fit;
  a.n_unvisited = s->N - s->n_visited;
  a.n_af = (int)afs.size();
  for (int q = 0; q < 3; ++q) a.af[q] = q < a.n_af ? afs[q] : 0;
  a.k = a.n_af;
  a.explore = s->desc.explore;
  a.lambda_const = s->desc.lambda_const;
  double mean, sd, ymin;
  y_stats(s, &mean, &sd, &ymin);
  a.fplus_t = (ymin - mean) / sd;
  a.fplus_raw = ymin;
  a.first_pass = 0;
  if (s->desc.explore == BO_EXPLORE_CV) {
    double mu_s = s->mu_s;
    if (!s->cv_set) {
      mu_s = 0;
      for (double y : s->fit_y) mu_s += y;
      mu_s /= (double)s->fit_y.size();
      a.first_pass = 1;
    }
    if (!(ymin > 0.0) || !(mu_s > 0.0))
      return fail(BO_ERR_NOT_POSITIVE,
                  "contextual variance needs a positive best observation (%g) and initial mean (%g)",
                  ymin, mu_s);
    a.mu_s_raw = mu_s;
    if (!s->cv_set) { s->mu_s = mu_s; s->cv_set = true; }
  }
  a.result_slot = slot;
  *out = a;
  return BO_OK;
}

int launch_pass(bo_space* s, const std::vector<int>& afs, int slot) {
  PassArgs a;
  const int rc = prepare_pass(s, afs, slot, &a);
  if (rc != BO_OK) return rc;
  if (s->desc.precision != BO_PREC_FP64 && s->fused_acquire) {
    const int k = launch_predict_acquire_tc(s->v, s->n_fit, a, s->stream);
    if (k > 0) {
      s->launches += k;
      return BO_OK;
    }
    if (k != -2) return fail(BO_ERR_CUDA, "prediction launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    s->fused_acquire = false;      // not launchable cooperatively here: two launches from now on
  }
  const int k1 = s->desc.precision == BO_PREC_FP64
                     ? launch_predict_f64(s->v, s->n_fit, a.n_unvisited, s->stream)
                     : launch_predict_tc(s->v, s->n_fit, a.n_unvisited, s->stream);
  if (k1 < 0) return fail(BO_ERR_CUDA, "prediction launch failed: %s",
                          cudaGetErrorString(cudaGetLastError()));
  const int k2 = launch_acquire(s->v, a, s->stream);
  if (k2 < 0) return fail(BO_ERR_CUDA, "acquisition launch failed: %s",
                          cudaGetErrorString(cudaGetLastError()));
  s->launches += k1 + k2;
  return BO_OK;
}

int fetch_result(bo_space* s, int slot) {
  BO_CUDA(cudaMemcpyAsync(s->host_result, s->v.results + slot, sizeof(bo_pass_result),
                          cudaMemcpyDeviceToHost, s->stream));
  BO_CUDA(cudaStreamSynchronize(s->stream));
  s->last = *s->host_result;
  if (s->host_result->status != BO_OK) {
    s->poisoned = s->host_result->status;
    return fail(s->poisoned, "device reported status %d (non-positive pivot or non-finite posterior)",
                s->poisoned);
  }
  return BO_OK;
}

int observe_host(bo_space* s, int64_t idx, double value, bool* fit, int* n_before, double* y_mean,
                 double* y_std) {
  if (idx < 0 || idx >= s->N) return fail(BO_ERR_INDEX, "index %lld out of range [0, %lld)",
                                          (long long)idx, (long long)s->N);
  if (s->visited[idx]) return fail(BO_ERR_DUPLICATE, "configuration %lld already observed",
                                   (long long)idx);
  const bool finite = std::isfinite(value);
  if (finite && s->n_fit >= s->n_cap)
    return fail(BO_ERR_CAPACITY, "more than n_max = %d valid observations", s->n_cap);
  s->visited[idx] = 1;
  ++s->n_visited;
  s->obs_idx.push_back(idx);
  s->obs_y.push_back(value);
  *fit = finite;
  *n_before = s->n_fit;
  if (finite) {
    s->fit_y.push_back(value);
    double ymin;
    y_stats(s, y_mean, y_std, &ymin);
    ++s->n_fit;
  }
  auto it = s->outstanding.find(idx);
  if (it != s->outstanding.end()) {
    if (finite) s->sel.credit(it->second, value);
    else if (!s->fit_y.empty()) s->sel.credit(it->second, median(s->fit_y));
    s->outstanding.erase(it);
  }
  return BO_OK;
}

int observe_impl(bo_space* s, int64_t idx, double value) {
  bool fit = false;
  int n_before = 0;
  double mean = 0.0, sd = 1.0;
  int rc = observe_host(s, idx, value, &fit, &n_before, &mean, &sd);
  if (rc != BO_OK) return rc;
  int k = 0;
  if (fit) {
    ObsNew o;
    make_obs_new(s, idx, value, mean, sd, &o);
    k = launch_observe_update(s->coop_update, s->v, n_before, o, s->stream);
  } else {
    k = launch_set_visited(s->v, idx, s->stream);
  }
  if (k < 0) return fail(BO_ERR_CUDA, "update launch failed");
  s->launches += k;
  return BO_OK;
}

int suggest_begin(bo_space* s, int64_t* idx_out, bo_suggest_info* info, bool* need_pass) {
  *need_pass = false;
  bo_suggest_info inf{};
  inf.af = -1;
  if (s->n_visited >= s->N) return fail(BO_ERR_EXHAUSTED, "every valid configuration was evaluated");
  if (s->n_fit < s->desc.n_init || s->n_fit == 0) {
    // initial sample (Sec. III-E): the Latin hypercube design first, then
    // random unobserved configurations until n_init valid observations exist
    if (s->desc.init_mode != BO_INIT_RANDOM && s->desc.n_init > 0 && !s->init_built) {
      s->init_built = true;
      const int count = (int)std::min<int64_t>(s->desc.n_init, s->N);
      std::vector<int64_t> design(count);
      auto valid_of = [s](int64_t flat) -> int64_t {   // binary search: the valid list is in flat order
        int64_t lo = 0, hi = s->N;
        while (lo < hi) {
          const int64_t mid = (lo + hi) / 2;
          int64_t f = 0;
          for (int p = 0; p < s->d; ++p) f = f * s->sizes[p] + s->codes[(size_t)p * s->N + mid];
          if (f < flat) lo = mid + 1; else hi = mid;
        }
        if (lo == s->N) return -1;
        int64_t f = 0;
        for (int p = 0; p < s->d; ++p) f = f * s->sizes[p] + s->codes[(size_t)p * s->N + lo];
        return f == flat ? lo : -1;
      };
      const int rc = initial_design(s->values, s->N, valid_of, count, s->desc.init_mode, s->desc.init_designs,
                                    s->rng, design.data());
      if (rc != BO_OK) return rc;
      s->init_queue.assign(design.begin(), design.end());
    }
    while (!s->init_queue.empty() && s->visited[s->init_queue.front()]) s->init_queue.pop_front();
    if (!s->init_queue.empty()) {
      inf.idx = s->init_queue.front();
      s->init_queue.pop_front();
      *idx_out = inf.idx;
      if (info) *info = inf;
      return BO_OK;
    }
    const int64_t free_count = s->N - s->n_visited;
    int64_t r = (int64_t)(splitmix64_next(s->rng) % (uint64_t)free_count);
    int64_t idx = -1;
    for (int64_t i = 0; i < s->N; ++i)
      if (!s->visited[i] && r-- == 0) { idx = i; break; }
    inf.idx = idx;
    *idx_out = idx;
    if (info) *info = inf;
    return BO_OK;
  }
  while (!s->queue.empty()) {
    Pick p = s->queue.front();
    s->queue.pop_front();
    if (s->visited[p.idx]) continue;
    s->outstanding[p.idx] = p.afs;
    inf.idx = p.idx;
    inf.af = p.afs[0];
    inf.predicted = 1;
    inf.mu = p.mu;
    inf.sigma = p.sigma;
    inf.score = p.score;
    inf.lambda = s->last.lambda;
    inf.mean_var = s->last.mean_var;
    inf.n_scored = 0;
    *idx_out = p.idx;
    if (info) *info = inf;
    return BO_OK;
  }
  s->sel.begin_round();
  s->outstanding.clear();
  *need_pass = true;
  return BO_OK;
}

int suggest_finish(bo_space* s, const bo_pass_result& r, int64_t* idx_out, bo_suggest_info* info) {
  s->last = r;
  if (r.status != BO_OK) {
    s->poisoned = r.status;
    return fail(r.status, "device reported status %d (non-positive pivot, non-finite posterior or timeout)",
                r.status);
  }
  std::vector<Pick> picks = s->sel.assign(r);
  if (picks.empty()) return fail(BO_ERR_EXHAUSTED, "no pick available");
  s->queue.assign(picks.begin() + 1, picks.end());
  const Pick& p = picks[0];
  s->outstanding[p.idx] = p.afs;
  bo_suggest_info inf{};
  inf.idx = p.idx;
  inf.af = p.afs[0];
  inf.predicted = 1;
  inf.mu = p.mu;
  inf.sigma = p.sigma;
  inf.score = p.score;
  inf.lambda = r.lambda;
  inf.mean_var = r.mean_var;
  inf.n_scored = r.n_scored;
  *idx_out = p.idx;
  if (info) *info = inf;
  return BO_OK;
}

// Every check of a space descriptor that needs no device: the fields, the
// value lists and the size of the product (*total_out); the mask's content is
// the caller's to check.  BO_OK, or BO_ERR_ARG with the message set.
int check_space_desc(const bo_space_desc& D, int64_t* total_out) {
  if (D.d < 1 || D.d > BO_MAX_PARAMS) return fail(BO_ERR_ARG, "d = %d not in [1, %d]", D.d, BO_MAX_PARAMS);
  if (!D.n_values || !D.values) return fail(BO_ERR_ARG, "n_values / values missing");
  if (!(D.nu == 1.5 || D.nu == 2.5)) return fail(BO_ERR_ARG, "nu must be 1.5 or 2.5");
  if (!(D.lengthscale > 0) || !(D.jitter >= 0)) return fail(BO_ERR_ARG, "bad lengthscale / jitter");
  if (D.af < BO_AF_EI || D.af > BO_AF_ADV_MULTI) return fail(BO_ERR_ARG, "bad af");
  if (D.explore != BO_EXPLORE_CV && D.explore != BO_EXPLORE_CONST) return fail(BO_ERR_ARG, "bad explore");
  if (D.precision < BO_PREC_FP64 || D.precision > BO_PREC_TF32X3) return fail(BO_ERR_ARG, "bad precision");
  if (D.n_max < 1 || D.n_max > BO_MAX_OBS) return fail(BO_ERR_ARG, "n_max not in [1, %d]", BO_MAX_OBS);
  if (D.skip_threshold < 0 || D.n_init < 0 || D.init_designs < 0) return fail(BO_ERR_ARG, "negative count");
  if (D.init_mode < BO_INIT_RANDOM || D.init_mode > BO_INIT_MAXIMIN) return fail(BO_ERR_ARG, "bad init_mode");
  int64_t total = 1;
  for (int p = 0; p < D.d; ++p) {
    if (D.n_values[p] < 1 || D.n_values[p] > BO_MAX_VALUES || !D.values[p])
      return fail(BO_ERR_ARG, "parameter %d: bad value list", p);
    for (int i = 0; i < D.n_values[p]; ++i)
      if (!(D.values[p][i] >= 0.0 && D.values[p][i] <= 1.0))
        return fail(BO_ERR_ARG, "parameter %d value %d not normalized to [0, 1]", p, i);
    total *= D.n_values[p];
    if (total > ((int64_t)1 << 40)) return fail(BO_ERR_ARG, "search space too large");
  }
  *total_out = total;
  return BO_OK;
}

}  // namespace host
}  // namespace bo

extern "C" {

void bo_space_desc_init(bo_space_desc* d) {
  if (!d) return;
  std::memset(d, 0, sizeof *d);
  d->nu = 1.5;
  d->lengthscale = 1.5;
  d->jitter = 1e-10;
  d->af = BO_AF_EI;
  d->explore = BO_EXPLORE_CV;
  d->lambda_const = 0.01;
  d->skip_threshold = 5;
  d->rif = 0.1;
  d->discount = 0.0;
  d->y_norm = BO_YNORM_STANDARDIZE;
  d->precision = BO_PREC_FP64;
  d->n_max = BO_MAX_OBS;
  d->init_mode = BO_INIT_MAXIMIN;
  d->init_designs = 100;
}

const char* bo_last_error(void) { return g_err.c_str(); }

int bo_space_create(const bo_space_desc* desc, bo_space** out) {
  g_err.clear();
  if (!desc || !out) return fail(BO_ERR_ARG, "null argument");
  *out = nullptr;
  const bo_space_desc& D = *desc;
  int64_t total = 0;
  if (const int rc = check_space_desc(D, &total); rc != BO_OK) return rc;

  bo_space* s = new (std::nothrow) bo_space();
  if (!s) return fail(BO_ERR_NOMEM, "host allocation failed");
  s->desc = D;
  s->desc.n_values = nullptr;
  s->desc.values = nullptr;
  s->desc.invalid_mask = nullptr;
  s->stream = (cudaStream_t)D.stream;
  cudaGetDevice(&s->device);
  s->d = D.d;
  s->n_cap = D.n_max;
  s->rng = D.seed;
  s->coop_update = getenv("BO_NO_COOP") == nullptr;
  s->fused_acquire = getenv("BO_FUSED_ACQ") != nullptr;
  s->sel.init(D.af, D.skip_threshold, D.discount, D.rif);
  for (int p = 0; p < D.d; ++p) {
    s->sizes.push_back(D.n_values[p]);
    s->values.emplace_back(D.values[p], D.values[p] + D.n_values[p]);
  }
  // valid list: row-major product, last parameter fastest, restricted removed
  int64_t nvalid = 0;
  for (int64_t f = 0; f < total; ++f) nvalid += !(D.invalid_mask && D.invalid_mask[f]);
  if (nvalid == 0) { delete s; return fail(BO_ERR_ARG, "no valid configuration"); }
  // the FP32 acquisition packs a valid-list index into 32 bits
  if (D.precision != BO_PREC_FP64 && nvalid >= (int64_t)0xFFFFFFFF) {
    delete s;
    return fail(BO_ERR_ARG, "reduced precision holds fewer than 2^32 - 1 valid configurations");
  }
  s->N = nvalid;
  const int64_t N_pad = (nvalid + kTileRows - 1) / kTileRows * kTileRows;
  std::vector<uint8_t> codes((size_t)D.d * N_pad, 0);
  {
    std::vector<int> digit(D.d, 0);
    int64_t i = 0;
    for (int64_t f = 0; f < total; ++f) {
      if (!(D.invalid_mask && D.invalid_mask[f])) {
        for (int p = 0; p < D.d; ++p) codes[(size_t)p * N_pad + i] = (uint8_t)digit[p];
        ++i;
      }
      for (int p = D.d - 1; p >= 0; --p) {
        if (++digit[p] < D.n_values[p]) break;
        digit[p] = 0;
      }
    }
  }
  s->codes.resize((size_t)D.d * nvalid);
  for (int p = 0; p < D.d; ++p)
    std::memcpy(&s->codes[(size_t)p * nvalid], &codes[(size_t)p * N_pad], nvalid);
  s->visited.assign(nvalid, 0);

  DevView& v = s->v;
  v.d = D.d;
  v.N = nvalid;
  v.N_pad = N_pad;
  const int n_alloc = (D.n_max + 31) / 32 * 32;
  v.n_max = n_alloc;
  v.precision = D.precision;
  v.nu = D.nu;
  v.lengthscale = D.lengthscale;
  v.jitter = D.jitter;
  v.kcoef = std::sqrt(2.0 * D.nu) / D.lengthscale;
  int num_sms = 152;
  cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, s->device);
  v.max_partials = (int)(N_pad / 32) + num_sms;
  v.max_acq_blocks = 4 * num_sms;
  v.num_sms = num_sms;
  v.max_results = 1024;
  const size_t fsz = D.precision == BO_PREC_FP64 ? 8 : 4;
  int rc = BO_OK;
  uint8_t* dcodes = nullptr;
  double* vt64 = nullptr;
  float* vt32 = nullptr;
  void* mu = nullptr;
  void* var = nullptr;
#define TRY(x) do { rc = (x); if (rc != BO_OK) { release(s); delete s; return rc; } } while (0)
  TRY(dalloc_n(s, (size_t)D.d * N_pad, &dcodes));
  TRY(dalloc_n(s, (size_t)D.d * 256, &vt64));
  TRY(dalloc_n(s, (size_t)D.d * 256, &vt32));
  TRY(dalloc_n(s, (size_t)N_pad / 32 + 1, &v.visited));
  TRY(dalloc_n(s, (size_t)n_alloc * D.d, &v.X));
  TRY(dalloc_n(s, (size_t)n_alloc * D.d, &v.Xc));
  // per-parameter tables of squared value differences, when they are small
  std::vector<int> sqd_meta(2 * D.d + 1, 0);
  size_t sqd_total = 0;
  for (int p = 0; p < D.d; ++p) {
    sqd_meta[p] = (int)sqd_total;
    sqd_meta[D.d + 1 + p] = D.n_values[p];
    sqd_total += (size_t)D.n_values[p] * D.n_values[p];
  }
  sqd_meta[D.d] = (int)sqd_total;
  double* dsqd = nullptr;
  int* dmeta = nullptr;
  if (sqd_total * sizeof(double) <= kSqdMaxBytes) {
    TRY(dalloc_n(s, sqd_total, &dsqd));
    TRY(dalloc_n(s, sqd_meta.size(), &dmeta));
  }
  v.ds = D.precision == BO_PREC_FP64 ? 0 : tc_dim_bucket(D.d);
  if (D.precision != BO_PREC_FP64) TRY(dalloc_n(s, (size_t)(v.ds + 2) * n_alloc, &v.xq));
  TRY(dalloc_n(s, (size_t)n_alloc, &v.y));
  TRY(dalloc_n(s, (size_t)n_alloc * n_alloc, &v.linv));
  TRY(dalloc_n(s, (size_t)n_alloc, &v.beta));
  TRY(dalloc_n(s, (size_t)n_alloc, &v.uvec));
  TRY(dalloc_n(s, (size_t)n_alloc, &v.evec));
  if (D.precision != BO_PREC_FP64) {
    TRY(dalloc_n(s, (size_t)n_alloc, &v.avec));
    TRY(dalloc_n(s, (size_t)n_alloc, &v.bvec));
  }
  if (D.precision != BO_PREC_FP64) {
    TRY(dalloc_n(s, lsplit_bytes(n_alloc, D.precision), &v.lsplit_hi));
    if (split_parts(D.precision) == 2) TRY(dalloc_n(s, lsplit_bytes(n_alloc, D.precision), &v.lsplit_lo));
  }
  TRY(dalloc(s, (size_t)N_pad * fsz, &mu));
  TRY(dalloc(s, (size_t)N_pad * fsz, &var));
  TRY(dalloc_n(s, (size_t)v.max_partials, &v.partial));
  TRY(dalloc_n(s, (size_t)n_alloc, &v.kvec));
  TRY(dalloc_n(s, (size_t)n_alloc, &v.lvec));
  TRY(dalloc_n(s, (size_t)8 * n_alloc, &v.wvec));
  TRY(dalloc_n(s, update_part_count(n_alloc), &v.upart));
  TRY(dalloc_n(s, 1, &v.stats));
  TRY(dalloc_n(s, (size_t)v.max_acq_blocks * 9, &v.acq_partial));
  TRY(dalloc_n(s, (size_t)v.max_results, &v.results));
#undef TRY
  v.codes = dcodes;
  v.vtab64 = vt64;
  v.sqd = dsqd;
  v.sqd_meta = dmeta;
  v.sqd_total = dsqd ? (int)sqd_total : 0;
  v.vtab32 = vt32;
  v.mu = mu;
  v.var = var;
  std::vector<double> t64((size_t)D.d * 256, 0.0);
  std::vector<float> t32((size_t)D.d * 256, 0.0f);
  const double cs = coord_scale(D.nu, D.lengthscale);
  for (int p = 0; p < D.d; ++p)
    for (int i = 0; i < D.n_values[p]; ++i) {
      t64[(size_t)p * 256 + i] = D.values[p][i];
      t32[(size_t)p * 256 + i] = (float)(D.values[p][i] * cs);
    }
  // (v_a - v_b)^2 rounded once, as the distance loops would form each term
  std::vector<double> sqd(dsqd ? sqd_total : 0);
  for (int p = 0; dsqd && p < D.d; ++p) {
    const int m = D.n_values[p];
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) {
        const double diff = D.values[p][a] - D.values[p][b];
        sqd[(size_t)sqd_meta[p] + (size_t)a * m + b] = diff * diff;
      }
  }
  cudaError_t e = cudaMemcpyAsync(dcodes, codes.data(), codes.size(), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess && dsqd)
    e = cudaMemcpyAsync(dsqd, sqd.data(), sqd.size() * 8, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess && dmeta)
    e = cudaMemcpyAsync(dmeta, sqd_meta.data(), sqd_meta.size() * 4, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(vt64, t64.data(), t64.size() * 8, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(vt32, t32.data(), t32.size() * 4, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMallocHost(&s->host_result, sizeof(bo_pass_result));
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) { rc = cuda_fail(e, "space upload"); release(s); delete s; return rc; }
  *out = s;
  return BO_OK;
}

int bo_space_destroy(bo_space* s) {
  if (!s) return fail(BO_ERR_ARG, "null space");
  cudaSetDevice(s->device);
  release(s);
  delete s;
  return BO_OK;
}

int bo_valid_count(const bo_space* s, int64_t* out) {
  if (!s || !out) return fail(BO_ERR_ARG, "null argument");
  *out = s->N;
  return BO_OK;
}

int bo_decode(const bo_space* s, int64_t idx, int32_t* value_idx_out) {
  if (!s || !value_idx_out) return fail(BO_ERR_ARG, "null argument");
  if (idx < 0 || idx >= s->N) return fail(BO_ERR_INDEX, "index out of range");
  for (int p = 0; p < s->d; ++p) value_idx_out[p] = s->codes[(size_t)p * s->N + idx];
  return BO_OK;
}

int bo_observe(bo_space* s, int64_t idx, double value) {
  if (!s) return fail(BO_ERR_ARG, "null space");
  if (s->poisoned) return fail(s->poisoned, "space is unusable after an earlier numeric failure");
  cudaSetDevice(s->device);
  return observe_impl(s, idx, value);
}

int bo_suggest(bo_space* s, int64_t* idx_out, bo_suggest_info* info) {
  if (!s || !idx_out) return fail(BO_ERR_ARG, "null argument");
  if (s->poisoned) return fail(s->poisoned, "space is unusable after an earlier numeric failure");
  cudaSetDevice(s->device);
  bool need_pass = false;
  int rc = suggest_begin(s, idx_out, info, &need_pass);
  if (rc != BO_OK || !need_pass) return rc;
  rc = launch_pass(s, s->sel.active, 0);
  if (rc != BO_OK) return rc;
  BO_CUDA(cudaMemcpyAsync(s->host_result, s->v.results, sizeof(bo_pass_result), cudaMemcpyDeviceToHost,
                          s->stream));
  BO_CUDA(cudaStreamSynchronize(s->stream));
  return suggest_finish(s, *s->host_result, idx_out, info);
}

int bo_last_posterior(bo_space* s, int64_t begin, int64_t count, double* mu_out, double* var_out) {
  if (!s || (!mu_out && !var_out)) return fail(BO_ERR_ARG, "null argument");
  if (begin < 0 || count < 0 || begin + count > s->N) return fail(BO_ERR_INDEX, "range out of bounds");
  cudaSetDevice(s->device);
  const size_t eb = s->desc.precision == BO_PREC_FP64 ? 8 : 4;
  std::vector<uint8_t> tmp((size_t)count * eb);
  for (int w = 0; w < 2; ++w) {
    double* dst = w ? var_out : mu_out;
    if (!dst) continue;
    const uint8_t* src = static_cast<const uint8_t*>(w ? s->v.var : s->v.mu) + (size_t)begin * eb;
    BO_CUDA(cudaMemcpyAsync(tmp.data(), src, (size_t)count * eb, cudaMemcpyDeviceToHost, s->stream));
    BO_CUDA(cudaStreamSynchronize(s->stream));
    for (int64_t i = 0; i < count; ++i)
      dst[i] = eb == 8 ? reinterpret_cast<const double*>(tmp.data())[i] : reinterpret_cast<const float*>(tmp.data())[i];
  }
  return BO_OK;
}

int bo_predict(bo_space* s, int64_t begin, int64_t count, double* mu_out, double* var_out) {
  if (!s || (!mu_out && !var_out)) return fail(BO_ERR_ARG, "null argument");
  if (begin < 0 || count < 0 || begin + count > s->N) return fail(BO_ERR_INDEX, "range out of bounds");
  cudaSetDevice(s->device);
  if (s->n_fit == 0) {   // the prior
    for (int64_t i = 0; i < count; ++i) {
      if (mu_out) mu_out[i] = 0.0;
      if (var_out) var_out[i] = 1.0;
    }
    return BO_OK;
  }
  const int k1 = s->desc.precision == BO_PREC_FP64
                     ? launch_predict_f64(s->v, s->n_fit, s->N - s->n_visited, s->stream)
                     : launch_predict_tc(s->v, s->n_fit, s->N - s->n_visited, s->stream);
  if (k1 < 0) return fail(BO_ERR_CUDA, "prediction launch failed");
  s->launches += k1;
  if (s->desc.precision == BO_PREC_FP64) {
    if (mu_out) BO_CUDA(cudaMemcpyAsync(mu_out, (double*)s->v.mu + begin, count * 8, cudaMemcpyDeviceToHost, s->stream));
    if (var_out) BO_CUDA(cudaMemcpyAsync(var_out, (double*)s->v.var + begin, count * 8, cudaMemcpyDeviceToHost, s->stream));
    BO_CUDA(cudaStreamSynchronize(s->stream));
  } else {
    std::vector<float> tmp(count);
    for (int w = 0; w < 2; ++w) {
      double* dst = w ? var_out : mu_out;
      if (!dst) continue;
      const float* src = (const float*)(w ? s->v.var : s->v.mu) + begin;
      BO_CUDA(cudaMemcpyAsync(tmp.data(), src, count * 4, cudaMemcpyDeviceToHost, s->stream));
      BO_CUDA(cudaStreamSynchronize(s->stream));
      for (int64_t i = 0; i < count; ++i) dst[i] = tmp[i];
    }
  }
  return BO_OK;
}

int bo_predict_enqueue(bo_space* s) {
  if (!s) return fail(BO_ERR_ARG, "null space");
  if (s->n_fit == 0) return fail(BO_ERR_STATE, "no valid observation to predict from");
  cudaSetDevice(s->device);
  const int k1 = s->desc.precision == BO_PREC_FP64
                     ? launch_predict_f64(s->v, s->n_fit, s->N - s->n_visited, s->stream)
                     : launch_predict_tc(s->v, s->n_fit, s->N - s->n_visited, s->stream);
  if (k1 < 0) return fail(BO_ERR_CUDA, "prediction launch failed");
  s->launches += k1;
  return BO_OK;
}

int bo_autotune(bo_space* s, int32_t reps, bo_tune_result* out) {
  if (!s) return fail(BO_ERR_ARG, "null space");
  if (s->desc.precision == BO_PREC_FP64) return fail(BO_ERR_ARG, "the FP64 pass has no tensor-core shapes");
  if (s->n_fit == 0) return fail(BO_ERR_STATE, "no valid observation to predict from");
  cudaSetDevice(s->device);
  BO_CUDA(cudaStreamSynchronize(s->stream));
  const TcSess ts = tc_session(s->v, s->n_fit);
  return autotune_shapes(s->stream, reps, s->desc.precision, s->desc.nu, tc_dim_bucket(s->d), ts.n_pad, false,
                         [&] { return launch_predict_tc(s->v, s->n_fit, s->N - s->n_visited, s->stream); }, out);
}

int bo_tuned_shape(const bo_space* s, bo_tune_result* out) {
  if (!s || !out) return fail(BO_ERR_ARG, "null argument");
  if (s->desc.precision == BO_PREC_FP64) return fail(BO_ERR_ARG, "the FP64 pass has no tensor-core shapes");
  if (s->n_fit == 0) return fail(BO_ERR_STATE, "no valid observation to predict from");
  const TcSess ts = tc_session(s->v, s->n_fit);
  TcShape sh{};
  std::memset(out, 0, sizeof *out);
  if (!tc_stored_shape(s->desc.precision, s->desc.nu, tc_dim_bucket(s->d), ts.n_pad, false, &sh))
    return fail(BO_ERR_STATE, "no shape stored for this launch key");
  out->stages_a = sh.stages_a;
  out->b_slots = sh.b_slots;
  out->b_resident = sh.b_resident;
  return BO_OK;
}

int bo_get_factor(bo_space* s, double* linv_out, double* beta_out, int32_t* n_out) {
  if (!s) return fail(BO_ERR_ARG, "null space");
  cudaSetDevice(s->device);
  const int n = s->n_fit;
  if (n_out) *n_out = n;
  if (n == 0) return BO_OK;
  if (linv_out)
    BO_CUDA(cudaMemcpy2DAsync(linv_out, (size_t)n * 8, s->v.linv, (size_t)s->v.n_max * 8, (size_t)n * 8, n,
                              cudaMemcpyDeviceToHost, s->stream));
  if (beta_out) BO_CUDA(cudaMemcpyAsync(beta_out, s->v.beta, (size_t)n * 8, cudaMemcpyDeviceToHost, s->stream));
  BO_CUDA(cudaStreamSynchronize(s->stream));
  return BO_OK;
}

int bo_sync(bo_space* s) {
  if (!s) return fail(BO_ERR_ARG, "null space");
  cudaSetDevice(s->device);
  BO_CUDA(cudaStreamSynchronize(s->stream));
  DevStats st;
  BO_CUDA(cudaMemcpy(&st, s->v.stats, sizeof st, cudaMemcpyDeviceToHost));
  if (st.status != BO_OK) {
    s->poisoned = st.status;
    return fail(st.status, "observation update failed (non-positive pivot)");
  }
  return BO_OK;
}

int bo_replay_enqueue(bo_space* s, const int64_t* idx, const double* y, int32_t steps) {
  if (!s || (steps > 0 && (!idx || !y))) return fail(BO_ERR_ARG, "null argument");
  if (steps < 0 || steps > s->v.max_results) return fail(BO_ERR_ARG, "steps not in [0, %d]", s->v.max_results);
  if (s->poisoned) return fail(s->poisoned, "space is unusable after an earlier numeric failure");
  cudaSetDevice(s->device);
  const std::vector<int> all = {kEI, kPI, kLCB};
  for (int32_t t = 0; t < steps; ++t) {
    int rc = observe_impl(s, idx[t], y[t]);
    if (rc != BO_OK) return rc;
    if (s->n_fit == 0) return fail(BO_ERR_STATE, "replay step %d has no valid observation yet", t);
    if (s->n_visited >= s->N) return fail(BO_ERR_EXHAUSTED, "search space exhausted at step %d", t);
    rc = launch_pass(s, all, t);
    if (rc != BO_OK) return rc;
  }
  s->replay_steps = steps;
  return BO_OK;
}

int bo_replay_fetch(bo_space* s, bo_pass_result* out, int32_t steps) {
  if (!s || (steps > 0 && !out)) return fail(BO_ERR_ARG, "null argument");
  if (steps > s->replay_steps) return fail(BO_ERR_ARG, "only %d replay results", s->replay_steps);
  cudaSetDevice(s->device);
  BO_CUDA(cudaMemcpyAsync(out, s->v.results, sizeof(bo_pass_result) * steps, cudaMemcpyDeviceToHost,
                          s->stream));
  BO_CUDA(cudaStreamSynchronize(s->stream));
  for (int32_t t = 0; t < steps; ++t)
    if (out[t].status != BO_OK) {
      s->poisoned = out[t].status;
      return fail(out[t].status, "replay step %d reported status %d", t, out[t].status);
    }
  return BO_OK;
}

int bo_selftest_waits(int32_t* mbar_status, int32_t* grid_status) {
  if (!mbar_status || !grid_status) return fail(BO_ERR_ARG, "null argument");
  // [0, 8): mbarrier status, [8, 16): its abort flag, [16, 16 + sizeof(DevStats)): grid barrier state
  static_assert(16 + sizeof(DevStats) <= 64, "scratch size");
  void* buf = nullptr;
  BO_CUDA(cudaMalloc(&buf, 64));
  cudaError_t e = cudaMemset(buf, 0, 64);
  auto* bytes = static_cast<uint8_t*>(buf);
  int32_t* st1 = reinterpret_cast<int32_t*>(bytes);
  int* abort1 = reinterpret_cast<int*>(bytes + 8);
  DevStats* st2 = reinterpret_cast<DevStats*>(bytes + 16);
  if (e == cudaSuccess && launch_selftest_mbar(st1, abort1, nullptr) < 0) e = cudaGetLastError();
  if (e == cudaSuccess && launch_selftest_grid(st2, nullptr) < 0) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  DevStats h2{};
  if (e == cudaSuccess) e = cudaMemcpy(mbar_status, st1, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&h2, st2, sizeof h2, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "self-test of the bounded waits");
  *grid_status = h2.status;
  return BO_OK;
}

int bo_selftest_exp(const double* t, double* out, double* ref, int32_t n) {
  if (!t || !out || !ref) return fail(BO_ERR_ARG, "null argument");
  if (n < 1 || n > (1 << 24)) return fail(BO_ERR_ARG, "n must be in [1, 2^24]");
  const size_t bytes = (size_t)n * sizeof(double);
  double* buf = nullptr;
  BO_CUDA(cudaMalloc(&buf, 3 * bytes));
  cudaError_t e = cudaMemcpy(buf, t, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && launch_selftest_exp(buf, buf + n, buf + 2 * (size_t)n, n, nullptr) < 0)
    e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(out, buf + n, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ref, buf + 2 * (size_t)n, bytes, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "self-test of the FP64 pass's exponential");
  return BO_OK;
}

int bo_launch_count(const bo_space* s, int64_t* out) {
  if (!s || !out) return fail(BO_ERR_ARG, "null argument");
  *out = s->launches;
  return BO_OK;
}

}  // extern "C"
