// Initial sample of a search space (paper Sec. III-E; Table I selects the
// maximin variant): a Latin hypercube over the parameters' value lists, or the
// best of several by the maximin criterion, mapped onto configurations, with
// restricted or repeated configurations replaced by random valid ones.  Host
// code: it runs once per session, before the first prediction pass.  The
// draw order is part of the interface (include/bo_suggest.h), so that every
// caller, and any other implementation, reproduces the same sample.
#include <algorithm>
#include <cmath>
#include <functional>
#include <unordered_set>
#include <vector>

#include "bo_space_impl.h"

namespace bo {
namespace host {

int initial_design(const std::vector<std::vector<double>>& values, int64_t n_valid,
                   const std::function<int64_t(int64_t)>& valid_of, int count, int mode, int designs,
                   uint64_t& rng, int64_t* out) {
  if (count < 1 || count > n_valid) return fail(BO_ERR_ARG, "initial sample of %d from %lld", count, (long long)n_valid);
  if (mode < BO_INIT_RANDOM || mode > BO_INIT_MAXIMIN) return fail(BO_ERR_ARG, "bad init_mode");
  std::unordered_set<int64_t> taken;
  auto random_valid = [&]() {
    for (;;) {
      const int64_t r = (int64_t)(splitmix64_next(rng) % (uint64_t)n_valid);
      if (taken.insert(r).second) return r;
    }
  };
  if (mode == BO_INIT_RANDOM) {
    for (int i = 0; i < count; ++i) out[i] = random_valid();
    return BO_OK;
  }
  const int d = (int)values.size();
  const int T = mode == BO_INIT_MAXIMIN ? std::max(designs, 1) : 1;
  std::vector<int> cur((size_t)count * d), best;
  std::vector<int> perm(count);
  double best_score = 0.0;
  const unsigned __int128 denom = (unsigned __int128)count << 53;
  for (int t = 0; t < T; ++t) {
    for (int p = 0; p < d; ++p) {
      for (int i = 0; i < count; ++i) perm[i] = i;
      for (int i = count - 1; i > 0; --i) {
        const int j = (int)(splitmix64_next(rng) % (uint64_t)(i + 1));
        std::swap(perm[i], perm[j]);
      }
      const unsigned __int128 m = (unsigned __int128)values[p].size();
      for (int i = 0; i < count; ++i) {
        const uint64_t r = splitmix64_next(rng) >> 11;             // U = r / 2^53
        const unsigned __int128 num = (((unsigned __int128)perm[i] << 53) + r) * m;
        cur[(size_t)i * d + p] = (int)(num / denom);              // floor((pi + U) m / count)
      }
    }
    double score = 0.0;
    if (T > 1 && count > 1) {                // smallest squared distance between two samples
      score = INFINITY;
      for (int i = 0; i < count; ++i)
        for (int j = i + 1; j < count; ++j) {
          double s = 0.0;
          for (int p = 0; p < d; ++p) {
            const double df = values[p][cur[(size_t)i * d + p]] - values[p][cur[(size_t)j * d + p]];
            s = s + df * df;
          }
          if (s < score) score = s;
        }
    }
    if (t == 0 || score > best_score) {
      best = cur;
      best_score = score;
    }
  }
  // configurations (row-major, last parameter fastest), then replacements in order
  std::vector<int64_t> idx(count, -1);
  for (int i = 0; i < count; ++i) {
    int64_t flat = 0;
    for (int p = 0; p < d; ++p) flat = flat * (int64_t)values[p].size() + best[(size_t)i * d + p];
    const int64_t v = valid_of(flat);
    if (v >= 0 && taken.insert(v).second) idx[i] = v;
  }
  for (int i = 0; i < count; ++i) {
    if (idx[i] < 0) idx[i] = random_valid();
    out[i] = idx[i];
  }
  return BO_OK;
}

}  // namespace host
}  // namespace bo

using namespace bo::host;

int bo_initial_design(const bo_space_desc* desc, int32_t count, int64_t* idx_out) {
  if (!desc || !idx_out) return fail(BO_ERR_ARG, "null argument");
  const bo_space_desc& D = *desc;
  if (D.d < 1 || D.d > BO_MAX_PARAMS || !D.n_values || !D.values) return fail(BO_ERR_ARG, "bad parameters");
  std::vector<std::vector<double>> values(D.d);
  int64_t total = 1;
  for (int p = 0; p < D.d; ++p) {
    if (D.n_values[p] < 1 || D.n_values[p] > BO_MAX_VALUES || !D.values[p])
      return fail(BO_ERR_ARG, "parameter %d: bad value list", p);
    values[p].assign(D.values[p], D.values[p] + D.n_values[p]);
    total *= D.n_values[p];
    if (total > ((int64_t)1 << 40)) return fail(BO_ERR_ARG, "search space too large");
  }
  // valid-list position of every valid flat index, by binary search over them
  std::vector<int64_t> valid_flats;
  for (int64_t f = 0; f < total; ++f)
    if (!(D.invalid_mask && D.invalid_mask[f])) valid_flats.push_back(f);
  const int64_t N = (int64_t)valid_flats.size();
  if (N == 0) return fail(BO_ERR_ARG, "no valid configuration");
  auto valid_of = [&](int64_t flat) -> int64_t {
    auto it = std::lower_bound(valid_flats.begin(), valid_flats.end(), flat);
    return (it != valid_flats.end() && *it == flat) ? (int64_t)(it - valid_flats.begin()) : -1;
  };
  uint64_t rng = D.seed;
  return initial_design(values, N, valid_of, count, D.init_mode, D.init_designs, rng, idx_out);
}
