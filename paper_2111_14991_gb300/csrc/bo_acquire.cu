// Acquisition and masked top-k over the predicted candidates.
//
// Reads the posterior mean / variance of every candidate and the evaluated
// bits, computes the exploration factor lambda from the pass's mean variance
// (contextual variance, paper Sec. III-F, or a constant), scores every valid,
// non-evaluated configuration with the active acquisition functions
// (minimization variants of EI, PI and LCB, Sec. III-C; larger is better) and
// keeps the k best (score, index) per function: per thread, then merged
// across the warp with shuffles, across the block in shared memory, and
// across blocks by the last block to finish.  Ties go to the lower index.
#include <algorithm>
#include <cfloat>
#include <cstdlib>
#include <climits>

#include "bo_acquire_dev.cuh"
#include "bo_internal.h"

namespace bo {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxK = 3;

template <typename T>
struct Lowest;
template <>
struct Lowest<double> {
  __device__ static double v() { return -DBL_MAX; }
};

template <typename T>
struct Top {
  T s[kMaxK];
  long long i[kMaxK];
};

template <typename T>
__device__ __forceinline__ bool better(T s1, long long i1, T s2, long long i2) {
  return s1 > s2 || (s1 == s2 && i1 < i2);
}

template <typename T>
__device__ __forceinline__ void top_init(Top<T>& t) {
#pragma unroll
  for (int r = 0; r < kMaxK; ++r) { t.s[r] = Lowest<T>::v(); t.i[r] = LLONG_MAX; }
}

template <typename T>
__device__ __forceinline__ void top_insert(Top<T>& t, T s, long long i) {
  if (!better(s, i, t.s[kMaxK - 1], t.i[kMaxK - 1])) return;
  if (better(s, i, t.s[0], t.i[0])) {
    t.s[2] = t.s[1]; t.i[2] = t.i[1]; t.s[1] = t.s[0]; t.i[1] = t.i[0]; t.s[0] = s; t.i[0] = i;
  } else if (better(s, i, t.s[1], t.i[1])) {
    t.s[2] = t.s[1]; t.i[2] = t.i[1]; t.s[1] = s; t.i[1] = i;
  } else {
    t.s[2] = s; t.i[2] = i;
  }
}

template <typename T>
__device__ __forceinline__ void top_merge(Top<T>& t, const Top<T>& o) {
#pragma unroll
  for (int r = 0; r < kMaxK; ++r) top_insert(t, o.s[r], o.i[r]);
}

// butterfly merge of each lane's lists across the warp
template <typename T>
__device__ __forceinline__ void warp_merge(Top<T>& t) {
  for (int o = 16; o > 0; o >>= 1) {
    Top<T> other;
#pragma unroll
    for (int r = 0; r < kMaxK; ++r) {
      other.s[r] = __shfl_xor_sync(0xffffffffu, t.s[r], o);
      other.i[r] = __shfl_xor_sync(0xffffffffu, t.i[r], o);
    }
    top_merge(t, other);
  }
}

template <typename T>
struct Math;
template <>
struct Math<double> {
  __device__ static double erfc_(double x) { return erfc(x); }
  __device__ static double exp_(double x) { return exp(x); }
  __device__ static double sqrt_(double x) { return sqrt(x); }
};

// the three scores at posterior (mu, sigma), larger is better: EI and PI share
// z and Phi (evaluated only when need_phi: EI or PI is active), LCB is
// -(mu - lam sigma)
template <typename T>
__device__ __forceinline__ void scores3(T mu, T sigma, T fplus, T lam, bool need_phi, T& ei, T& pi, T& lcb) {
  const T delta = fplus - mu - lam;
  lcb = lam * sigma - mu;
  if (!need_phi) {
    ei = pi = T(0);
    return;
  }
  if (!(sigma > T(0))) {
    ei = delta > T(0) ? delta : T(0);
    pi = delta > T(0) ? T(1) : T(0);
    return;
  }
  const T z = delta / sigma;
  const T Phi = T(0.5) * Math<T>::erfc_(-z * T(0.70710678118654752440));
  const T phi = Math<T>::exp_(T(-0.5) * z * z) * T(0.39894228040143267794);
  pi = Phi;
  ei = delta * Phi + sigma * phi;
}

// ---- FP32 posteriors: (score, index) packed into one 64-bit key ----------
// (bo_acquire_dev.cuh: the key order is the selection order of better()).
// acquire_body_f32: the scores in FP32 (EI and PI share z and Phi), kept as
// packed keys; block partials are keys (in TopEntry::idx), merged by the last
// block.
__device__ __forceinline__ void acquire_body_f32(const AcqDev& v, const PassArgs& a, const int block,
                                                 const int nblocks, const double sum_var) {
  __shared__ unsigned long long s_key[kThreads / 32][3][kMaxK];
  __shared__ bool s_last;
  __shared__ double s_lam[3];   // FP64 scalars formed once per block and broadcast
  const float* mu = static_cast<const float*>(v.mu);
  const float* var = static_cast<const float*>(v.var);
  if (threadIdx.x == 0) acq::pass_lambda(a, sum_var, a.first_pass ? 0.0 : *v.var_s, &s_lam[0], &s_lam[1], &s_lam[2]);
  __syncthreads();
  const double mean_var = s_lam[0], var_s = s_lam[1], lam = s_lam[2];
  const float lamT = (float)lam, fpT = (float)a.fplus_t;
  const int n_af = a.n_af;
  const int af0 = a.af[0], af1 = a.af[1], af2 = a.af[2];

  unsigned long long top[3][kMaxK];
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int r = 0; r < kMaxK; ++r) top[q][r] = 0ull;
  const int64_t stride = (int64_t)nblocks * kThreads;
  for (int64_t i = (int64_t)block * kThreads + threadIdx.x; i < v.N; i += stride) {
    if ((v.visited[i >> 5] >> (i & 31)) & 1u) continue;
    acq::score_f32(mu[i], var[i], fpT, lamT, n_af, af0, af1, af2, (long long)i, top);
  }
  acq::block_top3(top, &s_key[0][0][0], kThreads / 32);
  if (threadIdx.x < 32 && threadIdx.x < 3 * kMaxK) {
    const int q = threadIdx.x / kMaxK, r = threadIdx.x % kMaxK;
    unsigned long long k = 0ull;
#pragma unroll
    for (int qq = 0; qq < 3; ++qq)
#pragma unroll
      for (int rr = 0; rr < kMaxK; ++rr)
        if (qq == q && rr == r) k = top[qq][rr];
    TopEntry* out = v.partial + ((size_t)block * 3 + q) * kMaxK + r;
    out->score = (double)acq::key_score(k);
    out->idx = (long long)k;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int done = atomicAdd(v.counter, 1u);
    s_last = (done == (unsigned)nblocks - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last block: every thread gathers the keys of a strided slice of the block
  // partials (read past L1), then the block takes the three largest per AF;
  // the key order is total, so the result does not depend on the merge order
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int r = 0; r < kMaxK; ++r) top[q][r] = 0ull;
  for (int b = threadIdx.x; b < nblocks; b += kThreads)
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int r = 0; r < kMaxK; ++r)
        acq::key_insert(top[q], (unsigned long long)__ldcg(&v.partial[((size_t)b * 3 + q) * kMaxK + r].idx));
  acq::block_top3(top, &s_key[0][0][0], kThreads / 32);
  if (threadIdx.x < 32)
    acq::write_result_f32(v.result, top, a, mu, var, v.status_in ? *v.status_in : BO_OK, sum_var, mean_var, lam,
                          var_s);
  if (threadIdx.x == 0) {
    if (a.first_pass) *v.var_s = mean_var;
    *v.counter = 0;
  }
}

// One block's share of the acquisition pass over v: blocks [0, nblocks) of
// the pass stride over the candidates; the last one to finish merges.
template <typename T>
__device__ __forceinline__ void acquire_body(const AcqDev& v, const PassArgs& a, const int block, const int nblocks,
                                             const double sum_var) {
  static_assert(kMaxK == 3, "top_insert is written for three entries");
  __shared__ Top<T> s_top[kThreads / 32][3];
  __shared__ bool s_last;
  const T* mu = static_cast<const T*>(v.mu);
  const T* var = static_cast<const T*>(v.var);

  // lambda from the pass's mean variance (every block computes the same value,
  // one thread per block: FP64 scalars are broadcast, not repeated per thread)
  __shared__ double s_lam[3];
  if (threadIdx.x == 0) acq::pass_lambda(a, sum_var, a.first_pass ? 0.0 : *v.var_s, &s_lam[0], &s_lam[1], &s_lam[2]);
  __syncthreads();
  const double mean_var = s_lam[0], var_s = s_lam[1], lam = s_lam[2];
  const T lamT = (T)lam, fpT = (T)a.fplus_t;

  bool need_phi = false;
  for (int q = 0; q < a.n_af && q < 3; ++q) need_phi |= a.af[q] != kLCB;
  Top<T> top[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) top_init(top[q]);
  const int64_t stride = (int64_t)nblocks * kThreads;
  const int64_t first = v.spread ? block + (int64_t)nblocks * threadIdx.x : (int64_t)block * kThreads + threadIdx.x;
  for (int64_t i = first; i < v.N; i += stride) {
    if ((v.visited[i >> 5] >> (i & 31)) & 1u) continue;
    const T m = mu[i];
    const T vv = var[i];
    const T sg = Math<T>::sqrt_(vv > T(0) ? vv : T(0));
    T ei, pi, lcb;
    scores3<T>(m, sg, fpT, lamT, need_phi, ei, pi, lcb);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (q < a.n_af) {
        const int af = a.af[q];
        T sc = af == kEI ? ei : af == kPI ? pi : lcb;
        if (!(sc == sc)) sc = Lowest<T>::v() / T(2);   // NaN never wins
        top_insert(top[q], sc, (long long)i);
      }
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 3; ++q) warp_merge(top[q]);
  if (lane == 0)
    for (int q = 0; q < 3; ++q) s_top[warp][q] = top[q];
  __syncthreads();
  if (threadIdx.x < 3) {
    const int q = threadIdx.x;
    Top<T> t = s_top[0][q];
    for (int w = 1; w < kThreads / 32; ++w) top_merge(t, s_top[w][q]);
    TopEntry* out = v.partial + ((size_t)block * 3 + q) * kMaxK;
    for (int r = 0; r < kMaxK; ++r) { out[r].score = (double)t.s[r]; out[r].idx = t.i[r]; }
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int done = atomicAdd(v.counter, 1u);
    s_last = (done == (unsigned)nblocks - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last block: every thread merges a strided slice of the block partials, then
  // warp and block merges as above (the (score, index) order is total, so the
  // result does not depend on the merge order)
  Top<T> fin[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) top_init(fin[q]);
  for (int b = threadIdx.x; b < nblocks; b += kThreads)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const volatile TopEntry* in = v.partial + ((size_t)b * 3 + q) * kMaxK;
#pragma unroll
      for (int r = 0; r < kMaxK; ++r) top_insert(fin[q], (T)in[r].score, (long long)in[r].idx);
    }
#pragma unroll
  for (int q = 0; q < 3; ++q) warp_merge(fin[q]);
  __syncthreads();
  if (lane == 0)
    for (int q = 0; q < 3; ++q) s_top[warp][q] = fin[q];
  __syncthreads();
  if (threadIdx.x < 3) {
    const int q = threadIdx.x;
    Top<T> t = s_top[0][q];
    for (int w = 1; w < kThreads / 32; ++w) top_merge(t, s_top[w][q]);
    bo_pass_result* res = v.result;
    for (int r = 0; r < 3; ++r) {
      const bool ok = q < a.n_af && r < a.k && t.i[r] != LLONG_MAX;
      res->top_idx[q][r] = ok ? t.i[r] : -1;
      res->top_score[q][r] = ok ? (double)t.s[r] : 0.0;
      res->top_mu[q][r] = ok ? (double)mu[t.i[r]] : 0.0;
      const double vr = ok ? (double)var[t.i[r]] : 0.0;
      res->top_sigma[q][r] = ok ? sqrt(vr > 0.0 ? vr : 0.0) : 0.0;
    }
  }
  if (threadIdx.x == 0) {
    bo_pass_result* res = v.result;
    res->status = v.status_in ? *v.status_in : BO_OK;
    if (res->status == BO_OK && !(mean_var == mean_var)) res->status = BO_ERR_NUMERIC;
    res->n_fit = a.n;
    res->n_scored = a.n_unvisited;
    res->sum_var = sum_var;
    res->mean_var = mean_var;
    res->lambda = lam;
    res->mean_var_s = var_s;
    if (a.first_pass) *v.var_s = mean_var;
    *v.counter = 0;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) acquire_kernel(AcqDev v, PassArgs a) {
  __shared__ double red[kThreads / 32 + 1];
  pdl_wait();                 // the prediction pass has completed (dependent launch)
  // the variance sum: the prediction CTAs' sums added in CTA order (the same
  // value in every block), or a given total
  const double sum_var = v.var_parts ? block_sum_partials(v.var_parts, v.n_var_parts, red) : *v.sum_var;
  if constexpr (sizeof(T) == 4)
    acquire_body_f32(v, a, blockIdx.x, gridDim.x, sum_var);
  else
    acquire_body<T>(v, a, blockIdx.x, gridDim.x, sum_var);
}

// Many spaces in one launch: block b serves item block_item[b] as its
// block_local[b]-th block; the item's variance sum is the sum, in segment
// order, of the epilogue parts of its tensor-core segments.
template <typename T>
__global__ void __launch_bounds__(kThreads) acquire_batch_kernel(const AcqItem* items, const int* block_item,
                                                                 const int* block_local, const double* seg_part) {
  const AcqItem& it = items[block_item[blockIdx.x]];
  __shared__ double s_sum;        // formed once per block (FP64 is narrow on this GPU) and broadcast
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int g = it.seg0; g < it.seg1; ++g)
      for (int e = 0; e < 4; ++e) t += seg_part[(size_t)g * 4 + e];
    s_sum = t;
  }
  __syncthreads();
  const double sum_var = s_sum;
  if constexpr (sizeof(T) == 4)
    acquire_body_f32(it.dev, it.args, block_local[blockIdx.x], it.nblocks, sum_var);
  else
    acquire_body<T>(it.dev, it.args, block_local[blockIdx.x], it.nblocks, sum_var);
}

}  // namespace

bool pdl_enabled() {
  static const bool on = getenv("BO_NO_PDL") == nullptr;
  return on;
}

int acquire_grid(int64_t n_cand, int max_blocks, int per_thread) {
  const int64_t want = (n_cand + (int64_t)kThreads * per_thread - 1) / ((int64_t)kThreads * per_thread);
  return (int)(want < max_blocks ? (want < 1 ? 1 : want) : max_blocks);
}

int launch_acquire(const AcqDev& v, const PassArgs& a, bool f64, cudaStream_t s) {
  int grid = acquire_grid(v.N, v.max_blocks, 2);
  AcqDev w = v;
  if (f64 && v.min_blocks > grid) {
    // few candidates for the narrow FP64 pipes: one block per multiprocessor
    // (at least 16 candidates each), candidates dealt round-robin over them
    const int64_t want = std::max<int64_t>((v.N + 15) / 16, grid);
    grid = (int)std::min<int64_t>(std::min<int64_t>(v.max_blocks, v.min_blocks), want);
    w.spread = 1;
  }
  const cudaError_t e = f64 ? launch_ex(acquire_kernel<double>, dim3(grid), dim3(kThreads), 0, s, pdl_enabled(), w, a)
                            : launch_ex(acquire_kernel<float>, dim3(grid), dim3(kThreads), 0, s, pdl_enabled(), w, a);
  return e == cudaSuccess ? 1 : -1;
}

int launch_acquire_batch(const AcqItem* items, const int* block_item, const int* block_local,
                         const double* seg_part, int total_blocks, bool f64, cudaStream_t s) {
  if (f64)
    acquire_batch_kernel<double><<<total_blocks, kThreads, 0, s>>>(items, block_item, block_local, seg_part);
  else
    acquire_batch_kernel<float><<<total_blocks, kThreads, 0, s>>>(items, block_item, block_local, seg_part);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_acquire(const DevView& v, const PassArgs& a, cudaStream_t s) {
  AcqDev ad;
  ad.mu = v.mu;
  ad.var = v.var;
  ad.visited = v.visited;
  ad.N = v.N;
  ad.sum_var = nullptr;
  ad.var_parts = v.partial;
  ad.n_var_parts = v.precision == BO_PREC_FP64 ? predict_f64_grid(v, a.n) : predict_tc_grid(v);
  ad.var_s = &v.stats->var_s;
  ad.status_in = &v.stats->status;
  ad.partial = v.acq_partial;
  ad.counter = &v.stats->k2_done;
  ad.max_blocks = v.max_acq_blocks;
  ad.min_blocks = v.num_sms;
  ad.result = v.results + a.result_slot;
  return launch_acquire(ad, a, v.precision == BO_PREC_FP64, s);
}

}  // namespace bo
