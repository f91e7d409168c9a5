// Device pieces of the acquisition pass shared by the acquisition kernels
// (bo_acquire.cu) and the acquisition tail of the tensor-core prediction pass
// (bo_predict_tc.cu): the exploration factor, the FP32 scores of one candidate
// and the packed (score, index) keys of the masked top-3 (paper Sec. III-C,
// III-F).  Both callers use these functions, so the two forms of a pass score
// with the same arithmetic and select with the same order.
#pragma once

#include <cfloat>

#include "bo_internal.h"

namespace bo {
namespace acq {

constexpr int kTop = 3;   // entries kept per acquisition function

// lambda of a pass from its variance sum: contextual variance (Sec. III-F),
// lambda = (mean_var / (mu_s / f+)) / mean_var_s, with the baseline taken on
// the first pass, or the constant.
__device__ __forceinline__ void pass_lambda(const PassArgs& a, double sum_var, double var_s_stored,
                                            double* mean_var, double* var_s, double* lam) {
  *mean_var = a.n_unvisited > 0 ? sum_var / (double)a.n_unvisited : 0.0;
  *var_s = a.first_pass ? *mean_var : var_s_stored;
  *lam = a.lambda_const;
  if (a.explore == BO_EXPLORE_CV) *lam = *var_s > 0.0 ? (*mean_var / (a.mu_s_raw / a.fplus_raw)) / *var_s : 0.0;
}

// (score, index) as one 64-bit key: the high word maps the float score onto
// unsigned integers in the same order (negative values bit-inverted,
// positive ones with the sign bit set; -0 is first made +0), the low word
// holds 2^32 - 1 - index, so a larger key is a higher score, then a lower
// index.  Key 0 is "no candidate" (it would need a NaN score, which never
// enters).  Indices must stay below 2^32 - 1.
__device__ __forceinline__ unsigned long long pack_key(float s, long long i) {
  uint32_t u = __float_as_uint(s + 0.0f);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ((unsigned long long)u << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)i);
}
__device__ __forceinline__ float key_score(unsigned long long k) {
  const uint32_t u = (uint32_t)(k >> 32);
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}
__device__ __forceinline__ long long key_idx(unsigned long long k) {
  return (long long)(0xFFFFFFFFu - (uint32_t)k);
}

// keep the three largest keys, t[0] >= t[1] >= t[2] (real keys are distinct)
__device__ __forceinline__ void key_insert(unsigned long long (&t)[kTop], unsigned long long k) {
  if (k <= t[2]) return;
  if (k > t[0]) {
    t[2] = t[1]; t[1] = t[0]; t[0] = k;
  } else if (k > t[1]) {
    t[2] = t[1]; t[1] = k;
  } else {
    t[2] = k;
  }
}

// The largest key of the warp, in every lane: the hardware warp maximum
// (redux.sync) of the high words, then of the low words of the lanes that
// hold that high word.
__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long k) {
  const uint32_t hi = (uint32_t)(k >> 32), lo = (uint32_t)k;
  const uint32_t mh = __reduce_max_sync(0xffffffffu, hi);
  const uint32_t ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
  return ((unsigned long long)mh << 32) | ml;
}

// The three largest keys of the lanes' sorted lists, returned in every lane:
// three rounds of a warp maximum, the lane holding it popping its head.
__device__ __forceinline__ void warp_top3(unsigned long long (&t)[kTop]) {
  unsigned long long out[kTop];
#pragma unroll
  for (int r = 0; r < kTop; ++r) {
    const unsigned long long m = warp_max_key(t[0]);
    out[r] = m;
    if (m != 0ull && t[0] == m) { t[0] = t[1]; t[1] = t[2]; t[2] = 0ull; }
  }
#pragma unroll
  for (int r = 0; r < kTop; ++r) t[r] = out[r];
}

// Block-wide top-3 per AF for a block of `warps` warps (at most 32): each
// warp's three keys through shared memory s_key[warps][3][kTop], then warp 0
// takes the three largest (lane w holding warp w's sorted list).  Every
// thread calls it; the result is valid in warp 0.
__device__ __forceinline__ void block_top3(unsigned long long (&t)[3][kTop], unsigned long long* s_key, int warps) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 3; ++q) warp_top3(t[q]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int r = 0; r < kTop; ++r) s_key[(warp * 3 + q) * kTop + r] = t[q][r];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
#pragma unroll
      for (int r = 0; r < kTop; ++r) t[q][r] = lane < warps ? s_key[(lane * 3 + q) * kTop + r] : 0ull;
      warp_top3(t[q]);
    }
  }
}

// The scores of one candidate from its FP32 posterior (mu, var), larger is
// better: EI and PI (minimization variants, sharing z and Phi) and -LCB;
// each active AF's score enters its top-3 as a key.  NaN never wins.
__device__ __forceinline__ void score_f32(float m, float vv, float fpT, float lamT, int n_af, int af0, int af1,
                                          int af2, long long i, unsigned long long (&top)[3][kTop]) {
  const float sg = sqrtf(vv > 0.0f ? vv : 0.0f);
  const float delta = fpT - m - lamT;
  const float lcb = lamT * sg - m;
  float ei, pi;
  if (!(sg > 0.0f)) {
    ei = delta > 0.0f ? delta : 0.0f;
    pi = delta > 0.0f ? 1.0f : 0.0f;
  } else {
    const float z = delta / sg;
    const float Phi = 0.5f * erfcf(-z * 0.70710678118654752440f);
    const float phi = expf(-0.5f * z * z) * 0.39894228040143267794f;
    pi = Phi;
    ei = delta * Phi + sg * phi;
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (q < n_af) {
      const int af = q == 0 ? af0 : q == 1 ? af1 : af2;
      float x = af == kEI ? ei : af == kPI ? pi : lcb;
      if (!(x == x)) x = -FLT_MAX / 2.0f;
      key_insert(top[q], pack_key(x, i));
    }
  }
}

// Pass result of the three lists t (as warp 0 holds them after block_top3),
// written by lanes 0..2 (one AF each) and lane 0 (the scalars).
__device__ __forceinline__ void write_result_f32(bo_pass_result* res, const unsigned long long (&t)[3][kTop],
                                                 const PassArgs& a, const float* mu, const float* var,
                                                 int32_t status, double sum_var, double mean_var, double lam,
                                                 double var_s) {
  const int lane = threadIdx.x & 31;
  if (lane < 3) {
    const int q = lane;
    unsigned long long tt[kTop];
#pragma unroll
    for (int r = 0; r < kTop; ++r) tt[r] = q == 0 ? t[0][r] : q == 1 ? t[1][r] : t[2][r];
    for (int r = 0; r < kTop; ++r) {
      const bool ok = q < a.n_af && r < a.k && tt[r] != 0ull;
      const long long i = ok ? key_idx(tt[r]) : 0;
      res->top_idx[q][r] = ok ? i : -1;
      res->top_score[q][r] = ok ? (double)key_score(tt[r]) : 0.0;
      res->top_mu[q][r] = ok ? (double)mu[i] : 0.0;
      const float vr = ok ? var[i] : 0.0f;
      res->top_sigma[q][r] = ok ? (double)sqrtf(vr > 0.0f ? vr : 0.0f) : 0.0;   // as the scores' sigma
    }
  }
  if (lane == 0) {
    res->status = status;
    if (res->status == BO_OK && !(mean_var == mean_var)) res->status = BO_ERR_NUMERIC;
    res->n_fit = a.n;
    res->n_scored = a.n_unvisited;
    res->sum_var = sum_var;
    res->mean_var = mean_var;
    res->lambda = lam;
    res->mean_var_s = var_s;
  }
}

}  // namespace acq
}  // namespace bo
