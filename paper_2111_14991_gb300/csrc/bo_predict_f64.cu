// Prediction pass in FP64 on CUDA cores: the plain FP64 form of the hot path.
//
// Exhaustive prediction of every valid configuration (paper Sec. III-G): for a
// tile of BM candidates the Matern cross-covariance K*[BM x n] (Sec. III-B) is
// built in shared memory (never in HBM), then V = K* L^-T is formed one
// 64-column block at a time with register tiling, and reduced on the fly to
//   var = k(0) - sum_k V_ik^2   (clamped at 0),   mu = sum_k V_ik beta_k,
// which is the zero-mean GP posterior with beta = L^-1 y~.  Only entries
// j <= k of L^-1 are non-zero, so each column block stops at its diagonal,
// and inside it each 16-column group skips the slices above its own
// diagonal and the columns beyond n.
// Each CTA also writes the sum of the variances of its non-evaluated
// candidates; the acquisition adds those partial sums in block order
// (deterministic) for the exploration factor (Sec. III-F).
#include <algorithm>

#include "bo_internal.h"

namespace bo {

namespace {

constexpr int kThreads = 256;
constexpr int kBN = 64;   // output columns of V per pass
constexpr int kBK = 32;   // j per staged slice of L^-1

// e^-t for t >= 0 by a table-driven reduction after P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM Trans. Math. Softw. 15(2), 1989, in the form this kernel
// needs.  With N = round(-t 64 / ln 2) = 64 m + j (0 <= j < 64) and
// r = -t - N ln2/64 (|r| <= ln2/128; ln2/64 = L1 + L2, L1 with 36 significant
// bits so that N L1 is exact), e^-t = 2^m 2^(j/64) e^r with e^r = 1 + r + r^2/2
// + ... + r^5/120 (the dropped terms are below 4e-17) and 2^(j/64) from tab.
// N comes from the rounding of x + 1.5 2^52 (the integer sits in the low word),
// and 2^m is an add to the exponent field.  About 11 FP64 operations.  The
// Matern evaluation is the only FP64 work of the pass besides the contraction,
// and the FP64 pipe bounds the pass.  t > 700 gives 0 (e^-700 ~ 1e-304 lies far
// below every term of mu and sigma^2); NaN stays NaN.
__device__ __forceinline__ double exp_neg(double t, const double* tab) {
  const double x = -t * 0x1.71547652b82fep+6;           // -t 64 / ln 2
  const double sh = x + 0x1.8p52;
  const double N = sh - 0x1.8p52;
  const int ni = __double2loint(sh);
  const double r = fma(-N, 0x1.cf79abc9e3b3ap-46, fma(-N, 0x1.62e42fefa0000p-7, -t));
  double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  q = fma(q, r, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  const double p = fma(q, r * r, r);
  const double tj = tab[ni & 63];
  const double y = fma(tj, p, tj);                      // 2^(j/64) e^r, in [0.99, 2.02)
  const double e = __hiloint2double(__double2hiint(y) + (ni >> 6) * (1 << 20), __double2loint(y));
  return t <= 700.0 ? e : (t > 700.0 ? 0.0 : t);
}

// tab[j] = 2^(j/64), j < 64 (every block fills its own copy in shared memory).
__device__ __forceinline__ void fill_exp_tab(double* tab) {
  for (int j = threadIdx.x; j < 64; j += blockDim.x) tab[j] = exp2((double)j * (1.0 / 64.0));
}

__device__ __forceinline__ double matern64(double r, double nu, double c, const double* tab) {
  const double t = c * r;
  const double e = exp_neg(t, tab);
  return nu == 1.5 ? fma(t, e, e) : (1.0 + t + t * t * (1.0 / 3.0)) * e;
}

// acc[r][q] += K*[row r][j0 + jj] * L^-1[column q][j0 + jj] over the rows
// jj in [h, h + hn) of a staged slice, for the column groups q in [QLO, QHI)
// only (compile-time, so that no instruction is spent on the others).
template <int TM, int QLO, int QHI>
__device__ __forceinline__ void slice_fma(const double* Ks, const double* Ls, int ldk, int j0, int h, int hn,
                                          int tx, int ty, double (&acc)[TM][4]) {
  for (int jj = h; jj < h + hn; ++jj) {
    double a[TM], b[4];
#pragma unroll
    for (int r = 0; r < TM; ++r) a[r] = Ks[(ty + 16 * r) * ldk + j0 + jj];
#pragma unroll
    for (int q = QLO; q < QHI; ++q) b[q] = Ls[jj * (kBN + 1) + tx + 16 * q];
#pragma unroll
    for (int q = QLO; q < QHI; ++q)
#pragma unroll
      for (int r = 0; r < TM; ++r) acc[r][q] = fma(a[r], b[q], acc[r][q]);
  }
}

template <int TM>
__device__ __forceinline__ void slice_groups(int q_lo, int q_hi, const double* Ks, const double* Ls, int ldk,
                                             int j0, int h, int hn, int tx, int ty, double (&acc)[TM][4]) {
  switch (q_lo * 8 + q_hi) {
    case 0 * 8 + 4: slice_fma<TM, 0, 4>(Ks, Ls, ldk, j0, h, hn, tx, ty, acc); break;
    case 0 * 8 + 3: slice_fma<TM, 0, 3>(Ks, Ls, ldk, j0, h, hn, tx, ty, acc); break;
    case 0 * 8 + 2: slice_fma<TM, 0, 2>(Ks, Ls, ldk, j0, h, hn, tx, ty, acc); break;
    case 0 * 8 + 1: slice_fma<TM, 0, 1>(Ks, Ls, ldk, j0, h, hn, tx, ty, acc); break;
    case 1 * 8 + 4: slice_fma<TM, 1, 4>(Ks, Ls, ldk, j0, h, hn, tx, ty, acc); break;
    case 1 * 8 + 3: slice_fma<TM, 1, 3>(Ks, Ls, ldk, j0, h, hn, tx, ty, acc); break;
    case 1 * 8 + 2: slice_fma<TM, 1, 2>(Ks, Ls, ldk, j0, h, hn, tx, ty, acc); break;
    case 2 * 8 + 4: slice_fma<TM, 2, 4>(Ks, Ls, ldk, j0, h, hn, tx, ty, acc); break;
    case 2 * 8 + 3: slice_fma<TM, 2, 3>(Ks, Ls, ldk, j0, h, hn, tx, ty, acc); break;
    case 3 * 8 + 4: slice_fma<TM, 3, 4>(Ks, Ls, ldk, j0, h, hn, tx, ty, acc); break;
    default: break;   // q_lo >= q_hi: nothing in this half
  }
}

// TAB: the space keeps its per-parameter tables of squared value differences
// (small value lists): r^2 is then a sum of d table entries, addressed by the
// candidate's and the observation's value indices, instead of d differences
// and squares on the narrow FP64 pipe.
template <int BM, bool TAB>
__global__ void __launch_bounds__(kThreads, 1) predict_f64_kernel(DevView v, int n, int n_pad) {
  pdl_wait();                             // the observation update has completed (dependent launch)
  constexpr int TM = BM / 16;             // rows per thread
  extern __shared__ double smem[];
  const int d = v.d;
  const int ldk = n_pad + 1;
  double* Ks = smem;                      // [BM][ldk]
  double* Ls = Ks + BM * ldk;             // [kBK][kBN + 1]
  double* Bs = Ls + kBK * (kBN + 1);      // [n_pad]
  // coordinates (!TAB): Xs [d][n_pad], Cs [BM][d]; tables (TAB): Ts [sqd_total],
  // meta [2 d + 1] ints, then value indices Xc [d][n_pad] and Cc [BM][d] bytes
  double* Xs = Bs + n_pad;
  double* Cs = Xs + d * n_pad;
  double* Ts = Bs + n_pad;
  int* meta = reinterpret_cast<int*>(Ts + (TAB ? v.sqd_total : 0));
  uint8_t* Xc = reinterpret_cast<uint8_t*>(meta + 2 * d + 1);
  uint8_t* Cc = Xc + d * n_pad;
  __shared__ double red[kThreads / 32 + 1];
  __shared__ double exp_tab[64];

  const int tid = threadIdx.x;
  fill_exp_tab(exp_tab);
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const double c = sqrt(2.0 * v.nu) / v.lengthscale;

  if constexpr (TAB) {
    for (int e = tid; e < v.sqd_total; e += kThreads) Ts[e] = v.sqd[e];
    for (int e = tid; e < 2 * d + 1; e += kThreads) meta[e] = v.sqd_meta[e];
    for (int e = tid; e < d * n_pad; e += kThreads) {
      const int p = e / n_pad, j = e - p * n_pad;
      Xc[e] = j < n ? v.Xc[(size_t)j * d + p] : 0;
    }
    for (int e = tid; e < BM * d; e += kThreads) {
      const int i = e / d, p = e - i * d;
      Cc[e] = v.codes[(int64_t)p * v.N_pad + row0 + i];
    }
  } else {
    for (int e = tid; e < d * n_pad; e += kThreads) {
      const int p = e / n_pad, j = e - p * n_pad;
      Xs[e] = j < n ? v.X[(size_t)j * d + p] : 0.0;
    }
    for (int e = tid; e < BM * d; e += kThreads) {
      const int i = e / d, p = e - i * d;
      Cs[e] = v.vtab64[p * 256 + v.codes[(int64_t)p * v.N_pad + row0 + i]];
    }
  }
  for (int j = tid; j < n_pad; j += kThreads) Bs[j] = j < n ? v.beta[j] : 0.0;
  __syncthreads();

  // K*[i][j] = k(|x_i - X_j|); padded columns j >= n meet zero rows of L^-1.
  for (int e = tid; e < BM * n; e += kThreads) {
    const int i = e / n, j = e - i * n;
    double r2 = 0.0;
    if constexpr (TAB) {
      for (int p = 0; p < d; ++p)
        r2 += Ts[meta[p] + Cc[i * d + p] * meta[d + 1 + p] + Xc[p * n_pad + j]];
    } else {
      for (int p = 0; p < d; ++p) {
        const double diff = Cs[i * d + p] - Xs[p * n_pad + j];
        r2 = fma(diff, diff, r2);
      }
    }
    Ks[i * ldk + j] = matern64(sqrt(r2), v.nu, c, exp_tab);
  }
  for (int e = tid; e < BM * (n_pad - n); e += kThreads) {
    const int i = e / (n_pad - n), j = n + e % (n_pad - n);
    Ks[i * ldk + j] = 0.0;
  }
  __syncthreads();

  const int tx = tid & 15, ty = tid >> 4;
  double s2[TM], sm[TM];
#pragma unroll
  for (int r = 0; r < TM; ++r) s2[r] = sm[r] = 0.0;

  for (int kb = 0; kb < n; kb += kBN) {
    double acc[TM][4];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[r][q] = 0.0;
    const int jend = min(n, kb + kBN);      // L^-1[k][j] = 0 for j > k
    // column group q (columns kb + 16q .. kb + 16q + 15) holds real columns
    // only below n: groups from q_hi on are never touched
    const int q_hi = min(4, (n - kb + 15) / 16);
    for (int j0 = 0; j0 < jend; j0 += kBK) {
      __syncthreads();
      for (int e = tid; e < kBN * kBK; e += kThreads) {
        const int kk = e / kBK, jj = e - kk * kBK;
        const int k = kb + kk, j = j0 + jj;
        Ls[jj * (kBN + 1) + kk] = (k < n && j <= k) ? v.linv[(size_t)k * v.n_max + j] : 0.0;
      }
      __syncthreads();
      const int jn = min(kBK, jend - j0);
      // in 16-row halves of the slice: groups whose last column lies before
      // the half's first row j meet only zeros of L^-1 there (the triangle
      // inside the diagonal block); (q_lo, q_hi) is uniform across the CTA,
      // and the skipped products are exact zeros
      for (int h = 0; h < jn; h += 16) {
        const int j = j0 + h, q_lo = j > kb + 15 ? (j - kb) / 16 : 0;
        slice_groups<TM>(q_lo, q_hi, Ks, Ls, ldk, j0, h, min(16, jn - h), tx, ty, acc);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = kb + tx + 16 * q;
      const double bk = k < n_pad ? Bs[k] : 0.0;
#pragma unroll
      for (int r = 0; r < TM; ++r) {
        s2[r] = fma(acc[r][q], acc[r][q], s2[r]);
        sm[r] = fma(acc[r][q], bk, sm[r]);
      }
    }
  }

  // reduce over the 16 threads (tx) sharing a row: lanes differ in the low 4 bits
  double vsum = 0.0;
#pragma unroll
  for (int r = 0; r < TM; ++r) {
    for (int o = 8; o > 0; o >>= 1) {
      s2[r] += __shfl_xor_sync(0xffffffffu, s2[r], o);
      sm[r] += __shfl_xor_sync(0xffffffffu, sm[r], o);
    }
    const int64_t i = row0 + ty + 16 * r;
    if (tx == 0) {
      const double var = fmax(0.0, 1.0 - s2[r]);
      static_cast<double*>(v.mu)[i] = sm[r];
      static_cast<double*>(v.var)[i] = var;
      if (i < v.N && !((v.visited[i >> 5] >> (i & 31)) & 1u)) vsum += var;
    }
  }
  pdl_trigger();                           // the acquisition may be launched (it waits for completion)
  // block sum of variances in a fixed order; the acquisition adds the blocks' sums
  for (int o = 16; o > 0; o >>= 1) vsum += __shfl_xor_sync(0xffffffffu, vsum, o);
  if ((tid & 31) == 0) red[tid >> 5] = vsum;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    v.partial[blockIdx.x] = t;
  }
}

template <int BM, bool TAB>
size_t smem_bytes(int d, int n_pad, int sqd_total) {
  const size_t common = sizeof(double) * ((size_t)BM * (n_pad + 1) + kBK * (kBN + 1) + n_pad);
  if (!TAB) return common + sizeof(double) * ((size_t)d * n_pad + (size_t)BM * d);
  return common + sizeof(double) * (size_t)sqd_total + sizeof(int) * (2 * (size_t)d + 1) +
         (size_t)d * n_pad + (size_t)BM * d;
}

template <int BM, bool TAB>
int launch_bm(const DevView& v, int n, cudaStream_t s) {
  const int n_pad = ((n + kBK - 1) / kBK) * kBK;
  const size_t sm = smem_bytes<BM, TAB>(v.d, n_pad, v.sqd_total);
  static size_t configured[kMaxDevices] = {};
  if (!ensure_dynamic_smem((const void*)predict_f64_kernel<BM, TAB>, configured, sm)) return -1;
  const int grid = predict_f64_grid(v, n);
  if (grid > v.max_partials) return -1;
  return launch_ex(predict_f64_kernel<BM, TAB>, dim3(grid), dim3(kThreads), sm, s, pdl_enabled(), v, n, n_pad) ==
                 cudaSuccess
             ? 1
             : -1;
}

// Self-test of exp_neg: out[i] = exp_neg(t[i]), ref[i] = CUDA's exp(-t[i]).
__global__ void selftest_exp_kernel(const double* t, double* out, double* ref, int n) {
  __shared__ double tab[64];
  fill_exp_tab(tab);
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    out[i] = exp_neg(t[i], tab);
    ref[i] = exp(-t[i]);
  }
}

}  // namespace

int launch_selftest_exp(const double* t, double* out, double* ref, int n, cudaStream_t s) {
  if (n < 1) return -1;
  selftest_exp_kernel<<<std::min((n + 255) / 256, 1024), 256, 0, s>>>(t, out, ref, n);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

// Candidates per block: 64 while that still gives every multiprocessor a
// block, else 32 (a space of 2,560 candidates runs 80 blocks instead of 40 on
// the FP64 pipes); always 32 for n > 256, where 64 rows of K* no longer fit in
// shared memory.
int f64_rows_per_block(const DevView& v, int n) {
  if (n > 256) return 32;
  return v.N_pad / 64 >= (int64_t)v.num_sms ? 64 : 32;
}

int predict_f64_grid(const DevView& v, int n) { return (int)(v.N_pad / f64_rows_per_block(v, n)); }

int launch_predict_f64(const DevView& v, int n, int64_t /*n_unvisited*/, cudaStream_t s) {
  if (n < 1) return -1;
  const bool wide = f64_rows_per_block(v, n) == 64;
  if (v.sqd) return wide ? launch_bm<64, true>(v, n, s) : launch_bm<32, true>(v, n, s);
  return wide ? launch_bm<64, false>(v, n, s) : launch_bm<32, false>(v, n, s);
}

}  // namespace bo
