// Observation update of the GP surrogate (FP64), one valid observation at a time.
//
// With a fixed lengthscale (paper Sec. III-B) the kernel matrix of the
// observations only grows by one row and column per observation, so the
// Cholesky factor grows by one row and so does its inverse:
//   K_new = [[K, k], [k^T, k(0) + jitter]],  l = L^-1 k,  d = sqrt(k(0) + jitter - l.l)
//   L_new^-1 = [[L^-1, 0], [-(L^-T l)^T / d, 1 / d]].
// Rows of L^-1 never change once written.  beta = L^-1 y~ is recomputed in
// full because the standardization of y shifts with every observation.
// The reduced-precision contraction gets a per-row scaled, split copy of each
// new row (written once), see lsplit_offset().
#include <algorithm>

#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "bo_internal.h"

namespace bo {

__device__ __forceinline__ double matern64(double r, double nu, double c) {
  // c = sqrt(2 nu) / l; nu = 3/2: (1 + t) e^-t ; nu = 5/2: (1 + t + t^2/3) e^-t
  double t = c * r;
  double e = exp(-t);
  return nu == 1.5 ? (1.0 + t) * e : (1.0 + t + t * t * (1.0 / 3.0)) * e;
}

__device__ __forceinline__ double coord64(const DevView& v, int64_t idx, int p) {
  return v.vtab64[p * 256 + v.codes[(int64_t)p * v.N_pad + idx]];
}

// Byte offset of element (row k, column j) of L^-1 in the chunked copy.
// Chunk c holds columns [c*CW, (c+1)*CW) of rows k >= c*CW, in the K-major
// no-swizzle core-matrix layout the tensor core reads: 8-row x 16-byte core
// matrices, the CW/ (16/eb) core matrices of one 8-row group side by side
// (128 B apart), consecutive 8-row groups kChunkBytes*8 B apart.
__host__ __device__ __forceinline__ size_t lsplit_offset(int n_max, int eb, int k, int j) {
  const int cw = kChunkBytes / eb;
  const int c = j / cw;
  // sum over c' < c of (n_max - c' cw) * kChunkBytes
  const size_t base = (size_t)kChunkBytes * ((size_t)c * n_max - (size_t)cw * c * (c - 1) / 2);
  const int jj = j - c * cw;
  const int g = (k - c * cw) >> 3;
  return base + (size_t)g * (kChunkBytes * 8) + (size_t)((jj * eb) >> 4) * 128 +
         (size_t)(k & 7) * 16 + (size_t)((jj * eb) & 15);
}

size_t lsplit_bytes(int n_max, int precision) {
  if (precision == BO_PREC_FP64) return 0;
  const int eb = split_elem_bytes(precision);
  const int cw = kChunkBytes / eb;
  const int nc = n_max / cw;
  return (size_t)kChunkBytes * ((size_t)nc * n_max - (size_t)cw * nc * (nc - 1) / 2);
}

// --- K3a: X[n] = x(idx), y[n] = y, visited bit, k_j = k(|x - X_j|) --------------
__device__ __forceinline__ void obs_k_body(const DevView& v, int n, long long idx, double y_raw, int block) {
  const int j = block * blockDim.x + threadIdx.x;
  const double c = sqrt(2.0 * v.nu) / v.lengthscale;
  if (block == 0 && threadIdx.x < v.d) {
    const double x = coord64(v, idx, threadIdx.x);
    v.X[(size_t)n * v.d + threadIdx.x] = x;
    v.Xc[(size_t)n * v.d + threadIdx.x] = v.codes[(int64_t)threadIdx.x * v.N_pad + idx];
    if (v.xq) v.xq[xq_index(v.ds, n, threadIdx.x)] = (float)(x * (1.4426950408889634 * c));
  }
  if (block == 0 && threadIdx.x == 0) {
    v.y[n] = y_raw;
    atomicOr(&v.visited[idx >> 5], 1u << (idx & 31));
  }
  if (j < n) {
    double r2 = 0.0;
    if (v.sqd) {   // the prediction pass's arithmetic: a sum of tabulated squared differences
      for (int p = 0; p < v.d; ++p) {
        const int m = v.sqd_meta[v.d + 1 + p];
        const int a = v.codes[(int64_t)p * v.N_pad + idx], b = v.Xc[(size_t)j * v.d + p];
        r2 += v.sqd[v.sqd_meta[p] + a * m + b];
      }
    } else {
      for (int p = 0; p < v.d; ++p) {
        const double diff = coord64(v, idx, p) - v.X[(size_t)j * v.d + p];
        r2 = fma(diff, diff, r2);
      }
    }
    v.kvec[j] = matern64(sqrt(r2), v.nu, c);
  }
}

__global__ void obs_k_kernel(DevView v, int n, long long idx, double y_raw) {
  obs_k_body(v, n, idx, y_raw, blockIdx.x);
}

__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// --- K3b: l = L^-1 k (warp per row) -------------------------------------------
__device__ __forceinline__ void obs_l_body(const DevView& v, int n, int block) {
  const int warp = (block * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* row = v.linv + (size_t)warp * v.n_max;
  double s = 0.0;
#pragma unroll 4
  for (int j = lane; j <= warp; j += 32) s = fma(row[j], v.kvec[j], s);
  s = warp_sum(s);
  if (lane == 0) v.lvec[warp] = s;
}

__global__ void obs_l_kernel(DevView v, int n) { obs_l_body(v, n, blockIdx.x); }

// --- K3c: partial w = L^-T l over row segments of 64 ---------------------------
// Block (column block of 32, row segment of 64): lane = column, warp w sums
// rows seg*64 + 8w .. +8 with all eight loads in flight; L^-1[i][j] = 0 for j > i.
__device__ __forceinline__ void obs_w_body(const DevView& v, int n, int bx, int by) {
  __shared__ double part[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = bx * 32 + lane;
  const int i0 = by * 64 + w * 8;
  double s = 0.0;
  if (j < n) {
    double a[8], b[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = i0 + r;
      const bool in = i < n && i >= j;
      a[r] = in ? v.linv[(size_t)i * v.n_max + j] : 0.0;
      b[r] = in ? v.lvec[i] : 0.0;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) s = fma(a[r], b[r], s);
  }
  part[w][lane] = s;
  __syncthreads();
  if (w == 0 && j < n) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += part[q][lane];
    v.wvec[(size_t)by * v.n_max + j] = t;
  }
}

__global__ void obs_w_kernel(DevView v, int n) { obs_w_body(v, n, blockIdx.x, blockIdx.y); }

// --- K3d: pivot, new row n of L^-1 and its split copy (one block) --------------
__device__ __forceinline__ void obs_finish_body(const DevView& v, int n) {
  __shared__ double red[32];
  __shared__ double s_dinv;
  __shared__ float s_scale;
  const int tid = threadIdx.x;
  double ll = 0.0;
  for (int i = tid; i < n; i += blockDim.x) ll = fma(v.lvec[i], v.lvec[i], ll);
  ll = warp_sum(ll);
  if ((tid & 31) == 0) red[tid >> 5] = ll;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    const double d2 = 1.0 + v.jitter - t;
    s_dinv = (d2 > 0.0 && isfinite(d2)) ? 1.0 / sqrt(d2) : 0.0;
    if (s_dinv == 0.0) v.stats->status = BO_ERR_NUMERIC;
  }
  __syncthreads();
  const double dinv = s_dinv;
  if (dinv == 0.0) return;
  const int nseg = (n + 63) / 64;
  double* row = v.linv + (size_t)n * v.n_max;
  double amax = 0.0;
  for (int j = tid; j <= n; j += blockDim.x) {
    double val;
    if (j < n) {
      double w = 0.0;
#pragma unroll
      for (int s = 0; s < 8; ++s)
        if (s < nseg) w += v.wvec[(size_t)s * v.n_max + j];
      val = -w * dinv;
    } else {
      val = dinv;
    }
    row[j] = val;
    amax = fmax(amax, fabs(val));
  }
  if (v.precision == BO_PREC_FP64) return;
  // per-row power-of-two scale s with max |row| * s in [2^13, 2^14)
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = amax;
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    int e;
    frexp(m, &e);                       // m in [2^(e-1), 2^e)
    s_scale = ldexpf(1.0f, 14 - e);
    if (v.xq) v.xq[xq_index(v.ds, n, v.ds)] = 1.0f / (s_scale * s_scale);
  }
  __syncthreads();
  const float sc = s_scale;
  const int eb = split_elem_bytes(v.precision);
  for (int j = tid; j <= n; j += blockDim.x) {
    const float x = (float)row[j] * sc;
    const size_t off = lsplit_offset(v.n_max, eb, n, j);
    if (v.precision == BO_PREC_FP16X3) {
      const __half h = __float2half_rn(x);
      const __half l = __float2half_rn(x - __half2float(h));
      *reinterpret_cast<__half*>(v.lsplit_hi + off) = h;
      *reinterpret_cast<__half*>(v.lsplit_lo + off) = l;
    } else if (v.precision == BO_PREC_BF16X3) {
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
      *reinterpret_cast<__nv_bfloat16*>(v.lsplit_hi + off) = h;
      *reinterpret_cast<__nv_bfloat16*>(v.lsplit_lo + off) = l;
    } else {  // TF32: round to nearest (ties away) to 10 explicit mantissa bits
      uint32_t u;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
      *reinterpret_cast<uint32_t*>(v.lsplit_hi + off) = u;
      if (v.precision == BO_PREC_TF32X3) {   // lo = the rounding residual, itself rounded to TF32
        uint32_t w;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(w) : "f"(x - __uint_as_float(u)));
        *reinterpret_cast<uint32_t*>(v.lsplit_lo + off) = w;
      }
    }
  }
}

__global__ void obs_finish_kernel(DevView v, int n) { obs_finish_body(v, n); }


// --- K3e: beta = L^-1 y~ for rows 0..n ------------------------------------------
__device__ __forceinline__ void obs_beta_body(const DevView& v, int rows, double y_mean, double inv_std,
                                              int block) {
  const int warp = (block * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= rows) return;
  const double* row = v.linv + (size_t)warp * v.n_max;
  double s = 0.0;
  for (int j = lane; j <= warp; j += 32) s = fma(row[j], (v.y[j] - y_mean) * inv_std, s);
  s = warp_sum(s);
  if (lane == 0) v.beta[warp] = s;
}

// --- K3f (tensor-core forms): alpha = L^-T beta, so that mu = k* . alpha -------
// (warp per column j: lanes stride down the rows i >= j of L^-1, fixed-order
// reduction).  The prediction pass evaluates mu from K* and alpha directly:
// the FP32 error of mu is then bounded by sum_j |alpha_j k*_j| times the K*
// and accumulation rounding, and does not depend on the split contraction.
__device__ __forceinline__ void obs_alpha_body(const DevView& v, int rows, int block) {
  if (v.precision == BO_PREC_FP64) return;
  const int col = (block * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (col >= rows) return;
  double s = 0.0;
  for (int i = col + lane; i < rows; i += 32) s = fma(v.linv[(size_t)i * v.n_max + col], v.beta[i], s);
  s = warp_sum(s);
  if (lane == 0) v.xq[xq_index(v.ds, col, v.ds + 1)] = (float)s;
}

__global__ void obs_beta_kernel(DevView v, int rows, double y_mean, double inv_std) {
  obs_beta_body(v, rows, y_mean, inv_std, blockIdx.x);
}

__global__ void obs_alpha_kernel(DevView v, int rows) { obs_alpha_body(v, rows, blockIdx.x); }

// ---- the same phases over many spaces: block b serves item blocks[b].item ----
__global__ void obs_k_batch(const ObsItem* items, const ObsBlock* blocks) {
  const ObsBlock b = blocks[blockIdx.x];
  const ObsItem& it = items[b.item];
  obs_k_body(it.v, it.n, it.idx, it.y_raw, b.local);
}

__global__ void obs_l_batch(const ObsItem* items, const ObsBlock* blocks) {
  const ObsBlock b = blocks[blockIdx.x];
  const ObsItem& it = items[b.item];
  obs_l_body(it.v, it.n, b.local);
}

__global__ void obs_w_batch(const ObsItem* items, const ObsBlock* blocks) {
  const ObsBlock b = blocks[blockIdx.x];
  const ObsItem& it = items[b.item];
  const int gx = (it.n + 31) / 32;
  obs_w_body(it.v, it.n, b.local % gx, b.local / gx);
}

__global__ void obs_finish_batch(const ObsItem* items) {
  const ObsItem& it = items[blockIdx.x];
  obs_finish_body(it.v, it.n);
}

__global__ void obs_beta_batch(const ObsItem* items, const ObsBlock* blocks) {
  const ObsBlock b = blocks[blockIdx.x];
  const ObsItem& it = items[b.item];
  obs_beta_body(it.v, it.n + 1, it.y_mean, it.inv_std, b.local);
}

__global__ void obs_alpha_batch(const ObsItem* items, const ObsBlock* blocks) {
  const ObsBlock b = blocks[blockIdx.x];
  const ObsItem& it = items[b.item];
  obs_alpha_body(it.v, it.n + 1, b.local);
}

__global__ void set_visited_batch(const VisitItem* items, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) atomicOr(&items[i].visited[items[i].idx >> 5], 1u << (items[i].idx & 31));
}

__global__ void set_visited_kernel(uint32_t* visited, long long idx) {
  atomicOr(&visited[idx >> 5], 1u << (idx & 31));
}

void obs_batch_blocks(const int* n, int count, std::vector<ObsBlock>* blocks, int counts[5]) {
  // per phase, the blocks each space needs (as the single-space launch uses)
  blocks->clear();
  auto add = [&](int phase_blocks(int), int slot) {
    const size_t start = blocks->size();
    for (int i = 0; i < count; ++i)
      for (int b = 0; b < phase_blocks(n[i]); ++b) blocks->push_back(ObsBlock{i, b});
    counts[slot] = (int)(blocks->size() - start);
  };
  add([](int m) { return (m + 31) / 32 + (m == 0); }, 0);             // k: 32 threads
  add([](int m) { return (m + 7) / 8; }, 1);                          // l: warp per row
  add([](int m) { return ((m + 31) / 32) * ((m + 63) / 64); }, 2);    // w: 32 columns x 64 rows
  add([](int m) { return (m + 1 + 7) / 8; }, 3);                      // beta: warp per row
  add([](int m) { return (m + 1 + 7) / 8; }, 4);                      // alpha: warp per column
}

int launch_observe_batch(const ObsItem* items, int count, const ObsBlock* blocks, const int counts[5],
                         const VisitItem* visits, int n_visits, bool tc, cudaStream_t s) {
  int launches = 0;
  const ObsBlock* b = blocks;
  if (count > 0) {
    if (counts[0]) { obs_k_batch<<<counts[0], 32, 0, s>>>(items, b); ++launches; }
    b += counts[0];
    if (counts[1]) { obs_l_batch<<<counts[1], 256, 0, s>>>(items, b); ++launches; }
    b += counts[1];
    if (counts[2]) { obs_w_batch<<<counts[2], 256, 0, s>>>(items, b); ++launches; }
    b += counts[2];
    obs_finish_batch<<<count, 512, 0, s>>>(items);
    ++launches;
    if (counts[3]) { obs_beta_batch<<<counts[3], 256, 0, s>>>(items, b); ++launches; }
    b += counts[3];
    if (counts[4] && tc) { obs_alpha_batch<<<counts[4], 256, 0, s>>>(items, b); ++launches; }
  }
  if (n_visits > 0) {
    set_visited_batch<<<(n_visits + 127) / 128, 128, 0, s>>>(visits, n_visits);
    ++launches;
  }
  return cudaGetLastError() == cudaSuccess ? launches : -1;
}

int launch_set_visited(const DevView& v, int64_t idx, cudaStream_t s) {
  set_visited_kernel<<<1, 1, 0, s>>>(v.visited, (long long)idx);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

// ---- the whole update of one space in one cooperative launch ----------------
// The phases above run as virtual blocks of 256 threads over a co-resident
// grid, separated by grid barriers (arrival counter in DevStats, bounded wait:
// on expiry the update records BO_ERR_TIMEOUT and every block leaves).  One
// launch instead of six saves the launch gaps that dominate at small n.
constexpr int kFusedThreads = 256;
constexpr unsigned long long kCoopWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long coop_now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Arrive at grid barrier number `phase` (1, 2, ...) and wait for every block.
__device__ __forceinline__ bool coop_sync(DevStats* st, unsigned int phase) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&st->coop_count, 1u);
    const unsigned int target = phase * gridDim.x;
    const unsigned long long t0 = coop_now_ns();
    while (*(volatile unsigned int*)&st->coop_count < target) {
      if (*(volatile int32_t*)&st->coop_abort) break;
      if (coop_now_ns() - t0 > kCoopWaitNs) {
        atomicExch(&st->coop_abort, 1);
        atomicExch(&st->status, BO_ERR_TIMEOUT);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int32_t*)&st->coop_abort == 0;
}

__global__ void __launch_bounds__(kFusedThreads) obs_fused_kernel(DevView v, int n, long long idx, double y_raw,
                                                                  double y_mean, double inv_std) {
  DevStats* st = v.stats;
  const int G = (int)gridDim.x;
  const int rows = n + 1;
  unsigned int phase = 0;
  do {
    for (int b = blockIdx.x; b < (n + kFusedThreads - 1) / kFusedThreads + (n == 0); b += G)
      obs_k_body(v, n, idx, y_raw, b);
    if (n > 0) {
      if (!coop_sync(st, ++phase)) break;
      for (int b = blockIdx.x; b < (n + 7) / 8; b += G) obs_l_body(v, n, b);
      if (!coop_sync(st, ++phase)) break;
      const int gx = (n + 31) / 32, gy = (n + 63) / 64;
      for (int b = blockIdx.x; b < gx * gy; b += G) {
        obs_w_body(v, n, b % gx, b / gx);
        __syncthreads();                       // its shared partials are reused by the next one
      }
    }
    if (!coop_sync(st, ++phase)) break;
    if (blockIdx.x == 0) obs_finish_body(v, n);
    if (!coop_sync(st, ++phase)) break;
    for (int b = blockIdx.x; b < (rows + 7) / 8; b += G) obs_beta_body(v, rows, y_mean, inv_std, b);
    if (v.precision != BO_PREC_FP64) {
      if (!coop_sync(st, ++phase)) break;
      for (int b = blockIdx.x; b < (rows + 7) / 8; b += G) obs_alpha_body(v, rows, b);
    }
  } while (false);
  // the last block to leave resets the barrier state for the next update
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&st->coop_done, 1u) == (unsigned int)G - 1) {
      st->coop_count = 0;
      st->coop_abort = 0;
      st->coop_done = 0;
      __threadfence();
    }
  }
}

// Self-test of the fused update's grid barrier: block 1 of two never arrives,
// so block 0's bounded wait runs out and records BO_ERR_TIMEOUT in st.
__global__ void selftest_grid_kernel(DevStats* st) {
  if (blockIdx.x == 0) (void)coop_sync(st, 1);
}

int launch_selftest_grid(DevStats* st, cudaStream_t s) {
  void* args[] = {&st};
  return cudaLaunchCooperativeKernel((const void*)selftest_grid_kernel, dim3(2), dim3(kFusedThreads), args, 0, s) ==
                 cudaSuccess
             ? 1
             : -1;
}

// Blocks of the fused update for n fitted observations: the largest phase,
// capped by what is co-resident on the current device (-1 if the occupancy
// query fails).
int fused_update_grid(int n) {
  static int co_resident[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
  int max_blocks;
  {
    std::lock_guard<std::mutex> lk(launch_attr_mutex());
    if (co_resident[dev] == 0) {
      int sms = 0, per_sm = 0;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, obs_fused_kernel, kFusedThreads, 0) !=
              cudaSuccess ||
          per_sm < 1)
        return -1;
      co_resident[dev] = sms * per_sm;
    }
    max_blocks = co_resident[dev];
  }
  const int rows = n + 1;
  int want = std::max(1, (n + kFusedThreads - 1) / kFusedThreads);
  want = std::max(want, (n + 7) / 8);
  want = std::max(want, ((n + 31) / 32) * ((n + 63) / 64));
  want = std::max(want, (rows + 7) / 8);
  return std::min(want, max_blocks);
}

int launch_observe_update(bool cooperative, const DevView& v, int n, int64_t idx, double y_raw, double y_mean,
                          double y_std, cudaStream_t s) {
  // n = observations fitted before this one; the new one becomes row n.
  if (cooperative) {
    const int grid = fused_update_grid(n);
    if (grid > 0) {
      long long idx_ll = (long long)idx;
      double inv_std = 1.0 / y_std;
      DevView vv = v;
      void* args[] = {&vv, &n, &idx_ll, &y_raw, &y_mean, &inv_std};
      if (cudaLaunchCooperativeKernel((const void*)obs_fused_kernel, dim3(grid), dim3(kFusedThreads), args, 0, s) ==
          cudaSuccess)
        return 1;
      (void)cudaGetLastError();   // not launchable cooperatively here: the phase kernels below
    }
  }
  int launches = 0;
  obs_k_kernel<<<(n + 31) / 32 + (n == 0), 32, 0, s>>>(v, n, (long long)idx, y_raw);
  ++launches;
  if (n > 0) {
    obs_l_kernel<<<(n + 7) / 8, 256, 0, s>>>(v, n);
    dim3 gw((n + 31) / 32, (n + 63) / 64);
    obs_w_kernel<<<gw, 256, 0, s>>>(v, n);
    launches += 2;
  }
  obs_finish_kernel<<<1, 512, 0, s>>>(v, n);
  const int rows = n + 1;
  obs_beta_kernel<<<(rows + 7) / 8, 256, 0, s>>>(v, rows, y_mean, 1.0 / y_std);
  launches += 2;
  if (v.precision != BO_PREC_FP64) {
    obs_alpha_kernel<<<(rows + 7) / 8, 256, 0, s>>>(v, rows);
    ++launches;
  }
  return cudaGetLastError() == cudaSuccess ? launches : -1;
}

}  // namespace bo
