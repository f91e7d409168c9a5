// Observation update of the GP surrogate (FP64), one valid observation at a time.
//
// With a fixed lengthscale (paper Sec. III-B) the kernel matrix of the
// observations only grows by one row and column per observation, so the
// Cholesky factor grows by one row and so does its inverse:
//   K_new = [[K, k], [k^T, k(0) + jitter]],  l = L^-1 k,  d = sqrt(k(0) + jitter - l.l)
//   L_new^-1 = [[L^-1, 0], [-(L^-T l)^T / d, 1 / d]].
// Rows of L^-1 never change once written.  beta = L^-1 y~ and alpha = K^-1 y~
// change in every entry when the standardization of y shifts, but both are
// affine in its mean, so they follow from four vectors updated in O(n) per
// observation (see the finish phase).  The reduced-precision contraction gets
// a per-row scaled, split copy of each new row (written once), see
// lsplit_offset().
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
// (obs_record: the bookkeeping, by one block; obs_kj: one entry of k)
__device__ __forceinline__ void obs_record(const DevView& v, int n, const ObsNew& o) {
  if (threadIdx.x < v.d) {
    const int p = threadIdx.x;
    v.X[(size_t)n * v.d + p] = o.x[p];
    v.Xc[(size_t)n * v.d + p] = (uint8_t)o.a[p];
    if (v.xq) v.xq[xq_index(v.ds, n, p)] = (float)(o.x[p] * (1.4426950408889634 * v.kcoef));
  }
  if (threadIdx.x == 0) {
    v.y[n] = o.y_raw;
    atomicOr(&v.visited[o.idx >> 5], 1u << (o.idx & 31));
  }
}

// The new point's codes and coordinates and the table offsets (formed on the
// host), staged in shared memory once per block, so that an entry of k needs
// one round of loads (its observation's codes or coordinates, then the table
// entries).
struct KStage {
  int off[BO_MAX_PARAMS];      // table offset of parameter p (tabulated distances)
  int m[BO_MAX_PARAMS];        // value count of parameter p
  int a[BO_MAX_PARAMS];        // the new point's value index of parameter p
  double x[BO_MAX_PARAMS];     // the new point's coordinate of parameter p
};

__device__ __forceinline__ void k_stage(const DevView& v, const ObsNew& o, KStage& ks) {
  for (int p = threadIdx.x; p < v.d; p += blockDim.x) {
    ks.a[p] = o.a[p];
    ks.x[p] = o.x[p];
    ks.off[p] = o.off[p];
    ks.m[p] = o.m[p];
  }
  __syncthreads();
}

__device__ __forceinline__ void obs_kj(const DevView& v, const KStage& ks, int j) {
  const double c = v.kcoef;
  double r2 = 0.0;
  if (v.sqd) {   // the prediction pass's arithmetic: a sum of tabulated squared differences
#pragma unroll
    for (int p = 0; p < BO_MAX_PARAMS; ++p)
      if (p < v.d) r2 += v.sqd[ks.off[p] + ks.a[p] * ks.m[p] + v.Xc[(size_t)j * v.d + p]];
  } else {
#pragma unroll
    for (int p = 0; p < BO_MAX_PARAMS; ++p)
      if (p < v.d) {
        const double diff = ks.x[p] - v.X[(size_t)j * v.d + p];
        r2 = fma(diff, diff, r2);
      }
  }
  v.kvec[j] = matern64(sqrt(r2), v.nu, c);
}

__device__ __forceinline__ void obs_k_body(const DevView& v, int n, const ObsNew& o, int block) {
  __shared__ KStage ks;
  const int j = block * blockDim.x + threadIdx.x;
  if (block == 0) obs_record(v, n, o);
  k_stage(v, o, ks);
  if (j < n) obs_kj(v, ks, j);
}

__global__ void obs_k_kernel(DevView v, int n, const __grid_constant__ ObsNew o) { obs_k_body(v, n, o, blockIdx.x); }

__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// --- K3b: l = L^-1 k (warp per row, 8 rows per block of 256) ----------------------
// The block also writes its shares of three pivot sums over its rows i:
// l_i^2, k_i a_i and k_i b_i, each added in row order (upart[3 block + q]);
// the pivot phase adds the blocks' shares, so no single block reduces over n.
__device__ __forceinline__ void obs_l_body(const DevView& v, int n, int block) {
  __shared__ double s_part[8][3];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = block * 8 + w;
  double l = 0.0;
  if (row < n) {
    const double* r = v.linv + (size_t)row * v.n_max;
    double s = 0.0;
#pragma unroll 4
    for (int j = lane; j <= row; j += 32) s = fma(r[j], v.kvec[j], s);
    l = warp_sum(s);
    if (lane == 0) v.lvec[row] = l;
  }
  if (lane == 0) {
    const bool tc = row < n && v.avec != nullptr;
    s_part[w][0] = l * l;
    s_part[w][1] = tc ? v.kvec[row] * v.avec[row] : 0.0;
    s_part[w][2] = tc ? v.kvec[row] * v.bvec[row] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += s_part[q][threadIdx.x];
    v.upart[3 * block + threadIdx.x] = t;
  }
  __syncthreads();   // s_part is reused by the block's next row group
}

__global__ void obs_l_kernel(DevView v, int n) { obs_l_body(v, n, blockIdx.x); }

// --- K3c: partial w = L^-T l over row segments of 64 ---------------------------
// Block (column block of 32, row segment of 64): lane = column, warp w sums
// rows seg*64 + 8w .. +8 with all eight loads in flight; L^-1[i][j] = 0 for j > i.
// w.(y - y0) and w.1 are linear in these row-segment sums, so each block also
// writes its shares of both (upart[3 nl + 2 (by gx + bx) + q]).
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
  if (w == 0) {
    double t = 0.0;
    if (j < n) {
#pragma unroll
      for (int q = 0; q < 8; ++q) t += part[q][lane];
      v.wvec[(size_t)by * v.n_max + j] = t;
    }
    const double ty = warp_sum(j < n ? t * (v.y[j] - v.y[0]) : 0.0);
    const double t1 = warp_sum(t);
    if (lane == 0) {
      const int nl = (n + 7) / 8, gx = (n + 31) / 32;
      v.upart[3 * nl + 2 * (by * gx + bx)] = ty;
      v.upart[3 * nl + 2 * (by * gx + bx) + 1] = t1;
    }
  }
}

__global__ void obs_w_kernel(DevView v, int n) { obs_w_body(v, n, blockIdx.x, blockIdx.y); }

// --- K3d: pivot, new row n of L^-1 and its split copy, beta and alpha (one block)
// beta = L^-1 y~ and alpha = K^-1 y~ = L^-T beta change in every entry when the
// standardization y~ = (y - m) / std shifts, but both are affine in m:
//   beta  = (u - (m - y0) e) / std,   u = L^-1 (y - y0),  e = L^-1 1
//   alpha = (a - (m - y0) b) / std,   a = K^-1 (y - y0),  b = K^-1 1
// (y0 = the first fitted value, a fixed shift that keeps u and a small).  u and
// e grow by one entry per observation (rows of L^-1 never change): u_n =
// row_n . (y - y0), e_n = row_n . 1.  a and b follow the bordered inverse
//   K_new^-1 = [[K^-1 + w w^T / s, -w / s], [-w^T / s, 1 / s]],  w = K^-1 k,
//   s = k(0) + jitter - l.l:  a_new = [a - w g, g],  g = ((y_n - y0) - k.a) / s
// (the same for b with 1 - k.b), so the whole update of beta and alpha is O(n).

// The pivot and every scalar of the new row follow from five sums over the
// previous rows and max |w| (w = L^-T l):
//   l.l,  w.(y - y0),  w.1,  k.a,  k.b   (shares written by the l and w phases)
// d^2 = k(0) + jitter - l.l;  the new row is [-w / d, 1 / d], so
//   u_n = row . (y - y0) = ((y_n - y0) - w.(y - y0)) / d,  e_n = (1 - w.1) / d,
//   g_a = ((y_n - y0) - k.a) / d^2,  g_b = (1 - k.b) / d^2,
// and the row's largest magnitude, for the split copy's scale, is max|w| / d or 1 / d.
// FP64 is a narrow unit on this GPU (one warp instruction occupies it for ~64
// cycles), so no block reduces over n: each block adds the phases' block
// shares (warp q adds sum q in block order: the same value in every block),
// takes max |w| as an integer maximum of the bit patterns (non-negative doubles
// order as their bits), forms the scalars in one thread, and writes entries
// j = slice + nslices t of the row (slice 0 of nslices also the bookkeeping).
__device__ __forceinline__ void obs_finish_body(const DevView& v, int n, double y_mean, double inv_std, int slice,
                                                int nslices) {
  __shared__ double s_sum[5];  // l.l, k.a, k.b, w.(y - y0), w.1
  __shared__ unsigned long long s_wmax;
  __shared__ double s_sc[8];   // dinv, d2, u_n, e_n, g_a, g_b, amax
  __shared__ float s_scale;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool tc = v.precision != BO_PREC_FP64;
  const int nseg = (n + 63) / 64;
  const int nl = (n + 7) / 8, nw = ((n + 31) / 32) * nseg;
  const double y0 = v.y[0];
  auto w_of = [&](int j) {
    double w = 0.0;
#pragma unroll
    for (int s = 0; s < 8; ++s)
      if (s < nseg) w += v.wvec[(size_t)s * v.n_max + j];
    return w;
  };
  if (tid == 0) s_wmax = 0ull;
  __syncthreads();
  if (tc) {   // only the split copy's scale needs max |w|
    unsigned long long mx = 0ull;
    for (int j = tid; j < n; j += blockDim.x) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(w_of(j)));
      mx = b > mx ? b : mx;
    }
    const uint32_t hi = (uint32_t)(mx >> 32), mh = __reduce_max_sync(0xffffffffu, hi);
    const uint32_t ml = __reduce_max_sync(0xffffffffu, hi == mh ? (uint32_t)mx : 0u);
    if (lane == 0) atomicMax(&s_wmax, ((unsigned long long)mh << 32) | ml);
  }
  if (warp < 5) {
    const bool lq = warp < 3;   // an l-phase sum (3 per block) or a w-phase one (2 per block)
    const double* src = lq ? v.upart + warp : v.upart + 3 * nl + (warp - 3);
    const int cnt = lq ? nl : nw, stride = lq ? 3 : 2;
    double t = 0.0;
    for (int i = lane; i < cnt; i += 32) t += src[(size_t)i * stride];
    t = warp_sum(t);
    if (lane == 0) s_sum[warp] = t;
  }
  __syncthreads();
  if (tid == 0) {
    const double ll = s_sum[0], ka = s_sum[1], kb = s_sum[2], wy = s_sum[3], w1 = s_sum[4];
    const double wmax = __longlong_as_double((long long)s_wmax);
    const double d2 = 1.0 + v.jitter - ll;
    const double dinv = (d2 > 0.0 && isfinite(d2)) ? 1.0 / sqrt(d2) : 0.0;
    const double dinv2 = dinv * dinv;
    const double yn = v.y[n] - y0;
    s_sc[0] = dinv;
    s_sc[1] = d2;
    s_sc[2] = (yn - wy) * dinv;
    s_sc[3] = (1.0 - w1) * dinv;
    s_sc[4] = (yn - ka) * dinv2;
    s_sc[5] = (1.0 - kb) * dinv2;
    s_sc[6] = fmax(wmax, 1.0) * dinv;
    if (tc) {
      // per-row power-of-two scale s with max |row| * s in [2^13, 2^14)
      int e;
      frexp(s_sc[6], &e);                 // amax in [2^(e-1), 2^e)
      s_scale = ldexpf(1.0f, 14 - e);
    }
    if (slice == 0) {
      if (dinv == 0.0) v.stats->status = BO_ERR_NUMERIC;
      if (tc) v.xq[xq_index(v.ds, n, v.ds)] = 1.0f / (s_scale * s_scale);
      v.uvec[n] = s_sc[2];
      v.evec[n] = s_sc[3];
    }
  }
  __syncthreads();
  const double dinv = s_sc[0];
  if (dinv == 0.0) return;
  const double pu = s_sc[2], pe = s_sc[3], ga = s_sc[4], gb = s_sc[5];
  const double shift = y_mean - y0;
  const float sc = tc ? s_scale : 0.0f;
  const int eb = split_elem_bytes(v.precision);
  double* row = v.linv + (size_t)n * v.n_max;
  for (int j = slice + nslices * tid; j <= n; j += nslices * (int)blockDim.x) {
    const double w = j < n ? w_of(j) : 0.0;
    const double val = j < n ? -w * dinv : dinv;
    row[j] = val;
    const double u = j < n ? v.uvec[j] : pu, e = j < n ? v.evec[j] : pe;
    v.beta[j] = (u - shift * e) * inv_std;
    if (!tc) continue;
    const double a = j < n ? fma(-w, ga, v.avec[j]) : ga;
    const double b = j < n ? fma(-w, gb, v.bvec[j]) : gb;
    v.avec[j] = a;
    v.bvec[j] = b;
    v.xq[xq_index(v.ds, j, v.ds + 1)] = (float)((a - shift * b) * inv_std);
    // the split copy of row n, element j
    const float x = (float)val * sc;
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
      uint32_t hu;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hu) : "f"(x));
      *reinterpret_cast<uint32_t*>(v.lsplit_hi + off) = hu;
      if (v.precision == BO_PREC_TF32X3) {   // lo = the rounding residual, itself rounded to TF32
        uint32_t lu;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lu) : "f"(x - __uint_as_float(hu)));
        *reinterpret_cast<uint32_t*>(v.lsplit_lo + off) = lu;
      }
    }
  }
}

__global__ void obs_finish_kernel(DevView v, int n, double y_mean, double inv_std) {
  obs_finish_body(v, n, y_mean, inv_std, 0, 1);
}

// ---- the same phases over many spaces: block b serves item blocks[b].item ----
__global__ void obs_k_batch(const ObsItem* items, const ObsBlock* blocks) {
  const ObsBlock b = blocks[blockIdx.x];
  const ObsItem& it = items[b.item];
  obs_k_body(it.v, it.n, it.o, b.local);
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
  obs_finish_body(it.v, it.n, it.o.y_mean, it.o.inv_std, 0, 1);
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
  counts[3] = counts[4] = 0;                                          // beta, alpha: in the finish
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
  }
  (void)tc;
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
// The phases above (k, l, w, finish) run as virtual blocks of 256 threads over
// a co-resident grid, separated by three grid barriers (arrival counter in
// DevStats, bounded wait: on expiry the update records BO_ERR_TIMEOUT and
// every block leaves).  One launch instead of four saves the launch gaps that
// dominate at small n.
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

// L2 prefetch of this block's share (1 / parts) of [p, p + bytes), in whole 16-byte granules
// (a partial last granule is left out, so nothing past the range is touched).
__device__ __forceinline__ void l2_prefetch_share(const void* p, size_t bytes, int part, int parts) {
  if (!p) return;
  const size_t per = ((bytes + (size_t)parts - 1) / (size_t)parts + 15) & ~(size_t)15;
  size_t lo = per * (size_t)part;
  const size_t hi = min(bytes & ~(size_t)15, lo + per);
  while (lo < hi) {
    const uint32_t len = (uint32_t)min(hi - lo, (size_t)(1u << 20));
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(static_cast<const uint8_t*>(p) + lo), "r"(len)
                 : "memory");
    lo += len;
  }
}

__global__ void __launch_bounds__(kFusedThreads) obs_fused_kernel(DevView v, int n, const __grid_constant__ ObsNew o) {
  pdl_trigger();           // the prediction pass may be launched now (it waits for this update)
  // the phases' inputs into L2 first (an L2 flush between passes leaves them in HBM): the rows of
  // L^-1 (phases l, w), the observations' value indices / coordinates and tables (phase k), the
  // vectors the pivot phase reads; prefetches are hints, the phases read after their barriers
  if (threadIdx.x == 0) {
    const int G = (int)gridDim.x, b = (int)blockIdx.x;
    const size_t r8 = (size_t)n * 8;     // exact sizes: the prefetch stops at their last whole granule
    l2_prefetch_share(v.linv, (size_t)n * v.n_max * 8, b, G);
    if (b == G - 1) {
      l2_prefetch_share(v.Xc, (size_t)n * v.d, 0, 1);
      if (v.sqd) l2_prefetch_share(v.sqd, (size_t)v.sqd_total * 8, 0, 1);
      else l2_prefetch_share(v.X, (size_t)n * v.d * 8, 0, 1);
      l2_prefetch_share(v.y, r8, 0, 1);
      l2_prefetch_share(v.uvec, r8, 0, 1);
      l2_prefetch_share(v.evec, r8, 0, 1);
      l2_prefetch_share(v.avec, r8, 0, 1);
      l2_prefetch_share(v.bvec, r8, 0, 1);
    }
  }
  DevStats* st = v.stats;
  const int G = (int)gridDim.x;
  unsigned int phase = 0;
  do {
    // k over all blocks (entry j on block j mod G): its FP64 Matern chains run side by side
    if (blockIdx.x == 0) obs_record(v, n, o);
    {
      __shared__ KStage ks;
      k_stage(v, o, ks);
      for (int j = blockIdx.x + G * threadIdx.x; j < n; j += G * kFusedThreads) obs_kj(v, ks, j);
    }
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
    obs_finish_body(v, n, o.y_mean, o.inv_std, blockIdx.x, G);   // every block: its slice of the row
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
  int want = std::max(1, (n + kFusedThreads - 1) / kFusedThreads);
  want = std::max(want, (n + 7) / 8);
  want = std::max(want, ((n + 31) / 32) * ((n + 63) / 64));
  return std::min(want, max_blocks);
}

int launch_observe_update(bool cooperative, const DevView& v, int n, const ObsNew& o, cudaStream_t s) {
  // n = observations fitted before this one; the new one becomes row n.
  if (cooperative) {
    const int grid = fused_update_grid(n);
    if (grid > 0) {
      DevView vv = v;
      ObsNew oo = o;
      void* args[] = {&vv, &n, &oo};
      if (cudaLaunchCooperativeKernel((const void*)obs_fused_kernel, dim3(grid), dim3(kFusedThreads), args, 0, s) ==
          cudaSuccess)
        return 1;
      (void)cudaGetLastError();   // not launchable cooperatively here: the phase kernels below
    }
  }
  int launches = 0;
  obs_k_kernel<<<(n + 31) / 32 + (n == 0), 32, 0, s>>>(v, n, o);
  ++launches;
  if (n > 0) {
    obs_l_kernel<<<(n + 7) / 8, 256, 0, s>>>(v, n);
    dim3 gw((n + 31) / 32, (n + 63) / 64);
    obs_w_kernel<<<gw, 256, 0, s>>>(v, n);
    launches += 2;
  }
  obs_finish_kernel<<<1, 512, 0, s>>>(v, n, o.y_mean, o.inv_std);
  ++launches;
  return cudaGetLastError() == cudaSuccess ? launches : -1;
}

}  // namespace bo
