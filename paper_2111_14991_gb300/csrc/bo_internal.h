// Internal interfaces shared by the CUDA translation units and the host session.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "bo_suggest.h"

namespace bo {

// Candidates are processed in tiles of this many rows; per-candidate device
// arrays are padded to a multiple of it.
constexpr int kTileRows = 128;
// Columns of the reduced-precision L^-1 copy per K chunk, in bytes of one row.
constexpr int kChunkBytes = 64;

enum AfId { kEI = 0, kPI = 1, kLCB = 2 };

// Device-side scalars of one space.
struct DevStats {
  double sum_var;            // variance sum of the last pass with the acquisition as the prediction's tail
  double var_s;              // contextual-variance baseline (set by the first pass)
  unsigned int k1_done;      // grid-barrier and last-block counters (reset by the last block)
  unsigned int k2_done;
  int32_t status;            // sticky BO_ERR_* of observation updates
  int32_t pad;
  unsigned int coop_count;   // grid-barrier arrivals of the fused update (reset by its last block)
  unsigned int coop_done;    // blocks that left the fused update
  int32_t coop_abort;        // a grid-barrier wait of the fused update timed out
  int32_t pad2;
};

struct TopEntry {
  double score;
  long long idx;
};

// Every device pointer and size of a space, passed by value to launchers.
struct DevView {
  int d;
  int64_t N;                 // valid configurations
  int64_t N_pad;             // N rounded up to kTileRows
  int n_max;                 // capacity in fitted observations (multiple of 32)
  int precision;             // BO_PREC_*
  double nu, lengthscale, jitter;
  double kcoef;              // sqrt(2 nu) / lengthscale, formed once on the host

  const uint8_t* codes;      // [d][N_pad] value index per parameter, parameter-major
  const double* vtab64;      // [d][256] normalized values
  const float* vtab32;       // [d][256] values times sqrt(2 nu) / l * log2(e), rounded once
  uint32_t* visited;         // [ceil(N/32)] bit i = configuration i evaluated

  double* X;                 // [n_max][d] coordinates of fitted observations
  uint8_t* Xc;               // [n_max][d] value indices of fitted observations
  const double* sqd;         // per parameter p, [m_p][m_p] (v_a - v_b)^2 of its normalized values
  const int* sqd_meta;       // [2 d + 1]: offset of each parameter's table in sqd (then the
                             // total), then m_p
  int sqd_total;             // sum_p m_p^2
  float* xq;                 // [n_max / 8][ds + 2][8] per group of 8 observations: the FP32
                             // coordinates scaled as vtab32 (ds rows, rows >= d zero), then
                             // 1 / s_k^2 of the per-row power-of-two scale s_k of the split
                             // L^-1 copy, then alpha = L^-T beta (mu = k* . alpha); zero
                             // beyond n.  Reduced-precision spaces only.
  int ds;                    // coordinate rows per group: the space's dimension bucket
  double* y;                 // [n_max] raw fitted values
  double* linv;              // [n_max][n_max] L^-1, row-major, lower triangular
  double* beta;              // [n_max] L^-1 y~
  double* uvec;              // [n_max] L^-1 (y - y0), y0 = y[0] (beta is affine in the mean of y)
  double* evec;              // [n_max] L^-1 1
  double* avec;              // [n_max] K^-1 (y - y0) (tensor-core forms: alpha = K^-1 y~)
  double* bvec;              // [n_max] K^-1 1
  uint8_t* lsplit_hi;        // reduced-precision chunked copy of L^-1 (hi part, or the single tf32)
  uint8_t* lsplit_lo;        // (lo part; unused for the single tf32 form)

  void* mu;                  // [N_pad] posterior mean (double for FP64, else float)
  void* var;                 // [N_pad] posterior variance
  double* partial;           // [max_partials] per-block sums of variance
  int max_partials;

  double* kvec;              // [n_max] update scratch
  double* lvec;              // [n_max]
  double* wvec;              // [n_max]
  double* upart;             // [update_part_count(n_max)]: the l and w phases' block shares of the pivot sums

  DevStats* stats;
  TopEntry* acq_partial;     // [max_acq_blocks][3][3]
  int max_acq_blocks;
  int num_sms;               // multiprocessors of the space's device
  bo_pass_result* results;   // [max_results]
  int max_results;
};

// Float index of slot `slot` (coordinate row, ds = 1/s^2, ds + 1 = alpha) of observation j in xq.
__host__ __device__ inline size_t xq_index(int ds, int j, int slot) {
  return (size_t)(j >> 3) * (ds + 2) * 8 + (size_t)slot * 8 + (j & 7);
}

// Largest table of per-parameter squared value differences a space keeps (the
// FP64 distances then sum d table entries instead of d differences and squares).
constexpr size_t kSqdMaxBytes = 48 * 1024;

// Per-device launch attributes, set once and shared by every host thread:
// raise `kernel`'s dynamic shared-memory limit on the current device to at
// least `bytes` (configured[] remembers each device's value; one lock orders
// concurrent callers, so a smaller request never lowers a larger limit).
constexpr int kMaxDevices = 64;
inline std::mutex& launch_attr_mutex() {
  static std::mutex m;
  return m;
}
inline bool ensure_dynamic_smem(const void* kernel, size_t (&configured)[kMaxDevices], size_t bytes) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return false;
  std::lock_guard<std::mutex> lk(launch_attr_mutex());
  if (configured[dev] >= bytes) return true;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
    return false;
  configured[dev] = bytes;
  return true;
}

// Programmatic dependent launch: kernels of one pass (update -> prediction ->
// acquisition) may be launched as dependents of the previous kernel in the
// stream, so that their launch and prologue overlap its tail.  A dependent
// waits (pdl_wait) for the predecessor to complete, its memory visible,
// before it reads or writes anything the predecessor touches; a kernel
// launched without the attribute passes pdl_wait at once.  With BO_NO_PDL set
// in the environment (read once per process) they are launched plainly.
bool pdl_enabled();
// Launch `kernel` on s with the programmatic-serialization attribute when pdl.
template <typename... Params, typename... Args>
cudaError_t launch_ex(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                      Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Sum of count per-block partials (written by other blocks, made visible by
// the caller's fence / counter protocol), by every thread of a block: each
// thread adds its strided share in order, a fixed warp butterfly and a
// fixed-order sum of the warp results by one thread follow, so the value is
// the same in every run.  Loads go to L2 in parallel instead of one dependent
// chain.  (FP64 issues at 1/64 of the FP32 rate on this GPU: the scalar tail
// runs in one thread and is broadcast, not repeated by every thread.)  red:
// shared memory for blockDim.x / 32 + 1 doubles.  Every thread of the block
// must call it; every thread gets the sum.
__device__ __forceinline__ double block_sum_partials(const double* p, int count, double* red) {
  double t = 0.0;
  for (int b = threadIdx.x; b < count; b += blockDim.x) t += __ldcg(p + b);
  if ((int)(threadIdx.x & ~31u) < count)           // warps without partials add nothing
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  const int nw = (int)(blockDim.x >> 5);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    red[nw] = s;
  }
  __syncthreads();
  const double s = red[nw];
  __syncthreads();
  return s;
}
#endif

// Scalars of one prediction pass known to the host.
struct PassArgs {
  int n;                     // fitted observations
  int64_t n_unvisited;       // valid, non-evaluated configurations
  int n_af;                  // active acquisition functions (1..3), ids in af[]
  int af[3];
  int k;                     // entries kept per AF
  int explore;               // BO_EXPLORE_*
  double lambda_const;
  double fplus_t;            // best observation, standardized
  double fplus_raw, mu_s_raw;
  int first_pass;            // contextual-variance baseline is taken from this pass
  int result_slot;           // index into DevView::results
};

// Device operands of one acquisition pass.
struct AcqDev {
  const void* mu;            // [N] posterior mean (double or float)
  const void* var;           // [N] posterior variance
  const uint32_t* visited;   // [ceil(N/32)]
  int64_t N;
  const double* sum_var;     // sum of variances over the non-evaluated candidates (when var_parts is NULL)
  // or: the prediction pass's per-CTA variance sums, which every acquisition
  // block adds in the same fixed order (no last-CTA step in the prediction)
  const double* var_parts = nullptr;
  int n_var_parts = 0;
  double* var_s;             // contextual-variance baseline (written on a first pass)
  const int32_t* status_in;  // status folded into the result, or NULL
  TopEntry* partial;         // [max_blocks][3][3] scratch
  unsigned int* counter;     // last-block counter, 0 between launches
  int max_blocks;
  bo_pass_result* result;
  // FP64 posteriors of a small space: at least min_blocks blocks (one per
  // multiprocessor), candidates dealt round-robin over the blocks (spread), so
  // that the FP64 scoring runs on every FP64 pipe; 0 keeps the plain grid
  int min_blocks = 0;
  int spread = 0;
};

// One space as the tensor-core pass sees it (device pointers and sizes).
struct TcSess {
  const uint8_t* codes;      // [d][N_pad]
  const float* vtab32;       // [d][256] scaled values
  const uint32_t* visited;
  const float* xq;           // [n_max / 8][ds + 2][8] coordinates, 1/s^2, alpha per 8 observations
  const uint8_t* lhi;        // chunked split copy of L^-1
  const uint8_t* llo;
  float* mu;
  float* var;
  int64_t N, N_pad;
  int d, ds, n, n_pad, n_max, chunks, num_tiles;
};

// Tiles [tile0, tile1) of space sess, processed in order by one CTA.
struct TcSeg {
  int sess, tile0, tile1;
};

// Pipeline shape of a tensor-core launch (0 / -1 = the planner's default):
// A-ring depth, B-ring slots, resident B pieces allowed (-1 = never).
struct TcShape {
  int stages_a = 0;
  int b_slots = 0;
  int b_resident = 0;
};

// A batched tensor-core launch: device arrays the host planned and uploaded.
struct TcBatchLaunch {
  const TcSess* sess;        // [count]
  const TcSeg* segs;         // [num_segs]
  const int* seg_begin;      // [grid + 1]
  double* seg_part;          // [num_segs][4] variance sums written by the kernel
  int32_t* status;           // BO_ERR_TIMEOUT lands here
  int count, grid, precision, dmax, n_pad_max;
  double nu;
};

// One space of a batched acquisition launch.
struct AcqItem {
  AcqDev dev;                // dev.sum_var unused: the sum comes from seg_part[seg0, seg1)
  PassArgs args;
  int nblocks;               // blocks serving this space
  int seg0, seg1;            // its tensor-core segments
};

// One observation update of a batch (the arguments of the single-space launch).
// The new observation as the update reads it: its index and value, the fit's
// standardization, and the point's value indices, coordinates and distance
// table metadata, all formed on the host (the k phase starts without a chain
// of dependent loads).
struct ObsNew {
  long long idx;
  double y_raw, y_mean, inv_std;
  int32_t a[BO_MAX_PARAMS];     // value index of parameter p
  int32_t off[BO_MAX_PARAMS];   // offset of parameter p's table of squared differences
  int32_t m[BO_MAX_PARAMS];     // value count of parameter p
  double x[BO_MAX_PARAMS];      // coordinate of parameter p
};
struct ObsItem {
  DevView v;
  int n;                     // observations fitted before this one
  ObsNew o;
};
// Doubles of DevView::upart for n_max observations: three shares (l.l, k.a,
// k.b) per 8-row block of the l phase, two (w.(y - y0), w.1) per 32 x 64
// block of the w phase.
inline size_t update_part_count(int n_max) {
  const size_t nl = ((size_t)n_max + 7) / 8, nw = (((size_t)n_max + 31) / 32) * (((size_t)n_max + 63) / 64);
  return 3 * nl + 2 * nw;
}
struct ObsBlock {
  int item, local;           // space and its block index within one phase
};
struct VisitItem {
  uint32_t* visited;         // a non-finite observation only sets its evaluated bit
  long long idx;
};

// ---- launchers (each returns the number of kernels it launched, or -1) ----
// Self-tests of the bounded device waits (each returns 1 when launched).
// exp_neg of the FP64 pass and CUDA's exp(-t) for n arguments (device arrays).
int launch_selftest_exp(const double* t, double* out, double* ref, int n, cudaStream_t s);
int launch_selftest_mbar(int32_t* status, int* abort_flag, cudaStream_t s);
int launch_selftest_grid(DevStats* st, cudaStream_t s);
int launch_observe_update(bool cooperative, const DevView& v, int n, const ObsNew& o, cudaStream_t s);
int launch_set_visited(const DevView& v, int64_t idx, cudaStream_t s);
// Block tables of the batched update phases k, l, w, beta (concatenated) for spaces with
// n[i] observations fitted before their new one; counts[] receives each phase's block count.
void obs_batch_blocks(const int* n, int count, std::vector<ObsBlock>* blocks, int counts[5]);
int launch_observe_batch(const ObsItem* items, int count, const ObsBlock* blocks, const int counts[5],
                         const VisitItem* visits, int n_visits, bool tc, cudaStream_t s);
int launch_predict_f64(const DevView& v, int n, int64_t n_unvisited, cudaStream_t s);
int launch_predict_tc(const DevView& v, int n, int64_t n_unvisited, cudaStream_t s);
// CTAs of a single-space prediction launch: each writes one per-CTA variance
// sum to DevView::partial, which the acquisition adds up.
int predict_f64_grid(const DevView& v, int n);
int predict_tc_grid(const DevView& v);
// The tensor-core pass with the acquisition of `a` as its tail (one
// cooperative launch writing the pass result); -2 if the device does not
// launch it cooperatively (then predict + acquire as two launches).
int launch_predict_acquire_tc(const DevView& v, int n, const PassArgs& a, cudaStream_t s);
TcSess tc_session(const DevView& v, int n);
int tc_dim_bucket(int d);
// Cost-balanced segments of `count` spaces over `grid` CTAs; returns the segment count.
int tc_plan_batch(const TcSess* sess, int count, int dmax, int grid, std::vector<TcSeg>* segs,
                  std::vector<int>* seg_begin);
int launch_predict_tc_batch(const TcBatchLaunch& L, cudaStream_t s);
// Autotuner hooks: launches on this thread use `shape` while it is forced
// (nullptr ends it); a stored shape applies to every later launch of its key.
void tc_force_shape(const TcShape* shape);
void tc_store_shape(int precision, double nu, int dmax, int n_pad, bool batched, const TcShape& shape);
// The stored shape of a key, if the autotuner has chosen one.
bool tc_stored_shape(int precision, double nu, int dmax, int n_pad, bool batched, TcShape* shape);
int launch_acquire(const DevView& v, const PassArgs& a, cudaStream_t s);
int launch_acquire(const AcqDev& v, const PassArgs& a, bool f64, cudaStream_t s);
// Blocks of an acquisition pass over n_cand candidates, per_thread candidates
// per thread (a single space: few, so that the pass fills the GPU; a batch of
// spaces: many, the spaces together fill it), at most max_blocks.
int acquire_grid(int64_t n_cand, int max_blocks, int per_thread = 16);
int launch_acquire_batch(const AcqItem* items, const int* block_item, const int* block_local,
                         const double* seg_part, int total_blocks, bool f64, cudaStream_t s);

// Scale of the FP32 coordinate copies: distances in these units are
// u = sqrt(2 nu) r / l * log2(e), so e^-t = 2^-u with t = sqrt(2 nu) r / l.
inline double coord_scale(double nu, double lengthscale) {
  return 1.4426950408889634 * __builtin_sqrt(2.0 * nu) / lengthscale;
}

// Element width in bytes of the reduced-precision L^-1 copy and of the K*
// operand (4 for the TF32 forms, 2 for the 16-bit forms), and the number of
// parts of each (hi and lo, or a single TF32 part).
__host__ __device__ constexpr int split_elem_bytes(int precision) {
  return precision == BO_PREC_TF32 || precision == BO_PREC_TF32X3 ? 4 : 2;
}
__host__ __device__ constexpr int split_parts(int precision) { return precision == BO_PREC_TF32 ? 1 : 2; }

// Record an error for bo_last_error() on this thread; returns code.
int report_error(int code, const char* msg);

// Size in bytes of the reduced-precision chunked L^-1 copy (one of hi / lo).
size_t lsplit_bytes(int n_max, int precision);

}  // namespace bo
