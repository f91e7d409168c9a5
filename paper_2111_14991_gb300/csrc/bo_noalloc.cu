// Acquisition + masked top-k on caller-owned arrays, with no allocation.
//
// The acquisition kernel needs scratch for one partial top-k list per block
// and a last-block counter.  bo_suggest takes them from the space's device
// buffers; here they live in one file-scope device array of fixed size, so a
// caller that cannot allocate device memory can still score a posterior it
// already holds.  Host code reaches the array through its device address,
// looked up once per device with cudaGetSymbolAddress.
#include <cstdio>
#include <mutex>

#include "bo_internal.h"

namespace bo {
namespace {

// The array holds the partial top-k lists of kNoallocBlocks blocks, the most
// one call launches; the blocks stride over the candidates, so the array does
// not bound n_cand.  BO_NOALLOC_MAX_CAND bounds the work of one call instead:
// at the cap each thread of the 1,024 blocks of 256 threads scores 16 candidates.
constexpr int kNoallocBlocks = 1024;
constexpr int64_t kMaxCandPerThread = 16;

struct NoallocScratch {
  unsigned int counter;                        // last-block counter, zero before a launch
  int32_t pad0;
  double sum_var;                              // inputs the kernel reads through pointers
  double var_s;
  double pad1[5];
  TopEntry partial[kNoallocBlocks * 9];        // [block][af][rank]
};
static_assert(sizeof(NoallocScratch) == 147520, "documented scratch size");
static_assert((int64_t)kNoallocBlocks * 256 * kMaxCandPerThread == BO_NOALLOC_MAX_CAND, "documented limit");

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

std::mutex g_lookup_mu;
NoallocScratch* g_scratch_addr[kMaxDevices] = {};

__global__ void noalloc_prepare(NoallocScratch* s, double sum_var, double var_s) {
  s->counter = 0;
  s->sum_var = sum_var;
  s->var_s = var_s;
}

// Device address of the scratch array on the current device (set up on first use).
NoallocScratch* scratch_on_current_device(int* err) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *err = BO_ERR_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_lookup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      *err = BO_ERR_CUDA;
      return nullptr;
    }
    g_scratch_addr[dev] = static_cast<NoallocScratch*>(p);
  }
  return g_scratch_addr[dev];
}

}  // namespace
}  // namespace bo

using namespace bo;

extern "C" int bo_acquire_noalloc(const void* mu, const void* var, const uint32_t* visited, int32_t f64,
                                  const bo_acq_params* p, bo_pass_result* result, void* stream) {
  if (!mu || !var || !visited || !p || !result) return report_error(BO_ERR_ARG, "null argument");
  if (p->n_cand < 1) return report_error(BO_ERR_ARG, "n_cand must be positive");
  if (p->n_cand > BO_NOALLOC_MAX_CAND) {
    char msg[160];
    snprintf(msg, sizeof msg, "n_cand = %lld exceeds the %d candidates the fixed scratch serves",
             (long long)p->n_cand, BO_NOALLOC_MAX_CAND);
    return report_error(BO_ERR_CAPACITY, msg);
  }
  if (p->n_af < 1 || p->n_af > 3 || p->n_unvisited < 0 || p->n_unvisited > p->n_cand)
    return report_error(BO_ERR_ARG, "bad n_af or n_unvisited");
  for (int q = 0; q < p->n_af; ++q)
    if (p->af[q] < BO_AF_EI || p->af[q] > BO_AF_LCB) return report_error(BO_ERR_ARG, "bad af id");
  if (p->explore != BO_EXPLORE_CV && p->explore != BO_EXPLORE_CONST)
    return report_error(BO_ERR_ARG, "explore must be BO_EXPLORE_CV or BO_EXPLORE_CONST");
  if (p->explore == BO_EXPLORE_CV && !(p->fplus_raw > 0.0 && p->mu_s_raw > 0.0))
    return report_error(BO_ERR_NOT_POSITIVE, "contextual variance needs f+ > 0 and mu_s > 0");
  int err = BO_OK;
  NoallocScratch* s = scratch_on_current_device(&err);
  if (!s) return report_error(err, "cudaGetSymbolAddress of the acquisition scratch failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  noalloc_prepare<<<1, 1, 0, st>>>(s, p->sum_var, p->mean_var_s);
  if (cudaGetLastError() != cudaSuccess) return report_error(BO_ERR_CUDA, "scratch preparation launch failed");
  PassArgs a{};
  a.n = p->n_fit;
  a.n_unvisited = p->n_unvisited;
  a.n_af = p->n_af;
  for (int q = 0; q < 3; ++q) a.af[q] = q < p->n_af ? p->af[q] : 0;
  a.k = p->n_af;
  a.explore = p->explore;
  a.lambda_const = p->lambda_const;
  a.fplus_t = p->fplus;
  a.fplus_raw = p->fplus_raw;
  a.mu_s_raw = p->mu_s_raw;
  a.first_pass = p->mean_var_s > 0.0 ? 0 : 1;
  AcqDev ad;
  ad.mu = mu;
  ad.var = var;
  ad.visited = visited;
  ad.N = p->n_cand;
  ad.sum_var = &s->sum_var;
  ad.var_s = &s->var_s;
  ad.status_in = nullptr;
  ad.partial = s->partial;
  ad.counter = &s->counter;
  ad.max_blocks = kNoallocBlocks;
  ad.result = result;
  if (launch_acquire(ad, a, f64 != 0, st) < 0) return report_error(BO_ERR_CUDA, "acquisition launch failed");
  return BO_OK;
}
