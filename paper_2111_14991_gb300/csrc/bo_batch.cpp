// Batched observe / suggest over many spaces: the observation updates of all
// spaces in five launches, and the prediction passes of all spaces in one
// persistent tensor-core launch plus one acquisition launch, with one copy of
// all pass results back.  The host logic per space (checks, selection of
// acquisition functions, queues) is the same as bo_observe / bo_suggest.
#include <cstdlib>
#include <cstring>
#include <new>

#include "bo_space_impl.h"

using namespace bo;
using namespace bo::host;

struct bo_batch {
  std::vector<bo_space*> sp;
  int device = 0;
  cudaStream_t user = nullptr;   // the spaces' stream
  cudaStream_t bs = nullptr;     // the batch's own stream (graphs are captured on it)
  cudaEvent_t ev_user = nullptr, ev_done = nullptr;
  int precision = 0;
  double nu = 1.5;
  int dmax = 4, grid = 0, n_pad_cap = 32;
  int acq_cap = 0;               // acquisition blocks for all spaces at once
  int seg_cap = 0;               // segments of a tensor-core plan
  int obs_block_cap = 0;
  // device memory (one allocation) and its pinned host mirror for the uploads
  void* dev = nullptr;
  size_t dev_bytes = 0;
  uint8_t* stage = nullptr;      // pinned
  size_t off_sess = 0, off_segs = 0, off_seg_begin = 0, off_acq = 0, off_blk_item = 0, off_blk_local = 0;
  size_t pass_upload = 0;        // bytes [0, pass_upload) are the pass's upload
  size_t off_obs = 0, off_obs_blocks = 0, off_visits = 0, obs_upload_end = 0;
  size_t off_seg_part = 0, off_acq_partial = 0, off_counters = 0, off_results = 0, off_status = 0;
  bo_pass_result* h_results = nullptr;   // pinned copy of [off_results, off_status + 16)
  bo_space* owner = nullptr;             // whose allocator provided `dev`
  // graph of the pass (upload, two kernels, download) for one shape
  cudaGraphExec_t gexec = nullptr;
  std::vector<long long> gkey, seen_key;
  bool use_graph = true;
  int64_t launches = 0;
  TcBatchLaunch last{};          // the last batched prediction launch (for the autotuner)
  bool have_last = false;
};

namespace {

template <typename T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<uint8_t*>(base) + off);
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int phase_blocks_max(int n_max) {
  const int m = n_max - 1;   // the largest n an update can see before its new row
  return (m + 31) / 32 + 1 + (m + 7) / 8 + ((m + 31) / 32) * ((m + 63) / 64) + 2 * ((m + 8) / 8);
}

void release_batch(bo_batch* b) {
  if (b->bs) cudaStreamSynchronize(b->bs);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->dev) {
    const bo_space* o = b->owner;
    if (o && o->desc.alloc) {
      if (o->desc.free) o->desc.free(b->dev, b->dev_bytes, (void*)o->stream, o->desc.alloc_ctx);
    } else {
      cudaFreeAsync(b->dev, b->bs);
    }
  }
  if (b->stage) cudaFreeHost(b->stage);
  if (b->h_results) cudaFreeHost(b->h_results);
  if (b->ev_user) cudaEventDestroy(b->ev_user);
  if (b->ev_done) cudaEventDestroy(b->ev_done);
  if (b->bs) cudaStreamDestroy(b->bs);
}

// order the batch stream after the spaces' stream, and the spaces' stream after the batch
int begin_on_batch_stream(bo_batch* b) {
  BO_CUDA(cudaEventRecord(b->ev_user, b->user));
  BO_CUDA(cudaStreamWaitEvent(b->bs, b->ev_user, 0));
  return BO_OK;
}

int end_on_batch_stream(bo_batch* b) {
  BO_CUDA(cudaEventRecord(b->ev_done, b->bs));
  BO_CUDA(cudaStreamWaitEvent(b->user, b->ev_done, 0));
  return BO_OK;
}

// enqueue upload, kernels and download of one batched pass on the batch stream
int enqueue_pass(bo_batch* b, int count, int n_pad_max, int nsegs, int total_blocks) {
  BO_CUDA(cudaMemcpyAsync(b->dev, b->stage, b->pass_upload, cudaMemcpyHostToDevice, b->bs));
  TcBatchLaunch L{};
  L.sess = at<TcSess>(b->dev, b->off_sess);
  L.segs = at<TcSeg>(b->dev, b->off_segs);
  L.seg_begin = at<int>(b->dev, b->off_seg_begin);
  L.seg_part = at<double>(b->dev, b->off_seg_part);
  L.status = at<int32_t>(b->dev, b->off_status);
  L.count = count;
  L.grid = b->grid;
  L.precision = b->precision;
  L.dmax = b->dmax;
  L.n_pad_max = n_pad_max;
  L.nu = b->nu;
  (void)nsegs;
  b->last = L;
  b->have_last = true;
  if (launch_predict_tc_batch(L, b->bs) < 0) return fail(BO_ERR_CUDA, "batched prediction launch failed");
  if (launch_acquire_batch(at<AcqItem>(b->dev, b->off_acq), at<int>(b->dev, b->off_blk_item),
                           at<int>(b->dev, b->off_blk_local), at<double>(b->dev, b->off_seg_part), total_blocks,
                           false, b->bs) < 0)
    return fail(BO_ERR_CUDA, "batched acquisition launch failed");
  (void)count;
  BO_CUDA(cudaMemcpyAsync(b->h_results, at<void>(b->dev, b->off_results), b->off_status + 16 - b->off_results,
                          cudaMemcpyDeviceToHost, b->bs));
  return BO_OK;
}

}  // namespace

extern "C" {

int bo_batch_create(bo_space* const* spaces, int32_t count, bo_batch** out) {
  if (!spaces || !out || count < 1) return fail(BO_ERR_ARG, "null argument or empty batch");
  *out = nullptr;
  bo_batch* b = new (std::nothrow) bo_batch();
  if (!b) return fail(BO_ERR_NOMEM, "host allocation failed");
  b->sp.assign(spaces, spaces + count);
  const bo_space* s0 = spaces[0];
  for (int i = 0; i < count; ++i) {
    const bo_space* s = spaces[i];
    if (!s) { delete b; return fail(BO_ERR_ARG, "space %d is null", i); }
    if (s->device != s0->device || s->stream != s0->stream || s->desc.precision != s0->desc.precision ||
        s->desc.nu != s0->desc.nu) {
      delete b;
      return fail(BO_ERR_ARG, "space %d differs from space 0 in device, stream, precision or nu", i);
    }
  }
  b->device = s0->device;
  b->user = s0->stream;
  b->precision = s0->desc.precision;
  b->nu = s0->desc.nu;
  b->use_graph = getenv("BO_NO_GRAPH") == nullptr;
  cudaSetDevice(b->device);
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  b->grid = sms;
  int dmax_d = 1;
  for (int i = 0; i < count; ++i) {
    const bo_space* s = spaces[i];
    dmax_d = std::max(dmax_d, s->d);
    b->n_pad_cap = std::max(b->n_pad_cap, s->v.n_max);
    b->acq_cap += acquire_grid(s->N, 4 * sms);
    b->obs_block_cap += phase_blocks_max(s->v.n_max);
  }
  b->dmax = tc_dim_bucket(dmax_d);
  b->seg_cap = count + b->grid;
  // upload region of a pass, then of an observe, then device-only arrays
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = align_up(off + bytes, 256); return o; };
  b->off_sess = take(sizeof(TcSess) * count);
  b->off_segs = take(sizeof(TcSeg) * b->seg_cap);
  b->off_seg_begin = take(sizeof(int) * (b->grid + 1));
  b->off_acq = take(sizeof(AcqItem) * count);
  b->off_blk_item = take(sizeof(int) * b->acq_cap);
  b->off_blk_local = take(sizeof(int) * b->acq_cap);
  b->pass_upload = off;
  b->off_obs = take(sizeof(ObsItem) * count);
  b->off_obs_blocks = take(sizeof(ObsBlock) * b->obs_block_cap);
  b->off_visits = take(sizeof(VisitItem) * count);
  b->obs_upload_end = off;
  b->off_seg_part = take(sizeof(double) * 4 * b->seg_cap);
  b->off_acq_partial = take(sizeof(TopEntry) * 9 * b->acq_cap);
  b->off_counters = take(sizeof(unsigned) * count);
  b->off_results = take(sizeof(bo_pass_result) * count);
  b->off_status = take(16);                 // right after the results: one download
  b->dev_bytes = off;
  cudaError_t e = cudaStreamCreateWithFlags(&b->bs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_user, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming);
  b->owner = spaces[0];
  if (e == cudaSuccess) {
    if (s0->desc.alloc) {
      b->dev = s0->desc.alloc(b->dev_bytes, (void*)s0->stream, s0->desc.alloc_ctx);
      if (!b->dev) e = cudaErrorMemoryAllocation;
      else e = cudaStreamSynchronize(s0->stream);   // the memory is ready for the batch stream
    } else {
      e = cudaMallocAsync(&b->dev, b->dev_bytes, b->bs);
    }
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(b->dev, 0, b->dev_bytes, b->bs);
  if (e == cudaSuccess) e = cudaMallocHost(&b->stage, b->obs_upload_end);
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_results, b->off_status + 16 - b->off_results);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->bs);
  if (e != cudaSuccess) {
    const int rc = cuda_fail(e, "batch allocation");
    release_batch(b);
    delete b;
    return rc;
  }
  *out = b;
  return BO_OK;
}

int bo_batch_destroy(bo_batch* b) {
  if (!b) return fail(BO_ERR_ARG, "null batch");
  cudaSetDevice(b->device);
  release_batch(b);
  delete b;
  return BO_OK;
}

int bo_batch_observe(bo_batch* b, const int64_t* idx, const double* values, int32_t* status_out) {
  if (!b || !idx || !values) return fail(BO_ERR_ARG, "null argument");
  cudaSetDevice(b->device);
  const int count = (int)b->sp.size();
  BO_CUDA(cudaStreamSynchronize(b->bs));   // the staging buffer is free again
  ObsItem* items = at<ObsItem>(b->stage, b->off_obs);
  VisitItem* visits = at<VisitItem>(b->stage, b->off_visits);
  std::vector<int> n_before;
  int n_items = 0, n_visits = 0, first_err = BO_OK;
  for (int i = 0; i < count; ++i) {
    bo_space* s = b->sp[i];
    int rc = BO_OK;
    if (idx[i] >= 0) {
      if (s->poisoned) {
        rc = fail(s->poisoned, "space %d is unusable after an earlier numeric failure", i);
      } else {
        bool fit = false;
        int nb = 0;
        double mean = 0.0, sd = 1.0;
        rc = observe_host(s, idx[i], values[i], &fit, &nb, &mean, &sd);
        if (rc == BO_OK && fit) {
          ObsItem& it = items[n_items++];
          it.v = s->v;
          it.n = nb;
          make_obs_new(s, idx[i], values[i], mean, sd, &it.o);
          n_before.push_back(nb);
        } else if (rc == BO_OK) {
          visits[n_visits].visited = s->v.visited;
          visits[n_visits].idx = idx[i];
          ++n_visits;
        }
      }
    }
    if (status_out) status_out[i] = rc;
    if (rc != BO_OK && first_err == BO_OK) first_err = rc;
  }
  std::vector<ObsBlock> blocks;
  int counts[5] = {0, 0, 0, 0, 0};
  obs_batch_blocks(n_before.data(), n_items, &blocks, counts);
  if ((int)blocks.size() > b->obs_block_cap) return fail(BO_ERR_STATE, "update block table overflow");
  std::memcpy(at<void>(b->stage, b->off_obs_blocks), blocks.data(), sizeof(ObsBlock) * blocks.size());
  int rc = begin_on_batch_stream(b);
  if (rc != BO_OK) return rc;
  BO_CUDA(cudaMemcpyAsync(at<void>(b->dev, b->off_obs), b->stage + b->off_obs, b->obs_upload_end - b->off_obs,
                          cudaMemcpyHostToDevice, b->bs));
  const int k = launch_observe_batch(at<ObsItem>(b->dev, b->off_obs), n_items, at<ObsBlock>(b->dev, b->off_obs_blocks),
                                     counts, at<VisitItem>(b->dev, b->off_visits), n_visits,
                                     b->precision != BO_PREC_FP64, b->bs);
  if (k < 0) return fail(BO_ERR_CUDA, "batched update launch failed");
  b->launches += k;
  rc = end_on_batch_stream(b);
  if (rc != BO_OK) return rc;
  return first_err;
}

int bo_batch_suggest(bo_batch* b, int64_t* idx_out, int32_t* status_out, bo_suggest_info* info_out) {
  return bo_batch_suggest_some(b, nullptr, idx_out, status_out, info_out);
}

int bo_batch_suggest_some(bo_batch* b, const uint8_t* want, int64_t* idx_out, int32_t* status_out,
                          bo_suggest_info* info_out) {
  if (!b || !idx_out) return fail(BO_ERR_ARG, "null argument");
  cudaSetDevice(b->device);
  const int count = (int)b->sp.size();
  std::vector<int> pass;                     // spaces that need a prediction pass
  std::vector<PassArgs> args;
  int first_err = BO_OK;
  auto set_status = [&](int i, int rc) {
    if (status_out) status_out[i] = rc;
    if (rc != BO_OK && first_err == BO_OK) first_err = rc;
  };
  for (int i = 0; i < count; ++i) {
    bo_space* s = b->sp[i];
    idx_out[i] = -1;
    if (status_out) status_out[i] = BO_OK;
    if (want && !want[i]) continue;
    if (s->poisoned) { set_status(i, fail(s->poisoned, "space %d is unusable", i)); continue; }
    bool need = false;
    int rc = suggest_begin(s, &idx_out[i], info_out ? &info_out[i] : nullptr, &need);
    if (rc == BO_OK && need) {
      PassArgs a;
      rc = prepare_pass(s, s->sel.active, 0, &a);
      if (rc == BO_OK) { pass.push_back(i); args.push_back(a); }
    }
    set_status(i, rc);
  }
  if (pass.empty()) return first_err;
  const int np = (int)pass.size();
  if (b->precision == BO_PREC_FP64) {         // no batched FP64 kernel: one pass per space
    for (int k = 0; k < np; ++k) {
      bo_space* s = b->sp[pass[k]];
      int kk = launch_predict_f64(s->v, s->n_fit, args[k].n_unvisited, s->stream);
      int k2 = kk < 0 ? -1 : launch_acquire(s->v, args[k], s->stream);
      if (kk < 0 || k2 < 0) return fail(BO_ERR_CUDA, "prediction launch failed");
      s->launches += kk + k2;
      BO_CUDA(cudaMemcpyAsync(s->host_result, s->v.results, sizeof(bo_pass_result), cudaMemcpyDeviceToHost,
                              s->stream));
    }
    BO_CUDA(cudaStreamSynchronize(b->user));
    for (int k = 0; k < np; ++k) {
      const int i = pass[k];
      set_status(i, suggest_finish(b->sp[i], *b->sp[i]->host_result, &idx_out[i], info_out ? &info_out[i] : nullptr));
    }
    return first_err;
  }
  // ---- plan the batched pass on the host
  BO_CUDA(cudaStreamSynchronize(b->bs));     // the staging buffer is free again
  TcSess* sess = at<TcSess>(b->stage, b->off_sess);
  int n_pad_max = 32;
  for (int k = 0; k < np; ++k) {
    bo_space* s = b->sp[pass[k]];
    sess[k] = tc_session(s->v, s->n_fit);
    n_pad_max = std::max(n_pad_max, sess[k].n_pad);
  }
  std::vector<TcSeg> segs;
  std::vector<int> seg_begin;
  const int nsegs = tc_plan_batch(sess, np, b->dmax, b->grid, &segs, &seg_begin);
  if (nsegs > b->seg_cap) return fail(BO_ERR_STATE, "segment table overflow");
  std::memcpy(at<void>(b->stage, b->off_segs), segs.data(), sizeof(TcSeg) * segs.size());
  std::memcpy(at<void>(b->stage, b->off_seg_begin), seg_begin.data(), sizeof(int) * seg_begin.size());
  AcqItem* acq = at<AcqItem>(b->stage, b->off_acq);
  int* blk_item = at<int>(b->stage, b->off_blk_item);
  int* blk_local = at<int>(b->stage, b->off_blk_local);
  int total_blocks = 0, g = 0;
  size_t part_off = 0;
  for (int k = 0; k < np; ++k) {
    bo_space* s = b->sp[pass[k]];
    AcqItem& it = acq[k];
    it.nblocks = acquire_grid(s->N, 4 * b->grid);
    it.dev.mu = s->v.mu;
    it.dev.var = s->v.var;
    it.dev.visited = s->v.visited;
    it.dev.N = s->N;
    it.dev.sum_var = nullptr;
    it.dev.var_s = &s->v.stats->var_s;
    it.dev.status_in = &s->v.stats->status;
    it.dev.partial = at<TopEntry>(b->dev, b->off_acq_partial) + part_off;
    it.dev.counter = at<unsigned>(b->dev, b->off_counters) + k;
    it.dev.max_blocks = it.nblocks;
    it.dev.result = at<bo_pass_result>(b->dev, b->off_results) + k;
    it.args = args[k];
    it.seg0 = g;
    while (g < nsegs && segs[g].sess == k) ++g;
    it.seg1 = g;
    for (int q = 0; q < it.nblocks; ++q) {
      blk_item[total_blocks] = k;
      blk_local[total_blocks] = q;
      ++total_blocks;
    }
    part_off += (size_t)it.nblocks * 9;
  }
  if (total_blocks > b->acq_cap) return fail(BO_ERR_STATE, "acquisition block table overflow");
  // ---- run it: directly the first time a shape is seen, from a captured graph after that
  std::vector<long long> key = {np, n_pad_max, total_blocks, b->dmax};
  for (int k = 0; k < np; ++k) key.push_back(pass[k]);
  int rc = begin_on_batch_stream(b);
  if (rc != BO_OK) return rc;
  if (b->use_graph && b->gexec && key == b->gkey) {
    BO_CUDA(cudaGraphLaunch(b->gexec, b->bs));
  } else if (b->use_graph && key == b->seen_key) {
    cudaGraph_t graph = nullptr;
    BO_CUDA(cudaStreamBeginCapture(b->bs, cudaStreamCaptureModeThreadLocal));
    rc = enqueue_pass(b, np, n_pad_max, nsegs, total_blocks);
    const cudaError_t ce = cudaStreamEndCapture(b->bs, &graph);
    if (rc != BO_OK) return rc;
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate");
    b->gkey = key;
    BO_CUDA(cudaGraphLaunch(b->gexec, b->bs));
  } else {
    rc = enqueue_pass(b, np, n_pad_max, nsegs, total_blocks);
    if (rc != BO_OK) return rc;
    b->seen_key = key;
  }
  b->launches += 2;
  rc = end_on_batch_stream(b);
  if (rc != BO_OK) return rc;
  BO_CUDA(cudaStreamSynchronize(b->bs));
  const int32_t batch_status =
      *reinterpret_cast<const int32_t*>(reinterpret_cast<const uint8_t*>(b->h_results) + (b->off_status - b->off_results));
  for (int k = 0; k < np; ++k) {
    const int i = pass[k];
    bo_pass_result r = b->h_results[k];
    if (batch_status != BO_OK && r.status == BO_OK) r.status = batch_status;
    b->sp[i]->launches += 2;
    set_status(i, suggest_finish(b->sp[i], r, &idx_out[i], info_out ? &info_out[i] : nullptr));
  }
  return first_err;
}

int bo_batch_autotune(bo_batch* b, int32_t reps, bo_tune_result* out) {
  if (!b) return fail(BO_ERR_ARG, "null batch");
  if (b->precision == BO_PREC_FP64) return fail(BO_ERR_ARG, "the FP64 pass has no tensor-core shapes");
  if (!b->have_last) return fail(BO_ERR_STATE, "run bo_batch_suggest once before tuning");
  cudaSetDevice(b->device);
  BO_CUDA(cudaStreamSynchronize(b->bs));
  const TcBatchLaunch L = b->last;
  const int rc = autotune_shapes(b->bs, reps, b->precision, L.nu, L.dmax, L.n_pad_max, true,
                                 [&] { return launch_predict_tc_batch(L, b->bs); }, out);
  b->gkey.clear();               // captured graphs hold the old shape
  b->seen_key.clear();
  return rc;
}

int bo_batch_launch_count(const bo_batch* b, int64_t* out) {
  if (!b || !out) return fail(BO_ERR_ARG, "null argument");
  *out = b->launches;
  return BO_OK;
}

}  // extern "C"
