// Prediction pass on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Same mathematics as the FP64 pass (paper Sec. III-B, III-G): for every
// candidate c, v = L^-1 k*(c), var = k(0) - |v|^2, mu = v . beta.  Here the
// contraction V = K* L^-T runs on the tensor cores with FP32 accumulation in
// tensor memory, with the operands split to recover precision:
//   FP16X3 / BF16X3: K* = Kh + Kl and L^-1 = Lh + Ll (per-row power-of-two
//     scaled), V ~ Kh Lh + Kh Ll + Kl Lh  (three MMAs per k-step)
//   TF32: one MMA on TF32-rounded operands.
// The FP64 L^-1, beta and the update stay in FP64 (bo_update.cu), which
// writes the split copy of each new row once.
//
// CTA organisation (persistent, one CTA per SM, 128 candidates per tile):
//   warps 0-15   produce K* chunks: thread (row = t % 128, quarter = t / 128)
//                evaluates the Matern covariance of its candidate against a
//                quarter of the chunk's observations, splits it and stores it
//                in the K-major core-matrix layout.
//   warps 16-19  drain the accumulator (TMEM lane = row): sum acc_k^2 q_k and
//                acc_k b_k, write mu and var.  With n <= 256 the accumulator
//                is double-buffered, so a tile's MMAs overlap the previous
//                tile's drain.
//   warp 20      issues the MMAs (one thread) and owns the TMEM allocation.
//   warp 21      streams the L^-1 chunks with bulk copies (one thread), in
//                pieces of at most 256 rows: a 4-slot ring, or all pieces of a
//                tile kept resident when they fit (n <= ~256), loaded once.
// K chunk c covers observations j in [c CW, (c+1) CW); only output columns
// k >= c CW receive it (L^-1 is lower triangular), so the MMA N range
// shrinks along the chunks.  Every wait is bounded in time: on expiry the
// CTA records BO_ERR_TIMEOUT, drains its own copies / MMAs and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "bo_internal.h"

namespace bo {

namespace {

constexpr int kRows = 128;              // candidates per tile (MMA M)
constexpr int kProducerWarps = 16;
constexpr int kEpiWarp0 = 16;           // warps 16-19
constexpr int kMmaWarp = 20;
constexpr int kLoadWarp = 21;
constexpr int kThreads = 704;
constexpr int kPartBytes = kRows * kChunkBytes;   // one split part of an A stage: 8 KB
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s
constexpr int kPieceRows = 256;         // rows of L^-1 per B piece (= max MMA N)
constexpr int kMaxBSlots = 16;

struct TcParams {
  DevView v;
  int n, n_pad, chunks, cw, parts, stages_a;
  int tmem_cols;             // columns of one accumulator buffer
  int acc_stages;            // 1 or 2 accumulator buffers
  int num_tiles;
  // B (the split L^-1 chunks) in pieces of <= 256 rows: either a ring of
  // b_slots fixed-size slots, or every piece of a tile resident (loaded once)
  int b_resident, b_slots;
  size_t off_b, b_slot_bytes, off_x, off_q, off_bar;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
  return ok != 0;
}

// As mbar_test, but the thread may sleep up to ~0.1 ms for the phase instead
// of returning at once (waiting warps then leave the issue slots to others).
__device__ __forceinline__ bool mbar_test_sleep(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity), "r"(100000u) : "memory");
  return ok != 0;
}

// Bounded wait on a phase; false if it expired or another thread aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          int32_t* status) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  while (!mbar_test_sleep(bar, parity)) {
    if (*abort_flag) return false;
    if (now_ns() - t0 > kWaitNs) {
      *abort_flag = 1;
      atomicExch(status, BO_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// K-major, no-swizzle shared-memory matrix descriptor: core matrices of
// 8 rows x 16 bytes, `lbo` bytes apart along K, `sbo` bytes apart along M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor: D = F32, A/B format `fmt` (f16 0, bf16 1, tf32 2), K-major.
__host__ __device__ __forceinline__ uint32_t instr_desc(int fmt, int m, int n) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

template <int MODE>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (MODE == BO_PREC_TF32) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* r) {
  uint32_t u[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
        "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]),
        "=r"(u[15]), "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]),
        "=r"(u[22]), "=r"(u[23]), "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]),
        "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) r[i] = __uint_as_float(u[i]);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Packed pairs of FP32 (Blackwell f32x2 ALU): element 0 in the low word.
__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ void lds2x64(uint32_t addr, uint64_t& a, uint64_t& b) {
  asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(addr));
}

// Matern covariance in FP32 from u^2, the squared distance in units where
// u = t log2(e), t = sqrt(2 nu) r / l (the coordinate tables carry the scale):
// u from the hardware reciprocal square root and one Newton step, e^-t = 2^-u
// from the hardware exp2, then (1 + t) e^-t or (1 + t + t^2/3) e^-t.
template <bool NU52>
__device__ __forceinline__ float matern_u2(float u2) {
  u2 = fmaxf(u2, 1e-30f);
  const float rs = rsqrtf(u2);
  float u = u2 * rs;
  u = fmaf(fmaf(-u, u, u2), 0.5f * rs, u);
  const float e = ex2_approx(-u);
  const float t = u * 0.6931471805599453f;
  if constexpr (NU52)
    return fmaf(t * e, fmaf(t, 1.0f / 3.0f, 1.0f), e);
  else
    return fmaf(t, e, e);
}

// pack two values of the split parts: hi and lo 16-bit words, or one tf32 word
template <int MODE>
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  if constexpr (MODE == BO_PREC_FP16X3) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  }
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return u;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}

template <int MODE, int DMAX, bool NU52>
__global__ void __launch_bounds__(kThreads, 1) predict_tc_kernel(const __grid_constant__ TcParams P) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const DevView& v = P.v;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int d = v.d;
  const int n_pad = P.n_pad, chunks = P.chunks, cw = P.cw, parts = P.parts, SA = P.stages_a;
  uint8_t* sa = smem;                                   // [SA][parts][8 KB]
  uint8_t* sb = smem + P.off_b;                         // B slots or resident pieces
  float* Xs = reinterpret_cast<float*>(smem + P.off_x); // [DMAX][n_pad], rows >= d zero
  float* Qs = reinterpret_cast<float*>(smem + P.off_q); // [n_pad] 1/s_k^2
  float* Bs = Qs + n_pad;                               // [n_pad] beta_k/s_k
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + P.off_bar);
  uint64_t* a_full = bars;
  uint64_t* a_empty = bars + SA;
  uint64_t* b_full = bars + 2 * SA;                  // [kMaxBSlots]
  uint64_t* b_empty = bars + 2 * SA + kMaxBSlots;    // [kMaxBSlots]
  uint64_t* acc_full = bars + 2 * SA + 2 * kMaxBSlots;       // [2]
  uint64_t* acc_empty = bars + 2 * SA + 2 * kMaxBSlots + 2;  // [2]
  uint64_t* drain = bars + 2 * SA + 2 * kMaxBSlots + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * SA + 2 * kMaxBSlots + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  __shared__ double red[4];   // per epilogue warp
  __shared__ bool s_last;
  int32_t* status = &v.stats->status;

  // ---- setup: barriers, TMEM, observation coordinates, per-row factors
  if (threadIdx.x == 0) {
    for (int s = 0; s < SA; ++s) { mbar_init(&a_full[s], kProducerWarps); mbar_init(&a_empty[s], 1); }
    for (int s = 0; s < kMaxBSlots; ++s) { mbar_init(&b_full[s], 1); mbar_init(&b_empty[s], 1); }
    for (int s = 0; s < 2; ++s) { mbar_init(&acc_full[s], 1); mbar_init(&acc_empty[s], 4); }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(P.tmem_cols * P.acc_stages) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  for (int e = threadIdx.x; e < DMAX * n_pad; e += kThreads) {
    const int p = e / n_pad, j = e - p * n_pad;
    Xs[e] = (j < P.n && p < d) ? v.Xf[(size_t)j * d + p] : 0.0f;
  }
  for (int k = threadIdx.x; k < n_pad; k += kThreads) {
    Qs[k] = k < P.n ? v.rowq[k] : 0.0f;
    Bs[k] = k < P.n ? v.rowb[k] : 0.0f;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  double vsum = 0.0;

  if (warp < kProducerWarps) {
    // ===================== K* producers =====================
    const int row = threadIdx.x & (kRows - 1);
    const int quarter = threadIdx.x >> 7;
    const int jq = cw / 4;                       // observations per thread per chunk: 8 or 4
    const uint32_t a_base = smem_addr(sa);
    const uint32_t xs_base = smem_addr(Xs);
    const uint32_t row_off = (uint32_t)((row >> 3) * (kChunkBytes * 8) + (row & 7) * 16 + quarter * 128);
    bool ok = true;
    int s = 0;
    uint32_t ph = 0;                            // ring slot and its phase
    for (int tile = blockIdx.x; tile < P.num_tiles && ok; tile += gridDim.x) {
      const int64_t cand = (int64_t)tile * kRows + row;
      uint64_t xcp[DMAX];                      // candidate coordinate, twice per word
#pragma unroll
      for (int p = 0; p < DMAX; ++p) {
        const float x = p < d ? v.vtab32[p * 256 + v.codes[(int64_t)p * v.N_pad + cand]] : 0.0f;
        xcp[p] = pk2(x, x);
      }
      for (int c = 0; c < chunks && ok; ++c) {
        const int j0 = c * cw + quarter * jq;
        // K* for this thread's observations, computed before waiting for the ring slot:
        // squared distances two observations per packed instruction
        uint64_t r2p[4] = {0ull, 0ull, 0ull, 0ull};
        const uint32_t xrow = xs_base + (uint32_t)(j0 * 4);
#pragma unroll
        for (int p = 0; p < DMAX; ++p) {
          uint64_t o0, o1;
          lds2x64(xrow + (uint32_t)(p * n_pad * 4), o0, o1);
          uint64_t df = sub2(xcp[p], o0);
          r2p[0] = fma2(df, df, r2p[0]);
          df = sub2(xcp[p], o1);
          r2p[1] = fma2(df, df, r2p[1]);
          if constexpr (MODE != BO_PREC_TF32) {
            lds2x64(xrow + (uint32_t)(p * n_pad * 4 + 16), o0, o1);
            df = sub2(xcp[p], o0);
            r2p[2] = fma2(df, df, r2p[2]);
            df = sub2(xcp[p], o1);
            r2p[3] = fma2(df, df, r2p[3]);
          }
        }
        float kv[8];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          if (2 * w < jq) {
            float a, b;
            upk2(r2p[w], a, b);
            kv[2 * w] = matern_u2<NU52>(a);
            kv[2 * w + 1] = matern_u2<NU52>(b);
          }
        }
        if (!(ok = mbar_wait(&a_empty[s], ph ^ 1, abort_flag, status))) break;
        const uint32_t stage = a_base + (uint32_t)(s * parts * kPartBytes) + row_off;
        if constexpr (MODE == BO_PREC_TF32) {
          st_shared_v4(stage, to_tf32(kv[0]), to_tf32(kv[1]), to_tf32(kv[2]), to_tf32(kv[3]));
        } else {
          uint32_t h[4], l[4];
#pragma unroll
          for (int w = 0; w < 4; ++w) split2<MODE>(kv[2 * w], kv[2 * w + 1], h[w], l[w]);
          st_shared_v4(stage, h[0], h[1], h[2], h[3]);
          st_shared_v4(stage + kPartBytes, l[0], l[1], l[2], l[3]);
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&a_full[s]);
        if (++s == SA) { s = 0; ph ^= 1; }
      }
    }
  } else if (warp < kMmaWarp) {
    // ===================== epilogue: warp e owns TMEM lanes [32e, 32e+32) =====================
    const int e = warp - kEpiWarp0;
    const int row = e * 32 + lane;
    bool ok = true;
    int it = 0;
    for (int tile = blockIdx.x; tile < P.num_tiles && ok; tile += gridDim.x, ++it) {
      const int as = it % P.acc_stages;
      if (!(ok = mbar_wait(&acc_full[as], (it / P.acc_stages) & 1, abort_flag, status))) break;
      tc_fence_after();
      float s2 = 0.0f, sm = 0.0f;
      const uint32_t lane_base = tmem + (uint32_t)(as * P.tmem_cols) + ((uint32_t)(e * 32) << 16);
      for (int k0 = 0; k0 < n_pad; k0 += 32) {
        float acc[32];
        tmem_ld32(lane_base + (uint32_t)k0, acc);
#pragma unroll
        for (int i = 0; i < 32; i += 4) {
          const float4 q = *reinterpret_cast<const float4*>(&Qs[k0 + i]);
          const float4 b = *reinterpret_cast<const float4*>(&Bs[k0 + i]);
          s2 = fmaf(acc[i] * acc[i], q.x, s2);
          s2 = fmaf(acc[i + 1] * acc[i + 1], q.y, s2);
          s2 = fmaf(acc[i + 2] * acc[i + 2], q.z, s2);
          s2 = fmaf(acc[i + 3] * acc[i + 3], q.w, s2);
          sm = fmaf(acc[i], b.x, sm);
          sm = fmaf(acc[i + 1], b.y, sm);
          sm = fmaf(acc[i + 2], b.z, sm);
          sm = fmaf(acc[i + 3], b.w, sm);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[as]);
      const int64_t cand = (int64_t)tile * kRows + row;
      const float var = fmaxf(0.0f, 1.0f - s2);
      static_cast<float*>(v.mu)[cand] = sm;
      static_cast<float*>(v.var)[cand] = var;
      if (cand < v.N && !((v.visited[cand >> 5] >> (cand & 31)) & 1u)) vsum += (double)var;
    }
  } else if (warp == kMmaWarp) {
    // ===================== MMA issuer =====================
    if (lane == 0) {
      const int fmt = MODE == BO_PREC_FP16X3 ? 0 : MODE == BO_PREC_BF16X3 ? 1 : 2;
      const uint32_t a_base = smem_addr(sa), b_base = smem_addr(sb);
      bool ok = true, issued = false;
      int it = 0, sa_i = 0, tb = 0;
      uint32_t pha = 0, phb = 0;
      for (int tile = blockIdx.x; tile < P.num_tiles && ok; tile += gridDim.x, ++it) {
        const int as = it % P.acc_stages;
        if (!(ok = mbar_wait(&acc_empty[as], ((it / P.acc_stages) & 1) ^ 1, abort_flag, status))) break;
        tc_fence_after();
        const uint32_t d_base = tmem + (uint32_t)(as * P.tmem_cols);
        int q = 0;                  // piece index within the tile
        uint32_t packed = 0;        // resident byte offset of piece q
        for (int c = 0; c < chunks && ok; ++c) {
          const int s = sa_i;
          if (!(ok = mbar_wait(&a_full[s], pha, abort_flag, status))) break;
          tc_fence_after();
          const uint32_t a_st = a_base + (uint32_t)(s * parts * kPartBytes);
          for (int r0 = c * cw; r0 < n_pad && ok; r0 += kPieceRows, ++q) {
            const int w = min(kPieceRows, n_pad - r0);          // rows of this piece = MMA N
            const uint32_t part_bytes = (uint32_t)((w >> 3) * 512);
            const int slot = P.b_resident ? q : tb;
            if (!(ok = mbar_wait(&b_full[slot], P.b_resident ? 0u : phb, abort_flag, status))) break;
            tc_fence_after();
            const uint32_t b_st = b_base + (P.b_resident ? packed : (uint32_t)(tb * P.b_slot_bytes));
            const int nsplit = parts == 2 ? 3 : 1;
            for (int sp = 0; sp < nsplit; ++sp) {
              // products (hi, lo), (lo, hi), (hi, hi): small terms first
              const int pa = parts == 2 ? (sp == 1 ? 1 : 0) : 0;
              const int pb = parts == 2 ? (sp == 0 ? 1 : 0) : 0;
              for (int ks = 0; ks < 2; ++ks) {
                const uint64_t ad = smem_desc(a_st + (uint32_t)(pa * kPartBytes + ks * 256), 128, 512);
                const uint64_t bd = smem_desc(b_st + (uint32_t)(pb * part_bytes + ks * 256), 128, 512);
                const uint32_t acc = (c > 0 || sp > 0 || ks > 0) ? 1u : 0u;
                mma<MODE>(d_base + (uint32_t)r0, ad, bd, instr_desc(fmt, kRows, w), acc);
              }
            }
            issued = true;
            packed += part_bytes * (uint32_t)parts;
            if (!P.b_resident) {
              mma_commit(&b_empty[tb]);
              if (++tb == P.b_slots) { tb = 0; phb ^= 1; }
            }
          }
          if (!ok) break;
          mma_commit(&a_empty[s]);
          if (++sa_i == SA) { sa_i = 0; pha ^= 1; }
        }
        if (ok) mma_commit(&acc_full[as]);
      }
      if (issued) {   // every MMA of this CTA has completed before TMEM is released
        mma_commit(drain);
        unsigned long long t0 = now_ns();
        while (!mbar_test(drain, 0) && now_ns() - t0 < kWaitNs) {
        }
      }
    }
  } else if (warp == kLoadWarp) {
    // ===================== L^-1 chunk loader =====================
    if (lane == 0) {
      const int eb = MODE == BO_PREC_TF32 ? 4 : 2;
      const int ccw = kChunkBytes / eb;
      const uint32_t b_base = smem_addr(sb);
      bool ok = true;
      int issued[kMaxBSlots], last_phase[kMaxBSlots];
      for (int t = 0; t < kMaxBSlots; ++t) issued[t] = last_phase[t] = 0;
      int tb = 0;
      uint32_t phb = 0;
      for (int tile = blockIdx.x; tile < P.num_tiles && ok; tile += gridDim.x) {
        int q = 0;
        uint32_t packed = 0;
        for (int c = 0; c < chunks && ok; ++c) {
          const size_t goff = (size_t)kChunkBytes * ((size_t)c * v.n_max - (size_t)ccw * c * (c - 1) / 2);
          for (int r0 = c * ccw; r0 < n_pad && ok; r0 += kPieceRows, ++q) {
            const int w = min(kPieceRows, n_pad - r0);
            const uint32_t bytes = (uint32_t)((w >> 3) * 512);
            const size_t src = goff + (size_t)(r0 - c * ccw) / 8 * 512;
            const int slot = P.b_resident ? q : tb;
            if (!P.b_resident && !(ok = mbar_wait(&b_empty[tb], phb ^ 1, abort_flag, status))) break;
            const uint32_t dst = b_base + (P.b_resident ? packed : (uint32_t)(tb * P.b_slot_bytes));
            mbar_arrive_tx(&b_full[slot], bytes * parts);
            bulk_g2s(dst, v.lsplit_hi + src, bytes, &b_full[slot]);
            if (parts == 2) bulk_g2s(dst + bytes, v.lsplit_lo + src, bytes, &b_full[slot]);
            issued[slot] = 1;
            last_phase[slot] = P.b_resident ? 0 : (int)phb;
            packed += bytes * (uint32_t)parts;
            if (!P.b_resident && ++tb == P.b_slots) { tb = 0; phb ^= 1; }
          }
        }
        if (P.b_resident) break;   // every piece stays in shared memory for all tiles
      }
      // copies land on their own; wait for the last one of each slot before exit
      for (int t = 0; t < kMaxBSlots; ++t)
        if (issued[t]) {
          unsigned long long t0 = now_ns();
          while (!mbar_test(&b_full[t], (uint32_t)last_phase[t]) && now_ns() - t0 < kWaitNs) {
          }
        }
    }
  }

  // ---- teardown: per-CTA variance sum, TMEM release, last-block total
  for (int o = 16; o > 0; o >>= 1) vsum += __shfl_xor_sync(0xffffffffu, vsum, o);
  if (warp >= kEpiWarp0 && warp < kMmaWarp && lane == 0) red[warp - kEpiWarp0] = vsum;
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(P.tmem_cols * P.acc_stages) : "memory");
  }
  if (threadIdx.x == 0) {
    v.partial[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
    __threadfence();
    const unsigned int done = atomicAdd(&v.stats->k1_done, 1u);
    s_last = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    double t = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) t += ((volatile double*)v.partial)[b];
    v.stats->sum_var = t;
    v.stats->k1_done = 0;
  }
}

// dimension buckets: the distance loop runs over DMAX zero-padded coordinates
int dim_bucket(int d) { return d <= 4 ? 4 : d <= 7 ? 7 : d <= 9 ? 9 : 16; }

template <int MODE, int DMAX, bool NU52>
int launch_mode(const TcParams& P, size_t smem, int grid, cudaStream_t s) {
  static size_t configured = 0;
  if (configured < smem) {
    if (cudaFuncSetAttribute(predict_tc_kernel<MODE, DMAX, NU52>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return -1;
    configured = smem;
  }
  predict_tc_kernel<MODE, DMAX, NU52><<<grid, kThreads, smem, s>>>(P);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

template <int MODE, bool NU52>
int launch_dims(const TcParams& P, size_t smem, int grid, cudaStream_t s) {
  switch (dim_bucket(P.v.d)) {
    case 4: return launch_mode<MODE, 4, NU52>(P, smem, grid, s);
    case 7: return launch_mode<MODE, 7, NU52>(P, smem, grid, s);
    case 9: return launch_mode<MODE, 9, NU52>(P, smem, grid, s);
    default: return launch_mode<MODE, 16, NU52>(P, smem, grid, s);
  }
}

template <int MODE>
int launch_nu(const TcParams& P, size_t smem, int grid, cudaStream_t s) {
  return P.v.nu == 2.5 ? launch_dims<MODE, true>(P, smem, grid, s) : launch_dims<MODE, false>(P, smem, grid, s);
}

}  // namespace

int launch_predict_tc(const DevView& v, int n, int64_t /*n_unvisited*/, cudaStream_t s) {
  if (n < 1 || n > v.n_max || v.precision == BO_PREC_FP64 || v.d > 16) return -1;
  TcParams P;
  P.v = v;
  P.n = n;
  const int eb = v.precision == BO_PREC_TF32 ? 4 : 2;
  P.cw = kChunkBytes / eb;
  P.parts = v.precision == BO_PREC_TF32 ? 1 : 2;
  P.n_pad = (n + 31) / 32 * 32;
  if (P.n_pad > v.n_max) return -1;
  P.chunks = P.n_pad / P.cw;
  int cols = 32;
  while (cols < P.n_pad) cols <<= 1;
  if (cols > 512) return -1;
  P.tmem_cols = cols;
  P.acc_stages = 2 * cols <= 512 ? 2 : 1;
  P.num_tiles = (int)(v.N_pad / kRows);
  // shared memory plan
  const size_t a_stage = (size_t)P.parts * kPartBytes;
  const size_t x_bytes = (size_t)dim_bucket(v.d) * P.n_pad * 4;
  const size_t q_bytes = (size_t)2 * P.n_pad * 4;
  const size_t limit = 226 * 1024;   // dynamic part; the kernel's static shared memory is small
  size_t resident = 0;
  int pieces = 0;
  for (int c = 0; c < P.chunks; ++c)
    for (int r0 = c * P.cw; r0 < P.n_pad; r0 += kPieceRows, ++pieces)
      resident += (size_t)P.parts * (std::min(kPieceRows, P.n_pad - r0) / 8) * 512;
  P.b_resident = (pieces <= kMaxBSlots && resident <= (size_t)P.parts * 64 * 1024) ? 1 : 0;
  P.b_slots = 4;
  P.b_slot_bytes = (size_t)P.parts * (kPieceRows / 8) * 512;
  const size_t b_bytes = P.b_resident ? resident : P.b_slots * P.b_slot_bytes;
  const size_t fixed = ((b_bytes + 1023) / 1024) * 1024 + ((x_bytes + q_bytes + 1023) / 1024) * 1024 + 512;
  int sa = (int)((limit - fixed) / a_stage);
  sa = sa >= 8 ? 8 : sa >= 4 ? 4 : sa >= 2 ? 2 : 0;     // a power of two
  if (sa < 2) return -1;
  P.stages_a = sa;
  P.off_b = (size_t)sa * a_stage;
  P.off_x = P.off_b + ((b_bytes + 1023) / 1024) * 1024;
  P.off_q = P.off_x + x_bytes;
  P.off_bar = (P.off_q + q_bytes + 15) / 16 * 16;
  const size_t smem = P.off_bar + (size_t)(2 * sa + 2 * kMaxBSlots + 6) * 8 + 16;
  if (smem > limit) return -1;
  // every descriptor footprint stays inside its stage: A parts are 128 rows x
  // 64 B; a B piece [n0, n0 + w) of chunk c ends at row n_pad - c*cw of its part
  if ((size_t)15 * 512 + 256 + 255 >= (size_t)kPartBytes) return -1;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = P.num_tiles < sms ? P.num_tiles : sms;
  if (grid > v.max_partials) return -1;
  switch (v.precision) {
    case BO_PREC_FP16X3: return launch_nu<BO_PREC_FP16X3>(P, smem, grid, s);
    case BO_PREC_BF16X3: return launch_nu<BO_PREC_BF16X3>(P, smem, grid, s);
    default: return launch_nu<BO_PREC_TF32>(P, smem, grid, s);
  }
}

}  // namespace bo
