// Prediction pass on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Same mathematics as the FP64 pass (paper Sec. III-B, III-G): for every
// candidate c, v = L^-1 k*(c), var = k(0) - |v|^2, mu = k* . alpha with
// alpha = L^-T beta (the FP64 update provides it).  The producers that
// evaluate K* also accumulate mu (FP32 within a chunk, FP64 across chunks), so
// mu does not depend on the split contraction; the contraction V = K* L^-T,
// needed for the variance, runs on the tensor cores with FP32 accumulation in
// tensor memory, with the operands split to recover precision:
//   FP16X3 / BF16X3 / TF32X3: K* = Kh + Kl and L^-1 = Lh + Ll (per-row
//     power-of-two scaled), V ~ Kh Lh + Kh Ll + Kl Lh  (three MMAs per
//     k-step); a 16-bit or TF32 part has 11 (FP16, TF32) or 8 (BF16)
//     significant bits, so FP16X3 and TF32X3 carry about 22 bits
//   TF32: one MMA on TF32-rounded operands.
// The FP64 L^-1, beta and the update stay in FP64 (bo_update.cu), which
// writes the split copy of each new row once.
//
// One kernel serves one space (tiles strided over the CTAs) or a batch of
// spaces of different sizes in one persistent launch (each CTA walks a
// host-planned list of segments, i.e. runs of consecutive tiles of one
// space, balanced by estimated tile cost).
//
// CTA organisation (persistent, one CTA per SM, 128 candidates per tile):
//   warps 0-15   produce K* chunks: thread (row = t % 128, quarter = t / 128)
//                evaluates the Matern covariance of its candidate against a
//                quarter of the chunk's observations (packed f32x2, over the
//                space's own d coordinates), adds its share of k* . alpha,
//                splits it and stores it in the K-major core-matrix layout.
//                The next tile's candidate codes are fetched while the
//                current tile is computed (the first tile's before the
//                dependent wait).
//   warps 16-19  drain the accumulator (TMEM lane = row): sum acc_k^2 q_k
//                (q of the space in shared memory) and write var; add a
//                row's four quarter sums of k* . alpha (handed over in shared
//                memory) and write mu.  Each 32-column block is drained as
//                soon as the chunk that completes it has run, and a 256-column
//                region is handed back after its last block: the next tile's
//                first MMAs into a region wait only for that region.  With
//                n <= 256 the accumulator is double-buffered.
//   warps 20, 22 issue the MMAs (the whole warp runs the loop, one elected
//                lane issues each MMA and commit): warp 20 for accumulator
//                columns 0-255 (and owns the TMEM allocation), warp 22 for
//                columns 256-511 when n > 256, so that the two halves'
//                instruction streams overlap.
//   warp 21      streams, with bulk copies (one thread), each space's
//                observation coordinates, 1/s^2 and alpha into shared
//                memory (double-buffered across spaces) and the L^-1 chunks in pieces of at most 256
//                rows: a ring of slots, or, for one space whose pieces fit, all
//                pieces resident, loaded once.  With two issuers each region
//                has its own ring, and warp 23 streams region 1's pieces.
// K chunk c covers observations j in [c CW, (c+1) CW); only output columns
// k >= c CW receive it (L^-1 is lower triangular), so the MMA N range
// shrinks along the chunks.  Every wait is bounded in time: on expiry the
// CTA records BO_ERR_TIMEOUT, drains its own copies / MMAs and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <vector>

#include "bo_acquire_dev.cuh"
#include "bo_internal.h"

namespace bo {

namespace {

constexpr int kRows = 128;              // candidates per tile (MMA M)
constexpr int kProducerWarps = 16;
constexpr int kEpiWarp0 = 16;           // warps 16-19
constexpr int kMmaWarp = 20;
constexpr int kLoadWarp = 21;
constexpr int kMmaWarp2 = 22;           // second MMA issuer (columns 256..511)
constexpr int kLoadWarp2 = 23;          // loader of the second issuer's L^-1 pieces
constexpr int kThreads = 768;
constexpr int kPartBytes = kRows * kChunkBytes;   // one split part of an A stage: 8 KB
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s
constexpr int kPieceRows = 256;         // rows of L^-1 per B piece (= max MMA N)
constexpr int kMaxBSlots = 16;
constexpr int kAccBars = 32;            // per accumulator column block: 2 buffers x 16, or 1 x 32
constexpr int kMuPartBytes = 2 * 4 * kRows * 4;   // the four quarter sums of mu, two tiles

struct TcParams {
  TcSess s0;                 // the space, when batch == 0
  const TcSess* sess;        // batch > 0: [batch] device array
  const TcSeg* segs;         // batch > 0: segments; CTA b owns [seg_begin[b], seg_begin[b+1])
  const int* seg_begin;
  double* seg_part;          // batch > 0: [segment][4] variance sums of the epilogue warps
  double* partial;           // batch == 0: per-CTA variance sums
  DevStats* stats;           // batch == 0: the fused tail's counters; status word of the launch
  int32_t* status;
  int batch;
  int cw, parts, stages_a;
  int tmem_cols;             // columns of one accumulator buffer
  int acc_stages;            // 1 or 2 accumulator buffers
  int issuers;               // MMA issuing threads: 2 when some n_pad > 256 (one per 256-column region)
  int xs_bufs;               // 1 or 2 coordinate buffers
  // B (the split L^-1 chunks) in pieces of <= 256 rows: either a ring of
  // b_slots fixed-size slots, or every piece of the space resident (loaded once)
  int b_resident, b_slots;
  size_t off_b, b_slot_bytes, off_x, x_buf_bytes, off_mu, off_bar;
  // acquisition tail (one space, cooperative launch): after a grid barrier on
  // the variance partials every CTA scores the candidates of its own tiles
  int acq;
  PassArgs args;
  bo_pass_result* result;
  TopEntry* acq_partial;     // [grid][3][3] per-CTA top-3 keys (in TopEntry::idx)
  double* var_s;             // contextual-variance baseline
};

// Position in a CTA's work: one space with strided tiles, or a segment list.
struct Work {
  int seg, seg_end, sess, tile, tile_end;
};

__device__ __forceinline__ bool work_begin(const TcParams& P, Work& w) {
  if (P.batch == 0) {
    w.sess = 0;
    w.tile = blockIdx.x;
    w.tile_end = P.s0.num_tiles;
    w.seg = w.seg_end = 0;
    return w.tile < w.tile_end;
  }
  w.seg = P.seg_begin[blockIdx.x];
  w.seg_end = P.seg_begin[blockIdx.x + 1];
  if (w.seg >= w.seg_end) return false;
  const TcSeg g = P.segs[w.seg];
  w.sess = g.sess;
  w.tile = g.tile0;
  w.tile_end = g.tile1;
  return w.tile < w.tile_end;
}

__device__ __forceinline__ bool work_next(const TcParams& P, Work& w) {
  if (P.batch == 0) {
    w.tile += gridDim.x;
    return w.tile < w.tile_end;
  }
  if (++w.tile < w.tile_end) return true;
  if (++w.seg >= w.seg_end) return false;
  const TcSeg g = P.segs[w.seg];
  w.sess = g.sess;
  w.tile = g.tile0;
  w.tile_end = g.tile1;
  return w.tile < w.tile_end;
}

__device__ __forceinline__ const TcSess& sess_of(const TcParams& P, int s) {
  return P.batch == 0 ? P.s0 : P.sess[s];
}

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

// mbar_wait by every lane of a warp; the result is the same in all lanes
// (false if any lane's wait expired or saw the abort flag).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          int32_t* status) {
  return __all_sync(0xffffffffu, mbar_wait(bar, parity, abort_flag, status));
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// L2 prefetch of this CTA's share (1 / parts) of [p, p + bytes): the shares of
// all CTAs cover the range; 16-byte granules (the bulk prefetch's unit).
__device__ __forceinline__ void l2_prefetch_share(const void* p, size_t bytes, int part, int parts) {
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

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// Piece r of chunk c: the L^-1 rows [r0, r0 + wd) of accumulator region r
// (columns [256 r, 256 r + 256)) that chunk c reaches (rows >= c cw).  The
// loader and both issuers walk pieces in (chunk, region) order.
__device__ __forceinline__ bool piece_of(int c, int r, int cw, int n_pad, int* r0, int* wd) {
  const int lo = max(c * cw, r * kPieceRows), hi = min((r + 1) * kPieceRows, n_pad);
  *r0 = lo;
  *wd = hi - lo;
  return lo < hi;
}

// B slots of accumulator region r's ring: with one issuer a single ring of
// all slots; with two, the slots split between the regions.
__host__ __device__ __forceinline__ int ring_size(const TcParams& P, int r) {
  return P.issuers == 1 ? P.b_slots : (r == 0 ? P.b_slots - P.b_slots / 2 : P.b_slots / 2);
}
__host__ __device__ __forceinline__ int ring_base(const TcParams& P, int r) {
  return r == 0 ? 0 : ring_size(P, 0);
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

// The MMA-issuing warps run their loops with all 32 lanes, so that the loop
// state and the descriptors are warp-uniform; inside the same asm statement
// elect.sync picks the one lane that issues each MMA or commit.
template <int MODE>
__device__ __forceinline__ void mma_el(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (split_elem_bytes(MODE) == 4) {
    asm volatile(
        "{\n .reg .pred p, e;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
        " @e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p, e;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
        " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit_el(uint64_t* bar) {
  asm volatile(
      "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* r) {
  uint32_t u[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
        "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]),
        "=r"(u[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) r[i] = __uint_as_float(u[i]);
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

// Hardware reciprocal square root, flushing subnormals (inputs here are >= 1e-30).
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
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

__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t dup2(float x) { return pk2(x, x); }
// hi + lo += x by Knuth's TwoSum: a compensated FP32 running sum.  (FP64 is
// a narrow unit on this GPU; the per-tile sums stay off it.)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float t = hi + x;
  const float bp = t - hi;
  lo += (hi - (t - bp)) + (x - bp);
  hi = t;
}

__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}


// Matern covariance in FP32 for two squared distances at once (one packed
// word), in units where u = t log2(e), t = sqrt(2 nu) r / l (the coordinate
// tables carry the scale; the accumulators start at 1e-30 so u^2 > 0):
// u from the hardware reciprocal square root and one Newton step on the
// residual u0^2 - u^2, e^-t = 2^-u from the hardware exp2, then (1 + t) e^-t
// or (1 + t + t^2/3) e^-t.  Everything but the four MUFU operations runs on
// the packed f32x2 pipe.  (Without the Newton step the sigma error on the
// 7-parameter space at n = 220 grows from 9e-5 to 2.3e-4, for 2.5 % of the
// kernel time.)
template <bool NU52>
__device__ __forceinline__ uint64_t matern2(uint64_t u2p) {
  float a, b;
  upk2(u2p, a, b);
  const uint64_t rs = pk2(rsqrt_approx(a), rsqrt_approx(b));
  const uint64_t u0 = mul2(u2p, rs);
  const uint64_t nu2 = mul2(u2p, dup2(-1.0f));
  const uint64_t hn = mul2(rs, dup2(-0.5f));
  const uint64_t u = fma2(fma2(u0, u0, nu2), hn, u0);
  float ua, ub;
  upk2(u, ua, ub);
  const uint64_t e = pk2(ex2_approx(-ua), ex2_approx(-ub));
  const uint64_t t = mul2(u, dup2(0.6931471805599453f));
  if constexpr (NU52)
    return fma2(mul2(t, e), fma2(t, dup2(1.0f / 3.0f), dup2(1.0f)), e);
  else
    return fma2(t, e, e);
}

// Squared scaled distances of one candidate (xcp: its coordinates, twice per
// word) to this thread's observations of a chunk: `grp` is the shared-memory
// address of their coordinates inside a group of 8 observations (coordinate
// row p at + 32 p bytes), two observations per packed instruction;
// accumulators start at 1e-30 so that u^2 > 0.  CHECK: the space has fewer
// than DMAX coordinates (d, warp-uniform).
template <int MODE, int DMAX, bool CHECK>
__device__ __forceinline__ void sq_dist(const uint64_t* xcp, uint32_t grp, int d, uint64_t* r2p) {
  constexpr bool kWide = split_elem_bytes(MODE) == 2;   // 8 observations per thread and chunk, else 4
  const uint64_t eps = dup2(1e-30f);
  r2p[0] = r2p[1] = r2p[2] = r2p[3] = eps;
#pragma unroll
  for (int p = 0; p < DMAX; ++p) {
    if (CHECK && p >= d) break;
    uint64_t o0, o1;
    lds2x64(grp + (uint32_t)(p * 32), o0, o1);
    uint64_t df = sub2(xcp[p], o0);
    r2p[0] = fma2(df, df, r2p[0]);
    df = sub2(xcp[p], o1);
    r2p[1] = fma2(df, df, r2p[1]);
    if constexpr (kWide) {
      lds2x64(grp + (uint32_t)(p * 32 + 16), o0, o1);
      df = sub2(xcp[p], o0);
      r2p[2] = fma2(df, df, r2p[2]);
      df = sub2(xcp[p], o1);
      r2p[3] = fma2(df, df, r2p[3]);
    }
  }
}

// Split two K* values (one packed word, element 0 in the low half) into the
// hi and lo 16-bit words of the FP16X3 / BF16X3 forms: hi = round(k),
// lo = round(k - hi); each result holds element 0 in its low half.
template <int MODE>
__device__ __forceinline__ void split2(uint64_t kv, uint32_t& hi, uint32_t& lo) {
  float a, b;
  upk2(kv, a, b);
  float fa, fb;
  if constexpr (MODE == BO_PREC_FP16X3) {
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(b), "f"(a));
    asm("{\n .reg .b16 l, u;\n mov.b32 {l, u}, %2;\n cvt.f32.f16 %0, l;\n cvt.f32.f16 %1, u;\n}\n"
        : "=f"(fa), "=f"(fb) : "r"(hi));
  } else {
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(b), "f"(a));
    asm("{\n .reg .b16 l, u;\n mov.b32 {l, u}, %2;\n cvt.f32.bf16 %0, l;\n cvt.f32.bf16 %1, u;\n}\n"
        : "=f"(fa), "=f"(fb) : "r"(hi));
  }
  float ra, rb;
  upk2(sub2(kv, pk2(fa, fb)), ra, rb);
  if constexpr (MODE == BO_PREC_FP16X3)
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(rb), "f"(ra));
  else
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(rb), "f"(ra));
}

// x rounded to TF32 (10 explicit mantissa bits), to nearest with ties away from
// zero: half an ulp of the 10-bit mantissa added to the magnitude bits, the 13
// low bits cleared (a carry moves into the exponent as in any rounding).  Two
// integer operations; the same bits as cvt.rna.tf32.f32 for every finite x.
__device__ __forceinline__ uint32_t to_tf32(float x) {
  return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}

// Acquisition tail of a single-space pass (the kernel is launched
// cooperatively, so every CTA is resident): each CTA publishes its variance
// partial and waits, bounded in time, until all have; every CTA then forms
// the same variance sum (fixed order) and lambda, scores the candidates of its
// own tiles (FP32, bo_acquire_dev.cuh) into a block top-3 per AF, and the last
// CTA to finish merges the per-CTA lists into the pass result.  keys: shared
// memory for [24 warps][3][3] keys (the A stages, free by now).
__device__ __noinline__ void acquisition_tail(const TcParams& P, double my_vsum, unsigned long long* keys) {
  __shared__ double s_sum;
  __shared__ int s_ok;
  __shared__ bool s_last;
  const TcSess& S = P.s0;
  const int G = (int)gridDim.x;
  DevStats* st = P.stats;
  if (threadIdx.x == 0) {
    P.partial[blockIdx.x] = my_vsum;
    __threadfence();
    atomicAdd(&st->k1_done, 1u);
    const unsigned long long t0 = now_ns();
    int ok = 1;
    while (*(volatile unsigned int*)&st->k1_done < (unsigned int)G) {
      if (now_ns() - t0 > kWaitNs) {
        atomicExch(P.status, BO_ERR_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  {
    const double t = block_sum_partials(P.partial, G, reinterpret_cast<double*>(keys));
    if (threadIdx.x == 0) s_sum = s_ok ? t : 0.0;
  }
  __syncthreads();
  const PassArgs& a = P.args;
  __shared__ double s_lam[3];   // mean_var, var_s, lambda: FP64 scalars, formed once and broadcast
  if (threadIdx.x == 0) acq::pass_lambda(a, s_sum, a.first_pass ? 0.0 : *P.var_s, &s_lam[0], &s_lam[1], &s_lam[2]);
  __syncthreads();
  const double mean_var = s_lam[0], var_s = s_lam[1], lam = s_lam[2];
  unsigned long long top[3][acq::kTop];
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int r = 0; r < acq::kTop; ++r) top[q][r] = 0ull;
  if (s_ok) {
    const float lamT = (float)lam, fpT = (float)a.fplus_t;
    const int my_tiles = blockIdx.x < S.num_tiles ? (S.num_tiles - 1 - (int)blockIdx.x) / G + 1 : 0;
    for (int k = threadIdx.x; k < my_tiles * kRows; k += kThreads) {
      const int64_t i = (int64_t)(blockIdx.x + (k / kRows) * G) * kRows + (k % kRows);
      if (i >= S.N || ((S.visited[i >> 5] >> (i & 31)) & 1u)) continue;
      acq::score_f32(S.mu[i], S.var[i], fpT, lamT, a.n_af, a.af[0], a.af[1], a.af[2], (long long)i, top);
    }
  }
  acq::block_top3(top, keys, kThreads / 32);
  if (threadIdx.x < 3 * acq::kTop) {
    const int q = threadIdx.x / acq::kTop, r = threadIdx.x % acq::kTop;
    unsigned long long k = 0ull;
#pragma unroll
    for (int qq = 0; qq < 3; ++qq)
#pragma unroll
      for (int rr = 0; rr < acq::kTop; ++rr)
        if (qq == q && rr == r) k = top[qq][rr];
    P.acq_partial[((size_t)blockIdx.x * 3 + q) * acq::kTop + r].idx = (long long)k;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&st->k2_done, 1u) == (unsigned int)G - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last CTA: every CTA's lists, merged (the key order is total: any merge order gives the same result)
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int r = 0; r < acq::kTop; ++r) top[q][r] = 0ull;
  for (int b = threadIdx.x; b < G; b += kThreads)
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int r = 0; r < acq::kTop; ++r)
        acq::key_insert(top[q],
                        (unsigned long long)__ldcg(&P.acq_partial[((size_t)b * 3 + q) * acq::kTop + r].idx));
  acq::block_top3(top, keys, kThreads / 32);
  if (threadIdx.x < 32)
    acq::write_result_f32(P.result, top, a, S.mu, S.var, *(volatile int32_t*)P.status, s_sum, mean_var, lam,
                          var_s);
  if (threadIdx.x == 0) {
    if (a.first_pass) *P.var_s = mean_var;
    st->sum_var = s_sum;
    st->k1_done = 0;
    st->k2_done = 0;
  }
}

template <int MODE, int DMAX, bool NU52>
__global__ void __launch_bounds__(kThreads, 1) predict_tc_kernel(const __grid_constant__ TcParams P) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int CW = kChunkBytes / split_elem_bytes(MODE);   // observations per K chunk: 32 or 16
  const int cw = CW, parts = P.parts, SA = P.stages_a, XB = P.xs_bufs;
  uint8_t* sa = smem;                                   // [SA][parts][8 KB]
  uint8_t* sb = smem + P.off_b;                         // B slots or resident pieces
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + P.off_bar);
  uint64_t* a_full = bars;
  uint64_t* a_empty = bars + SA;
  uint64_t* b_full = bars + 2 * SA;                            // [kMaxBSlots]
  uint64_t* b_empty = bars + 2 * SA + kMaxBSlots;              // [kMaxBSlots]
  // acc_full[16 buffer + block]: one barrier per accumulator column block, so
  // that the MMA issuer is never more than one phase ahead of the epilogue on any
  uint64_t* acc_full = bars + 2 * SA + 2 * kMaxBSlots;                     // [kAccBars]
  uint64_t* acc_empty = bars + 2 * SA + 2 * kMaxBSlots + kAccBars;         // [2] regions
  uint64_t* xs_full = bars + 2 * SA + 2 * kMaxBSlots + kAccBars + 2;       // [2]
  uint64_t* xs_empty = bars + 2 * SA + 2 * kMaxBSlots + kAccBars + 4;      // [2]
  uint64_t* drain = bars + 2 * SA + 2 * kMaxBSlots + kAccBars + 6;
  uint64_t* mu_full = bars + 2 * SA + 2 * kMaxBSlots + kAccBars + 7;       // [2]
  uint64_t* mu_empty = bars + 2 * SA + 2 * kMaxBSlots + kAccBars + 9;      // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * SA + 2 * kMaxBSlots + kAccBars + 11);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  __shared__ double red[4];   // per epilogue warp
  int32_t* status = P.status;

  // ---- setup: barriers, TMEM
  if (threadIdx.x == 0) {
    for (int s = 0; s < SA; ++s) { mbar_init(&a_full[s], kProducerWarps); mbar_init(&a_empty[s], P.issuers); }
    for (int s = 0; s < kMaxBSlots; ++s) { mbar_init(&b_full[s], 1); mbar_init(&b_empty[s], 1); }
    for (int s = 0; s < kAccBars; ++s) mbar_init(&acc_full[s], 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&acc_empty[s], 4);
      mbar_init(&xs_full[s], 1);
      mbar_init(&xs_empty[s], kProducerWarps + 4);   // producers and epilogue warps
    }
    mbar_init(drain, P.issuers);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&mu_full[s], kProducerWarps);
      mbar_init(&mu_empty[s], 4);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(P.tmem_cols * P.acc_stages) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // one space, launched as a dependent of its observation update: while the update runs, pull
  // the inputs that the L2 flush between passes leaves in HBM (the split L^-1 copy, the
  // candidate codes) into L2; a prefetch is a hint only, every read follows pdl_wait below
  if (P.batch == 0 && warp == kLoadWarp && lane == 0) {
    const TcSess& S = P.s0;
    const size_t lbytes = (size_t)kChunkBytes * ((size_t)S.chunks * S.n_max -
                                                  (size_t)P.cw * S.chunks * (S.chunks - 1) / 2);
    l2_prefetch_share(S.lhi, lbytes, blockIdx.x, gridDim.x);
    if (P.parts == 2) l2_prefetch_share(S.llo, lbytes, blockIdx.x, gridDim.x);
    l2_prefetch_share(S.codes, (size_t)S.d * (size_t)S.N_pad, blockIdx.x, gridDim.x);
  }
  // the producers' candidate codes, four per word: the first tile's are read
  // here, before the dependent wait, while the update may still be running
  // (the codes and value tables are static: the update writes neither), with
  // the value-table entries they select pulled into L1; each later tile's are
  // fetched during the tile before it
  uint32_t code_next[(DMAX + 3) / 4];
#pragma unroll
  for (int p = 0; p < (DMAX + 3) / 4; ++p) code_next[p] = 0u;
  if (warp < kProducerWarps) {
    Work w0;
    if (work_begin(P, w0)) {
      const TcSess& S0 = sess_of(P, w0.sess);
      const int64_t cand0 = (int64_t)w0.tile * kRows + (threadIdx.x & (kRows - 1));
#pragma unroll
      for (int p = 0; p < DMAX; ++p)
        if (p < S0.d) {
          const uint32_t code = S0.codes[(int64_t)p * S0.N_pad + cand0];
          code_next[p >> 2] |= code << (8 * (p & 3));
          float t;
          asm volatile("ld.global.ca.f32 %0, [%1];" : "=f"(t) : "l"(S0.vtab32 + p * 256 + code));
        }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  pdl_wait();              // the observation update has completed (dependent launch); setup overlapped it
  const uint32_t tmem = *tmem_slot;
  const uint32_t xs_base = smem_addr(smem + P.off_x);
  double vsum = 0.0;

  if (warp < kProducerWarps) {
    // ===================== K* producers =====================
    const int row = threadIdx.x & (kRows - 1);
    const int quarter = threadIdx.x >> 7;
    const int jq = cw / 4;                       // observations per thread per chunk: 8 or 4
    const uint32_t a_base = smem_addr(sa);
    const uint32_t row_off = (uint32_t)((row >> 3) * (kChunkBytes * 8) + (row & 7) * 16 + quarter * 128);
    float* mu_part = reinterpret_cast<float*>(smem + P.off_mu);   // [2 tiles][4 quarters][128 rows]
    bool ok = true;
    int s = 0, ks = -1, prev = -1, tile_it = 0;
    uint32_t ph = 0;                             // ring slot and its phase
    int n_pad = 0, chunks = 0, d = 0, ds = 0, gstride = 0;
    const float* vt = nullptr;
    uint32_t xs = xs_base;
    Work w;
    for (bool more = work_begin(P, w); more && ok; more = work_next(P, w), ++tile_it) {
      if (w.sess != prev) {                      // next space: its coordinates, once copied in
        if (ks >= 0) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&xs_empty[ks % XB]);
        }
        ++ks;
        prev = w.sess;
        const TcSess& S = sess_of(P, w.sess);
        n_pad = S.n_pad;
        chunks = S.chunks;
        d = S.d;
        vt = S.vtab32;
        ds = S.ds;
        gstride = 32 * (ds + 2);
        xs = xs_base + (uint32_t)((ks % XB) * P.x_buf_bytes);
        if (!(ok = mbar_wait(&xs_full[ks % XB], (uint32_t)((ks / XB) & 1), abort_flag, status))) break;
      }
      // mu = k* . alpha: two packed FP32 sums over groups of 4 chunks, folded
      // into a compensated (hi, lo) pair by Knuth's TwoSum after each group
      uint64_t m2 = 0ull, mhi = 0ull, mlo = 0ull;
      {
        // this tile's candidate coordinates, from the codes in code_next
        uint64_t xcp[DMAX];                    // candidate coordinate, twice per word
#pragma unroll
        for (int p = 0; p < DMAX; ++p)
          xcp[p] = dup2(p < d ? vt[p * 256 + ((code_next[p >> 2] >> (8 * (p & 3))) & 0xFFu)] : 0.0f);
        {
          Work wn = w;
          if (work_next(P, wn)) {
            const TcSess& Sn = sess_of(P, wn.sess);
            const int64_t cn = (int64_t)wn.tile * kRows + row;
            const int dn = Sn.d;
            const int64_t Nn = Sn.N_pad;
            const uint8_t* cp = Sn.codes;
#pragma unroll
            for (int p = 0; p < (DMAX + 3) / 4; ++p) code_next[p] = 0u;
#pragma unroll
            for (int p = 0; p < DMAX; ++p)
              if (p < dn) code_next[p >> 2] |= (uint32_t)cp[(int64_t)p * Nn + cn] << (8 * (p & 3));
          }
        }
        for (int c = 0; c < chunks && ok; ++c) {
          const int j0 = c * cw + quarter * jq;
          // K* for this thread's observations, computed before waiting for the ring slot
          uint64_t r2p[4];
          // this thread's observations inside their group of 8 (coordinates, 1/s^2, alpha)
          const uint32_t grp = xs + (uint32_t)((j0 >> 3) * gstride + (j0 & 7) * 4);
          if (d == DMAX)
            sq_dist<MODE, DMAX, false>(xcp, grp, d, r2p);
          else
            sq_dist<MODE, DMAX, true>(xcp, grp, d, r2p);
          uint64_t kv[4];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (2 * q < jq) kv[q] = matern2<NU52>(r2p[q]);
          {
            const uint32_t arow = grp + (uint32_t)((ds + 1) * 32);
            uint64_t a0, a1;
            lds2x64(arow, a0, a1);
            m2 = fma2(kv[1], a1, fma2(kv[0], a0, m2));
            if constexpr (CW == 32) {
              lds2x64(arow + 16, a0, a1);
              m2 = fma2(kv[3], a1, fma2(kv[2], a0, m2));
            }
            if ((c & 3) == 3 || c + 1 == chunks) {
              const uint64_t t = add2(mhi, m2);
              const uint64_t bp = sub2(t, mhi);
              mlo = add2(mlo, add2(sub2(mhi, sub2(t, bp)), sub2(m2, bp)));
              mhi = t;
              m2 = 0ull;
            }
          }
          if (!(ok = mbar_wait(&a_empty[s], ph ^ 1, abort_flag, status))) break;
          const uint32_t stage = a_base + (uint32_t)(s * parts * kPartBytes) + row_off;
          if constexpr (MODE == BO_PREC_TF32) {
            float k0, k1, k2, k3;
            upk2(kv[0], k0, k1);
            upk2(kv[1], k2, k3);
            st_shared_v4(stage, to_tf32(k0), to_tf32(k1), to_tf32(k2), to_tf32(k3));
          } else if constexpr (MODE == BO_PREC_TF32X3) {
            // hi = TF32 rounding of k, lo = TF32 rounding of the (exact) residual k - hi
            float k0, k1, k2, k3;
            upk2(kv[0], k0, k1);
            upk2(kv[1], k2, k3);
            const uint32_t h0 = to_tf32(k0), h1 = to_tf32(k1), h2 = to_tf32(k2), h3 = to_tf32(k3);
            float r0, r1, r2, r3;
            upk2(sub2(kv[0], pk2(__uint_as_float(h0), __uint_as_float(h1))), r0, r1);
            upk2(sub2(kv[1], pk2(__uint_as_float(h2), __uint_as_float(h3))), r2, r3);
            st_shared_v4(stage, h0, h1, h2, h3);
            st_shared_v4(stage + kPartBytes, to_tf32(r0), to_tf32(r1), to_tf32(r2), to_tf32(r3));
          } else {
            uint32_t h[4], l[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) split2<MODE>(kv[q], h[q], l[q]);
            st_shared_v4(stage, h[0], h[1], h[2], h[3]);
            st_shared_v4(stage + kPartBytes, l[0], l[1], l[2], l[3]);
          }
          fence_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(&a_full[s]);
          if (++s == SA) { s = 0; ph ^= 1; }
        }
      }
      if (!ok) break;
      // tile end: this quarter's sum goes to the epilogue through shared memory
      // (double-buffered by tile, handed over with mbarriers)
      const int mb = tile_it & 1;
      if (!(ok = mbar_wait(&mu_empty[mb], ((uint32_t)(tile_it >> 1) & 1u) ^ 1u, abort_flag, status))) break;
      float h0, h1, l0, l1;
      upk2(mhi, h0, h1);
      upk2(mlo, l0, l1);
      mu_part[(mb * 4 + quarter) * kRows + row] = (h0 + h1) + (l0 + l1);
      __syncwarp();
      if (lane == 0) mbar_arrive(&mu_full[mb]);
    }
  } else if (warp < kMmaWarp) {
    // ===================== epilogue: warp e owns TMEM lanes [32e, 32e+32) =====================
    const int e = warp - kEpiWarp0;
    const int row = e * 32 + lane;
    bool ok = true;
    int it = 0, prev = -1, seg = -1, ks = -1;
    int n_pad = 0, chunks = 0;
    uint32_t par[2] = {0u, 0u};                  // phase parity of each block barrier, per buffer
    int64_t N = 0;
    const float* rq = nullptr;                   // 1/s_k^2 of the space, shared memory (group-strided)
    int gfloats = 0;                             // floats per group of 8 observations
    const uint32_t* visited = nullptr;
    float* var = nullptr;
    float* mu = nullptr;
    float vs_hi = 0.0f, vs_lo = 0.0f;           // this thread's variance sum (compensated)
    Work w;
    for (bool more = work_begin(P, w); more && ok; more = work_next(P, w), ++it) {
      if (P.batch && w.seg != seg) {             // segment boundary: hand in its variance sum
        if (seg >= 0) {
          double t = (double)vs_hi + (double)vs_lo;
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          if (lane == 0) P.seg_part[(size_t)seg * 4 + e] = t;
          vs_hi = vs_lo = 0.0f;
        }
        seg = w.seg;
      }
      if (w.sess != prev) {
        if (ks >= 0) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&xs_empty[ks % XB]);
        }
        ++ks;
        prev = w.sess;
        const TcSess& S = sess_of(P, w.sess);
        n_pad = S.n_pad;
        chunks = S.chunks;
        N = S.N;
        const float* xsb = reinterpret_cast<const float*>(smem + P.off_x + (size_t)(ks % XB) * P.x_buf_bytes);
        rq = xsb + (size_t)S.ds * 8;             // slot ds of each group of 8 observations
        gfloats = 8 * (S.ds + 2);
        visited = S.visited;
        var = S.var;
        mu = S.mu;
        if (!(ok = mbar_wait(&xs_full[ks % XB], (uint32_t)((ks / XB) & 1), abort_flag, status))) break;
      }
      // column block c (32 columns) of the accumulator is final once chunk c
      // completes (the issuer owning its region commits that block's barrier);
      // a 256-column region is handed back once its last block is drained
      const int as = it % P.acc_stages;
      const uint32_t lane_base = tmem + (uint32_t)(as * P.tmem_cols) + ((uint32_t)(e * 32) << 16);
      uint64_t s2p = 0ull;                       // two columns per packed word
      // (every column block is signalled as it becomes final, so earlier
      // blocks drain while later chunks are still being accumulated)
      for (int c = 0; c < chunks && ok; ++c) {
        {
          if (!(ok = mbar_wait(&acc_full[as * 16 + c], (par[as] >> c) & 1u, abort_flag, status))) break;
          par[as] ^= 1u << c;
          tc_fence_after();
        }
        const int k0 = c * CW;
        float acc[32];
        if constexpr (CW == 16)
          tmem_ld16(lane_base + (uint32_t)k0, acc);
        else
          tmem_ld32(lane_base + (uint32_t)k0, acc);
#pragma unroll
        for (int i = 0; i < CW; i += 4) {
          const int k = k0 + i;
          const float4 q = *reinterpret_cast<const float4*>(rq + (k >> 3) * gfloats + (k & 7));
          const uint64_t a01 = pk2(acc[i], acc[i + 1]), a23 = pk2(acc[i + 2], acc[i + 3]);
          s2p = fma2(mul2(a01, pk2(q.x, q.y)), a01, s2p);
          s2p = fma2(mul2(a23, pk2(q.z, q.w)), a23, s2p);
        }
        const int kend = k0 + CW;
        if (kend == n_pad || (kend & (kPieceRows - 1)) == 0) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[as + ((kend - 1) >> 8)]);
        }
      }
      if (!ok) break;
      float s2a, s2b;
      upk2(s2p, s2a, s2b);
      const float s2 = s2a + s2b;
      const int64_t cand = (int64_t)w.tile * kRows + row;
      const float vr = fmaxf(0.0f, 1.0f - s2);
      var[cand] = vr;
      {   // mu: the producers' four quarter sums of k* . alpha, added in a fixed order
        const int mb = it & 1;
        if (!(ok = mbar_wait(&mu_full[mb], (uint32_t)(it >> 1) & 1u, abort_flag, status))) break;
        const float* mp = reinterpret_cast<const float*>(smem + P.off_mu) + mb * 4 * kRows + row;
        mu[cand] = ((mp[0] + mp[kRows]) + mp[2 * kRows]) + mp[3 * kRows];
        __syncwarp();
        if (lane == 0) mbar_arrive(&mu_empty[mb]);
      }
      if (cand < N && !((visited[cand >> 5] >> (cand & 31)) & 1u)) two_sum_acc(vs_hi, vs_lo, vr);
    }
    if (P.batch && seg >= 0 && ok) {
      double t = (double)vs_hi + (double)vs_lo;
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) P.seg_part[(size_t)seg * 4 + e] = t;
      vs_hi = vs_lo = 0.0f;
    }
    vsum = (double)vs_hi + (double)vs_lo;
  } else if (warp == kMmaWarp || warp == kMmaWarp2) {
    // ===================== MMA issuers =====================
    // Issuer r (warp 20: r = 0, warp 22: r = 1) owns accumulator columns
    // [256 r, 256 r + 256): it issues the B pieces of that region, waits for
    // the region's drain, and hands over the column blocks it finalises.  Both
    // wait for every A stage and release it (a_empty counts both).
    const int r_me = warp == kMmaWarp ? 0 : 1;
    if (r_me < P.issuers) {       // all 32 lanes: the loop state stays warp-uniform
      const int fmt = MODE == BO_PREC_FP16X3 ? 0 : MODE == BO_PREC_BF16X3 ? 1 : 2;
      const uint32_t a_base = smem_addr(sa), b_base = smem_addr(sb);
      bool ok = true;
      int it = 0, sa_i = 0, tb = 0, prev = -1, n_pad = 0, chunks = 0;
      uint32_t pha = 0, phb = 0;
      uint32_t fill = 0;            // tiles started in this issuer's region (of buffer as)
      uint32_t fill2[2] = {0u, 0u};
      Work w;
      if (P.issuers == 1) {
        // n <= 256 everywhere: one region, one piece per chunk (rows [c cw, n_pad))
        for (bool more = work_begin(P, w); more && ok; more = work_next(P, w), ++it) {
          if (w.sess != prev) {
            prev = w.sess;
            const TcSess& S = sess_of(P, w.sess);
            n_pad = S.n_pad;
            chunks = S.chunks;
          }
          const int as = it % P.acc_stages;
          const uint32_t d_base = tmem + (uint32_t)(as * P.tmem_cols);
          uint32_t packed = 0;      // resident byte offset of chunk c's piece
          for (int c = 0; c < chunks && ok; ++c) {
            const int s = sa_i;
            if (!(ok = warp_wait(&a_full[s], pha, abort_flag, status))) break;
            tc_fence_after();
            if (c == 0) {           // the buffer's previous tile has been drained
              if (!(ok = warp_wait(&acc_empty[as], (fill2[as] & 1u) ^ 1u, abort_flag, status))) break;
              ++fill2[as];
              tc_fence_after();
            }
            const int r0 = c * cw, wd = n_pad - r0;
            const uint32_t part_bytes = (uint32_t)((wd >> 3) * 512);
            const int slot = P.b_resident ? c : tb;
            if (!(ok = warp_wait(&b_full[slot], P.b_resident ? 0u : phb, abort_flag, status))) break;
            tc_fence_after();
            const uint64_t ad0 = smem_desc(a_base + (uint32_t)(s * parts * kPartBytes), 128, 512);
            const uint64_t bd0 =
                smem_desc(b_base + (P.b_resident ? packed : (uint32_t)(tb * P.b_slot_bytes)), 128, 512);
            const uint32_t idesc = instr_desc(fmt, kRows, wd);
            const uint32_t dcol = d_base + (uint32_t)r0;
            const uint32_t first = c > 0 ? 1u : 0u;
            if (parts == 2) {
              const uint64_t pbo = (uint64_t)(part_bytes >> 4), pao = (uint64_t)(kPartBytes >> 4);
              mma_el<MODE>(dcol, ad0, bd0 + pbo, idesc, first);
              mma_el<MODE>(dcol, ad0 + 16, bd0 + pbo + 16, idesc, 1u);
              mma_el<MODE>(dcol, ad0 + pao, bd0, idesc, 1u);
              mma_el<MODE>(dcol, ad0 + pao + 16, bd0 + 16, idesc, 1u);
              mma_el<MODE>(dcol, ad0, bd0, idesc, 1u);
              mma_el<MODE>(dcol, ad0 + 16, bd0 + 16, idesc, 1u);
            } else {
              mma_el<MODE>(dcol, ad0, bd0, idesc, first);
              mma_el<MODE>(dcol, ad0 + 16, bd0 + 16, idesc, 1u);
            }
            packed += part_bytes * (uint32_t)parts;
            if (!P.b_resident) {
              mma_commit_el(&b_empty[tb]);
              if (++tb == P.b_slots) { tb = 0; phb ^= 1; }
            }
            mma_commit_el(&a_empty[s]);
            mma_commit_el(&acc_full[as * 16 + c]);   // column block c is final
            if (++sa_i == SA) { sa_i = 0; pha ^= 1; }
          }
        }
      } else {
      const int my_base = ring_base(P, r_me), my_size = ring_size(P, r_me);
      for (bool more = work_begin(P, w); more && ok; more = work_next(P, w), ++it) {
        if (w.sess != prev) {
          prev = w.sess;
          const TcSess& S = sess_of(P, w.sess);
          n_pad = S.n_pad;
          chunks = S.chunks;
        }
        const int as = it % P.acc_stages;
        const uint32_t d_base = tmem + (uint32_t)(as * P.tmem_cols);
        int q = 0;                  // piece index within the tile
        uint32_t packed = 0;        // resident byte offset of piece q
        for (int c = 0; c < chunks && ok; ++c) {
          const int s = sa_i;
          if (!(ok = warp_wait(&a_full[s], pha, abort_flag, status))) break;
          tc_fence_after();
          const uint64_t ad0 = smem_desc(a_base + (uint32_t)(s * parts * kPartBytes), 128, 512);
          for (int r = 0; r < 2 && ok; ++r) {
            int r0, wd;
            if (!piece_of(c, r, cw, n_pad, &r0, &wd)) continue;
            const uint32_t part_bytes = (uint32_t)((wd >> 3) * 512);
            // ring mode: region r has its own B ring (slots [ring_base(r), + ring_size(r))),
            // so each issuer waits only on pieces it consumes (a shared ring would
            // let an issuer that skips the other's pieces run phases ahead of the loader)
            const int slot = P.b_resident ? q : my_base + tb;
            const uint32_t b_st = b_base + (P.b_resident ? packed : (uint32_t)(slot * P.b_slot_bytes));
            ++q;
            packed += part_bytes * (uint32_t)parts;
            const bool mine = r == r_me;
            if (mine) {
              if (c == 0) {           // first write to this region since its last drain
                uint32_t& f = P.acc_stages == 2 ? fill2[as] : fill;
                if (!(ok = warp_wait(&acc_empty[as + r], (f & 1u) ^ 1u, abort_flag, status))) break;
                ++f;
                tc_fence_after();
              }
              if (!(ok = warp_wait(&b_full[slot], P.b_resident ? 0u : phb, abort_flag, status))) break;
              tc_fence_after();
              // descriptors advance by address >> 4: +16 is the next 16-element K step
              const uint64_t bd0 = smem_desc(b_st, 128, 512);
              const uint32_t idesc = instr_desc(fmt, kRows, wd);
              const uint32_t dcol = d_base + (uint32_t)r0;
              const uint32_t first = c > 0 ? 1u : 0u;
              if (parts == 2) {
                // products (hi, lo), (lo, hi), (hi, hi): small terms first
                const uint64_t pbo = (uint64_t)(part_bytes >> 4), pao = (uint64_t)(kPartBytes >> 4);
                mma_el<MODE>(dcol, ad0, bd0 + pbo, idesc, first);
                mma_el<MODE>(dcol, ad0 + 16, bd0 + pbo + 16, idesc, 1u);
                mma_el<MODE>(dcol, ad0 + pao, bd0, idesc, 1u);
                mma_el<MODE>(dcol, ad0 + pao + 16, bd0 + 16, idesc, 1u);
                mma_el<MODE>(dcol, ad0, bd0, idesc, 1u);
                mma_el<MODE>(dcol, ad0 + 16, bd0 + 16, idesc, 1u);
              } else {
                mma_el<MODE>(dcol, ad0, bd0, idesc, first);
                mma_el<MODE>(dcol, ad0 + 16, bd0 + 16, idesc, 1u);
              }
              if (!P.b_resident) {
                mma_commit_el(&b_empty[slot]);
                if (++tb == my_size) { tb = 0; phb ^= 1; }
              }
            }
          }
          if (!ok) break;
          mma_commit_el(&a_empty[s]);
          if (((c * cw) >> 8) == r_me) mma_commit_el(&acc_full[as * 16 + c]);  // block c is final
          if (++sa_i == SA) { sa_i = 0; pha ^= 1; }
        }
      }
      }
      // every MMA of this CTA has completed before TMEM is released (issuer 0 waits for both)
      mma_commit_el(drain);
      if (r_me == 0) {
        unsigned long long t0 = now_ns();
        while (!mbar_test(drain, 0) && now_ns() - t0 < kWaitNs) {
        }
      }
    }
  } else if (warp == kLoadWarp || warp == kLoadWarp2) {
    // ===================== coordinates and L^-1 pieces =====================
    // Loader 0 copies each space's coordinates in, and the L^-1 pieces of
    // every region; with two issuers and streamed pieces, loader 1 takes
    // region 1's ring, so that neither ring waits behind the other.
    const int l_me = warp == kLoadWarp ? 0 : 1;
    const bool split = P.issuers == 2 && !P.b_resident;
    if (lane == 0 && (l_me == 0 || split)) {
      const int ccw = kChunkBytes / split_elem_bytes(MODE);
      const uint32_t b_base = smem_addr(sb);
      bool ok = true, b_loaded = false;
      int issued[kMaxBSlots], last_phase[kMaxBSlots], xs_issued[2] = {0, 0}, xs_phase[2] = {0, 0};
      for (int t = 0; t < kMaxBSlots; ++t) issued[t] = last_phase[t] = 0;
      int ks = -1, prev = -1, n_pad = 0, chunks = 0, n_max = 0;
      int rtb[2] = {0, 0};                       // next slot of each region's ring, and its phase
      uint32_t rph[2] = {0u, 0u};
      const uint8_t* lhi = nullptr;
      const uint8_t* llo = nullptr;
      Work w;
      for (bool more = work_begin(P, w); more && ok; more = work_next(P, w)) {
        if (w.sess != prev) {                    // next space: copy its coordinates in
          ++ks;
          prev = w.sess;
          const TcSess& S = sess_of(P, w.sess);
          n_pad = S.n_pad;
          chunks = S.chunks;
          n_max = S.n_max;
          lhi = S.lhi;
          llo = S.llo;
          if (l_me == 0) {
            const int xb = ks % XB;
            if (!(ok = mbar_wait(&xs_empty[xb], (uint32_t)(((ks / XB) & 1) ^ 1), abort_flag, status))) break;
            const uint32_t bytes = (uint32_t)(n_pad / 8) * 32u * (uint32_t)(S.ds + 2);
            mbar_arrive_tx(&xs_full[xb], bytes);
            bulk_g2s(xs_base + (uint32_t)(xb * P.x_buf_bytes), S.xq, bytes, &xs_full[xb]);
            xs_issued[xb] = 1;
            xs_phase[xb] = (ks / XB) & 1;
          }
        }
        if (P.b_resident && b_loaded) continue;  // every piece stays in shared memory
        int q = 0;
        uint32_t packed = 0;
        for (int c = 0; c < chunks && ok; ++c) {
          const size_t goff = (size_t)kChunkBytes * ((size_t)c * n_max - (size_t)ccw * c * (c - 1) / 2);
          for (int r = 0; r < 2 && ok; ++r) {
            int r0, wd;
            if (split && r != l_me) continue;    // the other loader's region
            if (!piece_of(c, r, ccw, n_pad, &r0, &wd)) continue;
            const uint32_t bytes = (uint32_t)((wd >> 3) * 512);
            const size_t src = goff + (size_t)(r0 - c * ccw) / 8 * 512;
            const int slot = P.b_resident ? q : ring_base(P, r) + rtb[r];
            if (!P.b_resident && !(ok = mbar_wait(&b_empty[slot], rph[r] ^ 1u, abort_flag, status))) break;
            const uint32_t dst = b_base + (P.b_resident ? packed : (uint32_t)(slot * P.b_slot_bytes));
            mbar_arrive_tx(&b_full[slot], bytes * parts);
            bulk_g2s(dst, lhi + src, bytes, &b_full[slot]);
            if (parts == 2) bulk_g2s(dst + bytes, llo + src, bytes, &b_full[slot]);
            issued[slot] = 1;
            last_phase[slot] = P.b_resident ? 0 : (int)rph[r];
            packed += bytes * (uint32_t)parts;
            ++q;
            if (!P.b_resident && ++rtb[r] == ring_size(P, r)) { rtb[r] = 0; rph[r] ^= 1u; }
          }
        }
        b_loaded = true;
      }
      // copies land on their own; wait for the last one of each barrier before exit
      for (int t = 0; t < kMaxBSlots; ++t)
        if (issued[t]) {
          unsigned long long t0 = now_ns();
          while (!mbar_test(&b_full[t], (uint32_t)last_phase[t]) && now_ns() - t0 < kWaitNs) {
          }
        }
      for (int t = 0; t < 2; ++t)
        if (xs_issued[t]) {
          unsigned long long t0 = now_ns();
          while (!mbar_test(&xs_full[t], (uint32_t)xs_phase[t]) && now_ns() - t0 < kWaitNs) {
          }
        }
    }
  }

  // ---- teardown: TMEM release; one space: per-CTA variance sum
  pdl_trigger();           // the acquisition may be launched (it waits for completion)
  for (int o = 16; o > 0; o >>= 1) vsum += __shfl_xor_sync(0xffffffffu, vsum, o);
  if (warp >= kEpiWarp0 && warp < kMmaWarp && lane == 0) red[warp - kEpiWarp0] = vsum;
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(P.tmem_cols * P.acc_stages) : "memory");
  }
  if (P.batch) return;
  if (P.acq) {
    acquisition_tail(P, red[0] + red[1] + red[2] + red[3], reinterpret_cast<unsigned long long*>(smem));
    return;
  }
  if (threadIdx.x == 0) P.partial[blockIdx.x] = red[0] + red[1] + red[2] + red[3];   // the acquisition adds them
}

// dimension buckets: the distance loop runs over DMAX zero-padded coordinates
int dim_bucket(int d) { return d <= 4 ? 4 : d <= 7 ? 7 : d <= 9 ? 9 : 16; }

// Pipeline shapes chosen by the autotuner, per (precision, Matern nu = 5/2,
// dim bucket, padded n, batched): each key is its own kernel instantiation.
std::mutex g_tune_mu;
std::map<std::array<int, 5>, TcShape> g_tuned;
thread_local const TcShape* g_forced = nullptr;   // a shape being timed by the autotuner

TcShape shape_for(int precision, double nu, int dmax, int n_pad, bool batched) {
  if (g_forced) return *g_forced;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find({precision, nu == 2.5 ? 1 : 0, dmax, n_pad, batched ? 1 : 0});
  return it == g_tuned.end() ? TcShape{} : it->second;
}

// Launch one instantiation; cooperative launches (the acquisition tail's grid
// barrier needs every CTA resident) return -2 when the device refuses them.
template <int MODE, int DMAX, bool NU52>
int launch_mode(const TcParams& P, size_t smem, int grid, bool coop, cudaStream_t s) {
  static size_t configured[kMaxDevices] = {};
  if (!ensure_dynamic_smem((const void*)predict_tc_kernel<MODE, DMAX, NU52>, configured, smem)) return -1;
  if (!coop && P.batch == 0)   // one space: a dependent launch after its observation update
    return launch_ex(predict_tc_kernel<MODE, DMAX, NU52>, dim3(grid), dim3(kThreads), smem, s, pdl_enabled(), P) ==
                   cudaSuccess
               ? 1
               : -1;
  if (coop) {
    void* args[] = {const_cast<TcParams*>(&P)};
    if (cudaLaunchCooperativeKernel((const void*)predict_tc_kernel<MODE, DMAX, NU52>, dim3(grid), dim3(kThreads),
                                    args, smem, s) != cudaSuccess) {
      (void)cudaGetLastError();
      return -2;
    }
    return 1;
  }
  predict_tc_kernel<MODE, DMAX, NU52><<<grid, kThreads, smem, s>>>(P);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

template <int MODE, bool NU52>
int launch_dims(const TcParams& P, int dmax, size_t smem, int grid, bool coop, cudaStream_t s) {
  switch (dmax) {
    case 4: return launch_mode<MODE, 4, NU52>(P, smem, grid, coop, s);
    case 7: return launch_mode<MODE, 7, NU52>(P, smem, grid, coop, s);
    case 9: return launch_mode<MODE, 9, NU52>(P, smem, grid, coop, s);
    default: return launch_mode<MODE, 16, NU52>(P, smem, grid, coop, s);
  }
}

int dispatch(const TcParams& P, int precision, double nu, int dmax, size_t smem, int grid, cudaStream_t s,
             bool coop = false) {
  const bool nu52 = nu == 2.5;
  switch (precision) {
    case BO_PREC_FP16X3:
      return nu52 ? launch_dims<BO_PREC_FP16X3, true>(P, dmax, smem, grid, coop, s)
                  : launch_dims<BO_PREC_FP16X3, false>(P, dmax, smem, grid, coop, s);
    case BO_PREC_BF16X3:
      return nu52 ? launch_dims<BO_PREC_BF16X3, true>(P, dmax, smem, grid, coop, s)
                  : launch_dims<BO_PREC_BF16X3, false>(P, dmax, smem, grid, coop, s);
    case BO_PREC_TF32X3:
      return nu52 ? launch_dims<BO_PREC_TF32X3, true>(P, dmax, smem, grid, coop, s)
                  : launch_dims<BO_PREC_TF32X3, false>(P, dmax, smem, grid, coop, s);
    case BO_PREC_TF32:
      return nu52 ? launch_dims<BO_PREC_TF32, true>(P, dmax, smem, grid, coop, s)
                  : launch_dims<BO_PREC_TF32, false>(P, dmax, smem, grid, coop, s);
    default:
      return -1;
  }
}

// Shared-memory plan and pipeline depths for a launch whose spaces have at
// most n_pad_max padded observations and dmax coordinate rows.  resident_ok:
// the B pieces of the (single) space may stay resident.  Returns the dynamic
// shared-memory size, 0 if nothing fits.
size_t plan_smem(TcParams& P, int precision, int n_pad_max, int dmax, bool resident_ok, const TcShape& shape) {
  P.cw = kChunkBytes / split_elem_bytes(precision);
  P.parts = split_parts(precision);
  int cols = 32;
  while (cols < n_pad_max) cols <<= 1;
  if (cols > 512) return 0;
  P.tmem_cols = cols;
  P.acc_stages = 2 * cols <= 512 ? 2 : 1;
  P.issuers = n_pad_max > kPieceRows ? 2 : 1;
  const size_t a_stage = (size_t)P.parts * kPartBytes;
  P.x_buf_bytes = ((size_t)(dmax + 2) * n_pad_max * 4 + 127) / 128 * 128;   // coordinates, 1/s^2, alpha
  const size_t x_bytes = P.x_buf_bytes * P.xs_bufs;
  const size_t limit = 226 * 1024;   // dynamic part; the kernel's static shared memory is small
  size_t resident = 0;
  int pieces = 0;
  for (int c = 0; c < n_pad_max / P.cw; ++c)
    for (int r = 0; r < 2; ++r) {            // the pieces of piece_of(): region r of chunk c
      const int lo = std::max(c * P.cw, r * kPieceRows), hi = std::min((r + 1) * kPieceRows, n_pad_max);
      if (lo >= hi) continue;
      resident += (size_t)P.parts * ((hi - lo) / 8) * 512;
      ++pieces;
    }
  P.b_resident = (resident_ok && shape.b_resident >= 0 && pieces <= kMaxBSlots &&
                  resident <= (size_t)P.parts * 64 * 1024) ? 1 : 0;
  P.b_slots = shape.b_slots > 0 ? std::min(shape.b_slots, kMaxBSlots) : 4;
  if (P.issuers == 2 && P.b_slots < 2) return 0;   // one ring slot per region at least
  P.b_slot_bytes = (size_t)P.parts * (kPieceRows / 8) * 512;
  const size_t b_bytes = P.b_resident ? resident : P.b_slots * P.b_slot_bytes;
  const size_t fixed = ((b_bytes + 1023) / 1024) * 1024 + ((x_bytes + 1023) / 1024) * 1024 + kMuPartBytes + 512;
  if (fixed >= limit) return 0;
  int sa = (int)((limit - fixed) / a_stage);
  sa = std::min(sa, 8);          // ring slots advance by counters: any depth >= 2 works
  if (shape.stages_a > 0) sa = std::min(sa, shape.stages_a);
  if (sa < 2) return 0;
  P.stages_a = sa;
  P.off_b = (size_t)sa * a_stage;
  P.off_x = P.off_b + ((b_bytes + 1023) / 1024) * 1024;
  P.off_mu = (P.off_x + x_bytes + 15) / 16 * 16;
  P.off_bar = P.off_mu + kMuPartBytes;
  const size_t smem = P.off_bar + (size_t)(2 * sa + 2 * kMaxBSlots + kAccBars + 12) * 8 + 16;
  // every descriptor footprint stays inside its stage: A parts are 128 rows x
  // 64 B; a B piece [r0, r0 + w) ends at the end of its part
  if ((size_t)15 * 512 + 256 + 255 >= (size_t)kPartBytes) return 0;
  return smem <= limit ? smem : 0;
}

int num_sms() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

}  // namespace

// Self-test of the bounded mbarrier wait every role of the prediction kernel
// uses: one thread waits for a phase that nothing completes; the wait gives up
// after its limit, raises the abort flag and records BO_ERR_TIMEOUT.
__global__ void selftest_mbar_kernel(int32_t* status, int* abort_flag) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);                  // count 1, and no thread ever arrives
    (void)mbar_wait(&bar, 0, abort_flag, status);
  }
}

int launch_selftest_mbar(int32_t* status, int* abort_flag, cudaStream_t s) {
  selftest_mbar_kernel<<<1, 32, 0, s>>>(status, abort_flag);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

TcSess tc_session(const DevView& v, int n) {
  TcSess S{};
  S.codes = v.codes;
  S.vtab32 = v.vtab32;
  S.visited = v.visited;
  S.xq = v.xq;
  S.ds = v.ds;
  S.lhi = v.lsplit_hi;
  S.llo = v.lsplit_lo;
  S.mu = static_cast<float*>(v.mu);
  S.var = static_cast<float*>(v.var);
  S.N = v.N;
  S.N_pad = v.N_pad;
  S.d = v.d;
  S.n = n;
  S.n_pad = (n + 31) / 32 * 32;
  S.n_max = v.n_max;
  S.chunks = S.n_pad / (kChunkBytes / split_elem_bytes(v.precision));
  S.num_tiles = (int)(v.N_pad / kRows);
  return S;
}

namespace {

int launch_single(const DevView& v, int n, const PassArgs* a, cudaStream_t s) {
  if (n < 1 || n > v.n_max || v.precision == BO_PREC_FP64 || v.d > 16) return -1;
  TcParams P{};
  P.s0 = tc_session(v, n);
  if (P.s0.n_pad > v.n_max) return -1;
  P.batch = 0;
  P.xs_bufs = 1;
  P.partial = v.partial;
  P.stats = v.stats;
  P.status = &v.stats->status;
  const int dmax = dim_bucket(v.d);
  const size_t smem = plan_smem(P, v.precision, P.s0.n_pad, dmax, true,
                                shape_for(v.precision, v.nu, dmax, P.s0.n_pad, false));
  if (!smem) return -1;
  const int grid = predict_tc_grid(v);
  if (grid > v.max_partials) return -1;
  if (a) {
    if (grid > v.max_acq_blocks || a->result_slot < 0 || a->result_slot >= v.max_results) return -1;
    P.acq = 1;
    P.args = *a;
    P.result = v.results + a->result_slot;
    P.acq_partial = v.acq_partial;
    P.var_s = &v.stats->var_s;
  }
  return dispatch(P, v.precision, v.nu, dmax, smem, grid, s, a != nullptr);
}

}  // namespace

int predict_tc_grid(const DevView& v) { return std::min((int)(v.N_pad / kRows), num_sms()); }

int launch_predict_tc(const DevView& v, int n, int64_t /*n_unvisited*/, cudaStream_t s) {
  return launch_single(v, n, nullptr, s);
}

int launch_predict_acquire_tc(const DevView& v, int n, const PassArgs& a, cudaStream_t s) {
  return launch_single(v, n, &a, s);
}

int tc_plan_batch(const TcSess* sess, int count, int dmax, int grid, std::vector<TcSeg>* segs,
                  std::vector<int>* seg_begin) {
  // estimated time of one tile of space s, in microseconds on GB300: a
  // least-squares fit of per-CTA durations of a 256-space batched pass (1.3 %
  // residual) to per-tile, per-observation, per-observation-coordinate and
  // n^2 terms, plus a cost per segment (a space switch)
  (void)dmax;
  const double kSwitch = 0.55;
  std::vector<double> tile_cost(count);
  double total = 0.0;
  int nonempty = 0;
  for (int s = 0; s < count; ++s) {
    const double np = sess[s].n_pad;
    tile_cost[s] = 1.215 + 0.0272 * np + 3.53e-4 * np * sess[s].d + 1.61e-5 * np * np;
    total += tile_cost[s] * sess[s].num_tiles;
    nonempty += sess[s].num_tiles > 0;
  }
  total += kSwitch * (nonempty + grid);    // about one switch per space and per CTA
  segs->clear();
  seg_begin->assign(grid + 1, 0);
  int s = 0, t = 0;
  double acc = 0.0;
  for (int b = 0; b < grid; ++b) {
    (*seg_begin)[b] = (int)segs->size();
    const double goal = total * (b + 1) / grid;
    while (s < count) {
      if (t >= sess[s].num_tiles) { ++s; t = 0; continue; }
      // whole tiles of space s until this CTA's share is reached (the last CTA takes the rest)
      int take = sess[s].num_tiles - t;
      if (b + 1 < grid) {
        const double room = goal - acc;
        const int fit = (int)(room / tile_cost[s] + 0.5);
        take = std::min(take, std::max(fit, 0));
      }
      if (take <= 0) break;
      segs->push_back(TcSeg{s, t, t + take});
      acc += take * tile_cost[s] + kSwitch;
      t += take;
      if (t < sess[s].num_tiles) break;
    }
  }
  (*seg_begin)[grid] = (int)segs->size();
  return (int)segs->size();
}

int launch_predict_tc_batch(const TcBatchLaunch& L, cudaStream_t s) {
  if (L.count < 1 || L.precision == BO_PREC_FP64) return -1;
  TcParams P{};
  P.batch = L.count;
  P.sess = L.sess;
  P.segs = L.segs;
  P.seg_begin = L.seg_begin;
  P.seg_part = L.seg_part;
  P.status = L.status;
  P.xs_bufs = 2;
  const size_t smem = plan_smem(P, L.precision, L.n_pad_max, L.dmax, false,
                                shape_for(L.precision, L.nu, L.dmax, L.n_pad_max, true));
  if (!smem) return -1;
  return dispatch(P, L.precision, L.nu, L.dmax, smem, L.grid, s);
}

int tc_dim_bucket(int d) { return dim_bucket(d); }

void tc_force_shape(const TcShape* shape) { g_forced = shape; }

void tc_store_shape(int precision, double nu, int dmax, int n_pad, bool batched, const TcShape& shape) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[{precision, nu == 2.5 ? 1 : 0, dmax, n_pad, batched ? 1 : 0}] = shape;
}

bool tc_stored_shape(int precision, double nu, int dmax, int n_pad, bool batched, TcShape* shape) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find({precision, nu == 2.5 ? 1 : 0, dmax, n_pad, batched ? 1 : 0});
  if (it == g_tuned.end()) return false;
  *shape = it->second;
  return true;
}

}  // namespace bo
