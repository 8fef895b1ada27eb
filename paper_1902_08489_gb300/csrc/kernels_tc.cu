// Tensor-core (tcgen05, sm_103a) grouped complex block GEMM for the mixed
// precision contractions: C (M x N) = alpha * sum_terms op(A) op(B) (+ C).
//
// Complex arithmetic on the real tensor pipe: with A read as a real M x 2K
// matrix (re/im interleaved along K, the storage order of complex numbers)
// and B expanded to its 2K x 2N real representation
//     [ br  bi ]
//     [ -bi br ]   per complex entry,
// the real product is the complex product with re/im interleaved along N,
// i.e. exactly the storage of C.  A tile is 128 rows (the TMEM lanes) by up
// to 64 complex columns (128 real accumulator columns), K in stages of 8
// complex.  Split TF32 (3xTF32) splits each operand into a TF32 head and a
// TF32 tail and accumulates hi*hi + hi*lo + lo*hi; BF16 rounds both operands
// to BF16 (kind::f16, FP32 accumulation).
//
// The kernel is persistent (one CTA per SM walking a host-built tile list)
// and warp-specialised:
//   warps 0..7   producers.  The symmetry blocks are ragged and addressed
//                through arbitrary leading dimensions and operand modes, so
//                every element of a stage is fetched on its own: cp.async
//                copies the raw complex-float operands of a stage into a
//                ring of TC_NR raw slots (zero-filled past K) TC_NR - 1
//                stages ahead of use; a thread later reads back the elements
//                it fetched, applies the term coefficient and conjugation,
//                splits them into TF32 (or BF16) pieces with integer
//                operations and stores them in the canonical K-major
//                no-swizzle layout of a ring of TC_NS MMA stages
//                (full[s] / empty[s] mbarriers);
//   warp 12      issues tcgen05.mma for every stage into one of two TMEM
//                accumulators (acc_full[a] / acc_empty[a]) and commits;
//   warps 8..11  epilogue: drain an accumulator with tcgen05.ld (warp w
//                reads TMEM lanes 32 (w - 8) ..), scale by alpha and store
//                (split-K tasks store their slice of the partial buffer),
//                while the MMAs of the next tile run into the other
//                accumulator.
// FP64 work (device coefficients) is done by one lane per warp; the operand
// path issues no FP64 or conversion instruction (on this part the FP64 pipe,
// which also executes conversions, is the narrow one).
//
// Every wait is bounded: a timeout sets the error word and a CTA-wide abort
// flag, after which every role stops waiting and leaves, the MMA warp waits
// (bounded) for its issued MMAs, and the TMEM columns are released.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.hpp"

namespace tdmps {

namespace {

constexpr int TC_BM = 128;        // rows per tile (TMEM lanes)
constexpr int TC_BNC = 64;        // complex columns per tile
constexpr int TC_BKC = 8;         // complex K per stage
constexpr int TC_KR = 2 * TC_BKC; // real K per stage (16 tf32 = 2 MMA k-steps)
constexpr int TC_NREAL = 2 * TC_BNC;
constexpr uint32_t TC_SPIN_LIMIT = 1u << 22;

constexpr int TC_NS = 4;          // MMA stages in the ring
constexpr int TC_NR = 4;          // raw operand slots (prefetch depth + 1)
constexpr int TC_PROD_WARPS = 8;
constexpr int TC_PROD = TC_PROD_WARPS * 32;
constexpr int TC_EPI_WARP0 = 8;
constexpr int TC_MMA_WARP = 12;
constexpr int TC_THREADS = 13 * 32;
constexpr int TC_ACC_COLS = 128;  // real columns per accumulator
constexpr int TC_TMEM_ALLOC = 2 * TC_ACC_COLS;

// per producer thread and stage: 4 complex of A (one row) and 2 of B (one column)
constexpr int TC_AEL = TC_BM * TC_BKC / TC_PROD;    // 4
constexpr int TC_BEL = TC_BNC * TC_BKC / TC_PROD;   // 2
constexpr int RAW_BYTES = (TC_AEL + TC_BEL) * TC_PROD * 8;   // 12 KB per raw slot

// bytes of one staged operand tile (rows x 16 tf32)
constexpr int TILE_A_BYTES = TC_BM * TC_KR * 4;       // 8 KB
constexpr int TILE_B_BYTES = TC_NREAL * TC_KR * 4;    // 8 KB

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// canonical K-major, no-swizzle layout: element (r, k) of a rows x 16 tf32 tile
__device__ __forceinline__ int canon_off(int r, int k) {
  return ((r >> 3) * (TC_KR / 4) + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

// shared-memory matrix descriptor: start address, leading byte offset (next
// core matrix along K), stride byte offset (next 8-row group), version 1,
// no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  const uint64_t lbo = 128, sbo = (TC_KR / 4) * 128;
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// BF16 operands: element (r, k) of a rows x 16 tile, 2-byte elements
__device__ __forceinline__ int canon_off16(int r, int k) {
  return ((r >> 3) * 2 + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ uint64_t make_desc16(uint32_t saddr) {
  const uint64_t lbo = 128, sbo = 2 * 128;
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// instruction descriptor: F32 accumulator, BF16 A and B (kind::f16), K-major
__device__ __forceinline__ uint32_t make_idesc_bf16(int n_real) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n_real >> 3) << 17) |
         ((uint32_t)(TC_BM >> 4) << 24);
}
// instruction descriptor: F32 accumulator, TF32 A and B, both K-major
__device__ __forceinline__ uint32_t make_idesc_tf32(int n_real) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n_real >> 3) << 17) |
         ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      :
      : "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
      :
      : "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
               :
               : "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" : : "r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" : : "r"(mbar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(mbar), "r"(phase)
      : "memory");
  return done != 0;
}
// bounded wait that also gives up once another role aborted
__device__ __forceinline__ bool wait_or_abort(uint32_t mbar, uint32_t phase,
                                              volatile int* abort_flag, int* err) {
  for (uint32_t it = 0; it < TC_SPIN_LIMIT; ++it) {
    if (mbar_try(mbar, phase)) return true;
    if ((it & 255u) == 255u && *abort_flag) return false;
  }
  atomicExch(err, 2);
  *abort_flag = 1;
  return false;
}

// the same wait taken by lane 0 for the whole warp (every lane then sees the
// same outcome, so warp-collective instructions after it stay converged)
__device__ __forceinline__ bool warp_wait(uint32_t mbar, uint32_t phase, volatile int* abort_flag,
                                          int* err) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = wait_or_abort(mbar, phase, abort_flag, err) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}

// 8-byte asynchronous copy global -> shared; src_bytes = 0 fills zeros
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n"
               :
               : "r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" : : "n"(N) : "memory");
}

// x rounded to TF32 (nearest, ties away from zero) on the integer ALU: the
// tensor pipe reads the top 19 bits of a 32-bit operand, so adding half a
// unit of the 13 dropped bits to the magnitude and clearing them is the
// rounding.  The split of split TF32 is head = tf32(x), tail = tf32(x - head)
// (x - head is exact in FP32).
__device__ __forceinline__ float tf32_head(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
// BF16 bits of x rounded to nearest even (finite x)
__device__ __forceinline__ uint32_t bf16_bits(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}
// FP32 -> FP64 by exponent rebias on the integer ALU (the conversion
// instruction runs on the narrow FP64 pipe); subnormal, Inf and NaN inputs
// take the conversion instruction
__device__ __forceinline__ double f32_to_f64(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t e = (u >> 23) & 0xFFu;
  if ((u & 0x7FFFFFFFu) == 0u)   // signed zero
    return __longlong_as_double((long long)((unsigned long long)(u >> 31) << 63));
  if (e == 0u || e == 0xFFu) return (double)x;
  const unsigned long long b = ((unsigned long long)(u >> 31) << 63) |
                               ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)b);
}
__device__ __forceinline__ double2 f2_to_d2(float re, float im) {
  return make_double2(f32_to_f64(re), f32_to_f64(im));
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return bf16_bits(lo) | (bf16_bits(hi) << 16);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// address of element (r, c) of op(P), P complex float with leading dimension ld
__device__ __forceinline__ const float2* el_addr(const void* P, int ld, int op, int r, int c) {
  const size_t idx = (op == OP_N || op == OP_J) ? (size_t)r * ld + c : (size_t)c * ld + r;
  return (const float2*)P + idx;
}
__device__ __forceinline__ bool op_conj(int op) { return op == OP_C || op == OP_J; }

// One K stage of one tile, as a producer thread walks them
struct Item {
  int tile, s, e, k0;   // tile index, stage within the tile, term, complex K offset
};
// What the conversion of an issued stage needs (one per raw slot)
struct Pend {
  int valid, arow, bcol, conj_a, conj_b;
  float2 sc;
};

template <int MODE>   // 0: TF32, 1: 3xTF32, 2: BF16
__global__ void __launch_bounds__(TC_THREADS, 1) k_gemm_tc(const GemmTask* __restrict__ tasks,
                                                         const GemmTerm* __restrict__ terms,
                                                         const TcTile* __restrict__ tiles,
                                                         const GemmSeg* __restrict__ segs,
                                                         const SegOps* __restrict__ segops,
                                                         int ntiles, int* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr int NSPLIT = MODE == 1 ? 2 : 1;   // operand tiles per stage (hi[, lo])
  constexpr int A_BYTES = MODE == 2 ? TILE_A_BYTES / 2 : TILE_A_BYTES;
  constexpr int B_BYTES = MODE == 2 ? TILE_B_BYTES / 2 : TILE_B_BYTES;
  constexpr int STAGE_BYTES = NSPLIT * (A_BYTES + B_BYTES);
  unsigned char* raw = sm + TC_NS * STAGE_BYTES;
  __shared__ __align__(8) uint64_t full[TC_NS], empty[TC_NS], acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == TC_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 :
                 : "r"(smem_u32(&tmem_base)), "r"(TC_TMEM_ALLOC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (threadIdx.x == 0) {
    // one arrival per producer warp / epilogue warp (after __syncwarp): 256
    // arrivals on one barrier word per stage would serialise in shared memory
    for (int s = 0; s < TC_NS; ++s) {
      mbar_init(smem_u32(&full[s]), TC_PROD_WARPS);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&acc_full[a]), 1);
      mbar_init(smem_u32(&acc_empty[a]), 4);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp < TC_PROD_WARPS) {
    // ------------------------------------------------------------ producers
    const int p = threadIdx.x;
    const int ra_r = p & (TC_BM - 1);            // A: row of this thread
    const int ra_k = (p >> 7) * TC_AEL;          //    first complex K of its 4
    const int rb_n = p & (TC_BNC - 1);           // B: column of this thread
    const int rb_k = (p / TC_BNC) * TC_BEL;      //    first complex K of its TC_BEL
    // the stage being issued, with its tile's and term's fields kept in
    // registers while they stay the same (they are reloaded on a change only)
    Item cur{(int)blockIdx.x, 0, 0, 0};
    TcTile tl{};
    int tM = 0, topA = 0, topB = 0, tend = 0;
    // segmented task: this thread's A row (dim 0) or B column (dim 1) lies in
    // segment sseg at local index sidx; -1: not segmented
    int sdim = -1, sseg = 0, sidx = 0;
    const void* gA = nullptr;
    const void* gB = nullptr;
    int gK = 0, glda = 0, gldb = 0;
    float2 gsc = make_float2(1.f, 0.f);
    auto load_term = [&]() {
      const GemmTerm& g = terms[cur.e];
      gA = g.A;
      gB = g.B;
      gK = g.K;
      glda = g.lda;
      gldb = g.ldb;
      if (sdim >= 0) {   // this thread's segment block (null: zeros)
        const SegOps& so = segops[g.pad];
        if (sdim == 0) { gA = so.p[sseg]; glda = so.ld[sseg]; }
        else { gB = so.p[sseg]; gldb = so.ld[sseg]; }
      }
      gsc = g.fscale;
      if (g.scale_ptr) {   // a device coefficient: formed in FP64 by one lane
        float sx = 0.f, sy = 0.f;
        if (lane == 0) {
          const double2 q = *g.scale_ptr;
          sx = (float)(g.scale.x * q.x - g.scale.y * q.y);
          sy = (float)(g.scale.x * q.y + g.scale.y * q.x);
        }
        gsc = make_float2(__shfl_sync(0xffffffffu, sx, 0), __shfl_sync(0xffffffffu, sy, 0));
      }
    };
    auto first = [&]() {   // the first stage of the next tile that has K stages
      while (cur.tile < ntiles && tiles[cur.tile].count <= 0) cur.tile += gridDim.x;
      if (cur.tile >= ntiles) return;
      tl = tiles[cur.tile];
      const GemmTask& t = tasks[tl.task];
      tM = t.M;
      topA = t.opA;
      topB = t.opB;
      tend = t.term_end;
      sdim = -1;
      if (t.seg1) {
        const GemmSeg& sg = segs[t.seg1 - 1];
        sdim = sg.dim;
        const int x = sdim == 0 ? tl.m0 + ra_r : tl.n0 + rb_n;
        sseg = 0;
        while (sseg + 1 < sg.n && x >= sg.off[sseg + 1]) ++sseg;
        sidx = x - sg.off[sseg];
      }
      cur.s = 0;
      cur.e = tl.e0;
      cur.k0 = tl.k0;
      load_term();
    };
    first();
    // issue the copies of `cur` into raw slot r and step `cur` forward
    auto issue = [&](Pend& pd, int r) {
      pd.valid = cur.tile < ntiles;
      if (pd.valid) {
        pd.arow = tl.m0 + ra_r < tM;
        pd.bcol = rb_n < tl.ncols;
        pd.conj_a = op_conj(topA);
        pd.conj_b = op_conj(topB);
        pd.sc = gsc;
        const uint32_t base = smem_u32(raw + r * RAW_BYTES);
        if (pd.arow) {
          const int row = sdim == 0 ? sidx : tl.m0 + ra_r;
          const bool live = gA != nullptr;
#pragma unroll
          for (int j = 0; j < TC_AEL; ++j) {
            const int k = cur.k0 + ra_k + j;
            const bool in = live && k < gK;
            const void* src = in ? (const void*)el_addr(gA, glda, topA, row, k) : (const void*)tasks;
            cp_async8(base + (j * TC_PROD + p) * 8, src, in ? 8u : 0u);
          }
        }
        if (pd.bcol) {
          const int col = sdim == 1 ? sidx : tl.n0 + rb_n;
          const bool live = gB != nullptr;
#pragma unroll
          for (int j = 0; j < TC_BEL; ++j) {
            const int k = cur.k0 + rb_k + j;
            const bool in = live && k < gK;
            const void* src = in ? (const void*)el_addr(gB, gldb, topB, k, col) : (const void*)tasks;
            cp_async8(base + ((TC_AEL + j) * TC_PROD + p) * 8, src, in ? 8u : 0u);
          }
        }
        // next stage
        if (++cur.s >= tl.count) {
          cur.tile += gridDim.x;
          first();
        } else {
          cur.k0 += TC_BKC;
          if (cur.k0 >= gK) {
            do { ++cur.e; } while (cur.e < tend && terms[cur.e].K <= 0);
            cur.k0 = 0;
            if (cur.e < tend) load_term();
          }
        }
      }
      cp_async_commit();
    };
    uint32_t g = 0;   // stages converted so far (MMA ring position)
    // convert the oldest issued stage (raw slot r) into the MMA ring
    auto convert = [&](const Pend& pd, int r) -> bool {
      cp_async_wait<TC_NR - 1>();
      if (!pd.valid) return false;
      const int slot = g % TC_NS;
      const uint32_t use = g / TC_NS;
      if (!warp_wait(smem_u32(&empty[slot]), (use & 1u) ^ 1u, &abort_flag, err)) return false;
      unsigned char* sA = sm + slot * STAGE_BYTES;
      unsigned char* sB = sA + NSPLIT * A_BYTES;
      const float2* rw = (const float2*)(raw + r * RAW_BYTES);
      // A: 128 rows x 8 complex; rows past M are left as they are (they only
      // reach accumulator rows that are never stored)
      if (pd.arow) {
#pragma unroll
        for (int j = 0; j < TC_AEL; ++j) {
          const int kk = ra_k + j;
          float2 a0 = rw[j * TC_PROD + p];
          if (pd.conj_a) a0.y = -a0.y;
          const float2 a = make_float2(pd.sc.x * a0.x - pd.sc.y * a0.y,
                                       pd.sc.x * a0.y + pd.sc.y * a0.x);
          if (MODE == 2) {
            *(uint32_t*)(sA + canon_off16(ra_r, 2 * kk)) = pack_bf16(a.x, a.y);
            continue;
          }
          const float2 hi = make_float2(tf32_head(a.x), tf32_head(a.y));
          *(float2*)(sA + canon_off(ra_r, 2 * kk)) = hi;
          if (MODE == 1)
            *(float2*)(sA + A_BYTES + canon_off(ra_r, 2 * kk)) =
                make_float2(tf32_head(a.x - hi.x), tf32_head(a.y - hi.y));
        }
      }
      // B-tilde (K-major, rows = real N): column n -> rows 2n (br, -bi), 2n+1 (bi, br)
      if (pd.bcol) {
#pragma unroll
        for (int j = 0; j < TC_BEL; ++j) {
          const int kk = rb_k + j;
          float2 bv = rw[(TC_AEL + j) * TC_PROD + p];
          if (pd.conj_b) bv.y = -bv.y;
          if (MODE == 2) {
            *(uint32_t*)(sB + canon_off16(2 * rb_n, 2 * kk)) = pack_bf16(bv.x, -bv.y);
            *(uint32_t*)(sB + canon_off16(2 * rb_n + 1, 2 * kk)) = pack_bf16(bv.y, bv.x);
            continue;
          }
          const float2 r0 = make_float2(bv.x, -bv.y), r1 = make_float2(bv.y, bv.x);
          const float2 h0 = make_float2(tf32_head(r0.x), tf32_head(r0.y));
          const float2 h1 = make_float2(tf32_head(r1.x), tf32_head(r1.y));
          *(float2*)(sB + canon_off(2 * rb_n, 2 * kk)) = h0;
          *(float2*)(sB + canon_off(2 * rb_n + 1, 2 * kk)) = h1;
          if (MODE == 1) {
            *(float2*)(sB + B_BYTES + canon_off(2 * rb_n, 2 * kk)) =
                make_float2(tf32_head(r0.x - h0.x), tf32_head(r0.y - h0.y));
            *(float2*)(sB + B_BYTES + canon_off(2 * rb_n + 1, 2 * kk)) =
                make_float2(tf32_head(r1.x - h1.x), tf32_head(r1.y - h1.y));
          }
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&full[slot]));
      ++g;
      return true;
    };
    // TC_NR raw slots rotated through registers (the unrolled loop keeps
    // every index a constant): issue TC_NR - 1 stages ahead, then alternate
    // issue / convert
    Pend q[TC_NR];
#pragma unroll
    for (int j = 0; j < TC_NR - 1; ++j) issue(q[j], j);
    bool go = true;
    while (go) {
#pragma unroll
      for (int j = 0; j < TC_NR; ++j) {
        if (go) {
          issue(q[(j + TC_NR - 1) % TC_NR], (j + TC_NR - 1) % TC_NR);
          if (abort_flag || !convert(q[j], j)) go = false;
        }
      }
    }
    cp_async_wait<0>();
  } else if (warp == TC_MMA_WARP) {
    // ------------------------------------------------------------ MMA issuer
    uint32_t g = 0, v = 0;   // stages consumed, accumulator uses
    bool issued = false;
    uint32_t last_bar = 0, last_phase = 0;
    for (int tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x) {
      const TcTile tl = tiles[tile];
      if (tl.count <= 0) continue;
      const int acc = v & 1;
      const uint32_t vuse = v >> 1;
      if (!warp_wait(smem_u32(&acc_empty[acc]), (vuse & 1u) ^ 1u, &abort_flag, err)) break;
      tc_fence_after();
      const int nreal = ((2 * tl.ncols + 15) / 16) * 16;
      const uint32_t idesc = MODE == 2 ? make_idesc_bf16(nreal) : make_idesc_tf32(nreal);
      const uint32_t dacc = tmem + (uint32_t)(acc * TC_ACC_COLS);
      bool ok = true;
      for (int s = 0; s < tl.count; ++s, ++g) {
        const int slot = g % TC_NS;
        const uint32_t use = g / TC_NS;
        if (!warp_wait(smem_u32(&full[slot]), use & 1u, &abort_flag, err)) { ok = false; break; }
        tc_fence_after();
        if (lane == 0) {
          const uint32_t a0 = smem_u32(sm + slot * STAGE_BYTES);
          const uint32_t b0 = a0 + NSPLIT * A_BYTES;
          if (MODE == 2) {
            mma_bf16(dacc, make_desc16(a0), make_desc16(b0), idesc, s > 0 ? 1u : 0u);
          } else {
#pragma unroll
            for (int q = 0; q < TC_KR / 8; ++q) {
              const uint32_t off = q * 256;
              mma_tf32(dacc, make_desc(a0 + off), make_desc(b0 + off), idesc,
                       (s > 0 || q > 0) ? 1u : 0u);
              if (MODE == 1) {
                mma_tf32(dacc, make_desc(a0 + off), make_desc(b0 + B_BYTES + off), idesc, 1u);
                mma_tf32(dacc, make_desc(a0 + A_BYTES + off), make_desc(b0 + off), idesc, 1u);
              }
            }
          }
          mma_commit(smem_u32(&empty[slot]));
        }
        __syncwarp();
        issued = true;
        last_bar = smem_u32(&empty[slot]);
        last_phase = use & 1u;
      }
      if (!ok) break;
      if (lane == 0) mma_commit(smem_u32(&acc_full[acc]));
      __syncwarp();
      ++v;
    }
    // no MMA of this CTA may still run when the columns are released
    if (issued && abort_flag)
      for (uint32_t it = 0; it < TC_SPIN_LIMIT && !mbar_try(last_bar, last_phase); ++it) {
      }
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - TC_EPI_WARP0;      // TMEM lanes 32 ew .. 32 ew + 31
    uint32_t v = 0;
    for (int tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x) {
      // the task and its segments copied into registers: the stores below
      // then cannot force reloads of them
      const TcTile tl = tiles[tile];
      const GemmTask t = tasks[tl.task];
      const bool split = t.splits > 1;
      const bool have = tl.count > 0;
      // alpha in FP64 (device scalars) by one lane, shared by the warp
      float ax = 0.f, ay = 0.f;
      if (lane == 0) {
        double2 alpha = t.alpha;
        if (t.alpha_ptr) {
          const double2 q = *t.alpha_ptr;
          alpha = make_double2(alpha.x * q.x - alpha.y * q.y, alpha.x * q.y + alpha.y * q.x);
        }
        if (t.alpha_div) {
          const double2 q = *t.alpha_div;
          const double d = q.x * q.x + q.y * q.y;
          alpha = make_double2((alpha.x * q.x + alpha.y * q.y) / d,
                               (alpha.y * q.x - alpha.x * q.y) / d);
        }
        ax = (float)alpha.x;
        ay = (float)alpha.y;
      }
      const float fax = __shfl_sync(0xffffffffu, ax, 0), fay = __shfl_sync(0xffffffffu, ay, 0);
      const int acc = v & 1;
      const uint32_t vuse = v >> 1;
      if (have) {
        if (!warp_wait(smem_u32(&acc_full[acc]), vuse & 1u, &abort_flag, err)) break;
        tc_fence_after();
      }
      const int row = tl.m0 + 32 * ew + lane;
      const int nchunk = (2 * tl.ncols + 31) / 32;
      // segmented output: the segment of this lane's row (dim 0), or of each
      // column (dim 1)
      // segments in scalar registers: segment of index x = number of segment
      // starts at or below it (unused segments start at the total extent)
      int sdim = -1, o1 = 0, o2 = 0, o3 = 0, l0 = 0, l1 = 0, l2 = 0, l3 = 0;
      void *c0 = nullptr, *c1 = nullptr, *c2 = nullptr, *c3 = nullptr;
      if (t.seg1) {
        const GemmSeg& sg = segs[t.seg1 - 1];
        sdim = sg.dim;
        o1 = sg.off[1]; o2 = sg.off[2]; o3 = sg.off[3];
        c0 = sg.C[0]; c1 = sg.C[1]; c2 = sg.C[2]; c3 = sg.C[3];
        l0 = sg.ldc[0]; l1 = sg.ldc[1]; l2 = sg.ldc[2]; l3 = sg.ldc[3];
      }
      auto seg_of = [&](int x) { return (int)(x >= o1) + (int)(x >= o2) + (int)(x >= o3); };
      const int rseg = sdim == 0 ? seg_of(row) : 0;
      for (int c = 0; c < nchunk; ++c) {
        float vv[32];
        if (have) {
          tmem_ld32(tmem + (uint32_t)(acc * TC_ACC_COLS) + ((uint32_t)(32 * ew) << 16) +
                        (uint32_t)(32 * c),
                    vv);
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) vv[i] = 0.f;
        }
        if (have && c == nchunk - 1) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&acc_empty[acc]));
        }
        if (row >= t.M) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = tl.n0 + 16 * c + j;
          if (col >= tl.n0 + tl.ncols) break;
          const float xr = vv[2 * j], xi = vv[2 * j + 1];
          const float ore = fax * xr - fay * xi, oim = fax * xi + fay * xr;
          if (split) {   // this split's slice; launch_reduce_splits adds them in order
            const size_t o = ((size_t)tl.split * t.M + row) * t.N + col;
            ((float2*)t.part)[o] = make_float2(ore, oim);
            continue;
          }
          void* Cb = t.C;
          size_t o;
          if (sdim >= 0) {
            const int s = sdim == 0 ? rseg : seg_of(col);
            Cb = s == 0 ? c0 : s == 1 ? c1 : s == 2 ? c2 : c3;
            const int ld = s == 0 ? l0 : s == 1 ? l1 : s == 2 ? l2 : l3;
            const int base = s == 0 ? 0 : s == 1 ? o1 : s == 2 ? o2 : o3;
            o = sdim == 0 ? (size_t)(row - base) * ld + col : (size_t)row * ld + (col - base);
          } else {
            o = t.ct ? (size_t)col * t.ldc + row : (size_t)row * t.ldc + col;
          }
          if (t.tc == 0) {
            double2* C = (double2*)Cb + o;
            double2 out = f2_to_d2(ore, oim);
            if (t.beta) { out.x += C->x; out.y += C->y; }
            *C = out;
          } else {
            float2* C = (float2*)Cb + o;
            float2 out = make_float2(ore, oim);
            if (t.beta) { out.x += C->x; out.y += C->y; }
            *C = out;
          }
        }
      }
      if (have) ++v;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == TC_MMA_WARP) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n"
                 :
                 : "r"(tmem), "r"(TC_TMEM_ALLOC)
                 : "memory");
  }
}

// C of a split task = sum of its part slices in split order (+ C when beta):
// one CTA per chunk of a task's elements, the same summation order on every run
__global__ void k_reduce_splits(const GemmTask* __restrict__ tasks,
                                const GemmSeg* __restrict__ segs, const int* __restrict__ chunks,
                                int f32_parts) {
  const int* ch = chunks + 3 * blockIdx.x;
  const GemmTask t = tasks[ch[0]];
  GemmSeg sgv{};
  if (t.seg1) sgv = segs[t.seg1 - 1];
  const GemmSeg* sg = t.seg1 ? &sgv : nullptr;
  const size_t mn = (size_t)t.M * t.N;
  for (size_t i = (size_t)ch[1] + threadIdx.x; i < (size_t)ch[2]; i += blockDim.x) {
    const int r = (int)(i / t.N), c = (int)(i % t.N);
    void* Cb = t.C;
    size_t o;
    if (sg) {
      const int x = sg->dim == 0 ? r : c;
      int s = 0;
      while (s + 1 < sg->n && x >= sg->off[s + 1]) ++s;
      Cb = sg->C[s];
      o = sg->dim == 0 ? (size_t)(r - sg->off[s]) * sg->ldc[s] + c
                       : (size_t)r * sg->ldc[s] + (c - sg->off[s]);
    } else {
      o = t.ct ? (size_t)c * t.ldc + r : (size_t)r * t.ldc + c;
    }
    if (t.tc == 0 && !f32_parts) {
      // FP64 slices of the FP64 kernel
      const double2* P = (const double2*)t.part;
      double2 s = P[i];
      for (int q = 1; q < t.splits; ++q) {
        const double2 x = P[q * mn + i];
        s.x += x.x;
        s.y += x.y;
      }
      double2* C = (double2*)Cb + o;
      if (t.beta) { s.x += C->x; s.y += C->y; }
      *C = s;
    } else if (t.tc == 0) {
      // FP64 output: FP32 slices of the tensor-core kernel, added in FP64
      const float2* P = (const float2*)t.part;
      double2 s = f2_to_d2(P[i].x, P[i].y);
      for (int q = 1; q < t.splits; ++q) {
        const double2 x = f2_to_d2(P[q * mn + i].x, P[q * mn + i].y);
        s.x += x.x;
        s.y += x.y;
      }
      double2* C = (double2*)Cb + o;
      if (t.beta) { s.x += C->x; s.y += C->y; }
      *C = s;
    } else {
      const float2* P = (const float2*)t.part;
      float2 s = P[i];
      for (int q = 1; q < t.splits; ++q) {
        const float2 x = P[q * mn + i];
        s.x += x.x;
        s.y += x.y;
      }
      float2* C = (float2*)Cb + o;
      if (t.beta) { s.x += C->x; s.y += C->y; }
      *C = s;
    }
  }
}

}  // namespace

int tc_smem_bytes(int mode) {
  const int stage = mode == 1 ? 2 * (TILE_A_BYTES + TILE_B_BYTES)
                              : mode == 2 ? (TILE_A_BYTES + TILE_B_BYTES) / 2
                                          : TILE_A_BYTES + TILE_B_BYTES;
  return TC_NS * stage + TC_NR * RAW_BYTES;
}

void launch_gemm_tc(const GemmTask* d_tasks, const GemmTerm* d_terms, const TcTile* d_tiles,
                    const GemmSeg* d_segs, const SegOps* d_segops, int ntiles, int mode, int n_sm,
                    int* d_err, cudaStream_t st) {
  if (ntiles <= 0) return;
  const int grid = ntiles < n_sm ? ntiles : n_sm;
  const int smem = tc_smem_bytes(mode);
  if (mode == 2) {
    set_smem_limit((const void*)k_gemm_tc<2>, smem);
    k_gemm_tc<2><<<grid, TC_THREADS, smem, st>>>(d_tasks, d_terms, d_tiles, d_segs, d_segops, ntiles, d_err);
  } else if (mode == 0) {
    set_smem_limit((const void*)k_gemm_tc<0>, smem);
    k_gemm_tc<0><<<grid, TC_THREADS, smem, st>>>(d_tasks, d_terms, d_tiles, d_segs, d_segops, ntiles, d_err);
  } else {
    set_smem_limit((const void*)k_gemm_tc<1>, smem);
    k_gemm_tc<1><<<grid, TC_THREADS, smem, st>>>(d_tasks, d_terms, d_tiles, d_segs, d_segops, ntiles, d_err);
  }
}

void launch_reduce_splits(const GemmTask* d_tasks, const GemmSeg* d_segs, const int* d_chunks,
                          int n, int f32_parts, cudaStream_t st) {
  if (n <= 0) return;
  k_reduce_splits<<<n, 256, 0, st>>>(d_tasks, d_segs, d_chunks, f32_parts);
}

int tc_stage_k() { return TC_BKC; }
int tc_tile_m() { return TC_BM; }
int tc_tile_n() { return TC_BNC; }

}  // namespace tdmps
