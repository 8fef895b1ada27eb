// Tensor-core (tcgen05, sm_103a) grouped complex block GEMM for the mixed
// precision contractions: C (M x N) = alpha * sum_terms op(A) op(B) (+ C).
//
// Complex arithmetic on the real tensor pipe: with A read as a real M x 2K
// matrix (re/im interleaved along K, the storage order of complex numbers)
// and B expanded to its 2K x 2N real representation
//     [ br  bi ]
//     [ -bi br ]   per complex entry,
// the real product is the complex product with re/im interleaved along N,
// i.e. exactly the storage of C.  Each CTA computes a 128 x N' real tile
// (N' <= 128, 64 complex columns) in TMEM; operands are staged by the CTA's
// threads in the canonical K-major no-swizzle layout (8-row x 16-byte core
// matrices) because the symmetry blocks are ragged and addressed through
// arbitrary leading dimensions and operand modes; one elected thread issues
// tcgen05.mma and commits to an mbarrier.  3xTF32 splits each operand into
// a TF32 head and a TF32 tail and accumulates hi*hi + hi*lo + lo*hi.  The
// BF16 mode rounds both operands to BF16 (kind::f16, FP32 accumulation).
//
// Every wait is bounded: a stuck barrier sets the error word, the CTA waits
// (bounded) for its own MMAs, frees its TMEM and returns.
#include <cuda_runtime.h>

#include <cuda_bf16.h>

#include <cstdint>

#include "kernels.hpp"

namespace tdmps {

namespace {

constexpr int TC_BM = 128;        // rows per tile (TMEM lanes)
constexpr int TC_BNC = 64;        // complex columns per tile
constexpr int TC_BKC = 8;         // complex K per stage
constexpr int TC_KR = 2 * TC_BKC; // real K per stage (16 tf32 = 2 MMA k-steps)
constexpr int TC_NR = 2 * TC_BNC; // real N per tile
constexpr int TC_THREADS = 256;
constexpr int TC_TMEM_COLS = 128;
constexpr uint32_t TC_SPIN_LIMIT = 1u << 22;

// bytes of one staged operand tile (rows x 16 tf32)
constexpr int TILE_A_BYTES = TC_BM * TC_KR * 4;   // 8 KB
constexpr int TILE_B_BYTES = TC_NR * TC_KR * 4;   // 8 KB

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// canonical K-major, no-swizzle layout: element (r, k) of a rows x 32 tile
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
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      :
      : "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *(uint32_t*)&v;
}

// instruction descriptor: F32 accumulator, TF32 A and B, both K-major
__device__ __forceinline__ uint32_t make_idesc_tf32(int n_real) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n_real >> 3) << 17) |
         ((uint32_t)(TC_BM >> 4) << 24);
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

// bounded wait on an mbarrier phase; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (uint32_t it = 0; it < TC_SPIN_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
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

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
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

// element (r, c) of op(P) (R x C), P of element type t (0 double2, 1 float2)
__device__ __forceinline__ float2 load_el(const void* P, int t, int ld, int op, int r, int c, int R,
                                          int C) {
  if (r >= R || c >= C) return make_float2(0.f, 0.f);
  size_t idx;
  bool conj = false;
  switch (op) {
    case OP_N: idx = (size_t)r * ld + c; break;
    case OP_T: idx = (size_t)c * ld + r; break;
    case OP_C: idx = (size_t)c * ld + r; conj = true; break;
    default: idx = (size_t)r * ld + c; conj = true; break;
  }
  float2 v;
  if (t == 0) {
    double2 d = ((const double2*)P)[idx];
    v = make_float2((float)d.x, (float)d.y);
  } else {
    v = ((const float2*)P)[idx];
  }
  if (conj) v.y = -v.y;
  return v;
}

template <int MODE>   // 0: TF32, 1: 3xTF32, 2: BF16
__global__ void __launch_bounds__(TC_THREADS, 3) k_gemm_tc(const GemmTask* __restrict__ tasks,
                                                        const GemmTerm* __restrict__ terms,
                                                        const int* __restrict__ tile_task,
                                                        int* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr int NSPLIT = MODE == 1 ? 2 : 1;                 // operand tiles per stage (hi[, lo])
  constexpr int BUF_BYTES = NSPLIT * (TILE_A_BYTES + TILE_B_BYTES);
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ float2 alpha_sh;

  const int ti = tile_task[blockIdx.x];
  const GemmTask t = tasks[ti];
  const int local = blockIdx.x - t.tile_base;
  const int split = local % t.splits;
  const int rest = local / t.splits;
  const int m0 = (rest % t.tiles_m) * TC_BM;
  const int n0 = (rest / t.tiles_m) * TC_BNC;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ncols = min(TC_BNC, t.N - n0);
  const int nreal = ((2 * ncols + 15) / 16) * 16;   // MMA N: multiple of 16
  const uint32_t idesc = MODE == 2 ? make_idesc_bf16(nreal) : make_idesc_tf32(nreal);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 :
                 : "r"(smem_u32(&tmem_base)), "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&mbar[0]), 1);
    mbar_init(smem_u32(&mbar[1]), 1);
    abort_flag = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  // stages of this task: (term, k0) pairs of TC_BKC complex, this split's share
  int S = 0;
  for (int e = t.term_begin; e < t.term_end; ++e) S += (terms[e].K + TC_BKC - 1) / TC_BKC;
  const int lo = (int)((long long)split * S / t.splits);
  const int hi = (int)((long long)(split + 1) * S / t.splits);
  int e = t.term_begin, k0 = 0;
  {
    int idx = 0;
    while (e < t.term_end) {
      const int nk = (terms[e].K + TC_BKC - 1) / TC_BKC;
      if (idx + nk <= lo) { idx += nk; ++e; continue; }
      k0 = (lo - idx) * TC_BKC;
      break;
    }
  }
  const int count = hi - lo;

  uint32_t uses[2] = {0u, 0u};
  bool ok = true;
  // The global loads of stage s + 1 are issued right after the MMAs of stage
  // s, into registers, so their latency overlaps the MMAs and the wait for
  // the next shared-memory buffer.
  const int ra_r = threadIdx.x & (TC_BM - 1);
  const int ra_k = (threadIdx.x >> 7) * (TC_BKC / 2);
  const int rb_n = threadIdx.x & (TC_BNC - 1);
  const int rb_k = (threadIdx.x >> 6) * (TC_BKC / 4);
  float2 ra[TC_BKC / 2], rb[TC_BKC / 4];
  float2 sc = make_float2(1.f, 0.f);
  // the term coefficient is formed in FP64 once per term, not per stage (the
  // FP64 pipe is the scarce unit: every thread computes it)
  int sc_term = -1;
  auto load_stage = [&](int ee, int kk0) {
    const GemmTerm g = terms[ee];
    if (ee != sc_term) {
      if (g.scale_ptr) {   // a coefficient that lives on the device: form it in FP64
        const double2 p = *g.scale_ptr;
        const double2 scd = make_double2(g.scale.x * p.x - g.scale.y * p.y,
                                         g.scale.x * p.y + g.scale.y * p.x);
        sc = make_float2((float)scd.x, (float)scd.y);
      } else {             // FP32 copy made on the host: no FP64 instruction here
        sc = g.fscale;
      }
      sc_term = ee;
    }
#pragma unroll
    for (int j = 0; j < TC_BKC / 2; ++j)
      ra[j] = load_el(g.A, t.ta, g.lda, t.opA, m0 + ra_r, kk0 + ra_k + j, t.M, g.K);
#pragma unroll
    for (int j = 0; j < TC_BKC / 4; ++j)
      rb[j] = load_el(g.B, t.tb, g.ldb, t.opB, kk0 + rb_k + j, n0 + rb_n, g.K, t.N);
  };
  if (count > 0) load_stage(e, k0);
  for (int s = 0; s < count && ok; ++s) {
    const int b = s & 1;
    unsigned char* sA = sm + b * BUF_BYTES;
    unsigned char* sB = sA + NSPLIT * TILE_A_BYTES;
    if (uses[b] > 0) {   // the MMAs that last read this buffer must be done
      if (!mbar_wait(smem_u32(&mbar[b]), (uses[b] - 1) & 1u)) {
        if (lane == 0) atomicExch(err, 2);
        abort_flag = 1;
      }
    }
    // Rows past M and columns past N are zero in every stage: each of the
    // two buffers receives those zeros in its first stage and keeps them, so
    // later stages skip them (whole warps when the block is short -- the
    // local-matvec outputs fill only a fraction of a 128 x 64 tile).
    const bool a_stage = s < 2 || m0 + ra_r < t.M;
    const bool b_stage = s < 2 || n0 + rb_n < t.N;
    // ---- A: 128 rows x 8 complex; thread -> row, 4 complex of K
#pragma unroll
    for (int j = 0; j < TC_BKC / 2 && a_stage; ++j) {
      const int kk = ra_k + j;
      const float2 a0 = ra[j];
      const float2 a = make_float2(sc.x * a0.x - sc.y * a0.y, sc.x * a0.y + sc.y * a0.x);
      if (MODE == 2) {
        *(uint32_t*)(sA + canon_off16(ra_r, 2 * kk)) = pack_bf16(a.x, a.y);
        continue;
      }
      const float2 hi = make_float2(to_tf32(a.x), to_tf32(a.y));
      *(float2*)(sA + canon_off(ra_r, 2 * kk)) = hi;
      if (MODE == 1) {
        const float2 lo2 = make_float2(to_tf32(a.x - hi.x), to_tf32(a.y - hi.y));
        *(float2*)(sA + TILE_A_BYTES + canon_off(ra_r, 2 * kk)) = lo2;
      }
    }
    // ---- B-tilde (K-major, rows = real N): thread -> column n, 2 complex of K
#pragma unroll
    for (int j = 0; j < TC_BKC / 4 && b_stage; ++j) {
      const int kk = rb_k + j;
      const float2 bv = rb[j];
      if (MODE == 2) {
        *(uint32_t*)(sB + canon_off16(2 * rb_n, 2 * kk)) = pack_bf16(bv.x, -bv.y);
        *(uint32_t*)(sB + canon_off16(2 * rb_n + 1, 2 * kk)) = pack_bf16(bv.y, bv.x);
        continue;
      }
      const float2 hr = make_float2(to_tf32(bv.x), to_tf32(-bv.y));   // row 2n:   (br, -bi)
      const float2 hi2 = make_float2(to_tf32(bv.y), to_tf32(bv.x));   // row 2n+1: (bi,  br)
      *(float2*)(sB + canon_off(2 * rb_n, 2 * kk)) = hr;
      *(float2*)(sB + canon_off(2 * rb_n + 1, 2 * kk)) = hi2;
      if (MODE == 1) {
        const float2 lr = make_float2(to_tf32(bv.x - hr.x), to_tf32(-bv.y - hr.y));
        const float2 li = make_float2(to_tf32(bv.y - hi2.x), to_tf32(bv.x - hi2.y));
        *(float2*)(sB + TILE_B_BYTES + canon_off(2 * rb_n, 2 * kk)) = lr;
        *(float2*)(sB + TILE_B_BYTES + canon_off(2 * rb_n + 1, 2 * kk)) = li;
      }
    }
    fence_async_smem();
    __syncthreads();
    if (abort_flag) { ok = false; break; }
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      if (MODE == 2) {   // one K = 16 step covers the stage
        mma_bf16(tmem, make_desc16(a0), make_desc16(b0), idesc, s > 0 ? 1u : 0u);
      } else
#pragma unroll
      for (int q = 0; q < TC_KR / 8; ++q) {
        const uint32_t off = q * 256;   // two core matrices along K per k-step
        mma_tf32(tmem, make_desc(a0 + off), make_desc(b0 + off), idesc, (s > 0 || q > 0) ? 1u : 0u);
        if (MODE == 1) {
          mma_tf32(tmem, make_desc(a0 + off), make_desc(b0 + TILE_B_BYTES + off), idesc, 1u);
          mma_tf32(tmem, make_desc(a0 + TILE_A_BYTES + off), make_desc(b0 + off), idesc, 1u);
        }
      }
      mma_commit(smem_u32(&mbar[b]));
    }
    uses[b] += 1;
    k0 += TC_BKC;
    while (e < t.term_end && k0 >= terms[e].K) { ++e; k0 = 0; }
    if (s + 1 < count) load_stage(e, k0);
  }
  // the last commit covers every MMA issued before it
  uint32_t failed_bar = 0, failed_phase = 0;
  bool pending = false;
  if (count > 0) {
    const int b = (count - 1) & 1;
    failed_bar = smem_u32(&mbar[b]);
    failed_phase = (uses[b] - 1) & 1u;
    pending = true;
    if (ok && !mbar_wait(failed_bar, failed_phase)) {
      if (lane == 0) atomicExch(err, 2);
      abort_flag = 1;   // the epilogue's TMEM loads are warp-collective: fail as a CTA
      ok = false;
    }
  }
  __syncthreads();
  tc_fence_after();
  if (abort_flag) ok = false;

  if (threadIdx.x == 0) {   // alpha in FP64, once per CTA
    double2 alpha = t.alpha;
    if (t.alpha_ptr) {
      double2 p = *t.alpha_ptr;
      alpha = make_double2(alpha.x * p.x - alpha.y * p.y, alpha.x * p.y + alpha.y * p.x);
    }
    if (t.alpha_div) {
      double2 q = *t.alpha_div;
      double d = q.x * q.x + q.y * q.y;
      alpha = make_double2((alpha.x * q.x + alpha.y * q.y) / d, (alpha.y * q.x - alpha.x * q.y) / d);
    }
    alpha_sh = make_float2((float)alpha.x, (float)alpha.y);
  }
  __syncthreads();
  if (ok) {
    const bool atomic = t.splits > 1;
    const int quad = warp & 3, chalf = warp >> 2;
    const bool have = count > 0;
    const float fax = alpha_sh.x, fay = alpha_sh.y;
    // Each warp moves its 32 x 16-complex chunk through a 4 KB shared-memory
    // scratch (the operand buffers, free once the last MMA completed) so
    // that the global writes run along rows: 16 lanes per 128-byte row.
    // Slots are XOR-swizzled by row so neither side has bank conflicts.
    float2* scr = (float2*)(sm + warp * 4096);
    const int hrow = lane >> 4, jj = lane & 15;
    for (int c0 = 32 * chalf; c0 < 2 * ncols; c0 += 64) {
      float v[32];
      if (have) {
        tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) scr[lane * 16 + (j ^ (lane & 15))] = make_float2(v[2 * j], v[2 * j + 1]);
      __syncwarp();
      const int jn = min(16, ncols - c0 / 2);
      // transposed tasks (C^T computed) write along C's rows = this tile's
      // columns: lanes over the 32 tile rows, one tile column at a time
      for (int it = 0; it < 16; ++it) {
        int rl, jc;
        if (t.ct) { rl = lane; jc = it; } else { rl = 2 * it + hrow; jc = jj; }
        const int row = m0 + quad * 32 + rl;
        const float2 x = scr[rl * 16 + (jc ^ (rl & 15))];
        if (row >= t.M || jc >= jn || !(have || !atomic)) continue;
        const size_t col = (size_t)n0 + c0 / 2 + jc;
        const size_t o = t.ct ? col * t.ldc + row : (size_t)row * t.ldc + col;
        if (t.tc == 0) {
          double2* C = (double2*)t.C + o;
          double ore = (double)(fax * x.x - fay * x.y), oim = (double)(fax * x.y + fay * x.x);
          if (atomic) {
            atomicAdd(&C->x, ore);
            atomicAdd(&C->y, oim);
          } else {
            if (t.beta) { ore += C->x; oim += C->y; }
            *C = make_double2(ore, oim);
          }
        } else {
          float2* C = (float2*)t.C + o;
          float ore = fax * x.x - fay * x.y, oim = fax * x.y + fay * x.x;
          if (atomic) {
            atomicAdd(&C->x, ore);
            atomicAdd(&C->y, oim);
          } else {
            if (t.beta) { ore += C->x; oim += C->y; }
            *C = make_float2(ore, oim);
          }
        }
      }
      __syncwarp();
    }
  } else if (pending) {
    // give this CTA's MMAs one more bounded chance to drain before the
    // accumulator columns are released
    mbar_wait(failed_bar, failed_phase);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n"
                 :
                 : "r"(tmem), "r"(TC_TMEM_COLS)
                 : "memory");
  }
}

// zero a list of (pointer, bytes) regions (outputs of split-K tasks)
__global__ void k_zero_regions(const ZeroRegion* __restrict__ r) {
  const ZeroRegion z = r[blockIdx.x];
  uint32_t* p = (uint32_t*)z.p;
  const size_t n = z.bytes / 4;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) p[i] = 0u;
}

}  // namespace

void launch_gemm_tc(const GemmTask* d_tasks, const GemmTerm* d_terms, const int* d_tile_task,
                    int ntiles, int mode, int* d_err, cudaStream_t st) {
  if (ntiles <= 0) return;
  if (mode == 2) {
    const int smem = 2 * (TILE_A_BYTES + TILE_B_BYTES);
    set_smem_limit((const void*)k_gemm_tc<2>, smem);
    k_gemm_tc<2><<<ntiles, TC_THREADS, smem, st>>>(d_tasks, d_terms, d_tile_task, d_err);
  } else if (mode == 0) {
    const int smem = 2 * (TILE_A_BYTES + TILE_B_BYTES);
    set_smem_limit((const void*)k_gemm_tc<0>, smem);
    k_gemm_tc<0><<<ntiles, TC_THREADS, smem, st>>>(d_tasks, d_terms, d_tile_task, d_err);
  } else {
    const int smem = 2 * 2 * (TILE_A_BYTES + TILE_B_BYTES);
    set_smem_limit((const void*)k_gemm_tc<1>, smem);
    k_gemm_tc<1><<<ntiles, TC_THREADS, smem, st>>>(d_tasks, d_terms, d_tile_task, d_err);
  }
}

void launch_zero_regions(const ZeroRegion* d_regions, int n, cudaStream_t st) {
  if (n <= 0) return;
  k_zero_regions<<<n, 256, 0, st>>>(d_regions);
}

int tc_stage_k() { return TC_BKC; }
int tc_tile_m() { return TC_BM; }
int tc_tile_n() { return TC_BNC; }

}  // namespace tdmps
