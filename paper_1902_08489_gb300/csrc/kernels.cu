// FP64 device kernels of the tdmps library: grouped complex block GEMM, sparse
// MPO-tensor application, block gather/scatter, one-sided Jacobi SVD, Gram-Schmidt
// QR, the truncation rule, and the small Krylov algebra.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <set>
#include <tuple>

#include "kernels.hpp"

namespace tdmps {

// Raise a kernel's dynamic shared-memory limit once per (device, kernel, size).
// Thread-safe; a failure is left for the launch to report.
void set_smem_limit(const void* func, int bytes) {
  static std::mutex mu;
  static std::set<std::tuple<int, const void*, int>> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_tuple(dev, func, bytes);
  if (done.count(key)) return;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess)
    done.insert(key);
}


// ------------------------------------------------------------------ complex helpers

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {   // a*b + c
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ grouped GEMM

constexpr int GT = 32;    // output tile edge
constexpr int GK = 8;     // K chunk

__device__ __forceinline__ double2 load_op(const double2* P, int ld, int op, int r, int c,
                                           int R, int C) {
  // element (r, c) of op(P) where op(P) is R x C
  if (r >= R || c >= C) return make_double2(0.0, 0.0);
  switch (op) {
    case OP_N: return P[(size_t)r * ld + c];
    case OP_T: return P[(size_t)c * ld + r];
    case OP_C: return cconj(P[(size_t)c * ld + r]);
    default: return cconj(P[(size_t)r * ld + c]);
  }
}

__global__ void __launch_bounds__(256) k_gemm(const GemmTask* __restrict__ tasks,
                                              const GemmTerm* __restrict__ terms,
                                              const int* __restrict__ tile_task) {
  __shared__ double2 As[GK][GT + 1];
  __shared__ double2 Bs[GK][GT + 1];
  const int ti = tile_task[blockIdx.x];
  const GemmTask t = tasks[ti];
  const int local = blockIdx.x - t.tile_base;
  const int split = local % t.splits;
  const int rest = local / t.splits;
  const int m0 = (rest % t.tiles_m) * GT;
  const int n0 = (rest / t.tiles_m) * GT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  // rows past the block edge do no arithmetic (a warp covers 4 rows, so a
  // short block leaves whole warps idle instead of multiplying zeros)
  const bool rows_live = m0 + 2 * ty < t.M;
  double2 acc[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0.0, 0.0);
  // this split's share of the task's K chunks (GK each, over all terms)
  int S = 0;
  for (int e = t.term_begin; e < t.term_end; ++e) S += (terms[e].K + GK - 1) / GK;
  const int lo = (int)((long long)split * S / t.splits);
  const int hi = (int)((long long)(split + 1) * S / t.splits);
  int idx = 0;
  for (int e = t.term_begin; e < t.term_end && idx < hi; ++e) {
    const GemmTerm g = terms[e];
    const int nk = (g.K + GK - 1) / GK;
    if (idx + nk <= lo) { idx += nk; continue; }
    double2 sc = g.scale;
    if (g.scale_ptr) sc = cmul(sc, *g.scale_ptr);
    const int c0 = lo > idx ? lo - idx : 0;
    const int c1 = hi - idx < nk ? hi - idx : nk;
    for (int ch = c0; ch < c1; ++ch) {
      const int k0 = ch * GK;
      {
        int i = threadIdx.x >> 3, k = threadIdx.x & 7;      // A tile: 32 x 8
        As[k][i] = cmul(sc, load_op((const double2*)g.A, g.lda, t.opA, m0 + i, k0 + k, t.M, g.K));
        int kk = threadIdx.x >> 5, j = threadIdx.x & 31;    // B tile: 8 x 32
        Bs[kk][j] = load_op((const double2*)g.B, g.ldb, t.opB, k0 + kk, n0 + j, g.K, t.N);
      }
      __syncthreads();
      if (rows_live) {
        if (k0 + GK <= g.K) {
#pragma unroll
          for (int k = 0; k < GK; ++k) {
            double2 a0 = As[k][ty * 2], a1 = As[k][ty * 2 + 1];
            double2 b0 = Bs[k][tx * 2], b1 = Bs[k][tx * 2 + 1];
            acc[0][0] = cfma(a0, b0, acc[0][0]);
            acc[0][1] = cfma(a0, b1, acc[0][1]);
            acc[1][0] = cfma(a1, b0, acc[1][0]);
            acc[1][1] = cfma(a1, b1, acc[1][1]);
          }
        } else {   // ragged last chunk: only the valid K
          const int kl = g.K - k0;
          for (int k = 0; k < kl; ++k) {
            double2 a0 = As[k][ty * 2], a1 = As[k][ty * 2 + 1];
            double2 b0 = Bs[k][tx * 2], b1 = Bs[k][tx * 2 + 1];
            acc[0][0] = cfma(a0, b0, acc[0][0]);
            acc[0][1] = cfma(a0, b1, acc[0][1]);
            acc[1][0] = cfma(a1, b0, acc[1][0]);
            acc[1][1] = cfma(a1, b1, acc[1][1]);
          }
        }
      }
      __syncthreads();
    }
    idx += nk;
  }
  double2 alpha = t.alpha;
  if (t.alpha_ptr) alpha = cmul(alpha, *t.alpha_ptr);
  if (t.alpha_div) alpha = cdiv(alpha, *t.alpha_div);
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      int r = m0 + ty * 2 + i, c = n0 + tx * 2 + j;
      if (r < t.M && c < t.N) {
        double2* p = (double2*)t.C + (t.ct ? (size_t)c * t.ldc + r : (size_t)r * t.ldc + c);
        double2 v = cmul(alpha, acc[i][j]);
        if (t.splits > 1) {
          ((double2*)t.part)[((size_t)split * t.M + r) * t.N + c] = v;
        } else {
          if (t.beta) v = cadd(v, *p);
          *p = v;
        }
      }
    }
}

void launch_gemm(const GemmTask* d_tasks, int ntasks, const GemmTerm* d_terms,
                 const int* d_tile_task, int ntiles, cudaStream_t st) {
  (void)ntasks;
  if (ntiles <= 0) return;
  k_gemm<<<ntiles, 256, 0, st>>>(d_tasks, d_terms, d_tile_task);
}

// ------------------------------------------------------------------ W stage

template <class T>
__device__ __forceinline__ double2 ld2(const T* p, size_t i);
template <>
__device__ __forceinline__ double2 ld2<double2>(const double2* p, size_t i) { return p[i]; }
template <>
__device__ __forceinline__ double2 ld2<float2>(const float2* p, size_t i) {
  float2 v = p[i];
  return make_double2(v.x, v.y);
}
template <class T>
__device__ __forceinline__ void st2(T* p, size_t i, double2 v);
template <>
__device__ __forceinline__ void st2<double2>(double2* p, size_t i, double2 v) { p[i] = v; }
template <>
__device__ __forceinline__ void st2<float2>(float2* p, size_t i, double2 v) {
  p[i] = make_float2((float)v.x, (float)v.y);
}

// accumulation type of the MPO stage: FP64 for complex double data, FP32 for
// complex float data (the FP64 pipe is the scarce unit on this part)
template <class T> struct WAcc;
template <> struct WAcc<double2> { using R = double; };
template <> struct WAcc<float2> { using R = float; };

// One thread per (output channel w, column b) and group of up to WS_ROWS
// rows a of a block: the CSR row of w (entries w_in, value) is walked once
// and applied to all of those rows, so the entry loads, the loop control and
// the index arithmetic are shared by WS_ROWS outputs; consecutive threads
// take consecutive columns, so every X read and Y write is coalesced along b.
constexpr int WS_ROWS = 2;

template <class T>
__global__ void __launch_bounds__(256) k_wstage(const WTask* __restrict__ tasks, int ntasks,
                                                int64_t total, const int* __restrict__ rowptr,
                                                const int* __restrict__ ent_w,
                                                const typename WAcc<T>::R* __restrict__ ent_v) {
  using R = typename WAcc<T>::R;
  // each CTA owns one contiguous range of the flat work index, so a thread
  // finds its task once (binary search) and then only steps forward
  const int64_t per = (total + gridDim.x - 1) / gridDim.x;
  const int64_t beg = (int64_t)blockIdx.x * per;
  const int64_t end = beg + per < total ? beg + per : total;
  int lo = 0;
  if (beg + threadIdx.x < end) {
    int hi = ntasks - 1;
    const int64_t first = beg + threadIdx.x;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (tasks[mid].work_base <= first) lo = mid; else hi = mid - 1;
    }
  }
  for (int64_t idx = beg + threadIdx.x; idx < end; idx += blockDim.x) {
    while (lo + 1 < ntasks && tasks[lo + 1].work_base <= idx) ++lo;
    const WTask& t = tasks[lo];
    // 32-bit index split (a task holds fewer than 2^31 work items)
    const int loc = (int)(idx - t.work_base);
    const int cols = t.cols, wout = t.wout;
    const int rw = loc / cols;
    const int b = loc - rw * cols;
    const int q = rw / wout;            // row group
    const int w = rw - q * wout;
    const int a0 = q * WS_ROWS;
    const int nr = t.rows - a0 < WS_ROWS ? t.rows - a0 : WS_ROWS;
    R ax[WS_ROWS], ay[WS_ROWS];
#pragma unroll
    for (int r = 0; r < WS_ROWS; ++r) ax[r] = ay[r] = 0;
    for (int s = 0; s < 4; ++s) {
      if (t.csr[s] < 0) continue;
      const int* rp = rowptr + t.csr[s];
      const int win = t.win[s];
      const size_t rstride = (size_t)win * cols;
      const T* X = (const T*)t.X[s] + (size_t)a0 * rstride + b;
      const int e1 = rp[w + 1];
      for (int e = rp[w]; e < e1; ++e) {
        const R v = ent_v[e];
        const T* xp = X + (size_t)ent_w[e] * cols;
#pragma unroll
        for (int r = 0; r < WS_ROWS; ++r) {
          if (r < nr) {   // constant indices: the accumulators stay in registers
            const T x = xp[r * rstride];
            ax[r] = fma(v, (R)x.x, ax[r]);
            ay[r] = fma(v, (R)x.y, ay[r]);
          }
        }
      }
    }
    const size_t ystride = (size_t)wout * cols;
    T* y = (T*)t.Y + (size_t)a0 * ystride + (size_t)w * cols + b;
#pragma unroll
    for (int r = 0; r < WS_ROWS; ++r) {
      if (r < nr) {
        T* yr = y + r * ystride;
        R ox = ax[r], oy = ay[r];
        if (t.beta) { ox += (R)yr->x; oy += (R)yr->y; }
        yr->x = ox;
        yr->y = oy;
      }
    }
  }
}

int wstage_rows_per_item() { return WS_ROWS; }

void launch_wstage(const WTask* d_tasks, int ntasks, int64_t total_work, const int* d_rowptr,
                   const int* d_ent_w, const double* d_ent_v, const float* d_ent_vf, int et,
                   cudaStream_t st) {
  if (total_work <= 0) return;
  int64_t blocks = (total_work + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (et == 0)
    k_wstage<double2><<<(int)blocks, 256, 0, st>>>(d_tasks, ntasks, total_work, d_rowptr, d_ent_w, d_ent_v);
  else
    k_wstage<float2><<<(int)blocks, 256, 0, st>>>(d_tasks, ntasks, total_work, d_rowptr, d_ent_w, d_ent_vf);
}

template <class T>
__global__ void k_to_double(const T* in, double2* out, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = ld2(in, i);
}

void launch_to_double(const void* in, int et, double2* out, size_t n, cudaStream_t st) {
  if (n == 0) return;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (et == 0) k_to_double<double2><<<(unsigned)blocks, 256, 0, st>>>((const double2*)in, out, n);
  else k_to_double<float2><<<(unsigned)blocks, 256, 0, st>>>((const float2*)in, out, n);
}

__global__ void k_to_float(const double2* in, float2* out, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    out[i] = make_float2((float)v.x, (float)v.y);
  }
}

void launch_to_float(const double2* in, float2* out, size_t n, cudaStream_t st) {
  if (n == 0) return;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_to_float<<<(unsigned)blocks, 256, 0, st>>>(in, out, n);
}

__global__ void k_fill_one(void* p, int et) {
  if (et == 0) *(double2*)p = make_double2(1.0, 0.0);
  else *(float2*)p = make_float2(1.f, 0.f);
}

void launch_fill_one(void* p, int et, cudaStream_t st) { k_fill_one<<<1, 1, 0, st>>>(p, et); }

// ------------------------------------------------------------------ gather / scatter

__global__ void k_copy(const CopyTask* __restrict__ tasks, int to_work) {
  const CopyTask t = tasks[blockIdx.x];
  int n = t.rows * t.cols;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    int i = e / t.cols, j = e % t.cols;
    size_t w = t.conj_t ? (size_t)(t.row0 + i) * t.ldw + (t.col0 + j)
                        : (size_t)(t.col0 + j) * t.ldw + (t.row0 + i);
    double2* b = t.blk + (size_t)i * t.ld + j;
    if (to_work) {
      double2 v = cmul(t.scale, *b);
      t.work[w] = t.conj_t ? cconj(v) : v;
    } else {
      double2 v = t.work[w];
      if (t.conj_t) v = cconj(v);
      *b = cmul(t.scale, v);
    }
  }
}

void launch_copy(const CopyTask* d_tasks, int ntasks, int to_work, cudaStream_t st) {
  if (ntasks <= 0) return;
  k_copy<<<ntasks, 256, 0, st>>>(d_tasks, to_work);
}

__global__ void k_scatter(const ScatterTask* __restrict__ tasks) {
  const ScatterTask t = tasks[blockIdx.x];
  int n = t.rows * t.cols;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    int i = e / t.cols, j = e % t.cols;
    double2 v = t.conj_t ? cconj(t.src[(size_t)(t.c0 + i) * t.lds + t.r0 + j])
                         : t.src[(size_t)(t.c0 + j) * t.lds + t.r0 + i];
    if (t.scale_dim == 1) v = cscale(v, t.s[j]);
    else if (t.scale_dim == 2) v = cscale(v, t.s[i]);
    t.blk[(size_t)i * t.ld + j] = v;
  }
}

void launch_scatter(const ScatterTask* d_tasks, int ntasks, cudaStream_t st) {
  if (ntasks <= 0) return;
  k_scatter<<<ntasks, 256, 0, st>>>(d_tasks);
}

// dst = src^H for square column-major n x n matrices (one CTA per task)
__global__ void k_adjoint(const FactTask* __restrict__ src, const FactTask* __restrict__ dst) {
  const FactTask a = src[blockIdx.x], b = dst[blockIdx.x];
  const int n = b.n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    b.A[(size_t)j * n + i] = cconj(a.V[(size_t)i * n + j]);
  }
}

void launch_adjoint(const FactTask* d_src, const FactTask* d_dst, int n, cudaStream_t st) {
  if (n <= 0) return;
  k_adjoint<<<n, 256, 0, st>>>(d_src, d_dst);
}

__global__ void k_zero(double2* p, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    p[i] = make_double2(0.0, 0.0);
}

void launch_zero(double2* p, size_t n, cudaStream_t st) {
  if (n == 0) return;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_zero<<<(unsigned)blocks, 256, 0, st>>>(p, n);
}

__global__ void k_scale(double2* x, size_t n, double2 a) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    x[i] = cmul(a, x[i]);
}

void launch_scale(double2* x, size_t n, double2 a, cudaStream_t st) {
  if (n == 0) return;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_scale<<<(unsigned)blocks, 256, 0, st>>>(x, n, a);
}

__global__ void k_axpby(double2* y, const double2* x, size_t n, double2 a, double2 b) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    y[i] = cadd(cmul(a, y[i]), cmul(b, x[i]));
}

void launch_axpby(double2* y, const double2* x, size_t n, double2 a, double2 b, cudaStream_t st) {
  if (n == 0) return;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_axpby<<<(unsigned)blocks, 256, 0, st>>>(y, x, n, a, b);
}

// ------------------------------------------------------------------ Jacobi SVD

// One-sided (Hestenes) Jacobi on the columns of a column-major m x n matrix
// (n <= m): pairs of columns are rotated until mutually orthogonal to m*eps
// relative; round-robin pairing lets every warp rotate a disjoint pair.
// Columns below 1e-13 of the Frobenius norm are numerically zero and are not
// rotated (their singular values fall under the truncation floor).
// Afterwards sigma_j = |a_j|, u_j = a_j / sigma_j, columns sorted descending.
// The matrix and V live in shared memory when both fit (smem_budget bytes).
constexpr int SVD_THREADS = 1024;
constexpr int SVD_MAX_SWEEPS = 60;

// Rotation of the column pair with squared norms al, be and inner product
// gr + i gi (conj(a_p) a_q): c and s e^{i phi}, or false when the pair is
// already orthogonal to tol or a column is numerically zero.  Taken by one
// thread per pair: these square roots and divisions run on the FP64 pipe,
// which is the scarce unit on this part, and a warp that computed them on
// every lane would spend 32 times the pipe time.
__device__ __forceinline__ bool jacobi_rotation(double al, double be, double gr, double gi,
                                                double negl, double tol, double* c,
                                                double2* sph) {
  const double g = sqrt(gr * gr + gi * gi);
  if (g == 0.0 || al <= negl || be <= negl || g <= tol * sqrt(al * be)) return false;
  const double zeta = (be - al) / (2.0 * g);
  const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double cc = 1.0 / sqrt(1.0 + tt * tt), sn = cc * tt;
  *c = cc;
  *sph = cscale(make_double2(gr / g, gi / g), sn);   // s e^{i phi}
  return true;
}

__global__ void __launch_bounds__(SVD_THREADS) k_svd(const FactTask* __restrict__ tasks,
                                                     int* status, int smem_budget) {
  extern __shared__ double2 svd_sh[];
  const FactTask t = tasks[blockIdx.x];
  const int m = t.m, n = t.n;
  const bool a_sh = (size_t)m * n * sizeof(double2) <= (size_t)smem_budget && n <= 1024;
  const bool v_sh = a_sh && (size_t)(m * n + n * n) * sizeof(double2) <= (size_t)smem_budget;
  double2* A = a_sh ? svd_sh : t.A;
  double2* V = v_sh ? svd_sh + (size_t)m * n : t.V;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  __shared__ int rotated;
  __shared__ double fro2;
  __shared__ int perm[1024];
  __shared__ double2 pr[1024];   // per pair: sums, then rotation parameters
  if (threadIdx.x == 0) fro2 = 0.0;
  if (a_sh)
    for (size_t e = threadIdx.x; e < (size_t)m * n; e += blockDim.x) A[e] = t.A[e];
  for (int e = threadIdx.x; e < n * n; e += blockDim.x)
    V[e] = make_double2((e % n) == (e / n) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  {
    // Frobenius norm: warp partial sums added in warp order (the same
    // rounding on every run, so the negligibility threshold is reproducible)
    __shared__ double part[32];
    double s2 = 0.0;
    for (size_t e = threadIdx.x; e < (size_t)m * n; e += blockDim.x) s2 += cabs2(A[e]);
    s2 = warp_sum(s2);
    if (lane == 0) part[warp] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double f = 0.0;
      for (int w = 0; w < nwarp; ++w) f += part[w];
      fro2 = f;
    }
  }
  __syncthreads();
  const double negl = 1e-26 * fro2;
  // the computed inner product carries ~m eps relative rounding error
  const double tol = 2.2e-16 * fmax(16.0, (double)m);
  const int np = (n + 1) & ~1;   // even number of players
  int sweep = 0;
  for (; sweep < SVD_MAX_SWEEPS; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < np - 1; ++r) {
      // the pair sums and the rotation parameters (one thread per pair),
      // then the rotations (one thread per (pair, row)): no warp
      // reductions and no FP64 work repeated across lanes; pr holds each
      // pair's c and s e^{i phi}
      for (int k = threadIdx.x; k < np / 2; k += blockDim.x) {
        int pa = k, pb = np - 1 - k;
        int p = pa == 0 ? 0 : ((pa - 1 + r) % (np - 1)) + 1;
        int q = ((pb - 1 + r) % (np - 1)) + 1;
        double al = 0.0, be = 0.0, gr = 0.0, gi = 0.0;
        if (p < n && q < n) {
          if (p > q) { int tmp = p; p = q; q = tmp; }
          const double2* ap = A + (size_t)p * m;
          const double2* aq = A + (size_t)q * m;
          for (int i = 0; i < m; ++i) {
            double2 x = ap[i], y = aq[i];
            al += cabs2(x);
            be += cabs2(y);
            gr += x.x * y.x + x.y * y.y;     // conj(x) * y
            gi += x.x * y.y - x.y * y.x;
          }
        }
        double c = 1.0;
        double2 sph = make_double2(0.0, 0.0);
        const bool go = p < n && q < n && jacobi_rotation(al, be, gr, gi, negl, tol, &c, &sph);
        pr[2 * k] = make_double2(c, go ? 1.0 : 0.0);
        pr[2 * k + 1] = sph;
        if (go) rotated = 1;
      }
      __syncthreads();
      const int per = m + n;
      for (int idx = threadIdx.x; idx < (np / 2) * per; idx += blockDim.x) {
        const int k = idx / per, i = idx - k * per;
        if (pr[2 * k].y == 0.0) continue;
        int pa = k, pb = np - 1 - k;
        int p = pa == 0 ? 0 : ((pa - 1 + r) % (np - 1)) + 1;
        int q = ((pb - 1 + r) % (np - 1)) + 1;
        if (p > q) { int tmp = p; p = q; q = tmp; }
        const double c = pr[2 * k].x;
        const double2 sph = pr[2 * k + 1];                   // s e^{i phi}
        const double2 sphc = cconj(sph);                     // s e^{-i phi}
        double2* xp = i < m ? A + (size_t)p * m + i : V + (size_t)p * n + (i - m);
        double2* yp = i < m ? A + (size_t)q * m + i : V + (size_t)q * n + (i - m);
        const double2 x = *xp, y = *yp;
        *xp = csub(cscale(x, c), cmul(sphc, y));
        *yp = cadd(cmul(sph, x), cscale(y, c));
      }
      __syncthreads();
    }
    int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  if (threadIdx.x == 0 && sweep == SVD_MAX_SWEEPS) atomicExch(status, 1);
  // singular values
  for (int j = warp; j < n; j += nwarp) {
    const double2* aj = A + (size_t)j * m;
    double s2 = 0.0;
    for (int i = lane; i < m; i += 32) s2 += cabs2(aj[i]);
    s2 = warp_sum(s2);
    if (lane == 0) t.s[j] = sqrt(s2);
  }
  __syncthreads();
  if (a_sh) {
    // descending order (ties: lower index first) written straight out
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double sj = t.s[j];
      int rank = 0;
      for (int k = 0; k < n; ++k) {
        double sk = t.s[k];
        rank += (sk > sj) || (sk == sj && k < j);
      }
      perm[rank] = j;
      pr[j].x = sj > 0.0 ? 1.0 / sj : 0.0;   // 1/sigma once per column (pairs are done)
    }
    __syncthreads();
    for (size_t e = threadIdx.x; e < (size_t)m * n; e += blockDim.x) {
      int j = (int)(e / m), i = (int)(e % m);
      t.A[e] = cscale(A[(size_t)perm[j] * m + i], pr[perm[j]].x);
    }
    __syncthreads();
    if (!v_sh) {   // A's shared buffer is free: stage V there (n*n <= m*n)
      for (size_t e = threadIdx.x; e < (size_t)n * n; e += blockDim.x) svd_sh[e] = t.V[e];
      __syncthreads();
      V = svd_sh;
    }
    for (size_t e = threadIdx.x; e < (size_t)n * n; e += blockDim.x) {
      int j = (int)(e / n), i = (int)(e % n);
      t.V[e] = V[(size_t)perm[j] * n + i];
    }
    // permute the singular values: one thread per value (n <= 1024 = blockDim)
    double mine = threadIdx.x < n ? t.s[perm[threadIdx.x]] : 0.0;
    __syncthreads();
    if (threadIdx.x < n) t.s[threadIdx.x] = mine;
    return;
  }
  for (int j = warp; j < n; j += nwarp) {
    double2* aj = A + (size_t)j * m;
    double sv = t.s[j];
    double inv = sv > 0.0 ? 1.0 / sv : 0.0;
    for (int i = lane; i < m; i += 32) aj[i] = cscale(aj[i], inv);
  }
  __syncthreads();
  // selection sort in global memory, descending (ties: lower index first)
  __shared__ int sel;
  for (int j = 0; j < n - 1; ++j) {
    if (threadIdx.x == 0) {
      int b = j;
      for (int k = j + 1; k < n; ++k)
        if (t.s[k] > t.s[b]) b = k;
      sel = b;
    }
    __syncthreads();
    int b = sel;
    if (b != j) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double2 x = A[(size_t)j * m + i];
        A[(size_t)j * m + i] = A[(size_t)b * m + i];
        A[(size_t)b * m + i] = x;
      }
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double2 x = V[(size_t)j * n + i];
        V[(size_t)j * n + i] = V[(size_t)b * n + i];
        V[(size_t)b * n + i] = x;
      }
      if (threadIdx.x == 0) {
        double x = t.s[j];
        t.s[j] = t.s[b];
        t.s[b] = x;
      }
    }
    __syncthreads();
  }
}

// The same one-sided Jacobi SVD with one matrix spread over a cluster of
// SVDC_CS CTAs: CTA `rank` holds rows [rank*mc, rank*mc + mc) of A in shared
// memory and rows [rank*nc, rank*nc + nc) of V in global memory.  Each round
// of the round-robin ordering computes the partial inner products (|a_p|^2,
// |a_q|^2, a_p^H a_q) of all its n/2 disjoint column pairs over the local
// rows, sums them across the cluster in one reduction (slots in every CTA's
// shared memory, rank-ordered sums, so every CTA takes the same rotation
// decisions), and rotates its own rows.  One cluster barrier per round
// instead of one SM doing all of the FP64 work.
constexpr int SVDC_CS = 8;
constexpr int SVDC_THREADS = 512;

__host__ __device__ inline size_t svdc_elems(int m, int n) {
  const size_t mc = (m + SVDC_CS - 1) / SVDC_CS;
  const size_t np = (size_t)((n + 1) & ~1);
  const size_t SL = np > (size_t)n ? np : (size_t)n;
  return mc * n + SL + 2 * (size_t)SVDC_CS * SL + (size_t)n + 16;
}

__global__ void __launch_bounds__(SVDC_THREADS) k_svd_cl(const FactTask* __restrict__ tasks,
                                                         int* status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double2 shv[];
  const int rank = (int)cl.block_rank();
  const FactTask t = tasks[blockIdx.x / SVDC_CS];
  const int m = t.m, n = t.n;
  const int mc = (m + SVDC_CS - 1) / SVDC_CS, nc = (n + SVDC_CS - 1) / SVDC_CS;
  const int row0 = rank * mc, ml = max(0, min(mc, m - row0));
  const int vr0 = rank * nc, nl = max(0, min(nc, n - vr0));
  const int np = (n + 1) & ~1;
  const int SL = np > n ? np : n;
  double2* A = shv;                          // [n][mc]
  double2* part = A + (size_t)mc * n;        // [SL]: pair k -> (al, be), (gr, gi) at 2k, 2k+1
  double2* slots = part + SL;                // [2][CS][SL]
  double* sv = (double*)(slots + 2 * (size_t)SVDC_CS * SL);   // [n]
  int* perm = (int*)(sv + n);                // [n]
  __shared__ int rotated;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  int red = 0;
  auto allreduce = [&](double2* buf, int len) {
    const int b = red & 1;
    ++red;
    for (int r = 0; r < SVDC_CS; ++r) {
      double2* dst = cl.map_shared_rank(slots, r) + ((size_t)b * SVDC_CS + rank) * SL;
      for (int i = threadIdx.x; i < len; i += blockDim.x) dst[i] = buf[i];
    }
    cl.sync();
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      double2 acc = make_double2(0.0, 0.0);
      for (int r = 0; r < SVDC_CS; ++r) acc = cadd(acc, slots[((size_t)b * SVDC_CS + r) * SL + i]);
      buf[i] = acc;
    }
    __syncthreads();
  };
  for (int c = 0; c < n; ++c)
    for (int i = threadIdx.x; i < ml; i += blockDim.x) A[(size_t)c * mc + i] = t.A[(size_t)c * m + row0 + i];
  for (int c = 0; c < n; ++c)
    for (int i = threadIdx.x; i < nl; i += blockDim.x)
      t.V[(size_t)c * n + vr0 + i] = make_double2(vr0 + i == c ? 1.0 : 0.0, 0.0);
  // the rows were staged by every thread; warp 0 reads all of them
  __syncthreads();
  // Frobenius norm
  {
    if (warp == 0) {
      double s2 = 0.0;
      for (size_t e = lane; e < (size_t)ml * n; e += 32) {
        const size_t c = e / ml, i = e % ml;
        s2 += cabs2(A[c * mc + i]);
      }
      s2 = warp_sum(s2);
      if (lane == 0) part[0] = make_double2(s2, 0.0);
    }
    __syncthreads();
    allreduce(part, 1);
  }
  const double negl = 1e-26 * part[0].x;
  const double tol = 2.2e-16 * fmax(16.0, (double)m);
  __syncthreads();
  int sweep = 0;
  for (; sweep < SVD_MAX_SWEEPS; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < np - 1; ++r) {
      // the partial sums of every pair over the local rows, one thread per
      // pair (the local rows are few: no warp reduction, whose shuffles and
      // adds would cost the FP64 pipe on every lane)
      for (int k = threadIdx.x; k < np / 2; k += blockDim.x) {
        int pa = k, pb = np - 1 - k;
        int p = pa == 0 ? 0 : ((pa - 1 + r) % (np - 1)) + 1;
        int q = ((pb - 1 + r) % (np - 1)) + 1;
        double al = 0.0, be = 0.0, gr = 0.0, gi = 0.0;
        if (p < n && q < n) {
          if (p > q) { int tmp = p; p = q; q = tmp; }
          const double2* ap = A + (size_t)p * mc;
          const double2* aq = A + (size_t)q * mc;
          for (int i = 0; i < ml; ++i) {
            const double2 x = ap[i], y = aq[i];
            al += cabs2(x);
            be += cabs2(y);
            gr += x.x * y.x + x.y * y.y;     // conj(x) * y
            gi += x.x * y.y - x.y * y.x;
          }
        }
        part[2 * k] = make_double2(al, be);
        part[2 * k + 1] = make_double2(gr, gi);
      }
      __syncthreads();
      allreduce(part, np);
      // rotation parameters, one thread per pair, in place of the sums
      for (int k = threadIdx.x; k < np / 2; k += blockDim.x) {
        int pa = k, pb = np - 1 - k;
        int p = pa == 0 ? 0 : ((pa - 1 + r) % (np - 1)) + 1;
        int q = ((pb - 1 + r) % (np - 1)) + 1;
        double c = 1.0;
        double2 sph = make_double2(0.0, 0.0);
        const bool go = p < n && q < n &&
                        jacobi_rotation(part[2 * k].x, part[2 * k].y, part[2 * k + 1].x,
                                        part[2 * k + 1].y, negl, tol, &c, &sph);
        part[2 * k] = make_double2(c, go ? 1.0 : 0.0);
        part[2 * k + 1] = sph;
        if (go) rotated = 1;
      }
      __syncthreads();
      // the rotations, one thread per (pair, local row of A or V)
      const int per = ml + nl;
      for (int idx = threadIdx.x; idx < (np / 2) * per; idx += blockDim.x) {
        const int k = idx / per, i = idx - k * per;
        if (part[2 * k].y == 0.0) continue;
        int pa = k, pb = np - 1 - k;
        int p = pa == 0 ? 0 : ((pa - 1 + r) % (np - 1)) + 1;
        int q = ((pb - 1 + r) % (np - 1)) + 1;
        if (p > q) { int tmp = p; p = q; q = tmp; }
        const double c = part[2 * k].x;
        const double2 sph = part[2 * k + 1];                // s e^{i phi}
        const double2 sphc = cconj(sph);                    // s e^{-i phi}
        double2* xp;
        double2* yp;
        if (i < ml) {
          xp = A + (size_t)p * mc + i;
          yp = A + (size_t)q * mc + i;
        } else {
          xp = t.V + (size_t)p * n + vr0 + (i - ml);
          yp = t.V + (size_t)q * n + vr0 + (i - ml);
        }
        const double2 x = *xp, y = *yp;
        *xp = csub(cscale(x, c), cmul(sphc, y));
        *yp = cadd(cmul(sph, x), cscale(y, c));
      }
      __syncthreads();
    }
    const int any = rotated;   // identical in every CTA of the cluster
    __syncthreads();
    if (!any) break;
  }
  if (rank == 0 && threadIdx.x == 0 && sweep == SVD_MAX_SWEEPS) atomicExch(status, 1);
  // singular values: column norms over all rows
  for (int j = warp; j < n; j += nwarp) {
    const double2* aj = A + (size_t)j * mc;
    double s2 = 0.0;
    for (int i = lane; i < ml; i += 32) s2 += cabs2(aj[i]);
    s2 = warp_sum(s2);
    if (lane == 0) part[j] = make_double2(s2, 0.0);
  }
  __syncthreads();
  allreduce(part, n);
  for (int j = threadIdx.x; j < n; j += blockDim.x) sv[j] = sqrt(part[j].x);
  __syncthreads();
  // descending order, ties: lower index first
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double sj = sv[j];
    int rk = 0;
    for (int k = 0; k < n; ++k) rk += (sv[k] > sj) || (sv[k] == sj && k < j);
    perm[rk] = j;
    part[j].x = sj > 0.0 ? 1.0 / sj : 0.0;   // 1/sigma once per column
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const int pj = perm[j];
    const double inv = part[pj].x;
    for (int i = threadIdx.x; i < ml; i += blockDim.x)
      t.A[(size_t)j * m + row0 + i] = cscale(A[(size_t)pj * mc + i], inv);
  }
  if (rank == 0)
    for (int j = threadIdx.x; j < n; j += blockDim.x) t.s[j] = sv[perm[j]];
  // V columns permuted; each CTA owns its rows of V, staged through the A
  // buffer (free now; the launcher requires m >= n, so nc <= mc)
  __syncthreads();
  for (int c = 0; c < n; ++c)
    for (int i = threadIdx.x; i < nl; i += blockDim.x) A[(size_t)c * nc + i] = t.V[(size_t)c * n + vr0 + i];
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const int pj = perm[j];
    for (int i = threadIdx.x; i < nl; i += blockDim.x)
      t.V[(size_t)j * n + vr0 + i] = A[(size_t)pj * nc + i];
  }
  // no CTA may leave while others can still write into its slots
  cl.sync();
}

void launch_svd(const FactTask* d_tasks, int ntasks, int* d_status, cudaStream_t st,
                size_t max_bytes, const FactTask* h_tasks) {
  if (ntasks <= 0) return;
  {
    // the cluster kernel for square (or tall) matrices with a large one
    const size_t cap_cl = 200 * 1024;
    size_t need = 0;
    bool large = false, shape_ok = h_tasks != nullptr;
    for (int i = 0; h_tasks && i < ntasks; ++i) {
      need = std::max(need, svdc_elems(h_tasks[i].m, h_tasks[i].n) * sizeof(double2));
      if (h_tasks[i].m < h_tasks[i].n || h_tasks[i].n > 2048) shape_ok = false;
      if (h_tasks[i].n >= 24) large = true;
    }
    if (shape_ok && large && need <= cap_cl) {
      set_smem_limit((const void*)k_svd_cl, (int)cap_cl);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(ntasks * SVDC_CS));
      cfg.blockDim = dim3(SVDC_THREADS);
      cfg.dynamicSmemBytes = need;
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = SVDC_CS;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      cudaLaunchKernelEx(&cfg, k_svd_cl, d_tasks, d_status);
      return;
    }
  }
  // static shared: perm (4 KB), the pair array (16 KB) and scalars
  const size_t cap = 227 * 1024 - 21 * 1024;
  size_t dyn = max_bytes < cap ? max_bytes : cap;
  set_smem_limit((const void*)k_svd, (int)cap);
  k_svd<<<ntasks, SVD_THREADS, dyn, st>>>(d_tasks, d_status, (int)dyn);
}

// ------------------------------------------------------------------ Gram-Schmidt QR

// Classical Gram-Schmidt with re-orthogonalisation on a column-major m x n
// matrix.  The second projection pass runs when the first one removed more
// than 1 - 1/sqrt(2) of the column's norm (the Daniel-Gragg-Kaufman-Stewart
// criterion: otherwise one classical pass is already orthogonal to working
// precision); it halves the FP64 work on well-conditioned blocks.  Columns
// whose residual norm falls to <= 1e-12 times the largest input column norm
// are dependent: they add no new direction (such a column always lost far
// more than the criterion's share, so it always gets both passes).  The
// independent directions are stored compactly in the first columns (at most
// k = min(m, n)), the remaining of the first k columns are zero.  R (k x n,
// column-major, leading dimension n) holds the coefficients, so that
// A = Q R.
constexpr int QR_THREADS = 256;
constexpr int QR_SMEM = 200 * 1024;   // matrix held in shared memory when it fits

__global__ void __launch_bounds__(QR_THREADS) k_qr(const FactTask* __restrict__ tasks) {
  extern __shared__ double2 sh[];
  const FactTask t = tasks[blockIdx.x];
  const int m = t.m, n = t.n, kmax = m < n ? m : n;
  // layout: [v: m][coef: n][A: m*n][R: n*n] when they fit
  double2* v = sh;
  double2* coef = sh + m;
  const bool a_sh =
      (size_t)(m + n + (size_t)m * n + (size_t)n * n) * sizeof(double2) <= (size_t)QR_SMEM;
  double2* A = a_sh ? sh + m + n : t.A;
  double2* R = a_sh ? sh + m + n + (size_t)m * n : t.V;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  __shared__ double maxn, vn, vinv;
  __shared__ int nq;
  if (threadIdx.x == 0) { maxn = 0.0; nq = 0; }
  if (a_sh)
    for (size_t e = threadIdx.x; e < (size_t)m * n; e += blockDim.x) A[e] = t.A[e];
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) R[e] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int j = warp; j < n; j += nwarp) {
    double s2 = 0.0;
    for (int i = lane; i < m; i += 32) s2 += cabs2(A[(size_t)j * m + i]);
    s2 = warp_sum(s2);
    if (lane == 0) {
      // non-negative doubles order like their bit patterns
      atomicMax((unsigned long long*)&maxn, (unsigned long long)__double_as_longlong(sqrt(s2)));
    }
  }
  __syncthreads();
  const double tol = 1e-12 * maxn;
  for (int j = 0; j < n; ++j) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) v[i] = A[(size_t)j * m + i];
    __syncthreads();
    const int q = nq;
    double norm_before = 0.0;
    if (q > 0 && warp == 0) {
      double s2 = 0.0;
      for (int i = lane; i < m; i += 32) s2 += cabs2(v[i]);
      s2 = warp_sum(s2);
      if (lane == 0) vn = s2;
    }
    if (q > 0) {
      __syncthreads();
      norm_before = vn;
    }
    for (int pass = 0; pass < 2 && q > 0; ++pass) {
      for (int cc = warp; cc < q; cc += nwarp) {
        const double2* qc = A + (size_t)cc * m;
        double re = 0.0, im = 0.0;
        for (int i = lane; i < m; i += 32) {
          double2 a = qc[i], b = v[i];
          re += a.x * b.x + a.y * b.y;   // conj(q) * v
          im += a.x * b.y - a.y * b.x;
        }
        re = warp_sum(re); im = warp_sum(im);
        if (lane == 0) coef[cc] = make_double2(re, im);
      }
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double2 acc = v[i];
        for (int cc = 0; cc < q; ++cc) acc = csub(acc, cmul(coef[cc], A[(size_t)cc * m + i]));
        v[i] = acc;
      }
      for (int cc = threadIdx.x; cc < q; cc += blockDim.x) {
        double2* rr = R + (size_t)j * n + cc;   // R[c, j], leading dimension n
        *rr = cadd(*rr, coef[cc]);
      }
      __syncthreads();
      if (pass == 0) {
        if (warp == 0) {
          double s2 = 0.0;
          for (int i = lane; i < m; i += 32) s2 += cabs2(v[i]);
          s2 = warp_sum(s2);
          if (lane == 0) vn = s2;
        }
        __syncthreads();
        const bool again = vn < 0.5 * norm_before;   // |v'|^2 < |v|^2 / 2
        __syncthreads();
        if (!again) break;
      }
    }
    if (warp == 0) {
      double s2 = 0.0;
      for (int i = lane; i < m; i += 32) s2 += cabs2(v[i]);
      s2 = warp_sum(s2);
      if (lane == 0) {
        vn = sqrt(s2);
        vinv = vn > 0.0 ? 1.0 / vn : 0.0;   // once, not on every thread (FP64 pipe)
      }
    }
    __syncthreads();
    const double nrm = vn;
    if (nrm > tol && q < kmax) {
      const double inv = vinv;
      for (int i = threadIdx.x; i < m; i += blockDim.x) A[(size_t)q * m + i] = cscale(v[i], inv);
      if (threadIdx.x == 0) {
        R[(size_t)j * n + q] = make_double2(nrm, 0.0);
        nq = q + 1;
      }
    }
    __syncthreads();
  }
  const int nfin = nq;
  for (int cc = nfin; cc < kmax; ++cc)
    for (int i = threadIdx.x; i < m; i += blockDim.x) A[(size_t)cc * m + i] = make_double2(0.0, 0.0);
  if (a_sh) {
    __syncthreads();
    for (size_t e = threadIdx.x; e < (size_t)m * kmax; e += blockDim.x) t.A[e] = A[e];
    for (size_t e = threadIdx.x; e < (size_t)n * n; e += blockDim.x) t.V[e] = R[e];
  }
}

// The same Gram-Schmidt QR (dependency rule, conditional second pass)
// with one sector spread over a cluster of QRC_CS CTAs: CTA `rank` holds
// rows [rank*mc, rank*mc + mc) of the matrix in its shared memory, and every
// inner product (projection coefficients, norms) is a partial sum per CTA
// combined across the cluster through distributed shared memory.  Each CTA
// writes its partial vector into a slot of every CTA, the cluster barrier
// publishes them, and every CTA adds the slots in rank order -- so all CTAs
// hold bit-identical sums and take identical branch decisions.  Slots are
// double buffered: the barrier of reduction r also tells a CTA that every
// CTA has read the buffer of reduction r - 1, which reduction r + 1 reuses.
// A sector's FP64 work is divided by the cluster size, which is what limits
// the single-CTA kernel on large sectors (one SM's FP64 pipe).
constexpr int QRC_CS = 8;
constexpr int QRC_THREADS = 256;

__host__ __device__ inline int qrc_mc(int m) { return (m + QRC_CS - 1) / QRC_CS; }
// complex elements of dynamic shared memory per CTA
__host__ __device__ inline size_t qrc_elems(int m, int n) {
  const size_t mc = qrc_mc(m);
  return mc * n + mc + n + 2 * (size_t)QRC_CS * (n + 1) + 8;
}

__global__ void __launch_bounds__(QRC_THREADS) k_qr_cl(const FactTask* __restrict__ tasks) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double2 shc[];
  const int rank = (int)cl.block_rank();
  const FactTask t = tasks[blockIdx.x / QRC_CS];
  const int m = t.m, n = t.n, kmax = m < n ? m : n;
  const int mc = qrc_mc(m);
  const int row0 = rank * mc;
  const int ml = max(0, min(mc, m - row0));   // rows held here
  const int SL = n + 1;                       // slot length
  double2* A = shc;                           // [n][mc]
  double2* v = A + (size_t)mc * n;            // [mc]
  double2* coef = v + mc;                     // [n]
  double2* slots = coef + n;                  // [2][CS][SL]
  double2* scal = slots + 2 * (size_t)QRC_CS * SL;   // small scratch
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  int red = 0;
  // all-reduce of len values (mine may alias out)
  auto allreduce = [&](const double2* mine, int len, double2* out) {
    const int buf = red & 1;
    ++red;
    for (int r = 0; r < QRC_CS; ++r) {
      double2* dst = cl.map_shared_rank(slots, r) + ((size_t)buf * QRC_CS + rank) * SL;
      for (int i = threadIdx.x; i < len; i += blockDim.x) dst[i] = mine[i];
    }
    cl.sync();
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      double2 acc = make_double2(0.0, 0.0);
      for (int r = 0; r < QRC_CS; ++r) acc = cadd(acc, slots[((size_t)buf * QRC_CS + r) * SL + i]);
      out[i] = acc;
    }
    __syncthreads();
  };
  // squared norm of v over all rows
  auto vnorm2 = [&]() {
    if (warp == 0) {
      double s2 = 0.0;
      for (int i = lane; i < ml; i += 32) s2 += cabs2(v[i]);
      s2 = warp_sum(s2);
      if (lane == 0) scal[0] = make_double2(s2, 0.0);
    }
    __syncthreads();
    allreduce(scal, 1, scal + 1);
    return scal[1].x;
  };

  for (int c = 0; c < n; ++c)
    for (int i = threadIdx.x; i < ml; i += blockDim.x) A[(size_t)c * mc + i] = t.A[(size_t)c * m + row0 + i];
  if (rank == 0)
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) t.V[e] = make_double2(0.0, 0.0);
  // the rows were staged by every thread; each warp reads whole columns
  __syncthreads();
  // largest column norm
  for (int c = warp; c < n; c += nwarp) {
    double s2 = 0.0;
    for (int i = lane; i < ml; i += 32) s2 += cabs2(A[(size_t)c * mc + i]);
    s2 = warp_sum(s2);
    if (lane == 0) coef[c] = make_double2(s2, 0.0);
  }
  __syncthreads();
  allreduce(coef, n, coef);
  // sqrt is monotonic: the largest norm is the root of the largest square,
  // taken once (FP64 square roots on every thread would load the narrow pipe)
  if (threadIdx.x == 0) {
    double m2 = 0.0;
    for (int c = 0; c < n; ++c) m2 = fmax(m2, coef[c].x);
    scal[4] = make_double2(sqrt(m2), 0.0);
  }
  __syncthreads();
  const double tol = 1e-12 * scal[4].x;
  int nq = 0;
  for (int j = 0; j < n; ++j) {
    for (int i = threadIdx.x; i < ml; i += blockDim.x) v[i] = A[(size_t)j * mc + i];
    __syncthreads();
    const int q = nq;
    double nrm2;
    if (q == 0) {
      nrm2 = vnorm2();
    } else {
      // The first pass reduces the coefficients and |v|^2 together, and when
      // it removed less than half of |v|^2 the residual norm follows from
      // Pythagoras, |v'|^2 = |v|^2 - sum |c|^2 (accurate to a few ulp in that
      // regime) -- one cluster reduction per column instead of three.
      double before = 0.0;
      nrm2 = 0.0;
      for (int pass = 0; pass < 2; ++pass) {
        if (pass == 0 && warp == nwarp - 1) {
          double s2 = 0.0;
          for (int i = lane; i < ml; i += 32) s2 += cabs2(v[i]);
          s2 = warp_sum(s2);
          if (lane == 0) coef[q] = make_double2(s2, 0.0);
        }
        for (int cc = warp; cc < q; cc += nwarp) {
          const double2* qc = A + (size_t)cc * mc;
          double re = 0.0, im = 0.0;
          for (int i = lane; i < ml; i += 32) {
            const double2 a = qc[i], b = v[i];
            re += a.x * b.x + a.y * b.y;   // conj(q) * v
            im += a.x * b.y - a.y * b.x;
          }
          re = warp_sum(re);
          im = warp_sum(im);
          if (lane == 0) coef[cc] = make_double2(re, im);
        }
        __syncthreads();
        allreduce(coef, pass == 0 ? q + 1 : q, coef);
        if (pass == 0 && threadIdx.x == 0) {   // one thread; read after the barrier below
          double proj = 0.0;
          for (int cc = 0; cc < q; ++cc) proj += cabs2(coef[cc]);
          scal[2] = make_double2(coef[q].x, proj);
        }
        for (int i = threadIdx.x; i < ml; i += blockDim.x) {
          double2 acc = v[i];
          for (int cc = 0; cc < q; ++cc) acc = csub(acc, cmul(coef[cc], A[(size_t)cc * mc + i]));
          v[i] = acc;
        }
        if (rank == 0)
          for (int cc = threadIdx.x; cc < q; cc += blockDim.x) {
            double2* rr = t.V + (size_t)j * n + cc;   // R[cc, j], leading dimension n
            *rr = cadd(*rr, coef[cc]);
          }
        __syncthreads();
        if (pass == 0) {
          before = scal[2].x;
          const double est = before - scal[2].y;
          if (!(est < 0.5 * before)) {   // one pass was enough
            nrm2 = est;
            break;
          }
        } else {
          nrm2 = vnorm2();
        }
      }
    }
    // the column norm and its inverse, once
    if (threadIdx.x == 0) {
      const double r0 = sqrt(nrm2);
      scal[3] = make_double2(r0, r0 > 0.0 ? 1.0 / r0 : 0.0);
    }
    __syncthreads();
    const double nrm = scal[3].x;
    if (nrm > tol && q < kmax) {
      const double inv = scal[3].y;
      for (int i = threadIdx.x; i < ml; i += blockDim.x) A[(size_t)q * mc + i] = cscale(v[i], inv);
      if (rank == 0 && threadIdx.x == 0) t.V[(size_t)j * n + q] = make_double2(nrm, 0.0);
      nq = q + 1;
    }
    __syncthreads();
  }
  for (int c = 0; c < kmax; ++c)
    for (int i = threadIdx.x; i < ml; i += blockDim.x)
      t.A[(size_t)c * m + row0 + i] = c < nq ? A[(size_t)c * mc + i] : make_double2(0.0, 0.0);
  // no CTA may leave while others can still write into its slots
  cl.sync();
}

void launch_qr(const FactTask* d_tasks, int ntasks, cudaStream_t st, const FactTask* h_tasks) {
  if (ntasks <= 0) return;
  // the cluster kernel pays off when some sector is large and all fit
  size_t need = 0;
  bool large = false;
  for (int i = 0; h_tasks && i < ntasks; ++i) {
    need = std::max(need, qrc_elems(h_tasks[i].m, h_tasks[i].n) * sizeof(double2));
    if (h_tasks[i].n >= 16 && (long long)h_tasks[i].m * h_tasks[i].n >= 2048) large = true;
  }
  if (large && need <= (size_t)QR_SMEM) {
    set_smem_limit((const void*)k_qr_cl, QR_SMEM);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ntasks * QRC_CS));
    cfg.blockDim = dim3(QRC_THREADS);
    cfg.dynamicSmemBytes = need;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = QRC_CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_qr_cl, d_tasks);
    return;
  }
  set_smem_limit((const void*)k_qr, QR_SMEM);
  k_qr<<<ntasks, QR_THREADS, QR_SMEM, st>>>(d_tasks);
}



// ------------------------------------------------------------------ truncation rule

// Singular values of all sectors of one bond (each sector descending, sector
// ids ascending): sort descending with ties by position; drop values <=
// 1e-12 * max; keep at most D and the fewest whose discarded weight is <= eps
// of the total; move a cut inside a cluster (gaps <= 1e-10 * max) down to the
// cluster edge (up if the cluster starts at the top).
__global__ void k_trunc(const double* __restrict__ s, const int* __restrict__ sec, int nv,
                        int nsec, int D, double eps, int* kept, double* w, double* sorted,
                        int* sorted_sec) {
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    double si = s[i];
    int rank = 0;
    for (int j = 0; j < nv; ++j) {
      double sj = s[j];
      rank += (sj > si) || (sj == si && j < i);
    }
    sorted[rank] = si;
    sorted_sec[rank] = sec[i];
  }
  for (int i = threadIdx.x; i < nsec; i += blockDim.x) kept[i] = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    double total = 0.0;
    for (int i = nv - 1; i >= 0; --i) total += sorted[i] * sorted[i];
    int k = 0;
    double disc = total;
    if (nv > 0 && sorted[0] > 0.0) {
      const double smax = sorted[0];
      int nz = 0;
      while (nz < nv && sorted[nz] > 1e-12 * smax) ++nz;
      // tail[j] = sum_{i >= j} sorted[i]^2
      k = nz;
      double tail = 0.0;
      for (int i = nv - 1; i >= nz; --i) tail += sorted[i] * sorted[i];
      // try dropping index k-1 while allowed
      while (k > 1) {
        double t2 = tail + sorted[k - 1] * sorted[k - 1];
        if (t2 <= eps * total) { tail = t2; --k; } else break;
      }
      if (k > D) k = D;
      if (k < nz) {
        int j = k;
        while (j > 0 && sorted[j - 1] - sorted[j] <= 1e-10 * smax) --j;
        if (j > 0) k = j;
        else
          while (k < nz && sorted[k - 1] - sorted[k] <= 1e-10 * smax) ++k;
      }
      disc = 0.0;
      for (int i = nv - 1; i >= k; --i) disc += sorted[i] * sorted[i];
      for (int i = 0; i < k; ++i) kept[sorted_sec[i]] += 1;
    }
    w[0] = disc;
    w[1] = total;
  }
}

void launch_trunc(const double* d_s, const int* d_sec, int nv, int nsec, int D, double eps,
                  int* d_kept, double* d_w, double* d_sorted, int* d_sorted_sec, cudaStream_t st) {
  k_trunc<<<1, 1024, 0, st>>>(d_s, d_sec, nv, nsec, D, eps, d_kept, d_w, d_sorted, d_sorted_sec);
}

// ------------------------------------------------------------------ Krylov algebra

constexpr int KMAX = 16;

// Cyclic Jacobi eigen-decomposition of a Hermitian n x n matrix (row-major,
// in place); eigenvectors in columns of V.
__device__ void herm_eig(double2* A, double2* V, double* w, int n) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += cabs2(A[i * n + j]);
        if (i != j) off += cabs2(A[i * n + j]);
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double2 apq = A[p * n + q];
        double g = sqrt(cabs2(apq));
        if (g == 0.0) continue;
        double a = A[p * n + p].x, b = A[q * n + q].x;
        double2 ph = make_double2(apq.x / g, apq.y / g);   // e^{i phi}
        double zeta = (b - a) / (2.0 * g);
        double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + tt * tt), s = c * tt;
        // J = [[c, s],[ -s e^{-i phi}, c e^{-i phi}]] on (p, q); A <- J^H A J, V <- V J
        double2 phc = cconj(ph);
        for (int k = 0; k < n; ++k) {   // columns: A J
          double2 x = A[k * n + p], y = A[k * n + q];
          A[k * n + p] = csub(cscale(x, c), cmul(cscale(phc, s), y));
          A[k * n + q] = cadd(cscale(x, s), cmul(cscale(phc, c), y));
          double2 vx = V[k * n + p], vy = V[k * n + q];
          V[k * n + p] = csub(cscale(vx, c), cmul(cscale(phc, s), vy));
          V[k * n + q] = cadd(cscale(vx, s), cmul(cscale(phc, c), vy));
        }
        for (int k = 0; k < n; ++k) {   // rows: J^H (A J)
          double2 x = A[p * n + k], y = A[q * n + k];
          A[p * n + k] = csub(cscale(x, c), cmul(cscale(ph, s), y));
          A[q * n + k] = cadd(cscale(x, s), cmul(cscale(ph, c), y));
        }
        A[p * n + q] = make_double2(0.0, 0.0);
        A[q * n + p] = make_double2(0.0, 0.0);
      }
  }
  for (int i = 0; i < n; ++i) w[i] = A[i * n + i].x;
}

__global__ void k_krylov_small(const double2* Nm, const double2* Hm, int m, double dt,
                               double2* c, int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double2 A[KMAX * KMAX], V[KMAX * KMAX], X[KMAX * KMAX], M[KMAX * KMAX], U[KMAX * KMAX];
  double w[KMAX], lam[KMAX];
  int bad = 0;
  for (int i = 0; i < m * m; ++i) {
    if (!isfinite(Nm[i].x) || !isfinite(Nm[i].y) || !isfinite(Hm[i].x) || !isfinite(Hm[i].y)) bad = 1;
  }
  // N and H arrive with their upper triangles (i <= j) filled; complete them
  // as Hermitian matrices
  double2 Nf[KMAX * KMAX], Hf[KMAX * KMAX];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      double2 n = i <= j ? Nm[i * m + j] : cconj(Nm[j * m + i]);
      double2 h = i <= j ? Hm[i * m + j] : cconj(Hm[j * m + i]);
      if (i == j) { n.y = 0.0; h.y = 0.0; }
      Nf[i * m + j] = n;
      Hf[i * m + j] = h;
      A[i * m + j] = n;
    }
  herm_eig(A, V, w, m);
  double wmax = 0.0;
  for (int i = 0; i < m; ++i) wmax = fmax(wmax, w[i]);
  int r = 0;
  for (int k = 0; k < m; ++k)
    if (w[k] > 1e-12 * wmax) {
      double inv = 1.0 / sqrt(w[k]);
      for (int i = 0; i < m; ++i) X[i * KMAX + r] = cscale(V[i * m + k], inv);
      ++r;
    }
  // M = X^H H X  (r x r)
  for (int a = 0; a < r; ++a)
    for (int b = 0; b < r; ++b) {
      double2 acc = make_double2(0.0, 0.0);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
          acc = cadd(acc, cmul(cmul(cconj(X[i * KMAX + a]), Hf[i * m + j]), X[j * KMAX + b]));
        }
      M[a * r + b] = acc;
    }
  if (r > 0) herm_eig(M, U, lam, r);
  // b = X^H N e0
  double2 bvec[KMAX], tmp[KMAX];
  for (int a = 0; a < r; ++a) {
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < m; ++i) acc = cadd(acc, cmul(cconj(X[i * KMAX + a]), Nf[i * m + 0]));
    bvec[a] = acc;
  }
  for (int a = 0; a < r; ++a) {   // tmp = exp(-i dt lam) U^H b
    double2 acc = make_double2(0.0, 0.0);
    for (int b2 = 0; b2 < r; ++b2) acc = cadd(acc, cmul(cconj(U[b2 * r + a]), bvec[b2]));
    double ph = -dt * lam[a];
    tmp[a] = cmul(make_double2(cos(ph), sin(ph)), acc);
  }
  for (int i = 0; i < m; ++i) {
    double2 acc = make_double2(0.0, 0.0);
    for (int a = 0; a < r; ++a) {
      double2 ua = make_double2(0.0, 0.0);
      for (int b2 = 0; b2 < r; ++b2) ua = cadd(ua, cmul(U[a * r + b2], tmp[b2]));
      acc = cadd(acc, cmul(X[i * KMAX + a], ua));
    }
    c[i] = acc;
    if (!isfinite(acc.x) || !isfinite(acc.y)) bad = 1;
  }
  status[0] = m - r;
  status[1] = bad;
}

void launch_krylov_small(const double2* d_N, const double2* d_H, int m, double dt, double2* d_c,
                         int* d_status, cudaStream_t st) {
  k_krylov_small<<<1, 32, 0, st>>>(d_N, d_H, m, dt, d_c, d_status);
}

// ------------------------------------------------------------------ scalar helpers

__global__ void k_scalar_div_neg(const double2* num, const double2* den, double2* out) {
  double2 q = cdiv(*num, *den);
  *out = make_double2(-q.x, -q.y);
}

void launch_scalar_div_neg(const double2* num, const double2* den, double2* out, cudaStream_t st) {
  k_scalar_div_neg<<<1, 1, 0, st>>>(num, den, out);
}

__global__ void k_normalize(double2* x, size_t n, double2* norm_out) {
  __shared__ double part[32];
  double s2 = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) s2 += cabs2(x[i]);
  s2 = warp_sum(s2);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s2;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) part[0] = v;
  }
  __syncthreads();
  double nrm = sqrt(part[0]);
  double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) x[i] = cscale(x[i], inv);
  if (threadIdx.x == 0 && norm_out) *norm_out = make_double2(nrm, 0.0);
}

void launch_normalize(double2* x, size_t n, double2* d_norm_out, cudaStream_t st) {
  k_normalize<<<1, 1024, 0, st>>>(x, n, d_norm_out);
}

// out[w] += sum_{a, b} E[a][w][b] * R[a][b]   (rows x nch x cols and rows x cols)
template <class T>
__global__ void k_trace_channels(const T* E, int rows, int nch, int cols, const T* R,
                                 double2* out) {
  const int w = blockIdx.x;
  double re = 0.0, im = 0.0;
  for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
    int a = e / cols, b = e % cols;
    double2 v = cmul(ld2(E, ((size_t)a * nch + w) * cols + b), ld2(R, (size_t)a * cols + b));
    re += v.x;
    im += v.y;
  }
  __shared__ double pr[32], pi[32];
  re = warp_sum(re);
  im = warp_sum(im);
  if ((threadIdx.x & 31) == 0) { pr[threadIdx.x >> 5] = re; pi[threadIdx.x >> 5] = im; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sr = 0.0, si = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { sr += pr[k]; si += pi[k]; }
    out[w] = cadd(out[w], make_double2(sr, si));
  }
}

void launch_trace_channels(const void* E, int rows, int nch, int cols, const void* R, int et,
                           double2* out, cudaStream_t st) {
  if (nch <= 0 || rows * cols == 0) return;
  if (et == 0)
    k_trace_channels<double2><<<nch, 256, 0, st>>>((const double2*)E, rows, nch, cols, (const double2*)R, out);
  else
    k_trace_channels<float2><<<nch, 256, 0, st>>>((const float2*)E, rows, nch, cols, (const float2*)R, out);
}

}  // namespace tdmps
