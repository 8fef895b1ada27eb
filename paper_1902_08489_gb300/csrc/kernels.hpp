// Device kernel interfaces of the tdmps library.  All matrices are complex
// double (double2) unless stated; blocks are row-major unless stated.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace tdmps {

// op codes for grouped GEMM operands
enum : int { OP_N = 0, OP_T = 1, OP_C = 2, OP_J = 3 };   // none, transpose, conj-transpose, conj

// One product op(A) op(B) of a task; op(A) elements are multiplied by
// scale * (*scale_ptr if non-null) while staged (per-term coefficients).
struct GemmTerm {
  const void* A;
  const void* B;
  int K, lda, ldb, pad;
  double2 scale;
  const double2* scale_ptr;
  float2 fscale;   // scale rounded to FP32 on the host (tensor-core path, scale_ptr null)
};

// C (M x N, ldc) = alpha * sum_terms op(A) op(B) + beta * C;
// alpha = alpha_imm * (*alpha_ptr if non-null) * (alpha_inv ? 1 / *alpha_inv : 1).
struct GemmTask {
  void* C;
  const double2* alpha_ptr;
  const double2* alpha_div;
  double2 alpha;
  int M, N, ldc;
  int opA, opB, beta;
  int term_begin, term_end;
  int tiles_m, tile_base;
  int ta, tb, tc;        // element types of A, B, C: 0 double2, 1 float2 (tensor-core path)
  int splits;            // CTAs sharing the K range
  int ct;                // 1: the task computes C^T (M x N); element (r, c) goes to C[c][r]
  // splits > 1: split s stores alpha * (its partial sum) at part[(s M + r) N + c]
  // (task orientation; complex float from the tensor-core kernel, complex
  // double from the FP64 kernel) and launch_reduce_splits adds the slices in
  // split order into C, so results do not depend on timing
  void* part;
  // tensor-core path: 1 + index of this task's GemmSeg (0: not segmented)
  int seg1;
};

// A segmented task: the rows (dim 0) or the columns (dim 1) of C are the
// concatenation of n <= 4 output blocks, segment s covering [off[s], off[s+1])
// with its own output pointer C[s] and leading dimension ldc[s]; in every
// term the operand along that dimension (A for rows, B for columns) is one
// block per segment, listed in the term's SegOps (GemmTerm::pad = its index;
// a null block is zero), while the other operand is shared.  Used for the
// local states that share one operand of a contraction (e.g. the four
// output blocks (a, s) -> b of one right sector b), so that the shared
// operand is streamed once for all of them.
struct GemmSeg {
  int dim, n;
  int off[5];
  void* C[4];
  int ldc[4];
};
struct SegOps {
  const void* p[4];
  int ld[4];
};

// Sparse MPO-tensor application.  Output block Y[r][w][c] (rows r, W_out
// channels, c columns), Y[a][w][b] = sum over inputs s of
//   sum_{(w_in, v) in CSR_s[w]} v * X_s[a][w_in][b]   (X_s has W_in_s channels)
struct WTask {
  void* Y;
  const void* X[4];
  int win[4];
  int csr[4];          // row-pointer offset of the CSR for input s (-1: none)
  int rows, wout, cols, beta;
  int64_t work_base;   // first flat element index of this task
};

// Copy a (rows x cols, ld) row-major block into / out of a column-major work
// matrix (ldw) at (row0, col0); conj_t: the work matrix holds the conjugate
// transpose of the block.  scale multiplies on the way.
struct CopyTask {
  double2* blk;
  double2* work;
  int rows, cols, ld, ldw;
  int row0, col0, conj_t, zero_fill;
  double2 scale;
};

// One-sided Jacobi SVD / Gram-Schmidt QR on column-major matrices in global memory.
// blk(i, j) = src(r0 + i, c0 + j)            (conj_t = 0, src column-major, lds)
// blk(i, j) = conj(src(r0 + j, c0 + i))      (conj_t = 1)
// times s[j] (scale_dim = 1) or s[i] (scale_dim = 2)
struct ScatterTask {
  double2* blk;
  int rows, cols, ld;
  const double2* src;
  int lds, r0, c0, conj_t, scale_dim;
  const double* s;
};

struct FactTask {
  double2* A;       // m x n column-major (lda = m); overwritten by U (SVD) or Q (QR)
  double2* V;       // SVD: n x n column-major right singular vectors; QR: R (n x n col-major)
  double* s;        // SVD: n singular values (descending); QR: unused
  int m, n;
};

void launch_gemm(const GemmTask* d_tasks, int ntasks, const GemmTerm* d_terms,
                 const int* d_tile_task, int ntiles, cudaStream_t st);
// et: element type of X and Y (0 double2 with the FP64 values, 1 float2 with
// the FP32 copy of the values)
// rows a of a W-stage block that one work item covers (work per block:
// ceil(rows / this) x wout x cols)
int wstage_rows_per_item();
void launch_wstage(const WTask* d_tasks, int ntasks, int64_t total_work, const int* d_rowptr,
                   const int* d_ent_w, const double* d_ent_v, const float* d_ent_vf, int et,
                   cudaStream_t st);
// One tile of the tensor-core GEMM, built on the host: rows m0.. (tc_tile_m()
// of them), complex columns n0 .. n0 + ncols (ncols <= tc_tile_n()), and the
// K stages (tc_stage_k() complex each, counted over the task's terms in
// order) that this tile's split owns: `count` of them, the first in term e0
// at complex offset k0.
struct TcTile {
  int task;
  int m0, n0, ncols;
  int count, e0, k0;
  int split;
};
// tensor-core grouped GEMM (kernels_tc.cu); mode 0 TF32, 1 3xTF32, 2 BF16;
// operands complex float, C complex double (tc = 0) or float (tc = 1);
// persistent: min(ntiles, n_sm) CTAs walk the tile list
void launch_gemm_tc(const GemmTask* d_tasks, const GemmTerm* d_terms, const TcTile* d_tiles,
                    const GemmSeg* d_segs, const SegOps* d_segops, int ntiles, int mode, int n_sm,
                    int* d_err, cudaStream_t st);
int tc_smem_bytes(int mode);
int tc_tile_m();
int tc_tile_n();
int tc_stage_k();   // complex K per staged tile
// C of each listed split task = sum over s in order of its part slices
// (+ C when beta); d_chunks: n triples (index into d_tasks, first element,
// end element) of the task's flat M x N range, one CTA each.  f32_parts: the slices are
// complex float (tensor-core kernel; added in FP64 for a complex double C),
// else of C's element type (FP64 kernel).
void launch_reduce_splits(const GemmTask* d_tasks, const GemmSeg* d_segs, const int* d_chunks,
                          int n, int f32_parts, cudaStream_t st);
// out (float2) = in (double2), n elements
void launch_to_float(const double2* in, float2* out, size_t n, cudaStream_t st);
// out (double2) = in (element type et), n elements
void launch_to_double(const void* in, int et, double2* out, size_t n, cudaStream_t st);
void launch_fill_one(void* p, int et, cudaStream_t st);
// raise a kernel's dynamic shared-memory limit once per device (thread-safe)
void set_smem_limit(const void* func, int bytes);
void launch_copy(const CopyTask* d_tasks, int ntasks, int to_work, cudaStream_t st);
void launch_scatter(const ScatterTask* d_tasks, int ntasks, cudaStream_t st);
void launch_zero(double2* p, size_t n, cudaStream_t st);
// max_bytes: largest (m*n + n*n) * 16 of the tasks (shared-memory sizing)
// h_tasks: the same tasks on the host (shapes decide between the one-CTA and
// the cluster kernel)
void launch_svd(const FactTask* d_tasks, int ntasks, int* d_status, cudaStream_t st,
                size_t max_bytes, const FactTask* h_tasks);
// h_tasks: the same tasks on the host (shapes decide between the one-CTA and
// the cluster kernel)
void launch_qr(const FactTask* d_tasks, int ntasks, cudaStream_t st, const FactTask* h_tasks);
// dst[t].A (n x n) = src[t].V^H (the R factor of a QR), n = dst[t].n
void launch_adjoint(const FactTask* d_src, const FactTask* d_dst, int n, cudaStream_t st);
// truncation rule over nv singular values (grouped by sector, each sector
// descending; sector id per value): writes kept count per sector and the
// discarded / total weight to out_w[0..1].
void launch_trunc(const double* d_s, const int* d_sec, int nv, int nsec, int D, double eps,
                  int* d_kept, double* d_w, double* d_sorted, int* d_sorted_sec, cudaStream_t st);
constexpr int QR_MAX_ROWS = 4096;
constexpr int QR_MAX_COLS = 2048;
// Krylov: c = exp(-i dt N^-1 H) e_0 (canonical orthogonalisation of N);
// status[0] = number of dropped directions, status[1] = 1 if non-finite.
void launch_krylov_small(const double2* d_N, const double2* d_H, int m, double dt,
                         double2* d_c, int* d_status, cudaStream_t st);
// y[k] = a * x[k] / b[k] style scalar helpers on device scalars
void launch_scalar_div_neg(const double2* num, const double2* den, double2* out, cudaStream_t st);
// norm of a buffer (sqrt of sum |x|^2) and scaling of it by 1/norm
void launch_normalize(double2* x, size_t n, double2* d_norm_out, cudaStream_t st);
void launch_scale(double2* x, size_t n, double2 a, cudaStream_t st);
// y = a y + b x, n complex elements
void launch_axpby(double2* y, const double2* x, size_t n, double2 a, double2 b, cudaStream_t st);
void launch_trace_channels(const void* E, int rows, int nch, int cols, const void* R, int et,
                           double2* out, cudaStream_t st);

}  // namespace tdmps
