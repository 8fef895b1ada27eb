/*
 * tdmps.h -- C ABI of the GB300 library for MPS time evolution of the
 * ab-initio electronic Schroedinger equation (Frahm & Pfannkuche,
 * "Ultrafast ab-initio Quantum Chemistry Using Matrix Product States").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Units: atomic units, hbar = 1.
 * - Orbitals i = 0..L-1, spin orbitals ordered 0up, 0down, 1up, ... as in the
 *   paper's Eq. (fci).  Local states of one orbital: 0 = |0>, 1 = |up>,
 *   2 = |down>, 3 = |up down> (= c+_up c+_down |0>), charges (N, 2S_z) =
 *   (0,0), (1,1), (1,-1), (2,0).
 * - Hamiltonian, Eq. (hamil), with integrals read in chemist order:
 *     H = sum_{ij,s} h_ij c+_is c_js
 *       + 1/2 sum_{ijkl,s,t} (ij|kl) c+_is c+_kt c_lt c_js + e0.
 * - Handles own their memory; device memory comes from the context's stream
 *   ordered pool (cudaMallocAsync on the context stream).  Host arrays passed
 *   in are borrowed for the duration of the call and copied.
 * - All GPU work is enqueued on the context stream.  Calls that return host
 *   scalars or host arrays synchronise that stream before returning.
 * - Return value 0 on success, a negative TDMPS_ERR_* code otherwise; the
 *   message of the last error of a context is returned by tdmps_last_error.
 *   There is no CPU fallback: when a CUDA call fails the entry point returns
 *   TDMPS_ERR_CUDA.  A handle whose call failed stays valid and unchanged
 *   unless stated otherwise.  A NaN or Inf scalar argument (alpha, dt)
 *   returns TDMPS_ERR_NONFINITE, and a NULL handle or an out-of-range size
 *   TDMPS_ERR_INVALID_ARG, both before any work is enqueued.
 * - Complex numbers are passed as tdmps_complex {re, im} (layout of C99
 *   double complex).
 */
#ifndef TDMPS_H
#define TDMPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdmps_ctx_s* tdmps_ctx_t;
typedef struct tdmps_mpo_s* tdmps_mpo_t;
typedef struct tdmps_mps_s* tdmps_mps_t;
typedef struct tdmps_heff_s* tdmps_heff_t;

typedef struct {
  double re, im;
} tdmps_complex;

enum {
  TDMPS_OK = 0,
  TDMPS_ERR_INVALID_ARG = -1,
  TDMPS_ERR_SECTOR = -2,          /* quantum numbers of operands do not match */
  TDMPS_ERR_KRYLOV_SINGULAR = -3, /* Krylov overlap matrix has rank < 2      */
  TDMPS_ERR_NONFINITE = -4,       /* NaN or Inf in an input or a result      */
  TDMPS_ERR_CUDA = -5,            /* a CUDA runtime call or kernel failed    */
  TDMPS_ERR_OOM = -6,             /* device allocation failed                */
  TDMPS_ERR_ZERO_STATE = -7,      /* a fit target vanished on its sweep      */
  TDMPS_ERR_NUMERIC = -8          /* an iterative kernel did not converge    */
};

/* Arithmetic of the fit contractions (environments, local matvecs, sums)
 * and, if tdmps_set_krylov_fp64(ctx, 0) asks for it, of the Krylov inner
 * products <phi_i|phi_j>, <phi_i|H|phi_j>.  Factorisations (QR, SVD), the
 * Krylov matrices and their exponential, the centre-site norms and the
 * observables (tdmps_overlap, tdmps_expectation, tdmps_one_rdm,
 * tdmps_transition_rdm, tdmps_two_rdm) are always FP64. */
enum {
  TDMPS_FP64 = 0,   /* complex FP64 everywhere                               */
  TDMPS_TF32 = 1,   /* TF32 tensor-core products, FP32 accumulation          */
  TDMPS_TF32X3 = 2, /* split TF32 (hi*hi + hi*lo + lo*hi), FP32 accumulation */
  TDMPS_BF16 = 3    /* BF16 tensor-core products (kind::f16), FP32
                       accumulation; environments stored in FP32             */
};

/* ---------------------------------------------------------------- context */

/* Create a context on the current CUDA device.  cuda_stream: a cudaStream_t
 * (NULL = the legacy default stream).  precision: TDMPS_FP64, TDMPS_TF32,
 * TDMPS_TF32X3 or TDMPS_BF16 (the mixed modes keep environments and
 * intermediates in complex FP32 and run the block contractions on the
 * tcgen05 tensor cores).  The context allocates its staging ring (pinned
 * host and device memory) here.  Errors: INVALID_ARG (bad precision,
 * ctx == NULL; message in tdmps_create_error), CUDA, OOM. */
int tdmps_create(tdmps_ctx_t* ctx, void* cuda_stream, int precision);
/* Waits for the context stream, then releases the context: its staging
 * ring, caches and helper streams.  MPO and MPS handles made with it can
 * then only be freed; their memory is freed in stream order on the CUDA
 * stream the context was created on, which must still exist at that point.
 * Errors: INVALID_ARG for a NULL ctx. */
int tdmps_destroy(tdmps_ctx_t ctx);
/* Message of the last failed call on ctx ("" if none).  Owned by ctx. */
const char* tdmps_last_error(tdmps_ctx_t ctx);
/* Message of the last failed tdmps_create on this thread. */
const char* tdmps_create_error(void);
/* Precision of the following calls (TDMPS_FP64, _TF32, _TF32X3, _BF16).
 * Errors: INVALID_ARG for a NULL ctx or an unknown precision. */
int tdmps_set_precision(tdmps_ctx_t ctx, int precision);

/* Sweep schedule of every variational fit (Sec. 2.2.1, Eq. add_min; the
 * paper converges its fits in about ten sweeps): n_two_site two-site sweeps (each a
 * left-to-right and a right-to-left half sweep, truncated SVD of every
 * two-site tensor) followed by n_one_site one-site sweeps (QR / LQ gauge
 * moves, bond dimensions fixed).  Defaults: 2 and 2.  Errors: INVALID_ARG if
 * either is negative or both are 0. */
int tdmps_set_schedule(tdmps_ctx_t ctx, int n_two_site, int n_one_site);

/* The Krylov algebra in FP64 (on != 0, the default) or in the context
 * precision (on == 0).  It covers the inner products (Gram-Schmidt
 * coefficients and the N, H matrices of Eq. krylov_evo) and the fit of the
 * step's result sum_j c_j |phi_j>.  With on == 0 the TF32 modes run faster,
 * but the canonical orthogonalisation sees the TF32 rounding of N and H.
 * The Krylov basis vectors are always fitted in the context precision: N
 * and H are measured on the vectors as fitted, so their FP32-level errors
 * change the step only through the span they give.  The small matrices are
 * accumulated and processed in FP64 either way. */
int tdmps_set_krylov_fp64(tdmps_ctx_t ctx, int on);

/* Scheduling of the FP64 Krylov inner products of an orthogonal-basis step
 * (Eq. kry_orth).  Those of Gram-Schmidt step k depend on phi_0..phi_k only.
 * With on != 0 (the default) they run on a helper stream driven by a
 * second host thread, concurrently with the fit of H phi_k. With on == 0
 * they run after that fit, in order, on the context stream.  Both run the
 * same contractions with the same launch plans (fixed summation order).  The
 * serial order is for tools that serialise kernels across threads, such as
 * profilers.  It applies when the inner products are FP64
 * (tdmps_set_krylov_fp64) and m > 2.  The helper stream has the default,
 * lowest, priority: a context bound to a higher-priority stream keeps its
 * fits (the critical path of the step) ahead of the inner products.
 * Errors: INVALID_ARG for a NULL ctx. */
int tdmps_set_concurrent_inner(tdmps_ctx_t ctx, int on);

/* ------------------------------------------------------- orbital order */

/* Fiedler ordering of the orbitals (Sec. 3.2 sorts the molecular orbitals
 * along a Fiedler vector, which narrows the band of the Hamiltonian
 * matrix).  Graph weights W_ij = |h_ij| + |(ij|ji)| (symmetrised), Laplacian
 * D - W, and the orbitals sorted by the eigenvector of its second smallest
 * eigenvalue (ties by index; the eigenvector's sign is chosen so that its
 * correlation with the input order is >= 0).  perm[k] = input orbital placed
 * at position k; permute h and eri with it before tdmps_build_mpo.  Host
 * only, no context.  A graph whose second eigenvalue is degenerate (for
 * example a disconnected one) has no unique Fiedler vector; the result is
 * then one valid ordering.  Errors: INVALID_ARG (L < 1 or > 64, NULL),
 * NONFINITE. */
int tdmps_fiedler_order(const double* h, const double* eri, int L, int* perm);

/* ------------------------------------------------------------------- MPO */

/* Matrix product operator of Eq. (hamil) (paper Sec. 2.2 "Time Evolution
 * Methods").  h: L*L row-major, symmetric.  eri: L^4 row-major (ij|kl).
 * n_elec: electrons of the states it will act on (only checked by later
 * calls).  Terms are split at every bond into left and right operator
 * strings; a channel carries either the left string (coefficient applied
 * later) or the right string (coefficients already summed into the left
 * operator), whichever side holds fewer operators, ties going to the left
 * half of the chain; fermionic signs follow the Jordan-Wigner order of the
 * spin orbitals.  Errors: INVALID_ARG (L < 1 or > 64, NULL arrays),
 * NONFINITE, CUDA, OOM. */
int tdmps_build_mpo(tdmps_ctx_t ctx, const double* h, const double* eri, int L,
                    int n_elec, double e0, tdmps_mpo_t* out);
/* ctx may be NULL: the MPO is then built on the host only (no GPU needed);
 * its device tables are uploaded on first use by a context. */

/* Channel count of every bond (bond_dims[L+1]) and total stored elements.
 * Either output may be NULL.  Host only.  Errors: INVALID_ARG for a NULL
 * mpo. */
int tdmps_mpo_info(tdmps_mpo_t mpo, int* bond_dims, int64_t* n_elements);
/* Host copy of the stored elements of W_site, 0 <= site < L: entry e is the
 * matrix element <sig|W[w_in, w_out]|sigp> = v[e] between channel w_in of
 * bond `site` and channel w_out of bond site+1.  *count is the capacity on
 * entry and the number of elements on return; with win == NULL only the
 * number is returned.  No GPU is needed.  Errors: INVALID_ARG for a NULL
 * mpo or count, a site out of range, a NULL wout/sig/sigp/v when win is
 * given, or a capacity below the element count (*count then holds the
 * count needed). */
int tdmps_mpo_elements(tdmps_mpo_t mpo, int site, int64_t* count, int* win, int* wout, int* sig,
                       int* sigp, double* v);
/* Releases the MPO handle, its host tables and its device tables (freed in
 * stream order on the stream that uploaded them).  NULL is a no-op; always
 * returns 0. */
int tdmps_mpo_free(tdmps_mpo_t mpo);

/* ------------------------------------------------------------------- MPS */

/* Product state of one determinant (paper Eq. mps with bond dimension 1).
 * occ[L]: 0 = empty, 1 = up, 2 = down, 3 = both.  Errors: INVALID_ARG. */
int tdmps_mps_from_determinant(tdmps_ctx_t ctx, int L, const uint8_t* occ,
                               tdmps_mps_t* out);

/* Import dense site tensors with labelled bonds (Eq. mps).
 * bond_dims[L+1]: dimensions D_0..D_L (D_0 = 1 with label (0,0)).
 * labels: for k = 0..L, D_k pairs (N, 2S_z) concatenated (int32 pairs).
 * tensors[i]: host array D_i x 4 x D_{i+1}, row-major, complex.
 * Entries that violate charge conservation must be zero.
 * Errors: INVALID_ARG (NULL argument, L outside 1..63, a bond dimension
 * below 1, bond 0 not one-dimensional with label (0, 0), a non-zero entry
 * that violates charge conservation), SECTOR (D_L is not 1), NONFINITE (a
 * NaN or Inf entry), CUDA, OOM. */
int tdmps_mps_import(tdmps_ctx_t ctx, int L, const int* bond_dims, const int* labels,
                     const tdmps_complex* const* tensors, tdmps_mps_t* out);
/* Export: with tensors == NULL only bond_dims (L+1 entries) is written; then
 * call again with labels (sum D_k pairs) and tensors[i] of D_i*4*D_{i+1}.
 * Errors: INVALID_ARG (NULL mps or bond_dims, tensors without labels), CUDA. */
int tdmps_mps_export(tdmps_ctx_t ctx, tdmps_mps_t mps, int* bond_dims, int* labels,
                     tdmps_complex* const* tensors);
/* Length, total charge (N, 2S_z) and the largest bond dimension (sum over
 * the sectors of a bond, maximised over bonds).  Host only, no stream work;
 * any output pointer may be NULL.  Errors: INVALID_ARG for a NULL handle. */
int tdmps_mps_info(tdmps_mps_t mps, int* L, int* n_elec, int* two_sz, int* max_bond);
/* Deep copy of `in` (device to device on the context stream); *out is a new
 * handle owned by the caller.  Errors: INVALID_ARG, CUDA, OOM. */
int tdmps_mps_copy(tdmps_ctx_t ctx, tdmps_mps_t in, tdmps_mps_t* out);
/* Releases the MPS handle and its device memory (freed in stream order on
 * the stream it was allocated on).  NULL is a no-op; always returns 0. */
int tdmps_mps_free(tdmps_mps_t mps);

/* ---------------------------------------------------------- operations */

/* out ~ alpha * H |in> by variational fitting (Sec. 2.2.1, Eq. add_min) at
 * bond dimension <= D, discarding at most a relative weight eps per
 * truncation; n_sweeps > 0 overrides the one-site sweep count of the
 * schedule (n_sweeps <= 0 keeps it).  The initial guess is `in`.
 * The result is right-canonical with its norm on site 0.
 * Errors: INVALID_ARG (NULL argument, lengths differ, D < 1, eps outside [0,
 * 1), a symmetry block beyond the supported QR/SVD size), ZERO_STATE (the
 * fit target vanished on a sweep), NUMERIC (a Jacobi SVD did not converge,
 * or a tensor-core wait timed out), NONFINITE (non-finite scalar argument or
 * singular values), CUDA, OOM. */
int tdmps_apply_H(tdmps_ctx_t ctx, tdmps_mpo_t mpo, tdmps_mps_t in, tdmps_complex alpha,
                  int D, double eps, int n_sweeps, tdmps_mps_t* out);

/* out ~ sum_k coefs[k] |terms[k]> (Eqs. sum_exact, add_min), guess terms[0].
 * In the TF32/BF16 precisions the result is rescaled by <out|T>/<out|out>
 * (T the exact sum; FP64 overlaps), which the projection property of the
 * fit makes 1 in exact arithmetic and which removes the common shrink of
 * the tensor-core sums.
 * Errors: INVALID_ARG (n_terms < 1, NULL argument or term, lengths differ, D
 * < 1, eps outside [0, 1), a symmetry block beyond the supported QR/SVD
 * size), SECTOR (terms of different (N, 2S_z)), ZERO_STATE (the fit target
 * vanished on a sweep), NUMERIC (a Jacobi SVD did not converge, or a
 * tensor-core wait timed out), NONFINITE (non-finite scalar argument or
 * singular values), CUDA, OOM. */
int tdmps_sum(tdmps_ctx_t ctx, int n_terms, const tdmps_complex* coefs,
              const tdmps_mps_t* terms, int D, double eps, tdmps_mps_t* out);

/* The adjoint of the energy with respect to the state (Sec. 2.2.1: the
 * effective-Hamiltonian matvec of the local problem of Eq. add_min, applied
 * to the state's own sites).  For E = <psi|H|psi> / <psi|psi>:
 *     *energy = E,
 *     site i of *grad = dE/dconj(A_i) = (H_i A_i - E N_i A_i) / <psi|psi>,
 * where H_i A_i = sum L[a,w,a'] W[w,w',s,s'] A_i[a',s',b'] R[b,w',b'] with the
 * environments of <psi|H|psi> left and right of site i, and N_i A_i the same
 * with the identity operator (psi's gauge is not assumed).  A perturbation
 * dA_i changes E by 2 Re sum conj(G_i) dA_i to first order.  *grad is a new
 * handle with psi's bonds and block layout whose "sites" are the gradients
 * (read them with tdmps_mps_export; it is no physical state).  FP64 in every
 * context precision.  stride >= 1: right environments are kept at every
 * stride-th bond and rebuilt in between when the left-to-right pass needs
 * them (one extra right sweep; environment memory O(L/stride + stride)
 * instead of O(L)); stride = 1 keeps all.  env_bytes_peak (may be NULL)
 * receives the most device memory that environments held at once.
 * Errors: INVALID_ARG (NULL argument, stride < 1, lengths differ),
 * ZERO_STATE (psi = 0), CUDA. */
int tdmps_energy_gradient(tdmps_ctx_t ctx, tdmps_mpo_t mpo, tdmps_mps_t psi, int stride,
                          double* energy, tdmps_mps_t* grad, size_t* env_bytes_peak);

/* The one-site effective Hamiltonian of the local problem of Eq. add_min
 * (Sec. 2.2.1) at site `site` of psi, as an operator on that site's tensor:
 *     y[a,s,b] = sum L[a,w,a'] W_site[w,w',s,s'] x[a',s',b'] R[b,w',b'],
 * L and R the environments of <psi|H|psi> left and right of the site (the
 * product every one-site fit step forms).  psi's gauge is not assumed:
 * <psi(x)|H|psi(z)> = <x, H_site z> for psi with the site replaced, so in
 * psi's mixed-canonical gauge at the site the operator is H projected onto
 * the site's variational space.  Create builds the two environments once
 * (one sweep in from each end, in the context's precision) and keeps them
 * on the device; *env_bytes (may be NULL) receives their size.  The handle
 * copies what it needs of mpo and psi: both may be freed before it.  Free
 * it before its context.
 * Errors: INVALID_ARG (NULL argument, lengths differ, site outside
 * 0..L-1), SECTOR, CUDA. */
int tdmps_heff_create(tdmps_ctx_t ctx, tdmps_mpo_t mpo, tdmps_mps_t psi, int site,
                      tdmps_heff_t* out, size_t* env_bytes);

/* Replace site `site` of y with the operator applied to site `site` of x.
 * x and y need psi's (N, 2S_z), length and bonds at site and site + 1 (for
 * instance copies of psi; x == y is allowed).  Only that site of y changes,
 * and y is then in no canonical gauge.  One launch per stage (L-stage, MPO
 * stage, R-stage; a GEMM with split K is followed by its ordered reduction),
 * in the precision the operator was created in.
 * Errors: INVALID_ARG (NULL argument, context precision changed since
 * create), SECTOR (bonds differ), CUDA. */
int tdmps_heff_apply(tdmps_ctx_t ctx, tdmps_heff_t op, tdmps_mps_t x, tdmps_mps_t y);

/* Release the operator's environments (stream-ordered). */
int tdmps_heff_free(tdmps_heff_t op);

/* E = <psi|H|psi> / <psi|psi> (real part; H is Hermitian), FP64 chains.
 * Errors: INVALID_ARG, ZERO_STATE (psi = 0), CUDA. */
int tdmps_energy(tdmps_ctx_t ctx, tdmps_mpo_t mpo, tdmps_mps_t psi, double* energy);

/* The gradient of that energy with respect to the integrals of Eq. hamil
 * (E is linear in them): dE_dh[i*L + j] = Re gamma_ij / <psi|psi> and
 * dE_deri[((i*L + j)*L + k)*L + l] = Re Gamma_ijkl / (2 <psi|psi>), gamma and
 * Gamma as in tdmps_one_rdm and tdmps_two_rdm (chemist order); dE/de0 = 1.
 * Either output may be NULL (not both).  Host arrays of L^2 and L^4 doubles.
 * Errors: INVALID_ARG, ZERO_STATE, CUDA. */
int tdmps_integral_gradient(tdmps_ctx_t ctx, tdmps_mps_t psi, double* dE_dh, double* dE_deri);

/* <bra|ket> (the contraction of two chains of Eq. mps), FP64.  Errors:
 * INVALID_ARG (NULL argument, lengths differ), SECTOR (different (N, 2S_z)),
 * CUDA, OOM. */
int tdmps_overlap(tdmps_ctx_t ctx, tdmps_mps_t bra, tdmps_mps_t ket, tdmps_complex* out);

/* Overlap that allocates no device memory.  The paper has no counterpart:
 * this is a service for callers that must not allocate device memory while
 * they run -- applications whose caching allocator has to stay the only
 * owner of device memory, or loops on a fixed memory budget where an
 * allocation's latency or failure is not acceptable.  Same result as
 * tdmps_overlap (FP64 chain contraction); the environments and intermediate
 * blocks live in one file-scope device array of TDMPS_NOALLOC_SCRATCH_BYTES,
 * which every GPU that loads the library holds until the process exits.
 * The first call on a device resolves that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call
 * before any stream capture.  Task lists go through the staging ring that
 * tdmps_create allocated.  All calls on a device share the array and each
 * overwrites it, so calls that overlap on the GPU (several contexts or
 * streams at once) race.  A pair whose environments do not fit, or whose
 * task list for one launch exceeds a segment of the staging ring, returns
 * TDMPS_ERR_INVALID_ARG before any work is enqueued on the GPU; so does a
 * context whose device is not the current device.  Other errors: SECTOR
 * (different (N, 2S_z)), CUDA. */
#define TDMPS_NOALLOC_SCRATCH_BYTES (16u << 20)
int tdmps_overlap_noalloc(tdmps_ctx_t ctx, tdmps_mps_t bra, tdmps_mps_t ket, tdmps_complex* out);

/* <bra|H|ket> with the MPO (Sec. 2.2.3, H_ij of Eq. krylov_evo), FP64.
 * Errors: INVALID_ARG (NULL argument, lengths differ), SECTOR (different
 * (N, 2S_z)), CUDA, OOM. */
int tdmps_expectation(tdmps_ctx_t ctx, tdmps_mpo_t mpo, tdmps_mps_t bra, tdmps_mps_t ket,
                      tdmps_complex* out);

/* SVD compression in place (Sec. 2.1: keep the D largest singular values):
 * right-canonicalise, one left-to-right pass of truncated SVDs, exact LQ pass
 * back.  discarded_weight (may be NULL): sum over bonds of the relative
 * discarded weight.  Errors: INVALID_ARG (NULL argument, D < 1, eps outside
 * [0, 1)), ZERO_STATE (a zero state), NUMERIC, NONFINITE (the SVD), CUDA,
 * OOM; inout is unchanged on error. */
int tdmps_compress(tdmps_ctx_t ctx, tdmps_mps_t inout, int D, double eps,
                   double* discarded_weight);

/* One RK4 step in place (Sec. 2.2.2, stages k1..k4 with k = -i dt H(...),
 * Eq. rk_add): four fitted H applications and four fitted sums.
 * Errors: INVALID_ARG (NULL argument, lengths differ, D < 1, eps outside [0,
 * 1), a symmetry block beyond the supported QR/SVD size), ZERO_STATE (the
 * fit target vanished on a sweep), NUMERIC (a Jacobi SVD did not converge,
 * or a tensor-core wait timed out), NONFINITE (non-finite scalar argument or
 * singular values), CUDA, OOM; inout is unchanged on error. */
int tdmps_rk4_step(tdmps_ctx_t ctx, tdmps_mpo_t mpo, tdmps_mps_t inout, double dt, int D,
                   double eps);

/* One Krylov step in place (Sec. 2.2.3) with m >= 2 basis vectors including
 * phi_0 = psi.  orthogonal != 0: Eq. (kry_orth) (fit of H phi_k, then a
 * fitted sum subtracting <phi_j|H|phi_k>/<phi_j|phi_j> phi_j); otherwise
 * Eq. (kry_non).  Each new vector is normalised.  The new state is the fitted
 * sum of Eq. (krylov_evo) with N and H measured exactly; exp(-i dt N^-1 H) e0
 * uses canonical orthogonalisation of N (eigenvalues below 1e-12 * max are
 * dropped; KRYLOV_SINGULAR if fewer than 2 remain, inout unchanged).
 * Errors: INVALID_ARG (NULL argument, lengths differ, m outside [2, 16], D <
 * 1, eps outside [0, 1), a symmetry block beyond the supported QR/SVD size),
 * ZERO_STATE (the fit target vanished on a sweep), NUMERIC (a Jacobi SVD did
 * not converge, or a tensor-core wait timed out), NONFINITE (non-finite
 * scalar argument or singular values or Krylov matrices), CUDA, OOM,
 * KRYLOV_SINGULAR; inout is unchanged on error. */
int tdmps_krylov_step(tdmps_ctx_t ctx, tdmps_mpo_t mpo, tdmps_mps_t inout, double dt, int m,
                      int orthogonal, int D, double eps);

/* gamma_ij = sum_s <psi| c+_is c_js |psi> (Sec. 3.2, the 1BRDM), not
 * normalised by <psi|psi>.  gamma: host array L*L row-major.  FP64.
 * Errors: INVALID_ARG (NULL argument), CUDA, OOM. */
int tdmps_one_rdm(tdmps_ctx_t ctx, tdmps_mps_t psi, tdmps_complex* gamma);

/* T_ij = sum_s <bra| c+_is c_js |ket>: the 1BRDM between two states of the
 * same (N, 2S_z) (TDMPS_ERR_SECTOR otherwise), not normalised.  T: host
 * array L*L row-major.  FP64.  Errors: INVALID_ARG (NULL argument, lengths
 * differ), SECTOR, CUDA, OOM. */
int tdmps_transition_rdm(tdmps_ctx_t ctx, tdmps_mps_t bra, tdmps_mps_t ket, tdmps_complex* T);

/* Gamma_ijkl = sum_{s,t} <psi| c+_is c+_kt c_lt c_js |psi>, the partner of
 * the chemist-order integral (ij|kl) in Eq. hamil, so that
 * <psi|H|psi> = sum h_ij gamma_ij + 1/2 sum (ij|kl) Gamma_ijkl + e0 <psi|psi>
 * and dE/dh_ij = gamma_ij, dE/d(ij|kl) = Gamma_ijkl / 2.  Not normalised.
 * Gamma: host array L^4 row-major (index ((i*L + j)*L + k)*L + l).  Computed
 * as sum_s T[c_is psi, c_js psi]_kl from 2 L^2 transition 1BRDMs of the
 * exactly ionised states (tdmps_apply_site_op).  FP64.  Errors: INVALID_ARG
 * (NULL argument), CUDA, OOM. */
int tdmps_two_rdm(tdmps_ctx_t ctx, tdmps_mps_t psi, tdmps_complex* Gamma);

/* ------------------------------------------------------- site operators */

/* out = c_(site, spin)|in> (dagger = 0) or c+_(site, spin)|in> (dagger = 1),
 * exactly (no fit: the operator has bond dimension one).  spin: 0 up,
 * 1 down; site in [0, L).  Jordan-Wigner order 1up, 1down, 2up, ... (Eq.
 * fci): the parity (-1)^n of every earlier site and, for spin down, of the
 * up electron on the same site.  The result has (N -+ 1, 2S_z -+ 1 for up,
 * 2S_z +- 1 for down) and keeps the bond dimensions of `in`; it is neither
 * normalised nor canonical.  This is the ionisation step of the one-particle
 * Green's function (Eq. green_time: c_js|psi0>, propagated with a negative
 * time step, projected on c_is|psi0>).  Returns TDMPS_ERR_ZERO_STATE, with
 * *out untouched, when the operator annihilates every configuration of
 * `in` (for example c_up on a state with that orbital empty).  Other
 * errors: INVALID_ARG (NULL argument, site outside [0, L), spin not 0 or 1),
 * CUDA, OOM. */
int tdmps_apply_site_op(tdmps_ctx_t ctx, tdmps_mps_t in, int site, int spin, int dagger,
                        tdmps_mps_t* out);

/* One-particle Green's function of Eq. (green_time), spin-summed and
 * normalised, at tau = n dt for n = 0..n_steps:
 *   G_ij(tau) = -i sum_s <psi0| c+_is exp(+i H tau) c_js |psi0>
 *                  / sum_s <psi0| c+_is c_js |psi0>   (hbar = 1).
 * As in the paper: c_js|psi0> exactly (tdmps_apply_site_op), propagated
 * backwards in time (time step -dt) with method 0 = Krylov
 * (tdmps_krylov_step with m, orthogonal) or 1 = RK4 (tdmps_rk4_step; m and
 * orthogonal ignored), fitted at D / eps, and projected on c_is|psi0> after
 * every step (FP64 overlaps).  The MPO does not depend on the electron
 * number, so the MPO of psi0's Hamiltonian serves the ionised sectors.
 * G: host array of n_steps + 1 values.  Errors: INVALID_ARG (site, method,
 * n_steps < 0), ZERO_STATE (the denominator vanishes), and those of the
 * integrator. */
int tdmps_green_function(tdmps_ctx_t ctx, tdmps_mpo_t mpo, tdmps_mps_t psi0, int i, int j,
                         double dt, int n_steps, int method, int m, int orthogonal, int D,
                         double eps, tdmps_complex* G);

/* ------------------------------------------------------- instance batch */

/* Many independent time evolutions at once: item k advances states[k] in
 * place by n_steps[k] steps of dt[k] under mpos[k], fitted at D[k] / eps[k]
 * (method 0 = Krylov with m and orthogonal as in tdmps_krylov_step, 1 = RK4).
 * Items may differ in L, electrons and bond dimension; they may share MPOs
 * but not states.  n_workers host threads (<= 0: min(8, n)), each with its
 * own CUDA stream, staging ring and caches, take the next unfinished item
 * from a shared counter, so the kernels of several items overlap on the GPU.
 * The context's stream is ordered before the first and after the last
 * kernel of the batch; the context's precision and sweep schedule apply to
 * every item.  Each item runs the launch plans a separate tdmps_rk4_step /
 * tdmps_krylov_step call would run (the tests compare them to 1e-11).  status (may be NULL): n codes, 0 for every item that finished;
 * a failed item keeps its input state.  Returns 0 when every item finished,
 * else the code of the first failed item (message in tdmps_last_error with
 * its index).  The worker streams are created on the first call and live as
 * long as the context. */
int tdmps_evolve_batch(tdmps_ctx_t ctx, int n, const tdmps_mpo_t* mpos, tdmps_mps_t* states,
                       const double* dt, const int* n_steps, const int* D, const double* eps,
                       int method, int m, int orthogonal, int n_workers, int* status);

/* ------------------------------------------------------------ statistics */

/* Per-kernel-class timing with CUDA events on the context stream, and the
 * algorithmic work of every launch (block-sparse FLOPs / bytes, padding
 * excluded).  Classes: see TDMPS_KSTAT_*. */
enum {
  TDMPS_KSTAT_GEMM = 0,      /* block contractions on the tensor cores (TF32 modes) */
  TDMPS_KSTAT_WSTAGE = 1,    /* sparse MPO-tensor application                       */
  TDMPS_KSTAT_QR = 2,
  TDMPS_KSTAT_SVD = 3,
  TDMPS_KSTAT_OTHER = 4,
  TDMPS_KSTAT_GEMM_FP64 = 5, /* FP64 block contractions (FP64 mode, inner products,
                                observables, gauge moves)                          */
  TDMPS_KSTAT_HOST_PLAN = 6,   /* host wall time between consecutive launches inside
                                  one API call (planning, allocation, staging); no
                                  flops/bytes; launches = number of intervals      */
  TDMPS_KSTAT_HOST_LAUNCH = 7, /* host wall time inside the launch calls themselves */
  TDMPS_KSTAT_HOST_SYNC = 8,   /* host wall time blocked in stream synchronisations
                                  (part of HOST_PLAN when it falls between launches) */
  TDMPS_KSTAT_COUNT = 9
};
typedef struct {
  int64_t launches;
  double ms;        /* summed event time of those launches   */
  double flops;     /* algorithmic real FLOPs                */
  double bytes;     /* algorithmic bytes read + written      */
} tdmps_kstat;
/* Turns the recording on (enable != 0) or off.  Pending records are first
 * folded into the totals, which synchronises the context stream.  Recording
 * is off by default, and no events are recorded while it is off.
 * Errors: INVALID_ARG for a NULL ctx, CUDA. */
int tdmps_stats_enable(tdmps_ctx_t ctx, int enable);
/* Zeroes every class after folding in what is pending (synchronises the
 * context stream).  Errors: INVALID_ARG for a NULL ctx, CUDA. */
int tdmps_stats_reset(tdmps_ctx_t ctx);
/* Totals of class `kind` (0 <= kind < TDMPS_KSTAT_COUNT) since the last
 * reset.  Reading the event times synchronises the context stream.
 * Errors: INVALID_ARG for a NULL ctx or out, or a kind out of range. */
int tdmps_stats_get(tdmps_ctx_t ctx, int kind, tdmps_kstat* out);

#ifdef __cplusplus
}
#endif
#endif /* TDMPS_H */
