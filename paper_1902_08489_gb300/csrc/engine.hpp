// Host engine of the tdmps library: context, block-sparse intermediates,
// contraction planners and the algorithms of the paper built on them.
#pragma once

#include <chrono>
#include <complex>
#include <functional>
#include <map>
#include <unordered_map>
#include <vector>

#include "internal.hpp"
#include "kernels.hpp"

namespace tdmps {

using cplx = std::complex<double>;

// ------------------------------------------------------------------ context

struct KStat {
  int64_t launches = 0;
  double ms = 0.0, flops = 0.0, bytes = 0.0;
};

struct Context;

// A worker of the instance batch: its own non-blocking stream and context
// (staging ring, status words, MPO caches), used by one host thread at a time.
struct Worker {
  cudaStream_t st = nullptr;
  std::unique_ptr<Context> c;
  Worker(int precision, size_t ring_bytes);
  ~Worker();
};

struct Context {
  cudaStream_t st = nullptr;
  int device = 0;
  int precision = TDMPS_FP64;
  int n_two_site = 2, n_one_site = 2;
  bool krylov_fp64 = true;    // Krylov inner products and result fit in FP64 regardless of precision
  int n_sm = 0;               // streaming multiprocessors of the device
  std::string err;
  // staging ring for task lists
  // The staging ring is split into RING_SEGS segments.  Every staged array's
  // consumer is enqueued before the next stage() call, so when stage() leaves
  // a segment, an event recorded there marks the point after which the GPU no
  // longer reads it; re-entering that segment waits only for that event,
  // never for the whole stream, so the GPU keeps the work queued behind it.
  static constexpr int RING_SEGS = 8;
  char* h_ring = nullptr;
  char* d_ring = nullptr;
  size_t ring_cap = 0, ring_off = 0, seg_cap = 0;
  int cur_seg = 0;
  cudaEvent_t seg_ev[RING_SEGS] = {};
  bool seg_live[RING_SEGS] = {};
  std::vector<DevPtr> oversize;   // task lists larger than the ring, until the next sync()
  // statistics
  bool stats = false;
  KStat kstat[TDMPS_KSTAT_COUNT];
  struct Pending { int kind; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;   // recorded and read back events, reused
  std::vector<char> pack;                // host packing buffer for staged task lists
  // scratch for device status words
  DevPtr status;   // int[16]: [0] SVD convergence, [4..5] Krylov, [8] tensor-core waits
  std::unique_ptr<MPOd> ident;   // identity MPO cache (by L)
  std::unique_ptr<MPOd> rdm;     // density-matrix MPO cache (by L)
  std::unique_ptr<std::vector<MPOd>> rdm_read;   // its per-bond readouts (by L)

  std::vector<std::unique_ptr<Worker>> workers;   // instance-batch workers (lazy)
  std::unique_ptr<Worker> aux;    // helper for the concurrent Krylov inner products (lazy)
  bool overlap_inner = true;      // run those inner products beside the fits

  explicit Context(cudaStream_t s, int prec, size_t ring_bytes = (size_t)256 << 20);
  ~Context();

  // copy a host array into device memory valid until the stream passes it
  const void* stage(const void* src, size_t bytes);
  template <class T> const T* stage(const std::vector<T>& v) {
    return v.empty() ? nullptr : (const T*)stage(v.data(), v.size() * sizeof(T));
  }
  // kernel timing bracket
  // host timing: the end of the previous launch call inside the current API call
  std::chrono::steady_clock::time_point host_mark, launch_start;
  bool host_mark_valid = false;
  void api_enter() { host_mark_valid = false; }
  cudaEvent_t take_event();
  void kbegin(int kind, cudaEvent_t* a);
  void kend(int kind, cudaEvent_t a, double flops, double bytes);
  void collect_stats();
  void sync();
  void wait_stream();   // cudaStreamSynchronize(st), timed into HOST_SYNC
  void wait_event(cudaEvent_t e);   // cudaEventSynchronize, timed into HOST_SYNC
  void check_device_errors();
  const MPOd& identity_mpo(int L);
  int et() const { return precision == TDMPS_FP64 ? 0 : 1; }
  int* tc_err() const { return (int*)status->p + 8; }
  const MPOd& rdm_mpo(int L);
  const std::vector<MPOd>& rdm_readouts(int L);
};

// ------------------------------------------------------------------ intermediates

// Block-sparse tensor with blocks rows x W x cols keyed (row group, sigma,
// channel group, column sector); sigma = -1 for environments.
struct Inter {
  struct Blk {
    int rg, sig, g, k;
    int rows, W, cols;
    size_t off;
  };
  std::vector<Blk> blocks;
  std::unordered_map<uint64_t, int> index;   // key(rg, sig, g, k) -> block id
  size_t size = 0;
  int et = 0;   // element type: 0 complex double, 1 complex float
  DevPtr data;
  size_t esz() const { return et ? sizeof(float2) : sizeof(double2); }
  // sector, channel-group and local-state indices are small: 16 bits each
  static uint64_t key(int rg, int sig, int g, int k) {
    return ((uint64_t)(uint16_t)rg << 48) | ((uint64_t)(uint16_t)(sig + 1) << 32) |
           ((uint64_t)(uint16_t)g << 16) | (uint64_t)(uint16_t)k;
  }
  int find(int rg, int sig, int g, int k) const {
    auto it = index.find(key(rg, sig, g, k));
    return it == index.end() ? -1 : it->second;
  }
  int add(int rg, int sig, int g, int k, int rows, int W, int cols) {
    int id = (int)blocks.size();
    blocks.push_back({rg, sig, g, k, rows, W, cols, size});
    index[key(rg, sig, g, k)] = id;
    size += (size_t)rows * W * cols;
    return id;
  }
  void* ptr(int b) const { return (char*)data->p + blocks[b].off * esz(); }
  void alloc(cudaStream_t st, bool zero);
};

// Environment E[a, w, a'] at one bond: rows = bra row groups, channels = MPO
// bond groups, cols = ket bond sectors.  Block (rg, g) has ket sector
// q_rg - q_g.
struct Env {
  RowGroups rows;
  const MPOBond* mb = nullptr;
  const Bond* ket = nullptr;
  Bond ket_copy;
  Inter t;
};

// MPS handle contents
struct MPSh {
  MPSd m;
};

// ------------------------------------------------------------------ engine API

void upload_mpo_tables(MPOd& m, Context& c);
MPSd mps_determinant(Context& c, int L, const uint8_t* occ);
MPSd mps_import(Context& c, int L, const int* bond_dims, const int* labels,
                const tdmps_complex* const* tensors);
void mps_export(Context& c, const MPSd& m, int* bond_dims, int* labels, tdmps_complex* const* tensors);
MPSd mps_copy(Context& c, const MPSd& m);

// fit target term: coef * (H or identity) |ket>
struct FitTerm {
  const MPSd* ket;
  const MPOd* mpo;           // nullptr -> identity
  cplx coef = 1.0;
  const double2* coef_dev = nullptr;   // multiplies coef when set
};
struct FitOpts {
  int D = 0;
  double eps = 0.0;
  int n_two_site = 0, n_one_site = 0;
  double* max_discarded = nullptr;
};
MPSd fit(Context& c, const std::vector<FitTerm>& terms, const MPSd& guess, const FitOpts& o);
// Mixed-precision contexts: rescale a fit C of a sum of states (terms
// without MPO) by <C|T> / <C|C>, both from FP64 overlaps.  A no-op in exact
// arithmetic (the last local solve of a fit is an orthogonal projection, so
// <C|T> = <C|C>); it removes the common scale error of the tensor-core
// sums.  FP64 contexts: nothing.
void restore_fit_scale(Context& c, MPSd& C, const std::vector<FitTerm>& terms);

// <bra_p| O |ket_p> for many pairs into device scalars; FP64 contractions
// unless fp64 == false (then the context precision)
void sandwich_batch(Context& c, const MPOd* mpo,
                    const std::vector<std::pair<const MPSd*, const MPSd*>>& pairs,
                    const std::vector<double2*>& outs, bool fp64 = true);
// <bra| O |ket> into a device scalar (O = mpo or identity)
void sandwich_dev(Context& c, const MPOd* mpo, const MPSd& bra, const MPSd& ket, double2* out);
cplx sandwich(Context& c, const MPOd* mpo, const MPSd& bra, const MPSd& ket);

MPSd right_canonicalize(Context& c, const MPSd& m);
double compress(Context& c, MPSd& m, int D, double eps);
void normalize_center(Context& c, MPSd& m, double2* norm_out);

// E = <psi|H|psi> / <psi|psi> and dE/dconj(A_i) = (H_i A_i - E N_i A_i) /
// <psi|psi> for every site (H_i, N_i: one-site products with the
// environments of <psi|H|psi> and <psi|psi>), in FP64, as an MPS with the
// bonds of psi.  Right environments are kept every `stride` sites and the
// others recomputed when the left-to-right pass needs them (1: all kept).
MPSd energy_gradient(Context& c, const MPOd& H, const MPSd& psi, int stride, double* energy,
                     size_t* env_bytes_peak = nullptr);
// The one-site effective Hamiltonian of Eq. add_min's local problem at one
// site of psi: y = L W_site x R with the environments of <psi|H|psi> left
// and right of the site, built once in the context's precision at creation.
struct LocalOp {
  MPOd H;            // a copy (device tables shared): the environments point into it
  int site = 0, L = 0, precision = 0;
  QN tot;
  Bond left, right;  // psi's bonds at site and site + 1
  Env LE, RE;
  size_t env_bytes = 0;
};
std::unique_ptr<LocalOp> local_op_create(Context& c, const MPOd& H, const MPSd& psi, int site);
// y's site <- the operator applied to x's site (x, y on psi's bonds there)
void local_op_apply(Context& c, const LocalOp& op, const MPSd& x, MPSd& y);
MPSd rk4_step(Context& c, const MPOd& H, const MPSd& psi, double dt, const FitOpts& o);
MPSd krylov_step(Context& c, const MPOd& H, const MPSd& psi, double dt, int m, bool orth,
                 const FitOpts& o);
void one_rdm(Context& c, const MPSd& psi, cplx* gamma);
// T_ij = sum_s <bra| c+_is c_js |ket> (L*L row-major)
void transition_rdm(Context& c, const MPSd& bra, const MPSd& ket, cplx* T);
// Gamma_ijkl = sum_st <psi| c+_is c+_kt c_lt c_js |psi> (L^4 row-major)
void two_rdm(Context& c, const MPSd& psi, cplx* Gam);
// a_(site, spin)|in> (dagger false) or its adjoint, exactly; false if zero
bool apply_site_op(Context& c, const MPSd& in, int site, int spin, bool dagger, MPSd& out);
// Eq. (green_time) at tau = 0, dt, ..., n_steps dt (method 0 Krylov, 1 RK4)
void green_function(Context& c, const MPOd& H, const MPSd& psi0, int i, int j, double dt,
                    int n_steps, int method, int m, bool orth, const FitOpts& o, cplx* G);
// Many independent time evolutions at once (batch.cpp): item k advances
// *states[k] by n_steps[k] steps of dt[k] with its own MPO, D and eps;
// method 0 Krylov (m, orth), 1 RK4.  status[k] receives 0 or the item's
// error code (its state is then unchanged) and msgs[k] the message.
struct BatchItem {
  const MPOd* H;
  MPSd* state;
  double dt;
  int n_steps, D;
  double eps;
};
void evolve_batch(Context& c, const std::vector<BatchItem>& items, int method, int m, bool orth,
                  int n_workers, int* status, std::vector<std::string>& msgs);
// overlap with all blocks in a fixed device array (noalloc.cu)
cplx overlap_noalloc(Context& c, const MPSd& bra, const MPSd& ket);

}  // namespace tdmps
