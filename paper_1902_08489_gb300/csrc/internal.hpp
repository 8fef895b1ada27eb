// Internal data structures of the tdmps library (host side).
//
// Quantum numbers: every bond basis vector carries (N, 2S_z); site local
// states |0>, |up>, |down>, |up down> carry (0,0), (1,1), (1,-1), (2,0).
// Block sparsity: a site tensor A[a, sigma, b] has a dense block for every
// (left sector, sigma) whose charge sum is a right sector; environments
// E[a, w, a'] have a block for every (bra sector, MPO channel group) whose ket
// sector a' = q_a - q_w exists.  All blocks are row-major complex.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "../../include/tdmps.h"

namespace tdmps {

struct QN {
  int n = 0, s = 0;
  QN() = default;
  QN(int n_, int s_) : n(n_), s(s_) {}
  QN operator+(const QN& o) const { return {n + o.n, s + o.s}; }
  QN operator-(const QN& o) const { return {n - o.n, s - o.s}; }
  QN operator-() const { return {-n, -s}; }
  bool operator==(const QN& o) const { return n == o.n && s == o.s; }
  bool operator!=(const QN& o) const { return !(*this == o); }
  bool operator<(const QN& o) const { return n != o.n ? n < o.n : s < o.s; }
};

static const QN SITE_Q[4] = {QN(0, 0), QN(1, 1), QN(1, -1), QN(2, 0)};

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define TD_CHECK_CUDA(call)                                                          \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      throw ::tdmps::Error(e_ == cudaErrorMemoryAllocation ? TDMPS_ERR_OOM            \
                                                            : TDMPS_ERR_CUDA,        \
                           std::string(#call) + ": " + cudaGetErrorString(e_));      \
  } while (0)

// ------------------------------------------------------------------ memory

// Device allocation from the stream-ordered pool of the owning stream.
struct DevMem {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  DevMem(size_t b, cudaStream_t s);
  ~DevMem();
  DevMem(const DevMem&) = delete;
  DevMem& operator=(const DevMem&) = delete;
};
using DevPtr = std::shared_ptr<DevMem>;
DevPtr dev_alloc(size_t bytes, cudaStream_t st);

// ------------------------------------------------------------------ bonds

struct Bond {
  std::vector<QN> q;    // sectors, ascending
  std::vector<int> d;   // dimensions (> 0)
  int find(const QN& x) const;
  int total() const;
  int nsec() const { return (int)q.size(); }
};

// A "row group" list: the bra-side index of an environment or of a local
// tensor.  For ordinary tensors it is the bra bond; for the two-site step it
// is the fused pair (left sector, sigma_1).
struct RowGroups {
  std::vector<QN> q;
  std::vector<int> d;
  std::vector<int> sa, sig;  // origin: bond sector and local state (sig = -1 if plain)
  static RowGroups from_bond(const Bond& b);
  static RowGroups fused(const Bond& b);   // all (sector, sigma) pairs
  int n() const { return (int)q.size(); }
};

// ------------------------------------------------------------------ site tensor

// Blocks (row group r, sigma) -> right sector; block is rows(r) x d(right).
struct SiteT {
  struct Blk {
    int r, sig, sb, rows, cols;
    size_t off;   // element offset (complex elements)
  };
  std::vector<Blk> blocks;
  std::vector<int> index;  // [r*4 + sig] -> block id or -1
  size_t size = 0;         // complex elements
  DevPtr data;             // double2
  // float2 copy for the mixed-precision contractions, made on first use and
  // dropped whenever `data` is written in place
  mutable DevPtr data32;
  int block_of(int r, int sig) const { return index[(size_t)r * 4 + sig]; }
  double2* ptr(int b) const { return (double2*)data->p + blocks[b].off; }
};
SiteT make_site(const RowGroups& rows, const Bond& right, cudaStream_t st, bool zero);

struct MPSd {
  int L = 0;
  QN tot;
  std::vector<Bond> bonds;    // L+1
  std::vector<SiteT> sites;   // L, left index = plain row groups of bonds[i]
  // sites 1..L-1 are right-canonical (sum_s A^s A^s+ = 1 on their left bond):
  // set by the routines that produce that gauge (fits, compression,
  // right_canonicalize, determinants), cleared by anything else
  bool rcanon = false;
};

// ------------------------------------------------------------------ MPO

struct WElem {
  int win, wout, sig, sigp;   // W[w_in, w_out] maps local state sigp -> sig
  double v;
};

struct MPOBond {
  std::vector<QN> gq;          // channel group charges, ascending
  std::vector<int> gsize;      // channels per group
  std::vector<int> ch_group;   // channel -> group
  std::vector<int> ch_local;   // channel -> index inside its group
  int nch() const { return (int)ch_group.size(); }
  int find(const QN& x) const;
};

// Sparse application tables for one site: for each (sigma, sigma', g_out)
// a CSR over w_out listing (w_in, value) ("left" direction), and for each
// (sigma, sigma', g_in) a CSR over w_in listing (w_out, value) ("right").
struct WTable {
  int sig, sigp, g_out, g_in;
  int rows;         // rows of the CSR (W_gout for left, W_gin for right)
  int rowptr_off;   // offset into rowptr array
  int nnz;          // non-zero entries of the table
};

struct MPOd {
  int L = 0;
  bool identity = false;
  std::vector<MPOBond> bonds;                 // L+1
  std::vector<std::vector<WElem>> W;          // per site
  // device tables
  std::vector<std::vector<WTable>> tab_left, tab_right;
  std::vector<std::map<std::array<int, 3>, int>> tab_left_idx, tab_right_idx;
  // the same lookups as flat arrays: [(sig*4 + sigp) * ngroups + g] -> table or -1
  std::vector<std::vector<int>> tab_left_flat, tab_right_flat;
  DevPtr rowptr, ent_w, ent_v, ent_vf;        // int, int, double, float
  int64_t n_elem = 0;
};

// Host construction (mpo_build.cpp)
MPOd build_qc_mpo(const double* h, const double* eri, int L, double e0);
MPOd build_identity_mpo(int L);
MPOd build_rdm_mpo(int L);          // channels {I, c+_{i s}: i < k}; see rdm code
void upload_mpo(MPOd& m, cudaStream_t st);
// Fiedler ordering of the orbitals (ordering.cpp): perm[k] = orbital at position k
void fiedler_order(const double* h, const double* eri, int L, int* perm);

}  // namespace tdmps
