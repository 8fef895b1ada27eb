// Overlap <bra|ket> that allocates no device memory.
//
// Same contraction as tdmps_overlap (the chain of transfer steps
// E_{i+1} = sum_s B_i^s^H E_i A_i^s, FP64), but every environment and
// intermediate block lives in one file-scope device array instead of
// stream-ordered allocations, and the task lists go through the context's
// staging ring, which tdmps_create allocated up front.  Meant for callers
// that must not allocate device memory while they run: an application whose
// caching allocator has to remain the only owner of device memory, or a loop
// with a fixed device-memory budget where an allocation's latency or failure
// is not acceptable.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "engine.hpp"

namespace tdmps {
namespace {

constexpr size_t kScratchElems = TDMPS_NOALLOC_SCRATCH_BYTES / sizeof(double2);

// Shared by every call on a device and kept until the process exits; each
// call overwrites what it uses.
static __device__ __align__(256) double2 g_overlap_scratch[kScratchElems];

std::mutex g_mu;
double2* g_scratch_ptr[128] = {nullptr};

// Device address of the scratch array on the context's device, which must be
// the current device.  The first call on a device resolves it with
// cudaGetSymbolAddress (the host-side name of a __device__ array is not a
// device address).
double2* scratch_for_device(const Context& c) {
  int dev = 0;
  TD_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev != c.device)
    throw Error(TDMPS_ERR_INVALID_ARG, "the context's device is not the current device");
  if (dev < 0 || dev >= 128) throw Error(TDMPS_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_overlap_scratch);
    if (e != cudaSuccess)
      throw Error(TDMPS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = (double2*)p;
  }
  return g_scratch_ptr[dev];
}

// bytes a task list takes in the pre-allocated staging ring; a list larger
// than one ring segment would need a dedicated buffer and is rejected
size_t ring_bytes(size_t bytes) { return (bytes + 255) & ~(size_t)255; }

struct Blocks {   // per-sector dense blocks of one environment E[b][b']
  std::vector<size_t> off;   // element offset per bra sector (SIZE_MAX if absent)
  size_t size = 0;
};

}  // namespace

cplx overlap_noalloc(Context& c, const MPSd& bra, const MPSd& ket) {
  if (bra.L != ket.L) throw Error(TDMPS_ERR_INVALID_ARG, "MPS lengths differ");
  if (bra.tot != ket.tot) throw Error(TDMPS_ERR_SECTOR, "MPS quantum numbers (N, 2Sz) differ");
  double2* base = scratch_for_device(c);
  const int L = bra.L;
  auto env_layout = [&](int k, Blocks& b) {
    b.off.assign(bra.bonds[k].nsec(), SIZE_MAX);
    b.size = 0;
    for (int s = 0; s < bra.bonds[k].nsec(); ++s) {
      int sk = ket.bonds[k].find(bra.bonds[k].q[s]);
      if (sk < 0) continue;
      b.off[s] = b.size;
      b.size += (size_t)bra.bonds[k].d[s] * ket.bonds[k].d[sk];
    }
  };
  // Plan every launch on the host first: the scratch layout of each site and
  // the packed task lists.  A pair that does not fit is rejected here, before
  // anything is enqueued on the GPU.
  struct Launch { std::vector<char> pack; size_t o_terms, o_tiles; int ntask, ntile; };
  std::vector<Launch> plan;
  Blocks cur, nxt;
  env_layout(0, cur);
  if (cur.size != 1) throw Error(TDMPS_ERR_SECTOR, "left boundary bond must be one-dimensional");
  // environments alternate between the front and the back of the scratch;
  // the intermediate sits between them
  bool cur_front = true;
  double2* Ecur = base;
  double2* Efirst = base;
  const double2 one = make_double2(1.0, 0.0);
  for (int i = 0; i < L; ++i) {
    const SiteT& A = ket.sites[i];
    const SiteT& B = bra.sites[i];
    env_layout(i + 1, nxt);
    // intermediate X(sa, s) = E(sa) A(sa', s): bra rows of sa, ket columns of sb'
    std::vector<size_t> xoff(A.blocks.size(), SIZE_MAX);
    size_t xsize = 0;
    for (int kb = 0; kb < (int)A.blocks.size(); ++kb) {
      const SiteT::Blk& ab = A.blocks[kb];
      int sb_bra = bra.bonds[i].find(ket.bonds[i].q[ab.r]);
      if (sb_bra < 0 || cur.off[sb_bra] == SIZE_MAX) continue;
      xoff[kb] = xsize;
      xsize += (size_t)bra.bonds[i].d[sb_bra] * ab.cols;
    }
    if (cur.size + xsize + nxt.size > kScratchElems)
      throw Error(TDMPS_ERR_INVALID_ARG,
                  "overlap needs more than the fixed scratch of the no-allocation entry point");
    double2* X = cur_front ? base + cur.size : base + nxt.size;
    double2* Enext = cur_front ? base + (kScratchElems - nxt.size) : base;
    std::vector<GemmTask> tasks;
    std::vector<GemmTerm> terms;
    auto add_task = [&](double2* C, int M, int N, int opA, int opB) {
      GemmTask t{};
      t.C = C;
      t.alpha = one;
      t.M = M; t.N = N; t.ldc = N;
      t.opA = opA; t.opB = opB;
      t.term_begin = t.term_end = (int)terms.size();
      tasks.push_back(t);
    };
    auto add_term = [&](const double2* Ap, int lda, const double2* Bp, int ldb, int K) {
      terms.push_back({Ap, Bp, K, lda, ldb, 0, one, nullptr, make_float2(1.f, 0.f)});
      tasks.back().term_end = (int)terms.size();
    };
    // X = E A
    for (int kb = 0; kb < (int)A.blocks.size(); ++kb) {
      if (xoff[kb] == SIZE_MAX) continue;
      const SiteT::Blk& ab = A.blocks[kb];
      int sb_bra = bra.bonds[i].find(ket.bonds[i].q[ab.r]);
      int rows = bra.bonds[i].d[sb_bra];
      add_task(X + xoff[kb], rows, ab.cols, OP_N, OP_N);
      add_term(Ecur + cur.off[sb_bra], ab.rows, A.ptr(kb), ab.cols, ab.rows);
    }
    // E_next(sb) = sum_{(sa, s) -> sb} B(sa, s)^H X(sa, s)
    for (int s = 0; s < bra.bonds[i + 1].nsec(); ++s) {
      if (nxt.off[s] == SIZE_MAX) continue;
      int sk = ket.bonds[i + 1].find(bra.bonds[i + 1].q[s]);
      add_task(Enext + nxt.off[s], bra.bonds[i + 1].d[s], ket.bonds[i + 1].d[sk], OP_C, OP_N);
      for (int bb = 0; bb < (int)B.blocks.size(); ++bb) {
        const SiteT::Blk& blk = B.blocks[bb];
        if (blk.sb != s) continue;
        int ks = ket.bonds[i].find(bra.bonds[i].q[blk.r]);
        if (ks < 0) continue;
        int kb = A.block_of(ks, blk.sig);
        if (kb < 0 || xoff[kb] == SIZE_MAX) continue;
        add_term(B.ptr(bb), blk.cols, X + xoff[kb], A.blocks[kb].cols, blk.rows);
      }
    }
    // two launches: X first, then E_next (separate task lists)
    size_t nx = 0;
    for (size_t t = 0; t < tasks.size(); ++t)
      if (tasks[t].opA == OP_N) ++nx;
    for (int phase = 0; phase < 2; ++phase) {
      std::vector<GemmTask> tk;
      std::vector<int> tile_task;
      size_t lo = phase == 0 ? 0 : nx, hi = phase == 0 ? nx : tasks.size();
      for (size_t t = lo; t < hi; ++t) {
        GemmTask g = tasks[t];
        if (g.M <= 0 || g.N <= 0) continue;
        g.tiles_m = (g.M + 31) / 32;
        g.splits = 1;
        int tn = (g.N + 31) / 32;
        g.tile_base = (int)tile_task.size();
        int id = (int)tk.size();
        tk.push_back(g);
        for (int q = 0; q < g.tiles_m * tn; ++q) tile_task.push_back(id);
      }
      if (tile_task.empty()) continue;
      Launch ln;
      ln.o_terms = ring_bytes(tk.size() * sizeof(GemmTask));
      ln.o_tiles = ln.o_terms + ring_bytes(terms.size() * sizeof(GemmTerm));
      ln.pack.resize(ln.o_tiles + tile_task.size() * sizeof(int));
      std::memcpy(ln.pack.data(), tk.data(), tk.size() * sizeof(GemmTask));
      std::memcpy(ln.pack.data() + ln.o_terms, terms.data(), terms.size() * sizeof(GemmTerm));
      std::memcpy(ln.pack.data() + ln.o_tiles, tile_task.data(), tile_task.size() * sizeof(int));
      // a list larger than one ring segment would need a dedicated buffer
      if (ring_bytes(ln.pack.size()) > c.seg_cap)
        throw Error(TDMPS_ERR_INVALID_ARG, "task list exceeds the staging ring");
      ln.ntask = (int)tk.size();
      ln.ntile = (int)tile_task.size();
      plan.push_back(std::move(ln));
    }
    Ecur = Enext;
    cur_front = !cur_front;
    cur = nxt;
  }
  // Enqueue: the unit left boundary, then every launch, each with one staged
  // copy (the ring reuses a segment once the launches that read it are
  // enqueued).
  TD_CHECK_CUDA(cudaMemcpyAsync(Efirst, c.stage(&one, sizeof(one)), sizeof(double2),
                                cudaMemcpyDeviceToDevice, c.st));
  for (const Launch& ln : plan) {
    const char* p = (const char*)c.stage(ln.pack.data(), ln.pack.size());
    launch_gemm((const GemmTask*)p, ln.ntask, (const GemmTerm*)(p + ln.o_terms),
                (const int*)(p + ln.o_tiles), ln.ntile, c.st);
    TD_CHECK_CUDA(cudaGetLastError());
  }
  double2 h = make_double2(0.0, 0.0);
  if (cur.size == 1)
    TD_CHECK_CUDA(cudaMemcpyAsync(&h, Ecur, sizeof(double2), cudaMemcpyDeviceToHost, c.st));
  c.sync();
  return cplx(h.x, h.y);
}

}  // namespace tdmps
