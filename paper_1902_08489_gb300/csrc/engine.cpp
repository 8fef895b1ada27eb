// Host engine: block-sparse planners and the paper's algorithms.
//
// Environment and local-tensor contractions (paper Sec. 2.2.1, "Operations
// on MPS"): the local solution of Eq. (add_min) at site i in the
// mixed-canonical gauge is
//     C[a, s, b] = sum L[a, w, a'] W[w, w', s, s'] A[a', s', b'] R[b, w', b'],
// evaluated as three stages on symmetry blocks:
//   L-stage  X[a][w][s'][b'] = L[a][w][a'] A[a'][s'][b']        (block GEMM)
//   W-stage  Y[a][s][w'][b'] = sum W[w,w',s,s'] X[a][w][s'][b']  (sparse)
//   R-stage  C[a][s][b]      = sum_{w',b'} Y[a][s][w'][b'] R[b][w'][b']
// and the environment updates reuse the first two stages
//   L_new[b][w'][b'] = sum_{a,s} conj(C[a][s][b]) Y[a][s][w'][b'].
#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <thread>

#include "engine.hpp"

namespace tdmps {

// ------------------------------------------------------------------ memory, bonds

DevMem::DevMem(size_t b, cudaStream_t s) : bytes(b), st(s) {
  if (b == 0) return;
  cudaError_t e = cudaMallocAsync(&p, b, s);
  if (e != cudaSuccess) {
    p = nullptr;
    throw Error(e == cudaErrorMemoryAllocation ? TDMPS_ERR_OOM : TDMPS_ERR_CUDA,
                std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  }
}
DevMem::~DevMem() {
  if (p) cudaFreeAsync(p, st);
}
DevPtr dev_alloc(size_t bytes, cudaStream_t st) { return std::make_shared<DevMem>(bytes, st); }

int Bond::find(const QN& x) const {
  auto it = std::lower_bound(q.begin(), q.end(), x);
  if (it == q.end() || *it != x) return -1;
  return (int)(it - q.begin());
}
int Bond::total() const {
  int t = 0;
  for (int v : d) t += v;
  return t;
}
int MPOBond::find(const QN& x) const {
  auto it = std::lower_bound(gq.begin(), gq.end(), x);
  if (it == gq.end() || *it != x) return -1;
  return (int)(it - gq.begin());
}

RowGroups RowGroups::from_bond(const Bond& b) {
  RowGroups r;
  r.q = b.q;
  r.d = b.d;
  for (int i = 0; i < b.nsec(); ++i) { r.sa.push_back(i); r.sig.push_back(-1); }
  return r;
}
RowGroups RowGroups::fused(const Bond& b) {
  RowGroups r;
  for (int i = 0; i < b.nsec(); ++i)
    for (int s = 0; s < 4; ++s) {
      r.q.push_back(b.q[i] + SITE_Q[s]);
      r.d.push_back(b.d[i]);
      r.sa.push_back(i);
      r.sig.push_back(s);
    }
  return r;
}

SiteT make_site(const RowGroups& rows, const Bond& right, cudaStream_t st, bool zero) {
  SiteT t;
  t.index.assign((size_t)rows.n() * 4, -1);
  for (int r = 0; r < rows.n(); ++r)
    for (int s = 0; s < 4; ++s) {
      int sb = right.find(rows.q[r] + SITE_Q[s]);
      if (sb < 0) continue;
      t.index[(size_t)r * 4 + s] = (int)t.blocks.size();
      t.blocks.push_back({r, s, sb, rows.d[r], right.d[sb], t.size});
      t.size += (size_t)rows.d[r] * right.d[sb];
    }
  t.data = dev_alloc(std::max<size_t>(t.size, 1) * sizeof(double2), st);
  if (zero) launch_zero((double2*)t.data->p, t.size, st);
  return t;
}

void Inter::alloc(cudaStream_t st, bool zero) {
  data = dev_alloc(std::max<size_t>(size, 1) * esz(), st);
  if (zero) TD_CHECK_CUDA(cudaMemsetAsync(data->p, 0, size * esz(), st));
}

// ------------------------------------------------------------------ context

Context::Context(cudaStream_t s, int prec, size_t ring_bytes) : st(s), precision(prec) {
  seg_cap = ((ring_bytes / RING_SEGS) + 255) & ~(size_t)255;
  ring_cap = seg_cap * RING_SEGS;
  for (int k = 0; k < RING_SEGS; ++k)
    TD_CHECK_CUDA(cudaEventCreateWithFlags(&seg_ev[k], cudaEventDisableTiming));
  TD_CHECK_CUDA(cudaGetDevice(&device));
  TD_CHECK_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device));
  TD_CHECK_CUDA(cudaMallocHost((void**)&h_ring, ring_cap));
  TD_CHECK_CUDA(cudaMalloc((void**)&d_ring, ring_cap));
  status = dev_alloc(64, st);
  TD_CHECK_CUDA(cudaMemsetAsync(status->p, 0, 64, st));
}

Context::~Context() {
  aux.reset();
  workers.clear();
  cudaStreamSynchronize(st);
  for (auto& p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (auto e : event_pool) cudaEventDestroy(e);
  ident.reset();
  rdm.reset();
  status.reset();
  cudaStreamSynchronize(st);
  if (h_ring) cudaFreeHost(h_ring);
  if (d_ring) cudaFree(d_ring);
  for (int k = 0; k < RING_SEGS; ++k)
    if (seg_ev[k]) cudaEventDestroy(seg_ev[k]);
}

const void* Context::stage(const void* src, size_t bytes) {
  size_t need = (bytes + 255) & ~(size_t)255;
  if (need > seg_cap) {
    // oversize: dedicated buffer released after the stream passes it
    DevPtr b = dev_alloc(need, st);
    TD_CHECK_CUDA(cudaMemcpyAsync(b->p, src, bytes, cudaMemcpyHostToDevice, st));
    wait_stream();
    // its stream-ordered free is enqueued when the last holder lets go, so
    // keeping it here until the context's next synchronisation is enough
    oversize.push_back(b);
    return b->p;
  }
  if (ring_off - (size_t)cur_seg * seg_cap + need > seg_cap) {
    // leave the current segment (all its consumers are enqueued by now)
    TD_CHECK_CUDA(cudaEventRecord(seg_ev[cur_seg], st));
    seg_live[cur_seg] = true;
    const int next = (cur_seg + 1) % RING_SEGS;
    if (seg_live[next]) wait_event(seg_ev[next]);
    cur_seg = next;
    ring_off = (size_t)next * seg_cap;
  }
  std::memcpy(h_ring + ring_off, src, bytes);
  TD_CHECK_CUDA(cudaMemcpyAsync(d_ring + ring_off, h_ring + ring_off, bytes,
                                cudaMemcpyHostToDevice, st));
  const void* out = d_ring + ring_off;
  ring_off += need;
  return out;
}

// timing events come from a pool: creating an event costs more host time
// than recording it, and every launch of a timed region records two
cudaEvent_t Context::take_event() {
  if (!event_pool.empty()) {
    cudaEvent_t e = event_pool.back();
    event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  TD_CHECK_CUDA(cudaEventCreate(&e));
  return e;
}

void Context::kbegin(int kind, cudaEvent_t* a) {
  (void)kind;
  *a = nullptr;
  if (!stats) return;
  const auto now = std::chrono::steady_clock::now();
  if (host_mark_valid) {
    kstat[TDMPS_KSTAT_HOST_PLAN].launches += 1;
    kstat[TDMPS_KSTAT_HOST_PLAN].ms += std::chrono::duration<double, std::milli>(now - host_mark).count();
  }
  launch_start = now;
  *a = take_event();
  TD_CHECK_CUDA(cudaEventRecord(*a, st));
}

void Context::kend(int kind, cudaEvent_t a, double flops, double bytes) {
  TD_CHECK_CUDA(cudaGetLastError());
  if (!stats) return;
  cudaEvent_t b = take_event();
  TD_CHECK_CUDA(cudaEventRecord(b, st));
  pending.push_back({kind, a, b});
  kstat[kind].launches += 1;
  kstat[kind].flops += flops;
  kstat[kind].bytes += bytes;
  host_mark = std::chrono::steady_clock::now();
  host_mark_valid = true;
  kstat[TDMPS_KSTAT_HOST_LAUNCH].launches += 1;
  kstat[TDMPS_KSTAT_HOST_LAUNCH].ms +=
      std::chrono::duration<double, std::milli>(host_mark - launch_start).count();
}

void Context::collect_stats() {
  TD_CHECK_CUDA(cudaStreamSynchronize(st));
  for (auto& p : pending) {
    float ms = 0.f;
    TD_CHECK_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
    kstat[p.kind].ms += ms;
    event_pool.push_back(p.a);
    event_pool.push_back(p.b);
  }
  pending.clear();
}

void Context::wait_stream() {
  if (!stats) {
    TD_CHECK_CUDA(cudaStreamSynchronize(st));
    return;
  }
  const auto t0 = std::chrono::steady_clock::now();
  TD_CHECK_CUDA(cudaStreamSynchronize(st));
  kstat[TDMPS_KSTAT_HOST_SYNC].launches += 1;
  kstat[TDMPS_KSTAT_HOST_SYNC].ms +=
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

void Context::wait_event(cudaEvent_t e) {
  if (!stats) {
    TD_CHECK_CUDA(cudaEventSynchronize(e));
    return;
  }
  const auto t0 = std::chrono::steady_clock::now();
  TD_CHECK_CUDA(cudaEventSynchronize(e));
  kstat[TDMPS_KSTAT_HOST_SYNC].launches += 1;
  kstat[TDMPS_KSTAT_HOST_SYNC].ms +=
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

void Context::sync() {
  wait_stream();
  oversize.clear();
  check_device_errors();
}

// Error words written by kernels whose bounded waits ran out (read after a
// stream synchronisation; sticky until reported).
void Context::check_device_errors() {
  int h[16];
  TD_CHECK_CUDA(cudaMemcpyAsync(h, status->p, sizeof(h), cudaMemcpyDeviceToHost, st));
  TD_CHECK_CUDA(cudaStreamSynchronize(st));
  if (h[8]) {
    TD_CHECK_CUDA(cudaMemsetAsync((int*)status->p + 8, 0, sizeof(int), st));
    throw Error(TDMPS_ERR_NUMERIC, "a tensor-core barrier wait timed out");
  }
}

const MPOd& Context::identity_mpo(int L) {
  if (!ident || ident->L != L) {
    ident.reset(new MPOd(build_identity_mpo(L)));
    upload_mpo_tables(*ident, *this);
  }
  return *ident;
}

const MPOd& Context::rdm_mpo(int L) {
  if (!rdm || rdm->L != L) {
    rdm.reset(new MPOd(build_rdm_mpo(L)));
    upload_mpo_tables(*rdm, *this);
  }
  return *rdm;
}

// ------------------------------------------------------------------ MPO tables

void upload_mpo_tables(MPOd& m, Context& c) {
  std::vector<int> rowptr, ent_w;
  std::vector<double> ent_v;
  m.tab_left.assign(m.L, {});
  m.tab_right.assign(m.L, {});
  m.tab_left_idx.assign(m.L, {});
  m.tab_right_idx.assign(m.L, {});
  m.tab_left_flat.assign(m.L, {});
  m.tab_right_flat.assign(m.L, {});
  for (int i = 0; i < m.L; ++i) {
    const MPOBond& bi = m.bonds[i];
    const MPOBond& bo = m.bonds[i + 1];
    // left: key (sig, sigp, g_out) rows over w_out
    std::map<std::array<int, 3>, std::vector<const WElem*>> L, R;
    for (const WElem& e : m.W[i]) {
      L[{e.sig, e.sigp, bo.ch_group[e.wout]}].push_back(&e);
      R[{e.sig, e.sigp, bi.ch_group[e.win]}].push_back(&e);
    }
    for (auto& kv : L) {
      int gout = kv.first[2];
      int rows = bo.gsize[gout];
      int gin = bi.ch_group[kv.second[0]->win];
      std::vector<std::vector<std::pair<int, double>>> perrow(rows);
      for (auto* e : kv.second) {
        if (bi.ch_group[e->win] != gin) throw Error(TDMPS_ERR_SECTOR, "MPO charge inconsistency");
        perrow[bo.ch_local[e->wout]].push_back({bi.ch_local[e->win], e->v});
      }
      WTable t{kv.first[0], kv.first[1], gout, gin, rows, (int)rowptr.size(), 0};
      const int first = (int)ent_w.size();
      for (int r = 0; r < rows; ++r) {
        rowptr.push_back((int)ent_w.size());
        for (auto& pv : perrow[r]) { ent_w.push_back(pv.first); ent_v.push_back(pv.second); }
      }
      rowptr.push_back((int)ent_w.size());
      t.nnz = (int)ent_w.size() - first;
      m.tab_left_idx[i][kv.first] = (int)m.tab_left[i].size();
      m.tab_left[i].push_back(t);
    }
    for (auto& kv : R) {
      int gin = kv.first[2];
      int rows = bi.gsize[gin];
      int gout = bo.ch_group[kv.second[0]->wout];
      std::vector<std::vector<std::pair<int, double>>> perrow(rows);
      for (auto* e : kv.second) {
        if (bo.ch_group[e->wout] != gout) throw Error(TDMPS_ERR_SECTOR, "MPO charge inconsistency");
        perrow[bi.ch_local[e->win]].push_back({bo.ch_local[e->wout], e->v});
      }
      WTable t{kv.first[0], kv.first[1], gout, gin, rows, (int)rowptr.size(), 0};
      const int first = (int)ent_w.size();
      for (int r = 0; r < rows; ++r) {
        rowptr.push_back((int)ent_w.size());
        for (auto& pv : perrow[r]) { ent_w.push_back(pv.first); ent_v.push_back(pv.second); }
      }
      rowptr.push_back((int)ent_w.size());
      t.nnz = (int)ent_w.size() - first;
      m.tab_right_idx[i][kv.first] = (int)m.tab_right[i].size();
      m.tab_right[i].push_back(t);
    }
    const int ngo = (int)bo.gq.size(), ngi = (int)bi.gq.size();
    m.tab_left_flat[i].assign((size_t)16 * ngo, -1);
    m.tab_right_flat[i].assign((size_t)16 * ngi, -1);
    for (auto& kv : m.tab_left_idx[i])
      m.tab_left_flat[i][(size_t)(kv.first[0] * 4 + kv.first[1]) * ngo + kv.first[2]] = kv.second;
    for (auto& kv : m.tab_right_idx[i])
      m.tab_right_flat[i][(size_t)(kv.first[0] * 4 + kv.first[1]) * ngi + kv.first[2]] = kv.second;
  }
  m.rowptr = dev_alloc(std::max<size_t>(rowptr.size(), 1) * sizeof(int), c.st);
  m.ent_w = dev_alloc(std::max<size_t>(ent_w.size(), 1) * sizeof(int), c.st);
  m.ent_v = dev_alloc(std::max<size_t>(ent_v.size(), 1) * sizeof(double), c.st);
  m.ent_vf = dev_alloc(std::max<size_t>(ent_v.size(), 1) * sizeof(float), c.st);
  std::vector<float> ent_vf(ent_v.begin(), ent_v.end());
  if (!rowptr.empty())
    TD_CHECK_CUDA(cudaMemcpyAsync(m.rowptr->p, rowptr.data(), rowptr.size() * sizeof(int),
                                  cudaMemcpyHostToDevice, c.st));
  if (!ent_w.empty()) {
    TD_CHECK_CUDA(cudaMemcpyAsync(m.ent_w->p, ent_w.data(), ent_w.size() * sizeof(int),
                                  cudaMemcpyHostToDevice, c.st));
    TD_CHECK_CUDA(cudaMemcpyAsync(m.ent_v->p, ent_v.data(), ent_v.size() * sizeof(double),
                                  cudaMemcpyHostToDevice, c.st));
    TD_CHECK_CUDA(cudaMemcpyAsync(m.ent_vf->p, ent_vf.data(), ent_vf.size() * sizeof(float),
                                  cudaMemcpyHostToDevice, c.st));
  }
  // host vectors must outlive the async copies
  c.wait_stream();
}

// ------------------------------------------------------------------ batches

namespace {

// One grouped GEMM launch.  FP64 contexts (and every gauge-move GEMM) use
// the FP64 kernel; mixed-precision contexts use the tcgen05 kernel, which
// reads complex double or complex float operands and writes either.
struct GemmBatch {
  Context& c;
  bool fp64;
  std::vector<GemmTask> tasks;
  std::vector<GemmTerm> terms;
  std::vector<GemmSeg> segs;
  std::vector<SegOps> segops;
  double flops = 0.0, bytes = 0.0;
  // a segmented task of an FP64 batch, expanded into one plain task per
  // segment once its terms are known (the FP64 kernel has no segments)
  struct PendSeg {
    bool live = false;
    GemmSeg s;
    int other, tc, opA, ta, opB, tb;
    bool beta;
    cplx alpha;
    struct T { const void* shared; int ld; SegOps so; int K; cplx scale; const double2* sp; };
    std::vector<T> terms;
  } pend;
  explicit GemmBatch(Context& ctx, bool force_fp64 = false)
      : c(ctx), fp64(force_fp64 || ctx.precision == TDMPS_FP64) {}
  // A task whose rows (dim 0) or columns (dim 1) are n output blocks of the
  // given sizes (GemmSeg); `other` is the extent of the other dimension.
  void task_seg(int dim, int n, void* const* Cs, const int* ldcs, const int* sizes, int other,
                int tc, int opA, int ta, int opB, int tb, bool beta, cplx alpha) {
    flush();
    if (n < 1 || n > 4) throw Error(TDMPS_ERR_INVALID_ARG, "a GEMM task holds 1 to 4 segments");
    GemmSeg s{};
    s.dim = dim;
    s.n = n;
    for (int i = 0; i < n; ++i) {
      s.off[i + 1] = s.off[i] + sizes[i];
      s.C[i] = Cs[i];
      s.ldc[i] = ldcs[i];
    }
    for (int i = n; i < 4; ++i) s.off[i + 1] = s.off[i];
    if (fp64) {
      pend.live = true;
      pend.s = s;
      pend.other = other; pend.tc = tc; pend.opA = opA; pend.ta = ta; pend.opB = opB; pend.tb = tb;
      pend.beta = beta; pend.alpha = alpha;
      pend.terms.clear();
      return;
    }
    const int total = s.off[n];
    task(Cs[0], tc, dim == 0 ? total : other, dim == 0 ? other : total, ldcs[0], opA, ta, opB, tb,
         beta, alpha);
    tasks.back().seg1 = (int)segs.size() + 1;
    segs.push_back(s);
  }
  // One term of the current segmented task: the shared operand (B for row
  // segments, A for column segments) and one block per segment (null: none).
  void term_seg(const void* shared, int ld_shared, const void* const* segp, const int* segld,
                int K, cplx scale = 1.0, const double2* scale_ptr = nullptr) {
    if (K <= 0) return;
    SegOps so{};
    const void* any = nullptr;
    const GemmSeg& s = pend.live ? pend.s : segs[tasks.back().seg1 - 1];
    for (int i = 0; i < s.n; ++i) {
      so.p[i] = segp[i];
      so.ld[i] = segld[i];
      if (segp[i] && !any) any = segp[i];
    }
    if (!any) return;
    if (pend.live) {
      pend.terms.push_back({shared, ld_shared, so, K, scale, scale_ptr});
      return;
    }
    GemmTask& t = tasks.back();
    GemmTerm g{};
    if (s.dim == 0) { g.A = any; g.B = shared; g.ldb = ld_shared; }
    else { g.A = shared; g.lda = ld_shared; g.B = any; }
    g.K = K;
    g.pad = (int)segops.size();
    g.scale = make_double2(scale.real(), scale.imag());
    g.scale_ptr = scale_ptr;
    g.fscale = make_float2((float)scale.real(), (float)scale.imag());
    segops.push_back(so);
    terms.push_back(g);
    t.term_end = (int)terms.size();
    const int other = s.dim == 0 ? t.N : t.M;
    double live = 0.0;
    for (int i = 0; i < s.n; ++i)
      if (segp[i]) live += s.off[i + 1] - s.off[i];
    flops += 8.0 * live * other * K;
    bytes += 8.0 * (live * K + (double)other * K);
  }
  void flush() {
    if (!pend.live) return;
    pend.live = false;
    const GemmSeg& s = pend.s;
    for (int i = 0; i < s.n; ++i) {
      const int sz = s.off[i + 1] - s.off[i];
      if (sz <= 0) continue;
      task(s.C[i], pend.tc, s.dim == 0 ? sz : pend.other, s.dim == 0 ? pend.other : sz, s.ldc[i],
           pend.opA, pend.ta, pend.opB, pend.tb, pend.beta, pend.alpha);
      for (const auto& tm : pend.terms) {
        if (!tm.so.p[i]) continue;
        if (s.dim == 0) term(tm.so.p[i], tm.so.ld[i], tm.shared, tm.ld, tm.K, tm.scale, tm.sp);
        else term(tm.shared, tm.ld, tm.so.p[i], tm.so.ld[i], tm.K, tm.scale, tm.sp);
      }
    }
  }
  void task(void* C, int tc, int M, int N, int ldc, int opA, int ta, int opB, int tb, bool beta,
            cplx alpha, const double2* aptr = nullptr, const double2* adiv = nullptr) {
    flush();
    if (fp64 && (ta || tb || tc)) throw Error(TDMPS_ERR_INVALID_ARG, "FP64 GEMM on float data");
    if (!fp64 && (!ta || !tb))
      throw Error(TDMPS_ERR_INVALID_ARG, "tensor-core GEMM operands must be complex float");
    GemmTask t{};
    t.C = C;
    t.alpha_ptr = aptr;
    t.alpha_div = adiv;
    t.alpha = make_double2(alpha.real(), alpha.imag());
    t.M = M; t.N = N; t.ldc = ldc;
    t.opA = opA; t.opB = opB; t.beta = beta ? 1 : 0;
    t.ta = ta; t.tb = tb; t.tc = tc;
    t.term_begin = t.term_end = (int)terms.size();
    tasks.push_back(t);
    bytes += (tc ? 8.0 : 16.0) * M * N * (beta ? 2.0 : 1.0);
  }
  void term(const void* A, int lda, const void* B, int ldb, int K, cplx scale = 1.0,
            const double2* scale_ptr = nullptr) {
    if (K <= 0) return;
    GemmTask& t = tasks.back();
    terms.push_back({A, B, K, lda, ldb, 0, make_double2(scale.real(), scale.imag()), scale_ptr,
                     make_float2((float)scale.real(), (float)scale.imag())});
    t.term_end = (int)terms.size();
    flops += 8.0 * t.M * t.N * K;
    bytes += (t.ta ? 8.0 : 16.0) * t.M * K + (t.tb ? 8.0 : 16.0) * K * t.N;
  }
  // C^T = op(B)^T op(A)^T: the operand modes of the transposed product
  static int op_t(int op) {
    switch (op) {
      case OP_N: return OP_T;
      case OP_T: return OP_N;
      case OP_C: return OP_J;
      default: return OP_C;
    }
  }
  // FP64 tiles skip whole warps of rows past the block edge, so a task whose
  // N is the short side runs transposed (rows <- the short side).
  void orient_fp64() {
    for (auto& t : tasks) {
      if (t.M <= 0 || t.N <= 0 || t.N >= t.M || t.N >= 32) continue;
      for (int e = t.term_begin; e < t.term_end; ++e) {
        std::swap(terms[e].A, terms[e].B);
        std::swap(terms[e].lda, terms[e].ldb);
      }
      const int oa = t.opA;
      t.opA = op_t(t.opB);
      t.opB = op_t(oa);
      std::swap(t.ta, t.tb);
      std::swap(t.M, t.N);
      t.ct = 1;
    }
  }
  // Tensor-core tiles are 128 rows (the MMA M) by up to 64 complex columns
  // (the MMA N rounds to 8 complex), so a task with few rows and many
  // columns runs transposed: its long side fills the 128 TMEM lanes.
  void orient_tc() {
    for (auto& t : tasks) {
      if (t.seg1 || t.M <= 0 || t.N <= 0 || t.M >= tc_tile_m() || t.N <= t.M) continue;
      const long long pad_now = (long long)((t.M + 127) / 128) * 128 * ((t.N + 7) / 8) * 8;
      const long long pad_t = (long long)((t.N + 127) / 128) * 128 * ((t.M + 7) / 8) * 8;
      if (pad_t >= pad_now) continue;
      for (int e = t.term_begin; e < t.term_end; ++e) {
        std::swap(terms[e].A, terms[e].B);
        std::swap(terms[e].lda, terms[e].ldb);
      }
      const int oa = t.opA;
      t.opA = op_t(t.opB);
      t.opB = op_t(oa);
      std::swap(t.ta, t.tb);
      std::swap(t.M, t.N);
      t.ct = 1;
    }
  }
  void run() {
    flush();
    const int bm = fp64 ? 32 : tc_tile_m();
    const int bn = fp64 ? 32 : tc_tile_n();
    if (fp64) orient_fp64(); else orient_tc();
    std::vector<int> tile_task;
    std::vector<GemmTask> tk;
    std::vector<int> split_ids;
    std::vector<TcTile> tc_tiles;
    size_t part_elems = 0;
    // Split-K: long K runs are shared by several CTAs, each of which stores
    // its partial sum in a slice of a scratch buffer; a reduction adds the
    // slices in split order (deterministic).  The chunk count per CTA is chosen so
    // that the launch has about `per_sm` work units per SM (the FP64 pipe
    // and the tensor pipe are per-SM resources; a launch with fewer units
    // than SMs leaves the rest idle), with at least `min_chunks` K chunks
    // per unit to amortise the partial-slice store and its reduction.
    const int kc = fp64 ? 8 : tc_stage_k();
    const int per_sm = fp64 ? 4 : 3, min_chunks = fp64 ? 2 : 4;
    std::vector<long long> stages(tasks.size(), 0);
    long long total = 0;
    for (size_t i = 0; i < tasks.size(); ++i) {
      const GemmTask& t = tasks[i];
      if (t.M <= 0 || t.N <= 0) continue;
      for (int e = t.term_begin; e < t.term_end; ++e) stages[i] += (terms[e].K + kc - 1) / kc;
      total += (long long)((t.M + bm - 1) / bm) * ((t.N + bn - 1) / bn) * std::max(1LL, stages[i]);
    }
    const long long units = (long long)std::max(1, c.n_sm) * per_sm;
    const long long chunk = std::max<long long>(min_chunks, total / units);
    for (size_t i = 0; i < tasks.size(); ++i) {
      GemmTask& t = tasks[i];
      if (t.M <= 0 || t.N <= 0) continue;
      t.tiles_m = (t.M + bm - 1) / bm;
      int tn = (t.N + bn - 1) / bn;
      t.splits = (int)std::min<long long>(64, std::max<long long>(1, stages[i] / chunk));
      t.part = nullptr;
      t.tile_base = (int)tile_task.size();
      int id = (int)tk.size();
      if (!fp64) {
        // host-built tile descriptors: this task's K stages split evenly
        for (int sp = 0; sp < t.splits; ++sp) {
          const int lo = (int)((long long)sp * stages[i] / t.splits);
          const int hi = (int)((long long)(sp + 1) * stages[i] / t.splits);
          int e0 = t.term_begin, k0 = 0, idx = 0;
          while (e0 < t.term_end) {
            const int nk = (terms[e0].K + kc - 1) / kc;
            if (idx + nk <= lo) { idx += nk; ++e0; continue; }
            k0 = (lo - idx) * kc;
            break;
          }
          for (int q = 0; q < t.tiles_m * tn; ++q) {
            TcTile tl;
            tl.task = id;
            tl.m0 = (q % t.tiles_m) * bm;
            tl.n0 = (q / t.tiles_m) * bn;
            tl.ncols = std::min(bn, t.N - tl.n0);
            tl.count = hi - lo;
            tl.e0 = e0;
            tl.k0 = k0;
            tl.split = sp;
            tc_tiles.push_back(tl);
          }
        }
      }
      if (t.splits > 1) {
        split_ids.push_back(id);
        // element offset for now; made a pointer once the buffer exists
        t.part = (void*)(uintptr_t)part_elems;
        part_elems += (size_t)t.splits * t.M * t.N;
      }
      tk.push_back(t);
      for (int q = 0; q < t.tiles_m * tn * t.splits; ++q) tile_task.push_back(id);
    }
    if (tile_task.empty()) return;
    // the reduction of the split tasks in chunks of at most 512 elements (one
    // CTA of 256 threads each, two elements per thread): a few large tasks
    // still spread over every SM, with enough independent slice loads in
    // flight to cover their latency.  Every element is summed by one thread
    // in split order, so the chunking does not change the result.
    constexpr int red_chunk = 512;
    std::vector<int> red;
    for (int id : split_ids) {
      const int mn = tk[id].M * tk[id].N;
      for (int b = 0; b < mn; b += red_chunk) {
        red.push_back(id);
        red.push_back(b);
        red.push_back(std::min(mn, b + red_chunk));
      }
    }
    // partial-sum slices of the split tasks (freed in stream order after use)
    DevPtr part;
    if (part_elems) {
      // one buffer, slices addressed in units of the widest element type
      part = dev_alloc(part_elems * sizeof(double2), c.st);
      for (int id : split_ids) {
        GemmTask& t = tk[id];
        t.part = (char*)part->p + (size_t)(uintptr_t)t.part * sizeof(double2);
      }
    }
    // tasks, terms, the tile map and the split list go to the device in one
    // staged copy
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_terms = al(tk.size() * sizeof(GemmTask));
    const size_t o_split = o_terms + al(terms.size() * sizeof(GemmTerm));
    const size_t o_segs = o_split + al(red.size() * sizeof(int));
    const size_t o_segops = o_segs + al(segs.size() * sizeof(GemmSeg));
    const size_t o_tiles = o_segops + al(segops.size() * sizeof(SegOps));
    const size_t pk_bytes =
        o_tiles + (fp64 ? tile_task.size() * sizeof(int) : tc_tiles.size() * sizeof(TcTile));
    std::vector<char>& pk = c.pack;
    pk.resize(pk_bytes);
    std::memcpy(pk.data(), tk.data(), tk.size() * sizeof(GemmTask));
    if (!terms.empty()) std::memcpy(pk.data() + o_terms, terms.data(), terms.size() * sizeof(GemmTerm));
    if (!red.empty()) std::memcpy(pk.data() + o_split, red.data(), red.size() * sizeof(int));
    if (!segs.empty()) std::memcpy(pk.data() + o_segs, segs.data(), segs.size() * sizeof(GemmSeg));
    if (!segops.empty())
      std::memcpy(pk.data() + o_segops, segops.data(), segops.size() * sizeof(SegOps));
    if (fp64)
      std::memcpy(pk.data() + o_tiles, tile_task.data(), tile_task.size() * sizeof(int));
    else
      std::memcpy(pk.data() + o_tiles, tc_tiles.data(), tc_tiles.size() * sizeof(TcTile));
    const char* base = (const char*)c.stage(pk.data(), pk_bytes);
    const GemmTask* dt = (const GemmTask*)base;
    const GemmTerm* dm = terms.empty() ? nullptr : (const GemmTerm*)(base + o_terms);
    const int* dtt = (const int*)(base + o_tiles);
    cudaEvent_t ev;
    const int kind = fp64 ? TDMPS_KSTAT_GEMM_FP64 : TDMPS_KSTAT_GEMM;
    c.kbegin(kind, &ev);
    if (fp64)
      launch_gemm(dt, (int)tk.size(), dm, dtt, (int)tile_task.size(), c.st);
    else
      launch_gemm_tc(dt, dm, (const TcTile*)(base + o_tiles), (const GemmSeg*)(base + o_segs),
                     (const SegOps*)(base + o_segops), (int)tc_tiles.size(),
                     c.precision == TDMPS_TF32X3 ? 1 : c.precision == TDMPS_BF16 ? 2 : 0,
                     c.n_sm, c.tc_err(), c.st);
    if (!red.empty())
      launch_reduce_splits(dt, (const GemmSeg*)(base + o_segs), (const int*)(base + o_split),
                           (int)(red.size() / 3), fp64 ? 0 : 1, c.st);
    c.kend(kind, ev, flops, bytes);
  }
};

struct WBatch {
  const MPOd* mpo = nullptr;
  std::vector<WTask> tasks;
  int64_t work = 0;
  double flops = 0.0, bytes = 0.0;
  int et = 0;
  void run(Context& c) {
    if (!mpo) return;
    const MPOd& m = *mpo;
    if (tasks.empty() || work == 0) return;
    const WTask* dt = c.stage(tasks);
    cudaEvent_t ev;
    c.kbegin(TDMPS_KSTAT_WSTAGE, &ev);
    launch_wstage(dt, (int)tasks.size(), work, (const int*)m.rowptr->p, (const int*)m.ent_w->p,
                  (const double*)m.ent_v->p, (const float*)m.ent_vf->p, et, c.st);
    c.kend(TDMPS_KSTAT_WSTAGE, ev, flops, bytes);
  }
};

}  // namespace

// ------------------------------------------------------------------ environments

static Env env_left_boundary(Context& c, const MPSd& bra, const MPSd& ket, const MPOd& mpo) {
  if (bra.bonds[0].nsec() != 1 || ket.bonds[0].nsec() != 1)
    throw Error(TDMPS_ERR_SECTOR, "left boundary bond must be one-dimensional");
  Env e;
  e.rows = RowGroups::from_bond(bra.bonds[0]);
  e.mb = &mpo.bonds[0];
  e.ket_copy = ket.bonds[0];
  e.t.add(0, -1, 0, 0, 1, 1, 1);
  e.t.et = c.et();
  e.t.alloc(c.st, false);
  launch_fill_one(e.t.data->p, e.t.et, c.st);
  return e;
}

static Env env_right_boundary(Context& c, const MPSd& bra, const MPSd& ket, const MPOd& mpo) {
  int L = bra.L;
  if (bra.tot != ket.tot) throw Error(TDMPS_ERR_SECTOR, "bra and ket have different (N, 2Sz)");
  if (mpo.bonds[L].nch() != 1) throw Error(TDMPS_ERR_SECTOR, "MPO right boundary must have one channel");
  Env e;
  e.rows = RowGroups::from_bond(bra.bonds[L]);
  e.mb = &mpo.bonds[L];
  e.ket_copy = ket.bonds[L];
  e.t.add(0, -1, 0, 0, 1, 1, 1);
  e.t.et = c.et();
  e.t.alloc(c.st, false);
  launch_fill_one(e.t.data->p, e.t.et, c.st);
  return e;
}

// A site tensor as a GEMM operand: the FP64 blocks in FP64 mode, else an
// FP32 copy made once per tensor (the tensor-core kernels then convert no
// FP64 data per tile -- FP64 conversions run at the FP64 pipe's rate).
static const void* site_operand(Context& c, const SiteT& s, int b, int& et) {
  if (c.precision == TDMPS_FP64) {
    et = 0;
    return s.ptr(b);
  }
  if (!s.data32) {
    s.data32 = dev_alloc(std::max<size_t>(s.size, 1) * sizeof(float2), c.st);
    cudaEvent_t ev;
    c.kbegin(TDMPS_KSTAT_OTHER, &ev);
    launch_to_float((const double2*)s.data->p, (float2*)s.data32->p, s.size, c.st);
    c.kend(TDMPS_KSTAT_OTHER, ev, 0.0, 24.0 * s.size);
  }
  et = 1;
  return (const float2*)s.data32->p + s.blocks[b].off;
}
static int site_et(Context& c) { return c.precision == TDMPS_FP64 ? 0 : 1; }

// ---- stage planners: each appends its work to a batch; callers run one
// launch per stage for all terms of a fit or all pairs of a sandwich.

// Does the bra site have the block (row group rg, local state s)?
static bool bra_has(const SiteT& bra, int rg, int s) {
  return (size_t)rg * 4 + s < bra.index.size() && bra.block_of(rg, s) >= 0;
}

// X[rg][w][s'][b'] = E[rg][w][k] A[k][s'][b']
// In a sandwich (`bra` given, left-to-right), X[rg][g][s'] reaches the bra
// only through the MPO-stage outputs Y[rg][s] whose tables connect s' to s
// and for which the bra has the block (rg, s); X blocks with no such
// consumer are not computed.  With the identity MPO that is s = s'.
static Inter plan_lstage(Context& c, const Env& E, const SiteT& ket, const Bond& ket_right,
                         GemmBatch& gb, const SiteT* bra = nullptr, const MPOd* m = nullptr,
                         int site = 0) {
  auto consumed = [&](const Inter::Blk& eb, int sp) {
    if (!m || m->identity) return bra_has(*bra, eb.rg, sp);
    const MPOBond& bi = m->bonds[site];
    const MPOBond& bo = m->bonds[site + 1];
    const std::vector<int>& flat = m->tab_left_flat[site];
    const int ngy = (int)bo.gq.size();
    for (int s = 0; s < 4; ++s) {
      if (!bra_has(*bra, eb.rg, s)) continue;
      const int g = bo.find(bi.gq[eb.g] + SITE_Q[s] - SITE_Q[sp]);
      if (g >= 0 && flat[(size_t)(s * 4 + sp) * ngy + g] >= 0) return true;
    }
    return false;
  };
  Inter X;
  std::vector<std::pair<int, int>> src;   // (env block, ket block) per X block
  for (int b = 0; b < (int)E.t.blocks.size(); ++b) {
    const Inter::Blk& eb = E.t.blocks[b];
    for (int s = 0; s < 4; ++s) {
      int kb = ket.block_of(eb.k, s);
      if (kb < 0) continue;
      if (bra && !consumed(eb, s)) continue;
      int sb = ket.blocks[kb].sb;
      X.add(eb.rg, s, eb.g, sb, eb.rows, eb.W, ket_right.d[sb]);
      src.push_back({b, kb});
    }
  }
  X.et = E.t.et;
  X.alloc(c.st, false);
  // the X blocks of one environment block (one per local state s') share
  // that block as A: one task whose columns are the s' blocks side by side
  for (int x0 = 0; x0 < (int)X.blocks.size();) {
    int x1 = x0 + 1;
    while (x1 < (int)X.blocks.size() && x1 - x0 < 4 && src[x1].first == src[x0].first) ++x1;
    const Inter::Blk& eb = E.t.blocks[src[x0].first];
    void* Cs[4];
    int ld[4];
    const void* bp[4];
    int bet = 0;
    for (int x = x0; x < x1; ++x) {
      Cs[x - x0] = X.ptr(x);
      ld[x - x0] = X.blocks[x].cols;
      bp[x - x0] = site_operand(c, ket, src[x].second, bet);
    }
    gb.task_seg(1, x1 - x0, Cs, ld, ld, eb.rows * eb.W, X.et, OP_N, E.t.et, OP_N, bet, false, 1.0);
    gb.term_seg(E.t.ptr(src[x0].first), eb.cols, bp, ld, eb.cols);
    x0 = x1;
  }
  return X;
}

// Sparse MPO-tensor stage, either direction.
//   left:  Y[rg][s][w_out][b'] = sum_{s', w_in} W[w_in, w_out, s, s'] X[rg][w_in][s'][b']
//   right: Y[rb][s][w_in][a']  = sum_{s', w_out} W[w_in, w_out, s, s'] X[rb][w_out][s'][a']
// With `bra` given (a left-to-right sandwich), outputs Y[rg][s] for which the
// bra has no block (rg, s) are not computed: no environment term uses them.
static Inter plan_wstage(Context& c, Inter&& X, const MPOd& m, int site, bool left,
                         WBatch& wb, const SiteT* bra = nullptr) {
  if (m.identity) return std::move(X);   // no copy of the block index
  if (bra && !left) throw Error(TDMPS_ERR_INVALID_ARG, "bra filter is left-to-right only");
  if (wb.mpo && wb.mpo != &m) throw Error(TDMPS_ERR_INVALID_ARG, "mixed MPOs in one W batch");
  wb.mpo = &m;
  wb.et = X.et;
  const MPOBond& bi = m.bonds[site];
  const MPOBond& bo = m.bonds[site + 1];
  const MPOBond& bx = left ? bi : bo;   // channels of the input
  const MPOBond& by = left ? bo : bi;   // channels of the output
  // X blocks grouped by (row group, column sector), in that order; a flat
  // table replaces an ordered map (this runs for every launch)
  int nrg = 0, nk = 0;
  for (const auto& b : X.blocks) {
    nrg = std::max(nrg, b.rg + 1);
    nk = std::max(nk, b.k + 1);
  }
  std::vector<std::array<int, 4>> groups((size_t)nrg * nk, std::array<int, 4>{-1, -1, -1, -1});
  for (int x = 0; x < (int)X.blocks.size(); ++x)
    groups[(size_t)X.blocks[x].rg * nk + X.blocks[x].k][X.blocks[x].sig] = x;
  const std::vector<int>& flat = left ? m.tab_left_flat[site] : m.tab_right_flat[site];
  const int ngy = (int)by.gq.size();
  Inter Y;
  struct P { int xs[4]; int tabs[4]; };
  std::vector<P> pend;
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const std::array<int, 4>& grp = groups[gi];
    if (grp[0] < 0 && grp[1] < 0 && grp[2] < 0 && grp[3] < 0) continue;
    const int rg = (int)(gi / nk), kk = (int)(gi % nk);
    for (int s = 0; s < 4; ++s) {
      if (bra && !bra_has(*bra, rg, s)) continue;
      P p;
      int gy = -1, first = -1;
      for (int sp = 0; sp < 4; ++sp) {
        p.xs[sp] = -1;
        p.tabs[sp] = -1;
        int x = grp[sp];
        if (x < 0) continue;
        // charge of the output channel group
        QN qy = left ? bx.gq[X.blocks[x].g] + SITE_Q[s] - SITE_Q[sp]
                     : bx.gq[X.blocks[x].g] - SITE_Q[s] + SITE_Q[sp];
        int g = by.find(qy);
        if (g < 0) continue;
        const int tab = flat[(size_t)(s * 4 + sp) * ngy + g];
        if (tab < 0) continue;
        gy = g;
        p.xs[sp] = x;
        p.tabs[sp] = tab;
        if (first < 0) first = x;
      }
      if (first < 0) continue;
      Y.add(rg, s, gy, kk, X.blocks[first].rows, by.gsize[gy], X.blocks[first].cols);
      pend.push_back(p);
    }
  }
  Y.et = X.et;
  Y.alloc(c.st, false);
  for (int y = 0; y < (int)Y.blocks.size(); ++y) {
    const Inter::Blk& yb = Y.blocks[y];
    WTask t{};
    t.Y = Y.ptr(y);
    t.rows = yb.rows;
    t.wout = yb.W;
    t.cols = yb.cols;
    t.beta = 0;
    t.work_base = wb.work;
    int64_t nnz = 0;
    for (int sp = 0; sp < 4; ++sp) {
      int x = pend[y].xs[sp];
      if (x < 0) { t.X[sp] = nullptr; t.win[sp] = 0; t.csr[sp] = -1; continue; }
      t.X[sp] = X.ptr(x);
      t.win[sp] = X.blocks[x].W;
      const WTable& tb = (left ? m.tab_left[site] : m.tab_right[site])[pend[y].tabs[sp]];
      t.csr[sp] = tb.rowptr_off;
      nnz += tb.nnz;
      wb.bytes += (double)X.esz() * X.blocks[x].rows * X.blocks[x].W * X.blocks[x].cols;
    }
    int64_t n = (int64_t)yb.rows * yb.W * yb.cols;
    if (n >= ((int64_t)1 << 31)) throw Error(TDMPS_ERR_INVALID_ARG, "MPO-stage block too large");
    const int rpi = wstage_rows_per_item();
    wb.work += (int64_t)((yb.rows + rpi - 1) / rpi) * yb.W * yb.cols;
    wb.bytes += (double)Y.esz() * n;
    // one real x complex multiply-add per non-zero W entry, row and column
    wb.flops += 4.0 * (double)nnz * yb.rows * yb.cols;
    wb.tasks.push_back(t);
  }
  return Y;
}

// One term of a local tensor: coef * contraction of (Y, environment).
struct LocalTerm {
  const Inter* Y;
  const Env* E;
  cplx coef;
  const double2* coef_dev;
};

// out[r][s][b] = sum_t coef_t sum_{w', b'} Y_t[r][s][w'][b'] R_t[b][w'][b']
// Environment blocks of one local term grouped by row group (CSR over rg).
struct ByRow {
  std::vector<int> start, list;
  void build(const Inter& E) {
    int n = 0;
    for (const auto& b : E.blocks) n = std::max(n, b.rg + 1);
    start.assign((size_t)n + 1, 0);
    list.resize(E.blocks.size());
    for (const auto& b : E.blocks) start[(size_t)b.rg + 1]++;
    for (size_t i = 1; i < start.size(); ++i) start[i] += start[i - 1];
    std::vector<int> fill(start.begin(), start.end() - 1);
    for (int b = 0; b < (int)E.blocks.size(); ++b) list[fill[E.blocks[b].rg]++] = b;
  }
  int lo(int rg) const { return rg + 1 < (int)start.size() ? start[rg] : 0; }
  int hi(int rg) const { return rg + 1 < (int)start.size() ? start[rg + 1] : 0; }
};

// Output blocks of a site tensor grouped by their right sector (sb) or by
// their row group (r), in groups of at most four (the segments one GEMM task
// holds).  A plain tensor has at most four blocks per group, one per local
// state; a two-site tensor, whose rows are fused (sector, state) pairs, can
// have more, which then form several groups.
static std::vector<std::vector<int>> blocks_by(const SiteT& out, bool by_right) {
  int n = 0;
  for (const auto& b : out.blocks) n = std::max(n, (by_right ? b.sb : b.r) + 1);
  std::vector<std::vector<int>> g((size_t)n);
  for (int o = 0; o < (int)out.blocks.size(); ++o)
    g[(size_t)(by_right ? out.blocks[o].sb : out.blocks[o].r)].push_back(o);
  std::vector<std::vector<int>> out4;
  for (auto& v : g)
    for (size_t i = 0; i < v.size(); i += 4)
      out4.emplace_back(v.begin() + i, v.begin() + std::min(v.size(), i + 4));
  return out4;
}

// The blocks (a, s) -> b of one right sector b share every R block: one
// task whose rows are those blocks stacked (row segments).
static void plan_rstage(const std::vector<LocalTerm>& ts, SiteT& out, GemmBatch& gb) {
  std::vector<ByRow> rby(ts.size());
  for (size_t t = 0; t < ts.size(); ++t) rby[t].build(ts[t].E->t);
  for (const auto& grp : blocks_by(out, true)) {
    if (grp.empty()) continue;
    const int sb = out.blocks[grp[0]].sb, n = (int)grp.size();
    void* Cs[4];
    int ldc[4], rows[4];
    for (int i = 0; i < n; ++i) {
      Cs[i] = out.ptr(grp[i]);
      ldc[i] = out.blocks[grp[i]].cols;
      rows[i] = out.blocks[grp[i]].rows;
    }
    gb.task_seg(0, n, Cs, ldc, rows, out.blocks[grp[0]].cols, 0, OP_N, ts[0].Y->et, OP_T,
                ts[0].E->t.et, false, 1.0);
    for (size_t t = 0; t < ts.size(); ++t) {
      const Inter& R = ts[t].E->t;
      for (int q = rby[t].lo(sb); q < rby[t].hi(sb); ++q) {
        const int rb = rby[t].list[q];
        const Inter::Blk& r = R.blocks[rb];
        const int K = r.W * r.cols;
        const void* ap[4];
        int lda[4];
        for (int i = 0; i < n; ++i) {
          const SiteT::Blk& ob = out.blocks[grp[i]];
          const int y = ts[t].Y->find(ob.r, ob.sig, r.g, r.k);
          ap[i] = y < 0 ? nullptr : ts[t].Y->ptr(y);
          lda[i] = K;
        }
        gb.term_seg(R.ptr(rb), K, ap, lda, K, ts[t].coef, ts[t].coef_dev);
      }
    }
  }
}

// out[a][s][b] = sum_t coef_t sum_{w, a'} L_t[a][w][a'] Zp_t[b][s][w][a']
// The blocks (a, s) of one left sector a share every L block: one task
// whose columns are those blocks side by side (column segments).
static void plan_lcontract(const std::vector<LocalTerm>& ts, SiteT& out, GemmBatch& gb) {
  std::vector<ByRow> lby(ts.size());
  for (size_t t = 0; t < ts.size(); ++t) lby[t].build(ts[t].E->t);
  for (const auto& grp : blocks_by(out, false)) {
    if (grp.empty()) continue;
    const int r0 = out.blocks[grp[0]].r, n = (int)grp.size();
    void* Cs[4];
    int ldc[4];
    for (int i = 0; i < n; ++i) {
      Cs[i] = out.ptr(grp[i]);
      ldc[i] = out.blocks[grp[i]].cols;
    }
    gb.task_seg(1, n, Cs, ldc, ldc, out.blocks[grp[0]].rows, 0, OP_N, ts[0].E->t.et, OP_T,
                ts[0].Y->et, false, 1.0);
    for (size_t t = 0; t < ts.size(); ++t) {
      const Inter& Lt = ts[t].E->t;
      for (int q = lby[t].lo(r0); q < lby[t].hi(r0); ++q) {
        const int lb = lby[t].list[q];
        const Inter::Blk& l = Lt.blocks[lb];
        const int K = l.W * l.cols;
        const void* bp[4];
        int ldb[4];
        for (int i = 0; i < n; ++i) {
          const SiteT::Blk& ob = out.blocks[grp[i]];
          const int z = ts[t].Y->find(ob.sb, ob.sig, l.g, l.k);
          bp[i] = z < 0 ? nullptr : ts[t].Y->ptr(z);
          ldb[i] = K;
        }
        gb.term_seg(Lt.ptr(lb), K, bp, ldb, K, ts[t].coef, ts[t].coef_dev);
      }
    }
  }
}

// L_new[b][w'][b'] = sum_{a, s} conj(C[a][s][b]) Y[a][s][w'][b']
static Env plan_env_left(Context& c, const Inter& Y, const SiteT& bra, const Bond& bra_right,
                         const MPOBond& mb, const Bond& ket_right, GemmBatch& gb) {
  Env e;
  e.rows = RowGroups::from_bond(bra_right);
  e.mb = &mb;
  e.ket_copy = ket_right;
  // Y blocks by (row group, sigma), then the terms of every output block
  // (bra right sector, channel group) grouped in (sector, group) order --
  // counting sorts over flat index ranges instead of ordered maps
  int nrg = 0, ng = 0;
  for (const auto& y : Y.blocks) {
    nrg = std::max(nrg, y.rg + 1);
    ng = std::max(ng, y.g + 1);
  }
  std::vector<int> ystart((size_t)nrg * 4 + 1, 0), ylist(Y.blocks.size());
  for (const auto& y : Y.blocks) ystart[(size_t)y.rg * 4 + y.sig + 1]++;
  for (size_t i = 1; i < ystart.size(); ++i) ystart[i] += ystart[i - 1];
  {
    std::vector<int> fill(ystart.begin(), ystart.end() - 1);
    for (int y = 0; y < (int)Y.blocks.size(); ++y) ylist[fill[(size_t)Y.blocks[y].rg * 4 + Y.blocks[y].sig]++] = y;
  }
  struct T { int bra, y; };
  const size_t nkey = (size_t)bra_right.nsec() * ng;
  std::vector<int> cstart(nkey + 1, 0);
  auto ys_of = [&](const SiteT::Blk& cb, int& lo, int& hi) {
    lo = hi = 0;
    if (cb.r >= nrg) return;
    lo = ystart[(size_t)cb.r * 4 + cb.sig];
    hi = ystart[(size_t)cb.r * 4 + cb.sig + 1];
  };
  for (const auto& cb : bra.blocks) {
    int lo, hi;
    ys_of(cb, lo, hi);
    for (int q = lo; q < hi; ++q) cstart[(size_t)cb.sb * ng + Y.blocks[ylist[q]].g + 1]++;
  }
  for (size_t i = 1; i < cstart.size(); ++i) cstart[i] += cstart[i - 1];
  std::vector<T> terms(cstart[nkey]);
  {
    std::vector<int> fill(cstart.begin(), cstart.end() - 1);
    for (int b = 0; b < (int)bra.blocks.size(); ++b) {
      int lo, hi;
      ys_of(bra.blocks[b], lo, hi);
      for (int q = lo; q < hi; ++q) {
        const int y = ylist[q];
        terms[fill[(size_t)bra.blocks[b].sb * ng + Y.blocks[y].g]++] = {b, y};
      }
    }
  }
  for (size_t key = 0; key < nkey; ++key) {
    if (cstart[key] == cstart[key + 1]) continue;
    const Inter::Blk& y0 = Y.blocks[terms[cstart[key]].y];
    const int sb = (int)(key / ng), g = (int)(key % ng);
    e.t.add(sb, -1, g, y0.k, bra_right.d[sb], y0.W, y0.cols);
  }
  e.t.et = Y.et;
  e.t.alloc(c.st, false);
  int id = 0;
  for (size_t key = 0; key < nkey; ++key) {
    if (cstart[key] == cstart[key + 1]) continue;
    const Inter::Blk& eb = e.t.blocks[id];
    int N = eb.W * eb.cols;
    gb.task(e.t.ptr(id), e.t.et, eb.rows, N, N, OP_C, site_et(c), OP_N, Y.et, false, 1.0);
    for (int q = cstart[key]; q < cstart[key + 1]; ++q) {
      const SiteT::Blk& cb = bra.blocks[terms[q].bra];
      int aet;
      const void* ap = site_operand(c, bra, terms[q].bra, aet);
      gb.term(ap, cb.cols, Y.ptr(terms[q].y), N, cb.rows);
    }
    ++id;
  }
  return e;
}

// Z[rb][w'][s'][a'] = sum_b' R[rb][w'][b'] A[a'][s'][b']
static Inter plan_r1(Context& c, const Env& R, const SiteT& A, const Bond& ket_left,
                     GemmBatch& gb) {
  int nsb = 0;   // (right sector, sigma) -> ket block, flat
  for (const auto& b : A.blocks) nsb = std::max(nsb, b.sb + 1);
  std::vector<int> kby((size_t)nsb * 4, -1);
  for (int b = 0; b < (int)A.blocks.size(); ++b) kby[(size_t)A.blocks[b].sb * 4 + A.blocks[b].sig] = b;
  Inter Z;
  std::vector<std::pair<int, int>> src;
  for (int rb = 0; rb < (int)R.t.blocks.size(); ++rb) {
    const Inter::Blk& r = R.t.blocks[rb];
    if (r.k >= nsb) continue;
    for (int s = 0; s < 4; ++s) {
      const int kb = kby[(size_t)r.k * 4 + s];
      if (kb < 0) continue;
      const SiteT::Blk& ab = A.blocks[kb];
      Z.add(r.rg, s, r.g, ab.r, r.rows, r.W, ket_left.d[ab.r]);
      src.push_back({rb, kb});
    }
  }
  Z.et = R.t.et;
  Z.alloc(c.st, false);
  // the Z blocks of one environment block (one per local state s') share
  // that block as A: one task with the s' blocks as column segments
  for (int z0 = 0; z0 < (int)Z.blocks.size();) {
    int z1 = z0 + 1;
    while (z1 < (int)Z.blocks.size() && z1 - z0 < 4 && src[z1].first == src[z0].first) ++z1;
    const Inter::Blk& r = R.t.blocks[src[z0].first];
    void* Cs[4];
    int ldc[4], ldb[4];
    const void* bp[4];
    int bet = 0;
    for (int z = z0; z < z1; ++z) {
      Cs[z - z0] = Z.ptr(z);
      ldc[z - z0] = Z.blocks[z].cols;
      ldb[z - z0] = r.cols;
      bp[z - z0] = site_operand(c, A, src[z].second, bet);
    }
    gb.task_seg(1, z1 - z0, Cs, ldc, ldc, r.rows * r.W, Z.et, OP_N, R.t.et, OP_T, bet, false, 1.0);
    gb.term_seg(R.t.ptr(src[z0].first), r.cols, bp, ldb, r.cols);
    z0 = z1;
  }
  return Z;
}

// R_new[a][w][a'] = sum_{s, b} conj(C[a][s][b]) Zp[b][s][w][a']
static Env plan_env_right(Context& c, const Inter& Zp, const SiteT& bra, const Bond& bra_left,
                          const MPOBond& mb, const Bond& ket_left, GemmBatch& gb) {
  // Z' blocks by (row group = right sector, sigma); terms of every output
  // block (bra left sector, channel group) in (sector, group) order
  int nrg = 0, ng = 0;
  for (const auto& z : Zp.blocks) {
    nrg = std::max(nrg, z.rg + 1);
    ng = std::max(ng, z.g + 1);
  }
  std::vector<int> zstart((size_t)nrg * 4 + 1, 0), zlist(Zp.blocks.size());
  for (const auto& z : Zp.blocks) zstart[(size_t)z.rg * 4 + z.sig + 1]++;
  for (size_t i = 1; i < zstart.size(); ++i) zstart[i] += zstart[i - 1];
  {
    std::vector<int> fill(zstart.begin(), zstart.end() - 1);
    for (int z = 0; z < (int)Zp.blocks.size(); ++z) zlist[fill[(size_t)Zp.blocks[z].rg * 4 + Zp.blocks[z].sig]++] = z;
  }
  struct T { int bra, z; };
  const size_t nkey = (size_t)bra_left.nsec() * ng;
  std::vector<int> cstart(nkey + 1, 0);
  auto zs_of = [&](const SiteT::Blk& cb, int& lo, int& hi) {
    lo = hi = 0;
    if (cb.sb >= nrg) return;
    lo = zstart[(size_t)cb.sb * 4 + cb.sig];
    hi = zstart[(size_t)cb.sb * 4 + cb.sig + 1];
  };
  for (const auto& cb : bra.blocks) {
    int lo, hi;
    zs_of(cb, lo, hi);
    for (int q = lo; q < hi; ++q) cstart[(size_t)cb.r * ng + Zp.blocks[zlist[q]].g + 1]++;
  }
  for (size_t i = 1; i < cstart.size(); ++i) cstart[i] += cstart[i - 1];
  std::vector<T> terms(cstart[nkey]);
  {
    std::vector<int> fill(cstart.begin(), cstart.end() - 1);
    for (int b = 0; b < (int)bra.blocks.size(); ++b) {
      int lo, hi;
      zs_of(bra.blocks[b], lo, hi);
      for (int q = lo; q < hi; ++q) {
        const int z = zlist[q];
        terms[fill[(size_t)bra.blocks[b].r * ng + Zp.blocks[z].g]++] = {b, z};
      }
    }
  }
  Env e;
  e.rows = RowGroups::from_bond(bra_left);
  e.mb = &mb;
  e.ket_copy = ket_left;
  for (size_t key = 0; key < nkey; ++key) {
    if (cstart[key] == cstart[key + 1]) continue;
    const Inter::Blk& z0 = Zp.blocks[terms[cstart[key]].z];
    const int r = (int)(key / ng), g = (int)(key % ng);
    e.t.add(r, -1, g, z0.k, bra_left.d[r], z0.W, z0.cols);
  }
  e.t.et = Zp.et;
  e.t.alloc(c.st, false);
  int id = 0;
  for (size_t key = 0; key < nkey; ++key) {
    if (cstart[key] == cstart[key + 1]) continue;
    const Inter::Blk& eb = e.t.blocks[id];
    int N = eb.W * eb.cols;
    gb.task(e.t.ptr(id), e.t.et, eb.rows, N, N, OP_J, site_et(c), OP_N, Zp.et, false, 1.0);
    for (int q = cstart[key]; q < cstart[key + 1]; ++q) {
      const SiteT::Blk& cb = bra.blocks[terms[q].bra];
      int aet;
      const void* ap = site_operand(c, bra, terms[q].bra, aet);
      gb.term(ap, cb.cols, Zp.ptr(terms[q].z), N, cb.cols);
    }
    ++id;
  }
  return e;
}

// Single-term environment updates (density-matrix code, boundaries).
static Env env_update_left(Context& c, const Env& E, const SiteT& bra, const Bond& bra_right,
                           const MPSd& ket, int site, const MPOd& m) {
  GemmBatch g1(c);
  Inter X = plan_lstage(c, E, ket.sites[site], ket.bonds[site + 1], g1, &bra, &m, site);
  g1.run();
  WBatch wb;
  Inter Y = plan_wstage(c, std::move(X), m, site, true, wb, &bra);
  wb.run(c);
  GemmBatch g2(c);
  Env e = plan_env_left(c, Y, bra, bra_right, m.bonds[site + 1], ket.bonds[site + 1], g2);
  g2.run();
  return e;
}

static Env env_update_right(Context& c, const Env& R, const SiteT& bra, const Bond& bra_left,
                            const MPSd& ket, int site, const MPOd& m) {
  GemmBatch g1(c);
  Inter Z = plan_r1(c, R, ket.sites[site], ket.bonds[site], g1);
  g1.run();
  WBatch wb;
  Inter Zp = plan_wstage(c, std::move(Z), m, site, false, wb);
  wb.run(c);
  GemmBatch g2(c);
  Env e = plan_env_right(c, Zp, bra, bra_left, m.bonds[site], ket.bonds[site], g2);
  g2.run();
  return e;
}

// ------------------------------------------------------------------ factorisations

namespace {

struct FactWork {
  DevPtr buf;
  std::vector<FactTask> tasks;
  std::vector<size_t> a_off, v_off, s_off;
};

// allocate m x n work matrices (+ n x n V / R, + n values) for a list of shapes
FactWork fact_alloc(Context& c, const std::vector<std::pair<int, int>>& shapes) {
  FactWork fw;
  size_t off = 0;
  for (auto& sh : shapes) {
    fw.a_off.push_back(off);
    off += (size_t)sh.first * sh.second * sizeof(double2);
    off = (off + 255) & ~(size_t)255;
    fw.v_off.push_back(off);
    off += (size_t)sh.second * sh.second * sizeof(double2);
    off = (off + 255) & ~(size_t)255;
    fw.s_off.push_back(off);
    off += (size_t)sh.second * sizeof(double);
    off = (off + 255) & ~(size_t)255;
  }
  fw.buf = dev_alloc(std::max<size_t>(off, 256), c.st);
  char* base = (char*)fw.buf->p;
  for (size_t i = 0; i < shapes.size(); ++i)
    fw.tasks.push_back({(double2*)(base + fw.a_off[i]), (double2*)(base + fw.v_off[i]),
                        (double*)(base + fw.s_off[i]), shapes[i].first, shapes[i].second});
  return fw;
}

void run_copy(Context& c, const std::vector<CopyTask>& t, int to_work) {
  if (t.empty()) return;
  const CopyTask* d = c.stage(t);
  cudaEvent_t ev;
  c.kbegin(TDMPS_KSTAT_OTHER, &ev);
  launch_copy(d, (int)t.size(), to_work, c.st);
  double bytes = 0.0;
  for (auto& x : t) bytes += 32.0 * x.rows * x.cols;
  c.kend(TDMPS_KSTAT_OTHER, ev, 0.0, bytes);
}

void run_qr(Context& c, FactWork& fw) {
  if (fw.tasks.empty()) return;
  double fl = 0.0;
  for (auto& t : fw.tasks) {
    if (t.m > QR_MAX_ROWS || t.n > QR_MAX_COLS)
      throw Error(TDMPS_ERR_INVALID_ARG, "QR block exceeds the supported size");
    // algorithmic work: one classical Gram-Schmidt pass, 8 m n min(m, n)
    fl += 8.0 * t.m * t.n * std::min(t.m, t.n);
  }
  const FactTask* d = c.stage(fw.tasks);
  cudaEvent_t ev;
  c.kbegin(TDMPS_KSTAT_QR, &ev);
  launch_qr(d, (int)fw.tasks.size(), c.st, fw.tasks.data());
  c.kend(TDMPS_KSTAT_QR, ev, fl, 0.0);
}

void run_svd(Context& c, FactWork& fw) {
  if (fw.tasks.empty()) return;
  for (auto& t : fw.tasks)
    if (t.n > 1024) throw Error(TDMPS_ERR_INVALID_ARG, "SVD block exceeds the supported size");
  const FactTask* d = c.stage(fw.tasks);
  cudaEvent_t ev;
  c.kbegin(TDMPS_KSTAT_SVD, &ev);
  size_t mx = 0;
  for (auto& t : fw.tasks) mx = std::max(mx, (size_t)(t.m * t.n + t.n * t.n) * sizeof(double2));
  launch_svd(d, (int)fw.tasks.size(), (int*)c.status->p, c.st, mx, fw.tasks.data());
  double fl = 0.0;
  for (auto& t : fw.tasks) fl += 8.0 * 8.0 * t.m * t.n * t.n;
  c.kend(TDMPS_KSTAT_SVD, ev, fl, 0.0);
}

}  // namespace

// Block (r, s) -> sb of a site tensor seen as a matrix per right sector:
// rows = row groups r with their sigma, cols = d(sb).
struct RowLayout {
  std::vector<std::vector<std::pair<int, int>>> members;   // per sector: (block id, row offset)
  std::vector<int> m;
};
static RowLayout rows_by_right(const SiteT& t, int nsec_right) {
  RowLayout L;
  L.members.assign(nsec_right, {});
  L.m.assign(nsec_right, 0);
  for (int b = 0; b < (int)t.blocks.size(); ++b) {
    const SiteT::Blk& bl = t.blocks[b];
    L.members[bl.sb].push_back({b, L.m[bl.sb]});
    L.m[bl.sb] += bl.rows;
  }
  return L;
}

// One-site left-to-right gauge move: C -> Q (thin QR per right sector).
// Returns the new site tensor and the new right bond.
static std::pair<SiteT, Bond> qr_left(Context& c, const SiteT& C, const RowGroups& rows,
                                      const Bond& right) {
  RowLayout lay = rows_by_right(C, right.nsec());
  std::vector<std::pair<int, int>> shapes;
  std::vector<int> secs;
  for (int s = 0; s < right.nsec(); ++s)
    if (lay.m[s] > 0) { shapes.push_back({lay.m[s], right.d[s]}); secs.push_back(s); }
  FactWork fw = fact_alloc(c, shapes);
  std::vector<CopyTask> g;
  for (size_t i = 0; i < secs.size(); ++i)
    for (auto& mb : lay.members[secs[i]]) {
      const SiteT::Blk& bl = C.blocks[mb.first];
      g.push_back({C.ptr(mb.first), fw.tasks[i].A, bl.rows, bl.cols, bl.cols, shapes[i].first,
                   mb.second, 0, 0, 0, make_double2(1.0, 0.0)});
    }
  run_copy(c, g, 1);
  run_qr(c, fw);
  Bond nb;
  std::vector<int> kdim(right.nsec(), 0);
  for (size_t i = 0; i < secs.size(); ++i) kdim[secs[i]] = std::min(shapes[i].first, shapes[i].second);
  for (int s = 0; s < right.nsec(); ++s)
    if (kdim[s] > 0) { nb.q.push_back(right.q[s]); nb.d.push_back(kdim[s]); }
  SiteT Q = make_site(rows, nb, c.st, false);
  std::vector<CopyTask> sc;
  for (size_t i = 0; i < secs.size(); ++i) {
    int ns = nb.find(right.q[secs[i]]);
    for (auto& mb : lay.members[secs[i]]) {
      const SiteT::Blk& bl = C.blocks[mb.first];
      int qb = Q.block_of(bl.r, bl.sig);
      (void)ns;
      sc.push_back({Q.ptr(qb), fw.tasks[i].A, bl.rows, kdim[secs[i]], kdim[secs[i]],
                    shapes[i].first, mb.second, 0, 0, 0, make_double2(1.0, 0.0)});
    }
  }
  run_copy(c, sc, 0);
  return {std::move(Q), nb};
}

// One-site right-to-left gauge move: C = Lf Q per left sector (QR of C^H).
// Returns (Q site, new left bond); if absorb is given, also the factor work
// (R' of C^H = Q' R', with Lf = R'^H) for absorbing into the left neighbour.
struct LQResult {
  SiteT Q;
  Bond left;
  FactWork fw;
  std::vector<int> secs;   // old left sector per factor task
};
static LQResult lq_right(Context& c, const SiteT& C, const Bond& left, const Bond& right) {
  // per left sector: cols = (sig, sb) blocks concatenated
  std::vector<std::vector<std::pair<int, int>>> members(left.nsec());
  std::vector<int> ncol(left.nsec(), 0);
  for (int b = 0; b < (int)C.blocks.size(); ++b) {
    const SiteT::Blk& bl = C.blocks[b];
    members[bl.r].push_back({b, ncol[bl.r]});
    ncol[bl.r] += bl.cols;
  }
  LQResult res;
  std::vector<std::pair<int, int>> shapes;
  for (int s = 0; s < left.nsec(); ++s)
    if (ncol[s] > 0) { shapes.push_back({ncol[s], left.d[s]}); res.secs.push_back(s); }
  res.fw = fact_alloc(c, shapes);
  std::vector<CopyTask> g;
  for (size_t i = 0; i < res.secs.size(); ++i)
    for (auto& mb : members[res.secs[i]]) {
      const SiteT::Blk& bl = C.blocks[mb.first];
      // work = M^H (ncol x |sa|): block (i, j) of M at (0, off) -> conj_t
      g.push_back({C.ptr(mb.first), res.fw.tasks[i].A, bl.rows, bl.cols, bl.cols,
                   shapes[i].first, 0, mb.second, 1, 0, make_double2(1.0, 0.0)});
    }
  run_copy(c, g, 1);
  run_qr(c, res.fw);
  std::vector<int> kdim(left.nsec(), 0);
  for (size_t i = 0; i < res.secs.size(); ++i)
    kdim[res.secs[i]] = std::min(shapes[i].first, shapes[i].second);
  for (int s = 0; s < left.nsec(); ++s)
    if (kdim[s] > 0) { res.left.q.push_back(left.q[s]); res.left.d.push_back(kdim[s]); }
  res.Q = make_site(RowGroups::from_bond(res.left), right, c.st, false);
  std::vector<CopyTask> sc;
  for (size_t i = 0; i < res.secs.size(); ++i) {
    int s = res.secs[i];
    int ns = res.left.find(left.q[s]);
    for (auto& mb : members[s]) {
      const SiteT::Blk& bl = C.blocks[mb.first];
      int qb = res.Q.block_of(ns, bl.sig);
      // Q block (k x |sb|) = conj transpose of Q' rows [off, off+|sb|), cols [0, k)
      sc.push_back({res.Q.ptr(qb), res.fw.tasks[i].A, kdim[s], bl.cols, bl.cols, shapes[i].first,
                    0, mb.second, 1, 0, make_double2(1.0, 0.0)});
    }
  }
  run_copy(c, sc, 0);
  return res;
}

// new_prev[a'][s][k] = prev[a'][s][a] * Lf[a][k] with Lf = R'^H from lq_right
static SiteT absorb_left_factor(Context& c, const SiteT& prev, const RowGroups& rows,
                                const Bond& old_mid, const LQResult& lq) {
  SiteT out = make_site(rows, lq.left, c.st, false);
  std::map<int, int> task_of;   // old sector -> factor task
  for (size_t i = 0; i < lq.secs.size(); ++i) task_of[lq.secs[i]] = (int)i;
  GemmBatch gb(c, true);
  for (int o = 0; o < (int)out.blocks.size(); ++o) {
    const SiteT::Blk& ob = out.blocks[o];
    int old_sec = old_mid.find(lq.left.q[ob.sb]);
    int pb = prev.block_of(ob.r, ob.sig);
    gb.task(out.ptr(o), 0, ob.rows, ob.cols, ob.cols, OP_N, 0, OP_J, 0, false, 1.0);
    if (pb < 0 || old_sec < 0) continue;
    const FactTask& ft = lq.fw.tasks[task_of.at(old_sec)];
    // Lf[a][k] = conj(R[a*n + k]) with n = |sa| (leading dimension of R)
    gb.term(prev.ptr(pb), prev.blocks[pb].cols, ft.V, ft.n, ft.n);
  }
  gb.run();
  return out;
}

MPSd right_canonicalize(Context& c, const MPSd& m0) {
  MPSd m = m0;   // shares device buffers; every modified site is replaced
  for (int i = m.L - 1; i >= 1; --i) {
    LQResult lq = lq_right(c, m.sites[i], m.bonds[i], m.bonds[i + 1]);
    SiteT prev = absorb_left_factor(c, m.sites[i - 1], RowGroups::from_bond(m.bonds[i - 1]),
                                    m.bonds[i], lq);
    m.sites[i] = std::move(lq.Q);
    m.sites[i - 1] = std::move(prev);
    m.bonds[i] = lq.left;
  }
  m.rcanon = true;
  return m;
}

// Truncated SVD split of a tensor Th[(rg)][s2][c] whose row groups carry the
// middle charge.  Returns new left site (rows x middle), right site (middle x
// right) and the middle bond.  absorb_right: singular values go right.
struct SplitResult {
  SiteT A, B;
  Bond mid;
  double disc = 0.0, total = 0.0;
};
static SplitResult svd_split(Context& c, const SiteT& Th, const RowGroups& rows,
                             const RowGroups& left_rows_of_A, const Bond& right, int D, double eps,
                             bool absorb_right, int nsig2 = 4) {
  // middle charges
  std::map<QN, std::vector<std::pair<int, int>>> rmem;   // Q -> (row group, row offset)
  std::map<QN, int> mrows;
  for (int r = 0; r < rows.n(); ++r) {
    bool has = false;
    for (int s = 0; s < 4; ++s) has |= Th.block_of(r, s) >= 0;
    if (!has) continue;
    rmem[rows.q[r]].push_back({r, mrows[rows.q[r]]});
    mrows[rows.q[r]] += rows.d[r];
  }
  std::map<QN, std::vector<std::array<int, 3>>> cmem;    // Q -> (sig2, sc, col offset)
  std::map<QN, int> ncols;
  for (int s2 = 0; s2 < nsig2; ++s2)
    for (int sc = 0; sc < right.nsec(); ++sc) {
      QN Q = right.q[sc] - SITE_Q[s2];
      if (!mrows.count(Q)) continue;
      cmem[Q].push_back({s2, sc, ncols[Q]});
      ncols[Q] += right.d[sc];
    }
  std::vector<QN> qs;
  std::vector<std::pair<int, int>> shapes;
  std::vector<int> trans;
  for (auto& kv : mrows) {
    if (!ncols.count(kv.first)) continue;
    int m = kv.second, n = ncols[kv.first];
    qs.push_back(kv.first);
    bool t = n > m;
    trans.push_back(t);
    shapes.push_back(t ? std::make_pair(n, m) : std::make_pair(m, n));
  }
  SplitResult res;
  if (qs.empty()) throw Error(TDMPS_ERR_ZERO_STATE, "two-site tensor has no admissible sector");
  FactWork fw = fact_alloc(c, shapes);
  std::vector<CopyTask> g;
  for (size_t i = 0; i < qs.size(); ++i) {
    const QN& Q = qs[i];
    int ldw = shapes[i].first;
    for (auto& rm : rmem[Q])
      for (auto& cm : cmem[Q]) {
        int b = Th.block_of(rm.first, cm[0]);
        if (b < 0 || Th.blocks[b].sb != cm[1]) continue;
        const SiteT::Blk& bl = Th.blocks[b];
        g.push_back({Th.ptr(b), fw.tasks[i].A, bl.rows, bl.cols, bl.cols, ldw, rm.second, cm[2],
                     trans[i], 0, make_double2(1.0, 0.0)});
      }
  }
  // zero the work matrices first (blocks not present stay zero)
  for (size_t i = 0; i < qs.size(); ++i)
    launch_zero(fw.tasks[i].A, (size_t)shapes[i].first * shapes[i].second, c.st);
  run_copy(c, g, 1);
  // QR-preconditioned one-sided Jacobi: M = Q R, Jacobi on W = R^H gives
  // W J = U_w S, hence M = (Q J) S U_w^H; far fewer sweeps than Jacobi on M
  run_qr(c, fw);
  std::vector<std::pair<int, int>> sq;
  for (auto& sh : shapes) sq.push_back({sh.second, sh.second});
  FactWork fj = fact_alloc(c, sq);
  {
    std::vector<FactTask> both(fw.tasks);
    both.insert(both.end(), fj.tasks.begin(), fj.tasks.end());
    const FactTask* ds = c.stage(both);
    launch_adjoint(ds, ds + fw.tasks.size(), (int)fw.tasks.size(), c.st);
  }
  run_svd(c, fj);
  // U = Q J  (column-major m x n), computed as U^T = J^T Q^T in row-major terms
  DevPtr ubuf;
  std::vector<double2*> uptr(qs.size());
  {
    size_t tot = 0;
    for (auto& sh : shapes) tot += (size_t)sh.first * sh.second;
    ubuf = dev_alloc(std::max<size_t>(tot, 1) * sizeof(double2), c.st);
    size_t off = 0;
    GemmBatch gb(c, true);
    for (size_t i = 0; i < qs.size(); ++i) {
      const int m = shapes[i].first, n = shapes[i].second;
      uptr[i] = (double2*)ubuf->p + off;
      off += (size_t)m * n;
      gb.task(uptr[i], 0, n, m, m, OP_N, 0, OP_N, 0, false, 1.0);
      gb.term(fj.tasks[i].V, n, fw.tasks[i].A, m, n);
    }
    gb.run();
  }
  // truncation over all singular values of the bond
  std::vector<int> secid;
  int nv = 0;
  int ntot = 0;
  for (auto& sh : shapes) ntot += sh.second;
  DevPtr svals = dev_alloc(sizeof(double) * std::max(1, ntot) * 2 + 64, c.st);
  DevPtr sids = dev_alloc(sizeof(int) * std::max(1, ntot) * 2 + 64, c.st);
  for (size_t i = 0; i < qs.size(); ++i) {
    TD_CHECK_CUDA(cudaMemcpyAsync((double*)svals->p + nv, fj.tasks[i].s,
                                  sizeof(double) * shapes[i].second, cudaMemcpyDeviceToDevice, c.st));
    for (int k = 0; k < shapes[i].second; ++k) secid.push_back((int)i);
    nv += shapes[i].second;
  }
  const int* dsec = c.stage(secid);
  DevPtr kept = dev_alloc(sizeof(int) * (qs.size() + 2) + sizeof(double) * 4, c.st);
  int* dkept = (int*)kept->p;
  double* dw = (double*)((char*)kept->p + ((sizeof(int) * (qs.size() + 2) + 15) & ~(size_t)15));
  {
    cudaEvent_t ev;
    c.kbegin(TDMPS_KSTAT_OTHER, &ev);
    launch_trunc((const double*)svals->p, dsec, nv, (int)qs.size(), D, eps, dkept, dw,
                 (double*)svals->p + ntot, (int*)sids->p, c.st);
    c.kend(TDMPS_KSTAT_OTHER, ev, 0.0, 0.0);
  }
  std::vector<int> hk(qs.size());
  double hw[2];
  int hstat = 0;
  TD_CHECK_CUDA(cudaMemcpyAsync(hk.data(), dkept, sizeof(int) * qs.size(), cudaMemcpyDeviceToHost, c.st));
  TD_CHECK_CUDA(cudaMemcpyAsync(hw, dw, sizeof(double) * 2, cudaMemcpyDeviceToHost, c.st));
  TD_CHECK_CUDA(cudaMemcpyAsync(&hstat, c.status->p, sizeof(int), cudaMemcpyDeviceToHost, c.st));
  c.sync();
  if (hstat) throw Error(TDMPS_ERR_NUMERIC, "Jacobi SVD did not converge");
  if (!std::isfinite(hw[1])) throw Error(TDMPS_ERR_NONFINITE, "non-finite singular values");
  res.disc = hw[0];
  res.total = hw[1];
  for (size_t i = 0; i < qs.size(); ++i)
    if (hk[i] > 0) { res.mid.q.push_back(qs[i]); res.mid.d.push_back(hk[i]); }
  if (res.mid.q.empty()) throw Error(TDMPS_ERR_ZERO_STATE, "fit target vanished on this sweep");
  res.A = make_site(left_rows_of_A, res.mid, c.st, false);
  res.B = make_site(RowGroups::from_bond(res.mid), right, c.st, false);
  // scatter: A rows from U (or V' if transposed), B from V^H (or U'^H)
  std::vector<ScatterTask> ss;
  for (size_t i = 0; i < qs.size(); ++i) {
    int k = hk[i];
    if (k == 0) continue;
    const QN& Q = qs[i];
    int mid = res.mid.find(Q);
    const FactTask& ft = fw.tasks[i];
    // left factor Q J (m x n, ld m) and right factor U_w (n x n, ld n) of the
    // work matrix; the work matrix is M or M^H
    const double2* lf = uptr[i];
    const double2* rf = fj.tasks[i].A;
    const double2* usrc = trans[i] ? rf : lf;
    int ulds = trans[i] ? ft.n : ft.m;
    const double2* vsrc = trans[i] ? lf : rf;
    int vlds = trans[i] ? ft.m : ft.n;
    for (auto& rm : rmem[Q]) {
      int r = rm.first;
      int ab = res.A.block_of(rows.sa[r], rows.sig[r] < 0 ? 0 : rows.sig[r]);
      if (rows.sig[r] < 0) ab = res.A.block_of(rows.sa[r], 0);
      if (ab < 0 || res.A.blocks[ab].sb != mid) continue;
      ss.push_back({res.A.ptr(ab), rows.d[r], k, k, usrc, ulds, rm.second, 0, 0,
                    absorb_right ? 0 : 1, fj.tasks[i].s});
    }
    for (auto& cm : cmem[Q]) {
      int bb = res.B.block_of(mid, cm[0]);
      if (bb < 0 || res.B.blocks[bb].sb != cm[1]) continue;
      ss.push_back({res.B.ptr(bb), k, right.d[cm[1]], right.d[cm[1]], vsrc, vlds, cm[2], 0, 1,
                    absorb_right ? 2 : 0, fj.tasks[i].s});
    }
  }
  if (!ss.empty()) {
    const ScatterTask* d = c.stage(ss);
    cudaEvent_t ev;
    c.kbegin(TDMPS_KSTAT_OTHER, &ev);
    launch_scatter(d, (int)ss.size(), c.st);
    c.kend(TDMPS_KSTAT_OTHER, ev, 0.0, 0.0);
  }
  return res;
}

// ------------------------------------------------------------------ fit

namespace {

struct TermState {
  const MPSd* ket;
  const MPOd* mpo;
  cplx coef;
  const double2* coef_dev;
  std::vector<Env> LE, RE;
};

void check_same_space(const MPSd& a, const MPSd& b) {
  if (a.L != b.L) throw Error(TDMPS_ERR_INVALID_ARG, "MPS lengths differ");
  if (a.tot != b.tot) throw Error(TDMPS_ERR_SECTOR, "MPS quantum numbers (N, 2Sz) differ");
}

// MPO stage for all terms: one launch per distinct (non-identity) MPO
std::vector<Inter> wstage_all(Context& c, const std::vector<TermState>& ts,
                              std::vector<Inter>&& X, int site, bool left) {
  std::vector<Inter> Y(ts.size());
  std::vector<WBatch> batches;
  std::vector<const MPOd*> mpos;
  for (size_t t = 0; t < ts.size(); ++t) {
    if (ts[t].mpo->identity) { Y[t] = std::move(X[t]); continue; }
    size_t b = 0;
    while (b < mpos.size() && mpos[b] != ts[t].mpo) ++b;
    if (b == mpos.size()) { mpos.push_back(ts[t].mpo); batches.emplace_back(); }
    Y[t] = plan_wstage(c, std::move(X[t]), *ts[t].mpo, site, left, batches[b]);
  }
  for (auto& wb : batches) wb.run(c);
  return Y;
}

// right environments at bond i of all terms from bond i+1, bra site C[i]
void right_env_step(Context& c, std::vector<TermState>& ts, const MPSd& C, int i,
                    const std::vector<Inter>* zp = nullptr) {
  std::vector<Inter> Zp;
  if (!zp) {
    GemmBatch g1(c);
    std::vector<Inter> Z(ts.size());
    for (size_t t = 0; t < ts.size(); ++t)
      Z[t] = plan_r1(c, ts[t].RE[i + 1], ts[t].ket->sites[i], ts[t].ket->bonds[i], g1);
    g1.run();
    Zp = wstage_all(c, ts, std::move(Z), i, false);
    zp = &Zp;
  }
  GemmBatch g3(c);
  for (size_t t = 0; t < ts.size(); ++t)
    ts[t].RE[i] = plan_env_right(c, (*zp)[t], C.sites[i], C.bonds[i], ts[t].mpo->bonds[i],
                                 ts[t].ket->bonds[i], g3);
  g3.run();
}

void left_env_step(Context& c, std::vector<TermState>& ts, const MPSd& C, int i,
                   const std::vector<Inter>& Y) {
  GemmBatch g3(c);
  for (size_t t = 0; t < ts.size(); ++t)
    ts[t].LE[i + 1] = plan_env_left(c, Y[t], C.sites[i], C.bonds[i + 1], ts[t].mpo->bonds[i + 1],
                                    ts[t].ket->bonds[i + 1], g3);
  g3.run();
}

// Y_t = W_i (L_t[i] A_t[i]) for all terms
std::vector<Inter> left_stages(Context& c, std::vector<TermState>& ts, int i) {
  GemmBatch g1(c);
  std::vector<Inter> X(ts.size());
  for (size_t t = 0; t < ts.size(); ++t)
    X[t] = plan_lstage(c, ts[t].LE[i], ts[t].ket->sites[i], ts[t].ket->bonds[i + 1], g1);
  g1.run();
  return wstage_all(c, ts, std::move(X), i, true);
}

// Zp_t = W_i^right (R_t[i+1] A_t[i]^T) for all terms
std::vector<Inter> right_stages(Context& c, std::vector<TermState>& ts, int i) {
  GemmBatch g1(c);
  std::vector<Inter> Z(ts.size());
  for (size_t t = 0; t < ts.size(); ++t)
    Z[t] = plan_r1(c, ts[t].RE[i + 1], ts[t].ket->sites[i], ts[t].ket->bonds[i], g1);
  g1.run();
  return wstage_all(c, ts, std::move(Z), i, false);
}

}  // namespace

// Variational fit of Eq. (add_min): sum_t coef_t O_t |ket_t> into an MPS of
// bond dimension <= D, guess right-canonicalised first; schedule as in the
// header.  Left-to-right one-site steps contract L, A, W, then R, and reuse
// W(L A) for the new left environment; right-to-left steps contract R, A, W,
// then L, and reuse W(R A) for the new right environment.
MPSd fit(Context& c, const std::vector<FitTerm>& terms, const MPSd& guess, const FitOpts& o) {
  if (terms.empty()) throw Error(TDMPS_ERR_INVALID_ARG, "no fit terms");
  if (o.D < 1) throw Error(TDMPS_ERR_INVALID_ARG, "D must be >= 1");
  if (o.n_two_site < 0 || o.n_one_site < 0 || o.n_two_site + o.n_one_site < 1)
    throw Error(TDMPS_ERR_INVALID_ARG, "invalid sweep schedule");
  for (auto& t : terms) check_same_space(*t.ket, guess);
  const int L = guess.L;
  // the guess in right-canonical gauge; outputs of fits and compressions
  // already are, so they are used as they stand (every site is replaced
  // below, nothing is written in place)
  MPSd C = guess.rcanon ? guess : right_canonicalize(c, guess);
  C.rcanon = true;
  std::vector<TermState> ts(terms.size());
  for (size_t t = 0; t < terms.size(); ++t) {
    ts[t].ket = terms[t].ket;
    ts[t].mpo = terms[t].mpo ? terms[t].mpo : &c.identity_mpo(L);
    if (ts[t].mpo->L != L) throw Error(TDMPS_ERR_INVALID_ARG, "MPO length differs from MPS");
    ts[t].coef = terms[t].coef;
    ts[t].coef_dev = terms[t].coef_dev;
    ts[t].LE.resize(L + 1);
    ts[t].RE.resize(L + 1);
    ts[t].LE[0] = env_left_boundary(c, C, *ts[t].ket, *ts[t].mpo);
    ts[t].RE[L] = env_right_boundary(c, C, *ts[t].ket, *ts[t].mpo);
  }
  for (int i = L - 1; i >= 1; --i) right_env_step(c, ts, C, i);
  auto local_terms = [&](const std::vector<Inter>& Y, int env_bond, bool right_env) {
    std::vector<LocalTerm> lt;
    for (size_t t = 0; t < ts.size(); ++t)
      lt.push_back({&Y[t], right_env ? &ts[t].RE[env_bond] : &ts[t].LE[env_bond], ts[t].coef,
                    ts[t].coef_dev});
    return lt;
  };
  if (L == 1) {
    std::vector<Inter> Y = left_stages(c, ts, 0);
    SiteT out = make_site(RowGroups::from_bond(C.bonds[0]), C.bonds[1], c.st, false);
    GemmBatch g(c);
    plan_rstage(local_terms(Y, 1, true), out, g);
    g.run();
    C.sites[0] = std::move(out);
    return C;
  }
  double maxdisc = 0.0;
  for (int sw = 0; sw < o.n_two_site; ++sw) {
    for (int half = 0; half < 2; ++half) {
      for (int step = 0; step < L - 1; ++step) {
        const int i = half == 0 ? step : L - 2 - step;
        // two-site tensor: (L A_i W_i) viewed as an environment with fused
        // rows (a, s1), then A_{i+1}, W_{i+1} and R_{i+2}
        std::vector<Inter> Y1 = left_stages(c, ts, i);
        RowGroups fr = RowGroups::fused(C.bonds[i]);
        std::vector<Env> E2(ts.size());
        for (size_t t = 0; t < ts.size(); ++t) {
          E2[t].rows = fr;
          E2[t].mb = &ts[t].mpo->bonds[i + 1];
          E2[t].ket_copy = ts[t].ket->bonds[i + 1];
          E2[t].t.data = Y1[t].data;
          E2[t].t.size = Y1[t].size;
          E2[t].t.et = Y1[t].et;
          for (auto& b : Y1[t].blocks) {
            int id = (int)E2[t].t.blocks.size();
            E2[t].t.blocks.push_back({b.rg * 4 + b.sig, -1, b.g, b.k, b.rows, b.W, b.cols, b.off});
            E2[t].t.index[Inter::key(b.rg * 4 + b.sig, -1, b.g, b.k)] = id;
          }
        }
        GemmBatch g2(c);
        std::vector<Inter> X2(ts.size());
        for (size_t t = 0; t < ts.size(); ++t)
          X2[t] = plan_lstage(c, E2[t], ts[t].ket->sites[i + 1], ts[t].ket->bonds[i + 2], g2);
        g2.run();
        std::vector<Inter> Y2 = wstage_all(c, ts, std::move(X2), i + 1, true);
        SiteT Th = make_site(fr, C.bonds[i + 2], c.st, false);
        GemmBatch g3(c);
        plan_rstage(local_terms(Y2, i + 2, true), Th, g3);
        g3.run();
        SplitResult sp = svd_split(c, Th, fr, RowGroups::from_bond(C.bonds[i]), C.bonds[i + 2],
                                   o.D, o.eps, half == 0);
        if (sp.total > 0) maxdisc = std::max(maxdisc, sp.disc / sp.total);
        C.sites[i] = std::move(sp.A);
        C.sites[i + 1] = std::move(sp.B);
        C.bonds[i + 1] = sp.mid;
        if (half == 0) left_env_step(c, ts, C, i, Y1);
        else right_env_step(c, ts, C, i + 1);
      }
    }
  }
  for (int sw = 0; sw < o.n_one_site; ++sw) {
    for (int i = 0; i < L; ++i) {
      std::vector<Inter> Y = left_stages(c, ts, i);
      SiteT Ci = make_site(RowGroups::from_bond(C.bonds[i]), C.bonds[i + 1], c.st, false);
      GemmBatch g(c);
      plan_rstage(local_terms(Y, i + 1, true), Ci, g);
      g.run();
      if (i < L - 1) {
        auto qr = qr_left(c, Ci, RowGroups::from_bond(C.bonds[i]), C.bonds[i + 1]);
        C.sites[i] = std::move(qr.first);
        C.bonds[i + 1] = qr.second;
        left_env_step(c, ts, C, i, Y);
      } else {
        C.sites[i] = std::move(Ci);
      }
    }
    for (int i = L - 1; i >= 0; --i) {
      std::vector<Inter> Zp = right_stages(c, ts, i);
      SiteT Ci = make_site(RowGroups::from_bond(C.bonds[i]), C.bonds[i + 1], c.st, false);
      GemmBatch g(c);
      plan_lcontract(local_terms(Zp, i, false), Ci, g);
      g.run();
      if (i > 0) {
        LQResult lq = lq_right(c, Ci, C.bonds[i], C.bonds[i + 1]);
        C.sites[i] = std::move(lq.Q);
        C.bonds[i] = lq.left;
        right_env_step(c, ts, C, i, &Zp);
      } else {
        C.sites[0] = std::move(Ci);
      }
    }
  }
  if (o.max_discarded) *o.max_discarded = std::max(*o.max_discarded, maxdisc);
  return C;
}

// ------------------------------------------------------------------ sandwiches

namespace {
// Temporarily switch a context to FP64 contractions (Krylov inner products,
// observables and norms stay FP64 in every precision mode).
struct Fp64Scope {
  Context& c;
  int saved;
  explicit Fp64Scope(Context& ctx, bool on = true) : c(ctx), saved(ctx.precision) {
    if (on) c.precision = TDMPS_FP64;
  }
  ~Fp64Scope() { c.precision = saved; }
};
}  // namespace

// <bra_p| O |ket_p> for many pairs, one launch per stage and site for all.
void sandwich_batch(Context& c, const MPOd* mpo,
                    const std::vector<std::pair<const MPSd*, const MPSd*>>& pairs,
                    const std::vector<double2*>& outs, bool fp64) {
  if (pairs.empty()) return;
  Fp64Scope scope(c, fp64);
  const int L = pairs[0].first->L;
  for (auto& p : pairs) check_same_space(*p.first, *p.second);
  const MPOd& m = mpo ? *mpo : c.identity_mpo(L);
  std::vector<Env> E(pairs.size());
  for (size_t p = 0; p < pairs.size(); ++p) E[p] = env_left_boundary(c, *pairs[p].first, *pairs[p].second, m);
  for (int i = 0; i < L; ++i) {
    GemmBatch g1(c);
    std::vector<Inter> X(pairs.size());
    for (size_t p = 0; p < pairs.size(); ++p)
      X[p] = plan_lstage(c, E[p], pairs[p].second->sites[i], pairs[p].second->bonds[i + 1], g1,
                         &pairs[p].first->sites[i], &m, i);
    g1.run();
    WBatch wb;
    std::vector<Inter> Y(pairs.size());
    for (size_t p = 0; p < pairs.size(); ++p)
      Y[p] = plan_wstage(c, std::move(X[p]), m, i, true, wb, &pairs[p].first->sites[i]);
    wb.run(c);
    GemmBatch g2(c);
    for (size_t p = 0; p < pairs.size(); ++p)
      E[p] = plan_env_left(c, Y[p], pairs[p].first->sites[i], pairs[p].first->bonds[i + 1],
                           m.bonds[i + 1], pairs[p].second->bonds[i + 1], g2);
    g2.run();
  }
  for (size_t p = 0; p < pairs.size(); ++p) {
    const Env& e = E[p];
    if (e.t.blocks.empty()) {
      TD_CHECK_CUDA(cudaMemsetAsync(outs[p], 0, sizeof(double2), c.st));
      continue;
    }
    if (e.t.blocks.size() != 1 || e.t.blocks[0].rows != 1 || e.t.blocks[0].W != 1 ||
        e.t.blocks[0].cols != 1)
      throw Error(TDMPS_ERR_SECTOR, "final environment is not a scalar");
    launch_to_double(e.t.ptr(0), e.t.et, outs[p], 1, c.st);
  }
}

void sandwich_dev(Context& c, const MPOd* mpo, const MPSd& bra, const MPSd& ket, double2* out) {
  sandwich_batch(c, mpo, {{&bra, &ket}}, {out});
}

cplx sandwich(Context& c, const MPOd* mpo, const MPSd& bra, const MPSd& ket) {
  DevPtr d = dev_alloc(sizeof(double2), c.st);
  sandwich_dev(c, mpo, bra, ket, (double2*)d->p);
  double2 h;
  TD_CHECK_CUDA(cudaMemcpyAsync(&h, d->p, sizeof(double2), cudaMemcpyDeviceToHost, c.st));
  c.sync();
  return cplx(h.x, h.y);
}

// ------------------------------------------------------------------ energy gradient

// The adjoint of E = <psi|H|psi> / <psi|psi> with respect to the site tensors
// (the effective-Hamiltonian matvec of Eq. add_min's local problem, applied
// to psi's own site): dE/dconj(A_i) = (H_i A_i - E N_i A_i) / <psi|psi>.  H_i
// A_i and N_i A_i are the one-site products L W A R with the environments of
// <psi|H|psi> and <psi|psi> (bra = ket = psi, so no gauge is assumed).  The
// two terms share every launch of a pass.  Right environments from site L
// down; then a left-to-right pass forms the products site by site and
// advances the left environments, which are dropped once used.  With stride
// s > 1 only the right environments at bonds that are multiples of s (and L)
// are kept: the pass rebuilds the others of one segment from the next kept
// bond when it reaches it (one more right sweep in all, environment memory
// O(L/s + s) instead of O(L)).
MPSd energy_gradient(Context& c, const MPOd& H, const MPSd& psi, int stride, double* energy,
                     size_t* env_bytes_peak) {
  if (stride < 1) throw Error(TDMPS_ERR_INVALID_ARG, "stride must be >= 1");
  if (H.L != psi.L) throw Error(TDMPS_ERR_INVALID_ARG, "MPO length differs from MPS");
  Fp64Scope scope(c, true);
  const int L = psi.L;
  std::vector<TermState> ts(2);
  ts[0].mpo = &H;
  ts[1].mpo = &c.identity_mpo(L);
  for (auto& t : ts) {
    t.ket = &psi;
    t.coef = 1.0;
    t.coef_dev = nullptr;
    t.LE.resize(L + 1);
    t.RE.resize(L + 1);
    t.LE[0] = env_left_boundary(c, psi, psi, *t.mpo);
    t.RE[L] = env_right_boundary(c, psi, psi, *t.mpo);
  }
  auto kept = [&](int b) { return b == L || b % stride == 0; };
  size_t live = 0, peak = 0;
  auto env_bytes = [](const Env& e) { return e.t.size * e.t.esz(); };
  auto note = [&](long long delta) {
    live = (size_t)((long long)live + delta);
    peak = std::max(peak, live);
  };
  for (auto& t : ts) note((long long)(env_bytes(t.LE[0]) + env_bytes(t.RE[L])));
  // right environments RE[b] for b = hi - 1 down to lo from RE[hi]; those of
  // bonds that are not kept are dropped once the next one is formed, unless
  // keep_all (a segment rebuilt for the left-to-right pass)
  auto right_sweep = [&](int hi, int lo, bool keep_all) {
    for (int i = hi - 1; i >= lo; --i) {
      right_env_step(c, ts, psi, i);
      for (auto& t : ts) note((long long)env_bytes(t.RE[i]));
      if (!keep_all && !kept(i + 1))
        for (auto& t : ts) {
          note(-(long long)env_bytes(t.RE[i + 1]));
          t.RE[i + 1] = Env();
        }
    }
  };
  right_sweep(L, 0, false);
  // E and <psi|psi> from the bond-0 environments (1 x 1 x 1 blocks)
  DevPtr sc = dev_alloc(2 * sizeof(double2), c.st);
  for (int k = 0; k < 2; ++k) {
    const Env& e = ts[k].RE[0];
    if (e.t.blocks.size() != 1) throw Error(TDMPS_ERR_SECTOR, "final environment is not a scalar");
    launch_to_double(e.t.ptr(0), e.t.et, (double2*)sc->p + k, 1, c.st);
  }
  double2 hv[2];
  TD_CHECK_CUDA(cudaMemcpyAsync(hv, sc->p, sizeof(hv), cudaMemcpyDeviceToHost, c.st));
  c.sync();
  const double nrm = hv[1].x;
  if (!(nrm > 0.0)) throw Error(TDMPS_ERR_ZERO_STATE, "state has zero norm");
  const double E = hv[0].x / nrm;
  if (energy) *energy = E;
  for (auto& t : ts) {
    note(-(long long)env_bytes(t.RE[0]));
    t.RE[0] = Env();
  }
  MPSd G;
  G.L = L;
  G.tot = psi.tot;
  G.bonds = psi.bonds;
  G.sites.resize(L);
  for (int i = 0; i < L; ++i) {
    if (ts[0].RE[i + 1].t.blocks.empty() && !kept(i + 1)) {
      // rebuild the segment (i + 1 .. next kept bond - 1)
      const int hi = std::min(L, ((i + 1) / stride + 1) * stride);
      right_sweep(hi, i + 1, true);
    }
    std::vector<Inter> Y = left_stages(c, ts, i);
    SiteT gh = make_site(RowGroups::from_bond(psi.bonds[i]), psi.bonds[i + 1], c.st, false);
    SiteT gn = make_site(RowGroups::from_bond(psi.bonds[i]), psi.bonds[i + 1], c.st, false);
    {
      GemmBatch g(c);
      plan_rstage({{&Y[0], &ts[0].RE[i + 1], 1.0, nullptr}}, gh, g);
      plan_rstage({{&Y[1], &ts[1].RE[i + 1], 1.0, nullptr}}, gn, g);
      g.run();
    }
    // G_i = (H_i A_i - E N_i A_i) / <psi|psi>
    launch_axpby((double2*)gh.data->p, (const double2*)gn.data->p, gh.size,
                 make_double2(1.0 / nrm, 0.0), make_double2(-E / nrm, 0.0), c.st);
    G.sites[i] = std::move(gh);
    if (i + 1 < L) {
      left_env_step(c, ts, psi, i, Y);
      for (auto& t : ts) note((long long)env_bytes(t.LE[i + 1]));
    }
    for (auto& t : ts) {
      note(-(long long)(env_bytes(t.LE[i]) + env_bytes(t.RE[i + 1])));
      t.LE[i] = Env();
      t.RE[i + 1] = Env();
    }
  }
  if (env_bytes_peak) *env_bytes_peak = peak;
  c.sync();
  return G;
}

// ------------------------------------------------------------------ local operator

// The local problem of Eq. add_min at one site, as an operator on that site's
// tensor: L W x R, the product every one-site fit step forms, with the
// environments of <psi|H|psi> (no gauge assumed: <psi(x)|H|psi(z)> = <x, H_i z>
// for psi with site i replaced).  The environments come from one sweep in
// from each end, exactly as a fit builds them, and stay on the device.
std::unique_ptr<LocalOp> local_op_create(Context& c, const MPOd& H, const MPSd& psi, int site) {
  if (H.L != psi.L) throw Error(TDMPS_ERR_INVALID_ARG, "MPO length differs from MPS");
  if (site < 0 || site >= psi.L) throw Error(TDMPS_ERR_INVALID_ARG, "site out of range");
  const int L = psi.L;
  auto op = std::make_unique<LocalOp>();
  op->H = H;
  op->site = site;
  op->L = L;
  op->precision = c.precision;
  op->tot = psi.tot;
  op->left = psi.bonds[site];
  op->right = psi.bonds[site + 1];
  std::vector<TermState> ts(1);
  TermState& t = ts[0];
  t.ket = &psi;
  t.mpo = &op->H;
  t.coef = 1.0;
  t.coef_dev = nullptr;
  t.LE.resize(L + 1);
  t.RE.resize(L + 1);
  t.LE[0] = env_left_boundary(c, psi, psi, op->H);
  for (int j = 0; j < site; ++j) {
    std::vector<Inter> Y = left_stages(c, ts, j);
    left_env_step(c, ts, psi, j, Y);
    t.LE[j] = Env();
  }
  t.RE[L] = env_right_boundary(c, psi, psi, op->H);
  for (int j = L - 1; j > site; --j) {
    right_env_step(c, ts, psi, j);
    t.RE[j + 1] = Env();
  }
  op->LE = std::move(t.LE[site]);
  op->RE = std::move(t.RE[site + 1]);
  op->env_bytes = op->LE.t.size * op->LE.t.esz() + op->RE.t.size * op->RE.t.esz();
  return op;
}

void local_op_apply(Context& c, const LocalOp& op, const MPSd& x, MPSd& y) {
  if (c.precision != op.precision)
    throw Error(TDMPS_ERR_INVALID_ARG, "context precision differs from the operator's");
  auto on_bonds = [&](const MPSd& m) {
    const Bond& a = m.bonds[op.site];
    const Bond& b = m.bonds[op.site + 1];
    return m.L == op.L && m.tot == op.tot && a.q == op.left.q && a.d == op.left.d &&
           b.q == op.right.q && b.d == op.right.d;
  };
  if (!on_bonds(x) || !on_bonds(y))
    throw Error(TDMPS_ERR_SECTOR, "x and y must have the operator's bonds at its site");
  GemmBatch g1(c);
  Inter X = plan_lstage(c, op.LE, x.sites[op.site], op.right, g1);
  g1.run();
  WBatch wb;
  Inter Y = plan_wstage(c, std::move(X), op.H, op.site, true, wb);
  wb.run(c);
  SiteT out = make_site(RowGroups::from_bond(op.left), op.right, c.st, false);
  GemmBatch g2(c);
  plan_rstage({{&Y, &op.RE, 1.0, nullptr}}, out, g2);
  g2.run();
  y.sites[op.site] = std::move(out);
  y.rcanon = false;
}

void normalize_center(Context& c, MPSd& m, double2* norm_out) {
  cudaEvent_t ev;
  c.kbegin(TDMPS_KSTAT_OTHER, &ev);
  launch_normalize((double2*)m.sites[0].data->p, m.sites[0].size, norm_out, c.st);
  m.sites[0].data32.reset();
  c.kend(TDMPS_KSTAT_OTHER, ev, 0.0, 0.0);
}

// Mixed-precision fits come out scaled: at L = 16, D = 256 a fitted H|psi>
// is the FP64 fit times (1 - 1.7e-5) (the same factor on every 1-RDM entry
// to 2e-7), while its direction agrees to 1 - 4e-12 in fidelity.  The
// shrink grows with the length of the accumulation chains (cutting them to
// 4 K stages by split-K removes a third of it), the signature of FP32
// accumulators that drop the low bits of each MMA's sum instead of rounding
// them.  For a target T that is a sum of states, <C|T> and <C|C> are cheap
// FP64 overlaps, and the projection property of the last local solve
// (<C|T> = <C|C>) fixes the scale.
void restore_fit_scale(Context& c, MPSd& C, const std::vector<FitTerm>& terms) {
  if (c.precision == TDMPS_FP64 || terms.empty()) return;
  std::vector<std::pair<const MPSd*, const MPSd*>> pairs;
  for (auto& t : terms) {
    if (t.mpo) throw Error(TDMPS_ERR_INVALID_ARG, "scale restoration needs a sum of states");
    pairs.push_back({&C, t.ket});
  }
  pairs.push_back({&C, &C});
  const size_t n = pairs.size();
  DevPtr d = dev_alloc(sizeof(double2) * 2 * n, c.st);
  std::vector<double2*> outs;
  for (size_t k = 0; k < n; ++k) outs.push_back((double2*)d->p + k);
  sandwich_batch(c, nullptr, pairs, outs, true);
  // device coefficients next to the overlaps, one copy back
  for (size_t k = 0; k + 1 < n; ++k)
    if (terms[k].coef_dev)
      TD_CHECK_CUDA(cudaMemcpyAsync((double2*)d->p + n + k, terms[k].coef_dev, sizeof(double2),
                                    cudaMemcpyDeviceToDevice, c.st));
  std::vector<double2> h(2 * n);
  TD_CHECK_CUDA(cudaMemcpyAsync(h.data(), d->p, sizeof(double2) * 2 * n, cudaMemcpyDeviceToHost, c.st));
  c.sync();
  cplx ct = 0.0;
  for (size_t k = 0; k + 1 < n; ++k) {
    cplx a = terms[k].coef;
    if (terms[k].coef_dev) a *= cplx(h[n + k].x, h[n + k].y);
    ct += a * cplx(h[k].x, h[k].y);
  }
  const double cc = h[n - 1].x;
  if (!(cc > 0.0) || !std::isfinite(ct.real()) || !std::isfinite(ct.imag())) return;
  const cplx s = ct / cc;
  // the gauge centre of a fit result is site 0
  launch_scale((double2*)C.sites[0].data->p, C.sites[0].size, make_double2(s.real(), s.imag()), c.st);
  C.sites[0].data32.reset();
}

// ------------------------------------------------------------------ compress

double compress(Context& c, MPSd& m, int D, double eps) {
  if (D < 1) throw Error(TDMPS_ERR_INVALID_ARG, "D must be >= 1");
  MPSd C = m.rcanon ? m : right_canonicalize(c, m);
  double disc_sum = 0.0;
  for (int i = 0; i + 1 < C.L; ++i) {
    // SVD of site i as (rows = (a, s)) x b per right sector: reuse svd_split
    // with a one-site tensor whose "right" part is the bond itself.
    RowGroups rows = RowGroups::from_bond(C.bonds[i]);
    // build a tensor viewed as Th[(a,s)][s2=0][b]: express site i with fused
    // rows and sigma2 = 0 (charge 0) by re-keying its blocks.
    RowGroups fr = RowGroups::fused(C.bonds[i]);
    SiteT Th;
    Th.index.assign((size_t)fr.n() * 4, -1);
    Th.data = C.sites[i].data;
    Th.size = C.sites[i].size;
    for (auto& b : C.sites[i].blocks) {
      int r = b.r * 4 + b.sig;
      Th.index[(size_t)r * 4 + 0] = (int)Th.blocks.size();
      Th.blocks.push_back({r, 0, b.sb, b.rows, b.cols, b.off});
    }
    SplitResult sp = svd_split(c, Th, fr, rows, C.bonds[i + 1], D, eps, true, 1);
    if (sp.total > 0) disc_sum += sp.disc / sp.total;
    // sp.B is (mid x 0 x right bond) with sigma2 = 0: contract with site i+1
    const SiteT& nxt = C.sites[i + 1];
    SiteT out = make_site(RowGroups::from_bond(sp.mid), C.bonds[i + 2], c.st, false);
    GemmBatch gb(c, true);
    for (int o = 0; o < (int)out.blocks.size(); ++o) {
      const SiteT::Blk& ob = out.blocks[o];
      gb.task(out.ptr(o), 0, ob.rows, ob.cols, ob.cols, OP_N, 0, OP_N, 0, false, 1.0);
      // old middle sector with the same charge
      int old = C.bonds[i + 1].find(sp.mid.q[ob.r]);
      int sb = sp.B.block_of(ob.r, 0);
      int nb = nxt.block_of(old, ob.sig);
      if (sb < 0 || nb < 0) continue;
      gb.term(sp.B.ptr(sb), sp.B.blocks[sb].cols, nxt.ptr(nb), ob.cols, sp.B.blocks[sb].cols);
    }
    gb.run();
    C.sites[i] = std::move(sp.A);
    C.sites[i + 1] = std::move(out);
    C.bonds[i + 1] = sp.mid;
  }
  m = right_canonicalize(c, C);
  return disc_sum;
}

// ------------------------------------------------------------------ integrators

MPSd rk4_step(Context& c, const MPOd& H, const MPSd& psi, double dt, const FitOpts& o) {
  const cplx a(0.0, -dt);
  auto applyH = [&](const MPSd& x) { return fit(c, {{&x, &H, a}}, x, o); };
  auto sum2 = [&](cplx cb, const MPSd& b) { return fit(c, {{&psi, nullptr, 1.0}, {&b, nullptr, cb}}, psi, o); };
  MPSd k1 = applyH(psi);
  MPSd s1 = sum2(0.5, k1);
  MPSd k2 = applyH(s1);
  MPSd s2 = sum2(0.5, k2);
  MPSd k3 = applyH(s2);
  MPSd s3 = sum2(1.0, k3);
  MPSd k4 = applyH(s3);
  const std::vector<FitTerm> fin = {{&psi, nullptr, 1.0}, {&k1, nullptr, 1.0 / 6},
                                    {&k2, nullptr, 1.0 / 3}, {&k3, nullptr, 1.0 / 3},
                                    {&k4, nullptr, 1.0 / 6}};
  MPSd out = fit(c, fin, psi, o);
  restore_fit_scale(c, out, fin);
  return out;
}

MPSd krylov_step(Context& c, const MPOd& H, const MPSd& psi, double dt, int m, bool orth,
                 const FitOpts& o) {
  if (m < 2 || m > 16) throw Error(TDMPS_ERR_INVALID_ARG, "Krylov dimension must be in [2, 16]");
  std::vector<MPSd> phi;
  phi.reserve(m);
  phi.push_back(psi);
  DevPtr mats = dev_alloc(sizeof(double2) * (2 * m * m + 2 * m + 8), c.st);
  double2* Nd = (double2*)mats->p;
  double2* Hd = Nd + m * m;
  double2* cd = Hd + m * m;
  TD_CHECK_CUDA(cudaMemsetAsync(mats->p, 0, sizeof(double2) * (2 * m * m + 2 * m + 8), c.st));
  std::vector<char> haveN(m * m, 0), haveH(m * m, 0);
  // batched exact overlaps / H sandwiches for the pairs (i, j), i <= j, not yet known
  auto fill = [&](const std::vector<std::pair<int, int>>& want, bool withH) {
    std::vector<std::pair<const MPSd*, const MPSd*>> pn, ph;
    std::vector<double2*> on, oh;
    for (auto& ij : want) {
      int i = ij.first, j = ij.second;
      if (!haveN[i * m + j]) {
        pn.push_back({&phi[i], &phi[j]});
        on.push_back(Nd + i * m + j);
        haveN[i * m + j] = 1;
      }
      if (withH && !haveH[i * m + j]) {
        ph.push_back({&phi[i], &phi[j]});
        oh.push_back(Hd + i * m + j);
        haveH[i * m + j] = 1;
      }
    }
    sandwich_batch(c, nullptr, pn, on, c.krylov_fp64);
    sandwich_batch(c, &H, ph, oh, c.krylov_fp64);
  };
  // The inner products of a Gram-Schmidt step depend on phi_0..phi_k only,
  // not on the fit of H phi_k that precedes their use; with FP64 inner
  // products they run on a helper context (its own stream, staging ring and
  // caches) driven by a second host thread, while this thread plans and
  // launches the fit.  The fit keeps the tensor cores and the QR busy, the
  // inner products the FP64 pipe; events order both streams around the
  // hand-over.  (In other precisions the two would share the FP32 copies of
  // the site tensors, so they run one after the other.)
  const bool concurrent = orth && c.krylov_fp64 && c.overlap_inner && m > 2;
  Context* hc = nullptr;
  struct Events {
    cudaEvent_t in = nullptr, out = nullptr;
    ~Events() {
      if (in) cudaEventDestroy(in);
      if (out) cudaEventDestroy(out);
    }
  } ev;
  if (concurrent) {
    if (!c.aux) c.aux = std::make_unique<Worker>(TDMPS_FP64, (size_t)32 << 20);
    hc = c.aux->c.get();
    hc->precision = c.precision;
    hc->stats = c.stats;
    TD_CHECK_CUDA(cudaEventCreateWithFlags(&ev.in, cudaEventDisableTiming));
    TD_CHECK_CUDA(cudaEventCreateWithFlags(&ev.out, cudaEventDisableTiming));
  }
  for (int k = 0; k + 1 < m; ++k) {
    if (orth) {
      // Eq. (kry_orth): c_j = <phi_j|H|phi_k> / <phi_j|phi_j>; the overlaps
      // <phi_j|phi_k> of the Krylov matrix N are formed here too
      std::vector<std::pair<const MPSd*, const MPSd*>> pn, ph;
      std::vector<double2*> on, oh;
      for (int j = 0; j <= k; ++j) {
        if (!haveH[j * m + k]) { ph.push_back({&phi[j], &phi[k]}); oh.push_back(Hd + j * m + k); haveH[j * m + k] = 1; }
        if (!haveN[j * m + k]) { pn.push_back({&phi[j], &phi[k]}); on.push_back(Nd + j * m + k); haveN[j * m + k] = 1; }
      }
      MPSd u;
      if (concurrent) {
        TD_CHECK_CUDA(cudaEventRecord(ev.in, c.st));
        TD_CHECK_CUDA(cudaStreamWaitEvent(hc->st, ev.in, 0));
        std::exception_ptr err;
        const int dev = c.device;
        std::thread th([&, dev] {
          try {
            TD_CHECK_CUDA(cudaSetDevice(dev));
            hc->api_enter();
            sandwich_batch(*hc, &H, ph, oh, true);
            sandwich_batch(*hc, nullptr, pn, on, true);
          } catch (...) {
            err = std::current_exception();
          }
        });
        try {
          u = fit(c, {{&phi[k], &H, 1.0}}, phi[k], o);
        } catch (...) {
          th.join();
          throw;
        }
        th.join();
        if (err) std::rethrow_exception(err);
        TD_CHECK_CUDA(cudaEventRecord(ev.out, hc->st));
        TD_CHECK_CUDA(cudaStreamWaitEvent(c.st, ev.out, 0));
      } else {
        u = fit(c, {{&phi[k], &H, 1.0}}, phi[k], o);
        sandwich_batch(c, &H, ph, oh, c.krylov_fp64);
        sandwich_batch(c, nullptr, pn, on, c.krylov_fp64);
      }
      DevPtr cj = dev_alloc(sizeof(double2) * (k + 1), c.st);
      std::vector<FitTerm> terms;
      terms.push_back({&u, nullptr, 1.0});
      for (int j = 0; j <= k; ++j) {
        launch_scalar_div_neg(Hd + j * m + k, Nd + j * m + j, (double2*)cj->p + j, c.st);
        terms.push_back({&phi[j], nullptr, 1.0, (double2*)cj->p + j});
      }
      MPSd v = fit(c, terms, u, o);
      normalize_center(c, v, nullptr);
      phi.push_back(std::move(v));
    } else {
      MPSd u = fit(c, {{&phi[k], &H, 1.0}}, phi[k], o);
      normalize_center(c, u, nullptr);
      phi.push_back(std::move(u));
    }
  }
  if (hc && c.stats) {   // the helper's timings and work count as this context's
    hc->collect_stats();
    for (int q = 0; q < TDMPS_KSTAT_COUNT; ++q) {
      if (q == TDMPS_KSTAT_HOST_PLAN || q == TDMPS_KSTAT_HOST_LAUNCH) {
        hc->kstat[q] = KStat();   // host time of the helper thread overlaps this thread's
        continue;
      }
      c.kstat[q].launches += hc->kstat[q].launches;
      c.kstat[q].ms += hc->kstat[q].ms;
      c.kstat[q].flops += hc->kstat[q].flops;
      c.kstat[q].bytes += hc->kstat[q].bytes;
      hc->kstat[q] = KStat();
    }
  }
  std::vector<std::pair<int, int>> rest;
  for (int i = 0; i < m; ++i)
    for (int j = i; j < m; ++j) rest.push_back({i, j});
  fill(rest, true);
  int* st = (int*)c.status->p + 4;
  launch_krylov_small(Nd, Hd, m, dt, cd, st, c.st);
  int hs[2];
  TD_CHECK_CUDA(cudaMemcpyAsync(hs, st, sizeof(hs), cudaMemcpyDeviceToHost, c.st));
  c.sync();
  if (hs[1]) throw Error(TDMPS_ERR_NONFINITE, "non-finite Krylov matrices");
  if (m - hs[0] < 2) throw Error(TDMPS_ERR_KRYLOV_SINGULAR, "Krylov overlap matrix has rank < 2");
  std::vector<FitTerm> terms;
  for (int k = 0; k < m; ++k) terms.push_back({&phi[k], nullptr, 1.0, cd + k});
  // the step's result sum_j c_j |phi_j> is part of the Krylov algebra: with
  // FP64 inner products it is fitted in FP64 too (it is one of the 2m - 1
  // fits of the step, and the only one whose errors reach the next step
  // directly); otherwise in the context precision with its scale restored
  MPSd out;
  if (c.krylov_fp64) {
    Fp64Scope fs(c, true);
    out = fit(c, terms, phi[0], o);
  } else {
    out = fit(c, terms, phi[0], o);
    restore_fit_scale(c, out, terms);
  }
  return out;
}

// ------------------------------------------------------------------ density matrices

// Readout operators of the density-matrix MPO: at bond j they close the open
// creator channels c+_{is} (i < j) and the identity channel with c_{js} on
// site j into one channel per (i, s), i <= j.
const std::vector<MPOd>& Context::rdm_readouts(int L) {
  if (rdm_read && (int)rdm_read->size() == L) return *rdm_read;
  const MPOd& G = rdm_mpo(L);
  auto v = std::make_unique<std::vector<MPOd>>(L);
  for (int j = 0; j < L; ++j) {
    MPOd& R = (*v)[j];
    R.L = 1;
    R.bonds.resize(2);
    R.bonds[0] = G.bonds[j];
    MPOBond& rb = R.bonds[1];
    rb.gq = {QN()};
    rb.gsize = {2 * (j + 1)};
    for (int w = 0; w < 2 * (j + 1); ++w) { rb.ch_group.push_back(0); rb.ch_local.push_back(w); }
    R.W.assign(1, {});
    // local matrices: c_up |u>->|0>, |ud>->|d>; c_down |d>->|0>, |ud>->-|u>
    for (int s = 0; s < 2; ++s) {
      // channel of c+_{i s} at bond j: down spins 1 + i, up spins 1 + j + i
      for (int i = 0; i < j; ++i) {
        int win = s == 1 ? 1 + i : 1 + j + i;
        int wout = 2 * i + s;
        if (s == 0) { R.W[0].push_back({win, wout, 0, 1, 1.0}); R.W[0].push_back({win, wout, 2, 3, 1.0}); }
        else { R.W[0].push_back({win, wout, 0, 2, 1.0}); R.W[0].push_back({win, wout, 1, 3, -1.0}); }
      }
      // diagonal: n_s on site j from the identity channel
      int wout = 2 * j + s;
      if (s == 0) { R.W[0].push_back({0, wout, 1, 1, 1.0}); R.W[0].push_back({0, wout, 3, 3, 1.0}); }
      else { R.W[0].push_back({0, wout, 2, 2, 1.0}); R.W[0].push_back({0, wout, 3, 3, 1.0}); }
    }
    upload_mpo_tables(R, *this);
  }
  rdm_read = std::move(v);
  return *rdm_read;
}

// out[j][2 i + s] += <bra| c+_{is} c_{js} |ket> for i <= j (device, FP64 in
// the caller's scope).  Left environments carry the open creator channels of
// the density-matrix MPO; at every bond j the readout closes them with c_{js}
// and the result is traced against the right overlap environment.
static void rdm_upper(Context& c, const MPSd& bra, const MPSd& ket, double2* out) {
  const int L = bra.L;
  const MPOd& I = c.identity_mpo(L);
  const MPOd& G = c.rdm_mpo(L);
  const std::vector<MPOd>& R = c.rdm_readouts(L);
  std::vector<Env> RO(L + 1);
  RO[L] = env_right_boundary(c, bra, ket, I);
  for (int i = L - 1; i >= 1; --i)
    RO[i] = env_update_right(c, RO[i + 1], bra.sites[i], bra.bonds[i], ket, i, I);
  Env E = env_left_boundary(c, bra, ket, G);
  for (int j = 0; j < L; ++j) {
    GemmBatch g1(c);
    Inter X = plan_lstage(c, E, ket.sites[j], ket.bonds[j + 1], g1);
    g1.run();
    WBatch wb;
    Inter Y = plan_wstage(c, std::move(X), R[j], 0, true, wb);
    wb.run(c);
    GemmBatch g2(c);
    Env Eo = plan_env_left(c, Y, bra.sites[j], bra.bonds[j + 1], R[j].bonds[1], ket.bonds[j + 1], g2);
    g2.run();
    for (int b = 0; b < (int)Eo.t.blocks.size(); ++b) {
      const Inter::Blk& eb = Eo.t.blocks[b];
      int rb2 = RO[j + 1].t.find(eb.rg, -1, 0, eb.k);
      if (rb2 < 0) continue;
      launch_trace_channels(Eo.t.ptr(b), eb.rows, eb.W, eb.cols, RO[j + 1].t.ptr(rb2), Eo.t.et,
                            out + (size_t)j * 2 * L, c.st);
    }
    TD_CHECK_CUDA(cudaGetLastError());
    if (j + 1 < L) E = env_update_left(c, E, bra.sites[j], bra.bonds[j + 1], ket, j, G);
  }
}

static void check_rdm_pair(const MPSd& bra, const MPSd& ket) {
  if (bra.L != ket.L) throw Error(TDMPS_ERR_INVALID_ARG, "MPS lengths differ");
  if (bra.tot != ket.tot) throw Error(TDMPS_ERR_SECTOR, "bra and ket have different (N, 2Sz)");
}

void one_rdm(Context& c, const MPSd& psi, cplx* gamma) {
  Fp64Scope fp64(c);
  const int L = psi.L;
  DevPtr gd = dev_alloc(sizeof(double2) * (size_t)L * 2 * L, c.st);   // [j][2*i + s]
  TD_CHECK_CUDA(cudaMemsetAsync(gd->p, 0, sizeof(double2) * (size_t)L * 2 * L, c.st));
  rdm_upper(c, psi, psi, (double2*)gd->p);
  std::vector<double2> h((size_t)L * 2 * L);
  TD_CHECK_CUDA(cudaMemcpyAsync(h.data(), gd->p, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, c.st));
  c.sync();
  for (int i = 0; i < L * L; ++i) gamma[i] = 0.0;
  for (int j = 0; j < L; ++j)
    for (int i = 0; i <= j; ++i)
      for (int s = 0; s < 2; ++s) {
        double2 v = h[(size_t)j * 2 * L + 2 * i + s];
        gamma[i * L + j] += cplx(v.x, v.y);
      }
  for (int j = 0; j < L; ++j)
    for (int i = 0; i < j; ++i) gamma[j * L + i] = std::conj(gamma[i * L + j]);
}

void transition_rdm(Context& c, const MPSd& bra, const MPSd& ket, cplx* T) {
  check_rdm_pair(bra, ket);
  Fp64Scope fp64(c);
  const int L = bra.L;
  const size_t n = (size_t)L * 2 * L;
  DevPtr gd = dev_alloc(sizeof(double2) * 2 * n, c.st);
  TD_CHECK_CUDA(cudaMemsetAsync(gd->p, 0, sizeof(double2) * 2 * n, c.st));
  // upper triangle from <bra|..|ket>, lower from the conjugate of <ket|..|bra>
  rdm_upper(c, bra, ket, (double2*)gd->p);
  rdm_upper(c, ket, bra, (double2*)gd->p + n);
  std::vector<double2> h(2 * n);
  TD_CHECK_CUDA(cudaMemcpyAsync(h.data(), gd->p, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, c.st));
  c.sync();
  for (int i = 0; i < L * L; ++i) T[i] = 0.0;
  for (int j = 0; j < L; ++j)
    for (int i = 0; i <= j; ++i)
      for (int s = 0; s < 2; ++s) {
        double2 u = h[(size_t)j * 2 * L + 2 * i + s];
        T[i * L + j] += cplx(u.x, u.y);
        if (i < j) {
          double2 v = h[n + (size_t)j * 2 * L + 2 * i + s];
          T[j * L + i] += cplx(v.x, -v.y);
        }
      }
}

// Gamma_ijkl = sum_{s,t} <psi| c+_is c+_kt c_lt c_js |psi>
//            = sum_s T[c_is psi, c_js psi]_kl
// with T the spin-summed transition 1BRDM of the two ionised states.
void two_rdm(Context& c, const MPSd& psi, cplx* Gam) {
  Fp64Scope fp64(c);
  const int L = psi.L;
  const size_t L2 = (size_t)L * L, n = (size_t)L * 2 * L;
  for (size_t e = 0; e < L2 * L2; ++e) Gam[e] = 0.0;
  for (int s = 0; s < 2; ++s) {
    std::vector<MPSd> chi(L);
    std::vector<char> nz(L, 0);
    for (int i = 0; i < L; ++i) nz[i] = apply_site_op(c, psi, i, s, false, chi[i]);
    DevPtr gd = dev_alloc(sizeof(double2) * L2 * n, c.st);   // [(i, j)][l][2 k + t]
    TD_CHECK_CUDA(cudaMemsetAsync(gd->p, 0, sizeof(double2) * L2 * n, c.st));
    for (int i = 0; i < L; ++i)
      for (int j = 0; j < L; ++j)
        if (nz[i] && nz[j]) rdm_upper(c, chi[i], chi[j], (double2*)gd->p + ((size_t)i * L + j) * n);
    std::vector<double2> h(L2 * n);
    TD_CHECK_CUDA(cudaMemcpyAsync(h.data(), gd->p, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, c.st));
    c.sync();
    auto at = [&](int i, int j, int k, int l) {   // <chi_i| c+_k c_l |chi_j>, k <= l, spin-summed
      const double2* g = h.data() + ((size_t)i * L + j) * n + (size_t)l * 2 * L + 2 * k;
      return cplx(g[0].x + g[1].x, g[0].y + g[1].y);
    };
    for (int i = 0; i < L; ++i)
      for (int j = 0; j < L; ++j)
        for (int k = 0; k < L; ++k)
          for (int l = 0; l < L; ++l) {
            cplx v = k <= l ? at(i, j, k, l) : std::conj(at(j, i, l, k));
            Gam[((size_t)i * L + j) * L2 + (size_t)k * L + l] += v;
          }
  }
}

// ------------------------------------------------------------------ Green's function

// Eq. (green_time) for tau = n dt, n = 0..n_steps:
//   G_ij(tau) = -i sum_s <psi0| c+_is exp(+i H tau) c_js |psi0>
//                  / sum_s <psi0| c+_is c_js |psi0>,
// evaluated as the paper does: ionise exactly (c_js|psi0>), propagate the
// ionised state backwards in time with the integrator (time step -dt) and
// project on c_is|psi0> after every step.  Overlaps in FP64.
void green_function(Context& c, const MPOd& H, const MPSd& psi0, int i, int j, double dt,
                    int n_steps, int method, int m, bool orth, const FitOpts& o, cplx* G) {
  if (n_steps < 0) throw Error(TDMPS_ERR_INVALID_ARG, "n_steps must be >= 0");
  if (method != 0 && method != 1) throw Error(TDMPS_ERR_INVALID_ARG, "method must be 0 (Krylov) or 1 (RK4)");
  std::vector<cplx> num(n_steps + 1, 0.0);
  cplx den = 0.0;
  for (int s = 0; s < 2; ++s) {
    MPSd chi_i, chi;
    bool nzi = apply_site_op(c, psi0, i, s, false, chi_i);
    bool nzj = apply_site_op(c, psi0, j, s, false, chi);
    if (!nzi || !nzj) continue;
    cplx ov = sandwich(c, nullptr, chi_i, chi);
    den += ov;
    num[0] += ov;
    for (int n = 0; n < n_steps; ++n) {
      chi = method == 0 ? krylov_step(c, H, chi, -dt, m, orth, o) : rk4_step(c, H, chi, -dt, o);
      num[n + 1] += sandwich(c, nullptr, chi_i, chi);
    }
  }
  if (den == 0.0)
    throw Error(TDMPS_ERR_ZERO_STATE, "sum_s <psi0|c+_is c_js|psi0> vanishes");
  for (int n = 0; n <= n_steps; ++n) G[n] = cplx(0.0, -1.0) * num[n] / den;
}

// ------------------------------------------------------------------ site operators

// a_(site, spin)|in> or a+_(site, spin)|in>: a product operator (bond
// dimension one) -- the parity (-1)^n on every earlier site (Jordan-Wigner
// string over the spin orbitals before it), the local matrix on `site`, the
// identity after it.  Bonds right of `site` shift their charges by the
// operator's, which keeps their sector order.  Returns false when no block
// survives (the state is exactly zero).
bool apply_site_op(Context& c, const MPSd& in, int site, int spin, bool dagger, MPSd& out) {
  if (site < 0 || site >= in.L) throw Error(TDMPS_ERR_INVALID_ARG, "site out of range");
  if (spin < 0 || spin > 1) throw Error(TDMPS_ERR_INVALID_ARG, "spin must be 0 (up) or 1 (down)");
  const QN dq = dagger ? SITE_Q[1 + spin] : -SITE_Q[1 + spin];
  out = MPSd();
  out.L = in.L;
  out.tot = in.tot + dq;
  out.bonds = in.bonds;
  for (int k = site + 1; k <= in.L; ++k)
    for (auto& q : out.bonds[k].q) q = q + dq;
  const int bit = 1 << spin;
  std::vector<CopyTask> tasks;
  auto copy_block = [&](const SiteT& a, int b, const SiteT& o, int ob, double sign) {
    if (ob < 0 || o.blocks[ob].rows != a.blocks[b].rows || o.blocks[ob].cols != a.blocks[b].cols)
      throw Error(TDMPS_ERR_SECTOR, "site tensor blocks do not match their bonds");
    CopyTask t{};
    size_t n = (size_t)a.blocks[b].rows * a.blocks[b].cols;
    if (n > (size_t)INT32_MAX) throw Error(TDMPS_ERR_INVALID_ARG, "block too large");
    t.blk = a.ptr(b);
    t.work = o.ptr(ob);
    t.rows = 1;
    t.cols = (int)n;
    t.ld = (int)n;
    t.ldw = 1;
    t.scale = make_double2(sign, 0.0);
    tasks.push_back(t);
  };
  bool any = false;
  for (int k = 0; k < in.L; ++k) {
    const SiteT& a = in.sites[k];
    SiteT o = make_site(RowGroups::from_bond(out.bonds[k]), out.bonds[k + 1], c.st, k == site);
    for (int b = 0; b < (int)a.blocks.size(); ++b) {
      const SiteT::Blk& ab = a.blocks[b];
      if (k != site) {
        double sign = (k < site && (ab.sig == 1 || ab.sig == 2)) ? -1.0 : 1.0;
        copy_block(a, b, o, o.block_of(ab.r, ab.sig), sign);
      } else {
        bool occupied = (ab.sig & bit) != 0;
        if (occupied == dagger) continue;   // annihilated local state
        // the down operator passes the up creator of the same site
        double sign = (spin == 1 && (ab.sig & 1)) ? -1.0 : 1.0;
        copy_block(a, b, o, o.block_of(ab.r, ab.sig ^ bit), sign);
        any = true;
      }
    }
    out.sites.push_back(std::move(o));
  }
  if (!tasks.empty()) {
    const CopyTask* d = c.stage(tasks);
    cudaEvent_t ev;
    c.kbegin(TDMPS_KSTAT_OTHER, &ev);
    launch_copy(d, (int)tasks.size(), 1, c.st);
    TD_CHECK_CUDA(cudaGetLastError());
    double bytes = 0.0;
    for (auto& t : tasks) bytes += 32.0 * t.cols;
    c.kend(TDMPS_KSTAT_OTHER, ev, 0.0, bytes);
  }
  return any;
}

// ------------------------------------------------------------------ MPS creation

MPSd mps_determinant(Context& c, int L, const uint8_t* occ) {
  if (L < 1 || L > 63) throw Error(TDMPS_ERR_INVALID_ARG, "L must be in [1, 63]");
  MPSd m;
  m.L = L;
  m.bonds.resize(L + 1);
  m.bonds[0].q = {QN()};
  m.bonds[0].d = {1};
  QN q;
  for (int i = 0; i < L; ++i) {
    if (occ[i] > 3) throw Error(TDMPS_ERR_INVALID_ARG, "occupation codes must be 0..3");
    q = q + SITE_Q[occ[i]];
    m.bonds[i + 1].q = {q};
    m.bonds[i + 1].d = {1};
  }
  m.tot = q;
  std::vector<double2> ones(L, make_double2(1.0, 0.0));
  for (int i = 0; i < L; ++i) {
    m.sites.push_back(make_site(RowGroups::from_bond(m.bonds[i]), m.bonds[i + 1], c.st, false));
    TD_CHECK_CUDA(cudaMemcpyAsync(m.sites[i].data->p, c.stage(&ones[i], sizeof(double2)),
                                  sizeof(double2), cudaMemcpyDeviceToDevice, c.st));
  }
  m.rcanon = true;   // every site is a single unit entry
  return m;
}

MPSd mps_import(Context& c, int L, const int* bond_dims, const int* labels,
                const tdmps_complex* const* tensors) {
  if (L < 1 || L > 63) throw Error(TDMPS_ERR_INVALID_ARG, "L must be in [1, 63]");
  MPSd m;
  m.L = L;
  m.bonds.resize(L + 1);
  // per bond: map basis index -> (sector, position)
  std::vector<std::vector<std::pair<int, int>>> where(L + 1);
  const int* lab = labels;
  for (int k = 0; k <= L; ++k) {
    int D = bond_dims[k];
    if (D < 1) throw Error(TDMPS_ERR_INVALID_ARG, "bond dimensions must be >= 1");
    std::map<QN, int> cnt;
    std::vector<QN> qv(D);
    for (int x = 0; x < D; ++x) { qv[x] = QN(lab[2 * x], lab[2 * x + 1]); cnt[qv[x]]++; }
    lab += 2 * D;
    for (auto& kv : cnt) { m.bonds[k].q.push_back(kv.first); m.bonds[k].d.push_back(kv.second); }
    std::vector<int> pos(m.bonds[k].nsec(), 0);
    where[k].resize(D);
    for (int x = 0; x < D; ++x) {
      int s = m.bonds[k].find(qv[x]);
      where[k][x] = {s, pos[s]++};
    }
  }
  if (m.bonds[0].nsec() != 1 || m.bonds[0].q[0] != QN() || m.bonds[0].d[0] != 1)
    throw Error(TDMPS_ERR_INVALID_ARG, "bond 0 must be one-dimensional with label (0, 0)");
  if (m.bonds[L].nsec() != 1 || m.bonds[L].d[0] != 1)
    throw Error(TDMPS_ERR_SECTOR, "bond L must be one-dimensional");
  m.tot = m.bonds[L].q[0];
  for (int i = 0; i < L; ++i) {
    SiteT t = make_site(RowGroups::from_bond(m.bonds[i]), m.bonds[i + 1], c.st, false);
    std::vector<double2> h(t.size);
    int Dl = bond_dims[i], Dr = bond_dims[i + 1];
    const tdmps_complex* A = tensors[i];
    for (int a = 0; a < Dl; ++a)
      for (int s = 0; s < 4; ++s)
        for (int b = 0; b < Dr; ++b) {
          tdmps_complex v = A[((size_t)a * 4 + s) * Dr + b];
          if (!std::isfinite(v.re) || !std::isfinite(v.im))
            throw Error(TDMPS_ERR_NONFINITE, "MPS tensor contains NaN/Inf");
          int sa = where[i][a].first, sb = where[i + 1][b].first;
          int blk = t.block_of(sa, s);
          if (blk < 0 || t.blocks[blk].sb != sb) {
            if (v.re != 0.0 || v.im != 0.0)
              throw Error(TDMPS_ERR_INVALID_ARG, "non-zero entry violates charge conservation");
            continue;
          }
          const SiteT::Blk& bl = t.blocks[blk];
          h[bl.off + (size_t)where[i][a].second * bl.cols + where[i + 1][b].second] =
              make_double2(v.re, v.im);
        }
    if (t.size)
      TD_CHECK_CUDA(cudaMemcpyAsync(t.data->p, h.data(), t.size * sizeof(double2),
                                    cudaMemcpyHostToDevice, c.st));
    TD_CHECK_CUDA(cudaStreamSynchronize(c.st));
    m.sites.push_back(std::move(t));
  }
  return m;
}

void mps_export(Context& c, const MPSd& m, int* bond_dims, int* labels, tdmps_complex* const* tensors) {
  for (int k = 0; k <= m.L; ++k) bond_dims[k] = m.bonds[k].total();
  if (!tensors) return;
  int* lab = labels;
  for (int k = 0; k <= m.L; ++k)
    for (int s = 0; s < m.bonds[k].nsec(); ++s)
      for (int x = 0; x < m.bonds[k].d[s]; ++x) { *lab++ = m.bonds[k].q[s].n; *lab++ = m.bonds[k].q[s].s; }
  for (int i = 0; i < m.L; ++i) {
    const SiteT& t = m.sites[i];
    std::vector<double2> h(t.size);
    if (t.size)
      TD_CHECK_CUDA(cudaMemcpyAsync(h.data(), t.data->p, t.size * sizeof(double2),
                                    cudaMemcpyDeviceToHost, c.st));
    TD_CHECK_CUDA(cudaStreamSynchronize(c.st));
    int Dl = bond_dims[i], Dr = bond_dims[i + 1];
    std::vector<int> offl(m.bonds[i].nsec() + 1, 0), offr(m.bonds[i + 1].nsec() + 1, 0);
    for (int s = 0; s < m.bonds[i].nsec(); ++s) offl[s + 1] = offl[s] + m.bonds[i].d[s];
    for (int s = 0; s < m.bonds[i + 1].nsec(); ++s) offr[s + 1] = offr[s] + m.bonds[i + 1].d[s];
    tdmps_complex* A = tensors[i];
    for (size_t e = 0; e < (size_t)Dl * 4 * Dr; ++e) A[e] = {0.0, 0.0};
    for (auto& bl : t.blocks)
      for (int a = 0; a < bl.rows; ++a)
        for (int b = 0; b < bl.cols; ++b) {
          double2 v = h[bl.off + (size_t)a * bl.cols + b];
          A[((size_t)(offl[bl.r] + a) * 4 + bl.sig) * Dr + offr[bl.sb] + b] = {v.x, v.y};
        }
  }
}

MPSd mps_copy(Context& c, const MPSd& m) {
  MPSd o = m;
  for (int i = 0; i < m.L; ++i) {
    o.sites[i].data = dev_alloc(std::max<size_t>(m.sites[i].size, 1) * sizeof(double2), c.st);
    if (m.sites[i].size)
      TD_CHECK_CUDA(cudaMemcpyAsync(o.sites[i].data->p, m.sites[i].data->p,
                                    m.sites[i].size * sizeof(double2), cudaMemcpyDeviceToDevice, c.st));
  }
  return o;
}

}  // namespace tdmps
