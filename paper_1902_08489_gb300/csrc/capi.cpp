// extern "C" boundary of the tdmps library (declared in include/tdmps.h).
#include <cmath>
#include <cstring>
#include <memory>
#include <string>

#include "engine.hpp"

using namespace tdmps;

struct tdmps_ctx_s {
  std::unique_ptr<Context> c;
};
struct tdmps_mpo_s {
  MPOd m;
  int n_elec = 0;
  bool uploaded = false;
};
struct tdmps_mps_s {
  MPSd m;
};
struct tdmps_heff_s {
  std::unique_ptr<LocalOp> op;
};

namespace {

thread_local std::string g_create_err;

template <class F>
int guard(tdmps_ctx_t ctx, F&& f) {
  try {
    if (ctx) ctx->c->api_enter();
    f();
    if (ctx) ctx->c->err.clear();
    return TDMPS_OK;
  } catch (const Error& e) {
    if (ctx) ctx->c->err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->c->err = "host allocation failed";
    return TDMPS_ERR_OOM;
  } catch (const std::exception& e) {
    if (ctx) ctx->c->err = e.what();
    return TDMPS_ERR_INVALID_ARG;
  }
}

void need(bool cond, const char* msg) {
  if (!cond) throw Error(TDMPS_ERR_INVALID_ARG, msg);
}

// A scalar input that must be finite (NaN or Inf -> TDMPS_ERR_NONFINITE).
void need_finite(double x, const char* msg) {
  if (!std::isfinite(x)) throw Error(TDMPS_ERR_NONFINITE, msg);
}

void ensure_uploaded(tdmps_ctx_t ctx, tdmps_mpo_t mpo) {
  if (!mpo->uploaded) {
    upload_mpo_tables(mpo->m, *ctx->c);
    mpo->uploaded = true;
  }
}

FitOpts opts(tdmps_ctx_t ctx, int D, double eps) {
  need(D >= 1, "D must be >= 1");
  need(eps >= 0.0 && eps < 1.0, "eps must be in [0, 1)");
  FitOpts o;
  o.D = D;
  o.eps = eps;
  o.n_two_site = ctx->c->n_two_site;
  o.n_one_site = ctx->c->n_one_site;
  return o;
}

}  // namespace

extern "C" {

int tdmps_create(tdmps_ctx_t* ctx, void* cuda_stream, int precision) {
  if (!ctx) { g_create_err = "ctx is NULL"; return TDMPS_ERR_INVALID_ARG; }
  if (precision < TDMPS_FP64 || precision > TDMPS_BF16) {
    g_create_err = "unknown precision";
    return TDMPS_ERR_INVALID_ARG;
  }
  try {
    auto* h = new tdmps_ctx_s;
    h->c.reset(new Context((cudaStream_t)cuda_stream, precision));
    *ctx = h;
    g_create_err.clear();
    return TDMPS_OK;
  } catch (const Error& e) {
    g_create_err = e.what();
    return e.code;
  } catch (const std::exception& e) {
    g_create_err = e.what();
    return TDMPS_ERR_CUDA;
  }
}

int tdmps_destroy(tdmps_ctx_t ctx) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  delete ctx;
  return TDMPS_OK;
}

const char* tdmps_last_error(tdmps_ctx_t ctx) { return ctx ? ctx->c->err.c_str() : ""; }
const char* tdmps_create_error(void) { return g_create_err.c_str(); }

int tdmps_set_precision(tdmps_ctx_t ctx, int precision) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(precision >= TDMPS_FP64 && precision <= TDMPS_BF16, "unknown precision");
    ctx->c->precision = precision;
  });
}

int tdmps_set_schedule(tdmps_ctx_t ctx, int n_two_site, int n_one_site) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(n_two_site >= 0 && n_one_site >= 0 && n_two_site + n_one_site >= 1, "invalid schedule");
    ctx->c->n_two_site = n_two_site;
    ctx->c->n_one_site = n_one_site;
  });
}

int tdmps_set_krylov_fp64(tdmps_ctx_t ctx, int on) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  ctx->c->krylov_fp64 = on != 0;
  return TDMPS_OK;
}

int tdmps_set_concurrent_inner(tdmps_ctx_t ctx, int on) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  ctx->c->overlap_inner = on != 0;
  return TDMPS_OK;
}

int tdmps_build_mpo(tdmps_ctx_t ctx, const double* h, const double* eri, int L, int n_elec,
                    double e0, tdmps_mpo_t* out) {
  return guard(ctx, [&] {
    need(out && h && eri, "NULL argument");
    need(L >= 1 && L <= 63, "L must be in [1, 63]");
    need(n_elec >= 0 && n_elec <= 2 * L, "n_elec must be in [0, 2L]");
    auto* m = new tdmps_mpo_s;
    try {
      m->m = build_qc_mpo(h, eri, L, e0);
      m->n_elec = n_elec;
      if (ctx) ensure_uploaded(ctx, m);
    } catch (...) {
      delete m;
      throw;
    }
    *out = m;
  });
}

int tdmps_mpo_info(tdmps_mpo_t mpo, int* bond_dims, int64_t* n_elements) {
  if (!mpo) return TDMPS_ERR_INVALID_ARG;
  if (bond_dims)
    for (int k = 0; k <= mpo->m.L; ++k) bond_dims[k] = mpo->m.bonds[k].nch();
  if (n_elements) *n_elements = mpo->m.n_elem;
  return TDMPS_OK;
}

int tdmps_mpo_elements(tdmps_mpo_t mpo, int site, int64_t* count, int* win, int* wout, int* sig,
                       int* sigp, double* v) {
  if (!mpo || site < 0 || site >= mpo->m.L || !count) return TDMPS_ERR_INVALID_ARG;
  const auto& W = mpo->m.W[site];
  if (win) {
    if (!wout || !sig || !sigp || !v) return TDMPS_ERR_INVALID_ARG;
    if (*count < (int64_t)W.size()) {
      *count = (int64_t)W.size();
      return TDMPS_ERR_INVALID_ARG;
    }
    for (size_t e = 0; e < W.size(); ++e) {
      win[e] = W[e].win;
      wout[e] = W[e].wout;
      sig[e] = W[e].sig;
      sigp[e] = W[e].sigp;
      v[e] = W[e].v;
    }
  }
  *count = (int64_t)W.size();
  return TDMPS_OK;
}

int tdmps_mpo_free(tdmps_mpo_t mpo) {
  delete mpo;
  return TDMPS_OK;
}

int tdmps_mps_from_determinant(tdmps_ctx_t ctx, int L, const uint8_t* occ, tdmps_mps_t* out) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(out && occ, "NULL argument");
    auto* m = new tdmps_mps_s;
    try { m->m = mps_determinant(*ctx->c, L, occ); } catch (...) { delete m; throw; }
    *out = m;
  });
}

int tdmps_mps_import(tdmps_ctx_t ctx, int L, const int* bond_dims, const int* labels,
                     const tdmps_complex* const* tensors, tdmps_mps_t* out) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(out && bond_dims && labels && tensors, "NULL argument");
    auto* m = new tdmps_mps_s;
    try { m->m = mps_import(*ctx->c, L, bond_dims, labels, tensors); } catch (...) { delete m; throw; }
    *out = m;
  });
}

int tdmps_mps_export(tdmps_ctx_t ctx, tdmps_mps_t mps, int* bond_dims, int* labels,
                     tdmps_complex* const* tensors) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(mps && bond_dims, "NULL argument");
    need(!tensors || labels, "labels must be given with tensors");
    mps_export(*ctx->c, mps->m, bond_dims, labels, tensors);
  });
}

int tdmps_mps_info(tdmps_mps_t mps, int* L, int* n_elec, int* two_sz, int* max_bond) {
  if (!mps) return TDMPS_ERR_INVALID_ARG;
  if (L) *L = mps->m.L;
  if (n_elec) *n_elec = mps->m.tot.n;
  if (two_sz) *two_sz = mps->m.tot.s;
  if (max_bond) {
    int mb = 0;
    for (auto& b : mps->m.bonds) mb = std::max(mb, b.total());
    *max_bond = mb;
  }
  return TDMPS_OK;
}

int tdmps_mps_copy(tdmps_ctx_t ctx, tdmps_mps_t in, tdmps_mps_t* out) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(in && out, "NULL argument");
    auto* m = new tdmps_mps_s;
    m->m = mps_copy(*ctx->c, in->m);
    *out = m;
  });
}

int tdmps_mps_free(tdmps_mps_t mps) {
  delete mps;
  return TDMPS_OK;
}

int tdmps_apply_H(tdmps_ctx_t ctx, tdmps_mpo_t mpo, tdmps_mps_t in, tdmps_complex alpha, int D,
                  double eps, int n_sweeps, tdmps_mps_t* out) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(mpo && in && out, "NULL argument");
    need(mpo->m.L == in->m.L, "MPO and MPS lengths differ");
    need_finite(alpha.re, "alpha must be finite");
    need_finite(alpha.im, "alpha must be finite");
    ensure_uploaded(ctx, mpo);
    FitOpts o = opts(ctx, D, eps);
    if (n_sweeps > 0) o.n_one_site = n_sweeps;
    auto* r = new tdmps_mps_s;
    try {
      r->m = fit(*ctx->c, {{&in->m, &mpo->m, cplx(alpha.re, alpha.im)}}, in->m, o);
    } catch (...) { delete r; throw; }
    *out = r;
  });
}

int tdmps_energy_gradient(tdmps_ctx_t ctx, tdmps_mpo_t mpo, tdmps_mps_t psi, int stride,
                          double* energy, tdmps_mps_t* grad, size_t* env_bytes_peak) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(mpo && psi && grad, "NULL argument");
    need(mpo->m.L == psi->m.L, "MPO and MPS lengths differ");
    need(stride >= 1, "stride must be >= 1");
    ensure_uploaded(ctx, mpo);
    auto* r = new tdmps_mps_s;
    try {
      r->m = energy_gradient(*ctx->c, mpo->m, psi->m, stride, energy, env_bytes_peak);
    } catch (...) {
      delete r;
      throw;
    }
    *grad = r;
  });
}

int tdmps_heff_create(tdmps_ctx_t ctx, tdmps_mpo_t mpo, tdmps_mps_t psi, int site,
                      tdmps_heff_t* out, size_t* env_bytes) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(mpo && psi && out, "NULL argument");
    need(mpo->m.L == psi->m.L, "MPO and MPS lengths differ");
    need(site >= 0 && site < psi->m.L, "site out of range");
    ensure_uploaded(ctx, mpo);
    auto* r = new tdmps_heff_s;
    try {
      r->op = local_op_create(*ctx->c, mpo->m, psi->m, site);
    } catch (...) {
      delete r;
      throw;
    }
    if (env_bytes) *env_bytes = r->op->env_bytes;
    *out = r;
  });
}

int tdmps_heff_apply(tdmps_ctx_t ctx, tdmps_heff_t op, tdmps_mps_t x, tdmps_mps_t y) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(op && x && y, "NULL argument");
    local_op_apply(*ctx->c, *op->op, x->m, y->m);
  });
}

int tdmps_heff_free(tdmps_heff_t op) {
  delete op;
  return TDMPS_OK;
}

int tdmps_sum(tdmps_ctx_t ctx, int n_terms, const tdmps_complex* coefs, const tdmps_mps_t* terms,
              int D, double eps, tdmps_mps_t* out) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(n_terms >= 1 && coefs && terms && out, "invalid arguments");
    std::vector<FitTerm> ft;
    for (int k = 0; k < n_terms; ++k) {
      need(terms[k] != nullptr, "NULL term");
      ft.push_back({&terms[k]->m, nullptr, cplx(coefs[k].re, coefs[k].im)});
    }
    FitOpts o = opts(ctx, D, eps);
    auto* r = new tdmps_mps_s;
    try {
      r->m = fit(*ctx->c, ft, terms[0]->m, o);
      restore_fit_scale(*ctx->c, r->m, ft);
    } catch (...) {
      delete r;
      throw;
    }
    *out = r;
  });
}

int tdmps_overlap(tdmps_ctx_t ctx, tdmps_mps_t bra, tdmps_mps_t ket, tdmps_complex* out) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(bra && ket && out, "NULL argument");
    cplx v = sandwich(*ctx->c, nullptr, bra->m, ket->m);
    out->re = v.real();
    out->im = v.imag();
  });
}

int tdmps_overlap_noalloc(tdmps_ctx_t ctx, tdmps_mps_t bra, tdmps_mps_t ket, tdmps_complex* out) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(bra && ket && out, "NULL argument");
    cplx v = overlap_noalloc(*ctx->c, bra->m, ket->m);
    out->re = v.real();
    out->im = v.imag();
  });
}

int tdmps_expectation(tdmps_ctx_t ctx, tdmps_mpo_t mpo, tdmps_mps_t bra, tdmps_mps_t ket,
                      tdmps_complex* out) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(mpo && bra && ket && out, "NULL argument");
    need(mpo->m.L == bra->m.L, "MPO and MPS lengths differ");
    ensure_uploaded(ctx, mpo);
    cplx v = sandwich(*ctx->c, &mpo->m, bra->m, ket->m);
    out->re = v.real();
    out->im = v.imag();
  });
}

int tdmps_compress(tdmps_ctx_t ctx, tdmps_mps_t inout, int D, double eps, double* discarded_weight) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(inout != nullptr, "NULL argument");
    need(D >= 1, "D must be >= 1");
    need(eps >= 0.0 && eps < 1.0, "eps must be in [0, 1)");
    MPSd m = inout->m;
    double d = compress(*ctx->c, m, D, eps);
    inout->m = std::move(m);
    if (discarded_weight) *discarded_weight = d;
  });
}

int tdmps_rk4_step(tdmps_ctx_t ctx, tdmps_mpo_t mpo, tdmps_mps_t inout, double dt, int D, double eps) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(mpo && inout, "NULL argument");
    need(mpo->m.L == inout->m.L, "MPO and MPS lengths differ");
    need_finite(dt, "dt must be finite");
    ensure_uploaded(ctx, mpo);
    FitOpts o = opts(ctx, D, eps);
    MPSd r = rk4_step(*ctx->c, mpo->m, inout->m, dt, o);
    inout->m = std::move(r);
  });
}

int tdmps_krylov_step(tdmps_ctx_t ctx, tdmps_mpo_t mpo, tdmps_mps_t inout, double dt, int m,
                      int orthogonal, int D, double eps) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(mpo && inout, "NULL argument");
    need(mpo->m.L == inout->m.L, "MPO and MPS lengths differ");
    need_finite(dt, "dt must be finite");
    ensure_uploaded(ctx, mpo);
    FitOpts o = opts(ctx, D, eps);
    MPSd r = krylov_step(*ctx->c, mpo->m, inout->m, dt, m, orthogonal != 0, o);
    inout->m = std::move(r);
  });
}

int tdmps_one_rdm(tdmps_ctx_t ctx, tdmps_mps_t psi, tdmps_complex* gamma) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(psi && gamma, "NULL argument");
    std::vector<cplx> g((size_t)psi->m.L * psi->m.L);
    one_rdm(*ctx->c, psi->m, g.data());
    for (size_t i = 0; i < g.size(); ++i) gamma[i] = {g[i].real(), g[i].imag()};
  });
}

int tdmps_transition_rdm(tdmps_ctx_t ctx, tdmps_mps_t bra, tdmps_mps_t ket, tdmps_complex* T) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(bra && ket && T, "NULL argument");
    std::vector<cplx> g((size_t)bra->m.L * bra->m.L);
    transition_rdm(*ctx->c, bra->m, ket->m, g.data());
    for (size_t i = 0; i < g.size(); ++i) T[i] = {g[i].real(), g[i].imag()};
  });
}

int tdmps_two_rdm(tdmps_ctx_t ctx, tdmps_mps_t psi, tdmps_complex* Gamma) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(psi && Gamma, "NULL argument");
    size_t L2 = (size_t)psi->m.L * psi->m.L;
    std::vector<cplx> g(L2 * L2);
    two_rdm(*ctx->c, psi->m, g.data());
    for (size_t i = 0; i < g.size(); ++i) Gamma[i] = {g[i].real(), g[i].imag()};
  });
}

int tdmps_energy(tdmps_ctx_t ctx, tdmps_mpo_t mpo, tdmps_mps_t psi, double* energy) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(mpo && psi && energy, "NULL argument");
    need(mpo->m.L == psi->m.L, "MPO and MPS lengths differ");
    ensure_uploaded(ctx, mpo);
    const double n2 = sandwich(*ctx->c, nullptr, psi->m, psi->m).real();
    if (!(n2 > 0.0)) throw Error(TDMPS_ERR_ZERO_STATE, "state has zero norm");
    *energy = sandwich(*ctx->c, &mpo->m, psi->m, psi->m).real() / n2;
  });
}

int tdmps_integral_gradient(tdmps_ctx_t ctx, tdmps_mps_t psi, double* dE_dh, double* dE_deri) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(psi && (dE_dh || dE_deri), "NULL argument");
    const double n2 = sandwich(*ctx->c, nullptr, psi->m, psi->m).real();
    if (!(n2 > 0.0)) throw Error(TDMPS_ERR_ZERO_STATE, "state has zero norm");
    const size_t L2 = (size_t)psi->m.L * psi->m.L;
    if (dE_dh) {
      std::vector<cplx> g(L2);
      one_rdm(*ctx->c, psi->m, g.data());
      for (size_t i = 0; i < L2; ++i) dE_dh[i] = g[i].real() / n2;
    }
    if (dE_deri) {
      std::vector<cplx> g(L2 * L2);
      two_rdm(*ctx->c, psi->m, g.data());
      for (size_t i = 0; i < g.size(); ++i) dE_deri[i] = 0.5 * g[i].real() / n2;
    }
  });
}

int tdmps_apply_site_op(tdmps_ctx_t ctx, tdmps_mps_t in, int site, int spin, int dagger,
                        tdmps_mps_t* out) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(in && out, "NULL argument");
    auto m = std::make_unique<tdmps_mps_s>();
    if (!apply_site_op(*ctx->c, in->m, site, spin, dagger != 0, m->m))
      throw Error(TDMPS_ERR_ZERO_STATE, "the operator annihilates the state");
    *out = m.release();
  });
}

int tdmps_green_function(tdmps_ctx_t ctx, tdmps_mpo_t mpo, tdmps_mps_t psi0, int i, int j,
                         double dt, int n_steps, int method, int m, int orthogonal, int D,
                         double eps, tdmps_complex* G) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(mpo && psi0 && G, "NULL argument");
    need(mpo->m.L == psi0->m.L, "MPO and MPS lengths differ");
    need(i >= 0 && i < psi0->m.L && j >= 0 && j < psi0->m.L, "orbital index out of range");
    need_finite(dt, "dt must be finite");
    if (method == 0) need(m >= 2 && m <= 16, "Krylov dimension must be in [2, 16]");
    ensure_uploaded(ctx, mpo);
    std::vector<cplx> g((size_t)std::max(n_steps, 0) + 1);
    green_function(*ctx->c, mpo->m, psi0->m, i, j, dt, n_steps, method, m, orthogonal != 0,
                   opts(ctx, D, eps), g.data());
    for (size_t k = 0; k < g.size(); ++k) G[k] = {g[k].real(), g[k].imag()};
  });
}

int tdmps_evolve_batch(tdmps_ctx_t ctx, int n, const tdmps_mpo_t* mpos, tdmps_mps_t* states,
                       const double* dt, const int* n_steps, const int* D, const double* eps,
                       int method, int m, int orthogonal, int n_workers, int* status) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  int first = TDMPS_OK;
  int rc = guard(ctx, [&] {
    need(n >= 0, "n must be >= 0");
    if (n == 0) return;
    need(mpos && states && dt && n_steps && D && eps, "NULL argument");
    need(method == 0 || method == 1, "method must be 0 (Krylov) or 1 (RK4)");
    if (method == 0) need(m >= 2 && m <= 16, "Krylov dimension must be in [2, 16]");
    std::vector<BatchItem> items(n);
    for (int k = 0; k < n; ++k) {
      need(mpos[k] && states[k], "NULL MPO or state in the batch");
      need(mpos[k]->m.L == states[k]->m.L, "MPO and MPS lengths differ");
      need(n_steps[k] >= 0, "n_steps must be >= 0");
      need_finite(dt[k], "dt must be finite");
      opts(ctx, D[k], eps[k]);   // argument checks
      for (int q = 0; q < k; ++q) need(states[q] != states[k], "a state appears twice in the batch");
      ensure_uploaded(ctx, mpos[k]);
      items[k] = {&mpos[k]->m, &states[k]->m, dt[k], n_steps[k], D[k], eps[k]};
    }
    std::vector<int> st(n, TDMPS_OK);
    std::vector<std::string> msgs;
    evolve_batch(*ctx->c, items, method, m, orthogonal != 0, n_workers, st.data(), msgs);
    if (status) for (int k = 0; k < n; ++k) status[k] = st[k];
    for (int k = 0; k < n; ++k)
      if (st[k] != TDMPS_OK) {
        first = st[k];
        throw Error(st[k], "batch item " + std::to_string(k) + ": " + msgs[k]);
      }
  });
  return rc != TDMPS_OK ? rc : first;
}

int tdmps_fiedler_order(const double* h, const double* eri, int L, int* perm) {
  try {
    if (!h || !eri || !perm) return TDMPS_ERR_INVALID_ARG;
    fiedler_order(h, eri, L, perm);
    return TDMPS_OK;
  } catch (const Error& e) {
    g_create_err = e.what();
    return e.code;
  } catch (...) {
    return TDMPS_ERR_INVALID_ARG;
  }
}

int tdmps_stats_enable(tdmps_ctx_t ctx, int enable) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    ctx->c->collect_stats();
    ctx->c->stats = enable != 0;
  });
}

int tdmps_stats_reset(tdmps_ctx_t ctx) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    ctx->c->collect_stats();
    for (auto& k : ctx->c->kstat) k = KStat();
  });
}

int tdmps_stats_get(tdmps_ctx_t ctx, int kind, tdmps_kstat* out) {
  if (!ctx) return TDMPS_ERR_INVALID_ARG;
  return guard(ctx, [&] {
    need(kind >= 0 && kind < TDMPS_KSTAT_COUNT && out, "invalid arguments");
    ctx->c->collect_stats();
    const KStat& k = ctx->c->kstat[kind];
    out->launches = k.launches;
    out->ms = k.ms;
    out->flops = k.flops;
    out->bytes = k.bytes;
  });
}

}  // extern "C"
