// Matrix product operator of the quantum-chemistry Hamiltonian, paper Eq.
// (hamil), built on the host from the list of its terms.
//
// Every term (one-body h_ij c+ c, two-body 1/2 (ij|kl) c+ c+ c c) is brought
// to site order (Jordan-Wigner sign of the reordering) and, at each bond k,
// split into the operators on sites < k and on sites >= k.  A term lives in
// one channel per bond:
//   * I_L  if no operator is left of k,  H_L if none is right of k;
//   * otherwise a channel labelled by its LEFT string when the left side
//     holds fewer operators (ties: bonds in the left half of the chain), or
//     by its RIGHT string when the right side holds fewer.
// Left-labelled channels carry the bare operator string; right-labelled
// channels carry the integral-weighted sum of all left parts that share one
// right string.  The term's coefficient therefore enters the MPO exactly once,
// on the site where its channel switches from a left label to a right label.
// This yields the usual complementary-operator bond dimension
// ~ 2 + 4L + 8 min(k, L-k)^2 (spin orbitals counted per side).
//
// Fermionic signs: with operators in site order, the local factor on site j
// is (product of its own operators) * P_j^(number of operators right of j),
// P = (-1)^n the site parity; inside a site c_down carries the parity of the
// up spin orbital (Jordan-Wigner order up, down of Eq. fci).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "internal.hpp"

namespace tdmps {

namespace {

using M4 = std::array<double, 16>;   // [sigma][sigma']

M4 mzero() { M4 m; m.fill(0.0); return m; }
M4 meye() { M4 m = mzero(); for (int i = 0; i < 4; ++i) m[i * 4 + i] = 1.0; return m; }
M4 mmul(const M4& a, const M4& b) {
  M4 c = mzero();
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 4; ++k)
      if (a[i * 4 + k] != 0.0)
        for (int j = 0; j < 4; ++j) c[i * 4 + j] += a[i * 4 + k] * b[k * 4 + j];
  return c;
}

// local operators: code 0 = c+_up, 1 = c+_down, 2 = c_up, 3 = c_down
M4 local_op(int code) {
  M4 m = mzero();
  switch (code) {
    case 0: m[1 * 4 + 0] = 1.0; m[3 * 4 + 2] = 1.0; break;    // |0>->|u>, |d>->|ud>
    case 1: m[2 * 4 + 0] = 1.0; m[3 * 4 + 1] = -1.0; break;   // |0>->|d>, |u>->-|ud>
    case 2: m[0 * 4 + 1] = 1.0; m[2 * 4 + 3] = 1.0; break;    // transpose of code 0
    case 3: m[0 * 4 + 2] = 1.0; m[1 * 4 + 3] = -1.0; break;   // transpose of code 1
  }
  return m;
}
M4 parity() { M4 m = mzero(); m[0] = 1; m[5] = -1; m[10] = -1; m[15] = 1; return m; }

M4 mask_op(int mask) {   // canonical order c+_up c+_down c_up c_down
  M4 m = meye();
  for (int b = 0; b < 4; ++b)
    if (mask & (1 << b)) m = mmul(m, local_op(b));
  return m;
}
QN code_charge(int code) {
  switch (code) {
    case 0: return QN(1, 1);
    case 1: return QN(1, -1);
    case 2: return QN(-1, -1);
    default: return QN(-1, 1);
  }
}
QN mask_charge(int mask) {
  QN q;
  for (int b = 0; b < 4; ++b)
    if (mask & (1 << b)) q = q + code_charge(b);
  return q;
}

struct Term {
  int nsite;
  int site[4];
  int mask[4];
  double coef;
};

uint64_t term_key(const Term& t, int from, int to) {
  // (site, mask) pairs of entries [from, to) -> 10 bits each + count
  uint64_t k = (uint64_t)(to - from);
  for (int j = from; j < to; ++j) k = (k << 10) | ((uint64_t)t.site[j] << 4) | (uint64_t)t.mask[j];
  return k;
}

// Put the operator list in site order; returns false if the product vanishes.
bool canonical(const int* sites, const int* codes, int nops, double coef, Term& out) {
  int key[4];
  for (int i = 0; i < nops; ++i) key[i] = sites[i] * 4 + codes[i];
  int sign = 1;
  for (int i = 1; i < nops; ++i)
    for (int j = i; j > 0 && key[j - 1] > key[j]; --j) {
      std::swap(key[j - 1], key[j]);
      sign = -sign;
    }
  for (int i = 1; i < nops; ++i)
    if (key[i] == key[i - 1]) return false;
  out.nsite = 0;
  for (int i = 0; i < nops; ++i) {
    int s = key[i] / 4, c = key[i] % 4;
    if (out.nsite == 0 || out.site[out.nsite - 1] != s) {
      out.site[out.nsite] = s;
      out.mask[out.nsite] = 0;
      ++out.nsite;
    }
    out.mask[out.nsite - 1] |= 1 << c;
  }
  out.coef = sign * coef;
  return true;
}

enum ChanType { CH_IL = 0, CH_LEFT = 1, CH_RIGHT = 2, CH_HL = 3 };

struct ChanKey {
  int type;
  uint64_t key;
  bool operator==(const ChanKey& o) const { return type == o.type && key == o.key; }
};
struct ChanKeyHash {
  size_t operator()(const ChanKey& k) const { return std::hash<uint64_t>()(k.key * 4 + k.type); }
};

struct BondChannels {
  std::unordered_map<ChanKey, int, ChanKeyHash> idx;
  std::vector<ChanKey> keys;
  std::vector<QN> charge;
  int get(const ChanKey& k, const QN& q) {
    auto it = idx.find(k);
    if (it != idx.end()) return it->second;
    int id = (int)keys.size();
    idx.emplace(k, id);
    keys.push_back(k);
    charge.push_back(q);
    return id;
  }
};

// Sort channels of a bond by (charge, type, key) and fill MPOBond; returns
// old -> new index map.
std::vector<int> finalize_bond(const BondChannels& bc, MPOBond& mb) {
  int n = (int)bc.keys.size();
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) {
    if (bc.charge[a] != bc.charge[b]) return bc.charge[a] < bc.charge[b];
    if (bc.keys[a].type != bc.keys[b].type) return bc.keys[a].type < bc.keys[b].type;
    return bc.keys[a].key < bc.keys[b].key;
  });
  std::vector<int> newidx(n);
  mb.gq.clear(); mb.gsize.clear();
  mb.ch_group.assign(n, 0); mb.ch_local.assign(n, 0);
  for (int r = 0; r < n; ++r) {
    int o = ord[r];
    newidx[o] = r;
    const QN& q = bc.charge[o];
    if (mb.gq.empty() || mb.gq.back() != q) { mb.gq.push_back(q); mb.gsize.push_back(0); }
    mb.ch_group[r] = (int)mb.gq.size() - 1;
    mb.ch_local[r] = mb.gsize.back()++;
  }
  return newidx;
}

void push_elements(std::vector<WElem>& out, int win, int wout, const M4& m, double scale) {
  for (int s = 0; s < 4; ++s)
    for (int sp = 0; sp < 4; ++sp) {
      double v = m[s * 4 + sp] * scale;
      if (v != 0.0) out.push_back({win, wout, s, sp, v});
    }
}

void merge_elements(std::vector<WElem>& w) {
  std::sort(w.begin(), w.end(), [](const WElem& a, const WElem& b) {
    if (a.win != b.win) return a.win < b.win;
    if (a.wout != b.wout) return a.wout < b.wout;
    if (a.sig != b.sig) return a.sig < b.sig;
    return a.sigp < b.sigp;
  });
  std::vector<WElem> out;
  for (auto& e : w) {
    if (!out.empty() && out.back().win == e.win && out.back().wout == e.wout &&
        out.back().sig == e.sig && out.back().sigp == e.sigp)
      out.back().v += e.v;
    else
      out.push_back(e);
  }
  w.clear();
  for (auto& e : out)
    if (e.v != 0.0) w.push_back(e);
}

}  // namespace

MPOd build_qc_mpo(const double* h, const double* eri, int L, double e0) {
  if (L < 1 || L > 63) throw Error(TDMPS_ERR_INVALID_ARG, "L must be in [1, 63]");
  for (int64_t i = 0; i < (int64_t)L * L; ++i)
    if (!std::isfinite(h[i])) throw Error(TDMPS_ERR_NONFINITE, "h contains NaN/Inf");
  for (int64_t i = 0; i < (int64_t)L * L * L * L; ++i)
    if (!std::isfinite(eri[i])) throw Error(TDMPS_ERR_NONFINITE, "eri contains NaN/Inf");
  if (!std::isfinite(e0)) throw Error(TDMPS_ERR_NONFINITE, "e0 is not finite");

  // ---- terms, merged by canonical operator string
  std::unordered_map<uint64_t, size_t> seen;
  std::vector<Term> terms;
  auto add = [&](const int* sites, const int* codes, int n, double c) {
    if (c == 0.0) return;
    Term t;
    if (!canonical(sites, codes, n, c, t)) return;
    uint64_t k = term_key(t, 0, t.nsite);
    auto it = seen.find(k);
    if (it == seen.end()) { seen.emplace(k, terms.size()); terms.push_back(t); }
    else terms[it->second].coef += t.coef;
  };
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j)
      for (int s = 0; s < 2; ++s) {
        int sites[2] = {i, j}, codes[2] = {s, 2 + s};
        add(sites, codes, 2, h[i * L + j]);
      }
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j)
      for (int k = 0; k < L; ++k)
        for (int l = 0; l < L; ++l) {
          double v = eri[(((size_t)i * L + j) * L + k) * L + l];
          if (v == 0.0) continue;
          for (int s = 0; s < 2; ++s)
            for (int t = 0; t < 2; ++t) {
              int sites[4] = {i, k, l, j}, codes[4] = {s, t, 2 + t, 2 + s};
              add(sites, codes, 4, 0.5 * v);
            }
        }
  {
    std::vector<Term> kept;
    for (auto& t : terms)
      if (t.coef != 0.0) kept.push_back(t);
    terms.swap(kept);
  }

  // ---- channels per bond
  std::vector<BondChannels> bc(L + 1);
  const ChanKey KIL{CH_IL, 0}, KHL{CH_HL, 0};
  bc[0].get(KIL, QN());
  for (int k = 1; k <= L; ++k) bc[k].get(KHL, QN());   // E0 path, always present
  auto classify = [&](const Term& t, int k, int& ntotL, QN& q) -> ChanKey {
    int kl = 0, kr = 0, split = 0;
    for (int j = 0; j < t.nsite; ++j) {
      int c = __builtin_popcount(t.mask[j]);
      if (t.site[j] < k) { kl += c; split = j + 1; } else kr += c;
    }
    ntotL = kl;
    if (kr == 0) { q = QN(); return KHL; }
    if (kl == 0) { q = QN(); return KIL; }
    bool left = kl < kr || (kl == kr && 2 * k <= L);
    q = QN();
    if (left) {
      for (int j = 0; j < split; ++j) q = q + mask_charge(t.mask[j]);
      return ChanKey{CH_LEFT, term_key(t, 0, split)};
    }
    for (int j = split; j < t.nsite; ++j) q = q - mask_charge(t.mask[j]);
    return ChanKey{CH_RIGHT, term_key(t, split, t.nsite)};
  };

  // per term, channel id at each bond
  std::vector<int> chan((size_t)terms.size() * (L + 1));
  for (size_t ti = 0; ti < terms.size(); ++ti) {
    for (int k = 0; k <= L; ++k) {
      int nl;
      QN q;
      ChanKey key = classify(terms[ti], k, nl, q);
      chan[ti * (L + 1) + k] = bc[k].get(key, q);
    }
  }

  MPOd m;
  m.L = L;
  m.bonds.resize(L + 1);
  std::vector<std::vector<int>> remap(L + 1);
  for (int k = 0; k <= L; ++k) remap[k] = finalize_bond(bc[k], m.bonds[k]);

  // ---- W tensors
  m.W.assign(L, {});
  const M4 P = parity();
  for (int i = 0; i < L; ++i) {
    std::map<std::pair<int, int>, M4> setv;   // left->left and right->right (set once)
    std::map<std::pair<int, int>, M4> accv;   // transitions (accumulated)
    auto is_left = [&](int bond, int c) {
      int ty = bc[bond].keys[c].type;
      return ty == CH_IL || ty == CH_LEFT;
    };
    for (size_t ti = 0; ti < terms.size(); ++ti) {
      const Term& t = terms[ti];
      int cin = chan[ti * (L + 1) + i], cout = chan[ti * (L + 1) + i + 1];
      int mask = 0, nright = 0;
      for (int j = 0; j < t.nsite; ++j) {
        if (t.site[j] == i) mask = t.mask[j];
        if (t.site[j] > i) nright += __builtin_popcount(t.mask[j]);
      }
      M4 loc = mask_op(mask);
      if (nright & 1) loc = mmul(loc, P);
      bool lin = is_left(i, cin), lout = is_left(i + 1, cout);
      auto key = std::make_pair(cin, cout);
      if (lin && !lout) {
        auto it = accv.find(key);
        if (it == accv.end()) accv.emplace(key, mzero());
        M4& a = accv[key];
        for (int e = 0; e < 16; ++e) a[e] += t.coef * loc[e];
      } else {
        setv[key] = loc;
      }
    }
    // E0 path and the identity carriers of I_L / H_L
    {
      int il_in = bc[i].idx.count(KIL) ? bc[i].idx.at(KIL) : -1;
      int hl_out = bc[i + 1].idx.at(KHL);
      if (i == 0) {
        M4 e = meye();
        for (auto& x : e) x *= e0;
        auto key = std::make_pair(il_in, hl_out);
        if (!accv.count(key)) accv.emplace(key, mzero());
        for (int q = 0; q < 16; ++q) accv[key][q] += e[q];
      } else {
        int hl_in = bc[i].idx.at(KHL);
        setv[std::make_pair(hl_in, hl_out)] = meye();
      }
    }
    std::vector<WElem>& W = m.W[i];
    for (auto& kv : setv)
      push_elements(W, remap[i][kv.first.first], remap[i + 1][kv.first.second], kv.second, 1.0);
    for (auto& kv : accv)
      push_elements(W, remap[i][kv.first.first], remap[i + 1][kv.first.second], kv.second, 1.0);
    merge_elements(W);
    m.n_elem += (int64_t)W.size();
  }
  return m;
}

MPOd build_identity_mpo(int L) {
  MPOd m;
  m.L = L;
  m.identity = true;
  m.bonds.resize(L + 1);
  for (int k = 0; k <= L; ++k) {
    m.bonds[k].gq = {QN()};
    m.bonds[k].gsize = {1};
    m.bonds[k].ch_group = {0};
    m.bonds[k].ch_local = {0};
  }
  m.W.assign(L, {});
  for (int i = 0; i < L; ++i)
    for (int s = 0; s < 4; ++s) m.W[i].push_back({0, 0, s, s, 1.0});
  m.n_elem = 4 * L;
  return m;
}

// Channels of bond k: 0 = identity, then c+_{j,up}, c+_{j,down} for j < k
// (charges (1,1) and (1,-1)).  W_i: I->I (identity), I->c+_{i s} (local c+_s
// times P, the carried parity), c+_{j s}->c+_{j s} (P).  The open channels
// are read out by the one-body density-matrix code.
MPOd build_rdm_mpo(int L) {
  MPOd m;
  m.L = L;
  m.bonds.resize(L + 1);
  // channel numbering inside the bond: I first, then (j, s) in order
  for (int k = 0; k <= L; ++k) {
    BondChannels bcx;
    bcx.get(ChanKey{0, 0}, QN());
    for (int j = 0; j < k; ++j)
      for (int s = 0; s < 2; ++s) bcx.get(ChanKey{1, (uint64_t)(j * 2 + s)}, s == 0 ? QN(1, 1) : QN(1, -1));
    finalize_bond(bcx, m.bonds[k]);
  }
  const M4 P = parity();
  m.W.assign(L, {});
  // channel index of (j, s) at bond k after sorting by charge: group (1,-1)
  // holds down spins, group (1,1) holds up spins, each ordered by j.  Charges
  // sorted: (0,0) < (1,-1) < (1,1).
  auto ch = [&](int k, int j, int s) -> int {
    if (j < 0) return 0;
    return s == 1 ? 1 + j : 1 + k + j;
  };
  for (int i = 0; i < L; ++i) {
    std::vector<WElem>& W = m.W[i];
    push_elements(W, 0, 0, meye(), 1.0);
    for (int s = 0; s < 2; ++s) push_elements(W, 0, ch(i + 1, i, s), mmul(local_op(s), P), 1.0);
    for (int j = 0; j < i; ++j)
      for (int s = 0; s < 2; ++s) push_elements(W, ch(i, j, s), ch(i + 1, j, s), P, 1.0);
    merge_elements(W);
    m.n_elem += (int64_t)W.size();
  }
  return m;
}

}  // namespace tdmps
