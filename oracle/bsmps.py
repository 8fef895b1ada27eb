"""Oracle C: the MPS algorithm of Section 2.2 on U(1) x U(1) symmetry blocks
with the Hamiltonian as a matrix product operator (TEST INFRASTRUCTURE ONLY).

Only the test-suite, the smoke check and the benchmark's CPU-baseline and
``--impl reference`` legs may use this module.  It shares no code with the
CUDA library; it meets it only in the seeded inputs of ``synth``.

``oracle.mps`` solves every local problem of Eq. (add_min) by projecting the
exact 4^L target vector, which caps it at L ~ 8.  This module reaches the
benchmark size (L = 16, D = 256) by never forming that vector: the target
alpha H|A> is kept as the operator H (an MPO of Eq. hamil, built here) acting
on the MPS A, and the projection onto the left/right bases of the fitted MPS C
is taken through environments (the partial contractions <C|H|A> of the sites
left and right of the updated one), as Section 2.2.1 describes for the
variational fit.  The schedule, truncation rule and QR rule are those of
``oracle.mps`` (its module docstring), so on small systems the two oracles
return the same states; tests/test_oracle_bsmps.py checks that.

Data layout (plain dicts of numpy blocks, FP64 / complex128):
* a bond is {(n, 2Sz): dimension};
* a site tensor is {(left sector, sigma): block (d_left, d_right)} with right
  sector = left sector + charge(sigma); every other block is zero;
* an MPO bond lists the charge of every channel; the site tensor W_i is
  stored per pair of channel charges as a dense array [w_in, w_out, sigma,
  sigma'] (the matrix element <sigma| O |sigma'> of the local operator that
  takes channel w_in to w_out);
* an environment is {(bra sector, channel charge): block (d_bra, n_channels,
  d_ket)} with ket sector = bra sector - channel charge.

The MPO (reading of Eq. hamil; the paper builds its operators inside a
spin-adapted DMRG code and prints no MPO): every term of
H = sum h_ij c+_is c_js + 1/2 sum (ij|kl) c+_is c+_kt c_lt c_js + e0 is put
in spin-orbital order (1up, 1down, 2up, ... as in Eq. fci; each transposition
of two different spin orbitals flips the sign), terms with equal operator
strings are merged, and at every bond the term is carried by one channel: the
start channel while no operator is placed, the done channel once all are, in
between a channel named by the operators left of the bond when fewer of them
are there (ties: bonds in the left half of the chain), else by the operators
right of it.  Left-named channels carry bare operator strings; right-named
channels sum the left parts of every term that shares the right string, so a
term's coefficient enters on the site where its channel changes from a
left name (or start) to a right name (or done).  Jordan-Wigner signs: with
operators in spin-orbital order, the factor on site j is the product of its
own operators followed by the site parity (-1)^n once for every operator on a
later site.

Pins: tests/test_oracle_bsmps.py -- the MPO contracted to a matrix equals the
full-CI Hamiltonian of oracle.fci on the whole Fock space (L <= 4) and
H|psi> on a sector (L = 6); sandwiches and overlaps equal contracted vectors;
fits, sums, RK4 and Krylov steps equal oracle.mps and full CI (untruncated);
the 1-RDM equals the full-CI one; the FLOP count of an overlap equals
oracle.mps.overlap_flops; the energy gradient with respect to the site
tensors equals the full-CI projection M_i^+ (H v - E v) / |v|^2 and central
differences of the energy, and is orthogonal to its own site (E does not
change under A_i -> (1 + t) A_i); the one-site local operator equals the
full-CI projection M_i^+ H M_i, is Hermitian and gives <A_i, H_i A_i> =
<psi|H|psi> at every site; the two-site local product equals M_{i,i+1}^+ H v;
the sector QR / LQ factors reproduce their blocks with orthonormal factors,
right canonicalisation keeps the state, and the two-site split is the
truncated SVD of each middle sector (Eckart-Young); the identity MPO is the
identity and the site-operator MPOs of c_{j,s} (with their Jordan-Wigner
strings) obey the canonical anticommutation relations on the Fock space.  Parity unpinned, as in oracle.mps: whether
a truncated fit reaches the best truncated state.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import fci
from .mps import gram_schmidt_qr, truncation_rule

SITE_Q = ((0, 0), (1, 1), (1, -1), (2, 0))


def qadd(a, b):
    return (a[0] + b[0], a[1] + b[1])


def qsub(a, b):
    return (a[0] - b[0], a[1] - b[1])


# ---------------------------------------------------------------------------
# local operators of one spatial orbital (Eq. fci site basis)
# ---------------------------------------------------------------------------

def _two_mode_ops():
    """c_up, c_down on the site basis |0>, |up>, |down>, |up down> =
    c+_up c+_down |0>, from the two spin orbitals of the site in Jordan-Wigner
    order (up first): c_up = a (x) 1, c_down = Z (x) a, with a = |0><1| and
    Z = diag(1, -1) on one mode.  The mode basis |n_up n_down> maps to the
    site states as |00> -> |0>, |10> -> |up>, |01> -> |down>, |11> -> |up down>
    (c+_up c+_down |00> = +|11>)."""
    a = np.array([[0.0, 1.0], [0.0, 0.0]])
    Z = np.diag([1.0, -1.0])
    I2 = np.eye(2)
    cu = np.kron(a, I2)            # index n_up * 2 + n_down
    cd = np.kron(Z, a)
    # reorder mode index (n_up, n_down) -> site state 0, up, down, updown
    perm = [0, 2, 1, 3]            # site state s has mode index perm[s]
    P = np.zeros((4, 4))
    for s, m in enumerate(perm):
        P[s, m] = 1.0
    return P @ cu @ P.T, P @ cd @ P.T


_C_UP, _C_DN = _two_mode_ops()
PARITY = np.diag([1.0, -1.0, -1.0, 1.0])
IDENTITY = np.eye(4)


def local_op(spin: int, dagger: bool) -> np.ndarray:
    c = _C_UP if spin == 0 else _C_DN
    return c.T.copy() if dagger else c.copy()


def op_charge(spin: int, dagger: bool):
    q = SITE_Q[1 + spin]
    return q if dagger else (-q[0], -q[1])


# ---------------------------------------------------------------------------
# MPO of Eq. (hamil)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class MPO:
    L: int
    charges: list      # per bond: list of channel charges
    W: list            # per site: {(q_in, q_out): array [n_in, n_out, 4, 4]}
    groups: list       # per bond: {charge: array of channel indices}

    def bond_dims(self):
        return [len(c) for c in self.charges]

    def nnz(self, i: int) -> int:
        return int(sum(np.count_nonzero(b) for b in self.W[i].values()))


class WSite(dict):
    """One MPO site tensor {(q_in, q_out): [n_in, n_out, 4, 4]}.  ``passthrough``
    marks the identity operator, whose MPO stage copies its input and counts
    no arithmetic."""
    passthrough = False


def _finish_mpo(L, chan_lists, entries):
    """chan_lists[k]: list of (charge, name) per channel of bond k;
    entries[i]: {(ch_in, ch_out): 4x4 matrix}.  Channels are grouped by charge
    (order inside a group: first appearance)."""
    charges, groups, index = [], [], []
    for k in range(L + 1):
        qs = [c for c, _ in chan_lists[k]]
        order = sorted(range(len(qs)), key=lambda c: (qs[c], c))
        pos = {}
        g: dict = {}
        for c in order:
            g.setdefault(qs[c], []).append(c)
        for q, members in g.items():
            for r, c in enumerate(members):
                pos[c] = (q, r)
        charges.append(qs)
        groups.append({q: np.array(m, dtype=np.int64) for q, m in g.items()})
        index.append(pos)
    W = []
    for i in range(L):
        blocks = WSite()
        for (ci, co), m in entries[i].items():
            if not np.any(m):
                continue
            qi, ri = index[i][ci]
            qo, ro = index[i + 1][co]
            key = (qi, qo)
            if key not in blocks:
                blocks[key] = np.zeros((len(groups[i][qi]), len(groups[i + 1][qo]), 4, 4))
            blocks[key][ri, ro] += m
        W.append(blocks)
    return MPO(L, charges, W, groups)


def hamiltonian_mpo(h: np.ndarray, eri: np.ndarray, e0: float = 0.0) -> MPO:
    """The MPO of Eq. (hamil) with chemist-order integrals (ij|kl) (see the
    module docstring for the channel rule)."""
    L = h.shape[0]
    # ---- terms as operator strings (spin orbital p = 2 i + s, dagger flag)
    strings: dict = {}

    def add(ops, coef):
        if coef == 0.0:
            return
        ops = list(ops)
        sign = 1.0
        # stable insertion sort by spin orbital; swapping two different
        # spin orbitals anticommutes (equal ones keep their order)
        for a in range(1, len(ops)):
            b = a
            while b > 0 and 2 * ops[b - 1][0] + ops[b - 1][1] > 2 * ops[b][0] + ops[b][1]:
                ops[b - 1], ops[b] = ops[b], ops[b - 1]
                sign = -sign
                b -= 1
        # the same creator (or annihilator) twice in a row is the zero operator
        if any(ops[a] == ops[a - 1] for a in range(1, len(ops))):
            return
        key = tuple(ops)
        strings[key] = strings.get(key, 0.0) + sign * coef

    for i in range(L):
        for j in range(L):
            for s in range(2):
                add([(i, s, True), (j, s, False)], h[i, j])
    for i in range(L):
        for j in range(L):
            for k in range(L):
                for l in range(L):
                    v = eri[i, j, k, l]
                    if v == 0.0:
                        continue
                    for s in range(2):
                        for t in range(2):
                            add([(i, s, True), (k, t, True), (l, t, False), (j, s, False)],
                                0.5 * v)
    terms = [(ops, c) for ops, c in strings.items() if c != 0.0]

    START, DONE = ("start",), ("done",)
    chans = [dict() for _ in range(L + 1)]      # name -> (index, charge)
    chan_lists = [[] for _ in range(L + 1)]

    def channel(k, name, q):
        if name not in chans[k]:
            chans[k][name] = len(chan_lists[k])
            chan_lists[k].append((q, name))
        return chans[k][name]

    channel(0, START, (0, 0))
    for k in range(1, L + 1):
        channel(k, DONE, (0, 0))
    entries = [dict() for _ in range(L)]
    setonce = [dict() for _ in range(L)]

    def name_at(ops, k):
        left = [o for o in ops if o[0] < k]
        right = [o for o in ops if o[0] >= k]
        if not left:
            return START, (0, 0), True
        if not right:
            return DONE, (0, 0), False
        if len(left) < len(right) or (len(left) == len(right) and 2 * k <= L):
            q = (0, 0)
            for (_, s, d) in left:
                q = qadd(q, op_charge(s, d))
            return ("L",) + tuple(left), q, True
        q = (0, 0)
        for (_, s, d) in right:
            q = qsub(q, op_charge(s, d))
        return ("R",) + tuple(right), q, False

    for ops, coef in terms:
        names = [name_at(ops, k) for k in range(L + 1)]
        ids = [channel(k, names[k][0], names[k][1]) for k in range(L + 1)]
        for i in range(L):
            mine = [o for o in ops if o[0] == i]
            later = sum(1 for o in ops if o[0] > i)
            m = IDENTITY.copy()
            for (_, s, d) in mine:
                m = m @ local_op(s, d)
            if later % 2:
                m = m @ PARITY
            key = (ids[i], ids[i + 1])
            left_in, left_out = names[i][2], names[i + 1][2]
            if left_in and not left_out:
                entries[i][key] = entries[i].get(key, 0.0) + coef * m
            else:
                prev = setonce[i].get(key)
                if prev is not None and not np.array_equal(prev, m):
                    raise AssertionError("inconsistent shared MPO entry")
                setonce[i][key] = m
    # the constant e0 on site 0, and the done channel carried to the end
    if L >= 1:
        key = (chans[0][START], chans[1][DONE])
        entries[0][key] = entries[0].get(key, 0.0) + e0 * IDENTITY
    for i in range(1, L):
        setonce[i][(chans[i][DONE], chans[i + 1][DONE])] = IDENTITY.copy()
    for i in range(L):
        for key, m in setonce[i].items():
            entries[i][key] = entries[i].get(key, 0.0) + m
    return _finish_mpo(L, chan_lists, entries)


def identity_mpo(L: int) -> MPO:
    chan_lists = [[((0, 0), "id")] for _ in range(L + 1)]
    entries = [{(0, 0): IDENTITY.copy()} for _ in range(L)]
    mpo = _finish_mpo(L, chan_lists, entries)
    for w in mpo.W:
        w.passthrough = True
    return mpo


def site_operator_mpo(L: int, ops: dict) -> MPO:
    """Bond-dimension-one MPO of a product of single-site operators:
    ops = {site: (4x4 matrix, charge)}; sites not listed carry the identity.
    The channel charge at a bond is the summed charge of the operators left
    of it."""
    chan_lists, q = [], (0, 0)
    chan_lists.append([(q, "c")])
    for i in range(L):
        if i in ops:
            q = qadd(q, ops[i][1])
        chan_lists.append([(q, "c")])
    entries = [{(0, 0): (ops[i][0] if i in ops else IDENTITY).copy()} for i in range(L)]
    return _finish_mpo(L, chan_lists, entries)


def mpo_to_matrix(mpo: MPO) -> np.ndarray:
    """Contract the MPO to its 4^L x 4^L matrix (tiny L only); index
    sum_i sigma_i 4^(L-1-i) as in oracle.mps.to_fock."""
    L = mpo.L
    dense = []
    for i in range(L):
        nin, nout = len(mpo.charges[i]), len(mpo.charges[i + 1])
        Wd = np.zeros((nin, nout, 4, 4))
        for (qi, qo), b in mpo.W[i].items():
            Wd[np.ix_(mpo.groups[i][qi], mpo.groups[i + 1][qo])] += b
        dense.append(Wd)
    M = dense[0][0]                       # [w, s, s']
    for Wd in dense[1:]:
        M = np.einsum("wab,wvcd->vacbd", M, Wd)
        n = M.shape[1] * M.shape[2]
        M = M.reshape(M.shape[0], n, n)
    return M[0]


# ---------------------------------------------------------------------------
# block-sparse MPS
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class BMPS:
    bonds: list        # L+1 dicts {q: dim}
    sites: list        # L dicts {(q_left, sigma): array}

    @property
    def L(self) -> int:
        return len(self.sites)

    @property
    def total(self):
        (q,) = self.bonds[-1].keys()
        return q

    def copy(self) -> "BMPS":
        return BMPS([dict(b) for b in self.bonds],
                    [{k: v.copy() for k, v in s.items()} for s in self.sites])

    def bond_dims(self):
        return [sum(b.values()) for b in self.bonds]


def _rows_of(labels, q):
    return np.where((labels[:, 0] == q[0]) & (labels[:, 1] == q[1]))[0]


def from_dense(tensors, labels) -> BMPS:
    """Cut dense site tensors A[i] (D_l, 4, D_r) with bond labels (D, 2)
    into symmetry blocks; entries outside them must be zero."""
    labels = [np.asarray(q, dtype=np.int64).reshape(-1, 2) for q in labels]
    bonds = []
    for q in labels:
        b: dict = {}
        for x in map(tuple, q.tolist()):
            b[x] = b.get(x, 0) + 1
        bonds.append(dict(sorted(b.items())))
    sites = []
    for i, A in enumerate(tensors):
        A = np.asarray(A, dtype=np.complex128)
        s: dict = {}
        covered = np.zeros(A.shape, dtype=bool)
        for qa in bonds[i]:
            ia = _rows_of(labels[i], qa)
            for sig in range(4):
                qb = qadd(qa, SITE_Q[sig])
                if qb not in bonds[i + 1]:
                    continue
                ib = _rows_of(labels[i + 1], qb)
                s[(qa, sig)] = A[np.ix_(ia, [sig], ib)][:, 0, :].copy()
                covered[np.ix_(ia, [sig], ib)] = True
        if np.any(A[~covered] != 0):
            raise ValueError("site %d has entries outside its symmetry blocks" % i)
        sites.append(s)
    return BMPS(bonds, sites)


def to_dense(m: BMPS):
    """Dense site tensors and labels, bond vectors ordered by sector."""
    labels, offs = [], []
    for b in m.bonds:
        lab, off, o = [], {}, 0
        for q, d in b.items():
            off[q] = o
            lab.extend([q] * d)
            o += d
        labels.append(np.array(lab, dtype=np.int64).reshape(-1, 2))
        offs.append(off)
    tensors = []
    for i, s in enumerate(m.sites):
        A = np.zeros((len(labels[i]), 4, len(labels[i + 1])), dtype=np.complex128)
        for (qa, sig), blk in s.items():
            qb = qadd(qa, SITE_Q[sig])
            a0, b0 = offs[i][qa], offs[i + 1][qb]
            A[a0:a0 + blk.shape[0], sig, b0:b0 + blk.shape[1]] = blk
        tensors.append(A)
    return tensors, labels


def from_determinant(occ) -> BMPS:
    bonds, sites, q = [{(0, 0): 1}], [], (0, 0)
    for o in occ:
        sites.append({(q, o): np.ones((1, 1), dtype=np.complex128)})
        q = qadd(q, SITE_Q[o])
        bonds.append({q: 1})
    return BMPS(bonds, sites)


def _empty_site(left: dict, right: dict) -> dict:
    s = {}
    for qa, da in left.items():
        for sig in range(4):
            qb = qadd(qa, SITE_Q[sig])
            if qb in right:
                s[(qa, sig)] = np.zeros((da, right[qb]), dtype=np.complex128)
    return s


# ---------------------------------------------------------------------------
# FLOP bookkeeping (algorithmic count: a complex multiply-add is 8 real
# FLOPs, a real MPO entry times a complex number 4; only products of
# non-zero blocks and non-zero MPO entries are counted)
# ---------------------------------------------------------------------------

class Flops:
    def __init__(self):
        self.total = 0

    def add(self, n):
        self.total += int(n)


_NOCOUNT = Flops()


# ---------------------------------------------------------------------------
# environments (the three-layer transfer of <C| O |A>)
# ---------------------------------------------------------------------------

def left_boundary():
    return {((0, 0), (0, 0)): np.ones((1, 1, 1), dtype=np.complex128)}


def right_boundary(total):
    return {(total, (0, 0)): np.ones((1, 1, 1), dtype=np.complex128)}


def _acc(d: dict, key, val):
    if key in d:
        d[key] += val
    else:
        d[key] = val.copy()


def _mpo_stage(X: dict, W: dict, targets, fl: Flops):
    """Y[key_out] = sum over inputs of X[key_in] (x) W[w_in, w_out, s, s'] on the
    channel axis (axis 1 of X), for the (input, sigma, sigma', output) links
    listed by ``targets(key_in)`` as (s, sp, (q_w, q_w2), key_out)."""
    Y: dict = {}
    for kin, Xb in X.items():
        for s, sp, wkey, kout in targets(kin):
            Wb = W.get(wkey)
            if Wb is None:
                continue
            w = Wb[:, :, s, sp]
            nz = np.count_nonzero(w)
            if nz == 0:
                continue
            _acc(Y, kout, np.tensordot(Xb, w, axes=(1, 0)).transpose(0, 2, 1))
            if not getattr(W, "passthrough", False):
                fl.add(4 * nz * Xb.shape[0] * Xb.shape[2])
    return Y


def _consumed(W: dict, links) -> bool:
    """Does any (s, s', (q_w, q_w2), key) link have a non-zero MPO entry?
    Products that no later stage uses are not computed (nor counted)."""
    for s, sp, wkey, _ in links:
        Wb = W.get(wkey)
        if Wb is not None and np.any(Wb[:, :, s, sp]):
            return True
    return False


def env_left(E: dict, bra: dict, ket: dict, W: dict, fl: Flops = _NOCOUNT) -> dict:
    """E'[b, w', b'] = sum conj(B[a, s, b]) E[a, w, a'] W[w, w', s, s'] A[a', s', b'],
    in three stages: X = E A, Y = W X, E' = B^dagger Y."""
    def targets(k):
        qa, qw, sp = k
        qb2 = qadd(qsub(qa, qw), SITE_Q[sp])
        for s in range(4):
            if (qa, s) in bra:
                qb = qadd(qa, SITE_Q[s])
                qw2 = qsub(qb, qb2)
                yield s, sp, (qw, qw2), (qa, s, qw2)

    X: dict = {}                                   # (qa, qw, sp) -> [a, w, b']
    for (qa, qw), Eb in E.items():
        qa2 = qsub(qa, qw)
        for sp in range(4):
            Ab = ket.get((qa2, sp))
            if Ab is None or not _consumed(W, targets((qa, qw, sp))):
                continue
            X[(qa, qw, sp)] = np.tensordot(Eb, Ab, axes=(2, 0))
            fl.add(8 * Eb.size * Ab.shape[1])

    Y = _mpo_stage(X, W, targets, fl)              # (qa, s, qw2) -> [a, w', b']
    out: dict = {}
    for (qa, s, qw2), Yb in Y.items():
        Bb = bra[(qa, s)]
        qb = qadd(qa, SITE_Q[s])
        _acc(out, (qb, qw2), np.tensordot(Bb.conj(), Yb, axes=(0, 0)))
        fl.add(8 * Bb.shape[1] * Yb.size)
    return out


def env_right(R: dict, bra: dict, ket: dict, W: dict, fl: Flops = _NOCOUNT) -> dict:
    """R'[a, w, a'] = sum conj(B[a, s, b]) W[w, w', s, s'] A[a', s', b'] R[b, w', b'],
    in three stages: Z = R A^T, Y = W Z, R' = conj(B) Y."""
    def targets(k):
        qb, qw2, sp = k
        qa2 = qsub(qsub(qb, qw2), SITE_Q[sp])
        for s in range(4):
            qa = qsub(qb, SITE_Q[s])
            if (qa, s) in bra:
                yield s, sp, (qsub(qa, qa2), qw2), (qb, s, qsub(qa, qa2))

    Z: dict = {}                                   # (qb, qw2, sp) -> [b, w', a']
    for (qb, qw2), Rb in R.items():
        qb2 = qsub(qb, qw2)
        for sp in range(4):
            qa2 = qsub(qb2, SITE_Q[sp])
            Ab = ket.get((qa2, sp))
            if Ab is None or not _consumed(W, targets((qb, qw2, sp))):
                continue
            Z[(qb, qw2, sp)] = np.tensordot(Rb, Ab, axes=(2, 1))
            fl.add(8 * Rb.size * Ab.shape[0])

    # the MPO stage contracts the channel axis of Z with w_out: use W^T
    WT = WSite({(k[1], k[0]): v.transpose(1, 0, 2, 3) for k, v in W.items()})
    WT.passthrough = getattr(W, "passthrough", False)

    def targets_t(k):
        for s, sp, (qw, qw2), kout in targets(k):
            yield s, sp, (qw2, qw), kout

    Y = _mpo_stage(Z, WT, targets_t, fl)           # (qb, s, qw) -> [b, w, a']
    out: dict = {}
    for (qb, s, qw), Yb in Y.items():
        qa = qsub(qb, SITE_Q[s])
        Bb = bra[(qa, s)]
        _acc(out, (qa, qw), np.tensordot(Bb.conj(), Yb, axes=(1, 0)))
        fl.add(8 * Bb.shape[0] * Yb.size)
    return out


def local_one(Le: dict, Re: dict, ket: dict, W: dict, left: dict, right: dict,
              coef: complex = 1.0, out: dict | None = None, fl: Flops = _NOCOUNT) -> dict:
    """Local solution of Eq. (add_min) at one site in mixed-canonical gauge:
    C[a, s, b] += coef * sum L[a, w, a'] W[w, w', s, s'] A[a', s', b'] R[b, w', b']
    on the blocks of the bonds ``left`` x ``right``, in three stages:
    X = L A, Y = W X, C = Y R."""
    if out is None:
        out = _empty_site(left, right)

    def targets(k):
        qa, qw, sp = k
        qb2 = qadd(qsub(qa, qw), SITE_Q[sp])
        for s in range(4):
            if (qa, s) in out:
                qw2 = qsub(qadd(qa, SITE_Q[s]), qb2)
                if (qadd(qa, SITE_Q[s]), qw2) in Re:
                    yield s, sp, (qw, qw2), (qa, s, qw2)

    X: dict = {}
    for (qa, qw), Lb in Le.items():
        if qa not in left:
            continue
        qa2 = qsub(qa, qw)
        for sp in range(4):
            Ab = ket.get((qa2, sp))
            if Ab is None or not _consumed(W, targets((qa, qw, sp))):
                continue
            X[(qa, qw, sp)] = np.tensordot(Lb, Ab, axes=(2, 0))
            fl.add(8 * Lb.size * Ab.shape[1])

    Y = _mpo_stage(X, W, targets, fl)
    for (qa, s, qw2), Yb in Y.items():
        Rb = Re[(qadd(qa, SITE_Q[s]), qw2)]
        out[(qa, s)] += coef * np.tensordot(Yb, Rb, axes=([1, 2], [1, 2]))
        fl.add(8 * Yb.size * Rb.shape[0])
    return out


def local_two(Le: dict, Re: dict, ket1: dict, ket2: dict, W1: dict, W2: dict, left: dict,
              right: dict, coef: complex = 1.0, out: dict | None = None,
              fl: Flops = _NOCOUNT) -> dict:
    """Two-site local solution Th[(a, s1, s2)] (d_a x d_b), b = a + q(s1) + q(s2):
    sum L[a,w,a'] W1[w,m,s1,s1'] A1[a',s1',x'] W2[m,w',s2,s2'] A2[x',s2',b'] R[b,w',b'],
    staged as X1 = L A1, Y1 = W1 X1, X2 = Y1 A2, Y2 = W2 X2, Th = Y2 R."""
    if out is None:
        out = {}
        for qa, da in left.items():
            for s1 in range(4):
                for s2 in range(4):
                    qb = qadd(qadd(qa, SITE_Q[s1]), SITE_Q[s2])
                    if qb in right:
                        out[(qa, s1, s2)] = np.zeros((da, right[qb]), dtype=np.complex128)
    X1: dict = {}
    for (qa, qw), Lb in Le.items():
        if qa not in left:
            continue
        qa2 = qsub(qa, qw)
        for sp1 in range(4):
            A1 = ket1.get((qa2, sp1))
            if A1 is None:
                continue
            X1[(qa, qw, sp1)] = np.tensordot(Lb, A1, axes=(2, 0))
            fl.add(8 * Lb.size * A1.shape[1])

    def targets1(k):
        qa, qw, sp1 = k
        qm2 = qadd(qsub(qa, qw), SITE_Q[sp1])
        for s1 in range(4):
            qwm = qsub(qadd(qa, SITE_Q[s1]), qm2)
            yield s1, sp1, (qw, qwm), (qa, s1, qwm)

    Y1 = _mpo_stage(X1, W1, targets1, fl)           # (qa, s1, qwm) -> [a, m, x']
    X2: dict = {}
    for (qa, s1, qwm), Yb in Y1.items():
        qm2 = qsub(qadd(qa, SITE_Q[s1]), qwm)
        for sp2 in range(4):
            A2 = ket2.get((qm2, sp2))
            if A2 is None:
                continue
            X2[(qa, s1, qwm, sp2)] = np.tensordot(Yb, A2, axes=(2, 0))
            fl.add(8 * Yb.size * A2.shape[1])

    def targets2(k):
        qa, s1, qwm, sp2 = k
        qm = qadd(qa, SITE_Q[s1])
        qb2 = qadd(qsub(qm, qwm), SITE_Q[sp2])
        for s2 in range(4):
            if (qa, s1, s2) in out:
                qw2 = qsub(qadd(qm, SITE_Q[s2]), qb2)
                yield s2, sp2, (qwm, qw2), (qa, s1, s2, qw2)

    Y2 = _mpo_stage(X2, W2, targets2, fl)
    for (qa, s1, s2, qw2), Yb in Y2.items():
        qb = qadd(qadd(qa, SITE_Q[s1]), SITE_Q[s2])
        Rb = Re.get((qb, qw2))
        if Rb is None:
            continue
        out[(qa, s1, s2)] += coef * np.tensordot(Yb, Rb, axes=([1, 2], [1, 2]))
        fl.add(8 * Yb.size * Rb.shape[0])
    return out


# ---------------------------------------------------------------------------
# sector-wise factorisations (the rules of oracle.mps)
# ---------------------------------------------------------------------------

def _compact_qr(M):
    """gram_schmidt_qr with the zero columns of dependent directions removed:
    Q (m x r), R (r x n), r = number of independent directions."""
    Q, R = gram_schmidt_qr(M)
    keep = np.linalg.norm(Q, axis=0) > 0
    return Q[:, keep], R[keep]


def qr_left(C: dict, left: dict, right: dict):
    """Thin QR of C seen as (a, s) x b, one right sector at a time.
    Returns (Q site, new right bond, {q: (R, old right dim)})."""
    Q, newb, Rs = {}, {}, {}
    for qb, db in right.items():
        rows = [(qa, s) for s in range(4) for qa in [qsub(qb, SITE_Q[s])] if qa in left]
        rows.sort()
        if not rows:
            continue
        M = np.concatenate([C[k] for k in rows], axis=0)
        Qm, R = _compact_qr(M)
        r = Qm.shape[1]
        if r == 0:
            continue
        newb[qb] = r
        Rs[qb] = R
        o = 0
        for k in rows:
            Q[k] = Qm[o:o + C[k].shape[0]]
            o += C[k].shape[0]
    return Q, dict(sorted(newb.items())), Rs


def lq_right(C: dict, left: dict, right: dict):
    """Thin LQ of C seen as a x (s, b), one left sector at a time (QR of the
    conjugate transpose).  Returns (Q site, new left bond, {q: L factor})."""
    Q, newb, Ls = {}, {}, {}
    for qa, da in left.items():
        cols = [(qa, s) for s in range(4) if (qa, s) in C]
        if not cols:
            continue
        M = np.concatenate([C[k] for k in cols], axis=1)
        Qh, Rh = _compact_qr(M.conj().T)
        r = Qh.shape[1]
        if r == 0:
            continue
        newb[qa] = r
        Ls[qa] = Rh.conj().T                                        # da x r
        Qr = Qh.conj().T                                            # r x cols
        o = 0
        for k in cols:
            w = C[k].shape[1]
            Q[k] = Qr[:, o:o + w]
            o += w
    return Q, dict(sorted(newb.items())), Ls


def _restrict(site: dict, left: dict, right: dict) -> dict:
    return {k: v for k, v in site.items() if k[0] in left and qadd(k[0], SITE_Q[k[1]]) in right}


def right_canonicalize(m: BMPS) -> BMPS:
    """Sites 1..L-1 right-canonical by sector-wise LQ from the right, the
    factors pushed into the site on the left (no truncation)."""
    out = m.copy()
    for i in range(out.L - 1, 0, -1):
        Q, newb, Ls = lq_right(out.sites[i], out.bonds[i], out.bonds[i + 1])
        prev = out.sites[i - 1]
        new = {}
        for (qa, s), blk in prev.items():
            qb = qadd(qa, SITE_Q[s])
            if qb in Ls:
                new[(qa, s)] = blk @ Ls[qb]
        out.sites[i] = Q
        out.sites[i - 1] = new
        out.bonds[i] = newb
    return out


def split_two(Th: dict, left: dict, right: dict, D: int, eps: float, absorb: str):
    """SVD of the two-site tensor per middle sector, truncated by
    oracle.mps.truncation_rule.  absorb='right': (U, S V^H); 'left': (U S, V^H).
    Returns (A site, B site, middle bond, discarded, total)."""
    mids = {}
    for (qa, s1, s2) in Th:
        mids.setdefault(qadd(qa, SITE_Q[s1]), None)
    svd = {}
    for qm in sorted(mids):
        rows = sorted((qa, s1) for (qa, s1, s2) in Th if qadd(qa, SITE_Q[s1]) == qm)
        rows = sorted(set(rows))
        cols = sorted(set((s2, qadd(qm, SITE_Q[s2])) for (qa, s1, s2) in Th
                          if qadd(qa, SITE_Q[s1]) == qm))
        M = np.concatenate([np.concatenate([Th[(qa, s1, s2)] for (s2, qb) in cols], axis=1)
                            for (qa, s1) in rows], axis=0)
        U, sv, Vh = np.linalg.svd(M, full_matrices=False)
        svd[qm] = (U, sv, Vh, rows, cols)
    kept, disc, total = truncation_rule({q: v[1] for q, v in svd.items()}, D, eps)
    A, B, mid = {}, {}, {}
    for qm, (U, sv, Vh, rows, cols) in svd.items():
        k = kept[qm]
        if k == 0:
            continue
        mid[qm] = k
        Uk, Vk = U[:, :k], Vh[:k]
        if absorb == "right":
            Vk = sv[:k, None] * Vk
        else:
            Uk = Uk * sv[None, :k]
        o = 0
        for (qa, s1) in rows:
            da = left[qa]
            A[(qa, s1)] = Uk[o:o + da].copy()
            o += da
        o = 0
        for (s2, qb) in cols:
            db = right[qb]
            B[(qm, s2)] = Vk[:, o:o + db].copy()
            o += db
    if not mid:
        raise FloatingPointError("fit target is the zero state")
    return A, B, dict(sorted(mid.items())), disc, total


# ---------------------------------------------------------------------------
# sandwiches, overlaps, norms
# ---------------------------------------------------------------------------

def sandwich(mpo: MPO, bra: BMPS, ket: BMPS, fl: Flops = _NOCOUNT) -> complex:
    """<bra| O |ket> by the left-to-right chain of environments."""
    if bra.total != ket.total:
        return 0.0j
    E = left_boundary()
    for i in range(bra.L):
        E = env_left(E, bra.sites[i], ket.sites[i], mpo.W[i], fl)
    blk = E.get((bra.total, (0, 0)))
    return complex(blk[0, 0, 0]) if blk is not None else 0.0j


def overlap(bra: BMPS, ket: BMPS, fl: Flops = _NOCOUNT) -> complex:
    return sandwich(identity_mpo(bra.L), bra, ket, fl)


def norm(m: BMPS) -> float:
    return float(np.sqrt(max(overlap(m, m).real, 0.0)))


def _scaled(m: BMPS, factor: complex) -> BMPS:
    out = m.copy()
    out.sites[0] = {k: v * factor for k, v in out.sites[0].items()}
    return out


# ---------------------------------------------------------------------------
# variational fit (Eq. add_min)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Schedule:
    D: int
    eps: float = 0.0
    n_two_site: int = 1
    n_one_site: int = 2


def fit(terms, guess: BMPS, sch: Schedule, fl: Flops = _NOCOUNT, info: dict | None = None) -> BMPS:
    """Minimise ||C - sum_t coef_t O_t |ket_t>|| over MPS C of bond dimension
    <= D (Eq. add_min): terms = [(coef, MPO, ket)].  Schedule of oracle.mps:
    right-canonicalise the guess, n_two_site two-site sweeps (truncated SVD),
    n_one_site one-site sweeps (QR / LQ), no adaptive stop."""
    L = guess.L
    for _, _, k in terms:
        if k.total != guess.total:
            raise ValueError("terms and guess lie in different (N, 2Sz) sectors")
    C = right_canonicalize(guess)
    tot = C.total
    LE = [[None] * (L + 1) for _ in terms]
    RE = [[None] * (L + 1) for _ in terms]
    for t in range(len(terms)):
        LE[t][0] = left_boundary()
        RE[t][L] = right_boundary(tot)

    def right_update(i):
        for t, (_, mpo, ket) in enumerate(terms):
            RE[t][i] = env_right(RE[t][i + 1], C.sites[i], ket.sites[i], mpo.W[i], fl)

    def left_update(i):
        for t, (_, mpo, ket) in enumerate(terms):
            LE[t][i + 1] = env_left(LE[t][i], C.sites[i], ket.sites[i], mpo.W[i], fl)

    def solve_one(i):
        out = None
        for t, (coef, mpo, ket) in enumerate(terms):
            out = local_one(LE[t][i], RE[t][i + 1], ket.sites[i], mpo.W[i], C.bonds[i],
                            C.bonds[i + 1], coef, out, fl)
        return out

    def solve_two(i):
        out = None
        for t, (coef, mpo, ket) in enumerate(terms):
            out = local_two(LE[t][i], RE[t][i + 2], ket.sites[i], ket.sites[i + 1], mpo.W[i],
                            mpo.W[i + 1], C.bonds[i], C.bonds[i + 2], coef, out, fl)
        return out

    for i in range(L - 1, 0, -1):
        right_update(i)
    maxdisc = 0.0
    if L == 1:
        C.sites[0] = solve_one(0)
        return C
    for _ in range(sch.n_two_site):
        for i in range(L - 1):
            A, B, mid, disc, total = split_two(solve_two(i), C.bonds[i], C.bonds[i + 2],
                                               sch.D, sch.eps, "right")
            C.sites[i], C.sites[i + 1], C.bonds[i + 1] = A, B, mid
            if total > 0:
                maxdisc = max(maxdisc, disc / total)
            left_update(i)
        for i in range(L - 2, -1, -1):
            A, B, mid, disc, total = split_two(solve_two(i), C.bonds[i], C.bonds[i + 2],
                                               sch.D, sch.eps, "left")
            C.sites[i], C.sites[i + 1], C.bonds[i + 1] = A, B, mid
            if total > 0:
                maxdisc = max(maxdisc, disc / total)
            right_update(i + 1)
    for _ in range(sch.n_one_site):
        for i in range(L):
            Ci = solve_one(i)
            if i < L - 1:
                Q, newb, _ = qr_left(Ci, C.bonds[i], C.bonds[i + 1])
                C.sites[i], C.bonds[i + 1] = Q, newb
                C.sites[i + 1] = _restrict(C.sites[i + 1], newb, C.bonds[i + 2])
                left_update(i)
            else:
                C.sites[i] = Ci
        for i in range(L - 1, -1, -1):
            Ci = solve_one(i)
            if i > 0:
                Q, newb, _ = lq_right(Ci, C.bonds[i], C.bonds[i + 1])
                C.sites[i], C.bonds[i] = Q, newb
                C.sites[i - 1] = _restrict(C.sites[i - 1], C.bonds[i - 1], newb)
                right_update(i)
            else:
                C.sites[i] = Ci
    if info is not None:
        info["discarded"] = max(info.get("discarded", 0.0), maxdisc)
    return C


def apply_H(mpo: MPO, psi: BMPS, alpha: complex, sch: Schedule, fl: Flops = _NOCOUNT,
            info=None) -> BMPS:
    """C ~ alpha H |psi> (Sec. 2.2.1), guess = psi."""
    return fit([(alpha, mpo, psi)], psi, sch, fl, info)


def sum_fit(terms, sch: Schedule, fl: Flops = _NOCOUNT, info=None) -> BMPS:
    """C ~ sum_k c_k |psi_k> (Eqs. sum_exact, add_min), guess = first MPS."""
    ident = identity_mpo(terms[0][1].L)
    return fit([(c, ident, m) for c, m in terms], terms[0][1], sch, fl, info)


# ---------------------------------------------------------------------------
# integrators (Secs. 2.2.2 and 2.2.3)
# ---------------------------------------------------------------------------

def rk4_step(mpo: MPO, psi: BMPS, dt: float, sch: Schedule, fl: Flops = _NOCOUNT) -> BMPS:
    """Four fitted H applications k_n = -i dt H (psi + c k_{n-1}) and four
    fitted sums, the last one Eq. (rk_add)."""
    a = -1j * dt
    k1 = apply_H(mpo, psi, a, sch, fl)
    s1 = sum_fit([(1.0, psi), (0.5, k1)], sch, fl)
    k2 = apply_H(mpo, s1, a, sch, fl)
    s2 = sum_fit([(1.0, psi), (0.5, k2)], sch, fl)
    k3 = apply_H(mpo, s2, a, sch, fl)
    s3 = sum_fit([(1.0, psi), (1.0, k3)], sch, fl)
    k4 = apply_H(mpo, s3, a, sch, fl)
    return sum_fit([(1.0, psi), (1 / 6, k1), (1 / 3, k2), (1 / 3, k3), (1 / 6, k4)], sch, fl)


def krylov_step(mpo: MPO, psi: BMPS, dt: float, m: int, sch: Schedule,
                orthogonal: bool = True, fl: Flops = _NOCOUNT):
    """One Krylov step with m basis vectors (phi_0 = psi), as in
    oracle.mps.krylov_step: u = fit(H phi_k) (guess phi_k); with the
    orthogonal basis (Eq. kry_orth) phi_{k+1} = fit(u - sum_j c_j phi_j),
    c_j = <phi_j|H|phi_k>/<phi_j|phi_j> (guess u); each phi normalised.
    N_ij = <phi_i|phi_j> and H_ij = <phi_i|H|phi_j> by sandwiches for i <= j,
    the rest by Hermiticity; the new state is fitted to Eq. (krylov_evo) with
    guess phi_0.  Returns (MPS, c, N, H)."""
    phis = [psi]
    Hs: dict = {}
    for k in range(m - 1):
        u = apply_H(mpo, phis[k], 1.0, sch, fl)
        if orthogonal:
            terms = [(1.0, u)]
            for j in range(k + 1):
                hjk = sandwich(mpo, phis[j], phis[k], fl)
                Hs[(j, k)] = hjk
                terms.append((-hjk / overlap(phis[j], phis[j], fl), phis[j]))
            u = sum_fit(terms, sch, fl)
        phis.append(_scaled(u, 1.0 / norm(u)))
    N = np.zeros((m, m), dtype=np.complex128)
    Hk = np.zeros((m, m), dtype=np.complex128)
    for i in range(m):
        for j in range(i, m):
            N[i, j] = overlap(phis[i], phis[j], fl)
            Hk[i, j] = Hs[(i, j)] if (i, j) in Hs else sandwich(mpo, phis[i], phis[j], fl)
            N[j, i], Hk[j, i] = np.conj(N[i, j]), np.conj(Hk[i, j])
    c, _ = fci.krylov_coefficients(N, Hk, dt)
    out = sum_fit([(c[k], phis[k]) for k in range(m)], sch, fl)
    return out, c, N, Hk


# ---------------------------------------------------------------------------
# observables (Section 3.2)
# ---------------------------------------------------------------------------

def one_rdm(psi: BMPS) -> np.ndarray:
    """gamma_ij = sum_s <psi| c+_is c_js |psi> / <psi|psi> ... unnormalised:
    the plain expectation values <psi| c+_is c_js |psi>.

    For i < j the operator string is c+_is P_i on site i (the parity of the
    later operator c_js), P on every site between, c_js on site j, identity
    elsewhere; i = j is the number operator; j < i follows from Hermiticity.
    Left environments of the identity up to i and right ones from j+1 are
    shared by all pairs."""
    L = psi.L
    tot = psi.total
    ident = {((0, 0), (0, 0)): IDENTITY.reshape(1, 1, 4, 4)}
    Lid = [left_boundary()]
    for i in range(L):
        Lid.append(env_left(Lid[-1], psi.sites[i], psi.sites[i], ident))
    Rid = [None] * (L + 1)
    Rid[L] = right_boundary(tot)
    for i in range(L - 1, -1, -1):
        Rid[i] = env_right(Rid[i + 1], psi.sites[i], psi.sites[i], ident)

    def close(E, i, Rnext):
        # full contraction of a left environment at bond i+1 with the right one
        val = 0.0j
        for (qa, qw), blk in E.items():
            r = Rnext.get((qa, qw))
            if r is not None:
                val += np.sum(blk * r)
        return val

    gamma = np.zeros((L, L), dtype=np.complex128)
    for s in range(2):
        cd, c = local_op(s, True), local_op(s, False)
        qc = op_charge(s, True)
        for i in range(L):
            # diagonal: number operator on site i
            Wn = {((0, 0), (0, 0)): (cd @ c).reshape(1, 1, 4, 4)}
            E = env_left(Lid[i], psi.sites[i], psi.sites[i], Wn)
            gamma[i, i] += close(E, i, Rid[i + 1])
            # open channel c+_is P_i, charge qc
            Wo = {((0, 0), qc): (cd @ PARITY).reshape(1, 1, 4, 4)}
            G = env_left(Lid[i], psi.sites[i], psi.sites[i], Wo)
            for j in range(i + 1, L):
                Wc = {(qc, (0, 0)): c.reshape(1, 1, 4, 4)}
                E = env_left(G, psi.sites[j], psi.sites[j], Wc)
                gamma[i, j] += close(E, j, Rid[j + 1])
                Wp = {(qc, qc): PARITY.reshape(1, 1, 4, 4)}
                G = env_left(G, psi.sites[j], psi.sites[j], Wp)
    for i in range(L):
        for j in range(i):
            gamma[i, j] = np.conj(gamma[j, i])
    return gamma


def coefficients(m: BMPS, occs) -> np.ndarray:
    """<det|m> for configurations given as local states per site: the matrix
    product of Eq. (mps) along the blocks each configuration selects."""
    out = np.zeros(len(occs), dtype=np.complex128)
    for n, occ in enumerate(occs):
        v = np.ones((1, 1), dtype=np.complex128)
        q = (0, 0)
        ok = True
        for i, o in enumerate(occ):
            blk = m.sites[i].get((q, int(o)))
            if blk is None:
                ok = False
                break
            v = v @ blk
            q = qadd(q, SITE_Q[int(o)])
        out[n] = v[0, 0] if ok and v.shape == (1, 1) else 0.0
    return out


# ---------------------------------------------------------------------------
# gradient of the energy with respect to the site tensors
# ---------------------------------------------------------------------------

def energy_gradient(mpo: MPO, psi: BMPS):
    """E = <psi|H|psi> / <psi|psi> and its derivative with respect to the
    conjugated site tensors, site by site in the gauge psi is given in:

        dE / d conj(A_i) = (H_i A_i - E N_i A_i) / <psi|psi>,

    H_i A_i the one-site product of Eq. (add_min)'s local problem (left and
    right environments of <psi|H|psi> around site i, here with bra = ket =
    psi) and N_i A_i the same with the identity operator (the norm
    environments; no orthogonality of the other sites is assumed).  <psi|H|psi>
    is linear in A_i and in conj(A_i) separately, which is why its derivative
    with respect to conj(A_i) is H_i A_i.  Returns (E, [one block dict per
    site, blocks as in psi])."""
    L = psi.L
    ident = identity_mpo(L)
    RH, RN = [None] * (L + 1), [None] * (L + 1)
    RH[L] = right_boundary(psi.total)
    RN[L] = right_boundary(psi.total)
    for i in range(L - 1, -1, -1):
        RH[i] = env_right(RH[i + 1], psi.sites[i], psi.sites[i], mpo.W[i])
        RN[i] = env_right(RN[i + 1], psi.sites[i], psi.sites[i], ident.W[i])
    num = complex(RH[0][((0, 0), (0, 0))][0, 0, 0])
    nrm = RN[0][((0, 0), (0, 0))][0, 0, 0].real
    E = num.real / nrm
    LH, LN = left_boundary(), left_boundary()
    grads = []
    for i in range(L):
        gh = local_one(LH, RH[i + 1], psi.sites[i], mpo.W[i], psi.bonds[i], psi.bonds[i + 1])
        gn = local_one(LN, RN[i + 1], psi.sites[i], ident.W[i], psi.bonds[i], psi.bonds[i + 1])
        grads.append({k: (gh[k] - E * gn[k]) / nrm for k in gh})
        LH = env_left(LH, psi.sites[i], psi.sites[i], mpo.W[i])
        LN = env_left(LN, psi.sites[i], psi.sites[i], ident.W[i])
    return E, grads


def local_matvec(mpo: MPO, psi: BMPS, i: int, x: dict, fl: Flops = _NOCOUNT) -> dict:
    """The one-site effective Hamiltonian of Eq. (add_min)'s local problem at
    site i, applied to x (a site tensor on psi's bonds i and i+1):

        y[a, s, b] = sum L[a, w, a'] W_i[w, w', s, s'] x[a', s', b'] R[b, w', b'],

    L and R the environments of <psi|H|psi> left of site i and right of it.
    No gauge is assumed: <psi(x)|H|psi(z)> = <x, y(z)> for the states psi(x),
    psi(z) with site i replaced, so in psi's mixed-canonical gauge at i this is
    H projected onto the site's variational space.  The environments are
    built by plain sweeps from both ends; only the application is counted in
    ``fl``."""
    Le, Re = local_environments(mpo, psi, i)
    return local_one(Le, Re, x, mpo.W[i], psi.bonds[i], psi.bonds[i + 1], fl=fl)


def local_environments(mpo: MPO, psi: BMPS, i: int):
    """The environments of <psi|H|psi> left of site i and right of it."""
    Le = left_boundary()
    for j in range(i):
        Le = env_left(Le, psi.sites[j], psi.sites[j], mpo.W[j])
    Re = right_boundary(psi.total)
    for j in range(psi.L - 1, i, -1):
        Re = env_right(Re, psi.sites[j], psi.sites[j], mpo.W[j])
    return Le, Re
