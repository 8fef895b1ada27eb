"""Oracle B: the paper's MPS operations on small systems (TEST INFRASTRUCTURE ONLY).

Section 2.1 (Eq. mps) defines the state as a product of site matrices
A^{n_up n_down}; Section 2.2.1 (Eqs. sum_exact, add_min) obtains sums of MPS
and H|A> by variational fitting: the residual ||C - target||^2 is minimised
site by site, each local problem being linear, sweeping like DMRG, at a fixed
maximum bond dimension D.  Sections 2.2.2 / 2.2.3 build RK4 and Krylov steps
from those fits.

This module does all of that on dense site tensors A[i] of shape
(D_left, 4, D_right) whose bond basis vectors carry (N, 2S_z) labels, for L
small enough that the target state fits in memory as a vector over the 4^L
configurations.  The local linear problem of Eq. (add_min) in the
mixed-canonical gauge has the Gram matrices of the left and right bases equal
to the identity, so its solution is the projection of the target vector onto
those bases; this oracle computes exactly that projection from the target
vector itself.  It therefore needs no MPO and no environments, and shares no
arithmetic with the CUDA implementation, which reaches the same local tensors
through the Hamiltonian MPO and environment contractions.

Fixed schedule (the paper leaves it open; the same schedule runs on the GPU):
  0. right-canonicalise the initial guess (sector-wise LQ from the right);
  1. ``n_two_site`` two-site sweeps: pairs (0,1)..(L-2,L-1) left to right,
     then (L-2,L-1)..(0,1) right to left; each two-site tensor is split by
     SVD and truncated by ``truncation_rule``;
  2. ``n_one_site`` one-site sweeps: sites 0..L-1 left to right (thin QR per
     right sector moves the gauge), then L-1..0 right to left (thin LQ per
     left sector).  The result is right-canonical with its norm on site 0.
     The QR is ``gram_schmidt_qr``: dependent columns add no direction, so the
     new bond basis spans exactly the column space of the local solution.
The initial guess is the input MPS for H|A> and the first term's MPS for sums,
a deterministic stand-in for the paper's random initial MPS.

Truncation rule (Section 2.1 keeps the D largest singular values): singular values
of all sectors of a bond are sorted in descending order (ties: sector label
ascending, then index); values <= 1e-12 * max are dropped; at most D are kept
and, of those, the fewest whose discarded weight sum(s^2) stays <= eps *
sum(s^2); a cut inside a cluster of values within 1e-10 * max of each other
moves down to the cluster edge.

Pins (tests/test_oracle_mps.py, test_oracle_observables.py,
test_oracle_flops.py): untruncated fits and integrators equal the full-CI
results, compression of two sites equals the library SVD, the truncated
fit lowers its residual at every local solve, the sector QR / LQ factors
reproduce their blocks with orthonormal factors, the two-site split is the
truncated SVD of each sector, right canonicalisation keeps the vector, and
the local projections are the adjoints of the site maps.  Parity unpinned: whether a
truncated fit (D below the exact bond dimension) reaches the best truncated
state.  No closed form fixes that state, so the GPU is compared with this
oracle on the same schedule instead.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import fci

SITE_Q = np.array([(0, 0), (1, 1), (1, -1), (2, 0)], dtype=np.int64)
ZERO_FLOOR = 1e-12
CLUSTER_TOL = 1e-10


@dataclasses.dataclass
class MPS:
    tensors: list          # complex128 arrays (D_i, 4, D_{i+1})
    labels: list           # int64 arrays (D_k, 2), k = 0..L

    @property
    def L(self) -> int:
        return len(self.tensors)

    def copy(self) -> "MPS":
        return MPS([t.copy() for t in self.tensors], [q.copy() for q in self.labels])

    @property
    def bond_dims(self):
        return [len(q) for q in self.labels]


# ---------------------------------------------------------------------------
# construction and contraction
# ---------------------------------------------------------------------------

def from_arrays(tensors, labels) -> MPS:
    return MPS([np.asarray(t, dtype=np.complex128).copy() for t in tensors],
               [np.asarray(q, dtype=np.int64).reshape(-1, 2).copy() for q in labels])


def from_determinant(occ) -> MPS:
    """Product state of a determinant (bond dimension 1)."""
    tensors, labels = [], [np.zeros((1, 2), dtype=np.int64)]
    q = np.zeros(2, dtype=np.int64)
    for o in occ:
        A = np.zeros((1, 4, 1), dtype=np.complex128)
        A[0, o, 0] = 1.0
        tensors.append(A)
        q = q + SITE_Q[o]
        labels.append(q.reshape(1, 2).copy())
    return MPS(tensors, labels)


def to_fock(mps: MPS) -> np.ndarray:
    """Contract Eq. (mps) to the coefficient vector over all 4^L site
    configurations, index sum_i sigma_i 4^(L-1-i)."""
    v = np.ones((1, 1), dtype=np.complex128)
    for A in mps.tensors:
        Dl, d, Dr = A.shape
        v = (v @ A.reshape(Dl, d * Dr)).reshape(-1, Dr)
    return v[:, 0] if v.shape[1] == 1 else v.sum(axis=1)


def from_fock(v: np.ndarray, L: int, tol: float = 1e-14) -> MPS:
    """Exact MPS of a 4^L coefficient vector by successive SVDs (Sec. 2.1):
    split off one site at a time, keeping every singular value above
    tol * max of its bond; each bond sector is factorised on its own, so the
    bond labels are the (N, 2S_z) of the sites to the left."""
    rest = np.asarray(v, dtype=np.complex128).reshape(1, -1)
    lab = np.zeros((1, 2), dtype=np.int64)
    tensors, labels = [], [lab.copy()]
    for i in range(L - 1):
        Dl = rest.shape[0]
        M = rest.reshape(Dl * 4, -1)
        rowlab = (lab[:, None, :] + SITE_Q[None, :, :]).reshape(Dl * 4, 2)
        pieces = []
        for q in sorted({tuple(r) for r in rowlab}):
            rows = _rows_of(rowlab, q)
            U, sv, Vh = np.linalg.svd(M[rows], full_matrices=False)
            pieces.append((q, rows, U, sv, Vh))
        smax = max((p[3].max() for p in pieces if p[3].size), default=0.0)
        keep = [(q, rows, U[:, sv > tol * smax], sv[sv > tol * smax], Vh[sv > tol * smax])
                for q, rows, U, sv, Vh in pieces]
        keep = [k for k in keep if k[3].size]
        Dr = sum(k[3].size for k in keep)
        A = np.zeros((Dl * 4, Dr), dtype=np.complex128)
        nxt = np.zeros((Dr, M.shape[1]), dtype=np.complex128)
        newlab = np.zeros((Dr, 2), dtype=np.int64)
        c = 0
        for q, rows, U, sv, Vh in keep:
            k = sv.size
            A[rows, c:c + k] = U
            nxt[c:c + k] = sv[:, None] * Vh
            newlab[c:c + k] = q
            c += k
        tensors.append(A.reshape(Dl, 4, Dr))
        rest, lab = nxt, newlab
        labels.append(lab.copy())
    Dl = rest.shape[0]
    last = rest.reshape(Dl, 4, 1)
    rowlab = (lab[:, None, :] + SITE_Q[None, :, :])
    weight = {}
    for a in range(Dl):
        for s in range(4):
            q = tuple(rowlab[a, s])
            weight[q] = weight.get(q, 0.0) + abs(last[a, s, 0]) ** 2
    tot = max(weight, key=weight.get)
    if sum(weight.values()) - weight[tot] > 1e-24 * max(weight[tot], 1e-300):
        raise ValueError("vector is not an eigenvector of (N, 2S_z)")
    # entries of another total charge are SVD rounding noise of exact zeros
    mask = np.all(rowlab == np.array(tot)[None, None, :], axis=2)
    tensors.append(np.where(mask[:, :, None], last, 0.0))
    labels.append(np.array([tot], dtype=np.int64).reshape(1, 2))
    return MPS(tensors, labels)


def fock_index(dets: np.ndarray, L: int) -> np.ndarray:
    """Configuration index of each determinant mask (up bit -> 1, down -> 2)."""
    idx = np.zeros(len(dets), dtype=np.int64)
    for i in range(L):
        up = ((dets >> np.uint64(2 * i)) & np.uint64(1)).astype(np.int64)
        dn = ((dets >> np.uint64(2 * i + 1)) & np.uint64(1)).astype(np.int64)
        idx = idx * 4 + up + 2 * dn
    return idx


def to_sector(mps: MPS, dets: np.ndarray) -> np.ndarray:
    return to_fock(mps)[fock_index(dets, mps.L)]


def sector_to_fock(vec: np.ndarray, dets: np.ndarray, L: int) -> np.ndarray:
    out = np.zeros(4 ** L, dtype=np.complex128)
    out[fock_index(dets, L)] = vec
    return out


def coefficient(mps: MPS, occ) -> complex:
    """<det|mps>: the product A^{s_1} ... A^{s_L} of Eq. (mps) for one
    configuration (any L)."""
    v = np.ones((1,), dtype=np.complex128)
    for A, o in zip(mps.tensors, occ):
        v = v @ A[:, o, :]
    return complex(v[0])


def coefficients(mps: MPS, occs) -> np.ndarray:
    """<det|mps> for many configurations at once: the same products of
    Eq. (mps), evaluated site by site for all configurations together."""
    occs = np.asarray(occs, dtype=np.int64)
    v = np.ones((len(occs), 1), dtype=np.complex128)
    for i, A in enumerate(mps.tensors):
        nv = np.zeros((len(occs), A.shape[2]), dtype=np.complex128)
        for s in range(4):
            sel = occs[:, i] == s
            if sel.any():
                nv[sel] = v[sel] @ A[:, s, :]
        v = nv
    return v[:, 0]


def overlap(bra: MPS, ket: MPS) -> complex:
    """<bra|ket> by contracting the two chains site by site (any L)."""
    E = np.ones((1, 1), dtype=np.complex128)
    for B, A in zip(bra.tensors, ket.tensors):
        E = sum(B[:, s, :].conj().T @ (E @ A[:, s, :]) for s in range(4))
    return complex(E[0, 0])


def _sector_dims(labels: np.ndarray) -> dict:
    dims: dict = {}
    for q in map(tuple, labels.tolist()):
        dims[q] = dims.get(q, 0) + 1
    return dims


def overlap_flops(bra: MPS, ket: MPS) -> int:
    """Algorithmic real FLOPs of <bra|ket> by the transfer recursion of
    Section 2.1, E_{i+1} = sum_sigma B^sigma^dagger (E_i A^sigma), on the
    U(1) x U(1) blocks (a site tensor maps the left sector q to q + q(sigma);
    every other block is zero).  For each sector q that carries a non-zero
    block of E_i and each sigma whose q' = q + q(sigma) is a sector of both
    right bonds:
        E_i A^sigma            8 |bra_i(q)| |ket_i(q)| |ket_{i+1}(q')|
        B^sigma^dagger (E A)   8 |bra_{i+1}(q')| |bra_i(q)| |ket_{i+1}(q')|
    (a complex multiply-add is 8 real FLOPs).  Products that no later step
    uses (q' missing from the bra) are not algorithmic work."""
    live = {(0, 0)}          # the left boundary sector
    total = 0
    for i in range(bra.L):
        bl, kl = _sector_dims(bra.labels[i]), _sector_dims(ket.labels[i])
        br, kr = _sector_dims(bra.labels[i + 1]), _sector_dims(ket.labels[i + 1])
        nxt = set()
        for q in live:
            if q not in bl or q not in kl:
                continue
            for c in SITE_Q:
                qp = (q[0] + int(c[0]), q[1] + int(c[1]))
                if qp in br and qp in kr:
                    total += 8 * bl[q] * kl[q] * kr[qp] + 8 * br[qp] * bl[q] * kr[qp]
                    nxt.add(qp)
        live = nxt
    return total


def norm(mps: MPS) -> float:
    return float(np.sqrt(max(overlap(mps, mps).real, 0.0)))


def scale(mps: MPS, alpha: complex) -> MPS:
    """alpha|A>: the principal L-th root of alpha on every site (Sec. 2.2.1)."""
    out = mps.copy()
    r = complex(alpha) ** (1.0 / mps.L)
    out.tensors = [t * r for t in out.tensors]
    return out


def _site_op_matrix(spin: int, dagger: bool) -> np.ndarray:
    """4x4 matrix M[sigma_out, sigma_in] of a_(site, spin) or its adjoint on
    one site's local states |0>, |up>, |down>, |up down> = a+_up a+_down |0>.

    From the determinant convention of Eq. (fci): a local state is the
    ordered product of its creators (up before down), so removing or adding
    the down electron passes the up creator when the up orbital is occupied
    (sign -1); removing or adding the up electron passes nothing."""
    M = np.zeros((4, 4))
    bit = 1 << spin
    for s_in in range(4):
        occupied = bool(s_in & bit)
        if occupied == dagger:
            continue
        sign = -1.0 if (spin == 1 and (s_in & 1)) else 1.0
        M[s_in ^ bit, s_in] = sign
    return M


def apply_site_op(mps: MPS, site: int, spin: int, dagger: bool) -> MPS:
    """a_(site, spin)|mps> (dagger=False) or a+_(site, spin)|mps>, exactly.

    The operator is a product over sites (bond dimension one): the parity
    (-1)^n on every site before ``site`` (the electrons of all earlier spin
    orbitals of Eq. fci), the local matrix of ``_site_op_matrix`` on ``site``
    and the identity after it.  Bonds after ``site`` shift their (N, 2S_z)
    labels by the operator's charge."""
    out = mps.copy()
    parity = np.array([1.0, -1.0, -1.0, 1.0])
    for k in range(site):
        out.tensors[k] = out.tensors[k] * parity[None, :, None]
    M = _site_op_matrix(spin, dagger)
    out.tensors[site] = np.einsum("ts,asb->atb", M, out.tensors[site])
    dq = SITE_Q[1 + spin] * (1 if dagger else -1)
    for k in range(site + 1, mps.L + 1):
        out.labels[k] = out.labels[k] + dq[None, :]
    return out


# ---------------------------------------------------------------------------
# sector-wise factorisations
# ---------------------------------------------------------------------------

def _rows_of(labels: np.ndarray, q) -> np.ndarray:
    return np.where((labels[:, 0] == q[0]) & (labels[:, 1] == q[1]))[0]


def _sectors(labels: np.ndarray):
    return sorted({(int(a), int(b)) for a, b in labels})


QR_DEP_TOL = 1e-12


def gram_schmidt_qr(M: np.ndarray):
    """Thin QR by classical Gram-Schmidt with one re-orthogonalisation.

    A column whose residual norm is <= 1e-12 times the largest column norm of
    M adds no direction.  Q has k = min(m, n) columns: the independent
    directions in column order, then zero columns; R (k x n) satisfies
    M = Q R.  For full-rank M this spans the same space as any QR."""
    m, n = M.shape
    k = min(m, n)
    Q = np.zeros((m, k), dtype=np.complex128)
    R = np.zeros((k, n), dtype=np.complex128)
    tol = QR_DEP_TOL * (np.linalg.norm(M, axis=0).max() if n else 0.0)
    nq = 0
    for j in range(n):
        v = M[:, j].astype(np.complex128).copy()
        for _ in range(2):
            c = Q[:, :nq].conj().T @ v
            v = v - Q[:, :nq] @ c
            R[:nq, j] += c
        nrm = np.linalg.norm(v)
        if nrm > tol and nq < k:
            Q[:, nq] = v / nrm
            R[nq, j] = nrm
            nq += 1
    return Q, R


def qr_left(C: np.ndarray, ql: np.ndarray, qr: np.ndarray):
    """Thin QR of C viewed as a (left x sigma) by right matrix, one right
    sector at a time.  Returns (Q tensor, new right labels, R blocks)."""
    Dl, d, Dr = C.shape
    rowlab = (ql[:, None, :] + SITE_Q[None, :, :]).reshape(Dl * d, 2)
    M = C.reshape(Dl * d, Dr)
    cols_out, labs, Rs = [], [], {}
    for q in _sectors(qr):
        rows = _rows_of(rowlab, q)
        cols = _rows_of(qr, q)
        if len(rows) == 0 or len(cols) == 0:
            continue
        Q, R = gram_schmidt_qr(M[np.ix_(rows, cols)])
        full = np.zeros((Dl * d, Q.shape[1]), dtype=np.complex128)
        full[rows] = Q
        cols_out.append(full)
        labs.extend([q] * Q.shape[1])
        Rs[q] = (R, cols)
    Qt = np.concatenate(cols_out, axis=1) if cols_out else np.zeros((Dl * d, 0))
    return Qt.reshape(Dl, d, -1), np.array(labs, dtype=np.int64).reshape(-1, 2), Rs


def lq_right(C: np.ndarray, ql: np.ndarray, qr: np.ndarray):
    """Thin LQ of C viewed as a left by (sigma x right) matrix, one left sector
    at a time (QR of the conjugate transpose).  Returns (Q tensor, new left
    labels, dict sector -> (L factor, original row indices))."""
    Dl, d, Dr = C.shape
    collab = (qr[None, :, :] - SITE_Q[:, None, :]).reshape(d * Dr, 2)
    M = C.reshape(Dl, d * Dr)
    rows_out, labs, Ls = [], [], {}
    for q in _sectors(ql):
        rows = _rows_of(ql, q)
        cols = _rows_of(collab, q)
        if len(rows) == 0 or len(cols) == 0:
            continue
        Qh, Rh = gram_schmidt_qr(M[np.ix_(rows, cols)].conj().T)
        full = np.zeros((Qh.shape[1], d * Dr), dtype=np.complex128)
        full[:, cols] = Qh.conj().T
        rows_out.append(full)
        labs.extend([q] * Qh.shape[1])
        Ls[q] = (Rh.conj().T, rows)
    Qt = np.concatenate(rows_out, axis=0)
    return Qt.reshape(-1, d, Dr), np.array(labs, dtype=np.int64).reshape(-1, 2), Ls


def truncation_rule(svals: dict, D: int, eps: float):
    """Number of singular values kept per sector (see module docstring).
    svals: sector -> descending array.  Returns (kept dict, discarded weight,
    total weight)."""
    items = []
    for q in sorted(svals):
        for k, s in enumerate(svals[q]):
            items.append((-float(s), q, k))
    items.sort()
    s_all = np.array([-it[0] for it in items])
    total = float(np.sum(s_all ** 2))
    if len(s_all) == 0 or s_all[0] <= 0.0:
        return {q: 0 for q in svals}, total, total
    smax = s_all[0]
    n = int(np.sum(s_all > ZERO_FLOOR * smax))
    tail = np.concatenate([np.cumsum((s_all[::-1]) ** 2)[::-1], [0.0]])
    k = n
    while k > 1 and tail[k - 1] <= eps * total:
        k -= 1
    k = min(k, D)
    if k < n:
        j = k
        while j > 0 and s_all[j - 1] - s_all[j] <= CLUSTER_TOL * smax:
            j -= 1
        if j > 0:
            k = j
        else:
            while k < n and s_all[k - 1] - s_all[k] <= CLUSTER_TOL * smax:
                k += 1
    kept = {q: 0 for q in svals}
    for it in items[:k]:
        kept[it[1]] += 1
    disc = float(np.sum(s_all[k:] ** 2))
    return kept, disc, total


def split_two_site(Th: np.ndarray, ql: np.ndarray, qr: np.ndarray, D: int, eps: float,
                   absorb: str):
    """SVD of a two-site tensor Th[a, s1, s2, b] per middle-bond sector,
    truncated by ``truncation_rule``.  absorb='right': returns (U, S V^H);
    absorb='left': returns (U S, V^H).  Also the middle labels and the
    discarded weight."""
    Dl, _, _, Dr = Th.shape
    rowlab = (ql[:, None, :] + SITE_Q[None, :, :]).reshape(Dl * 4, 2)
    collab = (qr[None, :, :] - SITE_Q[:, None, :]).reshape(4 * Dr, 2)
    M = Th.reshape(Dl * 4, 4 * Dr)
    qs = sorted(set(_sectors(rowlab)) & set(_sectors(collab)))
    svd = {}
    for q in qs:
        rows, cols = _rows_of(rowlab, q), _rows_of(collab, q)
        U, s, Vh = np.linalg.svd(M[np.ix_(rows, cols)], full_matrices=False)
        svd[q] = (U, s, Vh, rows, cols)
    kept, disc, total = truncation_rule({q: v[1] for q, v in svd.items()}, D, eps)
    Ucols, Vrows, labs = [], [], []
    for q in qs:
        k = kept[q]
        if k == 0:
            continue
        U, s, Vh, rows, cols = svd[q]
        Uf = np.zeros((Dl * 4, k), dtype=np.complex128)
        Vf = np.zeros((k, 4 * Dr), dtype=np.complex128)
        if absorb == "right":
            Uf[rows] = U[:, :k]
            Vf[:, cols] = s[:k, None] * Vh[:k]
        else:
            Uf[rows] = U[:, :k] * s[None, :k]
            Vf[:, cols] = Vh[:k]
        Ucols.append(Uf)
        Vrows.append(Vf)
        labs.extend([q] * k)
    if not labs:
        raise FloatingPointError("fit target is the zero state")
    A = np.concatenate(Ucols, axis=1).reshape(Dl, 4, -1)
    B = np.concatenate(Vrows, axis=0).reshape(-1, 4, Dr)
    return A, B, np.array(labs, dtype=np.int64).reshape(-1, 2), disc, total


def right_canonicalize(mps: MPS) -> MPS:
    """Sites 1..L-1 right-canonical by sector-wise LQ from the right; the
    factors are pushed into site 0 (no truncation)."""
    out = mps.copy()
    for i in range(out.L - 1, 0, -1):
        Q, lab, Ls = lq_right(out.tensors[i], out.labels[i], out.labels[i + 1])
        prev = out.tensors[i - 1]
        new = np.zeros(prev.shape[:2] + (len(lab),), dtype=np.complex128)
        off = 0
        for q in _sectors(lab):
            Lf, rows = Ls[q]
            k = Lf.shape[1]
            new[:, :, off:off + k] = np.einsum("asb,bk->ask", prev[:, :, rows], Lf)
            off += k
        out.tensors[i] = Q
        out.tensors[i - 1] = new
        out.labels[i] = lab
    return out


# ---------------------------------------------------------------------------
# variational fit (Eq. add_min)
# ---------------------------------------------------------------------------

def _left_basis(C: MPS, i: int) -> np.ndarray:
    v = np.ones((1, 1), dtype=np.complex128)
    for A in C.tensors[:i]:
        Dl, d, Dr = A.shape
        v = (v @ A.reshape(Dl, d * Dr)).reshape(-1, Dr)
    return v


def _right_basis(C: MPS, i: int) -> np.ndarray:
    v = np.ones((1, 1), dtype=np.complex128)
    for A in reversed(C.tensors[i + 1:]):
        Dl, d, Dr = A.shape
        v = (A.reshape(Dl * d, Dr) @ v).reshape(Dl, -1)
    return v


def project_one(T: np.ndarray, C: MPS, i: int) -> np.ndarray:
    """Local solution at site i: <left basis, sigma, right basis | target>."""
    L = C.L
    Lb, Rb = _left_basis(C, i), _right_basis(C, i)
    Tr = T.reshape(4 ** i, 4, 4 ** (L - i - 1))
    return np.einsum("xa,xsy,by->asb", Lb.conj(), Tr, Rb.conj(), optimize=True)


def project_two(T: np.ndarray, C: MPS, i: int) -> np.ndarray:
    L = C.L
    Lb, Rb = _left_basis(C, i), _right_basis(C, i + 1)
    Tr = T.reshape(4 ** i, 4, 4, 4 ** (L - i - 2))
    return np.einsum("xa,xsty,by->astb", Lb.conj(), Tr, Rb.conj(), optimize=True)


@dataclasses.dataclass
class FitInfo:
    discarded: float = 0.0   # largest relative discarded weight of any split
    residuals: list = dataclasses.field(default_factory=list)


def fit(T: np.ndarray, guess: MPS, D: int, eps: float, n_two_site: int = 1,
        n_one_site: int = 2, info: FitInfo | None = None) -> MPS:
    """Minimise ||C - T|| over MPS C of bond dimension <= D (Eq. add_min),
    T given as a 4^L coefficient vector, with the fixed sweep schedule of the
    module docstring."""
    L = guess.L
    C = right_canonicalize(guess)
    tnorm2 = float(np.vdot(T, T).real)
    if L == 1:
        C.tensors[0] = project_one(T, C, 0)
        return C
    for _ in range(n_two_site):
        for i in range(L - 1):
            Th = project_two(T, C, i)
            A, B, lab, disc, tot = split_two_site(Th, C.labels[i], C.labels[i + 2], D, eps, "right")
            C.tensors[i], C.tensors[i + 1], C.labels[i + 1] = A, B, lab
            if info is not None and tot > 0:
                info.discarded = max(info.discarded, disc / tot)
        for i in range(L - 2, -1, -1):
            Th = project_two(T, C, i)
            A, B, lab, disc, tot = split_two_site(Th, C.labels[i], C.labels[i + 2], D, eps, "left")
            C.tensors[i], C.tensors[i + 1], C.labels[i + 1] = A, B, lab
            if info is not None and tot > 0:
                info.discarded = max(info.discarded, disc / tot)
    for _ in range(n_one_site):
        for i in range(L):
            Ci = project_one(T, C, i)
            if i < L - 1:
                Q, lab, _ = qr_left(Ci, C.labels[i], C.labels[i + 1])
                C.tensors[i], C.labels[i + 1] = Q, lab
            else:
                C.tensors[i] = Ci
        for i in range(L - 1, -1, -1):
            Ci = project_one(T, C, i)
            if i > 0:
                Q, lab, _ = lq_right(Ci, C.labels[i], C.labels[i + 1])
                C.tensors[i], C.labels[i] = Q, lab
            else:
                C.tensors[i] = Ci
        if info is not None:
            c2 = float(np.sum(np.abs(C.tensors[0]) ** 2))
            info.residuals.append(max(tnorm2 - c2, 0.0))
    return C


# ---------------------------------------------------------------------------
# the three operations and the two integrators
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class System:
    """Hamiltonian of one (N, 2S_z) sector as a dense FCI matrix (Oracle A)."""
    L: int
    dets: np.ndarray
    H: np.ndarray
    fidx: np.ndarray

    @classmethod
    def build(cls, h, eri, n_alpha, n_beta, e0=0.0):
        L = h.shape[0]
        dets = fci.basis(L, n_alpha, n_beta)
        return cls(L, dets, fci.hamiltonian(h, eri, dets, e0), fock_index(dets, L))

    def vec(self, mps: MPS) -> np.ndarray:
        return to_fock(mps)[self.fidx]

    def fock(self, v: np.ndarray) -> np.ndarray:
        out = np.zeros(4 ** self.L, dtype=np.complex128)
        out[self.fidx] = v
        return out


@dataclasses.dataclass
class Schedule:
    D: int
    eps: float = 0.0
    n_two_site: int = 1
    n_one_site: int = 2


def apply_H(sys: System, mps: MPS, alpha: complex, sch: Schedule, info=None) -> MPS:
    """C ~ alpha H |mps> (Sec. 2.2.1), guess = the input MPS."""
    T = sys.fock(alpha * (sys.H @ sys.vec(mps)))
    return fit(T, mps, sch.D, sch.eps, sch.n_two_site, sch.n_one_site, info)


def sum_fit(sys: System, terms, sch: Schedule, info=None) -> MPS:
    """C ~ sum_k c_k |mps_k> (Eqs. sum_exact, add_min), guess = first MPS."""
    v = sum(c * sys.vec(m) for c, m in terms)
    return fit(sys.fock(v), terms[0][1], sch.D, sch.eps, sch.n_two_site, sch.n_one_site, info)


def sandwich(sys: System, bra: MPS, ket: MPS) -> complex:
    return complex(np.vdot(sys.vec(bra), sys.H @ sys.vec(ket)))


def rk4_step(sys: System, psi: MPS, dt: float, sch: Schedule) -> MPS:
    """Sec. 2.2.2: four fitted H applications (k_n = -i dt H (psi + c k)) and
    four fitted sums, the last one Eq. (rk_add)."""
    a = -1j * dt
    k1 = apply_H(sys, psi, a, sch)
    s1 = sum_fit(sys, [(1.0, psi), (0.5, k1)], sch)
    k2 = apply_H(sys, s1, a, sch)
    s2 = sum_fit(sys, [(1.0, psi), (0.5, k2)], sch)
    k3 = apply_H(sys, s2, a, sch)
    s3 = sum_fit(sys, [(1.0, psi), (1.0, k3)], sch)
    k4 = apply_H(sys, s3, a, sch)
    return sum_fit(sys, [(1.0, psi), (1 / 6, k1), (1 / 3, k2), (1 / 3, k3), (1 / 6, k4)], sch)


def _normalise(m: MPS) -> MPS:
    nrm = norm(m)
    out = m.copy()
    out.tensors[0] = out.tensors[0] / nrm
    return out


def krylov_step(sys: System, psi: MPS, dt: float, m: int, sch: Schedule,
                orthogonal: bool = True):
    """Sec. 2.2.3 with m basis vectors, phi_0 = psi.

    For k = 0..m-2: u = fit(H phi_k) with guess phi_k; with the orthogonal
    basis (Eq. kry_orth) phi_{k+1} = fit(u - sum_{j<=k} c_j phi_j) with guess
    u and c_j = <phi_j|H|phi_k>/<phi_j|phi_j> (the N_K-1 additional sums the
    paper counts for this variant); with the plain basis (Eq. kry_non)
    phi_{k+1} = u.  Each phi_{k+1} is normalised.  N_ij = <phi_i|phi_j>,
    H_ij = <phi_i|H|phi_j> exactly, and the new state is fitted to
    Eq. (krylov_evo) with guess phi_0.  Returns (MPS, c, N, H)."""
    phis = [psi]
    for k in range(m - 1):
        u = apply_H(sys, phis[k], 1.0, sch)
        if orthogonal:
            terms = [(1.0, u)]
            for j in range(k + 1):
                cj = sandwich(sys, phis[j], phis[k]) / overlap(phis[j], phis[j])
                terms.append((-cj, phis[j]))
            u = sum_fit(sys, terms, sch)
        phis.append(_normalise(u))
    vs = [sys.vec(p) for p in phis]
    N = np.array([[np.vdot(a, b) for b in vs] for a in vs])
    Hk = np.array([[np.vdot(a, sys.H @ b) for b in vs] for a in vs])
    c, _ = fci.krylov_coefficients(N, Hk, dt)
    out = sum_fit(sys, [(c[k], phis[k]) for k in range(m)], sch)
    return out, c, N, Hk


def one_rdm(sys: System, mps: MPS) -> np.ndarray:
    return fci.one_rdm(sys.vec(mps), sys.dets, sys.L)


def two_rdm(sys: System, mps: MPS) -> np.ndarray:
    return fci.two_rdm(sys.vec(mps), sys.dets, sys.L)


def green_function(systems: dict, psi0: MPS, i: int, j: int, dt: float, n_steps: int, m: int,
                   sch: Schedule, orthogonal: bool = True, method: str = "krylov") -> np.ndarray:
    """Eq. (green_time) on MPS, as the paper evaluates it: annihilate an
    electron of spin s at orbital j (``apply_site_op``, exact), propagate the
    ionised state backwards in time with ``krylov_step`` or ``rk4_step``
    (time step -dt) and project on a_{is}|psi0> after every step.  ``systems[s]`` is the System
    of the sector with one electron of spin s fewer.  Returns G_ij at
    tau = 0, dt, ..., n_steps * dt."""
    num = np.zeros(n_steps + 1, dtype=np.complex128)
    den = 0.0 + 0.0j
    for s, sysm in systems.items():
        chi_i = apply_site_op(psi0, i, s, False)
        chi = apply_site_op(psi0, j, s, False)
        den += overlap(chi_i, chi)
        num[0] += overlap(chi_i, chi)
        for n in range(n_steps):
            if method == "krylov":
                chi = krylov_step(sysm, chi, -dt, m, sch, orthogonal)[0]
            else:
                chi = rk4_step(sysm, chi, -dt, sch)
            num[n + 1] += overlap(chi_i, chi)
    return -1j * num / den


def compress(mps: MPS, D: int, eps: float):
    """SVD compression (Sec. 2.1): right-canonicalise, then one left-to-right
    pass of truncated SVDs of each site (rows (a, sigma), columns b), then an
    exact LQ pass back.  Returns (MPS, summed relative discarded weight)."""
    C = right_canonicalize(mps)
    L = C.L
    disc_tot = 0.0
    for i in range(L - 1):
        A = C.tensors[i]
        Dl, d, Dr = A.shape
        rowlab = (C.labels[i][:, None, :] + SITE_Q[None, :, :]).reshape(Dl * d, 2)
        M = A.reshape(Dl * d, Dr)
        svd = {}
        for q in _sectors(C.labels[i + 1]):
            rows, cols = _rows_of(rowlab, q), _rows_of(C.labels[i + 1], q)
            if len(rows) == 0:
                continue
            U, s, Vh = np.linalg.svd(M[np.ix_(rows, cols)], full_matrices=False)
            svd[q] = (U, s, Vh, rows, cols)
        kept, disc, tot = truncation_rule({q: v[1] for q, v in svd.items()}, D, eps)
        disc_tot += disc / tot if tot > 0 else 0.0
        Ucols, SV, labs = [], [], []
        nxt = C.tensors[i + 1]
        for q in sorted(svd):
            k = kept[q]
            if k == 0:
                continue
            U, s, Vh, rows, cols = svd[q]
            Uf = np.zeros((Dl * d, k), dtype=np.complex128)
            Uf[rows] = U[:, :k]
            Ucols.append(Uf)
            SV.append(np.einsum("kb,bsc->ksc", s[:k, None] * Vh[:k], nxt[cols]))
            labs.extend([q] * k)
        C.tensors[i] = np.concatenate(Ucols, axis=1).reshape(Dl, d, -1)
        C.tensors[i + 1] = np.concatenate(SV, axis=0)
        C.labels[i + 1] = np.array(labs, dtype=np.int64).reshape(-1, 2)
    return right_canonicalize(C), disc_tot
