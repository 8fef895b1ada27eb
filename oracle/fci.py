"""Oracle A: full CI in the occupation-number basis (TEST INFRASTRUCTURE ONLY).

Follows the paper's Section 2.1 (Eq. fci) and Section 2.2 (Eqs. sg, hamil,
time_evo_opera, the RK4 stages k1..k4 with Eq. rk_add, and the Krylov
construction of Eqs. kry_orth / kry_non with Eq. krylov_evo).

Conventions
-----------
* Spin orbitals are ordered 1up, 1down, 2up, 2down, ... as in Eq. (fci); spin
  orbital (i, sigma) is bit ``2*i + s`` of a determinant's integer mask with
  s = 0 for up and 1 for down.  A determinant is the ordered product of
  creators in that order acting on the vacuum, so applying a_p or a_p^dagger
  costs the sign (-1)^(number of occupied spin orbitals below p).
* Hamiltonian (Eq. hamil), with the integrals read in chemist order:
      H = sum_{ij,s} h_ij a+_{is} a_{js}
        + 1/2 sum_{ijkl,s,t} (ij|kl) a+_{is} a+_{kt} a_{lt} a_{js} + E0,
  i.e. the paper's V_ijkl equals (ik|jl) (t_ij is h_ij).
* The RK4 stages use k = -i dt H (...) (hbar = 1); the paper's printed stages
  omit the factor -i, which the statement that RK4 equals the fourth-order
  Taylor expansion of exp(-i H dt) fixes.
* Krylov steps take m basis vectors including phi_0 = psi; phi_k (k >= 1) are
  normalised after construction; exp(-i dt N^-1 H) e_0 is evaluated by
  canonical orthogonalisation of N (eigenvalues of N below 1e-12 * max are
  discarded), which equals the plain formula whenever N is regular.

Pins (tests/test_oracle_fci.py, test_oracle_observables.py): the Hubbard-dimer
spectrum and Lehmann Green's function, the one-electron Rabi oscillation,
non-interacting spectra and dynamics, an independent Kronecker-product
Jordan-Wigner build of H, of the density matrices and of the Green's function,
[H, S^2] = 0, Slater-Condon diagonals, RK4 = fourth-order Taylor, Krylov exact
on the full space and norm- and energy-conserving below it.  No function here
is parity unpinned.
"""
from __future__ import annotations

from itertools import combinations

import numpy as np

EIG_DROP = 1e-12


# ---------------------------------------------------------------------------
# determinants
# ---------------------------------------------------------------------------

def basis(L: int, n_alpha: int, n_beta: int) -> np.ndarray:
    """All determinants with n_alpha up and n_beta down electrons, as sorted
    uint64 masks (Eq. fci restricted to one (N, S_z) sector)."""
    masks = []
    for ua in combinations(range(L), n_alpha):
        ma = sum(1 << (2 * i) for i in ua)
        for ub in combinations(range(L), n_beta):
            masks.append(ma | sum(1 << (2 * i + 1) for i in ub))
    return np.array(sorted(masks), dtype=np.uint64)


def occupation_mask(occ) -> int:
    """Mask of the determinant with per-orbital occupation codes
    0 = empty, 1 = up, 2 = down, 3 = both."""
    m = 0
    for i, o in enumerate(occ):
        if o & 1:
            m |= 1 << (2 * i)
        if o & 2:
            m |= 1 << (2 * i + 1)
    return m


def _popcount(x: np.ndarray) -> np.ndarray:
    return np.bitwise_count(x).astype(np.int64)


def apply_op(masks: np.ndarray, amp: np.ndarray, mode, dagger: bool):
    """Apply a_mode (dagger=False) or a+_mode to determinants.

    masks: uint64 array; amp: amplitude array (0 marks a vanished term);
    mode: int or int array broadcast against masks.  Returns new (masks, amp).
    """
    mode = np.asarray(mode, dtype=np.uint64)
    bit = np.left_shift(np.uint64(1), mode)
    occ = (masks & bit) != 0
    ok = ~occ if dagger else occ
    below = masks & (bit - np.uint64(1))
    sign = 1 - 2 * (_popcount(below) & 1)
    new = masks ^ bit
    return np.where(ok, new, masks), np.where(ok, amp * sign, 0.0)


def hamiltonian_terms(h: np.ndarray, eri: np.ndarray):
    """Yield (coef, [(mode, dagger), ...]) for every term of Eq. (hamil), the
    operator list written left to right (the rightmost acts first)."""
    L = h.shape[0]
    for i in range(L):
        for j in range(L):
            if h[i, j] != 0.0:
                for s in range(2):
                    yield h[i, j], [(2 * i + s, True), (2 * j + s, False)]
    for i in range(L):
        for j in range(L):
            for k in range(L):
                for l in range(L):
                    v = eri[i, j, k, l]
                    if v == 0.0:
                        continue
                    for s in range(2):
                        for t in range(2):
                            yield 0.5 * v, [(2 * i + s, True), (2 * k + t, True),
                                            (2 * l + t, False), (2 * j + s, False)]


def hamiltonian(h: np.ndarray, eri: np.ndarray, dets: np.ndarray, e0: float = 0.0) -> np.ndarray:
    """Dense Hamiltonian matrix <D_a|H|D_b> on the determinant list ``dets``,
    built by letting every term of Eq. (hamil) act on every determinant."""
    n = len(dets)
    H = np.zeros((n, n))
    col = np.arange(n)
    for coef, ops in hamiltonian_terms(h, eri):
        m = dets.copy()
        a = np.ones(n)
        for mode, dag in reversed(ops):
            m, a = apply_op(m, a, mode, dag)
        nz = a != 0.0
        if not nz.any():
            continue
        row = np.searchsorted(dets, m[nz])
        hit = (row < n)
        hit[hit] &= dets[row[hit]] == m[nz][hit]
        np.add.at(H, (row[hit], col[nz][hit]), coef * a[nz][hit])
    H[np.diag_indices(n)] += e0
    return H


def h_on_determinant(h: np.ndarray, eri: np.ndarray, mask: int, e0: float = 0.0):
    """H|D> for one determinant D at any L, as (masks, coefficients) with
    duplicates merged; every term of Eq. (hamil) is applied (vectorised over
    terms).  <D'|H|D> for all D' follows, and by hermiticity <D|H|D'>."""
    L = h.shape[0]
    I, J = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    out_m, out_c = [], []
    for s in range(2):
        coef = h[I, J].ravel()
        m = np.full(coef.shape, mask, dtype=np.uint64)
        a = np.ones(coef.shape)
        m, a = apply_op(m, a, (2 * J + s).ravel(), False)
        m, a = apply_op(m, a, (2 * I + s).ravel(), True)
        out_m.append(m)
        out_c.append(coef * a)
    idx = np.indices((L, L, L, L)).reshape(4, -1)
    i, j, k, l = idx
    v = 0.5 * eri.reshape(-1)
    for s in range(2):
        for t in range(2):
            m = np.full(v.shape, mask, dtype=np.uint64)
            a = np.ones(v.shape)
            m, a = apply_op(m, a, 2 * j + s, False)
            m, a = apply_op(m, a, 2 * l + t, False)
            m, a = apply_op(m, a, 2 * k + t, True)
            m, a = apply_op(m, a, 2 * i + s, True)
            out_m.append(m)
            out_c.append(v * a)
    m = np.concatenate(out_m)
    c = np.concatenate(out_c)
    keep = c != 0.0
    m, c = m[keep], c[keep]
    uniq, inv = np.unique(m, return_inverse=True)
    acc = np.zeros(len(uniq))
    np.add.at(acc, inv, c)
    if e0 != 0.0:
        hit = np.searchsorted(uniq, np.uint64(mask))
        if hit < len(uniq) and uniq[hit] == mask:
            acc[hit] += e0
        else:
            uniq = np.append(uniq, np.uint64(mask))
            acc = np.append(acc, e0)
    return uniq, acc


# ---------------------------------------------------------------------------
# observables
# ---------------------------------------------------------------------------

def one_rdm(psi: np.ndarray, dets: np.ndarray, L: int) -> np.ndarray:
    """gamma_ij = sum_s <psi| a+_{is} a_{js} |psi> (Section 3.2, 1BRDM)."""
    n = len(dets)
    g = np.zeros((L, L), dtype=np.complex128)
    for i in range(L):
        for j in range(L):
            for s in range(2):
                m, a = apply_op(dets, np.ones(n), 2 * j + s, False)
                m, a = apply_op(m, a, 2 * i + s, True)
                nz = a != 0.0
                row = np.searchsorted(dets, m[nz])
                g[i, j] += np.sum(np.conj(psi[row]) * a[nz] * psi[nz])
    return g


def two_rdm(psi: np.ndarray, dets: np.ndarray, L: int) -> np.ndarray:
    """Gamma_ijkl = sum_{s,t} <psi| a+_{is} a+_{kt} a_{lt} a_{js} |psi>, the
    chemist-order partner of (ij|kl) in Eq. (hamil)."""
    n = len(dets)
    G = np.zeros((L, L, L, L), dtype=np.complex128)
    for i in range(L):
        for j in range(L):
            for k in range(L):
                for l in range(L):
                    for s in range(2):
                        for t in range(2):
                            m, a = apply_op(dets, np.ones(n), 2 * j + s, False)
                            m, a = apply_op(m, a, 2 * l + t, False)
                            m, a = apply_op(m, a, 2 * k + t, True)
                            m, a = apply_op(m, a, 2 * i + s, True)
                            nz = a != 0.0
                            if not nz.any():
                                continue
                            row = np.searchsorted(dets, m[nz])
                            G[i, j, k, l] += np.sum(np.conj(psi[row]) * a[nz] * psi[nz])
    return G


def transition_rdm(bra: np.ndarray, ket: np.ndarray, dets: np.ndarray, L: int) -> np.ndarray:
    """T_ij = sum_s <bra| a+_{is} a_{js} |ket> for two vectors on the same
    determinant list (the 1BRDM of Section 3.2 between two states)."""
    n = len(dets)
    g = np.zeros((L, L), dtype=np.complex128)
    for i in range(L):
        for j in range(L):
            for s in range(2):
                m, a = apply_op(dets, np.ones(n), 2 * j + s, False)
                m, a = apply_op(m, a, 2 * i + s, True)
                nz = a != 0.0
                row = np.searchsorted(dets, m[nz])
                g[i, j] += np.sum(np.conj(bra[row]) * a[nz] * ket[nz])
    return g


def apply_to_vector(psi: np.ndarray, dets: np.ndarray, out_dets: np.ndarray, mode: int,
                    dagger: bool) -> np.ndarray:
    """a_mode psi or a+_mode psi, expressed on the determinant list
    ``out_dets`` of the target sector."""
    m, a = apply_op(dets, np.asarray(psi, dtype=np.complex128), mode, dagger)
    nz = a != 0.0
    out = np.zeros(len(out_dets), dtype=np.complex128)
    row = np.searchsorted(out_dets, m[nz])
    np.add.at(out, row, a[nz])
    return out


def green_function(h: np.ndarray, eri: np.ndarray, psi0: np.ndarray, dets: np.ndarray, L: int,
                   i: int, j: int, taus, e0: float = 0.0) -> np.ndarray:
    """Spin-summed, normalised one-particle Green's function of Eq. (green_time)
    for tau = t - t' >= 0 (hbar = 1):

        G_ij(tau) = -i sum_s <psi0| a+_{is} exp(+i H tau) a_{js} |psi0>
                       / sum_s <psi0| a+_{is} a_{js} |psi0>.

    a_{js}|psi0> lives in the sector with one electron of spin s fewer; it is
    propagated backwards in time there exactly (Eq. time_evo_opera with
    t -> -tau) and projected on a_{is}|psi0>."""
    na = int(np.bitwise_count(np.uint64(dets[0]) & np.uint64(0x5555555555555555)))
    nb = int(np.bitwise_count(np.uint64(dets[0]) & np.uint64(0xAAAAAAAAAAAAAAAA)))
    taus = np.atleast_1d(np.asarray(taus, dtype=float))
    num = np.zeros(len(taus), dtype=np.complex128)
    den = 0.0 + 0.0j
    for s in range(2):
        if (na, nb)[s] == 0:
            continue
        dm = basis(L, na - (s == 0), nb - (s == 1))
        Hm = hamiltonian(h, eri, dm, e0)
        chi_j = apply_to_vector(psi0, dets, dm, 2 * j + s, False)
        chi_i = apply_to_vector(psi0, dets, dm, 2 * i + s, False)
        den += np.vdot(chi_i, chi_j)
        for t, tau in enumerate(taus):
            num[t] += np.vdot(chi_i, exact_evolve(Hm, chi_j, -tau))
    return -1j * num / den


def energy(H: np.ndarray, psi: np.ndarray) -> float:
    return float(np.real(np.vdot(psi, H @ psi) / np.vdot(psi, psi)))


# ---------------------------------------------------------------------------
# time evolution on vectors
# ---------------------------------------------------------------------------

def exact_evolve(H: np.ndarray, psi: np.ndarray, t: float) -> np.ndarray:
    """exp(-i H t) psi by diagonalisation (Eq. time_evo_opera, hbar = 1)."""
    w, U = np.linalg.eigh(H)
    return U @ (np.exp(-1j * w * t) * (U.conj().T @ psi))


def rk4_step(H: np.ndarray, psi: np.ndarray, dt: float) -> np.ndarray:
    """One RK4 step: stages k1..k4 and Eq. (rk_add)."""
    k1 = -1j * dt * (H @ psi)
    k2 = -1j * dt * (H @ (psi + 0.5 * k1))
    k3 = -1j * dt * (H @ (psi + 0.5 * k2))
    k4 = -1j * dt * (H @ (psi + k3))
    return psi + (k1 + 2.0 * (k2 + k3) + k4) / 6.0


def krylov_coefficients(N: np.ndarray, Hk: np.ndarray, dt: float):
    """c = [exp(-i dt N^-1 H)]_{k0} of Eq. (krylov_evo) through canonical
    orthogonalisation.  Returns (c, number of discarded directions)."""
    n, V = np.linalg.eigh(N)
    keep = n > EIG_DROP * n.max()
    X = V[:, keep] / np.sqrt(n[keep])
    M = X.conj().T @ Hk @ X
    M = 0.5 * (M + M.conj().T)
    lam, U = np.linalg.eigh(M)
    b = X.conj().T @ N[:, 0]
    c = X @ (U @ (np.exp(-1j * dt * lam) * (U.conj().T @ b)))
    return c, int((~keep).sum())


def krylov_step(H: np.ndarray, psi: np.ndarray, dt: float, m: int,
                orthogonal: bool = True, return_basis: bool = False):
    """One Krylov step with m basis vectors (phi_0 = psi).

    orthogonal=True: Eq. (kry_orth), full Gram-Schmidt against all previous
    vectors; orthogonal=False: Eq. (kry_non), phi_{k+1} = H phi_k normalised.
    Then Eq. (krylov_evo) with the measured overlap matrix N.  Returns the new
    vector, and with return_basis=True also the basis (columns phi_0..phi_{m-1}).
    """
    phis = [psi.astype(np.complex128)]
    for k in range(m - 1):
        hv = H @ phis[k]
        v = hv.copy()
        if orthogonal:
            for j in range(k + 1):
                v = v - (np.vdot(phis[j], hv) / np.vdot(phis[j], phis[j])) * phis[j]
        v = v / np.linalg.norm(v)
        phis.append(v)
    P = np.array(phis).T
    N = P.conj().T @ P
    Hk = P.conj().T @ (H @ P)
    c, _ = krylov_coefficients(N, Hk, dt)
    return (P @ c, P) if return_basis else P @ c
