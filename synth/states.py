"""Seeded initial states: determinant occupations and random block-sparse MPS.

Local states of one spatial orbital, in the order used everywhere in this
project: 0 = |0>, 1 = |up>, 2 = |down>, 3 = |up down> (spin-orbital order
1up, 1down, 2up, ... of Eq. (1)).  Their charges (n, 2 S_z) are (0,0), (1,1),
(1,-1), (2,0).

``random_mps`` returns dense site tensors A[i] of shape (D_l, 4, D_r) together
with the charge label of every bond basis vector, so that any consumer can cut
them into symmetry blocks.  Entries outside the allowed blocks
(q_right = q_left + q_sigma) are zero.
"""
from __future__ import annotations

from math import comb

import numpy as np

SITE_CHARGE = ((0, 0), (1, 1), (1, -1), (2, 0))


def aufbau_occupation(L: int, n_elec: int) -> list[int]:
    """Lowest orbitals doubly occupied in index order; an odd electron is up."""
    occ = [0] * L
    for i in range(n_elec // 2):
        occ[i] = 3
    if n_elec % 2:
        occ[n_elec // 2] = 1
    return occ


def hole_occupation(L: int, n_elec: int, orbital: int, spin: str = "down") -> list[int]:
    """Aufbau determinant of n_elec electrons with one electron of the given
    spin removed from ``orbital`` (the sudden-ionisation initial state)."""
    occ = aufbau_occupation(L, n_elec)
    bit = 2 if spin == "down" else 1
    if not occ[orbital] & bit:
        raise ValueError("orbital %d has no %s electron" % (orbital, spin))
    occ[orbital] &= ~bit
    return occ


def occupation_charge(occ) -> tuple[int, int]:
    n = sum(SITE_CHARGE[o][0] for o in occ)
    s = sum(SITE_CHARGE[o][1] for o in occ)
    return n, s


def bond_sectors(L: int, n_elec: int, two_sz: int, k: int):
    """Charges (n, 2Sz) that can sit on bond k (after k sites) of a state with
    total charge (n_elec, two_sz), with the number of left and right
    configurations realising each: list of (n, s, dim_left, dim_right)."""
    na_tot = (n_elec + two_sz) // 2
    nb_tot = (n_elec - two_sz) // 2
    out = []
    for na in range(0, k + 1):
        for nb in range(0, k + 1):
            ra, rb = na_tot - na, nb_tot - nb
            if not (0 <= ra <= L - k and 0 <= rb <= L - k):
                continue
            out.append((na + nb, na - nb, comb(k, na) * comb(k, nb),
                        comb(L - k, ra) * comb(L - k, rb)))
    out.sort(key=lambda t: (t[0], t[1]))
    return out


def _allocate(maxdims: list[int], D: int) -> list[int]:
    tot = sum(maxdims)
    if tot <= D:
        return list(maxdims)
    raw = [D * m / tot for m in maxdims]
    dims = [min(m, int(np.floor(r))) for m, r in zip(maxdims, raw)]
    rest = D - sum(dims)
    order = sorted(range(len(raw)), key=lambda i: (-(raw[i] - np.floor(raw[i])), i))
    while rest > 0:
        progressed = False
        for i in order:
            if rest == 0:
                break
            if dims[i] < maxdims[i]:
                dims[i] += 1
                rest -= 1
                progressed = True
        if not progressed:
            break
    return dims


def random_mps(L: int, n_elec: int, two_sz: int, D: int, seed: int = 0):
    """Seeded random MPS with bond dimension <= D.

    Each bond's sector dimensions are proportional to min(#left, #right)
    configurations, capped by them (largest-remainder rounding to D), then
    clamped so that every sector is reachable from both neighbouring bonds.
    Entries of allowed blocks are complex normal; each site is scaled so that
    its columns have unit mean square norm.

    Returns (tensors, labels): tensors[i] is complex128 (D_i, 4, D_{i+1});
    labels[k] is int64 (D_k, 2) with the (n, 2Sz) of each bond basis vector.
    """
    rng = np.random.default_rng(seed)
    secs = [bond_sectors(L, n_elec, two_sz, k) for k in range(L + 1)]
    dims = []
    for k in range(L + 1):
        dims.append({(n, s): d for (n, s, _, _), d in
                     zip(secs[k], _allocate([min(a, b) for _, _, a, b in secs[k]], D))})
    for _ in range(2 * L + 2):
        changed = False
        for k in range(1, L + 1):
            for q in list(dims[k]):
                lim = sum(dims[k - 1].get((q[0] - c[0], q[1] - c[1]), 0) for c in SITE_CHARGE)
                if dims[k][q] > lim:
                    dims[k][q] = lim
                    changed = True
        for k in range(L - 1, -1, -1):
            for q in list(dims[k]):
                lim = sum(dims[k + 1].get((q[0] + c[0], q[1] + c[1]), 0) for c in SITE_CHARGE)
                if dims[k][q] > lim:
                    dims[k][q] = lim
                    changed = True
        if not changed:
            break
    labels = []
    for k in range(L + 1):
        rows = []
        for q in sorted(dims[k]):
            rows.extend([q] * dims[k][q])
        labels.append(np.array(rows, dtype=np.int64).reshape(-1, 2))
    tensors = []
    for i in range(L):
        ql, qr = labels[i], labels[i + 1]
        A = np.zeros((len(ql), 4, len(qr)), dtype=np.complex128)
        lsecs = sorted(dims[i])
        for qa in lsecs:
            if dims[i][qa] == 0:
                continue
            ia = np.where((ql[:, 0] == qa[0]) & (ql[:, 1] == qa[1]))[0]
            for sig, c in enumerate(SITE_CHARGE):
                qb = (qa[0] + c[0], qa[1] + c[1])
                ib = np.where((qr[:, 0] == qb[0]) & (qr[:, 1] == qb[1]))[0]
                if len(ib) == 0:
                    continue
                re = rng.standard_normal((len(ia), len(ib)))
                im = rng.standard_normal((len(ia), len(ib)))
                A[np.ix_(ia, [sig], ib)] = (re + 1j * im)[:, None, :] / np.sqrt(2.0)
        colnorm = np.sum(np.abs(A) ** 2, axis=(0, 1))
        A /= np.sqrt(max(colnorm.mean(), 1e-300))
        tensors.append(A)
    return tensors, labels
