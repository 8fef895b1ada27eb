"""Pins for the oracle's algorithmic FLOP count of the transfer-matrix overlap
(Section 2.1): a brute-force count over individual indices with structural
masks, and the closed form for two determinants."""
import numpy as np
import pytest

import synth
from oracle import fci
from oracle import mps as om


def _brute_overlap_flops(bra, ket):
    """Counts multiply-adds index by index.  E, A^sigma and B^sigma are
    replaced by 0/1 masks of their structurally non-zero entries (a site
    entry is allowed when the right label equals the left label plus the
    charge of sigma; E_0 is the 1x1 boundary); a product E[a,a'] A[a',b'] is
    counted when X[a,b'] reaches some bra entry, B[a,b] X[a,b'] whenever both
    factors are non-zero.  The next E is the mask of B^dagger X."""
    E = np.ones((1, 1), dtype=np.int64)
    total = 0
    for i in range(bra.L):
        ql, qr = bra.labels[i], bra.labels[i + 1]
        kl, kr = ket.labels[i], ket.labels[i + 1]
        same = (qr[:, None, :] == kr[None, :, :]).all(-1).astype(np.int64)
        En = np.zeros((len(qr), len(kr)), dtype=bool)
        for c in om.SITE_Q:
            Am = (kl[:, None, :] + c == kr[None, :, :]).all(-1).astype(np.int64)
            Bm = (ql[:, None, :] + c == qr[None, :, :]).all(-1).astype(np.int64)
            used = ((Bm @ same) > 0).astype(np.int64)
            total += 8 * int(np.einsum("ij,jk,ik->", E, Am, used))
            X = ((E @ Am) > 0).astype(np.int64)
            total += 8 * int(np.einsum("ab,ac->", Bm, X))
            En |= (Bm.T @ X) > 0
        E = En.astype(np.int64)
    return total


def _sparse_superposition(L, n_alpha, n_beta, k, rng):
    dets = fci.basis(L, n_alpha, n_beta)
    pick = rng.choice(len(dets), size=min(k, len(dets)), replace=False)
    vec = np.zeros(len(dets), dtype=np.complex128)
    vec[pick] = rng.normal(size=len(pick)) + 1j * rng.normal(size=len(pick))
    return om.from_fock(om.sector_to_fock(vec, dets, L), L)


@pytest.mark.parametrize("seed", range(4))
def test_overlap_flops_equal_brute_force_random_mps(seed):
    L = 6
    A, q = synth.random_mps(L, 5, 1, 12 + 4 * seed, seed=10 + seed)
    B, qb = synth.random_mps(L, 5, 1, 7 + 3 * seed, seed=20 + seed)
    ket, bra = om.from_arrays(A, q), om.from_arrays(B, qb)
    assert om.overlap_flops(bra, ket) == _brute_overlap_flops(bra, ket) > 0
    assert om.overlap_flops(ket, bra) == _brute_overlap_flops(ket, bra)


def test_overlap_flops_equal_brute_force_sparse_superpositions():
    """Superpositions of a few determinants have bond sectors that exist on
    both sides yet carry no non-zero block of E_i; the count must leave them
    out, and the brute force does so without a sector list."""
    rng = np.random.default_rng(5)
    seen_unreached = False
    for _ in range(30):
        ket = _sparse_superposition(5, 3, 2, 3, rng)
        bra = _sparse_superposition(5, 3, 2, 3, rng)
        n = om.overlap_flops(bra, ket)
        assert n == _brute_overlap_flops(bra, ket)
        # the same count with every common sector treated as reached
        full = 0
        for i in range(5):
            bl, kl = om._sector_dims(bra.labels[i]), om._sector_dims(ket.labels[i])
            br, kr = om._sector_dims(bra.labels[i + 1]), om._sector_dims(ket.labels[i + 1])
            for qs in set(bl) & set(kl):
                for c in om.SITE_Q:
                    qp = (qs[0] + int(c[0]), qs[1] + int(c[1]))
                    if qp in br and qp in kr:
                        full += 8 * bl[qs] * kl[qs] * kr[qp] + 8 * br[qp] * bl[qs] * kr[qp]
        seen_unreached |= full != n
    assert seen_unreached


def test_overlap_flops_of_determinants_closed_form():
    """Two determinants (bond dimension 1): a site adds 16 FLOPs (one 1x1x1
    product per stage) while the accumulated charges of both still agree."""
    rng = np.random.default_rng(9)
    L = 8
    for _ in range(40):
        da = rng.permutation([3, 3, 1, 2, 0, 0, 0, 0])
        db = rng.permutation([3, 3, 1, 2, 0, 0, 0, 0])
        qa = np.cumsum(om.SITE_Q[da], axis=0)
        qb = np.cumsum(om.SITE_Q[db], axis=0)
        agree = 0
        while agree < L and (qa[agree] == qb[agree]).all():
            agree += 1
        n = om.overlap_flops(om.from_determinant(db), om.from_determinant(da))
        assert n == 16 * agree
    same = om.from_determinant([3, 1, 0, 2])
    assert om.overlap_flops(same, same) == 16 * 4
