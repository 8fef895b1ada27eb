"""Pins for oracle C (block-sparse MPS with the Hamiltonian as an MPO) against
oracle A (full CI), oracle B (dense-projection MPS fits) and exact identities.

The MPO is pinned by contracting it to a matrix and comparing with the full-CI
Hamiltonian on the whole Fock space, with integrals that have no index
symmetry (so a transposed index or a dropped spin sum shows), and with a
constant e0.  The fit machinery is pinned by running the same schedules as
oracle B, which projects the exact target vector, and comparing the states.
"""
import numpy as np
import pytest

import synth
from oracle import bsmps as ob
from oracle import fci
from oracle import mps as om


def _fock_masks(L):
    """All 4^L determinant masks, listed in Fock index order of oracle.mps."""
    masks = np.arange(4 ** L, dtype=np.uint64)
    order = np.argsort(om.fock_index(masks, L))
    return masks[order]


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_mpo_matrix_equals_full_ci_on_fock_space(L):
    rng = np.random.default_rng(100 + L)
    h = rng.standard_normal((L, L))                 # no symmetry on purpose
    eri = rng.standard_normal((L, L, L, L))
    e0 = 0.37
    M = ob.mpo_to_matrix(ob.hamiltonian_mpo(h, eri, e0))
    dets = _fock_masks(L)
    srt = np.argsort(dets)
    Hs = fci.hamiltonian(h, eri, dets[srt], e0)     # rows/cols in sorted-mask order
    inv = np.empty_like(srt)
    inv[srt] = np.arange(len(srt))
    H = Hs[np.ix_(inv, inv)]
    assert np.max(np.abs(M - H)) < 1e-12


def test_mpo_bond_dimension_and_boundaries():
    I = synth.make_integrals(8, seed=0)
    mpo = ob.hamiltonian_mpo(I.h, I.eri)
    dims = mpo.bond_dims()
    assert dims[0] == 1 and dims[-1] == 1
    # complementary-operator count: start and done, 4L single operators,
    # O(8 min(k, L-k)^2) pairs on the smaller side (k spatial orbitals left)
    for k, d in enumerate(dims[1:-1], start=1):
        m = min(k, 8 - k)
        assert d <= 2 + 4 * 8 + 8 * m * m + 8 * m
    # bond 1 exactly: start, done, 4 single operators and 6 non-vanishing
    # pairs of site 0 (two-against-two splits are named on the left in the
    # left half), and the 28 single operators of sites 1..7 that close the
    # three-operator left parts
    assert dims[1] == 2 + 4 + 6 + 28
    # every channel charge is a difference of two site charges summed
    for qs in mpo.charges:
        for q in qs:
            assert abs(q[0]) <= 2 and abs(q[1]) <= 2


def _sector_system(L, n_elec, two_sz, seed):
    I = synth.make_integrals(L, seed=seed)
    na, nb = (n_elec + two_sz) // 2, (n_elec - two_sz) // 2
    return I, om.System.build(I.h, I.eri, na, nb)


def test_sandwich_and_overlap_equal_contracted_vectors():
    L = 6
    I, sys_ = _sector_system(L, 5, 1, 0)
    mpo = ob.hamiltonian_mpo(I.h, I.eri)
    A, qa = synth.random_mps(L, 5, 1, 20, seed=1)
    B, qb = synth.random_mps(L, 5, 1, 14, seed=2)
    a, b = ob.from_dense(A, qa), ob.from_dense(B, qb)
    va, vb = sys_.vec(om.from_arrays(A, qa)), sys_.vec(om.from_arrays(B, qb))
    ref = np.vdot(vb, sys_.H @ va)
    assert abs(ob.sandwich(mpo, b, a) - ref) < 1e-11 * abs(ref)
    ref2 = np.vdot(vb, va)
    assert abs(ob.overlap(b, a) - ref2) < 1e-12 * np.linalg.norm(va) * np.linalg.norm(vb)


def test_overlap_flop_count_equals_transfer_count():
    A, qa = synth.random_mps(8, 7, 1, 40, seed=3)
    B, qb = synth.random_mps(8, 7, 1, 25, seed=4)
    fl = ob.Flops()
    ob.overlap(ob.from_dense(B, qb), ob.from_dense(A, qa), fl)
    assert fl.total == om.overlap_flops(om.from_arrays(B, qb), om.from_arrays(A, qa))


def test_dense_roundtrip_and_coefficients():
    A, q = synth.random_mps(6, 6, 0, 16, seed=5)
    m = ob.from_dense(A, q)
    t, lab = ob.to_dense(m)
    v1 = om.to_fock(om.from_arrays(A, q))
    v2 = om.to_fock(om.from_arrays(t, lab))
    assert np.max(np.abs(v1 - v2)) < 1e-14
    rng = np.random.default_rng(0)
    dets = fci.basis(6, 3, 3)
    occs = []
    for msk in rng.choice(dets, 6):
        occs.append([((int(msk) >> (2 * i)) & 1) + 2 * ((int(msk) >> (2 * i + 1)) & 1)
                     for i in range(6)])
    ref = [om.coefficient(om.from_arrays(A, q), o) for o in occs]
    assert np.max(np.abs(ob.coefficients(m, occs) - ref)) < 1e-13


def _fid(u, v):
    return abs(np.vdot(u, v)) / (np.linalg.norm(u) * np.linalg.norm(v))


@pytest.mark.parametrize("sched,D", [((1, 2), 200), ((1, 2), 12), ((0, 2), 30)])
def test_apply_H_equals_projection_oracle(sched, D):
    L = 6
    I, sys_ = _sector_system(L, 5, 1, 1)
    mpo = ob.hamiltonian_mpo(I.h, I.eri)
    A, q = synth.random_mps(L, 5, 1, 30, seed=6)
    alpha = 0.3 - 0.7j
    ref = om.apply_H(sys_, om.from_arrays(A, q), alpha,
                     om.Schedule(D, 0.0, sched[0], sched[1]))
    got = ob.apply_H(mpo, ob.from_dense(A, q), alpha, ob.Schedule(D, 0.0, sched[0], sched[1]))
    vr = sys_.vec(ref)
    vg = sys_.vec(om.from_arrays(*ob.to_dense(got)))
    assert np.linalg.norm(vg - vr) < 1e-10 * np.linalg.norm(vr)
    assert got.bond_dims() == ref.bond_dims
    if D >= 200:   # untruncated: the exact alpha H |psi>
        exact = alpha * (sys_.H @ sys_.vec(om.from_arrays(A, q)))
        assert np.linalg.norm(vg - exact) < 1e-10 * np.linalg.norm(exact)


def test_sum_fit_equals_projection_oracle_truncated():
    L = 6
    _, sys_ = _sector_system(L, 6, 0, 2)
    A, qa = synth.random_mps(L, 6, 0, 20, seed=7)
    B, qb = synth.random_mps(L, 6, 0, 20, seed=8)
    terms_o = [(1.0, om.from_arrays(A, qa)), (0.4 - 0.2j, om.from_arrays(B, qb))]
    terms_b = [(1.0, ob.from_dense(A, qa)), (0.4 - 0.2j, ob.from_dense(B, qb))]
    for D, eps in ((10, 0.0), (40, 1e-6), (64, 0.0)):
        ref = om.sum_fit(sys_, terms_o, om.Schedule(D, eps, 1, 1))
        got = ob.sum_fit(terms_b, ob.Schedule(D, eps, 1, 1))
        vr = sys_.vec(ref)
        vg = sys_.vec(om.from_arrays(*ob.to_dense(got)))
        assert np.linalg.norm(vg - vr) < 1e-10 * np.linalg.norm(vr)


def test_rk4_and_krylov_steps_equal_projection_oracle_and_full_ci():
    L = 6
    I, sys_ = _sector_system(L, 5, 1, 3)
    mpo = ob.hamiltonian_mpo(I.h, I.eri)
    occ = synth.hole_occupation(L, 6, 2)
    sch_o, sch_b = om.Schedule(200, 0.0, 3, 1), ob.Schedule(200, 0.0, 3, 1)
    psi_o, psi_b = om.from_determinant(occ), ob.from_determinant(occ)
    v0 = sys_.vec(psi_o)
    r = ob.rk4_step(mpo, psi_b, 0.05, sch_b)
    vr = sys_.vec(om.from_arrays(*ob.to_dense(r)))
    assert np.linalg.norm(vr - fci.rk4_step(sys_.H, v0, 0.05)) < 1e-10
    assert np.linalg.norm(vr - sys_.vec(om.rk4_step(sys_, psi_o, 0.05, sch_o))) < 1e-10
    k, c, N, Hk = ob.krylov_step(mpo, psi_b, 0.1, 4, sch_b)
    vk = sys_.vec(om.from_arrays(*ob.to_dense(k)))
    ko, co, No, Hko = om.krylov_step(sys_, psi_o, 0.1, 4, sch_o)
    assert np.linalg.norm(vk - fci.krylov_step(sys_.H, v0, 0.1, 4)) < 1e-10
    assert np.linalg.norm(vk - sys_.vec(ko)) < 1e-10
    assert np.max(np.abs(N - No)) < 1e-11 and np.max(np.abs(Hk - Hko)) < 1e-11
    # the plain (non-orthogonal) basis of Eq. kry_non
    kn, _, _, _ = ob.krylov_step(mpo, psi_b, 0.1, 4, sch_b, orthogonal=False)
    kno, _, _, _ = om.krylov_step(sys_, psi_o, 0.1, 4, sch_o, orthogonal=False)
    assert np.linalg.norm(sys_.vec(om.from_arrays(*ob.to_dense(kn))) - sys_.vec(kno)) < 1e-10


def test_truncated_krylov_step_equals_projection_oracle():
    L = 6
    I, sys_ = _sector_system(L, 5, 1, 4)
    mpo = ob.hamiltonian_mpo(I.h, I.eri)
    A, q = synth.random_mps(L, 5, 1, 24, seed=9)
    sch_o, sch_b = om.Schedule(16, 1e-10, 1, 1), ob.Schedule(16, 1e-10, 1, 1)
    ko = om.krylov_step(sys_, om.from_arrays(A, q), 0.05, 3, sch_o)[0]
    kb = ob.krylov_step(mpo, ob.from_dense(A, q), 0.05, 3, sch_b)[0]
    vo, vb = sys_.vec(ko), sys_.vec(om.from_arrays(*ob.to_dense(kb)))
    assert np.linalg.norm(vb - vo) < 1e-9 * np.linalg.norm(vo)


def test_one_rdm_equals_full_ci():
    L = 6
    I, sys_ = _sector_system(L, 5, 1, 5)
    A, q = synth.random_mps(L, 5, 1, 20, seed=10)
    g = ob.one_rdm(ob.from_dense(A, q))
    ref = fci.one_rdm(sys_.vec(om.from_arrays(A, q)), sys_.dets, L)
    assert np.max(np.abs(g - ref)) < 1e-12 * np.max(np.abs(ref))
    # a determinant has its occupations on the diagonal and nothing else
    occ = [3, 1, 0, 2, 3, 0]
    gd = ob.one_rdm(ob.from_determinant(occ))
    assert np.max(np.abs(gd - np.diag([2, 1, 0, 1, 2, 0]))) < 1e-15


def test_energy_of_determinant_is_slater_condon():
    L = 8
    I = synth.make_integrals(L, seed=11)
    mpo = ob.hamiltonian_mpo(I.h, I.eri, 0.25)
    occ = synth.hole_occupation(L, 8, 3)
    d = ob.from_determinant(occ)
    e = ob.sandwich(mpo, d, d)
    dets = fci.basis(L, 4, 3)
    H = fci.hamiltonian(I.h, I.eri, dets, 0.25)
    col = np.searchsorted(dets, np.uint64(fci.occupation_mask(occ)))
    assert abs(e - H[col, col]) < 1e-12


def _energy(mpo, psi):
    return ob.sandwich(mpo, psi, psi).real / ob.overlap(psi, psi).real


def test_energy_gradient_equals_full_ci_projection():
    # dE/dconj(A_i) = M_i^+ (H v - E v) / |v|^2 with M_i = dv/dA_i, the
    # sector vector of the MPS differentiated by each entry of site i
    # (columns by unit perturbation: v is linear in A_i), H the full-CI
    # Hamiltonian of the sector
    L = 4
    I, sys_ = _sector_system(L, 4, 0, 12)
    mpo = ob.hamiltonian_mpo(I.h, I.eri)
    A, q = synth.random_mps(L, 4, 0, 8, seed=13)
    psi = ob.from_dense(A, q)
    E, G = ob.energy_gradient(mpo, psi)
    v = sys_.vec(om.from_arrays(A, q))
    Hv = sys_.H @ v
    n2 = np.vdot(v, v).real
    assert abs(E - np.vdot(v, Hv).real / n2) < 1e-12
    r = (Hv - E * v) / n2
    for i in range(L):
        for k, blk in psi.sites[i].items():
            for (a, b) in [(0, 0), (blk.shape[0] - 1, blk.shape[1] - 1)]:
                # column of M_i: the state with A_i replaced by the unit
                # tensor of entry (a, sigma, b) of this block
                unit = psi.copy()
                unit.sites[i] = {kk: np.zeros_like(x) for kk, x in unit.sites[i].items()}
                unit.sites[i][k][a, b] = 1.0
                col = sys_.vec(om.from_arrays(*ob.to_dense(unit)))
                ref = np.vdot(col, r)
                assert abs(G[i][k][a, b] - ref) < 1e-12 * max(1.0, abs(ref))


def test_energy_gradient_finite_differences_and_scale_invariance():
    L = 6
    I = synth.make_integrals(L, seed=14)
    mpo = ob.hamiltonian_mpo(I.h, I.eri, 0.1)
    A, q = synth.random_mps(L, 5, 1, 12, seed=15)
    psi = ob.from_dense(A, q)
    E, G = ob.energy_gradient(mpo, psi)
    rng = np.random.default_rng(16)
    h = 1e-6
    for i in (0, 2, L - 1):
        keys = list(psi.sites[i].keys())
        for _ in range(3):
            k = keys[rng.integers(len(keys))]
            a, b = rng.integers(psi.sites[i][k].shape[0]), rng.integers(psi.sites[i][k].shape[1])
            for d in (1.0, 1j):
                p, m = psi.copy(), psi.copy()
                p.sites[i][k][a, b] += h * d
                m.sites[i][k][a, b] -= h * d
                fd = (_energy(mpo, p) - _energy(mpo, m)) / (2 * h)
                # dE = 2 Re(conj(g) dz) for a real E of a complex z
                assert abs(fd - 2 * (np.conj(G[i][k][a, b]) * d).real) < 1e-7
    # E is invariant under A_i -> (1 + t) A_i: <A_i, dE/dconj(A_i)> = 0
    for i in range(L):
        s = sum(np.vdot(psi.sites[i][k], G[i][k]) for k in G[i])
        assert abs(s) < 1e-12 * abs(E)


def _random_site(site: dict, rng) -> dict:
    return {k: rng.standard_normal(b.shape) + 1j * rng.standard_normal(b.shape)
            for k, b in site.items()}


def _site_vectors(sys_, psi, i):
    """M_i: the sector vectors of psi with site i replaced by each unit tensor
    (one column per entry, entries in the order of _flat)."""
    cols = []
    for k, blk in psi.sites[i].items():
        for a in range(blk.shape[0]):
            for b in range(blk.shape[1]):
                unit = psi.copy()
                unit.sites[i] = {kk: np.zeros_like(x) for kk, x in unit.sites[i].items()}
                unit.sites[i][k][a, b] = 1.0
                cols.append(sys_.vec(om.from_arrays(*ob.to_dense(unit))))
    return np.array(cols).T


def _flat(site: dict, like: dict):
    return np.concatenate([site[k].reshape(-1) for k in like])


def test_local_matvec_equals_full_ci_projection():
    # y = M_i^+ H M_i x: the local operator is H in the coordinates of site i
    # (psi's other sites fixed, no gauge assumed), H the full-CI Hamiltonian
    L = 4
    I, sys_ = _sector_system(L, 4, 0, 40)
    mpo = ob.hamiltonian_mpo(I.h, I.eri, 0.3)
    A, q = synth.random_mps(L, 4, 0, 8, seed=41)
    psi = ob.from_dense(A, q)
    rng = np.random.default_rng(42)
    for i in range(L):
        x = _random_site(psi.sites[i], rng)
        y = ob.local_matvec(mpo, psi, i, x)
        assert set(y) == set(psi.sites[i])
        M = _site_vectors(sys_, psi, i)
        ref = M.conj().T @ ((sys_.H + 0.3 * np.eye(len(sys_.H))) @ (M @ _flat(x, psi.sites[i])))
        got = _flat(y, psi.sites[i])
        assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_local_matvec_hermitian_and_reproduces_the_energy():
    # <z, H_i x> = conj(<x, H_i z>), and with x = A_i the site's own tensor
    # <A_i, H_i A_i> = <psi|H|psi> at every site
    L = 6
    I = synth.make_integrals(L, seed=43)
    mpo = ob.hamiltonian_mpo(I.h, I.eri)
    A, q = synth.random_mps(L, 5, 1, 12, seed=44)
    psi = ob.from_dense(A, q)
    e = ob.sandwich(mpo, psi, psi)
    rng = np.random.default_rng(45)
    for i in range(L):
        keys = psi.sites[i]
        x, z = _random_site(keys, rng), _random_site(keys, rng)
        hx, hz = ob.local_matvec(mpo, psi, i, x), ob.local_matvec(mpo, psi, i, z)
        a = np.vdot(_flat(z, keys), _flat(hx, keys))
        b = np.vdot(_flat(x, keys), _flat(hz, keys))
        assert abs(a - np.conj(b)) < 1e-11 * abs(a)
        ha = ob.local_matvec(mpo, psi, i, psi.sites[i])
        assert abs(np.vdot(_flat(psi.sites[i], keys), _flat(ha, keys)) - e) < 1e-11 * abs(e)


def test_local_two_equals_full_ci_projection():
    # the two-site local product of the fit (sites i, i+1 of psi, environments
    # of <psi|H|psi> around them) = M_{i,i+1}^+ H v: each entry is the overlap
    # of H v with the state whose two-site tensor is the unit tensor of that
    # entry, built as a product through a one-dimensional middle bond
    L = 4
    I, sys_ = _sector_system(L, 4, 0, 46)
    mpo = ob.hamiltonian_mpo(I.h, I.eri, 0.2)
    A, q = synth.random_mps(L, 4, 0, 8, seed=47)
    psi = ob.from_dense(A, q)
    v = sys_.vec(om.from_arrays(A, q))
    Hv = (sys_.H + 0.2 * np.eye(len(v))) @ v
    for i in range(L - 1):
        Le = ob.local_environments(mpo, psi, i)[0]
        Re = ob.local_environments(mpo, psi, i + 1)[1]
        Th = ob.local_two(Le, Re, psi.sites[i], psi.sites[i + 1], mpo.W[i], mpo.W[i + 1],
                          psi.bonds[i], psi.bonds[i + 2])
        scale = max(np.abs(b).max() for b in Th.values())
        n = 0
        for (qa, s1, s2), blk in Th.items():
            qb = ob.qadd(ob.qadd(qa, ob.SITE_Q[s1]), ob.SITE_Q[s2])
            rows = np.flatnonzero((q[i] == qa).all(axis=1))
            cols = np.flatnonzero((q[i + 2] == qb).all(axis=1))
            for a in range(blk.shape[0]):
                for b in range(blk.shape[1]):
                    At = [x.copy() for x in A]
                    qt = [x.copy() for x in q]
                    At[i] = np.zeros((len(q[i]), 4, 1), dtype=complex)
                    At[i + 1] = np.zeros((1, 4, len(q[i + 2])), dtype=complex)
                    At[i][rows[a], s1, 0] = 1.0
                    At[i + 1][0, s2, cols[b]] = 1.0
                    qt[i + 1] = np.array([ob.qadd(qa, ob.SITE_Q[s1])])
                    col = sys_.vec(om.from_arrays(At, qt))
                    assert abs(blk[a, b] - np.vdot(col, Hv)) < 1e-12 * scale
                    n += 1
        assert n == sum(b.size for b in Th.values()) > 0


def _stack_rows(site, left, qb):
    rows = sorted((qa, s) for s in range(4) for qa in [ob.qsub(qb, ob.SITE_Q[s])] if qa in left
                  and (qa, s) in site)
    return rows, np.concatenate([site[k] for k in rows], axis=0)


def test_qr_left_and_lq_right_factor_each_sector():
    # Q R = C and orthonormal Q per right sector (QR); L Q = C and orthonormal
    # rows per left sector (LQ); a sector with a repeated column keeps rank r
    A, q = synth.random_mps(5, 5, 1, 12, seed=48)
    psi = ob.from_dense(A, q)
    i = 2
    C = {k: v.copy() for k, v in psi.sites[i].items()}
    left, right = psi.bonds[i], psi.bonds[i + 1]
    # make one right sector rank deficient: its last column repeats the first
    qb = max(right, key=lambda x: right[x])
    for (qa, s), blk in C.items():
        if ob.qadd(qa, ob.SITE_Q[s]) == qb:
            blk[:, -1] = blk[:, 0]
    Q, newb, Rs = ob.qr_left(C, left, right)
    for qr_, r in newb.items():
        rows, M = _stack_rows(C, left, qr_)
        Qm = np.concatenate([Q[k] for k in rows], axis=0)
        assert Qm.shape[1] == r == np.linalg.matrix_rank(M)
        assert np.abs(Qm.conj().T @ Qm - np.eye(r)).max() < 1e-13
        assert np.abs(Qm @ Rs[qr_] - M).max() < 1e-13 * np.abs(M).max()
    assert newb[qb] == right[qb] - 1 if right[qb] > 1 else True
    Q2, newl, Ls = ob.lq_right(C, left, right)
    for qa, r in newl.items():
        cols = [(qa, s) for s in range(4) if (qa, s) in C]
        M = np.concatenate([C[k] for k in cols], axis=1)
        Qr = np.concatenate([Q2[k] for k in cols], axis=1)
        assert Qr.shape[0] == r == np.linalg.matrix_rank(M)
        assert np.abs(Qr @ Qr.conj().T - np.eye(r)).max() < 1e-13
        assert np.abs(Ls[qa] @ Qr - M).max() < 1e-13 * np.abs(M).max()


def test_right_canonicalize_keeps_the_state_and_makes_sites_isometric():
    L = 5
    A, q = synth.random_mps(L, 5, 1, 12, seed=49)
    psi = ob.from_dense(A, q)
    rc = ob.right_canonicalize(psi)
    sys_ = om.System.build(np.zeros((L, L)), np.zeros((L,) * 4), 3, 2)
    v0 = sys_.vec(om.from_arrays(A, q))
    v1 = sys_.vec(om.from_arrays(*ob.to_dense(rc)))
    assert np.abs(v1 - v0).max() < 1e-12 * np.abs(v0).max()
    for i in range(1, L):
        for qa, da in rc.bonds[i].items():
            acc = np.zeros((da, da), dtype=complex)
            for s in range(4):
                if (qa, s) in rc.sites[i]:
                    b = rc.sites[i][(qa, s)]
                    acc += b @ b.conj().T
            assert np.abs(acc - np.eye(da)).max() < 1e-12


def test_split_two_is_the_truncated_svd_of_each_middle_sector():
    # untruncated: A B = Th exactly; truncated to D: per middle sector the
    # best rank-k approximation (Eckart-Young) with the kept counts, and the
    # discarded weight is the sum of the dropped squared singular values
    A, q = synth.random_mps(5, 5, 1, 12, seed=50)
    psi = ob.from_dense(A, q)
    i = 1
    left, right = psi.bonds[i], psi.bonds[i + 2]
    Th = {}
    for (qa, s1), B1 in psi.sites[i].items():
        qm = ob.qadd(qa, ob.SITE_Q[s1])
        for s2 in range(4):
            B2 = psi.sites[i + 1].get((qm, s2))
            if B2 is not None and ob.qadd(qm, ob.SITE_Q[s2]) in right:
                Th[(qa, s1, s2)] = B1 @ B2
    Dfull = sum(psi.bonds[i + 1].values())

    def product(Aa, Bb):
        out = {}
        for (qa, s1, s2) in Th:
            qm = ob.qadd(qa, ob.SITE_Q[s1])
            if (qa, s1) in Aa and (qm, s2) in Bb:
                out[(qa, s1, s2)] = Aa[(qa, s1)] @ Bb[(qm, s2)]
            else:
                out[(qa, s1, s2)] = np.zeros_like(Th[(qa, s1, s2)])
        return out

    Aa, Bb, mid, disc, total = ob.split_two(Th, left, right, Dfull, 0.0, "right")
    P = product(Aa, Bb)
    assert max(np.abs(P[k] - Th[k]).max() for k in Th) < 1e-12 * max(np.abs(t).max() for t in Th.values())
    assert abs(total - sum(np.sum(np.abs(t) ** 2) for t in Th.values())) < 1e-10 * total
    D = Dfull // 2
    Aa, Bb, mid, disc, total = ob.split_two(Th, left, right, D, 0.0, "left")
    assert sum(mid.values()) <= D
    P = product(Aa, Bb)
    dropped = 0.0
    for qm in {ob.qadd(qa, ob.SITE_Q[s1]) for (qa, s1, s2) in Th}:
        rows = sorted({(qa, s1) for (qa, s1, s2) in Th if ob.qadd(qa, ob.SITE_Q[s1]) == qm})
        cols = sorted({(s2, ob.qadd(qm, ob.SITE_Q[s2])) for (qa, s1, s2) in Th
                       if ob.qadd(qa, ob.SITE_Q[s1]) == qm})
        M = np.block([[Th[(qa, s1, s2)] for (s2, qb) in cols] for (qa, s1) in rows])
        Mp = np.block([[P[(qa, s1, s2)] for (s2, qb) in cols] for (qa, s1) in rows])
        U, sv, Vh = np.linalg.svd(M, full_matrices=False)
        k = mid.get(qm, 0)
        best = (U[:, :k] * sv[:k]) @ Vh[:k]
        assert np.abs(Mp - best).max() < 1e-10 * max(1.0, sv[0])
        dropped += np.sum(sv[k:] ** 2)
    assert abs(disc - dropped) < 1e-10 * total


@pytest.mark.parametrize("L", [1, 2, 3])
def test_identity_and_site_operator_mpos_on_the_fock_space(L):
    # the identity MPO contracts to the identity; the site-operator MPOs of
    # c_{j,s} with Jordan-Wigner parities on the sites before j satisfy the
    # canonical anticommutation relations on the whole Fock space, and
    # c+_{j,s} c_{j,s} is diagonal with the occupation of spin orbital (j, s)
    # in the Fock index sum_i sigma_i 4^(L-1-i)
    assert np.array_equal(ob.mpo_to_matrix(ob.identity_mpo(L)), np.eye(4 ** L))
    C = {}
    for j in range(L):
        for s in range(2):
            ops = {k: (ob.PARITY, (0, 0)) for k in range(j)}
            ops[j] = (ob.local_op(s, False), ob.op_charge(s, False))
            C[(j, s)] = ob.mpo_to_matrix(ob.site_operator_mpo(L, ops))
            Cd = ob.mpo_to_matrix(ob.site_operator_mpo(
                L, {**{k: (ob.PARITY, (0, 0)) for k in range(j)},
                    j: (ob.local_op(s, True), ob.op_charge(s, True))}))
            assert np.array_equal(Cd, C[(j, s)].T)
    eye = np.eye(4 ** L)
    for p, Cp in C.items():
        for q_, Cq in C.items():
            assert np.abs(Cp @ Cq.T + Cq.T @ Cp - (eye if p == q_ else 0)).max() < 1e-14
            assert np.abs(Cp @ Cq + Cq @ Cp).max() < 1e-14
        j, s = p
        digit = (np.arange(4 ** L) // 4 ** (L - 1 - j)) % 4
        occ = np.isin(digit, (1, 3) if s == 0 else (2, 3)).astype(float)
        assert np.array_equal(Cp.T @ Cp, np.diag(occ))
