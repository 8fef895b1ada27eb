"""Pins for oracle B (MPS operations) against oracle A, library SVDs and
exact properties of the fit (Eq. add_min) and of SVD truncation."""
import numpy as np
import pytest

import synth
from oracle import fci
from oracle import mps as om


def _system(L, n_elec, two_sz, seed):
    I = synth.make_integrals(L, seed=seed)
    na, nb = (n_elec + two_sz) // 2, (n_elec - two_sz) // 2
    return om.System.build(I.h, I.eri, na, nb)


def test_determinant_mps_is_unit_vector():
    occ = [3, 1, 0, 2, 3, 0]
    m = om.from_determinant(occ)
    na, nb = 3, 3
    dets = fci.basis(6, na, nb)
    v = om.to_sector(m, dets)
    ref = np.zeros(len(dets))
    ref[np.searchsorted(dets, np.uint64(fci.occupation_mask(occ)))] = 1.0
    assert np.allclose(v, ref)
    assert om.coefficient(m, occ) == 1.0


def test_transfer_overlap_equals_vector_overlap_and_coefficients():
    A, q = synth.random_mps(6, 6, 0, 12, seed=1)
    B, qb = synth.random_mps(6, 6, 0, 9, seed=2)
    a, b = om.from_arrays(A, q), om.from_arrays(B, qb)
    va, vb = om.to_fock(a), om.to_fock(b)
    assert abs(om.overlap(b, a) - np.vdot(vb, va)) < 1e-12 * np.linalg.norm(va) * np.linalg.norm(vb)
    rng = np.random.default_rng(0)
    dets = fci.basis(6, 3, 3)
    for m in rng.choice(dets, 5):
        occ = [((int(m) >> (2 * i)) & 1) + 2 * ((int(m) >> (2 * i + 1)) & 1) for i in range(6)]
        idx = om.fock_index(np.array([m], dtype=np.uint64), 6)[0]
        assert abs(om.coefficient(a, occ) - va[idx]) < 1e-13
        assert abs(om.coefficients(a, [occ])[0] - va[idx]) < 1e-13


def test_compress_two_sites_is_library_svd():
    # L = 2: one bond; truncation to D is the Eckart-Young truncation of the
    # 4 x 4 coefficient matrix, computed here by numpy's SVD.
    A, q = synth.random_mps(2, 2, 0, 4, seed=3)
    m = om.from_arrays(A, q)
    M = om.to_fock(m).reshape(4, 4)
    s = np.linalg.svd(M, compute_uv=False)
    for D in (1, 2):
        c, disc = om.compress(m, D, 0.0)
        err2 = np.linalg.norm(om.to_fock(c).reshape(4, 4) - M) ** 2
        assert abs(err2 - np.sum(s[D:] ** 2)) < 1e-12
        assert abs(disc - np.sum(s[D:] ** 2) / np.sum(s ** 2)) < 1e-12


def test_compress_exact_and_single_bond_truncation_weight():
    A, q = synth.random_mps(6, 5, 1, 30, seed=4)
    m = om.from_arrays(A, q)
    v = om.to_fock(m)
    c, disc = om.compress(m, 10 ** 6, 0.0)
    assert np.linalg.norm(om.to_fock(c) - v) < 1e-12 * np.linalg.norm(v)
    assert disc < 1e-24
    # normalised state, truncation only at the middle bond (others are small
    # enough to stay exact): <psi'|psi'> = 1 - discarded, |psi - psi'|^2 = discarded
    mn = om.scale(c, 1.0 / om.norm(c))
    D = 6
    t, disc = om.compress(mn, D, 0.0)
    dims = t.bond_dims
    assert max(dims) <= D
    vn, vt = om.to_fock(mn), om.to_fock(t)
    assert abs(np.vdot(vn - vt, vn - vt).real - (1 - np.vdot(vt, vt).real)) < 1e-12


def test_truncation_rule_eps_D_and_clusters():
    s = {(0, 0): np.array([1.0, 0.5, 0.1]), (1, 1): np.array([0.5 + 1e-13, 1e-3]),
         (1, -1): np.array([1e-14])}
    kept, disc, tot = om.truncation_rule(s, D=10, eps=0.0)
    assert kept == {(0, 0): 3, (1, 1): 2, (1, -1): 0}          # zero floor
    kept, disc, tot = om.truncation_rule(s, D=10, eps=2e-6 / tot)
    assert kept == {(0, 0): 3, (1, 1): 1, (1, -1): 0}          # drops 1e-3 (weight 1e-6)
    kept, _, _ = om.truncation_rule(s, D=2, eps=0.0)            # cut inside 0.5 cluster
    assert kept == {(0, 0): 1, (1, 1): 0, (1, -1): 0}
    kept, _, _ = om.truncation_rule(s, D=3, eps=0.0)
    assert kept == {(0, 0): 2, (1, 1): 1, (1, -1): 0}
    # a degenerate cluster at the very top is kept whole even beyond D (there
    # is no cluster edge below the cut); spin symmetry makes such clusters
    # span sectors
    top = {(1, 1): np.array([1.0]), (1, -1): np.array([1.0 - 1e-13]), (2, 0): np.array([0.3])}
    kept, disc, tot = om.truncation_rule(top, D=1, eps=0.0)
    assert kept == {(1, 1): 1, (1, -1): 1, (2, 0): 0}
    assert abs(disc - 0.09) < 1e-12


@pytest.mark.parametrize("n_two,n_one", [(3, 1), (4, 0)])
def test_untruncated_apply_h_is_exact(n_two, n_one):
    # (4, 0): two-site sweeps alone (their projections decide the result)
    sys_ = _system(6, 6, 0, seed=5)
    psi = om.from_determinant([3, 3, 0, 0, 1, 2])
    sch = om.Schedule(D=500, eps=0.0, n_two_site=n_two, n_one_site=n_one)
    c = om.apply_H(sys_, psi, 0.7 - 0.2j, sch)
    ref = (0.7 - 0.2j) * (sys_.H @ sys_.vec(psi))
    assert np.linalg.norm(sys_.vec(c) - ref) < 1e-12 * np.linalg.norm(ref)


def test_untruncated_integrators_equal_full_ci_integrators():
    sys_ = _system(6, 5, 1, seed=6)
    psi = om.from_determinant(synth.hole_occupation(6, 6, 2))
    sch = om.Schedule(D=500, eps=0.0, n_two_site=3, n_one_site=1)
    v = sys_.vec(psi).astype(complex)
    p = om.rk4_step(sys_, psi, 0.03, sch)
    assert np.linalg.norm(sys_.vec(p) - fci.rk4_step(sys_.H, v, 0.03)) < 1e-11
    k, c, N, Hk = om.krylov_step(sys_, p, 0.05, 5, sch)
    # Eq. (kry_orth): the fitted, normalised basis is orthonormal when nothing
    # is truncated (p is complex, so a conjugated coefficient would show)
    assert np.allclose(N, np.eye(5), atol=1e-10)
    ref = fci.krylov_step(sys_.H, sys_.vec(p), 0.05, 5)
    assert np.linalg.norm(sys_.vec(k) - ref) < 1e-10
    assert abs(om.norm(k) - om.norm(p)) < 1e-12
    g = om.one_rdm(sys_, k)
    assert np.allclose(g, fci.one_rdm(ref, sys_.dets, 6), atol=1e-10)


def test_truncated_fit_residual_monotone_and_projection_property():
    sys_ = _system(6, 6, 0, seed=7)
    A, q = synth.random_mps(6, 6, 0, 24, seed=8)
    psi = om.from_arrays(A, q)
    psi = om.scale(psi, 1.0 / om.norm(psi))
    info = om.FitInfo()
    sch = om.Schedule(D=8, eps=0.0, n_two_site=1, n_one_site=4)
    T = sys_.fock(sys_.H @ sys_.vec(psi))
    c = om.fit(T, psi, sch.D, sch.eps, sch.n_two_site, sch.n_one_site, info)
    r = info.residuals
    assert all(r[i + 1] <= r[i] + 1e-12 for i in range(len(r) - 1))
    # after the last local solve, C is the projection of T on its own tangent
    # space: <C|C> = <C|T>, and the residual equals |T|^2 - |C|^2
    vc = om.to_fock(c)
    assert abs(np.vdot(vc, vc) - np.vdot(vc, T)) < 1e-12 * np.vdot(T, T).real
    assert abs(np.vdot(T - vc, T - vc).real - r[-1]) < 1e-10 * np.vdot(T, T).real
    assert max(c.bond_dims) <= 8


def test_scale_uses_lth_root():
    A, q = synth.random_mps(4, 4, 0, 6, seed=9)
    m = om.from_arrays(A, q)
    s = om.scale(m, -2.0 + 1.0j)
    assert np.allclose(om.to_fock(s), (-2.0 + 1.0j) * om.to_fock(m))


def test_gram_schmidt_qr_against_library_qr():
    rng = np.random.default_rng(5)
    for m, n in [(9, 4), (4, 9), (6, 6)]:
        M = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
        Q, R = om.gram_schmidt_qr(M)
        Ql, _ = np.linalg.qr(M, mode="reduced")
        assert np.allclose(Q @ R, M, atol=1e-12)
        assert np.allclose(Q.conj().T @ Q, np.eye(min(m, n)), atol=1e-12)
        assert np.allclose(Q @ Q.conj().T, Ql @ Ql.conj().T, atol=1e-12)   # same span
    # a dependent column adds no direction; the last column of Q is zero
    M = rng.standard_normal((6, 3))
    M[:, 1] = 2.0 * M[:, 0]
    Q, R = om.gram_schmidt_qr(M)
    assert np.allclose(Q @ R, M, atol=1e-12)
    assert np.abs(Q[:, 2]).max() == 0.0


def _row_labels(ql):
    return (ql[:, None, :] + om.SITE_Q[None, :, :]).reshape(-1, 2)


def test_sector_qr_and_lq_factor_each_sector_with_orthonormal_factors():
    A, q = synth.random_mps(5, 5, 1, 12, seed=60)
    i = 2
    C = np.asarray(A[i], dtype=complex).copy()
    ql, qr = np.asarray(q[i]), np.asarray(q[i + 1])
    Dl, d, Dr = C.shape
    M = C.reshape(Dl * d, Dr)
    Q, lab, Rs = om.qr_left(C, ql, qr)
    Qm = Q.reshape(Dl * d, -1)
    assert np.abs(Qm.conj().T @ Qm - np.eye(Qm.shape[1])).max() < 1e-13
    rowlab = _row_labels(ql)
    for sec, (R, cols) in Rs.items():
        k = np.flatnonzero((lab == sec).all(axis=1))
        rows = np.flatnonzero((rowlab == sec).all(axis=1))
        outside = np.setdiff1d(np.arange(Dl * d), rows)
        assert np.abs(Qm[np.ix_(outside, k)]).max(initial=0.0) == 0.0
        assert np.abs(Qm[:, k] @ R - M[:, cols]).max() < 1e-13 * np.abs(M).max()
    Q2, lab2, Ls = om.lq_right(C, ql, qr)
    Q2m = Q2.reshape(-1, d * Dr)
    assert np.abs(Q2m @ Q2m.conj().T - np.eye(Q2m.shape[0])).max() < 1e-13
    Mr = C.reshape(Dl, d * Dr)
    for sec, (Lf, rows) in Ls.items():
        k = np.flatnonzero((lab2 == sec).all(axis=1))
        assert np.abs(Lf @ Q2m[k] - Mr[rows]).max() < 1e-13 * np.abs(Mr).max()


def test_split_two_site_is_the_truncated_svd_of_each_sector():
    A, q = synth.random_mps(5, 5, 1, 12, seed=61)
    i = 1
    Th = np.einsum("asx,xtb->astb", A[i], A[i + 1])
    ql, qr = np.asarray(q[i]), np.asarray(q[i + 2])
    Dl, _, _, Dr = Th.shape
    M = Th.reshape(Dl * 4, 4 * Dr)
    rowlab = _row_labels(ql)
    collab = (qr[None, :, :] - om.SITE_Q[:, None, :]).reshape(4 * Dr, 2)
    total = np.sum(np.abs(M) ** 2)
    U, V, lab, disc, tot = om.split_two_site(Th, ql, qr, 10 ** 6, 0.0, "right")
    assert np.abs(np.einsum("asx,xtb->astb", U, V) - Th).max() < 1e-12 * np.abs(Th).max()
    assert abs(tot - total) < 1e-10 * total
    D = len(q[i + 1]) // 2
    U, V, lab, disc, tot = om.split_two_site(Th, ql, qr, D, 0.0, "left")
    assert len(lab) <= D
    P = np.einsum("asx,xtb->astb", U, V).reshape(Dl * 4, 4 * Dr)
    dropped = 0.0
    for sec in {tuple(x) for x in rowlab} & {tuple(x) for x in collab}:
        rows = np.flatnonzero((rowlab == sec).all(axis=1))
        cols = np.flatnonzero((collab == sec).all(axis=1))
        u, s, vh = np.linalg.svd(M[np.ix_(rows, cols)], full_matrices=False)
        k = int(np.sum((lab == sec).all(axis=1)))
        best = (u[:, :k] * s[:k]) @ vh[:k]
        assert np.abs(P[np.ix_(rows, cols)] - best).max() < 1e-10 * max(1.0, s[0])
        dropped += np.sum(s[k:] ** 2)
    assert abs(disc - dropped) < 1e-10 * total


def test_right_canonicalize_keeps_the_vector_and_makes_sites_isometric():
    A, q = synth.random_mps(5, 5, 1, 12, seed=62)
    m = om.from_arrays(A, q)
    rc = om.right_canonicalize(m)
    v0, v1 = om.to_fock(m), om.to_fock(rc)
    assert np.abs(v1 - v0).max() < 1e-12 * np.abs(v0).max()
    for t in rc.tensors[1:]:
        Dl = t.shape[0]
        Mt = t.reshape(Dl, -1)
        assert np.abs(Mt @ Mt.conj().T - np.eye(Dl)).max() < 1e-12


def test_projections_are_the_adjoint_of_the_site_maps():
    # project_one(T) = M_i^+ T and project_two(T) = M_{i,i+1}^+ T, M the
    # linear maps from the site (pair) tensor to the Fock vector of C with
    # that site (pair) replaced
    L = 4
    A, q = synth.random_mps(L, 4, 0, 6, seed=63)
    C = om.from_arrays(A, q)
    rng = np.random.default_rng(64)
    T = rng.standard_normal(4 ** L) + 1j * rng.standard_normal(4 ** L)
    for i in range(L):
        P = om.project_one(T, C, i)
        Dl, _, Dr = C.tensors[i].shape
        for a, s, b in [(0, 0, 0), (Dl - 1, 3, Dr - 1), (Dl // 2, 1, Dr // 2)]:
            U = C.copy()
            U.tensors[i] = np.zeros_like(C.tensors[i])
            U.tensors[i][a, s, b] = 1.0
            assert abs(P[a, s, b] - np.vdot(om.to_fock(U), T)) < 1e-12 * np.abs(T).max()
    for i in range(L - 1):
        P2 = om.project_two(T, C, i)
        Dl, Dr = C.tensors[i].shape[0], C.tensors[i + 1].shape[2]
        for a, s, t, b in [(0, 0, 3, 0), (Dl - 1, 2, 1, Dr - 1)]:
            U = C.copy()
            U.tensors[i] = np.zeros((Dl, 4, 1), dtype=complex)
            U.tensors[i + 1] = np.zeros((1, 4, Dr), dtype=complex)
            U.tensors[i][a, s, 0] = 1.0
            U.tensors[i + 1][0, t, b] = 1.0
            assert abs(P2[a, s, t, b] - np.vdot(om.to_fock(U), T)) < 1e-12 * np.abs(T).max()


def test_untruncated_sum_fit_is_the_exact_sum():
    L = 4
    sys_ = _system(L, 4, 0, 65)
    A1, q1 = synth.random_mps(L, 4, 0, 6, seed=66)
    A2, q2 = synth.random_mps(L, 4, 0, 6, seed=67)
    m1, m2 = om.from_arrays(A1, q1), om.from_arrays(A2, q2)
    c1, c2 = 0.7 - 0.2j, -1.1 + 0.4j
    out = om.sum_fit(sys_, [(c1, m1), (c2, m2)], om.Schedule(D=36, n_two_site=3, n_one_site=1))
    ref = c1 * sys_.vec(m1) + c2 * sys_.vec(m2)
    assert np.abs(sys_.vec(out) - ref).max() < 1e-11 * np.abs(ref).max()
