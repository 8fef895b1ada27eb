"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs (FP64 contractions, tolerance 1e-10 unless stated).

Small systems (L <= 8) compare whole states element by element through the
oracle's full-CI vectors; L = 16, D = 256 (the benchmark size) compares
sampled outputs the oracle computes one by one: overlaps by chain
contraction and <D|H|psi> by Slater-Condon expansion of H|D>.
"""
import numpy as np
import pytest

import synth
from oracle import fci
from oracle import mps as om

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def td():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_08489_gb300 as mod
    mod.lib()
    return mod


@pytest.fixture(scope="module")
def ctx(td):
    c = td.Context("fp64")
    yield c
    c.close()


def _to_oracle(m):
    t, q = m.export()
    return om.from_arrays(t, q)


def _system(L, n_elec, two_sz, seed):
    I = synth.make_integrals(L, seed=seed)
    na, nb = (n_elec + two_sz) // 2, (n_elec - two_sz) // 2
    return I, om.System.build(I.h, I.eri, na, nb)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- basic ops

def test_determinant_roundtrip_and_energy(td, ctx):
    L = 8
    I, sys_ = _system(L, 7, 1, 0)
    occ = synth.hole_occupation(8, 8, 3)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=7)
    psi = td.mps_from_determinant(ctx, occ)
    assert abs(td.overlap(ctx, psi, psi) - 1.0) < 1e-14
    e = td.expectation(ctx, mpo, psi, psi)
    col = np.searchsorted(sys_.dets, np.uint64(fci.occupation_mask(occ)))
    assert abs(e - sys_.H[col, col]) < 1e-11
    o = _to_oracle(psi)
    assert np.allclose(sys_.vec(o)[col], 1.0)


def test_import_export_and_overlap_random_mps(td, ctx):
    A, q = synth.random_mps(8, 7, 1, 40, seed=3)
    B, qb = synth.random_mps(8, 7, 1, 25, seed=4)
    a = td.mps_import(ctx, A, q)
    b = td.mps_import(ctx, B, qb)
    oa, ob = om.from_arrays(A, q), om.from_arrays(B, qb)
    ta, la = a.export()
    assert all(np.allclose(x, y) for x, y in zip(ta, om.from_arrays(A, q).tensors))
    ref = om.overlap(ob, oa)
    assert abs(td.overlap(ctx, b, a) - ref) < TOL * max(1.0, abs(ref))


def test_sandwich_matches_full_ci(td, ctx):
    L = 8
    I, sys_ = _system(L, 7, 1, 1)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=7)
    A, q = synth.random_mps(L, 7, 1, 48, seed=5)
    B, qb = synth.random_mps(L, 7, 1, 30, seed=6)
    a, b = td.mps_import(ctx, A, q), td.mps_import(ctx, B, qb)
    va, vb = sys_.vec(om.from_arrays(A, q)), sys_.vec(om.from_arrays(B, qb))
    ref = np.vdot(vb, sys_.H @ va)
    got = td.expectation(ctx, mpo, b, a)
    assert abs(got - ref) < TOL * max(1.0, abs(ref))
    # hermiticity through the GPU path
    assert abs(td.expectation(ctx, mpo, a, b) - np.conj(got)) < TOL * max(1.0, abs(ref))


def test_full_size_sandwich_sampled_determinants(td, ctx):
    # L = 16, D = 256: <D|H|psi> for sampled determinants D; the oracle sums
    # <D|H|D'> psi(D') over the Slater-Condon expansion of H|D>.
    L, N, S = 16, 15, 1
    I = synth.make_integrals(L, seed=0)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=N)
    A, q = synth.random_mps(L, N, S, 256, seed=0)
    psi = td.mps_import(ctx, A, q)
    opsi = om.from_arrays(A, q)
    rng = np.random.default_rng(7)
    base = synth.hole_occupation(L, 16, 7)
    dets = [base]
    for _ in range(2):
        occ = list(base)
        i, j = rng.choice(L, 2, replace=False)
        occ[i], occ[j] = occ[j], occ[i]
        dets.append(occ)
    for occ in dets:
        d = td.mps_from_determinant(ctx, occ)
        got = td.expectation(ctx, mpo, d, psi)
        masks, coefs = fci.h_on_determinant(I.h, I.eri, fci.occupation_mask(occ))
        occs = [[((int(mk) >> (2 * i)) & 1) + 2 * ((int(mk) >> (2 * i + 1)) & 1) for i in range(L)]
                for mk in masks]
        ref = np.sum(coefs * om.coefficients(opsi, occs))
        assert abs(got - ref) < 1e-9 * max(1.0, abs(ref)), (got, ref)


def test_full_size_overlap(td, ctx):
    A, q = synth.random_mps(16, 15, 1, 256, seed=1)
    B, qb = synth.random_mps(16, 15, 1, 256, seed=2)
    a, b = td.mps_import(ctx, A, q), td.mps_import(ctx, B, qb)
    ref = om.overlap(om.from_arrays(B, qb), om.from_arrays(A, q))
    assert abs(td.overlap(ctx, b, a) - ref) < TOL * max(1.0, abs(ref))


def test_full_size_apply_h_projection_property(td, ctx):
    # L = 16, D = 256, the benchmark's apply_H (one one-site sweep) in FP64.
    # The fit ends with the local solve at site 0, which is the projection of
    # the target alpha H|psi> on the orthonormal bases of the other sites
    # (Eq. add_min in the mixed-canonical gauge).  So <C|C> = <C|alpha H|psi>
    # at any size; the oracle pins the same identity on small systems.
    L, N, S = 16, 15, 1
    I = synth.make_integrals(L, seed=0)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=N)
    A, q = synth.random_mps(L, N, S, 256, seed=3)
    psi = td.mps_import(ctx, A, q)
    ctx.set_schedule(0, 1)
    alpha = 0.4 - 0.9j
    c = td.apply_H(ctx, mpo, psi, alpha, 256, 0.0)
    cc = td.overlap(ctx, c, c)
    ct = alpha * td.expectation(ctx, mpo, c, psi)
    assert abs(cc.imag) < 1e-12 * abs(cc)
    assert abs(cc - ct) < 1e-9 * abs(cc), (cc, ct)


# ---------------------------------------------------------------- fits

@pytest.mark.parametrize("n2,n1,D", [(3, 1, 500), (1, 2, 12), (0, 3, 64)])
def test_apply_h_matches_oracle_schedule(td, ctx, n2, n1, D):
    L = 6
    I, sys_ = _system(L, 5, 1, 2)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=5)
    A, q = synth.random_mps(L, 5, 1, 10, seed=8)
    psi = td.mps_import(ctx, A, q)
    ctx.set_schedule(n2, n1)
    alpha = 0.3 - 0.7j
    out = td.apply_H(ctx, mpo, psi, alpha, D, 0.0)
    ref = om.apply_H(sys_, om.from_arrays(A, q), alpha, om.Schedule(D=D, eps=0.0, n_two_site=n2,
                                                                    n_one_site=n1))
    v_gpu = sys_.vec(_to_oracle(out))
    v_ref = sys_.vec(ref)
    assert _rel(v_gpu, v_ref) < TOL
    if D >= 500:
        exact = alpha * (sys_.H @ sys_.vec(om.from_arrays(A, q)))
        assert _rel(v_gpu, exact) < TOL


def test_apply_h_from_determinant_exact(td, ctx):
    L = 6
    I, sys_ = _system(L, 6, 0, 3)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=6)
    occ = [3, 3, 0, 0, 1, 2]
    psi = td.mps_from_determinant(ctx, occ)
    ctx.set_schedule(3, 1)
    out = td.apply_H(ctx, mpo, psi, 1.0, 500, 0.0)
    exact = sys_.H @ sys_.vec(om.from_determinant(occ))
    assert _rel(sys_.vec(_to_oracle(out)), exact) < TOL


def test_sum_fit_and_compress(td, ctx):
    L = 6
    I, sys_ = _system(L, 5, 1, 4)
    A, q = synth.random_mps(L, 5, 1, 10, seed=9)
    B, qb = synth.random_mps(L, 5, 1, 8, seed=10)
    a, b = td.mps_import(ctx, A, q), td.mps_import(ctx, B, qb)
    oa, ob = om.from_arrays(A, q), om.from_arrays(B, qb)
    ctx.set_schedule(1, 2)
    s = td.mps_sum(ctx, [1.0, -0.4 + 0.2j], [a, b], 9, 0.0)
    ref = om.sum_fit(sys_, [(1.0, oa), (-0.4 + 0.2j, ob)], om.Schedule(D=9, n_two_site=1, n_one_site=2))
    assert _rel(sys_.vec(_to_oracle(s)), sys_.vec(ref)) < TOL
    c = a.copy()
    disc = td.compress(ctx, c, 5, 0.0)
    rc, rdisc = om.compress(oa, 5, 0.0)
    assert _rel(sys_.vec(_to_oracle(c)), sys_.vec(rc)) < TOL
    assert abs(disc - rdisc) < 1e-10


def test_truncation_with_eps(td, ctx):
    L = 6
    I, sys_ = _system(L, 6, 0, 5)
    A, q = synth.random_mps(L, 6, 0, 20, seed=11)
    a = td.mps_import(ctx, A, q)
    c = a.copy()
    disc = td.compress(ctx, c, 100, 1e-3)
    rc, rdisc = om.compress(om.from_arrays(A, q), 100, 1e-3)
    assert _rel(sys_.vec(_to_oracle(c)), sys_.vec(rc)) < TOL
    assert _to_oracle(c).bond_dims == rc.bond_dims
    assert abs(disc - rdisc) < 1e-10


# ---------------------------------------------------------------- integrators

def test_rk4_step_matches_oracle_truncated_and_exact(td, ctx):
    L = 6
    I, sys_ = _system(L, 5, 1, 6)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=5)
    occ = synth.hole_occupation(6, 6, 2)
    for D, n2, n1 in [(500, 3, 1), (10, 2, 1)]:
        psi = td.mps_from_determinant(ctx, occ)
        ctx.set_schedule(n2, n1)
        td.rk4_step(ctx, mpo, psi, 0.05, D, 0.0)
        ref = om.rk4_step(sys_, om.from_determinant(occ), 0.05, om.Schedule(D=D, n_two_site=n2, n_one_site=n1))
        assert _rel(sys_.vec(_to_oracle(psi)), sys_.vec(ref)) < TOL
        if D == 500:
            exact = fci.rk4_step(sys_.H, sys_.vec(om.from_determinant(occ)).astype(complex), 0.05)
            assert _rel(sys_.vec(_to_oracle(psi)), exact) < TOL


def test_krylov_step_matches_oracle(td, ctx):
    L = 6
    I, sys_ = _system(L, 5, 1, 7)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=5)
    A, q = synth.random_mps(L, 5, 1, 12, seed=12)
    oa = om.from_arrays(A, q)
    oa = om.scale(oa, 1.0 / om.norm(oa))
    t0, q0 = oa.tensors, oa.labels
    for D, n2, n1, m in [(500, 3, 1, 4), (10, 1, 2, 5)]:
        psi = td.mps_import(ctx, t0, q0)
        ctx.set_schedule(n2, n1)
        td.krylov_step(ctx, mpo, psi, 0.05, m, True, D, 0.0)
        ref, *_ = om.krylov_step(sys_, om.from_arrays(t0, q0), 0.05, m,
                                 om.Schedule(D=D, n_two_site=n2, n_one_site=n1))
        assert _rel(sys_.vec(_to_oracle(psi)), sys_.vec(ref)) < 1e-9
        if D == 500:
            exact = fci.krylov_step(sys_.H, sys_.vec(om.from_arrays(t0, q0)), 0.05, m)
            assert _rel(sys_.vec(_to_oracle(psi)), exact) < 1e-9
            assert abs(td.overlap(ctx, psi, psi) - 1.0) < 1e-10


def test_krylov_step_serial_inner_products_match_oracle(td, ctx):
    """The truncated step above with the inner products run after each fit on
    the context stream (tdmps_set_concurrent_inner(ctx, 0)) instead of beside
    it on the helper thread."""
    L = 6
    I, sys_ = _system(L, 5, 1, 7)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=5)
    A, q = synth.random_mps(L, 5, 1, 12, seed=12)
    oa = om.from_arrays(A, q)
    oa = om.scale(oa, 1.0 / om.norm(oa))
    ctx.set_schedule(1, 2)
    ctx.set_concurrent_inner(False)
    try:
        psi = td.mps_import(ctx, oa.tensors, oa.labels)
        td.krylov_step(ctx, mpo, psi, 0.05, 5, True, 10, 0.0)
    finally:
        ctx.set_concurrent_inner(True)
    ref, *_ = om.krylov_step(sys_, oa.copy(), 0.05, 5,
                             om.Schedule(D=10, n_two_site=1, n_one_site=2))
    assert _rel(sys_.vec(_to_oracle(psi)), sys_.vec(ref)) < 1e-9


def test_one_rdm_matches_oracle(td, ctx):
    L = 6
    I, sys_ = _system(L, 5, 1, 8)
    A, q = synth.random_mps(L, 5, 1, 14, seed=13)
    a = td.mps_import(ctx, A, q)
    g = td.one_rdm(ctx, a)
    ref = fci.one_rdm(sys_.vec(om.from_arrays(A, q)), sys_.dets, L)
    assert np.abs(g - ref).max() < TOL * max(1.0, np.abs(ref).max())


def test_rk4_trajectory_equals_full_ci_untruncated(td, ctx):
    # configuration of the first workload: L = 8, 8 electrons minus one
    # down electron in orbital 3, dt = 0.01; exact bond dimension (<= 256).
    L = 8
    I, sys_ = _system(L, 7, 1, 0)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=7)
    occ = synth.hole_occupation(8, 8, 3)
    psi = td.mps_from_determinant(ctx, occ)
    ctx.set_schedule(4, 1)
    v = sys_.vec(om.from_determinant(occ)).astype(complex)
    for step in range(3):
        td.rk4_step(ctx, mpo, psi, 0.01, 256, 0.0)
        v = fci.rk4_step(sys_.H, v, 0.01)
        g = td.one_rdm(ctx, psi)
        gref = fci.one_rdm(v, sys_.dets, L)
        assert np.abs(g - gref).max() < 1e-10
    assert _rel(sys_.vec(_to_oracle(psi)), v) < 1e-10
