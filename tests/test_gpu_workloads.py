"""GPU runs of the paper's integrators on the small configurations, against
the oracle: the first workload's RK4 trajectory (L = 8, 8 electrons minus the
down electron of orbital 3, dt = 0.01) untruncated against full CI over its
full length of 200 steps and truncated at D = 64 against the MPS oracle, and the plain
(non-orthogonal) Krylov basis of Eq. (kry_non)."""
import numpy as np
import pytest

import synth
from oracle import fci
from oracle import mps as om

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def td():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_08489_gb300 as mod
    mod.lib()
    return mod


def _system(L, n_elec, two_sz, seed):
    I = synth.make_integrals(L, seed=seed)
    na, nb = (n_elec + two_sz) // 2, (n_elec - two_sz) // 2
    return I, om.System.build(I.h, I.eri, na, nb)


def _vec(sys_, m):
    return sys_.vec(om.from_arrays(*m.export()))


def test_first_workload_rk4_trajectory_untruncated(td):
    # D = 160 is the exact bond dimension of the propagated sector, so the
    # MPS trajectory is the full-CI RK4 trajectory; after 200 steps (t = 2
    # a.u.) it also stays within the RK4 error of the exact propagation
    L, dt, steps = 8, 0.01, 200
    I, sys_ = _system(L, 7, 1, 0)
    ctx = td.Context("fp64")
    ctx.set_schedule(4, 1)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=7)
    occ = synth.hole_occupation(8, 8, 3)
    psi = td.mps_from_determinant(ctx, occ)
    v = sys_.vec(om.from_determinant(occ)).astype(complex)
    v0 = v.copy()
    Hc = sys_.H.astype(complex)   # exact copy; saves a conversion per product
    worst = 0.0
    for step in range(steps):
        td.rk4_step(ctx, mpo, psi, dt, 160, 0.0)
        v = fci.rk4_step(Hc, v, dt)
        if step % 10 == 9:
            g = td.one_rdm(ctx, psi)
            worst = max(worst, np.abs(g - fci.one_rdm(v, sys_.dets, L)).max())
    print("first workload, %d RK4 steps: max 1-RDM error vs full CI %.2e" % (steps, worst))
    assert worst < 1e-10
    assert np.linalg.norm(_vec(sys_, psi) - v) < 1e-9
    exact = fci.exact_evolve(sys_.H, v0, dt * steps)
    lam = np.linalg.eigvalsh(sys_.H)
    bound = steps * (np.abs(lam).max() * dt) ** 5 / 120
    assert np.linalg.norm(v - exact) < bound
    ctx.close()


def test_first_workload_truncated_matches_oracle(td):
    L, dt = 8, 0.01
    I, sys_ = _system(L, 7, 1, 0)
    ctx = td.Context("fp64")
    ctx.set_schedule(3, 1)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=7)
    occ = synth.hole_occupation(8, 8, 3)
    psi = td.mps_from_determinant(ctx, occ)
    ref = om.from_determinant(occ)
    sch = om.Schedule(D=64, eps=0.0, n_two_site=3, n_one_site=1)
    for _ in range(3):
        td.rk4_step(ctx, mpo, psi, dt, 64, 0.0)
        ref = om.rk4_step(sys_, ref, dt, sch)
    a, b = _vec(sys_, psi), sys_.vec(ref)
    assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)
    assert max(om.from_arrays(*psi.export()).bond_dims) <= 64
    ctx.close()


def test_plain_krylov_basis_matches_oracle_and_full_ci(td):
    L = 6
    I, sys_ = _system(L, 5, 1, 7)
    ctx = td.Context("fp64")
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=5)
    A, q = synth.random_mps(L, 5, 1, 12, seed=12)
    oa = om.from_arrays(A, q)
    oa = om.scale(oa, 1.0 / om.norm(oa))
    for D, n2, n1, m in [(500, 3, 1, 4), (10, 1, 2, 5)]:
        psi = td.mps_import(ctx, oa.tensors, oa.labels)
        ctx.set_schedule(n2, n1)
        td.krylov_step(ctx, mpo, psi, 0.05, m, False, D, 0.0)
        ref, *_ = om.krylov_step(sys_, oa, 0.05, m,
                                 om.Schedule(D=D, n_two_site=n2, n_one_site=n1), orthogonal=False)
        got = _vec(sys_, psi)
        assert np.linalg.norm(got - sys_.vec(ref)) <= 1e-9 * np.linalg.norm(sys_.vec(ref))
        if D == 500:
            exact = fci.krylov_step(sys_.H, sys_.vec(oa), 0.05, m, orthogonal=False)
            assert np.linalg.norm(got - exact) < 1e-9
    ctx.close()
