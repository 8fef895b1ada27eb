"""GPU parity of the observables beyond the 1BRDM: exact site operators,
transition and two-body density matrices, the one-particle Green's function
of Eq. (green_time) and the energy gradient (torch.autograd), against the
CPU oracle on the same seeded inputs (FP64, tolerance 1e-10 unless stated)."""
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


def _sector(n_elec, two_sz):
    return (n_elec + two_sz) // 2, (n_elec - two_sz) // 2


def test_site_ops_equal_oracle_and_zero_state(td, ctx):
    L = 5
    A, q = synth.random_mps(L, 5, 1, 12, seed=21)
    psi = td.mps_import(ctx, A, q)
    ref = om.from_arrays(A, q)
    for site in range(L):
        for spin in range(2):
            for dagger in (False, True):
                out = td.apply_site_op(ctx, psi, site, spin, dagger)
                want = om.apply_site_op(ref, site, spin, dagger)
                got = _to_oracle(out)
                assert np.abs(om.to_fock(got) - om.to_fock(want)).max() < 1e-15
                info = out.info()
                assert info["n_elec"] == 5 + (1 if dagger else -1)
                assert info["two_sz"] == 1 + (1 if dagger else -1) * (1 if spin == 0 else -1)
    det = td.mps_from_determinant(ctx, [3, 0, 1, 2])
    with pytest.raises(td.TdmpsError) as e:
        td.apply_site_op(ctx, det, 1, 0, False)
    assert e.value.name == "ZERO_STATE"
    with pytest.raises(td.TdmpsError) as e:
        td.apply_site_op(ctx, det, 0, 1, True)
    assert e.value.name == "ZERO_STATE"
    with pytest.raises(td.TdmpsError):
        td.apply_site_op(ctx, det, 4, 0, False)


def test_transition_rdm_equals_oracle(td, ctx):
    L = 6
    na, nb = _sector(5, -1)
    dets = fci.basis(L, na, nb)
    A, q = synth.random_mps(L, 5, -1, 20, seed=22)
    B, qb = synth.random_mps(L, 5, -1, 14, seed=23)
    a, b = td.mps_import(ctx, A, q), td.mps_import(ctx, B, qb)
    va = om.to_sector(om.from_arrays(A, q), dets)
    vb = om.to_sector(om.from_arrays(B, qb), dets)
    ref = fci.transition_rdm(vb, va, dets, L)
    got = td.transition_rdm(ctx, b, a)
    assert np.abs(got - ref).max() < TOL * max(1.0, np.abs(ref).max())
    # the diagonal case is the 1BRDM
    assert np.abs(td.transition_rdm(ctx, a, a) - td.one_rdm(ctx, a)).max() < 1e-12
    C, qc = synth.random_mps(L, 5, 1, 8, seed=24)
    with pytest.raises(td.TdmpsError) as e:
        td.transition_rdm(ctx, a, td.mps_import(ctx, C, qc))
    assert e.value.name == "SECTOR"


@pytest.mark.parametrize("L,n_elec,two_sz,D,seed", [(4, 4, 0, 16, 25), (6, 5, 1, 24, 26)])
def test_two_rdm_equals_oracle_and_energy(td, ctx, L, n_elec, two_sz, D, seed):
    na, nb = _sector(n_elec, two_sz)
    dets = fci.basis(L, na, nb)
    A, q = synth.random_mps(L, n_elec, two_sz, D, seed=seed)
    psi = td.mps_import(ctx, A, q)
    v = om.to_sector(om.from_arrays(A, q), dets)
    ref = fci.two_rdm(v, dets, L)
    got = td.two_rdm(ctx, psi)
    assert np.abs(got - ref).max() < TOL * max(1.0, np.abs(ref).max())
    I = synth.make_integrals(L, seed=seed)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=n_elec, e0=0.3)
    g = td.one_rdm(ctx, psi)
    e = np.einsum("ij,ij->", I.h, g) + 0.5 * np.einsum("ijkl,ijkl->", I.eri, got) \
        + 0.3 * td.overlap(ctx, psi, psi)
    assert abs(e - td.expectation(ctx, mpo, psi, psi)) < 1e-10 * max(1.0, abs(e))


def _ground_state(I, L, na, nb):
    dets = fci.basis(L, na, nb)
    w, U = np.linalg.eigh(fci.hamiltonian(I.h, I.eri, dets))
    v = U[:, 0].astype(complex)
    return dets, v, om.from_fock(om.sector_to_fock(v, dets, L), L)


@pytest.mark.parametrize("method", ["krylov", "rk4"])
def test_green_function_equals_oracle_and_full_ci(td, ctx, method):
    L = 4
    I = synth.make_integrals(L, seed=27)
    dets, v, psi0 = _ground_state(I, L, 2, 2)
    psi = td.mps_import(ctx, psi0.tensors, psi0.labels)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=4)
    td_ctx = ctx
    td_ctx.set_schedule(1, 1)
    dt, n, m = 0.1, 3, 6
    systems = {0: om.System.build(I.h, I.eri, 1, 2), 1: om.System.build(I.h, I.eri, 2, 1)}
    sch = om.Schedule(D=64, eps=0.0, n_two_site=1, n_one_site=1)
    for i, j in [(1, 1), (0, 2)]:
        got = td.green_function(ctx, mpo, psi, i, j, dt, n, method=method, m=m, D=64)
        ref = om.green_function(systems, psi0, i, j, dt, n, m, sch, method=method)
        assert np.abs(got - ref).max() < 1e-9
        exact = fci.green_function(I.h, I.eri, v, dets, L, i, j, dt * np.arange(n + 1))
        # integrator error only: Krylov with m = 6 in a 24-dimensional sector,
        # RK4 local error (|H| dt)^5 / 120
        tol = 1e-7 if method == "krylov" else 5e-3
        assert np.abs(got - exact).max() < tol
        assert abs(got[0] + 1j) < 1e-12


def test_energy_gradient_is_density_matrices_and_finite_differences(td, ctx):
    torch = pytest.importorskip("torch")
    from paper_1902_08489_gb300 import grad
    L = 4
    I = synth.make_integrals(L, seed=28)
    A, q = synth.random_mps(L, 3, 1, 12, seed=29)
    psi = td.mps_import(ctx, A, q)
    h = torch.tensor(I.h, dtype=torch.float64, requires_grad=True)
    eri = torch.tensor(I.eri, dtype=torch.float64, requires_grad=True)
    e0 = torch.tensor(0.2, dtype=torch.float64, requires_grad=True)
    E = grad.energy(h, eri, e0, ctx, psi)
    E.backward()
    na, nb = _sector(3, 1)
    dets = fci.basis(L, na, nb)
    v = om.to_sector(om.from_arrays(A, q), dets)
    nrm = np.vdot(v, v).real
    H = fci.hamiltonian(I.h, I.eri, dets, 0.2)
    assert abs(E.item() - np.vdot(v, H @ v).real / nrm) < 1e-11
    assert np.abs(h.grad.numpy() - fci.one_rdm(v, dets, L).real / nrm).max() < 1e-11
    assert np.abs(eri.grad.numpy() - 0.5 * fci.two_rdm(v, dets, L).real / nrm).max() < 1e-11
    assert abs(e0.grad.item() - 1.0) < 1e-15

    # central differences along symmetry orbits of the integrals (E is linear
    # in them, so the difference quotient is exact up to rounding)
    def e_at(hh, ee):
        return grad.energy(torch.tensor(hh), torch.tensor(ee), 0.2, ctx, psi).item()
    d = 1e-3
    for (i, j) in [(0, 0), (1, 3)]:
        P = np.zeros((L, L)); P[i, j] = P[j, i] = 1.0
        fd = (e_at(I.h + d * P, I.eri) - e_at(I.h - d * P, I.eri)) / (2 * d)
        assert abs(fd - (h.grad.numpy() * P).sum()) < 1e-9
    for (i, j, k, l) in [(0, 1, 2, 3), (1, 1, 2, 2), (0, 2, 0, 2)]:
        P = np.zeros((L,) * 4)
        for a, b, c, e in [(i, j, k, l), (j, i, k, l), (i, j, l, k), (j, i, l, k),
                           (k, l, i, j), (l, k, i, j), (k, l, j, i), (l, k, j, i)]:
            P[a, b, c, e] = 1.0
        fd = (e_at(I.h, I.eri + d * P) - e_at(I.h, I.eri - d * P)) / (2 * d)
        assert abs(fd - (eri.grad.numpy() * P).sum()) < 1e-9
