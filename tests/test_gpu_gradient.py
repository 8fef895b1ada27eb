"""The adjoint of the energy (tdmps_energy_gradient, grad.state_energy) and the
integral gradient (grad.energy) on the GPU.

* dE/dconj(A_i) = (H_i A_i - E N_i A_i) / <psi|psi> against the oracle's
  (oracle.bsmps.energy_gradient, pinned on the CPU against full CI and finite
  differences), element by element; environments kept at every bond or
  rebuilt between checkpoints give the same bits.
* The differentiation workload: a Krylov trajectory of L = 12 orbitals, 12
  electrons (2S_z = 0) from the aufbau determinant (a correlation quench),
  D = 128, at 50 time points.  At three of them the gradients with respect to
  h_ij, (ij|kl) and the site tensors are checked against central finite
  differences with step 1e-6 in FP64, to <= 1e-6 relative; the hole density
  per orbital (gamma_ii(0) - gamma_ii(t)) is printed against time.
"""
import numpy as np
import pytest

import synth
from oracle import bsmps as ob

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def td():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_08489_gb300 as mod
    mod.lib()
    return mod


def test_state_gradient_matches_block_sparse_oracle(td):
    L = 8
    I = synth.make_integrals(L, seed=30)
    A, q = synth.random_mps(L, 7, 1, 40, seed=31)
    ctx = td.Context("tf32x3")          # the adjoint runs in FP64 in every precision
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=7, e0=0.4)
    psi = td.mps_import(ctx, A, q)
    E, G, _ = td.energy_gradient(ctx, mpo, psi)
    gt, gq = G.export()
    Eo, Go = ob.energy_gradient(ob.hamiltonian_mpo(I.h, I.eri, 0.4), ob.from_dense(A, q))
    got = ob.from_dense(gt, gq)
    assert abs(E - Eo) < 1e-12 * abs(Eo)
    scale = max(np.abs(b).max() for s in Go for b in s.values())
    err = max(np.abs(got.sites[i][k] - Go[i][k]).max() for i in range(L) for k in Go[i])
    print("state gradient L=8 D=40 vs oracle: max abs error %.2e (max |G| %.2e)" % (err, scale))
    assert err < 1e-11 * scale
    ctx.close()


def test_recomputed_environments_give_the_same_gradient(td):
    L = 12
    I = synth.make_integrals(L, seed=32)
    A, q = synth.random_mps(L, 12, 0, 64, seed=33)
    ctx = td.Context("fp64")
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=12)
    psi = td.mps_import(ctx, A, q)
    E1, G1, peak1 = td.energy_gradient(ctx, mpo, psi, stride=1)
    E4, G4, peak4 = td.energy_gradient(ctx, mpo, psi, stride=4)
    t1, _ = G1.export()
    t4, _ = G4.export()
    print("environment memory: all kept %.1f MB, every 4th bond kept %.1f MB"
          % (peak1 / 1e6, peak4 / 1e6))
    assert E1 == E4
    assert all(np.array_equal(a, b) for a, b in zip(t1, t4))
    assert peak4 < peak1
    with pytest.raises(td.TdmpsError):
        td.energy_gradient(ctx, mpo, psi, stride=0)
    ctx.close()


def test_state_energy_autograd(td):
    torch = pytest.importorskip("torch")
    from paper_1902_08489_gb300 import grad
    L = 6
    I = synth.make_integrals(L, seed=34)
    A, q = synth.random_mps(L, 5, 1, 16, seed=35)
    # the caller's vector order need not be the library's (sectors grouped):
    # reverse every inner bond
    rev = [np.arange(len(x))[::-1] if 0 < i < L else np.arange(len(x)) for i, x in enumerate(q)]
    A = [a[np.ix_(rev[i], np.arange(4), rev[i + 1])] for i, a in enumerate(A)]
    q = [x[r] for x, r in zip(q, rev)]
    ctx = td.Context("fp64")
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=5)
    ts = [torch.tensor(a, dtype=torch.complex128, requires_grad=True) for a in A]
    E = grad.state_energy(ctx, mpo, q, ts)
    E.backward()
    psi_o = ob.from_dense(A, q)
    Eo, Go = ob.energy_gradient(ob.hamiltonian_mpo(I.h, I.eri), psi_o)
    assert abs(E.item() - Eo) < 1e-12 * abs(Eo)
    # the oracle's gradient back in the caller's dense layout
    ref_t, ref_q = ob.to_dense(ob.BMPS(psi_o.bonds, Go))
    from paper_1902_08489_gb300.grad import _vector_order
    perm = [_vector_order(a, b) for a, b in zip(q, ref_q)]
    # torch's gradient of a real function of complex z is 2 dE/dconj(z)
    for i in range(L):
        ref = ref_t[i][np.ix_(perm[i], np.arange(4), perm[i + 1])]
        assert np.abs(ts[i].grad.numpy() - 2 * ref).max() < 1e-11 * max(1.0, np.abs(ref).max())
    ctx.close()


def _fd_rel(fd, an, scale):
    return abs(fd - an) / scale


def test_differentiation_workload_L12_D128_trajectory(td):
    L, N = 12, 12
    I = synth.make_integrals(L, seed=0)
    occ = synth.aufbau_occupation(L, N)
    ctx = td.Context("fp64")
    ctx.set_schedule(1, 1)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=N)
    psi = td.mps_from_determinant(ctx, occ)
    g0 = np.real(np.diag(td.one_rdm(ctx, psi)))
    rng = np.random.default_rng(36)
    step, h_fd = 1e-6, 1e-6
    worst = 0.0
    holes = []
    for t in range(1, 51):
        td.krylov_step(ctx, mpo, psi, 0.05, 6, True, 128, 1e-10)
        n2 = td.overlap(ctx, psi, psi).real
        holes.append(g0 - np.real(np.diag(td.one_rdm(ctx, psi))) / n2)
        if t not in (10, 30, 50):
            continue
        dh, deri = td.integral_gradient(ctx, psi)

        def e_of(hh, ee):
            m = td.build_mpo(ctx, hh, ee, n_elec=N)
            e = td.energy(ctx, m, psi)
            m.free()
            return e
        for _ in range(3):
            i, j = rng.integers(L, size=2)
            P = np.zeros((L, L))
            P[i, j] = P[j, i] = 1.0
            fd = (e_of(I.h + h_fd * P, I.eri) - e_of(I.h - h_fd * P, I.eri)) / (2 * h_fd)
            worst = max(worst, _fd_rel(fd, (dh * P).sum(), np.abs(dh).max()))
        for _ in range(3):
            i, j, k, l = rng.integers(L, size=4)
            P = np.zeros((L,) * 4)
            for a, b, c, e in [(i, j, k, l), (j, i, k, l), (i, j, l, k), (j, i, l, k),
                               (k, l, i, j), (l, k, i, j), (k, l, j, i), (l, k, j, i)]:
                P[a, b, c, e] = 1.0
            fd = (e_of(I.h, I.eri + h_fd * P) - e_of(I.h, I.eri - h_fd * P)) / (2 * h_fd)
            worst = max(worst, _fd_rel(fd, (deri * P).sum(), np.abs(deri).max()))
        # the state gradient: central differences of E along single entries
        E, G, _ = td.energy_gradient(ctx, mpo, psi, stride=3)
        gt, _ = G.export()
        A, q = psi.export()
        for _ in range(4):
            s = int(rng.integers(L))
            nz = np.argwhere(np.abs(gt[s]) > 0.1 * np.abs(gt[s]).max())
            idx = tuple(nz[rng.integers(len(nz))])
            for d in (1.0, 1j):
                Ap = [a.copy() for a in A]
                Am = [a.copy() for a in A]
                Ap[s][idx] += step * d
                Am[s][idx] -= step * d
                pp, pm = td.mps_import(ctx, Ap, q), td.mps_import(ctx, Am, q)
                fd = (td.energy(ctx, mpo, pp) - td.energy(ctx, mpo, pm)) / (2 * step)
                pp.free()
                pm.free()
                an = 2 * (np.conj(gt[s][idx]) * d).real
                worst = max(worst, _fd_rel(fd, an, np.abs(gt[s]).max()))
        print("t = %d: max relative gradient error vs central differences %.2e" % (t, worst))
    holes = np.array(holes)
    print("hole density per orbital (gamma_ii(0) - gamma_ii(t)), every 10th of 50 steps:")
    for t in range(9, 50, 10):
        print("  t = %.2f a.u.: %s" % (0.05 * (t + 1), np.array2string(holes[t], precision=4)))
    assert abs(holes[-1].sum()) < 1e-8          # particle number is conserved
    assert worst <= 1e-6
    ctx.close()


def test_integral_gradient_equals_full_ci_rdms_L8(td):
    # dE/dh = Re gamma / <psi|psi>, dE/d(ij|kl) = Re Gamma / (2 <psi|psi>) against
    # the full-CI density matrices of the contracted state (L = 8, 7 electrons)
    from oracle import fci
    from oracle import mps as om
    L = 8
    I = synth.make_integrals(L, seed=37)
    A, q = synth.random_mps(L, 7, 1, 40, seed=38)
    ctx = td.Context("tf32x3")          # the density matrices are FP64 in every precision
    psi = td.mps_import(ctx, A, q)
    dh, deri = td.integral_gradient(ctx, psi)
    dets = fci.basis(L, 4, 3)
    v = om.to_sector(om.from_arrays(A, q), dets)
    n2 = np.vdot(v, v).real
    g = fci.one_rdm(v, dets, L).real / n2
    G = 0.5 * fci.two_rdm(v, dets, L).real / n2
    e1, e2 = np.abs(dh - g).max(), np.abs(deri - G).max()
    print("integral gradient L=8 vs full CI: dE/dh %.2e, dE/deri %.2e" % (e1, e2))
    assert e1 < 1e-11 * np.abs(g).max() and e2 < 1e-11 * np.abs(G).max()
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=7)
    H = fci.hamiltonian(I.h, I.eri, dets)
    assert abs(td.energy(ctx, mpo, psi) - np.vdot(v, H @ v).real / n2) < 1e-11
    ctx.close()


@pytest.mark.parametrize("L,stride", [(1, 1), (2, 1), (3, 2), (4, 9)])
def test_state_gradient_short_chains_and_wide_strides(td, L, stride):
    # the boundaries of the adjoint: one and two sites, a checkpoint stride
    # that does not divide L, one longer than the chain
    I = synth.make_integrals(L, seed=40 + L)
    n = max(1, L - 1)
    A, q = synth.random_mps(L, n, n % 2, 8, seed=41 + L)
    ctx = td.Context("fp64")
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=n)
    psi = td.mps_import(ctx, A, q)
    E, G, _ = td.energy_gradient(ctx, mpo, psi, stride=stride)
    gt, gq = G.export()
    Eo, Go = ob.energy_gradient(ob.hamiltonian_mpo(I.h, I.eri), ob.from_dense(A, q))
    got = ob.from_dense(gt, gq)
    assert abs(E - Eo) < 1e-12 * max(1.0, abs(Eo))
    scale = max(np.abs(b).max() for s in Go for b in s.values())
    err = max(np.abs(got.sites[i][k] - Go[i][k]).max() for i in range(L) for k in Go[i])
    # (at L = 1 the one-dimensional sector makes the gradient vanish)
    assert err <= 1e-11 * max(scale, abs(Eo))
    ctx.close()
