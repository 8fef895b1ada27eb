"""Pins for the oracle's site operators, MPS-from-vector decomposition,
transition and two-body density matrices and one-particle Green's function
(Eq. green_time) against Kronecker-product Jordan-Wigner operators, closed
forms of the non-interacting problem and exact identities."""
import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import fci
from oracle import mps as om
from jw_kron import site_config_index, spin_orbital_ops


def _rand_sector_vector(dets, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(len(dets)) + 1j * rng.standard_normal(len(dets))
    return v / np.linalg.norm(v)


def _labels_consistent(m):
    for i, A in enumerate(m.tensors):
        ql, qr = m.labels[i], m.labels[i + 1]
        for a, s, b in zip(*np.nonzero(np.abs(A) > 0)):
            if not np.array_equal(ql[a] + om.SITE_Q[s], qr[b]):
                return False
    return True


@pytest.mark.parametrize("dagger", [False, True])
def test_site_op_matches_kronecker_operators(dagger):
    L = 3
    A, q = synth.random_mps(L, 3, 1, 6, seed=4)
    m = om.from_arrays(A, q)
    a = spin_orbital_ops(L)
    idx = site_config_index(L)
    vk = om.to_fock(m)[idx]
    for i in range(L):
        for s in range(2):
            op = a[2 * i + s].T if dagger else a[2 * i + s]
            out = om.apply_site_op(m, i, s, dagger)
            assert _labels_consistent(out)
            assert np.allclose(om.to_fock(out)[idx], op @ vk, atol=1e-14)
            sign = 1 if dagger else -1
            assert np.array_equal(out.labels[-1][0], m.labels[-1][0] + sign * om.SITE_Q[1 + s])


def test_site_ops_anticommute():
    L = 3
    A, q = synth.random_mps(L, 3, -1, 6, seed=5)
    m = om.from_arrays(A, q)
    v = om.to_fock(m)
    for p in range(2 * L):
        for r in range(2 * L):
            x = om.apply_site_op(om.apply_site_op(m, r // 2, r % 2, True), p // 2, p % 2, False)
            y = om.apply_site_op(om.apply_site_op(m, p // 2, p % 2, False), r // 2, r % 2, True)
            assert np.allclose(om.to_fock(x) + om.to_fock(y), v * (p == r), atol=1e-14)


def test_from_fock_contracts_back_with_full_ci_bond_profile():
    L = 5
    dets = fci.basis(L, 3, 2)
    v = _rand_sector_vector(dets, 6)
    m = om.from_fock(om.sector_to_fock(v, dets, L), L)
    assert np.abs(om.to_sector(m, dets) - v).max() < 1e-14
    assert _labels_consistent(m)
    # a generic vector has the full rank at every cut: the number of
    # (left, right) configuration pairs of matching charge, bounded by 4^k
    for k, D in enumerate(m.bond_dims):
        assert D <= min(4 ** k, 4 ** (L - k))
    assert m.bond_dims[2] == 16 and m.bond_dims[3] == 16


def test_transition_and_two_rdm_match_kronecker_operators():
    L = 3
    a = spin_orbital_ops(L)
    ad = [x.T for x in a]
    dets = fci.basis(L, 2, 1)
    bra, ket = _rand_sector_vector(dets, 7), _rand_sector_vector(dets, 8)
    full = lambda v: (lambda o: (o.__setitem__(dets.astype(np.int64), v), o)[1])(
        np.zeros(4 ** L, dtype=complex))
    B, K = full(bra), full(ket)
    T = fci.transition_rdm(bra, ket, dets, L)
    for i in range(L):
        for j in range(L):
            ref = sum(np.vdot(B, ad[2 * i + s] @ a[2 * j + s] @ K) for s in range(2))
            assert abs(T[i, j] - ref) < 1e-13
    assert np.allclose(fci.transition_rdm(ket, ket, dets, L), fci.one_rdm(ket, dets, L), atol=1e-15)
    G = fci.two_rdm(ket, dets, L)
    for i, j, k, l in np.ndindex(L, L, L, L):
        ref = sum(np.vdot(K, ad[2 * i + s] @ ad[2 * k + t] @ a[2 * l + t] @ a[2 * j + s] @ K)
                  for s in range(2) for t in range(2))
        assert abs(G[i, j, k, l] - ref) < 1e-13


def test_two_rdm_energy_trace_and_symmetries():
    L = 4
    I = synth.make_integrals(L, seed=9, n_chol=3)
    dets = fci.basis(L, 2, 1)
    v = _rand_sector_vector(dets, 10)
    H = fci.hamiltonian(I.h, I.eri, dets, 0.37)
    g = fci.one_rdm(v, dets, L)
    G = fci.two_rdm(v, dets, L)
    e = np.einsum("ij,ij->", I.h, g) + 0.5 * np.einsum("ijkl,ijkl->", I.eri, G) + 0.37
    assert abs(e - np.vdot(v, H @ v)) < 1e-12
    n = 3
    assert np.allclose(np.einsum("ijkk->ij", G), (n - 1) * g, atol=1e-13)
    assert np.allclose(G, G.transpose(2, 3, 0, 1), atol=1e-14)
    assert np.allclose(G, G.transpose(1, 0, 3, 2).conj(), atol=1e-14)


def test_green_function_noninteracting_closed_form():
    # V = 0 and psi0 an eigenstate (E0): exp(iH tau) a_j exp(-iH tau) =
    # sum_q [exp(-i h tau)]_jq a_q, so the numerator of Eq. (green_time) is
    # exp(i E0 tau) [gamma exp(-i h tau)]_ij with the spin-summed 1BRDM gamma.
    L = 4
    I = synth.make_integrals(L, seed=12, n_chol=3)
    eri0 = np.zeros_like(I.eri)
    dets = fci.basis(L, 2, 2)
    H = fci.hamiltonian(I.h, eri0, dets, 0.25)
    w, U = np.linalg.eigh(H)
    psi0 = U[:, 0].astype(complex)
    g = fci.one_rdm(psi0, dets, L)
    taus = np.array([0.0, 0.3, 1.1])
    for i, j in [(0, 0), (1, 2), (3, 1)]:
        G = fci.green_function(I.h, eri0, psi0, dets, L, i, j, taus, 0.25)
        ref = np.array([-1j * np.exp(1j * w[0] * t) * (g @ scipy.linalg.expm(-1j * I.h * t))[i, j]
                        / g[i, j] for t in taus])
        assert np.allclose(G, ref, atol=1e-11)
        assert abs(G[0] + 1j) < 1e-13


@pytest.mark.parametrize("t,U", [(1.0, 4.0), (0.3, 1.7), (2.0, 0.5), (1.0, 0.0)])
def test_green_function_hubbard_dimer_lehmann_closed_form(t, U):
    """Interacting pin (textbook Hubbard dimer: hopping -t, on-site U, two
    electrons in the singlet ground state, E0 = (U - sqrt(U^2 + 16 t^2))/2).
    The ground state is C |covalent> + I |ionic> with I / C = r = |E0| / (2t).
    Removing an electron leaves one electron, whose states are the bonding
    (energy -t) and antibonding (+t) orbitals, reached with the Lehmann weights
    w_b = (1 + r)^2 / (2 (1 + r^2)) and w_a = (1 - r)^2 / (2 (1 + r^2))
    (w_b + w_a = 1 = the occupation of one site).  So
        G_11(tau) = -i (w_b e^{-i t tau} + w_a e^{+i t tau}),
        G_12(tau) = -i (w_b e^{-i t tau} - w_a e^{+i t tau}) / (w_b - w_a):
    the antibonding orbital changes sign between the sites, and any sign
    convention multiplies numerator and normalisation alike."""
    h = np.array([[0.0, -t], [-t, 0.0]])
    eri = np.zeros((2, 2, 2, 2))
    eri[0, 0, 0, 0] = eri[1, 1, 1, 1] = U
    dets = fci.basis(2, 1, 1)
    w, V = np.linalg.eigh(fci.hamiltonian(h, eri, dets))
    E0 = 0.5 * (U - np.sqrt(U * U + 16 * t * t))
    assert abs(w[0] - E0) < 1e-13 and w[1] - w[0] > 1e-6
    psi0 = V[:, 0].astype(complex)
    r = abs(E0) / (2 * t)
    wb = (1 + r) ** 2 / (2 * (1 + r * r))
    wa = (1 - r) ** 2 / (2 * (1 + r * r))
    taus = np.array([0.0, 0.4, 1.3, 2.9])
    G11 = fci.green_function(h, eri, psi0, dets, 2, 0, 0, taus)
    assert np.allclose(G11, -1j * (wb * np.exp(-1j * t * taus) + wa * np.exp(1j * t * taus)),
                       atol=1e-12)
    G12 = fci.green_function(h, eri, psi0, dets, 2, 0, 1, taus)
    assert np.allclose(G12, -1j * (wb * np.exp(-1j * t * taus) - wa * np.exp(1j * t * taus))
                       / (wb - wa), atol=1e-12)


def test_green_function_equals_kronecker_fock_space():
    """Eq. (green_time) on the whole Fock space with Kronecker-product
    Jordan-Wigner operators and scipy's matrix exponential, for a random
    complex state with unequal spin counts (so neither the i <-> j exchange
    nor the two spins are related by a symmetry)."""
    L = 3
    I = synth.make_integrals(L, seed=21, n_chol=3)
    dets = fci.basis(L, 2, 1)
    psi0 = _rand_sector_vector(dets, 22)
    a = spin_orbital_ops(L)
    ad = [x.T for x in a]
    H = np.zeros((4 ** L, 4 ** L))
    for i in range(L):
        for j in range(L):
            for s in range(2):
                H += I.h[i, j] * ad[2 * i + s] @ a[2 * j + s]
    for i in range(L):
        for j in range(L):
            for k in range(L):
                for l in range(L):
                    for s in range(2):
                        for u in range(2):
                            H += 0.5 * I.eri[i, j, k, l] * (ad[2 * i + s] @ ad[2 * k + u]
                                                           @ a[2 * l + u] @ a[2 * j + s])
    v = np.zeros(4 ** L, dtype=complex)
    v[dets.astype(np.int64)] = psi0        # a determinant mask is its Kronecker index
    taus = np.array([0.0, 0.35, 1.2])
    for i, j in [(0, 2), (2, 0), (1, 1), (2, 1)]:
        den = sum(np.vdot(a[2 * i + s] @ v, a[2 * j + s] @ v) for s in range(2))
        ref = np.array([-1j * sum(np.vdot(a[2 * i + s] @ v,
                                          scipy.linalg.expm(1j * H * t) @ (a[2 * j + s] @ v))
                                  for s in range(2)) / den for t in taus])
        G = fci.green_function(I.h, I.eri, psi0, dets, L, i, j, taus)
        assert np.allclose(G, ref, atol=1e-11)


def test_mps_green_function_matches_full_ci():
    L = 4
    I = synth.make_integrals(L, seed=13, n_chol=3)
    dets = fci.basis(L, 2, 2)
    w, U = np.linalg.eigh(fci.hamiltonian(I.h, I.eri, dets))
    psi0 = om.from_fock(om.sector_to_fock(U[:, 0].astype(complex), dets, L), L)
    systems = {0: om.System.build(I.h, I.eri, 1, 2), 1: om.System.build(I.h, I.eri, 2, 1)}
    sch = om.Schedule(D=64, eps=0.0, n_two_site=1, n_one_site=1)
    dt, n = 0.1, 3
    G = om.green_function(systems, psi0, 1, 2, dt, n, 6, sch)
    ref = fci.green_function(I.h, I.eri, U[:, 0], dets, L, 1, 2, dt * np.arange(n + 1))
    assert np.allclose(G, ref, atol=1e-9)
    # RK4 variant: untruncated, it equals the same backward steps taken by the
    # vector RK4 (time step -dt) on the ionised full-CI vectors
    G4 = om.green_function(systems, psi0, 1, 2, dt, n, 6, sch, method="rk4")
    num = np.zeros(n + 1, dtype=complex)
    den = 0.0
    for s, (na, nb) in ((0, (1, 2)), (1, (2, 1))):
        dm = fci.basis(L, na, nb)
        Hm = fci.hamiltonian(I.h, I.eri, dm)
        chi_i = fci.apply_to_vector(U[:, 0], dets, dm, 2 * 1 + s, False)
        chi = fci.apply_to_vector(U[:, 0], dets, dm, 2 * 2 + s, False)
        den += np.vdot(chi_i, chi)
        num[0] += np.vdot(chi_i, chi)
        for k in range(n):
            chi = fci.rk4_step(Hm, chi, -dt)
            num[k + 1] += np.vdot(chi_i, chi)
    assert np.allclose(G4, -1j * num / den, atol=1e-9)
    assert np.abs(G4 - ref).max() > 1e-9    # RK4 is not the exact propagation
