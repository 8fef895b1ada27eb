"""Pins for oracle A (full CI) against closed forms, brute force and invariants.

Each pin checks the oracle against something it does not compute itself:
textbook spectra, an independent Kronecker-product (Jordan-Wigner) build of
Eq. (hamil), the Slater-Condon diagonal, one-body closed-form dynamics, the
RK4 amplification factor, and library matrix exponentials.
"""
import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import fci


def _spin_orbital_ops(L):
    """Jordan-Wigner annihilators a_p on the 2^(2L) Fock space, mode order
    1up, 1down, 2up, ... (Eq. fci); basis index = sum_p n_p 2^p."""
    n = 2 * L
    a1 = np.array([[0.0, 1.0], [0.0, 0.0]])   # |0><1| on one mode (basis |0>,|1>)
    z = np.diag([1.0, -1.0])
    eye = np.eye(2)
    ops = []
    for p in range(n):
        mats = [z] * p + [a1] + [eye] * (n - p - 1)
        # kron with mode 0 as the least significant bit: kron(m_{n-1}, ..., m_0)
        M = np.array([[1.0]])
        for m in reversed(mats):
            M = np.kron(M, m)
        ops.append(M)
    return ops


def _kron_hamiltonian(h, eri):
    L = h.shape[0]
    a = _spin_orbital_ops(L)
    ad = [x.T for x in a]
    dim = 4 ** L
    H = np.zeros((dim, dim))
    for i in range(L):
        for j in range(L):
            for s in range(2):
                H += h[i, j] * ad[2 * i + s] @ a[2 * j + s]
    for i in range(L):
        for j in range(L):
            for k in range(L):
                for l in range(L):
                    for s in range(2):
                        for t in range(2):
                            H += 0.5 * eri[i, j, k, l] * (ad[2 * i + s] @ ad[2 * k + t]
                                                          @ a[2 * l + t] @ a[2 * j + s])
    return H, a


def _random_integrals(L, seed):
    return synth.make_integrals(L, seed=seed, n_chol=3)


def test_hubbard_dimer_closed_form():
    # Two sites, hopping -t, on-site U, two electrons with S_z = 0:
    # E = {0, U, (U +- sqrt(U^2 + 16 t^2))/2} (textbook Hubbard dimer).
    for t, U in [(1.0, 4.0), (0.3, 1.7), (2.0, 0.5)]:
        h = np.array([[0.0, -t], [-t, 0.0]])
        eri = np.zeros((2, 2, 2, 2))
        eri[0, 0, 0, 0] = eri[1, 1, 1, 1] = U
        dets = fci.basis(2, 1, 1)
        w = np.linalg.eigvalsh(fci.hamiltonian(h, eri, dets))
        ref = sorted([0.0, U, 0.5 * (U + np.sqrt(U * U + 16 * t * t)),
                      0.5 * (U - np.sqrt(U * U + 16 * t * t))])
        assert np.allclose(w, ref, atol=1e-13)


def test_one_electron_rabi_oscillation():
    # Two orbitals (h = [[e1, -t], [-t, e2]]), one up electron started in
    # orbital 0: orbital 1 holds it with the textbook Rabi probability
    # (4 t^2 / W^2) sin^2(W tau / 2), W = sqrt((e1 - e2)^2 + 4 t^2).
    for e1, e2, t in [(0.0, 0.0, 1.0), (-0.3, 0.5, 0.7)]:
        h = np.array([[e1, -t], [-t, e2]])
        eri = np.zeros((2, 2, 2, 2))
        eri[0, 0, 1, 1] = eri[1, 1, 0, 0] = 0.4     # no second electron: no effect
        dets = fci.basis(2, 1, 0)
        H = fci.hamiltonian(h, eri, dets)
        psi = np.zeros(len(dets), dtype=complex)
        psi[np.searchsorted(dets, np.uint64(fci.occupation_mask([1, 0])))] = 1.0
        W = np.sqrt((e1 - e2) ** 2 + 4 * t * t)
        for tau in (0.0, 0.37, 1.9):
            g = fci.one_rdm(fci.exact_evolve(H, psi, tau), dets, 2)
            assert abs(g[1, 1].real - 4 * t * t / W ** 2 * np.sin(W * tau / 2) ** 2) < 1e-13
            assert abs(np.trace(g).real - 1.0) < 1e-13


@pytest.mark.parametrize("L,na,nb", [(4, 2, 1), (5, 2, 2), (3, 3, 1)])
def test_noninteracting_spectrum_is_sum_of_orbital_energies(L, na, nb):
    I = _random_integrals(L, 3)
    eps = np.linalg.eigvalsh(I.h)
    from itertools import combinations
    ref = sorted(sum(eps[list(a)]) + sum(eps[list(b)])
                 for a in combinations(range(L), na) for b in combinations(range(L), nb))
    w = np.linalg.eigvalsh(fci.hamiltonian(I.h, np.zeros_like(I.eri), fci.basis(L, na, nb)))
    assert np.allclose(w, ref, atol=1e-12)


@pytest.mark.parametrize("L,seed", [(2, 0), (3, 1)])
def test_matches_kronecker_jordan_wigner_build(L, seed):
    I = _random_integrals(L, seed)
    Hk, _ = _kron_hamiltonian(I.h, I.eri)
    for na in range(L + 1):
        for nb in range(L + 1):
            dets = fci.basis(L, na, nb)
            # Fock index of a mask in the Kronecker basis is the mask itself
            idx = dets.astype(np.int64)
            ref = Hk[np.ix_(idx, idx)]
            assert np.allclose(fci.hamiltonian(I.h, I.eri, dets), ref, atol=1e-13)


def test_commutes_with_total_spin():
    L = 3
    I = _random_integrals(L, 5)
    Hk, a = _kron_hamiltonian(I.h, I.eri)
    ad = [x.T for x in a]
    Sp = sum(ad[2 * i] @ a[2 * i + 1] for i in range(L))
    Sz = sum(0.5 * (ad[2 * i] @ a[2 * i] - ad[2 * i + 1] @ a[2 * i + 1]) for i in range(L))
    S2 = Sp.T @ Sp + Sz @ Sz + Sz
    assert np.abs(Hk @ S2 - S2 @ Hk).max() < 1e-12
    # and the oracle's sector matrix equals the Kronecker one on that sector
    dets = fci.basis(L, 2, 1)
    idx = dets.astype(np.int64)
    assert np.allclose(fci.hamiltonian(I.h, I.eri, dets), Hk[np.ix_(idx, idx)], atol=1e-13)


def test_hermitian_and_slater_condon_diagonal():
    L = 5
    I = _random_integrals(L, 7)
    dets = fci.basis(L, 3, 2)
    H = fci.hamiltonian(I.h, I.eri, dets)
    assert np.abs(H - H.T).max() < 1e-13
    for row, m in enumerate(dets[:25]):
        occ = [(p // 2, p % 2) for p in range(2 * L) if (int(m) >> p) & 1]
        e = sum(I.h[i, i] for i, _ in occ)
        for x, (i, s) in enumerate(occ):
            for y, (j, t) in enumerate(occ):
                if x == y:
                    continue
                e += 0.5 * I.eri[i, i, j, j]
                if s == t:
                    e -= 0.5 * I.eri[i, j, j, i]
        assert abs(H[row, row] - e) < 1e-12


def test_h_on_determinant_matches_dense_columns():
    I = synth.make_integrals(6, seed=2)
    dets = fci.basis(6, 3, 2)
    for e0 in (0.0, 0.37):
        H = fci.hamiltonian(I.h, I.eri, dets, e0)
        for col in (0, 17, 101):
            m, c = fci.h_on_determinant(I.h, I.eri, int(dets[col]), e0)
            full = np.zeros(len(dets))
            full[np.searchsorted(dets, m)] = c
            assert np.allclose(full, H[:, col], atol=1e-13)


def test_one_rdm_of_determinant_and_trace():
    L = 5
    occ = [3, 1, 0, 2, 0]
    dets = fci.basis(L, 2, 2)
    psi = np.zeros(len(dets), dtype=complex)
    psi[np.searchsorted(dets, np.uint64(fci.occupation_mask(occ)))] = 1.0
    g = fci.one_rdm(psi, dets, L)
    assert np.allclose(g, np.diag([2, 1, 0, 1, 0]), atol=1e-15)
    rng = np.random.default_rng(0)
    v = rng.standard_normal(len(dets)) + 1j * rng.standard_normal(len(dets))
    v /= np.linalg.norm(v)
    g = fci.one_rdm(v, dets, L)
    assert abs(np.trace(g) - 4) < 1e-12
    assert np.abs(g - g.conj().T).max() < 1e-13
    w = np.linalg.eigvalsh(g)
    assert w.min() > -1e-12 and w.max() < 2 + 1e-12


def test_noninteracting_dynamics_closed_form():
    # V = 0: gamma(t) = conj(U) gamma(0) U^T with U = exp(-i h t).
    L = 5
    I = _random_integrals(L, 11)
    dets = fci.basis(L, 2, 2)
    H = fci.hamiltonian(I.h, np.zeros_like(I.eri), dets)
    occ = [3, 2, 1, 0, 0]
    psi = np.zeros(len(dets), dtype=complex)
    psi[np.searchsorted(dets, np.uint64(fci.occupation_mask(occ)))] = 1.0
    g0 = fci.one_rdm(psi, dets, L)
    for t in (0.3, 2.0):
        U = scipy.linalg.expm(-1j * I.h * t)
        ref = U.conj() @ g0 @ U.T
        gt = fci.one_rdm(fci.exact_evolve(H, psi, t), dets, L)
        assert np.allclose(gt, ref, atol=1e-12)


def test_rk4_is_fourth_order_taylor_and_norm_factor():
    L = 4
    I = _random_integrals(L, 13)
    dets = fci.basis(L, 2, 1)
    H = fci.hamiltonian(I.h, I.eri, dets)
    rng = np.random.default_rng(1)
    psi = rng.standard_normal(len(dets)) + 1j * rng.standard_normal(len(dets))
    psi /= np.linalg.norm(psi)
    dt = 0.37
    from math import factorial
    taylor = sum(np.linalg.matrix_power(-1j * dt * H, p) @ psi / factorial(p) for p in range(5))
    out = fci.rk4_step(H, psi, dt)
    assert np.allclose(out, taylor, atol=1e-12)
    # per eigencomponent |r(x)|^2 = 1 - x^6/72 + x^8/576 with x = lambda dt
    lam, V = np.linalg.eigh(H)
    c = V.conj().T @ psi
    x = lam * dt
    pred = np.sum(np.abs(c) ** 2 * (1 - x ** 6 / 72 + x ** 8 / 576))
    assert abs(np.vdot(out, out).real - pred) < 1e-12


def test_krylov_full_space_is_exact_and_conserves_norm():
    L = 3
    I = _random_integrals(L, 17)
    dets = fci.basis(L, 2, 1)
    H = fci.hamiltonian(I.h, I.eri, dets)
    rng = np.random.default_rng(2)
    psi = rng.standard_normal(len(dets)) + 1j * rng.standard_normal(len(dets))
    psi /= np.linalg.norm(psi)
    n = len(dets)
    out = fci.krylov_step(H, psi, 0.9, n)
    assert np.allclose(out, scipy.linalg.expm(-1j * 0.9 * H) @ psi, atol=1e-10)
    out5 = fci.krylov_step(H, psi, 0.1, 5)
    assert abs(np.linalg.norm(out5) - 1.0) < 1e-13


def test_krylov_conserves_energy_and_beats_rk4_at_equal_cost():
    """Sec. 2.2.3: the Krylov step conserves norm and energy even with m below
    the space dimension -- the new state lies in the Krylov space, where the
    propagator is a function of the projected H.  With N_K = 5 (four H
    applications, the cost of one RK4 step) it is far more accurate than RK4
    over the same time (the paper's comparison, here with a wide margin)."""
    I = _random_integrals(4, 17)
    dets = fci.basis(4, 2, 2)
    H = fci.hamiltonian(I.h, I.eri, dets)
    rng = np.random.default_rng(17)
    psi = rng.standard_normal(len(dets)) + 1j * rng.standard_normal(len(dets))
    psi /= np.linalg.norm(psi)
    out = fci.krylov_step(H, psi, 0.2, 5)
    assert abs(np.linalg.norm(out) - 1.0) < 1e-13
    assert abs(fci.energy(H, out) - fci.energy(H, psi)) < 1e-12
    a, b = psi.copy(), psi.copy()
    for _ in range(10):
        a = fci.rk4_step(H, a, 0.1)
        b = fci.krylov_step(H, b, 0.1, 5)
    exact = fci.exact_evolve(H, psi, 1.0)
    assert np.linalg.norm(b - exact) < 1e-2 * np.linalg.norm(a - exact)


def test_krylov_orthogonal_and_plain_bases_agree():
    # Both constructions span the same Krylov space; Eq. (krylov_evo) with the
    # measured N is basis independent in exact arithmetic.
    L = 4
    I = _random_integrals(L, 19)
    dets = fci.basis(L, 2, 2)
    H = fci.hamiltonian(I.h, I.eri, dets)
    rng = np.random.default_rng(3)
    psi = rng.standard_normal(len(dets)) + 1j * rng.standard_normal(len(dets))
    a, P = fci.krylov_step(H, psi, 0.05, 4, orthogonal=True, return_basis=True)
    b, Q = fci.krylov_step(H, psi, 0.05, 4, orthogonal=False, return_basis=True)
    assert np.allclose(a, b, atol=1e-10)
    # Eq. (kry_orth) makes the basis orthogonal, and phi_1.. are normalised
    # (phi_0 = psi keeps its norm); Eq. (kry_non) is not orthogonal
    G = P.conj().T @ P
    assert np.allclose(G - np.diag(np.diag(G)), 0.0, atol=1e-12)
    assert np.allclose(np.diag(G)[1:], 1.0, atol=1e-12)
    G2 = Q.conj().T @ Q
    assert np.abs(G2 - np.diag(np.diag(G2))).max() > 1e-3


def test_krylov_coefficients_match_expm_and_scaling_invariance():
    rng = np.random.default_rng(4)
    m = 5
    A = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    Hk = A + A.conj().T
    c, dropped = fci.krylov_coefficients(np.eye(m), Hk, 0.3)
    assert dropped == 0
    assert np.allclose(c, scipy.linalg.expm(-0.3j * Hk)[:, 0], atol=1e-13)
    # non-orthogonal basis P = Q S: coefficients transform with S^-1
    S = np.triu(rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) + 3 * np.eye(m)
    S[0, 0] = 1.0       # column 0 = e_0: phi_0 unchanged; the later vectors keep
    #                     complex phi_0 components, so N[:, 0] is complex
    N = S.conj().T @ S
    assert np.abs(N[1:, 0].imag).max() > 1e-2
    H2 = S.conj().T @ Hk @ S
    c2, _ = fci.krylov_coefficients(N, H2, 0.3)
    assert np.allclose(S @ c2, c, atol=1e-12)
    # the definition of Eq. (krylov_evo) for a regular N
    assert np.allclose(c2, scipy.linalg.expm(-0.3j * np.linalg.solve(N, H2))[:, 0], atol=1e-11)


def test_krylov_error_decreases_with_time_step():
    L = 4
    I = _random_integrals(L, 23)
    dets = fci.basis(L, 2, 2)
    H = fci.hamiltonian(I.h, I.eri, dets)
    psi = np.zeros(len(dets), dtype=complex)
    psi[3] = 1.0
    errs = []
    for dt in (0.2, 0.1):
        errs.append(np.linalg.norm(fci.krylov_step(H, psi, dt, 4) - fci.exact_evolve(H, psi, dt)))
    # local error O(dt^m): halving dt shrinks it by ~2^4
    assert errs[1] < errs[0] / 8


@pytest.mark.parametrize("L", [1, 2, 3])
def test_apply_op_equals_kronecker_operators(L):
    # a_p and a+_p on determinant bit strings (mask = sum_p n_p 2^p) equal the
    # Jordan-Wigner Kronecker matrices of every spin orbital
    ops = _spin_orbital_ops(L)
    masks = np.arange(4 ** L, dtype=np.uint64)
    for p in range(2 * L):
        for dagger in (False, True):
            new, amp = fci.apply_op(masks, np.ones(len(masks)), p, dagger)
            M = np.zeros((4 ** L, 4 ** L))
            for old, (n, a) in enumerate(zip(new, amp)):
                if a != 0.0:
                    M[int(n), old] += a
            ref = ops[p].T if dagger else ops[p]
            assert np.array_equal(M, ref), (p, dagger)
