"""GPU edge cases against the oracle and closed forms: a single orbital,
the empty and the full sector (one-dimensional Hilbert spaces), the largest
orbital count the oracle's determinant masks cover (L = 32, the size of the
iodoacetylene-like active space), ragged odd bond dimensions, compression to
D = 1, and argument errors."""
from math import factorial

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


@pytest.fixture(scope="module")
def ctx(td):
    c = td.Context("fp64")
    yield c
    c.close()


def _taylor4(x):
    """RK4 amplification r(x) = sum_{p<=4} x^p / p! (x = -i E dt)."""
    return sum(x ** p / factorial(p) for p in range(5))


def _vec(m):
    t, q = m.export()
    return om.to_fock(om.from_arrays(t, q))


def test_single_orbital(td, ctx):
    h = np.array([[-1.3]])
    eri = np.array([[[[0.8]]]])
    mpo = td.build_mpo(ctx, h, eri, n_elec=2, e0=0.1)
    for occ, E in [([1], -1.3 + 0.1), ([2], -1.3 + 0.1), ([3], 2 * -1.3 + 0.8 + 0.1)]:
        psi = td.mps_from_determinant(ctx, occ)
        assert abs(td.expectation(ctx, mpo, psi, psi) - E) < 1e-14
        out = td.apply_H(ctx, mpo, psi, 0.3 - 0.2j, 4, 0.0)
        assert abs(td.overlap(ctx, psi, out) - (0.3 - 0.2j) * E) < 1e-13
        td.rk4_step(ctx, mpo, psi, 0.05, 4)
        assert abs(td.overlap(ctx, td.mps_from_determinant(ctx, occ), psi) - _taylor4(-1j * E * 0.05)) < 1e-13
        g = td.one_rdm(ctx, psi)
        assert abs(g[0, 0] - bin(occ[0]).count("1") * abs(_taylor4(-1j * E * 0.05)) ** 2) < 1e-12
    # a one-dimensional sector has no second Krylov direction
    psi = td.mps_from_determinant(ctx, [3])
    with pytest.raises(td.TdmpsError) as e:
        td.krylov_step(ctx, mpo, psi, 0.05, 2, True, 4)
    assert e.value.name in ("KRYLOV_SINGULAR", "ZERO_STATE", "NONFINITE")


def test_empty_and_full_sectors(td, ctx):
    L = 4
    I = synth.make_integrals(L, seed=41)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=0, e0=0.7)
    vac = td.mps_from_determinant(ctx, [0] * L)
    out = td.apply_H(ctx, mpo, vac, 2.0, 8, 0.0)
    assert abs(td.overlap(ctx, vac, out) - 1.4) < 1e-13
    assert np.abs(td.one_rdm(ctx, vac)).max() == 0.0
    # the full sector: one determinant, an eigenstate with the closed-form energy
    full = td.mps_from_determinant(ctx, [3] * L)
    m, c = fci.h_on_determinant(I.h, I.eri, fci.occupation_mask([3] * L), 0.7)
    assert len(m) == 1
    E = c[0]
    assert abs(td.expectation(ctx, mpo, full, full) - E) < 1e-12
    td.rk4_step(ctx, mpo, full, 0.02, 8)
    ref = td.mps_from_determinant(ctx, [3] * L)
    assert abs(td.overlap(ctx, ref, full) - _taylor4(-1j * E * 0.02)) < 1e-12
    assert np.allclose(td.one_rdm(ctx, full), 2 * abs(_taylor4(-1j * E * 0.02)) ** 2 * np.eye(L), atol=1e-12)
    # H|0> = 0 without e0: a vanished target is either an exact zero state or ZERO_STATE
    mpo0 = td.build_mpo(ctx, I.h, I.eri, n_elec=0)
    try:
        z = td.apply_H(ctx, mpo0, vac, 1.0, 8, 0.0)
        assert abs(td.overlap(ctx, z, z)) == 0.0
    except td.TdmpsError as e:
        assert e.name == "ZERO_STATE"


def test_largest_orbital_count_determinant_matrix_elements(td, ctx):
    # L = 32 (64 spin orbitals fill the oracle's 64-bit masks), 23 electrons,
    # the localised-block integrals of the large active space
    L = 32
    I = synth.make_integrals(L, seed=5, n_chol=16, localised_block=True)
    occ = [3] * 11 + [1] + [0] * 20
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=23)
    psi = td.mps_from_determinant(ctx, occ)
    masks, coefs = fci.h_on_determinant(I.h, I.eri, fci.occupation_mask(occ))
    col = dict(zip((int(x) for x in masks), coefs))
    mask0 = fci.occupation_mask(occ)
    assert abs(td.expectation(ctx, mpo, psi, psi).real - col[mask0]) < 1e-10 * max(1, abs(col[mask0]))
    # a few single and double excitations <D'|H|D>
    picks = [x for x in col if x != mask0][:: max(1, len(col) // 6)][:6]
    for mk in picks:
        o = [((mk >> (2 * i)) & 1) | (((mk >> (2 * i + 1)) & 1) << 1) for i in range(L)]
        bra = td.mps_from_determinant(ctx, o)
        assert abs(td.expectation(ctx, mpo, bra, psi) - col[mk]) < 1e-11


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("tf32x3", 2e-5)])
def test_ragged_odd_bond_dimensions(td, prec, tol):
    L, N, S, D = 7, 6, 0, 37
    I = synth.make_integrals(L, seed=43)
    sys_ = om.System.build(I.h, I.eri, 3, 3)
    A, q = synth.random_mps(L, N, S, D, seed=44)
    c = td.Context(prec)
    c.set_schedule(0, 2)
    mpo = td.build_mpo(c, I.h, I.eri, n_elec=N)
    out = td.apply_H(c, mpo, td.mps_import(c, A, q), 0.5j, D, 0.0)
    ref = om.apply_H(sys_, om.from_arrays(A, q), 0.5j, om.Schedule(D=D, n_two_site=0, n_one_site=2))
    got = sys_.vec(om.from_arrays(*out.export()))
    assert np.linalg.norm(got - sys_.vec(ref)) <= tol * np.linalg.norm(sys_.vec(ref))
    c.close()


def test_compress_to_bond_dimension_one(td, ctx):
    A, q = synth.random_mps(6, 6, 0, 20, seed=45)
    psi = td.mps_import(ctx, A, q)
    disc = td.compress(ctx, psi, 1, 0.0)
    ref, rdisc = om.compress(om.from_arrays(A, q), 1, 0.0)
    assert max(om.from_arrays(*psi.export()).bond_dims) == 1
    v, r = _vec(psi), om.to_fock(ref)
    assert abs(abs(np.vdot(v, r)) - np.linalg.norm(v) * np.linalg.norm(r)) < 1e-10 * np.linalg.norm(r) ** 2
    assert abs(disc - rdisc) < 1e-10


def test_argument_errors(td, ctx):
    I = synth.make_integrals(4, seed=46)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=4)
    psi = td.mps_from_determinant(ctx, [3, 3, 0, 0])
    for bad in (lambda: td.krylov_step(ctx, mpo, psi, 0.1, 1, True, 8),
                lambda: td.krylov_step(ctx, mpo, psi, 0.1, 17, True, 8),
                lambda: td.apply_H(ctx, mpo, psi, 1.0, 0, 0.0),
                lambda: td.apply_H(ctx, mpo, psi, 1.0, 8, 1.5),
                lambda: td.mps_from_determinant(ctx, []),
                lambda: td.mps_from_determinant(ctx, [4, 0])):
        with pytest.raises(td.TdmpsError) as e:
            bad()
        assert e.value.name == "INVALID_ARG"
    # non-finite scalar inputs are rejected on the host before any launch
    for bad in (lambda: td.apply_H(ctx, mpo, psi, complex(float("nan"), 0.0), 8, 0.0),
                lambda: td.rk4_step(ctx, mpo, psi, float("inf"), 8),
                lambda: td.krylov_step(ctx, mpo, psi, float("nan"), 4, True, 8)):
        with pytest.raises(td.TdmpsError) as e:
            bad()
        assert e.value.name == "NONFINITE"
    other = td.mps_from_determinant(ctx, [3, 1, 0, 0])
    with pytest.raises(td.TdmpsError) as e:
        td.overlap(ctx, psi, other)
    assert e.value.name == "SECTOR"


def test_compress_keeps_a_degenerate_top_cluster_whole(td, ctx):
    # Two orbitals, one up and one down electron in an equal-weight
    # superposition of |up, down> and |down, up>: the middle bond has two
    # one-dimensional sectors, (1, 1) and (1, -1), with equal singular values.
    # Compressing to D = 1 would cut inside that top cluster, so the rule
    # keeps both (like the oracle), the state is unchanged, nothing is
    # discarded.
    dets = fci.basis(2, 1, 1)
    v = np.zeros(len(dets), dtype=complex)
    for occ, amp in (([1, 2], 1 / np.sqrt(2)), ([2, 1], -1 / np.sqrt(2))):
        v[np.searchsorted(dets, np.uint64(fci.occupation_mask(occ)))] = amp
    m = om.from_fock(om.sector_to_fock(v, dets, 2), 2)
    psi = td.mps_import(ctx, m.tensors, m.labels)
    disc = td.compress(ctx, psi, 1, 0.0)
    ref, rdisc = om.compress(m, 1, 0.0)
    assert om.from_arrays(*psi.export()).bond_dims == ref.bond_dims == [1, 2, 1]
    assert abs(disc) < 1e-12 and abs(rdisc) < 1e-12
    assert abs(abs(td.overlap(ctx, td.mps_import(ctx, m.tensors, m.labels), psi)) - 1.0) < 1e-12
