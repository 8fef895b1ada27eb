"""Mixed precision (tcgen05 TF32 / split 3xTF32 contractions, FP32
accumulation, FP64 factorisations) against the FP64 GPU path and the oracle.

Tolerances follow from the arithmetic: a TF32 product carries a relative
rounding of 2^-11 per operand, so sums of K ~ 10^3 terms land near 1e-3
relative; the split 3xTF32 product keeps ~21 mantissa bits, and FP32
accumulation plus FP32 storage of the environments (2^-24 per element,
~sqrt(K) growth per contraction, chained over ~2L environment updates) bound
a fitted state at ~2e-5 relative.
"""
import numpy as np
import pytest

import synth
from oracle import fci
from oracle import mps as om

pytestmark = pytest.mark.gpu

TOLS = {"tf32": 3e-3, "tf32x3": 2e-5}


@pytest.fixture(scope="module")
def td():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_08489_gb300 as mod
    mod.lib()
    return mod


def _to_oracle(m):
    t, q = m.export()
    return om.from_arrays(t, q)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("prec", ["tf32x3", "tf32"])
def test_small_sandwich_tensor_core(td, prec):
    L = 6
    I = synth.make_integrals(L, seed=1)
    sys_ = om.System.build(I.h, I.eri, 3, 2)
    ctx = td.Context(prec)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=5)
    A, q = synth.random_mps(L, 5, 1, 20, seed=2)
    B, qb = synth.random_mps(L, 5, 1, 14, seed=3)
    a, b = td.mps_import(ctx, A, q), td.mps_import(ctx, B, qb)
    ref = np.vdot(sys_.vec(om.from_arrays(B, qb)), sys_.H @ sys_.vec(om.from_arrays(A, q)))
    got = td.expectation(ctx, mpo, b, a)
    assert abs(got - ref) < TOLS[prec] * max(1.0, abs(ref)), (got, ref)
    ov = td.overlap(ctx, b, a)
    oref = om.overlap(om.from_arrays(B, qb), om.from_arrays(A, q))
    assert abs(ov - oref) < TOLS[prec] * max(1.0, abs(oref))
    ctx.close()


@pytest.mark.parametrize("prec", ["tf32x3", "tf32"])
def test_apply_h_mixed_vs_fp64(td, prec):
    L = 8
    I = synth.make_integrals(L, seed=0)
    sys_ = om.System.build(I.h, I.eri, 4, 3)
    A, q = synth.random_mps(L, 7, 1, 64, seed=4)
    res = {}
    for p in ("fp64", prec):
        ctx = td.Context(p)
        ctx.set_schedule(0, 2)
        mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=7)
        psi = td.mps_import(ctx, A, q)
        out = td.apply_H(ctx, mpo, psi, -0.05j, 64, 0.0)
        res[p] = sys_.vec(_to_oracle(out))
        ctx.close()
    ref = om.apply_H(sys_, om.from_arrays(A, q), -0.05j, om.Schedule(D=64, n_two_site=0, n_one_site=2))
    assert _rel(res["fp64"], sys_.vec(ref)) < 1e-10
    assert _rel(res[prec], res["fp64"]) < TOLS[prec]


def test_full_size_sandwich_tf32x3(td):
    L, N, S = 16, 15, 1
    I = synth.make_integrals(L, seed=0)
    ctx = td.Context("tf32x3")
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=N)
    A, q = synth.random_mps(L, N, S, 256, seed=0)
    psi = td.mps_import(ctx, A, q)
    opsi = om.from_arrays(A, q)
    occ = synth.hole_occupation(L, 16, 7)
    d = td.mps_from_determinant(ctx, occ)
    got = td.expectation(ctx, mpo, d, psi)
    masks, coefs = fci.h_on_determinant(I.h, I.eri, fci.occupation_mask(occ))
    occs = [[((int(mk) >> (2 * i)) & 1) + 2 * ((int(mk) >> (2 * i + 1)) & 1) for i in range(L)]
            for mk in masks]
    ref = np.sum(coefs * om.coefficients(opsi, occs))
    assert abs(got - ref) < 1e-5 * max(1.0, abs(ref)), (got, ref)
    ctx.close()


def test_krylov_trajectory_mixed_observables(td):
    # Krylov steps in split TF32 follow the FP64 GPU run: 1-RDM and energy
    L = 8
    I = synth.make_integrals(L, seed=0)
    occ = synth.hole_occupation(8, 8, 3)
    out = {}
    for p in ("fp64", "tf32x3"):
        ctx = td.Context(p)
        ctx.set_schedule(2, 1)
        mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=7)
        psi = td.mps_from_determinant(ctx, occ)
        gs, es = [], []
        for _ in range(3):
            td.krylov_step(ctx, mpo, psi, 0.05, 6, True, 128, 1e-10)
            gs.append(td.one_rdm(ctx, psi))
            es.append(td.expectation(ctx, mpo, psi, psi).real)
        out[p] = (np.array(gs), np.array(es))
        ctx.close()
    assert np.abs(out["fp64"][0] - out["tf32x3"][0]).max() < 1e-5
    assert np.abs(out["fp64"][1] - out["tf32x3"][1]).max() < 1e-5
