"""Mixed precision (tcgen05 TF32 / split 3xTF32 contractions, FP32
accumulation, FP64 factorisations) against the FP64 GPU path and the oracle.

Tolerances follow from the arithmetic: a TF32 product carries a relative
rounding of 2^-11 per operand, so sums of K ~ 10^3 terms land near 1e-3
relative; a BF16 operand carries 2^-8 (about 4e-3 per product, chained over
~2L environment updates: a few 1e-2); the split 3xTF32 product keeps ~21
mantissa bits, and FP32
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

TOLS = {"tf32": 3e-3, "tf32x3": 2e-5, "bf16": 5e-2}


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


@pytest.mark.parametrize("prec", ["tf32x3", "tf32", "bf16"])
def test_small_apply_tensor_core_vs_oracle(td, prec):
    # the fit contractions run on the tensor cores; compare with the oracle
    L = 6
    I = synth.make_integrals(L, seed=1)
    sys_ = om.System.build(I.h, I.eri, 3, 2)
    ctx = td.Context(prec)
    ctx.set_schedule(1, 2)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=5)
    A, q = synth.random_mps(L, 5, 1, 20, seed=2)
    a = td.mps_import(ctx, A, q)
    out = td.apply_H(ctx, mpo, a, 0.4 + 0.3j, 14, 0.0)
    ref = om.apply_H(sys_, om.from_arrays(A, q), 0.4 + 0.3j,
                     om.Schedule(D=14, n_two_site=1, n_one_site=2))
    assert _rel(sys_.vec(_to_oracle(out)), sys_.vec(ref)) < TOLS[prec]
    ctx.close()


@pytest.mark.parametrize("prec", ["tf32x3", "tf32", "bf16"])
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


def test_full_size_apply_tf32x3_vs_fp64(td):
    # L = 16, D = 256: the split-TF32 fit and the FP64 fit of the same H|psi>
    # agree to the mixed tolerance (fidelity and norm, FP64 overlaps)
    L, N, S = 16, 15, 1
    I = synth.make_integrals(L, seed=0)
    A, q = synth.random_mps(L, N, S, 256, seed=0)
    outs = {}
    ctx = td.Context("fp64")
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=N)
    ctx.set_schedule(0, 1)
    psi = td.mps_import(ctx, A, q)
    outs["fp64"] = td.apply_H(ctx, mpo, psi, -0.05j, 256, 0.0)
    ctx.set_precision("tf32x3")
    outs["tf32x3"] = td.apply_H(ctx, mpo, psi, -0.05j, 256, 0.0)
    a, b = outs["fp64"], outs["tf32x3"]
    aa, bb, ab = td.overlap(ctx, a, a).real, td.overlap(ctx, b, b).real, td.overlap(ctx, a, b)
    assert 1.0 - abs(ab) ** 2 / (aa * bb) < TOLS["tf32x3"] ** 2
    assert abs(np.sqrt(bb / aa) - 1.0) < TOLS["tf32x3"]
    ctx.close()


def test_krylov_trajectory_mixed_observables(td):
    # Krylov steps in split TF32 follow the FP64 GPU run: 1-RDM and energy.
    # The fits contract in split TF32 with FP32 accumulation, so the energy
    # is conserved to ~1e-6 relative per step (FP64 conserves it exactly);
    # three steps of |E| ~ 5.6 stay within 3e-5.
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
    assert np.abs(out["fp64"][1] - out["tf32x3"][1]).max() < 3e-5
    # FP64 Krylov conserves the energy up to the truncation (eps = 1e-10 weight)
    assert np.ptp(out["fp64"][1]) < 1e-8


def test_full_size_krylov_step_mixed_vs_fp64_physical(td):
    # The benchmark's Krylov step at full size (L = 16, D = 256, m = 10,
    # dt = 0.05, eps = 1e-8) on the physical beta-hole state, one two-site +
    # one one-site sweep per fit: split 3xTF32 against FP64 on the GPU.  The
    # energy stays within 1e-6 (the accuracy target of the mixed mode); the
    # 1-RDM within the FP32 class of the products (~1e-5 per step).
    L = 16
    I = synth.make_integrals(L, seed=0)
    occ = synth.hole_occupation(L, 16, 7)
    res = {}
    for p in ("fp64", "tf32x3"):
        ctx = td.Context(p)
        ctx.set_schedule(1, 1)
        mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=15)
        psi = td.mps_from_determinant(ctx, occ)
        td.krylov_step(ctx, mpo, psi, 0.05, 10, True, 256, 1e-8)
        nrm = td.overlap(ctx, psi, psi).real
        e = td.expectation(ctx, mpo, psi, psi).real / nrm
        g = td.one_rdm(ctx, psi)
        res[p] = (g, e)
        ctx.close()
        # properties of any 15-electron state, at full size: the particle
        # number is exact (one block-sparse sector), and the occupations of a
        # spatial orbital (eigenvalues of the spin-summed 1-RDM) lie in [0, 2]
        assert abs(np.trace(g).real / nrm - 15.0) < 1e-9
        lam = np.linalg.eigvalsh(g / nrm)
        assert lam.min() > -1e-9 and lam.max() < 2.0 + 1e-9
    assert abs(res["fp64"][1] - res["tf32x3"][1]) < 1e-6
    assert np.abs(res["fp64"][0] - res["tf32x3"][0]).max() < 2e-5
