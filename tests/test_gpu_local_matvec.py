"""The one-site local operator of the fit (tdmps_heff_*, the product L W x R of
Eq. add_min's local problem) on the GPU.

* FP64 equals the oracle (oracle.bsmps.local_matvec, pinned on the CPU against
  the full-CI projection M_i^+ H M_i) element by element at every site of an
  L = 8 chain: the first and last sites (boundary environments), the centre.
* Split TF32 and BF16 against the same oracle.  The product carries the FP32
  environment chains of up to L - 1 sites, the case the fitted-state bounds
  of the mixed tests cover (2e-5 relative for split TF32, 5e-2 for BF16).
* At the benchmark size (L = 16, 15 electrons, 2S_z = 1, D = 256, centre
  site): FP64 against the oracle on every element of the site (1e-10 of the
  largest entry, the FP64 observable bound), <A_c, H_c A_c> = <psi|H|psi>
  (the FP64 sandwich), and split TF32 against FP64 on every element.
* Only the operator's site of y changes; wrong bonds and a changed context
  precision are refused before any work.
"""
import numpy as np
import pytest

import synth
from oracle import bsmps as ob

pytestmark = pytest.mark.gpu

MIXED_TOL = {"tf32x3": 2e-5, "bf16": 5e-2}


@pytest.fixture(scope="module")
def td():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_08489_gb300 as mod
    mod.lib()
    return mod


def _perturbed(A, i, seed):
    """psi's tensors with site i multiplied entry-wise by random complex
    factors: the symmetry pattern is kept, the values are new."""
    rng = np.random.default_rng(seed)
    B = [a.copy() for a in A]
    B[i] = B[i] * (rng.standard_normal(B[i].shape) + 1j * rng.standard_normal(B[i].shape))
    return B


def _flat(site, like):
    return np.concatenate([site[k].reshape(-1) for k in like])


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _run_site(td, ctx, mpo, A, q, i, seed):
    psi = td.mps_import(ctx, A, q)
    X = _perturbed(A, i, seed)
    x = td.mps_import(ctx, X, q)
    y = td.mps_import(ctx, A, q)
    op = td.local_hamiltonian(ctx, mpo, psi, i)
    op.apply(x, y)
    yt, yq = y.export()
    op.free()
    for m in (psi, x, y):
        m.free()
    return X, yt, yq


def test_local_operator_matches_oracle_every_site_fp64(td):
    L = 8
    I = synth.make_integrals(L, seed=50)
    A, q = synth.random_mps(L, 7, 1, 40, seed=51)
    ctx = td.Context("fp64")
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=7, e0=0.2)
    mpo_o = ob.hamiltonian_mpo(I.h, I.eri, 0.2)
    psi_o = ob.from_dense(A, q)
    worst = 0.0
    for i in range(L):
        X, yt, yq = _run_site(td, ctx, mpo, A, q, i, 52 + i)
        got = ob.from_dense(yt, yq)
        ref = ob.local_matvec(mpo_o, psi_o, i, ob.from_dense(X, q).sites[i])
        keys = psi_o.sites[i]
        err = np.abs(_flat(got.sites[i], keys) - _flat(ref, keys)).max()
        scale = np.abs(_flat(ref, keys)).max()
        worst = max(worst, err / scale)
        assert err <= 1e-12 * scale
        # the other sites of y are psi's
        for j in range(L):
            if j != i:
                assert all(np.array_equal(got.sites[j][k], psi_o.sites[j][k]) for k in psi_o.sites[j])
    print("local operator L=8 D=40, FP64 vs oracle: max relative error %.2e" % worst)
    ctx.close()


@pytest.mark.parametrize("prec", ["tf32x3", "bf16"])
def test_local_operator_tensor_core_vs_oracle(td, prec):
    L = 8
    I = synth.make_integrals(L, seed=53)
    A, q = synth.random_mps(L, 7, 1, 64, seed=54)
    ctx = td.Context(prec)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=7)
    mpo_o = ob.hamiltonian_mpo(I.h, I.eri)
    psi_o = ob.from_dense(A, q)
    worst = 0.0
    for i in (0, 3, L - 1):
        X, yt, yq = _run_site(td, ctx, mpo, A, q, i, 55 + i)
        got = ob.from_dense(yt, yq)
        ref = ob.local_matvec(mpo_o, psi_o, i, ob.from_dense(X, q).sites[i])
        keys = psi_o.sites[i]
        worst = max(worst, _rel(_flat(got.sites[i], keys), _flat(ref, keys)))
    print("local operator L=8 D=64, %s vs oracle: relative error %.2e" % (prec, worst))
    assert worst < MIXED_TOL[prec]
    ctx.close()


def test_local_operator_at_bench_size_centre_site(td):
    L, N, S, D = 16, 15, 1, 256
    I = synth.make_integrals(L, seed=0)
    A, q = synth.random_mps(L, N, S, D, seed=0)
    c = L // 2
    out = {}
    for prec in ("fp64", "tf32x3"):
        ctx = td.Context(prec)
        mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=N)
        psi = td.mps_import(ctx, A, q)
        y = psi.copy()
        op = td.local_hamiltonian(ctx, mpo, psi, c)
        op.apply(psi, y)
        yt, yq = y.export()
        pt, pq = psi.export()
        out[prec] = (ob.from_dense(yt, yq).sites[c], ob.from_dense(pt, pq).sites[c])
        if prec == "fp64":
            e = td.expectation(ctx, mpo, psi, psi)
            env_mb = op.env_bytes / 1e6
        op.free()
        ctx.close()
    y64, a64 = out["fp64"]
    keys = a64
    # the oracle's local operator on the same state, every entry of the site
    psi_o = ob.from_dense(A, q)
    ref = ob.local_matvec(ob.hamiltonian_mpo(I.h, I.eri), psi_o, c, psi_o.sites[c])
    err = np.abs(_flat(y64, keys) - _flat(ref, keys)).max()
    scale = np.abs(_flat(ref, keys)).max()
    print("centre site of L=16 D=256: FP64 vs oracle, max abs error %.2e (max |y| %.2e)"
          % (err, scale))
    assert err <= 1e-10 * scale
    ea = np.vdot(_flat(a64, keys), _flat(y64, keys))
    print("centre site of L=16 D=256: <A,H_c A> - <psi|H|psi> = %.2e (|E| %.3e), "
          "environments %.1f MB (FP64)" % (abs(ea - e), abs(e), env_mb))
    assert abs(ea - e) <= 1e-11 * abs(e)
    r = _rel(_flat(out["tf32x3"][0], keys), _flat(y64, keys))
    print("centre site of L=16 D=256: split TF32 vs FP64 relative error %.2e" % r)
    assert r < MIXED_TOL["tf32x3"]


def test_local_operator_refuses_other_bonds_and_precision(td):
    L = 6
    I = synth.make_integrals(L, seed=56)
    A, q = synth.random_mps(L, 5, 1, 16, seed=57)
    B, qb = synth.random_mps(L, 5, 1, 12, seed=58)
    ctx = td.Context("fp64")
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=5)
    psi = td.mps_import(ctx, A, q)
    other = td.mps_import(ctx, B, qb)
    y = psi.copy()
    op = td.local_hamiltonian(ctx, mpo, psi, 2)
    with pytest.raises(td.TdmpsError):
        op.apply(other, y)
    with pytest.raises(td.TdmpsError):
        td.local_hamiltonian(ctx, mpo, psi, L)
    ctx.set_precision("tf32x3")
    with pytest.raises(td.TdmpsError):
        op.apply(psi, y)
    ctx.set_precision("fp64")
    op.apply(psi, y)          # x == y's source state, y a copy: allowed
    op.apply(y, y)            # x == y: allowed
    op.free()
    ctx.close()
