"""Repeatability: the same call on the same inputs gives the same bits.

Every reduction on the path adds in a fixed order (split-K slices in split
order, cluster and warp partial sums in rank order, no floating-point
atomics), so two runs of a fit or a time step -- including the concurrent
inner products, the two-site sweeps with their SVD truncation and the
tensor-core contractions -- must agree bit for bit.  Without that, FP64
results could not be compared run to run and an ill-conditioned step (such
as the benchmark's Krylov step from a random start) would not be
reproducible.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def td():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_08489_gb300 as mod
    mod.lib()
    return mod


def _states_equal(a, b):
    (ta, la), (tb, lb) = a, b
    return (all(np.array_equal(x, y) for x, y in zip(la, lb))
            and all(np.array_equal(x, y) for x, y in zip(ta, tb)))


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_bench_size_krylov_step_is_bitwise_repeatable(td, prec):
    I = synth.make_integrals(16, seed=0)
    A, q = synth.random_mps(16, 15, 1, 256, seed=0)
    outs = []
    for _ in range(2):
        ctx = td.Context(prec)
        ctx.set_schedule(0, 2)
        mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=15)
        psi = td.mps_import(ctx, A, q)
        td.krylov_step(ctx, mpo, psi, 0.05, 4, True, 256, 1e-8)
        outs.append(psi.export())
        ctx.close()
    assert _states_equal(outs[0], outs[1])


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_two_site_trajectory_is_bitwise_repeatable(td, prec):
    # two-site sweeps with SVD truncation (eps and D both active), the
    # physical beta-hole start, three Krylov steps
    L = 10
    I = synth.make_integrals(L, seed=1)
    occ = synth.hole_occupation(L, L, 4)
    outs = []
    for _ in range(2):
        ctx = td.Context(prec)
        ctx.set_schedule(1, 1)
        mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=L - 1)
        psi = td.mps_from_determinant(ctx, occ)
        for _ in range(3):
            td.krylov_step(ctx, mpo, psi, 0.05, 6, True, 48, 1e-9)
        outs.append((psi.export(), td.one_rdm(ctx, psi)))
        ctx.close()
    assert _states_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
